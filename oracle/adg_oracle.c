/*
 * adg_oracle.c -- the FP64 CPU oracle for the AutoDiffGeo shape->material map
 * and its adjoint-gradient sum reduction (arXiv 2311.05646).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * loads this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or constant with the CUDA path.
 *
 * It is deliberately plain: every cell, every component and every primitive is
 * evaluated with straight loops (no binning, no tiling, no culling), in double
 * precision, following the paper's definitions:
 *
 *   sigma_k(x) = sigma(k x)                        Sec. 4, Table "Nonlinear
 *                                                  function definitions"
 *   primitives (Step/Rect/Poly/Circ/GeneralCartesian2D)
 *                                                  Table "AutoDiffGeo definitions"
 *   union / intersection                           Eqs. union, intersection and
 *                                                  Appendix B.2 (union_2, int_2)
 *   eps = eps_b + (eps_s - eps_b) * fill           Sec. 5.1 (volumetric average)
 *   grad f = Re sum_j w * (d eps_j / d v) E_j E_j^adj   Eq. 1 (eps term); the
 *            reverse sweep follows Eqs. AD / jaceps: the seed eta_P = E (.) E_adj
 *            is pulled back through each stage of the composition in turn.
 *   central finite differences of the loss         the FD baseline of Sec. 3
 *
 * Exactness of the axis-aligned box: the paper (Sec. 5.1, Eq. linear) shows the
 * piecewise-linear sigma with k = 1/dx gives the exact area fraction of an
 * axis-parallel edge.  The default box here is that exact form written as the
 * overlap of the box with the cell's averaging window, factor by factor.
 *
 * Readings where the paper is silent (the same list is kept in the design
 * notes): sample offsets are inputs; kinks take the closed interval; the
 * polygon normal points inward whatever the winding; difference(a,b) =
 * intersection(a, 1-b); clamp subgradients pass through at the boundary;
 * a circle's derivative w.r.t. its centre is 0 at r = 0, and so is a polar
 * shape's (whose angle is then taken as 0); a rotation / aspect transform
 * (Sec. 4, item iii) evaluates the primitive at p + S^-1 R(-theta) (r - p).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- description enums (the input format; see the design notes) ---------- */
enum { OD_BOX = 0, OD_CIRCLE = 1, OD_POLYGON = 2, OD_GRAPH = 3, OD_POLAR = 4 };
enum { OD_LINEAR = 0, OD_SIGMOID = 1, OD_QUADRATIC = 2, OD_SIN = 3, OD_ERF = 4 };
enum { OD_PRODUCT = 0, OD_CLAMP = 1 };
enum {
  OD_BOUND_X = 1, OD_BOUND_Y = 2, OD_BOUND_Z = 4, /* box: which axes are bounded */
  OD_RECT_SIGMA = 8,   /* box uses the paper's Rect product of sigma_k factors */
  OD_GRAPH_ABOVE = 16, /* graph: region y > f(x) instead of y < f(x)          */
  OD_XFORM = 64        /* in-plane rotation + aspect transform (last 5 scalars) */
};
enum { OD_OP_PUSH = 0, OD_OP_UNION = 1, OD_OP_INTERSECT = 2, OD_OP_DIFF = 3 };

typedef struct {
  int32_t nx, ny, nz, ncomp;
  double d[3];   /* grid spacing per axis                                    */
  double o[3];   /* origin per axis                                          */
  double off[9]; /* off[3*c + axis]: sample offset of component c, in cells   */
  double eps_bg, eps_fg;
  int32_t logic;
  int32_t nparam;
  int32_t nq;
  int32_t nprim;
  int32_t nops;
  int32_t pad_;
  const double *q_base, *q_coeff; /* q_j = q_base[j] + q_coeff[j] * p[q_param[j]] */
  const int32_t *q_param;         /* -1: constant geometric scalar           */
  const int32_t *kind, *sigma, *flags, *q0, *nqp; /* per primitive            */
  const double *kr;               /* per primitive: k = kr / spacing          */
  const int32_t *ops;             /* postfix program: (code << 24) | arg      */
} od_design;

/* ------------------------------------------------------------------------- */
/* sigma(u): the [0,1]-bounded building blocks of Table "Nonlinear function
 * definitions", in the unit variable u = k x.  Returns sigma, writes d sigma/du.
 * Kinks take the closed interval (the derivative of the inner branch).        */
double od_sigma(int kind, double u, double *dsdu) {
  const double r2 = 1.0 / sqrt(2.0);
  double s = 0.0, ds = 0.0;
  switch (kind) {
  case OD_LINEAR: /* max{0, min{1, u + 1/2}} */
    if (u < -0.5) { s = 0.0; ds = 0.0; }
    else if (u > 0.5) { s = 1.0; ds = 0.0; }
    else { s = u + 0.5; ds = 1.0; }
    break;
  case OD_SIGMOID: /* (1 + exp(-u))^-1; derivative sigma (1 - sigma) (Sec. 3.1) */
    if (u >= 0.0) { double e = exp(-u); s = 1.0 / (1.0 + e); }
    else { double e = exp(u); s = e / (1.0 + e); }
    ds = s * (1.0 - s);
    break;
  case OD_QUADRATIC: /* piecewise quadratic, exact for a 45-degree edge (Eq. quadratic) */
    if (u < -r2) { s = 0.0; ds = 0.0; }
    else if (u < 0.0) { s = (r2 + u) * (r2 + u); ds = 2.0 * (r2 + u); }
    else if (u <= r2) { s = 1.0 - (r2 - u) * (r2 - u); ds = 2.0 * (r2 - u); }
    else { s = 1.0; ds = 0.0; }
    break;
  case OD_SIN: /* (1 + sin u)/2 on [-pi/2, pi/2], clamped outside */
    if (u < -M_PI / 2) { s = 0.0; ds = 0.0; }
    else if (u > M_PI / 2) { s = 1.0; ds = 0.0; }
    else { s = 0.5 * (1.0 + sin(u)); ds = 0.5 * cos(u); }
    break;
  case OD_ERF: /* (1 + Erf(u))/2 */
    s = 0.5 * (1.0 + erf(u));
    ds = exp(-u * u) / sqrt(M_PI);
    break;
  default:
    s = 0.0; ds = 0.0;
  }
  if (dsdu) *dsdu = ds;
  return s;
}

/* Exact fraction of the window [c - h/2, c + h/2] covered by [a, b], and its
 * derivatives w.r.t. a and b (the exact volumetric average of an axis-aligned
 * slab; Sec. 5.1, Eq. linear / dlinear).                                      */
static double overlap1d(double a, double b, double c, double h, double *dda, double *ddb) {
  double lo = fmax(a, c - 0.5 * h);
  double hi = fmin(b, c + 0.5 * h);
  double len = hi - lo;
  if (len > 0.0) {
    if (dda) *dda = (a >= c - 0.5 * h) ? -1.0 / h : 0.0;
    if (ddb) *ddb = (b <= c + 0.5 * h) ? 1.0 / h : 0.0;
    return len / h;
  }
  if (dda) *dda = 0.0;
  if (ddb) *ddb = 0.0;
  return 0.0;
}

/* Evaluate primitive `pi` (flags fl, nq scalars Q) at the point r (physical
 * coordinates).  Writes s and, if dsdq != NULL, d s / d Q for every scalar. */
static int prim_eval(const od_design *D, int pi, int fl, int nq, const double *Q,
                     const double r[3], double *s_out, double *dsdq) {
  const int kind = D->kind[pi], sk = D->sigma[pi];
  if (dsdq)
    for (int t = 0; t < nq; ++t) dsdq[t] = 0.0;

  if (kind == OD_BOX) {
    /* Rect1D / Rect2D / RectdD: product of per-axis factors (Table, Rect*D).
     * q = x0, x1, y0, y1, z0, z1. */
    if (nq != 6) return -1;
    double f[3], dfa[3], dfb[3];
    for (int ax = 0; ax < 3; ++ax) {
      f[ax] = 1.0; dfa[ax] = 0.0; dfb[ax] = 0.0;
      if (!(fl & (1 << ax))) continue;
      double a = Q[2 * ax], b = Q[2 * ax + 1], h = D->d[ax];
      if (fl & OD_RECT_SIGMA) {
        double k = D->kr[pi] / h, d1, d2;
        double s1 = od_sigma(sk, k * (r[ax] - a), &d1);
        double s2 = od_sigma(sk, k * (b - r[ax]), &d2);
        f[ax] = s1 * s2;
        dfa[ax] = -k * d1 * s2;
        dfb[ax] = s1 * k * d2;
      } else {
        f[ax] = overlap1d(a, b, r[ax], h, &dfa[ax], &dfb[ax]);
      }
    }
    double s = f[0] * f[1] * f[2];
    *s_out = s;
    if (dsdq) {
      for (int ax = 0; ax < 3; ++ax) {
        double other = 1.0;
        for (int bx = 0; bx < 3; ++bx)
          if (bx != ax) other *= f[bx];
        dsdq[2 * ax] = dfa[ax] * other;
        dsdq[2 * ax + 1] = dfb[ax] * other;
      }
    }
    return 0;
  }

  /* extrusion along z for the 2D primitives: exact overlap (planarity, Sec. 5.2) */
  double zf = 1.0, dz0 = 0.0, dz1 = 0.0;
  int zq0 = -1;

  if (kind == OD_CIRCLE) {
    /* Circ2D: sigma_k(R - r(x, y, x0, y0)); q = cx, cy, R, z0, z1 */
    if (nq != 5) return -1;
    double cx = Q[0], cy = Q[1], R = Q[2];
    zq0 = 3;
    if (fl & OD_BOUND_Z) zf = overlap1d(Q[3], Q[4], r[2], D->d[2], &dz0, &dz1);
    double ddx = r[0] - cx, ddy = r[1] - cy;
    double rr = sqrt(ddx * ddx + ddy * ddy);
    double k = D->kr[pi] / D->d[0], ds;
    double sg = od_sigma(sk, k * (R - rr), &ds);
    *s_out = sg * zf;
    if (dsdq) {
      double g = k * ds * zf; /* d s / d (R - r) */
      dsdq[2] = g;
      if (rr > 0.0) {
        dsdq[0] = g * (ddx / rr); /* d(-r)/d cx = (x - cx)/r */
        dsdq[1] = g * (ddy / rr);
      }
    }
  } else if (kind == OD_POLAR) {
    /* Polar2D (Table 4) with the Fourier boundary of the PSGC scatterers:
     * sigma_k(R(theta) - r), R(theta) = R0 + sum_n c_n cos(n theta) + s_n sin(n theta),
     * theta and r the polar angle and radius about (cx, cy);
     * q = cx, cy, R0, z0, z1, c_1, s_1, ..., c_N, s_N */
    if (nq < 5 || (nq - 5) % 2) return -1;
    const int N = (nq - 5) / 2;
    double cx = Q[0], cy = Q[1];
    zq0 = 3;
    if (fl & OD_BOUND_Z) zf = overlap1d(Q[3], Q[4], r[2], D->d[2], &dz0, &dz1);
    double ddx = r[0] - cx, ddy = r[1] - cy;
    double rr = sqrt(ddx * ddx + ddy * ddy);
    double th = rr > 0.0 ? atan2(ddy, ddx) : 0.0;
    double Rth = Q[2], dR = 0.0; /* R(theta), dR / dtheta */
    for (int n = 1; n <= N; ++n) {
      double cn = Q[3 + 2 * n], sn = Q[4 + 2 * n];
      Rth += cn * cos(n * th) + sn * sin(n * th);
      dR += n * (sn * cos(n * th) - cn * sin(n * th));
    }
    double k = D->kr[pi] / D->d[0], ds;
    double sg = od_sigma(sk, k * (Rth - rr), &ds);
    *s_out = sg * zf;
    if (dsdq) {
      double g = k * ds * zf; /* d s / d (R(theta) - r) */
      dsdq[2] = g;
      for (int n = 1; n <= N; ++n) {
        dsdq[3 + 2 * n] = g * cos(n * th);
        dsdq[4 + 2 * n] = g * sin(n * th);
      }
      if (rr > 0.0) {
        /* d theta / d cx = (y - cy) / r^2, d theta / d cy = -(x - cx) / r^2 */
        dsdq[0] = g * (ddx / rr + dR * ddy / (rr * rr));
        dsdq[1] = g * (ddy / rr - dR * ddx / (rr * rr));
      }
    }
  } else if (kind == OD_POLYGON) {
    /* Poly2D: product over edges of Step2D with the edge's inward unit normal;
     * q = z0, z1, x1, y1, ..., xN, yN. */
    int N = (nq - 2) / 2;
    if (N < 3 || nq != 2 + 2 * N) return -1;
    zq0 = 0;
    if (fl & OD_BOUND_Z) zf = overlap1d(Q[0], Q[1], r[2], D->d[2], &dz0, &dz1);
    const double *V = Q + 2;
    double area2 = 0.0; /* twice the signed area: fixes which side is inside */
    for (int e = 0; e < N; ++e) {
      int e1 = (e + 1) % N;
      area2 += V[2 * e] * V[2 * e1 + 1] - V[2 * e1] * V[2 * e + 1];
    }
    double sgn = area2 >= 0.0 ? 1.0 : -1.0;
    double k = D->kr[pi] / D->d[0];
    if (N > 4096) return -1;
    double sig[N], dsig[N];
    double prod = 1.0;
    for (int e = 0; e < N; ++e) {
      int e1 = (e + 1) % N;
      double ex = V[2 * e1] - V[2 * e], ey = V[2 * e1 + 1] - V[2 * e + 1];
      double L = sqrt(ex * ex + ey * ey);
      double rx = r[0] - V[2 * e], ry = r[1] - V[2 * e + 1];
      double cross = ex * ry - ey * rx; /* left normal (-ey, ex) . (r - v_e) * L */
      double dist = sgn * cross / L;
      sig[e] = od_sigma(sk, k * dist, &dsig[e]);
      prod *= sig[e];
    }
    *s_out = prod * zf;
    if (dsdq) {
      for (int e = 0; e < N; ++e) {
        if (dsig[e] == 0.0) continue;
        double others = zf;
        for (int f2 = 0; f2 < N; ++f2)
          if (f2 != e) others *= sig[f2];
        double g = others * k * dsig[e]; /* d s / d dist_e */
        int e1 = (e + 1) % N;
        double ex = V[2 * e1] - V[2 * e], ey = V[2 * e1 + 1] - V[2 * e + 1];
        double L = sqrt(ex * ex + ey * ey);
        double rx = r[0] - V[2 * e], ry = r[1] - V[2 * e + 1];
        double cross = ex * ry - ey * rx;
        /* d cross and d L w.r.t. (x_e, y_e, x_e1, y_e1) */
        double dc[4] = {-ry + ey, -ex + rx, ry, -rx};
        double dL[4] = {-ex / L, -ey / L, ex / L, ey / L};
        int idx[4] = {2 + 2 * e, 2 + 2 * e + 1, 2 + 2 * e1, 2 + 2 * e1 + 1};
        for (int t = 0; t < 4; ++t) {
          double dd = sgn * (dc[t] / L - cross * dL[t] / (L * L));
          dsdq[idx[t]] += g * dd;
        }
      }
    }
  } else if (kind == OD_GRAPH) {
    /* GeneralCartesian2D: sigma_k(+-(f(x) - y)) with f the piecewise-linear
     * interpolant through (X_j, Y_j); q = z0, z1, X_1..X_M, Y_1..Y_M. */
    int M = (nq - 2) / 2;
    if (M < 2 || nq != 2 + 2 * M) return -1;
    zq0 = 0;
    if (fl & OD_BOUND_Z) zf = overlap1d(Q[0], Q[1], r[2], D->d[2], &dz0, &dz1);
    const double *X = Q + 2, *Y = Q + 2 + M;
    double x = r[0], f, dfdX[2] = {0, 0}, dfdY[2] = {0, 0};
    int j0 = 0, j1 = 0;
    if (x <= X[0]) { f = Y[0]; dfdY[0] = 1.0; j0 = j1 = 0; }
    else if (x >= X[M - 1]) { f = Y[M - 1]; dfdY[0] = 1.0; j0 = j1 = M - 1; }
    else {
      int j = 0;
      while (j + 1 < M - 1 && x >= X[j + 1]) ++j;
      double dX = X[j + 1] - X[j], dY = Y[j + 1] - Y[j], t = (x - X[j]) / dX;
      f = Y[j] + dY * t;
      dfdY[0] = 1.0 - t; dfdY[1] = t;
      dfdX[0] = dY * (x - X[j + 1]) / (dX * dX);
      dfdX[1] = -dY * (x - X[j]) / (dX * dX);
      j0 = j; j1 = j + 1;
    }
    double sgn = (fl & OD_GRAPH_ABOVE) ? -1.0 : 1.0;
    double k = D->kr[pi] / D->d[1], ds;
    double sg = od_sigma(sk, k * sgn * (f - r[1]), &ds);
    *s_out = sg * zf;
    if (dsdq) {
      double g = zf * k * ds * sgn; /* d s / d f */
      if (j0 == j1) {
        dsdq[2 + M + j0] += g * dfdY[0];
      } else {
        dsdq[2 + j0] += g * dfdX[0];
        dsdq[2 + j1] += g * dfdX[1];
        dsdq[2 + M + j0] += g * dfdY[0];
        dsdq[2 + M + j1] += g * dfdY[1];
      }
    }
  } else {
    return -1;
  }

  /* z derivatives: the in-plane factor times d(overlap)/d(z0, z1); with zero
   * overlap both derivatives of the overlap are zero as well. */
  if (dsdq && (fl & OD_BOUND_Z) && zf > 0.0) {
    double base = *s_out / zf;
    dsdq[zq0] += base * dz0;
    dsdq[zq0 + 1] += base * dz1;
  }
  return 0;
}

/* Rotation and aspect-ratio transform of a 2D primitive (Sec. 4, item iii:
 * the primitives support parameterized aspect-ratio and rotation
 * transforms; the paper gives no formula -- this is the reading).  The last
 * five scalars are the pivot (px, py), the angle theta (radians) and the
 * aspect (sx, sy > 0); the primitive, drawn with its own scalars, is stretched
 * by (sx, sy) along its own axes and rotated by theta about the pivot, i.e.
 * it is evaluated at the local point
 *     u = p + S^-1 R(-theta) (r - p),   S = diag(sx, sy),
 * with z untouched; its sigma_k acts on distances in local units.  Boxes take
 * the paper's sigma-product form (the exact window overlap is for
 * axis-aligned boxes), graphs are not transformed, and the grid must have
 * dx == dy.  Derivatives: the primitive's own scalars are those of the base
 * primitive at u; a transform scalar xi gives grad_u s . du/dxi, where the
 * spatial gradient grad_u s is minus the derivative of s w.r.t. a rigid
 * translation of the shape (the sum over its x, resp. y, position scalars). */
static int prim_xform(const od_design *D, int pi, int fl, int nq, const double *Q,
                      const double r[3], double *s_out, double *dsdq) {
  const int kind = D->kind[pi], nb = nq - 5;
  if (nb < 1 || kind == OD_GRAPH) return -1;
  if (kind == OD_BOX && !(fl & OD_RECT_SIGMA)) return -1;
  const double px = Q[nb], py = Q[nb + 1], th = Q[nb + 2], sx = Q[nb + 3], sy = Q[nb + 4];
  if (!(sx > 0.0) || !(sy > 0.0)) return -1;
  const double c = cos(th), s = sin(th);
  const double dx = r[0] - px, dy = r[1] - py;
  const double vx = c * dx + s * dy, vy = -s * dx + c * dy; /* R(-theta) (r - p) */
  const double u[3] = {px + vx / sx, py + vy / sy, r[2]};
  if (nb > 4096) return -1;
  double db[nb];
  int rc = prim_eval(D, pi, fl & ~OD_XFORM, nb, Q, u, s_out, dsdq ? db : NULL);
  if (rc || !dsdq) return rc;
  double gx = 0.0, gy = 0.0; /* grad_u s */
  if (kind == OD_BOX) {
    gx = -(db[0] + db[1]);
    gy = -(db[2] + db[3]);
  } else if (kind == OD_CIRCLE || kind == OD_POLAR) {
    gx = -db[0];
    gy = -db[1];
  } else { /* polygon: q = z0, z1, x1, y1, ... */
    for (int t = 2; t + 1 < nb; t += 2) { gx -= db[t]; gy -= db[t + 1]; }
  }
  for (int t = 0; t < nb; ++t) dsdq[t] = db[t];
  dsdq[nb] = gx * (1.0 - c / sx) + gy * (s / sy);                       /* d/d px    */
  dsdq[nb + 1] = gx * (-s / sx) + gy * (1.0 - c / sy);                  /* d/d py    */
  dsdq[nb + 2] = gx * ((-s * dx + c * dy) / sx) + gy * ((-c * dx - s * dy) / sy); /* theta */
  dsdq[nb + 3] = gx * (-vx / (sx * sx));                                 /* d/d sx    */
  dsdq[nb + 4] = gy * (-vy / (sy * sy));                                 /* d/d sy    */
  return 0;
}

/* Evaluate primitive `pi` at sample point r (physical coordinates).  `q` is the
 * full geometric-scalar vector; the primitive reads q[q0 .. q0 + nq - 1].
 * Writes s and, if dsdq != NULL, d s / d q_local for every local scalar.    */
int od_prim(const od_design *D, int pi, const double *q, const double r[3], double *s_out,
            double *dsdq) {
  const int fl = D->flags[pi], nq = D->nqp[pi];
  const double *Q = q + D->q0[pi];
  if (fl & OD_XFORM) return prim_xform(D, pi, fl, nq, Q, r, s_out, dsdq);
  return prim_eval(D, pi, fl, nq, Q, r, s_out, dsdq);
}

/* ---- the CSG program as an explicit tree --------------------------------- */
typedef struct {
  int n;          /* nodes = ops */
  int *code, *arg;
  int *cstart, *ccount; /* children of node i: child[cstart[i] .. + ccount[i]] */
  int *child;
  int root;
} od_tree;

static void tree_free(od_tree *T) {
  free(T->code);
  free(T->child);
}

/* Parse the postfix program into a tree.  Returns 0 on success. */
static int tree_build(const od_design *D, od_tree *T) {
  int n = D->nops;
  memset(T, 0, sizeof(*T));
  if (n <= 0) return -1;
  T->n = n;
  T->code = (int *)calloc((size_t)5 * n, sizeof(int));
  T->arg = T->code + n;
  T->cstart = T->code + 2 * n;
  T->ccount = T->code + 3 * n;
  int *stack = T->code + 4 * n;
  T->child = (int *)calloc((size_t)n + 1, sizeof(int));
  int sp = 0, nc = 0;
  for (int i = 0; i < n; ++i) {
    int code = (D->ops[i] >> 24) & 0xff, arg = D->ops[i] & 0xffffff;
    T->code[i] = code;
    T->arg[i] = arg;
    int need = 0;
    if (code == OD_OP_PUSH) {
      if (arg < 0 || arg >= D->nprim) { tree_free(T); return -2; }
      need = 0;
    } else if (code == OD_OP_UNION || code == OD_OP_INTERSECT) {
      need = arg;
      if (need < 1) { tree_free(T); return -3; }
    } else if (code == OD_OP_DIFF) {
      need = 2;
    } else { tree_free(T); return -4; }
    if (sp < need) { tree_free(T); return -5; }
    T->cstart[i] = nc;
    T->ccount[i] = need;
    for (int t = 0; t < need; ++t) T->child[nc + t] = stack[sp - need + t];
    nc += need;
    sp -= need;
    stack[sp++] = i;
  }
  if (sp != 1) { tree_free(T); return -6; }
  T->root = n - 1;
  return 0;
}

/* Forward value of one logic node from its children's values (Eqs. union,
 * intersection, and union_2 / intersection_2 of Appendix B.2). */
static double node_forward(int logic, int code, int nch, const double *cv) {
  if (code == OD_OP_UNION) {
    if (logic == OD_PRODUCT) { /* union_2: 1 - prod(1 - s_i), i.e. a + b - ab */
      double p = 1.0;
      for (int t = 0; t < nch; ++t) p *= (1.0 - cv[t]);
      return 1.0 - p;
    } else { /* min{1, sum s_i} */
      double s = 0.0;
      for (int t = 0; t < nch; ++t) s += cv[t];
      return fmin(1.0, s);
    }
  } else if (code == OD_OP_INTERSECT) {
    if (logic == OD_PRODUCT) { /* intersection_2: prod s_i */
      double p = 1.0;
      for (int t = 0; t < nch; ++t) p *= cv[t];
      return p;
    } else { /* max{N-1, sum s_i} - (N-1) */
      double s = 0.0;
      for (int t = 0; t < nch; ++t) s += cv[t];
      return fmax((double)(nch - 1), s) - (double)(nch - 1);
    }
  } else { /* difference(a, b) = intersection(a, 1 - b) */
    if (logic == OD_PRODUCT) return cv[0] * (1.0 - cv[1]);
    return fmax(0.0, cv[0] - cv[1]);
  }
}

/* Local partials d node / d child_t for every child. */
static void node_backward(int logic, int code, int nch, const double *cv, double *dcv) {
  if (code == OD_OP_UNION) {
    if (logic == OD_PRODUCT) {
      for (int t = 0; t < nch; ++t) {
        double p = 1.0;
        for (int u = 0; u < nch; ++u)
          if (u != t) p *= (1.0 - cv[u]);
        dcv[t] = p;
      }
    } else {
      double s = 0.0;
      for (int t = 0; t < nch; ++t) s += cv[t];
      for (int t = 0; t < nch; ++t) dcv[t] = (s <= 1.0) ? 1.0 : 0.0;
    }
  } else if (code == OD_OP_INTERSECT) {
    if (logic == OD_PRODUCT) {
      for (int t = 0; t < nch; ++t) {
        double p = 1.0;
        for (int u = 0; u < nch; ++u)
          if (u != t) p *= cv[u];
        dcv[t] = p;
      }
    } else {
      double s = 0.0;
      for (int t = 0; t < nch; ++t) s += cv[t];
      for (int t = 0; t < nch; ++t) dcv[t] = (s >= (double)(nch - 1)) ? 1.0 : 0.0;
    }
  } else {
    if (logic == OD_PRODUCT) { dcv[0] = 1.0 - cv[1]; dcv[1] = -cv[0]; }
    else {
      double on = (cv[0] - cv[1] >= 0.0) ? 1.0 : 0.0;
      dcv[0] = on; dcv[1] = -on;
    }
  }
}

/* Geometric scalars from parameters: q_j = b_j + a_j p_{idx_j}. */
static void param_map(const od_design *D, const double *p, double *q) {
  for (int j = 0; j < D->nq; ++j) {
    q[j] = D->q_base[j];
    if (D->q_param[j] >= 0) q[j] += D->q_coeff[j] * p[D->q_param[j]];
  }
}

static void sample_point(const od_design *D, int c, int i, int j, int k, double r[3]) {
  r[0] = D->o[0] + ((double)i + D->off[3 * c + 0]) * D->d[0];
  r[1] = D->o[1] + ((double)j + D->off[3 * c + 1]) * D->d[1];
  r[2] = D->o[2] + ((double)k + D->off[3 * c + 2]) * D->d[2];
}

static int max_nqp(const od_design *D) {
  int m = 1;
  for (int t = 0; t < D->nprim; ++t)
    if (D->nqp[t] > m) m = D->nqp[t];
  return m;
}

int od_validate(const od_design *D) {
  if (D->nx < 1 || D->ny < 1 || D->nz < 1 || D->ncomp < 1 || D->ncomp > 3) return -1;
  for (int t = 0; t < D->nprim; ++t) {
    if (D->q0[t] < 0 || D->q0[t] + D->nqp[t] > D->nq) return -2;
    if ((D->flags[t] & OD_XFORM) &&
        (D->kind[t] == OD_GRAPH || D->nqp[t] < 6 || fabs(D->d[0] - D->d[1]) > 1e-12 * D->d[0] ||
         (D->kind[t] == OD_BOX && !(D->flags[t] & OD_RECT_SIGMA))))
      return -4;
  }
  for (int j = 0; j < D->nq; ++j)
    if (D->q_param[j] >= D->nparam) return -3;
  od_tree T;
  int rc = tree_build(D, &T);
  if (rc) return -10 + rc;
  tree_free(&T);
  return 0;
}

/* Per-cell forward: leaf values, then node values in postfix order. */
static double cell_forward(const od_design *D, const od_tree *T, const double *q,
                           const double r[3], double *val, double *cvbuf) {
  for (int i = 0; i < T->n; ++i) {
    if (T->code[i] == OD_OP_PUSH) {
      double s;
      od_prim(D, T->arg[i], q, r, &s, NULL);
      val[i] = s;
    } else {
      int nch = T->ccount[i];
      for (int t = 0; t < nch; ++t) cvbuf[t] = val[T->child[T->cstart[i] + t]];
      val[i] = node_forward(D->logic, T->code[i], nch, cvbuf);
    }
  }
  return val[T->root];
}

/* fill[c][k][j][i] for all cells (the forward map v -> fill). */
int od_fill(const od_design *D, const double *p, double *fill) {
  if (od_validate(D)) return -1;
  od_tree T;
  tree_build(D, &T);
  double *q = (double *)malloc(sizeof(double) * (D->nq + 1));
  param_map(D, p, q);
  const int nplanes = D->ncomp * D->nz;
#pragma omp parallel
  {
    double *val = (double *)malloc(sizeof(double) * 2 * (T.n + 1));
    double *cvb = val + T.n + 1;
#pragma omp for schedule(dynamic, 1)
    for (int pl = 0; pl < nplanes; ++pl) {
      int c = pl / D->nz, k = pl % D->nz;
      for (int j = 0; j < D->ny; ++j)
        for (int i = 0; i < D->nx; ++i) {
          double r[3];
          sample_point(D, c, i, j, k, r);
          size_t idx = (((size_t)c * D->nz + k) * D->ny + j) * D->nx + i;
          fill[idx] = cell_forward(D, &T, q, r, val, cvb);
        }
    }
    free(val);
  }
  free(q);
  tree_free(&T);
  return 0;
}

/* fill at a list of flat indices ((c*nz + k)*ny + j)*nx + i. */
int od_fill_at(const od_design *D, const double *p, int64_t n, const int64_t *flat,
               double *out) {
  if (od_validate(D)) return -1;
  od_tree T;
  tree_build(D, &T);
  double *q = (double *)malloc(sizeof(double) * (D->nq + 1));
  param_map(D, p, q);
  double *val = (double *)malloc(sizeof(double) * 2 * (T.n + 1));
  double *cvb = val + T.n + 1;
  for (int64_t t = 0; t < n; ++t) {
    int64_t f = flat[t];
    int i = (int)(f % D->nx); f /= D->nx;
    int j = (int)(f % D->ny); f /= D->ny;
    int k = (int)(f % D->nz); f /= D->nz;
    int c = (int)f;
    double r[3];
    sample_point(D, c, i, j, k, r);
    out[t] = cell_forward(D, &T, q, r, val, cvb);
  }
  free(val);
  free(q);
  tree_free(&T);
  return 0;
}

/* The reverse sweep of Eqs. AD / jaceps for one design.
 *   seed mode 0: eta = Re(w_c E_adj E_fwd) (complex fields, no conjugate, Eq. 1)
 *   seed mode 1: eta = G (a real cotangent dL/deps, the autograd form)
 * g[n] receives d L / d p, with L = sum_c sum_cells eta * eps_c.
 * Per-plane partial sums are combined in plane order (deterministic). */
static int grad_impl(const od_design *D, const double *p, int mode, const float *ef,
                     const float *ea, const double *w, const float *G, double *g,
                     double *loss) {
  if (od_validate(D)) return -1;
  od_tree T;
  tree_build(D, &T);
  const int n = D->nparam, nq = D->nq, mq = max_nqp(D);
  double *q = (double *)malloc(sizeof(double) * (nq + 1));
  param_map(D, p, q);
  const int nplanes = D->ncomp * D->nz;
  double *gq_pl = (double *)calloc((size_t)nplanes * (nq + 1), sizeof(double));
  double *L_pl = (double *)calloc((size_t)nplanes, sizeof(double));
  const double deps = D->eps_fg - D->eps_bg;
#pragma omp parallel
  {
    double *val = (double *)malloc(sizeof(double) * (4 * (T.n + 1) + mq + 1));
    double *cvb = val + T.n + 1;
    double *dcv = cvb + T.n + 1;
    double *adj = dcv + T.n + 1;
    double *dsdq = adj + T.n + 1;
#pragma omp for schedule(dynamic, 1)
    for (int pl = 0; pl < nplanes; ++pl) {
      int c = pl / D->nz, k = pl % D->nz;
      double *gq = gq_pl + (size_t)pl * (nq + 1);
      double Lsum = 0.0;
      for (int j = 0; j < D->ny; ++j)
        for (int i = 0; i < D->nx; ++i) {
          size_t idx = (((size_t)c * D->nz + k) * D->ny + j) * D->nx + i;
          double eta;
          if (mode == 0) {
            /* eta_P = E (.) E_adj, weighted by w_c, real part (Eq. 1) */
            double fr = ef[2 * idx], fi = ef[2 * idx + 1];
            double ar = ea[2 * idx], ai = ea[2 * idx + 1];
            double pr = fr * ar - fi * ai, pi = fr * ai + fi * ar;
            double wr = w[2 * c], wi = w[2 * c + 1];
            eta = wr * pr - wi * pi;
          } else {
            eta = (double)G[idx];
          }
          double r[3];
          sample_point(D, c, i, j, k, r);
          double fillv = cell_forward(D, &T, q, r, val, cvb);
          Lsum += eta * (D->eps_bg + deps * fillv);
          if (eta == 0.0) continue;
          /* eps = eps_bg + deps * fill  ->  eta_fill = deps * eta */
          for (int t = 0; t < T.n; ++t) adj[t] = 0.0;
          adj[T.root] = deps * eta;
          /* logic nodes, root first (reverse postfix order) */
          for (int t = T.n - 1; t >= 0; --t) {
            if (T.code[t] == OD_OP_PUSH || adj[t] == 0.0) continue;
            int nch = T.ccount[t];
            for (int u = 0; u < nch; ++u) cvb[u] = val[T.child[T.cstart[t] + u]];
            node_backward(D->logic, T.code[t], nch, cvb, dcv);
            for (int u = 0; u < nch; ++u) adj[T.child[T.cstart[t] + u]] += adj[t] * dcv[u];
          }
          /* primitives: d s / d q_local, then into the geometric scalars */
          for (int t = 0; t < T.n; ++t) {
            if (T.code[t] != OD_OP_PUSH || adj[t] == 0.0) continue;
            int pi = T.arg[t];
            double s;
            od_prim(D, pi, q, r, &s, dsdq);
            for (int u = 0; u < D->nqp[pi]; ++u) gq[D->q0[pi] + u] += adj[t] * dsdq[u];
          }
        }
      L_pl[pl] = Lsum;
    }
    free(val);
  }
  /* parameter map: g_p[idx_j] += a_j dL/dq_j, planes combined in order */
  for (int t = 0; t < n; ++t) g[t] = 0.0;
  double L = 0.0;
  for (int pl = 0; pl < nplanes; ++pl) {
    const double *gq = gq_pl + (size_t)pl * (nq + 1);
    for (int jq = 0; jq < nq; ++jq)
      if (D->q_param[jq] >= 0) g[D->q_param[jq]] += D->q_coeff[jq] * gq[jq];
    L += L_pl[pl];
  }
  if (loss) *loss = L;
  free(gq_pl);
  free(L_pl);
  free(q);
  tree_free(&T);
  return 0;
}

int od_grad(const od_design *D, const double *p, const float *efwd, const float *eadj,
            const double *w, double *g, double *loss) {
  return grad_impl(D, p, 0, efwd, eadj, w, NULL, g, loss);
}

int od_grad_real(const od_design *D, const double *p, const float *G, double *g,
                 double *loss) {
  return grad_impl(D, p, 1, NULL, NULL, NULL, G, g, loss);
}

/* L(p) = Re sum_c sum_cells w_c E_adj E_fwd eps_c(p): forward only. */
double od_loss(const od_design *D, const double *p, const float *ef, const float *ea,
               const double *w) {
  size_t m = (size_t)D->ncomp * D->nz * D->ny * D->nx;
  double *fill = (double *)malloc(sizeof(double) * m);
  if (od_fill(D, p, fill)) { free(fill); return NAN; }
  const double deps = D->eps_fg - D->eps_bg;
  double L = 0.0;
  for (size_t idx = 0; idx < m; ++idx) {
    int c = (int)(idx / ((size_t)D->nz * D->ny * D->nx));
    double fr = ef[2 * idx], fi = ef[2 * idx + 1];
    double ar = ea[2 * idx], ai = ea[2 * idx + 1];
    double pr = fr * ar - fi * ai, pi = fr * ai + fi * ar;
    double eta = w[2 * c] * pr - w[2 * c + 1] * pi;
    L += eta * (D->eps_bg + deps * fill[idx]);
  }
  free(fill);
  return L;
}

/* Derivatives of the same L with respect to the two material levels of
 * eps = eps_b + (eps_s - eps_b) * fill (Sec. 5.1): L is linear in both, with
 *   dL/d eps_b = sum eta (1 - fill),   dL/d eps_s = sum eta fill,
 * eta = Re(w E_adj E_fwd) per sample.  out[0] = dL/d eps_bg, out[1] = dL/d eps_fg. */
int od_grad_material(const od_design *D, const double *p, const float *ef, const float *ea,
                     const double *w, double *out) {
  size_t m = (size_t)D->ncomp * D->nz * D->ny * D->nx;
  double *fill = (double *)malloc(sizeof(double) * m);
  if (od_fill(D, p, fill)) { free(fill); return -1; }
  double gb = 0.0, gf = 0.0;
  for (size_t idx = 0; idx < m; ++idx) {
    int c = (int)(idx / ((size_t)D->nz * D->ny * D->nx));
    double fr = ef[2 * idx], fi = ef[2 * idx + 1];
    double ar = ea[2 * idx], ai = ea[2 * idx + 1];
    double pr = fr * ar - fi * ai, pi = fr * ai + fi * ar;
    double eta = w[2 * c] * pr - w[2 * c + 1] * pi;
    gb += eta * (1.0 - fill[idx]);
    gf += eta * fill[idx];
  }
  free(fill);
  out[0] = gb;
  out[1] = gf;
  return 0;
}

/* The paper's baseline: central finite differences of L, one parameter at a
 * time (n + n re-evaluations of the material map; Sec. 3, Eq. 1 by FD). */
int od_grad_fd(const od_design *D, const double *p, const float *ef, const float *ea,
               const double *w, double h, double *g) {
  if (od_validate(D)) return -1;
  double *pp = (double *)malloc(sizeof(double) * (D->nparam + 1));
  for (int t = 0; t < D->nparam; ++t) {
    memcpy(pp, p, sizeof(double) * D->nparam);
    pp[t] = p[t] + h;
    double Lp = od_loss(D, pp, ef, ea, w);
    pp[t] = p[t] - h;
    double Lm = od_loss(D, pp, ef, ea, w);
    g[t] = (Lp - Lm) / (2.0 * h);
  }
  free(pp);
  return 0;
}

int od_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void od_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
