// adg_kernels.cu -- sm_103a kernels of libadg.
//
//   k_bin       one warp per tile: classify every primitive against the tile
//               (outside / inside / edge band) and fold the chained logic
//               program with the constants, leaving only the band primitives
//               (the restriction of work to the non-zero material-Jacobian
//               support that the paper suggests, Sec. 3 footnote, Sec. 7).
//   k_build     eps_c = eps_bg + deps * fill_c at every Yee sample (Eq. eps;
//               Table 4; Eqs. union / intersection; Sec. 5.1): persistent,
//               warp-specialised blocks -- band warps evaluate the folded
//               program of band tiles, a fill warp streams constant tiles.
//   k_vjp       per band tile (k_vjp_polar: the same for job tables that hold
//               Polar2D primitives): the reverse sweep of Eqs. AD / jaceps seeded
//               with Re(w E_adj E) (Eq. 1): forward tape, reverse logic
//               adjoints, primitive derivatives, warp-shuffle reduction per
//               (primitive, scalar) slot into compensated block partials.
//   k_finalize  per parameter: fixed-order sum of the block partials through
//               the parameter map (deterministic, FP64); it clears every
//               partial it reads, so the next VJP starts from zero.
//   k_dense,    the dense form's field stream: Re(w E_adj E) and its product
//   k_dense_final  with fill summed over every sample, per chunk, then in
//               chunk order.
// The build and the VJP take band tiles from a counter of their launch, so
// that tiles of very different cost balance over the blocks.
#include <limits.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "adg_internal.h"

namespace adg {
namespace {

constexpr float kMargin = 4e-3f;  // cells; classification is conservative by this much
enum : int { cOUT = 0, cIN = 1, cBND = 2 };

// ---------------------------------------------------------------- sigma ----
// Table "Nonlinear function definitions" in the unit variable u = k x.
__device__ __forceinline__ float sigma_f(int kind, float u, float& ds) {
  switch (kind) {
    case kLinear:
      if (u < -0.5f) { ds = 0.f; return 0.f; }
      if (u > 0.5f) { ds = 0.f; return 1.f; }
      ds = 1.f;
      return u + 0.5f;
    case kSigmoid: {
      // beyond |u| = 20 the tail (< 2.1e-9) is dropped, matching the binner's
      // band, so derivatives vanish exactly outside the derivative tile box
      if (u > 20.f) { ds = 0.f; return 1.f; }
      if (u < -20.f) { ds = 0.f; return 0.f; }
      const float t = expf(-fabsf(u));
      const float r = 1.f / (1.f + t);
      ds = t * r * r;  // sigma (1 - sigma)
      return u >= 0.f ? r : t * r;
    }
    case kQuadratic: {
      const float r2 = 0.70710678118654752f;
      if (u < -r2) { ds = 0.f; return 0.f; }
      if (u < 0.f) { const float a = r2 + u; ds = 2.f * a; return a * a; }
      if (u <= r2) { const float a = r2 - u; ds = 2.f * a; return 1.f - a * a; }
      ds = 0.f;
      return 1.f;
    }
    case kSin: {
      const float h = 1.57079632679489662f;
      if (u < -h) { ds = 0.f; return 0.f; }
      if (u > h) { ds = 0.f; return 1.f; }
      float s, c;
      sincosf(u, &s, &c);
      ds = 0.5f * c;
      return 0.5f * (1.f + s);
    }
    default:  // erf (tail beyond |u| = 4.5 below 1.1e-10, dropped as for the sigmoid)
      if (u > 4.5f) { ds = 0.f; return 1.f; }
      if (u < -4.5f) { ds = 0.f; return 0.f; }
      ds = 0.56418958354775629f * expf(-u * u);
      return 0.5f * (1.f + erff(u));
  }
}

struct Cell {
  int i, j, k;
  float ox, oy, oz;
};

// Exact int -> float for |v| < 2^22 by the IEEE-754 magic-number method:
// placing v in the mantissa of 1.5 * 2^23 (integer add) and subtracting that
// constant (float add).  Both run on the integer / FP32 pipes; a plain
// conversion instruction goes through a much narrower pipe on this part.
// Larger |v| are clamped: such a coordinate difference lies far outside any
// sample window, so its clamped value gives the same overlap / sigma.
__device__ __forceinline__ float i2f(int v) {
  v = min(max(v, -(1 << 21)), 1 << 21);
  return __int_as_float(v + 0x4B400000) - 12582912.0f;
}

// Exact fraction of the cell window [u - 1/2, u + 1/2] covered by [a, b]
// (Sec. 5.1, Eq. linear), a = ai0 + af0, b = ai1 + af1, u = i + off; da, db
// are its derivatives w.r.t. a and b in cells.
__device__ __forceinline__ float ov_exact(int ai0, float af0, int ai1, float af1, int i,
                                          float off, float& da, float& db) {
  const float ta = i2f(ai0 - i) + (af0 - off);
  const float tb = i2f(ai1 - i) + (af1 - off);
  const float len = fminf(tb, 0.5f) - fmaxf(ta, -0.5f);
  if (len > 0.f) {
    da = (ta >= -0.5f) ? -1.f : 0.f;
    db = (tb <= 0.5f) ? 1.f : 0.f;
    return len;
  }
  da = 0.f;
  db = 0.f;
  return 0.f;
}

__device__ __forceinline__ float zfactor(const PrimRec& P, const Cell& c, float& dz0, float& dz1) {
  if (!(P.flags & kBoundZ)) { dz0 = 0.f; dz1 = 0.f; return 1.f; }
  return ov_exact(P.ai[4], P.af[4], P.ai[5], P.af[5], c.k, c.oz, dz0, dz1);
}

// ------------------------------------------------------------ primitives ---
// Box (Rect1D / Rect2D / RectdD): product of per-axis factors.
__device__ __forceinline__ void box_axes(const PrimRec& P, const Cell& c, float f[3], float fa[3],
                                         float fb[3]) {
  const int idx[3] = {c.i, c.j, c.k};
  const float off[3] = {c.ox, c.oy, c.oz};
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    f[ax] = 1.f; fa[ax] = 0.f; fb[ax] = 0.f;
    if (!(P.flags & (1 << ax))) continue;
    if (P.flags & kRectSigma) {
      const float ta = i2f(P.ai[2 * ax] - idx[ax]) + (P.af[2 * ax] - off[ax]);
      const float tb = i2f(P.ai[2 * ax + 1] - idx[ax]) + (P.af[2 * ax + 1] - off[ax]);
      float d1, d2;
      const float s1 = sigma_f(P.sigma, -P.kr * ta, d1);
      const float s2 = sigma_f(P.sigma, P.kr * tb, d2);
      f[ax] = s1 * s2;
      fa[ax] = -P.kr * d1 * s2;
      fb[ax] = s1 * P.kr * d2;
    } else {
      f[ax] = ov_exact(P.ai[2 * ax], P.af[2 * ax], P.ai[2 * ax + 1], P.af[2 * ax + 1], idx[ax],
                       off[ax], fa[ax], fb[ax]);
    }
  }
}

// Circ2D: d = R - r in cells, with R^2 - r^2 formed from exact integer parts
// so that d keeps ~1e-7-cell accuracy for radii of hundreds of cells.
__device__ __forceinline__ float circle_dist(const PrimRec& P, const Cell& c, float& dxr,
                                             float& dyr, float& r) {
  const float fxi = i2f(c.i - P.ai[0]), fyi = i2f(c.j - P.ai[1]);
  const float dxf = c.ox - P.af[0], dyf = c.oy - P.af[1];
  const float ii2 = fxi * fxi + fyi * fyi;
  const float cr = 2.f * (fxi * dxf + fyi * dyf) + (dxf * dxf + dyf * dyf);
  r = sqrtf(fmaxf(ii2 + cr, 0.f));
  dxr = fxi + dxf;
  dyr = fyi + dyf;
  const float R = P.g[0];
  if (P.g[3] != 0.f) return R - r;
  const float den = R + r;
  return den > 0.f ? ((P.g[1] - ii2) + (P.g[2] - cr)) / den : 0.f;
}

// Polar2D with a Fourier boundary: R(theta) - r in cells, FP64 (R0 and the
// coefficients come from auxf as hi + lo float pairs: R0, c_1, s_1, ..., c_N,
// s_N).  cos(n theta),
// sin(n theta) by the angle-addition recurrence from cos, sin theta = (dx,
// dy) / r; at r = 0 theta is taken as 0.  Out: cos, sin theta, 1 / r (0 at
// r = 0) and dR / dtheta.
__device__ __forceinline__ double polar_coef(const float* F, int j) {
  return (double)F[2 * j] + (double)F[2 * j + 1];
}

__device__ __forceinline__ double polar_geom(const PrimRec& P, const Cell& c, const float* auxf,
                                             double& cth, double& sth, double& ir, double& dR) {
  const double dx = (double)(c.i - P.ai[0]) + ((double)c.ox - (double)P.af[0]);
  const double dy = (double)(c.j - P.ai[1]) + ((double)c.oy - (double)P.af[1]);
  const double r = sqrt(dx * dx + dy * dy);
  if (r > 0.0) { ir = 1.0 / r; cth = dx * ir; sth = dy * ir; }
  else { ir = 0.0; cth = 1.0; sth = 0.0; }
  const float* F = auxf + P.auxf_off;
  double R = polar_coef(F, 0), d1 = 0.0, cn = cth, sn = sth;
  for (int n = 1; n <= P.naux; ++n) {
    const double a = polar_coef(F, 2 * n - 1), b = polar_coef(F, 2 * n);
    R += a * cn + b * sn;
    d1 += (double)n * (b * cn - a * sn);
    const double c2 = cn * cth - sn * sth, s2 = sn * cth + cn * sth;
    cn = c2;
    sn = s2;
  }
  dR = d1;
  return R - r;
}

// The value-only form for the build and the tables.  Not inlined, like
// graph_dist: its FP64 work and outputs stay off the other kinds' paths.
__device__ __noinline__ float polar_dist(const PrimRec& P, const Cell& c, const float* auxf) {
  double cth, sth, ir, dR;
  return (float)polar_geom(P, c, auxf, cth, sth, ir, dR);
}

// GeneralCartesian2D: segment of the piecewise-linear f containing u_x.
__device__ __forceinline__ int graph_seg(const float* Xf, int M, float ux) {
  if (ux <= Xf[0]) return -1;
  if (ux >= Xf[M - 1]) return M - 1;
  int lo = 0, hi = M - 1;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (Xf[mid] <= ux) lo = mid; else hi = mid;
  }
  return lo;
}

// signed vertical distance f(x) - y (or y - f(x)) in cells, FP64 where it cancels.
// Not inlined: its FP64 conversions must not be hoisted into the box path.
__device__ __noinline__ float graph_dist(const PrimRec& P, const Cell& c, const float* auxf,
                                            const double* auxd, int& seg, double& t) {
  const int M = P.naux;
  const double* X = auxd + P.auxd_off;
  const double* Y = X + M;
  const double* iX = Y + M;
  const double uxd = (double)c.i + (double)c.ox;
  seg = graph_seg(auxf + P.auxf_off, M, (float)uxd);
  double f;
  t = 0.0;
  if (seg < 0) f = Y[0];
  else if (seg >= M - 1) f = Y[M - 1];
  else {
    t = (uxd - X[seg]) * iX[seg];
    f = Y[seg] + t * (Y[seg + 1] - Y[seg]);
  }
  const double d = f - ((double)c.j + (double)c.oy);
  return (float)((P.flags & kGraphAbove) ? -d : d);
}

// Poly2D: signed distance of the sample to edge e's line, inward positive, in
// cells (FP64 line equation: coordinates reach thousands of cells).
// Error-free sum (Knuth): a + b = s + e exactly (no contraction into fma).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Signed distance (cells, positive inside) of a sample from the line of one
// polygon edge (Table 4, Poly2D): n . (u - v_e), with u relative to the
// polygon's anchor cell (exact in fp32) and v_e, n stored as hi + lo pairs;
// the products are split exactly with fma, so the distance carries about 48
// bits however far the sample is from the anchor -- no FP64, whose rate on
// this part is a small fraction of fp32.
__device__ __forceinline__ float poly_d(const float* E, float ux, float uy) {
  float dxh, dxl, dyh, dyl;
  two_sum(ux, -E[0], dxh, dxl);
  two_sum(uy, -E[2], dyh, dyl);
  dxl = __fsub_rn(dxl, E[1]);
  dyl = __fsub_rn(dyl, E[3]);
  const float p1 = __fmul_rn(E[4], dxh), e1 = fmaf(E[4], dxh, -p1);
  const float p2 = __fmul_rn(E[6], dyh), e2 = fmaf(E[6], dyh, -p2);
  float sh, sl;
  two_sum(p1, p2, sh, sl);
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(sl, e1), e2),
                             __fadd_rn(fmaf(E[4], dxl, E[5] * dxh), fmaf(E[6], dyl, E[7] * dyh)));
  return __fadd_rn(sh, lo);
}

// Sample position relative to the polygon's anchor cell (exact in fp32).
__device__ __forceinline__ void poly_rel(const PrimRec& P, const Cell& c, float& ux, float& uy) {
  ux = (float)(c.i - P.ai[0]) + c.ox;
  uy = (float)(c.j - P.ai[1]) + c.oy;
}

__device__ __noinline__ float poly_value(const PrimRec& P, const Cell& c, const float* auxf) {
  const int N = P.naux;
  const float* E = auxf + P.auxf_off;
  float ux, uy;
  poly_rel(P, c, ux, uy);
  float prod = 1.f, ds;
  for (int e = 0; e < N && prod != 0.f; ++e)
    prod *= sigma_f(P.sigma, P.kr * poly_d(E + kPolyEdgeFloats * e, ux, uy), ds);
  return prod;
}

// ---- rotation / aspect transforms (Sec. 4, item iii) -----------------------------
// A transformed primitive (kXform; base kind in flags bits 8..11) is its base
// evaluated at the local point u = p + S^-1 R(-theta)(r - p), with its
// geometry in FP64 cells relative to the pivot (auxd, see kXformHead).  The
// local point and every distance are FP64 (a sample far from the pivot must
// keep sub-1e-7-cell accuracy); sigma and the products are fp32.  With
// derivatives, add(key, v, unit) receives d s / d q_key per cell (unit 0: x /
// y cells, 2: z cells, 3: dimensionless), keys in description order -- the
// base scalars, then px, py, theta, sx, sy through the spatial gradient
// grad_u s (minus the derivative w.r.t. a rigid translation of the shape).
__device__ __forceinline__ int xform_base(const PrimRec& P) { return (P.flags >> 8) & 15; }

struct NoAdd {
  __device__ __forceinline__ void operator()(int, float, int) const {}
};

template <bool kD, class Add>
__device__ __forceinline__ float xform_core(const PrimRec& P, const Cell& c, const double* auxd,
                                            const Add& add) {
  const double* A = auxd + P.auxd_off;
  const double* B = A + kXformHead;
  const double wx = (double)(c.i - P.ai[0]) + ((double)c.ox - A[6]);  // r - p, cells
  const double wy = (double)(c.j - P.ai[1]) + ((double)c.oy - A[7]);
  const double vx = A[0] * wx + A[1] * wy, vy = A[0] * wy - A[1] * wx;  // R(-theta)(r - p)
  const double ux = vx * A[2], uy = vy * A[3];                            // local, rel. pivot
  const int base = xform_base(P);
  const float kr = P.kr;
  double gx = 0.0, gy = 0.0;  // grad_u s (per local cell)
  int nb = 0;
  float s;
  if (base == kBox) {  // the paper's Rect form per bounded axis, z untransformed
    nb = 6;
    float f[3] = {1.f, 1.f, 1.f}, fa[3] = {0.f, 0.f, 0.f}, fb[3] = {0.f, 0.f, 0.f};
    const double pos[3] = {ux, uy, (double)c.k + (double)c.oz};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      if (!(P.flags & (1 << ax))) continue;
      float d1, d2;
      const float s1 = sigma_f(P.sigma, kr * (float)(pos[ax] - B[2 * ax]), d1);
      const float s2 = sigma_f(P.sigma, kr * (float)(B[2 * ax + 1] - pos[ax]), d2);
      f[ax] = s1 * s2;
      fa[ax] = -kr * d1 * s2;
      fb[ax] = s1 * kr * d2;
    }
    s = f[0] * f[1] * f[2];
    if (kD) {
      const float o0 = f[1] * f[2], o1 = f[0] * f[2], o2 = f[0] * f[1];
      add(0, fa[0] * o0, 0);
      add(1, fb[0] * o0, 0);
      add(2, fa[1] * o1, 0);
      add(3, fb[1] * o1, 0);
      add(4, fa[2] * o2, 2);
      add(5, fb[2] * o2, 2);
      gx = -(double)((fa[0] + fb[0]) * o0);
      gy = -(double)((fa[1] + fb[1]) * o1);
    }
  } else {
    float dz0 = 0.f, dz1 = 0.f;
    const float zf = zfactor(P, c, dz0, dz1);
    if (base == kCircle || base == kPolar) {
      const double dx = ux - B[0], dy = uy - B[1];
      const double r = sqrt(dx * dx + dy * dy);
      double Rt = B[2], dR = 0.0, cth = 1.0, sth = 0.0;
      const int N = base == kPolar ? P.naux : 0;
      nb = base == kPolar ? 5 + 2 * N : 5;
      if (r > 0.0) { cth = dx / r; sth = dy / r; }
      double cn = cth, sn = sth;
      for (int n = 1; n <= N; ++n) {
        Rt += B[1 + 2 * n] * cn + B[2 + 2 * n] * sn;
        dR += n * (B[2 + 2 * n] * cn - B[1 + 2 * n] * sn);
        const double c2 = cn * cth - sn * sth, s2 = sn * cth + cn * sth;
        cn = c2;
        sn = s2;
      }
      float ds;
      const float sg = sigma_f(P.sigma, kr * (float)(Rt - r), ds);
      s = sg * zf;
      if (kD) {
        const float gg = kr * ds * zf;  // d s / d (R(theta) - r)
        float dcx = 0.f, dcy = 0.f;
        if (r > 0.0) {
          dcx = gg * (float)(cth + dR * sth / r);
          dcy = gg * (float)(sth - dR * cth / r);
        }
        add(0, dcx, 0);
        add(1, dcy, 0);
        add(2, gg, 0);
        add(3, sg * dz0, 2);
        add(4, sg * dz1, 2);
        cn = cth;
        sn = sth;
        for (int n = 1; n <= N; ++n) {
          add(3 + 2 * n, gg * (float)cn, 0);
          add(4 + 2 * n, gg * (float)sn, 0);
          const double c2 = cn * cth - sn * sth, s2 = sn * cth + cn * sth;
          cn = c2;
          sn = s2;
        }
        gx = -(double)dcx;
        gy = -(double)dcy;
      }
    } else {  // polygon: product over edges of sigma of the inward distance
      const int N = P.naux;
      nb = 2 + 2 * N;
      const double sgn = B[0];
      const double* V = B + 1;
      float prod = 1.f, ds;
      int nzero = 0;
      if (zf != 0.f) {
        for (int e = 0; e < N; ++e) {
          const int e1 = e + 1 == N ? 0 : e + 1;
          const double ex = V[2 * e1] - V[2 * e], ey = V[2 * e1 + 1] - V[2 * e + 1];
          const double L = sqrt(ex * ex + ey * ey);
          const double dist = sgn * (ex * (uy - V[2 * e + 1]) - ey * (ux - V[2 * e])) / L;
          const float se = sigma_f(P.sigma, kr * (float)dist, ds);
          if (se == 0.f) { if (++nzero > 1) break; }
          else prod *= se;
        }
      }
      s = (zf != 0.f && nzero == 0) ? prod * zf : 0.f;
      if (kD) {
        const float inplane = (zf != 0.f && nzero == 0) ? prod : 0.f;
        add(0, inplane * dz0, 2);
        add(1, inplane * dz1, 2);
        const bool live = zf != 0.f && nzero <= 1;
        for (int e = 0; e < N; ++e) {
          const int e1 = e + 1 == N ? 0 : e + 1;
          float ge = 0.f;
          double ex = 0.0, ey = 0.0, L = 1.0, rx = 0.0, ry = 0.0, cross = 0.0;
          if (live) {
            ex = V[2 * e1] - V[2 * e];
            ey = V[2 * e1 + 1] - V[2 * e + 1];
            L = sqrt(ex * ex + ey * ey);
            rx = ux - V[2 * e];
            ry = uy - V[2 * e + 1];
            cross = ex * ry - ey * rx;
            const float se = sigma_f(P.sigma, kr * (float)(sgn * cross / L), ds);
            const float other = nzero == 0 ? prod / se : (se == 0.f ? prod : 0.f);
            ge = kr * ds * other * zf;  // d s / d dist_e
          }
          // d dist_e / d (x_e, y_e, x_e1, y_e1) (as the oracle's Poly2D)
          const double il = 1.0 / L, cl = cross * il * il * il;
          add(2 + 2 * e, ge * (float)(sgn * ((ey - ry) * il + cl * ex)), 0);
          add(3 + 2 * e, ge * (float)(sgn * ((rx - ex) * il + cl * ey)), 0);
          add(2 + 2 * e1, ge * (float)(sgn * (ry * il - cl * ex)), 0);
          add(3 + 2 * e1, ge * (float)(sgn * (-rx * il - cl * ey)), 0);
          gx += (double)ge * (-sgn * ey * il);
          gy += (double)ge * (sgn * ex * il);
        }
      }
    }
  }
  if (kD) {  // pivot, angle and aspect through grad_u s
    const double cth = A[0], sth = A[1], isx = A[2], isy = A[3];
    add(nb, (float)(gx * (1.0 - cth * isx) + gy * (sth * isy)), 0);
    add(nb + 1, (float)(gx * (-sth * isx) + gy * (1.0 - cth * isy)), 0);
    add(nb + 2, (float)(gx * ((-sth * wx + cth * wy) * isx) + gy * ((-cth * wx - sth * wy) * isy)), 3);
    add(nb + 3, (float)(gx * (-vx * isx * isx)), 3);
    add(nb + 4, (float)(gy * (-vy * isy * isy)), 3);
  }
  return s;
}

__device__ __noinline__ float xform_value(const PrimRec& P, const Cell& c, const double* auxd) {
  return xform_core<false>(P, c, auxd, NoAdd{});
}

// kX: the job table may hold transformed primitives (the kernels compiled
// for such tables; the others carry no transform code at all).
template <bool kX = false>
__device__ __forceinline__ float leaf_value(const PrimRec& P, const Cell& c, const float* auxf,
                                            const double* auxd) {
  if constexpr (kX) {
    if (P.kind == kXform) return xform_value(P, c, auxd);
  }
  float ds;
  if (P.kind == kBox) {
    float f[3], fa[3], fb[3];
    box_axes(P, c, f, fa, fb);
    return f[0] * f[1] * f[2];
  }
  float dz0, dz1;
  const float zf = zfactor(P, c, dz0, dz1);
  if (zf == 0.f) return 0.f;
  if (P.kind == kCircle) {
    float dxr, dyr, r;
    const float d = circle_dist(P, c, dxr, dyr, r);
    return sigma_f(P.sigma, P.kr * d, ds) * zf;
  }
  if (P.kind == kGraph) {
    int seg;
    double t;
    const float d = graph_dist(P, c, auxf, auxd, seg, t);
    return sigma_f(P.sigma, P.kr * d, ds) * zf;
  }
  if (P.kind == kPolar) return sigma_f(P.sigma, P.kr * polar_dist(P, c, auxf), ds) * zf;
  return poly_value(P, c, auxf) * zf;
}

// Nonzero d s / d q (physical units) of one leaf at one cell, times `a`, as
// (active slot, value) pairs in ascending slot order.  Columns of stride kBlock.
// Slots are per (primitive, parameter): a scalar's term is scaled by its
// coefficient and merged with the previous pair when both hit the same slot.
__device__ __forceinline__ int push_pair(const int* actp, const float* actcp, int key, float v,
                                         int n, int* pk, float* pv) {
  const int s = actp[key];
  if (s < 0 || v == 0.f) return n;
  v *= actcp[key];
  if (n > 0 && pk[(n - 1) * kBlock] == s) {
    pv[(n - 1) * kBlock] += v;
    return n;
  }
  if (n < kMaxPairs) {
    pk[n * kBlock] = s;
    pv[n * kBlock] = v;
    return n + 1;
  }
  return n;
}

// GeneralCartesian2D derivative pairs (z0, z1, X_j, X_j+1, Y_j, Y_j+1).  Not
// inlined, like graph_dist, to keep its FP64 work off the box path.
__device__ __noinline__ int graph_pairs(const PrimRec& P, const Cell& c, float a, const GridDev& g,
                                      const int* actp, const float* actcp, const float* auxf,
                                      const double* auxd, int* pk, float* pv) {
  int n = 0;
  float dz0, dz1, ds;
  const float zf = zfactor(P, c, dz0, dz1);
  int seg;
  double t;
  const float d = graph_dist(P, c, auxf, auxd, seg, t);
  const float s = sigma_f(P.sigma, P.kr * d, ds);
  const float sgn = (P.flags & kGraphAbove) ? -1.f : 1.f;
  const float gg = P.kr * ds * zf * sgn * a;  // d s / d f (per y-cell) times a
  const int M = P.naux;
  n = push_pair(actp, actcp, 0, s * dz0 * a * g.invd[2], n, pk, pv);
  n = push_pair(actp, actcp, 1, s * dz1 * a * g.invd[2], n, pk, pv);
  if (seg < 0) {
    n = push_pair(actp, actcp, 2 + M, gg * g.invd[1], n, pk, pv);
  } else if (seg >= M - 1) {
    n = push_pair(actp, actcp, 2 + M + M - 1, gg * g.invd[1], n, pk, pv);
  } else {
    const double* X = auxd + P.auxd_off;
    const double* Y = X + M;
    const double* iX = Y + M;
    const double ux = (double)c.i + (double)c.ox;
    const float dY = (float)(Y[seg + 1] - Y[seg]);
    const float ix = (float)iX[seg];
    const float e0 = (float)(ux - X[seg + 1]), e1 = (float)(ux - X[seg]);
    n = push_pair(actp, actcp, 2 + seg, gg * dY * e0 * ix * ix * g.invd[0], n, pk, pv);
    n = push_pair(actp, actcp, 3 + seg, -gg * dY * e1 * ix * ix * g.invd[0], n, pk, pv);
    n = push_pair(actp, actcp, 2 + M + seg, gg * (float)(1.0 - t) * g.invd[1], n, pk, pv);
    n = push_pair(actp, actcp, 3 + M + seg, gg * (float)t * g.invd[1], n, pk, pv);
  }
  return n;
}

__device__ __forceinline__ int leaf_pairs(const PrimRec& P, const Cell& c, float a, const GridDev& g,
                          const int* act, const float* actc, const float* auxf,
                          const double* auxd, int* pk, float* pv) {
  const int* actp = act + P.act_off;
  const float* actcp = actc + P.act_off;
  int n = 0;
  if (P.kind == kXform) return n;  // every scalar goes through xform_accumulate
  if (P.kind == kBox) {
    float f[3], fa[3], fb[3];
    box_axes(P, c, f, fa, fb);
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const float other = f[(ax + 1) % 3] * f[(ax + 2) % 3] * a * g.invd[ax];
      n = push_pair(actp, actcp, 2 * ax, fa[ax] * other, n, pk, pv);
      n = push_pair(actp, actcp, 2 * ax + 1, fb[ax] * other, n, pk, pv);
    }
    return n;
  }
  float dz0, dz1;
  const float zf = zfactor(P, c, dz0, dz1);
  float ds;
  if (P.kind == kCircle) {
    float dxr, dyr, r;
    const float d = circle_dist(P, c, dxr, dyr, r);
    const float s = sigma_f(P.sigma, P.kr * d, ds);
    const float gg = P.kr * ds * zf * a * g.invd[0];
    const float ir = r > 0.f ? 1.f / r : 0.f;
    n = push_pair(actp, actcp, 0, gg * dxr * ir, n, pk, pv);
    n = push_pair(actp, actcp, 1, gg * dyr * ir, n, pk, pv);
    n = push_pair(actp, actcp, 2, gg, n, pk, pv);
    n = push_pair(actp, actcp, 3, s * dz0 * a * g.invd[2], n, pk, pv);
    n = push_pair(actp, actcp, 4, s * dz1 * a * g.invd[2], n, pk, pv);
    return n;
  }
  if (P.kind == kGraph) return graph_pairs(P, c, a, g, actp, actcp, auxf, auxd, pk, pv);
  if (P.kind == kPolar) return n;  // every scalar goes through polar_accumulate
  // polygon: only the extrusion scalars here; vertices go through poly_accumulate
  if (actp[0] < 0 && actp[1] < 0) return n;
  const float s = poly_value(P, c, auxf);
  n = push_pair(actp, actcp, 0, s * dz0 * a * g.invd[2], n, pk, pv);
  n = push_pair(actp, actcp, 1, s * dz1 * a * g.invd[2], n, pk, pv);
  return n;
}

// ---------------------------------------------------------- classification --
__device__ __forceinline__ int cls_and(int a, int b) {
  if (a == cOUT || b == cOUT) return cOUT;
  if (a == cIN && b == cIN) return cIN;
  return cBND;
}

// exact-overlap axis: windows of samples in [lo, hi]
__device__ __forceinline__ int cls_exact(int ai0, float af0, int ai1, float af1, float lo,
                                         float hi) {
  const float a = (float)ai0 + af0, b = (float)ai1 + af1;
  if (b < lo - 0.5f - kMargin || a > hi + 0.5f + kMargin) return cOUT;
  if (a < lo - 0.5f - kMargin && b > hi + 0.5f + kMargin) return cIN;
  return cBND;
}

// sigma(u - a) sigma(b - u) at point samples u in [lo, hi], transition +-beta
__device__ __forceinline__ int cls_sigma(float a, float b, float beta, float lo, float hi) {
  if (hi < a - beta - kMargin || lo > b + beta + kMargin) return cOUT;
  if (lo > a + beta + kMargin && hi < b - beta - kMargin) return cIN;
  return cBND;
}

__device__ __forceinline__ int classify(const PrimRec& P, const float lo[3], const float hi[3],
                                        const double* auxd, const float* auxf) {
  if (P.kind == kXform) return cBND;  // inside its value tile box: evaluated per sample
  int z = cIN;
  if (P.kind != kBox && (P.flags & kBoundZ))
    z = cls_exact(P.ai[4], P.af[4], P.ai[5], P.af[5], lo[2], hi[2]);
  if (z == cOUT) return cOUT;
  if (P.kind == kBox) {
    int cl = cIN;
    for (int ax = 0; ax < 3; ++ax) {
      if (!(P.flags & (1 << ax))) continue;
      int ca;
      if (P.flags & kRectSigma)
        ca = cls_sigma((float)P.ai[2 * ax] + P.af[2 * ax], (float)P.ai[2 * ax + 1] + P.af[2 * ax + 1],
                       P.band, lo[ax], hi[ax]);
      else
        ca = cls_exact(P.ai[2 * ax], P.af[2 * ax], P.ai[2 * ax + 1], P.af[2 * ax + 1], lo[ax], hi[ax]);
      cl = cls_and(cl, ca);
      if (cl == cOUT) return cOUT;
    }
    return cl;
  }
  if (P.kind == kCircle) {
    const float cx = (float)P.ai[0] + P.af[0], cy = (float)P.ai[1] + P.af[1];
    const float nx = fmaxf(fmaxf(lo[0] - cx, cx - hi[0]), 0.f);
    const float ny = fmaxf(fmaxf(lo[1] - cy, cy - hi[1]), 0.f);
    const float fx = fmaxf(fabsf(lo[0] - cx), fabsf(hi[0] - cx));
    const float fy = fmaxf(fabsf(lo[1] - cy), fabsf(hi[1] - cy));
    const float rmin = sqrtf(nx * nx + ny * ny), rmax = sqrtf(fx * fx + fy * fy);
    const float R = P.g[0];
    if (rmin > R + P.band + kMargin) return cOUT;
    if (rmax < R - P.band - kMargin) return cls_and(cIN, z);
    return cBND;
  }
  if (P.kind == kPolar) {  // the annulus g[2] <= R(theta) <= g[1]
    const float cx = (float)P.ai[0] + P.af[0], cy = (float)P.ai[1] + P.af[1];
    const float nx = fmaxf(fmaxf(lo[0] - cx, cx - hi[0]), 0.f);
    const float ny = fmaxf(fmaxf(lo[1] - cy, cy - hi[1]), 0.f);
    const float fx = fmaxf(fabsf(lo[0] - cx), fabsf(hi[0] - cx));
    const float fy = fmaxf(fabsf(lo[1] - cy), fabsf(hi[1] - cy));
    const float rmin = sqrtf(nx * nx + ny * ny), rmax = sqrtf(fx * fx + fy * fy);
    const float slack = P.band + kMargin + 1e-5f * (1.f + fabsf(P.g[1]));
    if (rmin > P.g[1] + slack) return cOUT;
    if (rmax < P.g[2] - slack) return cls_and(cIN, z);
    return cBND;
  }
  if (P.kind == kGraph) {
    const int M = P.naux;
    const double* X = auxd + P.auxd_off;
    const double* Y = X + M;
    double fmn = 1e300, fmx = -1e300;
    for (int e = 0; e < 2; ++e) {  // f at both ends of the tile's x range
      const double x = e ? hi[0] : lo[0];
      double f;
      if (x <= X[0]) f = Y[0];
      else if (x >= X[M - 1]) f = Y[M - 1];
      else {
        int j = 0;
        while (j + 1 < M - 1 && x >= X[j + 1]) ++j;
        f = Y[j] + (Y[j + 1] - Y[j]) * (x - X[j]) / (X[j + 1] - X[j]);
      }
      fmn = fmin(fmn, f);
      fmx = fmax(fmx, f);
    }
    for (int j = 0; j < M; ++j)
      if (X[j] > lo[0] && X[j] < hi[0]) { fmn = fmin(fmn, Y[j]); fmx = fmax(fmx, Y[j]); }
    const float b = P.band + kMargin;
    if (!(P.flags & kGraphAbove)) {  // region y < f(x)
      if ((float)fmx - lo[1] < -b) return cOUT;
      if ((float)fmn - hi[1] > b) return cls_and(cIN, z);
    } else {                          // region y > f(x)
      if (hi[1] - (float)fmn < -b) return cOUT;
      if (lo[1] - (float)fmx > b) return cls_and(cIN, z);
    }
    return cBND;
  }
  if (P.kind == kPolygon) {
    // each edge's line function over the tile's sample box, relative to the
    // anchor cell; fp32 rounding (~1e-7 of the polygon's extent) stays far
    // inside the classification margin
    const int N = P.naux;
    const float* E = auxf + P.auxf_off;
    const float lx = lo[0] - (float)P.ai[0], hx = hi[0] - (float)P.ai[0];
    const float ly = lo[1] - (float)P.ai[1], hy = hi[1] - (float)P.ai[1];
    const float b = P.band + kMargin;
    bool all_in = true;
    for (int e = 0; e < N; ++e) {
      const float* Ee = E + kPolyEdgeFloats * e;
      const float nx = Ee[4], ny = Ee[6], rx = Ee[0], ry = Ee[2];
      const float ax = nx >= 0.f ? nx * (lx - rx) : nx * (hx - rx);
      const float bx = nx >= 0.f ? nx * (hx - rx) : nx * (lx - rx);
      const float ay = ny >= 0.f ? ny * (ly - ry) : ny * (hy - ry);
      const float by = ny >= 0.f ? ny * (hy - ry) : ny * (ly - ry);
      const float dmin = ax + ay, dmax = bx + by;
      if (dmax < -b) return cOUT;
      if (dmin <= b) all_in = false;
    }
    return all_in ? cls_and(cIN, z) : cBND;
  }
  return cBND;
}

// The same classification by a whole warp (every lane, same result): a
// polygon's edges or a graph's breakpoints spread over the lanes (the
// binner's walk hands these kinds to the warp; one lane takes the others).
__device__ __forceinline__ int classify_warp(const PrimRec& P, const float lo[3],
                                             const float hi[3], const double* auxd,
                                             const float* auxf, int lane) {
  if (P.kind != kPolygon && P.kind != kGraph) return classify(P, lo, hi, auxd, auxf);
  int z = cIN;
  if (P.flags & kBoundZ) z = cls_exact(P.ai[4], P.af[4], P.ai[5], P.af[5], lo[2], hi[2]);
  if (z == cOUT) return cOUT;
  if (P.kind == kPolygon) {
    const int N = P.naux;
    const float* E = auxf + P.auxf_off;
    const float lx = lo[0] - (float)P.ai[0], hx = hi[0] - (float)P.ai[0];
    const float ly = lo[1] - (float)P.ai[1], hy = hi[1] - (float)P.ai[1];
    const float b = P.band + kMargin;
    bool out = false, all_in = true;
    for (int e = lane; e < N; e += 32) {
      const float* Ee = E + kPolyEdgeFloats * e;
      const float nx = Ee[4], ny = Ee[6], rx = Ee[0], ry = Ee[2];
      const float ax = nx >= 0.f ? nx * (lx - rx) : nx * (hx - rx);
      const float bx = nx >= 0.f ? nx * (hx - rx) : nx * (lx - rx);
      const float ay = ny >= 0.f ? ny * (ly - ry) : ny * (hy - ry);
      const float by = ny >= 0.f ? ny * (hy - ry) : ny * (ly - ry);
      const float dmin = ax + ay, dmax = bx + by;
      if (dmax < -b) out = true;
      if (dmin <= b) all_in = false;
    }
    if (__any_sync(0xffffffffu, out)) return cOUT;
    return __all_sync(0xffffffffu, all_in) ? cls_and(cIN, z) : cBND;
  }
  // graph: f at both ends of the tile's x range (segment found by counting
  // breakpoints, as the sequential search does) and at the interior ones
  const int M = P.naux;
  const double* X = auxd + P.auxd_off;
  const double* Y = X + M;
  double fmn = 1e300, fmx = -1e300;
  for (int e = 0; e < 2; ++e) {
    const double x = e ? hi[0] : lo[0];
    double f;
    if (x <= X[0]) f = Y[0];
    else if (x >= X[M - 1]) f = Y[M - 1];
    else {
      int j = 0;  // the number of breakpoints 1 .. M-2 at or left of x
      for (int k0 = 1; k0 < M - 1; k0 += 32) {
        const int k = k0 + lane;
        j += __popc(__ballot_sync(0xffffffffu, k < M - 1 && x >= X[k]));
      }
      f = Y[j] + (Y[j + 1] - Y[j]) * (x - X[j]) / (X[j + 1] - X[j]);
    }
    fmn = fmin(fmn, f);
    fmx = fmax(fmx, f);
  }
  for (int j = lane; j < M; j += 32)
    if (X[j] > lo[0] && X[j] < hi[0]) { fmn = fmin(fmn, Y[j]); fmx = fmax(fmx, Y[j]); }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    fmn = fmin(fmn, __shfl_xor_sync(0xffffffffu, fmn, o));
    fmx = fmax(fmx, __shfl_xor_sync(0xffffffffu, fmx, o));
  }
  const float b = P.band + kMargin;
  if (!(P.flags & kGraphAbove)) {
    if ((float)fmx - lo[1] < -b) return cOUT;
    if ((float)fmn - hi[1] > b) return cls_and(cIN, z);
  } else {
    if (hi[1] - (float)fmn < -b) return cOUT;
    if (lo[1] - (float)fmx > b) return cls_and(cIN, z);
  }
  return cBND;
}

// Vertex derivatives of one Poly2D leaf at one sample, accumulated edge by
// edge.  s = zf prod_e sigma(k d_e); d s / d d_e uses the product of the other
// factors (with an exact zero count, no division by zero).  Each edge adds to
// the slots of its two vertices' x and y scalars; slots are warp-uniform, so a
// two-entry register cache merges consecutive edges on the same parameter
// (a translated polygon needs two warp reductions per sample, not 4 N).
__device__ __forceinline__ void flush_slot(int& slot, float& v, float* acc, float* cmp, int lane);

__device__ __noinline__ void poly_accumulate(const PrimRec& P, const Cell& c, float a, const GridDev& g,
                                const int* act, const float* actc, const float* auxf,
                                float* acc, float* cmp, int lane) {
  const int N = P.naux;
  const float* E = auxf + P.auxf_off;
  const int* actp = act + P.act_off;
  const float* actcp = actc + P.act_off;
  float ux, uy;
  poly_rel(P, c, ux, uy);
  float dz0, dz1;
  const float zf = a != 0.f ? zfactor(P, c, dz0, dz1) : 0.f;
  float prod = 1.f, ds;
  int nz = 0;
  if (zf != 0.f) {
    for (int e = 0; e < N; ++e) {
      const float s = sigma_f(P.sigma, P.kr * poly_d(E + kPolyEdgeFloats * e, ux, uy), ds);
      if (s == 0.f) { if (++nz > 1) break; }
      else prod *= s;
    }
  }
  const bool live = zf != 0.f && nz <= 1;
  const float sgn = P.g[0];
  const float scale = a * zf * P.kr * g.invd[0];
  int cs0 = -1, cs1 = -1;
  float cv0 = 0.f, cv1 = 0.f;
  for (int e = 0; e < N; ++e) {
    const int e1 = e + 1 == N ? 0 : e + 1;
    float ge = 0.f, d = 0.f;
    const float* Ee = E + kPolyEdgeFloats * e;
    if (live) {
      d = poly_d(Ee, ux, uy);
      const float se = sigma_f(P.sigma, P.kr * d, ds);
      const float other = nz == 0 ? prod / se : (se == 0.f ? prod : 0.f);
      ge = scale * ds * other;
    }
    if (!__any_sync(0xffffffffu, ge != 0.f)) continue;
    // d(d_e)/d(x_e, y_e, x_e1, y_e1) in cells (see the oracle's Poly2D)
    const float ex = Ee[8], ey = Ee[9];
    const float rx = (ux - Ee[0]) - Ee[1], ry = (uy - Ee[2]) - Ee[3];
    const float il = Ee[10];
    const float dil = d * il * il;
    const float t[4] = {sgn * (ey - ry) * il + dil * ex, sgn * (rx - ex) * il + dil * ey,
                        sgn * ry * il - dil * ex, -sgn * rx * il - dil * ey};
    const int key[4] = {2 + 2 * e, 3 + 2 * e, 2 + 2 * e1, 3 + 2 * e1};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int slot = actp[key[u]];
      if (slot < 0) continue;
      const float v = ge * t[u] * actcp[key[u]];
      if (slot == cs0) cv0 += v;
      else if (slot == cs1) cv1 += v;
      else {
        flush_slot(cs0, cv0, acc, cmp, lane);
        cs0 = cs1; cv0 = cv1;
        cs1 = slot; cv1 = v;
      }
    }
  }
  flush_slot(cs0, cv0, acc, cmp, lane);
  flush_slot(cs1, cv1, acc, cmp, lane);
}

// Polar2D's derivative terms at one sample, every scalar (keys cx, cy, R0, z0,
// z1, c_1, s_1, ..., c_N, s_N): d/dR0 = 1, d/dc_n = cos(n theta), d/ds_n =
// sin(n theta), d/dcx = cos theta + R'(theta) sin theta / r and d/dcy =
// sin theta - R'(theta) cos theta / r (0 at r = 0), times kr sigma' zf a / d;
// z0, z1 through the extrusion.  The distance inside sigma is FP64
// (polar_dist); the angle factors are fp32 (hi parts of the coefficients).
// Warp-uniform slots, merged by the same two-entry cache as the polygon's.
__device__ __forceinline__ void polar_accumulate(const PrimRec& P, const Cell& c, float a,
                                              const GridDev& g, const int* act, const float* actc,
                                              const float* auxf, float* acc, float* cmp,
                                              int lane) {
  const int* actp = act + P.act_off;
  const float* actcp = actc + P.act_off;
  float dz0 = 0.f, dz1 = 0.f, s = 0.f, ds = 0.f;
  const float zf = a != 0.f ? zfactor(P, c, dz0, dz1) : 0.f;
  if (zf != 0.f) s = sigma_f(P.sigma, P.kr * polar_dist(P, c, auxf), ds);
  const float gg = P.kr * ds * zf * a * g.invd[0];
  const float gz = s * a * g.invd[2];
  if (!__any_sync(0xffffffffu, gg != 0.f || gz != 0.f)) return;
  // the angle terms in fp32: they scale derivatives, not the distance
  const float dx = i2f(c.i - P.ai[0]) + (c.ox - P.af[0]);
  const float dy = i2f(c.j - P.ai[1]) + (c.oy - P.af[1]);
  const float r = sqrtf(dx * dx + dy * dy);
  const float ir = r > 0.f ? 1.f / r : 0.f;
  const float cth = r > 0.f ? dx * ir : 1.f, sth = r > 0.f ? dy * ir : 0.f;
  const float* F = auxf + P.auxf_off;
  float dR = 0.f, cn = cth, sn = sth;
  for (int n = 1; n <= P.naux; ++n) {
    dR += (float)n * (F[4 * n] * cn - F[4 * n - 2] * sn);
    const float c2 = cn * cth - sn * sth, s2 = sn * cth + cn * sth;
    cn = c2;
    sn = s2;
  }
  // one warp reduction per driven scalar, in key order (slots are warp-uniform)
  const int nq = 5 + 2 * P.naux;
  cn = cth;
  sn = sth;
  for (int key = 0; key < nq; ++key) {
    float v;
    if (key == 0) v = gg * (r > 0.f ? cth + dR * sth * ir : 0.f);
    else if (key == 1) v = gg * (r > 0.f ? sth - dR * cth * ir : 0.f);
    else if (key == 2) v = gg;
    else if (key == 3) v = gz * dz0;
    else if (key == 4) v = gz * dz1;
    else if (key & 1) v = gg * cn;
    else {
      v = gg * sn;
      const float c2 = cn * cth - sn * sth, s2 = sn * cth + cn * sth;
      cn = c2;
      sn = s2;
    }
    int slot = actp[key];
    if (slot < 0) continue;
    v *= actcp[key];
    flush_slot(slot, v, acc, cmp, lane);
  }
}

// The VJP's call for the kinds whose scalars are not all keyed, in designs
// with Polar2D primitives: polygon vertices and every Polar2D scalar (other
// designs call poly_accumulate directly, so their sample loop is unchanged).
// A transformed primitive's terms at one sample (every scalar, key order,
// from xform_core) times a, to physical units; one warp reduction per
// driven slot, merged by the same two-entry cache as the polygon's.
__device__ __forceinline__ void xform_accumulate(const PrimRec& P, const Cell& c, float a,
                                                 const GridDev& g, const int* act,
                                                 const float* actc, const double* auxd,
                                                 float* acc, float* cmp, int lane) {
  const int* actp = act + P.act_off;
  const float* actcp = actc + P.act_off;
  int cs0 = -1, cs1 = -1;
  float cv0 = 0.f, cv1 = 0.f;
  const float unit[4] = {g.invd[0] * a, g.invd[1] * a, g.invd[2] * a, a};
  auto add = [&](int key, float v, int u) {
    const int slot = actp[key];
    if (slot < 0) return;
    v *= unit[u] * actcp[key];
    if (slot == cs0) cv0 += v;
    else if (slot == cs1) cv1 += v;
    else {
      flush_slot(cs0, cv0, acc, cmp, lane);
      cs0 = cs1; cv0 = cv1;
      cs1 = slot; cv1 = v;
    }
  };
  xform_core<true>(P, c, auxd, add);
  flush_slot(cs0, cv0, acc, cmp, lane);
  flush_slot(cs1, cv1, acc, cmp, lane);
}

// The VJP's one out-of-line call for the kinds whose scalars are not all
// keyed: polygon vertices, every Polar2D scalar (job tables with Polar2D
// only) and every scalar of a transformed primitive.
__device__ __noinline__ void shape_accumulate(const PrimRec& P, const Cell& c, float a,
                                              const GridDev& g, const int* act, const float* actc,
                                              const float* auxf, const double* auxd, float* acc,
                                              float* cmp, int lane) {
  if (P.kind == kPolar) polar_accumulate(P, c, a, g, act, actc, auxf, acc, cmp, lane);
  else if (P.kind == kXform) xform_accumulate(P, c, a, g, act, actc, auxd, acc, cmp, lane);
  else poly_accumulate(P, c, a, g, act, actc, auxf, acc, cmp, lane);
}

// --------------------------------------------------------------- kernels ---
// Fold-stack entry (16 bits): kind (0 = const 0, 1 = const 1, 2 = expression)
// | root << 2 | start << 9 (root: position of the expression's last op;
// start: its first; 7-bit fields, both < kMaxOps).
__device__ __forceinline__ int mkE(int root, int start) { return 2 | (root << 2) | (start << 9); }

// Folded op words (code 2 bits, operands 7 bits; complement = difference(kOne, b)).
__device__ __forceinline__ int mk_op(int code, int a, int b) { return code | (a << 2) | (b << 9); }
struct FoldOp {
  int code, a, b;  // complement: code fCompl, operand in a
};
__device__ __forceinline__ FoldOp fold_op(int op) {
  FoldOp f{op & 3, (op >> 2) & 127, (op >> 9) & 127};
  if (f.code == fDiff && f.a == kOne) { f.code = fCompl; f.a = f.b; }
  return f;
}

// First job whose range end exceeds idx (ends are nondecreasing).
__device__ __forceinline__ int job_by_tile(const Job* jobs, int n, int idx) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const Job& J = jobs[mid];
    const int end = J.tile_base + (((J.g.T + 127) >> 7) << 7);
    if (end > idx) hi = mid; else lo = mid + 1;
  }
  return lo;
}

__device__ __forceinline__ int job_by_param(const Job* jobs, int n, int idx) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const Job& J = jobs[mid];
    if (J.param_base + (J.do_grad ? J.nparam : 0) > idx) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// Programmatic dependent launch: the build, the VJP and the finalize may be
// launched to overlap the tail of the kernel before them on the stream (the
// launch, block scheduling and a prologue that reads only tables uploaded
// before that kernel).  They wait here for it to complete, and for its
// memory to be visible, before reading anything it may have written; a
// kernel launched without the attribute returns from this at once.
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---- binner: one warp per tile ------------------------------------------------
// A block takes kBinWarps consecutive tiles of one job (y fastest: tiles that
// differ only in y usually see the same primitives).  The chain is walked in
// segments: the block first drops, for all its tiles at once, the push of a
// primitive that misses the block's tile box together with a union or
// difference right after it (union(A, 0) = difference(A, 0) = A); then each
// warp walks the rest for its tile 32 words at a time -- the lanes test the
// tile box, drop the same pairs for the tile, and classify the remaining
// pushes in parallel -- and lane 0 folds them with the constants (the fold
// is sequential, the classification is not).
constexpr int kBinWarps = 16;
constexpr int kBinThreads = 32 * kBinWarps;
constexpr int kBinSeg = 4096;  // chain words compacted per block pass
static_assert(kBinSeg % kBinThreads == 0 && 128 % kBinWarps == 0, "binner layout");
struct BinWarpBuf {
  int word[32];              // the round's kept chain words
  unsigned char cls[32];     // their classes (pushes)
  uint16_t stk[kMaxDepth];   // fold stack below the three register entries
  uint16_t leaf[kMaxLeaves];
  uint16_t ops[kMaxOps];
};
// the tile boxes of the first kBinTbCache primitives, cached per block
constexpr int kBinTbCache = kBinThreads;
constexpr size_t kBinSmem =
    sizeof(int) * kBinSeg + sizeof(BinWarpBuf) * kBinWarps + sizeof(int) * 6 * kBinTbCache;

__device__ __forceinline__ bool tb_hits(const int* tb, int x0, int x1, int y0, int y1, int z0,
                                        int z1) {  // tile box [x0, x1] x ... against tb
  return x0 < __ldg(tb + 1) && x1 >= __ldg(tb) && y0 < __ldg(tb + 3) && y1 >= __ldg(tb + 2) &&
         z0 < __ldg(tb + 5) && z1 >= __ldg(tb + 4);
}
__device__ __forceinline__ bool is_ud(int word) {
  const int c = (word >> 24) & 0xff;
  return c == cUnion || c == cDiff;
}

// Lane 0's fold state of one tile.
struct Fold {
  int sp, r0, r1, r2;  // stack depth; top three entries (deeper ones in stk)
  int nops, nleaf, e;
};

// One chain word of the tile (lane 0): a push with its class, or a logic op
// folded with the constants (Eqs. union / intersection / difference on 0/1).
// uniq: no primitive is pushed twice by the chain, so a band push is a new leaf.
__device__ __forceinline__ void fold_word(Fold& f, int word, int cl, BinWarpBuf& B, bool uniq) {
  const int code = (word >> 24) & 0xff, arg = word & 0xffffff;
  if (code == cPush) {
    int ent = 0;
    if (cl == cBND) {
      int slot = -1;
      if (!uniq)
        for (int l = 0; l < f.nleaf; ++l)
          if (B.leaf[l] == arg) { slot = l; break; }
      if (slot < 0) {
        if (f.nleaf < kMaxLeaves) { B.leaf[f.nleaf] = (uint16_t)arg; slot = f.nleaf++; }
        else f.e |= eLeafOverflow;
      }
      if (slot >= 0 && f.nops < kMaxOps) {
        B.ops[f.nops] = (uint16_t)mk_op(fPush, slot, 0);
        ent = mkE(f.nops, f.nops);
        ++f.nops;
      } else {
        f.e |= eOpsOverflow;
      }
    } else {
      ent = (cl == cIN) ? 1 : 0;
    }
    if (f.sp < kMaxDepth) {
      if (f.sp >= 3) B.stk[f.sp - 3] = (uint16_t)f.r2;
      f.r2 = f.r1;
      f.r1 = f.r0;
      f.r0 = ent;
      ++f.sp;
    } else {
      f.e |= eDepthOverflow;
    }
    return;
  }
  if (f.sp < 2) { f.e |= eBadProgram; return; }
  const int B0 = f.r0, A = f.r1;
  const int ka = A & 3, kb = B0 & 3;
  const int ra = (A >> 2) & 127, sa = (A >> 9) & 127;
  const int rb = (B0 >> 2) & 127, sb = (B0 >> 9) & 127;
  int res = 0, emit = -1, unary = 0;
  bool discard = false;
  if (code == cUnion) {
    if (ka == 1 || kb == 1) { res = 1; discard = true; }
    else if (ka == 0) res = B0;
    else if (kb == 0) res = A;
    else emit = fUnion;
  } else if (code == cInter) {
    if (ka == 0 || kb == 0) { res = 0; discard = true; }
    else if (ka == 1) res = B0;
    else if (kb == 1) res = A;
    else emit = fInter;
  } else {  // difference
    if (ka == 0 || kb == 1) { res = 0; discard = true; }
    else if (kb == 0) res = A;
    else if (ka == 1) { emit = fCompl; unary = 1; }
    else emit = fDiff;
  }
  if (discard) {  // the dropped operand's ops were the last ones emitted
    if (ka == 2) f.nops = sa;
    else if (kb == 2) f.nops = sb;
  }
  if (emit >= 0) {
    if (f.nops < kMaxOps) {
      if (unary) {
        B.ops[f.nops] = (uint16_t)mk_op(fDiff, kOne, rb);
        res = mkE(f.nops, sb);
      } else {
        B.ops[f.nops] = (uint16_t)mk_op(emit, ra, rb);
        res = mkE(f.nops, sa);
      }
      ++f.nops;
    } else {
      f.e |= eOpsOverflow;
      res = 0;
    }
  }
  f.r0 = res;  // two popped, one pushed: the fourth entry comes back from memory
  f.r1 = f.r2;
  f.r2 = f.sp >= 4 ? (int)B.stk[f.sp - 4] : 0;
  --f.sp;
}

__global__ void __launch_bounds__(kBinThreads) k_bin(const Job* __restrict__ jobs, int njobs,
                                                     int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem[];
  int* schain = reinterpret_cast<int*>(smem);
  BinWarpBuf* wbuf = reinterpret_cast<BinWarpBuf*>(schain + kBinSeg);
  int* stb = reinterpret_cast<int*>(wbuf + kBinWarps);  // cached primitive tile boxes
  __shared__ int wtot[kBinWarps];
  __shared__ int sband[kBinWarps];  // the block's band tiles
  __shared__ int sagg[4];           // band tiles, longest program, band cells, list base
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g0 = blockIdx.x * kBinWarps;  // first tile (padded numbering) of the block
  const Job& J = jobs[job_by_tile(jobs, njobs, g0)];
  if (!J.do_bin) return;  // uniform over the block
  // this binning counts into J.counters (zeroed by the previous one) and
  // clears the other set for the next
  if (tid < 4 && g0 == J.tile_base) J.counters_next[tid] = 0;
  const int nty = J.g.nty, ntx = J.g.ntx;
  const int ub0 = g0 - J.tile_base;
  if (ub0 >= J.g.T) return;  // padding block (uniform)
  const int ub1 = min(ub0 + kBinWarps, J.g.T) - 1;
  const PrimRec* __restrict__ prims = J.prims;
  const int* __restrict__ chain = J.chain;
  // the block's box of tile coordinates
  int bx0 = 0, bx1 = ntx - 1, by0 = 0, by1 = nty - 1;
  const int bz0 = ub0 / (nty * ntx), bz1 = ub1 / (nty * ntx);
  if (bz0 == bz1) {
    bx0 = (ub0 / nty) % ntx;
    bx1 = (ub1 / nty) % ntx;
    if (bx0 == bx1) { by0 = ub0 % nty; by1 = ub1 % nty; }
  }
  if (tid < 4) sagg[tid] = 0;
  // the first kBinTbCache primitives' tile boxes into shared memory (one per
  // thread), testing them against the block's box on the way
  const int nprims = J.g.nprims;
  auto box_hits = [](const int* b, int x0, int x1, int y0, int y1, int z0, int z1) {
    return x0 < b[1] && x1 >= b[0] && y0 < b[3] && y1 >= b[2] && z0 < b[5] && z1 >= b[4];
  };
  bool hit = false;
  if (tid < nprims && tid < kBinTbCache) {
    int b[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      b[k] = __ldg(prims[tid].tb + k);
      stb[6 * tid + k] = b[k];
    }
    hit = box_hits(b, bx0, bx1, by0, by1, bz0, bz1);
  }
  for (int q = tid + kBinTbCache; q < nprims && !hit; q += kBinThreads)
    hit = tb_hits(prims[q].tb, bx0, bx1, by0, by1, bz0, bz1);
  const bool any = __syncthreads_or(hit);  // also publishes the cache
  const int u = ub0 + warp;
  const bool live = u < J.g.T;  // warp-uniform
  const int ty = u % nty, tx = (u / nty) % ntx, tz = u / (nty * ntx);
  const int t = (tz * nty + ty) * ntx + tx;
  if (!any) {  // no primitive reaches the block: every tile folds to the constant 0
    if (live && lane == 0) J.tclass[t] = 0;  // build and VJP read only the class and the list
    return;
  }
  const int lx = J.g.lx, ly = J.g.ly, lz = J.g.lz;
  const int i0 = tx << lx, j0 = ty << ly, k0 = tz << lz;
  const int i1 = min(J.g.nx, (tx + 1) << lx), j1 = min(J.g.ny, (ty + 1) << ly),
            k1 = min(J.g.nz, (tz + 1) << lz);
  const float lo[3] = {i0 + J.g.offmin[0], j0 + J.g.offmin[1], k0 + J.g.offmin[2]};
  const float hi[3] = {(i1 - 1) + J.g.offmax[0], (j1 - 1) + J.g.offmax[1], (k1 - 1) + J.g.offmax[2]};
  BinWarpBuf& B = wbuf[warp];
  Fold f{0, 0, 0, 0, 0, 0, 0};
  const int nchain = J.g.nchain;
  auto hits = [&](int p, int x0, int x1, int y0, int y1, int z0, int z1) {
    return p < kBinTbCache ? box_hits(stb + 6 * p, x0, x1, y0, y1, z0, z1)
                           : tb_hits(prims[p].tb, x0, x1, y0, y1, z0, z1);
  };
  auto misses_block = [&](int word) {
    return ((word >> 24) & 0xff) == cPush && !hits(word & 0xffffff, bx0, bx1, by0, by1, bz0, bz1);
  };
  auto misses_tile = [&](int word) {
    return ((word >> 24) & 0xff) == cPush && !hits(word & 0xffffff, tx, tx, ty, ty, tz, tz);
  };
  const bool uniq = J.g.unique_push != 0;
  for (int s0 = 0; s0 < nchain; s0 += kBinSeg) {
    const int s1 = min(nchain, s0 + kBinSeg);
    // block pass, one word per thread and slab: the segment's words minus
    // the pairs that miss the block, in order
    int n = 0;
    __syncthreads();  // the previous segment's walks are done with schain
    for (int w0 = s0; w0 < s1; w0 += kBinThreads) {
      const int w = w0 + tid;
      int word = 0;
      bool keep = false;
      if (w < s1) {
        word = __ldg(chain + w);
        keep = !((w + 1 < nchain && is_ud(__ldg(chain + w + 1)) && misses_block(word)) ||
                 (w >= 1 && is_ud(word) && misses_block(__ldg(chain + w - 1))));
      }
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (lane == 0) wtot[warp] = __popc(m);
      __syncthreads();  // warp counts of this slab
      int off = n, tot = 0;
      for (int v = 0; v < kBinWarps; ++v) {
        if (v < warp) off += wtot[v];
        tot += wtot[v];
      }
      if (keep) schain[off + __popc(m & ((1u << lane) - 1u))] = word;
      n += tot;
      __syncthreads();  // this slab's words are in place; wtot is free again
    }
    if (live) {
      for (int r = 0; r < n; r += 32) {
        const int i = r + lane;
        int word = 0, cl = cOUT;
        bool kept = false, defer = false;
        if (i < n) {
          word = schain[i];
          if (((word >> 24) & 0xff) == cPush) {
            const bool miss = misses_tile(word);
            kept = !miss || !(i + 1 < n && is_ud(schain[i + 1]));
            if (!miss) {
              const PrimRec& R = prims[word & 0xffffff];
              const int kind = R.kind;
              if (kind == kPolygon || kind == kGraph) defer = true;
              else cl = classify(R, lo, hi, J.auxd, J.auxf);
            }
          } else {
            kept = !(i >= 1 && is_ud(word) && misses_tile(schain[i - 1]));
          }
        }
        // polygons and graphs: classified by the whole warp, one at a time
        for (unsigned dm = __ballot_sync(0xffffffffu, defer); dm; dm &= dm - 1) {
          const int src = __ffs(dm) - 1;
          const int wd = __shfl_sync(0xffffffffu, word, src);
          const int c = classify_warp(prims[wd & 0xffffff], lo, hi, J.auxd, J.auxf, lane);
          if (lane == src) cl = c;
        }
        const unsigned km = __ballot_sync(0xffffffffu, kept);
        if (kept) {
          const int p = __popc(km & ((1u << lane) - 1u));
          B.word[p] = word;
          B.cls[p] = (unsigned char)cl;
        }
        __syncwarp();
        if (lane == 0)
          for (int j = 0; j < __popc(km); ++j) fold_word(f, B.word[j], B.cls[j], B, uniq);
        __syncwarp();
      }
    }
  }
  // the tile's program: constant, or band ops over its leaves
  int nops = 0, nleaf = 0, e = 0;
  float cval = 0.f;
  if (lane == 0) {
    if (f.sp != 1) f.e |= eBadProgram;
    const int fin = f.sp >= 1 ? f.r0 : 0;
    nops = f.nops;
    if ((fin & 3) != 2) { nops = 0; cval = (fin & 3) ? 1.f : 0.f; }
    nleaf = f.nleaf;
    e = f.e;
  }
  nops = __shfl_sync(0xffffffffu, nops, 0);
  nleaf = __shfl_sync(0xffffffffu, nleaf, 0);
  e = __shfl_sync(0xffffffffu, e, 0);
  cval = __shfl_sync(0xffffffffu, cval, 0);
  int nslot = 0;
  bool pairs = false;  // a graph or polygon leaf: the VJP reserves pair columns
  if (live && nops > 0) {
    for (int l = lane; l < nleaf; l += 32) {
      const PrimRec& L = prims[B.leaf[l]];
      nslot += L.nact;
      pairs |= L.kind == kGraph || L.kind == kPolygon;
    }
    nslot = __reduce_add_sync(0xffffffffu, nslot);
    pairs = __any_sync(0xffffffffu, pairs);
    if (nslot > kMaxSlots) e |= eSlotOverflow;
    if (pool_need(nleaf, kWarps * nslot, nops) + (pairs ? kPairFloats : 0) + kPoolSpare > kVjpPool)
      e |= ePoolOverflow;
  }
  if (live && e) {
    if (lane == 0) atomicOr(err, e);
    nops = 0;
    cval = 0.f;
  }
  const bool band = live && nops > 0;
  if (band) {  // constant tiles keep only their class
    TileProg* out = J.progs + t;
    for (int l = lane; l < nleaf; l += 32) out->leaf[l] = B.leaf[l];
    for (int q = lane; q < nops; q += 32) out->ops[q] = B.ops[q];
    if (lane == 0) {
      out->nops = nops;
      out->nleaf = nleaf;
      out->cval = cval;
      out->nslot = nslot;
      out->pairs = pairs;
      const int pos = atomicAdd(&sagg[0], 1);
      sband[pos] = t;
      atomicMax(&sagg[1], nops);
      atomicAdd(&sagg[2], (i1 - i0) * (j1 - j0) * (k1 - k0));
    }
  }
  if (live && lane == 0) J.tclass[t] = band ? 2 : (cval != 0.f ? 1 : 0);
  // the block's band tiles into the list: one set of global atomics per block
  // (the list order is free)
  __syncthreads();
  const int nb = sagg[0];
  if (nb == 0) return;  // uniform
  if (tid == 0) {
    sagg[3] = atomicAdd(&J.counters[0], nb);
    atomicMax(&J.counters[1], sagg[1]);
    atomicAdd(&J.counters[2], sagg[2]);
  }
  __syncthreads();
  if (tid < nb && ADG_CHECK(sagg[3] + tid < J.g.T, J.err)) J.list[sagg[3] + tid] = sband[tid];
}

// Threads [tid0, tid0 + nthr) of the block, one 16-byte word at a time:
// the tile's primitive records into shared memory.
__device__ __forceinline__ void stage_tile(const TileProg* P, const PrimRec* prims, int nleaf,
                                           PrimRec* sl, int tid, int nthr) {
  constexpr int W = sizeof(PrimRec) / 16;
  for (int q = tid; q < nleaf * W; q += nthr) {
    const int l = q / W, w = q - l * W;
    reinterpret_cast<int4*>(sl + l)[w] = reinterpret_cast<const int4*>(prims + P->leaf[l])[w];
  }
}

// ---- per-tile factor tables ------------------------------------------------
// Late projection to the grid (Sec. 3, item (iii)): a leaf's value factors as
// s(c, x, y, z) = A(c, x, y) * Z(c, z), and for a box A = X(c, x) * Y(c, y)
// (Table 4: RectdD is a product of Rect1D factors; Sec. 5.2: planarity is a
// z factor).  Each tile evaluates every factor once per (component,
// coordinate) into shared memory; a sample's leaf value is then two or three
// table reads.  Leaves that do not fit the table pool are evaluated directly.
struct __align__(16) LeafTab {
  int4 v;         // value tables x, y, z, xy (offsets in floats), -1 if absent
  int4 d;         // derivative tables dx, dy, dz (lo, hi per component); w = flags
  int slot[6];    // box: accumulator slot and map coefficient of scalar k
  float coef[6];
};
// LeafTab.d.w flags
constexpr int tOK = 1, tBOX = 2, tACT = 4;  // tabled, box, drives some parameter
constexpr int tKEYS = 8;                     // bits 8..13: box scalars driving a parameter

// Axis factor of a box along axis `ax` at cell index i with offset off:
// exact overlap, or the paper's sigma product; unbounded axes give 1.
__device__ __forceinline__ float box_axis(const PrimRec& P, int ax, int i, float off, float& da,
                                          float& db) {
  if (!(P.flags & (1 << ax))) { da = 0.f; db = 0.f; return 1.f; }
  if (P.flags & kRectSigma) {
    const float ta = i2f(P.ai[2 * ax] - i) + (P.af[2 * ax] - off);
    const float tb = i2f(P.ai[2 * ax + 1] - i) + (P.af[2 * ax + 1] - off);
    float d1, d2;
    const float s1 = sigma_f(P.sigma, -P.kr * ta, d1);
    const float s2 = sigma_f(P.sigma, P.kr * tb, d2);
    da = -P.kr * d1 * s2;
    db = s1 * P.kr * d2;
    return s1 * s2;
  }
  return ov_exact(P.ai[2 * ax], P.af[2 * ax], P.ai[2 * ax + 1], P.af[2 * ax + 1], i, off, da, db);
}

// In-plane factor of a circle / graph / polar shape / polygon at (i, j) (no z factor).
__device__ __forceinline__ float plane_value(const PrimRec& P, const Cell& c, const float* auxf,
                                             const double* auxd) {
  float ds;
  if (P.kind == kCircle) {
    float dxr, dyr, r;
    return sigma_f(P.sigma, P.kr * circle_dist(P, c, dxr, dyr, r), ds);
  }
  if (P.kind == kGraph) {
    int seg;
    double t;
    return sigma_f(P.sigma, P.kr * graph_dist(P, c, auxf, auxd, seg, t), ds);
  }
  if (P.kind == kPolar) return sigma_f(P.sigma, P.kr * polar_dist(P, c, auxf), ds);
  return poly_value(P, c, auxf);  // (transformed leaves are never tabled)
}

// All threads: fill the planned tables of the tile with origin (X0, Y0, Z0).
// On the way, each thread checks its y and z entries of boxes and z entries
// of the other leaves against the entry at y = 0 (z = 0), recomputed (the
// same function of the same inputs, so bitwise what that thread wrote):
// okY / okZ start the collapse test that uniform_finish completes.  With
// act1 (VJP), a box entry whose keyed derivative is nonzero marks its
// (axis, component, coordinate) active; act1 is cleared beforehand.
__device__ __forceinline__ void tables_fill(const PrimRec* sl, int nleaf, const GridDev& g,
                                            const LeafTab* lt, bool derivs, int X0, int Y0,
                                            int Z0, float* tab, int tid, const float* auxf,
                                            const double* auxd, unsigned char* act1, bool& okY,
                                            bool& okZ) {
  const int TX = 1 << g.lx, TY = 1 << g.ly, TZ = 1 << g.lz, C = g.C;
  okY = true;
  okZ = true;
  // boxes: every (leaf, entry) pair of the tabled boxes over all the threads at
  // once (a leaf's entries alone leave most threads idle in its last round)
  const int tbx = C * (TX + TY + TZ);
  for (int q = tid; q < nleaf * tbx; q += kBlock) {
    const int l = q / tbx, e = q - l * tbx;
    const int4 tv = lt[l].v, td = lt[l].d;
    if ((td.w & (tOK | tBOX)) != (tOK | tBOX)) continue;
    const PrimRec& P = sl[l];
    // axis, component and coordinate of entry e (x block, y block, z block)
    int ax = 0, r = e, T = TX, O = X0;
    if (r >= C * TX) { r -= C * TX; ax = 1; T = TY; O = Y0; }
    if (ax == 1 && r >= C * TY) { r -= C * TY; ax = 2; T = TZ; O = Z0; }
    const int c = r / T, u = r - c * T;
    float da, db;
    const float f = box_axis(P, ax, O + u, g.off[c][ax], da, db);
    const int vt = ax == 0 ? tv.x : (ax == 1 ? tv.y : tv.z);
    tab[vt + c * T + u] = f;
    if (derivs) {
      const int dt = ax == 0 ? td.x : (ax == 1 ? td.y : td.z);
      tab[dt + (2 * c) * T + u] = da;
      tab[dt + (2 * c + 1) * T + u] = db;
      const int k = (td.w >> (3 + 2 * ax)) & 3;
      if (act1 && (td.w & tACT) && (((k & 1) && da != 0.f) || ((k & 2) && db != 0.f)))
        act1[e] = 1;
    }
    if (ax > 0 && u > 0) {
      float da0, db0;
      const float f0 = box_axis(P, ax, O, g.off[c][ax], da0, db0);
      const bool same = f == f0 && (!derivs || (da == da0 && db == db0));
      if (ax == 1) okY &= same; else okZ &= same;
    }
  }
  // the other tabled leaves: in-plane table and z factor
  for (int l = 0; l < nleaf; ++l) {
    const int4 tv = lt[l].v, td = lt[l].d;
    if ((td.w & (tOK | tBOX)) != tOK) continue;
    const PrimRec& P = sl[l];
    {
      const int nxy = C * TX * TY;
      for (int e = tid; e < nxy + C * TZ; e += kBlock) {
        if (e < nxy) {
          const int c = e / (TX * TY), r = e - c * TX * TY, v = r / TX, u = r - v * TX;
          const Cell cc{X0 + u, Y0 + v, Z0, g.off[c][0], g.off[c][1], g.off[c][2]};
          tab[tv.w + e] = plane_value(P, cc, auxf, auxd);
        } else {
          const int r = e - nxy, c = r / TZ, u = r - c * TZ;
          const Cell cc{X0, Y0, Z0 + u, g.off[c][0], g.off[c][1], g.off[c][2]};
          float dz0, dz1;
          const float zf = zfactor(P, cc, dz0, dz1);
          tab[tv.z + r] = zf;
          if (derivs) {
            tab[td.z + (2 * c) * TZ + u] = dz0;
            tab[td.z + (2 * c + 1) * TZ + u] = dz1;
          }
          if (u > 0) {
            const Cell c0{X0, Y0, Z0, g.off[c][0], g.off[c][1], g.off[c][2]};
            float e0, e1;
            const float z0 = zfactor(P, c0, e0, e1);
            okZ &= zf == z0 && (!derivs || (dz0 == e0 && dz1 == e1));
          }
        }
      }
    }
  }
}

struct TileLoc {
  int x, y, z, c;  // local coordinates of the sample in the tile
  int TX, TY, TZ;
};

static_assert(sizeof(LeafTab) == kLeafTabBytes, "pool accounting");
// job-prefix entries in shared memory: a class for small tables, one for any
__host__ __device__ constexpr int spre_len(int njobs) { return (njobs + 16) & ~15; }
constexpr size_t kBuildFixed = (size_t)kMaxDepth * kBlock * 4 + (size_t)kBuildPool * 4 +
                               kMaxOps * 16 + 16;
size_t build_smem(int njobs) { return kBuildFixed + 2 * (size_t)spre_len(njobs) * 4; }

// Pool carve of one tile: staged leaves, descriptors, then (VJP) accumulators.
struct TilePool {
  PrimRec* sl;
  LeafTab* lt;
  float* acc;
  float* cmp;
  float* tab;
  int cap;
};
__device__ __forceinline__ TilePool carve_pool(float* pool, int size, int nleaf, int nacc) {
  TilePool t;
  t.sl = reinterpret_cast<PrimRec*>(pool);
  t.lt = reinterpret_cast<LeafTab*>(t.sl + nleaf);
  t.acc = reinterpret_cast<float*>(t.lt + nleaf);
  t.cmp = t.acc + nacc;
  const int used = pool_need(nleaf, nacc, 0);  // <= size - kPoolSpare
  t.tab = pool + used;
  t.cap = size - used;
  return t;
}

// All threads (a block-wide scan; ends with a barrier): spre[j] = prefix of
// the band-tile counts of the jobs that take part, spre[njobs] = the total;
// with rpre, also rpre[j] = job j's first fill unit, rpre[njobs] = nfill.
__device__ __forceinline__ void job_prefix(const Job* jobs, int njobs, bool grad, int* spre,
                                           int* rpre = nullptr, int nfill = 0) {
  __shared__ int wsum[kWarps];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool part = tid < kBlock;  // threads past the first kBlock only meet the barriers
  int run = 0;
  for (int b0 = 0; b0 < njobs; b0 += kBlock) {
    const int j = b0 + tid;
    int cnt = 0;
    if (part && j < njobs) {
      const Job& J = jobs[j];
      if (grad ? J.do_grad : J.do_build) cnt = J.counters[0];
      if (rpre) rpre[j] = J.row_base;
    }
    int inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += u;
    }
    if (part && lane == 31) wsum[warp] = inc;
    __syncthreads();
    int off = run;
    for (int w = 0; w < warp && w < kWarps; ++w) off += wsum[w];
    if (part && j < njobs) spre[j] = off + inc - cnt;
    for (int w = 0; w < kWarps; ++w) run += wsum[w];
    __syncthreads();
  }
  if (tid == 0) {
    spre[njobs] = run;
    if (rpre) rpre[njobs] = nfill;
  }
  __syncthreads();
}

// Last job whose prefix is <= i (zero-width ranges never end last).
__device__ __forceinline__ int job_of(const int* spre, int njobs, int i) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (spre[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Stores of the build's outputs (fill, eps), cache-streaming (evict first):
// hundreds of MB written once, whose lines would otherwise crowd L2 and
// drain to HBM under the next kernel's field loads.
__device__ __forceinline__ void out_st(float4* p, float4 v) { __stcs(p, v); }
__device__ __forceinline__ void out_st(float* p, float v) { __stcs(p, v); }

// Streaming fill of the constant tiles of one group of kFillRows x-rows: fill
// = 0 or 1, eps = eps_bg or eps_fg, 16-byte stores (a store instruction
// covers 512 contiguous bytes); band tiles are left to the band evaluation.
// One warp, row after row.
__device__ __forceinline__ void fill_rows(const Job* __restrict__ jobs, int jb, int unit,
                                          int lane) {
  const Job& J = jobs[jb];
  if (!J.do_build) return;
  const int nx = J.g.nx, ny = J.g.ny, nz = J.g.nz;
  const int lx = J.g.lx, ly = J.g.ly, lz = J.g.lz, ntx = J.g.ntx, nty = J.g.nty;
  const int rows = J.g.C * nz * ny;
  const float e0 = J.g.eps_bg, e1 = J.g.eps_bg + J.g.deps;
  float* __restrict__ fill = J.fill;
  float* __restrict__ eps = J.eps;
  const bool vec = (nx & 3) == 0 &&
                   ((reinterpret_cast<uintptr_t>(eps) | reinterpret_cast<uintptr_t>(fill)) & 15) == 0;
  for (int wr = 0; wr < kFillRows; ++wr) {
    const int row = (unit - J.row_base) * kFillRows + wr;
    if (row >= rows) break;
    const int j = row % ny, k = (row / ny) % nz;
    const size_t base = (size_t)row * nx;
    const unsigned char* __restrict__ tcl = J.tclass + ((k >> lz) * nty + (j >> ly)) * ntx;
    if (vec) {
      float4* f4 = reinterpret_cast<float4*>(fill + base);
      float4* e4 = reinterpret_cast<float4*>(eps + base);
      const int n4 = nx >> 2;
      for (int v0 = lane; v0 < n4; v0 += 128) {  // four tile classes in flight, then the stores
        int cls[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int v = v0 + 32 * u;
          cls[u] = v < n4 ? __ldg(tcl + ((4 * v) >> lx)) : 2;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (cls[u] == 2) continue;
          const int v = v0 + 32 * u;
          const float f = cls[u] ? 1.f : 0.f, e = cls[u] ? e1 : e0;
          if (fill) out_st(f4 + v, make_float4(f, f, f, f));
          out_st(e4 + v, make_float4(e, e, e, e));
        }
      }
    } else {
      for (int i = lane; i < nx; i += 32) {
        const int cls = __ldg(tcl + (i >> lx));
        if (cls == 2) continue;
        if (fill) out_st(fill + base + i, cls ? 1.f : 0.f);
        out_st(eps + base + i, cls ? e1 : e0);
      }
    }
  }
}

// ---- axis collapse -------------------------------------------------------------
// Whether a band tile's folded program has the same value at every y of the
// tile (okY), and at every z (okZ): every leaf is tabled and its y (z)
// factors are bitwise equal along the axis -- for the VJP also the derivative
// entries, and a parameter-driven in-plane leaf (whose derivatives are not
// tabled) blocks the y collapse.  Then the build evaluates one y (z) and
// writes it to all, and the VJP sums the seeds along the axis first (the
// projection to the grid comes last, Sec. 3; extruded and planar designs
// are uniform along whole axes, Sec. 3.1).  All threads, after the tables
// (which checked the box and z entries); per-thread flags, to be voted.
__device__ __forceinline__ void uniform_finish(const LeafTab* lt, int nleaf, const GridDev& g,
                                               const float* tab, bool derivs, int tid, bool& okY,
                                               bool& okZ) {
  const int TX = 1 << g.lx, TY = 1 << g.ly, C = g.C;
  const int lane = tid & 31;
  // axes that cannot collapse (the flags are read by the lanes of every warp
  // in parallel; the result is the same for every thread)
  bool untabled = false, planeAct = false, plane = false;
  for (int l = lane; l < nleaf; l += 32) {
    const int f = lt[l].d.w;
    untabled |= !(f & tOK);
    plane |= !(f & tBOX);
    planeAct |= derivs && !(f & tBOX) && (f & tACT);
  }
  if (__any_sync(0xffffffffu, untabled)) { okY = false; okZ = false; return; }
  if (__any_sync(0xffffffffu, planeAct)) okY = false;
  if (!__any_sync(0xffffffffu, plane)) return;
  // in-plane tables of the non-box leaves along y
  if (okY || !derivs)
    for (int l = 0; l < nleaf; ++l) {
      const int4 v = lt[l].v;
      if (lt[l].d.w & tBOX) continue;
      for (int e = tid; e < C * TX * TY; e += kBlock) {
        const int c = e / (TX * TY), r = e - c * TX * TY, y = r / TX, x = r - y * TX;
        if (y == 0) continue;
        okY &= tab[v.w + (c * TY + y) * TX + x] == tab[v.w + c * TY * TX + x];
      }
    }
}

// ---- forward-only evaluation (build) ----------------------------------------
// The folded program is postfix: every op takes the top two values of a
// stack (the complement the top one) and pushes one, so the build, which
// needs no tape, runs it on a four-deep register stack.  Each op is resolved
// once per tile into a descriptor: x = kind (0 tabled box, 1 tabled in-plane
// leaf, 2 direct leaf, 8 + logic code), y/z/w = table offsets or the leaf.
constexpr int kRegStack = 4;
constexpr int dBox = 0, dPlane = 1, dDirect = 2, dLogic = 8;

template <int LOGIC>
__device__ __forceinline__ float logic_fwd(int code, float a, float b) {
  if (code == fUnion) return LOGIC == 0 ? (a + b - a * b) : fminf(1.f, a + b);
  if (code == fInter) return LOGIC == 0 ? a * b : fmaxf(0.f, a + b - 1.f);
  return LOGIC == 0 ? a * (1.f - b) : fmaxf(0.f, a - b);
}

// Table offsets of one sample: x, y, z blocks and the in-plane block.
struct SampleOff {
  int x, y, z, xy;
};

// The same program on a stack in shared memory (column of stride kBlock), for
// programs deeper than the register stack; depth <= kMaxDepth by construction.
template <int LOGIC, bool kX>
__device__ __forceinline__ float eval_stack_smem(const int4* desc, int nops, const float* tab,
                                                 const PrimRec* sl, const SampleOff& o, int4 p,
                                                 const GridDev& g, const float* auxf,
                                                 const double* auxd, float* stk) {
  int sp = 0;
  for (int pos = 0; pos < nops; ++pos) {
    const int4 d = desc[pos];
    if (d.x < dLogic) {
      float v;
      if (d.x == dBox) {
        v = tab[d.y + o.x] * tab[d.z + o.y] * tab[d.w + o.z];
      } else if (d.x == dPlane) {
        v = tab[d.y + o.xy] * tab[d.w + o.z];
      } else {
        const Cell c{p.x, p.y, p.z, g.off[p.w][0], g.off[p.w][1], g.off[p.w][2]};
        v = leaf_value<kX>(sl[d.y], c, auxf, auxd);
      }
      if (sp < kMaxDepth) stk[(sp++) * kBlock] = v;
    } else if (sp >= 1) {
      const int code = d.x - dLogic;
      float* top = stk + (sp - 1) * kBlock;
      if (code == fCompl) {
        *top = 1.f - *top;
      } else if (sp >= 2) {
        const float b = *top;
        --sp;
        top -= kBlock;
        *top = logic_fwd<LOGIC>(code, *top, b);
      }
    }
  }
  return sp >= 1 ? stk[0] : 0.f;
}

template <int LOGIC, bool kX>
__device__ __forceinline__ void eval_stack2(const int4* desc, int nops, const float* tab,
                                            const PrimRec* sl, const SampleOff& o0,
                                            const SampleOff& o1, int4 p0, int4 p1,
                                            const GridDev& g, const float* auxf,
                                            const double* auxd, float& r0, float& r1) {
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;  // stack of sample 0, a0 on top
  float b0 = 0.f, b1 = 0.f, b2 = 0.f, b3 = 0.f;  // stack of sample 1
  for (int pos = 0; pos < nops; ++pos) {
    const int4 d = desc[pos];
    if (d.x < dLogic) {
      float v0, v1;
      if (d.x == dBox) {
        v0 = tab[d.y + o0.x] * tab[d.z + o0.y] * tab[d.w + o0.z];
        v1 = tab[d.y + o1.x] * tab[d.z + o1.y] * tab[d.w + o1.z];
      } else if (d.x == dPlane) {
        v0 = tab[d.y + o0.xy] * tab[d.w + o0.z];
        v1 = tab[d.y + o1.xy] * tab[d.w + o1.z];
      } else {  // cells built here only: the direct path takes them by reference
        const Cell c0{p0.x, p0.y, p0.z, g.off[p0.w][0], g.off[p0.w][1], g.off[p0.w][2]};
        const Cell c1{p1.x, p1.y, p1.z, g.off[p1.w][0], g.off[p1.w][1], g.off[p1.w][2]};
        v0 = leaf_value<kX>(sl[d.y], c0, auxf, auxd);
        v1 = leaf_value<kX>(sl[d.y], c1, auxf, auxd);
      }
      a3 = a2; a2 = a1; a1 = a0; a0 = v0;
      b3 = b2; b2 = b1; b1 = b0; b0 = v1;
    } else {
      const int code = d.x - dLogic;
      if (code == fCompl) {
        a0 = 1.f - a0;
        b0 = 1.f - b0;
      } else {
        a0 = logic_fwd<LOGIC>(code, a1, a0);
        b0 = logic_fwd<LOGIC>(code, b1, b0);
        a1 = a2; a2 = a3;
        b1 = b2; b2 = b3;
      }
    }
  }
  r0 = a0;
  r1 = b0;
}

// Warp 0 of a build band tile, straight from the records in global memory
// (while the other band warps stage them): the leaves' value-table offsets
// (prefix over the lanes; a leaf past `cap` is evaluated directly) and
// flags, the op descriptors, and the largest stack depth of the program.
__device__ __forceinline__ int build_plan_warp(const TileProg* P, const Job& J, int nleaf, int nops,
                                               int cap, LeafTab* lt, int4* desc, int lane) {
  const GridDev& g = J.g;
  const int TX = 1 << g.lx, TY = 1 << g.ly, TZ = 1 << g.lz, C = g.C;
  uint16_t opw[(kMaxOps + 31) / 32];
#pragma unroll
  for (int i = 0; i < (kMaxOps + 31) / 32; ++i) {
    const int pos = i * 32 + lane;
    opw[i] = pos < nops ? P->ops[pos] : (uint16_t)0;
  }
  int tbase = 0;
  for (int l0 = 0; l0 < nleaf; l0 += 32) {
    const int l = l0 + lane;
    const bool on = l < nleaf;
    const int kind = on ? J.prims[P->leaf[l]].kind : -1;
    const bool box = kind == kBox;
    const int need = !on ? 0 : (box ? C * (TX + TY + TZ) : C * TX * TY + C * TZ);
    int inc = need;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    const int off = tbase + inc - need;
    tbase += __shfl_sync(0xffffffffu, inc, 31);
    if (!on) continue;
    int4 v = make_int4(-1, -1, -1, -1), d = make_int4(-1, -1, -1, 0);
    if (off + need <= cap && kind != kXform) {  // transformed leaves are evaluated directly
      if (box) { v.x = off; v.y = v.x + C * TX; v.z = v.y + C * TY; }
      else { v.w = off; v.z = v.w + C * TX * TY; }
      d.w |= tOK;
    }
    if (box) d.w |= tBOX;
    lt[l].v = v;
    lt[l].d = d;
  }
  __syncwarp();  // lt of every leaf, for the descriptors
  int depth = 0, maxd = 0;
#pragma unroll
  for (int i = 0; i < (kMaxOps + 31) / 32; ++i) {
    const int p0 = i * 32;
    if (p0 >= nops) break;
    const int pos = p0 + lane;
    int delta = 0;
    if (pos < nops) {
      const FoldOp fo = fold_op(opw[i]);
      if (fo.code == fPush) {
        const int f = lt[fo.a].d.w;
        const int4 v = lt[fo.a].v;
        desc[pos] = !(f & tOK) ? make_int4(dDirect, fo.a, 0, 0)
                  : (f & tBOX) ? make_int4(dBox, v.x, v.y, v.z) : make_int4(dPlane, v.w, 0, v.z);
        delta = 1;
      } else {
        desc[pos] = make_int4(dLogic + fo.code, 0, 0, 0);
        delta = fo.code != fCompl ? -1 : 0;
      }
    }
    int inc = delta;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += u;
    }
    maxd = max(maxd, __reduce_max_sync(0xffffffffu, depth + inc));
    depth += __shfl_sync(0xffffffffu, inc, 31);
  }
  return maxd;
}

// Barriers of the build's band warps (warps 0 .. kWarps-1; named barrier 1):
// the fill warps of the block never wait on them.
__device__ __forceinline__ void band_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kBlock) : "memory"); }
__device__ __forceinline__ bool band_sync_and(bool p) {
  int r;
  asm volatile(
      "{\n\t.reg .pred a, b;\n\tsetp.ne.s32 a, %1, 0;\n\tbar.red.and.pred b, 1, %2, a;\n\t"
      "selp.s32 %0, 1, 0, b;\n\t}"
      : "=r"(r)
      : "r"((int)p), "n"(kBlock)
      : "memory");
  return r != 0;
}

// One band tile of the build (the kBlock threads of the band warps).
template <bool kX>
__device__ __forceinline__ void build_band_tile(const Job* __restrict__ jobs, int njobs,
                                                const int* spre, int gi_, unsigned char* smem) {
  float* stk = reinterpret_cast<float*>(smem);  // stack of the deep-program fallback
  float* pool = stk + kMaxDepth * kBlock;
  int4* desc = reinterpret_cast<int4*>(pool + kBuildPool);
  int* sdepth = reinterpret_cast<int*>(desc + kMaxOps);
  const int tid = threadIdx.x;
  {
    const int jb = job_of(spre, njobs, gi_);
    const Job& J = jobs[jb];
    const GridDev& g = J.g;
    const int t = J.list[gi_ - spre[jb]];
    if (!ADG_CHECK(t >= 0 && t < g.T, J.err)) return;  // uniform over the band warps
    const TileProg* P = J.progs + t;
    const int nops = P->nops, nleaf = P->nleaf;
    const int tx = t % g.ntx, ty = (t / g.ntx) % g.nty, tz = t / (g.ntx * g.nty);
    const TilePool tp = carve_pool(pool, kBuildPool, nleaf, 0);
    band_sync();  // the previous tile is done with the staged program
    if (tid < 32) {  // warp 0 plans from the records while warps 1.. stage them
      const int depth = build_plan_warp(P, J, nleaf, nops, tp.cap, tp.lt, desc, tid);
      if (tid == 0) {
        sdepth[0] = depth;
        sdepth[1] = 1;  // z collapse until a thread finds otherwise
      }
    } else {
      stage_tile(P, J.prims, nleaf, tp.sl, tid - 32, kBlock - 32);
    }
    band_sync();
    bool okY, okZ;
    tables_fill(tp.sl, nleaf, g, tp.lt, false, tx << g.lx, ty << g.ly, tz << g.lz, tp.tab, tid,
                J.auxf, J.auxd, nullptr, okY, okZ);
    band_sync();
    uniform_finish(tp.lt, nleaf, g, tp.tab, false, tid, okY, okZ);
    if (!okZ) sdepth[1] = 0;
    const bool uy = band_sync_and(okY);
    const bool uz = sdepth[1] != 0;
    // evaluated lattice: x, then y (one row if y collapses), z, component
    const int lyr = uy ? 0 : g.ly, lzr = uz ? 0 : g.lz;
    const int lxy = g.lx + lyr, lxyz = lxy + lzr;
    const int ncc = g.C << lxyz;
    const int TXm = (1 << g.lx) - 1, TYm = (1 << lyr) - 1, TZm = (1 << lzr) - 1;
    const int X0 = tx << g.lx, Y0 = ty << g.ly, Z0 = tz << g.lz;
    // the y and z each evaluated sample stands for (in the grid)
    const int ny_r = uy ? min(1 << g.ly, g.ny - Y0) : 1, nz_r = uz ? min(1 << g.lz, g.nz - Z0) : 1;
    const size_t plane = (size_t)g.nx * g.ny * g.nz;
    float* __restrict__ fill = J.fill;
    float* __restrict__ eps = J.eps;
    auto store = [&](int x, int y, int z, int c, float v) {
      if (X0 + x >= g.nx || Y0 + y >= g.ny || Z0 + z >= g.nz) return;
      const float e = g.eps_bg + g.deps * v;
      if (!uy && !uz) {  // uniform over the block
        const size_t o = (size_t)c * plane + ((size_t)(Z0 + z) * g.ny + (Y0 + y)) * g.nx + (X0 + x);
        if (fill) out_st(fill + o, v);
        out_st(eps + o, e);
        return;
      }
      for (int zz = 0; zz < nz_r; ++zz)
        for (int yy = 0; yy < ny_r; ++yy) {
          const size_t o = (size_t)c * plane + ((size_t)(Z0 + z + zz) * g.ny + (Y0 + y + yy)) * g.nx +
                           (X0 + x);
          if (fill) out_st(fill + o, v);
          out_st(eps + o, e);
        }
    };
    if (sdepth[0] <= kRegStack) {
      const int half = ncc >> 1;  // even: TX >= 32
      for (int l = tid; l < half; l += kBlock) {
        SampleOff o[2];
        int4 pc[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int m = l + h * half;
          const int x = m & TXm, y = (m >> g.lx) & TYm, z = (m >> lxy) & TZm, c = m >> lxyz;
          o[h] = SampleOff{(c << g.lx) + x, (c << g.ly) + y, (c << g.lz) + z,
                           (((c << g.ly) + y) << g.lx) + x};
          pc[h] = make_int4(X0 + x, Y0 + y, Z0 + z, c);
        }
        float v0, v1;
        if (g.logic == 0)
          eval_stack2<0, kX>(desc, nops, tp.tab, tp.sl, o[0], o[1], pc[0], pc[1], g, J.auxf, J.auxd, v0, v1);
        else
          eval_stack2<1, kX>(desc, nops, tp.tab, tp.sl, o[0], o[1], pc[0], pc[1], g, J.auxf, J.auxd, v0, v1);
        store(pc[0].x - X0, pc[0].y - Y0, pc[0].z - Z0, pc[0].w, v0);
        store(pc[1].x - X0, pc[1].y - Y0, pc[1].z - Z0, pc[1].w, v1);
      }
      return;
    }
    for (int l = tid; l < ncc; l += kBlock) {
      const int x = l & TXm, y = (l >> g.lx) & TYm, z = (l >> lxy) & TZm, c = l >> lxyz;
      if (X0 + x >= g.nx || Y0 + y >= g.ny || Z0 + z >= g.nz) continue;
      const SampleOff so{(c << g.lx) + x, (c << g.ly) + y, (c << g.lz) + z,
                         (((c << g.ly) + y) << g.lx) + x};
      const int4 pc = make_int4(X0 + x, Y0 + y, Z0 + z, c);
      const float v = g.logic == 0
          ? eval_stack_smem<0, kX>(desc, nops, tp.tab, tp.sl, so, pc, g, J.auxf, J.auxd, stk + tid)
          : eval_stack_smem<1, kX>(desc, nops, tp.tab, tp.sl, so, pc, g, J.auxf, J.auxd, stk + tid);
      store(x, y, z, c, v);
    }
  }
}

// The build (constant and band tiles of every build job), persistent: band
// tiles from the binner's compacted list -- the tile's primitives staged with
// their factor tables, the folded program run at every sample (two samples
// per thread, register stack; a shared-memory stack for deeper programs) --
// and the streaming fill of the constant tiles.
// 80 registers: four blocks of 160 or 192 threads per SM.  kX: compiled twice,
// k_build_x for job tables with transformed primitives (FP64 evaluation)
template <bool kX>
__device__ __forceinline__ void build_body(const Job* __restrict__ jobs, int njobs, int nfill,
                                           int* work) {
  extern __shared__ __align__(16) unsigned char smem[];
  // layout: deep-program stack, pool, descriptors, four words (depth, z flag,
  // unused, next band tile), job prefix
  int* spre = reinterpret_cast<int*>(smem + (size_t)kMaxDepth * kBlock * 4 + (size_t)kBuildPool * 4 +
                                     kMaxOps * 16) + 4;
  int* rpre = spre + spre_len(njobs);  // first fill unit of each job
  const int tid = threadIdx.x;
  wait_prior_grid();  // the binner's counters, lists and programs
  job_prefix(jobs, njobs, false, spre, rpre, nfill);  // ends with a barrier
  const int total = spre[njobs];
  // Warp-specialised: the band warps take band tiles (latency-bound, with
  // their own barriers) while the fill warps stream the rows of constant
  // tiles (store-bound), so that neither waits for the other.  Fill units
  // are handed out by a counter of the launch; band warps that run out of
  // band tiles take fill units too.  Each unit is written by exactly one
  // warp, so the output does not depend on who.
  const int G = gridDim.x;
  if (tid < kBlock) {  // band tiles: as in the VJP, the rest from work[2]
    int* sgi = spre - 1;
    int nxt = blockIdx.x;
    bool have = true;
    for (;;) {
      if (tid == 0) {
        if (!have) nxt = G + atomicAdd(work + 2, 1);
        *sgi = nxt;
      }
      band_sync();
      const int gi_ = *sgi;
      if (gi_ >= total) break;
      if (tid == 0) {
        have = gi_ + 2 * G < total;
        if (have) nxt = G + atomicAdd(work + 2, 1);
      }
      build_band_tile<kX>(jobs, njobs, spre, gi_, smem);  // starts with a band barrier
    }
    if (tid == 0) {
      __threadfence();
      if (atomicAdd(work + 3, 1) == G - 1) {
        work[2] = 0;
        work[3] = 0;
        __threadfence();
      }
    }
  }
  // fill units from the launch's counter (work[4]), so that warps of blocks
  // whose band tiles ended early take more of them
  const int lane = tid & 31;
  while (true) {
    int fu = 0;
    if (lane == 0) fu = atomicAdd(work + 4, 1);
    fu = __shfl_sync(0xffffffffu, fu, 0);
    if (fu >= nfill) break;
    fill_rows(jobs, job_of(rpre, njobs, fu), fu, lane);
  }
  // every warp of the block has made its last fetch: the last block resets
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(work + 5, 1) == G - 1) {
      work[4] = 0;
      work[5] = 0;
      __threadfence();
    }
  }
}

__global__ void __maxnreg__(80) k_build(const Job* __restrict__ jobs, int njobs, int nfill,
                                        int* work) {
  build_body<false>(jobs, njobs, nfill, work);
}

__global__ void __maxnreg__(80) k_build_x(const Job* __restrict__ jobs, int njobs, int nfill,
                                          int* work) {
  build_body<true>(jobs, njobs, nfill, work);
}

__device__ __forceinline__ void neumaier(float& s, float& c, float v) {
  const float t = s + v;
  if (fabsf(s) >= fabsf(v)) c += (s - t) + v;
  else c += (v - t) + s;
  s = t;
}

__device__ __forceinline__ void flush_slot(int& slot, float& v, float* acc, float* cmp, int lane) {
  if (slot >= 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) neumaier(acc[slot], cmp[slot], v);
  }
  slot = -1;
  v = 0.f;
}

// Warp-cooperative, deterministic accumulation of the lanes' (slot, value)
// pairs: each distinct slot present in the warp is reduced with a fixed
// xor-shuffle tree and added by lane 0 into the warp's compensated row.
__device__ __forceinline__ void warp_accumulate(int n, int sb, const int* pk, const float* pv,
                                                float* acc, float* cmp, int lane) {
  int ptr = 0;
  while (true) {
    const int my = ptr < n ? pk[ptr * kBlock] : INT_MAX;
    const int k = __reduce_min_sync(0xffffffffu, my);
    if (k == INT_MAX) break;
    float v = 0.f;
    if (my == k) { v = pv[ptr * kBlock]; ++ptr; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) neumaier(acc[sb + k], cmp[sb + k], v);
  }
}

// One key of a tabled box: the warp's values reduced with a fixed xor tree,
// added by lane 0 into the warp's compensated row (warp-uniform call).
__device__ __forceinline__ void key_reduce(int slot, float v, float* acc, float* cmp, int lane) {
  if (__ballot_sync(0xffffffffu, v != 0.f) == 0u) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) neumaier(acc[slot], cmp[slot], v);
}

// Where a keyed leaf's terms go: a per-thread column of the tile's
// accumulators (col[slot * kBlock], summed once per tile), or, when the tile
// has too many slots for columns, a warp reduction per key into the warp's
// compensated row.  `pt` is uniform over the block.
struct KeySink {
  float* col;
  float* acc;
  float* cmp;
  int lane;
  bool pt;
  __device__ __forceinline__ void add(int slot, float v) const {
    if (pt) col[slot * kBlock] += v;
    else key_reduce(slot, v, acc, cmp, lane);
  }
};

// d s / d (box scalar k) * a for the six scalars of a tabled box leaf
// (keys 0..5 = x0, x1, y0, y1, z0, z1).
__device__ __forceinline__ void box_tab_reduce(const LeafTab& t, const TileLoc& q, const float* tab,
                                               float a, const GridDev& g, const KeySink& ks) {
  const int4 v = t.v, d = t.d;
  const float fx = tab[v.x + q.c * q.TX + q.x], fy = tab[v.y + q.c * q.TY + q.y],
              fz = tab[v.z + q.c * q.TZ + q.z];
  const int k = d.w >> 3;
  if (k & 3) {
    const float ax = a * fy * fz * g.invd[0];
    if (k & 1) ks.add(t.slot[0], tab[d.x + (2 * q.c) * q.TX + q.x] * ax * t.coef[0]);
    if (k & 2) ks.add(t.slot[1], tab[d.x + (2 * q.c + 1) * q.TX + q.x] * ax * t.coef[1]);
  }
  if (k & 12) {
    const float ay = a * fx * fz * g.invd[1];
    if (k & 4) ks.add(t.slot[2], tab[d.y + (2 * q.c) * q.TY + q.y] * ay * t.coef[2]);
    if (k & 8) ks.add(t.slot[3], tab[d.y + (2 * q.c + 1) * q.TY + q.y] * ay * t.coef[3]);
  }
  if (k & 48) {
    const float az = a * fx * fy * g.invd[2];
    if (k & 16) ks.add(t.slot[4], tab[d.z + (2 * q.c) * q.TZ + q.z] * az * t.coef[4]);
    if (k & 32) ks.add(t.slot[5], tab[d.z + (2 * q.c + 1) * q.TZ + q.z] * az * t.coef[5]);
  }
}

// The same for a box whose factors are not tabled (evaluated at the sample).
__device__ __forceinline__ void box_direct_reduce(const PrimRec& P, const LeafTab& t, const Cell& c,
                                                  float a, const GridDev& g, const KeySink& ks) {
  float f[3], fa[3], fb[3];
  box_axes(P, c, f, fa, fb);
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const float other = f[(ax + 1) % 3] * f[(ax + 2) % 3] * a * g.invd[ax];
    if (t.slot[2 * ax] >= 0) ks.add(t.slot[2 * ax], fa[ax] * other * t.coef[2 * ax]);
    if (t.slot[2 * ax + 1] >= 0) ks.add(t.slot[2 * ax + 1], fb[ax] * other * t.coef[2 * ax + 1]);
  }
}

// Circ2D (Table 4) extruded in z: keys cx, cy, r, z0, z1, each reduced over the
// warp (every lane holds the same leaf, so the slots are warp-uniform).
__device__ __forceinline__ void circle_reduce(const PrimRec& P, const LeafTab& t, const Cell& c,
                                              float a, const GridDev& g, const KeySink& ks) {
  float dz0, dz1, dxr, dyr, r, ds;
  const float zf = zfactor(P, c, dz0, dz1);
  const float s = sigma_f(P.sigma, P.kr * circle_dist(P, c, dxr, dyr, r), ds);
  const float gg = P.kr * ds * zf * a * g.invd[0];
  const float ir = r > 0.f ? 1.f / r : 0.f;
  if (t.slot[0] >= 0) ks.add(t.slot[0], gg * dxr * ir * t.coef[0]);
  if (t.slot[1] >= 0) ks.add(t.slot[1], gg * dyr * ir * t.coef[1]);
  if (t.slot[2] >= 0) ks.add(t.slot[2], gg * t.coef[2]);
  if (t.slot[3] >= 0) ks.add(t.slot[3], s * dz0 * a * g.invd[2] * t.coef[3]);
  if (t.slot[4] >= 0) ks.add(t.slot[4], s * dz1 * a * g.invd[2] * t.coef[4]);
}

// Poly2D (Table 4) translated rigidly by its parameters: moving every vertex
// by dx changes each edge distance by -n_x dx, so the vertex terms collapse to
// two sums over the edges; keys z0, z1, x, y (slots staged as 0..3).
__device__ __noinline__ void poly_rigid_reduce(const PrimRec& P, const LeafTab& t, const Cell& c,
                                               float a, const GridDev& g, const float* auxf,
                                               const KeySink& ks) {
  const int N = P.naux;
  const float* E = auxf + P.auxf_off;
  float ux, uy, dz0 = 0.f, dz1 = 0.f, ds;
  poly_rel(P, c, ux, uy);
  const float zf = zfactor(P, c, dz0, dz1);
  // one pass: prod = product of the nonzero factors, (sx, sy) = sum of
  // (sigma'/sigma) n over them; an exactly-zero factor keeps only its own
  // term (sigma' n times the others), two of them zero the derivative
  float prod = 1.f, gx = 0.f, gy = 0.f;
  int nz = 0;
  if (a != 0.f) {
    float sx = 0.f, sy = 0.f, zx = 0.f, zy = 0.f;
    for (int e = 0; e < N; ++e) {
      const float* Ee = E + kPolyEdgeFloats * e;
      const float se = sigma_f(P.sigma, P.kr * poly_d(Ee, ux, uy), ds);
      if (se == 0.f) {
        if (++nz > 1) break;
        zx = ds * Ee[4];
        zy = ds * Ee[6];
      } else {
        prod *= se;
        const float r = ds / se;
        sx += r * Ee[4];
        sy += r * Ee[6];
      }
    }
    if (nz == 0) { gx = -prod * sx; gy = -prod * sy; }
    else if (nz == 1) { gx = -prod * zx; gy = -prod * zy; }
  }
  const float v = nz == 0 ? prod : 0.f;  // the in-plane factor
  const float scale = a * zf * P.kr * g.invd[0];
  if (t.slot[0] >= 0) ks.add(t.slot[0], v * dz0 * a * g.invd[2] * t.coef[0]);
  if (t.slot[1] >= 0) ks.add(t.slot[1], v * dz1 * a * g.invd[2] * t.coef[1]);
  if (t.slot[2] >= 0) ks.add(t.slot[2], scale * gx * t.coef[2]);
  if (t.slot[3] >= 0) ks.add(t.slot[3], scale * gy * t.coef[3]);
}

// Activity of the tile's samples, per axis: a sample can have a nonzero
// Jacobian row only where some parameter-driven scalar of a tabled box has a
// nonzero derivative-table entry at its x, y or z (each scalar moves one
// face), or anywhere when a parameter-driven leaf is not a tabled box.
// act1 holds one byte per (component, coordinate) of the x, y, z blocks
// (set by the tables).
constexpr int kAct1 = 3 * (64 + 16 + 8);

// ---- VJP helpers ---------------------------------------------------------------
// Warp 0 of the VJP, straight from the records in global memory (while the
// other warps stage them): per leaf (one lane each) the accumulator slot and
// map coefficient of each keyed scalar -- the box's 6, the circle's 5, a
// rigid polygon's z0, z1 and shared vertex x, y -- the table offsets with
// derivatives (prefix over the lanes; a leaf past `cap` is evaluated
// directly) and flags, the slot bases (prefix of nact), the all-active flag,
// and the op descriptors with the parameter-driven pushes.  Writes lt,
// sbase, desc, dl and misc[1..3].
__device__ __forceinline__ void vjp_plan_warp(const TileProg* P, const Job& J, int nleaf, int nops,
                                              int cap, LeafTab* lt, int4* desc, int* dl,
                                              int* sbase, int* misc, int lane) {
  const GridDev& g = J.g;
  const int TX = 1 << g.lx, TY = 1 << g.ly, TZ = 1 << g.lz, C = g.C;
  uint16_t opw[(kMaxOps + 31) / 32];  // the program, one op per lane and round
#pragma unroll
  for (int i = 0; i < (kMaxOps + 31) / 32; ++i) {
    const int pos = i * 32 + lane;
    opw[i] = pos < nops ? P->ops[pos] : (uint16_t)0;
  }
  int tbase = 0, sb = 0;
  bool all = false;
  for (int l0 = 0; l0 < nleaf; l0 += 32) {
    const int l = l0 + lane;
    const bool on = l < nleaf;
    int kind = 0, flags = 0, nact = 0, aoff = 0;
    if (on) {
      const PrimRec* R = J.prims + P->leaf[l];
      kind = R->kind;
      flags = R->flags;
      nact = R->nact;
      aoff = R->act_off;
    }
    int keys = 0;
    if (on) {
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const bool keyed = kind == kBox || (kind == kCircle && k < 5) ||
                           (kind == kPolygon && (flags & kPolyRigid) && k < 4);
        const int slot = keyed ? __ldg(J.act + aoff + k) : -1;
        lt[l].slot[k] = slot;
        lt[l].coef[k] = keyed ? __ldg(J.actc + aoff + k) : 0.f;
        if (slot >= 0) keys |= tKEYS << k;
      }
    }
    const bool box = on && kind == kBox;
    const int need = !on ? 0 : (box ? 3 * C * (TX + TY + TZ) : C * TX * TY + 3 * C * TZ);
    int inc = need, ninc = on ? nact : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, inc, o);
      const int u = __shfl_up_sync(0xffffffffu, ninc, o);
      if (lane >= o) { inc += t; ninc += u; }
    }
    const int off = tbase + inc - need;
    tbase += __shfl_sync(0xffffffffu, inc, 31);
    if (on) sbase[l] = sb + ninc - nact;
    sb += __shfl_sync(0xffffffffu, ninc, 31);
    if (!on) continue;
    int4 v = make_int4(-1, -1, -1, -1), d = make_int4(-1, -1, -1, 0);
    if (off + need <= cap && kind != kXform) {  // transformed leaves are evaluated directly
      if (box) {
        v.x = off; v.y = v.x + C * TX; v.z = v.y + C * TY;
        d.x = v.z + C * TZ; d.y = d.x + 2 * C * TX; d.z = d.y + 2 * C * TY;
      } else {
        v.w = off; v.z = v.w + C * TX * TY;
        d.z = v.z + C * TZ;
      }
      d.w |= tOK;
    }
    if (box) d.w |= tBOX | keys;
    if (nact > 0) d.w |= tACT;
    lt[l].v = v;
    lt[l].d = d;
    if ((d.w & tACT) && (d.w & (tOK | tBOX)) != (tOK | tBOX)) all = true;
  }
  all = __any_sync(0xffffffffu, all);
  __syncwarp();  // lt of every leaf, for the descriptors
  int n = 0;
#pragma unroll
  for (int i = 0; i < (kMaxOps + 31) / 32; ++i) {
    const int p0 = i * 32;
    if (p0 >= nops) break;
    const int pos = p0 + lane;
    bool act = false;
    int leaf = 0;
    if (pos < nops) {
      const FoldOp fo = fold_op(opw[i]);
      if (fo.code == fPush) {
        const int f = lt[fo.a].d.w;
        const int4 v = lt[fo.a].v;
        desc[pos] = !(f & tOK) ? make_int4(dDirect, fo.a, 0, 0)
                  : (f & tBOX) ? make_int4(dBox, v.x, v.y, v.z) : make_int4(dPlane, v.w, 0, v.z);
        act = (f & tACT) != 0;
        leaf = fo.a;
      } else {
        desc[pos] = make_int4(dLogic + fo.code, fo.a, fo.b, 0);
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, act);
    if (act) dl[n + __popc(m & ((1u << lane) - 1u))] = pos | (leaf << 8);
    n += __popc(m);
  }
  if (lane == 0) {
    sbase[nleaf] = sb;
    misc[1] = all;
    misc[2] = n;
    misc[3] = 1;  // z collapse until a thread finds otherwise
  }
}

template <int LOGIC>
__device__ __forceinline__ void logic_bwd(int code, float a, float b, float& da, float& db) {
  if (code == fUnion) {
    if (LOGIC == 0) { da = 1.f - b; db = 1.f - a; }
    else { const float on = (a + b <= 1.f) ? 1.f : 0.f; da = on; db = on; }
  } else if (code == fInter) {
    if (LOGIC == 0) { da = b; db = a; }
    else { const float on = (a + b >= 1.f) ? 1.f : 0.f; da = on; db = on; }
  } else {
    if (LOGIC == 0) { da = 1.f - b; db = -a; }
    else { const float on = (a - b >= 0.f) ? 1.f : 0.f; da = on; db = -on; }
  }
}

// Forward tape (value of every op at the sample), then the reverse sweep
// through the logic (Eqs. AD / jaceps): afterwards tap[pos] holds d fill / d
// value(pos).  tap: this thread's column, stride kBlock.
template <int LOGIC, bool kX>
__device__ __forceinline__ void vjp_tape(const int4* desc, int nops, const float* tab,
                                         const SampleOff& o, const PrimRec* sl, int4 pc,
                                         const GridDev& g, const float* auxf, const double* auxd,
                                         float* tap) {
  for (int pos = 0; pos < nops; ++pos) {
    const int4 d = desc[pos];
    float v;
    if (d.x == dBox) {
      v = tab[d.y + o.x] * tab[d.z + o.y] * tab[d.w + o.z];
    } else if (d.x == dPlane) {
      v = tab[d.y + o.xy] * tab[d.w + o.z];
    } else if (d.x == dDirect) {
      const Cell c{pc.x, pc.y, pc.z, g.off[pc.w][0], g.off[pc.w][1], g.off[pc.w][2]};
      v = leaf_value<kX>(sl[d.y], c, auxf, auxd);
    } else if (d.x == dLogic + fCompl) {
      v = 1.f - tap[d.y * kBlock];
    } else {
      v = logic_fwd<LOGIC>(d.x - dLogic, tap[d.y * kBlock], tap[d.z * kBlock]);
    }
    tap[pos * kBlock] = v;
  }
  tap[(nops - 1) * kBlock] = 1.f;
  for (int pos = nops - 1; pos >= 0; --pos) {
    const int4 d = desc[pos];
    if (d.x < dLogic) continue;
    const float adj = tap[pos * kBlock];
    if (d.x == dLogic + fCompl) {
      tap[d.y * kBlock] = -adj;
      continue;
    }
    float da, db;
    logic_bwd<LOGIC>(d.x - dLogic, tap[d.y * kBlock], tap[d.z * kBlock], da, db);
    tap[d.y * kBlock] = adj * da;
    tap[d.z * kBlock] = adj * db;
  }
}

constexpr int kSeedChunk = 512;  // active samples whose seeds are staged at once

// Seeds of active samples [c0, c1) of a tile: deps Re(w E_adj E_fwd) (Eq. 1,
// no conjugate) or deps G, summed over the ny_r x nz_r positions an evaluated
// sample stands for.  geo = (X0, Y0, Z0, lx | lyr << 8 | lzr << 16).  Once
// per chunk, out of line: its values stay out of the sample loop's registers.
__device__ __noinline__ void tile_seeds(const Job* J, const uint16_t* slist, float* zsb, int c0,
                                        int c1, int4 geo, int ny_r, int nz_r) {
  const GridDev& g = J->g;
  const VjpArgs& va = J->va;
  const int lx = geo.w & 255, lyr = (geo.w >> 8) & 255, lzr = geo.w >> 16;
  const int TXm = (1 << lx) - 1, TYm = (1 << lyr) - 1, TZm = (1 << lzr) - 1;
  const int lxy = lx + lyr, lxyz = lxy + lzr;
  const size_t plane = (size_t)g.nx * g.ny * g.nz;
  const int npos = ny_r * nz_r;
  if (npos == 1) {  // one position per sample: several samples' loads in flight
#pragma unroll 4
    for (int i = c0 + (int)threadIdx.x; i < c1; i += kBlock) {
      const int l = slist[i];
      const int x = l & TXm, y = (l >> lx) & TYm, z = (l >> lxy) & TZm, c = l >> lxyz;
      const size_t o = ((size_t)(geo.z + z) * g.ny + (geo.y + y)) * g.nx + (geo.x + x);
      float zs;
      if (va.G) {
        zs = __ldg(va.G + (size_t)c * plane + o);
      } else {
        const float2 f = __ldg(va.ef[c] + o), a = __ldg(va.ea[c] + o);
        const float pr = f.x * a.x - f.y * a.y, pi = f.x * a.y + f.y * a.x;
        zs = 0.f + (va.w[c].x * pr - va.w[c].y * pi);
      }
      zsb[i - c0] = zs * g.deps;
    }
    return;
  }
  for (int i = c0 + (int)threadIdx.x; i < c1; i += kBlock) {
    const int l = slist[i];
    const int x = l & TXm, y = (l >> lx) & TYm, z = (l >> lxy) & TZm, c = l >> lxyz;
    const size_t o0 = ((size_t)(geo.z + z) * g.ny + (geo.y + y)) * g.nx + (geo.x + x);
    float zs = 0.f;
    // positions in groups of four: the group's loads are all issued before
    // the first product, and the sum runs through the positions in order
    for (int p0 = 0; p0 < npos; p0 += 4) {
      float2 f[4], a[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int p = p0 + k;
        f[k] = make_float2(0.f, 0.f);
        a[k] = make_float2(0.f, 0.f);
        if (p < npos) {
          const int zz = p / ny_r, yy = p - zz * ny_r;
          const size_t o = o0 + ((size_t)zz * g.ny + yy) * g.nx;
          if (va.G) f[k].x = __ldg(va.G + (size_t)c * plane + o);
          else { f[k] = __ldg(va.ef[c] + o); a[k] = __ldg(va.ea[c] + o); }
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (p0 + k >= npos) break;
        if (va.G) {
          zs += f[k].x;
        } else {
          const float pr = f[k].x * a[k].x - f[k].y * a[k].y, pi = f[k].x * a[k].y + f[k].y * a[k].x;
          zs += va.w[c].x * pr - va.w[c].y * pi;
        }
      }
    }
    zsb[i - c0] = zs * g.deps;  // eps = eps_bg + deps fill
  }
}
// a warp's share of a tile's x-rows (C * TY * TZ <= 3 * 16 * 8) fits kRowRounds
// rounds of its lanes
constexpr int kRowRounds = 3;
static_assert((3 * 16 * 8 + kWarps - 1) / kWarps <= 32 * kRowRounds, "rows per warp");
constexpr size_t kVjpFixed = (size_t)kSmemOps * kBlock * 4 + (size_t)kVjpPool * 4 +
                             (size_t)kSeedChunk * 4 + (kMaxLeaves + 1) * 4 + kAct1 + 32 * 4;
// the job prefix, then the active-sample list (C x cells entries of 16 bits)
__host__ __device__ constexpr size_t vjp_list_off(int njobs) {
  return ((kVjpFixed + 15) & ~(size_t)15) + (((size_t)spre_len(njobs) * 4 + 15) & ~(size_t)15);
}
__host__ __device__ constexpr size_t vjp_smem(int njobs, int cells) {
  return vjp_list_off(njobs) + (size_t)cells * 3 * 2;
}
// five blocks per SM up to 1024-cell tiles (228 KB of shared memory, 1 KB
// reserved per block); 2048-cell tiles run four
static_assert(5 * (vjp_smem(1, 1024) + 1024) <= 228 * 1024, "VJP shared memory for five blocks per SM");
static_assert(4 * (vjp_smem(1, kMaxTileCells) + 1024) <= 228 * 1024, "VJP shared memory, largest tiles");

// The VJP body; kPolarT: the job table holds Polar2D primitives (k_vjp_polar),
// else k_vjp, whose sample loop carries no Polar2D code at all.
template <bool kPolarT>
__device__ __forceinline__ void vjp_body(const Job* __restrict__ jobs, int njobs,
                                         int* __restrict__ err, float* __restrict__ gtape,
                                         int* work) {
  extern __shared__ __align__(16) unsigned char smem[];
  wait_prior_grid();  // the binner's output, the fields, the partials' last clearing
  float* tape = reinterpret_cast<float*>(smem);
  float* pool = tape + kSmemOps * kBlock;
  float* zsb = pool + kVjpPool;  // seeds of a chunk
  int* sbase = reinterpret_cast<int*>(zsb + kSeedChunk);
  unsigned char* act1 = reinterpret_cast<unsigned char*>(sbase + kMaxLeaves + 1);
  // misc words: [1] all-active flag, [2] parameter-driven pushes, [3]
  // z-collapse flag, [12..15] active samples per warp's rows
  int* misc = reinterpret_cast<int*>(act1 + kAct1);
  int* spre = reinterpret_cast<int*>(smem + ((kVjpFixed + 15) & ~(size_t)15));
  uint16_t* slist = reinterpret_cast<uint16_t*>(smem + vjp_list_off(njobs));  // active samples
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  job_prefix(jobs, njobs, true, spre);
  const int total = spre[njobs];
  // Tiles: the first by block index, the rest from the launch's counter
  // (work[0]); tiles cost very different amounts, so blocks balance.  While
  // more than two waves of tiles are left the next one is fetched a tile
  // ahead (the atomic's latency hides behind the tile); near the end only
  // when free, so that no block holds a tile while it works on another.
  __shared__ int s_gi[2];  // by iteration parity: a skipped tile has no barrier after the read
  int nxt = blockIdx.x;    // thread 0's next tile
  bool have = true;        // thread 0 holds it already
  for (int it = 0;; ++it) {
    if (tid == 0) {
      if (!have) nxt = (int)gridDim.x + atomicAdd(work, 1);
      s_gi[it & 1] = nxt;
    }
    __syncthreads();
    const int gi_ = s_gi[it & 1];
    if (gi_ >= total) break;
    if (tid == 0) {  // fetch ahead while much is left; near the end, when free
      have = gi_ + 2 * (int)gridDim.x < total;
      if (have) nxt = (int)gridDim.x + atomicAdd(work, 1);
    }
    const int jb = job_of(spre, njobs, gi_);
    const Job& J = jobs[jb];
    const GridDev& g = J.g;
    const int t = J.list[gi_ - spre[jb]];
    if (!ADG_CHECK(t >= 0 && t < g.T, err)) continue;  // uniform over the block
    const TileProg* P = J.progs + t;
    const int nops = P->nops, nleaf = P->nleaf, nslot = P->nslot;
    const int tx = t % g.ntx, ty = (t / g.ntx) % g.nty, tz = t / (g.ntx * g.nty);
    if (nslot > kMaxSlots) {  // flagged by the binner too; uniform over the block
      if (tid == 0) atomicOr(err, eSlotOverflow);
      continue;
    }
    // No leaf of the tile is driven by a parameter: d eps / d p is zero on
    // it (no slot, no active sample, no partial), so the tile is skipped.
    if (nslot == 0) continue;
    // pool: staged leaves, descriptors, op descriptors, pushes list,
    // accumulator rows, then per-thread columns and factor tables
    PrimRec* slw = reinterpret_cast<PrimRec*>(pool);
    LeafTab* ltw = reinterpret_cast<LeafTab*>(slw + nleaf);
    int4* desc = reinterpret_cast<int4*>(ltw + nleaf);
    int* dl = reinterpret_cast<int*>(desc + nops);
    float* racc = reinterpret_cast<float*>(dl + nops);
    float* rcmp = racc + kWarps * nslot;
    const int used = pool_need(nleaf, kWarps * nslot, nops);
    const PrimRec* sl = slw;
    const LeafTab* lt = ltw;
    // After the rows: pair columns (tiles with graph or polygon leaves), then
    // per-thread accumulator columns (nslot x kBlock) when they take at most
    // half of what is left, then the factor tables.  The binner checked that
    // the rows and the pair columns leave at least kPoolSpare floats.
    const bool pairs = P->pairs != 0;
    float* pv = pool + used;
    int* pk = reinterpret_cast<int*>(pv + kMaxPairs * kBlock);
    const int used2 = used + (pairs ? kPairFloats : 0);
    const int cap = kVjpPool - used2;
    const bool pt = nslot * kBlock <= cap / 2;
    float* tcol = pool + used2;
    float* tabw = pt ? tcol + nslot * kBlock : tcol;
    const int tcap = pt ? cap - nslot * kBlock : cap;
    const float* tab = tabw;
    __syncthreads();  // the previous tile is done with the pool
    // warp 0 plans from the records in global memory while the other warps
    // stage them and clear the accumulator rows
    if (warp == 0) {
      vjp_plan_warp(P, J, nleaf, nops, tcap, ltw, desc, dl, sbase, misc, lane);
    } else {
      stage_tile(P, J.prims, nleaf, slw, tid - 32, kBlock - 32);
      for (int q = tid - 32; q < 2 * kWarps * nslot; q += kBlock - 32) racc[q] = 0.f;  // rows and compensation
      for (int q = tid - 32; q < g.C * ((1 << g.lx) + (1 << g.ly) + (1 << g.lz)); q += kBlock - 32)
        act1[q] = 0;  // activity, set by the tables
    }
    if (pt)
      for (int q = 0; q < nslot; ++q) tcol[q * kBlock + tid] = 0.f;  // this thread's column
    __syncthreads();
    bool okY, okZ;
    tables_fill(sl, nleaf, g, lt, true, tx << g.lx, ty << g.ly, tz << g.lz, tabw, tid, J.auxf,
                J.auxd, act1, okY, okZ);
    __syncthreads();
    uniform_finish(lt, nleaf, g, tab, true, tid, okY, okZ);
    if (!okZ) misc[3] = 0;  // set to 1 by warp 0 before the last barrier
    const bool uy = __syncthreads_and(okY);
    const bool uz = misc[3] != 0;
    float* wacc = racc + warp * nslot;
    float* wcmp = rcmp + warp * nslot;
    const int TX = 1 << g.lx, TY = 1 << g.ly, TZ = 1 << g.lz, C = g.C;
    // evaluated lattice (x, y, z, c) with y and/or z collapsed to one
    // position; each evaluated sample's seed sums the positions it stands for
    const int lyr = uy ? 0 : g.ly, lzr = uz ? 0 : g.lz;
    const int TYr = 1 << lyr, TZr = 1 << lzr;
    const int lxy = g.lx + lyr, lxyz = lxy + lzr;
    const int TXm = TX - 1, TYm = TYr - 1, TZm = TZr - 1;
    const int X0 = tx << g.lx, Y0 = ty << g.ly, Z0 = tz << g.lz;
    const int ny_r = uy ? min(TY, g.ny - Y0) : 1, nz_r = uz ? min(TZ, g.nz - Z0) : 1;
    const int nrows = C * TYr * TZr;
    const int nw = TX >> 5;  // 32-bit words per x-row
    // Active samples, per x-row (c, z, y): the whole row when the sample's y
    // or z moves a face (or a non-box leaf drives a parameter), else the
    // component's x-pattern; out-of-grid samples never.  Each warp takes a
    // contiguous quarter of the rows: their counts, a warp prefix, the warp
    // totals through shared memory, then the rows' entries -- so the list
    // runs through the samples in order and the accumulation order is fixed.
    unsigned xm[3][2], xi[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int x = h * 32 + lane;
      const bool in = h < nw && X0 + x < g.nx;
      xi[h] = __ballot_sync(0xffffffffu, in);
#pragma unroll
      for (int c = 0; c < 3; ++c) xm[c][h] = __ballot_sync(0xffffffffu, in && c < C && act1[c * TX + x]);
    }
    const bool all = misc[1] != 0;
    const int rpw = (nrows + kWarps - 1) / kWarps;  // <= 32 kRowRounds
    const int ra = warp * rpw, rb = min(nrows, ra + rpw);
    // the warp's rows in rounds of 32 (row ra + 32 j + lane): per row its kind
    // (0 none, 1 whole, 2 pattern), first list entry within the warp and
    // (c, z, y) packed as c << 16 | z << 8 | y
    int rkind[kRowRounds], rbase[kRowRounds], rpack[kRowRounds];
    int run = 0;
#pragma unroll
    for (int j = 0; j < kRowRounds; ++j) {
      rkind[j] = 0;
      rbase[j] = 0;
      rpack[j] = 0;
      if (ra + 32 * j >= rb) continue;  // warp-uniform
      const int r = ra + 32 * j + lane;
      int cnt = 0;
      if (r < rb) {
        const int rc = r / (TYr * TZr);
        const int rem = r - rc * TYr * TZr;
        const int rz = rem / TYr;
        const int ry = rem - rz * TYr;
        rpack[j] = (rc << 16) | (rz << 8) | ry;
        if (Y0 + ry < g.ny && Z0 + rz < g.nz) {
          const bool full = all || act1[C * TX + rc * TY + ry] || act1[C * (TX + TY) + rc * TZ + rz];
          rkind[j] = full ? 1 : 2;
#pragma unroll
          for (int h = 0; h < 2; ++h)
            cnt += __popc(full ? xi[h] : (rc == 0 ? xm[0][h] : rc == 1 ? xm[1][h] : xm[2][h]));
        }
      }
      int inc = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
      }
      rbase[j] = run + inc - cnt;
      run += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) misc[12 + warp] = run;
    __syncthreads();  // warp totals
    int wbase = 0, nact_cells = 0;
#pragma unroll
    for (int v = 0; v < kWarps; ++v) {
      const int tv = misc[12 + v];
      if (v < warp) wbase += tv;
      nact_cells += tv;
    }
#pragma unroll
    for (int j = 0; j < kRowRounds; ++j) {  // this warp's rows, all lanes per row
      const int nr = min(32, rb - ra - 32 * j);
      for (int rr = 0; rr < nr; ++rr) {
        const int kd = __shfl_sync(0xffffffffu, rkind[j], rr);
        int off = wbase + __shfl_sync(0xffffffffu, rbase[j], rr);
        const int pk = __shfl_sync(0xffffffffu, rpack[j], rr);
        if (!kd) continue;
        const int c = pk >> 16, z = (pk >> 8) & 255, y = pk & 255;
        const int lrow = ((c * TZr + z) * TYr + y) << g.lx;
        for (int h = 0; h < nw; ++h) {
          const unsigned m = kd == 1 ? xi[h] : (c == 0 ? xm[0][h] : c == 1 ? xm[1][h] : xm[2][h]);
          if ((m >> lane) & 1u) slist[off + __popc(m & ((1u << lane) - 1u))] = (uint16_t)(lrow + h * 32 + lane);
          off += __popc(m);
        }
      }
    }
    __syncthreads();  // the list is complete; misc[12..] free again
    const int ndl = misc[2];
    if (tid == 0) atomicAdd(&J.counters[3], nact_cells * ny_r * nz_r);  // grid samples
    for (int c0 = 0; c0 < nact_cells; c0 += kSeedChunk) {
      const int c1 = min(nact_cells, c0 + kSeedChunk);
      tile_seeds(&J, slist, zsb, c0, c1, make_int4(X0, Y0, Z0, g.lx | (lyr << 8) | (lzr << 16)),
                 ny_r, nz_r);
      // The tape: shared memory for short programs, else this block's slice of
      // the global tape; the logic family is a template parameter.  The
      // variants are separate instantiations, so the shared one keeps
      // shared-memory addressing.
      auto samples = [&](auto big, auto logic, auto polar) {
        constexpr bool kBig = decltype(big)::value;
        constexpr int kLogic = decltype(logic)::value;
        constexpr bool kPolarT = decltype(polar)::value;
        float* tap = (kBig ? gtape + (size_t)blockIdx.x * kTapeBlockFloats : tape) + tid;
        for (int i0 = c0; i0 < c1; i0 += kBlock) {
          if (i0 + warp * 32 >= c1) continue;  // no live lane in this warp (warp-uniform)
          const int i = i0 + tid;
          const bool live = i < c1;
          const int l = live ? slist[i] : 0;
          const int x = l & TXm, y = (l >> g.lx) & TYm, z = (l >> lxy) & TZm, c = l >> lxyz;
          const float zs = live ? zsb[i - c0] : 0.f;
          const int4 pc = make_int4(X0 + x, Y0 + y, Z0 + z, c);
          const SampleOff so{(c << g.lx) + x, (c << g.ly) + y, (c << g.lz) + z,
                             (((c << g.ly) + y) << g.lx) + x};  // tables keep full TY, TZ
          vjp_tape<kLogic, kPolarT>(desc, nops, tab, so, sl, pc, g, J.auxf, J.auxd, tap);
          const Cell cc{pc.x, pc.y, pc.z, g.off[c][0], g.off[c][1], g.off[c][2]};
          const TileLoc q{x, y, z, c, TX, TY, TZ};
          // primitives: d s / d q times the seed
          for (int k = 0; k < ndl; ++k) {
            const int e = dl[k];
            const int pos = e & 255, lf = e >> 8;
            const float a = zs * tap[pos * kBlock];
            if (__ballot_sync(0xffffffffu, a != 0.f) == 0u) continue;
            const int fl = lt[lf].d.w;
            float* la = wacc + sbase[lf];
            float* lc = wcmp + sbase[lf];
            const KeySink ks{tcol + sbase[lf] * kBlock + tid, la, lc, lane, pt};
            if ((fl & (tOK | tBOX)) == (tOK | tBOX)) {
              box_tab_reduce(lt[lf], q, tab, a, g, ks);
              continue;
            }
            const int kind = sl[lf].kind;
            if (kind == kBox) {
              box_direct_reduce(sl[lf], lt[lf], cc, a, g, ks);
              continue;
            }
            // a tabled in-plane factor of exactly 0 means sigma is 0 with zero
            // slope on every edge (truncated tails; not for the linear kind,
            // whose closed-interval kink has slope 1 at 0): nothing to add
            float an = a;
            if ((fl & tOK) && sl[lf].sigma != kLinear &&
                tab[lt[lf].v.w + (c * TY + y) * TX + x] == 0.f)
              an = 0.f;
            if (__ballot_sync(0xffffffffu, an != 0.f) == 0u) continue;
            if (kind == kCircle) {
              circle_reduce(sl[lf], lt[lf], cc, an, g, ks);
              continue;
            }
            if (kind == kPolygon && (sl[lf].flags & kPolyRigid)) {
              poly_rigid_reduce(sl[lf], lt[lf], cc, an, g, J.auxf, ks);
              continue;
            }
            int n = 0;
            if (an != 0.f)
              n = leaf_pairs(sl[lf], cc, an, g, J.act, J.actc, J.auxf, J.auxd, pk + tid, pv + tid);
            warp_accumulate(n, 0, pk + tid, pv + tid, la, lc, lane);
            if constexpr (kPolarT) {
              if (kind == kPolygon || kind == kPolar || kind == kXform)
                shape_accumulate(sl[lf], cc, an, g, J.act, J.actc, J.auxf, J.auxd, la, lc, lane);
            } else {
              if (kind == kPolygon)
                poly_accumulate(sl[lf], cc, an, g, J.act, J.actc, J.auxf, la, lc, lane);
            }
          }
        }
      };
      using kS = std::false_type;
      using kG = std::true_type;
      using kP = std::integral_constant<int, 0>;
      using kC = std::integral_constant<int, 1>;
      using kPol = std::integral_constant<bool, kPolarT>;
      if (nops > kSmemOps) {
        if (g.logic == 0) samples(kG{}, kP{}, kPol{}); else samples(kG{}, kC{}, kPol{});
      } else {
        if (g.logic == 0) samples(kS{}, kP{}, kPol{}); else samples(kS{}, kC{}, kPol{});
      }
    }  // chunks of active samples
    __syncthreads();
    if (pt) {  // each slot's column sum, one warp per slot, fixed order
      for (int s2 = warp; s2 < nslot; s2 += kWarps) {
        const float* c = tcol + s2 * kBlock;
        float v = ((c[lane] + c[lane + 32]) + c[lane + 64]) + c[lane + 96];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) tcol[s2 * kBlock] = v;  // only this warp reads slot s2's column
      }
      __syncthreads();
    }
    for (int s2 = tid; s2 < nslot; s2 += kBlock) {
      int lf = 0;
      while (lf + 1 < nleaf && sbase[lf + 1] <= s2) ++lf;
      const int qa = s2 - sbase[lf];
      float tot = pt ? tcol[s2 * kBlock] : 0.f;
      for (int w = 0; w < kWarps; ++w) tot += racc[w * nslot + s2] + rcmp[w * nslot + s2];
      const PrimRec& R = sl[lf];
      if (tx >= R.pb[0] && tx < R.pb[1] && ty >= R.pb[2] && ty < R.pb[3] && tz >= R.pb[4] &&
          tz < R.pb[5]) {
        const int rel = ((tz - R.pb[4]) * (R.pb[3] - R.pb[2]) + (ty - R.pb[2])) * (R.pb[1] - R.pb[0]) +
                        (tx - R.pb[0]);
        const size_t idx = (size_t)R.part_off + (size_t)qa * R.npb + rel;
        if (ADG_CHECK(idx < (size_t)J.partial_n, err)) J.partial[idx] = tot;
      } else if (tot != 0.f) {
        atomicOr(err, ePartialRange);
      }
    }
  }
  // every block has made its last fetch: the last one to get here resets
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(work + 1, 1) == (int)gridDim.x - 1) {
      work[0] = 0;
      work[1] = 0;
      __threadfence();
    }
  }
}

__global__ void __launch_bounds__(kBlock, 5) k_vjp(const Job* __restrict__ jobs, int njobs,
                                                   int* __restrict__ err,
                                                   float* __restrict__ gtape, int* work) {
  vjp_body<false>(jobs, njobs, err, gtape, work);
}

__global__ void __launch_bounds__(kBlock, 5) k_vjp_polar(const Job* __restrict__ jobs, int njobs,
                                                         int* __restrict__ err,
                                                         float* __restrict__ gtape, int* work) {
  vjp_body<true>(jobs, njobs, err, gtape, work);
}

// ---- the dense field stream --------------------------------------------------
// Each warp takes chunks of kDenseChunk samples from the counter and streams
// E_fwd, E_adj (complex64) and fill with 16-byte loads
// (cache-streaming: read once), accumulating z = Re(w E_adj E_fwd) and
// z * fill in compensated fp32 per lane, then in FP64 over the warp.  The
// chunk's partial goes to its own slot, so the order of the final sum does not
// depend on which warp took which chunk.
__device__ __forceinline__ float dense_z(float fr, float fi, float ar, float ai, float2 w) {
  const float pr = fr * ar - fi * ai, pi = fr * ai + fi * ar;
  return w.x * pr - w.y * pi;
}

constexpr int kDenseBlock = 256;
__global__ void __launch_bounds__(kDenseBlock, 4) k_dense(DenseArgs a) {
  const int lane = threadIdx.x & 31;
  const int nch = a.C * a.chunks_per_c;
  while (true) {
    int ch = 0;
    if (lane == 0) ch = atomicAdd(a.ctr, 1);
    ch = __shfl_sync(0xffffffffu, ch, 0);
    if (ch >= nch) break;
    const int c = ch / a.chunks_per_c;
    const long long i0 = (long long)(ch - c * a.chunks_per_c) * kDenseChunk;
    const long long i1 = min(a.plane, i0 + kDenseChunk);
    // component c's arrays, selected without indexing the parameter block
    const float2 w = c == 0 ? a.w[0] : (c == 1 ? a.w[1] : a.w[2]);
    const float2* __restrict__ ef = c == 0 ? a.ef[0] : (c == 1 ? a.ef[1] : a.ef[2]);
    const float2* __restrict__ ea = c == 0 ? a.ea[0] : (c == 1 ? a.ea[1] : a.ea[2]);
    const float* __restrict__ fl = a.fill + (size_t)c * a.plane;
    float sz = 0.f, cz = 0.f, sf = 0.f, cf = 0.f;
    const bool vec = ((a.plane & 3) == 0) &&
                     (((reinterpret_cast<uintptr_t>(ef) | reinterpret_cast<uintptr_t>(ea) |
                        reinterpret_cast<uintptr_t>(fl)) & 15) == 0);
    if (vec) {  // i0, i1 are multiples of 4
      const float4* __restrict__ e4 = reinterpret_cast<const float4*>(ef);
      const float4* __restrict__ a4 = reinterpret_cast<const float4*>(ea);
      const float4* __restrict__ f4 = reinterpret_cast<const float4*>(fl);
#pragma unroll 8
      for (long long q = (i0 >> 2) + lane; q < (i1 >> 2); q += 32) {
        const float4 e0 = __ldcs(e4 + 2 * q), e1 = __ldcs(e4 + 2 * q + 1);
        const float4 g0 = __ldcs(a4 + 2 * q), g1 = __ldcs(a4 + 2 * q + 1);
        const float4 f = __ldcs(f4 + q);
        const float z0 = dense_z(e0.x, e0.y, g0.x, g0.y, w), z1 = dense_z(e0.z, e0.w, g0.z, g0.w, w);
        const float z2 = dense_z(e1.x, e1.y, g1.x, g1.y, w), z3 = dense_z(e1.z, e1.w, g1.z, g1.w, w);
        neumaier(sz, cz, (z0 + z1) + (z2 + z3));
        neumaier(sf, cf, (z0 * f.x + z1 * f.y) + (z2 * f.z + z3 * f.w));
      }
    } else {
      for (long long i = i0 + lane; i < i1; i += 32) {
        const float2 e = __ldcs(ef + i), g = __ldcs(ea + i);
        const float z = dense_z(e.x, e.y, g.x, g.y, w);
        neumaier(sz, cz, z);
        neumaier(sf, cf, z * __ldcs(fl + i));
      }
    }
    double vz = (double)sz + (double)cz, vf = (double)sf + (double)cf;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      vz += __shfl_xor_sync(0xffffffffu, vz, o);
      vf += __shfl_xor_sync(0xffffffffu, vf, o);
    }
    if (lane == 0) a.part[ch] = make_double2(vz, vf);
  }
}

// One block: the chunk partials in index order (per-thread strided sums, then
// a fixed shared-memory tree).
__global__ void __launch_bounds__(256) k_dense_final(DenseArgs a) {
  __shared__ double sz[256], sf[256];
  const int t = threadIdx.x, nch = a.C * a.chunks_per_c;
  double z = 0.0, f = 0.0;
  for (int ch = t; ch < nch; ch += 256) {
    const double2 v = a.part[ch];
    z += v.x;
    f += v.y;
  }
  sz[t] = z;
  sf[t] = f;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (t < h) {
      sz[t] += sz[t + h];
      sf[t] += sf[t + h];
    }
    __syncthreads();
  }
  if (t == 0) {
    a.gmat[0] = sz[0] - sf[0];  // sum z (1 - fill)
    a.gmat[1] = sf[0];          // sum z fill
  }
}

// One block per parameter: its (primitive, slot) partials over the derivative
// tile boxes, in a fixed order -- each warp takes every fourth partial of each
// reference (compensated fp32 per lane), FP64 across lanes, references and
// the four warps.
// Also clears what the VJP accumulated: each (primitive, scalar) partial row
// belongs to exactly one parameter, so the block that sums a row zeroes it,
// and the first block of a job moves the active-sample count to
// counters_last.
__global__ void __launch_bounds__(128) k_finalize(const Job* __restrict__ jobs, int njobs, int nparams) {
  __shared__ double wsum[4];
  const int wid = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const Job& J = jobs[job_by_param(jobs, njobs, wid)];
  const int k = wid - J.param_base;
  const int r0 = J.ref_off[k], r1 = J.ref_off[k + 1];  // tables uploaded before the VJP
  wait_prior_grid();  // the VJP's partials and counters
  if (k == 0 && threadIdx.x == 0) {
    *J.counters_last = J.counters[3];
    J.counters[3] = 0;
  }
  double total = 0.0;
  for (int r = r0; r < r1; ++r) {
    const PrimRec& P = J.prims[J.ref_prim[r]];
    if (!ADG_CHECK((size_t)P.part_off + (size_t)(J.ref_qa[r] + 1) * P.npb <= (size_t)J.partial_n,
                   J.err))
      continue;  // uniform over the block
    float* src = J.partial + P.part_off + (size_t)J.ref_qa[r] * P.npb;
    float s = 0.f, c = 0.f;
    // eight loads in flight per thread, summed in tile order; the nonzero
    // ones (tiles the VJP wrote) are cleared
    for (int t0 = threadIdx.x; t0 < P.npb; t0 += 8 * 128) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = t0 + u * 128 < P.npb ? src[t0 + u * 128] : 0.f;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (t0 + u * 128 < P.npb) {
          neumaier(s, c, v[u]);
          if (v[u] != 0.f) src[t0 + u * 128] = 0.f;
        }
    }
    double v = (double)s + (double)c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    total += J.ref_coeff[r] * v;
  }
  if (lane == 0) wsum[warp] = total;
  __syncthreads();
  if (threadIdx.x == 0) J.grad[k] = (float)(((wsum[0] + wsum[1]) + wsum[2]) + wsum[3]);
}

}  // namespace

cudaError_t init_kernel_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_bin, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kBinSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_build, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)build_smem(kMaxJobs));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_build_x, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)build_smem(kMaxJobs));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_vjp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)vjp_smem(kMaxJobs, kMaxTileCells));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_vjp_polar, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)vjp_smem(kMaxJobs, kMaxTileCells));
  return e;
}

// Resident blocks per SM for a job table of njobs jobs (the job prefix in
// shared memory grows with it), cached per job count.
int build_blocks_per_sm(int njobs, int fill_warps, bool xform) {
  static int v[2][kMaxFillWarps][kMaxJobs + 1] = {};
  njobs = std::min(std::max(njobs, 1), kMaxJobs);
  fill_warps = std::min(std::max(fill_warps, 1), kMaxFillWarps);
  int& r = v[xform ? 1 : 0][fill_warps - 1][njobs];
  if (!r) {
    if (xform)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_build_x, kBlock + 32 * fill_warps,
                                                    build_smem(njobs));
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_build, kBlock + 32 * fill_warps,
                                                    build_smem(njobs));
    if (r < 1) r = 1;
  }
  return r;
}

// cells: the largest tile of the table (a power of two, 128 .. kMaxTileCells).
int vjp_blocks_per_sm(int njobs, bool polar, int cells) {
  constexpr int kCellClasses = 5;  // 128, 256, ..., 2048 cells
  static_assert(128 << (kCellClasses - 1) == kMaxTileCells, "tile cell classes");
  static int v[2][kCellClasses][kMaxJobs + 1] = {};
  njobs = std::min(std::max(njobs, 1), kMaxJobs);
  int cls = 0;
  while (cls + 1 < kCellClasses && (128 << cls) < cells) ++cls;
  cells = 128 << cls;
  int& r = v[polar ? 1 : 0][cls][njobs];
  if (!r) {
    if (polar)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_vjp_polar, kBlock, vjp_smem(njobs, cells));
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_vjp, kBlock, vjp_smem(njobs, cells));
    if (r < 1) r = 1;
  }
  return r;
}

cudaError_t launch_bin(const Job* jobs, const JobTotals& t, int* err, cudaStream_t s) {
  if (t.tiles_padded <= 0) return cudaSuccess;
  k_bin<<<t.tiles_padded / kBinWarps, kBinThreads, kBinSmem, s>>>(jobs, t.njobs, err);
  return cudaGetLastError();
}

// A launch, with programmatic stream serialisation when pdl is set (the
// kernel then starts as the one before it drains; see wait_prior_grid).
template <typename... P, typename... A>
cudaError_t launch_k(bool pdl, void (*k)(P...), int grid, int block, size_t smem, cudaStream_t s,
                     A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? at : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

cudaError_t launch_build(const Job* jobs, const JobTotals& t, int sms, cudaStream_t s) {
  if (!t.work || t.fill_warps < 1 || t.fill_warps > kMaxFillWarps) return cudaErrorInvalidValue;
  const int grid = sms * build_blocks_per_sm(t.njobs, t.fill_warps, t.xform != 0);
  return launch_k(t.pdl != 0, t.xform ? k_build_x : k_build, grid, kBlock + 32 * t.fill_warps,
                  build_smem(t.njobs), s, jobs, t.njobs, t.fill_blocks, t.work);
}

cudaError_t launch_vjp(const Job* jobs, const JobTotals& t, int* err, int sms, float* gtape,
                       int gtape_blocks, cudaStream_t s) {
  // Polar2D and transformed primitives: the VJP compiled with their code
  const bool shapes = t.polar || t.xform;
  const int cells = t.max_cells > 0 ? std::min(t.max_cells, kMaxTileCells) : kMaxTileCells;
  const int grid = std::min(sms * vjp_blocks_per_sm(t.njobs, shapes, cells), gtape_blocks);
  if (grid < 1 || !gtape || !t.work) return cudaErrorInvalidValue;
  return launch_k(t.pdl != 0, shapes ? k_vjp_polar : k_vjp, grid, kBlock, vjp_smem(t.njobs, cells),
                  s, jobs, t.njobs, err, gtape, t.work);
}

cudaError_t launch_dense(const DenseArgs& a, int sms, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(a.ctr, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const int nch = a.C * a.chunks_per_c;
  const int warps = kDenseBlock / 32;
  const int grid = std::max(1, std::min((nch + warps - 1) / warps, sms * 4));
  k_dense<<<grid, kDenseBlock, 0, s>>>(a);
  k_dense_final<<<1, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const Job* jobs, const JobTotals& t, cudaStream_t s) {
  if (t.params <= 0) return cudaSuccess;
  return launch_k(t.pdl != 0, k_finalize, t.params, 128, 0, s, jobs, t.njobs, t.params);
}

}  // namespace adg
