// adg_kernels.cu -- sm_103a kernels of libadg.
//
//   k_bin       per tile: classify every primitive against the tile (outside /
//               inside / edge band) and fold the chained logic program with
//               the constants, leaving only the band primitives (hot-path row
//               "binner"; the paper's suggestion of restricting work to the
//               non-zero material-Jacobian support, Sec. 3 footnote, Sec. 7).
//   k_build     per tile: eps_c = eps_bg + deps * fill_c, fill from the folded
//               program evaluated at every Yee sample (Eq. eps; Table 4;
//               Eqs. union / intersection; Sec. 5.1).
//   k_vjp       per band tile: the reverse sweep of Eqs. AD / jaceps seeded
//               with Re(w E_adj E) (Eq. 1): forward tape, reverse logic
//               adjoints, primitive derivatives, warp-shuffle reduction per
//               (primitive, scalar) slot into compensated block partials.
//   k_finalize  per parameter: fixed-order sum of the block partials through
//               the parameter map (deterministic, FP64).
#include <limits.h>
#include <math.h>

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

// Exact fraction of the cell window [u - 1/2, u + 1/2] covered by [a, b]
// (Sec. 5.1, Eq. linear), a = ai0 + af0, b = ai1 + af1, u = i + off; da, db
// are its derivatives w.r.t. a and b in cells.
__device__ __forceinline__ float ov_exact(int ai0, float af0, int ai1, float af1, int i,
                                          float off, float& da, float& db) {
  const float ta = (float)(ai0 - i) + (af0 - off);
  const float tb = (float)(ai1 - i) + (af1 - off);
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
      const float ta = (float)(P.ai[2 * ax] - idx[ax]) + (P.af[2 * ax] - off[ax]);
      const float tb = (float)(P.ai[2 * ax + 1] - idx[ax]) + (P.af[2 * ax + 1] - off[ax]);
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
  const float fxi = (float)(c.i - P.ai[0]), fyi = (float)(c.j - P.ai[1]);
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

// signed vertical distance f(x) - y (or y - f(x)) in cells, FP64 where it cancels
__device__ __forceinline__ float graph_dist(const PrimRec& P, const Cell& c, const float* auxf,
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

__device__ __forceinline__ float leaf_value(const PrimRec& P, const Cell& c, const float* auxf,
                                            const double* auxd) {
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
  return 0.f;
}

// Nonzero d s / d q (physical units) of one leaf at one cell, times `a`, as
// (active slot, value) pairs in ascending slot order.  Columns of stride kBlock.
__device__ __forceinline__ int push_pair(const int* actp, int key, float v, int n, int* pk,
                                         float* pv) {
  const int s = actp[key];
  if (s >= 0 && v != 0.f && n < kMaxPairs) {
    pk[n * kBlock] = s;
    pv[n * kBlock] = v;
    return n + 1;
  }
  return n;
}

__device__ int leaf_pairs(const PrimRec& P, const Cell& c, float a, const GridDev& g,
                          const int* act, const float* auxf, const double* auxd, int* pk,
                          float* pv) {
  const int* actp = act + P.act_off;
  int n = 0;
  if (P.kind == kBox) {
    float f[3], fa[3], fb[3];
    box_axes(P, c, f, fa, fb);
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const float other = f[(ax + 1) % 3] * f[(ax + 2) % 3] * a * g.invd[ax];
      n = push_pair(actp, 2 * ax, fa[ax] * other, n, pk, pv);
      n = push_pair(actp, 2 * ax + 1, fb[ax] * other, n, pk, pv);
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
    n = push_pair(actp, 0, gg * dxr * ir, n, pk, pv);
    n = push_pair(actp, 1, gg * dyr * ir, n, pk, pv);
    n = push_pair(actp, 2, gg, n, pk, pv);
    n = push_pair(actp, 3, s * dz0 * a * g.invd[2], n, pk, pv);
    n = push_pair(actp, 4, s * dz1 * a * g.invd[2], n, pk, pv);
    return n;
  }
  if (P.kind == kGraph) {
    int seg;
    double t;
    const float d = graph_dist(P, c, auxf, auxd, seg, t);
    const float s = sigma_f(P.sigma, P.kr * d, ds);
    const float sgn = (P.flags & kGraphAbove) ? -1.f : 1.f;
    const float gg = P.kr * ds * zf * sgn * a;  // d s / d f (per y-cell) times a
    const int M = P.naux;
    n = push_pair(actp, 0, s * dz0 * a * g.invd[2], n, pk, pv);
    n = push_pair(actp, 1, s * dz1 * a * g.invd[2], n, pk, pv);
    if (seg < 0) {
      n = push_pair(actp, 2 + M, gg * g.invd[1], n, pk, pv);
    } else if (seg >= M - 1) {
      n = push_pair(actp, 2 + M + M - 1, gg * g.invd[1], n, pk, pv);
    } else {
      const double* X = auxd + P.auxd_off;
      const double* Y = X + M;
      const double* iX = Y + M;
      const double ux = (double)c.i + (double)c.ox;
      const float dY = (float)(Y[seg + 1] - Y[seg]);
      const float ix = (float)iX[seg];
      const float e0 = (float)(ux - X[seg + 1]), e1 = (float)(ux - X[seg]);
      n = push_pair(actp, 2 + seg, gg * dY * e0 * ix * ix * g.invd[0], n, pk, pv);
      n = push_pair(actp, 3 + seg, -gg * dY * e1 * ix * ix * g.invd[0], n, pk, pv);
      n = push_pair(actp, 2 + M + seg, gg * (float)(1.0 - t) * g.invd[1], n, pk, pv);
      n = push_pair(actp, 3 + M + seg, gg * (float)t * g.invd[1], n, pk, pv);
    }
    return n;
  }
  return 0;
}

// ------------------------------------------------------------------ logic ---
__device__ __forceinline__ float op_fwd(int code, int logic, float a, float b) {
  switch (code) {
    case fUnion: return logic == 0 ? (a + b - a * b) : fminf(1.f, a + b);
    case fInter: return logic == 0 ? a * b : fmaxf(0.f, a + b - 1.f);
    case fDiff: return logic == 0 ? a * (1.f - b) : fmaxf(0.f, a - b);
    default: return 1.f - a;  // complement: difference(1, a)
  }
}

__device__ __forceinline__ void op_bwd(int code, int logic, float a, float b, float& da,
                                       float& db) {
  switch (code) {
    case fUnion:
      if (logic == 0) { da = 1.f - b; db = 1.f - a; }
      else { const float on = (a + b <= 1.f) ? 1.f : 0.f; da = on; db = on; }
      break;
    case fInter:
      if (logic == 0) { da = b; db = a; }
      else { const float on = (a + b >= 1.f) ? 1.f : 0.f; da = on; db = on; }
      break;
    case fDiff:
      if (logic == 0) { da = 1.f - b; db = -a; }
      else { const float on = (a - b >= 0.f) ? 1.f : 0.f; da = on; db = -on; }
      break;
    default: da = -1.f; db = 0.f;
  }
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

__device__ int classify(const PrimRec& P, const float lo[3], const float hi[3],
                        const double* auxd) {
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
      if ((float)fmx - hi[1] < -b && (float)fmx - lo[1] < -b) return cOUT;
      if ((float)fmn - hi[1] > b) return cls_and(cIN, z);
    } else {                          // region y > f(x)
      if (hi[1] - (float)fmn < -b) return cOUT;
      if (lo[1] - (float)fmx > b) return cls_and(cIN, z);
    }
    return cBND;
  }
  return cBND;
}

// --------------------------------------------------------------- kernels ---
// Fold-stack entry: kind (0 = const 0, 1 = const 1, 2 = expression) | root << 2
// | start << 10 (root: position of the expression's last op; start: its first).
__device__ __forceinline__ int mkE(int root, int start) { return 2 | (root << 2) | (start << 10); }

__global__ void __launch_bounds__(128) k_bin(GridDev g, const int* __restrict__ chain,
                                             const PrimRec* __restrict__ prims,
                                             const float* __restrict__ auxf,
                                             const double* __restrict__ auxd,
                                             TileProg* __restrict__ progs, int* __restrict__ list,
                                             int* __restrict__ counters, int* __restrict__ err) {
  __shared__ int stk[kMaxDepth][128];
  __shared__ uint16_t sleaf[kMaxLeaves][128];
  const int tid = threadIdx.x;
  const int t = blockIdx.x * blockDim.x + tid;
  if (t >= g.T) return;
  const int tx = t % g.ntx, ty = (t / g.ntx) % g.nty, tz = t / (g.ntx * g.nty);
  const int i0 = tx << g.lx, j0 = ty << g.ly, k0 = tz << g.lz;
  const int i1 = min(g.nx, (tx + 1) << g.lx), j1 = min(g.ny, (ty + 1) << g.ly),
            k1 = min(g.nz, (tz + 1) << g.lz);
  const float lo[3] = {i0 + g.offmin[0], j0 + g.offmin[1], k0 + g.offmin[2]};
  const float hi[3] = {(i1 - 1) + g.offmax[0], (j1 - 1) + g.offmax[1], (k1 - 1) + g.offmax[2]};
  TileProg* out = progs + t;
  int nops = 0, nleaf = 0, sp = 0, e = 0;
  for (int w = 0; w < g.nchain; ++w) {
    const int word = chain[w];
    const int code = (word >> 24) & 0xff, arg = word & 0xffffff;
    int ent = 0;
    if (code == cPush) {
      const PrimRec& P = prims[arg];
      int cl = cOUT;
      if (tx >= P.tb[0] && tx < P.tb[1] && ty >= P.tb[2] && ty < P.tb[3] && tz >= P.tb[4] &&
          tz < P.tb[5])
        cl = classify(P, lo, hi, auxd);
      if (cl == cBND) {
        int slot = -1;
        for (int l = 0; l < nleaf; ++l)
          if (sleaf[l][tid] == arg) { slot = l; break; }
        if (slot < 0) {
          if (nleaf < kMaxLeaves) { sleaf[nleaf][tid] = (uint16_t)arg; slot = nleaf++; }
          else e |= eLeafOverflow;
        }
        if (slot >= 0 && nops < kMaxOps) {
          out->ops[nops] = (uint16_t)(fPush | (slot << 3));
          ent = mkE(nops, nops);
          ++nops;
        } else {
          e |= eOpsOverflow;
          ent = 0;
        }
      } else {
        ent = (cl == cIN) ? 1 : 0;
      }
      if (sp < kMaxDepth) stk[sp++][tid] = ent;
      else e |= eDepthOverflow;
    } else {
      if (sp < 2) { e |= eBadProgram; break; }
      const int B = stk[--sp][tid];
      const int A = stk[--sp][tid];
      const int ka = A & 3, kb = B & 3;
      const int ra = (A >> 2) & 0xff, sa = (A >> 10) & 0xff;
      const int rb = (B >> 2) & 0xff, sb = (B >> 10) & 0xff;
      int res = 0, emit = -1, unary = 0;
      bool discard = false;
      if (code == cUnion) {
        if (ka == 1 || kb == 1) { res = 1; discard = true; }
        else if (ka == 0) res = B;
        else if (kb == 0) res = A;
        else emit = fUnion;
      } else if (code == cInter) {
        if (ka == 0 || kb == 0) { res = 0; discard = true; }
        else if (ka == 1) res = B;
        else if (kb == 1) res = A;
        else emit = fInter;
      } else {  // difference
        if (ka == 0 || kb == 1) { res = 0; discard = true; }
        else if (kb == 0) res = A;
        else if (ka == 1) { emit = fCompl; unary = 1; }
        else emit = fDiff;
      }
      if (discard) {
        if (ka == 2) nops = sa;
        else if (kb == 2) nops = sb;
      }
      if (emit >= 0) {
        if (nops < kMaxOps) {
          if (unary) {
            out->ops[nops] = (uint16_t)(fCompl | (rb << 3));
            res = mkE(nops, sb);
          } else {
            out->ops[nops] = (uint16_t)(emit | (ra << 3) | (rb << 9));
            res = mkE(nops, sa);
          }
          ++nops;
        } else {
          e |= eOpsOverflow;
          res = 0;
        }
      }
      stk[sp++][tid] = res;
    }
  }
  if (sp != 1) e |= eBadProgram;
  const int fin = sp >= 1 ? stk[sp - 1][tid] : 0;
  float cval = 0.f;
  if ((fin & 3) != 2) { nops = 0; cval = (float)(fin & 3); }
  int nslot = 0;
  for (int l = 0; l < nleaf; ++l) {
    out->leaf[l] = sleaf[l][tid];
    nslot += prims[sleaf[l][tid]].nact;
  }
  if (nops > 0 && nslot > kMaxSlots) e |= eSlotOverflow;
  if (e) {
    atomicOr(err, e);
    nops = 0;
    cval = 0.f;
  }
  out->nops = nops;
  out->nleaf = nleaf;
  out->cval = cval;
  out->nslot = nslot;
  if (nops > 0) {
    const int idx = atomicAdd(&counters[0], 1);
    list[idx] = t;
    atomicMax(&counters[1], nops);
    atomicAdd(&counters[2], (i1 - i0) * (j1 - j0) * (k1 - k0));
  }
}

__device__ __forceinline__ void stage_tile(const TileProg* P, const PrimRec* prims, int nops,
                                           int nleaf, uint16_t* sops, PrimRec* sl, int tid) {
  for (int q = tid; q < nops; q += kBlock) sops[q] = P->ops[q];
  constexpr int W = sizeof(PrimRec) / 16;
  for (int q = tid; q < nleaf * W; q += kBlock) {
    const int l = q / W, w = q - l * W;
    reinterpret_cast<int4*>(sl + l)[w] = reinterpret_cast<const int4*>(prims + P->leaf[l])[w];
  }
}

__device__ __forceinline__ float eval_forward(const uint16_t* sops, int nops, const PrimRec* sl,
                                              const Cell& cc, int logic, float* tape, int tid,
                                              const float* auxf, const double* auxd) {
  float v = 0.f;
  for (int pos = 0; pos < nops; ++pos) {
    const int op = sops[pos];
    const int code = op & 7, a = (op >> 3) & 63, b = (op >> 9) & 63;
    if (code == fPush) v = leaf_value(sl[a], cc, auxf, auxd);
    else v = op_fwd(code, logic, tape[a * kBlock + tid], code == fCompl ? 0.f : tape[b * kBlock + tid]);
    tape[pos * kBlock + tid] = v;
  }
  return v;
}

constexpr size_t kBuildSmem = (size_t)kMaxOps * kBlock * 4 + kMaxLeaves * sizeof(PrimRec) +
                              kMaxOps * 2 + 16;

__global__ void __launch_bounds__(kBlock) k_build(GridDev g, const TileProg* __restrict__ progs,
                                                  const PrimRec* __restrict__ prims,
                                                  const float* __restrict__ auxf,
                                                  const double* __restrict__ auxd,
                                                  float* __restrict__ fill, float* __restrict__ eps) {
  extern __shared__ __align__(16) unsigned char smem[];
  float* tape = reinterpret_cast<float*>(smem);
  PrimRec* sl = reinterpret_cast<PrimRec*>(tape + kMaxOps * kBlock);
  uint16_t* sops = reinterpret_cast<uint16_t*>(sl + kMaxLeaves);
  const int tid = threadIdx.x;
  const int lxy = g.lx + g.ly, lxyz = lxy + g.lz;
  const int ncc = g.C << lxyz;
  const size_t plane = (size_t)g.nx * g.ny * g.nz;
  for (int t = blockIdx.x; t < g.T; t += gridDim.x) {
    const TileProg* P = progs + t;
    const int nops = P->nops, nleaf = P->nleaf;
    const float cval = P->cval;
    const int tx = t % g.ntx, ty = (t / g.ntx) % g.nty, tz = t / (g.ntx * g.nty);
    if (nops > 0) {
      __syncthreads();
      stage_tile(P, prims, nops, nleaf, sops, sl, tid);
      __syncthreads();
    }
    for (int l = tid; l < ncc; l += kBlock) {
      const int x = l & ((1 << g.lx) - 1), y = (l >> g.lx) & ((1 << g.ly) - 1),
                z = (l >> lxy) & ((1 << g.lz) - 1), c = l >> lxyz;
      const int gi = (tx << g.lx) + x, gj = (ty << g.ly) + y, gk = (tz << g.lz) + z;
      if (gi >= g.nx || gj >= g.ny || gk >= g.nz) continue;
      float v = cval;
      if (nops > 0) {
        const Cell cc{gi, gj, gk, g.off[c][0], g.off[c][1], g.off[c][2]};
        v = eval_forward(sops, nops, sl, cc, g.logic, tape, tid, auxf, auxd);
      }
      const size_t o = (size_t)c * plane + ((size_t)gk * g.ny + gj) * g.nx + gi;
      if (fill) fill[o] = v;
      eps[o] = g.eps_bg + g.deps * v;
    }
  }
}

__device__ __forceinline__ void neumaier(float& s, float& c, float v) {
  const float t = s + v;
  if (fabsf(s) >= fabsf(v)) c += (s - t) + v;
  else c += (v - t) + s;
  s = t;
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

constexpr size_t kVjpSmem = (size_t)kMaxOps * kBlock * 4 + 2 * (size_t)kWarps * kMaxSlots * 4 +
                            2 * (size_t)kMaxPairs * kBlock * 4 + kMaxLeaves * sizeof(PrimRec) +
                            kMaxOps * 2 + (kMaxLeaves + 1) * 4 + 16;

__global__ void __launch_bounds__(kBlock) k_vjp(GridDev g, const TileProg* __restrict__ progs,
                                                const int* __restrict__ list,
                                                const int* __restrict__ counters,
                                                const PrimRec* __restrict__ prims,
                                                const int* __restrict__ act,
                                                const float* __restrict__ auxf,
                                                const double* __restrict__ auxd, VjpArgs va,
                                                float* __restrict__ partial, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem[];
  float* tape = reinterpret_cast<float*>(smem);
  float* acc = tape + kMaxOps * kBlock;
  float* cmp = acc + kWarps * kMaxSlots;
  float* pv = cmp + kWarps * kMaxSlots;
  int* pk = reinterpret_cast<int*>(pv + kMaxPairs * kBlock);
  PrimRec* sl = reinterpret_cast<PrimRec*>(pk + kMaxPairs * kBlock);
  uint16_t* sops = reinterpret_cast<uint16_t*>(sl + kMaxLeaves);
  int* sbase = reinterpret_cast<int*>(sops + kMaxOps);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int lxy = g.lx + g.ly, lxyz = lxy + g.lz;
  const int ncc = g.C << lxyz;
  const size_t plane = (size_t)g.nx * g.ny * g.nz;
  const int nprog = counters[0];
  for (int li = blockIdx.x; li < nprog; li += gridDim.x) {
    const int t = list[li];
    const TileProg* P = progs + t;
    const int nops = P->nops, nleaf = P->nleaf;
    const int tx = t % g.ntx, ty = (t / g.ntx) % g.nty, tz = t / (g.ntx * g.nty);
    __syncthreads();
    stage_tile(P, prims, nops, nleaf, sops, sl, tid);
    __syncthreads();
    if (tid == 0) {
      int s = 0;
      for (int l = 0; l < nleaf; ++l) { sbase[l] = s; s += sl[l].nact; }
      sbase[nleaf] = s;
    }
    __syncthreads();
    const int nslot = sbase[nleaf];
    if (nslot > kMaxSlots) {
      if (tid == 0) atomicOr(err, eSlotOverflow);
      continue;
    }
    for (int q = tid; q < kWarps * nslot; q += kBlock) { acc[q] = 0.f; cmp[q] = 0.f; }
    __syncthreads();
    float* wacc = acc + warp * nslot;
    float* wcmp = cmp + warp * nslot;
    for (int l0 = 0; l0 < ncc; l0 += kBlock) {
      const int l = l0 + tid;
      const int x = l & ((1 << g.lx) - 1), y = (l >> g.lx) & ((1 << g.ly) - 1),
                z = (l >> lxy) & ((1 << g.lz) - 1), c = l >> lxyz;
      const int gi = (tx << g.lx) + x, gj = (ty << g.ly) + y, gk = (tz << g.lz) + z;
      const bool valid = gi < g.nx && gj < g.ny && gk < g.nz;
      float zs = 0.f;
      if (valid) {
        const size_t o = ((size_t)gk * g.ny + gj) * g.nx + gi;
        if (va.G) {
          zs = va.G[(size_t)c * plane + o];
        } else {
          const float2 f = va.ef[c][o], a = va.ea[c][o];
          const float pr = f.x * a.x - f.y * a.y, pi = f.x * a.y + f.y * a.x;
          zs = va.w[c].x * pr - va.w[c].y * pi;  // Re(w E_adj E), no conjugate (Eq. 1)
        }
        zs *= g.deps;  // eps = eps_bg + deps fill
      }
      const Cell cc{gi, gj, gk, g.off[c][0], g.off[c][1], g.off[c][2]};
      eval_forward(sops, nops, sl, cc, g.logic, tape, tid, auxf, auxd);
      // reverse sweep through the logic: tape slots become adjoints d fill / d node
      tape[(nops - 1) * kBlock + tid] = 1.f;
      for (int pos = nops - 1; pos >= 0; --pos) {
        const int op = sops[pos];
        const int code = op & 7;
        if (code == fPush) continue;
        const int a = (op >> 3) & 63, b = (op >> 9) & 63;
        const float adj = tape[pos * kBlock + tid];
        const float vb = code == fCompl ? 0.f : tape[b * kBlock + tid];
        float da, db;
        op_bwd(code, g.logic, tape[a * kBlock + tid], vb, da, db);
        tape[a * kBlock + tid] = adj * da;
        if (code != fCompl) tape[b * kBlock + tid] = adj * db;
      }
      // primitives: d s / d q times the seed, reduced per slot
      for (int pos = 0; pos < nops; ++pos) {
        const int op = sops[pos];
        if ((op & 7) != fPush) continue;
        const int lf = (op >> 3) & 63;
        const float a = zs * tape[pos * kBlock + tid];
        int n = 0;
        if (a != 0.f && sl[lf].nact > 0)
          n = leaf_pairs(sl[lf], cc, a, g, act, auxf, auxd, pk + tid, pv + tid);
        if (sl[lf].nact > 0) warp_accumulate(n, sbase[lf], pk + tid, pv + tid, wacc, wcmp, lane);
      }
    }
    __syncthreads();
    for (int s = tid; s < nslot; s += kBlock) {
      int lf = 0;
      while (lf + 1 < nleaf && sbase[lf + 1] <= s) ++lf;
      const int qa = s - sbase[lf];
      float tot = 0.f;
      for (int w = 0; w < kWarps; ++w) tot += acc[w * nslot + s] + cmp[w * nslot + s];
      const PrimRec& R = sl[lf];
      if (tx >= R.pb[0] && tx < R.pb[1] && ty >= R.pb[2] && ty < R.pb[3] && tz >= R.pb[4] &&
          tz < R.pb[5]) {
        const int rel = ((tz - R.pb[4]) * (R.pb[3] - R.pb[2]) + (ty - R.pb[2])) * (R.pb[1] - R.pb[0]) +
                        (tx - R.pb[0]);
        partial[(size_t)R.part_off + (size_t)qa * R.npb + rel] = tot;
      } else if (tot != 0.f) {
        atomicOr(err, ePartialRange);
      }
    }
  }
}

__global__ void k_finalize(int n, const int* __restrict__ ref_off, const int* __restrict__ ref_prim,
                           const int* __restrict__ ref_qa, const double* __restrict__ ref_coeff,
                           const PrimRec* __restrict__ prims, const float* __restrict__ partial,
                           float* __restrict__ grad) {
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (wid >= n) return;
  double total = 0.0;
  for (int r = ref_off[wid]; r < ref_off[wid + 1]; ++r) {
    const PrimRec& P = prims[ref_prim[r]];
    const float* src = partial + P.part_off + (size_t)ref_qa[r] * P.npb;
    double s = 0.0, c = 0.0;
    for (int t = lane; t < P.npb; t += 32) {
      const double v = src[t];
      const double u = s + v;
      c += (fabs(s) >= fabs(v)) ? (s - u) + v : (v - u) + s;
      s = u;
    }
    s += c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    total += ref_coeff[r] * s;
  }
  if (lane == 0) grad[wid] = (float)total;
}

}  // namespace

int build_blocks_per_sm() {
  static int v = 0;
  if (!v) {
    cudaFuncSetAttribute(k_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBuildSmem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_build, kBlock, kBuildSmem);
    if (v < 1) v = 1;
  }
  return v;
}

int vjp_blocks_per_sm() {
  static int v = 0;
  if (!v) {
    cudaFuncSetAttribute(k_vjp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kVjpSmem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_vjp, kBlock, kVjpSmem);
    if (v < 1) v = 1;
  }
  return v;
}

cudaError_t launch_bin(const GridDev& g, const int* chain, const PrimRec* prims,
                       const float* auxf, const double* auxd, TileProg* progs, int* list,
                       int* counters, int* err, cudaStream_t s) {
  const int blocks = (g.T + 127) / 128;
  k_bin<<<blocks, 128, 0, s>>>(g, chain, prims, auxf, auxd, progs, list, counters, err);
  return cudaGetLastError();
}

cudaError_t launch_build(const GridDev& g, const TileProg* progs, const PrimRec* prims,
                         const float* auxf, const double* auxd, float* fill, float* eps,
                         int grid, cudaStream_t s) {
  build_blocks_per_sm();
  k_build<<<grid, kBlock, kBuildSmem, s>>>(g, progs, prims, auxf, auxd, fill, eps);
  return cudaGetLastError();
}

cudaError_t launch_vjp(const GridDev& g, const TileProg* progs, const int* list,
                       const int* counters, const PrimRec* prims, const int* act,
                       const float* auxf, const double* auxd, const VjpArgs& a,
                       float* partial, int* err, int grid, cudaStream_t s) {
  vjp_blocks_per_sm();
  k_vjp<<<grid, kBlock, kVjpSmem, s>>>(g, progs, list, counters, prims, act, auxf, auxd, a,
                                       partial, err);
  return cudaGetLastError();
}

cudaError_t launch_finalize(int nparam, const int* ref_off, const int* ref_prim,
                            const int* ref_qa, const double* ref_coeff, const PrimRec* prims,
                            const float* partial, float* grad, cudaStream_t s) {
  if (nparam <= 0) return cudaSuccess;
  const int blocks = (nparam * 32 + 127) / 128;
  k_finalize<<<blocks, 128, 0, s>>>(nparam, ref_off, ref_prim, ref_qa, ref_coeff, prims, partial,
                                    grad);
  return cudaGetLastError();
}

}  // namespace adg
