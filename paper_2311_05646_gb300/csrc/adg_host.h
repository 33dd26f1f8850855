// adg_host.h -- host-side compilation of a design description and the FP64
// parameter map, on caller-provided storage (no allocation), shared by the
// regular entry points (adg_api.cu) and the no-allocation one (adg_noalloc.cu).
#pragma once
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include "../../include/adg.h"
#include "adg_internal.h"

namespace adg {
namespace host {

// transition half-widths of the sigma kinds in the unit variable u = k x;
// beyond them the kernels treat sigma as exactly 0 or 1 with zero slope
constexpr double kBand[5] = {0.5, 20.0, 0.70710678118654752, 1.5707963267948966, 4.5};

struct Msg {
  char text[512];
  adg_status set(adg_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(text, sizeof(text), fmt, ap);
    va_end(ap);
    return st;
  }
};

inline bool fin(double v) { return std::isfinite(v); }

inline int vertices_of(int kind, int nq) {
  if (kind == ADG_PRIM_POLYGON) return (nq - 2) / 2;
  if (kind == ADG_PRIM_GRAPH) return (nq - 2) / 2;
  return 0;
}

// Description checks shared by every entry point that takes a description.
inline adg_status validate(const adg_design_desc* D, Msg& m) {
  const adg_grid& G = D->grid;
  if (G.nx < 1 || G.ny < 1 || G.nz < 1 || G.nx > 8192 || G.ny > 8192 || G.nz > 8192)
    return m.set(ADG_EINVAL, "grid %dx%dx%d outside 1..8192 per axis", G.nx, G.ny, G.nz);
  if (G.ncomp < 1 || G.ncomp > 3) return m.set(ADG_EINVAL, "ncomp %d not in 1..3", G.ncomp);
  if (!(G.dx > 0) || !(G.dy > 0) || !(G.dz > 0) || !fin(G.dx) || !fin(G.dy) || !fin(G.dz))
    return m.set(ADG_EINVAL, "grid spacing must be positive and finite");
  if (!fin(G.ox) || !fin(G.oy) || !fin(G.oz)) return m.set(ADG_EINVAL, "grid origin must be finite");
  for (int c = 0; c < G.ncomp; ++c)
    for (int a = 0; a < 3; ++a)
      if (!(fabs(G.off[c][a]) <= 1.0))
        return m.set(ADG_EINVAL, "offset off[%d][%d] not in [-1, 1]", c, a);
  if (!fin(D->eps_bg) || !fin(D->eps_fg)) return m.set(ADG_EINVAL, "eps levels must be finite");
  if (D->logic != ADG_LOGIC_PRODUCT && D->logic != ADG_LOGIC_CLAMP)
    return m.set(ADG_EINVAL, "logic %d unknown", D->logic);
  if (D->reserved != 0) return m.set(ADG_EINVAL, "reserved must be 0");
  if (D->n_params < 0 || D->n_q < 0 || D->n_prims < 1 || D->n_ops < 1 || D->n_prims > 65535)
    return m.set(ADG_EINVAL, "counts: params %d, q %d, prims %d (1..65535), ops %d", D->n_params,
                 D->n_q, D->n_prims, D->n_ops);
  if ((D->n_q > 0 && (!D->q_base || !D->q_coeff || !D->q_param)) || !D->prim_kind ||
      !D->prim_sigma || !D->prim_flags || !D->prim_q0 || !D->prim_nq || !D->prim_kr || !D->ops)
    return m.set(ADG_EINVAL, "description array is NULL");
  for (int j = 0; j < D->n_q; ++j) {
    if (D->q_param[j] < -1 || D->q_param[j] >= D->n_params)
      return m.set(ADG_EINVAL, "q_param[%d] = %d out of range", j, D->q_param[j]);
    if (!fin(D->q_base[j]) || !fin(D->q_coeff[j]))
      return m.set(ADG_EINVAL, "q_base / q_coeff[%d] not finite", j);
  }
  for (int p = 0; p < D->n_prims; ++p) {
    const int k = D->prim_kind[p], s = D->prim_sigma[p], q0 = D->prim_q0[p];
    const bool xf = (D->prim_flags[p] & ADG_XFORM) != 0;
    const int n = D->prim_nq[p] - (xf ? 5 : 0);  // the base primitive's scalars
    if (q0 < 0 || D->prim_nq[p] < 0 || q0 + D->prim_nq[p] > D->n_q)
      return m.set(ADG_EINVAL, "primitive %d: scalars [%d, %d) outside [0, %d)", p, q0,
                   q0 + D->prim_nq[p], D->n_q);
    if (xf && (k == ADG_PRIM_GRAPH || (k == ADG_PRIM_BOX && !(D->prim_flags[p] & ADG_RECT_SIGMA))))
      return m.set(ADG_EINVAL, "primitive %d: a transform applies to sigma-form boxes, circles, "
                               "polygons and polar shapes", p);
    if (xf && fabs(G.dx - G.dy) > 1e-12 * G.dx)
      return m.set(ADG_EINVAL, "primitive %d: a transformed primitive needs dx == dy", p);
    if (s < 0 || s > 4) return m.set(ADG_EINVAL, "primitive %d: sigma kind %d unknown", p, s);
    if (!(D->prim_kr[p] > 0) || !fin(D->prim_kr[p]))
      return m.set(ADG_EINVAL, "primitive %d: kr must be positive", p);
    if (k == ADG_PRIM_BOX) {
      if (n != 6) return m.set(ADG_EINVAL, "box %d needs 6 scalars, has %d", p, n);
    } else if (k == ADG_PRIM_CIRCLE) {
      if (n != 5) return m.set(ADG_EINVAL, "circle %d needs 5 scalars, has %d", p, n);
    } else if (k == ADG_PRIM_GRAPH) {
      if (n < 6 || (n - 2) % 2) return m.set(ADG_EINVAL, "graph %d needs 2 + 2M scalars, M >= 2", p);
    } else if (k == ADG_PRIM_POLAR) {
      if (n < 5 || (n - 5) % 2 || (n - 5) / 2 > kMaxPolarHarm)
        return m.set(ADG_EINVAL, "polar %d needs 5 + 2N scalars, 0 <= N <= %d", p, kMaxPolarHarm);
    } else if (k == ADG_PRIM_POLYGON) {
      if (n < 8 || (n - 2) % 2 || (n - 2) / 2 > kMaxPolyVerts)
        return m.set(ADG_EINVAL, "polygon %d needs 2 + 2N scalars, 3 <= N <= %d", p, kMaxPolyVerts);
    } else {
      return m.set(ADG_EINVAL, "primitive %d: kind %d unknown", p, k);
    }
    if ((k == ADG_PRIM_CIRCLE || k == ADG_PRIM_POLYGON || k == ADG_PRIM_POLAR) &&
        fabs(G.dx - G.dy) > 1e-12 * G.dx)
      return m.set(ADG_EINVAL, "primitive %d (circle / polygon / polar) needs dx == dy", p);
  }
  return ADG_OK;
}

// Postfix program -> tree -> chain of binary ops.  n-ary union / intersection
// become left-to-right chains (the recursive form of union_2, Appendix B.2).
// Storage: node_* and kids of n_ops entries, stack of n_ops, chain of 2 n_ops.
struct ChainWork {
  int *node_code, *node_arg, *node_k0, *node_nk, *kids, *stack;
};

inline bool emit_chain(const ChainWork& w, int id, int* chain, int& n, int depth) {
  if (depth > 4096) return false;
  const int code = w.node_code[id];
  if (code == ADG_OP_PUSH) {
    chain[n++] = (cPush << 24) | w.node_arg[id];
    return true;
  }
  const int* k = w.kids + w.node_k0[id];
  const int nk = w.node_nk[id];
  if (code == ADG_OP_DIFF) {
    if (!emit_chain(w, k[0], chain, n, depth + 1) || !emit_chain(w, k[1], chain, n, depth + 1))
      return false;
    chain[n++] = cDiff << 24;
    return true;
  }
  const int c = code == ADG_OP_UNION ? cUnion : cInter;
  if (!emit_chain(w, k[0], chain, n, depth + 1)) return false;
  for (int t = 1; t < nk; ++t) {
    if (!emit_chain(w, k[t], chain, n, depth + 1)) return false;
    chain[n++] = c << 24;
  }
  return true;
}

inline adg_status compile_chain(const adg_design_desc* D, const ChainWork& w, int* chain,
                                int* nchain, Msg& m) {
  int sp = 0, nk = 0;
  for (int i = 0; i < D->n_ops; ++i) {
    const int wd = D->ops[i], code = (wd >> 24) & 0xff, arg = wd & 0xffffff;
    int need = 0;
    if (code == ADG_OP_PUSH) {
      if (arg < 0 || arg >= D->n_prims)
        return m.set(ADG_EINVAL, "program op %d pushes primitive %d (have %d)", i, arg, D->n_prims);
    } else if (code == ADG_OP_UNION || code == ADG_OP_INTERSECT) {
      need = arg;
      if (need < 1) return m.set(ADG_EINVAL, "program op %d: operand count %d", i, need);
    } else if (code == ADG_OP_DIFF) {
      need = 2;
    } else {
      return m.set(ADG_EINVAL, "program op %d: unknown code %d", i, code);
    }
    if (sp < need) return m.set(ADG_EINVAL, "program op %d: stack underflow", i);
    w.node_code[i] = code;
    w.node_arg[i] = arg;
    w.node_k0[i] = nk;
    w.node_nk[i] = need;
    for (int t = 0; t < need; ++t) w.kids[nk + t] = w.stack[sp - need + t];
    nk += need;
    sp -= need;
    w.stack[sp++] = i;
  }
  if (sp != 1) return m.set(ADG_EINVAL, "program leaves %d values on the stack (need 1)", sp);
  int n = 0;
  if (!emit_chain(w, w.stack[0], chain, n, 0)) return m.set(ADG_EINVAL, "program nesting too deep");
  int s2 = 0, mx = 0;
  for (int t = 0; t < n; ++t) {
    s2 += ((chain[t] >> 24) == cPush) ? 1 : -1;
    mx = std::max(mx, s2);
  }
  if (mx > kMaxDepth)
    return m.set(ADG_EINVAL, "program nesting %d exceeds the supported depth %d", mx, kMaxDepth);
  *nchain = n;
  return ADG_OK;
}

// Accumulator slots: one per (primitive, parameter).  Every scalar q of a
// primitive driven by parameter k (coefficient a != 0) maps to the slot of k
// within that primitive and carries a; the kernels accumulate a dL/dq there.
// act / actc hold n_q-per-primitive entries at act_off[p]; refs list, per
// parameter, its (primitive, slot) pairs.  count is scratch of n_params + 1.
struct SlotTables {
  int *act, *nact, *act_off;
  float* actc;
  int *ref_off, *ref_prim, *ref_qa;
  double* ref_coeff;
  int *auxd_off, *auxf_off;
  int nact_table, nrefs, auxd_n, auxf_n;
};

inline int aux_doubles(int kind, int nq, int flags = 0) {
  if (flags & ADG_XFORM) {  // see kXformHead
    const int nb = nq - 5;
    if (kind == ADG_PRIM_BOX) return kXformHead + 6;
    if (kind == ADG_PRIM_CIRCLE) return kXformHead + 3;
    if (kind == ADG_PRIM_POLAR) return kXformHead + nb - 2;  // cx, cy, R0, c_n, s_n
    return kXformHead + 1 + (nb - 2);                       // polygon: sign, vertices
  }
  const int N = vertices_of(kind, nq);
  if (kind == ADG_PRIM_GRAPH) return 3 * N;    // X, Y, 1/dX
  if (kind == ADG_PRIM_POLYGON) return 6 * N;  // X, Y, nx, ny, c, 1/L
  return 0;
}

inline int aux_floats(int kind, int nq, int flags = 0) {
  if (flags & ADG_XFORM) return 0;
  if (kind == ADG_PRIM_POLAR) return 2 * (nq - 4);  // R0, c_n, s_n (cells) as hi + lo pairs
  if (kind == ADG_PRIM_GRAPH) return vertices_of(kind, nq);
  if (kind == ADG_PRIM_POLYGON) return kPolyEdgeFloats * vertices_of(kind, nq);
  return 0;
}

inline void build_slots(const adg_design_desc* D, SlotTables& t, int* count) {
  int na_tab = 0, auxd = 0, auxf = 0;
  for (int k = 0; k <= D->n_params; ++k) count[k] = 0;
  for (int p = 0; p < D->n_prims; ++p) {
    t.act_off[p] = na_tab;
    t.auxd_off[p] = auxd;
    t.auxf_off[p] = auxf;
    auxd += aux_doubles(D->prim_kind[p], D->prim_nq[p], D->prim_flags[p]);
    auxf += aux_floats(D->prim_kind[p], D->prim_nq[p], D->prim_flags[p]);
    int na = 0;
    for (int u = 0; u < D->prim_nq[p]; ++u) {
      const int j = D->prim_q0[p] + u;
      const int k = D->q_param[j];
      t.act[na_tab + u] = -1;
      t.actc[na_tab + u] = 0.f;
      if (k < 0 || D->q_coeff[j] == 0.0) continue;
      int slot = -1;
      for (int v = 0; v < u; ++v) {  // an earlier scalar of this primitive on the same parameter
        const int jv = D->prim_q0[p] + v;
        if (t.act[na_tab + v] >= 0 && D->q_param[jv] == k) { slot = t.act[na_tab + v]; break; }
      }
      if (slot < 0) {
        slot = na++;
        count[k]++;
      }
      t.act[na_tab + u] = slot;
      t.actc[na_tab + u] = (float)D->q_coeff[j];
    }
    t.nact[p] = na;
    na_tab += D->prim_nq[p];
  }
  t.nact_table = na_tab;
  t.auxd_n = auxd;
  t.auxf_n = auxf;
  t.ref_off[0] = 0;
  for (int k = 0; k < D->n_params; ++k) t.ref_off[k + 1] = t.ref_off[k] + count[k];
  t.nrefs = t.ref_off[D->n_params];
  for (int k = 0; k < D->n_params; ++k) count[k] = t.ref_off[k];
  for (int p = 0; p < D->n_prims; ++p) {
    int seen = 0;
    for (int u = 0; u < D->prim_nq[p]; ++u) {
      const int s = t.act[t.act_off[p] + u];
      if (s < 0 || s < seen) continue;  // slots are numbered in first-appearance order
      const int k = D->q_param[D->prim_q0[p] + u];
      const int r = count[k]++;
      t.ref_prim[r] = p;
      t.ref_qa[r] = s;
      t.ref_coeff[r] = 1.0;
      seen = s + 1;
    }
  }
}

inline void set_grid(const adg_design_desc* D, int tx, int ty, int tz, int nchain, GridDev& g) {
  auto lg = [](int v) { int l = 0; while ((1 << l) < v) ++l; return l; };
  const adg_grid& G = D->grid;
  g = GridDev{};
  g.nx = G.nx; g.ny = G.ny; g.nz = G.nz; g.C = G.ncomp;
  g.lx = lg(tx); g.ly = lg(ty); g.lz = lg(tz);
  g.ntx = (G.nx + tx - 1) / tx; g.nty = (G.ny + ty - 1) / ty; g.ntz = (G.nz + tz - 1) / tz;
  g.T = g.ntx * g.nty * g.ntz;
  for (int a = 0; a < 3; ++a) { g.offmin[a] = 1e9f; g.offmax[a] = -1e9f; }
  for (int c = 0; c < 3; ++c)
    for (int a = 0; a < 3; ++a) {
      g.off[c][a] = c < G.ncomp ? (float)G.off[c][a] : 0.f;
      if (c < G.ncomp) {
        g.offmin[a] = std::min(g.offmin[a], g.off[c][a]);
        g.offmax[a] = std::max(g.offmax[a], g.off[c][a]);
      }
    }
  const double dd[3] = {G.dx, G.dy, G.dz};
  for (int a = 0; a < 3; ++a) g.invd[a] = (float)(1.0 / dd[a]);
  g.eps_bg = (float)D->eps_bg;
  g.deps = (float)(D->eps_fg - D->eps_bg);
  g.logic = D->logic;
  g.nchain = nchain;
  g.nprims = D->n_prims;
  g.polar = 0;
  g.xform = 0;
  for (int p = 0; p < D->n_prims; ++p) {
    g.polar |= D->prim_kind[p] == ADG_PRIM_POLAR && !(D->prim_flags[p] & ADG_XFORM);
    g.xform |= (D->prim_flags[p] & ADG_XFORM) != 0;
  }
}

inline bool tile_ok(int tx, int ty, int tz) {
  auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
  return (tx == 32 || tx == 64) && pow2(ty) && ty <= 16 && pow2(tz) && tz <= 8 &&
         tx * ty * tz >= kBlock && tx * ty * tz <= kMaxTileCells;
}

// Static per-primitive facts the parameter map needs (the description's
// primitive table, kept by the caller).
struct PrimTable {
  const int *kind, *sigma, *flags, *q0, *nq;
  const double* kr;
  int n;
};

inline void anchor(double v, int& ai, float& af) {
  v = std::min(std::max(v, -1e8), 1e8);
  const double f = floor(v);
  ai = (int)f;
  af = (float)(v - f);
}

// inclusive cell-index range whose samples u = i + off (any component) can
// fall in [ulo, uhi], clipped to [0, n-1]; empty as lo > hi
inline void cell_range(double ulo, double uhi, float offmin, float offmax, int n, int& lo, int& hi) {
  const double a = floor(ulo - offmax - 1.0), b = ceil(uhi - offmin + 1.0);
  lo = (int)std::max(0.0, std::min((double)n, a));
  hi = (int)std::min((double)(n - 1), std::max(-1.0, b));
}

// The parameter map (hot-path step a1), FP64: q = b + a p; each primitive's
// cell-local anchors, value / derivative tile boxes and partial offset.
inline adg_status prepare_prims(const GridDev& g, const double d[3], const double o[3],
                                const PrimTable& P, const SlotTables& t, const double* q,
                                PrimRec* out, double* auxd, float* auxf, size_t* part_total,
                                Msg& m) {
  const int nn[3] = {g.nx, g.ny, g.nz};
  const int lt[3] = {g.lx, g.ly, g.lz};
  size_t part = 0;
  for (int pi = 0; pi < P.n; ++pi) {
    PrimRec R;
    memset(&R, 0, sizeof(R));
    R.kind = P.kind[pi];
    R.sigma = P.sigma[pi];
    R.flags = P.flags[pi];
    R.nact = t.nact[pi];
    R.act_off = t.act_off[pi];
    R.kr = (float)P.kr[pi];
    const double beta = kBand[R.sigma] / P.kr[pi];
    R.band = (float)beta;
    R.auxd_off = t.auxd_off[pi];
    R.auxf_off = t.auxf_off[pi];
    const double* Q = q + P.q0[pi];
    auto cellc = [&](double v, int ax) { return (v - o[ax]) / d[ax]; };
    int vlo[3], vhi[3], plo[3], phi[3];
    for (int a = 0; a < 3; ++a) { vlo[a] = 0; vhi[a] = nn[a] - 1; }
    auto zrange = [&]() {
      if (!(R.flags & kBoundZ)) return;
      const bool c5 = R.kind == kCircle || R.kind == kPolar;  // z0, z1 after cx, cy, R
      const double a = cellc(Q[c5 ? 3 : 0], 2);
      const double b = cellc(Q[c5 ? 4 : 1], 2);
      anchor(a, R.ai[4], R.af[4]);
      anchor(b, R.ai[5], R.af[5]);
      cell_range(a - 0.5, b + 0.5, g.offmin[2], g.offmax[2], g.nz, vlo[2], vhi[2]);
    };
    if (R.flags & kXformFlag) {
      // rotation / aspect transform (Sec. 4, item iii): the base evaluated at
      // the local point u = p + S^-1 R(-theta)(r - p); geometry in FP64 cells
      // relative to the pivot (dx == dy), see kXformHead
      const int base = R.kind;
      const int nb = P.nq[pi] - 5;
      const double* X5 = Q + nb;  // px, py, theta, sx, sy
      const double sx = X5[3], sy = X5[4];
      if (!(sx > 0.0) || !(sy > 0.0) || !fin(sx) || !fin(sy) || !fin(X5[2]))
        return m.set(ADG_EINVAL, "primitive %d: transform needs sx, sy > 0 and a finite angle", pi);
      R.kind = kXform;
      R.flags |= base << 8;
      const double cth = cos(X5[2]), sth = sin(X5[2]);
      const double pcx = cellc(X5[0], 0), pcy = cellc(X5[1], 1);
      double* A = auxd + R.auxd_off;
      A[0] = cth; A[1] = sth; A[2] = 1.0 / sx; A[3] = 1.0 / sy; A[4] = sx; A[5] = sy;
      R.ai[0] = (int)floor(std::min(std::max(pcx, -1e8), 1e8));
      R.ai[1] = (int)floor(std::min(std::max(pcy, -1e8), 1e8));
      A[6] = pcx - R.ai[0];
      A[7] = pcy - R.ai[1];
      double* B = A + kXformHead;
      auto lxy = [&](double v, int ax) { return (v - X5[ax]) / d[0]; };  // local cells
      // points whose hull holds every sample where the base can be nonzero
      double pts[2 * kMaxPolyVerts + 8];
      int npt = 0;
      auto square = [&](double cx, double cy, double h) {
        const double sq[8] = {cx - h, cy - h, cx + h, cy - h, cx + h, cy + h, cx - h, cy + h};
        for (int u = 0; u < 8; ++u) pts[npt++] = sq[u];
      };
      auto zext = [&](int iz0, int iz1) {  // exact z overlap (2D bases)
        if (!(R.flags & kBoundZ)) return;
        const double a = cellc(Q[iz0], 2), b = cellc(Q[iz1], 2);
        anchor(a, R.ai[4], R.af[4]);
        anchor(b, R.ai[5], R.af[5]);
        cell_range(a - 0.5, b + 0.5, g.offmin[2], g.offmax[2], g.nz, vlo[2], vhi[2]);
      };
      const double big = 1e7;
      if (base == kBox) {
        const bool bx = R.flags & kBoundX, by = R.flags & kBoundY;
        B[0] = bx ? lxy(Q[0], 0) : 0.0;
        B[1] = bx ? lxy(Q[1], 0) : 0.0;
        B[2] = by ? lxy(Q[2], 1) : 0.0;
        B[3] = by ? lxy(Q[3], 1) : 0.0;
        B[4] = cellc(Q[4], 2);
        B[5] = cellc(Q[5], 2);
        const double x0 = bx ? B[0] - beta : -big, x1 = bx ? B[1] + beta : big;
        const double y0 = by ? B[2] - beta : -big, y1 = by ? B[3] + beta : big;
        const double c4[8] = {x0, y0, x1, y0, x1, y1, x0, y1};
        for (int u = 0; u < 8; ++u) pts[npt++] = c4[u];
        if (R.flags & kBoundZ)
          cell_range(B[4] - beta, B[5] + beta, g.offmin[2], g.offmax[2], g.nz, vlo[2], vhi[2]);
      } else if (base == kCircle) {
        B[0] = lxy(Q[0], 0);
        B[1] = lxy(Q[1], 1);
        B[2] = Q[2] / d[0];
        square(B[0], B[1], fabs(B[2]) + beta);
        zext(3, 4);
      } else if (base == kPolar) {
        const int N = (nb - 5) / 2;
        R.naux = N;
        B[0] = lxy(Q[0], 0);
        B[1] = lxy(Q[1], 1);
        B[2] = Q[2] / d[0];
        double amp = 0.0;
        for (int n = 1; n <= N; ++n) {
          B[1 + 2 * n] = Q[3 + 2 * n] / d[0];
          B[2 + 2 * n] = Q[4 + 2 * n] / d[0];
          amp += fabs(B[1 + 2 * n]) + fabs(B[2 + 2 * n]);
        }
        square(B[0], B[1], std::max(B[2] + amp, 0.0) + beta);
        zext(3, 4);
      } else {  // polygon
        const int N = (nb - 2) / 2;
        R.naux = N;
        double* V = B + 1;
        double area2 = 0.0;
        for (int j = 0; j < N; ++j) {
          V[2 * j] = lxy(Q[2 + 2 * j], 0);
          V[2 * j + 1] = lxy(Q[3 + 2 * j], 1);
        }
        for (int j = 0; j < N; ++j) {
          const int j1 = (j + 1) % N;
          area2 += V[2 * j] * V[2 * j1 + 1] - V[2 * j1] * V[2 * j + 1];
        }
        const double sgn = area2 >= 0.0 ? 1.0 : -1.0;
        B[0] = sgn;
        // the polygon grown by beta along every edge normal: its vertices are
        // the crossings of consecutive offset edge lines n_e . x = c_e - beta
        for (int j = 0; j < N; ++j) {
          const int jp = (j + N - 1) % N, j1 = (j + 1) % N;
          double nx[2], ny[2], cc[2];
          const int es[2] = {jp, j};
          for (int u = 0; u < 2; ++u) {
            const int e = es[u], e1 = (e + 1) % N;
            const double ex = V[2 * e1] - V[2 * e], ey = V[2 * e1 + 1] - V[2 * e + 1];
            const double L = sqrt(ex * ex + ey * ey);
            if (!(L > 0.0)) return m.set(ADG_EINVAL, "polygon %d: repeated vertex %d", pi, e);
            nx[u] = -sgn * ey / L;
            ny[u] = sgn * ex / L;
            cc[u] = nx[u] * V[2 * e] + ny[u] * V[2 * e + 1] - beta;
          }
          const double det = nx[0] * ny[1] - ny[0] * nx[1];
          if (fabs(det) > 1e-3) {
            pts[npt++] = (cc[0] * ny[1] - ny[0] * cc[1]) / det;
            pts[npt++] = (nx[0] * cc[1] - cc[0] * nx[1]) / det;
          } else {  // nearly straight at vertex j: the vertex moved out by beta
            pts[npt++] = V[2 * j] - beta * nx[1];
            pts[npt++] = V[2 * j + 1] - beta * ny[1];
          }
          (void)j1;
        }
        zext(0, 1);
      }
      // the hull's image in world cells: r = p + R(theta) S u
      double wx0 = 1e300, wx1 = -1e300, wy0 = 1e300, wy1 = -1e300;
      for (int u = 0; u < npt; u += 2) {
        const double ux = sx * pts[u], uy = sy * pts[u + 1];
        const double wx = pcx + cth * ux - sth * uy, wy = pcy + sth * ux + cth * uy;
        wx0 = std::min(wx0, wx); wx1 = std::max(wx1, wx);
        wy0 = std::min(wy0, wy); wy1 = std::max(wy1, wy);
      }
      cell_range(wx0, wx1, g.offmin[0], g.offmax[0], g.nx, vlo[0], vhi[0]);
      cell_range(wy0, wy1, g.offmin[1], g.offmax[1], g.ny, vlo[1], vhi[1]);
      for (int a = 0; a < 3; ++a) { plo[a] = vlo[a]; phi[a] = vhi[a]; }
    } else if (R.kind == kBox) {
      for (int ax = 0; ax < 3; ++ax) {
        if (!(R.flags & (1 << ax))) continue;
        const double a = cellc(Q[2 * ax], ax), b = cellc(Q[2 * ax + 1], ax);
        anchor(a, R.ai[2 * ax], R.af[2 * ax]);
        anchor(b, R.ai[2 * ax + 1], R.af[2 * ax + 1]);
        const double w = (R.flags & kRectSigma) ? beta : 0.5;
        cell_range(a - w, b + w, g.offmin[ax], g.offmax[ax], nn[ax], vlo[ax], vhi[ax]);
      }
      for (int a = 0; a < 3; ++a) { plo[a] = vlo[a]; phi[a] = vhi[a]; }
    } else if (R.kind == kCircle) {
      const double cx = cellc(Q[0], 0), cy = cellc(Q[1], 1), Rc = Q[2] / d[0];
      anchor(cx, R.ai[0], R.af[0]);
      anchor(cy, R.ai[1], R.af[1]);
      const double R2 = Rc * Rc;
      R.g[0] = (float)Rc;
      R.g[1] = (float)R2;
      R.g[2] = (float)(R2 - (double)R.g[1]);
      R.g[3] = Rc < 0 ? 1.f : 0.f;
      const double ext = fabs(Rc) + beta;
      cell_range(cx - ext, cx + ext, g.offmin[0], g.offmax[0], g.nx, vlo[0], vhi[0]);
      cell_range(cy - ext, cy + ext, g.offmin[1], g.offmax[1], g.ny, vlo[1], vhi[1]);
      zrange();
      for (int a = 0; a < 3; ++a) { plo[a] = vlo[a]; phi[a] = vhi[a]; }
    } else if (R.kind == kPolar) {
      // Polar2D: R0 and the Fourier coefficients in cells (FP64 on the
      // device); g[1] / g[2] bound R(theta) from above / below for the binner
      const int N = (P.nq[pi] - 5) / 2;
      R.naux = N;
      const double cx = cellc(Q[0], 0), cy = cellc(Q[1], 1);
      anchor(cx, R.ai[0], R.af[0]);
      anchor(cy, R.ai[1], R.af[1]);
      double A[1 + 2 * kMaxPolarHarm];  // N <= kMaxPolarHarm (validated)
      A[0] = Q[2] / d[0];
      double amp = 0.0;
      for (int n = 1; n <= N; ++n) {
        A[2 * n - 1] = Q[3 + 2 * n] / d[0];
        A[2 * n] = Q[4 + 2 * n] / d[0];
        amp += fabs(A[2 * n - 1]) + fabs(A[2 * n]);
      }
      float* F = auxf + R.auxf_off;  // hi + lo pairs: about 48 bits, read back in FP64
      for (int j = 0; j <= 2 * N; ++j) {
        F[2 * j] = (float)A[j];
        F[2 * j + 1] = (float)(A[j] - (double)F[2 * j]);
      }
      const double rmax = A[0] + amp, rmin = A[0] - amp;
      R.g[0] = (float)A[0];
      R.g[1] = (float)rmax;
      R.g[2] = (float)rmin;
      const double ext = std::max(rmax, 0.0) + beta + 1e-6 * (1.0 + fabs(rmax));
      cell_range(cx - ext, cx + ext, g.offmin[0], g.offmax[0], g.nx, vlo[0], vhi[0]);
      cell_range(cy - ext, cy + ext, g.offmin[1], g.offmax[1], g.ny, vlo[1], vhi[1]);
      zrange();
      for (int a = 0; a < 3; ++a) { plo[a] = vlo[a]; phi[a] = vhi[a]; }
    } else if (R.kind == kGraph) {
      const int M = vertices_of(R.kind, P.nq[pi]);
      R.naux = M;
      double* X = auxd + R.auxd_off;
      double* Y = X + M;
      double* iX = Y + M;
      float* Xf = auxf + R.auxf_off;
      double ymin = 1e300, ymax = -1e300;
      for (int j = 0; j < M; ++j) {
        X[j] = cellc(Q[2 + j], 0);
        Y[j] = cellc(Q[2 + M + j], 1);
        Xf[j] = (float)X[j];
        ymin = std::min(ymin, Y[j]);
        ymax = std::max(ymax, Y[j]);
        if (j > 0 && !(X[j] > X[j - 1]))
          return m.set(ADG_EINVAL, "graph %d: knots must increase strictly in x", pi);
      }
      for (int j = 0; j + 1 < M; ++j) iX[j] = 1.0 / (X[j + 1] - X[j]);
      iX[M - 1] = 0.0;
      zrange();
      for (int a = 0; a < 3; ++a) { plo[a] = vlo[a]; phi[a] = vhi[a]; }
      int lo, hi;
      cell_range(ymin - beta, ymax + beta, g.offmin[1], g.offmax[1], g.ny, lo, hi);
      plo[1] = lo;
      phi[1] = hi;
      if (R.flags & kGraphAbove) vlo[1] = lo; else vhi[1] = hi;
    } else {  // polygon
      const int N = vertices_of(R.kind, P.nq[pi]);
      R.naux = N;
      double* X = auxd + R.auxd_off;
      double* Y = X + N;
      double* NX = Y + N;
      double* NY = NX + N;
      double* C = NY + N;
      double* IL = C + N;
      double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300, area2 = 0.0;
      for (int j = 0; j < N; ++j) {
        X[j] = cellc(Q[2 + 2 * j], 0);
        Y[j] = cellc(Q[3 + 2 * j], 1);
        xmin = std::min(xmin, X[j]); xmax = std::max(xmax, X[j]);
        ymin = std::min(ymin, Y[j]); ymax = std::max(ymax, Y[j]);
      }
      for (int j = 0; j < N; ++j) {
        const int j1 = (j + 1) % N;
        area2 += X[j] * Y[j1] - X[j1] * Y[j];
      }
      const double sgn = area2 >= 0.0 ? 1.0 : -1.0;
      R.g[0] = (float)sgn;
      for (int j = 0; j < N; ++j) {
        const int j1 = (j + 1) % N;
        const double ex = X[j1] - X[j], ey = Y[j1] - Y[j];
        const double L = sqrt(ex * ex + ey * ey);
        if (!(L > 0.0)) return m.set(ADG_EINVAL, "polygon %d: repeated vertex %d", pi, j);
        NX[j] = -sgn * ey / L;  // inward unit normal
        NY[j] = sgn * ex / L;
        C[j] = NX[j] * X[j] + NY[j] * Y[j];
        IL[j] = 1.0 / L;
      }
      {  // rigid: all vertex x scalars share one slot and coefficient, all y too
        const int* ac = t.act + t.act_off[pi];
        const float* cc = t.actc + t.act_off[pi];
        bool rigid = true;
        for (int j = 1; j < N && rigid; ++j)
          rigid = ac[2 + 2 * j] == ac[2] && cc[2 + 2 * j] == cc[2] && ac[3 + 2 * j] == ac[3] &&
                  cc[3 + 2 * j] == cc[3];
        if (rigid) R.flags |= kPolyRigid;
      }
      // fp32 edge table for the device: vertex relative to the anchor cell and
      // the normal as hi + lo pairs (about 48 bits), so that a sample's edge
      // distance needs no FP64
      R.ai[0] = (int)std::floor(X[0]);
      R.ai[1] = (int)std::floor(Y[0]);
      float* E = auxf + R.auxf_off;
      auto split = [](double v, float* hl) {
        hl[0] = (float)v;
        hl[1] = (float)(v - (double)hl[0]);
      };
      for (int j = 0; j < N; ++j) {
        const int j1 = (j + 1) % N;
        float* e = E + kPolyEdgeFloats * j;
        split(X[j] - R.ai[0], e + 0);
        split(Y[j] - R.ai[1], e + 2);
        split(NX[j], e + 4);
        split(NY[j], e + 6);
        e[8] = (float)(X[j1] - X[j]);
        e[9] = (float)(Y[j1] - Y[j]);
        e[10] = (float)IL[j];
      }
      cell_range(xmin - beta, xmax + beta, g.offmin[0], g.offmax[0], g.nx, vlo[0], vhi[0]);
      cell_range(ymin - beta, ymax + beta, g.offmin[1], g.offmax[1], g.ny, vlo[1], vhi[1]);
      zrange();
      for (int a = 0; a < 3; ++a) { plo[a] = vlo[a]; phi[a] = vhi[a]; }
    }
    int np = 1;
    for (int a = 0; a < 3; ++a) {
      if (vlo[a] > vhi[a]) { R.tb[2 * a] = 0; R.tb[2 * a + 1] = 0; }
      else { R.tb[2 * a] = vlo[a] >> lt[a]; R.tb[2 * a + 1] = (vhi[a] >> lt[a]) + 1; }
      if (plo[a] > phi[a]) { R.pb[2 * a] = 0; R.pb[2 * a + 1] = 0; }
      else { R.pb[2 * a] = plo[a] >> lt[a]; R.pb[2 * a + 1] = (phi[a] >> lt[a]) + 1; }
      np *= R.pb[2 * a + 1] - R.pb[2 * a];
    }
    R.npb = R.nact > 0 ? np : 0;
    R.part_off = (int)part;
    part += (size_t)R.nact * R.npb;
    if (part > ((size_t)1 << 31)) return m.set(ADG_EINVAL, "partial buffer exceeds 2^31 entries");
    out[pi] = R;
  }
  *part_total = part;
  return ADG_OK;
}

inline adg_status map_params(int n_q, const double* qb, const double* qa, const int* qp,
                             const double* p, double* q, Msg& m) {
  for (int j = 0; j < n_q; ++j) {
    q[j] = qb[j];
    if (qp[j] >= 0) q[j] += qa[j] * p[qp[j]];
    if (!std::isfinite(q[j])) return m.set(ADG_EINVAL, "geometric scalar %d is not finite", j);
  }
  return ADG_OK;
}

}  // namespace host
}  // namespace adg
