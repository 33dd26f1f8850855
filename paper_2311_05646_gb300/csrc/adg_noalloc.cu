// adg_noalloc.cu -- adg_grad_noalloc: the Eq. 1 gradient for callers that
// cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is unavailable or forbidden --
// for example a host process whose device memory is owned by another runtime
// with a fixed arena, plug-ins loaded into a simulator that must not grow its
// footprint after start-up, or callers working under a strict device-memory
// budget.  adg_grad (the regular path) allocates per-design tables and a
// growing partial buffer; this variant allocates nothing.
//
// How: every device-side table and scratch buffer of the gradient (design
// tables, primitive records, per-tile programs, band-tile list, partial sums,
// error word) lives in one file-scope static device array of fixed size,
// kNoAllocScratchBytes (32 MiB).  Every GPU that loads libadg holds that array
// until the process exits.  Host-side tables live in fixed static host buffers
// guarded by a mutex; nothing is taken from the heap either.  The caller passes
// the design description, the parameters, the fields, w and the output.
//
// Set-up: the first call on each device (with that device current) obtains
// the array's device address with cudaGetSymbolAddress; make that first call
// before any stream capture.  In host code the array's name is only a
// host-side stand-in, never passed to a kernel.
//
// Sharing: all calls use the same array, which keeps the last call's contents;
// each call clears what must start at zero (error word, counters, partials).
// Calls that overlap on the GPU (different streams, or another host thread
// between enqueue and completion) race on the array -- serialise them.  The
// call returns after its stream work has completed, so that device-side
// checks can be reported.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "../../include/adg.h"
#include "adg_internal.h"

using namespace adg;

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// fixed host-side limits of this variant
constexpr int kNAMaxPrims = 4096;
constexpr int kNAMaxQ = 32768;
constexpr int kNAMaxOps = 16384;
constexpr int kNAMaxParams = 16384;
constexpr int kNAMaxDevices = 64;

struct NoAllocHost {
  // description compile
  int node_code[kNAMaxOps], node_arg[kNAMaxOps], node_k0[kNAMaxOps], node_nk[kNAMaxOps];
  int kids[kNAMaxOps], stack[kNAMaxOps];
  int chain[2 * kNAMaxOps];
  int act[kNAMaxQ], nact[kNAMaxPrims], act_off[kNAMaxPrims];
  int auxd_off[kNAMaxPrims], auxf_off[kNAMaxPrims];
  int ref_count[kNAMaxParams + 1], ref_off[kNAMaxParams + 1], ref_prim[kNAMaxQ], ref_qa[kNAMaxQ];
  double ref_coeff[kNAMaxQ];
  // per call
  double q[kNAMaxQ];
  PrimRec prims[kNAMaxPrims];
  double auxd[3 * kNAMaxQ];
  float auxf[kNAMaxQ];
};

NoAllocHost g_host;
std::mutex g_mu;
void* g_sym[kNAMaxDevices];
bool g_sym_ok[kNAMaxDevices];

const double kBandNA[5] = {0.5, 20.0, 0.70710678118654752, 1.5707963267948966, 4.5};

adg_status na_fail(adg_status st, const char* fmt, ...);

#define NACU(call)                                                                            \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return na_fail(ADG_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

int na_nchain = 0;

bool na_emit(int id, int depth) {
  if (depth > 4096) return false;
  const int code = g_host.node_code[id];
  if (code == ADG_OP_PUSH) {
    g_host.chain[na_nchain++] = (cPush << 24) | g_host.node_arg[id];
    return true;
  }
  const int* k = g_host.kids + g_host.node_k0[id];
  const int nk = g_host.node_nk[id];
  if (code == ADG_OP_DIFF) {
    if (!na_emit(k[0], depth + 1) || !na_emit(k[1], depth + 1)) return false;
    g_host.chain[na_nchain++] = cDiff << 24;
    return true;
  }
  const int c = code == ADG_OP_UNION ? cUnion : cInter;
  if (!na_emit(k[0], depth + 1)) return false;
  for (int t = 1; t < nk; ++t) {
    if (!na_emit(k[t], depth + 1)) return false;
    g_host.chain[na_nchain++] = c << 24;
  }
  return true;
}

void na_anchor(double v, int& ai, float& af) {
  v = std::min(std::max(v, -1e8), 1e8);
  const double f = floor(v);
  ai = (int)f;
  af = (float)(v - f);
}

void na_range(double ulo, double uhi, float offmin, float offmax, int n, int& lo, int& hi) {
  const double a = floor(ulo - offmax - 1.0), b = ceil(uhi - offmin + 1.0);
  lo = (int)std::max(0.0, std::min((double)n, a));
  hi = (int)std::min((double)(n - 1), std::max(-1.0, b));
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

namespace {
// messages go to the library's thread-local adg_last_error()
adg_status na_fail(adg_status st, const char* fmt, ...) {
  char msg[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof(msg), fmt, ap);
  va_end(ap);
  set_last_error(msg);
  return st;
}
}  // namespace

extern "C" adg_status adg_grad_noalloc(const adg_design_desc* D, const adg_tile_opts* tiles,
                                       const double* h_params, const float* const d_efwd[3],
                                       const float* const d_eadj[3], const float* w,
                                       float* d_grad, void* stream) {
  std::lock_guard<std::mutex> lock(g_mu);
  NoAllocHost& H = g_host;
  if (!D || !d_efwd || !d_eadj || !w) return na_fail(ADG_EINVAL, "adg_grad_noalloc: NULL argument");
  const adg_grid& G = D->grid;
  // ---- validation (the same rules as adg_design_create) ----
  if (G.nx < 1 || G.ny < 1 || G.nz < 1 || G.nx > 8192 || G.ny > 8192 || G.nz > 8192 ||
      G.ncomp < 1 || G.ncomp > 3)
    return na_fail(ADG_EINVAL, "grid %dx%dx%d x %d components not supported", G.nx, G.ny, G.nz,
                   G.ncomp);
  if (!(G.dx > 0) || !(G.dy > 0) || !(G.dz > 0) || !std::isfinite(G.dx) || !std::isfinite(G.dy) ||
      !std::isfinite(G.dz) || !std::isfinite(G.ox) || !std::isfinite(G.oy) || !std::isfinite(G.oz))
    return na_fail(ADG_EINVAL, "grid spacing / origin invalid");
  for (int c = 0; c < G.ncomp; ++c)
    for (int a = 0; a < 3; ++a)
      if (!(fabs(G.off[c][a]) <= 1.0)) return na_fail(ADG_EINVAL, "offset off[%d][%d] invalid", c, a);
  if (D->logic != ADG_LOGIC_PRODUCT && D->logic != ADG_LOGIC_CLAMP)
    return na_fail(ADG_EINVAL, "logic %d unknown", D->logic);
  if (!std::isfinite(D->eps_bg) || !std::isfinite(D->eps_fg) || D->reserved != 0)
    return na_fail(ADG_EINVAL, "eps levels / reserved invalid");
  if (D->n_prims < 1 || D->n_prims > kNAMaxPrims || D->n_q < 0 || D->n_q > kNAMaxQ ||
      D->n_ops < 1 || D->n_ops > kNAMaxOps || D->n_params < 0 || D->n_params > kNAMaxParams)
    return na_fail(ADG_EINVAL,
                   "adg_grad_noalloc limits: primitives 1..%d, scalars <= %d, ops 1..%d, "
                   "params <= %d (got %d, %d, %d, %d)",
                   kNAMaxPrims, kNAMaxQ, kNAMaxOps, kNAMaxParams, D->n_prims, D->n_q, D->n_ops,
                   D->n_params);
  if ((D->n_q > 0 && (!D->q_base || !D->q_coeff || !D->q_param)) || !D->prim_kind ||
      !D->prim_sigma || !D->prim_flags || !D->prim_q0 || !D->prim_nq || !D->prim_kr || !D->ops ||
      (D->n_params > 0 && (!h_params || !d_grad)))
    return na_fail(ADG_EINVAL, "description array or parameter pointer is NULL");
  for (int c = 0; c < G.ncomp; ++c)
    if (!d_efwd[c] || !d_eadj[c]) return na_fail(ADG_EINVAL, "field of component %d is NULL", c);
  for (int j = 0; j < D->n_q; ++j)
    if (D->q_param[j] < -1 || D->q_param[j] >= D->n_params || !std::isfinite(D->q_base[j]) ||
        !std::isfinite(D->q_coeff[j]))
      return na_fail(ADG_EINVAL, "geometric scalar %d invalid", j);
  for (int p = 0; p < D->n_prims; ++p) {
    const int k = D->prim_kind[p], n = D->prim_nq[p], q0 = D->prim_q0[p], s = D->prim_sigma[p];
    if (q0 < 0 || n < 0 || q0 + n > D->n_q || s < 0 || s > 4 || !(D->prim_kr[p] > 0) ||
        !std::isfinite(D->prim_kr[p]))
      return na_fail(ADG_EINVAL, "primitive %d invalid", p);
    if ((k == ADG_PRIM_BOX && n != 6) || (k == ADG_PRIM_CIRCLE && n != 5) ||
        (k == ADG_PRIM_GRAPH && (n < 6 || (n - 2) % 2)) || k == ADG_PRIM_POLYGON || k < 0 ||
        k > ADG_PRIM_GRAPH)
      return na_fail(ADG_EINVAL, "primitive %d: kind %d with %d scalars not supported", p, k, n);
    if (k == ADG_PRIM_CIRCLE && fabs(G.dx - G.dy) > 1e-12 * G.dx)
      return na_fail(ADG_EINVAL, "circle %d needs dx == dy", p);
  }
  // ---- program: postfix -> tree -> binary chain ----
  int sp = 0, nk = 0;
  for (int i = 0; i < D->n_ops; ++i) {
    const int wd = D->ops[i], code = (wd >> 24) & 0xff, arg = wd & 0xffffff;
    int need = 0;
    if (code == ADG_OP_PUSH) {
      if (arg < 0 || arg >= D->n_prims) return na_fail(ADG_EINVAL, "op %d: bad primitive", i);
    } else if (code == ADG_OP_UNION || code == ADG_OP_INTERSECT) {
      need = arg;
      if (need < 1) return na_fail(ADG_EINVAL, "op %d: operand count %d", i, need);
    } else if (code == ADG_OP_DIFF) {
      need = 2;
    } else {
      return na_fail(ADG_EINVAL, "op %d: unknown code %d", i, code);
    }
    if (sp < need) return na_fail(ADG_EINVAL, "op %d: stack underflow", i);
    H.node_code[i] = code;
    H.node_arg[i] = arg;
    H.node_k0[i] = nk;
    H.node_nk[i] = need;
    for (int t = 0; t < need; ++t) H.kids[nk + t] = H.stack[sp - need + t];
    nk += need;
    sp -= need;
    H.stack[sp++] = i;
  }
  if (sp != 1) return na_fail(ADG_EINVAL, "program leaves %d values on the stack", sp);
  na_nchain = 0;
  if (!na_emit(H.stack[0], 0)) return na_fail(ADG_EINVAL, "program nesting too deep");
  {
    int s2 = 0, mx = 0;
    for (int t = 0; t < na_nchain; ++t) {
      s2 += ((H.chain[t] >> 24) == cPush) ? 1 : -1;
      mx = std::max(mx, s2);
    }
    if (mx > kMaxDepth) return na_fail(ADG_EINVAL, "program nesting %d > %d", mx, kMaxDepth);
  }
  // ---- tile shape and grid ----
  int tx = 32, ty = 4, tz = 4;
  if (tiles && (tiles->tx || tiles->ty || tiles->tz)) { tx = tiles->tx; ty = tiles->ty; tz = tiles->tz; }
  auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
  if (!(tx == 32 || tx == 64) || !pow2(ty) || ty > 16 || !pow2(tz) || tz > 8 || tx * ty * tz < kBlock)
    return na_fail(ADG_EINVAL, "tile %dx%dx%d not supported", tx, ty, tz);
  auto lg = [](int v) { int l = 0; while ((1 << l) < v) ++l; return l; };
  GridDev g{};
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
  const double dd[3] = {G.dx, G.dy, G.dz}, oo[3] = {G.ox, G.oy, G.oz};
  for (int a = 0; a < 3; ++a) g.invd[a] = (float)(1.0 / dd[a]);
  g.eps_bg = (float)D->eps_bg;
  g.deps = (float)(D->eps_fg - D->eps_bg);
  g.logic = D->logic;
  g.nchain = na_nchain;
  // ---- active scalars, parameter references, aux layout ----
  int auxd_n = 0, auxf_n = 0;
  for (int k = 0; k <= D->n_params; ++k) H.ref_count[k] = 0;
  for (int p = 0; p < D->n_prims; ++p) {
    H.auxd_off[p] = auxd_n;
    H.auxf_off[p] = auxf_n;
    if (D->prim_kind[p] == ADG_PRIM_GRAPH) {
      const int M = (D->prim_nq[p] - 2) / 2;
      auxd_n += 3 * M;
      auxf_n += M;
    }
  }
  int nact_table = 0;
  for (int p = 0; p < D->n_prims; ++p) {
    H.act_off[p] = nact_table;
    int na = 0;
    for (int t = 0; t < D->prim_nq[p]; ++t) {
      const int j = D->prim_q0[p] + t;
      if (nact_table >= kNAMaxQ) return na_fail(ADG_EINVAL, "too many primitive scalars (> %d)", kNAMaxQ);
      if (D->q_param[j] >= 0 && D->q_coeff[j] != 0.0) {
        H.act[nact_table++] = na++;
        H.ref_count[D->q_param[j]]++;
      } else {
        H.act[nact_table++] = -1;
      }
    }
    H.nact[p] = na;
  }
  if (auxd_n > 3 * kNAMaxQ || auxf_n > kNAMaxQ) return na_fail(ADG_EINVAL, "graph knots exceed limits");
  H.ref_off[0] = 0;
  for (int k = 0; k < D->n_params; ++k) H.ref_off[k + 1] = H.ref_off[k] + H.ref_count[k];
  const int nrefs = D->n_params > 0 ? H.ref_off[D->n_params] : 0;
  if (nrefs > kNAMaxQ) return na_fail(ADG_EINVAL, "too many parameter references");
  for (int k = 0; k < D->n_params; ++k) H.ref_count[k] = H.ref_off[k];
  for (int p = 0; p < D->n_prims; ++p) {
    int na = 0;
    for (int t = 0; t < D->prim_nq[p]; ++t) {
      const int j = D->prim_q0[p] + t;
      if (D->q_param[j] >= 0 && D->q_coeff[j] != 0.0) {
        const int r = H.ref_count[D->q_param[j]]++;
        H.ref_prim[r] = p;
        H.ref_qa[r] = na++;
        H.ref_coeff[r] = D->q_coeff[j];
      }
    }
  }
  // ---- parameter map (FP64) and primitive records ----
  for (int j = 0; j < D->n_q; ++j) {
    H.q[j] = D->q_base[j];
    if (D->q_param[j] >= 0) H.q[j] += D->q_coeff[j] * h_params[D->q_param[j]];
    if (!std::isfinite(H.q[j])) return na_fail(ADG_EINVAL, "geometric scalar %d not finite", j);
  }
  const int nn[3] = {g.nx, g.ny, g.nz};
  const int lt[3] = {g.lx, g.ly, g.lz};
  size_t part = 0;
  for (int pi = 0; pi < D->n_prims; ++pi) {
    PrimRec& R = H.prims[pi];
    memset(&R, 0, sizeof(R));
    R.kind = D->prim_kind[pi];
    R.sigma = D->prim_sigma[pi];
    R.flags = D->prim_flags[pi];
    R.nact = H.nact[pi];
    R.act_off = H.act_off[pi];
    R.kr = (float)D->prim_kr[pi];
    const double beta = kBandNA[R.sigma] / D->prim_kr[pi];
    R.band = (float)beta;
    R.auxd_off = H.auxd_off[pi];
    R.auxf_off = H.auxf_off[pi];
    const double* Q = H.q + D->prim_q0[pi];
    auto cellc = [&](double v, int ax) { return (v - oo[ax]) / dd[ax]; };
    int vlo[3], vhi[3], plo[3], phi[3];
    for (int a = 0; a < 3; ++a) { vlo[a] = 0; vhi[a] = nn[a] - 1; }
    auto zrange = [&]() {
      if (!(R.flags & kBoundZ)) return;
      const double a = cellc(Q[R.kind == kCircle ? 3 : 0], 2);
      const double b = cellc(Q[R.kind == kCircle ? 4 : 1], 2);
      na_anchor(a, R.ai[4], R.af[4]);
      na_anchor(b, R.ai[5], R.af[5]);
      na_range(a - 0.5, b + 0.5, g.offmin[2], g.offmax[2], g.nz, vlo[2], vhi[2]);
    };
    if (R.kind == kBox) {
      for (int ax = 0; ax < 3; ++ax) {
        if (!(R.flags & (1 << ax))) continue;
        const double a = cellc(Q[2 * ax], ax), b = cellc(Q[2 * ax + 1], ax);
        na_anchor(a, R.ai[2 * ax], R.af[2 * ax]);
        na_anchor(b, R.ai[2 * ax + 1], R.af[2 * ax + 1]);
        const double wd = (R.flags & kRectSigma) ? beta : 0.5;
        na_range(a - wd, b + wd, g.offmin[ax], g.offmax[ax], nn[ax], vlo[ax], vhi[ax]);
      }
      for (int a = 0; a < 3; ++a) { plo[a] = vlo[a]; phi[a] = vhi[a]; }
    } else if (R.kind == kCircle) {
      const double cx = cellc(Q[0], 0), cy = cellc(Q[1], 1), Rc = Q[2] / dd[0];
      na_anchor(cx, R.ai[0], R.af[0]);
      na_anchor(cy, R.ai[1], R.af[1]);
      const double R2 = Rc * Rc;
      R.g[0] = (float)Rc;
      R.g[1] = (float)R2;
      R.g[2] = (float)(R2 - (double)R.g[1]);
      R.g[3] = Rc < 0 ? 1.f : 0.f;
      const double ext = fabs(Rc) + beta;
      na_range(cx - ext, cx + ext, g.offmin[0], g.offmax[0], g.nx, vlo[0], vhi[0]);
      na_range(cy - ext, cy + ext, g.offmin[1], g.offmax[1], g.ny, vlo[1], vhi[1]);
      zrange();
      for (int a = 0; a < 3; ++a) { plo[a] = vlo[a]; phi[a] = vhi[a]; }
    } else {
      const int M = (D->prim_nq[pi] - 2) / 2;
      R.naux = M;
      double* X = H.auxd + R.auxd_off;
      double* Y = X + M;
      double* iX = Y + M;
      float* Xf = H.auxf + R.auxf_off;
      double ymin = 1e300, ymax = -1e300;
      for (int j = 0; j < M; ++j) {
        X[j] = cellc(Q[2 + j], 0);
        Y[j] = cellc(Q[2 + M + j], 1);
        Xf[j] = (float)X[j];
        ymin = std::min(ymin, Y[j]);
        ymax = std::max(ymax, Y[j]);
        if (j > 0 && !(X[j] > X[j - 1]))
          return na_fail(ADG_EINVAL, "graph %d: knots must increase strictly in x", pi);
      }
      for (int j = 0; j + 1 < M; ++j) iX[j] = 1.0 / (X[j + 1] - X[j]);
      iX[M - 1] = 0.0;
      zrange();
      for (int a = 0; a < 3; ++a) { plo[a] = vlo[a]; phi[a] = vhi[a]; }
      int lo, hi;
      na_range(ymin - beta, ymax + beta, g.offmin[1], g.offmax[1], g.ny, lo, hi);
      plo[1] = lo;
      phi[1] = hi;
      if (R.flags & kGraphAbove) vlo[1] = lo; else vhi[1] = hi;
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
  }
  // ---- carve the static scratch; reject what does not fit ----
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off = align256(off + bytes); return o; };
  const size_t o_err = take(sizeof(int));
  const size_t o_cnt = take(4 * sizeof(int));
  const size_t o_chain = take(sizeof(int) * na_nchain);
  const size_t o_act = take(sizeof(int) * std::max(nact_table, 1));
  const size_t o_roff = take(sizeof(int) * (D->n_params + 1));
  const size_t o_rprim = take(sizeof(int) * std::max(nrefs, 1));
  const size_t o_rqa = take(sizeof(int) * std::max(nrefs, 1));
  const size_t o_rcoef = take(sizeof(double) * std::max(nrefs, 1));
  const size_t o_prims = take(sizeof(PrimRec) * D->n_prims);
  const size_t o_auxd = take(sizeof(double) * std::max(auxd_n, 1));
  const size_t o_auxf = take(sizeof(float) * std::max(auxf_n, 1));
  const size_t o_progs = take(sizeof(TileProg) * (size_t)g.T);
  const size_t o_list = take(sizeof(int) * (size_t)g.T);
  const size_t o_part = take(sizeof(float) * std::max<size_t>(part, 1));
  if (off > kNoAllocScratchBytes)
    return na_fail(ADG_EINVAL,
                   "adg_grad_noalloc: this design needs %zu bytes of scratch (%d tiles, %zu "
                   "partials); the static scratch holds %zu bytes -- use a larger tile shape or "
                   "adg_grad",
                   off, g.T, part, kNoAllocScratchBytes);
  // ---- set-up once per device: the array's device address ----
  int dev = 0;
  NACU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNAMaxDevices) return na_fail(ADG_EINVAL, "device %d out of range", dev);
  if (!g_sym_ok[dev]) {
    void* ptr = nullptr;
    NACU(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    g_sym[dev] = ptr;
    g_sym_ok[dev] = true;
  }
  unsigned char* base = static_cast<unsigned char*>(g_sym[dev]);
  cudaStream_t s = (cudaStream_t)stream;
  int* d_err = reinterpret_cast<int*>(base + o_err);
  int* d_cnt = reinterpret_cast<int*>(base + o_cnt);
  int* d_chain = reinterpret_cast<int*>(base + o_chain);
  int* d_act = reinterpret_cast<int*>(base + o_act);
  int* d_roff = reinterpret_cast<int*>(base + o_roff);
  int* d_rprim = reinterpret_cast<int*>(base + o_rprim);
  int* d_rqa = reinterpret_cast<int*>(base + o_rqa);
  double* d_rcoef = reinterpret_cast<double*>(base + o_rcoef);
  PrimRec* d_prims = reinterpret_cast<PrimRec*>(base + o_prims);
  double* d_auxd = reinterpret_cast<double*>(base + o_auxd);
  float* d_auxf = reinterpret_cast<float*>(base + o_auxf);
  TileProg* d_progs = reinterpret_cast<TileProg*>(base + o_progs);
  int* d_list = reinterpret_cast<int*>(base + o_list);
  float* d_part = reinterpret_cast<float*>(base + o_part);
  // ---- upload, clear, launch (binner -> VJP -> finalize) ----
  NACU(cudaMemsetAsync(d_err, 0, sizeof(int), s));
  NACU(cudaMemsetAsync(d_cnt, 0, 4 * sizeof(int), s));
  NACU(cudaMemcpyAsync(d_chain, H.chain, sizeof(int) * na_nchain, cudaMemcpyHostToDevice, s));
  if (nact_table)
    NACU(cudaMemcpyAsync(d_act, H.act, sizeof(int) * nact_table, cudaMemcpyHostToDevice, s));
  NACU(cudaMemcpyAsync(d_roff, H.ref_off, sizeof(int) * (D->n_params + 1), cudaMemcpyHostToDevice, s));
  if (nrefs) {
    NACU(cudaMemcpyAsync(d_rprim, H.ref_prim, sizeof(int) * nrefs, cudaMemcpyHostToDevice, s));
    NACU(cudaMemcpyAsync(d_rqa, H.ref_qa, sizeof(int) * nrefs, cudaMemcpyHostToDevice, s));
    NACU(cudaMemcpyAsync(d_rcoef, H.ref_coeff, sizeof(double) * nrefs, cudaMemcpyHostToDevice, s));
  }
  NACU(cudaMemcpyAsync(d_prims, H.prims, sizeof(PrimRec) * D->n_prims, cudaMemcpyHostToDevice, s));
  if (auxd_n) NACU(cudaMemcpyAsync(d_auxd, H.auxd, sizeof(double) * auxd_n, cudaMemcpyHostToDevice, s));
  if (auxf_n) NACU(cudaMemcpyAsync(d_auxf, H.auxf, sizeof(float) * auxf_n, cudaMemcpyHostToDevice, s));
  if (part) NACU(cudaMemsetAsync(d_part, 0, sizeof(float) * part, s));
  VjpArgs va{};
  for (int c = 0; c < G.ncomp; ++c) {
    va.ef[c] = reinterpret_cast<const float2*>(d_efwd[c]);
    va.ea[c] = reinterpret_cast<const float2*>(d_eadj[c]);
    va.w[c] = make_float2(w[2 * c], w[2 * c + 1]);
  }
  int sms = 1;
  NACU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  NACU(launch_bin(g, d_chain, d_prims, d_auxf, d_auxd, d_progs, d_list, d_cnt, d_err, s));
  NACU(launch_vjp(g, d_progs, d_list, d_cnt, d_prims, d_act, d_auxf, d_auxd, va, d_part, d_err,
                  sms * vjp_blocks_per_sm(), s));
  NACU(launch_finalize(D->n_params, d_roff, d_rprim, d_rqa, d_rcoef, d_prims, d_part, d_grad, s));
  // ---- wait and report device-side checks ----
  int herr = 0;
  NACU(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  NACU(cudaStreamSynchronize(s));
  if (herr)
    return na_fail(ADG_EDEVICE, "device check failed (bits 0x%x); use a smaller tile shape", herr);
  return ADG_OK;
}
