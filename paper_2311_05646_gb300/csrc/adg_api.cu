// adg_api.cu -- host side of libadg: the C ABI of include/adg.h.
//
// Design creation validates the description and compiles it (chained logic
// program, active-scalar table, parameter -> (primitive, scalar) references).
// Each build / gradient call runs the parameter map in FP64 on the host
// (q = b + a p, cell-local anchors, value- and derivative-support tile boxes,
// partial-buffer offsets; O(primitives), microseconds), uploads the primitive
// records, then enqueues binner -> build, or binner -> VJP -> finalize, on the
// caller's stream.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/adg.h"
#include "adg_internal.h"

using namespace adg;

namespace {

thread_local std::string g_err = "no error";

adg_status fail(adg_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define CU(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(e_ == cudaErrorMemoryAllocation ? ADG_ENOMEM : ADG_ECUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                  \
  } while (0)

// transition half-widths of the sigma kinds in the unit variable (beyond them
// the function is 0 or 1 with zero slope; the sigmoid's tail is below 2.1e-9)
const double kBand[5] = {0.5, 20.0, 0.70710678118654752, 1.5707963267948966, 4.5};

int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

template <class T>
cudaError_t upload(T** dptr, const std::vector<T>& h) {
  *dptr = nullptr;
  size_t n = std::max<size_t>(h.size(), 1);
  cudaError_t e = cudaMalloc((void**)dptr, n * sizeof(T));
  if (e != cudaSuccess) return e;
  if (!h.empty()) e = cudaMemcpy(*dptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

}  // namespace

struct adg_ctx {
  int device = 0;
  int sms = 1;
  int* d_err = nullptr;
  // measurement: event pairs around launches while profiling is on
  bool prof = false;
  struct Rec { int kernel; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  int64_t launches[ADG_K_COUNT] = {};
  double ms[ADG_K_COUNT] = {};
};

namespace {

cudaEvent_t take_event(adg_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets one kernel launch with events on its stream when profiling is on.
struct ProfScope {
  adg_ctx* c;
  int k;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  ProfScope(adg_ctx* c_, int k_, cudaStream_t s_) : c(c_), k(k_), s(s_) {
    if (c->prof) {
      a = take_event(c);
      cudaEventRecord(a, s);
    }
  }
  ~ProfScope() {
    if (c->prof && a) {
      cudaEvent_t b = take_event(c);
      cudaEventRecord(b, s);
      c->recs.push_back({k, a, b});
    }
  }
};

}  // namespace

struct adg_design {
  adg_ctx* ctx = nullptr;
  GridDev g{};
  double d[3]{}, o[3]{};
  int n_params = 0, n_q = 0, n_prims = 0;
  std::vector<double> q_base, q_coeff, kr;
  std::vector<int> q_param, kind, sigma, flags, q0, nq;
  std::vector<int> chain;
  std::vector<int> nact, act_off, act;
  std::vector<int> auxd_off, auxf_off;
  int auxd_n = 0, auxf_n = 0;
  std::vector<int> ref_off, ref_prim, ref_qa;
  std::vector<double> ref_coeff;
  // device
  int *d_chain = nullptr, *d_act = nullptr, *d_ref_off = nullptr, *d_ref_prim = nullptr,
      *d_ref_qa = nullptr;
  double* d_ref_coeff = nullptr;
  PrimRec* d_prims = nullptr;
  double* d_auxd = nullptr;
  float* d_auxf = nullptr;
  TileProg* d_progs = nullptr;
  int* d_list = nullptr;
  int* d_counters = nullptr;
  float* d_partial = nullptr;
  size_t partial_cap = 0;
  // per-call host staging
  std::vector<PrimRec> h_prims;
  std::vector<double> h_auxd, q;
  std::vector<float> h_auxf;
  size_t part_total = 0;
  std::vector<double> last_params;
  bool bins_valid = false;
};

// ------------------------------------------------------------------ context -
extern "C" adg_status adg_ctx_create(int32_t device, adg_ctx** out) {
  if (!out) return fail(ADG_EINVAL, "adg_ctx_create: out is NULL");
  *out = nullptr;
  int ndev = 0;
  CU(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev)
    return fail(ADG_EINVAL, "adg_ctx_create: device %d out of range (%d devices)", device, ndev);
  CU(cudaSetDevice(device));
  adg_ctx* c = new adg_ctx();
  c->device = device;
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
  cudaError_t e = cudaMalloc((void**)&c->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int));
  if (e != cudaSuccess) {
    delete c;
    return fail(ADG_ECUDA, "adg_ctx_create: %s", cudaGetErrorString(e));
  }
  *out = c;
  return ADG_OK;
}

extern "C" adg_status adg_ctx_destroy(adg_ctx* ctx) {
  if (!ctx) return ADG_OK;
  cudaSetDevice(ctx->device);
  for (auto& r : ctx->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : ctx->pool) cudaEventDestroy(e);
  cudaFree(ctx->d_err);
  delete ctx;
  return ADG_OK;
}

// ------------------------------------------------------------------- design -
namespace {

// postfix -> tree -> chain of binary ops (n-ary union / intersection become
// left-to-right chains, the recursive form of union_2 in Appendix B.2)
struct Node {
  int code, arg;
  std::vector<int> kids;
};

void emit_chain(const std::vector<Node>& nodes, int id, std::vector<int>& out) {
  const Node& n = nodes[id];
  if (n.code == ADG_OP_PUSH) {
    out.push_back((cPush << 24) | n.arg);
    return;
  }
  if (n.code == ADG_OP_DIFF) {
    emit_chain(nodes, n.kids[0], out);
    emit_chain(nodes, n.kids[1], out);
    out.push_back(cDiff << 24);
    return;
  }
  const int c = n.code == ADG_OP_UNION ? cUnion : cInter;
  emit_chain(nodes, n.kids[0], out);
  for (size_t t = 1; t < n.kids.size(); ++t) {
    emit_chain(nodes, n.kids[t], out);
    out.push_back(c << 24);
  }
}

adg_status compile_program(const adg_design_desc* D, std::vector<int>& chain) {
  std::vector<Node> nodes;
  std::vector<int> st;
  for (int i = 0; i < D->n_ops; ++i) {
    const int w = D->ops[i];
    const int code = (w >> 24) & 0xff, arg = w & 0xffffff;
    Node nd{code, arg, {}};
    int need = 0;
    if (code == ADG_OP_PUSH) {
      if (arg < 0 || arg >= D->n_prims)
        return fail(ADG_EINVAL, "program op %d pushes primitive %d (have %d)", i, arg, D->n_prims);
    } else if (code == ADG_OP_UNION || code == ADG_OP_INTERSECT) {
      need = arg;
      if (need < 1) return fail(ADG_EINVAL, "program op %d: operand count %d", i, need);
    } else if (code == ADG_OP_DIFF) {
      need = 2;
    } else {
      return fail(ADG_EINVAL, "program op %d: unknown code %d", i, code);
    }
    if ((int)st.size() < need) return fail(ADG_EINVAL, "program op %d: stack underflow", i);
    nd.kids.assign(st.end() - need, st.end());
    st.resize(st.size() - need);
    nodes.push_back(nd);
    st.push_back((int)nodes.size() - 1);
  }
  if (st.size() != 1)
    return fail(ADG_EINVAL, "program leaves %zu values on the stack (need 1)", st.size());
  chain.clear();
  emit_chain(nodes, st[0], chain);
  int sp = 0, mx = 0;
  for (int w : chain) {
    sp += ((w >> 24) == cPush) ? 1 : -1;
    mx = std::max(mx, sp);
  }
  if (mx > kMaxDepth)
    return fail(ADG_EINVAL, "program nesting %d exceeds the supported depth %d", mx, kMaxDepth);
  return ADG_OK;
}

void free_design(adg_design* d) {
  cudaFree(d->d_chain);
  cudaFree(d->d_act);
  cudaFree(d->d_ref_off);
  cudaFree(d->d_ref_prim);
  cudaFree(d->d_ref_qa);
  cudaFree(d->d_ref_coeff);
  cudaFree(d->d_prims);
  cudaFree(d->d_auxd);
  cudaFree(d->d_auxf);
  cudaFree(d->d_progs);
  cudaFree(d->d_list);
  cudaFree(d->d_counters);
  cudaFree(d->d_partial);
  delete d;
}

bool is_fin(double v) { return std::isfinite(v); }

}  // namespace

extern "C" adg_status adg_design_create(adg_ctx* ctx, const adg_design_desc* D,
                                        const adg_tile_opts* tiles, adg_design** out) {
  if (!ctx || !D || !out) return fail(ADG_EINVAL, "adg_design_create: NULL argument");
  *out = nullptr;
  const adg_grid& G = D->grid;
  if (G.nx < 1 || G.ny < 1 || G.nz < 1 || G.nx > 8192 || G.ny > 8192 || G.nz > 8192)
    return fail(ADG_EINVAL, "grid %dx%dx%d outside 1..8192 per axis", G.nx, G.ny, G.nz);
  if (G.ncomp < 1 || G.ncomp > 3) return fail(ADG_EINVAL, "ncomp %d not in 1..3", G.ncomp);
  if (!(G.dx > 0) || !(G.dy > 0) || !(G.dz > 0) || !is_fin(G.dx) || !is_fin(G.dy) || !is_fin(G.dz))
    return fail(ADG_EINVAL, "grid spacing must be positive and finite");
  if (!is_fin(G.ox) || !is_fin(G.oy) || !is_fin(G.oz))
    return fail(ADG_EINVAL, "grid origin must be finite");
  for (int c = 0; c < G.ncomp; ++c)
    for (int a = 0; a < 3; ++a)
      if (!(fabs(G.off[c][a]) <= 1.0)) return fail(ADG_EINVAL, "offset off[%d][%d] not in [-1, 1]", c, a);
  if (!is_fin(D->eps_bg) || !is_fin(D->eps_fg)) return fail(ADG_EINVAL, "eps levels must be finite");
  if (D->logic != ADG_LOGIC_PRODUCT && D->logic != ADG_LOGIC_CLAMP)
    return fail(ADG_EINVAL, "logic %d unknown", D->logic);
  if (D->reserved != 0) return fail(ADG_EINVAL, "reserved must be 0");
  if (D->n_params < 0 || D->n_q < 0 || D->n_prims < 1 || D->n_ops < 1 || D->n_prims > 65535)
    return fail(ADG_EINVAL, "counts: params %d, q %d, prims %d (1..65535), ops %d", D->n_params,
                D->n_q, D->n_prims, D->n_ops);
  if ((D->n_q > 0 && (!D->q_base || !D->q_coeff || !D->q_param)) || !D->prim_kind ||
      !D->prim_sigma || !D->prim_flags || !D->prim_q0 || !D->prim_nq || !D->prim_kr || !D->ops)
    return fail(ADG_EINVAL, "description array is NULL");
  for (int j = 0; j < D->n_q; ++j) {
    if (D->q_param[j] < -1 || D->q_param[j] >= D->n_params)
      return fail(ADG_EINVAL, "q_param[%d] = %d out of range", j, D->q_param[j]);
    if (!is_fin(D->q_base[j]) || !is_fin(D->q_coeff[j]))
      return fail(ADG_EINVAL, "q_base / q_coeff[%d] not finite", j);
  }
  for (int p = 0; p < D->n_prims; ++p) {
    const int k = D->prim_kind[p], s = D->prim_sigma[p], n = D->prim_nq[p], q0 = D->prim_q0[p];
    if (q0 < 0 || n < 0 || q0 + n > D->n_q)
      return fail(ADG_EINVAL, "primitive %d: scalars [%d, %d) outside [0, %d)", p, q0, q0 + n, D->n_q);
    if (s < 0 || s > 4) return fail(ADG_EINVAL, "primitive %d: sigma kind %d unknown", p, s);
    if (!(D->prim_kr[p] > 0) || !is_fin(D->prim_kr[p]))
      return fail(ADG_EINVAL, "primitive %d: kr must be positive", p);
    if (k == ADG_PRIM_BOX) {
      if (n != 6) return fail(ADG_EINVAL, "box %d needs 6 scalars, has %d", p, n);
    } else if (k == ADG_PRIM_CIRCLE) {
      if (n != 5) return fail(ADG_EINVAL, "circle %d needs 5 scalars, has %d", p, n);
      if (fabs(G.dx - G.dy) > 1e-12 * G.dx) return fail(ADG_EINVAL, "circle %d needs dx == dy", p);
    } else if (k == ADG_PRIM_GRAPH) {
      if (n < 6 || (n - 2) % 2) return fail(ADG_EINVAL, "graph %d needs 2 + 2M scalars, M >= 2", p);
    } else if (k == ADG_PRIM_POLYGON) {
      return fail(ADG_EINVAL, "primitive %d: polygons are not supported by this build", p);
    } else {
      return fail(ADG_EINVAL, "primitive %d: kind %d unknown", p, k);
    }
  }
  std::vector<int> chain;
  adg_status st = compile_program(D, chain);
  if (st != ADG_OK) return st;

  CU(cudaSetDevice(ctx->device));
  adg_design* d = new adg_design();
  d->ctx = ctx;
  d->chain = chain;
  d->n_params = D->n_params;
  d->n_q = D->n_q;
  d->n_prims = D->n_prims;
  d->d[0] = G.dx; d->d[1] = G.dy; d->d[2] = G.dz;
  d->o[0] = G.ox; d->o[1] = G.oy; d->o[2] = G.oz;
  d->q_base.assign(D->q_base, D->q_base + D->n_q);
  d->q_coeff.assign(D->q_coeff, D->q_coeff + D->n_q);
  d->q_param.assign(D->q_param, D->q_param + D->n_q);
  d->kind.assign(D->prim_kind, D->prim_kind + D->n_prims);
  d->sigma.assign(D->prim_sigma, D->prim_sigma + D->n_prims);
  d->flags.assign(D->prim_flags, D->prim_flags + D->n_prims);
  d->q0.assign(D->prim_q0, D->prim_q0 + D->n_prims);
  d->nq.assign(D->prim_nq, D->prim_nq + D->n_prims);
  d->kr.assign(D->prim_kr, D->prim_kr + D->n_prims);

  // tile shape
  int tx = 32, ty = 4, tz = 4;
  if (tiles && (tiles->tx || tiles->ty || tiles->tz)) { tx = tiles->tx; ty = tiles->ty; tz = tiles->tz; }
  auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
  if (!(tx == 32 || tx == 64) || !pow2(ty) || ty > 16 || !pow2(tz) || tz > 8 || tx * ty * tz < kBlock) {
    delete d;
    return fail(ADG_EINVAL, "tile %dx%dx%d: tx in {32,64}, ty in {1..16}, tz in {1..8}, powers of 2, >= %d cells",
                tx, ty, tz, kBlock);
  }
  GridDev& g = d->g;
  g.nx = G.nx; g.ny = G.ny; g.nz = G.nz; g.C = G.ncomp;
  g.lx = ilog2(tx); g.ly = ilog2(ty); g.lz = ilog2(tz);
  g.ntx = (G.nx + tx - 1) / tx; g.nty = (G.ny + ty - 1) / ty; g.ntz = (G.nz + tz - 1) / tz;
  const long long T = (long long)g.ntx * g.nty * g.ntz;
  if (T > (1LL << 30)) { delete d; return fail(ADG_EINVAL, "too many tiles"); }
  g.T = (int)T;
  for (int a = 0; a < 3; ++a) { g.offmin[a] = 1e9f; g.offmax[a] = -1e9f; }
  for (int c = 0; c < 3; ++c)
    for (int a = 0; a < 3; ++a) {
      g.off[c][a] = c < G.ncomp ? (float)G.off[c][a] : 0.f;
      if (c < G.ncomp) {
        g.offmin[a] = std::min(g.offmin[a], g.off[c][a]);
        g.offmax[a] = std::max(g.offmax[a], g.off[c][a]);
      }
    }
  for (int a = 0; a < 3; ++a) g.invd[a] = (float)(1.0 / d->d[a]);
  g.eps_bg = (float)D->eps_bg;
  g.deps = (float)(D->eps_fg - D->eps_bg);
  g.logic = D->logic;
  g.nchain = (int)chain.size();

  // active scalars and parameter references
  d->nact.assign(d->n_prims, 0);
  d->act_off.assign(d->n_prims, 0);
  d->auxd_off.assign(d->n_prims, 0);
  d->auxf_off.assign(d->n_prims, 0);
  std::vector<std::vector<int>> rp(d->n_params), rq(d->n_params);
  std::vector<std::vector<double>> rc(d->n_params);
  for (int p = 0; p < d->n_prims; ++p) {
    d->act_off[p] = (int)d->act.size();
    int na = 0;
    for (int t = 0; t < d->nq[p]; ++t) {
      const int j = d->q0[p] + t;
      if (d->q_param[j] >= 0 && d->q_coeff[j] != 0.0) {
        d->act.push_back(na);
        rp[d->q_param[j]].push_back(p);
        rq[d->q_param[j]].push_back(na);
        rc[d->q_param[j]].push_back(d->q_coeff[j]);
        ++na;
      } else {
        d->act.push_back(-1);
      }
    }
    d->nact[p] = na;
    if (d->kind[p] == ADG_PRIM_GRAPH) {
      const int M = (d->nq[p] - 2) / 2;
      d->auxd_off[p] = d->auxd_n;
      d->auxd_n += 3 * M;
      d->auxf_off[p] = d->auxf_n;
      d->auxf_n += M;
    }
  }
  d->ref_off.push_back(0);
  for (int k = 0; k < d->n_params; ++k) {
    for (size_t t = 0; t < rp[k].size(); ++t) {
      d->ref_prim.push_back(rp[k][t]);
      d->ref_qa.push_back(rq[k][t]);
      d->ref_coeff.push_back(rc[k][t]);
    }
    d->ref_off.push_back((int)d->ref_prim.size());
  }
  d->h_prims.resize(d->n_prims);
  d->h_auxd.resize(d->auxd_n);
  d->h_auxf.resize(d->auxf_n);
  d->q.resize(std::max(d->n_q, 1));

  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = upload(&d->d_chain, d->chain);
  if (e == cudaSuccess) e = upload(&d->d_act, d->act);
  if (e == cudaSuccess) e = upload(&d->d_ref_off, d->ref_off);
  if (e == cudaSuccess) e = upload(&d->d_ref_prim, d->ref_prim);
  if (e == cudaSuccess) e = upload(&d->d_ref_qa, d->ref_qa);
  if (e == cudaSuccess) e = upload(&d->d_ref_coeff, d->ref_coeff);
  if (e == cudaSuccess) e = upload(&d->d_prims, d->h_prims);
  if (e == cudaSuccess) e = upload(&d->d_auxd, d->h_auxd);
  if (e == cudaSuccess) e = upload(&d->d_auxf, d->h_auxf);
  if (e == cudaSuccess) e = cudaMalloc((void**)&d->d_progs, sizeof(TileProg) * (size_t)g.T);
  if (e == cudaSuccess) e = cudaMalloc((void**)&d->d_list, sizeof(int) * (size_t)g.T);
  if (e == cudaSuccess) e = cudaMalloc((void**)&d->d_counters, sizeof(int) * 4);
  if (e != cudaSuccess) {
    free_design(d);
    return fail(e == cudaErrorMemoryAllocation ? ADG_ENOMEM : ADG_ECUDA, "adg_design_create: %s",
                cudaGetErrorString(e));
  }
  *out = d;
  return ADG_OK;
}

extern "C" adg_status adg_design_destroy(adg_ctx* ctx, adg_design* d) {
  if (!d) return ADG_OK;
  if (ctx) cudaSetDevice(ctx->device);
  free_design(d);
  return ADG_OK;
}

// ------------------------------------------------------ parameter map (a1) -
namespace {

void anchor(double v, int& ai, float& af) {
  v = std::min(std::max(v, -1e8), 1e8);
  const double f = floor(v);
  ai = (int)f;
  af = (float)(v - f);
}

// inclusive cell-index range whose samples u = i + off (any component) can
// fall in [ulo, uhi], clipped to [0, n-1]; empty as lo > hi
void cell_range(double ulo, double uhi, float offmin, float offmax, int n, int& lo, int& hi) {
  const double a = floor(ulo - offmax - 1.0), b = ceil(uhi - offmin + 1.0);
  lo = (int)std::max(0.0, std::min((double)n, a));
  hi = (int)std::min((double)(n - 1), std::max(-1.0, b));
}

adg_status prepare_prims(adg_design* d, const double* p) {
  const GridDev& g = d->g;
  for (int j = 0; j < d->n_q; ++j) {
    d->q[j] = d->q_base[j];
    if (d->q_param[j] >= 0) d->q[j] += d->q_coeff[j] * p[d->q_param[j]];
    if (!std::isfinite(d->q[j])) return fail(ADG_EINVAL, "geometric scalar %d is not finite", j);
  }
  const int nn[3] = {g.nx, g.ny, g.nz};
  const int lt[3] = {g.lx, g.ly, g.lz};
  size_t part = 0;
  for (int pi = 0; pi < d->n_prims; ++pi) {
    PrimRec R;
    memset(&R, 0, sizeof(R));
    R.kind = d->kind[pi];
    R.sigma = d->sigma[pi];
    R.flags = d->flags[pi];
    R.nact = d->nact[pi];
    R.act_off = d->act_off[pi];
    R.kr = (float)d->kr[pi];
    const double beta = kBand[R.sigma] / d->kr[pi];
    R.band = (float)beta;
    R.auxd_off = d->auxd_off[pi];
    R.auxf_off = d->auxf_off[pi];
    const double* Q = d->q.data() + d->q0[pi];
    auto cellc = [&](double v, int ax) { return (v - d->o[ax]) / d->d[ax]; };
    int vlo[3], vhi[3], plo[3], phi[3];
    for (int a = 0; a < 3; ++a) { vlo[a] = 0; vhi[a] = nn[a] - 1; }
    auto zrange = [&]() {
      if (!(R.flags & kBoundZ)) return;
      const double a = cellc(Q[R.kind == kCircle ? 3 : 0], 2);
      const double b = cellc(Q[R.kind == kCircle ? 4 : 1], 2);
      anchor(a, R.ai[4], R.af[4]);
      anchor(b, R.ai[5], R.af[5]);
      cell_range(a - 0.5, b + 0.5, g.offmin[2], g.offmax[2], g.nz, vlo[2], vhi[2]);
    };
    if (R.kind == kBox) {
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
      const double cx = cellc(Q[0], 0), cy = cellc(Q[1], 1), Rc = Q[2] / d->d[0];
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
    } else {  // graph
      const int M = (d->nq[pi] - 2) / 2;
      R.naux = M;
      double* X = d->h_auxd.data() + R.auxd_off;
      double* Y = X + M;
      double* iX = Y + M;
      float* Xf = d->h_auxf.data() + R.auxf_off;
      double ymin = 1e300, ymax = -1e300;
      for (int j = 0; j < M; ++j) {
        X[j] = cellc(Q[2 + j], 0);
        Y[j] = cellc(Q[2 + M + j], 1);
        Xf[j] = (float)X[j];
        ymin = std::min(ymin, Y[j]);
        ymax = std::max(ymax, Y[j]);
        if (j > 0 && !(X[j] > X[j - 1]))
          return fail(ADG_EINVAL, "graph %d: knots must increase strictly in x", pi);
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
    if (part > (size_t)1 << 31) return fail(ADG_EINVAL, "partial buffer exceeds 2^31 entries");
    d->h_prims[pi] = R;
  }
  d->part_total = part;
  return ADG_OK;
}

adg_status ensure_bins(adg_ctx* ctx, adg_design* d, const double* h_params, cudaStream_t s) {
  if (d->n_params > 0 && !h_params) return fail(ADG_EINVAL, "h_params is NULL");
  if (d->bins_valid && (int)d->last_params.size() == d->n_params &&
      (d->n_params == 0 ||
       memcmp(d->last_params.data(), h_params, sizeof(double) * d->n_params) == 0))
    return ADG_OK;
  d->bins_valid = false;
  adg_status st = prepare_prims(d, h_params);
  if (st != ADG_OK) return st;
  CU(cudaMemcpyAsync(d->d_prims, d->h_prims.data(), sizeof(PrimRec) * d->n_prims,
                     cudaMemcpyHostToDevice, s));
  if (d->auxd_n)
    CU(cudaMemcpyAsync(d->d_auxd, d->h_auxd.data(), sizeof(double) * d->auxd_n,
                       cudaMemcpyHostToDevice, s));
  if (d->auxf_n)
    CU(cudaMemcpyAsync(d->d_auxf, d->h_auxf.data(), sizeof(float) * d->auxf_n,
                       cudaMemcpyHostToDevice, s));
  CU(cudaMemsetAsync(d->d_counters, 0, sizeof(int) * 4, s));
  ProfScope ps(ctx, ADG_K_BIN, s);
  CU(launch_bin(d->g, d->d_chain, d->d_prims, d->d_auxf, d->d_auxd, d->d_progs, d->d_list,
                d->d_counters, ctx->d_err, s));
  d->last_params.assign(h_params, h_params + d->n_params);
  d->bins_valid = true;
  return ADG_OK;
}

adg_status run_vjp(adg_ctx* ctx, adg_design* d, const VjpArgs& va, float* d_grad, cudaStream_t s) {
  if (d->part_total > d->partial_cap) {
    if (d->d_partial) CU(cudaFreeAsync(d->d_partial, s));
    d->d_partial = nullptr;
    const size_t cap = d->part_total + d->part_total / 2 + 1024;
    CU(cudaMallocAsync((void**)&d->d_partial, cap * sizeof(float), s));
    d->partial_cap = cap;
  }
  if (d->part_total) CU(cudaMemsetAsync(d->d_partial, 0, d->part_total * sizeof(float), s));
  const int grid = ctx->sms * vjp_blocks_per_sm();
  {
    ProfScope ps(ctx, ADG_K_VJP, s);
    CU(launch_vjp(d->g, d->d_progs, d->d_list, d->d_counters, d->d_prims, d->d_act, d->d_auxf,
                  d->d_auxd, va, d->d_partial, ctx->d_err, grid, s));
  }
  ProfScope ps(ctx, ADG_K_FINALIZE, s);
  CU(launch_finalize(d->n_params, d->d_ref_off, d->d_ref_prim, d->d_ref_qa, d->d_ref_coeff,
                     d->d_prims, d->d_partial, d_grad, s));
  return ADG_OK;
}

}  // namespace

// ------------------------------------------------------------------- calls --
extern "C" adg_status adg_build_eps(adg_ctx* ctx, adg_design* d, const double* h_params,
                                    float* d_fill, float* d_eps, void* stream) {
  if (!ctx || !d || !d_eps) return fail(ADG_EINVAL, "adg_build_eps: NULL argument");
  CU(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  adg_status st = ensure_bins(ctx, d, h_params, s);
  if (st != ADG_OK) return st;
  const int grid = std::min(d->g.T, ctx->sms * build_blocks_per_sm());
  ProfScope ps(ctx, ADG_K_BUILD, s);
  CU(launch_build(d->g, d->d_progs, d->d_prims, d->d_auxf, d->d_auxd, d_fill, d_eps, grid, s));
  return ADG_OK;
}

extern "C" adg_status adg_grad(adg_ctx* ctx, adg_design* d, const double* h_params,
                               const float* const d_efwd[3], const float* const d_eadj[3],
                               const float* w, float* d_grad, void* stream) {
  if (!ctx || !d || !d_efwd || !d_eadj || !w || (!d_grad && d->n_params > 0))
    return fail(ADG_EINVAL, "adg_grad: NULL argument");
  VjpArgs va{};
  for (int c = 0; c < d->g.C; ++c) {
    if (!d_efwd[c] || !d_eadj[c]) return fail(ADG_EINVAL, "adg_grad: field of component %d is NULL", c);
    va.ef[c] = reinterpret_cast<const float2*>(d_efwd[c]);
    va.ea[c] = reinterpret_cast<const float2*>(d_eadj[c]);
    va.w[c] = make_float2(w[2 * c], w[2 * c + 1]);
  }
  va.G = nullptr;
  CU(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  adg_status st = ensure_bins(ctx, d, h_params, s);
  if (st != ADG_OK) return st;
  return run_vjp(ctx, d, va, d_grad, s);
}

extern "C" adg_status adg_grad_real(adg_ctx* ctx, adg_design* d, const double* h_params,
                                    const float* d_G, float* d_grad, void* stream) {
  if (!ctx || !d || !d_G || (!d_grad && d->n_params > 0))
    return fail(ADG_EINVAL, "adg_grad_real: NULL argument");
  VjpArgs va{};
  va.G = d_G;
  CU(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  adg_status st = ensure_bins(ctx, d, h_params, s);
  if (st != ADG_OK) return st;
  return run_vjp(ctx, d, va, d_grad, s);
}

extern "C" adg_status adg_sync(adg_ctx* ctx, void* stream) {
  if (!ctx) return fail(ADG_EINVAL, "adg_sync: NULL context");
  CU(cudaSetDevice(ctx->device));
  CU(cudaStreamSynchronize((cudaStream_t)stream));
  int e = 0;
  CU(cudaMemcpy(&e, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    CU(cudaMemset(ctx->d_err, 0, sizeof(int)));
    return fail(ADG_EDEVICE,
                "device check failed (bits 0x%x: 1 leaves/tile, 2 ops/tile, 4 depth, 8 slots/tile, "
                "16 partial range, 32 program); use a smaller tile shape",
                e);
  }
  return ADG_OK;
}

extern "C" adg_status adg_design_stats(adg_ctx* ctx, adg_design* d, void* stream, adg_stats* out) {
  if (!ctx || !d || !out) return fail(ADG_EINVAL, "adg_design_stats: NULL argument");
  CU(cudaSetDevice(ctx->device));
  CU(cudaStreamSynchronize((cudaStream_t)stream));
  int c[4] = {0, 0, 0, 0};
  CU(cudaMemcpy(c, d->d_counters, sizeof(c), cudaMemcpyDeviceToHost));
  out->tiles = d->g.T;
  out->program_tiles = c[0];
  out->max_ops = c[1];
  out->band_cells = c[2];
  out->cells = (int64_t)d->g.nx * d->g.ny * d->g.nz;
  out->tile[0] = 1 << d->g.lx;
  out->tile[1] = 1 << d->g.ly;
  out->tile[2] = 1 << d->g.lz;
  return ADG_OK;
}

extern "C" adg_status adg_profile_enable(adg_ctx* ctx, int32_t on) {
  if (!ctx) return fail(ADG_EINVAL, "adg_profile_enable: NULL context");
  ctx->prof = on != 0;
  return ADG_OK;
}

extern "C" adg_status adg_profile_read(adg_ctx* ctx, adg_profile_data* out, int32_t reset) {
  if (!ctx || !out) return fail(ADG_EINVAL, "adg_profile_read: NULL argument");
  CU(cudaSetDevice(ctx->device));
  for (auto& r : ctx->recs) {
    CU(cudaEventSynchronize(r.b));
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, r.a, r.b));
    ctx->ms[r.kernel] += ms;
    ctx->launches[r.kernel] += 1;
    ctx->pool.push_back(r.a);
    ctx->pool.push_back(r.b);
  }
  ctx->recs.clear();
  for (int k = 0; k < ADG_K_COUNT; ++k) {
    out->launches[k] = ctx->launches[k];
    out->ms[k] = ctx->ms[k];
    if (reset) { ctx->launches[k] = 0; ctx->ms[k] = 0.0; }
  }
  return ADG_OK;
}

namespace adg {
void set_last_error(const char* msg) { g_err = msg; }
}  // namespace adg

extern "C" const char* adg_last_error(void) { return g_err.c_str(); }
