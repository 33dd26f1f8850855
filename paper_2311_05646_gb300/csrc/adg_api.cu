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
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/adg.h"
#include "adg_host.h"
#include "adg_internal.h"

using namespace adg;

namespace {

// The last error message of this thread: a fixed buffer, so that reporting
// an error allocates nothing (adg_grad_noalloc relies on it).
thread_local char g_err[512] = "no error";

adg_status fail(adg_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

#define CU(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(e_ == cudaErrorMemoryAllocation ? ADG_ENOMEM : ADG_ECUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                  \
  } while (0)

// ---- allocation accounting and host-side fault injection ----------------------
// Every device and pinned-host allocation of the library goes through these,
// so that a test can make one fail as if memory were exhausted
// (adg_debug_alloc) and count what the library still holds afterwards.
std::atomic<int> g_fail_after{-1};  // allocations to let through before one fails; -1: none
std::atomic<long long> g_live{0};   // live allocations made by the library

bool injected_failure() {
  int b = g_fail_after.load();
  while (b >= 0)
    if (g_fail_after.compare_exchange_weak(b, b - 1)) return b == 0;
  return false;
}
template <class T>
cudaError_t lib_malloc(T** p, size_t bytes) {
  if (injected_failure()) { *p = nullptr; return cudaErrorMemoryAllocation; }
  const cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e == cudaSuccess) ++g_live;
  return e;
}
template <class T>
cudaError_t lib_malloc_async(T** p, size_t bytes, cudaStream_t s) {
  if (injected_failure()) { *p = nullptr; return cudaErrorMemoryAllocation; }
  const cudaError_t e = cudaMallocAsync((void**)p, bytes, s);
  if (e == cudaSuccess) ++g_live;
  return e;
}
cudaError_t lib_malloc_host(void** p, size_t bytes) {
  if (injected_failure()) { *p = nullptr; return cudaErrorMemoryAllocation; }
  const cudaError_t e = cudaMallocHost(p, bytes);
  if (e == cudaSuccess) ++g_live;
  return e;
}
cudaError_t lib_free(void* p) {
  if (!p) return cudaSuccess;
  --g_live;
  return cudaFree(p);
}
cudaError_t lib_free_async(void* p, cudaStream_t s) {
  if (!p) return cudaSuccess;
  --g_live;
  return cudaFreeAsync(p, s);
}
cudaError_t lib_free_host(void* p) {
  if (!p) return cudaSuccess;
  --g_live;
  return cudaFreeHost(p);
}

template <class T>
cudaError_t upload(T** dptr, const std::vector<T>& h) {
  *dptr = nullptr;
  size_t n = std::max<size_t>(h.size(), 1);
  cudaError_t e = lib_malloc((void**)dptr, n * sizeof(T));
  if (e != cudaSuccess) return e;
  if (!h.empty()) e = cudaMemcpy(*dptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

}  // namespace

struct adg_ctx {
  int device = 0;
  int sms = 1;
  int* d_err = nullptr;
  float* d_gtape = nullptr;  // VJP tape for programs longer than the shared-memory tape
  void* d_mesh = nullptr;  // adg_mesh_*: polygon records, vertices, region buffers, sums
  size_t mesh_cap = 0;     // bytes
  int gtape_blocks = 0;
  // measurement: event pairs around launches while profiling is on
  bool prof = false;
  struct Rec { int kernel; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  int64_t launches[ADG_K_COUNT] = {};
  double ms[ADG_K_COUNT] = {};
  // batches: two alternating arenas (device table + pinned staging), each
  // with the CUDA graph of its last captured batch shape
  struct Arena {
    void* d = nullptr;
    void* h = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;
    bool used = false;
    cudaGraphExec_t exec = nullptr;
    uint64_t sig = 0;
    int* d_work = nullptr;  // the batch launches' tile counters (zero between launches)
  };
  Arena arenas[2];
  int next_arena = 0;
  cudaStream_t capture = nullptr;  // graphs are captured here, launched on the caller's stream
  cudaStream_t upload = nullptr;   // designs' primitive records go to the device here
  struct Ticket { uint64_t id; cudaEvent_t ev; };
  std::vector<Ticket> tickets;
  uint64_t next_ticket = 1;
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

// Brackets one kernel launch with an NVTX range on the host (named after the
// kernel; free when no tool is attached) and, when profiling is on, with
// events on its stream.
const char* const kKernelNames[ADG_K_COUNT] = {"adg/k_bin", "adg/k_build", "adg/k_vjp",
                                               "adg/k_finalize", "adg/prepare", "adg/fill",
                                               "adg/k_dense", "adg/k_levels"};
struct ProfScope {
  adg_ctx* c;
  int k;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  ProfScope(adg_ctx* c_, int k_, cudaStream_t s_) : c(c_), k(k_), s(s_) {
    nvtxRangePushA(kKernelNames[k]);
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
    nvtxRangePop();
  }
};

// An NVTX range over one entry point (host side).
struct CallRange {
  explicit CallRange(const char* name) { nvtxRangePushA(name); }
  ~CallRange() { nvtxRangePop(); }
};

}  // namespace

struct adg_design {
  adg_ctx* ctx = nullptr;
  GridDev g{};
  int fill_warps = 1;  // build: warps streaming constant tiles per block
  double d[3]{}, o[3]{};
  int n_params = 0, n_q = 0, n_prims = 0;
  std::vector<double> q_base, q_coeff, kr;
  std::vector<int> q_param, kind, sigma, flags, q0, nq;
  std::vector<int> chain;
  std::vector<int> nact, act_off, act, auxd_off, auxf_off;
  std::vector<float> actc;
  std::vector<int> ref_off, ref_prim, ref_qa;
  std::vector<double> ref_coeff;
  host::SlotTables st{};
  // device
  int *d_chain = nullptr, *d_act = nullptr, *d_ref_off = nullptr, *d_ref_prim = nullptr,
      *d_ref_qa = nullptr;
  float* d_actc = nullptr;
  double* d_ref_coeff = nullptr;
  // primitive records, two buffers (one per counter set, below): a binning's
  // records are uploaded on the context's upload stream into the buffer of
  // its set while kernels of the binning before still read the other one
  PrimRec* d_prims = nullptr;  // 2 n_prims
  double* d_auxd = nullptr;    // 2 auxd_stride
  float* d_auxf = nullptr;     // 2 auxf_stride
  size_t auxd_stride = 1, auxf_stride = 1;
  void* h_pin[2] = {};             // pinned staging of each buffer: prims, auxd, auxf
  cudaEvent_t up_done[2] = {};     // the last copy out of staging b
  cudaEvent_t used[2] = {};        // after the last kernels that read buffer b (recorded
                                   // when a binning moves to the other buffer)
  bool side_upload = false;        // copies on the upload stream (large grids), else
                                   // on the caller's stream (launch-bound small ones)
  TileProg* d_progs = nullptr;
  unsigned char* d_tclass = nullptr;
  int* d_list = nullptr;
  int* d_counters = nullptr;  // two sets of 4 (the binning alternates between them),
                              // the active samples of the last VJP, then (from
                              // int 12) the persistent kernels' 6 work counters
  int gen = 0;                // the set of the last binning
  float* d_partial = nullptr;  // all zero between calls (the finalize clears what it sums)
  size_t partial_cap = 0;
  bool partial_dirty = false;  // a call that enqueued the VJP did not complete its enqueue
  // the one-job tables of single-design calls, one slot per (build?, gradient?,
  // counter set): in an optimisation loop each call finds its table already
  // uploaded, so no copy sits between the kernels of consecutive calls
  static constexpr int kJobSlots = 8;
  Job* d_job = nullptr;
  Job jobs_h[kJobSlots]{};
  bool job_ok[kJobSlots] = {};
  // dense field stream (adg_grad_dense): per-chunk partials and work counter
  double2* d_dense_part = nullptr;
  int* d_dense_ctr = nullptr;
  // finite-difference baseline (adg_grad_fd): z, fill+, fill-, eps scratch;
  // chunk partials; one FP64 sum per parameter
  float* d_fd_buf = nullptr;
  double* d_fd_part = nullptr;
  double* d_fd_acc = nullptr;
  float* d_row = nullptr;  // n_params floats: this design's term of a sum
                           // (adg_grad_eh, adg_levels_grad)
  float* d_lv_buf = nullptr;  // adg_levels_*: fills and cotangents (first set)
  size_t lv_cap = 0;          // floats
  // per-call host staging
  std::vector<PrimRec> h_prims;
  std::vector<double> h_auxd, q;
  std::vector<float> h_auxf;
  size_t part_total = 0;
  std::vector<double> last_params;
  bool bins_valid = false;
  // a call failed between flipping the counter set and enqueueing its binning:
  // both sets are cleared before the next binning
  bool counters_dirty = false;
};

// Grids from this many samples up copy their records on the upload stream:
// their kernels run long enough for the copy to hide behind the ones before.
// Smaller grids are launch-bound: the fewer runtime calls of a copy on the
// caller's stream win there.
constexpr size_t kSideUploadSamples = (size_t)1 << 21;

// Bytes of one record buffer: primitive records, FP64 and fp32 auxiliary
// tables (the pinned staging lays them out in this order).
size_t record_bytes(const adg_design* d) {
  return sizeof(PrimRec) * d->n_prims + sizeof(double) * d->auxd_stride +
         sizeof(float) * d->auxf_stride;
}

// After a call that had prepared a new binning failed before enqueueing all
// of its work: the bins may not have been written, and the counter set the
// design now points at may hold an older binning's counts.
void invalidate_bins(adg_design* d) {
  d->bins_valid = false;
  d->counters_dirty = true;
}

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
  cudaError_t e = init_kernel_attributes();
  c->gtape_blocks = c->sms * std::max(vjp_blocks_per_sm(1, false, 128), vjp_blocks_per_sm(1, true, 128));
  if (e == cudaSuccess) e = lib_malloc((void**)&c->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int));
  if (e == cudaSuccess)
    e = lib_malloc((void**)&c->d_gtape, sizeof(float) * kTapeBlockFloats * c->gtape_blocks);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->upload, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    lib_free(c->d_err);
    lib_free(c->d_gtape);
    if (c->upload) cudaStreamDestroy(c->upload);
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
  for (auto& a : ctx->arenas) {
    if (a.exec) cudaGraphExecDestroy(a.exec);
    if (a.done) cudaEventDestroy(a.done);
    lib_free(a.d);
    lib_free_host(a.h);
    lib_free(a.d_work);
  }
  for (auto& t : ctx->tickets) cudaEventDestroy(t.ev);
  if (ctx->capture) cudaStreamDestroy(ctx->capture);
  if (ctx->upload) cudaStreamDestroy(ctx->upload);
  lib_free(ctx->d_err);
  lib_free(ctx->d_gtape);
  lib_free(ctx->d_mesh);
  delete ctx;
  return ADG_OK;
}

// ------------------------------------------------------------------- design -
namespace {

void free_design(adg_design* d) {
  for (int b = 0; b < 2; ++b) {
    if (d->up_done[b]) {
      cudaEventSynchronize(d->up_done[b]);  // no copy from the staging in flight
      cudaEventDestroy(d->up_done[b]);
    }
    if (d->used[b]) cudaEventDestroy(d->used[b]);
    lib_free_host(d->h_pin[b]);
  }
  lib_free(d->d_chain);
  lib_free(d->d_act);
  lib_free(d->d_actc);
  lib_free(d->d_ref_off);
  lib_free(d->d_ref_prim);
  lib_free(d->d_ref_qa);
  lib_free(d->d_ref_coeff);
  lib_free(d->d_prims);
  lib_free(d->d_auxd);
  lib_free(d->d_auxf);
  lib_free(d->d_progs);
  lib_free(d->d_tclass);
  lib_free(d->d_list);
  lib_free(d->d_counters);
  lib_free(d->d_partial);
  lib_free(d->d_job);
  lib_free(d->d_dense_part);
  lib_free(d->d_dense_ctr);
  lib_free(d->d_fd_buf);
  lib_free(d->d_fd_part);
  lib_free(d->d_fd_acc);
  lib_free(d->d_row);
  lib_free(d->d_lv_buf);
  delete d;
}

}  // namespace

extern "C" adg_status adg_design_create(adg_ctx* ctx, const adg_design_desc* D,
                                        const adg_tile_opts* tiles, adg_design** out) {
  CallRange nvtx_range("adg_design_create");
  if (!ctx || !D || !out) return fail(ADG_EINVAL, "adg_design_create: NULL argument");
  *out = nullptr;
  host::Msg m;
  if (host::validate(D, m) != ADG_OK) return fail(ADG_EINVAL, "%s", m.text);
  int tx = 32, ty = 4, tz = 4;
  if (tiles && (tiles->tx || tiles->ty || tiles->tz)) { tx = tiles->tx; ty = tiles->ty; tz = tiles->tz; }
  const int fill_warps = tiles && tiles->fill_warps ? tiles->fill_warps : 1;
  if (fill_warps < 1 || fill_warps > kMaxFillWarps)
    return fail(ADG_EINVAL, "fill_warps %d: 1 or 2 (0 = 1)", tiles->fill_warps);
  if (!host::tile_ok(tx, ty, tz))
    return fail(ADG_EINVAL,
                "tile %dx%dx%d: tx in {32,64}, ty in {1..16}, tz in {1..8}, powers of 2, %d..%d cells",
                tx, ty, tz, kBlock, kMaxTileCells);
  const adg_grid& G = D->grid;
  if ((long long)((G.nx + tx - 1) / tx) * ((G.ny + ty - 1) / ty) * ((G.nz + tz - 1) / tz) >
      (1LL << 30))
    return fail(ADG_EINVAL, "too many tiles");

  // program -> chain
  std::vector<int> w(6 * (size_t)D->n_ops), chain(2 * (size_t)D->n_ops);
  host::ChainWork cw{w.data(), w.data() + D->n_ops, w.data() + 2 * D->n_ops,
                     w.data() + 3 * D->n_ops, w.data() + 4 * D->n_ops, w.data() + 5 * D->n_ops};
  int nchain = 0;
  if (host::compile_chain(D, cw, chain.data(), &nchain, m) != ADG_OK)
    return fail(ADG_EINVAL, "%s", m.text);
  chain.resize(nchain);

  CU(cudaSetDevice(ctx->device));
  adg_design* d = new adg_design();
  d->fill_warps = fill_warps;
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
  host::set_grid(D, tx, ty, tz, nchain, d->g);
  {
    std::vector<unsigned char> pushed(D->n_prims, 0);
    bool unique = true;
    for (int i = 0; i < nchain && unique; ++i)
      if (((chain[i] >> 24) & 0xff) == cPush) unique = pushed[chain[i] & 0xffffff]++ == 0;
    d->g.unique_push = unique ? 1 : 0;
  }

  // accumulator slots per (primitive, parameter) and parameter references
  size_t nqs = 0;
  for (int p = 0; p < D->n_prims; ++p) nqs += D->prim_nq[p];
  d->act.resize(std::max<size_t>(nqs, 1));
  d->actc.resize(std::max<size_t>(nqs, 1));
  d->nact.resize(D->n_prims);
  d->act_off.resize(D->n_prims);
  d->auxd_off.resize(D->n_prims);
  d->auxf_off.resize(D->n_prims);
  d->ref_off.resize(D->n_params + 1);
  d->ref_prim.resize(std::max<size_t>(nqs, 1));
  d->ref_qa.resize(std::max<size_t>(nqs, 1));
  d->ref_coeff.resize(std::max<size_t>(nqs, 1));
  std::vector<int> count(D->n_params + 1);
  host::SlotTables st{d->act.data(), d->nact.data(), d->act_off.data(), d->actc.data(),
                      d->ref_off.data(), d->ref_prim.data(), d->ref_qa.data(), d->ref_coeff.data(),
                      d->auxd_off.data(), d->auxf_off.data(), 0, 0, 0, 0};
  host::build_slots(D, st, count.data());
  d->st = st;
  d->ref_prim.resize(std::max(st.nrefs, 1));
  d->ref_qa.resize(std::max(st.nrefs, 1));
  d->ref_coeff.resize(std::max(st.nrefs, 1));
  d->st.ref_prim = d->ref_prim.data();
  d->st.ref_qa = d->ref_qa.data();
  d->st.ref_coeff = d->ref_coeff.data();
  d->h_prims.resize(d->n_prims);
  d->h_auxd.resize(std::max(st.auxd_n, 1));
  d->h_auxf.resize(std::max(st.auxf_n, 1));
  d->q.resize(std::max(d->n_q, 1));

  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = upload(&d->d_chain, d->chain);
  if (e == cudaSuccess) e = upload(&d->d_act, d->act);
  if (e == cudaSuccess) e = upload(&d->d_actc, d->actc);
  if (e == cudaSuccess) e = upload(&d->d_ref_off, d->ref_off);
  if (e == cudaSuccess) e = upload(&d->d_ref_prim, d->ref_prim);
  if (e == cudaSuccess) e = upload(&d->d_ref_qa, d->ref_qa);
  if (e == cudaSuccess) e = upload(&d->d_ref_coeff, d->ref_coeff);
  d->auxd_stride = d->h_auxd.size();
  d->auxf_stride = d->h_auxf.size();
  d->side_upload = (size_t)G.nx * G.ny * G.nz * G.ncomp >= kSideUploadSamples;
  if (e == cudaSuccess) e = lib_malloc((void**)&d->d_prims, 2 * sizeof(PrimRec) * d->n_prims);
  if (e == cudaSuccess) e = lib_malloc((void**)&d->d_auxd, 2 * sizeof(double) * d->auxd_stride);
  if (e == cudaSuccess) e = lib_malloc((void**)&d->d_auxf, 2 * sizeof(float) * d->auxf_stride);
  for (int b = 0; b < 2; ++b) {
    if (e == cudaSuccess) e = lib_malloc_host(&d->h_pin[b], record_bytes(d));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d->up_done[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d->used[b], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = lib_malloc((void**)&d->d_progs, sizeof(TileProg) * (size_t)d->g.T);
  if (e == cudaSuccess) e = lib_malloc((void**)&d->d_tclass, (size_t)d->g.T);
  if (e == cudaSuccess) e = lib_malloc((void**)&d->d_list, sizeof(int) * (size_t)d->g.T);
  if (e == cudaSuccess) e = lib_malloc((void**)&d->d_counters, sizeof(int) * 20);
  if (e == cudaSuccess) e = cudaMemset(d->d_counters, 0, sizeof(int) * 20);
  if (e == cudaSuccess) e = lib_malloc((void**)&d->d_job, sizeof(Job) * adg_design::kJobSlots);
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

adg_status prepare_prims(adg_design* d, const double* p) {
  host::Msg m;
  if (host::map_params(d->n_q, d->q_base.data(), d->q_coeff.data(), d->q_param.data(), p,
                       d->q.data(), m) != ADG_OK)
    return fail(ADG_EINVAL, "%s", m.text);
  host::PrimTable P{d->kind.data(), d->sigma.data(), d->flags.data(), d->q0.data(), d->nq.data(),
                    d->kr.data(), d->n_prims};
  if (host::prepare_prims(d->g, d->d, d->o, P, d->st, d->q.data(), d->h_prims.data(),
                          d->h_auxd.data(), d->h_auxf.data(), &d->part_total, m) != ADG_OK)
    return fail(ADG_EINVAL, "%s", m.text);
  return ADG_OK;
}

// Parameter map + record upload when the parameters changed since the last
// binning of this design; *rebin tells whether the binner must run.
adg_status ensure_records(adg_design* d, const double* h_params, cudaStream_t s, bool* rebin) {
  if (d->n_params > 0 && !h_params) return fail(ADG_EINVAL, "h_params is NULL");
  *rebin = false;
  if (d->bins_valid && (int)d->last_params.size() == d->n_params &&
      (d->n_params == 0 ||
       memcmp(d->last_params.data(), h_params, sizeof(double) * d->n_params) == 0))
    return ADG_OK;
  d->bins_valid = false;
  adg_status st = prepare_prims(d, h_params);
  if (st != ADG_OK) return st;
#ifdef ADG_DEBUG
  // Test hook of the debug build (ADG_DEBUG_PLANT=partials): the last
  // primitive with partials is moved one entry past the design's range --
  // still inside the buffer, which keeps at least 1024 spare entries -- so
  // that the kernels' bound checks must catch it.
  if (const char* pl = getenv("ADG_DEBUG_PLANT"))
    if (!strcmp(pl, "partials"))
      for (int p = d->n_prims - 1; p >= 0; --p)
        if (d->h_prims[p].npb > 0) { d->h_prims[p].part_off += 1; break; }
#endif
  if (d->counters_dirty) {
    CU(cudaMemsetAsync(d->d_counters, 0, sizeof(int) * 8, s));  // both counter sets
    d->counters_dirty = false;
  }
  // this binning counts into the other set (cleared by the last one) and
  // reads the records of the other buffer
  const int b = d->gen ^ 1;
  PrimRec* dp = d->d_prims + (size_t)b * d->n_prims;
  double* dd = d->d_auxd + (size_t)b * d->auxd_stride;
  float* df = d->d_auxf + (size_t)b * d->auxf_stride;
  const size_t np = sizeof(PrimRec) * d->n_prims, nd = sizeof(double) * d->st.auxd_n,
               nf = sizeof(float) * d->st.auxf_n;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (d->side_upload) CU(cudaStreamIsCapturing(s, &cap));
  if (d->side_upload && cap == cudaStreamCaptureStatusNone) {
    // Large grids: from pinned staging b (once its last copy has left it) on
    // the upload stream, after the kernels that read buffer b (two binnings
    // ago) -- usually long before the kernels ahead of this call's binner
    // finish, so no copy sits between them.
    unsigned char* hp = static_cast<unsigned char*>(d->h_pin[b]);
    const size_t od = sizeof(PrimRec) * d->n_prims, of = od + sizeof(double) * d->auxd_stride;
    CU(cudaEventSynchronize(d->up_done[b]));
    memcpy(hp, d->h_prims.data(), np);
    memcpy(hp + od, d->h_auxd.data(), nd);
    memcpy(hp + of, d->h_auxf.data(), nf);
    cudaStream_t up = d->ctx->upload;
    CU(cudaEventRecord(d->used[d->gen], s));  // the binning being left: its kernels
    CU(cudaStreamWaitEvent(up, d->used[b], 0));
    CU(cudaMemcpyAsync(dp, hp, np, cudaMemcpyHostToDevice, up));
    if (nd) CU(cudaMemcpyAsync(dd, hp + od, nd, cudaMemcpyHostToDevice, up));
    if (nf) CU(cudaMemcpyAsync(df, hp + of, nf, cudaMemcpyHostToDevice, up));
    CU(cudaEventRecord(d->up_done[b], up));
    CU(cudaStreamWaitEvent(s, d->up_done[b], 0));
  } else {  // small (launch-bound) grids, or captured into a graph: on the caller's stream
    CU(cudaMemcpyAsync(dp, d->h_prims.data(), np, cudaMemcpyHostToDevice, s));
    if (nd) CU(cudaMemcpyAsync(dd, d->h_auxd.data(), nd, cudaMemcpyHostToDevice, s));
    if (nf) CU(cudaMemcpyAsync(df, d->h_auxf.data(), nf, cudaMemcpyHostToDevice, s));
  }
  d->last_params.assign(h_params, h_params + d->n_params);
  d->bins_valid = true;
  d->gen = b;
  *rebin = true;
  return ADG_OK;
}

// The partial buffer starts zeroed and stays so: the VJP writes only
// partials that the finalize then sums and clears.  A call whose enqueue
// stopped between the two leaves it dirty; the next call clears it.
adg_status ensure_partials(adg_design* d, cudaStream_t s) {
  if (d->part_total > d->partial_cap) {
    if (d->d_partial) CU(lib_free_async(d->d_partial, s));
    d->d_partial = nullptr;
    const size_t cap = d->part_total + d->part_total / 2 + 1024;
    CU(lib_malloc_async((void**)&d->d_partial, cap * sizeof(float), s));
    d->partial_cap = cap;
    d->partial_dirty = true;
  }
  if (d->partial_dirty) {
    CU(cudaMemsetAsync(d->d_partial, 0, d->partial_cap * sizeof(float), s));
    d->partial_dirty = false;
  }
  return ADG_OK;
}

// The job of one design (device pointers of its tables and bins).
Job design_job(adg_design* d) {
  Job J{};
  J.g = d->g;
  J.err = d->ctx ? d->ctx->d_err : nullptr;
  J.chain = d->d_chain;
  J.prims = d->d_prims + (size_t)d->gen * d->n_prims;
  J.act = d->d_act;
  J.actc = d->d_actc;
  J.auxf = d->d_auxf + (size_t)d->gen * d->auxf_stride;
  J.auxd = d->d_auxd + (size_t)d->gen * d->auxd_stride;
  J.ref_off = d->d_ref_off;
  J.ref_prim = d->d_ref_prim;
  J.ref_qa = d->d_ref_qa;
  J.ref_coeff = d->d_ref_coeff;
  J.progs = d->d_progs;
  J.tclass = d->d_tclass;
  J.list = d->d_list;
  J.counters = d->d_counters + 4 * d->gen;
  J.counters_next = d->d_counters + 4 * (d->gen ^ 1);
  J.counters_last = d->d_counters + 8;
  J.partial = d->d_partial;
  J.partial_n = (long long)d->part_total;
  J.nparam = d->n_params;
  return J;
}

// Enqueue bin -> build / VJP -> finalize for a job table.
adg_status run_jobs(adg_ctx* ctx, const Job* d_jobs, const JobTotals& t_in, bool any_bin,
                    bool any_build, bool any_grad, int max_tiles, cudaStream_t s) {
  // Programmatic dependent launch for the kernels after the first: not while
  // profiling (events sit between the launches) or capturing a graph.
  JobTotals t = t_in;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CU(cudaStreamIsCapturing(s, &cap));
  t.pdl = (!ctx->prof && cap == cudaStreamCaptureStatusNone) ? 1 : 0;
  if (any_bin) {
    ProfScope ps(ctx, ADG_K_BIN, s);
    CU(launch_bin(d_jobs, t, ctx->d_err, s));
  }
  if (any_build) {  // constant-tile fill and band tiles in one launch
    ProfScope ps(ctx, ADG_K_BUILD, s);
    CU(launch_build(d_jobs, t, ctx->sms, s));
  }
  if (any_grad) {
    {
      ProfScope ps(ctx, ADG_K_VJP, s);
      CU(launch_vjp(d_jobs, t, ctx->d_err, ctx->sms, ctx->d_gtape, ctx->gtape_blocks, s));
    }
    ProfScope ps(ctx, ADG_K_FINALIZE, s);
    CU(launch_finalize(d_jobs, t, s));
  }
  return ADG_OK;
}

adg_status run_single_enqueue(adg_ctx* ctx, adg_design* d, bool rebin, float* d_fill,
                              float* d_eps, const VjpArgs* va, float* d_grad, cudaStream_t s);

adg_status run_single(adg_ctx* ctx, adg_design* d, const double* h_params, float* d_fill,
                      float* d_eps, const VjpArgs* va, float* d_grad, cudaStream_t s) {
  bool rebin = false;
  adg_status st = ensure_records(d, h_params, s, &rebin);
  if (st != ADG_OK) return st;
  st = run_single_enqueue(ctx, d, rebin, d_fill, d_eps, va, d_grad, s);
  if (st != ADG_OK && rebin) invalidate_bins(d);
  return st;
}

adg_status run_single_enqueue(adg_ctx* ctx, adg_design* d, bool rebin, float* d_fill,
                              float* d_eps, const VjpArgs* va, float* d_grad, cudaStream_t s) {
  adg_status st = ADG_OK;
  const bool grad = va != nullptr;
  if (grad) {
    st = ensure_partials(d, s);
    if (st != ADG_OK) return st;
  }
  Job J = design_job(d);
  J.do_bin = rebin ? 1 : 0;
  J.do_build = d_eps ? 1 : 0;
  J.do_grad = grad ? 1 : 0;
  J.fill = d_fill;
  J.eps = d_eps;
  if (grad) J.va = *va;
  J.grad = d_grad;
  J.partial_n = grad ? (long long)d->part_total : 0;
  if (grad) d->partial_dirty = true;  // until the finalize is enqueued
  const int slot = (d_eps ? 1 : 0) | (grad ? 2 : 0) | (d->gen << 2);
  if (!d->job_ok[slot] || memcmp(&d->jobs_h[slot], &J, sizeof(Job)) != 0) {
    d->job_ok[slot] = false;
    memcpy(&d->jobs_h[slot], &J, sizeof(Job));
    CU(cudaMemcpyAsync(d->d_job + slot, &d->jobs_h[slot], sizeof(Job), cudaMemcpyHostToDevice, s));
    d->job_ok[slot] = true;
  }
  JobTotals t{};
  t.njobs = 1;
  t.tiles_padded = ((d->g.T + 127) / 128) * 128;
  t.bin_blocks = t.tiles_padded / 128;
  t.fill_blocks = d_eps ? (d->g.C * d->g.nz * d->g.ny + kFillRows - 1) / kFillRows : 0;
  t.params = grad ? d->n_params : 0;
  t.work = d->d_counters + 12;
  t.fill_warps = d->fill_warps;
  t.polar = d->g.polar;
  t.xform = d->g.xform;
  t.max_cells = 1 << (d->g.lx + d->g.ly + d->g.lz);
  st = run_jobs(ctx, d->d_job + slot, t, rebin, d_eps != nullptr, grad, d->g.T, s);
  if (st == ADG_OK) d->partial_dirty = false;
  return st;
}

}  // namespace

// ------------------------------------------------------------------- calls --
extern "C" adg_status adg_build_eps(adg_ctx* ctx, adg_design* d, const double* h_params,
                                    float* d_fill, float* d_eps, void* stream) {
  CallRange nvtx_range("adg_build_eps");
  if (!ctx || !d || !d_eps) return fail(ADG_EINVAL, "adg_build_eps: NULL argument");
  CU(cudaSetDevice(ctx->device));
  return run_single(ctx, d, h_params, d_fill, d_eps, nullptr, nullptr, (cudaStream_t)stream);
}

extern "C" adg_status adg_grad(adg_ctx* ctx, adg_design* d, const double* h_params,
                               const float* const d_efwd[3], const float* const d_eadj[3],
                               const float* w, float* d_grad, void* stream) {
  CallRange nvtx_range("adg_grad");
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
  return run_single(ctx, d, h_params, nullptr, nullptr, &va, d_grad, (cudaStream_t)stream);
}

extern "C" adg_status adg_grad_real(adg_ctx* ctx, adg_design* d, const double* h_params,
                                    const float* d_G, float* d_grad, void* stream) {
  CallRange nvtx_range("adg_grad_real");
  if (!ctx || !d || !d_G || (!d_grad && d->n_params > 0))
    return fail(ADG_EINVAL, "adg_grad_real: NULL argument");
  VjpArgs va{};
  va.G = d_G;
  CU(cudaSetDevice(ctx->device));
  return run_single(ctx, d, h_params, nullptr, nullptr, &va, d_grad, (cudaStream_t)stream);
}

extern "C" adg_status adg_grad_dense(adg_ctx* ctx, adg_design* d, const double* h_params,
                                     const float* const d_efwd[3], const float* const d_eadj[3],
                                     const float* w, const float* d_fill, float* d_grad,
                                     double* d_gmat, void* stream) {
  CallRange nvtx_range("adg_grad_dense");
  if (!ctx || !d || !d_efwd || !d_eadj || !w || !d_fill || !d_gmat || (!d_grad && d->n_params > 0))
    return fail(ADG_EINVAL, "adg_grad_dense: NULL argument");
  VjpArgs va{};
  DenseArgs da{};
  const GridDev& g = d->g;
  for (int c = 0; c < g.C; ++c) {
    if (!d_efwd[c] || !d_eadj[c])
      return fail(ADG_EINVAL, "adg_grad_dense: field of component %d is NULL", c);
    va.ef[c] = da.ef[c] = reinterpret_cast<const float2*>(d_efwd[c]);
    va.ea[c] = da.ea[c] = reinterpret_cast<const float2*>(d_eadj[c]);
    va.w[c] = da.w[c] = make_float2(w[2 * c], w[2 * c + 1]);
  }
  va.G = nullptr;
  da.fill = d_fill;
  da.plane = (long long)g.nx * g.ny * g.nz;
  da.C = g.C;
  da.chunks_per_c = (int)((da.plane + kDenseChunk - 1) / kDenseChunk);
  da.gmat = d_gmat;
  CU(cudaSetDevice(ctx->device));
  if (!d->d_dense_part) {
    CU(lib_malloc((void**)&d->d_dense_part, sizeof(double2) * (size_t)da.C * da.chunks_per_c));
    CU(lib_malloc((void**)&d->d_dense_ctr, sizeof(int)));
  }
  da.part = d->d_dense_part;
  da.ctr = d->d_dense_ctr;
  cudaStream_t s = (cudaStream_t)stream;
  // the band gradient, then the field stream at full occupancy: run side by
  // side on one SM the two slow each other (shared-memory and load pipes)
  const adg_status st = run_single(ctx, d, h_params, nullptr, nullptr, &va, d_grad, s);
  if (st != ADG_OK) return st;
  ProfScope ps(ctx, ADG_K_DENSE, s);
  CU(launch_dense(da, ctx->sms, s));
  return ADG_OK;
}

// ------------------------------------------------------- topology (Sec. 3.1) -
namespace {

adg_status topo_args(const adg_grid* grid, const adg_topo_region* r, const float* d_v,
                     const char* who, TopoArgs& a) {
  if (!grid || !r || !d_v) return fail(ADG_EINVAL, "%s: NULL argument", who);
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || grid->ncomp < 1 || grid->ncomp > 3)
    return fail(ADG_EINVAL, "%s: grid %dx%dx%d with %d components", who, grid->nx, grid->ny,
                grid->nz, grid->ncomp);
  if (r->nx < 1 || r->ny < 1 || r->x0 < 0 || r->y0 < 0 || r->x0 + r->nx > grid->nx ||
      r->y0 + r->ny > grid->ny || r->z0 < 0 || r->z1 <= r->z0 || r->z1 > grid->nz ||
      (long long)r->nx * r->ny > (1LL << 30))
    return fail(ADG_EINVAL, "%s: region x [%d, %d) y [%d, %d) z [%d, %d) outside the %dx%dx%d grid",
                who, r->x0, r->x0 + r->nx, r->y0, r->y0 + r->ny, r->z0, r->z1, grid->nx, grid->ny,
                grid->nz);
  a = TopoArgs{};
  a.nx = grid->nx;
  a.ny = grid->ny;
  a.nz = grid->nz;
  a.C = grid->ncomp;
  a.x0 = r->x0;
  a.y0 = r->y0;
  a.rx = r->nx;
  a.ry = r->ny;
  a.z0 = r->z0;
  a.z1 = r->z1;
  a.v = d_v;
  return ADG_OK;
}

}  // namespace

extern "C" adg_status adg_topo_eps(adg_ctx* ctx, const adg_grid* grid, const adg_topo_region* r,
                                   const float* d_v, double eps_l, double deps, float* d_eps,
                                   void* stream) {
  CallRange nvtx_range("adg_topo_eps");
  if (!ctx || !d_eps) return fail(ADG_EINVAL, "adg_topo_eps: NULL argument");
  TopoArgs a;
  const adg_status st = topo_args(grid, r, d_v, "adg_topo_eps", a);
  if (st != ADG_OK) return st;
  a.eps_l = (float)eps_l;
  a.deps = (float)deps;
  a.eps = d_eps;
  CU(cudaSetDevice(ctx->device));
  CU(launch_topo_eps(a, ctx->sms, (cudaStream_t)stream));
  return ADG_OK;
}

extern "C" adg_status adg_topo_grad(adg_ctx* ctx, const adg_grid* grid, const adg_topo_region* r,
                                    const float* d_v, double deps, const float* const d_efwd[3],
                                    const float* const d_eadj[3], const float* w, float* d_grad,
                                    void* stream) {
  CallRange nvtx_range("adg_topo_grad");
  if (!ctx || !d_efwd || !d_eadj || !w || !d_grad)
    return fail(ADG_EINVAL, "adg_topo_grad: NULL argument");
  TopoArgs a;
  const adg_status st = topo_args(grid, r, d_v, "adg_topo_grad", a);
  if (st != ADG_OK) return st;
  for (int c = 0; c < a.C; ++c) {
    if (!d_efwd[c] || !d_eadj[c])
      return fail(ADG_EINVAL, "adg_topo_grad: field of component %d is NULL", c);
    a.ef[c] = reinterpret_cast<const float2*>(d_efwd[c]);
    a.ea[c] = reinterpret_cast<const float2*>(d_eadj[c]);
    a.w[c] = make_float2(w[2 * c], w[2 * c + 1]);
  }
  a.deps = (float)deps;
  a.grad = d_grad;
  CU(cudaSetDevice(ctx->device));
  CU(launch_topo_grad(a, ctx->sms, (cudaStream_t)stream));
  return ADG_OK;
}

extern "C" adg_status adg_grad_eh(adg_ctx* ctx, adg_design* d_eps, adg_design* d_mu,
                                  const double* h_params, const float* const d_efwd[3],
                                  const float* const d_eadj[3], const float* w_e,
                                  const float* const d_hfwd[3], const float* const d_hadj[3],
                                  const float* w_h, float* d_grad, void* stream) {
  CallRange nvtx_range("adg_grad_eh");
  if (!ctx || !d_eps || !d_mu || !d_efwd || !d_eadj || !w_e || !d_hfwd || !d_hadj || !w_h ||
      (!d_grad && d_eps->n_params > 0))
    return fail(ADG_EINVAL, "adg_grad_eh: NULL argument");
  if (d_eps->n_params != d_mu->n_params)
    return fail(ADG_EINVAL, "adg_grad_eh: the eps design has %d parameters, the mu design %d",
                d_eps->n_params, d_mu->n_params);
  VjpArgs ve{}, vh{};
  for (int c = 0; c < d_eps->g.C; ++c) {
    if (!d_efwd[c] || !d_eadj[c]) return fail(ADG_EINVAL, "adg_grad_eh: E of component %d is NULL", c);
    ve.ef[c] = reinterpret_cast<const float2*>(d_efwd[c]);
    ve.ea[c] = reinterpret_cast<const float2*>(d_eadj[c]);
    ve.w[c] = make_float2(w_e[2 * c], w_e[2 * c + 1]);
  }
  for (int c = 0; c < d_mu->g.C; ++c) {
    if (!d_hfwd[c] || !d_hadj[c]) return fail(ADG_EINVAL, "adg_grad_eh: H of component %d is NULL", c);
    vh.ef[c] = reinterpret_cast<const float2*>(d_hfwd[c]);
    vh.ea[c] = reinterpret_cast<const float2*>(d_hadj[c]);
    vh.w[c] = make_float2(w_h[2 * c], w_h[2 * c + 1]);
  }
  CU(cudaSetDevice(ctx->device));
  const int n = d_eps->n_params;
  if (!d_mu->d_row && n > 0) CU(lib_malloc((void**)&d_mu->d_row, sizeof(float) * n));
  cudaStream_t s = (cudaStream_t)stream;
  adg_status st = run_single(ctx, d_eps, h_params, nullptr, nullptr, &ve, d_grad, s);  // eps term
  if (st != ADG_OK) return st;
  st = run_single(ctx, d_mu, h_params, nullptr, nullptr, &vh, d_mu->d_row, s);      // mu term
  if (st != ADG_OK) return st;
  CU(launch_add(d_mu->d_row, d_grad, n, s));
  return ADG_OK;
}

namespace {

// Validates a list of level sets (App. B, Alg. 1) and fills the parts of
// LevelArgs that do not depend on the pass; sizes the first set's scratch
// to `slices` fill-sized slices.
adg_status levels_setup(adg_ctx* ctx, adg_design* const* sets, int K, const double* levels,
                        const char* who, int slices, LevelArgs& a) {
  if (!ctx || !sets || !levels) return fail(ADG_EINVAL, "%s: NULL argument", who);
  if (K < 1 || K > kMaxLevels)
    return fail(ADG_EINVAL, "%s: %d sets (1 .. %d supported)", who, K, kMaxLevels);
  for (int k = 0; k < K; ++k) {
    if (!sets[k]) return fail(ADG_EINVAL, "%s: set %d is NULL", who, k);
    if (!std::isfinite(levels[k]) || !(levels[k] > 0.0) || (k > 0 && levels[k] < levels[k - 1]))
      return fail(ADG_EINVAL, "%s: levels must be finite, positive and ascending (level %d = %g)",
                  who, k, levels[k]);
    const GridDev &g = sets[k]->g, &g0 = sets[0]->g;
    if (g.eps_bg != 0.0f || g.deps != 1.0f)
      return fail(ADG_EINVAL, "%s: set %d needs material slots eps_bg = 0, eps_fg = 1", who, k);
    bool same = g.nx == g0.nx && g.ny == g0.ny && g.nz == g0.nz && g.C == g0.C &&
                g.logic == g0.logic && sets[k]->n_params == sets[0]->n_params;
    for (int c = 0; c < 3 && same; ++c)
      same = sets[k]->d[c] == sets[0]->d[c] && sets[k]->o[c] == sets[0]->o[c];
    for (int c = 0; c < g.C && same; ++c)
      for (int x = 0; x < 3; ++x) same = same && g.off[c][x] == g0.off[c][x];
    if (!same)
      return fail(ADG_EINVAL, "%s: set %d differs from set 0 in its grid, logic or parameters",
                  who, k);
  }
  const GridDev& g = sets[0]->g;
  a = LevelArgs{};
  a.plane = (long long)g.nx * g.ny * g.nz;
  a.C = g.C;
  a.K = K;
  a.logic = g.logic;
  a.stride = (a.plane * g.C + 63) / 64 * 64;  // 256-byte aligned slices
  a.lv_top = (float)levels[K - 1];
  for (int k = 1; k < K; ++k) a.r[k] = (float)(levels[k - 1] / levels[k]);
  const size_t need = (size_t)a.stride * slices;
  CU(cudaSetDevice(ctx->device));
  adg_design* d0 = sets[0];
  if (d0->lv_cap < need) {
    if (d0->d_lv_buf) {
      CU(cudaDeviceSynchronize());
      CU(lib_free(d0->d_lv_buf));
      d0->d_lv_buf = nullptr;
      d0->lv_cap = 0;
    }
    CU(lib_malloc((void**)&d0->d_lv_buf, sizeof(float) * need));
    d0->lv_cap = need;
  }
  a.fill = d0->d_lv_buf;
  return ADG_OK;
}

}  // namespace

extern "C" adg_status adg_levels_eps(adg_ctx* ctx, adg_design* const* sets, int32_t K,
                                     const double* levels, double eps_bg, const double* h_params,
                                     float* d_eps, void* stream) {
  CallRange nvtx_range("adg_levels_eps");
  LevelArgs a;
  adg_status st = levels_setup(ctx, sets, K, levels, "adg_levels_eps", K, a);
  if (st != ADG_OK) return st;
  if (!d_eps) return fail(ADG_EINVAL, "adg_levels_eps: NULL eps");
  if (!std::isfinite(eps_bg)) return fail(ADG_EINVAL, "adg_levels_eps: eps_bg not finite");
  cudaStream_t s = (cudaStream_t)stream;
  float* fills = sets[0]->d_lv_buf;
  for (int k = 0; k < K; ++k) {  // each set's fill; d_eps is the builds' eps scratch
    st = run_single(ctx, sets[k], h_params, fills + k * a.stride, d_eps, nullptr, nullptr, s);
    if (st != ADG_OK) return st;
  }
  a.out = d_eps;
  a.eps_bg = (float)eps_bg;
  {
    ProfScope ps(ctx, ADG_K_LEVELS, s);
    CU(launch_levels(a, false, ctx->sms, s));
  }
  return ADG_OK;
}

extern "C" adg_status adg_levels_grad(adg_ctx* ctx, adg_design* const* sets, int32_t K,
                                      const double* levels, const double* h_params,
                                      const float* const d_efwd[3], const float* const d_eadj[3],
                                      const float* w, float* d_grad, void* stream) {
  CallRange nvtx_range("adg_levels_grad");
  LevelArgs a;
  adg_status st = levels_setup(ctx, sets, K, levels, "adg_levels_grad", 2 * K, a);
  if (st != ADG_OK) return st;
  const int n = sets[0]->n_params;
  if (!d_efwd || !d_eadj || !w || (!d_grad && n > 0))
    return fail(ADG_EINVAL, "adg_levels_grad: NULL argument");
  for (int c = 0; c < a.C; ++c) {
    if (!d_efwd[c] || !d_eadj[c])
      return fail(ADG_EINVAL, "adg_levels_grad: field of component %d is NULL", c);
    a.ef[c] = reinterpret_cast<const float2*>(d_efwd[c]);
    a.ea[c] = reinterpret_cast<const float2*>(d_eadj[c]);
    a.w[c] = make_float2(w[2 * c], w[2 * c + 1]);
  }
  for (int k = 1; k < K; ++k)
    if (!sets[k]->d_row && n > 0) CU(lib_malloc((void**)&sets[k]->d_row, sizeof(float) * n));
  cudaStream_t s = (cudaStream_t)stream;
  float* fills = sets[0]->d_lv_buf;
  float* cots = fills + (size_t)K * a.stride;
  for (int k = 0; k < K; ++k) {  // each set's fill; the first cotangent slice is eps scratch
    st = run_single(ctx, sets[k], h_params, fills + k * a.stride, cots, nullptr, nullptr, s);
    if (st != ADG_OK) return st;
  }
  a.out = cots;
  {
    ProfScope ps(ctx, ADG_K_LEVELS, s);
    CU(launch_levels(a, true, ctx->sms, s));
  }
  for (int k = 0; k < K; ++k) {  // each set's sweep with its cotangent, then the sum
    VjpArgs va{};
    va.G = cots + k * a.stride;
    st = run_single(ctx, sets[k], h_params, nullptr, nullptr, &va, k ? sets[k]->d_row : d_grad, s);
    if (st != ADG_OK) return st;
    if (k) CU(launch_add(sets[k]->d_row, d_grad, n, s));
  }
  return ADG_OK;
}

namespace {

size_t al256b(size_t v) { return (v + 255) & ~size_t(255); }

adg_status mesh_grid(const adg_grid* g, const char* who) {
  if (!g) return fail(ADG_EINVAL, "%s: NULL grid", who);
  if (g->nx < 1 || g->ny < 1 || g->nz < 1 || g->ncomp < 1 || g->ncomp > 3)
    return fail(ADG_EINVAL, "%s: grid %dx%dx%d with %d components", who, g->nx, g->ny, g->nz,
                g->ncomp);
  if (!(g->dx > 0) || !(g->dy > 0) || !(g->dz > 0) || !std::isfinite(g->dx) ||
      !std::isfinite(g->dy) || !std::isfinite(g->dz) || !std::isfinite(g->ox) ||
      !std::isfinite(g->oy) || !std::isfinite(g->oz))
    return fail(ADG_EINVAL, "%s: spacing must be positive and finite", who);
  return ADG_OK;
}

adg_status mesh_region(const adg_grid* g, const adg_topo_region* r, const char* who,
                       adg_topo_region& out) {
  if (!r) {
    out = adg_topo_region{0, 0, g->nx, g->ny, 0, g->nz};
    return ADG_OK;
  }
  if (r->nx < 1 || r->ny < 1 || r->x0 < 0 || r->y0 < 0 || r->x0 + r->nx > g->nx ||
      r->y0 + r->ny > g->ny || r->z0 < 0 || r->z1 <= r->z0 || r->z1 > g->nz)
    return fail(ADG_EINVAL, "%s: region x [%d, %d) y [%d, %d) z [%d, %d) outside the grid", who,
                r->x0, r->x0 + r->nx, r->y0, r->y0 + r->ny, r->z0, r->z1);
  out = *r;
  return ADG_OK;
}

// One public layer -> device records in cell units, keeping only polygons
// whose box can reach an averaging cell of the region.  The records' offsets
// are relative to the packed arrays; the pointers are set after the upload.
adg_status mesh_pack(const adg_grid* g, const adg_mesh_layer* L, const adg_topo_region& r,
                     const char* who, std::vector<MeshPoly>& polys, std::vector<double2>& verts,
                     MeshLayerDev& dev, int& first) {
  if (!L) return fail(ADG_EINVAL, "%s: NULL layer", who);
  if (L->n_polys < 0 || (L->n_polys > 0 && (!L->vert_off || !L->xy)))
    return fail(ADG_EINVAL, "%s: layer with %d polygons and NULL arrays", who, L->n_polys);
  if (L->bound_z && !(L->z0 <= L->z1 && std::isfinite(L->z0) && std::isfinite(L->z1)))
    return fail(ADG_EINVAL, "%s: layer z range [%g, %g]", who, L->z0, L->z1);
  double omin[2] = {1e300, 1e300}, omax[2] = {-1e300, -1e300};
  for (int c = 0; c < g->ncomp; ++c)
    for (int a = 0; a < 2; ++a) {
      omin[a] = std::min(omin[a], g->off[c][a]);
      omax[a] = std::max(omax[a], g->off[c][a]);
    }
  const double rx0 = r.x0 + omin[0] - 0.5, rx1 = r.x0 + r.nx - 1 + omax[0] + 0.5;
  const double ry0 = r.y0 + omin[1] - 0.5, ry1 = r.y0 + r.ny - 1 + omax[1] + 0.5;
  first = (int)polys.size();
  for (int p = 0; p < L->n_polys; ++p) {
    const int v0 = L->vert_off[p], v1 = L->vert_off[p + 1];
    if (v0 < 0 || v1 - v0 < 3 || (p == 0 && v0 != 0))
      return fail(ADG_EINVAL, "%s: polygon %d has vertices [%d, %d) (need >= 3, offsets from 0)",
                  who, p, v0, v1);
    MeshPoly P{};
    P.bx0 = P.by0 = 1e300;
    P.bx1 = P.by1 = -1e300;
    P.v0 = (int)verts.size();
    P.nv = v1 - v0;
    double area2 = 0.0;
    for (int v = v0; v < v1; ++v) {
      const double x = (L->xy[2 * v] - g->ox) / g->dx, y = (L->xy[2 * v + 1] - g->oy) / g->dy;
      if (!std::isfinite(x) || !std::isfinite(y))
        return fail(ADG_EINVAL, "%s: polygon %d vertex %d not finite", who, p, v - v0);
      verts.push_back(make_double2(x, y));
      P.bx0 = std::min(P.bx0, x);
      P.bx1 = std::max(P.bx1, x);
      P.by0 = std::min(P.by0, y);
      P.by1 = std::max(P.by1, y);
    }
    for (int v = 0; v < P.nv; ++v) {
      const double2 a = verts[P.v0 + v], b = verts[P.v0 + (v + 1) % P.nv];
      area2 += a.x * b.y - b.x * a.y;
    }
    P.sgn = area2 > 0.0 ? -1.0 : 1.0;
    if (P.bx1 <= rx0 || P.bx0 >= rx1 || P.by1 <= ry0 || P.by0 >= ry1) {
      verts.resize(P.v0);  // never reaches the region
      continue;
    }
    polys.push_back(P);
  }
  dev = MeshLayerDev{};
  dev.npolys = (int)polys.size() - first;
  dev.bound_z = L->bound_z ? 1 : 0;
  dev.zl0 = (L->z0 - g->oz) / g->dz;
  dev.zl1 = (L->z1 - g->oz) / g->dz;
  return ADG_OK;
}

// Device scratch of the mesher calls: grown on demand (which synchronises the
// device), never shrunk.
adg_status mesh_reserve(adg_ctx* ctx, size_t need) {
  if (ctx->mesh_cap >= need) return ADG_OK;
  if (ctx->d_mesh) {
    CU(cudaDeviceSynchronize());
    CU(lib_free(ctx->d_mesh));
    ctx->d_mesh = nullptr;
    ctx->mesh_cap = 0;
  }
  CU(lib_malloc(&ctx->d_mesh, need));
  ctx->mesh_cap = need;
  return ADG_OK;
}

MeshGridDev mesh_grid_dev(const adg_grid* g) {
  MeshGridDev m{};
  m.C = g->ncomp;
  for (int c = 0; c < 3; ++c)
    for (int x = 0; x < 3; ++x) m.off[c][x] = c < g->ncomp ? g->off[c][x] : 0.0;
  return m;
}

// Host image of the device records, laid out as on the device: polygons,
// vertices, mesh jobs, dot jobs, chunk table (each 256-byte aligned).
struct MeshImage {
  size_t o_poly = 0, o_vert = 0, o_job = 0, o_dot = 0, o_chunk = 0, bytes = 0;
  std::vector<char> h;
  void layout(size_t np, size_t nv, size_t nj, size_t nd, size_t nc) {
    o_poly = 0;
    o_vert = al256b(sizeof(MeshPoly) * np);
    o_job = o_vert + al256b(sizeof(double2) * nv);
    o_dot = o_job + al256b(sizeof(MeshJob) * nj);
    o_chunk = o_dot + al256b(sizeof(MeshDotJob) * nd);
    bytes = o_chunk + al256b(sizeof(int2) * nc);
    h.assign(bytes, 0);
  }
};

}  // namespace

extern "C" adg_status adg_mesh_fill(adg_ctx* ctx, const adg_grid* grid, const adg_mesh_layer* layer,
                                    const adg_topo_region* region, float* d_fill, void* stream) {
  CallRange nvtx_range("adg_mesh_fill");
  if (!ctx || !d_fill) return fail(ADG_EINVAL, "adg_mesh_fill: NULL argument");
  adg_status st = mesh_grid(grid, "adg_mesh_fill");
  if (st != ADG_OK) return st;
  adg_topo_region r;
  st = mesh_region(grid, region, "adg_mesh_fill", r);
  if (st != ADG_OK) return st;
  std::vector<MeshPoly> polys;
  std::vector<double2> verts;
  MeshLayerDev L;
  int first = 0;
  st = mesh_pack(grid, layer, r, "adg_mesh_fill", polys, verts, L, first);
  if (st != ADG_OK) return st;
  CU(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  MeshImage im;
  im.layout(polys.size(), verts.size(), 1, 0, 0);
  st = mesh_reserve(ctx, im.bytes);
  if (st != ADG_OK) return st;
  char* base = static_cast<char*>(ctx->d_mesh);
  if (!polys.empty()) memcpy(im.h.data() + im.o_poly, polys.data(), sizeof(MeshPoly) * polys.size());
  if (!verts.empty()) memcpy(im.h.data() + im.o_vert, verts.data(), sizeof(double2) * verts.size());
  MeshJob J{};
  J.L = L;
  J.L.polys = reinterpret_cast<const MeshPoly*>(base + im.o_poly) + first;
  J.L.verts = reinterpret_cast<const double2*>(base + im.o_vert);
  J.x0 = r.x0;
  J.y0 = r.y0;
  J.z0 = r.z0;
  J.rx = r.nx;
  J.ry = r.ny;
  J.rz = r.z1 - r.z0;
  J.s_j = grid->nx;
  J.s_k = (long long)grid->nx * grid->ny;
  J.s_c = J.s_k * grid->nz;
  J.out = d_fill + (long long)r.z0 * J.s_k + (long long)r.y0 * J.s_j + r.x0;
  memcpy(im.h.data() + im.o_job, &J, sizeof(J));
  CU(cudaMemcpyAsync(base, im.h.data(), im.bytes, cudaMemcpyHostToDevice, s));
  CU(launch_mesh_fill(reinterpret_cast<const MeshJob*>(base + im.o_job), 1,
                      (long long)r.nx * r.ny * grid->ncomp, mesh_grid_dev(grid), ctx->sms, s));
  return ADG_OK;
}

extern "C" adg_status adg_mesh_grad_fd(adg_ctx* ctx, const adg_grid* grid, int32_t n_params,
                                       const adg_mesh_layer* plus, const adg_mesh_layer* minus,
                                       const adg_topo_region* regions, double h, double deps,
                                       const float* const d_efwd[3], const float* const d_eadj[3],
                                       const float* w, float* d_grad, void* stream) {
  CallRange nvtx_range("adg_mesh_grad_fd");
  const char* who = "adg_mesh_grad_fd";
  if (!ctx || n_params < 0 || (n_params > 0 && (!plus || !minus || !d_grad)) || !d_efwd ||
      !d_eadj || !w)
    return fail(ADG_EINVAL, "%s: NULL argument", who);
  if (!(h > 0.0) || !std::isfinite(h) || !std::isfinite(deps))
    return fail(ADG_EINVAL, "%s: step h = %g, deps = %g", who, h, deps);
  adg_status st = mesh_grid(grid, who);
  if (st != ADG_OK) return st;
  MeshDotFields f{};
  for (int c = 0; c < grid->ncomp; ++c) {
    if (!d_efwd[c] || !d_eadj[c]) return fail(ADG_EINVAL, "%s: field of component %d is NULL", who, c);
    f.ef[c] = reinterpret_cast<const float2*>(d_efwd[c]);
    f.ea[c] = reinterpret_cast<const float2*>(d_eadj[c]);
    f.w[c] = make_float2(w[2 * c], w[2 * c + 1]);
  }
  f.nx = grid->nx;
  f.ny = grid->ny;
  if (n_params == 0) return ADG_OK;
  std::vector<adg_topo_region> rs(n_params);
  std::vector<long long> ns(n_params);
  for (int k = 0; k < n_params; ++k) {
    st = mesh_region(grid, regions ? regions + k : nullptr, who, rs[k]);
    if (st != ADG_OK) return st;
    ns[k] = (long long)grid->ncomp * (rs[k].z1 - rs[k].z0) * rs[k].ny * rs[k].nx;
    if (ns[k] > (1LL << 30))
      return fail(ADG_EINVAL, "%s: region of parameter %d holds %lld samples (at most 2^30)", who,
                  k, ns[k]);
  }
  CU(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const MeshGridDev gd = mesh_grid_dev(grid);
  // Parameters go in groups whose two meshes per region fit the scratch
  // budget; each group is three launches over all of its parameters.
  const long long budget = 1LL << 28;  // floats of region scratch per group (1 GiB)
  for (int k0 = 0; k0 < n_params;) {
    int k1 = k0;
    long long tot = 0;
    while (k1 < n_params && (k1 == k0 || tot + 2 * ns[k1] <= budget)) tot += 2 * ns[k1++];
    const int nk = k1 - k0;
    std::vector<MeshPoly> polys;
    std::vector<double2> verts;
    std::vector<MeshLayerDev> lp(nk), lm(nk);
    std::vector<int> fp(nk), fm(nk);
    long long max_cols = 0, nch = 0;
    for (int k = k0; k < k1; ++k) {
      st = mesh_pack(grid, plus + k, rs[k], who, polys, verts, lp[k - k0], fp[k - k0]);
      if (st != ADG_OK) return st;
      st = mesh_pack(grid, minus + k, rs[k], who, polys, verts, lm[k - k0], fm[k - k0]);
      if (st != ADG_OK) return st;
      max_cols = std::max(max_cols, (long long)rs[k].nx * rs[k].ny * grid->ncomp);
      nch += (ns[k] + kMeshChunk - 1) / kMeshChunk;
    }
    MeshImage im;
    im.layout(polys.size(), verts.size(), 2 * nk, nk, (size_t)nch);
    const size_t b_part = al256b(sizeof(double) * (size_t)std::max<long long>(nch, 1));
    st = mesh_reserve(ctx, im.bytes + b_part + sizeof(float) * (size_t)tot);
    if (st != ADG_OK) return st;
    char* base = static_cast<char*>(ctx->d_mesh);
    double* part = reinterpret_cast<double*>(base + im.bytes);
    float* buf = reinterpret_cast<float*>(base + im.bytes + b_part);
    const MeshPoly* dpol = reinterpret_cast<const MeshPoly*>(base + im.o_poly);
    const double2* dver = reinterpret_cast<const double2*>(base + im.o_vert);
    if (!polys.empty())
      memcpy(im.h.data() + im.o_poly, polys.data(), sizeof(MeshPoly) * polys.size());
    if (!verts.empty())
      memcpy(im.h.data() + im.o_vert, verts.data(), sizeof(double2) * verts.size());
    MeshJob* jobs = reinterpret_cast<MeshJob*>(im.h.data() + im.o_job);
    MeshDotJob* dots = reinterpret_cast<MeshDotJob*>(im.h.data() + im.o_dot);
    int2* chunks = reinterpret_cast<int2*>(im.h.data() + im.o_chunk);
    long long off = 0;
    int ch = 0;
    for (int k = k0; k < k1; ++k) {
      const int i = k - k0;
      const adg_topo_region& r = rs[k];
      float* A = buf + off;
      float* B = A + ns[k];
      off += 2 * ns[k];
      for (int side = 0; side < 2; ++side) {
        MeshJob& J = jobs[2 * i + side];
        J.L = side ? lm[i] : lp[i];
        J.L.polys = dpol + (side ? fm[i] : fp[i]);
        J.L.verts = dver;
        J.out = side ? B : A;
        J.x0 = r.x0;
        J.y0 = r.y0;
        J.z0 = r.z0;
        J.rx = r.nx;
        J.ry = r.ny;
        J.rz = r.z1 - r.z0;
        J.s_j = r.nx;
        J.s_k = (long long)r.nx * r.ny;
        J.s_c = J.s_k * (r.z1 - r.z0);
      }
      MeshDotJob& D = dots[i];
      D.a = A;
      D.b = B;
      D.x0 = r.x0;
      D.y0 = r.y0;
      D.z0 = r.z0;
      D.rx = r.nx;
      D.ry = r.ny;
      D.rz = r.z1 - r.z0;
      D.n = (int)ns[k];
      D.param = k;
      D.chunk0 = ch;
      for (long long q = 0; q < ns[k]; q += kMeshChunk) chunks[ch++] = make_int2(i, (int)q);
      D.chunk1 = ch;
    }
    CU(cudaMemcpyAsync(base, im.h.data(), im.bytes, cudaMemcpyHostToDevice, s));
    const MeshJob* djobs = reinterpret_cast<const MeshJob*>(base + im.o_job);
    const MeshDotJob* ddots = reinterpret_cast<const MeshDotJob*>(base + im.o_dot);
    const int2* dchunks = reinterpret_cast<const int2*>(base + im.o_chunk);
    CU(launch_mesh_fill(djobs, 2 * nk, max_cols, gd, ctx->sms, s));
    CU(launch_mesh_dot(ddots, nk, dchunks, ch, f, part, deps / (2.0 * h), d_grad, ctx->sms, s));
    k0 = k1;
  }
  return ADG_OK;
}

extern "C" adg_status adg_grad_fd(adg_ctx* ctx, adg_design* d, const double* h_params,
                                  const float* const d_efwd[3], const float* const d_eadj[3],
                                  const float* w, double h, float* d_grad, void* stream) {
  CallRange nvtx_range("adg_grad_fd");
  if (!ctx || !d || !d_efwd || !d_eadj || !w || (!d_grad && d->n_params > 0) ||
      (!h_params && d->n_params > 0))
    return fail(ADG_EINVAL, "adg_grad_fd: NULL argument");
  if (!(h > 0.0)) return fail(ADG_EINVAL, "adg_grad_fd: step h = %g must be positive", h);
  const GridDev& g = d->g;
  FdSeedArgs sa{};
  for (int c = 0; c < g.C; ++c) {
    if (!d_efwd[c] || !d_eadj[c])
      return fail(ADG_EINVAL, "adg_grad_fd: field of component %d is NULL", c);
    sa.ef[c] = reinterpret_cast<const float2*>(d_efwd[c]);
    sa.ea[c] = reinterpret_cast<const float2*>(d_eadj[c]);
    sa.w[c] = make_float2(w[2 * c], w[2 * c + 1]);
  }
  sa.plane = (long long)g.nx * g.ny * g.nz;
  sa.C = g.C;
  const long long ns = sa.plane * g.C;  // samples
  const int n = d->n_params;
  CU(cudaSetDevice(ctx->device));
  if (!d->d_fd_buf) {
    CU(lib_malloc((void**)&d->d_fd_buf, sizeof(float) * (size_t)ns * 4));
    CU(lib_malloc((void**)&d->d_fd_part, sizeof(double) * (size_t)std::max(fd_chunks(ns), 1)));
    CU(lib_malloc((void**)&d->d_fd_acc, sizeof(double) * (size_t)std::max(n, 1)));
  }
  float* z = d->d_fd_buf;
  float* fa = z + ns;
  float* fb = fa + ns;
  float* es = fb + ns;
  sa.z = z;
  cudaStream_t s = (cudaStream_t)stream;
  CU(launch_fd_seed(sa, ctx->sms, s));
  std::vector<double> p(h_params, h_params + n);
  for (int k = 0; k < n; ++k) {  // two builds per parameter, then one dot product
    const double p0 = p[k];
    p[k] = p0 + h;
    adg_status st = run_single(ctx, d, p.data(), fa, es, nullptr, nullptr, s);
    if (st != ADG_OK) return st;
    p[k] = p0 - h;
    st = run_single(ctx, d, p.data(), fb, es, nullptr, nullptr, s);
    if (st != ADG_OK) return st;
    p[k] = p0;
    CU(launch_fd_dot(z, fa, fb, ns, d->d_fd_part, d->d_fd_acc + k, s));
  }
  CU(launch_fd_scale(d->d_fd_acc, n, (double)g.deps / (2.0 * h), d_grad, s));
  return ADG_OK;
}

// ------------------------------------------------------------------ batches -
namespace {

size_t al256(size_t v) { return (v + 255) & ~size_t(255); }

uint64_t mix(uint64_t h, uint64_t v) {
  h ^= v + 0x9e3779b97f4a7c15ULL + (h << 6) + (h >> 2);
  return h;
}

}  // namespace

extern "C" adg_status adg_batch_submit(adg_ctx* ctx, const adg_batch_item* items, int32_t n,
                                       int32_t flags, void* stream, uint64_t* ticket) {
  CallRange nvtx_range("adg_batch_submit");
  if (!ctx || !items || !ticket) return fail(ADG_EINVAL, "adg_batch_submit: NULL argument");
  if (n < 1 || n > kMaxJobs) return fail(ADG_EINVAL, "batch of %d items (1..%d)", n, kMaxJobs);
  if (flags & ~ADG_BATCH_GRAPH) return fail(ADG_EINVAL, "unknown batch flags 0x%x", flags);
  cudaStream_t s = (cudaStream_t)stream;
  CU(cudaSetDevice(ctx->device));
  for (int i = 0; i < n; ++i) {
    const adg_batch_item& it = items[i];
    adg_design* d = it.design;
    if (!d || d->ctx != ctx) return fail(ADG_EINVAL, "item %d: design missing or of another context", i);
    if (it.reserved != 0 || it.ops <= 0 || (it.ops & ~7) ||
        ((it.ops & ADG_BATCH_GRAD) && (it.ops & ADG_BATCH_GRAD_REAL)))
      return fail(ADG_EINVAL, "item %d: ops 0x%x invalid", i, it.ops);
    if ((it.ops & ADG_BATCH_BUILD) && !it.d_eps) return fail(ADG_EINVAL, "item %d: d_eps is NULL", i);
    if ((it.ops & (ADG_BATCH_GRAD | ADG_BATCH_GRAD_REAL)) && !it.d_grad && d->n_params > 0)
      return fail(ADG_EINVAL, "item %d: d_grad is NULL", i);
    if ((it.ops & ADG_BATCH_GRAD_REAL) && !it.d_G) return fail(ADG_EINVAL, "item %d: d_G is NULL", i);
    if (it.ops & ADG_BATCH_GRAD)
      for (int c = 0; c < d->g.C; ++c)
        if (!it.d_efwd[c] || !it.d_eadj[c]) return fail(ADG_EINVAL, "item %d: field %d is NULL", i, c);
    if (d->n_params > 0 && !it.h_params) return fail(ADG_EINVAL, "item %d: h_params is NULL", i);
    for (int k = 0; k < i; ++k)
      if (items[k].design == d) return fail(ADG_EINVAL, "items %d and %d share a design", k, i);
  }
  adg_ctx::Arena& A = ctx->arenas[ctx->next_arena];
  const int arena_id = ctx->next_arena;
  ctx->next_arena ^= 1;
  if (A.used) CU(cudaEventSynchronize(A.done));  // the batch two back released this arena
  // parameter maps (host, FP64) and sizes of the packed upload
  size_t nprim = 0, nauxd = 0, nauxf = 0;
  // until the launches are enqueued, a failure leaves every flipped design to
  // be re-binned from cleared counters
  struct Flipped {
    const adg_batch_item* items;
    int n = 0;
    bool done = false;
    ~Flipped() {
      if (!done)
        for (int k = 0; k < n; ++k) invalidate_bins(items[k].design);
    }
  } flipped{items};
  for (int i = 0; i < n; ++i) {
    adg_design* d = items[i].design;
    adg_status st = prepare_prims(d, items[i].h_params);
    if (st != ADG_OK) return st;
    if (d->counters_dirty) {
      CU(cudaMemsetAsync(d->d_counters, 0, sizeof(int) * 8, s));  // both counter sets
      d->counters_dirty = false;
    }
    d->bins_valid = false;  // the batch re-bins this design with its own records
    // the design's single-call kernels so far read record buffer gen: a later
    // upload into it waits for them
    CU(cudaEventRecord(d->used[d->gen], s));
    d->gen ^= 1;            // into the other counter set (cleared by the last binning)
    flipped.n = i + 1;
    if (items[i].ops & (ADG_BATCH_GRAD | ADG_BATCH_GRAD_REAL)) {
      st = ensure_partials(d, s);
      if (st != ADG_OK) return st;
    }
    nprim += d->n_prims;
    nauxd += d->st.auxd_n;
    nauxf += d->st.auxf_n;
  }
  const size_t o_jobs = 0;
  const size_t o_prims = al256(o_jobs + sizeof(Job) * n);
  const size_t o_auxd = al256(o_prims + sizeof(PrimRec) * nprim);
  const size_t o_auxf = al256(o_auxd + sizeof(double) * nauxd);
  const size_t bytes = al256(o_auxf + sizeof(float) * nauxf);
  if (bytes > A.cap) {
    if (A.exec) { cudaGraphExecDestroy(A.exec); A.exec = nullptr; A.sig = 0; }
    lib_free(A.d);
    lib_free_host(A.h);
    A.d = nullptr;
    A.h = nullptr;
    A.cap = 0;
    const size_t cap = bytes + bytes / 2 + 4096;
    CU(lib_malloc(&A.d, cap));
    CU(lib_malloc_host(&A.h, cap));
    A.cap = cap;
  }
  if (!A.done) CU(cudaEventCreateWithFlags(&A.done, cudaEventDisableTiming));
  if (!A.d_work) {
    CU(lib_malloc((void**)&A.d_work, sizeof(int) * 8));
    CU(cudaMemset(A.d_work, 0, sizeof(int) * 8));
  }
  unsigned char* hb = static_cast<unsigned char*>(A.h);
  unsigned char* db = static_cast<unsigned char*>(A.d);
  Job* hj = reinterpret_cast<Job*>(hb + o_jobs);
  size_t po = 0, ado = 0, afo = 0;
  int tile_base = 0, param_base = 0, max_tiles = 0, row_base = 0, max_cells = 128;
  bool any_build = false, any_grad = false, any_polar = false, any_xform = false;
  uint64_t sig = mix(0, (uint64_t)arena_id);
  sig = mix(sig, (uint64_t)n);
  for (int i = 0; i < n; ++i) {
    const adg_batch_item& it = items[i];
    adg_design* d = it.design;
    PrimRec* hp = reinterpret_cast<PrimRec*>(hb + o_prims) + po;
    memcpy(hp, d->h_prims.data(), sizeof(PrimRec) * d->n_prims);
    if (d->st.auxd_n)
      memcpy(reinterpret_cast<double*>(hb + o_auxd) + ado, d->h_auxd.data(), sizeof(double) * d->st.auxd_n);
    if (d->st.auxf_n)
      memcpy(reinterpret_cast<float*>(hb + o_auxf) + afo, d->h_auxf.data(), sizeof(float) * d->st.auxf_n);
    Job J = design_job(d);
    J.prims = reinterpret_cast<const PrimRec*>(db + o_prims) + po;
    J.auxd = reinterpret_cast<const double*>(db + o_auxd) + ado;
    J.auxf = reinterpret_cast<const float*>(db + o_auxf) + afo;
    J.do_bin = 1;
    J.do_build = (it.ops & ADG_BATCH_BUILD) ? 1 : 0;
    J.do_grad = (it.ops & (ADG_BATCH_GRAD | ADG_BATCH_GRAD_REAL)) ? 1 : 0;
    J.fill = it.d_fill;
    J.eps = it.d_eps;
    J.grad = it.d_grad;
    if (it.ops & ADG_BATCH_GRAD) {
      for (int c = 0; c < d->g.C; ++c) {
        J.va.ef[c] = reinterpret_cast<const float2*>(it.d_efwd[c]);
        J.va.ea[c] = reinterpret_cast<const float2*>(it.d_eadj[c]);
        J.va.w[c] = make_float2(it.w[2 * c], it.w[2 * c + 1]);
      }
    } else if (it.ops & ADG_BATCH_GRAD_REAL) {
      J.va.G = it.d_G;
    }
    J.partial_n = J.do_grad ? (long long)d->part_total : 0;
    J.param_base = param_base;
    J.tile_base = tile_base;
    J.row_base = row_base;
    if (J.do_build) row_base += (d->g.C * d->g.nz * d->g.ny + kFillRows - 1) / kFillRows;
    if (J.do_grad) {
      param_base += d->n_params;
      d->partial_dirty = true;  // until the finalize is enqueued
    }
    tile_base += ((d->g.T + 127) / 128) * 128;
    max_tiles = std::max(max_tiles, d->g.T);
    if (J.do_grad) max_cells = std::max(max_cells, 1 << (d->g.lx + d->g.ly + d->g.lz));
    any_build = any_build || J.do_build;
    any_grad = any_grad || J.do_grad;
    any_polar = any_polar || (J.do_grad && d->g.polar);
    any_xform = any_xform || d->g.xform;
    hj[i] = J;
    po += d->n_prims;
    ado += d->st.auxd_n;
    afo += d->st.auxf_n;
    sig = mix(sig, (uint64_t)d->g.T);
    sig = mix(sig, (uint64_t)it.ops);
  }
  JobTotals t{};
  t.njobs = n;
  t.tiles_padded = tile_base;
  t.bin_blocks = tile_base / 128;
  t.fill_blocks = row_base;
  t.params = param_base;
  t.work = A.d_work;
  t.fill_warps = 1;
  t.polar = any_polar ? 1 : 0;
  t.xform = any_xform ? 1 : 0;
  t.max_cells = max_cells;
  sig = mix(sig, (uint64_t)t.polar);  // the captured VJP kernel depends on it
  sig = mix(sig, (uint64_t)t.xform);  // and the build and VJP kernels on this
  sig = mix(sig, (uint64_t)t.max_cells);  // the VJP's shared memory and grid
  sig = mix(sig, (uint64_t)bytes);
  sig = mix(sig, (uint64_t)tile_base);
  sig = mix(sig, (uint64_t)param_base);
  build_blocks_per_sm(t.njobs, t.fill_warps, t.xform != 0);  // set before any capture
  vjp_blocks_per_sm(t.njobs, t.polar || t.xform, t.max_cells);
  const bool graph = (flags & ADG_BATCH_GRAPH) && !ctx->prof;
  if (graph && A.exec && A.sig == sig) {
    CU(cudaGraphLaunch(A.exec, s));
  } else if (graph) {
    if (A.exec) { cudaGraphExecDestroy(A.exec); A.exec = nullptr; A.sig = 0; }
    // capture on the context's own stream (the legacy default stream cannot
    // be captured); the graph itself is launched on the caller's stream
    if (!ctx->capture) CU(cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking));
    cudaStream_t cs = ctx->capture;
    CU(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemcpyAsync(A.d, A.h, bytes, cudaMemcpyHostToDevice, cs);
    adg_status st = e == cudaSuccess ? run_jobs(ctx, reinterpret_cast<const Job*>(db + o_jobs), t,
                                                true, any_build, any_grad, max_tiles, cs)
                                     : ADG_ECUDA;
    cudaGraph_t gr = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &gr);
    if (st != ADG_OK) { if (gr) cudaGraphDestroy(gr); return st; }
    if (e != cudaSuccess || e2 != cudaSuccess)
      return fail(ADG_ECUDA, "batch capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    e = cudaGraphInstantiate(&A.exec, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) { A.exec = nullptr; return fail(ADG_ECUDA, "graph instantiate: %s", cudaGetErrorString(e)); }
    A.sig = sig;
    CU(cudaGraphLaunch(A.exec, s));
  } else {
    CU(cudaMemcpyAsync(A.d, A.h, bytes, cudaMemcpyHostToDevice, s));
    adg_status st = run_jobs(ctx, reinterpret_cast<const Job*>(db + o_jobs), t, true, any_build,
                             any_grad, max_tiles, s);
    if (st != ADG_OK) return st;
  }
  flipped.done = true;  // every design's binning is enqueued
  for (int i = 0; i < n; ++i)  // the finalize of every gradient item is enqueued
    if (items[i].ops & (ADG_BATCH_GRAD | ADG_BATCH_GRAD_REAL)) items[i].design->partial_dirty = false;
  CU(cudaEventRecord(A.done, s));
  A.used = true;
  cudaEvent_t ev = nullptr;
  CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  CU(cudaEventRecord(ev, s));
  const uint64_t id = ctx->next_ticket++;
  ctx->tickets.push_back({id, ev});
  *ticket = id;
  return ADG_OK;
}

extern "C" adg_status adg_batch_poll(adg_ctx* ctx, uint64_t ticket, int32_t* done) {
  if (!ctx || !done) return fail(ADG_EINVAL, "adg_batch_poll: NULL argument");
  CU(cudaSetDevice(ctx->device));
  for (size_t k = 0; k < ctx->tickets.size(); ++k) {
    if (ctx->tickets[k].id != ticket) continue;
    const cudaError_t e = cudaEventQuery(ctx->tickets[k].ev);
    if (e == cudaErrorNotReady) { *done = 0; return ADG_OK; }
    cudaEventDestroy(ctx->tickets[k].ev);
    ctx->tickets.erase(ctx->tickets.begin() + k);
    if (e != cudaSuccess) return fail(ADG_ECUDA, "batch %llu: %s", (unsigned long long)ticket, cudaGetErrorString(e));
    *done = 1;
    return ADG_OK;
  }
  if (ticket == 0 || ticket >= ctx->next_ticket) return fail(ADG_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
  *done = 1;  // already collected
  return ADG_OK;
}

extern "C" adg_status adg_batch_wait(adg_ctx* ctx, uint64_t ticket, uint64_t timeout_ns) {
  if (!ctx) return fail(ADG_EINVAL, "adg_batch_wait: NULL context");
  const auto t0 = std::chrono::steady_clock::now();
  while (true) {
    int32_t done = 0;
    adg_status st = adg_batch_poll(ctx, ticket, &done);
    if (st != ADG_OK || done) return st;
    const auto el = std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0);
    if ((uint64_t)el.count() >= timeout_ns)
      return fail(ADG_ETIMEOUT, "batch %llu still running after %llu ns", (unsigned long long)ticket,
                  (unsigned long long)timeout_ns);
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
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
                "16 partial range, 32 program, 64 tile pool, 128 debug bound check); use a "
                "smaller tile shape",
                e);
  }
  return ADG_OK;
}

extern "C" adg_status adg_design_stats(adg_ctx* ctx, adg_design* d, void* stream, adg_stats* out) {
  if (!ctx || !d || !out) return fail(ADG_EINVAL, "adg_design_stats: NULL argument");
  CU(cudaSetDevice(ctx->device));
  CU(cudaStreamSynchronize((cudaStream_t)stream));
  int c[4] = {0, 0, 0, 0}, last = 0;
  CU(cudaMemcpy(c, d->d_counters + 4 * d->gen, sizeof(c), cudaMemcpyDeviceToHost));
  CU(cudaMemcpy(&last, d->d_counters + 8, sizeof(int), cudaMemcpyDeviceToHost));
  out->tiles = d->g.T;
  out->program_tiles = c[0];
  out->max_ops = c[1];
  out->band_cells = c[2];
  out->active_samples = last;
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
void set_last_error(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }
}  // namespace adg

extern "C" const char* adg_last_error(void) { return g_err; }

// Device bytes a design holds: its tables, bins and counters, the partial
// buffer at the size its current parameters need (or its capacity, if
// larger), and the scratch of the optional calls it has made.
size_t design_bytes(const adg_design* d) {
  auto vb = [](const auto& v) { return std::max<size_t>(v.size(), 1) * sizeof(v[0]); };
  size_t b = vb(d->chain) + vb(d->act) + vb(d->actc) + vb(d->ref_off) + vb(d->ref_prim) +
             vb(d->ref_qa) + vb(d->ref_coeff) + 2 * record_bytes(d);
  const size_t T = (size_t)d->g.T;
  b += T * (sizeof(TileProg) + 1 + sizeof(int)) + 20 * sizeof(int) +
       sizeof(Job) * adg_design::kJobSlots;
  b += std::max(d->partial_cap, d->part_total) * sizeof(float);
  const size_t plane = (size_t)d->g.nx * d->g.ny * d->g.nz, ns = plane * d->g.C;
  if (d->d_dense_part)
    b += sizeof(double2) * d->g.C * ((plane + kDenseChunk - 1) / kDenseChunk) + sizeof(int);
  if (d->d_fd_buf)
    b += sizeof(float) * ns * 4 + sizeof(double) * std::max(fd_chunks((long long)ns), 1) +
         sizeof(double) * std::max(d->n_params, 1);
  if (d->d_row) b += sizeof(float) * d->n_params;
  b += sizeof(float) * d->lv_cap;
  return b;
}

extern "C" adg_status adg_design_bytes(adg_ctx* ctx, adg_design* d, int64_t* bytes) {
  if (!ctx || !d || !bytes) return fail(ADG_EINVAL, "adg_design_bytes: NULL argument");
  *bytes = (int64_t)design_bytes(d);
  return ADG_OK;
}

extern "C" adg_status adg_debug_alloc(int32_t fail_after, int64_t* live) {
  if (fail_after >= -1) g_fail_after.store(fail_after);
  if (live) *live = g_live.load();
  return ADG_OK;
}
