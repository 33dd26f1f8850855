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

#include "adg_host.h"
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
  int work[6 * kNAMaxOps];
  int chain[2 * kNAMaxOps];
  int act[kNAMaxQ], nact[kNAMaxPrims], act_off[kNAMaxPrims];
  float actc[kNAMaxQ];
  int auxd_off[kNAMaxPrims], auxf_off[kNAMaxPrims];
  int count[kNAMaxParams + 1], ref_off[kNAMaxParams + 1], ref_prim[kNAMaxQ], ref_qa[kNAMaxQ];
  double ref_coeff[kNAMaxQ];
  double q[kNAMaxQ];
  PrimRec prims[kNAMaxPrims];
  double auxd[6 * kNAMaxQ];
  float auxf[6 * kNAMaxQ];
  Job job;
};

NoAllocHost g_host;
std::mutex g_mu;
void* g_sym[kNAMaxDevices];
bool g_sym_ok[kNAMaxDevices];

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

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

#define NACU(call)                                                                            \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return na_fail(ADG_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

extern "C" adg_status adg_grad_noalloc(const adg_design_desc* D, const adg_tile_opts* tiles,
                                       const double* h_params, const float* const d_efwd[3],
                                       const float* const d_eadj[3], const float* w,
                                       float* d_grad, void* stream) {
  std::lock_guard<std::mutex> lock(g_mu);
  NoAllocHost& H = g_host;
  if (!D || !d_efwd || !d_eadj || !w) return na_fail(ADG_EINVAL, "adg_grad_noalloc: NULL argument");
  host::Msg m;
  if (host::validate(D, m) != ADG_OK) return na_fail(ADG_EINVAL, "%s", m.text);
  size_t nqs = 0;
  for (int p = 0; p < D->n_prims; ++p) nqs += D->prim_nq[p];
  if (D->n_prims > kNAMaxPrims || D->n_q > kNAMaxQ || (int64_t)nqs > kNAMaxQ ||
      D->n_ops > kNAMaxOps || D->n_params > kNAMaxParams)
    return na_fail(ADG_EINVAL,
                   "adg_grad_noalloc limits: primitives <= %d, scalars <= %d, ops <= %d, "
                   "params <= %d (got %d, %d, %d, %d)",
                   kNAMaxPrims, kNAMaxQ, kNAMaxOps, kNAMaxParams, D->n_prims, (int)nqs, D->n_ops,
                   D->n_params);
  if (D->n_params > 0 && (!h_params || !d_grad))
    return na_fail(ADG_EINVAL, "h_params / d_grad is NULL");
  for (int c = 0; c < D->grid.ncomp; ++c)
    if (!d_efwd[c] || !d_eadj[c]) return na_fail(ADG_EINVAL, "field of component %d is NULL", c);
  int tx = 32, ty = 4, tz = 4;
  if (tiles && (tiles->tx || tiles->ty || tiles->tz)) { tx = tiles->tx; ty = tiles->ty; tz = tiles->tz; }
  if (!host::tile_ok(tx, ty, tz)) return na_fail(ADG_EINVAL, "tile %dx%dx%d not supported", tx, ty, tz);
  // ---- compile: chain, slots, references (static host storage) ----
  const int n = D->n_ops;
  host::ChainWork cw{H.work, H.work + n, H.work + 2 * n, H.work + 3 * n, H.work + 4 * n,
                     H.work + 5 * n};
  int nchain = 0;
  if (host::compile_chain(D, cw, H.chain, &nchain, m) != ADG_OK)
    return na_fail(ADG_EINVAL, "%s", m.text);
  host::SlotTables st{H.act, H.nact, H.act_off, H.actc, H.ref_off, H.ref_prim, H.ref_qa,
                      H.ref_coeff, H.auxd_off, H.auxf_off, 0, 0, 0, 0};
  for (int p = 0; p < D->n_prims; ++p)
    if (host::aux_doubles(D->prim_kind[p], D->prim_nq[p], D->prim_flags[p]) > 6 * kNAMaxQ)
      return na_fail(ADG_EINVAL, "primitive %d has too many vertices", p);
  host::build_slots(D, st, H.count);
  if (st.auxd_n > 6 * kNAMaxQ || st.auxf_n > 6 * kNAMaxQ)
    return na_fail(ADG_EINVAL, "graph / polygon vertices exceed the static limits");
  GridDev g;
  host::set_grid(D, tx, ty, tz, nchain, g);
  // ---- parameter map (FP64) and primitive records ----
  if (host::map_params(D->n_q, D->q_base, D->q_coeff, D->q_param, h_params, H.q, m) != ADG_OK)
    return na_fail(ADG_EINVAL, "%s", m.text);
  const double dd[3] = {D->grid.dx, D->grid.dy, D->grid.dz};
  const double oo[3] = {D->grid.ox, D->grid.oy, D->grid.oz};
  host::PrimTable P{D->prim_kind, D->prim_sigma, D->prim_flags, D->prim_q0, D->prim_nq,
                    D->prim_kr, D->n_prims};
  size_t part = 0;
  if (host::prepare_prims(g, dd, oo, P, st, H.q, H.prims, H.auxd, H.auxf, &part, m) != ADG_OK)
    return na_fail(ADG_EINVAL, "%s", m.text);
  // ---- carve the static scratch; reject what does not fit ----
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off = align256(off + bytes); return o; };
  const size_t o_err = take(sizeof(int));
  const size_t o_job = take(sizeof(Job));
  // this call's counter set, the one its binning clears, the moved active-sample
  // count, the persistent kernels' tile counters
  const size_t o_cnt = take(20 * sizeof(int));
  const size_t o_chain = take(sizeof(int) * nchain);
  const size_t o_act = take(sizeof(int) * std::max(st.nact_table, 1));
  const size_t o_actc = take(sizeof(float) * std::max(st.nact_table, 1));
  const size_t o_roff = take(sizeof(int) * (D->n_params + 1));
  const size_t o_rprim = take(sizeof(int) * std::max(st.nrefs, 1));
  const size_t o_rqa = take(sizeof(int) * std::max(st.nrefs, 1));
  const size_t o_rcoef = take(sizeof(double) * std::max(st.nrefs, 1));
  const size_t o_prims = take(sizeof(PrimRec) * D->n_prims);
  const size_t o_auxd = take(sizeof(double) * std::max(st.auxd_n, 1));
  const size_t o_auxf = take(sizeof(float) * std::max(st.auxf_n, 1));
  const size_t o_progs = take(sizeof(TileProg) * (size_t)g.T);
  const size_t o_list = take(sizeof(int) * (size_t)g.T);
  const size_t o_tcls = take((size_t)g.T);
  const size_t o_part = take(sizeof(float) * std::max<size_t>(part, 1));
  // the VJP's long-program tape: one slice per block, one block per SM
  int dev = 0, sms = 1;
  NACU(cudaGetDevice(&dev));
  NACU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const size_t o_gtape = take(sizeof(float) * kTapeBlockFloats * (size_t)sms);
  if (off > kNoAllocScratchBytes)
    return na_fail(ADG_EINVAL,
                   "adg_grad_noalloc: this design needs %zu bytes of scratch (%d tiles, %zu "
                   "partials); the static scratch holds %zu bytes -- use a larger tile shape or "
                   "adg_grad",
                   off, g.T, part, kNoAllocScratchBytes);
  // ---- set-up once per device: the array's device address ----
  if (dev < 0 || dev >= kNAMaxDevices) return na_fail(ADG_EINVAL, "device %d out of range", dev);
  if (!g_sym_ok[dev]) {
    NACU(init_kernel_attributes());
    void* ptr = nullptr;
    NACU(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    g_sym[dev] = ptr;
    g_sym_ok[dev] = true;
  }
  unsigned char* base = static_cast<unsigned char*>(g_sym[dev]);
  cudaStream_t s = (cudaStream_t)stream;
  // From the first enqueue on, every return waits for this call's stream work
  // before the lock is released (the guard is destroyed first): a failed
  // enqueue must not leave kernels reading the shared array while the next
  // call overwrites it.
  struct DrainOnExit {
    cudaStream_t s;
    ~DrainOnExit() { cudaStreamSynchronize(s); }
  } drain{s};
  int* d_err = reinterpret_cast<int*>(base + o_err);
  Job* d_job = reinterpret_cast<Job*>(base + o_job);
  int* d_cnt = reinterpret_cast<int*>(base + o_cnt);
  int* d_chain = reinterpret_cast<int*>(base + o_chain);
  int* d_act = reinterpret_cast<int*>(base + o_act);
  float* d_actc = reinterpret_cast<float*>(base + o_actc);
  int* d_roff = reinterpret_cast<int*>(base + o_roff);
  int* d_rprim = reinterpret_cast<int*>(base + o_rprim);
  int* d_rqa = reinterpret_cast<int*>(base + o_rqa);
  double* d_rcoef = reinterpret_cast<double*>(base + o_rcoef);
  PrimRec* d_prims = reinterpret_cast<PrimRec*>(base + o_prims);
  double* d_auxd = reinterpret_cast<double*>(base + o_auxd);
  float* d_auxf = reinterpret_cast<float*>(base + o_auxf);
  TileProg* d_progs = reinterpret_cast<TileProg*>(base + o_progs);
  int* d_list = reinterpret_cast<int*>(base + o_list);
  unsigned char* d_tcls = base + o_tcls;
  float* d_part = reinterpret_cast<float*>(base + o_part);
  float* d_gtape = reinterpret_cast<float*>(base + o_gtape);
  // ---- upload, clear, launch (binner -> VJP -> finalize) ----
  NACU(cudaMemsetAsync(d_err, 0, sizeof(int), s));
  NACU(cudaMemsetAsync(d_cnt, 0, 4 * sizeof(int), s));
  NACU(cudaMemsetAsync(d_cnt + 12, 0, 8 * sizeof(int), s));  // the space is shared by all calls
  // the partials' space held other tables in earlier calls
  NACU(cudaMemsetAsync(d_part, 0, sizeof(float) * std::max<size_t>(part, 1), s));
  NACU(cudaMemcpyAsync(d_chain, H.chain, sizeof(int) * nchain, cudaMemcpyHostToDevice, s));
  if (st.nact_table) {
    NACU(cudaMemcpyAsync(d_act, H.act, sizeof(int) * st.nact_table, cudaMemcpyHostToDevice, s));
    NACU(cudaMemcpyAsync(d_actc, H.actc, sizeof(float) * st.nact_table, cudaMemcpyHostToDevice, s));
  }
  NACU(cudaMemcpyAsync(d_roff, H.ref_off, sizeof(int) * (D->n_params + 1), cudaMemcpyHostToDevice, s));
  if (st.nrefs) {
    NACU(cudaMemcpyAsync(d_rprim, H.ref_prim, sizeof(int) * st.nrefs, cudaMemcpyHostToDevice, s));
    NACU(cudaMemcpyAsync(d_rqa, H.ref_qa, sizeof(int) * st.nrefs, cudaMemcpyHostToDevice, s));
    NACU(cudaMemcpyAsync(d_rcoef, H.ref_coeff, sizeof(double) * st.nrefs, cudaMemcpyHostToDevice, s));
  }
  NACU(cudaMemcpyAsync(d_prims, H.prims, sizeof(PrimRec) * D->n_prims, cudaMemcpyHostToDevice, s));
  if (st.auxd_n)
    NACU(cudaMemcpyAsync(d_auxd, H.auxd, sizeof(double) * st.auxd_n, cudaMemcpyHostToDevice, s));
  if (st.auxf_n)
    NACU(cudaMemcpyAsync(d_auxf, H.auxf, sizeof(float) * st.auxf_n, cudaMemcpyHostToDevice, s));
  Job& J = H.job;
  J = Job{};
  J.g = g;
  J.chain = d_chain;
  J.prims = d_prims;
  J.act = d_act;
  J.actc = d_actc;
  J.auxf = d_auxf;
  J.auxd = d_auxd;
  J.ref_off = d_roff;
  J.ref_prim = d_rprim;
  J.ref_qa = d_rqa;
  J.ref_coeff = d_rcoef;
  J.progs = d_progs;
  J.tclass = d_tcls;
  J.list = d_list;
  J.counters = d_cnt;
  J.counters_next = d_cnt + 4;
  J.counters_last = d_cnt + 8;
  J.partial = d_part;
  J.partial_n = (long long)part;
  J.err = d_err;
  J.grad = d_grad;
  J.nparam = D->n_params;
  J.do_bin = 1;
  J.do_grad = 1;
  for (int c = 0; c < D->grid.ncomp; ++c) {
    J.va.ef[c] = reinterpret_cast<const float2*>(d_efwd[c]);
    J.va.ea[c] = reinterpret_cast<const float2*>(d_eadj[c]);
    J.va.w[c] = make_float2(w[2 * c], w[2 * c + 1]);
  }
  NACU(cudaMemcpyAsync(d_job, &J, sizeof(Job), cudaMemcpyHostToDevice, s));
  JobTotals t{};
  t.njobs = 1;
  t.tiles_padded = ((g.T + 127) / 128) * 128;
  t.bin_blocks = t.tiles_padded / 128;
  t.params = D->n_params;
  t.work = d_cnt + 12;
  t.polar = g.polar;
  t.xform = g.xform;
  t.max_cells = 1 << (g.lx + g.ly + g.lz);
  NACU(launch_bin(d_job, t, d_err, s));
  NACU(launch_vjp(d_job, t, d_err, sms, d_gtape, sms, s));
  NACU(launch_finalize(d_job, t, s));
  // ---- wait and report device-side checks ----
  int herr = 0;
  NACU(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  NACU(cudaStreamSynchronize(s));
  if (herr)
    return na_fail(ADG_EDEVICE, "device check failed (bits 0x%x); use a smaller tile shape", herr);
  return ADG_OK;
}
