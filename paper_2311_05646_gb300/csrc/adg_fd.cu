// adg_fd.cu -- sm_103a kernels of the finite-difference gradient baseline
// (Sec. 3: the per-parameter finite differences of the material map that
// the paper's AutoDiff replaces).  With the library's own build as the
// mesher, dL/dp_k = deps sum_c sum_samples z (fill(p + h e_k) -
// fill(p - h e_k)) / 2h, z = Re(w E_adj E) (Eq. 1, eps term):
//
//   k_fd_seed   z_c = Re(w_c E_adj,c E_fwd,c) at every sample, once.
//   k_fd_dot    sum z (a - b) over every sample: one block per chunk of
//               kFdChunk samples (16-byte loads), a fixed-order tree in the
//               block, FP64 chunk partials; k_fd_final adds them in chunk
//               order, so the result is reproducible bit for bit.
// All three are HBM streams.  k_add (b += a, for the two terms of Eq. 1) is
// kept here with the other small helpers.
#include <cuda_runtime.h>
#include <stdint.h>

#include "adg_internal.h"

namespace adg {
namespace {

__global__ void __launch_bounds__(256) k_fd_seed(FdSeedArgs a) {
  const long long n = a.plane;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n * a.C;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / n);
    const long long s = i - (long long)c * n;
    const float2 f = __ldcs(a.ef[c] + s), e = __ldcs(a.ea[c] + s);
    const float pr = f.x * e.x - f.y * e.y, pi = f.x * e.y + f.y * e.x;
    a.z[i] = a.w[c].x * pr - a.w[c].y * pi;
  }
}

__global__ void __launch_bounds__(256) k_fd_dot(const float* __restrict__ z,
                                                const float* __restrict__ pa,
                                                const float* __restrict__ pb, long long n,
                                                bool vec, double* __restrict__ part) {
  __shared__ double ws[8];
  const long long c0 = (long long)blockIdx.x * kFdChunk;
  const long long c1 = c0 + kFdChunk < n ? c0 + kFdChunk : n;
  float s = 0.f;
  if (vec) {  // 16-byte loads (n a multiple of 4, arrays 16-byte aligned)
    const float4* z4 = reinterpret_cast<const float4*>(z);
    const float4* a4 = reinterpret_cast<const float4*>(pa);
    const float4* b4 = reinterpret_cast<const float4*>(pb);
#pragma unroll 4
    for (long long q = c0 / 4 + threadIdx.x; q < c1 / 4; q += blockDim.x) {
      const float4 zz = __ldcs(z4 + q), aa = __ldcs(a4 + q), bb = __ldcs(b4 + q);
      s += zz.x * (aa.x - bb.x) + zz.y * (aa.y - bb.y) + zz.z * (aa.z - bb.z) + zz.w * (aa.w - bb.w);
    }
  } else {
    for (long long q = c0 + threadIdx.x; q < c1; q += blockDim.x) s += z[q] * (pa[q] - pb[q]);
  }
  double d = s;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += ws[k];
    part[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(256) k_fd_final(const double* __restrict__ part, int nchunks,
                                                  double* __restrict__ out) {
  __shared__ double ws[8];
  double d = 0.0;
  for (int k = threadIdx.x; k < nchunks; k += blockDim.x) d += part[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += ws[k];
    *out = t;
  }
}

__global__ void k_fd_scale(const double* __restrict__ acc, int n, double scale,
                           float* __restrict__ grad) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) grad[k] = (float)(scale * acc[k]);
}

}  // namespace

__global__ void k_add(const float* __restrict__ a, float* __restrict__ b, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) b[k] += a[k];
}

cudaError_t launch_add(const float* a, float* b, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_add<<<(n + 255) / 256, 256, 0, s>>>(a, b, n);
  return cudaGetLastError();
}

cudaError_t launch_fd_scale(const double* acc, int n, double scale, float* grad, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_fd_scale<<<(n + 255) / 256, 256, 0, s>>>(acc, n, scale, grad);
  return cudaGetLastError();
}

cudaError_t launch_fd_seed(const FdSeedArgs& a, int sms, cudaStream_t s) {
  const long long total = a.plane * a.C;
  if (total <= 0) return cudaSuccess;
  const long long want = (total + 255) / 256;
  const int grid = (int)(want < (long long)sms * 8 ? want : (long long)sms * 8);
  k_fd_seed<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

int fd_chunks(long long n) { return (int)((n + kFdChunk - 1) / kFdChunk); }

cudaError_t launch_fd_dot(const float* z, const float* a, const float* b, long long n,
                          double* part, double* out, cudaStream_t s) {
  const int nch = fd_chunks(n);
  if (nch <= 0) return cudaMemsetAsync(out, 0, sizeof(double), s);
  const bool vec = (n & 3) == 0 &&
                   ((reinterpret_cast<uintptr_t>(z) | reinterpret_cast<uintptr_t>(a) |
                     reinterpret_cast<uintptr_t>(b)) & 15) == 0;
  k_fd_dot<<<nch, 256, 0, s>>>(z, a, b, n, vec, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_fd_final<<<1, 256, 0, s>>>(part, nch, out);
  return cudaGetLastError();
}

}  // namespace adg
