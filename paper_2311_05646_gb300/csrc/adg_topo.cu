// adg_topo.cu -- sm_103a kernels of the bi-level topology special case
// (Sec. 3.1): every pixel of a 2D design region is its own parameter,
// broadcast along z over the region's cells (the matrix B of Eq. TO_example).
//
//   k_topo_eps   eps = eps_l + deps sigma(v) at every sample of the region
//                (Eq. TO_example; sigma the logistic sigmoid), one thread
//                per pixel writing all of the pixel's samples.
//   k_topo_grad  g_p = deps sigma(v_p) (1 - sigma(v_p)) sum over the
//                components and the region's z cells of Re(w E_adj E)
//                (Eq. top_AD; B^T is that sum).  One thread per pixel, the
//                threads of a warp on consecutive x, so every field load of a
//                warp is 256 contiguous bytes; the sum runs through the
//                components and z in order (compensated fp32), so g is
//                reproducible bit for bit.
// Both are HBM-bound streams.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "adg_internal.h"

namespace adg {
namespace {

__device__ __forceinline__ float logistic(float v) { return 1.f / (1.f + expf(-v)); }

__device__ __forceinline__ void neumaier_add(float& s, float& c, float v) {
  const float t = s + v;
  if (fabsf(s) >= fabsf(v)) c += (s - t) + v;
  else c += (v - t) + s;
  s = t;
}

// One thread per pixel: sigma once, then the pixel's value into every
// (component, z) slab of the region (the warp's stores of a slab are
// contiguous along x).
__global__ void __launch_bounds__(256) k_topo_eps(TopoArgs a) {
  const int npix = a.rx * a.ry;
  const long long plane = (long long)a.nx * a.ny * a.nz;
  const long long slab = (long long)a.nx * a.ny;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) {
    const int px = p % a.rx, py = p / a.rx;
    const float e = a.eps_l + a.deps * logistic(__ldg(a.v + p));
    float* __restrict__ out = a.eps + ((long long)a.z0 * a.ny + (a.y0 + py)) * a.nx + (a.x0 + px);
    for (int c = 0; c < a.C; ++c)
#pragma unroll 4
      for (int k = 0; k < a.z1 - a.z0; ++k) __stcs(out + c * plane + k * slab, e);
  }
}

__global__ void __launch_bounds__(256) k_topo_grad(TopoArgs a) {
  const int npix = a.rx * a.ry;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) {
    const int px = p % a.rx, py = p / a.rx;
    const long long base = (long long)(a.y0 + py) * a.nx + (a.x0 + px);
    float s = 0.f, cmp = 0.f;
    for (int c = 0; c < a.C; ++c) {
      const float2* __restrict__ ef = a.ef[c];
      const float2* __restrict__ ea = a.ea[c];
      const float wr = a.w[c].x, wi = a.w[c].y;
      int k = a.z0;
      for (; k + 8 <= a.z1; k += 8) {  // eight cells' loads in flight, summed in order
        float2 f[8], e[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const long long o = (long long)(k + u) * a.nx * a.ny + base;
          f[u] = __ldcs(ef + o);
          e[u] = __ldcs(ea + o);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float pr = f[u].x * e[u].x - f[u].y * e[u].y, pi = f[u].x * e[u].y + f[u].y * e[u].x;
          neumaier_add(s, cmp, wr * pr - wi * pi);
        }
      }
      for (; k < a.z1; ++k) {
        const long long o = (long long)k * a.nx * a.ny + base;
        const float2 f = __ldcs(ef + o), e = __ldcs(ea + o);
        const float pr = f.x * e.x - f.y * e.y, pi = f.x * e.y + f.y * e.x;
        neumaier_add(s, cmp, wr * pr - wi * pi);
      }
    }
    const float sg = logistic(__ldg(a.v + p));
    a.grad[p] = a.deps * sg * (1.f - sg) * (s + cmp);
  }
}

}  // namespace

cudaError_t launch_topo_eps(const TopoArgs& a, int sms, cudaStream_t s) {
  const int npix = a.rx * a.ry;
  if (npix <= 0) return cudaSuccess;
  const int want = (npix + 255) / 256;
  const int grid = want < sms * 16 ? want : sms * 16;
  k_topo_eps<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_topo_grad(const TopoArgs& a, int sms, cudaStream_t s) {
  const int npix = a.rx * a.ry;
  if (npix <= 0) return cudaSuccess;
  const int want = (npix + 255) / 256;
  const int grid = want < sms * 16 ? want : sms * 16;
  k_topo_grad<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace adg
