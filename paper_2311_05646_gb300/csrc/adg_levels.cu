// adg_levels.cu -- sm_103a kernels of the union over non-binary material
// levels (App. B, Alg. 1).  K sets of shapes, set k with material level eps^k
// above the background (0 < eps^1 <= ... <= eps^K); s^k is set k's fill, the
// output of that set's own build.  Per sample:
//
//   k_levels<VEC, false>  s <- s^1; s <- union(r_k s, s^k) for k = 2..K with
//                         r_k = eps^{k-1} / eps^k; eps = eps_bg + eps^K s.
//                         Reads K fills, writes eps.
//   k_levels<VEC, true>   the same forward, then its reverse from the seed
//                         eps^K Re(w E_adj E): one real cotangent per set,
//                         which that set's VJP (the real-cotangent sweep)
//                         maps to the parameters.  Reads K fills and the two
//                         fields, writes K cotangents.
//
// union is the sets' logic family: Eq. union (min{1, a + b}, derivative
// passed through at a + b = 1 inclusive) or App. B.2's product form
// a + b - a b.  Both are HBM streams: each thread takes VEC consecutive
// samples of one component (VEC = 4, 16-byte loads, when the component plane
// is a multiple of 4 and every pointer is 16-byte aligned), in a grid-stride
// loop over at most 8 blocks of 256 threads per SM.
#include <cuda_runtime.h>
#include <stdint.h>

#include "adg_internal.h"

namespace adg {
namespace {

template <int VEC>
__device__ __forceinline__ void load_vec(const float* p, float* v) {
  if constexpr (VEC == 4) {
    const float4 t = __ldcs(reinterpret_cast<const float4*>(p));
    v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
  } else {
    v[0] = __ldcs(p);
  }
}

template <int VEC>
__device__ __forceinline__ void store_vec(float* p, const float* v) {
  if constexpr (VEC == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    p[0] = v[0];
  }
}

// Re(w E_adj E_fwd) for VEC consecutive samples of one component
template <int VEC>
__device__ __forceinline__ void seed_vec(const float2* ef, const float2* ea, float2 w, float* g) {
  float2 f[VEC], e[VEC];
  if constexpr (VEC == 4) {
    const float4 f0 = __ldcs(reinterpret_cast<const float4*>(ef));
    const float4 f1 = __ldcs(reinterpret_cast<const float4*>(ef) + 1);
    const float4 e0 = __ldcs(reinterpret_cast<const float4*>(ea));
    const float4 e1 = __ldcs(reinterpret_cast<const float4*>(ea) + 1);
    f[0] = make_float2(f0.x, f0.y), f[1] = make_float2(f0.z, f0.w);
    f[2] = make_float2(f1.x, f1.y), f[3] = make_float2(f1.z, f1.w);
    e[0] = make_float2(e0.x, e0.y), e[1] = make_float2(e0.z, e0.w);
    e[2] = make_float2(e1.x, e1.y), e[3] = make_float2(e1.z, e1.w);
  } else {
    f[0] = __ldcs(ef);
    e[0] = __ldcs(ea);
  }
#pragma unroll
  for (int v = 0; v < VEC; ++v) {
    const float pr = f[v].x * e[v].x - f[v].y * e[v].y, pi = f[v].x * e[v].y + f[v].y * e[v].x;
    g[v] = w.x * pr - w.y * pi;
  }
}

template <int VEC, bool COT>
__global__ void __launch_bounds__(256) k_levels(LevelArgs a) {
  const long long nq = a.plane / VEC;  // thread items per component
  const long long total = nq * a.C;
  const bool clamp = a.logic == kLogicClamp;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const long long i = q * VEC;  // first sample (component-major, as the fills)
    float S[kMaxLevels][VEC], A[kMaxLevels][VEC], s[VEC];
#pragma unroll
    for (int k = 0; k < kMaxLevels; ++k)
      if (k < a.K) load_vec<VEC>(a.fill + k * a.stride + i, S[k]);
#pragma unroll
    for (int v = 0; v < VEC; ++v) s[v] = S[0][v];
#pragma unroll
    for (int k = 1; k < kMaxLevels; ++k) {
      if (k < a.K) {
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          const float x = a.r[k] * s[v], y = S[k][v];
          A[k][v] = x;
          s[v] = clamp ? fminf(1.0f, x + y) : x + y - x * y;
        }
      }
    }
    if constexpr (!COT) {
      float e[VEC];
#pragma unroll
      for (int v = 0; v < VEC; ++v) e[v] = a.eps_bg + a.lv_top * s[v];
      store_vec<VEC>(a.out + i, e);
    } else {
      const int c = (int)(q / nq);
      const long long o = i - (long long)c * a.plane;
      float sb[VEC];
      seed_vec<VEC>(a.ef[c] + o, a.ea[c] + o, a.w[c], sb);
#pragma unroll
      for (int v = 0; v < VEC; ++v) sb[v] *= a.lv_top;
#pragma unroll
      for (int k = kMaxLevels - 1; k >= 1; --k) {
        if (k < a.K) {
          float ck[VEC];
#pragma unroll
          for (int v = 0; v < VEC; ++v) {
            const float x = A[k][v], y = S[k][v];
            const float pass = (x + y <= 1.0f) ? 1.0f : 0.0f;
            const float dx = clamp ? pass : 1.0f - y, dy = clamp ? pass : 1.0f - x;
            ck[v] = sb[v] * dy;
            sb[v] = sb[v] * dx * a.r[k];
          }
          store_vec<VEC>(a.out + k * a.stride + i, ck);
        }
      }
      store_vec<VEC>(a.out + i, sb);
    }
  }
}

bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace

cudaError_t launch_levels(const LevelArgs& a, bool cot, int sms, cudaStream_t s) {
  if (a.plane <= 0 || a.C <= 0) return cudaSuccess;
  bool vec = (a.plane & 3) == 0 && (a.stride & 3) == 0 && al16(a.fill) && al16(a.out);
  if (cot)
    for (int c = 0; c < a.C; ++c) vec = vec && al16(a.ef[c]) && al16(a.ea[c]);
  const long long items = (vec ? a.plane / 4 : a.plane) * a.C;
  const long long want = (items + 255) / 256;
  const int grid = (int)(want < (long long)sms * 8 ? want : (long long)sms * 8);
  if (vec)
    cot ? k_levels<4, true><<<grid, 256, 0, s>>>(a) : k_levels<4, false><<<grid, 256, 0, s>>>(a);
  else
    cot ? k_levels<1, true><<<grid, 256, 0, s>>>(a) : k_levels<1, false><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace adg
