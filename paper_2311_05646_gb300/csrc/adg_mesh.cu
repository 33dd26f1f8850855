// adg_mesh.cu -- sm_103a kernels of the exact polygon mesher (Prop. 2's
// standard, exact shape representation: the volume-averaged material of a
// layer of polygons on the Yee grid) and of the finite-difference gradient
// that re-meshes the layer per parameter perturbation (Sec. 6.3's FD
// baseline).
//
//   k_mesh_fill  one thread per (component, y, x) column of a region: the
//                exact area of every polygon inside the sample's averaging
//                cell, summed and clamped to 1, times the exact z overlap of
//                the layer, written down the column.  FP64 throughout.
//                blockIdx.y picks the job (one layer over one region).
//   The FD gradient runs every parameter at once, in three launches:
//   k_mesh_fill over 2n jobs (the region of parameter k meshed at p + h e_k
//   and at p - h e_k into its own scratch), k_mesh_dot over every region's
//   chunks of kMeshChunk samples (Re(w E_adj E) (a - b), an FP64 fixed-order
//   tree per chunk), and k_mesh_final (one block per parameter: its chunks
//   in order, times deps / 2h).
//
// The area of polygon P inside the cell R = [x0, x1] x [y0, y1] comes from
// Green's theorem: the boundary integral of F dx with F(x, y) =
// (clamp(y, y0, y1) - y0) for x in [x0, x1] (0 outside) is minus the area of
// P n R for a counter-clockwise P.  Each edge contributes the integral of F
// along it: its x range clipped to [x0, x1], and clamp(y) integrated exactly
// by splitting the clipped edge where y crosses y0 and y1 (on each piece the
// clamp is linear, so its mean is its midpoint value).  No clipping buffers:
// every edge is one closed-form term.
#include <cuda_runtime.h>
#include <stdint.h>

#include "adg_internal.h"

namespace adg {
namespace {

__device__ __forceinline__ double clampd(double v, double lo, double hi) {
  return fmin(fmax(v, lo), hi);
}

// integral over the edge (xa, ya) -> (xb, yb) of (clamp(y, y0, y1) - y0) dx,
// x restricted to [x0, x1] (signed by the edge's x direction)
__device__ __forceinline__ double edge_term(double xa, double ya, double xb, double yb,
                                            double x0, double x1, double y0, double y1) {
  if (xa == xb) return 0.0;
  const bool fwd = xb > xa;
  const double lx = fmax(fwd ? xa : xb, x0), hx = fmin(fwd ? xb : xa, x1);
  if (!(hx > lx)) return 0.0;
  const double sl = (yb - ya) / (xb - xa);
  const double a = ya + sl * (lx - xa), b = ya + sl * (hx - xa);
  double mean;
  if (a == b) {
    mean = clampd(a, y0, y1) - y0;
  } else {
    const double inv = 1.0 / (b - a);
    double f1 = clampd((y0 - a) * inv, 0.0, 1.0), f2 = clampd((y1 - a) * inv, 0.0, 1.0);
    if (f1 > f2) {
      const double t = f1;
      f1 = f2;
      f2 = t;
    }
    const double d = b - a;
    mean = f1 * (clampd(a + d * (0.5 * f1), y0, y1) - y0) +
           (f2 - f1) * (clampd(a + d * (0.5 * (f1 + f2)), y0, y1) - y0) +
           (1.0 - f2) * (clampd(a + d * (0.5 * (f2 + 1.0)), y0, y1) - y0);
  }
  const double len = (hx - lx) * mean;
  return fwd ? len : -len;
}

__global__ void __launch_bounds__(256) k_mesh_fill(const MeshJob* __restrict__ jobs, int njobs,
                                                   MeshGridDev g) {
  for (int jb = blockIdx.y; jb < njobs; jb += gridDim.y) {
    const MeshJob J = jobs[jb];
    const MeshLayerDev L = J.L;
    const long long cols = (long long)J.rx * J.ry * g.C;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < cols;
         t += (long long)gridDim.x * blockDim.x) {
      const int li = (int)(t % J.rx);
      const int lj = (int)((t / J.rx) % J.ry);
      const int c = (int)(t / ((long long)J.rx * J.ry));
      const double cx0 = (double)(J.x0 + li) + g.off[c][0] - 0.5, cx1 = cx0 + 1.0;
      const double cy0 = (double)(J.y0 + lj) + g.off[c][1] - 0.5, cy1 = cy0 + 1.0;
      double A = 0.0;
      for (int p = 0; p < L.npolys; ++p) {
        const MeshPoly P = L.polys[p];
        if (P.bx1 <= cx0 || P.bx0 >= cx1 || P.by1 <= cy0 || P.by0 >= cy1) continue;
        const double2* V = L.verts + P.v0;
        double s = 0.0;
        double2 u = V[P.nv - 1];
        for (int e = 0; e < P.nv; ++e) {
          const double2 v = V[e];
          s += edge_term(u.x, u.y, v.x, v.y, cx0, cx1, cy0, cy1);
          u = v;
        }
        A += P.sgn * s;
      }
      A = clampd(A, 0.0, 1.0);
      float* col = J.out + (long long)c * J.s_c + (long long)lj * J.s_j + li;
      for (int lk = 0; lk < J.rz; ++lk) {
        double zf = 1.0;
        if (L.bound_z) {
          const double cz0 = (double)(J.z0 + lk) + g.off[c][2] - 0.5;
          zf = fmax(0.0, fmin(cz0 + 1.0, L.zl1) - fmax(cz0, L.zl0));
        }
        col[(long long)lk * J.s_k] = (float)(A * zf);
      }
    }
  }
}

// One block per chunk: the chunk's samples of its parameter's region.
__global__ void __launch_bounds__(256) k_mesh_dot(const MeshDotJob* __restrict__ jobs,
                                                  const int2* __restrict__ chunks, int nchunks,
                                                  MeshDotFields f, double* __restrict__ part) {
  __shared__ double ws[256];
  for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const int2 cj = chunks[ch];  // (job, first sample)
    const MeshDotJob J = jobs[cj.x];
    const int q1 = min(cj.y + kMeshChunk, J.n);
    double acc = 0.0;
    for (int q = cj.y + threadIdx.x; q < q1; q += blockDim.x) {
      const int li = q % J.rx;
      const int r1 = q / J.rx;
      const int lj = r1 % J.ry;
      const int r2 = r1 / J.ry;
      const int lk = r2 % J.rz;
      const int c = r2 / J.rz;
      const long long gi = ((long long)(J.z0 + lk) * f.ny + (J.y0 + lj)) * f.nx + (J.x0 + li);
      const float2 a = f.ef[c][gi], e = f.ea[c][gi];
      const float pr = a.x * e.x - a.y * e.y, pi = a.x * e.y + a.y * e.x;
      const float z = f.w[c].x * pr - f.w[c].y * pi;
      acc += (double)z * ((double)J.a[q] - (double)J.b[q]);
    }
    ws[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) ws[threadIdx.x] += ws[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[ch] = ws[0];
    __syncthreads();
  }
}

// One block per parameter: its chunks' partials in chunk order, scaled.
__global__ void __launch_bounds__(128) k_mesh_final(const MeshDotJob* __restrict__ jobs, int njobs,
                                                    const double* __restrict__ part, double scale,
                                                    float* __restrict__ grad) {
  __shared__ double ws[128];
  for (int k = blockIdx.x; k < njobs; k += gridDim.x) {
    const MeshDotJob J = jobs[k];
    double acc = 0.0;
    for (int i = J.chunk0 + threadIdx.x; i < J.chunk1; i += blockDim.x) acc += part[i];
    ws[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) ws[threadIdx.x] += ws[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) grad[J.param] = (float)(scale * ws[0]);
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_mesh_fill(const MeshJob* jobs, int njobs, long long max_cols,
                             const MeshGridDev& g, int sms, cudaStream_t s) {
  if (njobs <= 0 || max_cols <= 0) return cudaSuccess;
  const long long want = (max_cols + 255) / 256;
  const int gx = (int)(want < (long long)sms * 8 ? want : (long long)sms * 8);
  const int gy = njobs < 65535 ? njobs : 65535;
  k_mesh_fill<<<dim3(gx, gy), 256, 0, s>>>(jobs, njobs, g);
  return cudaGetLastError();
}

cudaError_t launch_mesh_dot(const MeshDotJob* jobs, int njobs, const int2* chunks, int nchunks,
                            const MeshDotFields& f, double* part, double scale, float* grad,
                            int sms, cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  if (nchunks > 0) {
    const int gd = nchunks < sms * 16 ? nchunks : sms * 16;
    k_mesh_dot<<<gd, 256, 0, s>>>(jobs, chunks, nchunks, f, part);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int gf = njobs < sms * 8 ? njobs : sms * 8;
  k_mesh_final<<<gf, 128, 0, s>>>(jobs, njobs, part, scale, grad);
  return cudaGetLastError();
}

}  // namespace adg
