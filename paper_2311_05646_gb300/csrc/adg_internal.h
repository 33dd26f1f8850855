// adg_internal.h -- device records and launch interfaces shared by the host
// side (adg_api.cu) and the kernels (adg_kernels.cu) of libadg.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace adg {

// Per-tile capacities of the binned kernels.  A tile that would exceed one of
// them is reported through the device error word (never written out of range).
constexpr int kMaxLeaves = 64;  // primitives whose edge band crosses the tile
constexpr int kMaxOps = 120;    // folded logic program length (7-bit operand fields)
constexpr int kSmemOps = 16;    // VJP tape entries kept in shared memory; longer
                                // programs use a per-block slice of a global tape
constexpr int kMaxDepth = 32;   // fold stack depth (checked at design creation)
constexpr int kMaxSlots = 384;  // (primitive, active scalar) accumulators
constexpr int kMaxPairs = 6;    // d s / d q terms one cell yields per leaf (box, graph 6; circle 5)
constexpr int kBlock = 128;     // threads per CTA of the build / VJP kernels
constexpr int kMaxTileCells = 2048;  // cells per tile (per component)
constexpr int kWarps = kBlock / 32;
constexpr int kMaxPolyVerts = 256;  // vertices of one convex polygon
// Polygon edge table (fp32, kPolyEdgeFloats per edge): the edge's start vertex
// relative to the polygon's integer anchor cell (PrimRec ai[0], ai[1]) as
// (hi, lo) pairs, the unit inward normal as (hi, lo) pairs, the edge vector
// and its inverse length (cells).
constexpr int kPolyEdgeFloats = 11;
static_assert(kMaxOps < 127 && kMaxLeaves < 127, "op operands are 7-bit fields, 127 = constant 1");
// Per-tile pools of the band kernels (floats): staged leaves (PrimRec) and
// their table descriptors (80 B each), the VJP's per-warp accumulator rows,
// then factor tables in what is left (at least kPoolSpare floats).
constexpr int kBuildPool = 4096;
constexpr int kVjpPool = 7040;
constexpr int kPoolSpare = 192;
constexpr int kLeafTabBytes = 80;
constexpr size_t kTapeBlockFloats = (size_t)kMaxOps * kBlock;  // global tape per VJP block

enum : int32_t { kBox = 0, kCircle = 1, kPolygon = 2, kGraph = 3, kPolar = 4,
                 kXform = 5 /* a box (sigma form), circle, polygon or polar shape under a
                               rotation / aspect transform; base kind in flags bits 8..11 */ };
constexpr int kMaxPolarHarm = 32;  // Fourier harmonics of one Polar2D boundary
enum : int32_t { kLinear = 0, kSigmoid = 1, kQuadratic = 2, kSin = 3, kErf = 4 };
enum : int32_t { kBoundX = 1, kBoundY = 2, kBoundZ = 4, kRectSigma = 8, kGraphAbove = 16,
                 kPolyRigid = 32 /* every vertex x (y) is the same scalar of one parameter */,
                 kXformFlag = 64 /* ADG_XFORM: the last five scalars are px, py, theta, sx, sy */ };
// FP64 record of a transformed primitive in auxd: cos theta, sin theta, 1/sx,
// 1/sy, sx, sy, the pivot's fractional cell parts (x, y), then the base
// geometry in cells relative to the pivot (local frame): box x0, x1, y0, y1
// and z0, z1 (grid cells); circle cx, cy, R; polar cx, cy, R0, c_1, s_1, ...;
// polygon the winding sign, then x_1, y_1, ...
constexpr int kXformHead = 8;
// chained (binary) design program, one int32 word per op: (code << 24) | arg
enum : int32_t { cPush = 0, cUnion = 1, cInter = 2, cDiff = 3 };
// folded per-tile program, one uint16 per op: code | a << 2 | b << 9 (code 2
// bits, operands 7 bits); the complement of b is stored as difference(kOne, b)
enum : int32_t { fPush = 0, fUnion = 1, fInter = 2, fDiff = 3, fCompl = 4 };
constexpr int kOne = 127;
// device error bits
enum : int32_t {
  eLeafOverflow = 1,
  eOpsOverflow = 2,
  eDepthOverflow = 4,
  eSlotOverflow = 8,
  ePartialRange = 16,
  eBadProgram = 32,
  ePoolOverflow = 64,
  eDebugBound = 128  // ADG_DEBUG builds: an index failed its bound check (the access was skipped)
};
// ADG_DEBUG builds (compiled with -DADG_DEBUG) check the indices of the
// kernels' main global accesses -- band-tile list entries, tile programs,
// partial sums -- against the ranges their buffers were sized for; a failed
// check records eDebugBound in the error word and the access is skipped.
// Release builds compile the checks away.
#ifdef ADG_DEBUG
#define ADG_CHECK(cond, err) ((cond) ? true : (atomicOr((err), eDebugBound), false))
#else
#define ADG_CHECK(cond, err) true
#endif

struct GridDev {
  int nx, ny, nz, C;
  int lx, ly, lz;  // log2 of the tile shape
  int ntx, nty, ntz, T;
  float off[3][3];  // [component][axis] sample offsets (cells)
  float offmin[3], offmax[3];
  float invd[3];  // 1 / spacing
  float eps_bg, deps;
  int logic;
  int nchain;
  int nprims;
  int polar;  // some primitive is Polar2D (its gradient runs on k_vjp_polar)
  int xform;  // some primitive is transformed (k_build_x and k_vjp_polar)
  int unique_push;  // no primitive is pushed twice by the chain (the binner's
                    // fold then gives each push its own leaf without a search)
};

// One primitive after the parameter map, in cell units of each axis:
// a coordinate q along axis a becomes (q - o_a) / d_a = ai + af with ai an
// integer and af in [0, 1), so that per-cell differences stay exact in fp32.
struct alignas(16) PrimRec {
  int kind, sigma, flags, nact;
  float kr;    // sigma_k(x) = sigma(kr * x / d): kr in per-cell units
  float band;  // transition half-width in cells (beyond it sigma is 0/1, flat)
  int act_off; // act[act_off + local q] = accumulator slot (or -1), actc = its coefficient
  int auxd_off, auxf_off, naux;
  int part_off;  // first partial of this primitive
  int npb;       // tiles in the partial box
  int tb[6];     // tile box of the value support   [x0,x1) [y0,y1) [z0,z1)
  int pb[6];     // tile box of the derivative support (partials)
  int ai[6];     // box: x0,x1,y0,y1,z0,z1; circle: cx, cy in [0],[1]; z0,z1 in [4],[5]
  float af[6];
  float g[4];  // circle: R, R^2 (hi, lo) in cells, [3] = 1 if R < 0; polygon: [0] = winding sign
};

// Floats of a tile's pool taken by nleaf staged leaves with their table
// descriptors, nops op descriptors (16 B) with a list entry each (4 B), and
// nacc accumulators (plus as many compensation terms).
__host__ __device__ constexpr int pool_need(int nleaf, int nacc, int nops) {
  return (nleaf * ((int)sizeof(PrimRec) + kLeafTabBytes) / 4 + 5 * nops + 2 * nacc + 3) & ~3;
}
static_assert(pool_need(kMaxLeaves, 0, 0) + kPoolSpare <= kBuildPool,
              "the build pool holds any tile's leaves");
// the VJP's (slot, value) pair columns of graph and polygon leaves, taken from
// the pool only by tiles that have such leaves
constexpr int kPairFloats = 2 * kMaxPairs * kBlock;

struct TileProg {
  int nops;   // 0: constant tile, value cval
  int nleaf;
  float cval;
  int nslot;
  int pairs;  // a graph or polygon leaf: the VJP reserves pair columns
  int pad[3];
  uint16_t ops[kMaxOps];
  uint16_t leaf[kMaxLeaves];
};

struct VjpArgs {
  const float2* ef[3];
  const float2* ea[3];
  float2 w[3];
  const float* G;  // real-seed mode when non-null
};

// The finite-difference baseline (Sec. 3): z = Re(w E_adj E) once, then
// sum z (a - b) per pair of fills, in kFdChunk-sample chunks summed in order.
constexpr int kFdChunk = 8192;
struct FdSeedArgs {
  const float2* ef[3];
  const float2* ea[3];
  float2 w[3];
  long long plane;  // nx ny nz
  int C;
  float* z;         // [C][plane]
};
cudaError_t launch_fd_seed(const FdSeedArgs& a, int sms, cudaStream_t s);
int fd_chunks(long long n);
cudaError_t launch_fd_scale(const double* acc, int n, double scale, float* grad, cudaStream_t s);
cudaError_t launch_add(const float* a, float* b, int n, cudaStream_t s);  // b += a

// Union over non-binary material levels (App. B, Alg. 1), adg_levels.cu.
constexpr int kMaxLevels = 8;
constexpr int kLogicClamp = 1;  // GridDev::logic of the clamped family (0: product)
struct LevelArgs {
  const float* fill;  // K fill slices, `stride` floats apart, each [C][plane]
  float* out;         // eps [C][plane], or K cotangent slices `stride` apart
  long long stride, plane;
  int C, K, logic;
  float lv_top, eps_bg;   // eps^K, the background
  float r[kMaxLevels];    // r[k] = eps^{k-1} / eps^k for k >= 1
  const float2* ef[3];    // cotangent pass: fields and weights
  const float2* ea[3];
  float2 w[3];
};
cudaError_t launch_levels(const LevelArgs& a, bool cot, int sms, cudaStream_t s);

// Exact polygon mesher and its finite-difference gradient, adg_mesh.cu.
// Coordinates in cell units of the grid: x -> (x - o_x) / dx and so on.
struct MeshPoly {
  double bx0, bx1, by0, by1;  // bounding box
  double sgn;                 // -1 for a counter-clockwise polygon, +1 clockwise
  int v0, nv;                 // vertices [v0, v0 + nv) of the layer's vertex array
};
struct MeshLayerDev {
  const MeshPoly* polys;
  const double2* verts;
  int npolys;
  int bound_z;
  double zl0, zl1;
};
struct MeshGridDev {
  int C;
  double off[3][3];
};
// One mesh of one layer over one region: sample (c, x0 + i, y0 + j, z0 + k)
// goes to out + c s_c + k s_k + j s_j + i.
struct MeshJob {
  MeshLayerDev L;
  float* out;
  int x0, y0, z0, rx, ry, rz;
  long long s_c, s_k, s_j;
};
// One parameter's dot product over its region (compact [C][rz][ry][rx]
// buffers a = fill at p + h e_k, b = at p - h e_k); chunks [chunk0, chunk1).
struct MeshDotJob {
  const float* a;
  const float* b;
  int x0, y0, z0, rx, ry, rz, n;
  int chunk0, chunk1, param;
};
struct MeshDotFields {
  const float2* ef[3];
  const float2* ea[3];
  float2 w[3];
  int nx, ny;
};
constexpr int kMeshChunk = 2048;  // samples per dot-product block
cudaError_t launch_mesh_fill(const MeshJob* jobs, int njobs, long long max_cols,
                             const MeshGridDev& g, int sms, cudaStream_t s);
// part: one double per chunk; grad[param] <- scale * (the job's chunks in order)
cudaError_t launch_mesh_dot(const MeshDotJob* jobs, int njobs, const int2* chunks, int nchunks,
                            const MeshDotFields& f, double* part, double scale, float* grad,
                            int sms, cudaStream_t s);
// part: fd_chunks(n) doubles of scratch; out: one double
cudaError_t launch_fd_dot(const float* z, const float* a, const float* b, long long n,
                          double* part, double* out, cudaStream_t s);

// The topology special case (Sec. 3.1): a region of rx x ry pixels at
// (x0, y0) broadcast along z over [z0, z1), one parameter v per pixel.
struct TopoArgs {
  int nx, ny, nz, C;
  int x0, y0, rx, ry, z0, z1;
  const float* v;     // rx ry, x fastest
  float eps_l, deps;
  float* eps;         // [C][nz][ny][nx] (eps build)
  const float2* ef[3];
  const float2* ea[3];
  float2 w[3];
  float* grad;        // rx ry (gradient)
};
cudaError_t launch_topo_eps(const TopoArgs& a, int sms, cudaStream_t s);
cudaError_t launch_topo_grad(const TopoArgs& a, int sms, cudaStream_t s);

// The dense field stream of adg_grad_dense: every sample's
// z = Re(w E_adj E_fwd) and z * fill, summed per chunk of kDenseChunk
// samples (chunks handed out by an atomic counter, partials stored by chunk
// index, summed in index order by one block).
constexpr int kDenseChunk = 8192;
struct DenseArgs {
  const float2* ef[3];
  const float2* ea[3];
  float2 w[3];
  const float* fill;  // [C][plane]
  long long plane;    // nx ny nz
  int C;
  int chunks_per_c;   // ceil(plane / kDenseChunk)
  int* ctr;           // work counter, zeroed by the launcher
  double2* part;      // C * chunks_per_c partials (sum z, sum z fill)
  double* gmat;       // out: dL/d eps_bg, dL/d eps_fg
};

// One unit of device work: one design with the operations asked of it.  All
// kernels take a table of jobs; a single-design call is a one-job table and a
// batch of designs of uneven size runs through the same launches.
struct Job {
  GridDev g;
  // design tables
  const int* chain;
  const PrimRec* prims;
  const int* act;
  const float* actc;
  const float* auxf;
  const double* auxd;
  const int* ref_off;
  const int* ref_prim;
  const int* ref_qa;
  const double* ref_coeff;
  // bins
  TileProg* progs;
  unsigned char* tclass;  // per tile: 0 / 1 constant fill, 2 band (program) tile
  int* list;
  int* counters;       // [band tiles, longest program, band cells, active samples]
  int* counters_next;  // the other set: zeroed by this binning for the next one
  int* counters_last;  // active samples of the last VJP (moved here by the finalize)
  // outputs and inputs of the operations
  float* fill;
  float* eps;
  VjpArgs va;
  float* partial;
  float* grad;
  long long partial_n;  // partials of the job (zero between calls: the finalize clears them)
  int* err;             // the context's device error word
  int nparam;
  int param_base;  // prefix over the table (finalize)
  int tile_base;   // prefix over the table, multiple of 128 (binner blocks)
  int row_base;    // prefix over build jobs of kFillRows-row groups (streaming fill)
  int do_bin, do_build, do_grad;
};

constexpr int kFillRows = 4;  // x-rows per work unit of the streaming fill (a shorter tail
                              // than 8; 2 costs more in fetches than it saves)

struct JobTotals {
  int njobs;
  int fill_blocks;       // fill work units: sum over build jobs of ceil(C nz ny / kFillRows)
  int bin_blocks;        // sum over binned jobs of ceil(T / 128)
  int tiles_padded;      // tile_base of one past the last job
  int params;            // sum of nparam over gradient jobs
  // Work counters of the persistent kernels, 6 ints: VJP next tile, VJP blocks
  // done, build next band tile, build blocks done with band tiles, build next
  // fill unit, build blocks done with fill units.  Zero between launches: the
  // last block of a launch resets each pair.  One launch at a time per array.
  int* work;
  int fill_warps;  // build: warps per block streaming constant tiles (1 .. kMaxFillWarps)
  int polar;       // some job's design has Polar2D primitives: the VJP is k_vjp_polar
  int xform;       // some job's design has transformed primitives: k_build_x, k_vjp_polar
  int pdl;         // launch the build, VJP and finalize with programmatic dependent launch
  int max_cells;   // largest tile (cells) of the table's jobs: sizes the VJP's sample list
};

constexpr int kMaxJobs = 1024;  // jobs in one table (one batch)
constexpr int kMaxFillWarps = 2;

cudaError_t launch_bin(const Job* jobs, const JobTotals& t, int* err, cudaStream_t s);
cudaError_t launch_build(const Job* jobs, const JobTotals& t, int sms, cudaStream_t s);
// gtape: kTapeBlockFloats floats per block for gtape_blocks blocks; the grid
// never exceeds gtape_blocks.
cudaError_t launch_vjp(const Job* jobs, const JobTotals& t, int* err, int sms, float* gtape,
                       int gtape_blocks, cudaStream_t s);
cudaError_t launch_finalize(const Job* jobs, const JobTotals& t, cudaStream_t s);
// the dense field stream (zero the counter, stream, fixed-order sum) on `s`
cudaError_t launch_dense(const DenseArgs& a, int sms, cudaStream_t s);
// Shared-memory limits of the kernels; call once per device before any capture.
cudaError_t init_kernel_attributes();
int build_blocks_per_sm(int njobs, int fill_warps, bool xform);
int vjp_blocks_per_sm(int njobs, bool polar, int cells);
void set_last_error(const char* msg);  // the thread-local text of adg_last_error()

}  // namespace adg
