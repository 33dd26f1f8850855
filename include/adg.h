/*
 * adg.h -- C ABI of libadg: a GB300 (sm_103a) implementation of the
 * differentiable shape-to-material map ("AutoDiffGeo") and of the adjoint
 * gradient sum reduction of arXiv 2311.05646 (Hooten et al.).
 *
 * The paper's problem statement (Sec. 2, the 7-step adjoint protocol): given
 * shape parameters v (here `params`), compute the material distribution eps(v)
 * (step 2) and, with the forward and adjoint fields treated as given
 * quantities, the gradient of Eq. 1 (step 5).  libadg implements exactly those
 * two steps; the simulators are outside its scope (Sec. 2, last paragraph).
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are DEVICE pointers owned by the caller; the library
 *     never frees or retains them beyond the call's stream work.  Pointers
 *     named h_* and every array inside adg_design_desc are HOST pointers; the
 *     library copies what it needs before returning.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     All device work of a call is enqueued on it and is asynchronous.
 *   - Every call returns adg_status; nothing throws or aborts across the ABI.
 *     adg_last_error() returns a thread-local message for the last failure.
 *   - Arguments are validated before any launch (ADG_EINVAL).  Device-side
 *     checks (tile capacity) set an error word that adg_sync() reports as
 *     ADG_EDEVICE; no kernel traps or faults on bad data.  Per tile, at most
 *     64 primitives may have an edge band crossing it, its folded logic
 *     program at most 120 ops (fold stack depth 32), with at most 384
 *     (primitive, parameter) accumulators, and its staged primitives plus
 *     accumulators must fit the VJP's 27.5 KB tile pool (7040 floats); a
 *     smaller tile shape lowers all of these.
 *   - Layout of every per-cell array: [ncomp][nz][ny][nx], x fastest, fp32
 *     (fields: complex64 = interleaved (re, im) fp32 pairs).
 */
#ifndef ADG_H
#define ADG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ADG_OK = 0,
  ADG_EINVAL = 1,   /* invalid argument or design description            */
  ADG_ENOMEM = 2,   /* device or host allocation failed                  */
  ADG_ECUDA = 3,    /* a CUDA runtime call failed                        */
  ADG_ETIMEOUT = 4, /* a bounded wait ran out                            */
  ADG_EBUSY = 5,    /* resource in use (e.g. batch queue full)           */
  ADG_EDEVICE = 6   /* a device-side check tripped (see adg_last_error)  */
} adg_status;

/* ---- design description format ----------------------------------------
 * Primitive kinds (Table "AutoDiffGeo definitions"; geometric scalars q in
 * physical units, listed in the order the primitive reads them):
 *   BOX      Rect1D/2D/dD: q = x0, x1, y0, y1, z0, z1; ADG_BOUND_* flags say
 *            which axes are bounded.  Default: exact overlap of the box with
 *            each cell's averaging window (Sec. 5.1, Eq. linear; zero error vs
 *            volumetric averaging).  ADG_RECT_SIGMA: the paper's product
 *            sigma_k(x - x0) sigma_k(x1 - x) per bounded axis, k = kr / d_axis.
 *   CIRCLE   Circ2D: q = cx, cy, R, z0, z1; s = sigma_k(R - r), k = kr / dx.
 *   POLYGON  Poly2D (convex): q = z0, z1, x1, y1, ..., xN, yN; product over edges
 *            of sigma_k(n . (r - v_e)) with the inward normal whatever the
 *            winding; k = kr / dx.
 *   GRAPH    GeneralCartesian2D: q = z0, z1, X1..XM, Y1..YM; s = sigma_k(f(x) - y)
 *            (or y - f(x) with ADG_GRAPH_ABOVE), f the piecewise-linear
 *            interpolant through (X_j, Y_j), constant beyond the end knots;
 *            k = kr / dy.
 *   POLAR    Polar2D (star-convex) with a Fourier boundary (the PSGC
 *            scatterers' R(theta) = R0 + sum_n c_n cos(n theta) + s_n sin(n theta)):
 *            q = cx, cy, R0, z0, z1, c1, s1, ..., cN, sN (0 <= N <= 32);
 *            s = sigma_k(R(theta) - r), r and theta polar about (cx, cy);
 *            k = kr / dx.  N = 0 is CIRCLE.  With ADG_PRIM_POLAR the derivative
 *            w.r.t. the centre is 0 at r = 0.
 *   CIRCLE/POLYGON/GRAPH/POLAR are extruded along z by the exact overlap of
 *   [z0, z1] when ADG_BOUND_Z is set (planarity, Sec. 5.2).  CIRCLE, POLYGON
 *   and POLAR need dx == dy.
 *   ADG_XFORM (rotation and aspect ratio, Sec. 4 item iii): five more
 *   scalars after the primitive's own, px, py, theta, sx, sy (pivot in
 *   physical units, angle in radians, aspect > 0).  The primitive drawn with
 *   its own scalars is stretched by (sx, sy) along its own axes and rotated
 *   by theta about (px, py): it is evaluated at the local point
 *   u = p + S^-1 R(-theta)(r - p), S = diag(sx, sy), z unchanged, its sigma_k
 *   acting on local distances.  For BOX with ADG_RECT_SIGMA (the paper's
 *   Rect form; the exact overlap is for axis-aligned boxes), CIRCLE (an
 *   ellipse with an aspect), POLYGON and POLAR; not GRAPH; needs dx == dy.
 *   All five scalars may be driven by parameters: the gradient goes through
 *   the spatial gradient of the primitive at u.  Evaluated in FP64 on the
 *   device.
 * Sigma kinds: Table "Nonlinear function definitions", sigma_k(x) = sigma(k x).
 * Logic (Eqs. union/intersection, Appendix B.2):
 *   PRODUCT: union a + b - ab, intersection ab, difference a (1 - b)
 *   CLAMP:   union min{1, a + b}, intersection max{0, a + b - 1},
 *            difference max{0, a - b}
 *   n-ary operations are evaluated as left-to-right chains of binary ones
 *   (the paper's recursive definition of union_2).
 * Program: postfix int32 words (code << 24) | arg; PUSH arg = primitive id,
 *   UNION/INTERSECT arg = operand count (>= 1), DIFF arg ignored (2 operands).
 * Parameter map: q_j = q_base[j] + q_coeff[j] * params[q_param[j]], or
 *   q_base[j] when q_param[j] = -1 (a fixed scalar).
 */
enum { ADG_PRIM_BOX = 0, ADG_PRIM_CIRCLE = 1, ADG_PRIM_POLYGON = 2, ADG_PRIM_GRAPH = 3,
       ADG_PRIM_POLAR = 4 };
enum {
  ADG_SIGMA_LINEAR = 0,
  ADG_SIGMA_SIGMOID = 1,
  ADG_SIGMA_QUADRATIC = 2,
  ADG_SIGMA_SIN = 3,
  ADG_SIGMA_ERF = 4
};
enum { ADG_LOGIC_PRODUCT = 0, ADG_LOGIC_CLAMP = 1 };
enum {
  ADG_BOUND_X = 1,
  ADG_BOUND_Y = 2,
  ADG_BOUND_Z = 4,
  ADG_RECT_SIGMA = 8,
  ADG_GRAPH_ABOVE = 16,
  ADG_XFORM = 64
};
enum { ADG_OP_PUSH = 0, ADG_OP_UNION = 1, ADG_OP_INTERSECT = 2, ADG_OP_DIFF = 3 };

/* Rectilinear grid.  Cell (i, j, k) of component c is sampled at
 * o + ((i + off[c][0]) dx, (j + off[c][1]) dy, (k + off[c][2]) dz); its
 * averaging window is the cell-sized box centred there.  The paper asks for
 * eps at the Yee half-steps of each polarisation (Sec. 3) but does not fix
 * them; the offsets are the caller's. */
typedef struct {
  int32_t nx, ny, nz, ncomp; /* nz = 1 for 2D; ncomp in {1, 2, 3}          */
  double dx, dy, dz;         /* spacing                                     */
  double ox, oy, oz;         /* origin                                      */
  double off[3][3];          /* [component][axis] sample offset in cells    */
} adg_grid;

typedef struct {
  adg_grid grid;
  double eps_bg, eps_fg;     /* eps = eps_bg + (eps_fg - eps_bg) fill (Sec. 5.1) */
  int32_t logic;             /* ADG_LOGIC_*                                 */
  int32_t n_params;
  int32_t n_q;
  int32_t n_prims;
  int32_t n_ops;
  int32_t reserved;          /* must be 0                                   */
  const double *q_base, *q_coeff;
  const int32_t *q_param;
  const int32_t *prim_kind, *prim_sigma, *prim_flags, *prim_q0, *prim_nq;
  const double *prim_kr;
  const int32_t *ops;
} adg_design_desc;

/* Tile shape (cells) of the binned kernels.  tx in {32, 64}, ty in
 * {1, 2, 4, 8, 16}, tz in {1, 2, 4, 8}, 128 <= tx*ty*tz <= 2048.  All zero =
 * library default (32 x 4 x 4).  fill_warps: warps of each build block that
 * stream the constant tiles beside its four band warps, 1 or 2 (0 = 1); a
 * design with much constant area and few band tiles builds faster with 2.
 * Batched builds use 1. */
typedef struct {
  int32_t tx, ty, tz;
  int32_t fill_warps;
} adg_tile_opts;

/* Counters of the last binned call, for measurement (read with a sync). */
typedef struct {
  int64_t tiles;          /* tiles covering the grid                        */
  int64_t program_tiles;  /* tiles where some primitive's edge band lies     */
  int64_t cells;          /* nx * ny * nz                                   */
  int64_t band_cells;     /* cells (per component) inside program tiles     */
  int32_t tile[3];        /* tile shape in use                              */
  int32_t max_ops;        /* longest folded per-tile program                */
  int64_t active_samples; /* samples the last VJP swept (a derivative of a
                             parameter-driven primitive may be nonzero)     */
} adg_stats;

typedef struct adg_ctx adg_ctx;       /* opaque: device, error word         */
typedef struct adg_design adg_design; /* opaque: compiled design, scratch   */

/* Create a context on CUDA device `device` (makes it current on this thread).
 * Out: *out, owned by the caller, released by adg_ctx_destroy. */
adg_status adg_ctx_create(int32_t device, adg_ctx **out);
adg_status adg_ctx_destroy(adg_ctx *ctx);

/* Compile a design: validates the description (primitive table, parameter map,
 * postfix program), converts the program to its chained form and uploads the
 * static tables.  `tiles` may be NULL.  Host arrays are copied. */
adg_status adg_design_create(adg_ctx *ctx, const adg_design_desc *desc,
                             const adg_tile_opts *tiles, adg_design **out);
adg_status adg_design_destroy(adg_ctx *ctx, adg_design *design);

/* Step 2 of the protocol (Sec. 2): v -> eps.  Eq. eps realised as
 * parameter map -> primitives (sigma_k, Table 4) -> logic (Eqs. union,
 * intersection) -> eps = eps_bg + deps * fill (Sec. 5.1).
 * h_params: n_params host doubles.  d_fill (nullable) and d_eps: device fp32
 * [ncomp][nz][ny][nx].  Asynchronous on `stream`. */
adg_status adg_build_eps(adg_ctx *ctx, adg_design *design, const double *h_params,
                         float *d_fill, float *d_eps, void *stream);

/* Step 5 (Eq. 1, eps term): for every parameter k,
 *   g_k = Re sum_c sum_cells w_c * E_adj,c * E_fwd,c * d eps_c / d p_k
 * (no complex conjugate, as in Eq. 1; w_c = -2 i omega gives 2 omega Im(.)).
 * Computed as the vector-Jacobian product of Eqs. AD/jaceps: the material
 * Jacobian is never formed and fill is recomputed, not read.
 * d_efwd[c], d_eadj[c]: device complex64 [nz][ny][nx] per component c.
 * w: 2 * ncomp host floats (re, im per component).  d_grad: n_params device
 * floats, overwritten.  Asynchronous on `stream`. */
adg_status adg_grad(adg_ctx *ctx, adg_design *design, const double *h_params,
                    const float *const d_efwd[3], const float *const d_eadj[3],
                    const float *w, float *d_grad, void *stream);

/* The same sweep seeded with a real cotangent G = dL/deps (the autograd form):
 *   g_k = sum_c sum_cells G_c * d eps_c / d p_k.
 * d_G: device fp32 [ncomp][nz][ny][nx]. */
adg_status adg_grad_real(adg_ctx *ctx, adg_design *design, const double *h_params,
                         const float *d_G, float *d_grad, void *stream);

/* The dense form of step 5: the same g as adg_grad (bit for bit), plus the
 * derivatives of the same L with respect to the two material levels of
 * eps = eps_bg + (eps_fg - eps_bg) * fill (Sec. 5.1):
 *   d_gmat[0] = dL/d eps_bg = sum_c sum_cells Re(w_c E_adj,c E_fwd,c) (1 - fill_c)
 *   d_gmat[1] = dL/d eps_fg = sum_c sum_cells Re(w_c E_adj,c E_fwd,c) fill_c
 * These depend on every cell, so every cell's fields are streamed (no band
 * culling of the field reads); g still comes from the band tiles, the only
 * place where d eps / d p can be nonzero.  d_fill: the design's fill at the
 * same h_params (as written by adg_build_eps), device fp32
 * [ncomp][nz][ny][nx].  d_gmat: 2 device doubles, overwritten.  The field
 * stream follows the band kernels on `stream`; its sums are formed in a
 * fixed order (reproducible bit for bit).  Asynchronous on `stream`. */
adg_status adg_grad_dense(adg_ctx *ctx, adg_design *design, const double *h_params,
                          const float *const d_efwd[3], const float *const d_eadj[3],
                          const float *w, const float *d_fill, float *d_grad, double *d_gmat,
                          void *stream);

/* Union over non-binary material levels (App. B, Alg. 1).  sets[0..K-1] are
 * K designs, set k being one set of shapes with its own program (the set's
 * union), all on one grid with one logic family and one parameter vector,
 * each with material slots eps_bg = 0, eps_fg = 1 (so its fill is the set's
 * union s^k).  levels[k] is set k's material level above the background,
 * finite, with 0 < levels[0] <= ... <= levels[K-1]; 1 <= K <= 8.  Per sample:
 *   s <- s^1;  s <- union((levels[k-1] / levels[k]) s, s^k), k = 2..K;
 *   eps = eps_bg + levels[K-1] s,
 * union being the sets' logic (Eq. union, or App. B.2's product form).
 * ADG_EINVAL for a NULL argument, K outside [1, 8], unsorted or non-positive
 * levels, or sets that differ in grid, logic, parameter count or material
 * slots.  The first set owns the scratch: K fill-sized float slices for
 * adg_levels_eps, 2K for adg_levels_grad, allocated on first use or growth
 * (growth synchronises the device).  Asynchronous on `stream`; the K sets
 * must not be used concurrently on another stream. */
adg_status adg_levels_eps(adg_ctx *ctx, adg_design *const *sets, int32_t K, const double *levels,
                          double eps_bg, const double *h_params, float *d_eps, void *stream);

/* Eq. 1 (eps term) through Alg. 1: g = Re sum_c w_c E_adj,c E_fwd,c d eps_c / dp
 * with eps the map of adg_levels_eps.  Each set's build, one pass turning
 * the seed levels[K-1] Re(w E_adj E) into one real cotangent per set (the
 * reverse of the loop), each set's real-cotangent sweep (as adg_grad_real),
 * and the sum of the K rows into d_grad (n_params floats, overwritten).
 * Fields and weights as for adg_grad; errors and scratch as above (sets 2..K
 * also hold one n_params float row each). */
adg_status adg_levels_grad(adg_ctx *ctx, adg_design *const *sets, int32_t K, const double *levels,
                           const double *h_params, const float *const d_efwd[3],
                           const float *const d_eadj[3], const float *w, float *d_grad,
                           void *stream);

/* Both terms of Eq. 1: the permittivity term through d_eps (fields E) plus
 * the permeability term through d_mu (fields H), the reverse sweeps of
 * Eqs. jaceps and jacmu seeded with E_adj E and H_adj H:
 *   g = Re sum w_e E_adj E d eps/dp + Re sum w_h H_adj H d mu/dp.
 * d_mu is a design of the composition mu(v) of Eq. mu: its own shapes and
 * program over the same parameters, its grid offsets those of the H samples,
 * and its eps_bg / eps_fg fields holding mu_bg / mu_fg.  Both designs must
 * have the same n_params (ADG_EINVAL otherwise).  Fields, weights and d_grad
 * as for adg_grad (w_h = -2 i omega gives the paper's mu term).  Allocates
 * n_params floats on d_mu on first use.  Asynchronous on `stream`. */
adg_status adg_grad_eh(adg_ctx *ctx, adg_design *d_eps, adg_design *d_mu, const double *h_params,
                       const float *const d_efwd[3], const float *const d_eadj[3],
                       const float *w_e, const float *const d_hfwd[3],
                       const float *const d_hadj[3], const float *w_h, float *d_grad,
                       void *stream);

/* The finite-difference gradient that AutoDiff replaces (Sec. 3; the paper's
 * baseline), on the GPU with the library's own build as the mesher:
 *   g_k = deps sum_c sum_samples Re(w_c E_adj,c E_fwd,c)
 *         (fill(p + h e_k) - fill(p - h e_k)) / 2h,
 * two builds per parameter and one fixed-order dot product each.  Arguments
 * as for adg_grad; h > 0 in parameter units.  Allocates, per design and on
 * first use, four fp32 arrays of the grid (ncomp nz ny nx samples each).
 * Asynchronous on `stream`; reproducible bit for bit.  For measurement and
 * comparison, not for optimisation loops. */
adg_status adg_grad_fd(adg_ctx *ctx, adg_design *design, const double *h_params,
                       const float *const d_efwd[3], const float *const d_eadj[3],
                       const float *w, double h, float *d_grad, void *stream);

/* ---- the bi-level topology special case (Sec. 3.1) ------------------------
 * Every pixel of a 2D design region is its own parameter v_p, broadcast along z
 * over the region's cells (the matrix B of Eq. TO_example):
 *   eps_c(x, y, z) = eps_l + deps sigma(v_p), sigma the logistic sigmoid, for
 *   every component c, pixel p = (x - x0, y - y0) and z0 <= z < z1;
 *   g_p = deps sigma(v_p) (1 - sigma(v_p)) sum_c sum_{z0 <= z < z1}
 *         Re(w_c E_adj,c E_fwd,c)(x, y, z)                       (Eq. top_AD)
 * (w = -2 i omega gives the paper's 2 omega Im(E E_adj); no conjugate).
 * grid: the field layout (nx, ny, nz, ncomp; spacing and offsets unused).
 * d_v, d_grad: device fp32 [ny][nx] of the region (x fastest), caller-owned.
 * d_eps: device fp32 [ncomp][nz][ny][nx]; only the region's samples are
 * written.  d_efwd / d_eadj / w: as for adg_grad.  A region outside the grid,
 * an empty one or a NULL argument returns ADG_EINVAL before any launch.
 * Asynchronous on `stream`; g is reproducible bit for bit. */
typedef struct {
  int32_t x0, y0;  /* first pixel (cells)                               */
  int32_t nx, ny;  /* pixels; v has nx * ny entries                      */
  int32_t z0, z1;  /* the cells [z0, z1) every pixel is broadcast to     */
} adg_topo_region;
adg_status adg_topo_eps(adg_ctx *ctx, const adg_grid *grid, const adg_topo_region *region,
                        const float *d_v, double eps_l, double deps, float *d_eps,
                        void *stream);
adg_status adg_topo_grad(adg_ctx *ctx, const adg_grid *grid, const adg_topo_region *region,
                         const float *d_v, double deps, const float *const d_efwd[3],
                         const float *const d_eadj[3], const float *w, float *d_grad,
                         void *stream);

/* ---- the exact polygon mesher (Prop. 2) and its FD gradient (Sec. 6.3) ----
 * Prop. 2 simulates on the standard, exact shape representation: the
 * volume-averaged material of the layout on the Yee grid.  A layer is a set
 * of simple polygons (convex or concave, either winding, not overlapping one
 * another) extruded over [z0, z1] (bound_z = 1) or over every z (bound_z = 0).
 * The fill of the sample of component c at cell (i, j, k) is the exact
 * average of the layer over the averaging cell centred at the sample
 * (x_s +- dx/2, y_s +- dy/2, z_s +- dz/2; x_s = ox + (i + off[c][0]) dx):
 *   fill = min(1, sum_p area(P_p n cell_xy) / (dx dy)) * |[z0, z1] n cell_z| / dz.
 * Computed in FP64, written as float. */
typedef struct {
  int32_t n_polys;
  const int32_t *vert_off; /* n_polys + 1 offsets into xy, from 0; >= 3 vertices each */
  const double *xy;        /* x, y of every vertex (physical units), host memory     */
  int32_t bound_z;         /* 1: the layer spans [z0, z1]; 0: every z                */
  double z0, z1;
} adg_mesh_layer;

/* d_fill [ncomp][nz][ny][nx] <- the layer's fill over `region` (cells; NULL:
 * the whole grid); samples outside the region are not written.  The layer is
 * copied to the context's scratch (grown on demand, which synchronises the
 * device): calls of one context must not run concurrently on two streams.
 * ADG_EINVAL for a NULL argument, a bad grid or region, a polygon with fewer
 * than 3 vertices, a non-finite coordinate or a reversed z range. */
adg_status adg_mesh_fill(adg_ctx *ctx, const adg_grid *grid, const adg_mesh_layer *layer,
                         const adg_topo_region *region, float *d_fill, void *stream);

/* The finite-difference gradient with the exact mesher (Sec. 6.3's FD
 * baseline): for each parameter k, plus[k] and minus[k] are the layer at
 * p + h e_k and p - h e_k (built by the caller's parameterisation), and
 * regions[k] (NULL: the whole grid for every k) a region outside which the
 * two meshes agree.  g_k = deps sum_{c, samples in region} Re(w_c E_adj,c
 * E_fwd,c) (fill(plus[k]) - fill(minus[k])) / 2h, each region meshed twice
 * into scratch and reduced in a fixed order (reproducible bit for bit).
 * d_grad: n_params floats.  Fields and weights as for adg_grad.  Errors and
 * scratch as above; h must be positive. */
adg_status adg_mesh_grad_fd(adg_ctx *ctx, const adg_grid *grid, int32_t n_params,
                            const adg_mesh_layer *plus, const adg_mesh_layer *minus,
                            const adg_topo_region *regions, double h, double deps,
                            const float *const d_efwd[3], const float *const d_eadj[3],
                            const float *w, float *d_grad, void *stream);

/* ---- batched work ---------------------------------------------------------
 * Many (design, operation) items run as ONE job table: four launches (bin,
 * build, VJP, finalize) whatever the number of designs, their grid sizes or
 * primitive counts.  The binner covers every item's tiles in one grid; the
 * build and VJP kernels are persistent and walk a work list of (design, tile)
 * pairs.  The batched form of the same computation as adg_build_eps /
 * adg_grad / adg_grad_real (Sec. 2, steps 2 and 5), for many designs. */
enum { ADG_BATCH_BUILD = 1, ADG_BATCH_GRAD = 2, ADG_BATCH_GRAD_REAL = 4 };
enum { ADG_BATCH_GRAPH = 1 }; /* submit flag: capture the launches once as a CUDA
                                 graph and replay it for batches of the same shape */
typedef struct {
  adg_design *design;  /* each design at most once per batch                  */
  int32_t ops;         /* ADG_BATCH_* bitmask (GRAD and GRAD_REAL exclusive)   */
  int32_t reserved;    /* must be 0                                           */
  const double *h_params;               /* n_params host doubles              */
  float *d_fill, *d_eps;                /* BUILD outputs (d_fill nullable)    */
  const float *d_efwd[3], *d_eadj[3];   /* GRAD fields, as for adg_grad       */
  float w[6];                           /* GRAD weights (re, im per component) */
  const float *d_G;                     /* GRAD_REAL cotangent                */
  float *d_grad;                        /* GRAD / GRAD_REAL output            */
} adg_batch_item;

/* Enqueue a batch on `stream`; returns a ticket for adg_batch_poll/wait.
 * The library keeps two batch arenas per context, so a third submit waits
 * (host side) for the batch two back to finish uploading.  Host arrays are
 * copied before return.  Batches of one context must share one stream (or be
 * ordered by the caller). */
adg_status adg_batch_submit(adg_ctx *ctx, const adg_batch_item *items, int32_t n_items,
                            int32_t flags, void *stream, uint64_t *ticket);
/* *done = 1 once the batch's device work has completed. */
adg_status adg_batch_poll(adg_ctx *ctx, uint64_t ticket, int32_t *done);
/* Wait at most timeout_ns for the batch; ADG_ETIMEOUT if it is still running. */
adg_status adg_batch_wait(adg_ctx *ctx, uint64_t ticket, uint64_t timeout_ns);

/* Wait for `stream` and report device-side errors (ADG_EDEVICE) recorded by
 * any call of this context since the last adg_sync. */
adg_status adg_sync(adg_ctx *ctx, void *stream);

/* Counters of the design's last binning (synchronises `stream`). */
adg_status adg_design_stats(adg_ctx *ctx, adg_design *design, void *stream, adg_stats *out);

/* Device memory the design holds, in bytes (host-side bookkeeping, no
 * synchronisation): its tables, bins and counters, the partial buffer at the
 * size its current parameters need (or its capacity, if larger), and the
 * scratch of the optional calls it has made (dense form, FD, levels, E+H).
 * Caller buffers (fields, eps, fill, gradients) are not included.  For
 * admission control by a memory budget. */
adg_status adg_design_bytes(adg_ctx *ctx, adg_design *design, int64_t *bytes);

/* Per-kernel timing for measurement.  While enabled, every kernel launch of
 * the context is bracketed by CUDA events recorded on the launching stream.
 * adg_profile_read waits for the recorded events and returns, per kernel
 * (index ADG_K_*), the launch count and the summed device time; `reset`
 * clears the accumulators. */
enum { ADG_K_BIN = 0, ADG_K_BUILD = 1, ADG_K_VJP = 2, ADG_K_FINALIZE = 3,
       ADG_K_PREPARE = 4 /* reserved, not launched: the finalize clears the partials */,
       ADG_K_FILL = 5 /* reserved, not launched: the build fills the constant tiles */,
       ADG_K_DENSE = 6 /* field stream + its fixed-order sum */,
       ADG_K_LEVELS = 7 /* the per-sample pass of Alg. 1 (adg_levels_*) */,
       ADG_K_COUNT = 8 };
typedef struct {
  int64_t launches[ADG_K_COUNT];
  double ms[ADG_K_COUNT];
} adg_profile_data;
adg_status adg_profile_enable(adg_ctx *ctx, int32_t on);
adg_status adg_profile_read(adg_ctx *ctx, adg_profile_data *out, int32_t reset);

/* The gradient of adg_grad for callers that cannot allocate device memory
 * (a process whose device memory belongs to another runtime's fixed arena, a
 * plug-in that must not grow its footprint after start-up, a strict memory
 * budget).  The paper has no counterpart: this is a deployment variant.
 *   - It allocates nothing: no cudaMalloc / cudaFree / allocating library
 *     routine, no host heap.  All device scratch (design tables, primitive
 *     records, per-tile programs, partials, error word) lives in one static
 *     device array of 32 MiB that every GPU loading libadg holds until exit.
 *   - desc, tiles (nullable), h_params: host, as for adg_design_create and
 *     adg_grad; d_efwd, d_eadj, w, d_grad: as for adg_grad (caller-owned).
 *   - Designs needing more than 32 MiB of scratch (tiles x 405 B + partials +
 *     tables), or beyond 4096 primitives / 32768 scalars / 16384 program ops
 *     or parameters, are rejected with ADG_EINVAL and a message saying why.
 *   - The first call on a device sets up the scratch address for that device
 *     (cudaGetSymbolAddress with the device current); make it before any
 *     stream capture.
 *   - Calls share the array and it keeps the last call's contents; each call
 *     clears what must start at zero.  Calls that overlap on the GPU race on
 *     it: serialise them.  The call returns after its work on `stream` has
 *     completed -- also when it fails after enqueueing some of it -- and
 *     reports device-side checks as ADG_EDEVICE.  Error messages go to a
 *     fixed per-thread buffer (adg_last_error), so failures allocate nothing
 *     either. */
adg_status adg_grad_noalloc(const adg_design_desc *desc, const adg_tile_opts *tiles,
                            const double *h_params, const float *const d_efwd[3],
                            const float *const d_eadj[3], const float *w, float *d_grad,
                            void *stream);

/* For tests of the error paths (host-side fault injection; the paper has no
 * counterpart).  Every device and pinned-host allocation libadg makes goes
 * through one counter: with fail_after = n >= 0, the next n allocations
 * succeed and the one after fails as if memory were exhausted (the call that
 * made it returns ADG_ENOMEM), after which injection is off again;
 * fail_after = -1 switches injection off, -2 leaves it as it is.  *live
 * (nullable) receives the number of allocations libadg holds now, so that a
 * test can check that a failed call released what it had taken.
 * Process-wide; not for production use. */
adg_status adg_debug_alloc(int32_t fail_after, int64_t *live);

/* Thread-local description of the last error (never NULL). */
const char *adg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ADG_H */
