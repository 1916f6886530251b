/*
 * vt_gb300.h -- C ABI of the GB300 (sm_103a) Voronoi-cell library.
 *
 * What the library computes follows PARAVT (R. E. Gonzalez, "PARAVT: Parallel
 * Voronoi Tessellation code", arXiv:1601.06429):
 *   - the Voronoi cell of every particle, i.e. the region nearer to it than
 *     to any other particle (Introduction), in a periodic box (Abstract and
 *     Discussion: periodic conditions) or a bounded box;
 *   - from each cell its volume and the density mass/volume (Implementation
 *     section: volume from the cell facets, density from particle mass and
 *     cell volume), the immediate neighbours, i.e. the particles that share a
 *     facet (Implementation section), the density gradient from densities and
 *     neighbours (Implementation section) and densities on a regular grid
 *     (Implementation section);
 *   - outputs are in input order and neighbour indices are real particle
 *     indices, never periodic images (Implementation section: re-indexing of
 *     boundary particles to real indices, output in input order).
 * The backward pass (vt_backward) has no counterpart in the paper; it is the
 * derivative of the cell volumes with respect to the particle positions.
 *
 * Conventions for every entry point:
 *   - Pointers marked "device" are CUDA device memory on the current device,
 *     owned by the caller, and must stay valid until the call's work on the
 *     handle's stream has finished.  Pointers marked "host" are read or written
 *     before the call returns.
 *   - Positions are [N][3] row-major (x,y,z per particle), FP32 or FP64 as
 *     given by `dtype`; every floating-point output uses the same dtype.
 *   - Return value: VT_OK (0) or a negative VT_ERR_* code.  No exception and
 *     no device trap crosses this boundary; errors detected on the device are
 *     recorded in the handle and returned by the next call that synchronises
 *     (vt_build, the size query of vt_cells, vt_status).
 *   - Work is enqueued on the stream given to vt_build.  vt_build synchronises
 *     that stream to read a few status words back (and to grow the facet pool
 *     when a set needs more); the other calls are asynchronous unless stated.
 *     Status words are read through mapped pinned host memory that a small
 *     kernel on the handle's stream writes, not by a copy: a synchronising
 *     call never waits for copies that other streams have queued on the copy
 *     engines.  Each live handle holds one such block (a few hundred bytes,
 *     reused by later handles).
 *   - A handle is not thread-safe; distinct handles are independent.
 */
#ifndef VT_GB300_H
#define VT_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define VT_OK 0
#define VT_ERR_INVALID -1     /* bad argument, NaN/out-of-box position, bad handle */
#define VT_ERR_OOM -2         /* device allocation failed */
#define VT_ERR_CUDA -3        /* a CUDA runtime call failed */
#define VT_ERR_DUPLICATE -4   /* two particles at the same position */
#define VT_ERR_SECURITY -5    /* the security-radius test did not pass within max_passes */
#define VT_ERR_UNSUPPORTED -6 /* e.g. a periodic cell wider than a quarter box, FP32 filter with a box length not representable in FP32 */
#define VT_ERR_CAPACITY -7    /* a cell exceeded the per-cell plane, vertex or candidate capacity */
#define VT_ERR_NUMERIC -8     /* an exact-arithmetic expansion exceeded its workspace */

/* position / output dtypes */
#define VT_F32 0
#define VT_F64 1

/* clipping precision */
#define VT_PLAIN64 0  /* FP64 geometry; FP64 error-bounded predicates, exact fallback */
#define VT_FILTER32 1 /* FP32 geometry; FP32 error-bounded predicates, FP64 then exact fallback */

typedef struct vt_params {
    int precision;  /* VT_PLAIN64 or VT_FILTER32 (default VT_FILTER32) */
    int k_target;   /* particles aimed for in a cell's first candidate pass (default 24) */
    int max_passes; /* candidate radius passes per cell before VT_ERR_SECURITY (default 1000) */
    int face_pool;  /* facet records reserved per particle (default 24; grown on demand) */
    int threads_per_cell; /* VT_FILTER32 only: 32 = one warp per cell (default; 0 means 32); 1 = one thread
                             per cell first, 32 cells of a search-tree bucket per warp; 4 or 8 = that many
                             lanes per cell first (8 or 4 cells per warp, the cell in shared memory, the
                             side tests split by vertex); in each case the cells the first kernel cannot
                             finish are then taken by a warp each (same cells) */
    int reserved[3]; /* [0]: candidate pass sizing, 0 = radius doubling up to 2R, 1 = also limited (default)
                        by the density seen so far; others must be 0 */
} vt_params;

typedef struct vt_stats {
    int64_t n;                /* particles */
    int64_t n_faces;          /* facets between particles (each counted from both sides) */
    int64_t n_cut;            /* bisector planes that cut a cell */
    int64_t n_tested;         /* bisector planes tested against a cell */
    int64_t n_passes;         /* candidate radius passes, summed over cells */
    int64_t n_fp64_fallbacks; /* FP32 predicates re-decided in FP64 */
    int64_t n_exact_cells;    /* cells re-run with the exact predicate */
    int64_t n_exact_preds;    /* predicates decided by exact expansion arithmetic */
    int64_t n_exact_zero;     /* exact predicates that were zero (degenerate input) */
    int64_t max_faces;        /* largest facet count of a cell */
    int32_t device_error;     /* first VT_ERR_* recorded on the device, or VT_OK */
    int32_t error_particle;   /* an input index that raised it, or -1 */
    int64_t n_launches;       /* CUDA kernels launched through this handle so far */
    double t_sort_ms;         /* device time of vt_build's key, sort, gather and tree kernels (CUDA events) */
    double t_clip_ms;         /* device time of vt_build's clipping kernels, last attempt (CUDA events) */
    int64_t reserved[3];      /* diagnostics: [0] internal detail of device_error, [1] candidate collections,
                                 [2] candidates collected */
    int64_t n_handed_over;    /* FP32 filter: cells the thread-per-cell kernel handed to the warp-per-cell kernel */
    int64_t n_bucket_passes;  /* FP32 filter: radius passes of the thread-per-cell kernel, summed over buckets */
    int64_t n_grid_failed;    /* cell/voxel parts the last vt_grid_density_volume could not compute (0 normally) */
} vt_stats;

typedef struct vt_handle_s *vt_handle;

/* Fill *p with the defaults.  Returns VT_OK or VT_ERR_INVALID (p == NULL). */
int vt_default_params(vt_params *p);

/*
 * vt_build -- Voronoi cells of all N particles (Implementation section: the
 * tessellation step; here per cell, by clipping with bisector planes).
 *   h       host out: new handle (NULL on failure)
 *   pos     device [N][3], dtype VT_F32 or VT_F64.  Periodic: every coordinate
 *           in [box_lo, box_hi); bounded: in [box_lo, box_hi].
 *   mass    device [N] of the same dtype, or NULL for unit masses
 *   box_lo, box_hi  host [3]: box corners (box_hi > box_lo)
 *   periodic 1: periodic box; 0: cells clipped by the box walls
 *   p       host params or NULL for defaults
 *   stream  cudaStream_t (NULL: legacy default stream)
 * The handle owns its workspace (sorted particles, search tree, facet records)
 * until vt_destroy.  `pos` and `mass` are read during the call only.  Errors:
 * VT_ERR_INVALID (arguments, NaN or out-of-box coordinates), VT_ERR_DUPLICATE,
 * VT_ERR_SECURITY, VT_ERR_UNSUPPORTED, VT_ERR_CAPACITY, VT_ERR_NUMERIC,
 * VT_ERR_OOM, VT_ERR_CUDA; on error *h is NULL and nothing is leaked.
 */
int vt_build(vt_handle *h, const void *pos, int dtype, const void *mass, int64_t N, const double box_lo[3],
             const double box_hi[3], int periodic, const vt_params *p, void *stream);

/*
 * vt_build_owned -- the cells of the first n_owned particles only, the other N - n_owned being buffer
 * particles that bound those cells but get none of their own (Implementation section: each task computes
 * the cells of its sub-volume from its own particles plus the boundary particles of a buffer zone around
 * it).  Arguments as vt_build, plus
 *   n_owned  1 <= n_owned <= N: input rows [0, n_owned) are the particles whose cells are computed
 * The handle answers every call of a vt_build handle; the rows of buffer particles have volume 0, density 0,
 * no neighbours, a zero gradient and radius 0, while the neighbour lists of computed cells may name them (input
 * row indices).  A computed cell is the true cell of its particle when every particle within twice its radius
 * (vt_cell_radius) is in pos; the caller checks that against the extent of its buffer zone (the library
 * cannot: it sees only the particles it is given).  vt_rebuild keeps n_owned.  Errors as vt_build.
 */
int vt_build_owned(vt_handle *h, const void *pos, int dtype, const void *mass, int64_t N, int64_t n_owned,
                   const double box_lo[3], const double box_hi[3], int periodic, const vt_params *p, void *stream);

/*
 * vt_rebuild -- the cells of new positions for the same particles, in the
 * handle's workspace (the tessellation step again, e.g. for the next Lloyd
 * iteration or the next batch of sets of the same sizes).
 *   pos   device [N][3], the handle's N and dtype; a batched handle keeps its
 *         set offsets and boxes
 *   mass  device [N] or NULL for unit masses
 * Allocates nothing and does not synchronise: every step is a kernel launch or
 * an asynchronous device memset on the handle's stream, so the call may be
 * captured in a CUDA graph (make the vt_build that created the handle before
 * the capture).  Errors found on the device are sticky and come back from
 * vt_status: VT_ERR_INVALID (NaN or out-of-box coordinates; no cell is
 * computed), VT_ERR_CAPACITY (the facet pool of the handle is full: build a
 * new handle, with a larger vt_params.face_pool), VT_ERR_DUPLICATE,
 * VT_ERR_SECURITY, VT_ERR_NUMERIC.  Returns VT_ERR_INVALID (NULL argument) or
 * VT_ERR_CUDA (a launch failed), else VT_OK.
 */
int vt_rebuild(vt_handle h, const void *pos, const void *mass);

/*
 * vt_probe_fp32_tflops -- measured FP32 FMA throughput of this GPU (TFLOP/s,
 * one FMA = 2 flops): eight independent FMA chains per thread on every SM,
 * best of three timed launches after one untimed (CUDA events).  The
 * denominator of the clipping kernel's ALU roofline (the paper has no
 * counterpart).  Synchronises; allocates 32 KB of device memory for the call.
 * Errors: VT_ERR_INVALID (tflops NULL), VT_ERR_OOM, VT_ERR_CUDA.
 */
int vt_probe_fp32_tflops(double *tflops, void *stream);

/*
 * vt_probe_fp64_tflops -- measured FP64 FMA throughput of this GPU (TFLOP/s), by the same method as
 * vt_probe_fp32_tflops on the FP64 pipe (fewer iterations per thread): the denominator of the roofline of the
 * plain FP64 clipping path.  Synchronises; allocates 32 KB of device memory for the call.  Errors as
 * vt_probe_fp32_tflops.
 */
int vt_probe_fp64_tflops(double *tflops, void *stream);

/* most independent sets one vt_build_batched call takes */
#define VT_MAX_SETS 65536

/*
 * vt_build_batched -- Voronoi cells of many independent point sets in one
 * build (Parallel implementation section: the volume is split into
 * sub-volumes that are tessellated independently; here each set is its own
 * bounded sub-volume, with no buffer particles, and all sets share one sort,
 * one search tree and one persistent clipping launch whose work queue runs
 * over the cells of every set).
 *   h        host out: new handle (NULL on failure)
 *   pos      device [N][3], dtype VT_F32 or VT_F64, N = set_off[n_sets]; set s
 *            is the rows [set_off[s], set_off[s+1]), every coordinate inside
 *            its own box (walls included)
 *   mass     device [N] of the same dtype, or NULL for unit masses
 *   set_off  host [n_sets+1], set_off[0] = 0, non-decreasing (empty sets allowed)
 *   n_sets   1 .. VT_MAX_SETS
 *   boxes    host [n_sets][6]: lo x,y,z then hi x,y,z of each set's box; the
 *            cells of a set are clipped by its box walls (no periodic images)
 *   set_k    host [n_sets] k_target of each set, or NULL (p's k_target)
 *   set_tpc  host [n_sets] threads_per_cell of each set (1, 4, 8 or 32; 0 means 32),
 *            or NULL (p's threads_per_cell); see vt_autotune_batched
 *   p, stream  as for vt_build
 * A particle's neighbours are particles of its own set only.  The handle
 * answers vt_cells, vt_density, vt_gradient, vt_moments, vt_backward and
 * vt_status exactly as a vt_build handle over the concatenated sets would, with
 * input indices into `pos`; vt_grid_density returns VT_ERR_UNSUPPORTED.
 * Errors: those of vt_build; VT_ERR_INVALID also for a bad set_off or box.
 */
int vt_build_batched(vt_handle *h, const void *pos, int dtype, const void *mass, const int64_t *set_off,
                     int n_sets, const double *boxes, const int32_t *set_k, const int32_t *set_tpc,
                     const vt_params *p, void *stream);

/*
 * vt_autotune_batched -- per-set clipping parameters for vt_build_batched,
 * chosen by timing (the paper has no counterpart: its parameters are set by
 * hand).  Sets are grouped by size class [2^c, 2^(c+1)); for each class, whole
 * sets spread evenly through it, about `sample` points in all (<= 0: 262144),
 * are copied to a temporary device buffer and built as one batch for every
 * k_target in {16, 24, 32, 48, 64} and (FP32 filter) threads_per_cell in
 * {32, 1, 4, 8}; the configuration with the shortest clipping time (CUDA events)
 * wins for every set of the class.
 *   pos, dtype, set_off, n_sets, boxes, p, stream  as for vt_build_batched
 *   k_out, tpc_out  host out [n_sets]: the chosen k_target and
 *                   threads_per_cell of each set (empty sets: p's k_target, 32)
 * Synchronises; allocates and frees device memory.  The choice only changes
 * the speed: the cells do not depend on it.  Errors: those of vt_build_batched.
 */
int vt_autotune_batched(const void *pos, int dtype, const int64_t *set_off, int n_sets, const double *boxes,
                        const vt_params *p, int64_t sample, int32_t *k_out, int32_t *tpc_out, void *stream);

/*
 * vt_cells -- cell volumes and neighbour lists (Implementation section:
 * volume from the facets; neighbours are the particles sharing a facet;
 * output in input order with real indices).
 *   vol          device [N] (dtype of pos) or NULL
 *   nbr_off      device int64 [N+1] CSR offsets or NULL
 *   nbr_id       device int32 [nnz]: neighbours of particle i, ascending, at
 *                nbr_id[nbr_off[i] .. nbr_off[i+1]); NULL = size query
 *   n_faces_out  host out: nnz (always written when non-NULL; the size query
 *                needs no synchronisation on a handle that was never passed to
 *                vt_rebuild, and synchronises the handle's stream on one that was)
 * After a vt_rebuild, nbr_id needs room for the new nnz: ask for it first.
 * Inside a stream capture pass nbr_id = NULL and n_faces_out = NULL.
 */
int vt_cells(vt_handle h, void *vol, int64_t *nbr_off, int32_t *nbr_id, int64_t *n_faces_out);

/*
 * vt_cell_radius -- the radius of every cell: an upper bound (within about 1e-6 relative) of the largest
 * distance from the particle to a vertex of its cell (no counterpart in the paper; the security-radius test
 * stops on it, and a buffer zone must reach twice it).  rad: device [N], input order, dtype of pos;
 * asynchronous.  Rows whose cell was not computed (vt_build_owned) get 0.
 */
int vt_cell_radius(vt_handle h, void *rad);

/*
 * vt_cell_flags -- which cells needed the fallbacks of the error-bounded predicates (diagnostics; the paper
 * has no counterpart, its Qhull runs in one precision).  flags: device uint8 [N], input order, written
 * asynchronously on the handle's stream: bit 0 (VT_CELL_FP64) some side test of the cell that the FP32
 * filter could not decide was decided in FP64; bit 1 (VT_CELL_EXACT) the cell was finished by the
 * exact-predicate kernel (an FP64 test stayed undecided, or the cell outgrew the fast kernel's capacity).
 * The cells do not depend on the path taken; tests use the flags to make sure such cells are compared.
 */
#define VT_CELL_FP64 1
#define VT_CELL_EXACT 2
int vt_cell_flags(vt_handle h, uint8_t *flags);

/* vt_density -- density mass/volume (Implementation section).  dens: device [N]. */
int vt_density(vt_handle h, void *dens);

/*
 * vt_gradient -- density gradient at each particle from the densities of its
 * Voronoi neighbours (Implementation section; the paper gives no formula):
 * the least-squares linear fit  (sum_j d d^T) g = sum_j d (rho_j - rho_i),
 * d = x_j - x_i the facet's image displacement.  grad: device [N][3].
 */
int vt_gradient(vt_handle h, void *grad);

/*
 * vt_gradient_gg -- the Green-Gauss form of the density gradient, as used by
 * the moving-mesh code the Introduction cites among uses of the tessellation:
 *   grad rho_i = (1/V_i) sum_f A_f (rho_j - rho_i) c_f / |d_f|
 * over the facets between particles (c_f the facet centroid relative to x_i,
 * d_f the neighbour image's displacement); exact for a linear density field;
 * on a wall of a bounded box rho is taken as rho_i.  grad: device [N][3].
 */
int vt_gradient_gg(vt_handle h, void *grad);

/*
 * vt_grid_density -- densities on a regular G^3 grid over the box
 * (Implementation section; the paper gives no formula): node (a,b,c) takes
 * the mean, over its S^3 stratified sub-points
 * lo + (a + (u+1/2)/S) L/G ..., of the density of the cell containing the
 * sub-point (the nearest particle; ties to the lower index).
 * grid: device [G][G][G] indexed [c][b][a] (x fastest).  1 <= G <= 4096, 1 <= S <= 8.
 * VT_ERR_UNSUPPORTED on a vt_build_batched handle.
 */
int vt_grid_density(vt_handle h, int G, int S, void *grid);

/*
 * vt_grid_density_volume -- densities on a regular G^3 grid over the box as
 * volume-weighted averages of the cell densities (Implementation section,
 * "average Voronoi densities on a regular grid", read exactly):
 *   grid[v] = sum_i rho_i |V_i intersect voxel v| / |voxel v|,
 * voxel (a, b, c) = [lo + a L/G, lo + (a+1) L/G] per axis (x fastest in grid,
 * device [G][G][G], dtype of pos); periodic boxes wrap.  Each cell is rebuilt
 * from its facet planes and clipped by the walls of every voxel it meets, in
 * FP32 (volumes to about 1e-6 relative).  1 <= G <= 1024.  Allocates, on the
 * first call (and for a larger G), an FP64 accumulator of G^3 and a retry
 * list; parts that cannot be computed are counted in vt_stats.n_grid_failed.
 * VT_ERR_UNSUPPORTED on a vt_build_batched handle.
 */
int vt_grid_density_volume(vt_handle h, int G, void *grid);

/*
 * vt_backward_weighted -- gradient of the weighted centroidal energy
 *   E_w = sum_i w_i integral over V_i of |y - x_i|^2
 * (the paper has no counterpart; the unweighted form is vt_backward's energy
 * term): moving x_k changes cell k's integrand and moves each facet between k
 * and a neighbour j, across which the energy density jumps by
 * (w_k - w_j) |y - x_k|^2, so
 *   dE_w/dx_k = 2 w_k V_k (x_k - z_k)
 *             + sum_j (w_k - w_j) / |x_j - x_k| integral_f |y - x_k|^2 (y - x_k) dA.
 *   w        device [N] weights, input order, dtype of pos
 *   dE_dpos  device [N][3] out, input order
 * Each cell is rebuilt from its facet planes in FP32 and the facet integrals
 * taken with an exact cubic triangle rule.  Cells that cannot be rebuilt are
 * counted in vt_stats.n_grid_failed (their rows are then not written).
 */
int vt_backward_weighted(vt_handle h, const void *w, void *dE_dpos);

/*
 * vt_moments -- first and second moments of every cell (no counterpart in the paper; they define the
 * centroidal Voronoi energy used with vt_backward).
 *   centroid  device [N][3] or NULL: the cell's centroid, in the frame of the positions (wrapped into
 *             [box_lo, box_hi) for periodic boxes)
 *   energy    device [N] or NULL: E_i = integral over cell i of |y - x_i|^2
 */
int vt_moments(vt_handle h, void *centroid, void *energy);

/*
 * vt_backward -- adjoint of the cell volumes (no counterpart in the paper).
 * For a loss L with dL/dV_i = dL_dV[i] and, optionally, a uniform weight
 * dL_dE on the centroidal (CVT) energy E = sum_i integral_{cell i} |y - x_i|^2:
 *   dL/dx_k = sum_{j in N(k)} (A_kj/|r_kj|) (g_k - g_j) (c_kj - x_k)
 *             + dL_dE * 2 V_k (x_k - z_k),
 * with A, c the facet area and centroid, r the separation and z the cell
 * centroid.  dL_dV: device [N] or NULL; dL_dpos: device [N][3] (overwritten).
 */
int vt_backward(vt_handle h, const void *dL_dV, double dL_dE, void *dL_dpos);

/*
 * vt_volumes_noalloc -- cell volumes of a small periodic or bounded point set without any device
 * allocation.  The paper has no counterpart: this is for callers that cannot call cudaMalloc (inside
 * another library's memory pool, on hosts that forbid allocation after start-up, or where an allocation
 * would synchronise the device).  It runs the same kernels as vt_build + vt_cells with the default
 * parameters (FP32-filtered clipping, one warp per cell), so the volumes equal theirs bit for bit.  All
 * of its scratch memory lives in one file-scope device array of about 8 MB that every GPU using the
 * library holds until the process exits.
 *   pos      device [N][3] (dtype VT_F32 or VT_F64), same rules as vt_build
 *   N        1 <= N <= VT_NOALLOC_MAX_N; larger sets return VT_ERR_CAPACITY
 *   box_lo, box_hi, periodic: as vt_build (periodic boxes need lengths representable in FP32)
 *   vol      device [N] output, dtype of pos
 *   stream   cudaStream_t; the call synchronises it once (to read the status words)
 * All calls share the array and it keeps the last call's contents; calls whose work overlaps on the GPU
 * (other streams or host threads) race and must be serialised by the caller.  The first call on a device
 * looks up the array's device address with that device current: make that first call before any stream
 * capture; the address is kept, so the entry point must not be used after a cudaDeviceReset of that device.
 * It calls no cudaMalloc, cudaFree or allocating library routine.  Errors as vt_build, plus
 * VT_ERR_CAPACITY when the set is too large or its facets do not fit the fixed pool.
 */
#define VT_NOALLOC_MAX_N 8192
int vt_volumes_noalloc(const void *pos, int dtype, int64_t N, const double box_lo[3], const double box_hi[3],
                       int periodic, void *vol, void *stream);

/* vt_status -- counters and the sticky device error; synchronises the stream. */
int vt_status(vt_handle h, vt_stats *out);

/*
 * vt_last_error_detail -- diagnostics of the last vt_build on the calling host thread that failed with a
 * device-detected error: returns an internal reason code (0 if none; for VT_ERR_CAPACITY: -101 planes,
 * -102 vertices, -103 boundary edges, -104 candidates, -105 search stack) and stores in *particle (if not
 * NULL) an input index whose cell raised it, or -1.  Not part of the paper's method.
 */
int vt_last_error_detail(int *particle);

/*
 * vt_debug_fail_alloc -- fault injection for tests (no counterpart in the paper): the nth device allocation
 * that vt_build or vt_build_batched makes for a handle's workspace from now on (counting from 1) fails as if
 * cudaMalloc had run out of memory, and the call returns VT_ERR_OOM after freeing what it had allocated.  The
 * hook fires once and disarms; nth <= 0 disarms it.  Process-wide (all host threads, all devices); returns the
 * previous setting (0 if the hook was disarmed or has fired).  Touches no device.
 */
int vt_debug_fail_alloc(int nth);

/* vt_error_string -- static description of a VT_* code. */
const char *vt_error_string(int code);

/*
 * vt_destroy -- frees the handle and its workspace (NULL is ignored).  Asynchronous: the workspace goes back to
 * the library's memory pool in order on the handle's stream, after the work already enqueued there.
 */
void vt_destroy(vt_handle h);

/*
 * vt_release_memory -- handle workspaces come from a stream-ordered memory pool per device that the library
 * creates on first use (cudaMallocFromPoolAsync / cudaFreeAsync on the handle's stream), which keeps freed memory
 * for the next build instead of returning it to the device; this call synchronises the current device and gives
 * the pool's unused memory back, and frees the pinned host blocks kept for the status reads of destroyed
 * handles.  Returns VT_OK or VT_ERR_CUDA.  (Not part of the paper's method.)
 */
int vt_release_memory(void);

#ifdef __cplusplus
}
#endif
#endif /* VT_GB300_H */
