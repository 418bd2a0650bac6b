/*
 * octfuse -- octree TV-L1 range-data fusion on one GB300 (sm_103a).
 *
 * C ABI of the library.  Every entry point takes plain pointers and sizes; no
 * PyTorch or C++ type crosses it.  Pointers marked "host or device" may point
 * to either (the library copies with cudaMemcpyDefault); pointers marked
 * "device" must be device memory of the context's GPU.
 *
 * The method (Kehl et al., "An Octree-Based Approach towards Efficient
 * Variational Range Data Fusion", BMVC 2016):
 *   - Eq. 1 (Sec. 3.1): per frame i a truncated signed distance
 *       f_i(x) = clamp((D_i(pi_i(x)) - ||x - C_i||) / delta, -1, 1)
 *     and a binary weight w_i(x) (observed unless phi_i(x) < -eta);
 *   - Eq. 2 (Sec. 3.1): top-down octree construction, a node splitting while
 *     the spread max f - min f over it exceeds tau;
 *   - Eq. 3-5 (Sec. 3.2): the fused field u* minimises
 *       E(u) = integral of  sum_i w_i |u - f_i| / (sum_i w_i + gamma)
 *                           + lambda |grad u|
 *     over the leaves of an adaptive octree;
 *   - Sec. 3.2 "Optimization on the Octree": leaves with |u| < tau_split are
 *     split, subtrees whose leaves all hold |u| > tau_join with one sign are
 *     joined.
 * The minimiser here is the first-order primal-dual method the paper names as
 * future work (Sec. 5, Chambolle & Pock), applied to the exact L1 energy;
 * ofu_descend runs the paper's own gradient descent on the eps-L1 energy
 * (Eq. 4-6) on the same leaves and operators.
 *
 * Data layout (all owned by the context, in HBM):
 *   leaves sorted by Morton key of their minimum corner in finest-voxel units
 *   (x bit k -> key bit 3k, y -> 3k+1, z -> 3k+2); level 0 = root,
 *   max_depth = finest voxel; structure of arrays for key, level, u, ubar,
 *   p_x, p_y, p_z, tau, sigma; per-leaf Eq. 1 samples as a sorted CSR.
 *
 * Streams: every call enqueues its work on the stream given at creation and
 * is ordered with respect to earlier calls.  Calls that return host values
 * (restructure, energy, export_*, num_leaves, solve) synchronise that stream.
 *
 * Errors: every call returns an ofu_status; ofu_last_error() describes the
 * last failure.  OFU_EINVAL / OFU_ESTATE / OFU_ECAPACITY leave the context as
 * it was, except where a call has already replaced the frames or the
 * structure when it finds the problem (ofu_integrate_frames when the
 * construction exceeds a cap, ofu_load on a malformed file): the context then
 * holds no octree until a call that builds one succeeds.  OFU_ECUDA and
 * OFU_ENOMEM poison the context: only ofu_destroy is valid after them.  No
 * call aborts the process or traps on the device.
 */
#ifndef OCTFUSE_H
#define OCTFUSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ofu_ctx ofu_ctx;

typedef enum {
  OFU_OK = 0,
  OFU_EINVAL = 1,      /* bad argument */
  OFU_ENOMEM = 2,      /* device allocation failed */
  OFU_ECUDA = 3,       /* CUDA error; context poisoned */
  OFU_ESTATE = 4,      /* call not valid in the context's current state */
  OFU_ECAPACITY = 5,   /* result would exceed max_leaves or a 32-bit index */
  OFU_ETIMEOUT = 6     /* reserved: a bounded device wait gave up */
} ofu_status;

/* Solver and scene parameters.  Lengths in metres. */
typedef struct {
  double origin[3];    /* minimum corner of the cubic domain */
  double extent;       /* edge length of the domain (> 0) */
  int32_t max_depth;   /* D_max, 1..15: finest voxel = extent / 2^D_max */
  int32_t sample_fp16; /* 0: Eq. 1 samples stored as float32, 1: as float16 */
  double delta;        /* truncation band of Eq. 1 (> 0) */
  double eta;          /* observation threshold of Sec. 3.1 (>= 0) */
  double lambda;       /* TV weight of Eq. 3/5 (>= 0) */
  double gamma;        /* normaliser offset of Eq. 5 (> 0) */
  double tau_split;    /* split a leaf when |u| < tau_split */
  double tau_join;     /* join a subtree when all |u| > tau_join (>= tau_split) */
  double spread_tau;   /* Eq. 2 construction threshold (the paper uses 0.1) */
  int64_t max_leaves;  /* hard cap on the leaf count (0 = 2^27, the maximum) */
  int32_t data_term;   /* source of each leaf's frame samples: 0 = Eq. 1 at the leaf
                          centre; 1 = the per-frame TSDF octrees of Sec. 3.1 read by
                          the Fig. 4 rule (see ofu_integrate_frames) */
  int32_t reserved;    /* 0 */
} ofu_params;

/* Fills `p` with the defaults: origin (-0.5,-0.5,-0.5), extent 1, max_depth 6,
 * float32 samples, delta 4 voxels, eta 2 delta, lambda 0.5, gamma 1e-3,
 * tau_split 0.95, tau_join 0.99, spread_tau 0.1, max_leaves 0, data_term 0. */
void ofu_default_params(ofu_params* p);

/* Creates an empty context on the current CUDA device.  `cuda_stream` is a
 * cudaStream_t (NULL = legacy default stream), borrowed for the context's
 * lifetime.  Device memory is allocated by the library (cudaMalloc; see
 * ofu_create_octree_ex for a caller's allocator) and released by
 * ofu_destroy.  EINVAL for out-of-range parameters. */
ofu_status ofu_create_octree(const ofu_params* params, void* cuda_stream, ofu_ctx** out);

/* Device allocator supplied by the caller (for example a framework's caching
 * allocator).  alloc returns `bytes` of device memory on the current device,
 * or NULL on failure; free_fn gives back a block that alloc returned, with its
 * size.  The library may give a block back while work it enqueued earlier on
 * the context's stream still uses it, and may use a new block from work
 * enqueued on that stream right away: the allocator must order reuse after
 * the stream's pending work (a stream-ordered allocator bound to that stream,
 * as PyTorch's caching allocator is, or one that synchronises). */
typedef void* (*ofu_alloc_fn)(size_t bytes, void* user);
typedef void (*ofu_free_fn)(void* ptr, size_t bytes, void* user);

/* ofu_create_octree with every device buffer of the context (leaves, samples,
 * neighbour lists, voxel map, frames, scratch) taken from alloc and given back
 * through free_fn; pinned host staging is the library's own.  Both callbacks
 * must be given (EINVAL otherwise); `user` is passed through.  A NULL from
 * alloc fails the call that needed the memory with ENOMEM and poisons the
 * context (only ofu_destroy is valid after it).  ofu_destroy gives back every
 * block still held, after synchronising the stream. */
ofu_status ofu_create_octree_ex(const ofu_params* params, void* cuda_stream, ofu_alloc_fn alloc,
                                ofu_free_fn free_fn, void* user, ofu_ctx** out);

/* Releases everything the context owns.  NULL is ignored. */
void ofu_destroy(ofu_ctx* ctx);

/* Text of the last error of `ctx` (empty if none); valid until the next call
 * on ctx.  With ctx == NULL, the last error of a failed ofu_create_octree. */
const char* ofu_last_error(const ofu_ctx* ctx);

/* Eq. 1-2, Sec. 3.1: takes F range frames and builds the initial octree.
 *   depth: host or device, float32 [F][H][W], z-depth in metres along the
 *          optical axis; 0, negative or NaN = invalid pixel (w = 0);
 *          +inf = the ray saw no surface (f = +1, w = 1).
 *   intr:  host or device, float64 [F][4] = fx, fy, cx, cy; pixel (px, py)
 *          has its centre at (px + 0.5, py + 0.5).
 *   pose:  host or device, float64 [F][16], camera-to-world 4x4 row-major,
 *          camera axes x right, y down, z forward.
 * The frames are copied into the context (re-integration after restructuring
 * reads them).  Then: the median of the Eq. 1 samples at every finest-voxel
 * centre (-1 where no frame observes it) is reduced top-down by Eq. 2 into
 * the leaves; every leaf gets its sorted samples at its centre; face
 * neighbours and step sizes are built; u = ubar = per-leaf median, p = 0.
 * Replaces any earlier structure.  EINVAL for F, H, W < 1 or null pointers;
 * ECAPACITY when leaves or samples exceed the caps. */
ofu_status ofu_integrate_frames(ofu_ctx* ctx, int32_t F, int32_t H, int32_t W,
                                const float* depth, const double* intr, const double* pose);

/* n >= 0 primal-dual iterations on the current structure (Sec. 3.2 energy):
 *   p    <- proj_{|p_l| <= lambda}(p + sigma_l grad ubar)
 *   u'   <- clamp(prox of the L1 data term at u + tau_l div p, -1, 1)
 *   ubar <- 2 u' - u,  u <- u'
 * Asynchronous.  ESTATE before ofu_integrate_frames. */
ofu_status ofu_iterate(ofu_ctx* ctx, int32_t n);

/* Split/join pass (Sec. 3.2): leaves below max_depth with |u| < tau_split are
 * replaced by all their finest descendants (children inherit u and p); every
 * maximal subtree whose leaves all hold |u| > tau_join with one sign becomes
 * one leaf holding the volume-weighted means of u and p.  New leaves get
 * their Eq. 1 samples; neighbours and step sizes are rebuilt; ubar = u.
 * Outputs (host pointers, each may be NULL): number of split leaves, of
 * joined subtrees, and the new leaf count.  Synchronises the stream. */
ofu_status ofu_restructure(ofu_ctx* ctx, int64_t* n_split, int64_t* n_join, int64_t* n_leaves);

/* Energy of Eq. 5 (exact L1 terms) at the current u, the value of the dual
 * problem at the current p, and their difference (the primal-dual gap, >= 0
 * up to rounding), all accumulated in float64 in a fixed order.  Host
 * pointers, each may be NULL.  Synchronises the stream. */
ofu_status ofu_energy(ofu_ctx* ctx, double* primal, double* dual, double* gap);

/* Current leaf count (host pointer). */
ofu_status ofu_num_leaves(ofu_ctx* ctx, int64_t* n);

/* Copies the leaves in key order: keys (uint64 Morton keys), levels (uint8)
 * and u (float32).  Each destination is host or device and may be NULL;
 * `cap` is the element capacity of each.  *n receives the leaf count;
 * ECAPACITY (nothing copied) when cap < count.  Synchronises the stream. */
ofu_status ofu_export_leaves(ofu_ctx* ctx, uint64_t* keys, uint8_t* levels, float* u,
                             int64_t cap, int64_t* n);

/* The whole hot path after ofu_integrate_frames: runs `iters` iterations in
 * windows of `restructure_every` (0 = never restructure), restructuring after
 * every window but the last; every `check_every` iterations (0 = never) it
 * evaluates the energy and stops early once gap / max(|primal|, 1) < gap_tol.
 * Outputs (host, may be NULL): iterations run, sum over iterations of the leaf
 * count (leaf-iterations), and the final primal, dual, gap (energies3[3];
 * evaluated once at the end when check_every = 0).  Synchronises. */
ofu_status ofu_solve(ofu_ctx* ctx, int32_t iters, int32_t restructure_every, int32_t check_every,
                     double gap_tol, int32_t* iters_done, int64_t* leaf_iters, double* energies3);

/* The paper's own solver (Eq. 4-6; step schedule of Sec. 4): n iterations of
 * gradient descent on the eps-L1-smoothed normalised energy
 *   E_eps(u) = sum_l h_l^3 [c_l sum_k G(u_l - f_k) + lambda G(|grad u (l)|)],
 *   G(x) = sqrt(x^2 + eps^2),  c_l = 1 / (W_l + gamma),
 * on the current structure, with the same level-aware gradient and divergence
 * as ofu_iterate.  Iteration t0 + i (0-based) takes the step
 * xi = xi0 * 0.5^floor((t0 + i) / halve_every) (the paper: xi0 = 0.1, halved
 * every 20, 100 iterations):
 *   q    <- grad u / sqrt(|grad u|^2 + eps^2)
 *   u    <- u - xi [c sum_k (u - f_k) / sqrt((u - f_k)^2 + eps^2) - lambda div q]
 *   ubar <- u;  p is not touched; u is not clamped.
 * Restructuring stays a separate call (ofu_restructure).  Asynchronous.
 * EINVAL for n < 0, t0 < 0, eps <= 0, xi0 <= 0 or halve_every < 1 (or NaN);
 * ESTATE before ofu_integrate_frames. */
ofu_status ofu_descend(ofu_ctx* ctx, int32_t n, int32_t t0, double eps, double xi0,
                       int32_t halve_every);

/* Eq. 7 (Sec. 4.2, split and join): the quantisation error between a field
 * on the finest voxels and the current leaves,
 *   err = sum over leaves n of | u(n) - mean of fine over the voxels of n |.
 * fine: host or device, float32 [n_fine], n_fine = 8^max_depth, indexed by the
 * Morton key of each finest voxel -- the u of a fully refined run exported in
 * key order.  err: host double.  Means are differences of float64 prefix
 * sums; the terms are summed in a fixed order.  Synchronises.  EINVAL for
 * NULL pointers or a wrong n_fine; ESTATE before ofu_integrate_frames. */
ofu_status ofu_quantisation_error(ofu_ctx* ctx, const float* fine, int64_t n_fine, double* err);

/* ---- per-frame TSDF octrees (data_term = 1) ------------------------------
 *
 * With data_term = 1, ofu_integrate_frames (and ofu_load) also turns each
 * frame's TSDF into an octree f_i* (Sec. 3.1, "Octree construction"): Eq. 1
 * at every finest-voxel centre for that frame alone, then top-down, a node is
 * split while its voxels do not all share one weight, or while all are
 * observed and the spread of f over them exceeds spread_tau (Eq. 2); every
 * node holds the mean of the observed f below it and weight 1 when any voxel
 * below it is observed.  A leaf of the iterate at level L then takes, from
 * each frame, the deepest node of that frame's tree on its path at a level
 * <= L (Fig. 4: the node at the leaf's level, else the tree leaf containing
 * it) as its sample, unobserved when that node's weight is 0; this replaces
 * Eq. 1 at the leaf centre for every sample (construction's median field
 * still uses Eq. 1 at the finest voxels).  Means are float64 quotients of
 * float64 sums, stored as float32 (or float16) samples. */

/* Leaves of frame `frame`'s tree, sorted by Morton key (keys uint64,
 * levels uint8; host or device; NULL to size).  *n receives the count;
 * ECAPACITY when cap is too small; ESTATE without data_term = 1 frames.
 * Synchronises. */
ofu_status ofu_export_frame_tree(ofu_ctx* ctx, int32_t frame, uint64_t* keys, uint8_t* levels,
                                 int64_t cap, int64_t* n);

/* Memory of the data term, Table 1's comparison: dense_bytes = frames x
 * 8^max_depth voxels x (a float distance + a float weight); octree_bytes =
 * nodes of all frame trees x (9 pointers + 3 floats, the node layout of
 * Sec. 4.1); device_bytes = what this library keeps on the device for the
 * trees; nodes (int64 [frames], host, may be NULL) per frame.  Any output
 * may be NULL.  ESTATE without data_term = 1 frames. */
ofu_status ofu_data_term_memory(ofu_ctx* ctx, int64_t* nodes, int64_t* dense_bytes,
                                int64_t* octree_bytes, int64_t* device_bytes);

/* Zero level set of the current field as a triangle mesh (Sec. 3.3: the
 * fused result is meshed by marching cubes).  The field is sampled at every
 * finest-voxel centre (each voxel takes its leaf's u); cubes have eight
 * neighbouring centres as corners; u < 0 is inside.  One vertex per grid edge
 * whose ends differ in sign, at t = a / (a - b) from the edge's lower end
 * (float64, then stored as float32 world coordinates origin + (i + 1/2 +
 * t e) * extent / 2^max_depth); vertices are shared between cubes.  Each
 * cube's triangles follow from its faces (no case table): on each face, seen
 * from outside with corners counter-clockwise, a contour segment starts at
 * every crossing where the walk goes from outside to inside and ends at the
 * walk's next crossing; the segments close into loops, taken in the order
 * found (faces -x, +x, -y, +y, -z, +z) and fanned from their first vertex, so
 * triangle normals point outside (u >= 0) and the mesh is closed.
 *
 * Output order: vertices by voxel (x-major index (x n + y) n + z, n =
 * 2^max_depth) then axis; triangles by cube (the same index of its lowest
 * voxel), then loop, then fan.  verts: float32 [V][3], tris: int32 [T][3]
 * (host or device; either may be NULL); *n_verts and *n_tris receive V and T
 * (call with NULL buffers to size them).  ECAPACITY, nothing written, when a
 * given buffer is smaller than the mesh.  Scratch: about 13 bytes per finest
 * voxel, kept by the context.  Synchronises. */
ofu_status ofu_extract_mesh(ofu_ctx* ctx, float* verts, int64_t vcap, int32_t* tris, int64_t tcap,
                            int64_t* n_verts, int64_t* n_tris);

/* ---- inspection and test hooks ----------------------------------------- */

typedef enum {
  OFU_FIELD_U = 0,          /* float32 [N] */
  OFU_FIELD_UBAR = 1,       /* float32 [N] */
  OFU_FIELD_P = 2,          /* float32 [3][N]: p_x then p_y then p_z */
  OFU_FIELD_TAU = 3,        /* float32 [N] primal step sizes */
  OFU_FIELD_SIGMA = 4,      /* float32 [N] dual step sizes */
  OFU_FIELD_W = 5,          /* int32 [N] observed-sample counts */
  OFU_FIELD_SAMPLE_OFF = 6, /* uint32 [N+1] CSR offsets of the samples */
  OFU_FIELD_SAMPLES = 7     /* float32 [total]: sorted samples (float16 ones widened) */
} ofu_field;

/* Copies one per-leaf array to `dst` (host or device) holding `cap_items`
 * elements of the field's type.  *n_items receives the element count;
 * ECAPACITY (nothing copied) when cap_items is too small.  Synchronises. */
ofu_status ofu_export_field(ofu_ctx* ctx, int32_t field, void* dst, int64_t cap_items,
                            int64_t* n_items);

/* Face-neighbour lists of one face (0..5 = +x, +y, +z, -x, -y, -z) as CSR:
 * off int64 [N+1] and idx int64 [nnz] (host or device; either may be NULL to
 * query nnz).  The neighbours across a face are the leaves containing a
 * finest voxel that touches the face from outside, ascending in index; an
 * empty list is the domain boundary.  ECAPACITY when cap < nnz. */
ofu_status ofu_export_neighbours(ofu_ctx* ctx, int32_t face, int64_t* off, int64_t* idx,
                                 int64_t cap, int64_t* nnz);

/* Replaces the structure by n leaves given in ascending key order (keys
 * uint64, levels uint8; host or device; they must tile the domain), takes
 * their Eq. 1 samples from the stored frames and rebuilds neighbours and step
 * sizes.  u (float32 [N]) and p (float32 [3][N]) are optional (NULL: u =
 * median, p = 0); ubar = u.  ESTATE before ofu_integrate_frames, EINVAL when
 * the leaves do not tile the domain. */
ofu_status ofu_import_leaves(ofu_ctx* ctx, const uint64_t* keys, const uint8_t* levels, int64_t n,
                             const float* u, const float* p);

/* Overwrites u, ubar and p (float32 [N], [N], [3][N]; host or device; ubar
 * may be NULL for ubar = u) on the current structure. */
ofu_status ofu_set_state(ofu_ctx* ctx, const float* u, const float* ubar, const float* p, int64_t n);

/* ---- checkpoint / resume ------------------------------------------------- */

/* Writes the context to a file: parameters, the frames (as the range maps
 * the integration uses) and cameras, the leaves (keys, levels) and the
 * iterate (u, ubar, p).  Synchronises the stream.  EINVAL if the file cannot
 * be written. */
ofu_status ofu_save(ofu_ctx* ctx, const char* path);

/* Restores a file written by ofu_save into `ctx` (created with any
 * parameters; they are replaced by the file's).  Samples, neighbours and
 * step sizes are rebuilt from the stored frames and leaves, so iterating
 * after a load gives bit for bit what the saved context would have given.
 * EINVAL for a missing or malformed file (the context is then without an
 * octree). */
ofu_status ofu_load(ofu_ctx* ctx, const char* path);

/* ---- learned warm start (not in the paper) ----------------------------- */
/*
 * A per-leaf network replaces the median initialisation of observed leaves
 * by a learned initial u.  The paper has no learned component; its
 * initialisation is the plain per-point data (Sec. 3.1).
 *
 * Features, 39 float32 per leaf (row-major [N][39]):
 *   x[0..31]  nearest-rank quantiles f_(r_j) of the leaf's sorted samples,
 *             r_j = ceil((2j - 1) W / 64) for j = 1..32 (0 when W = 0);
 *   x[32]     level / max_depth;
 *   x[33..38] per face (+x, +y, +z, -x, -y, -z) the mean of the neighbours'
 *             current u weighted by the share of the face each covers,
 *             min(1, (h_m / h_l)^2); the leaf's own u on the domain boundary.
 * Network: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = tanh(w3 . h2 + b3),
 * W1 [64][39], W2 [64][64]; the 6785 float32 parameters are packed in the
 * order W1, b1, W2, b2, w3, b3 (row-major).
 * Training loss over a batch: sum_i w_i (y_i - t_i)^2 / sum_i w_i; Adam with
 * beta1 = 0.9, beta2 = 0.999, eps = 1e-8 and bias correction. */
typedef struct ofu_mlp ofu_mlp;

/* Number of packed parameters (6785). */
int64_t ofu_mlp_num_params(void);

/* Creates a network with all parameters 0 on the current device; work runs
 * on `cuda_stream`.  ofu_last_error(NULL) describes a failure. */
ofu_status ofu_mlp_create(void* cuda_stream, ofu_mlp** out);
void ofu_mlp_destroy(ofu_mlp* net);
const char* ofu_mlp_last_error(const ofu_mlp* net);

/* Copies the packed parameters in (host or device; resets Adam's moments and
 * step count) or out.  Synchronise the network's stream. */
ofu_status ofu_mlp_set_params(ofu_mlp* net, const float* params);
ofu_status ofu_mlp_get_params(ofu_mlp* net, float* params);

/* y[B] = network(X[B][39]); device pointers; asynchronous. */
ofu_status ofu_mlp_forward(ofu_mlp* net, const float* X, int64_t B, float* y);

/* Gradient of the batch loss with respect to the packed parameters and the
 * loss itself.  X [*][39], t [*], w [*] are device arrays; `rows` (device,
 * int32 [B], may be NULL for rows 0..B-1) selects the batch.  `grad` (host or
 * device, 6785 floats) and `loss` (host) may be NULL.  Per-block partial
 * gradients are summed in a fixed order, so results are reproducible.
 * Synchronises the network's stream. */
ofu_status ofu_mlp_gradient(ofu_mlp* net, const float* X, const float* t, const float* w,
                            const int32_t* rows, int64_t B, float* grad, double* loss);

/* One Adam step (learning rate lr > 0) on the batch's gradient.  With a
 * non-NULL `loss` (host) the batch loss before the step is returned and the
 * stream is synchronised; otherwise the call is asynchronous. */
ofu_status ofu_mlp_train_step(ofu_mlp* net, const float* X, const float* t, const float* w,
                              const int32_t* rows, int64_t B, float lr, double* loss);

/* Features of the current leaves from the current u into X (device, at
 * least cap_rows >= N rows of 39 floats); asynchronous. */
ofu_status ofu_features(ofu_ctx* ctx, float* X, int64_t cap_rows);

/* Warm start: u = ubar = network(features) for leaves with W > 0 whose
 * output is finite; other leaves keep their value (the median, -1 where
 * unobserved).  Features are taken from the current u, so call it right after
 * ofu_integrate_frames.  The dual variable is started consistently with the
 * new field: p = lambda grad u / |grad u| where |grad u| >= 0.05 (truncation
 * units per finest voxel; a TSDF ramp has 1/4 at delta = 4 voxels), p = 0
 * elsewhere -- the optimal dual wherever the field has an edge.  With p = 0
 * the first primal steps would pull u back towards the median.  Asynchronous
 * on the context's stream (it first waits for the network's stream). */
ofu_status ofu_warm_start(ofu_ctx* ctx, const ofu_mlp* net);

/* ---- allocation-free variant -------------------------------------------- */

/* ofu_energy for callers that must not cause a device allocation: a caller
 * whose GPU memory is already owned by another allocator (a framework's
 * caching allocator that has reserved the device, a fixed memory budget), or
 * a latency-critical loop that forbids cudaMalloc / cudaFree, which
 * synchronise the device, once it is running.  ofu_energy may allocate its
 * reduction buffer on first use; this variant allocates nothing.  The paper
 * has no counterpart: this is an interface convenience, the arithmetic is
 * that of ofu_energy (same per-leaf float64 terms, partials summed in a fixed
 * order, so results agree to rounding).
 *
 * Input: the context's current iterate.  Output: out3[3] = primal energy,
 * dual value, gap; host or device memory.  Synchronises the stream.
 *
 * Scratch: a file-scope device array of 8192 x 2 + 3 doubles (about 128 KiB),
 * present on every GPU that loads the library until the process exits.  One
 * partial pair per block of 2048 leaves, so at most 16,777,216 leaves:
 * larger octrees get OFU_ECAPACITY with a message naming the limit.  Every
 * call looks up the array's device address (cudaGetSymbolAddress, which
 * allocates nothing) with the context's device current; the device that was
 * current at ofu_create_octree must be current here, else OFU_EINVAL.  The
 * first call on a device may load the library's device code there, so make
 * it before any stream capture.
 * All calls share the array and each overwrites it, so calls that overlap on
 * the GPU (several streams or threads at once) race and must be serialised
 * by the caller. */
ofu_status ofu_energy_static(ofu_ctx* ctx, double* out3);

/* ---- measurement hooks --------------------------------------------------- */

/* Number of CUDA kernels this library has launched in this process. */
int64_t ofu_kernel_launches(void);

/* enable >= 1 clears and starts per-launch timing of the two iteration
 * kernels (dual step, primal step) with CUDA events recorded on the context's
 * stream around each launch made by ofu_iterate / ofu_solve; enable = 0 stops
 * it.  The event pool is created here (outside any timed work) for
 * max(enable, 8192) iterations and kept; iterations beyond the pool are not
 * timed (and not counted by ofu_profile_read) until the next enable.  EINVAL
 * for enable < 0 or > 2^20. */
ofu_status ofu_profile(ofu_ctx* ctx, int32_t enable);

/* Reads the timing since ofu_profile(ctx, 1) (synchronises): per kernel
 * (index 0 = dual step, 1 = primal step) the summed device time in ms, the
 * launch count, and the summed algorithmic bytes, i.e. every array element
 * the kernel must read or write once per leaf (neighbour values re-read
 * through the cache are not counted):
 *   dual   45 B per leaf: ubar, level, three +face entries, p read and
 *          written, sigma;
 *   primal 57 B per leaf + each observed sample (4 B, or 2 B in float16):
 *          u read and written, ubar written, level, six face entries, p,
 *          tau, sample offset, and the samples the prox is defined over.
 *          The kernel's search starts at the leaf's rank of the previous
 *          iteration, so a settled leaf reads only the two samples that
 *          bracket its prox (one 32-byte sector) and the DRAM bytes fall
 *          below this count.
 * Any output pointer may be NULL. */
ofu_status ofu_profile_read(ofu_ctx* ctx, double* ms, int64_t* launches, double* bytes);

#ifdef __cplusplus
}
#endif

#endif /* OCTFUSE_H */
