/*
 * pot.h -- C ABI of the GB300 PlenOctree renderer (libpot.so).
 *
 * Method: PlenOctrees for Real-time Rendering of Neural Radiance Fields
 * (Yu, Li, Tancik, Li, Ng, Kanazawa; ICCV 2021).  A sparse octree stores, in
 * every leaf at the deepest level, a density sigma and real spherical-harmonic
 * coefficients k_l^m in R^3 (Sec. 3.1, Sec. 3.2).  A pixel is rendered by
 * cutting its ray at the voxel boundaries of the octree into segments of
 * constant density and colour, colouring each leaf with the sigmoid of its SH
 * expansion at the ray direction, and compositing with the NeRF quadrature
 * (Eq. 1) plus a background term (App. B.3.2), stopping early once the
 * transmittance falls below gamma (Sec. 3.2 "Rendering").
 *
 * Conventions shared by every entry point:
 *   - Grid: depth D (1..12), R = 2^D voxels per axis over the cube
 *     [bbox_lo, bbox_lo + bbox_size)^3; voxel k on an axis is the half-open
 *     interval [lo + k h, lo + (k+1) h), h = bbox_size / 2^D (exact).
 *   - Morton code of voxel (x,y,z): bits interleaved with x most significant
 *     in each triple, m = sum_b x_b<<(3b+2) | y_b<<(3b+1) | z_b<<3b.
 *   - Canonical tree arrays (pot_tree_export): nodes in breadth-first order
 *     (root = 0; each level by ascending Morton prefix); child[n][s] with slot
 *     s = (x_bit<<2)|(y_bit<<1)|z_bit of the node's level, value 0 = empty,
 *     > 0 node index, < 0 -(leaf+1); leaves numbered by ascending Morton code.
 *   - SH: K = (sh_degree+1)^2 coefficients per channel, index k = l^2 + l + m,
 *     RGB innermost ([K][3]); real basis from the complex Y_l^m with the
 *     Condon-Shortley phase (App. B.1), theta from +z, phi = atan2(y, x),
 *     evaluated at the unit ray direction.  Degree 1 is (+y, +z, +x) * sqrt(3/4pi).
 *   - Distances (near, far, segment length delta) are world units along the ray.
 *   - Pixel ray of a pinhole camera (column i, row j), fp32 in this order, each
 *     operation IEEE round-to-nearest, no contraction:
 *       xc = ((float)i + 0.5 - cx) / fx;  yc = -(((float)j + 0.5 - cy) / fy)
 *       d_r = (c2w[r][0]*xc + c2w[r][1]*yc) - c2w[r][2];   o_r = c2w[r][3]
 *     (camera looks along its -z axis; the direction need not be unit length).
 *
 * Memory and streams.  Every call is asynchronous on the caller's stream
 * unless stated otherwise; a NULL stream is the legacy default stream.  Array
 * arguments may live in host or device memory where a function says so (the
 * library detects which); when an output is in host memory the call
 * synchronises the stream before returning.  Inputs are read-only and owned by
 * the caller; trees are owned by the library and released by pot_tree_free.
 * Per-call scratch (tile counters, staged inputs, staging buffers of host
 * outputs) is stream-ordered memory from a pool the library keeps per device,
 * which holds on to up to 1 GiB of freed scratch for later calls; host-output
 * renders also use two library-owned streams per device (a second render
 * stream and a copy stream) and join them back to the caller's stream.
 *
 * Errors.  Every entry point returns a pot_status; POT_OK is 0.  The message
 * of the last failure on the calling thread is returned by pot_last_error().
 * A render whose traversal exceeds its step bound (3 * 2^D + 16 cells per
 * ray, never expected for a well formed tree) stops that ray and raises a
 * device error word, which pot_check() reports as POT_ERR_TRAVERSAL.
 */
#ifndef POT_H
#define POT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st *pot_stream;

typedef enum pot_status {
    POT_OK = 0,
    POT_ERR_INVALID_ARG = 1,
    POT_ERR_OOM = 2,
    POT_ERR_CUDA = 3,
    POT_ERR_TRAVERSAL = 4,
    POT_ERR_BUDGET = 5,
    POT_ERR_UNSUPPORTED = 6
} pot_status;

/* Storage type of leaf values (density and SH).  Arithmetic is fp32 always;
 * the paper optimises in float32 and stores the tree in float16 (App. B.5,
 * PlenOctree optimisation details). */
typedef enum pot_dtype {
    POT_F32 = 0,
    POT_F16 = 1,
    POT_BF16 = 2,
    POT_CB16 = 3 /* codebook-quantised SH (pot_tree_quantize only): float32 sigma, uint16 codes */
} pot_dtype;

typedef struct pot_tree pot_tree;

typedef struct pot_build_desc {
    int32_t depth;         /* D, 1..12 (1..10 for pot_build from a dense grid) */
    int32_t sh_degree;     /* 0..4 */
    int32_t leaf_dtype;    /* pot_dtype */
    float sigma_threshold; /* pot_build keeps voxel iff sigma > threshold */
    float bbox_lo[3];
    float bbox_size;       /* > 0 */
} pot_build_desc;

/* 80 bytes.  c2w: rows of the camera-to-world matrix; columns are the camera
 * right, up and back (= -viewing direction) axes and the eye position. */
typedef struct pot_camera {
    float c2w[3][4];
    float fx, fy, cx, cy;
    int32_t width, height;
    float near, far;
} pot_camera;

typedef struct pot_render_opts {
    float bg[3];      /* background colour c_N (App. B.3.2); default 0 */
    float gamma;      /* early stop when transmittance < gamma; 0 disables */
    float near, far;  /* pot_render_rays only: clip range (world distance) */
    uint32_t flags;   /* reserved, must be 0 */
    int32_t max_steps; /* cells visited per ray before the ray is stopped and the
                          device error word raised; 0 = 3 * 2^D + 16, which no
                          ray of a well formed tree can reach */
    /* Optional device outputs for measurement (NULL to skip):
     *   seg_count[ray]   number of leaf segments composited
     *   leaf_touched[L]  set to 1 for every leaf composited by some ray   */
    int32_t *seg_count;
    uint8_t *leaf_touched;
} pot_render_opts;

typedef struct pot_tree_info {
    int32_t depth, sh_degree, sh_dim, leaf_dtype;
    int64_t n_nodes, n_leaves;
    int64_t bytes;        /* device bytes held by the tree */
    int64_t leaf_bytes;   /* bytes of one leaf record as stored (sigma + SH, padding included) */
    float bbox_lo[3];
    float bbox_size;
    int32_t saturated;    /* 1 if some value overflowed fp16/bf16 and was clamped */
    int32_t device;
    int64_t index_bytes;  /* device bytes of the cell index (pot_tree_set_cell_index), 0 if none;
                             included in bytes */
    int32_t index_kind;   /* pot_cells layout of the cell index */
} pot_tree_info;

/* ---------------------------------------------------------------- build ---
 * Sec. 3.2 "Filtering": the kept voxels become leaves at the deepest level
 * and the tree is empty elsewhere.  A node exists iff it has a kept
 * descendant; leaf values are copied (rounded to nearest even and saturated
 * for fp16 / bf16 storage).
 *
 * pot_build: dense grids, host or device memory, indexed [x][y][z]:
 *   sigma [R][R][R] float32, sh [R][R][R][K][3] float32.
 *   A voxel is kept iff sigma > desc->sigma_threshold.  A NaN or infinite
 *   sigma gives POT_ERR_INVALID_ARG.
 * pot_build_sparse: n kept voxels, host or device memory:
 *   morton [n] uint64 strictly increasing and < 8^D (else
 *   POT_ERR_INVALID_ARG), sigma [n] float32 (finite), sh [n][K][3] float32.
 * *out receives a new tree on the current device.  Synchronises the stream. */
pot_status pot_build(const pot_build_desc *desc, const float *sigma, const float *sh, pot_tree **out,
                     pot_stream stream);
pot_status pot_build_sparse(const pot_build_desc *desc, int64_t n, const uint64_t *morton,
                            const float *sigma, const float *sh, pot_tree **out, pot_stream stream);

pot_status pot_tree_get_info(const pot_tree *tree, pot_tree_info *info);

/* Canonical arrays (conventions above) into caller buffers in host or device
 * memory: child [n_nodes][8] int32, sigma [n_leaves] float32, sh
 * [n_leaves][K][3] float32 (stored values widened exactly), morton
 * [n_leaves] uint64.  Any pointer may be NULL. */
pot_status pot_tree_export(const pot_tree *tree, int32_t *child, float *sigma, float *sh,
                           uint64_t *morton, pot_stream stream);

/* Overwrites leaf values from caller arrays (same layouts as pot_build_sparse,
 * host or device memory); the structure is unchanged. */
pot_status pot_tree_set_values(pot_tree *tree, const float *sigma, const float *sh, pot_stream stream);

/* Synchronises the tree's device and frees it.  NULL is accepted. */
pot_status pot_tree_free(pot_tree *tree);

/* Cell index of a tree (the paper has no counterpart: an acceleration
 * structure of this library).  It gives, for every voxel of the 2^D grid, the
 * leaf holding it (>= 0) -- what the descent of the child array (Sec. 3.2
 * "Rendering") finds -- or, for an empty voxel, a box of empty space around
 * it that a ray crosses in one step:
 *   -(2 + 2 l)   the empty octree node of level l that contains it, or
 *   -(3 + 2 e)   the cube of (2e+1)^3 voxels centred on it (every voxel within
 *                Chebyshev distance e is empty; e <= 63), recorded where
 *                2e + 2 > 2^(D-l).
 * Two layouts:
 *   POT_CELLS_DENSE  one int32 entry per voxel: 4 * 8^D bytes (537 MB at
 *                    D = 9, 4.3 GB at D = 10); D <= 10 (the build also needs
 *                    2 * 8^D bytes of scratch); e is the voxel's own
 *                    Chebyshev distance to the nearest leaf - 1.  A cell is
 *                    one 4-byte load.
 *   POT_CELLS_BRICK  one int32 per 4 x 4 x 4 brick of voxels (4 * 8^(D-2)
 *                    bytes: 8 MB at D = 9, 67 MB at D = 10, 537 MB at
 *                    D = 11) plus 64 entries (256 bytes) for each brick that
 *                    holds a leaf; D in 3..11.  A brick without a leaf has
 *                    one entry for all its voxels: the empty node around
 *                    the brick, or the cube of half-extent 4 (b - 1) where b
 *                    is the brick's Chebyshev distance, in bricks, to the
 *                    nearest brick holding a leaf; inside a brick with a leaf
 *                    empty voxels get their empty node.  A cell is two
 *                    dependent 4-byte loads.
 * A leaf's segment is bounded by the crossing times of its own faces however
 * the empty space before it was stepped over, so renders, gradients and
 * visibility weights are bit-identical with either index and without one.
 *   Every tree that pot_build, pot_build_sparse, pot_tree_prune or
 *   pot_tree_quantize creates gets the default layout for its depth (dense
 *   for D <= 9, brick for 10 <= D <= 11) when the device has room for it
 *   (pot_tree_info.index_bytes / index_kind say which it has).
 *   enable = 0 synchronises the device and frees it; 1 builds the default
 *   layout, 2 the dense, 3 the brick layout (replacing another layout;
 *   POT_ERR_UNSUPPORTED outside the layout's depths, POT_ERR_OOM when the
 *   device is full).  The tree's structure is never changed after
 *   creation, so the index stays valid under pot_tree_set_values and
 *   pot_step.  Not thread-safe against renders of the same tree from other
 *   host threads. */
typedef enum pot_cells { POT_CELLS_NONE = 0, POT_CELLS_DENSE = 2, POT_CELLS_BRICK = 3 } pot_cells;
pot_status pot_tree_set_cell_index(pot_tree *tree, int32_t enable, pot_stream stream);

/* The cell index (entries as above, each voxel's own entry in either layout)
 * as a dense [R][R][R] int32 array indexed [x][y][z] (R = 2^D) into caller
 * memory (host or device); POT_ERR_INVALID_ARG if the tree has none.  (No
 * counterpart in the paper.) */
pot_status pot_tree_export_cell_index(const pot_tree *tree, int32_t *out, pot_stream stream);

/* ---------------------------------------------------------------- query ---
 * Leaf containing each point xyz [n][3] float32: leaf index >= 0, -1 for
 * empty space inside the box, -2 outside the box (or NaN).  Exact membership
 * (conventions above).  xyz and leaf_out in device memory. */
pot_status pot_query(const pot_tree *tree, int64_t n, const float *xyz, int32_t *leaf_out,
                     pot_stream stream);

/* Real SH basis Y_k, k < K, at the directions dirs [n][3] (normalised
 * inside) into Y [n][K] float32, K in {1, 4, 9, 16, 25}; device memory.
 * App. B.1. */
pot_status pot_sh_basis(int32_t K, int64_t n, const float *dirs, float *Y, pot_stream stream);

/* --------------------------------------------------------------- render ---
 * Sec. 3.2 "Rendering", Eq. 1, App. B.3.2: for every pixel of every camera,
 *   C = sum_i T_i (1 - exp(-max(sigma_i,0) delta_i)) c_i + T_N bg,
 *   T_i = exp(-sum_{j<i} max(sigma_j,0) delta_j),
 *   c_i = sigmoid(sum_k k_{i,k} Y_k(d)),
 * over the leaf segments of the ray clipped to the box and to [near, far];
 * stops after the first segment that leaves T < gamma.
 *   cams [n_cams] in host memory, all with the same width and height;
 *   rgb [n_cams][H][W][3] float32 and t_final [n_cams][H][W] float32 (final
 *   transmittance T_N; may be NULL), host or device memory.               */
pot_status pot_render(const pot_tree *tree, const pot_camera *cams, int32_t n_cams,
                      const pot_render_opts *opts, float *rgb, float *t_final, pot_stream stream);

/* Same for arbitrary rays: origins [n][3], dirs [n][3] (not necessarily unit)
 * float32; rgb [n][3], t_final [n]; host or device memory.               */
pot_status pot_render_rays(const pot_tree *tree, int64_t n, const float *origins, const float *dirs,
                           const pot_render_opts *opts, float *rgb, float *t_final, pot_stream stream);

/* ------------------------------------------------------------- backward ---
 * App. B.3.2: gradients of L = sum_rays <grad_rgb, C> with respect to the
 * stored leaf values, for the rays of pot_render_rays with the same opts:
 *   dC/dk_{i,k}  = w_i c_i (1 - c_i) Y_k            (per channel)
 *   dC/dsigma_i  = delta_i [ c_i T_{i+1} - (C - sum_{j<=i} w_j c_j) ]
 * (zero where the stored sigma <= 0), summed over channels, rays and segments.
 * rgb_fwd is the forward colour C of each ray (pot_render_rays output, same
 * tree and opts); NULL makes the kernel recompute it in a first pass.
 * ACCUMULATES (+=) into grad_sigma [n_leaves] and grad_sh [n_leaves][K][3]
 * (float32, canonical layout); the caller zeroes them.  grad_sh must be
 * 16-byte aligned when 3K is a multiple of 4 (rows are added in 16-byte
 * vectors), else POT_ERR_INVALID_ARG.  All arrays in device memory.
 * Summation order of the float atomics is not deterministic.               */
pot_status pot_render_backward(const pot_tree *tree, int64_t n, const float *origins, const float *dirs,
                               const float *grad_rgb, const float *rgb_fwd, const pot_render_opts *opts,
                               float *grad_sigma, float *grad_sh, pot_stream stream);

/* Sec. 3.3 / App. B.3.2 in one launch, for a training batch: each ray is
 * rendered as by pot_render_rays (C, same opts), the MSE loss
 *   L = sum over rays and channels of (C - target)^2 / (3 n)
 * (the loss of pot_loss_mse) is WRITTEN to *loss (one float), and its
 * gradients (pot_render_backward with grad_rgb = 2 (C - target) / (3 n)) are
 * ACCUMULATED into grad_sigma [n_leaves] and grad_sh [n_leaves][K][3].  rgb
 * [n][3] receives C when not NULL.  Each ray is walked twice in the same
 * launch (colour, then gradients), so no colour buffer or second launch is
 * needed.  target [n][3] float32; every array in device memory; grad_sh
 * aligned as for pot_render_backward.  Float atomic summation order
 * (gradients, loss) is not deterministic.                                  */
pot_status pot_render_mse_backward(const pot_tree *tree, int64_t n, const float *origins, const float *dirs,
                                   const float *target, const pot_render_opts *opts, float *rgb, float *loss,
                                   float *grad_sigma, float *grad_sh, pot_stream stream);

/* ----------------------------------------------------------------- step ---
 * Sec. 3.3 / App. B.5: gradient step on the leaf values with the structure
 * fixed (the paper uses SGD; RMSprop and Adam are offered too), in place on a
 * float32 tree (other dtypes: POT_ERR_UNSUPPORTED).  Element-wise, separate
 * learning rates for sigma and SH:
 *   SGD      x -= lr g
 *   RMSprop  v = alpha v + (1 - alpha) g^2;  x -= lr g / (sqrt(v) + eps)
 *   Adam     m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 *            x -= lr (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps)
 * (the torch.optim definitions).  state: caller-owned float32 device buffer of
 * pot_step_state_floats(tree, kind) floats, zero before the first step;
 * layout [sigma part n_leaves][SH part n_leaves*3K] (Adam: m then v).     */
typedef enum pot_optimizer { POT_SGD = 0, POT_RMSPROP = 1, POT_ADAM = 2 } pot_optimizer;

typedef struct pot_step_desc {
    int32_t kind;            /* pot_optimizer */
    float lr_sigma, lr_sh;
    float alpha;             /* RMSprop smoothing, e.g. 0.99 */
    float beta1, beta2;      /* Adam, e.g. 0.9, 0.999 */
    float eps;               /* e.g. 1e-8 */
    int32_t step;            /* Adam: 1 for the first step */
} pot_step_desc;

int64_t pot_step_state_floats(const pot_tree *tree, int32_t kind);
pot_status pot_step(pot_tree *tree, const pot_step_desc *desc, const float *grad_sigma, const float *grad_sh,
                    float *state, pot_stream stream);

/* Sec. 3, NeRF loss, as a mean: loss = (1/(3n)) sum (rgb - target)^2 and
 * grad_rgb = 2 (rgb - target) / (3n) (grad_rgb may be NULL).  rgb, target,
 * grad_rgb [n][3]; loss: one float; all device memory.                    */
pot_status pot_loss_mse(int64_t n, const float *rgb, const float *target, float *grad_rgb, float *loss,
                        pot_stream stream);

/* Pixel rays of cameras (the camera expression above): for k < n, pixel
 * index pixels[k] = cam * H * W + row * W + col (pixels NULL: k itself), into
 * origins / dirs [n][3].  cams in host memory (same width/height); pixels,
 * origins, dirs in device memory.  An index outside the cameras gives
 * POT_ERR_INVALID_ARG (checked after the launch; synchronises).           */
pot_status pot_camera_rays(const pot_camera *cams, int32_t n_cams, int64_t n, const int64_t *pixels,
                           float *origins, float *dirs, pot_stream stream);

/* pot_render for callers that may not allocate GPU memory (the paper has no
 * counterpart; this is a deployment variant).  Applications that embed the
 * renderer and own all GPU memory -- a viewer on a fixed memory budget, a host
 * whose allocator hooks refuse allocations by libraries, a frame loop that
 * cannot pay for an allocator call -- cannot use pot_render, which allocates a
 * small scratch buffer (tile counter + device copy of the cameras) per call.
 * This call takes that scratch from one fixed array inside the library
 * (256 B + 1024 camera records = 82,176 B per GPU, held until the process
 * exits) and makes no allocation at all.
 *   - Same arguments and results as pot_render, except: at most 1024 cameras
 *     per call (more gives POT_ERR_INVALID_ARG), and rgb / t_final (and
 *     opts->seg_count / leaf_touched, when given) must be device memory
 *     (nothing is staged; host arrays give POT_ERR_INVALID_ARG before any
 *     launch); cams are in host memory and are copied to the array by every
 *     call.
 *   - The first call on a device looks up the array's device address (with
 *     that device current) and caches it; make that first call before any
 *     stream capture on the device.
 *   - All calls share the array and it keeps the last call's contents (the
 *     tile counter is cleared by every call).  Calls whose GPU work overlaps
 *     (other streams, other host threads) race on it: serialise them.       */
pot_status pot_render_noalloc(const pot_tree *tree, const pot_camera *cams, int32_t n_cams,
                              const pot_render_opts *opts, float *rgb, float *t_final, pot_stream stream);

/* ------------------------------------------------------------ filtering ---
 * Sec. 3.2 "Filtering": render the cameras and keep, for every leaf, the
 * largest ray weight w_i = T_i (1 - exp(-max(sigma_i,0) delta_i)) it receives
 * (compositing and early stop as in pot_render; bg unused).  Updates
 * max_weight [n_leaves] (device memory, float32) to max(old, new): the caller
 * initialises it (zeros) and may accumulate over several calls.  cams: host
 * memory, same width and height.                                           */
pot_status pot_visibility(const pot_tree *tree, const pot_camera *cams, int32_t n_cams,
                          const pot_render_opts *opts, float *max_weight, pot_stream stream);

/* A new tree holding the leaves of `tree` whose score >= threshold (score
 * [n_leaves] in device memory, e.g. pot_visibility's max_weight), with the
 * same depth, box, SH degree, dtype and leaf values; the tree is empty
 * elsewhere, so empty space grows where leaves were dropped.  Synchronises. */
pot_status pot_tree_prune(const pot_tree *tree, const float *score, float threshold, pot_tree **out,
                          pot_stream stream);

/* --------------------------------------------------------- quantisation ---
 * App. B.2: a copy of `tree` whose SH coefficients are quantised, separately
 * for each SH basis function, into a codebook of 2^bits RGB entries (float16)
 * by median cut, each leaf keeping one uint16 code per basis function; sigma
 * is kept as it is (stored as float32: the source tree's values exactly,
 * whatever its dtype).  Median cut here: every box splits at every
 * level; the split axis is the box's longest extent (ties: lowest channel);
 * its points are ordered by (value on that axis, leaf index) and split at
 * floor(n/2); a box of fewer than two points keeps them.  An entry is the mean
 * of its box (float64, summed in box order, rounded once to float16).  The
 * result has leaf_dtype POT_CB16; it renders, batches, filters and exports
 * (values = the codebook entries) like any tree; no gradients or set_values.
 * bits: 1..16.  Runs on the host (threads over basis functions); synchronises. */
pot_status pot_tree_quantize(const pot_tree *tree, int32_t bits, pot_tree **out, pot_stream stream);

/* ---------------------------------------------------------------- batch ---
 * Many render requests in one call -- the work list of a continuous-batching
 * server (the paper's real-time viewer renders one view at a time, Sec. 4.5;
 * this is its multi-request form).  Each item names its own tree, camera
 * (any resolution), background, early-stop threshold and outputs; items may
 * use different trees, SH degrees and leaf dtypes.  Items are grouped by
 * (SH degree, dtype) and each group is one kernel launch on the stream, whose
 * warps draw 8x4-pixel tiles from all the group's items.  Per-ray arithmetic
 * is pot_render's: a request's pixels are identical alone or in a batch.
 * items: host array; rgb [H][W][3] and t_final [H][W] (may be NULL) in device
 * memory; trees on the current device.                                    */
typedef struct pot_render_item {
    const pot_tree *tree;
    pot_camera cam;
    float bg[3];
    float gamma;
    float *rgb;
    float *t_final;
} pot_render_item;

pot_status pot_render_batch(const pot_render_item *items, int32_t n_items, pot_stream stream);

/* ---------------------------------------------------------- measurement ---
 * L2 read bandwidth of this GPU (the paper has no counterpart: a measurement
 * kernel for the render path's L2 roofline).  Allocates a `bytes` device
 * buffer (1 MiB .. 1 GiB; pick one that fits in L2, e.g. 32 MiB), fills it,
 * reads it twice to make it L2-resident, then times `reps` (1..10000) full
 * passes of 16-byte loads that bypass L1 (CUDA events on `stream`) and writes
 * the bytes read per second / 1e9 to *gbs.  Synchronises; frees the buffer. */
pot_status pot_probe_l2_read(int64_t bytes, int32_t reps, double *gbs, pot_stream stream);

/* Number of CUDA kernels launched by this library in this process since it
 * was loaded (a counter for benchmarks). */
int64_t pot_launch_count(void);

/* Synchronises the stream and returns POT_ERR_TRAVERSAL if any render on
 * this device raised the device error word since the last check (the word
 * is cleared), POT_ERR_CUDA on a CUDA error, else POT_OK. */
pot_status pot_check(pot_stream stream);

const char *pot_last_error(void);
int32_t pot_version(void);

#ifdef __cplusplus
}
#endif
#endif /* POT_H */
