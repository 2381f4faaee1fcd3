/*
 * sdg.h -- C ABI of libsdg: differentiable volume rendering of an SDF (with
 * colour and semantic channels) stored in a globally sparse, locally dense
 * voxel-block grid, on one NVIDIA B300 (sm_103a).
 *
 * Paper: "Fast Monocular Scene Reconstruction with Global-Sparse Local-Dense
 * Grids" (arXiv 2305.13220).  Each entry point cites the passage that defines
 * the operation it performs.
 *
 * Conventions shared by every call
 * --------------------------------
 *  * Every call returns an int status (SDG_OK = 0 or an SDG_ERR_* code); no
 *    exception crosses the ABI.  sdg_last_error() returns a thread-local
 *    message for the last failing call of the calling thread.
 *  * Pointers named *_dev are device pointers on the grid's device; all other
 *    pointers are host pointers.  Device arrays are dense and row-major, FP32
 *    unless stated.  The caller owns every buffer it passes in and must keep
 *    it alive until the work enqueued on the grid's stream has finished.
 *  * The grid owns its hash table, voxel channels, gradients, optimiser
 *    state, neighbour table and dense block-index grid.  sdg_grid_channel exposes
 *    channels zero-copy; those pointers stay valid until sdg_grid_destroy.
 *  * All work is enqueued on the stream given in sdg_grid_desc.  Calls are
 *    asynchronous, except those that return a count to the host
 *    (activation's n_new, sdg_grid_num_blocks) and save/load, which
 *    synchronise that stream.
 *  * Voxel layout: grid point (voxel) v in Z^3 sits at world position
 *    v * voxel_size.  Its block key is b = floor(v / 8) per axis, its local
 *    coordinate l = v - 8b in [0,8)^3, stored at linear position
 *    lz*64 + ly*8 + lx inside block index i, i.e. element i*512 + that.
 *  * Block indices are dense in [0, num_blocks).  Each activation batch
 *    appends its new blocks after the existing ones, in ascending
 *    (z, y, x) key order.
 *  * Ray records are 8 floats: ox, oy, oz, tnear, dx, dy, dz, tfar.
 *  * Block keys are limited to [-2^20, 2^20) per axis.
 */
#ifndef SDG_H
#define SDG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------------- */
/* Status codes                                                             */
/* ----------------------------------------------------------------------- */
#define SDG_OK 0
#define SDG_ERR_ARG 1       /* invalid argument (null pointer, bad size, wrong layout) */
#define SDG_ERR_OOM 2       /* a device or host allocation failed */
#define SDG_ERR_CAPACITY 3  /* a fixed capacity would be exceeded; the object is unchanged */
#define SDG_ERR_CUDA 4      /* a CUDA runtime call or kernel launch failed */
#define SDG_ERR_TIMEOUT 5   /* a wait ran out of time */
#define SDG_ERR_BUSY 6      /* not now: a result not ready yet (poll again), or a grid registered with a server */
#define SDG_ERR_IO 7        /* file read/write failed or the file is malformed */
#define SDG_ERR_NOT_FOUND 8 /* unknown ticket / scene id */

/* Storage types of the colour channel. */
#define SDG_F32 0
#define SDG_BF16 1

/* Channel groups (sdg_grid_channel). */
#define SDG_GROUP_GEO 0    /* SDG_F32 grids: float4 {sdf, r, g, b} per voxel, [max_blocks][512][4] */
#define SDG_GROUP_SDF 1    /* SDG_BF16 grids: float sdf, [max_blocks][512] */
#define SDG_GROUP_RGB 2    /* SDG_BF16 grids: bfloat16 {r, g, b, 0}, [max_blocks][512][4] */
#define SDG_GROUP_SEM 3    /* bfloat16 semantic logits, [max_blocks][512][n_sem] (n_sem > 0 only) */
#define SDG_GROUP_WEIGHT 4 /* float fusion weight, [max_blocks][512] (not read by the renderer) */

/* Channel kinds. */
#define SDG_KIND_VALUE 0
#define SDG_KIND_GRAD 1   /* float, same element count as the value (the RGB group keeps 4 lanes) */
#define SDG_KIND_ADAM_M 2 /* float first moment (unused by RMSProp) */
#define SDG_KIND_ADAM_V 3 /* float second moment (RMSProp's running mean of g^2) */

/* Backward modes (sdg_render_opts.mode). */
#define SDG_MODE_RECOMPUTE 0 /* backward re-traverses and re-samples each ray: O(rays) saved state */
#define SDG_MODE_STORE 1     /* forward keeps every sample's position and values for the backward */

/* Optimisers (sdg_adam_opts.algo). */
#define SDG_OPT_ADAM 0
#define SDG_OPT_RMSPROP 1

typedef struct sdg_grid_s* sdg_grid;
typedef struct sdg_ctx_s* sdg_ctx;
typedef struct sdg_server_s* sdg_server;

/* ----------------------------------------------------------------------- */
/* Grid                                                                     */
/* ----------------------------------------------------------------------- */

/* Sec. 3.2 ("Sparse-Dense Data Structure"): voxels exist only inside
 * allocated 8^3 blocks, indexed by a collision-free hash map; each voxel
 * stores an SDF (theta_d), a colour (theta_c) and optionally semantic logits
 * (theta_s).  Sec. 4.1 uses 8^3 blocks. */
typedef struct {
    float voxel_size;   /* metres, > 0 */
    float beta;         /* Laplace scale of the SDF-to-density transform (Sec. 3.5.1), metres;
                           <= 0 selects voxel_size / 2 */
    int64_t max_blocks; /* block capacity, at most 2^22 (voxel addresses are 32-bit in the kernels); every
                           per-block array is allocated for it up front */
    int32_t rgb_dtype;  /* SDG_F32 or SDG_BF16 */
    int32_t n_sem;      /* semantic channels per voxel: 0 or a multiple of 4, at most 32 */
    int32_t device;     /* CUDA device ordinal */
    int32_t reserved;   /* must be 0 */
    void* stream;       /* cudaStream_t for all work on this grid; NULL = the legacy default stream */
} sdg_grid_desc;

/* Creates an empty grid; all channels, gradients and optimiser state start at zero.
 * Errors: SDG_ERR_ARG (bad descriptor), SDG_ERR_OOM, SDG_ERR_CUDA. */
int sdg_grid_create(const sdg_grid_desc* desc, sdg_grid* out);

/* Frees every device buffer the grid owns.  Safe on NULL. */
int sdg_grid_destroy(sdg_grid g);

/* Block activation, Sec. 3.4.1 Eq. 7-8 (phi = 1): for every point x, the
 * voxel v = floor(x * (1/voxel_size)) (FP32, (1/voxel_size) rounded to FP32)
 * is grown to the cube v + [-dilate_voxels, dilate_voxels]^3 and every block
 * touched by that cube is activated.  dilate_voxels = 8R reproduces the
 * supplement's block dilation Dilate_R exactly (R = 2 in the paper).
 * xyz_dev: [n][3] float device points.  Points whose scaled coordinates are
 * non-finite or beyond 8e6 voxels are skipped.  0 <= dilate_voxels <= 64.
 * n_new (host, may be NULL): number of blocks added.  Synchronises.
 * All-or-nothing: on SDG_ERR_CAPACITY (more than max_blocks in total, or a
 * block bounding box of more than 2^31 blocks: the traversal keeps a 4-byte
 * block index for every block cell of the box) the grid is unchanged. */
int sdg_grid_activate_points(sdg_grid g, const float* xyz_dev, int64_t n, int32_t dilate_voxels, int64_t* n_new);

/* Same as sdg_grid_activate_points on the points of a depth map, unprojected
 * per Eq. 8 with this exact FP32 operation order (no fused multiply-add):
 *   xc = (((u + 0.5f) - cx) * (1/fx)) * d;  yc = (((v + 0.5f) - cy) * (1/fy)) * d;  zc = d
 *   x_i = ((Twc[i][0]*xc + Twc[i][1]*yc) + Twc[i][2]*zc) + Twc[i][3]
 * depth_dev: [H][W] float z-depth; pixels with non-finite or non-positive
 * depth are skipped.  K (host): fx, fy, cx, cy.  Twc (host): row-major 3x4
 * camera-to-world.  Synchronises; all-or-nothing like activate_points. */
int sdg_grid_activate_depth(sdg_grid g, const float* depth_dev, int32_t H, int32_t W, const float K[4],
                            const float Twc[12], int32_t dilate_voxels, int64_t* n_new);

/* sdg_grid_activate_depth over F depth maps as ONE activation batch: the
 * union of their blocks is inserted at once, new blocks indexed in ascending
 * packed-key order over the whole batch (F sequential calls give the same
 * block set, indexed map by map).  depth_dev: [F][H][W] float z-depth.
 * K (host): [F][4] fx, fy, cx, cy.  Twc (host): [F][12] row-major 3x4
 * camera-to-world.  The per-map unprojection is sdg_grid_activate_depth's.
 * F = 0 adds nothing.  Synchronises once; all-or-nothing over the batch. */
int sdg_grid_activate_depth_frames(sdg_grid g, const float* depth_dev, int32_t F, int32_t H, int32_t W,
                                   const float* K, const float* Twc, int32_t dilate_voxels, int64_t* n_new);

/* Activates an explicit list of block keys keys_dev [n][3] int32 (duplicates
 * and already active keys allowed).  Synchronises; all-or-nothing. */
int sdg_grid_activate_keys(sdg_grid g, const int32_t* keys_dev, int64_t n, int64_t* n_new);

/* Number of active blocks (host).  Synchronises. */
int sdg_grid_num_blocks(sdg_grid g, int64_t* n);

/* Copies the active keys, in index order, to keys_dev [num_blocks][3] int32. */
int sdg_grid_keys(sdg_grid g, int32_t* keys_dev);

/* Hash-map lookup (Sec. 3.2, the collision-free block index): keys_dev [n][3]
 * int32 -> idx_dev [n] int32 block index, -1 if the block is not active. */
int sdg_grid_lookup(sdg_grid g, const int32_t* keys_dev, int64_t n, int32_t* idx_dev);

/* Zero-copy view of one channel: *dev_ptr and its size in bytes (for
 * max_blocks blocks; only the first num_blocks are meaningful).
 * SDG_ERR_ARG if the group/kind does not exist in this grid's layout. */
int sdg_grid_channel(sdg_grid g, int32_t group, int32_t kind, void** dev_ptr, int64_t* bytes);

/* Sets every gradient channel to zero (enqueued). */
int sdg_grid_zero_grad(sdg_grid g);

/* Writes / reads the grid: header (voxel size, beta, layout, block count,
 * optimiser step), keys in index order, then every value, gradient and
 * optimiser-state channel of the active blocks.  Load creates a new grid; a
 * non-NULL desc overrides device, stream and max_blocks (which must be at
 * least the stored block count).  Both synchronise.  SDG_ERR_IO on failure. */
int sdg_grid_save(sdg_grid g, const char* path);
int sdg_grid_load(const char* path, const sdg_grid_desc* desc, sdg_grid* out);

/* Optimiser step counter kept with the grid (saved and loaded with it). */
int sdg_grid_get_step(sdg_grid g, int32_t* step);
int sdg_grid_set_step(sdg_grid g, int32_t step);

/* Profiling aid (the paper has no counterpart).  With start and stop two
 * cudaEvent_t handles (not owned; created by the caller on the grid's
 * device), every render pass enqueued on this grid afterwards -- forward,
 * backward, training passes -- records start on the grid's stream just
 * before its render kernels (after the traversal pass and any ray ordering)
 * and stop just after them, so cudaEventElapsedTime(start, stop) is the
 * duration of the render kernels of the last pass.  NULL, NULL stops the
 * recording.  Errors: SDG_ERR_ARG (one of the two NULL). */
int sdg_grid_set_pass_events(sdg_grid g, void* start_event, void* stop_event);

/* Bounds-checked build (the paper has no counterpart; a debugging aid).  A
 * library compiled with -DSDG_CHECKED checks in its render, traversal and
 * query kernels every block index, trilinear-corner voxel address,
 * dense-grid cell and ray row they derive before using it; the first index
 * out of range is recorded in a status word per device (code << 48 | the
 * index's low 48 bits; codes SDG_CHECK_*) -- never a trap -- and the access is
 * skipped (the stencil counts as invalid, the cell as unallocated, the ray as
 * ray 0).  This call synchronises the device, reads that word into *status
 * (0: no violation) and clears it if `clear`; *checked tells whether the
 * loaded library is the checked build (in the normal build *status is 0). */
#define SDG_CHECK_BLOCK 1
#define SDG_CHECK_VOXEL 2
#define SDG_CHECK_DENSE 3
#define SDG_CHECK_RAY 4
int sdg_checked_status(int32_t device, int32_t clear, uint64_t* status, int32_t* checked);

/* Blocks the host until all work on the grid's stream has finished. */
int sdg_grid_sync(sdg_grid g);

/* ----------------------------------------------------------------------- */
/* Rendering                                                                */
/* ----------------------------------------------------------------------- */

/* Sec. 3.5.1, Eq. 12-15.  For each ray x(t) = o + t d on [tnear, tfar]
 * (clipped to the box of active blocks), the allocated stretches
 * [t_in, t_out) are found by a block-level traversal that skips
 * unallocated space; their total length S defines a skip-space coordinate
 * s.  Sample k of N sits at s_k = (k + u_k) S / N (u_k = 0.5, or a PCG hash
 * of (seed, ray_id0 + ray, k) when stratified), mapped back to t_k.
 * delta_k = s_{k+1} - s_k, delta_{N-1} = S - s_{N-1}.  At each sample the
 * SDF, colour and logits are trilinear interpolations of the 8 surrounding
 * voxels (Eq. 17); a sample whose 8 voxels are not all allocated is invalid
 * (density 0, no gradient).  Density: sigma = Psi_beta(-d) / beta (the
 * Laplace CDF transform of VolSDF).  Weights w_k = T_k (1 - exp(-sigma_k
 * delta_k)), T_k = exp(-sum_{j<k} sigma_j delta_j) (Eq. 15).  Outputs per
 * ray: rgb = sum w c + T_N bg, depth = sum w t, opac = sum w, sem = sum w s. */
typedef struct {
    int32_t n_samples;  /* N per ray, 1..256 */
    uint32_t seed;      /* stratification seed */
    uint32_t ray_id0;   /* hash id of ray 0 of this call (ray i uses ray_id0 + i) */
    int32_t stratified; /* 1: jittered u_k; 0: u_k = 0.5 */
    int32_t mode;       /* SDG_MODE_RECOMPUTE or SDG_MODE_STORE */
    float bg[3];        /* background colour, weighted by T_N */
} sdg_render_opts;

typedef struct {
    float* rgb;   /* [n][3] device */
    float* depth; /* [n] device */
    float* opac;  /* [n] device */
    float* sem;   /* [n][n_sem] device, or NULL to skip the semantic output */
} sdg_render_out;

/* Forward render of n rays (rays_dev [n][8]).  When ctx is non-NULL, a
 * context for sdg_render_backward is returned; it refers to rays_dev, which
 * must stay unchanged until the backward has run.  In SDG_MODE_STORE the
 * context holds 6 words per sample slot (t, sdf, colour, block index;
 * 32*ceil(N/32) slots per ray, device memory allocated on the grid's stream,
 * freed by sdg_ctx_release); the backward then re-reads no voxel values.  Errors: SDG_ERR_ARG, SDG_ERR_OOM,
 * SDG_ERR_CUDA. */
int sdg_render_forward(sdg_grid g, const float* rays_dev, int64_t n, const sdg_render_opts* opts,
                       const sdg_render_out* out, sdg_ctx* ctx);

/* Backward of sdg_render_forward: given dL/d(rgb, depth, opac, sem) per ray
 * (device, [n][3], [n], [n], [n][n_sem]; depth/opac/sem may be NULL = 0),
 * ACCUMULATES (+=) dL/dtheta into the grid's gradient channels:
 *   dL/dtau_k = T_{k+1} v_k - sum_{j>k} w_j v_j - T_N (g_rgb . bg),
 *   v_k = g_rgb . c_k + g_depth t_k + g_opac + g_sem . s_k,
 *   dL/dd_k = delta_k sigma'(d_k) dL/dtau_k,  dL/dc_k = w_k g_rgb,  dL/ds_k = w_k g_sem,
 * each scattered to the 8 voxels with the trilinear weights (Eq. 17). */
int sdg_render_backward(sdg_ctx ctx, const float* g_rgb_dev, const float* g_depth_dev, const float* g_opac_dev,
                        const float* g_sem_dev);

/* Debug export of where a render placed every sample (Sec. 3.5.1: the
 * allocated stretches, S, and the samples t_k mapped back from skip space;
 * Eq. 17: the trilinear cell of each sample).  It runs the forward pass with
 * the same traversal and placement code as the other passes and writes, for
 * each ray i (row i of rays_dev) and sample k, to device buffers:
 *   n_cells [n]      allocated block cells in the ray's traversal record, or -1
 *                    when the ray crossed more than SDG_TRACE_CELLS of them
 *                    (rendered from up to twice as many records two per lane,
 *                    beyond that walked in-warp) or walk = SDG_WALK_IN_WARP;
 *   S [n]            total allocated length (0: the ray meets no block);
 *   t [n][N]         ray parameter t_k of sample k;
 *   cell [n][N][3]   voxel coordinates of the base corner of the sample's cell
 *                    (floor of x / voxel_size, decided in FP32);
 *   block [n][N]     index of the block holding that corner, -1 if none;
 *   valid [n][N]     1 if all 8 corners of the cell are allocated;
 *   seg [n][SDG_TRACE_CELLS][2]  (may be NULL) t_in and length of each
 *                    recorded cell, in order (first n_cells[i] entries);
 *   rgb, depth, opac forward outputs, as sdg_render_forward.
 * Samples of a ray with S = 0 read t = 0, cell = 0, block = -1, valid = 0.
 * walk: SDG_WALK_PASS (the traversal pass used by sdg_render_forward,
 * sdg_render_backward, the training passes and the serving loop) or
 * SDG_WALK_IN_WARP (the in-warp traversal used by the allocation-free pass and
 * for the rays that cross more than 2 * SDG_TRACE_CELLS allocated cells).
 * Asynchronous on the grid's stream.  Errors: SDG_ERR_ARG (null or
 * misaligned buffer, bad walk), SDG_ERR_OOM, SDG_ERR_CUDA. */
#define SDG_TRACE_CELLS 32
#define SDG_WALK_PASS 0
#define SDG_WALK_IN_WARP 1
typedef struct {
    int32_t* n_cells;
    float* S;
    float* t;
    int32_t* cell;
    int32_t* block;
    uint8_t* valid;
    float* seg;
    float *rgb, *depth, *opac;
} sdg_trace_out;
int sdg_debug_trace(sdg_grid g, const float* rays_dev, int64_t n, const sdg_render_opts* opts, int32_t walk,
                    const sdg_trace_out* out);

/* Same export for the H x W pinhole view that the serving loop renders for a
 * request (K = {fx, fy, cx, cy}, T row-major 3x4 camera-to-world, host
 * arrays; pixel (u, v) is ray v * W + u, its direction normalised): the rays
 * are formed by the serving kernels' own code (ray id = pixel index; the
 * options' ray_id0 is not used) and walked by the traversal pass as the
 * serving loop walks them, so the outputs equal the served request's bit for
 * bit.  rays_out [H*W][8] (device) receives the rays {o, tnear, d, tfar}. */
int sdg_debug_trace_view(sdg_grid g, int32_t H, int32_t W, const float K[4], const float T[12], float tnear,
                         float tfar, const sdg_render_opts* opts, float* rays_out_dev, const sdg_trace_out* out);

/* Releases a context (enqueues the release of its device memory).  Safe on NULL. */
int sdg_ctx_release(sdg_ctx ctx);

/* Loss weights.  Eq. 12-13 and the supplement's hyper-parameters
 * (lambda_d = 0.1); the colour loss is L1 per channel, the depth loss L1 on
 * metric depth (scale a = 1, shift b = 0), and the semantic loss the squared
 * L2 of rendered logits (following the L2 label fusion of Eq. 11), weighted
 * lambda_s. */
typedef struct {
    float lambda_depth; /* 0.1 */
    float lambda_sem;   /* 0.1 */
    int32_t ray_order;  /* SDG_ORDER_*; used by sdg_train_step_rays only */
    int32_t learn_beta; /* sdg_train_step_rays: also accumulate dL/dbeta (see below) */
    int64_t norm_rays;  /* the n of the means "over rays" in the training passes; 0 = the call's own ray count.
                           A data-parallel step that splits a batch of M rays over ranks passes M, so that the
                           ranks' gradients sum to the whole batch's */
    int32_t prepared;   /* sdg_train_step_rays: 0, or 1 + the slot sdg_train_prepare prepared these rays in */
    int32_t reserved;   /* must be 0 */
} sdg_loss_opts;

/* Prepares a training batch ahead (the paper has no counterpart; a scheduling aid): enqueues the ray
 * ordering (lo->ray_order, as sdg_train_step_rays would apply it) and the traversal pass of these n rays on the
 * grid's auxiliary stream, into preparation slot `slot` (0 or 1), after everything already enqueued on the
 * grid's stream.  The next sdg_train_step_rays of the same rays_dev and n with lo->prepared = slot + 1 uses them
 * and waits for them on the grid's stream.  Issued after one step's training pass and before its optimiser step,
 * the next batch's traversal (issue-bound) runs beside the optimiser (HBM-bound).  The rays and t_depth must not
 * change before that call; preparing a slot again replaces its batch.  Per-ray results are those of an
 * unprepared call.  Errors: SDG_ERR_ARG (bad slot or size, null argument), SDG_ERR_OOM, SDG_ERR_CUDA. */
int sdg_train_prepare(sdg_grid g, const float* rays_dev, int64_t n, const float* t_depth_dev,
                      const sdg_loss_opts* lo, int32_t slot);

/* Learnable Laplace scale (beta of Sec. 3.5.1 as a parameter, as VolSDF
 * learns it).  With lo->learn_beta set, sdg_train_step_rays also accumulates
 *   dL/dbeta = sum_k dL/dtau_k delta_k dsigma_k/dbeta
 *            = -(1/beta) sum_k dL/dtau_k (tau_k + d_k delta_k dsigma_k/dd)
 * (sigma = Psi(-d/beta)/beta, so dsigma/dbeta = -sigma/beta - (d/beta) dsigma/dd)
 * into a grid-owned device scalar; the next sdg_adam_step reads it back (the
 * one host synchronisation such a step needs), updates beta on the host with
 * the same optimiser, hyper-parameters and step index as the voxels (moments
 * kept in the grid and in checkpoints), clamps beta >= 1e-3 voxel sizes and
 * zeroes the scalar.  sdg_grid_beta_grad reads the pending gradient
 * (synchronises); sdg_grid_get_beta / sdg_grid_set_beta read and set beta. */
int sdg_grid_get_beta(sdg_grid g, float* beta);
int sdg_grid_set_beta(sdg_grid g, float beta);
int sdg_grid_beta_grad(sdg_grid g, float* grad);

/* Order in which sdg_train_step_rays processes a batch's rays.  The result of
 * each ray (its samples, its loss term, its gradient contributions) does not
 * depend on the order; only the order of the floating-point gradient
 * accumulation, which is unordered in every mode, and the speed do.
 *   SDG_ORDER_AUTO    surface order for batches of at least 65536 rays,
 *                     the given order below that;
 *   SDG_ORDER_GIVEN   the rays' order in rays_dev;
 *   SDG_ORDER_SURFACE rays grouped by the coarse cell (4x4x4 blocks, Morton
 *                     order) that holds their target surface point
 *                     o + t_depth d, so that rays updating the same voxels
 *                     run together and their gradient updates meet in L2.
 *                     Rays with a non-finite or non-positive target depth go
 *                     last.  Needs a grid-owned scratch of 8 bytes per ray
 *                     plus 128 KiB, grown on demand. */
#define SDG_ORDER_AUTO 0
#define SDG_ORDER_GIVEN 1
#define SDG_ORDER_SURFACE 2

/* Per-ray loss and gradient seeds for n rays:
 *   loss_i = sum_c |rgb - t_rgb| / (3n) + lambda_d |depth - t_depth| / n + lambda_s ||sem - t_sem||^2 / n
 *   g_rgb = sign(rgb - t_rgb) / (3n), g_depth = lambda_d sign(depth - t_depth) / n,
 *   g_sem = 2 lambda_s (sem - t_sem) / n,  sign(0) = 0.
 * sem/t_sem/g_sem may be NULL (no semantic term).  loss_dev [n] per-ray
 * terms (may be NULL). */
int sdg_loss_l1(sdg_grid g, int64_t n, const float* rgb_dev, const float* depth_dev, const float* sem_dev,
                const float* t_rgb_dev, const float* t_depth_dev, const float* t_sem_dev, const sdg_loss_opts* lo,
                float* g_rgb_dev, float* g_depth_dev, float* g_sem_dev, float* loss_dev);

/* The fused training pass with the normal loss of Eq. 14 added:
 *   N_i = sum_k w_k grad f(x_k)  (the rendered normal; grad f in closed form,
 *         Eq. 17, from the same 8 corner values as f; world frame, unnormalised)
 *   loss_i += lambda_normal |N_i - N^_i|_1 / (3n),  dL/dN = lambda_normal sign(N - N^) / (3n)
 * The normal seeds enter the backward twice: through the weights
 * (v_k += g_N . grad f(x_k)) and through grad f itself (the SDF of each
 * corner e gains w_k g_N . grad_x r(x_k, x_e)).  t_normal_dev [n][3] world-
 * frame target normals (e.g. a monocular normal prior rotated to the world);
 * the paper uses lambda_normal = 0.05.  Other arguments as
 * sdg_train_step_rays; grids with logits and lo->learn_beta are not
 * supported here (SDG_ERR_ARG). */
int sdg_train_step_rays_normal(sdg_grid g, const float* rays_dev, int64_t n, const float* t_rgb_dev,
                               const float* t_depth_dev, const float* t_normal_dev, const sdg_render_opts* opts,
                               const sdg_loss_opts* lo, float lambda_normal, float* loss_dev, float* loss_sum_dev);

/* Scale- and shift-invariant depth loss (Eq. 13 with the per-batch least
 * squares scale a and shift b of MiDaS): (a, b) = argmin sum_i (a t_i + b - D_i)^2
 * over the n rays (t = target depth, D = rendered depth), from FP64 sums in a
 * fixed order (deterministic); targets without spread leave the scale
 * undetermined and give a = 1, b = mean(D - t).
 *   loss_i = (lambda / n) (D_i - a t_i - b)^2,  g_depth_i = 2 lambda (D_i - a t_i - b) / n
 * (at the optimum dL/da = dL/db = 0, so the dependence of a and b on D adds
 * nothing).  depth_dev, t_depth_dev [n]; g_depth_dev [n], loss_dev [n],
 * loss_sum_dev [1] may each be NULL; ab (host, 2 doubles, may be NULL)
 * receives (a, b) and makes the call synchronise.  Use with
 * sdg_render_forward / sdg_render_backward (g_depth as the depth seed). */
int sdg_loss_depth_ssi(sdg_grid g, int64_t n, const float* depth_dev, const float* t_depth_dev, float lambda,
                       float* g_depth_dev, float* loss_dev, float* loss_sum_dev, double* ab);

/* One fused training pass (forward, sdg_loss_l1 and backward of the same
 * rays in a single kernel; no per-sample state leaves the SM): accumulates
 * the gradients and writes the per-ray loss terms to loss_dev [n] (may be
 * NULL) and their sum to loss_sum_dev [1] (may be NULL; deterministic
 * reduction).  t_sem_dev may be NULL when the grid has no semantics or the
 * semantic term is not wanted.  opts->mode is ignored.  lo->ray_order picks
 * the processing order (SDG_ORDER_*); an unknown value is SDG_ERR_ARG. */
int sdg_train_step_rays(sdg_grid g, const float* rays_dev, int64_t n, const float* t_rgb_dev,
                        const float* t_depth_dev, const float* t_sem_dev, const sdg_render_opts* opts,
                        const sdg_loss_opts* lo, float* loss_dev, float* loss_sum_dev);

/* Allocation-free variant of sdg_train_step_rays (the paper has no
 * counterpart; this is a deployment aid).  Some callers cannot let the
 * library allocate device memory: processes whose whole device-memory budget
 * is owned by another allocator, and latency-critical loops that cannot
 * afford cudaMalloc/cudaFree, which synchronise the device.
 * sdg_train_step_rays allocates a per-ray loss buffer the first time only the
 * summed loss is requested; this entry point instead keeps that scratch in a
 * fixed array built into the library (4 MiB, held on every GPU that loads
 * the library until the process exits) and calls no allocating routine.
 * Same arguments and results as sdg_train_step_rays without loss_dev: the
 * gradients accumulate into the grid and loss_sum_dev [1] (may be NULL)
 * receives the summed loss.  lo->ray_order is ignored: the rays run in the
 * given order (surface ordering would need a further scratch).
 * lo->learn_beta must be 0 (dL/dbeta needs a per-ray partial buffer):
 * SDG_ERR_ARG otherwise.  n may be at most 1048576 rays; larger n returns
 * SDG_ERR_CAPACITY before any work is enqueued.  The first call on each
 * device looks up the array's device address (a one-time set-up); make that
 * first call before any stream capture.  Every call on a device shares the
 * one array and overwrites its first n entries before reading them, so calls
 * whose work overlaps on the GPU (other streams or host threads) race: order
 * them on one stream or serialise them. */
int sdg_train_step_rays_noalloc(sdg_grid g, const float* rays_dev, int64_t n, const float* t_rgb_dev,
                                const float* t_depth_dev, const float* t_sem_dev, const sdg_render_opts* opts,
                                const sdg_loss_opts* lo, float* loss_sum_dev);

/* ----------------------------------------------------------------------- */
/* Optimiser                                                                */
/* ----------------------------------------------------------------------- */

/* Sec. 3.5.4 optimises theta_d, theta_c, theta_s with RMSProp at learning
 * rate 1e-3; Adam is the default here (SDG_OPT_RMSPROP selects RMSProp with
 * alpha = beta2).  One step over every voxel of the active blocks and every
 * trainable channel (SDF, colour, semantics; not the fusion weight), in FP32;
 * BF16 channels are updated in FP32 and rounded to nearest-even on store.
 * Gradients are zeroed.  Adam: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * theta -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 * step <= 0 uses (and increments) the grid's own step counter. */
typedef struct {
    double lr;    /* 1e-3 */
    double beta1; /* 0.9 */
    double beta2; /* 0.999 (RMSProp: alpha, 0.99) */
    double eps;   /* 1e-8 */
    int32_t step;
    int32_t algo; /* SDG_OPT_ADAM or SDG_OPT_RMSPROP */
} sdg_adam_opts;
/* (Hyper-parameters are doubles so that 1 - beta is exact to FP32 rounding;
 * the update itself runs in FP32.) */

int sdg_adam_step(sdg_grid g, const sdg_adam_opts* a);

/* ---------------------------------------------------------------------------
 * Volumetric fusion, Sec. 3.4.2 (Eq. 9-11) with the supplement's truncation
 * psi(x, mu) = min(x, mu): initialises the voxels from RGB-D (+ logit) frames.
 * Every voxel v of every allocated block b (world x = (8b + l) * voxel_size)
 * is associated with each frame i whose pixel it projects into; the decision
 * is taken in FP32 in this exact order (no fused multiply-add):
 *   x_a = (float)(8 b_a + l_a) * voxel_size;  e_a = x_a - t_a
 *   c_j = (R_0j e_0 + R_1j e_1) + R_2j e_2      (camera coordinates, c = R^T (x - t))
 *   kept only if c_2 > 0;  r = 1 / c_2 (correctly rounded);  pu = fx (c_0 r) + cx,
 *   pv = fy (c_1 r) + cy
 *   pixel (floor pu, floor pv) inside the image (pixel centres at +0.5, as in
 *   activation); D = depth there finite and > 0;  o = D - c_2 (the SDF seen
 *   from frame i, positive in front of the surface); kept only if o >= -mu
 *   (farther behind the surface is occlusion);  psi = min(o, mu).
 * The least-squares solutions of Eq. 9-11 are averages over the kept
 * associations: SDF = mean psi, colour = mean pixel colour, logits
 * s* = mean pixel logits and theta_s = s* / |s*| (Eq. 11).  They are kept as
 * running means with the association count in the WEIGHT channel, so frames
 * may be fused over any number of calls: theta' = (w theta + sum) / (w + n).
 * Where the running means live until sdg_fuse_finalize:
 *   SDF: the SDF value channel (FP32 in both layouts);
 *   colour: the RGB value channel in the SDG_F32 layout; for SDG_BF16 the FP32
 *     colour gradient channel, rounded into the BF16 value channel by
 *     sdg_fuse_finalize;
 *   logits: the FP32 semantic gradient channel; sdg_fuse_finalize writes
 *     theta_s (rounded to BF16) into the semantic value channel.
 * Fusion therefore precedes training: finalize (which zeroes those gradient
 * channels) before the first training pass.  Colour and logits should be given
 * on every call or on none, since the count is shared.
 *   F frames of H x W pixels; depth_dev [F][H][W] float z-depth (m);
 *   rgb_dev [F][H][W][3] float or NULL; sem_dev [F][H][W][n_sem] float logits
 *   or NULL (SDG_ERR_ARG if the grid has no semantic channel);
 *   K (host) [F][4] fx, fy, cx, cy (fx, fy > 0); Twc (host) [F][12] row-major
 *   3x4 camera-to-world [R | t]; mu > 0 the truncation distance (m).
 * Asynchronous on the grid's stream; the host arrays may be reused on return.
 * Voxels with no kept association are not written. */
int sdg_fuse_frames(sdg_grid g, int64_t F, int32_t H, int32_t W, const float* depth_dev, const float* rgb_dev,
                    const float* sem_dev, const float* K, const float* Twc, float mu);

/* ---------------------------------------------------------------------------
 * SDF and its gradient at points, in one pass (Sec. 3.5.2, Eq. 16-17):
 *   f(x) = sum_i r(x, x_i) theta_d(x_i),  grad f(x) = sum_i grad_x r(x, x_i) theta_d(x_i)
 * over the 8 grid points x_i of the voxel cell holding x; r is the trilinear
 * weight, whose derivative along an axis is +-1/voxel_size times the other two
 * axes' factors.  The cell is floor(x * (1/voxel_size)) in FP32.
 *   xyz_dev [n][3] float points; sdf_dev [n] and grad_dev [n][3] float outputs
 *   (either may be NULL).  A point whose 8 grid points are not all allocated
 *   (or outside the block-key range, or NaN) gets NaN.  Asynchronous. */
int sdg_query(sdg_grid g, const float* xyz_dev, int64_t n, float* sdf_dev, float* grad_dev);

/* Eikonal regulariser (Sec. 3.5.3) at n points:
 *   L = (lambda / n) * sum_k (|grad f(x_k)| - 1)^2, invalid points contributing 0,
 * and its gradient with respect to the stored SDF values,
 *   dL/dtheta_d(x_i) = (lambda / n) 2 (|grad f| - 1) (grad f / |grad f|) . grad_x r(x, x_i)
 * (0 where |grad f| < 1e-4: in a flat, e.g. truncated, region the direction
 * of grad f is rounding noise), ADDED into the SDF gradient channel (the SDF lane of
 * the FP32 gradient record, or the SDF gradient array of the BF16 layout) with
 * atomics.  terms_dev [n] receives the per-point terms (may be NULL);
 * loss_sum_dev [1] their sum (may be NULL; deterministic reduction).  The
 * points are the caller's: surface samples, uniform samples in the allocated
 * blocks, or both, as the paper combines them.  Asynchronous. */
int sdg_eikonal(sdg_grid g, const float* xyz_dev, int64_t n, float lambda, float* terms_dev, float* loss_sum_dev);

/* ---------------------------------------------------------------------------
 * Continuous CRF message passing (Sec. 3.5.3, Eq. 19-22): the Gaussian edge
 * potential's sum over all sample points is evaluated with a permutohedral
 * lattice (Adams, Baek and Davis 2010) on a hash map of lattice points.
 *   elevation: x = (d+1) sqrt(2/3) sum_i p_i u_i on the hyperplane sum x = 0 of
 *     R^(d+1), u_i = (1, .., 1, -i, 0, ..) / sqrt(i (i+1)), computed in FP64 in
 *     a fixed order (the lattice point set is exactly that of an FP64 evaluation);
 *   splat onto the d + 1 vertices of the enclosing simplex (barycentric weights);
 *   blur along each of the d + 1 lattice directions with [1 2 1]/4 over the
 *     splatted lattice points; slice back with the same weights.
 * out = slice(blur(splat(val))), divided by the same filter of ones when
 * normalize is set (a Gaussian-weighted mean of unit standard deviation in the
 * scaled features, to a few per cent).
 *   pos_dev [n][d] float features already divided by their standard deviations
 *   (the paper concatenates positions, colours, normals and logits), 1 <= d <= 16;
 *   val_dev [n][c], out_dev [n][c] float, 1 <= c <= 64.  n_lattice (host, may be
 *   NULL) receives the number of lattice points.  Uses grid-owned scratch and the
 *   grid's stream; synchronises once (the lattice size sizes the blur).
 * SDG_ERR_ARG for non-finite or out-of-range features; a 64-bit fingerprint
 * collision between distinct lattice points is detected and reported. */
int sdg_lattice_filter(sdg_grid g, int64_t n, int32_t d, const float* pos_dev, int32_t c, const float* val_dev,
                       float* out_dev, int32_t normalize, int64_t* n_lattice);

/* CRF losses (Sec. 3.5.3, Eq. 22 reads "L_prop = D_f(x_prop || Q(x_prop))"):
 * the divergence between a property at surface points and its CRF
 * message-passed value, the latter a fixed target (e.g. from
 * sdg_crf_meanfield for labels, or a normalised sdg_lattice_filter of the
 * colours / normals):
 *   prop 0, labels: (lambda/n) sum_i KL(Q_i || softmax(s(x_i))), s the
 *     trilinear logits; dL/ds_i = (lambda/n)(softmax(s_i) - Q_i);
 *     target [n][n_sem] distributions (SDG_ERR_ARG without logits);
 *   prop 1, colour: (lambda/n) sum_i |c(x_i) - t_i|^2, target [n][3];
 *   prop 2, normal: (lambda/n) sum_i |grad f(x_i) - t_i|^2, target [n][3]
 *     (grad f of Eq. 17).
 * The gradients are ADDED to the matching gradient channel through the
 * trilinear weights (their x-gradients for the normal); points whose 8 grid
 * points are not all allocated contribute 0.  terms_dev [n] (may be NULL),
 * loss_sum_dev [1] (may be NULL; deterministic).  Asynchronous. */
int sdg_crf_loss(sdg_grid g, int32_t prop, int64_t n, const float* xyz_dev, const float* target_dev, float lambda,
                 float* terms_dev, float* loss_sum_dev);

/* One mean-field update of per-point label distributions with a Potts
 * compatibility (Eq. 22, after Krahenbuhl and Koltun 2011): with F the
 * (unnormalised) lattice filter above and Qt = F(Q) - Q,
 *   E_i(l) = U_i(l) + w (sum_l' Qt_i(l') - Qt_i(l)),   Q_i^+ = softmax(-E_i).
 * unary_dev, q_dev, q_out_dev [n][L] float, 1 <= L <= 64. */
int sdg_crf_meanfield(sdg_grid g, int64_t n, int32_t d, const float* pos_dev, int32_t L, const float* unary_dev,
                      const float* q_dev, float w, float* q_out_dev);

/* Ends a fusion: for every voxel with a non-zero weight writes the BF16
 * colour (SDG_BF16 layout) and theta_s = s* / |s*| (grids with logits) into
 * the value channels, then zeroes the FP32 accumulators (colour and semantic
 * gradient channels).  No-op for an SDG_F32 grid without logits. */
int sdg_fuse_finalize(sdg_grid g);

/* ----------------------------------------------------------------------- */
/* Serving: continuous batching of render requests over several grids       */
/* ----------------------------------------------------------------------- */

/* Inference rendering (Sec. 4.2, colour and depth of whole images) as a
 * service.  A host scheduler thread admits requests while slots and the
 * device-memory budget allow, splits each into ray chunks, and launches
 * batches that mix chunks of different requests, resolutions and scenes on
 * several streams, so batches overlap on the device.  A request's result
 * does not depend on what it was batched with: every ray is computed by the
 * same per-ray code, from its own pixel index (a traversal pass over the
 * batch, then the records kernels -- one record per lane up to
 * SDG_TRACE_CELLS allocated cells, two up to twice that -- and rays crossing
 * more walked in-warp).  Besides the output pool the server holds
 * traversal records for max_batch_rays rays per stream: 8 + 40 *
 * SDG_TRACE_CELLS + 8 bytes a ray (about 340 MB per stream at 2^18 rays). */
typedef struct {
    int64_t hbm_budget_bytes; /* device memory for in-flight outputs (the server allocates it once) */
    int32_t max_slots;        /* requests in flight at once, >= 1 */
    int32_t n_streams;        /* 1..8 */
    int32_t chunk_rays;       /* rays per chunk, multiple of 32 */
    int32_t max_batch_rays;   /* rays per launch, multiple of chunk_rays */
    int32_t device;
    int32_t reserved;
} sdg_server_opts;

typedef struct {
    int32_t scene_id;  /* from sdg_server_add_scene */
    int32_t H, W;      /* image size */
    float K[4];        /* fx, fy, cx, cy */
    float Twc[12];     /* row-major camera-to-world; ray of pixel (u, v) has direction
                          normalize(R ((u+0.5-cx)/fx, (v+0.5-cy)/fy, 1)), origin Twc[:,3] */
    int32_t n_samples; /* samples per ray */
    uint32_t seed;     /* stratification seed; ray id = pixel index v*W + u */
    int32_t stratified;
    float tnear, tfar;
} sdg_request;

typedef struct {
    int32_t status;     /* SDG_OK when done */
    int32_t H, W;
    const float* rgb;   /* device [H*W][3], owned by the server until sdg_server_release */
    const float* depth; /* device [H*W] */
    const float* opac;  /* device [H*W] */
    double t_submit_ms; /* host clock (monotonic, ms) */
    double t_admit_ms;
    double t_done_ms;   /* when the scheduler saw the last chunk complete */
} sdg_result;

typedef struct {
    int64_t submitted, admitted, completed, launches, rays_rendered;
    int64_t bytes_in_use, peak_bytes_in_use;
    int32_t in_flight, queued;
} sdg_server_stats;

int sdg_server_create(const sdg_server_opts* o, sdg_server* out);
/* Registers a grid (not owned).  All scenes of a server must share rgb_dtype
 * and n_sem (SDG_ERR_ARG otherwise).  Not allowed once requests exist.  From
 * registration until sdg_server_destroy the grid's block structure is fixed:
 * activation calls and sdg_grid_destroy on it return SDG_ERR_BUSY (the
 * scheduler reads the block tables of every scene at any time).  Calls that
 * change voxel values (training, fusion, optimiser steps, set_beta) remain
 * allowed and memory-safe, but race with batches in flight: a request may
 * render old or new values. */
int sdg_server_add_scene(sdg_server s, sdg_grid g, int32_t* scene_id);
/* Queues a request; SDG_ERR_CAPACITY if its outputs can never fit the budget. */
int sdg_server_submit(sdg_server s, const sdg_request* q, uint64_t* ticket);
/* Non-blocking: SDG_OK and a filled result when done, SDG_ERR_BUSY before. */
int sdg_server_poll(sdg_server s, uint64_t ticket, sdg_result* r);
/* Blocks up to timeout_ms (host clock); SDG_ERR_TIMEOUT if not done by then. */
int sdg_server_wait(sdg_server s, uint64_t ticket, int64_t timeout_ms, sdg_result* r);
/* Frees a completed request's outputs; cancels a queued one. */
int sdg_server_release(sdg_server s, uint64_t ticket);
int sdg_server_get_stats(sdg_server s, sdg_server_stats* st);
/* Waits for in-flight work, stops the scheduler, frees everything. */
int sdg_server_destroy(sdg_server s);

/* Test support (no counterpart in the paper): from now on, the n-th device
 * allocation made by grid creation, activation or loading fails as if the
 * device were out of memory (n = 0: the next one; n < 0: switch off).  Used
 * to check that every such failure returns SDG_ERR_OOM and leaks nothing. */
int sdg_debug_fail_alloc_after(int64_t n);

/* Thread-local message of the calling thread's last error ("" if none). */
const char* sdg_last_error(void);

/* Library version string. */
const char* sdg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SDG_H */
