// Host-side grid object shared by the .cu files of libsdg (not part of the ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "render_core.cuh"

// Grid-owned scratch of the permutohedral lattice filter (lattice.cu), grown on demand.
struct LatticeScratch {
    unsigned long long* fp = nullptr;  // slot fingerprints
    unsigned* fp2 = nullptr;           // second slot fingerprints
    int* idx = nullptr;                // slot -> lattice index
    int* skey = nullptr;               // slot -> coordinates
    int* keys = nullptr;               // lattice index -> coordinates
    int* vidx = nullptr;               // point -> vertex lattice indices
    float* vbary = nullptr;            // point -> barycentric weights
    float *val0 = nullptr, *val1 = nullptr;  // lattice values (double buffer)
    int* nb = nullptr;                 // lattice neighbours per direction
    int* counters = nullptr;           // lattice size, status
    float* fq = nullptr;               // mean field: filtered label distributions
    int* sr = nullptr;                 // point -> remainder-0 vertex of its simplex
    signed char* srank = nullptr;      // point -> ranks of its residual
    int* vslot = nullptr;              // point -> table slots of its vertices
    int64_t cap_fp = 0, cap_idx = 0, cap_skey = 0, cap_keys = 0, cap_vidx = 0, cap_vbary = 0, cap_val0 = 0,
            cap_val1 = 0, cap_nb = 0, cap_counters = 0, cap_fq = 0, cap_sr = 0, cap_srank = 0, cap_vslot = 0,
            cap_fp2 = 0;
};

// Per-batch scratch of a pass: the surface ordering of its rays and the records of its traversal pass.
struct BatchBufs {
    int* order_keys = nullptr;  // per-ray bucket [order_cap]
    int* order_perm = nullptr;  // processing order [order_cap]
    int* order_hist = nullptr;  // bucket counts, then offsets [kOrderBuckets]
    int64_t order_cap = 0;
    // traversal records for up to walk_cap rays: header, skip-space offsets, cell records
    int2* walk_hdr = nullptr;
    float* walk_s0 = nullptr;
    int4* walk_rec = nullptr;
    int* walk_over = nullptr;  // overflow list [walk_cap], mid list [walk_cap], their lengths [2] (WalkBufs)
    int64_t walk_cap = 0;
};

// A training batch whose ordering and traversal ran ahead on the auxiliary stream.
struct PreparedBatch {
    BatchBufs b;
    cudaEvent_t fence = nullptr;  // recorded on the grid's stream when the preparation is enqueued
    cudaEvent_t ready = nullptr;  // recorded on the auxiliary stream when the preparation is done
    const float* rays = nullptr;
    int64_t n = 0;
    const int* perm = nullptr;  // NULL: given order
    bool valid = false;
};

namespace sdg {

// Blocks of the deterministic sums (reduce.cuh: k_sum), one per SM.
constexpr int kSumBlocks = 148;
// Device status word of the bounds-checked build (SDG_CHECKED) on `device`, allocated on first use; NULL in the
// normal build.
unsigned long long* checked_status_word(int device);
}  // namespace sdg

struct sdg_grid_s {
    sdg_grid_desc desc;
    cudaStream_t stream = nullptr;
    int device = 0;
    int64_t max_blocks = 0;
    int64_t n_blocks = 0;
    uint32_t cap = 0, mask = 0;  // hash capacity (power of two) and cap - 1
    float beta = 0.f;
    int32_t step = 0;

    // hash map (main) and the de-duplication set used by activation
    ulonglong2* table = nullptr;
    ulonglong2* tmp_table = nullptr;
    int4* keys = nullptr;  // [max_blocks] {x, y, z, 0} in index order
    int4* nbr = nullptr;   // [max_blocks][2]
    int32_t* dense = nullptr;  // block index of every cell of the block AABB (-1: not allocated), x fastest
    int64_t dense_cells = 0, dense_cap = 0;
    int bmin[3] = {0, 0, 0}, bdim[3] = {0, 0, 0};

    // channels
    float4 *geo = nullptr, *ggeo = nullptr, *m_geo = nullptr, *v_geo = nullptr;                  // SDG_F32
    float *sdf = nullptr, *gsdf = nullptr, *m_sdf = nullptr, *v_sdf = nullptr;                   // SDG_BF16
    uint2* rgbh = nullptr;                                                                        // SDG_BF16
    float4 *grgb = nullptr, *m_rgb = nullptr, *v_rgb = nullptr;                                   // SDG_BF16
    __nv_bfloat16* sem = nullptr;
    float *gsem = nullptr, *m_sem = nullptr, *v_sem = nullptr;
    float* weight = nullptr;

    // activation scratch
    uint64_t* sort_buf = nullptr;  // [sort_cap]
    int64_t sort_cap = 0;
    unsigned long long* counters = nullptr;    // device [8]
    unsigned long long* h_counters = nullptr;  // pinned host [8]
    int* minmax = nullptr;                     // device [6]
    int* h_minmax = nullptr;                   // pinned host [6]
    int* h_over = nullptr;  // pinned host [2]: overflow- and mid-list lengths of the last pass (launch hints)
    float* loss_buf = nullptr;                 // per-ray loss scratch of the fused training pass
    float* sum_scratch = nullptr;              // device [kSumBlocks + 1]: partials and ticket of the loss sums
    int64_t loss_cap = 0;
    BatchBufs batch;     // ordering and traversal scratch of the passes enqueued on `stream`
    PreparedBatch prep[2];  // training batches prepared ahead on `aux` (sdg_train_prepare)
    cudaStream_t aux = nullptr;  // auxiliary stream of the preparations, created on first use
    void* fuse_cams = nullptr;  // per-frame cameras of a fusion call [fuse_cam_cap]
    int64_t fuse_cam_cap = 0;
    // learnable Laplace scale: dL/dbeta accumulates on the device until the next optimiser step
    float* beta_grad = nullptr;  // device [1]
    float* beta_part = nullptr;  // per-ray dL/dbeta [beta_part_cap]
    int64_t beta_part_cap = 0;
    bool beta_grad_pending = false;
    double beta_m = 0.0, beta_v = 0.0;  // the scale's optimiser moments
    double ssi_ab[2] = {0.0, 0.0};
    double* ssi_dev = nullptr;  // device [2]: (a, b) of the last scale/shift-invariant depth loss
    LatticeScratch lat;

    cudaEvent_t pass_ev[2] = {nullptr, nullptr};  // recorded around the render kernels of every pass (not owned)
    std::mutex mu;  // serialises host-side mutation (activation, load) of this grid
    int served = 0;  // servers this grid is registered with (under mu): its block structure is then fixed

    GridDev dev() const {
        GridDev d{};
        d.table = table;
        d.nbr = nbr;
        d.dense = dense;
        d.keys = keys;
        d.mask = mask;
        d.n_sem = desc.n_sem;
        for (int a = 0; a < 3; ++a) {
            d.bmin[a] = bmin[a];
            d.bdim[a] = bdim[a];
        }
        d.vs = desc.voxel_size;
        d.inv_vs = 1.0f / desc.voxel_size;
        d.L = 8.0f * desc.voxel_size;
        d.inv_L = 1.0f / d.L;
        d.beta = beta;
        d.inv_beta = 1.0f / beta;
        d.n_blocks = n_blocks;
        d.geo = geo;
        d.ggeo = ggeo;
        d.sdf = sdf;
        d.rgbh = rgbh;
        d.gsdf = gsdf;
        d.grgb = grgb;
        d.sem = sem;
        d.gsem = gsem;
        d.dense_cells = dense_cells;
        d.status = sdg::checked_status_word(device);
        return d;
    }
};

namespace sdg {
// Makes g's device current for the calling thread.
int use_device(sdg_grid g);

// Grid-owned per-item loss scratch of at least n floats (grown on demand; valid until the next call on g).
int loss_scratch(sdg_grid g, int64_t n, float** out);

// Enqueues the traversal pass (k_walk) of n rays, processed in order perm (NULL: as given), into the grid-owned
// walk records and points a.walk at them (render.cu).
int walk_rays(sdg_grid g, const float* rays, const int* perm, int64_t n, PassArgs& a);
// The same into the batch scratch b on stream s (every buffer growth first drains the grid's streams).
int walk_rays_into(sdg_grid g, BatchBufs& b, cudaStream_t s, const float* rays, const int* perm, int64_t n,
                   PassArgs& a);
// Frees a batch scratch (the caller has drained the streams that use it).
void free_batch(BatchBufs& b);
// Blocks until the grid's stream and its auxiliary stream are idle.
int drain_streams(sdg_grid g);

// Buckets of the surface ordering of a training batch (order.cu).
constexpr int kOrderBuckets = 1 << 15;

// Enqueues on g's stream the surface ordering of n training rays (SDG_ORDER_SURFACE) and sets *perm to the
// grid-owned processing order (valid until the next call on this grid).  Sets *perm to NULL, with nothing
// enqueued, when the grid holds no block.
int order_rays_by_surface(sdg_grid g, const float* rays, const float* tdepth, int64_t n, const int** perm);
// The same into the batch scratch b on stream s.
int order_rays_into(sdg_grid g, BatchBufs& b, cudaStream_t s, const float* rays, const float* tdepth, int64_t n,
                    const int** perm);
}  // namespace sdg
