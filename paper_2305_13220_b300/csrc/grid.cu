// Grid life cycle, block activation (Sec. 3.4.1, Eq. 7-8), hash lookups, the
// neighbour table and dense block-index grid derived from the hash map, and
// checkpointing.  Paper: arXiv 2305.13220.
#include <atomic>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace sdg {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}
int cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SDG_ERR_OOM : SDG_ERR_CUDA;
}
int use_device(sdg_grid g) {
    SDG_CUDA_TRY(cudaSetDevice(g->device));
    return SDG_OK;
}

// Host-side fault injection for tests: the n-th device allocation made by grid creation or activation from
// now on fails with cudaErrorMemoryAllocation (n < 0: off).
static std::atomic<long long> g_fail_alloc_countdown{-1};

cudaError_t device_malloc(void** p, size_t bytes) {
    long long c = g_fail_alloc_countdown.load();
    if (c >= 0) {
        if (g_fail_alloc_countdown.fetch_sub(1) == 0) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
    }
    return cudaMalloc(p, bytes);
}

}  // namespace sdg

extern "C" int sdg_debug_fail_alloc_after(int64_t n) {
    sdg::g_fail_alloc_countdown.store(n < 0 ? -1 : n);
    return SDG_OK;
}

using namespace sdg;

extern "C" const char* sdg_last_error(void) { return g_last_error.c_str(); }
extern "C" const char* sdg_version(void) { return "sdg 0.1 (sm_103a)"; }

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------
namespace {

constexpr int kThreads = 256;
// Largest block capacity: the render and query kernels form voxel addresses (block * 512 + local) in 32 bits.
constexpr int64_t kMaxBlocks = 1ll << 22;

__device__ __forceinline__ int floordiv8(int v) { return v >> 3; }  // arithmetic shift = floor division

// Records candidate block key `key` in the de-duplication set unless it is
// already active.  counters[0] counts keys new to this batch; counters[1] is
// the overflow flag.
__device__ __forceinline__ void offer_key(uint64_t key, const ulonglong2* table, uint32_t mask, ulonglong2* tmp,
                                          unsigned long long* counters, unsigned long long room) {
    if (sdg_table_find_rw(table, mask, key) >= 0) return;
    if (counters[0] > room) {  // cannot fit anyway: stop filling the set
        counters[1] = 1;
        return;
    }
    int r = sdg_table_insert(tmp, mask, key, 0);
    if (r == 1) atomicAdd(counters, 1ull);
    if (r < 0) counters[1] = 1;
}

// Eq. 7: all blocks touched by the voxel cube v + [-r, r]^3 of one voxel v.
__device__ __forceinline__ void offer_voxel_cube(int vx, int vy, int vz, int r, const ulonglong2* table,
                                                 uint32_t mask, ulonglong2* tmp, unsigned long long* counters,
                                                 unsigned long long room) {
    int x0 = floordiv8(vx - r), x1 = floordiv8(vx + r);
    int y0 = floordiv8(vy - r), y1 = floordiv8(vy + r);
    int z0 = floordiv8(vz - r), z1 = floordiv8(vz + r);
    for (int z = z0; z <= z1; ++z)
        for (int y = y0; y <= y1; ++y)
            for (int x = x0; x <= x1; ++x) offer_key(sdg_pack_key(x, y, z), table, mask, tmp, counters, room);
}

// v = floor(x * inv_vs) in FP32; false if the point is unusable.
__device__ __forceinline__ bool quantise(float x, float inv_vs, int* v) {
    float q = __fmul_rn(x, inv_vs);
    if (!isfinite(q) || fabsf(q) > 8.0e6f) return false;
    *v = (int)floorf(q);
    return true;
}

__global__ void k_candidates_points(const float* __restrict__ xyz, int64_t n, float inv_vs, int r,
                                    const ulonglong2* table, uint32_t mask, ulonglong2* tmp,
                                    unsigned long long* counters, unsigned long long room) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int v[3];
        bool ok = true;
        for (int a = 0; a < 3; ++a) ok = quantise(xyz[3 * i + a], inv_vs, &v[a]) && ok;
        if (ok) offer_voxel_cube(v[0], v[1], v[2], r, table, mask, tmp, counters, room);
    }
}

struct Cam {
    float fx_inv, fy_inv, cx, cy;
    float T[12];
};

// Eq. 8 (phi = 1), FP32 with the operation order stated in sdg.h; every
// operation is an explicitly rounded intrinsic, so no multiply-add is fused.
__global__ void k_candidates_depth(const float* __restrict__ depth, int H, int W, Cam cam, float inv_vs, int r,
                                   const ulonglong2* table, uint32_t mask, ulonglong2* tmp,
                                   unsigned long long* counters, unsigned long long room) {
    int64_t n = (int64_t)H * W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float d = depth[i];
        if (!(isfinite(d) && d > 0.0f)) continue;
        int u;
        const int v = (int)sdg_divmod(i, W, u);
        float xc = __fmul_rn(__fmul_rn(__fadd_rn(__fadd_rn((float)u, 0.5f), -cam.cx), cam.fx_inv), d);
        float yc = __fmul_rn(__fmul_rn(__fadd_rn(__fadd_rn((float)v, 0.5f), -cam.cy), cam.fy_inv), d);
        float zc = d;
        int q[3];
        bool ok = true;
        for (int a = 0; a < 3; ++a) {
            float p0 = __fmul_rn(cam.T[a * 4 + 0], xc);
            float p1 = __fmul_rn(cam.T[a * 4 + 1], yc);
            float p2 = __fmul_rn(cam.T[a * 4 + 2], zc);
            float x = __fadd_rn(__fadd_rn(__fadd_rn(p0, p1), p2), cam.T[a * 4 + 3]);
            ok = quantise(x, inv_vs, &q[a]) && ok;
        }
        if (ok) offer_voxel_cube(q[0], q[1], q[2], r, table, mask, tmp, counters, room);
    }
}

__global__ void k_candidates_keys(const int32_t* __restrict__ keys, int64_t n, const ulonglong2* table, uint32_t mask,
                                  ulonglong2* tmp, unsigned long long* counters, unsigned long long room) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int x = keys[3 * i], y = keys[3 * i + 1], z = keys[3 * i + 2];
        if (x < -SDG_KEY_BIAS || x >= SDG_KEY_BIAS || y < -SDG_KEY_BIAS || y >= SDG_KEY_BIAS || z < -SDG_KEY_BIAS ||
            z >= SDG_KEY_BIAS) {
            counters[3] = 1;  // bad key
            continue;
        }
        offer_key(sdg_pack_key(x, y, z), table, mask, tmp, counters, room);
    }
}

// Moves the keys of the de-duplication set to a list and empties the set.
__global__ void k_compact(ulonglong2* tmp, uint32_t cap, uint64_t* out, unsigned long long* counter) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x) {
        uint64_t k = tmp[i].x;
        if (k != SDG_EMPTY_KEY) {
            unsigned long long p = atomicAdd(counter, 1ull);
            out[p] = k;
            tmp[i].x = SDG_EMPTY_KEY;
            tmp[i].y = 0;
        }
    }
}

__global__ void k_fill_u64(uint64_t* a, int64_t from, int64_t to, uint64_t v) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = from + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < to; i += stride)
        a[i] = v;
}

// Bitonic sort (ascending) of a power-of-two array.  Direction of a
// compare-exchange is set by bit k of the global index, so the shared-memory
// stages and the global stages compose into one sorting network.
constexpr int kSortTile = 2048;

__device__ __forceinline__ void cmp_swap(uint64_t& a, uint64_t& b, bool asc) {
    if ((a > b) == asc) {
        uint64_t t = a;
        a = b;
        b = t;
    }
}

// All stages k <= 2048 inside one tile.
__global__ void k_bitonic_tile_sort(uint64_t* a) {
    __shared__ uint64_t s[kSortTile];
    const uint32_t base = blockIdx.x * kSortTile;
    for (int i = threadIdx.x; i < kSortTile; i += blockDim.x) s[i] = a[base + i];
    __syncthreads();
    for (uint32_t k = 2; k <= kSortTile; k <<= 1)
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < kSortTile; i += blockDim.x) {
                uint32_t ixj = i ^ j;
                if (ixj > i) cmp_swap(s[i], s[ixj], ((base + i) & k) == 0);
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < kSortTile; i += blockDim.x) a[base + i] = s[i];
}

// One global stage (k, j) with j >= 2048.
__global__ void k_bitonic_global(uint64_t* a, uint32_t n, uint32_t j, uint32_t k) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t ixj = i ^ j;
    if (ixj > i) {
        uint64_t x = a[i], y = a[ixj];
        if ((x > y) == ((i & k) == 0)) {
            a[i] = y;
            a[ixj] = x;
        }
    }
}

// Stages j = 1024 .. 1 of one k > 2048, inside one tile.
__global__ void k_bitonic_tile_merge(uint64_t* a, uint32_t k) {
    __shared__ uint64_t s[kSortTile];
    const uint32_t base = blockIdx.x * kSortTile;
    for (int i = threadIdx.x; i < kSortTile; i += blockDim.x) s[i] = a[base + i];
    __syncthreads();
    for (uint32_t j = kSortTile >> 1; j > 0; j >>= 1) {
        for (uint32_t i = threadIdx.x; i < kSortTile; i += blockDim.x) {
            uint32_t ixj = i ^ j;
            if (ixj > i) cmp_swap(s[i], s[ixj], ((base + i) & k) == 0);
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < kSortTile; i += blockDim.x) a[base + i] = s[i];
}

__global__ void k_minmax(const uint64_t* __restrict__ list, int64_t n, int* mm) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int3 k = sdg_unpack_key(list[i]);
        atomicMin(mm + 0, k.x);
        atomicMin(mm + 1, k.y);
        atomicMin(mm + 2, k.z);
        atomicMax(mm + 3, k.x);
        atomicMax(mm + 4, k.y);
        atomicMax(mm + 5, k.z);
    }
}

// Inserts list[i] with block index base + i (keys are unique and absent).
__global__ void k_insert(const uint64_t* __restrict__ list, int64_t n, int64_t base, ulonglong2* table, uint32_t mask,
                         int4* keys, unsigned long long* counters) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = list[i];
        if (sdg_table_insert(table, mask, k, (uint64_t)(base + i)) != 1) counters[4] = 1;
        int3 c = sdg_unpack_key(k);
        keys[base + i] = make_int4(c.x, c.y, c.z, 0);
    }
}

__global__ void k_keys_to_list(const int4* __restrict__ keys, int64_t n, uint64_t* list) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int4 k = keys[i];
        list[i] = sdg_pack_key(k.x, k.y, k.z);
    }
}

// Dense block-index grid over the block AABB: cell (x, y, z) holds the index of that block (-1 elsewhere), so
// the traversal reads occupancy and block index with one load per cell.
__global__ void k_dense(const int4* __restrict__ keys, int64_t n, int bx, int by, int bz, int dx, int dy,
                        int32_t* dense) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int4 k = keys[i];
        int64_t cell = ((int64_t)(k.z - bz) * dy + (k.y - by)) * (int64_t)dx + (k.x - bx);
        dense[cell] = (int32_t)i;
    }
}

// nbr[b] = block indices of b + {0, x, y, xy, z, xz, yz, xyz} (bit 0 = +x, bit 1 = +y, bit 2 = +z).
__global__ void k_neighbours(const int4* __restrict__ keys, int64_t n, const ulonglong2* table, uint32_t mask,
                             int4* nbr) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
        int4 k = keys[b];
        int v[8];
        v[0] = (int)b;
        for (int m = 1; m < 8; ++m)
            v[m] = sdg_table_find_rw(table, mask, sdg_pack_key(k.x + (m & 1), k.y + ((m >> 1) & 1), k.z + (m >> 2)));
        nbr[2 * b] = make_int4(v[0], v[1], v[2], v[3]);
        nbr[2 * b + 1] = make_int4(v[4], v[5], v[6], v[7]);
    }
}

__global__ void k_lookup(const int32_t* __restrict__ keys, int64_t n, const ulonglong2* table, uint32_t mask,
                         int32_t* idx) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int x = keys[3 * i], y = keys[3 * i + 1], z = keys[3 * i + 2];
        bool ok = x >= -SDG_KEY_BIAS && x < SDG_KEY_BIAS && y >= -SDG_KEY_BIAS && y < SDG_KEY_BIAS &&
                  z >= -SDG_KEY_BIAS && z < SDG_KEY_BIAS;
        idx[i] = ok ? sdg_table_find(table, mask, sdg_pack_key(x, y, z)) : -1;
    }
}

__global__ void k_keys_out(const int4* __restrict__ keys, int64_t n, int32_t* out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int4 k = keys[i];
        out[3 * i] = k.x;
        out[3 * i + 1] = k.y;
        out[3 * i + 2] = k.z;
    }
}

int grid_blocks(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    if (b > 148 * 32) b = 148 * 32;
    return (int)b;
}

uint64_t next_pow2(uint64_t v) {
    uint64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

template <class T>
int dalloc(T** p, size_t count, cudaStream_t s) {
    if (count == 0) {
        *p = nullptr;
        return SDG_OK;
    }
    SDG_CUDA_TRY(device_malloc((void**)p, count * sizeof(T)));
    SDG_CUDA_TRY(cudaMemsetAsync(*p, 0, count * sizeof(T), s));
    return SDG_OK;
}

void free_grid_buffers(sdg_grid g) {
    void* ptrs[] = {g->table, g->tmp_table, g->keys, g->nbr, g->dense, g->geo, g->ggeo, g->m_geo, g->v_geo,
                    g->sdf, g->gsdf, g->m_sdf, g->v_sdf, g->rgbh, g->grgb, g->m_rgb, g->v_rgb, g->sem, g->gsem,
                    g->m_sem, g->v_sem, g->weight, g->sort_buf, g->counters, g->minmax, g->loss_buf, g->sum_scratch,
                    g->fuse_cams, g->beta_grad, g->beta_part,
                    g->ssi_dev, g->lat.fp, g->lat.idx, g->lat.skey, g->lat.keys, g->lat.vidx, g->lat.vbary,
                    g->lat.val0, g->lat.val1, g->lat.nb, g->lat.counters, g->lat.fq, g->lat.sr, g->lat.srank,
                    g->lat.vslot, g->lat.fp2};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    free_batch(g->batch);
    for (PreparedBatch& pb : g->prep) {
        free_batch(pb.b);
        if (pb.fence) cudaEventDestroy(pb.fence);
        if (pb.ready) cudaEventDestroy(pb.ready);
    }
    if (g->aux) cudaStreamDestroy(g->aux);
    if (g->h_counters) cudaFreeHost(g->h_counters);
    if (g->h_minmax) cudaFreeHost(g->h_minmax);
    if (g->h_over) cudaFreeHost(g->h_over);
}

// Sorts sort_buf[0, n) ascending (pads to a power of two >= 2048 with all-ones).
int sort_keys(sdg_grid g, int64_t n) {
    uint64_t np = next_pow2((uint64_t)n);
    if (np < (uint64_t)kSortTile) np = kSortTile;
    if ((int64_t)np > g->sort_cap) return fail(SDG_ERR_CAPACITY, "sort buffer too small");
    k_fill_u64<<<grid_blocks(np - n), kThreads, 0, g->stream>>>(g->sort_buf, n, (int64_t)np, ~0ull);
    uint32_t tiles = (uint32_t)(np / kSortTile);
    k_bitonic_tile_sort<<<tiles, 1024, 0, g->stream>>>(g->sort_buf);
    for (uint32_t k = 2 * kSortTile; k <= np; k <<= 1) {
        for (uint32_t j = k >> 1; j >= (uint32_t)kSortTile; j >>= 1)
            k_bitonic_global<<<(uint32_t)((np + kThreads - 1) / kThreads), kThreads, 0, g->stream>>>(
                g->sort_buf, (uint32_t)np, j, k);
        k_bitonic_tile_merge<<<tiles, 1024, 0, g->stream>>>(g->sort_buf, k);
    }
    SDG_LAUNCH_CHECK("bitonic sort");
    return SDG_OK;
}

// Makes the dense block-index grid hold at least `cells` cells (the old contents are not kept).
int reserve_dense(sdg_grid g, int64_t cells) {
    if (cells <= g->dense_cap) return SDG_OK;
    int32_t* nd = nullptr;
    SDG_CUDA_TRY(device_malloc((void**)&nd, cells * sizeof(int32_t)));
    if (g->dense) cudaFree(g->dense);
    g->dense = nd;
    g->dense_cap = cells;
    return SDG_OK;
}

// Recomputes the AABB (from all keys), the dense block-index grid and the neighbour table.
int rebuild_derived(sdg_grid g) {
    const int64_t N = g->n_blocks;
    if (N == 0) {
        for (int a = 0; a < 3; ++a) g->bmin[a] = g->bdim[a] = 0;
        g->dense_cells = 0;
        return SDG_OK;
    }
    int init[6] = {INT32_MAX, INT32_MAX, INT32_MAX, INT32_MIN, INT32_MIN, INT32_MIN};
    std::memcpy(g->h_minmax, init, sizeof(init));
    SDG_CUDA_TRY(cudaMemcpyAsync(g->minmax, g->h_minmax, sizeof(init), cudaMemcpyHostToDevice, g->stream));
    k_keys_to_list<<<grid_blocks(N), kThreads, 0, g->stream>>>(g->keys, N, g->sort_buf);
    k_minmax<<<grid_blocks(N), kThreads, 0, g->stream>>>(g->sort_buf, N, g->minmax);
    SDG_LAUNCH_CHECK("minmax");
    SDG_CUDA_TRY(cudaMemcpyAsync(g->h_minmax, g->minmax, sizeof(init), cudaMemcpyDeviceToHost, g->stream));
    SDG_CUDA_TRY(cudaStreamSynchronize(g->stream));
    int64_t cells = 1;
    for (int a = 0; a < 3; ++a) {
        g->bmin[a] = g->h_minmax[a];
        g->bdim[a] = g->h_minmax[3 + a] - g->h_minmax[a] + 1;
        cells *= g->bdim[a];
    }
    int rc = reserve_dense(g, cells);
    if (rc) return rc;
    g->dense_cells = cells;
    SDG_CUDA_TRY(cudaMemsetAsync(g->dense, 0xFF, cells * sizeof(int32_t), g->stream));
    k_dense<<<grid_blocks(N), kThreads, 0, g->stream>>>(g->keys, N, g->bmin[0], g->bmin[1], g->bmin[2], g->bdim[0],
                                                        g->bdim[1], g->dense);
    k_neighbours<<<grid_blocks(N), kThreads, 0, g->stream>>>(g->keys, N, g->table, g->mask, g->nbr);
    SDG_LAUNCH_CHECK("block index/neighbours");
    return SDG_OK;
}

// Largest block AABB the dense block-index grid may cover (cells; 4 bytes each).
constexpr int64_t kMaxDenseCells = 1ll << 31;

// Second half of every activation: the candidate kernel has filled tmp_table and counters.
int finish_activation(sdg_grid g, int64_t* n_new) {
    SDG_LAUNCH_CHECK("activation candidates");
    SDG_CUDA_TRY(cudaMemcpyAsync(g->h_counters, g->counters, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                 g->stream));
    SDG_CUDA_TRY(cudaStreamSynchronize(g->stream));
    unsigned long long cnt = g->h_counters[0];
    bool overflow = g->h_counters[1] != 0;
    bool bad_key = g->h_counters[3] != 0;
    auto clear_tmp = [&]() -> int {
        SDG_CUDA_TRY(cudaMemsetAsync(g->tmp_table, 0xFF, (size_t)g->cap * sizeof(ulonglong2), g->stream));
        return SDG_OK;
    };
    if (bad_key) {
        int rc = clear_tmp();
        return rc ? rc : fail(SDG_ERR_ARG, "activation: block key outside [-2^20, 2^20)");
    }
    if (overflow || (int64_t)cnt > g->max_blocks - g->n_blocks) {
        int rc = clear_tmp();
        if (rc) return rc;
        return fail(SDG_ERR_CAPACITY, "activation would exceed max_blocks (" + std::to_string(g->max_blocks) +
                                          "); grid unchanged");
    }
    if (n_new) *n_new = (int64_t)cnt;
    if (cnt == 0) return SDG_OK;
    // compact + sort the new keys; the set is emptied by the compaction
    SDG_CUDA_TRY(cudaMemsetAsync(g->counters + 2, 0, sizeof(unsigned long long), g->stream));
    k_compact<<<grid_blocks(g->cap), kThreads, 0, g->stream>>>(g->tmp_table, g->cap, g->sort_buf, g->counters + 2);
    SDG_LAUNCH_CHECK("compact");
    int rc = sort_keys(g, (int64_t)cnt);
    if (rc) return rc;
    // the AABB of old + new keys must stay within the block-index grid's limit (checked before any insertion)
    int init[6] = {INT32_MAX, INT32_MAX, INT32_MAX, INT32_MIN, INT32_MIN, INT32_MIN};
    if (g->n_blocks > 0)
        for (int a = 0; a < 3; ++a) {
            init[a] = g->bmin[a];
            init[3 + a] = g->bmin[a] + g->bdim[a] - 1;
        }
    std::memcpy(g->h_minmax, init, sizeof(init));
    SDG_CUDA_TRY(cudaMemcpyAsync(g->minmax, g->h_minmax, sizeof(init), cudaMemcpyHostToDevice, g->stream));
    k_minmax<<<grid_blocks(cnt), kThreads, 0, g->stream>>>(g->sort_buf, (int64_t)cnt, g->minmax);
    SDG_CUDA_TRY(cudaMemcpyAsync(g->h_minmax, g->minmax, sizeof(init), cudaMemcpyDeviceToHost, g->stream));
    SDG_CUDA_TRY(cudaStreamSynchronize(g->stream));
    int64_t cells = 1;
    for (int a = 0; a < 3; ++a) cells *= (int64_t)g->h_minmax[3 + a] - g->h_minmax[a] + 1;
    if (cells > kMaxDenseCells)
        return fail(SDG_ERR_CAPACITY, "activation: block bounding box exceeds 2^31 blocks; grid unchanged");
    // every allocation happens before the first insertion, so a failure leaves the grid unchanged
    rc = reserve_dense(g, cells);
    if (rc) return rc;
    k_insert<<<grid_blocks(cnt), kThreads, 0, g->stream>>>(g->sort_buf, (int64_t)cnt, g->n_blocks, g->table, g->mask,
                                                            g->keys, g->counters);
    SDG_LAUNCH_CHECK("insert");
    // the insertion status comes back with the synchronisation the rebuild already makes
    SDG_CUDA_TRY(cudaMemcpyAsync(g->h_counters + 4, g->counters + 4, sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, g->stream));
    g->n_blocks += (int64_t)cnt;
    rc = rebuild_derived(g);
    if (rc) return rc;
    // A probe sequence that met no empty slot: impossible at a load factor <= 0.5 (every sequence ends at an
    // empty slot), reported rather than assumed.
    if (g->h_counters[4] != 0) return fail(SDG_ERR_CAPACITY, "activation: hash table full during insertion");
    return SDG_OK;
}

Cam make_cam(const float K[4], const float T[12]) {
    Cam cam;
    cam.fx_inv = 1.0f / K[0];
    cam.fy_inv = 1.0f / K[1];
    cam.cx = K[2];
    cam.cy = K[3];
    for (int i = 0; i < 12; ++i) cam.T[i] = T[i];
    return cam;
}

// Called with g->mu held.
int begin_activation(sdg_grid g) {
    if (!g) return fail(SDG_ERR_ARG, "null grid");
    if (g->served)
        return fail(SDG_ERR_BUSY, "activation: the grid is registered with a server, whose batches read its block "
                                  "structure at any time; destroy the server first");
    int rc = use_device(g);
    if (rc) return rc;
    SDG_CUDA_TRY(cudaMemsetAsync(g->counters, 0, 8 * sizeof(unsigned long long), g->stream));
    return SDG_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------
extern "C" int sdg_grid_create(const sdg_grid_desc* d, sdg_grid* out) {
    if (!d || !out) return fail(SDG_ERR_ARG, "sdg_grid_create: null argument");
    *out = nullptr;
    if (!(d->voxel_size > 0.f) || d->max_blocks <= 0 || d->max_blocks > kMaxBlocks ||
        (d->rgb_dtype != SDG_F32 && d->rgb_dtype != SDG_BF16) || d->n_sem < 0 || d->n_sem > 32 || d->n_sem % 4 ||
        d->reserved != 0)
        return fail(SDG_ERR_ARG, "sdg_grid_create: invalid descriptor");
    sdg_grid g = new (std::nothrow) sdg_grid_s();
    if (!g) return fail(SDG_ERR_OOM, "host allocation");
    g->desc = *d;
    g->device = d->device;
    g->stream = (cudaStream_t)d->stream;
    g->max_blocks = d->max_blocks;
    g->beta = d->beta > 0.f ? d->beta : 0.5f * d->voxel_size;
    g->cap = (uint32_t)next_pow2((uint64_t)(2 * d->max_blocks));
    if (g->cap < 1024) g->cap = 1024;
    g->mask = g->cap - 1;
    int rc = SDG_OK;
    auto run = [&]() -> int {
        SDG_CUDA_TRY(cudaSetDevice(g->device));
        cudaStream_t s = g->stream;
        const size_t V = (size_t)g->max_blocks * 512;
        SDG_CUDA_TRY(device_malloc((void**)&g->table, (size_t)g->cap * sizeof(ulonglong2)));
        SDG_CUDA_TRY(device_malloc((void**)&g->tmp_table, (size_t)g->cap * sizeof(ulonglong2)));
        SDG_CUDA_TRY(cudaMemsetAsync(g->table, 0xFF, (size_t)g->cap * sizeof(ulonglong2), s));
        SDG_CUDA_TRY(cudaMemsetAsync(g->tmp_table, 0xFF, (size_t)g->cap * sizeof(ulonglong2), s));
        int r;
        if ((r = dalloc(&g->keys, g->max_blocks, s))) return r;
        if ((r = dalloc(&g->nbr, 2 * g->max_blocks, s))) return r;
        if (d->rgb_dtype == SDG_F32) {
            if ((r = dalloc(&g->geo, V, s)) || (r = dalloc(&g->ggeo, V, s)) || (r = dalloc(&g->m_geo, V, s)) ||
                (r = dalloc(&g->v_geo, V, s)))
                return r;
        } else {
            if ((r = dalloc(&g->sdf, V, s)) || (r = dalloc(&g->gsdf, V, s)) || (r = dalloc(&g->m_sdf, V, s)) ||
                (r = dalloc(&g->v_sdf, V, s)) || (r = dalloc(&g->rgbh, V, s)) || (r = dalloc(&g->grgb, V, s)) ||
                (r = dalloc(&g->m_rgb, V, s)) || (r = dalloc(&g->v_rgb, V, s)))
                return r;
        }
        if (d->n_sem) {
            size_t S = V * d->n_sem;
            if ((r = dalloc(&g->sem, S, s)) || (r = dalloc(&g->gsem, S, s)) || (r = dalloc(&g->m_sem, S, s)) ||
                (r = dalloc(&g->v_sem, S, s)))
                return r;
        }
        if ((r = dalloc(&g->weight, V, s))) return r;
        g->sort_cap = (int64_t)next_pow2((uint64_t)g->max_blocks);
        if (g->sort_cap < kSortTile) g->sort_cap = kSortTile;
        if ((r = dalloc(&g->sort_buf, g->sort_cap, s))) return r;
        if ((r = dalloc(&g->counters, 8, s))) return r;
        if ((r = dalloc(&g->sum_scratch, kSumBlocks + 1, s))) return r;
        if ((r = dalloc(&g->minmax, 6, s))) return r;
        if ((r = dalloc(&g->beta_grad, 1, s))) return r;
        if ((r = dalloc(&g->ssi_dev, 2, s))) return r;
        SDG_CUDA_TRY(cudaMallocHost((void**)&g->h_counters, 8 * sizeof(unsigned long long)));
        SDG_CUDA_TRY(cudaMallocHost((void**)&g->h_minmax, 6 * sizeof(int)));
        SDG_CUDA_TRY(cudaMallocHost((void**)&g->h_over, 2 * sizeof(int)));
        g->h_over[0] = g->h_over[1] = 0;
        SDG_CUDA_TRY(cudaStreamSynchronize(s));
        return SDG_OK;
    };
    rc = run();
    if (rc) {
        std::string msg = g_last_error;
        free_grid_buffers(g);
        delete g;
        return fail(rc, msg);
    }
    *out = g;
    return SDG_OK;
}

extern "C" int sdg_grid_destroy(sdg_grid g) {
    if (!g) return SDG_OK;
    {
        std::lock_guard<std::mutex> lk(g->mu);
        if (g->served) return fail(SDG_ERR_BUSY, "sdg_grid_destroy: the grid is registered with a server");
    }
    cudaSetDevice(g->device);
    cudaStreamSynchronize(g->stream);
    if (g->aux) cudaStreamSynchronize(g->aux);
    free_grid_buffers(g);
    delete g;
    return SDG_OK;
}

extern "C" int sdg_grid_activate_points(sdg_grid g, const float* xyz, int64_t n, int32_t r, int64_t* n_new) {
    if (n_new) *n_new = 0;
    if (!g || (n > 0 && !xyz) || n < 0 || r < 0 || r > 64) return fail(SDG_ERR_ARG, "sdg_grid_activate_points");
    std::lock_guard<std::mutex> lk(g->mu);
    int rc = begin_activation(g);
    if (rc) return rc;
    const float inv_vs = 1.0f / g->desc.voxel_size;
    if (n > 0)
        k_candidates_points<<<grid_blocks(n), kThreads, 0, g->stream>>>(
            xyz, n, inv_vs, r, g->table, g->mask, g->tmp_table, g->counters,
            (unsigned long long)(g->max_blocks - g->n_blocks));
    return finish_activation(g, n_new);
}

extern "C" int sdg_grid_activate_depth(sdg_grid g, const float* depth, int32_t H, int32_t W, const float K[4],
                                       const float T[12], int32_t r, int64_t* n_new) {
    if (n_new) *n_new = 0;
    if (!g || !depth || !K || !T || H <= 0 || W <= 0 || r < 0 || r > 64 || !(K[0] != 0.f) || !(K[1] != 0.f))
        return fail(SDG_ERR_ARG, "sdg_grid_activate_depth");
    std::lock_guard<std::mutex> lk(g->mu);
    int rc = begin_activation(g);
    if (rc) return rc;
    const float inv_vs = 1.0f / g->desc.voxel_size;
    k_candidates_depth<<<grid_blocks((int64_t)H * W), kThreads, 0, g->stream>>>(
        depth, H, W, make_cam(K, T), inv_vs, r, g->table, g->mask, g->tmp_table, g->counters,
        (unsigned long long)(g->max_blocks - g->n_blocks));
    return finish_activation(g, n_new);
}

// All frames' candidates go into the one de-duplication set, then a single compaction, sort and insertion: one
// activation batch (new blocks indexed in ascending packed-key order over the whole batch), one synchronisation.
extern "C" int sdg_grid_activate_depth_frames(sdg_grid g, const float* depth, int32_t F, int32_t H, int32_t W,
                                              const float* K, const float* T, int32_t r, int64_t* n_new) {
    if (n_new) *n_new = 0;
    if (!g || F < 0 || (F > 0 && (!depth || !K || !T)) || H <= 0 || W <= 0 || r < 0 || r > 64)
        return fail(SDG_ERR_ARG, "sdg_grid_activate_depth_frames");
    for (int32_t f = 0; f < F; ++f)
        if (!(K[4 * f] != 0.f) || !(K[4 * f + 1] != 0.f))
            return fail(SDG_ERR_ARG, "sdg_grid_activate_depth_frames: fx and fy must be non-zero");
    std::lock_guard<std::mutex> lk(g->mu);
    int rc = begin_activation(g);
    if (rc) return rc;
    const float inv_vs = 1.0f / g->desc.voxel_size;
    const unsigned long long room = (unsigned long long)(g->max_blocks - g->n_blocks);
    const int64_t HW = (int64_t)H * W;
    for (int32_t f = 0; f < F; ++f)
        k_candidates_depth<<<grid_blocks(HW), kThreads, 0, g->stream>>>(
            depth + f * HW, H, W, make_cam(K + 4 * f, T + 12 * f), inv_vs, r, g->table, g->mask, g->tmp_table,
            g->counters, room);
    return finish_activation(g, n_new);
}

extern "C" int sdg_grid_activate_keys(sdg_grid g, const int32_t* keys, int64_t n, int64_t* n_new) {
    if (n_new) *n_new = 0;
    if (!g || (n > 0 && !keys) || n < 0) return fail(SDG_ERR_ARG, "sdg_grid_activate_keys");
    std::lock_guard<std::mutex> lk(g->mu);
    int rc = begin_activation(g);
    if (rc) return rc;
    if (n > 0) {
        const unsigned long long room = (unsigned long long)(g->max_blocks - g->n_blocks);
        k_candidates_keys<<<grid_blocks(n), kThreads, 0, g->stream>>>(keys, n, g->table, g->mask, g->tmp_table,
                                                                      g->counters, room);
    }
    return finish_activation(g, n_new);
}

extern "C" int sdg_grid_num_blocks(sdg_grid g, int64_t* n) {
    if (!g || !n) return fail(SDG_ERR_ARG, "sdg_grid_num_blocks");
    std::lock_guard<std::mutex> lk(g->mu);
    int rc = use_device(g);
    if (rc) return rc;
    SDG_CUDA_TRY(cudaStreamSynchronize(g->stream));
    *n = g->n_blocks;
    return SDG_OK;
}

extern "C" int sdg_grid_keys(sdg_grid g, int32_t* out) {
    if (!g || (!out && g->n_blocks)) return fail(SDG_ERR_ARG, "sdg_grid_keys");
    int rc = use_device(g);
    if (rc) return rc;
    if (g->n_blocks) k_keys_out<<<grid_blocks(g->n_blocks), kThreads, 0, g->stream>>>(g->keys, g->n_blocks, out);
    SDG_LAUNCH_CHECK("sdg_grid_keys");
    return SDG_OK;
}

extern "C" int sdg_grid_lookup(sdg_grid g, const int32_t* keys, int64_t n, int32_t* idx) {
    if (!g || n < 0 || (n > 0 && (!keys || !idx))) return fail(SDG_ERR_ARG, "sdg_grid_lookup");
    int rc = use_device(g);
    if (rc) return rc;
    if (n) k_lookup<<<grid_blocks(n), kThreads, 0, g->stream>>>(keys, n, g->table, g->mask, idx);
    SDG_LAUNCH_CHECK("sdg_grid_lookup");
    return SDG_OK;
}

namespace {
struct ChannelInfo {
    void* ptr;
    int64_t elem_bytes;  // per voxel
};

ChannelInfo channel_info(sdg_grid g, int group, int kind) {
    const bool f32 = g->desc.rgb_dtype == SDG_F32;
    const int ns = g->desc.n_sem;
    switch (group) {
        case SDG_GROUP_GEO:
            if (!f32) break;
            if (kind == SDG_KIND_VALUE) return {g->geo, 16};
            if (kind == SDG_KIND_GRAD) return {g->ggeo, 16};
            if (kind == SDG_KIND_ADAM_M) return {g->m_geo, 16};
            if (kind == SDG_KIND_ADAM_V) return {g->v_geo, 16};
            break;
        case SDG_GROUP_SDF:
            if (f32) break;
            if (kind == SDG_KIND_VALUE) return {g->sdf, 4};
            if (kind == SDG_KIND_GRAD) return {g->gsdf, 4};
            if (kind == SDG_KIND_ADAM_M) return {g->m_sdf, 4};
            if (kind == SDG_KIND_ADAM_V) return {g->v_sdf, 4};
            break;
        case SDG_GROUP_RGB:
            if (f32) break;
            if (kind == SDG_KIND_VALUE) return {g->rgbh, 8};
            if (kind == SDG_KIND_GRAD) return {g->grgb, 16};
            if (kind == SDG_KIND_ADAM_M) return {g->m_rgb, 16};
            if (kind == SDG_KIND_ADAM_V) return {g->v_rgb, 16};
            break;
        case SDG_GROUP_SEM:
            if (!ns) break;
            if (kind == SDG_KIND_VALUE) return {g->sem, 2 * ns};
            if (kind == SDG_KIND_GRAD) return {g->gsem, 4 * ns};
            if (kind == SDG_KIND_ADAM_M) return {g->m_sem, 4 * ns};
            if (kind == SDG_KIND_ADAM_V) return {g->v_sem, 4 * ns};
            break;
        case SDG_GROUP_WEIGHT:
            if (kind == SDG_KIND_VALUE) return {g->weight, 4};
            break;
    }
    return {nullptr, 0};
}
}  // namespace

extern "C" int sdg_grid_channel(sdg_grid g, int32_t group, int32_t kind, void** ptr, int64_t* bytes) {
    if (!g || !ptr) return fail(SDG_ERR_ARG, "sdg_grid_channel: null argument");
    ChannelInfo c = channel_info(g, group, kind);
    if (!c.ptr) return fail(SDG_ERR_ARG, "sdg_grid_channel: no such channel in this grid's layout");
    *ptr = c.ptr;
    if (bytes) *bytes = c.elem_bytes * 512 * g->max_blocks;
    return SDG_OK;
}

extern "C" int sdg_grid_zero_grad(sdg_grid g) {
    if (!g) return fail(SDG_ERR_ARG, "null grid");
    int rc = use_device(g);
    if (rc) return rc;
    const size_t V = (size_t)g->n_blocks * 512;
    if (!V) return SDG_OK;
    if (g->ggeo) SDG_CUDA_TRY(cudaMemsetAsync(g->ggeo, 0, V * 16, g->stream));
    if (g->gsdf) SDG_CUDA_TRY(cudaMemsetAsync(g->gsdf, 0, V * 4, g->stream));
    if (g->grgb) SDG_CUDA_TRY(cudaMemsetAsync(g->grgb, 0, V * 16, g->stream));
    if (g->gsem) SDG_CUDA_TRY(cudaMemsetAsync(g->gsem, 0, V * 4 * g->desc.n_sem, g->stream));
    return SDG_OK;
}

extern "C" int sdg_grid_get_step(sdg_grid g, int32_t* step) {
    if (!g || !step) return fail(SDG_ERR_ARG, "sdg_grid_get_step");
    *step = g->step;
    return SDG_OK;
}
extern "C" int sdg_grid_set_step(sdg_grid g, int32_t step) {
    if (!g || step < 0) return fail(SDG_ERR_ARG, "sdg_grid_set_step");
    g->step = step;
    return SDG_OK;
}

extern "C" int sdg_grid_get_beta(sdg_grid g, float* beta) {
    if (!g || !beta) return fail(SDG_ERR_ARG, "sdg_grid_get_beta: null argument");
    *beta = g->beta;
    return SDG_OK;
}

extern "C" int sdg_grid_set_beta(sdg_grid g, float beta) {
    if (!g || !(beta > 0.f)) return fail(SDG_ERR_ARG, "sdg_grid_set_beta: beta must be > 0");
    g->beta = beta;
    return SDG_OK;
}

extern "C" int sdg_grid_beta_grad(sdg_grid g, float* grad) {
    if (!g || !grad) return fail(SDG_ERR_ARG, "sdg_grid_beta_grad: null argument");
    int rc = use_device(g);
    if (rc) return rc;
    SDG_CUDA_TRY(cudaMemcpyAsync(grad, g->beta_grad, sizeof(float), cudaMemcpyDeviceToHost, g->stream));
    SDG_CUDA_TRY(cudaStreamSynchronize(g->stream));
    return SDG_OK;
}

extern "C" int sdg_grid_sync(sdg_grid g) {
    if (!g) return fail(SDG_ERR_ARG, "null grid");
    int rc = use_device(g);
    if (rc) return rc;
    SDG_CUDA_TRY(cudaStreamSynchronize(g->stream));
    return SDG_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint
// ---------------------------------------------------------------------------
namespace {
struct FileHeader {
    char magic[8];  // "SDGGRID2" ("SDGGRID1": the same without the fields after `reserved`)
    float voxel_size, beta;
    int32_t rgb_dtype, n_sem;
    int64_t n_blocks;
    int32_t step, reserved;
    double beta_m, beta_v;  // optimiser moments of the learnable Laplace scale
};
constexpr size_t kHeaderV1 = offsetof(FileHeader, beta_m);

// (group, kind) pairs saved, in file order.
const int kSaved[][2] = {{SDG_GROUP_GEO, SDG_KIND_VALUE},  {SDG_GROUP_GEO, SDG_KIND_GRAD},
                         {SDG_GROUP_GEO, SDG_KIND_ADAM_M}, {SDG_GROUP_GEO, SDG_KIND_ADAM_V},
                         {SDG_GROUP_SDF, SDG_KIND_VALUE},  {SDG_GROUP_SDF, SDG_KIND_GRAD},
                         {SDG_GROUP_SDF, SDG_KIND_ADAM_M}, {SDG_GROUP_SDF, SDG_KIND_ADAM_V},
                         {SDG_GROUP_RGB, SDG_KIND_VALUE},  {SDG_GROUP_RGB, SDG_KIND_GRAD},
                         {SDG_GROUP_RGB, SDG_KIND_ADAM_M}, {SDG_GROUP_RGB, SDG_KIND_ADAM_V},
                         {SDG_GROUP_SEM, SDG_KIND_VALUE},  {SDG_GROUP_SEM, SDG_KIND_GRAD},
                         {SDG_GROUP_SEM, SDG_KIND_ADAM_M}, {SDG_GROUP_SEM, SDG_KIND_ADAM_V},
                         {SDG_GROUP_WEIGHT, SDG_KIND_VALUE}};
}  // namespace

extern "C" int sdg_grid_save(sdg_grid g, const char* path) {
    if (!g || !path) return fail(SDG_ERR_ARG, "sdg_grid_save");
    std::lock_guard<std::mutex> lk(g->mu);
    int rc = use_device(g);
    if (rc) return rc;
    SDG_CUDA_TRY(cudaStreamSynchronize(g->stream));
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(SDG_ERR_IO, std::string("cannot open ") + path);
    FileHeader h{};
    std::memcpy(h.magic, "SDGGRID2", 8);
    h.beta_m = g->beta_m;
    h.beta_v = g->beta_v;
    h.voxel_size = g->desc.voxel_size;
    h.beta = g->beta;
    h.rgb_dtype = g->desc.rgb_dtype;
    h.n_sem = g->desc.n_sem;
    h.n_blocks = g->n_blocks;
    h.step = g->step;
    bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1;
    std::vector<char> buf;
    if (ok && g->n_blocks) {
        buf.resize((size_t)g->n_blocks * sizeof(int4));
        if (cudaMemcpy(buf.data(), g->keys, buf.size(), cudaMemcpyDeviceToHost) != cudaSuccess) ok = false;
        ok = ok && std::fwrite(buf.data(), 1, buf.size(), f) == buf.size();
        for (auto& gk : kSaved) {
            ChannelInfo c = channel_info(g, gk[0], gk[1]);
            if (!c.ptr || !ok) continue;
            buf.resize((size_t)g->n_blocks * 512 * c.elem_bytes);
            if (cudaMemcpy(buf.data(), c.ptr, buf.size(), cudaMemcpyDeviceToHost) != cudaSuccess) ok = false;
            ok = ok && std::fwrite(buf.data(), 1, buf.size(), f) == buf.size();
        }
    }
    ok = (std::fclose(f) == 0) && ok;
    return ok ? SDG_OK : fail(SDG_ERR_IO, std::string("write failed: ") + path);
}

extern "C" int sdg_grid_load(const char* path, const sdg_grid_desc* over, sdg_grid* out) {
    if (!path || !out) return fail(SDG_ERR_ARG, "sdg_grid_load");
    *out = nullptr;
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(SDG_ERR_IO, std::string("cannot open ") + path);
    FileHeader h{};
    bool head = std::fread(&h, kHeaderV1, 1, f) == 1 && h.n_blocks >= 0;
    const bool v2 = head && std::memcmp(h.magic, "SDGGRID2", 8) == 0;
    if (v2) head = std::fread(reinterpret_cast<char*>(&h) + kHeaderV1, sizeof(h) - kHeaderV1, 1, f) == 1;
    if (!head || (!v2 && std::memcmp(h.magic, "SDGGRID1", 8) != 0)) {
        std::fclose(f);
        return fail(SDG_ERR_IO, "not a grid file");
    }
    sdg_grid_desc d{};
    if (over) d = *over;
    d.voxel_size = h.voxel_size;
    d.beta = h.beta;
    d.rgb_dtype = h.rgb_dtype;
    d.n_sem = h.n_sem;
    if (!over) d.max_blocks = h.n_blocks > 0 ? h.n_blocks : 1;
    if (d.max_blocks < h.n_blocks) {
        std::fclose(f);
        return fail(SDG_ERR_CAPACITY, "max_blocks smaller than the stored block count");
    }
    sdg_grid g = nullptr;
    int rc = sdg_grid_create(&d, &g);
    if (rc) {
        std::fclose(f);
        return rc;
    }
    bool ok = true;
    std::vector<char> buf;
    if (h.n_blocks) {
        buf.resize((size_t)h.n_blocks * sizeof(int4));
        ok = std::fread(buf.data(), 1, buf.size(), f) == buf.size();
        ok = ok && cudaMemcpy(g->keys, buf.data(), buf.size(), cudaMemcpyHostToDevice) == cudaSuccess;
        for (auto& gk : kSaved) {
            ChannelInfo c = channel_info(g, gk[0], gk[1]);
            if (!c.ptr || !ok) continue;
            buf.resize((size_t)h.n_blocks * 512 * c.elem_bytes);
            ok = std::fread(buf.data(), 1, buf.size(), f) == buf.size();
            ok = ok && cudaMemcpy(c.ptr, buf.data(), buf.size(), cudaMemcpyHostToDevice) == cudaSuccess;
        }
    }
    std::fclose(f);
    if (!ok) {
        sdg_grid_destroy(g);
        return fail(SDG_ERR_IO, "truncated grid file");
    }
    // re-insert the keys with their stored indices
    if (h.n_blocks) {
        g->n_blocks = 0;
        SDG_CUDA_TRY(cudaMemsetAsync(g->counters, 0, 8 * sizeof(unsigned long long), g->stream));
        k_keys_to_list<<<grid_blocks(h.n_blocks), kThreads, 0, g->stream>>>(g->keys, h.n_blocks, g->sort_buf);
        k_insert<<<grid_blocks(h.n_blocks), kThreads, 0, g->stream>>>(g->sort_buf, h.n_blocks, 0, g->table, g->mask,
                                                                       g->keys, g->counters);
        SDG_LAUNCH_CHECK("load insert");
        g->n_blocks = h.n_blocks;
        rc = rebuild_derived(g);
        if (rc) {
            sdg_grid_destroy(g);
            return rc;
        }
    }
    g->step = h.step;
    g->beta_m = v2 ? h.beta_m : 0.0;
    g->beta_v = v2 ? h.beta_v : 0.0;
    SDG_CUDA_TRY(cudaStreamSynchronize(g->stream));
    *out = g;
    return SDG_OK;
}

// ---------------------------------------------------------------------------
// Bounds-checked build: one status word per device
// ---------------------------------------------------------------------------
#ifdef SDG_CHECKED
namespace {
std::mutex g_checked_mu;
unsigned long long* g_checked_word[64] = {};
}  // namespace
#endif

namespace sdg {
unsigned long long* checked_status_word(int device) {
#ifdef SDG_CHECKED
    if (device < 0 || device >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_checked_mu);
    if (!g_checked_word[device]) {
        unsigned long long* p = nullptr;
        if (cudaMalloc((void**)&p, sizeof(unsigned long long)) != cudaSuccess) return nullptr;
        if (cudaMemset(p, 0, sizeof(unsigned long long)) != cudaSuccess) {
            cudaFree(p);
            return nullptr;
        }
        g_checked_word[device] = p;
    }
    return g_checked_word[device];
#else
    (void)device;
    return nullptr;
#endif
}
}  // namespace sdg

extern "C" int sdg_checked_status(int32_t device, int32_t clear, uint64_t* status, int32_t* checked) {
    if (!status || !checked) return fail(SDG_ERR_ARG, "sdg_checked_status: null argument");
    *status = 0;
#ifdef SDG_CHECKED
    *checked = 1;
    int prev = 0;
    SDG_CUDA_TRY(cudaGetDevice(&prev));
    SDG_CUDA_TRY(cudaSetDevice(device));
    unsigned long long* w = sdg::checked_status_word(device);
    int rc = SDG_OK;
    if (!w) {
        rc = fail(SDG_ERR_OOM, "sdg_checked_status: no status word");
    } else {
        unsigned long long v = 0;
        cudaError_t e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaMemcpy(&v, w, sizeof(v), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && clear) e = cudaMemset(w, 0, sizeof(v));
        if (e != cudaSuccess) rc = cuda_fail(e, "sdg_checked_status");
        *status = v;
    }
    cudaSetDevice(prev);
    return rc;
#else
    (void)device;
    (void)clear;
    *checked = 0;
    return SDG_OK;
#endif
}
