// Surface ordering of a training batch.  Rays are grouped by the coarse cell
// (4x4x4 blocks) holding the surface point o + t_depth d that their target
// depth names, the cells taken in Morton order; rays that update the same
// voxels then run in the same wave of warps, so their gradient updates and
// voxel reads meet in L2 instead of each missing to DRAM.  The rendering and
// the loss of a ray do not change: the fused pass reads ray perm[i] in warp
// slot i and keeps the ray's own index for its samples and outputs.
//
// Counting sort over at most 2^15 buckets: per-ray bucket and histogram in
// one pass, an exclusive scan of the histogram in one block, and a scatter
// in which each warp claims the places of its rays with one atomic per
// distinct bucket.  The order of rays within a bucket is not fixed.
#include <algorithm>

#include "internal.h"

namespace sdg {
namespace {

constexpr int kThreads = 256;

// Spreads the low 10 bits of v to bits 0, 3, 6, ... (Morton interleave).
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
    v &= 0x3FFu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

struct OrderParams {
    float inv_L;
    int bmin[3], bdim[3];
    int cshift;  // block coordinate -> coarse cell coordinate (>= 2)
    int bshift;  // Morton code -> bucket
    int last;    // bucket of rays without a usable target depth
};

__device__ __forceinline__ int surface_bucket(const OrderParams& p, const float4 r0, const float4 r1, float D) {
    if (!(D > 0.f) || !(D < 3.0e38f)) return p.last;  // NaN, inf, <= 0
    const float x[3] = {fmaf(D, r1.x, r0.x), fmaf(D, r1.y, r0.y), fmaf(D, r1.z, r0.z)};
    uint32_t c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float b = floorf(x[a] * p.inv_L) - (float)p.bmin[a];
        b = fminf(fmaxf(b, 0.f), (float)(p.bdim[a] - 1));  // also maps a NaN coordinate to 0
        c[a] = (uint32_t)b >> p.cshift;
    }
    const uint32_t m = spread3(c[0]) | (spread3(c[1]) << 1) | (spread3(c[2]) << 2);
    return (int)(m >> p.bshift);
}

// Adds `count` to *counter once per distinct value of `key` in the active lanes; returns the counter's value
// before this warp's addition plus the calling lane's rank among the lanes with its key.
__device__ __forceinline__ int warp_claim(int* counter_base, int key) {
    const unsigned active = __activemask();
    const unsigned peers = __match_any_sync(active, key);
    const int leader = __ffs(peers) - 1;
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == leader) base = atomicAdd(counter_base + key, __popc(peers));
    base = __shfl_sync(peers, base, leader);
    return base + __popc(peers & ((1u << lane) - 1u));
}

__global__ void k_surface_keys(const float* __restrict__ rays, const float* __restrict__ tdepth, int64_t n,
                               OrderParams p, int* __restrict__ keys, int* __restrict__ hist) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 r0 = __ldg(reinterpret_cast<const float4*>(rays) + 2 * i);
    const float4 r1 = __ldg(reinterpret_cast<const float4*>(rays) + 2 * i + 1);
    const int k = surface_bucket(p, r0, r1, __ldg(tdepth + i));
    keys[i] = k;
    warp_claim(hist, k);
}

// In-place exclusive scan of hist[0, kOrderBuckets) by one block of 1024 threads: the counts are staged in
// shared memory with coalesced 16-byte loads, each warp scans its contiguous 1/32 of the buckets 32 at a time,
// and the warps' totals are scanned by warp 0 and added on the way back out.
__global__ void __launch_bounds__(1024) k_scan_buckets(int* hist) {
    extern __shared__ int4 sh4[];
    __shared__ int wsum[32];
    int* sh = reinterpret_cast<int*>(sh4);
    int4* h4 = reinterpret_cast<int4*>(hist);
    constexpr int kV = kOrderBuckets / 4 / 1024;  // int4 per thread
    constexpr int kSeg = kOrderBuckets / 32;      // buckets per warp
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    int4 v[kV];
#pragma unroll
    for (int q = 0; q < kV; ++q) v[q] = h4[q * 1024 + t];
#pragma unroll
    for (int q = 0; q < kV; ++q) sh4[q * 1024 + t] = v[q];
    __syncthreads();
    int carry = 0;
    for (int r = 0; r < kSeg / 32; ++r) {
        int* p = sh + w * kSeg + r * 32 + lane;
        const int x = *p;
        int inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int nb = __shfl_up_sync(0xFFFFFFFFu, inc, o);
            if (lane >= o) inc += nb;
        }
        *p = carry + inc - x;
        carry += __shfl_sync(0xFFFFFFFFu, inc, 31);
    }
    if (lane == 0) wsum[w] = carry;
    __syncthreads();
    if (w == 0) {
        const int x = wsum[lane];
        int inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int nb = __shfl_up_sync(0xFFFFFFFFu, inc, o);
            if (lane >= o) inc += nb;
        }
        wsum[lane] = inc - x;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kV; ++q) {
        const int i4 = q * 1024 + t;
        int4 a = sh4[i4];
        const int off = wsum[(i4 * 4) / kSeg];
        a.x += off;
        a.y += off;
        a.z += off;
        a.w += off;
        h4[i4] = a;
    }
}

__global__ void k_scatter_rays(const int* __restrict__ keys, int64_t n, int* offs, int* __restrict__ perm) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    perm[warp_claim(offs, __ldg(keys + i))] = (int)i;
}

int bit_length(uint32_t v) { return v ? 32 - __builtin_clz(v) : 0; }

}  // namespace

int order_rays_into(sdg_grid g, BatchBufs& b, cudaStream_t st, const float* rays, const float* tdepth, int64_t n,
                    const int** perm) {
    *perm = nullptr;
    if (g->n_blocks == 0 || n == 0) return SDG_OK;
    if (n > ((int64_t)1 << 31) - 1) return fail(SDG_ERR_ARG, "surface ordering: at most 2^31 - 1 rays");
    if (b.order_cap < n) {
        if (b.order_keys || b.order_perm) {
            int rc = drain_streams(g);  // earlier work may still read them
            if (rc) return rc;
        }
        if (b.order_keys) cudaFree(b.order_keys);
        if (b.order_perm) cudaFree(b.order_perm);
        b.order_keys = b.order_perm = nullptr;
        b.order_cap = 0;
        SDG_CUDA_TRY(cudaMalloc((void**)&b.order_keys, sizeof(int) * n));
        SDG_CUDA_TRY(cudaMalloc((void**)&b.order_perm, sizeof(int) * n));
        b.order_cap = n;
    }
    if (!b.order_hist) SDG_CUDA_TRY(cudaMalloc((void**)&b.order_hist, sizeof(int) * kOrderBuckets));

    OrderParams p{};
    p.inv_L = 1.0f / (8.0f * g->desc.voxel_size);
    int maxc = 0;
    for (int a = 0; a < 3; ++a) {
        p.bmin[a] = g->bmin[a];
        p.bdim[a] = g->bdim[a];
    }
    p.cshift = 2;
    for (;;) {  // coarse coordinates must fit the 10 bits per axis of the Morton code
        maxc = 0;
        for (int a = 0; a < 3; ++a) maxc = std::max(maxc, (g->bdim[a] - 1) >> p.cshift);
        if (maxc < 1024) break;
        ++p.cshift;
    }
    const int bits = 3 * bit_length((uint32_t)maxc);
    p.bshift = bits > 15 ? bits - 15 : 0;
    const int used = 1 << (bits - p.bshift);  // buckets that Morton codes can reach
    p.last = used < kOrderBuckets ? used : kOrderBuckets - 1;

    const unsigned blocks = (unsigned)((n + kThreads - 1) / kThreads);
    SDG_CUDA_TRY(cudaMemsetAsync(b.order_hist, 0, sizeof(int) * kOrderBuckets, st));
    k_surface_keys<<<blocks, kThreads, 0, st>>>(rays, tdepth, n, p, b.order_keys, b.order_hist);
    SDG_LAUNCH_CHECK("surface keys");
    SDG_CUDA_TRY(cudaFuncSetAttribute(k_scan_buckets, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(sizeof(int) * kOrderBuckets)));  // per device, so set on every call
    k_scan_buckets<<<1, 1024, sizeof(int) * kOrderBuckets, st>>>(b.order_hist);
    SDG_LAUNCH_CHECK("bucket scan");
    k_scatter_rays<<<blocks, kThreads, 0, st>>>(b.order_keys, n, b.order_hist, b.order_perm);
    SDG_LAUNCH_CHECK("ray scatter");
    *perm = b.order_perm;
    return SDG_OK;
}

int order_rays_by_surface(sdg_grid g, const float* rays, const float* tdepth, int64_t n, const int** perm) {
    return order_rays_into(g, g->batch, g->stream, rays, tdepth, n, perm);
}

}  // namespace sdg
