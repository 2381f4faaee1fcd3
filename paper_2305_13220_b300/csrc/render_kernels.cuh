// Render kernel template and its launcher, instantiated per (layout, semantics,
// pass) in the render_inst_*.cu files so that they compile in parallel.
#pragma once

#include <algorithm>

#include "render_core.cuh"

namespace sdg {

// Resident 256-thread blocks per SM requested from the register allocator: three (80 registers) where the
// program fits with no or a few bytes of spill (measured on the room training step: 1.69 -> 1.49 ms), fewer
// for the larger per-lane sample counts and the semantic variants (NSC > 0), which need more registers.
template <int MODE, int NSC, int Q>
constexpr int render_min_blocks() {
#ifdef SDG_RENDER_MIN_BLOCKS
    return SDG_RENDER_MIN_BLOCKS;
#else
    return NSC > 0 ? (Q >= 6 ? 1 : 2) : (MODE == PASS_TRAIN_NRM || Q >= 6 ? 2 : 3);
#endif
}

// Ray of processing slot `slot` (ray perm[slot], or ray slot) into j.
__device__ __forceinline__ void load_job(const GridDev& g, const float* rays, const int* perm, uint32_t ray_id0,
                                         int64_t slot, int64_t n, RayJob& j) {
    int64_t r = perm ? (int64_t)__ldg(perm + slot) : slot;
    if (!sdg_in_range(g.status, r, n, SDG_CHECK_RAY)) r = 0;  // checked build: a bad order row reads ray 0
    const float4 r0 = __ldg(reinterpret_cast<const float4*>(rays) + 2 * r);
    const float4 r1 = __ldg(reinterpret_cast<const float4*>(rays) + 2 * r + 1);
    j.o = make_float3(r0.x, r0.y, r0.z);
    j.tn = r0.w;
    j.d = make_float3(r1.x, r1.y, r1.z);
    j.tf = r1.w;
    j.ray_id = ray_id0 + (uint32_t)r;
    j.idx = r;
    j.slot = slot;
}

// Warps per block: 4 for the records kernels without logits (a block holds its SM slots until its slowest ray
// ends, so small blocks keep an SM fuller: 0.950 -> 0.938 ms per room step against 8, 0.989 with 12; the unfused
// forward 0.695 -> 0.626 ms), 8 for the semantic ones (5.80 ms with 4 against 5.70) and for the in-warp kernels
// (the shared memory of their walk is per warp).  Blocks per SM scale so the registers per thread stay the same.
template <int NSC, bool INWARP>
constexpr int render_wpb() { return INWARP || NSC > 0 ? kWarpsPerBlock : 4; }
template <int MODE, int NSC, int Q, bool INWARP>
constexpr int render_blocks_per_sm() {
    return render_min_blocks<MODE, NSC, Q>() * kWarpsPerBlock / render_wpb<NSC, INWARP>();
}

// One warp per ray.  !INWARP: every slot, cells from the traversal pass's records (a slot with more than kWalkCap
// is skipped: the mid- and overflow-list kernels render it).  INWARP: every slot, the warp walking its ray (a pass
// without traversal records).  Kept apart, the records kernel needs no shared memory, which leaves L1 to the voxel
// gathers.
template <int MODE, bool BF16, int NSC, int Q, bool INWARP>
__global__ void __launch_bounds__(32 * render_wpb<NSC, INWARP>(), (render_blocks_per_sm<MODE, NSC, Q, INWARP>()))
    k_render(GridDev g, const float* __restrict__ rays, uint32_t ray_id0, PassArgs a) {
    // the semantic records program keeps a voxel table per warp for at most kWarpsPerBlock warps
    static_assert(render_wpb<NSC, INWARP>() <= kWarpsPerBlock, "warps per block");
    __shared__ WarpSmem smem[INWARP ? kWarpsPerBlock : 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * render_wpb<NSC, INWARP>() + warp;
    if (w >= a.n) return;  // warp-uniform
    RayJob j;
    load_job(g, rays, a.perm, ray_id0, w, a.n, j);
    ray_program<MODE, BF16, NSC, Q, INWARP>(g, a, j, smem[INWARP ? warp : 0], lane);
}

// Rays beyond the records kernel, of a pass with traversal records: the mid list a.walk.mid[0, *a.walk.n_mid)
// (kWalkCap + 1 .. kWalkSlot allocated cells, rendered from their records two per lane) and the overflow list
// a.walk.over[0, *a.walk.n_over) (more cells, walked in-warp).  A long list -- longer than k_render_rest takes in
// one turn, going by the length the grid's previous pass left in its pinned words (PassArgs::over_out) -- first
// goes to a kernel with one warp per entry (no loop, so the program keeps the register budget of the records
// kernel without spilling: full occupancy for a scene where many rays cross walls, a large apartment); what is
// left of both lists (normally all of a short list, none of a long one) to k_render_rest, a grid of at most
// kRestBlocks blocks striding over them that runs alone after the records kernel (2 blocks per SM, no spills).
constexpr unsigned kRestBlocks = 296;

template <int MODE, bool BF16, int NSC, int Q>
__global__ void __launch_bounds__(32 * render_wpb<NSC, false>(), (render_blocks_per_sm<MODE, NSC, Q, false>()))
    k_render_mid_list(GridDev g, const float* __restrict__ rays, uint32_t ray_id0, PassArgs a) {
    __shared__ WarpSmem smem[1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * render_wpb<NSC, false>() + warp;
    if (q >= (int64_t)__ldg(a.walk.n_mid)) return;  // warp-uniform
    RayJob j;
    load_job(g, rays, a.perm, ray_id0, (int64_t)__ldg(a.walk.mid + q), a.n, j);
    ray_program<MODE, BF16, NSC, Q, false, 2>(g, a, j, smem[0], lane);
}

template <int MODE, bool BF16, int NSC, int Q>
__global__ void __launch_bounds__(256, (render_min_blocks<MODE, NSC, Q>()))
    k_render_over_list(GridDev g, const float* __restrict__ rays, uint32_t ray_id0, PassArgs a) {
    __shared__ WarpSmem smem[kWarpsPerBlock];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
    if (q >= (int64_t)__ldg(a.walk.n_over)) return;  // warp-uniform
    RayJob j;
    load_job(g, rays, a.perm, ray_id0, (int64_t)__ldg(a.walk.over + q), a.n, j);
    ray_program<MODE, BF16, NSC, Q, true>(g, a, j, smem[warp], lane);
}

template <int MODE, bool BF16, int NSC, int Q>
__global__ void __launch_bounds__(256, 2) k_render_rest(GridDev g, const float* __restrict__ rays, uint32_t ray_id0,
                                                        PassArgs a, int64_t first_mid, int64_t first_over) {
    __shared__ WarpSmem smem[kWarpsPerBlock];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n_mid = (int64_t)__ldg(a.walk.n_mid), n_over = (int64_t)__ldg(a.walk.n_over);
    const int64_t w = (int64_t)blockIdx.x * kWarpsPerBlock + warp, stride = (int64_t)gridDim.x * kWarpsPerBlock;
    if (a.over_out && blockIdx.x == 0 && threadIdx.x == 0) {  // the next pass's hints
        a.over_out[0] = (int)n_over;
        a.over_out[1] = (int)n_mid;
    }
    for (int64_t q = first_mid + w; q < n_mid; q += stride) {
        RayJob j;
        load_job(g, rays, a.perm, ray_id0, (int64_t)__ldg(a.walk.mid + q), a.n, j);
        ray_program<MODE, BF16, NSC, Q, false, 2>(g, a, j, smem[warp], lane);
    }
    for (int64_t q = first_over + w; q < n_over; q += stride) {
        RayJob j;
        load_job(g, rays, a.perm, ray_id0, (int64_t)__ldg(a.walk.over + q), a.n, j);
        ray_program<MODE, BF16, NSC, Q, true>(g, a, j, smem[warp], lane);
    }
}

// Blocks of a list kernel for a list the hint says is long (0: leave the list to k_render_rest).
inline unsigned list_blocks(int64_t hint, int warps_per_block, unsigned cap) {
    if (hint <= 2 * (int64_t)kRestBlocks * kWarpsPerBlock) return 0;
    const int64_t want = hint + hint / 4 + 64;  // a margin for a longer list than the last pass's
    return (unsigned)std::min<int64_t>((want + warps_per_block - 1) / warps_per_block, cap);
}

template <int MODE, bool BF16, int NSC, int Q>
int launch_one(const GridDev& gd, const float* rays, uint32_t id0, const PassArgs& a, cudaStream_t s) {
    const unsigned blocks = (unsigned)((a.n + kWarpsPerBlock - 1) / kWarpsPerBlock);
    constexpr bool kNoWalk = MODE == PASS_BWD_STORE;  // samples come from the forward's stored records
    if (kNoWalk || a.walk.hdr) {
        constexpr int R = render_wpb<NSC, false>();
        const unsigned rblocks = (unsigned)((a.n + R - 1) / R);
        k_render<MODE, BF16, NSC, Q, false><<<rblocks, 32 * R, 0, s>>>(gd, rays, id0, a);
        if constexpr (!kNoWalk) {
            const unsigned lm = list_blocks(a.mid_hint, R, rblocks);
            const unsigned lo = list_blocks(a.over_hint, kWarpsPerBlock, blocks);
            if (lm) k_render_mid_list<MODE, BF16, NSC, Q><<<lm, 32 * R, 0, s>>>(gd, rays, id0, a);
            if (lo) k_render_over_list<MODE, BF16, NSC, Q><<<lo, 256, 0, s>>>(gd, rays, id0, a);
            k_render_rest<MODE, BF16, NSC, Q><<<blocks < kRestBlocks ? blocks : kRestBlocks, 256, 0, s>>>(
                gd, rays, id0, a, (int64_t)lm * R, (int64_t)lo * kWarpsPerBlock);
        }
    } else {
        k_render<MODE, BF16, NSC, Q, true><<<blocks, 256, 0, s>>>(gd, rays, id0, a);
    }
    return SDG_OK;
}

template <int MODE, bool BF16, int NSC>
int launch_q(const GridDev& gd, const float* rays, uint32_t id0, const PassArgs& a, int Q, cudaStream_t s) {
    int rc;
    switch (Q) {
        case 2: rc = launch_one<MODE, BF16, NSC, 2>(gd, rays, id0, a, s); break;
        case 4: rc = launch_one<MODE, BF16, NSC, 4>(gd, rays, id0, a, s); break;
        case 6: rc = launch_one<MODE, BF16, NSC, 6>(gd, rays, id0, a, s); break;
        default: rc = launch_one<MODE, BF16, NSC, 8>(gd, rays, id0, a, s); break;
    }
    if (rc) return rc;
    SDG_LAUNCH_CHECK("render kernel");
    return SDG_OK;
}


}  // namespace sdg

#define SDG_INSTANTIATE_LAUNCH(MODE, BF16, NSC)                                                         \
    template int sdg::launch_q<MODE, BF16, NSC>(const GridDev&, const float*, uint32_t, const PassArgs&, int, \
                                                cudaStream_t);
#define SDG_EXTERN_LAUNCH(MODE, BF16, NSC)                                                                   \
    extern template int sdg::launch_q<MODE, BF16, NSC>(const GridDev&, const float*, uint32_t, const PassArgs&, \
                                                       int, cudaStream_t);
