// Render kernel template and its launcher, instantiated per (layout, semantics,
// pass) in the render_inst_*.cu files so that they compile in parallel.
#pragma once

#include "render_core.cuh"

namespace sdg {

// Resident 256-thread blocks per SM requested from the register allocator: three (80 registers) where the
// program fits with no or a few bytes of spill (measured on the room training step: 1.69 -> 1.49 ms), fewer
// for the larger per-lane sample counts and the semantic variants, which need more registers.
template <int MODE, bool SEM, int Q>
constexpr int render_min_blocks() {
#ifdef SDG_RENDER_MIN_BLOCKS
    return SDG_RENDER_MIN_BLOCKS;
#else
    return SEM ? (Q >= 6 ? 1 : 2) : (MODE == PASS_TRAIN_NRM || Q >= 6 ? 2 : 3);
#endif
}

template <int MODE, bool BF16, bool SEM, int Q>
__global__ void __launch_bounds__(256, (render_min_blocks<MODE, SEM, Q>()))
    k_render(GridDev g, const float* __restrict__ rays, uint32_t ray_id0, PassArgs a) {
    __shared__ WarpSmem smem[kWarpsPerBlock];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t slot = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
    if (slot >= a.n) return;  // warp-uniform
    const int64_t r = a.perm ? (int64_t)__ldg(a.perm + slot) : slot;
    const float4 r0 = __ldg(reinterpret_cast<const float4*>(rays) + 2 * r);
    const float4 r1 = __ldg(reinterpret_cast<const float4*>(rays) + 2 * r + 1);
    RayJob j;
    j.o = make_float3(r0.x, r0.y, r0.z);
    j.tn = r0.w;
    j.d = make_float3(r1.x, r1.y, r1.z);
    j.tf = r1.w;
    j.ray_id = ray_id0 + (uint32_t)r;
    j.idx = r;
    j.slot = slot;
    ray_program<MODE, BF16, SEM, Q>(g, a, j, smem[warp], lane);
}

template <int MODE, bool BF16, bool SEM>
int launch_q(const GridDev& gd, const float* rays, uint32_t id0, const PassArgs& a, int Q, cudaStream_t s) {
    const unsigned blocks = (unsigned)((a.n + kWarpsPerBlock - 1) / kWarpsPerBlock);
    switch (Q) {
        case 2: k_render<MODE, BF16, SEM, 2><<<blocks, 256, 0, s>>>(gd, rays, id0, a); break;
        case 4: k_render<MODE, BF16, SEM, 4><<<blocks, 256, 0, s>>>(gd, rays, id0, a); break;
        case 6: k_render<MODE, BF16, SEM, 6><<<blocks, 256, 0, s>>>(gd, rays, id0, a); break;
        default: k_render<MODE, BF16, SEM, 8><<<blocks, 256, 0, s>>>(gd, rays, id0, a); break;
    }
    SDG_LAUNCH_CHECK("render kernel");
    return SDG_OK;
}


}  // namespace sdg

#define SDG_INSTANTIATE_LAUNCH(MODE, BF16, SEM)                                                         \
    template int sdg::launch_q<MODE, BF16, SEM>(const GridDev&, const float*, uint32_t, const PassArgs&, int, \
                                                cudaStream_t);
