// Point queries of the SDF and its closed-form gradient (Sec. 3.5.2, Eq.
// 16-17) and the Eikonal regulariser built on them (Sec. 3.5.3).  The
// trilinear weight of a stencil corner is a product over the axes of f_a (far
// corner) or 1 - f_a (near corner); its derivative along axis a swaps that
// factor for +-1/vs, so value and gradient come from the same 8 corner loads
// in one pass, without a second differentiation.
//
// One thread per point: FP32 cell and block of the point, the block's index
// from the hash map, corner addresses through the neighbour table (corners
// past the block's +x/+y/+z faces live in the neighbour blocks).  A point with
// a corner in an unallocated block, or outside the block-key range, is invalid.
#include "internal.h"
#include "reduce.cuh"
#include "render_core.cuh"

namespace sdg {
namespace {

constexpr int kThreads = 256;
// Below this |grad f| (a flat, e.g. truncated, region) the direction of grad f is rounding noise, so the
// Eikonal gradient is taken as 0 there (its loss term is still counted).
constexpr float kFlatGrad = 1e-4f;
// Largest |cell coordinate| whose block key (21 bits per axis) is representable.
constexpr float kMaxCell = 8.0f * (float)(1 << 20) - 16.0f;

struct PointStencil {
    bool valid;
    int addr[8];
    float f[3];
};

__device__ __forceinline__ PointStencil point_stencil(const GridDev& g, float x, float y, float z) {
    PointStencil s;
    s.valid = false;
    const float gx = x * g.inv_vs, gy = y * g.inv_vs, gz = z * g.inv_vs;
    if (!(fabsf(gx) < kMaxCell && fabsf(gy) < kMaxCell && fabsf(gz) < kMaxCell)) return s;  // also NaN
    const float fx = floorf(gx), fy = floorf(gy), fz = floorf(gz);
    const int cx = (int)fx, cy = (int)fy, cz = (int)fz;
    s.f[0] = gx - fx;
    s.f[1] = gy - fy;
    s.f[2] = gz - fz;
    const int blk = sdg_table_find(g.table, g.mask, sdg_pack_key(cx >> 3, cy >> 3, cz >> 3));
    if (blk < 0) return s;
    const int lcell = (cx & 7) | ((cy & 7) << 3) | ((cz & 7) << 6);
    s.valid = corner_addresses(g, blk, lcell, s.addr);
    return s;
}

template <bool BF16>
__device__ __forceinline__ float corner_sdf(const GridDev& g, int addr) {
    if constexpr (BF16) return __ldg(g.sdf + addr);
    else return __ldg(&g.geo[addr].x);
}

// f and grad f at a valid stencil; dr[e][a] = d r_e / d x_a.
template <bool BF16>
__device__ __forceinline__ void sdf_and_grad(const GridDev& g, const PointStencil& s, float& f, float grad[3],
                                             float dr[8][3]) {
    float th[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) th[e] = corner_sdf<BF16>(g, s.addr[e]);
    f = 0.f;
    grad[0] = grad[1] = grad[2] = 0.f;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        float fac[3], dfac[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const bool far = (e >> a) & 1;
            fac[a] = far ? s.f[a] : 1.f - s.f[a];
            dfac[a] = far ? g.inv_vs : -g.inv_vs;
        }
        dr[e][0] = dfac[0] * fac[1] * fac[2];
        dr[e][1] = fac[0] * dfac[1] * fac[2];
        dr[e][2] = fac[0] * fac[1] * dfac[2];
        f = fmaf(fac[0] * fac[1] * fac[2], th[e], f);
#pragma unroll
        for (int a = 0; a < 3; ++a) grad[a] = fmaf(dr[e][a], th[e], grad[a]);
    }
}

template <bool BF16>
__global__ void __launch_bounds__(kThreads) k_query(GridDev g, const float* __restrict__ xyz, int64_t n,
                                                    float* __restrict__ sdf, float* __restrict__ grad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const PointStencil s =
            point_stencil(g, __ldg(xyz + 3 * i), __ldg(xyz + 3 * i + 1), __ldg(xyz + 3 * i + 2));
        float f = __int_as_float(0x7fc00000), gr[3] = {f, f, f};
        if (s.valid) {
            float dr[8][3];
            sdf_and_grad<BF16>(g, s, f, gr, dr);
        }
        if (sdf) sdf[i] = f;
        if (grad) {
            grad[3 * i] = gr[0];
            grad[3 * i + 1] = gr[1];
            grad[3 * i + 2] = gr[2];
        }
    }
}

// Eikonal term (lambda/n)(|grad f| - 1)^2 per point and its gradient w.r.t. the stencil's stored SDF values,
// (lambda/n) 2 (|grad f| - 1) (grad f / |grad f|) . grad r_e, added to the SDF gradient channel (0 below kFlatGrad).
template <bool BF16>
__global__ void __launch_bounds__(kThreads) k_eikonal(GridDev g, const float* __restrict__ xyz, int64_t n,
                                                      float lam_over_n, float* __restrict__ terms) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const PointStencil s =
            point_stencil(g, __ldg(xyz + 3 * i), __ldg(xyz + 3 * i + 1), __ldg(xyz + 3 * i + 2));
        float term = 0.f;
        if (s.valid) {
            float f, gr[3], dr[8][3];
            sdf_and_grad<BF16>(g, s, f, gr, dr);
            const float norm = sqrtf(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
            term = lam_over_n * (norm - 1.f) * (norm - 1.f);
            if (norm >= kFlatGrad) {
                const float c = lam_over_n * 2.f * (norm - 1.f) / norm;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const float v = c * (gr[0] * dr[e][0] + gr[1] * dr[e][1] + gr[2] * dr[e][2]);
                    if constexpr (BF16) atomicAdd(g.gsdf + s.addr[e], v);
                    else atomicAdd(&g.ggeo[s.addr[e]].x, v);
                }
            }
        }
        terms[i] = term;
    }
}

int grid_blocks(int64_t n) { return (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 148 * 32); }

bool aligned4(const void* p) { return ((uintptr_t)p & 3u) == 0; }

}  // namespace
}  // namespace sdg

using namespace sdg;

extern "C" int sdg_query(sdg_grid g, const float* xyz, int64_t n, float* sdf, float* grad) {
    if (!g || n < 0 || (n > 0 && !xyz)) return fail(SDG_ERR_ARG, "sdg_query: null argument");
    if (n > 0 && (!aligned4(xyz) || (sdf && !aligned4(sdf)) || (grad && !aligned4(grad))))
        return fail(SDG_ERR_ARG, "sdg_query: arrays must be 4-byte aligned");
    int rc = use_device(g);
    if (rc) return rc;
    if (n == 0 || (!sdf && !grad)) return SDG_OK;
    const GridDev gd = g->dev();
    if (g->desc.rgb_dtype == SDG_BF16)
        k_query<true><<<grid_blocks(n), kThreads, 0, g->stream>>>(gd, xyz, n, sdf, grad);
    else
        k_query<false><<<grid_blocks(n), kThreads, 0, g->stream>>>(gd, xyz, n, sdf, grad);
    SDG_LAUNCH_CHECK("sdf query");
    return SDG_OK;
}

extern "C" int sdg_eikonal(sdg_grid g, const float* xyz, int64_t n, float lambda, float* terms, float* loss_sum) {
    if (!g || n < 0 || (n > 0 && !xyz)) return fail(SDG_ERR_ARG, "sdg_eikonal: null argument");
    if (n > 0 && !aligned4(xyz)) return fail(SDG_ERR_ARG, "sdg_eikonal: xyz must be 4-byte aligned");
    int rc = use_device(g);
    if (rc) return rc;
    if (n == 0) {
        if (loss_sum) SDG_CUDA_TRY(cudaMemsetAsync(loss_sum, 0, sizeof(float), g->stream));
        return SDG_OK;
    }
    float* per_point = terms;
    if (!per_point && (rc = loss_scratch(g, n, &per_point))) return rc;
    const GridDev gd = g->dev();
    const float lam_n = lambda / (float)n;
    if (g->desc.rgb_dtype == SDG_BF16)
        k_eikonal<true><<<grid_blocks(n), kThreads, 0, g->stream>>>(gd, xyz, n, lam_n, per_point);
    else
        k_eikonal<false><<<grid_blocks(n), kThreads, 0, g->stream>>>(gd, xyz, n, lam_n, per_point);
    SDG_LAUNCH_CHECK("eikonal");
    if (loss_sum) {
        k_sum<<<1, 1024, 0, g->stream>>>(per_point, n, loss_sum);
        SDG_LAUNCH_CHECK("eikonal loss sum");
    }
    return SDG_OK;
}
