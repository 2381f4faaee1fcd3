// Point queries of the SDF and its closed-form gradient (Sec. 3.5.2, Eq.
// 16-17) and the Eikonal regulariser built on them (Sec. 3.5.3).  The
// trilinear weight of a stencil corner is a product over the axes of f_a (far
// corner) or 1 - f_a (near corner); its derivative along axis a swaps that
// factor for +-1/vs, so value and gradient come from the same 8 corner loads
// in one pass, without a second differentiation.
//
// One thread per point: FP32 cell and block of the point, the block's index
// from the dense block-index grid (one load), corner addresses through the
// neighbour table (corners past the block's +x/+y/+z faces live in the
// neighbour blocks).  A point with a corner in an unallocated block, or
// outside the block-key range, is invalid.
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
    const int blk = block_at(g, cx >> 3, cy >> 3, cz >> 3);  // dense block-index grid: one load, -1 if absent
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

// CRF losses (Sec. 3.5.3, Eq. 22): the divergence between a property at surface points and its fixed CRF target.
//   PROP 0, labels: (lambda/n) KL(Q || softmax(s)), dL/ds = (lambda/n)(softmax(s) - Q), s the trilinear logits;
//   PROP 1, colour: (lambda/n) |c - t|^2;  PROP 2, normal: (lambda/n) |grad f - t|^2.
// Gradients go through the trilinear weights (their x-gradients for the normal) into the gradient channels.
template <bool BF16, int PROP>
__global__ void __launch_bounds__(kThreads) k_crf_loss(GridDev g, const float* __restrict__ xyz, int64_t n,
                                                       const float* __restrict__ target, float k,
                                                       float* __restrict__ terms) {
    const int ns = g.n_sem;
    const int ch = PROP == 0 ? ns : 3;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const PointStencil s =
            point_stencil(g, __ldg(xyz + 3 * i), __ldg(xyz + 3 * i + 1), __ldg(xyz + 3 * i + 2));
        float term = 0.f;
        if (s.valid) {
            const float* t = target + (int64_t)ch * i;
            float r[8];
            trilinear_weights(s.f[0], s.f[1], s.f[2], r);
            if constexpr (PROP == 0) {
                float lg[32];
#pragma unroll
                for (int c = 0; c < 32; ++c) lg[c] = 0.f;
#pragma unroll
                for (int e = 0; e < 8; ++e)
#pragma unroll
                    for (int c4 = 0; c4 < 8; ++c4)
                        if (4 * c4 < ns) {
                            float v[4];
                            sem_load4(g, s.addr[e], 4 * c4, v);
#pragma unroll
                            for (int q = 0; q < 4; ++q) lg[4 * c4 + q] = fmaf(r[e], v[q], lg[4 * c4 + q]);
                        }
                float mx = -3.0e38f;
#pragma unroll
                for (int c = 0; c < 32; ++c)
                    if (c < ns) mx = fmaxf(mx, lg[c]);
                float z = 0.f;
#pragma unroll
                for (int c = 0; c < 32; ++c)
                    if (c < ns) z += __expf(lg[c] - mx);
                const float lz = __logf(z);
#pragma unroll
                for (int c = 0; c < 32; ++c)
                    if (c < ns) {
                        const float logp = lg[c] - mx - lz;
                        const float tc = __ldg(t + c);
                        if (tc > 0.f) term += k * tc * (__logf(tc) - logp);
                        lg[c] = k * (__expf(logp) - tc);  // now dL/ds_c
                    }
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    float* gs = g.gsem + (int64_t)s.addr[e] * ns;
#pragma unroll
                    for (int c4 = 0; c4 < 8; ++c4)
                        if (4 * c4 < ns)
                            red_add_v4(reinterpret_cast<float4*>(gs) + c4, r[e] * lg[4 * c4], r[e] * lg[4 * c4 + 1],
                                       r[e] * lg[4 * c4 + 2], r[e] * lg[4 * c4 + 3]);
                }
            } else if constexpr (PROP == 1) {
                float cv[3] = {0.f, 0.f, 0.f};
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    float c0, c1, c2;
                    if constexpr (BF16) {
                        const uint2 u = __ldg(g.rgbh + s.addr[e]);
                        c0 = sdg_bf16_lo(u.x);
                        c1 = sdg_bf16_hi(u.x);
                        c2 = sdg_bf16_lo(u.y);
                    } else {
                        const float4 v = __ldg(g.geo + s.addr[e]);
                        c0 = v.y;
                        c1 = v.z;
                        c2 = v.w;
                    }
                    cv[0] = fmaf(r[e], c0, cv[0]);
                    cv[1] = fmaf(r[e], c1, cv[1]);
                    cv[2] = fmaf(r[e], c2, cv[2]);
                }
                float gp[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float dlt = cv[c] - __ldg(t + c);
                    term += k * dlt * dlt;
                    gp[c] = 2.f * k * dlt;
                }
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    if constexpr (BF16) red_add_v4(g.grgb + s.addr[e], r[e] * gp[0], r[e] * gp[1], r[e] * gp[2], 0.f);
                    else red_add_v4(g.ggeo + s.addr[e], 0.f, r[e] * gp[0], r[e] * gp[1], r[e] * gp[2]);
                }
            } else {
                float f, gr[3], dr[8][3];
                sdf_and_grad<BF16>(g, s, f, gr, dr);
                float gp[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float dlt = gr[a] - __ldg(t + a);
                    term += k * dlt * dlt;
                    gp[a] = 2.f * k * dlt;
                }
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const float v = gp[0] * dr[e][0] + gp[1] * dr[e][1] + gp[2] * dr[e][2];
                    if constexpr (BF16) atomicAdd(g.gsdf + s.addr[e], v);
                    else atomicAdd(&g.ggeo[s.addr[e]].x, v);
                }
            }
        }
        terms[i] = term;
    }
}

int grid_blocks(int64_t n) { return (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 148 * 32); }

// One resident wave of CTAs (the SM count times the CTAs per SM that the kernel's registers allow), fewer when n
// needs fewer: every thread then loops over an equal share of the points and no partial last wave leaves SMs idle
// (the SDF query at 512^3 points: 1.59 -> 1.31 ms).  The atomic-bound Eikonal and CRF-loss kernels run faster with
// one point per thread over more CTAs (grid_blocks).
template <class Kernel>
int wave_blocks(Kernel kernel, int64_t n) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0) || sms <= 0 || per_sm <= 0) {
        (void)cudaGetLastError();
        sms = 148;
        per_sm = 4;
    }
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, (int64_t)sms * per_sm));
}

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
        k_query<true><<<wave_blocks(k_query<true>, n), kThreads, 0, g->stream>>>(gd, xyz, n, sdf, grad);
    else
        k_query<false><<<wave_blocks(k_query<false>, n), kThreads, 0, g->stream>>>(gd, xyz, n, sdf, grad);
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
        launch_sum(per_point, n, loss_sum, g->sum_scratch, g->stream);
        SDG_LAUNCH_CHECK("eikonal loss sum");
    }
    return SDG_OK;
}

extern "C" int sdg_crf_loss(sdg_grid g, int32_t prop, int64_t n, const float* xyz, const float* target, float lambda,
                            float* terms, float* loss_sum) {
    if (!g || n < 0 || prop < 0 || prop > 2 || (n > 0 && (!xyz || !target)))
        return fail(SDG_ERR_ARG, "sdg_crf_loss: bad argument (prop 0 labels, 1 colour, 2 normal)");
    if (prop == 0 && g->desc.n_sem == 0) return fail(SDG_ERR_ARG, "sdg_crf_loss: the grid has no logits");
    if (n > 0 && (!aligned4(xyz) || !aligned4(target))) return fail(SDG_ERR_ARG, "sdg_crf_loss: misaligned arrays");
    int rc = use_device(g);
    if (rc) return rc;
    if (n == 0) {
        if (loss_sum) SDG_CUDA_TRY(cudaMemsetAsync(loss_sum, 0, sizeof(float), g->stream));
        return SDG_OK;
    }
    float* per_point = terms;
    if (!per_point && (rc = loss_scratch(g, n, &per_point))) return rc;
    const GridDev gd = g->dev();
    const float k = lambda / (float)n;
    const bool bf16 = g->desc.rgb_dtype == SDG_BF16;
    cudaStream_t st = g->stream;
    const int nb = grid_blocks(n);
    auto launch = [&](auto kernel) { kernel<<<nb, kThreads, 0, st>>>(gd, xyz, n, target, k, per_point); };
    if (prop == 0) {
        if (bf16) launch(k_crf_loss<true, 0>);
        else launch(k_crf_loss<false, 0>);
    } else if (prop == 1) {
        if (bf16) launch(k_crf_loss<true, 1>);
        else launch(k_crf_loss<false, 1>);
    } else {
        if (bf16) launch(k_crf_loss<true, 2>);
        else launch(k_crf_loss<false, 2>);
    }
    SDG_LAUNCH_CHECK("crf loss");
    if (loss_sum) {
        launch_sum(per_point, n, loss_sum, g->sum_scratch, st);
        SDG_LAUNCH_CHECK("crf loss sum");
    }
    return SDG_OK;
}
