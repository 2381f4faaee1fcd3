// Optimiser step over the voxel parameters (Sec. 3.5.4: theta_d, theta_c,
// theta_s optimised directly; RMSProp at lr 1e-3 in the paper, Adam by
// default here).  A streaming kernel: every parameter is read and written once
// per step (theta, g, m, v in; theta, m, v out; g zeroed), so it is bound by
// HBM bandwidth.  Paper: arXiv 2305.13220.
#include <algorithm>
#include <cmath>

#include "internal.h"

using namespace sdg;

// Streaming (evict-first) cache hints on the once-read, once-written optimiser streams.
#define SDG_LD(p) __ldcs(p)
#define SDG_ST(p, v) __stcs(p, v)

namespace {

struct OptParams {
    float lr, b1, b2, eps;
    float omb1, omb2;   // 1 - b1, 1 - b2 (rounded from double)
    float step_size;    // lr / (1 - b1^step)
    float inv_sqrt_c2;  // 1 / sqrt(1 - b2^step)
};

// theta -= lr (m / c1) / (sqrt(v / c2) + eps), written as step_size * m / (sqrt(v) / sqrt(c2) + eps) with the
// bias corrections folded on the host: one square root and one division per parameter.
template <int ALGO>
__device__ __forceinline__ float update(float th, float g, float& m, float& v, const OptParams& p) {
    if (ALGO == SDG_OPT_ADAM) {
        m = fmaf(p.b1, m, p.omb1 * g);
        v = fmaf(p.b2, v, p.omb2 * g * g);
        const float denom = fmaf(sqrtf(v), p.inv_sqrt_c2, p.eps);
        return th - __fdividef(p.step_size * m, denom);
    } else {  // RMSProp, alpha = b2
        v = fmaf(p.b2, v, p.omb2 * g * g);
        return th - __fdividef(p.lr * g, sqrtf(v) + p.eps);
    }
}

// FP32 parameters, four per thread-iteration (16-byte streaming accesses).
template <int ALGO>
__global__ void __launch_bounds__(256) k_opt_f32(float4* __restrict__ th, float4* __restrict__ gr,
                                                 float4* __restrict__ m, float4* __restrict__ v, int64_t n4,
                                                 OptParams p) {
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        // RMSProp has no first moment: m is neither read nor written
        float4 t = SDG_LD(th + i), g = SDG_LD(gr + i), mm = ALGO == SDG_OPT_ADAM ? SDG_LD(m + i) : z,
               vv = SDG_LD(v + i);
        t.x = update<ALGO>(t.x, g.x, mm.x, vv.x, p);
        t.y = update<ALGO>(t.y, g.y, mm.y, vv.y, p);
        t.z = update<ALGO>(t.z, g.z, mm.z, vv.z, p);
        t.w = update<ALGO>(t.w, g.w, mm.w, vv.w, p);
        SDG_ST(th + i, t);
        SDG_ST(gr + i, z);
        if (ALGO == SDG_OPT_ADAM) SDG_ST(m + i, mm);
        SDG_ST(v + i, vv);
    }
}

__device__ __forceinline__ float bf_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf_hi(uint32_t u) { return __uint_as_float(u & 0xFFFF0000u); }
__device__ __forceinline__ uint32_t pack_bf2(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);  // round to nearest even
    return *reinterpret_cast<uint32_t*>(&h);
}

// BF16 parameters in groups of four (uint2) with FP32 gradient and moments;
// lanes >= nlanes of each group are padding and left untouched.
template <int ALGO>
__global__ void __launch_bounds__(256) k_opt_bf16(uint2* __restrict__ th, float4* __restrict__ gr,
                                                  float4* __restrict__ m, float4* __restrict__ v, int64_t n4,
                                                  int nlanes, OptParams p) {
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        uint2 t = SDG_LD(th + i);
        float4 g = SDG_LD(gr + i), mm = ALGO == SDG_OPT_ADAM ? SDG_LD(m + i) : z, vv = SDG_LD(v + i);
        float a0 = bf_lo(t.x), a1 = bf_hi(t.x), a2 = bf_lo(t.y), a3 = bf_hi(t.y);
        a0 = update<ALGO>(a0, g.x, mm.x, vv.x, p);
        a1 = update<ALGO>(a1, g.y, mm.y, vv.y, p);
        a2 = update<ALGO>(a2, g.z, mm.z, vv.z, p);
        if (nlanes == 4) a3 = update<ALGO>(a3, g.w, mm.w, vv.w, p);
        t.x = pack_bf2(a0, a1);
        t.y = pack_bf2(a2, a3);
        SDG_ST(th + i, t);
        SDG_ST(gr + i, z);
        if (ALGO == SDG_OPT_ADAM) SDG_ST(m + i, mm);
        SDG_ST(v + i, vv);
    }
}

int opt_blocks(int64_t n) {
    int64_t b = (n + 255) / 256;
    const int64_t cap = 148 * 8;  // enough resident warps to saturate HBM; grid-stride beyond
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <int ALGO>
int run(sdg_grid g, const OptParams& p) {
    const int64_t V = g->n_blocks * 512;
    cudaStream_t s = g->stream;
    if (g->desc.rgb_dtype == SDG_F32) {
        k_opt_f32<ALGO><<<opt_blocks(V), 256, 0, s>>>(g->geo, g->ggeo, g->m_geo, g->v_geo, V, p);
    } else {
        k_opt_f32<ALGO><<<opt_blocks(V / 4), 256, 0, s>>>((float4*)g->sdf, (float4*)g->gsdf, (float4*)g->m_sdf,
                                                           (float4*)g->v_sdf, V / 4, p);
        k_opt_bf16<ALGO><<<opt_blocks(V), 256, 0, s>>>(g->rgbh, g->grgb, g->m_rgb, g->v_rgb, V, 3, p);
    }
    if (g->desc.n_sem) {
        const int64_t n4 = V * g->desc.n_sem / 4;
        k_opt_bf16<ALGO><<<opt_blocks(n4), 256, 0, s>>>((uint2*)g->sem, (float4*)g->gsem, (float4*)g->m_sem,
                                                         (float4*)g->v_sem, n4, 4, p);
    }
    SDG_LAUNCH_CHECK("optimiser");
    return SDG_OK;
}

// The learnable Laplace scale (a single parameter) is updated on the host with the same optimiser and step
// index: its gradient, accumulated on the device by the training passes since the last step, is read back (the
// one synchronisation a step with a learnable scale needs), then zeroed.  beta stays >= 1e-3 voxel sizes.
int beta_step(sdg_grid g, const sdg_adam_opts* a, int32_t step) {
    float grad = 0.f;
    SDG_CUDA_TRY(cudaMemcpyAsync(&grad, g->beta_grad, sizeof(float), cudaMemcpyDeviceToHost, g->stream));
    SDG_CUDA_TRY(cudaMemsetAsync(g->beta_grad, 0, sizeof(float), g->stream));
    SDG_CUDA_TRY(cudaStreamSynchronize(g->stream));
    g->beta_grad_pending = false;
    const double gb = grad;
    double beta = g->beta;
    if (a->algo == SDG_OPT_ADAM) {
        g->beta_m = a->beta1 * g->beta_m + (1.0 - a->beta1) * gb;
        g->beta_v = a->beta2 * g->beta_v + (1.0 - a->beta2) * gb * gb;
        const double mh = g->beta_m / (1.0 - std::pow(a->beta1, step));
        const double vh = g->beta_v / (1.0 - std::pow(a->beta2, step));
        beta -= a->lr * mh / (std::sqrt(vh) + a->eps);
    } else {
        g->beta_v = a->beta2 * g->beta_v + (1.0 - a->beta2) * gb * gb;
        beta -= a->lr * gb / (std::sqrt(g->beta_v) + a->eps);
    }
    g->beta = (float)std::max(beta, 1e-3 * (double)g->desc.voxel_size);
    return SDG_OK;
}

}  // namespace

extern "C" int sdg_adam_step(sdg_grid g, const sdg_adam_opts* a) {
    if (!g || !a || !(a->lr >= 0.0) || !(a->beta1 >= 0.0 && a->beta1 < 1.0) || !(a->beta2 >= 0.0 && a->beta2 < 1.0) ||
        !(a->eps > 0.0) || (a->algo != SDG_OPT_ADAM && a->algo != SDG_OPT_RMSPROP))
        return fail(SDG_ERR_ARG, "sdg_adam_step: invalid options");
    int rc = use_device(g);
    if (rc) return rc;
    const int32_t step = a->step > 0 ? a->step : g->step + 1;
    g->step = step;
    if (g->beta_grad_pending && (rc = beta_step(g, a, step))) return rc;
    if (g->n_blocks == 0) return SDG_OK;
    OptParams p;
    p.lr = (float)a->lr;
    p.b1 = (float)a->beta1;
    p.b2 = (float)a->beta2;
    p.eps = (float)a->eps;
    p.omb1 = (float)(1.0 - a->beta1);
    p.omb2 = (float)(1.0 - a->beta2);
    p.step_size = (float)(a->lr / (1.0 - std::pow(a->beta1, step)));
    p.inv_sqrt_c2 = (float)(1.0 / std::sqrt(1.0 - std::pow(a->beta2, step)));
    return a->algo == SDG_OPT_ADAM ? run<SDG_OPT_ADAM>(g, p) : run<SDG_OPT_RMSPROP>(g, p);
}
