// Volumetric fusion of depth, colour and semantic-logit frames into the
// allocated voxels: Sec. 3.4.2 (Eq. 9-11) and the supplement's truncation psi.
// The least-squares problems of Eq. 9-11 are solved by averages over the
// voxel-pixel associations, kept here as running means with a per-voxel count
// (the WEIGHT channel), so that frames can be fused in any number of calls.
//
// One CTA per voxel block, one thread per voxel (cameras are read as four
// 16-byte loads, logits as float4 when their count allows).  The CTA first
// finds the frames whose view frustum can contain the block (a conservative
// bounding-sphere test, one frame per thread, then an order-preserving
// compaction in shared memory), so each voxel only projects itself into those
// frames.  The association itself is decided in FP32 with a fixed operation
// order (round-to-nearest intrinsics, no contraction) so that the integer
// decisions -- which pixel, kept or not -- are exactly those of any FP32
// evaluation of the same order:
//   x_a = (float)(8 b_a + l_a) * vs;  e_a = x_a - t_a;
//   c_j = (R_0j e_0 + R_1j e_1) + R_2j e_2        (c = R^T (x - t));  need c_2 > 0
//   r = 1 / c_2;  pu = fx (c_0 r) + cx, pv = fy (c_1 r) + cy; pixel (floor pu, floor pv) inside the image
//   D = depth there, finite and > 0;  o = D - c_2;  need o >= -mu;  psi = min(o, mu)
// The sums of one call accumulate in FP32 in frame order and are folded into
// the running mean once: theta' = (w theta + sum) / (w + n).
#include <vector>

#include "internal.h"

namespace sdg {
namespace {

constexpr int kFuseThreads = 512;     // one voxel block
constexpr int kFuseMaxFrames = 1024;  // frames per launch (their visible subset is listed in shared memory)
constexpr int kSemCap = 32;

struct __align__(16) FuseCam {
    float R[9];  // camera to world rotation, row-major
    float t[3];
    float fx, fy, cx, cy;
};

// A camera as four 16-byte loads (uniform across the CTA) instead of sixteen scalar ones.
__device__ __forceinline__ FuseCam load_cam(const FuseCam* p) {
    const float4* q = reinterpret_cast<const float4*>(p);
    const float4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2), d = __ldg(q + 3);
    FuseCam r;
    r.R[0] = a.x; r.R[1] = a.y; r.R[2] = a.z; r.R[3] = a.w;
    r.R[4] = b.x; r.R[5] = b.y; r.R[6] = b.z; r.R[7] = b.w;
    r.R[8] = c.x; r.t[0] = c.y; r.t[1] = c.z; r.t[2] = c.w;
    r.fx = d.x; r.fy = d.y; r.cx = d.z; r.cy = d.w;
    return r;
}

struct FuseArgs {
    const int4* keys;
    float vs, mu;
    int F, H, W;
    const FuseCam* cams;
    const float* depth;  // [F][H][W]
    const float* rgb;    // [F][H][W][3] or NULL
    const float* sem;    // [F][H][W][ns] or NULL
    int ns;
    bool sem4;  // ns a multiple of 4 and sem 16-byte aligned: a pixel's logits load as float4
    float4* geo;   // FP32 layout: (sdf, r, g, b) running means
    float* sdf;    // BF16 layout: SDF running mean
    float4* racc;  // BF16 layout: FP32 colour running mean (the colour gradient channel)
    float* sacc;   // FP32 logit running mean [voxel][ns] (the semantic gradient channel)
    float* weight;
};

// Conservative test: may the sphere (centre p in camera coordinates, radius r) hold a point that projects
// inside the W x H image in front of the camera?  The four side planes of the frustum pass through the
// camera centre; u >= 0 is fx x + cx z >= 0, u <= W is (W - cx) z - fx x >= 0, and likewise for v.
__device__ __forceinline__ bool sphere_in_frustum(const float p[3], float r, const FuseCam& c, int W, int H) {
    if (p[2] < -r) return false;
    const float a0 = c.fx * p[0] + c.cx * p[2], n0 = sqrtf(c.fx * c.fx + c.cx * c.cx);
    const float rw = (float)W - c.cx, rh = (float)H - c.cy;
    const float a1 = rw * p[2] - c.fx * p[0], n1 = sqrtf(c.fx * c.fx + rw * rw);
    const float a2 = c.fy * p[1] + c.cy * p[2], n2 = sqrtf(c.fy * c.fy + c.cy * c.cy);
    const float a3 = rh * p[2] - c.fy * p[1], n3 = sqrtf(c.fy * c.fy + rh * rh);
    return a0 >= -r * n0 && a1 >= -r * n1 && a2 >= -r * n2 && a3 >= -r * n3;
}

template <bool COLOUR_IN_GEO, bool SEM>
__global__ void __launch_bounds__(kFuseThreads) k_fuse(FuseArgs a) {
    __shared__ short vis[kFuseMaxFrames];
    __shared__ int warp_count[kFuseThreads / 32];
    __shared__ int n_vis;
    const int blk = blockIdx.x;
    const int l = threadIdx.x, lane = l & 31, warp = l >> 5;
    const int4 key = __ldg(a.keys + blk);

    // ---- frames that can see this block, in frame order ----
    {
        const float half = 3.5f * a.vs;
        const float ctr[3] = {fmaf(8.0f * a.vs, (float)key.x, half), fmaf(8.0f * a.vs, (float)key.y, half),
                              fmaf(8.0f * a.vs, (float)key.z, half)};
        const float r = 1.01f * 1.7320508f * half + 1e-4f;  // half-diagonal of the voxel positions, with slack
        int base = 0;
        for (int f0 = 0; f0 < a.F; f0 += kFuseThreads) {
            const int f = f0 + l;
            bool in = false;
            if (f < a.F) {
                const FuseCam c = load_cam(a.cams + f);
                const float e[3] = {ctr[0] - c.t[0], ctr[1] - c.t[1], ctr[2] - c.t[2]};
                float p[3];
                for (int j = 0; j < 3; ++j) p[j] = c.R[j] * e[0] + c.R[3 + j] * e[1] + c.R[6 + j] * e[2];
                in = sphere_in_frustum(p, r, c, a.W, a.H);
            }
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, in);
            if (lane == 0) warp_count[warp] = __popc(bal);
            __syncthreads();
            int before = base;
            for (int w = 0; w < warp; ++w) before += warp_count[w];
            if (in) vis[before + __popc(bal & ((1u << lane) - 1u))] = (short)f;
            int total = 0;
            for (int w = 0; w < kFuseThreads / 32; ++w) total += warp_count[w];
            base += total;
            __syncthreads();
        }
        if (l == 0) n_vis = base;
        __syncthreads();
    }
    const int nv = n_vis;
    if (nv == 0) return;

    // ---- this voxel's associations ----
    const int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
    const float x0 = __fmul_rn((float)(8 * key.x + lx), a.vs);
    const float x1 = __fmul_rn((float)(8 * key.y + ly), a.vs);
    const float x2 = __fmul_rn((float)(8 * key.z + lz), a.vs);
    const int64_t HW = (int64_t)a.H * a.W;
    float cnt = 0.f, sd = 0.f, s0 = 0.f, s1 = 0.f, s2 = 0.f;
    float ss[SEM ? kSemCap : 1];
#pragma unroll
    for (int q = 0; q < (SEM ? kSemCap : 1); ++q) ss[q] = 0.f;
    for (int k = 0; k < nv; ++k) {
        const int i = vis[k];
        const FuseCam c = load_cam(a.cams + i);
        const float e0 = __fsub_rn(x0, c.t[0]), e1 = __fsub_rn(x1, c.t[1]), e2 = __fsub_rn(x2, c.t[2]);
        const float c0 = __fadd_rn(__fadd_rn(__fmul_rn(c.R[0], e0), __fmul_rn(c.R[3], e1)), __fmul_rn(c.R[6], e2));
        const float c1 = __fadd_rn(__fadd_rn(__fmul_rn(c.R[1], e0), __fmul_rn(c.R[4], e1)), __fmul_rn(c.R[7], e2));
        const float c2 = __fadd_rn(__fadd_rn(__fmul_rn(c.R[2], e0), __fmul_rn(c.R[5], e1)), __fmul_rn(c.R[8], e2));
        if (!(c2 > 0.f)) continue;
        const float rz = __frcp_rn(c2);  // one correctly rounded reciprocal, two products
        const float pu = __fadd_rn(__fmul_rn(c.fx, __fmul_rn(c0, rz)), c.cx);
        const float pv = __fadd_rn(__fmul_rn(c.fy, __fmul_rn(c1, rz)), c.cy);
        const float fu = floorf(pu), fv = floorf(pv);
        if (!(fu >= 0.f && fu < (float)a.W && fv >= 0.f && fv < (float)a.H)) continue;
        // pixel within the frame in 32 bits (a frame holds < 2^31 pixels), frame offset in 64
        const int64_t pix = (int64_t)i * HW + ((int)fv * a.W + (int)fu);
        const float D = __ldg(a.depth + pix);
        if (!(isfinite(D) && D > 0.f)) continue;
        const float o = __fsub_rn(D, c2);
        if (!(o >= -a.mu)) continue;
        cnt += 1.f;
        sd += fminf(o, a.mu);
        if (a.rgb) {
            s0 += __ldg(a.rgb + 3 * pix);
            s1 += __ldg(a.rgb + 3 * pix + 1);
            s2 += __ldg(a.rgb + 3 * pix + 2);
        }
        if constexpr (SEM) {
            if (a.sem) {
                const float* sp = a.sem + (int64_t)a.ns * pix;
                if (a.sem4) {
#pragma unroll
                    for (int q4 = 0; q4 < kSemCap / 4; ++q4)
                        if (4 * q4 < a.ns) {
                            const float4 v = __ldg(reinterpret_cast<const float4*>(sp) + q4);
                            ss[4 * q4] += v.x;
                            ss[4 * q4 + 1] += v.y;
                            ss[4 * q4 + 2] += v.z;
                            ss[4 * q4 + 3] += v.w;
                        }
                } else {
#pragma unroll
                    for (int q = 0; q < kSemCap; ++q)
                        if (q < a.ns) ss[q] += __ldg(sp + q);
                }
            }
        }
    }
    if (cnt == 0.f) return;

    // ---- fold into the running means ----
    const int64_t v = (int64_t)blk * 512 + l;
    const float w = a.weight[v], w2 = w + cnt;
    a.weight[v] = w2;
    if constexpr (COLOUR_IN_GEO) {
        float4 g = a.geo[v];
        g.x = w > 0.f ? (w * g.x + sd) / w2 : sd / w2;
        if (a.rgb) {
            g.y = w > 0.f ? (w * g.y + s0) / w2 : s0 / w2;
            g.z = w > 0.f ? (w * g.z + s1) / w2 : s1 / w2;
            g.w = w > 0.f ? (w * g.w + s2) / w2 : s2 / w2;
        }
        a.geo[v] = g;
    } else {
        a.sdf[v] = w > 0.f ? (w * a.sdf[v] + sd) / w2 : sd / w2;
        if (a.rgb) {
            float4 r = a.racc[v];
            r.x = w > 0.f ? (w * r.x + s0) / w2 : s0 / w2;
            r.y = w > 0.f ? (w * r.y + s1) / w2 : s1 / w2;
            r.z = w > 0.f ? (w * r.z + s2) / w2 : s2 / w2;
            a.racc[v] = r;
        }
    }
    if constexpr (SEM) {
        if (a.sem) {
            float* sp = a.sacc + (int64_t)a.ns * v;
#pragma unroll
            for (int q = 0; q < kSemCap; ++q)
                if (q < a.ns) sp[q] = w > 0.f ? (w * sp[q] + ss[q]) / w2 : ss[q] / w2;
        }
    }
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);  // round to nearest even
    return *reinterpret_cast<uint32_t*>(&h);
}

// Writes the fused colour (BF16 layout) and theta_s = s* / |s*| (Eq. 11) of every voxel with a kept
// association into the BF16 value channels, then zeroes the FP32 accumulators (the gradient channels).
// n_sem is a multiple of 4: logits move as 16-byte groups (FP32 accumulators) and 8-byte groups (BF16 values).
template <int NS4>
__global__ void k_fuse_finalize(int64_t V, const float* __restrict__ weight, float4* racc, uint2* rgbh,
                                float4* sacc, uint2* sem, int ns4_rt) {
    const int ns4 = NS4 > 0 ? NS4 : ns4_rt;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        const bool fused = __ldg(weight + v) > 0.f;
        if (racc) {
            const float4 r = racc[v];
            if (fused) rgbh[v] = make_uint2(pack_bf16x2(r.x, r.y), pack_bf16x2(r.z, 0.f));
            __stcs(racc + v, make_float4(0.f, 0.f, 0.f, 0.f));
        }
        if (sacc) {
            constexpr int kCap = NS4 > 0 ? NS4 : 8;  // n_sem <= 32
            float4* sp = sacc + (int64_t)ns4 * v;
            float4 x[kCap];
            float nn = 0.f;
#pragma unroll
            for (int q = 0; q < kCap; ++q) {
                x[q] = q < ns4 ? __ldcs(sp + q) : make_float4(0.f, 0.f, 0.f, 0.f);
                nn += x[q].x * x[q].x + x[q].y * x[q].y + x[q].z * x[q].z + x[q].w * x[q].w;
            }
            const float inv = nn > 0.f ? 1.0f / sqrtf(nn) : 0.f;
#pragma unroll
            for (int q = 0; q < kCap; ++q) {
                if (q < ns4) {
                    if (fused)
                        sem[(int64_t)ns4 * v + q] = make_uint2(pack_bf16x2(x[q].x * inv, x[q].y * inv),
                                                               pack_bf16x2(x[q].z * inv, x[q].w * inv));
                    __stcs(sp + q, make_float4(0.f, 0.f, 0.f, 0.f));
                }
            }
        }
    }
}

}  // namespace
}  // namespace sdg

using namespace sdg;

extern "C" int sdg_fuse_frames(sdg_grid g, int64_t F, int H, int W, const float* depth, const float* rgb,
                               const float* sem, const float* K, const float* Twc, float mu) {
    if (!g || F < 0 || H <= 0 || W <= 0 || (F > 0 && (!depth || !K || !Twc)))
        return fail(SDG_ERR_ARG, "sdg_fuse_frames: null argument or empty image size");
    if (!(mu > 0.f)) return fail(SDG_ERR_ARG, "sdg_fuse_frames: mu must be > 0");
    if ((int64_t)H * W > ((int64_t)1 << 31))
        return fail(SDG_ERR_ARG, "sdg_fuse_frames: at most 2^31 pixels per frame");
    if (sem && g->desc.n_sem == 0) return fail(SDG_ERR_ARG, "sdg_fuse_frames: logits given but the grid has none");
    int rc = use_device(g);
    if (rc) return rc;
    if (F == 0 || g->n_blocks == 0) return SDG_OK;
    std::vector<FuseCam> cams((size_t)F);
    for (int64_t i = 0; i < F; ++i) {
        FuseCam& c = cams[(size_t)i];
        const float* T = Twc + 12 * i;
        for (int r = 0; r < 3; ++r) {
            for (int j = 0; j < 3; ++j) c.R[3 * r + j] = T[4 * r + j];
            c.t[r] = T[4 * r + 3];
        }
        c.fx = K[4 * i];
        c.fy = K[4 * i + 1];
        c.cx = K[4 * i + 2];
        c.cy = K[4 * i + 3];
        if (!(c.fx > 0.f && c.fy > 0.f)) return fail(SDG_ERR_ARG, "sdg_fuse_frames: fx and fy must be > 0");
    }
    if (g->fuse_cam_cap < F) {
        if (g->fuse_cams) {
            SDG_CUDA_TRY(cudaStreamSynchronize(g->stream));
            cudaFree(g->fuse_cams);
        }
        g->fuse_cams = nullptr;
        g->fuse_cam_cap = 0;
        SDG_CUDA_TRY(cudaMalloc(&g->fuse_cams, sizeof(FuseCam) * (size_t)F));
        g->fuse_cam_cap = F;
    }
    // from pageable memory: returns once the host array has been staged, so it may go out of scope
    SDG_CUDA_TRY(cudaMemcpyAsync(g->fuse_cams, cams.data(), sizeof(FuseCam) * (size_t)F, cudaMemcpyHostToDevice,
                                 g->stream));
    const bool bf16 = g->desc.rgb_dtype == SDG_BF16;
    const bool with_sem = sem != nullptr;
    FuseArgs a{};
    a.keys = g->keys;
    a.vs = g->desc.voxel_size;
    a.mu = mu;
    a.H = H;
    a.W = W;
    a.ns = g->desc.n_sem;
    a.sem4 = with_sem && a.ns % 4 == 0 && ((uintptr_t)sem & 15u) == 0;
    a.geo = g->geo;
    a.sdf = g->sdf;
    a.racc = g->grgb;
    a.sacc = g->gsem;
    a.weight = g->weight;
    const int64_t HW = (int64_t)H * W;
    for (int64_t f0 = 0; f0 < F; f0 += kFuseMaxFrames) {
        a.F = (int)std::min<int64_t>(kFuseMaxFrames, F - f0);
        a.cams = reinterpret_cast<const FuseCam*>(g->fuse_cams) + f0;
        a.depth = depth + f0 * HW;
        a.rgb = rgb ? rgb + f0 * HW * 3 : nullptr;
        a.sem = with_sem ? sem + f0 * HW * a.ns : nullptr;
        const unsigned blocks = (unsigned)g->n_blocks;
        if (!bf16 && !with_sem) k_fuse<true, false><<<blocks, kFuseThreads, 0, g->stream>>>(a);
        else if (!bf16) k_fuse<true, true><<<blocks, kFuseThreads, 0, g->stream>>>(a);
        else if (!with_sem) k_fuse<false, false><<<blocks, kFuseThreads, 0, g->stream>>>(a);
        else k_fuse<false, true><<<blocks, kFuseThreads, 0, g->stream>>>(a);
        SDG_LAUNCH_CHECK("fuse");
    }
    return SDG_OK;
}

extern "C" int sdg_fuse_finalize(sdg_grid g) {
    if (!g) return fail(SDG_ERR_ARG, "sdg_fuse_finalize: null grid");
    int rc = use_device(g);
    if (rc) return rc;
    const bool bf16 = g->desc.rgb_dtype == SDG_BF16;
    const int ns = g->desc.n_sem;
    if ((!bf16 && ns == 0) || g->n_blocks == 0) return SDG_OK;
    const int64_t V = g->n_blocks * 512;
    const int blocks = (int)std::min<int64_t>((V + 255) / 256, 148 * 16);
    float4* racc = bf16 ? g->grgb : nullptr;
    float4* sacc = ns ? reinterpret_cast<float4*>(g->gsem) : nullptr;
    uint2* sem = reinterpret_cast<uint2*>(g->sem);
    if (ns == 20) k_fuse_finalize<5><<<blocks, 256, 0, g->stream>>>(V, g->weight, racc, g->rgbh, sacc, sem, 5);
    else k_fuse_finalize<0><<<blocks, 256, 0, g->stream>>>(V, g->weight, racc, g->rgbh, sacc, sem, ns / 4);
    SDG_LAUNCH_CHECK("fuse finalize");
    return SDG_OK;
}
