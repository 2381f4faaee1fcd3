// Debug export of the sample placement (Sec. 3.5.1 skip-space sampling, Eq. 17 trilinear cells): the forward
// pass in PASS_FWD_TRACE mode writes, per sample, t_k, its cell and block and its validity, so that a test can
// feed exactly these samples to an independent implementation of the rest of the method.
#include "internal.h"
#include "render_kernels.cuh"

// Instantiated in the render_inst_*_fwd.cu files.
SDG_EXTERN_LAUNCH(sdg::PASS_FWD_TRACE, false, 0)
SDG_EXTERN_LAUNCH(sdg::PASS_FWD_TRACE, true, 0)
SDG_EXTERN_LAUNCH(sdg::PASS_FWD_TRACE, false, sdg::kSemCapSmall)
SDG_EXTERN_LAUNCH(sdg::PASS_FWD_TRACE, true, sdg::kSemCapSmall)
SDG_EXTERN_LAUNCH(sdg::PASS_FWD_TRACE, false, 32)
SDG_EXTERN_LAUNCH(sdg::PASS_FWD_TRACE, true, 32)

using namespace sdg;

namespace {

// The rays of an H x W pinhole view, one thread per pixel, formed by pinhole_ray as the serving kernels form them.
__global__ void __launch_bounds__(256) k_view_rays(int H, int W, Cam6 cam, float tnear, float tfar, float* rays_out) {
    const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= (int64_t)H * W) return;
    float3 o, d;
    pinhole_ray(cam.K, cam.T, (int)(pix % W), (int)(pix / W), o, d);
    float4* r = reinterpret_cast<float4*>(rays_out) + 2 * pix;
    r[0] = make_float4(o.x, o.y, o.z, tnear);
    r[1] = make_float4(d.x, d.y, d.z, tfar);
}

int pick_q(int N) { return N <= 64 ? 2 : N <= 128 ? 4 : N <= 192 ? 6 : 8; }

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int check_out(const sdg_trace_out* out, int64_t n) {
    if (!out) return fail(SDG_ERR_ARG, "trace: null output");
    if (n > 0 && (!out->n_cells || !out->S || !out->t || !out->cell || !out->block || !out->valid || !out->rgb ||
                  !out->depth || !out->opac))
        return fail(SDG_ERR_ARG, "trace: null output buffer");
    return SDG_OK;
}

PassArgs trace_args(const sdg_render_opts* o, int64_t n, const sdg_trace_out* out) {
    PassArgs a{};
    a.N = o->n_samples;
    a.seed = o->seed;
    a.strat = o->stratified ? 1 : 0;
    for (int c = 0; c < 3; ++c) a.bg[c] = o->bg[c];
    a.n = n;
    a.out_rgb = out->rgb;
    a.out_depth = out->depth;
    a.out_opac = out->opac;
    a.tr_ncell = out->n_cells;
    a.tr_S = out->S;
    a.tr_t = out->t;
    a.tr_cell = out->cell;
    a.tr_blk = out->block;
    a.tr_valid = out->valid;
    a.tr_seg = out->seg;
    return a;
}

int check_opts(const sdg_render_opts* o) {
    if (!o || o->n_samples < 1 || o->n_samples > 256) return fail(SDG_ERR_ARG, "trace: n_samples must be in [1, 256]");
    return SDG_OK;
}

}  // namespace

extern "C" int sdg_debug_trace(sdg_grid g, const float* rays, int64_t n, const sdg_render_opts* o, int32_t walk,
                               const sdg_trace_out* out) {
    if (!g || n < 0 || (n > 0 && !rays)) return fail(SDG_ERR_ARG, "sdg_debug_trace: null argument");
    int rc = check_opts(o);
    if (rc || (rc = check_out(out, n))) return rc;
    if (walk != SDG_WALK_PASS && walk != SDG_WALK_IN_WARP) return fail(SDG_ERR_ARG, "sdg_debug_trace: bad walk");
    if (n > 0 && !aligned16(rays)) return fail(SDG_ERR_ARG, "sdg_debug_trace: rays must be 16-byte aligned");
    if (n > (int64_t)1 << 31) return fail(SDG_ERR_ARG, "sdg_debug_trace: at most 2^31 rays per call");
    if ((rc = use_device(g))) return rc;
    if (n == 0) return SDG_OK;
    PassArgs a = trace_args(o, n, out);
    if (walk == SDG_WALK_PASS && (rc = walk_rays(g, rays, nullptr, n, a))) return rc;
    const GridDev gd = g->dev();
    const int Q = pick_q(o->n_samples);
    return launch_layout<PASS_FWD_TRACE>(g->desc.rgb_dtype == SDG_BF16, g->desc.n_sem, gd, rays, o->ray_id0, a, Q,
                                         g->stream);
}

extern "C" int sdg_debug_trace_view(sdg_grid g, int32_t H, int32_t W, const float K[4], const float T[12],
                                    float tnear, float tfar, const sdg_render_opts* o, float* rays_out,
                                    const sdg_trace_out* out) {
    if (!g || !K || !T || H <= 0 || W <= 0 || !rays_out || !(K[0] != 0.f) || !(K[1] != 0.f))
        return fail(SDG_ERR_ARG, "sdg_debug_trace_view: bad argument");
    const int64_t n = (int64_t)H * W;
    int rc = check_opts(o);
    if (rc || (rc = check_out(out, n))) return rc;
    if (!aligned16(rays_out)) return fail(SDG_ERR_ARG, "sdg_debug_trace_view: rays_out must be 16-byte aligned");
    if (n > (int64_t)1 << 31) return fail(SDG_ERR_ARG, "sdg_debug_trace_view: at most 2^31 pixels");
    if ((rc = use_device(g))) return rc;
    PassArgs a = trace_args(o, n, out);
    Cam6 cam;
    for (int i = 0; i < 4; ++i) cam.K[i] = K[i];
    for (int i = 0; i < 12; ++i) cam.T[i] = T[i];
    k_view_rays<<<(unsigned)((n + 255) / 256), 256, 0, g->stream>>>(H, W, cam, tnear, tfar, rays_out);
    SDG_LAUNCH_CHECK("view rays");
    // then as the serving loop renders them: the traversal pass, the records kernel and, for rays crossing more
    // than kWalkCap allocated cells, the in-warp kernel; the jitter's ray id is the pixel index
    if ((rc = walk_rays(g, rays_out, nullptr, n, a))) return rc;
    return launch_layout<PASS_FWD_TRACE>(g->desc.rgb_dtype == SDG_BF16, g->desc.n_sem, g->dev(), rays_out, 0u, a,
                                         pick_q(o->n_samples), g->stream);
}
