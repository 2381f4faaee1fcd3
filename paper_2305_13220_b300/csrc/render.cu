// Rendering entry points: forward, backward (recompute or stored samples),
// rendering losses and the fused training pass.  Paper: arXiv 2305.13220,
// Sec. 3.5.1 (Eq. 12-15), Sec. 3.5.4 and the supplement's hyper-parameters.
#include <mutex>
#include <new>

#include "internal.h"
#include "reduce.cuh"
#include "render_core.cuh"

using namespace sdg;

struct sdg_ctx_s {
    sdg_grid g;
    const float* rays;
    int64_t n;
    sdg_render_opts opts;
    int Q;
    float* rec;  // store mode
    float* rec_S;
};

namespace {

// Smallest batch that SDG_ORDER_AUTO puts in surface order.
constexpr int64_t kAutoSurfaceOrderRays = 65536;

int pick_q(int N) { return N <= 64 ? 2 : N <= 128 ? 4 : N <= 192 ? 6 : 8; }

// Records the grid's pass event `which` (sdg_grid_set_pass_events) on its stream, if one is set.
int pass_event(sdg_grid g, int which) {
    if (g->pass_ev[which]) SDG_CUDA_TRY(cudaEventRecord(g->pass_ev[which], g->stream));
    return SDG_OK;
}

// a with the list sizing hints: the overflow- and mid-list lengths the grid's last pass with traversal records
// stored in its pinned words h_over (a kernel writes them as it runs, the host reads whatever is there: they only
// size launches)
PassArgs with_over_hint(sdg_grid g, const PassArgs& a) {
    PassArgs b = a;
    if (a.walk.hdr && g->h_over) {
        b.over_hint = reinterpret_cast<volatile int*>(g->h_over)[0];
        b.mid_hint = reinterpret_cast<volatile int*>(g->h_over)[1];
        b.over_out = g->h_over;
    }
    return b;
}

template <int MODE>
int launch_pass(sdg_grid g, const float* rays, uint32_t id0, const PassArgs& a) {
    if (a.n == 0) return SDG_OK;
    const GridDev gd = g->dev();
    const int Q = pick_q(a.N);
    int rc = pass_event(g, 0);
    if (rc) return rc;
    rc = launch_layout<MODE>(g->desc.rgb_dtype == SDG_BF16, g->desc.n_sem, gd, rays, id0, with_over_hint(g, a), Q,
                             g->stream);
    return rc ? rc : pass_event(g, 1);
}

// Same for passes instantiated only for grids without logits.
template <int MODE>
int launch_pass_nosem(sdg_grid g, const float* rays, uint32_t id0, const PassArgs& a) {
    if (a.n == 0) return SDG_OK;
    const GridDev gd = g->dev();
    const int Q = pick_q(a.N);
    int rc = pass_event(g, 0);
    if (rc) return rc;
    const PassArgs b = with_over_hint(g, a);
    if (g->desc.rgb_dtype == SDG_BF16) rc = launch_q<MODE, true, 0>(gd, rays, id0, b, Q, g->stream);
    else rc = launch_q<MODE, false, 0>(gd, rays, id0, b, Q, g->stream);
    return rc ? rc : pass_event(g, 1);
}

int check_opts(const sdg_render_opts* o) {
    if (!o || o->n_samples < 1 || o->n_samples > 256 || (o->mode != SDG_MODE_RECOMPUTE && o->mode != SDG_MODE_STORE))
        return fail(SDG_ERR_ARG, "render opts: n_samples must be in [1, 256] and mode RECOMPUTE or STORE");
    return SDG_OK;
}

PassArgs base_args(const sdg_render_opts* o, int64_t n) {
    PassArgs a{};
    a.N = o->n_samples;
    a.seed = o->seed;
    a.strat = o->stratified ? 1 : 0;
    a.bg[0] = o->bg[0];
    a.bg[1] = o->bg[1];
    a.bg[2] = o->bg[2];
    a.n = n;
    return a;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// ---------------------------------------------------------------------------
// Traversal pass (Sec. 3.5.1: samples only where blocks are allocated): one thread walks the whole ray through
// the dense block-index grid and writes the allocated cells it crosses, in order, with their skip-space offsets.
// A warp of the render kernel then places its ray's samples by a binary search over these records instead of
// walking the ray itself (a ray crossing more than kWalkCap allocated cells -- 0.15% of the room step's rays --
// keeps the in-warp traversal).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_walk(GridDev g, const float* __restrict__ rays, const int* __restrict__ perm,
                                              int64_t n, WalkBufs w) {
    const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= n) return;
    int64_t r = perm ? (int64_t)__ldg(perm + slot) : slot;
    if (!sdg_in_range(g.status, r, n, SDG_CHECK_RAY)) r = 0;  // checked build: a bad order row reads ray 0
    const float4 r0 = __ldg(reinterpret_cast<const float4*>(rays) + 2 * r);
    const float4 r1 = __ldg(reinterpret_cast<const float4*>(rays) + 2 * r + 1);
    walk_ray_records(g, make_float3(r0.x, r0.y, r0.z), make_float3(r1.x, r1.y, r1.z), r0.w, r1.w, w, slot);
}

}  // namespace

namespace sdg {
// Blocks until the grid's stream and its auxiliary stream are idle.
int drain_streams(sdg_grid g) {
    SDG_CUDA_TRY(cudaStreamSynchronize(g->stream));
    if (g->aux) SDG_CUDA_TRY(cudaStreamSynchronize(g->aux));
    return SDG_OK;
}

void free_batch(BatchBufs& b) {
    void* ptrs[] = {b.order_keys, b.order_perm, b.order_hist, b.walk_hdr, b.walk_s0, b.walk_rec, b.walk_over};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    b = BatchBufs{};
}

// Grows the walk records of b to n rays (valid until the next pass that uses b).
int walk_scratch(sdg_grid g, BatchBufs& b, int64_t n) {
    if (b.walk_cap >= n) return SDG_OK;
    if (b.walk_hdr || b.walk_s0 || b.walk_rec || b.walk_over) {
        int rc = drain_streams(g);  // earlier work may still read them
        if (rc) return rc;
        cudaFree(b.walk_hdr);
        cudaFree(b.walk_s0);
        cudaFree(b.walk_rec);
        cudaFree(b.walk_over);
    }
    b.walk_hdr = nullptr;
    b.walk_s0 = nullptr;
    b.walk_rec = nullptr;
    b.walk_over = nullptr;
    b.walk_cap = 0;
    SDG_CUDA_TRY(cudaMalloc((void**)&b.walk_hdr, sizeof(int2) * n));
    SDG_CUDA_TRY(cudaMalloc((void**)&b.walk_s0, sizeof(float) * kWalkSlot * n));
    SDG_CUDA_TRY(cudaMalloc((void**)&b.walk_rec, sizeof(int4) * kWalkSlot * n));
    // the overflow list [n], the mid list [n], their lengths at [2n] and [2n + 1]
    SDG_CUDA_TRY(cudaMalloc((void**)&b.walk_over, sizeof(int) * (2 * n + 2)));
    b.walk_cap = n;
    return SDG_OK;
}

// The records of b as the render kernels read them.
WalkBufs walk_bufs(const BatchBufs& b) {
    const int64_t n = b.walk_cap;
    return WalkBufs{b.walk_hdr,          b.walk_s0,         b.walk_rec,         b.walk_over,
                    b.walk_over + 2 * n, b.walk_over + n,   b.walk_over + 2 * n + 1};
}

int walk_rays_into(sdg_grid g, BatchBufs& b, cudaStream_t st, const float* rays, const int* perm, int64_t n,
                   PassArgs& a) {
    a.walk = WalkBufs{};
    if (n == 0) return SDG_OK;
    int rc = walk_scratch(g, b, n);
    if (rc) return rc;
    const WalkBufs w = walk_bufs(b);
    SDG_CUDA_TRY(cudaMemsetAsync(w.n_over, 0, 2 * sizeof(int), st));  // n_over and n_mid
    k_walk<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g->dev(), rays, perm, n, w);
    SDG_LAUNCH_CHECK("traversal pass");
    a.walk = w;
    return SDG_OK;
}

// Enqueues the traversal pass of n rays (processing order perm, or the given order) on the grid's stream into its
// batch scratch and points a.walk at the records.
int walk_rays(sdg_grid g, const float* rays, const int* perm, int64_t n, PassArgs& a) {
    return walk_rays_into(g, g->batch, g->stream, rays, perm, n, a);
}
}  // namespace sdg

namespace {

// ---------------------------------------------------------------------------
// Losses
// ---------------------------------------------------------------------------
__global__ void k_loss_l1(int64_t n, int ns, const float* __restrict__ rgb, const float* __restrict__ depth,
                          const float* __restrict__ sem, const float* __restrict__ trgb,
                          const float* __restrict__ tdepth, const float* __restrict__ tsem, float lam_d, float lam_s,
                          float inv_n, float* grgb, float* gdepth, float* gsem, float* loss) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float third = inv_n * (1.0f / 3.0f);
        float L = 0.f;
        for (int c = 0; c < 3; ++c) {
            const float e = rgb[3 * i + c] - trgb[3 * i + c];
            L += fabsf(e) * third;
            grgb[3 * i + c] = sgnf(e) * third;
        }
        const float ed = depth[i] - tdepth[i];
        L += lam_d * fabsf(ed) * inv_n;
        gdepth[i] = lam_d * sgnf(ed) * inv_n;
        if (sem && tsem)
            for (int c = 0; c < ns; ++c) {
                const float es = sem[i * ns + c] - tsem[i * ns + c];
                L += lam_s * es * es * inv_n;
                if (gsem) gsem[i * ns + c] = 2.f * lam_s * es * inv_n;
            }
        if (loss) loss[i] = L;
    }
}

// Least-squares alignment (a, b) of the targets t to the rendered depths D (scale/shift-invariant depth loss):
// FP64 sums of t, D, t^2, t D in a fixed order by one block, then the 2x2 normal equations; targets without
// spread leave the scale undetermined, and a = 1, b = mean(D - t).
__global__ void __launch_bounds__(1024) k_ssi_fit(const float* __restrict__ D, const float* __restrict__ t,
                                                  int64_t n, double* ab) {
    __shared__ double s[4][1024];
    double st = 0.0, sd = 0.0, stt = 0.0, std_ = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 1024) {
        const double ti = t[i], di = D[i];
        st += ti;
        sd += di;
        stt += ti * ti;
        std_ += ti * di;
    }
    s[0][threadIdx.x] = st;
    s[1][threadIdx.x] = sd;
    s[2][threadIdx.x] = stt;
    s[3][threadIdx.x] = std_;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < 4; ++q) s[q][threadIdx.x] += s[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double nn = (double)n, T = s[0][0], Dd = s[1][0], TT = s[2][0], TD = s[3][0];
        const double det = nn * TT - T * T;
        double a = 1.0, b = (Dd - T) / nn;
        if (det > 1e-12 * nn * TT) {
            a = (nn * TD - T * Dd) / det;
            b = (Dd - a * T) / nn;
        }
        ab[0] = a;
        ab[1] = b;
    }
}

// (lambda/n)(D - a t - b)^2 per ray and its derivative 2 lambda (D - a t - b)/n (the envelope theorem: a and b
// are at their optimum, so their own dependence on D adds nothing).
__global__ void k_ssi_seeds(const float* __restrict__ D, const float* __restrict__ t, int64_t n,
                            const double* __restrict__ ab, float lam_over_n, float* __restrict__ g_depth,
                            float* __restrict__ loss) {
    const float a = (float)ab[0], b = (float)ab[1];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float r = D[i] - fmaf(a, t[i], b);
        if (g_depth) g_depth[i] = 2.f * lam_over_n * r;
        if (loss) loss[i] = lam_over_n * r * r;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------
namespace sdg {
int loss_scratch(sdg_grid g, int64_t n, float** out) {
    if (g->loss_cap < n) {
        if (g->loss_buf) {
            SDG_CUDA_TRY(cudaStreamSynchronize(g->stream));  // earlier work on the stream may still read it
            cudaFree(g->loss_buf);
        }
        g->loss_buf = nullptr;
        g->loss_cap = 0;
        SDG_CUDA_TRY(cudaMalloc((void**)&g->loss_buf, sizeof(float) * n));
        g->loss_cap = n;
    }
    *out = g->loss_buf;
    return SDG_OK;
}
}  // namespace sdg

extern "C" int sdg_render_forward(sdg_grid g, const float* rays, int64_t n, const sdg_render_opts* o,
                                  const sdg_render_out* out, sdg_ctx* ctx) {
    if (ctx) *ctx = nullptr;
    if (!g || !out || n < 0 || (n > 0 && (!rays || !out->rgb || !out->depth || !out->opac)))
        return fail(SDG_ERR_ARG, "sdg_render_forward: null argument");
    int rc = check_opts(o);
    if (rc) return rc;
    if (n > 0 && !aligned16(rays)) return fail(SDG_ERR_ARG, "sdg_render_forward: rays must be 16-byte aligned");
    if (n > (int64_t)1 << 31) return fail(SDG_ERR_ARG, "sdg_render_forward: at most 2^31 rays per call");
    if ((rc = use_device(g))) return rc;
    PassArgs a = base_args(o, n);
    a.out_rgb = out->rgb;
    a.out_depth = out->depth;
    a.out_opac = out->opac;
    a.out_sem = g->desc.n_sem ? out->sem : nullptr;
    const int Q = pick_q(o->n_samples);
    float *rec = nullptr, *rec_S = nullptr;
    const bool store = o->mode == SDG_MODE_STORE && ctx;
    if (store && n > 0) {
        SDG_CUDA_TRY(cudaMallocAsync((void**)&rec, sizeof(float) * kRecChannels * (size_t)n * 32 * Q, g->stream));
        cudaError_t e = cudaMallocAsync((void**)&rec_S, sizeof(float) * (size_t)n, g->stream);
        if (e != cudaSuccess) {
            cudaFreeAsync(rec, g->stream);
            return cuda_fail(e, "cudaMallocAsync(store records)");
        }
        a.rec = rec;
        a.rec_S = rec_S;
        rc = walk_rays(g, rays, nullptr, n, a);
        if (!rc) rc = launch_pass<PASS_FWD_STORE>(g, rays, o->ray_id0, a);
    } else {
        rc = walk_rays(g, rays, nullptr, n, a);
        if (!rc) rc = launch_pass<PASS_FWD>(g, rays, o->ray_id0, a);
    }
    if (rc) {
        if (rec) cudaFreeAsync(rec, g->stream);
        if (rec_S) cudaFreeAsync(rec_S, g->stream);
        return rc;
    }
    if (ctx) {
        sdg_ctx c = new (std::nothrow) sdg_ctx_s{g, rays, n, *o, Q, rec, rec_S};
        if (!c) {
            if (rec) cudaFreeAsync(rec, g->stream);
            if (rec_S) cudaFreeAsync(rec_S, g->stream);
            return fail(SDG_ERR_OOM, "context");
        }
        c->opts.mode = store ? SDG_MODE_STORE : SDG_MODE_RECOMPUTE;
        *ctx = c;
    }
    return SDG_OK;
}

extern "C" int sdg_render_backward(sdg_ctx c, const float* g_rgb, const float* g_depth, const float* g_opac,
                                   const float* g_sem) {
    if (!c || (c->n > 0 && !g_rgb)) return fail(SDG_ERR_ARG, "sdg_render_backward: null argument");
    sdg_grid g = c->g;
    int rc = use_device(g);
    if (rc) return rc;
    PassArgs a = base_args(&c->opts, c->n);
    a.g_rgb = g_rgb;
    a.g_depth = g_depth;
    a.g_opac = g_opac;
    a.g_sem = g->desc.n_sem ? g_sem : nullptr;
    if (c->opts.mode == SDG_MODE_STORE && c->rec) {
        a.rec = c->rec;
        a.rec_S = c->rec_S;
        return launch_pass<PASS_BWD_STORE>(g, c->rays, c->opts.ray_id0, a);
    }
    if ((rc = walk_rays(g, c->rays, nullptr, c->n, a))) return rc;  // the forward's records, recomputed
    return launch_pass<PASS_BWD>(g, c->rays, c->opts.ray_id0, a);
}

extern "C" int sdg_ctx_release(sdg_ctx c) {
    if (!c) return SDG_OK;
    cudaSetDevice(c->g->device);
    if (c->rec) cudaFreeAsync(c->rec, c->g->stream);
    if (c->rec_S) cudaFreeAsync(c->rec_S, c->g->stream);
    delete c;
    return SDG_OK;
}

extern "C" int sdg_loss_l1(sdg_grid g, int64_t n, const float* rgb, const float* depth, const float* sem,
                           const float* trgb, const float* tdepth, const float* tsem, const sdg_loss_opts* lo,
                           float* grgb, float* gdepth, float* gsem, float* loss) {
    if (!g || !lo || n < 0 || (n > 0 && (!rgb || !depth || !trgb || !tdepth || !grgb || !gdepth)))
        return fail(SDG_ERR_ARG, "sdg_loss_l1: null argument");
    int rc = use_device(g);
    if (rc) return rc;
    if (n == 0) return SDG_OK;
    const int ns = g->desc.n_sem;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 16);
    k_loss_l1<<<blocks, 256, 0, g->stream>>>(n, ns, rgb, depth, ns ? sem : nullptr, trgb, tdepth, ns ? tsem : nullptr,
                                             lo->lambda_depth, lo->lambda_sem, 1.0f / (float)n, grgb, gdepth,
                                             ns ? gsem : nullptr, loss);
    SDG_LAUNCH_CHECK("loss");
    return SDG_OK;
}

extern "C" int sdg_train_step_rays(sdg_grid g, const float* rays, int64_t n, const float* trgb, const float* tdepth,
                                   const float* tsem, const sdg_render_opts* o, const sdg_loss_opts* lo, float* loss,
                                   float* loss_sum) {
    if (!g || !lo || n < 0 || (n > 0 && (!rays || !trgb || !tdepth)))
        return fail(SDG_ERR_ARG, "sdg_train_step_rays: null argument");
    int rc = check_opts(o);
    if (rc) return rc;
    if (n > 0 && !aligned16(rays)) return fail(SDG_ERR_ARG, "sdg_train_step_rays: rays must be 16-byte aligned");
    if (n > (int64_t)1 << 31) return fail(SDG_ERR_ARG, "sdg_train_step_rays: at most 2^31 rays per call");
    if (lo->ray_order != SDG_ORDER_AUTO && lo->ray_order != SDG_ORDER_GIVEN && lo->ray_order != SDG_ORDER_SURFACE)
        return fail(SDG_ERR_ARG, "sdg_train_step_rays: unknown ray_order");
    if (lo->prepared < 0 || lo->prepared > 2 || lo->reserved != 0)
        return fail(SDG_ERR_ARG, "sdg_train_step_rays: prepared must be 0, 1 or 2 and reserved 0");
    if ((rc = use_device(g))) return rc;
    if (n == 0) {
        if (loss_sum) SDG_CUDA_TRY(cudaMemsetAsync(loss_sum, 0, sizeof(float), g->stream));
        return SDG_OK;
    }
    float* per_ray = loss;
    if (!per_ray && loss_sum) {
        if ((rc = loss_scratch(g, n, &per_ray))) return rc;
    }
    PassArgs a = base_args(o, n);
    a.t_rgb = trgb;
    a.t_depth = tdepth;
    a.t_sem = g->desc.n_sem ? tsem : nullptr;
    a.lam_d = lo->lambda_depth;
    a.lam_s = lo->lambda_sem;
    a.inv_n = 1.0f / (float)(lo->norm_rays > 0 ? lo->norm_rays : n);
    a.loss = per_ray;
    if (lo->prepared) {
        PreparedBatch& P = g->prep[lo->prepared - 1];
        if (!P.valid || P.rays != rays || P.n != n)
            return fail(SDG_ERR_ARG, "sdg_train_step_rays: the prepared slot does not hold these rays");
        SDG_CUDA_TRY(cudaStreamWaitEvent(g->stream, P.ready, 0));
        a.perm = P.perm;
        a.walk = walk_bufs(P.b);
        P.valid = false;
    } else {
        if (lo->ray_order == SDG_ORDER_SURFACE || (lo->ray_order == SDG_ORDER_AUTO && n >= kAutoSurfaceOrderRays)) {
            if ((rc = order_rays_by_surface(g, rays, tdepth, n, &a.perm))) return rc;
        }
        if ((rc = walk_rays(g, rays, a.perm, n, a))) return rc;
    }
    if (lo->learn_beta) {
        if (g->beta_part_cap < n) {
            if (g->beta_part) {
                SDG_CUDA_TRY(cudaStreamSynchronize(g->stream));
                cudaFree(g->beta_part);
            }
            g->beta_part = nullptr;
            g->beta_part_cap = 0;
            SDG_CUDA_TRY(cudaMalloc((void**)&g->beta_part, sizeof(float) * n));
            g->beta_part_cap = n;
        }
        a.beta_part = g->beta_part;
        rc = launch_pass<PASS_TRAIN_BETA>(g, rays, o->ray_id0, a);
        if (rc) return rc;
        launch_sum<true>(g->beta_part, n, g->beta_grad, g->sum_scratch, g->stream);  // dL/dbeta += sum over rays
        SDG_LAUNCH_CHECK("beta gradient sum");
        g->beta_grad_pending = true;
    } else {
        rc = launch_pass<PASS_TRAIN>(g, rays, o->ray_id0, a);
        if (rc) return rc;
    }
    if (loss_sum) {
        launch_sum(per_ray, n, loss_sum, g->sum_scratch, g->stream);
        SDG_LAUNCH_CHECK("loss sum");
    }
    return SDG_OK;
}

extern "C" int sdg_train_step_rays_normal(sdg_grid g, const float* rays, int64_t n, const float* trgb,
                                          const float* tdepth, const float* tnormal, const sdg_render_opts* o,
                                          const sdg_loss_opts* lo, float lambda_normal, float* loss,
                                          float* loss_sum) {
    if (!g || !lo || n < 0 || (n > 0 && (!rays || !trgb || !tdepth || !tnormal)))
        return fail(SDG_ERR_ARG, "sdg_train_step_rays_normal: null argument");
    int rc = check_opts(o);
    if (rc) return rc;
    if (n > 0 && !aligned16(rays))
        return fail(SDG_ERR_ARG, "sdg_train_step_rays_normal: rays must be 16-byte aligned");
    if (n > (int64_t)1 << 31) return fail(SDG_ERR_ARG, "sdg_train_step_rays_normal: at most 2^31 rays per call");
    if (g->desc.n_sem) return fail(SDG_ERR_ARG, "sdg_train_step_rays_normal: grids with logits are not supported");
    if (lo->learn_beta) return fail(SDG_ERR_ARG, "sdg_train_step_rays_normal: learn_beta is not supported");
    if (lo->prepared) return fail(SDG_ERR_ARG, "sdg_train_step_rays_normal: prepared batches are not supported");
    if (lo->ray_order != SDG_ORDER_AUTO && lo->ray_order != SDG_ORDER_GIVEN && lo->ray_order != SDG_ORDER_SURFACE)
        return fail(SDG_ERR_ARG, "sdg_train_step_rays_normal: unknown ray_order");
    if ((rc = use_device(g))) return rc;
    if (n == 0) {
        if (loss_sum) SDG_CUDA_TRY(cudaMemsetAsync(loss_sum, 0, sizeof(float), g->stream));
        return SDG_OK;
    }
    float* per_ray = loss;
    if (!per_ray && loss_sum && (rc = loss_scratch(g, n, &per_ray))) return rc;
    PassArgs a = base_args(o, n);
    a.t_rgb = trgb;
    a.t_depth = tdepth;
    a.t_normal = tnormal;
    a.lam_d = lo->lambda_depth;
    a.lam_n = lambda_normal;
    a.inv_n = 1.0f / (float)(lo->norm_rays > 0 ? lo->norm_rays : n);
    a.loss = per_ray;
    if (lo->ray_order == SDG_ORDER_SURFACE || (lo->ray_order == SDG_ORDER_AUTO && n >= kAutoSurfaceOrderRays)) {
        if ((rc = order_rays_by_surface(g, rays, tdepth, n, &a.perm))) return rc;
    }
    if ((rc = walk_rays(g, rays, a.perm, n, a))) return rc;
    rc = launch_pass_nosem<PASS_TRAIN_NRM>(g, rays, o->ray_id0, a);
    if (rc) return rc;
    if (loss_sum) {
        launch_sum(per_ray, n, loss_sum, g->sum_scratch, g->stream);
        SDG_LAUNCH_CHECK("loss sum");
    }
    return SDG_OK;
}

extern "C" int sdg_loss_depth_ssi(sdg_grid g, int64_t n, const float* depth, const float* t_depth, float lambda,
                                  float* g_depth, float* loss, float* loss_sum, double* ab_host) {
    if (!g || n < 0 || (n > 0 && (!depth || !t_depth))) return fail(SDG_ERR_ARG, "sdg_loss_depth_ssi: null argument");
    int rc = use_device(g);
    if (rc) return rc;
    if (n == 0) {
        if (loss_sum) SDG_CUDA_TRY(cudaMemsetAsync(loss_sum, 0, sizeof(float), g->stream));
        return SDG_OK;
    }
    k_ssi_fit<<<1, 1024, 0, g->stream>>>(depth, t_depth, n, g->ssi_dev);
    SDG_LAUNCH_CHECK("depth alignment");
    float* per_ray = loss;
    if (!per_ray && loss_sum && (rc = loss_scratch(g, n, &per_ray))) return rc;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 16);
    k_ssi_seeds<<<blocks, 256, 0, g->stream>>>(depth, t_depth, n, g->ssi_dev, lambda / (float)n, g_depth, per_ray);
    SDG_LAUNCH_CHECK("depth loss");
    if (loss_sum) {
        launch_sum(per_ray, n, loss_sum, g->sum_scratch, g->stream);
        SDG_LAUNCH_CHECK("depth loss sum");
    }
    if (ab_host) {
        SDG_CUDA_TRY(cudaMemcpyAsync(ab_host, g->ssi_dev, 2 * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
        SDG_CUDA_TRY(cudaStreamSynchronize(g->stream));
    }
    return SDG_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free fused training pass: the per-ray loss scratch is a fixed
// array in the library image instead of a cudaMalloc'd buffer.
// ---------------------------------------------------------------------------
namespace {
constexpr int64_t kNoAllocMaxRays = 1 << 20;  // 4 MiB of FP32 per-ray loss terms
static __device__ __align__(256) float g_noalloc_loss[kNoAllocMaxRays];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
float* g_noalloc_ptr[kNoAllocMaxDevices] = {};  // device address of g_noalloc_loss, per device ordinal

// Resolves (once per device, with that device current) the device address of
// the scratch array; host code must not pass the symbol itself to a kernel.
int noalloc_scratch(int device, float** out) {
    if (device < 0 || device >= kNoAllocMaxDevices) return fail(SDG_ERR_ARG, "no-alloc scratch: bad device ordinal");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        float* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_loss);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_noalloc_ptr[device] = p;
    }
    *out = g_noalloc_ptr[device];
    return SDG_OK;
}
}  // namespace

extern "C" int sdg_train_step_rays_noalloc(sdg_grid g, const float* rays, int64_t n, const float* trgb,
                                           const float* tdepth, const float* tsem, const sdg_render_opts* o,
                                           const sdg_loss_opts* lo, float* loss_sum) {
    if (!g || !lo || n < 0 || (n > 0 && (!rays || !trgb || !tdepth)))
        return fail(SDG_ERR_ARG, "sdg_train_step_rays_noalloc: null argument");
    if (lo->learn_beta)  // dL/dbeta needs a per-ray partial buffer this entry point does not have
        return fail(SDG_ERR_ARG, "sdg_train_step_rays_noalloc: learn_beta is not supported");
    if (lo->prepared)  // a prepared batch lives in grid-owned scratch
        return fail(SDG_ERR_ARG, "sdg_train_step_rays_noalloc: prepared batches are not supported");
    if (n > kNoAllocMaxRays)
        return fail(SDG_ERR_CAPACITY, "sdg_train_step_rays_noalloc: n = " + std::to_string(n) +
                                          " rays exceeds the fixed scratch capacity of 1048576 rays");
    int rc = check_opts(o);
    if (rc) return rc;
    if (n > 0 && !aligned16(rays))
        return fail(SDG_ERR_ARG, "sdg_train_step_rays_noalloc: rays must be 16-byte aligned");
    if ((rc = use_device(g))) return rc;
    float* scratch = nullptr;
    if ((rc = noalloc_scratch(g->device, &scratch))) return rc;
    if (n == 0) {
        if (loss_sum) SDG_CUDA_TRY(cudaMemsetAsync(loss_sum, 0, sizeof(float), g->stream));
        return SDG_OK;
    }
    PassArgs a = base_args(o, n);
    a.t_rgb = trgb;
    a.t_depth = tdepth;
    a.t_sem = g->desc.n_sem ? tsem : nullptr;
    a.lam_d = lo->lambda_depth;
    a.lam_s = lo->lambda_sem;
    a.inv_n = 1.0f / (float)(lo->norm_rays > 0 ? lo->norm_rays : n);
    a.loss = loss_sum ? scratch : nullptr;  // every ray writes its entry before the sum reads it
    rc = launch_pass<PASS_TRAIN>(g, rays, o->ray_id0, a);
    if (rc) return rc;
    if (loss_sum) {
        launch_sum(scratch, n, loss_sum, g->sum_scratch, g->stream);
        SDG_LAUNCH_CHECK("no-alloc loss sum");
    }
    return SDG_OK;
}

extern "C" int sdg_grid_set_pass_events(sdg_grid g, void* start, void* stop) {
    if (!g || (!start) != (!stop)) return fail(SDG_ERR_ARG, "sdg_grid_set_pass_events: both events or neither");
    g->pass_ev[0] = (cudaEvent_t)start;
    g->pass_ev[1] = (cudaEvent_t)stop;
    return SDG_OK;
}

extern "C" int sdg_train_prepare(sdg_grid g, const float* rays, int64_t n, const float* tdepth,
                                 const sdg_loss_opts* lo, int32_t slot) {
    if (!g || !lo || n <= 0 || !rays || !tdepth || slot < 0 || slot > 1)
        return fail(SDG_ERR_ARG, "sdg_train_prepare: null argument, n <= 0 or slot not 0 or 1");
    if (!aligned16(rays)) return fail(SDG_ERR_ARG, "sdg_train_prepare: rays must be 16-byte aligned");
    if (n > (int64_t)1 << 31) return fail(SDG_ERR_ARG, "sdg_train_prepare: at most 2^31 rays per call");
    if (lo->ray_order != SDG_ORDER_AUTO && lo->ray_order != SDG_ORDER_GIVEN && lo->ray_order != SDG_ORDER_SURFACE)
        return fail(SDG_ERR_ARG, "sdg_train_prepare: unknown ray_order");
    int rc = use_device(g);
    if (rc) return rc;
    if (!g->aux) SDG_CUDA_TRY(cudaStreamCreateWithFlags(&g->aux, cudaStreamNonBlocking));
    PreparedBatch& P = g->prep[slot];
    if (!P.fence) SDG_CUDA_TRY(cudaEventCreateWithFlags(&P.fence, cudaEventDisableTiming));
    if (!P.ready) SDG_CUDA_TRY(cudaEventCreateWithFlags(&P.ready, cudaEventDisableTiming));
    P.valid = false;
    // after everything already on the grid's stream: the inputs, and the last pass that read this slot
    SDG_CUDA_TRY(cudaEventRecord(P.fence, g->stream));
    SDG_CUDA_TRY(cudaStreamWaitEvent(g->aux, P.fence, 0));
    const int* perm = nullptr;
    if (lo->ray_order == SDG_ORDER_SURFACE || (lo->ray_order == SDG_ORDER_AUTO && n >= kAutoSurfaceOrderRays)) {
        if ((rc = order_rays_into(g, P.b, g->aux, rays, tdepth, n, &perm))) return rc;
    }
    PassArgs a{};
    if ((rc = walk_rays_into(g, P.b, g->aux, rays, perm, n, a))) return rc;
    SDG_CUDA_TRY(cudaEventRecord(P.ready, g->aux));
    P.rays = rays;
    P.n = n;
    P.perm = perm;
    P.valid = true;
    return SDG_OK;
}
