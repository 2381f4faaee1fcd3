// Per-ray warp program of the renderer: empty-space-skipping traversal,
// stratified sampling in allocated space, trilinear fetch, Laplace density,
// compositing and its backward.  Paper: arXiv 2305.13220, Sec. 3.5.1
// (Eq. 12-15) and Sec. 3.5.2 (Eq. 17, trilinear interpolation).
//
// Work decomposition (one warp = one ray):
//  * traversal: the ray's clipped range [t0, t1] is cut into 32 equal pieces;
//    lane j walks the block cells of piece j (a block-level Amanatides-Woo
//    walk against the occupancy bitmap) and sums the allocated length S_j.
//    A sequential shuffle prefix gives each lane its skip-space interval
//    [P_j, P_{j+1}) (monotone, so the lanes partition [0, S) exactly).
//  * sampling: lane j walks its piece again and writes t_k for the samples
//    whose s_k falls in its interval into the warp's shared-memory slots.
//  * sample work: lane l owns the Q consecutive samples l*Q .. l*Q+Q-1, so
//    consecutive samples of a lane usually share a voxel cell: the cell's 8
//    corners (one 16-byte load each in the FP32 layout) are fetched once
//    per cell, and in the backward the gradient of a run of same-cell
//    samples is summed in registers and sent with one vector atomic per
//    corner.  Transmittance is a warp scan over the lanes' optical depths.
#pragma once

#include "common.cuh"

namespace sdg {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kWarpsPerBlock = 8;

enum PassMode { PASS_FWD = 0, PASS_FWD_STORE = 1, PASS_BWD = 2, PASS_BWD_STORE = 3, PASS_TRAIN = 4 };

struct PassArgs {
    int N;  // samples per ray
    uint32_t seed;
    int strat;
    float bg[3];
    int64_t n;  // rays in this launch
    float *out_rgb, *out_depth, *out_opac, *out_sem;
    float* rec;    // store mode: [5][n][32*Q] (t, sdf or NaN if invalid, r, g, b)
    float* rec_S;  // store mode: [n]
    const float *g_rgb, *g_depth, *g_opac, *g_sem;
    const float *t_rgb, *t_depth, *t_sem;
    float lam_d, lam_s, inv_n;
    float* loss;
};

struct RayJob {
    float3 o, d;
    float tn, tf;
    uint32_t ray_id;
    int64_t idx;  // row of this ray in per-ray arrays
};

// ---------------------------------------------------------------------------
// Counter-based jitter: PCG hash (Jarzynski & Olano, JCGT 2020), nested over
// (seed, ray, k); u = top 24 bits * 2^-24.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pcg_hash(uint32_t v) {
    uint32_t state = v * 747796405u + 2891336453u;
    uint32_t word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
    return (word >> 22u) ^ word;
}
__device__ __forceinline__ float sample_u(uint32_t seed_h, uint32_t ray_id, int k) {
    uint32_t h = pcg_hash((uint32_t)k + pcg_hash(ray_id + seed_h));
    return (float)(h >> 8) * 5.9604644775390625e-8f;
}

struct SampleGen {
    float s_over_n, s_max;
    uint32_t seed_h, ray_id;
    int strat;
    __device__ __forceinline__ float s(int k) const {
        float u = strat ? sample_u(seed_h, ray_id, k) : 0.5f;
        return fminf(((float)k + u) * s_over_n, s_max);
    }
};

// ---------------------------------------------------------------------------
// Traversal
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool clip_to_grid(const GridDev& g, const float3& o, const float3& d, float& t0,
                                             float& t1) {
    if (g.n_blocks == 0) return false;
    const float oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float lo = (float)g.bmin[a] * g.L, hi = (float)(g.bmin[a] + g.bdim[a]) * g.L;
        if (dd[a] == 0.0f) {
            if (oo[a] < lo || oo[a] > hi) return false;
            continue;
        }
        float inv = 1.0f / dd[a];
        float ta = (lo - oo[a]) * inv, tb = (hi - oo[a]) * inv;
        t0 = fmaxf(t0, fminf(ta, tb));
        t1 = fminf(t1, fmaxf(ta, tb));
    }
    return t0 < t1;
}

__device__ __forceinline__ bool occupied(const GridDev& g, int cx, int cy, int cz) {
    int64_t bit = ((int64_t)cz * g.bdim[1] + cy) * (int64_t)g.bdim[0] + cx;
    return (__ldg(g.bitmap + (bit >> 5)) >> (bit & 31)) & 1u;
}

// Calls f(a, b) for every allocated stretch [a, b) of the ray inside [ta, tb),
// one call per allocated block cell, in order of increasing t.
template <class F>
__device__ __forceinline__ void walk_cells(const GridDev& g, const float3& o, const float3& d, const float3& invd,
                                           float ta, float tb, F&& f) {
    if (!(tb > ta)) return;
    const float INF = __int_as_float(0x7f800000);
    int cx = (int)floorf(fmaf(ta, d.x, o.x) * g.inv_L) - g.bmin[0];
    int cy = (int)floorf(fmaf(ta, d.y, o.y) * g.inv_L) - g.bmin[1];
    int cz = (int)floorf(fmaf(ta, d.z, o.z) * g.inv_L) - g.bmin[2];
    cx = min(max(cx, 0), g.bdim[0] - 1);
    cy = min(max(cy, 0), g.bdim[1] - 1);
    cz = min(max(cz, 0), g.bdim[2] - 1);
    const int sx = d.x > 0.f ? 1 : (d.x < 0.f ? -1 : 0);
    const int sy = d.y > 0.f ? 1 : (d.y < 0.f ? -1 : 0);
    const int sz = d.z > 0.f ? 1 : (d.z < 0.f ? -1 : 0);
    float tcur = ta;
    const int maxit = g.bdim[0] + g.bdim[1] + g.bdim[2] + 3;
    for (int it = 0; it < maxit; ++it) {
        float tx = sx ? ((float)(g.bmin[0] + cx + (sx > 0)) * g.L - o.x) * invd.x : INF;
        float ty = sy ? ((float)(g.bmin[1] + cy + (sy > 0)) * g.L - o.y) * invd.y : INF;
        float tz = sz ? ((float)(g.bmin[2] + cz + (sz > 0)) * g.L - o.z) * invd.z : INF;
        float te = fminf(tx, fminf(ty, tz));
        float b = fminf(te, tb);
        if (b > tcur && occupied(g, cx, cy, cz)) f(tcur, b);
        if (!(te < tb)) break;
        if (tx == te) cx += sx;
        if (ty == te) cy += sy;
        if (tz == te) cz += sz;
        tcur = fmaxf(te, ta);
        if ((unsigned)cx >= (unsigned)g.bdim[0] || (unsigned)cy >= (unsigned)g.bdim[1] ||
            (unsigned)cz >= (unsigned)g.bdim[2])
            break;
    }
}

// Traversal + sample placement.  Writes t_k and s_k (k < N) to ts/ss and
// s_N = S; returns S (0 when the ray sees no allocated block).
__device__ __forceinline__ float place_samples(const GridDev& g, const PassArgs& a, const RayJob& j, float* ts,
                                               float* ss, int lane, SampleGen& gen) {
    float t0 = j.tn, t1 = j.tf;
    float S_j = 0.f;
    const float3 invd = make_float3(1.0f / j.d.x, 1.0f / j.d.y, 1.0f / j.d.z);
    float ta = 0.f, tb = 0.f;
    const bool hit = clip_to_grid(g, j.o, j.d, t0, t1);
    if (hit) {
        const float dt = (t1 - t0) * (1.0f / 32.0f);
        ta = fmaf((float)lane, dt, t0);
        tb = lane == 31 ? t1 : fmaf((float)(lane + 1), dt, t0);
        walk_cells(g, j.o, j.d, invd, ta, tb, [&](float x0, float x1) { S_j += x1 - x0; });
    }
    // sequential prefix: P_{j+1} = fl(P_j + S_j) exactly, so the intervals tile [0, S)
    float P = 0.f;
#pragma unroll
    for (int i = 0; i < 31; ++i) {
        float v = __shfl_sync(kFull, S_j, i);
        if (i < lane) P += v;
    }
    const float S = __shfl_sync(kFull, P + S_j, 31);
    float hi = __shfl_down_sync(kFull, P, 1);
    if (lane == 31) hi = S;
    gen.s_over_n = S / (float)a.N;
    gen.s_max = __int_as_float(__float_as_int(S) - 1);  // largest float below S (S > 0)
    if (!(S > 0.f)) return 0.f;
    const int N = a.N;
    if (hi > P) {
        int k = max(0, (int)(P / gen.s_over_n) - 1);
        while (k < N && gen.s(k) < P) ++k;
        float scur = P, pa = 0.f, ps = 0.f, plen = 0.f;
        bool have = false;
        auto flush = [&](float bound) {
            while (k < N) {
                float sk = gen.s(k);
                if (!(sk < bound && sk < hi)) break;
                ts[k] = pa + fminf(fmaxf(sk - ps, 0.f), plen);
                ss[k] = sk;
                ++k;
            }
        };
        walk_cells(g, j.o, j.d, invd, ta, tb, [&](float x0, float x1) {
            if (have) flush(ps + plen);
            pa = x0;
            ps = scur;
            plen = x1 - x0;
            scur += plen;
            have = true;
        });
        if (have) flush(hi);
    }
    if (lane == 0) ss[N] = S;
    __syncwarp();
    return S;
}

// ---------------------------------------------------------------------------
// Voxel stencil of a cell (Eq. 17): the 8 grid points around x
// ---------------------------------------------------------------------------
struct BlockCache {
    uint64_t key;
    int32_t blk;
};

// Resolves the 8 corner voxel addresses of the cell whose base grid point is
// (cx, cy, cz).  False if any corner's block is not allocated.
__device__ __forceinline__ bool cell_addresses(const GridDev& g, int cx, int cy, int cz, BlockCache& bc, int addr[8]) {
    const uint64_t key = sdg_pack_key(cx >> 3, cy >> 3, cz >> 3);
    if (key != bc.key) {
        bc.key = key;
        bc.blk = sdg_table_find(g.table, g.mask, key);
    }
    const int b = bc.blk;
    if (b < 0) return false;
    const int lx = cx & 7, ly = cy & 7, lz = cz & 7;
    const int ovf = (lx == 7) | ((ly == 7) << 1) | ((lz == 7) << 2);
    int nb[8];
    if (ovf) {
        int4 n0 = __ldg(g.nbr + 2 * b), n1 = __ldg(g.nbr + 2 * b + 1);
        nb[0] = n0.x; nb[1] = n0.y; nb[2] = n0.z; nb[3] = n0.w;
        nb[4] = n1.x; nb[5] = n1.y; nb[6] = n1.z; nb[7] = n1.w;
    } else {
#pragma unroll
        for (int m = 0; m < 8; ++m) nb[m] = b;
    }
    bool ok = true;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int ex = e & 1, ey = (e >> 1) & 1, ez = e >> 2;
        const int be = nb[e & ovf];
        ok = ok && be >= 0;
        addr[e] = be * 512 + (((lz + ez) & 7) << 6) + (((ly + ey) & 7) << 3) + ((lx + ex) & 7);
    }
    return ok;
}

template <bool BF16>
__device__ __forceinline__ void load_corners(const GridDev& g, const int addr[8], float s[8], float r[8], float gg[8],
                                             float b[8]) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        if constexpr (!BF16) {
            float4 v = __ldg(g.geo + addr[e]);
            s[e] = v.x; r[e] = v.y; gg[e] = v.z; b[e] = v.w;
        } else {
            s[e] = __ldg(g.sdf + addr[e]);
            uint2 c = __ldg(g.rgbh + addr[e]);
            r[e] = sdg_bf16_lo(c.x); gg[e] = sdg_bf16_hi(c.x); b[e] = sdg_bf16_lo(c.y);
        }
    }
}

__device__ __forceinline__ void trilinear_weights(float fx, float fy, float fz, float w[8]) {
    const float gx = 1.f - fx, gy = 1.f - fy, gz = 1.f - fz;
    w[0] = gx * gy * gz; w[1] = fx * gy * gz; w[2] = gx * fy * gz; w[3] = fx * fy * gz;
    w[4] = gx * gy * fz; w[5] = fx * gy * fz; w[6] = gx * fy * fz; w[7] = fx * fy * fz;
}

// sum over 4 semantic channels c0..c0+3 of one corner, weighted
__device__ __forceinline__ void sem_load4(const GridDev& g, int addr, int c0, float v[4]) {
    uint2 u = __ldg(reinterpret_cast<const uint2*>(g.sem + (int64_t)addr * g.n_sem + c0));
    v[0] = sdg_bf16_lo(u.x); v[1] = sdg_bf16_hi(u.x); v[2] = sdg_bf16_lo(u.y); v[3] = sdg_bf16_hi(u.y);
}

__device__ __forceinline__ void red_add_v4(float4* p, float a, float b, float c, float d) {
    atomicAdd(p, make_float4(a, b, c, d));
}

// ---------------------------------------------------------------------------
// Warp collectives
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ float warp_incl_scan(float v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        float n = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += n;
    }
    return v;
}
// sum of v over lanes > lane
__device__ __forceinline__ float warp_excl_suffix(float v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        float n = __shfl_down_sync(kFull, v, o);
        if (lane + o < 32) v += n;
    }
    float r = __shfl_down_sync(kFull, v, 1);
    return lane == 31 ? 0.f : r;
}

__device__ __forceinline__ float sgnf(float x) { return (float)((x > 0.f) - (x < 0.f)); }

// ---------------------------------------------------------------------------
// The per-ray program
// ---------------------------------------------------------------------------
template <int MODE, bool BF16, bool SEM, int Q>
__device__ __forceinline__ void ray_program(const GridDev& g, const PassArgs& a, const RayJob& j, float* ts,
                                            float* ss, int lane) {
    constexpr bool kStoreIn = MODE == PASS_BWD_STORE;
    constexpr bool kStoreOut = MODE == PASS_FWD_STORE;
    constexpr bool kBwd = MODE == PASS_BWD || MODE == PASS_BWD_STORE || MODE == PASS_TRAIN;
    constexpr bool kFwdOut = MODE == PASS_FWD || MODE == PASS_FWD_STORE;
    constexpr int SEMCAP = SEM ? 32 : 0;
    const int N = a.N;
    const int ns = SEM ? g.n_sem : 0;
    const int64_t RS = 32 * Q;  // record stride per ray

    SampleGen gen;
    gen.seed_h = pcg_hash(a.seed);
    gen.ray_id = j.ray_id;
    gen.strat = a.strat;
    float S;
    if constexpr (kStoreIn) {
        S = a.rec_S[j.idx];
        gen.s_over_n = S / (float)N;
        gen.s_max = __int_as_float(__float_as_int(S) - 1);
    } else {
        S = place_samples(g, a, j, ts, ss, lane, gen);
    }
    if constexpr (kStoreOut) {
        if (lane == 0) a.rec_S[j.idx] = S;
    }
    const bool any = S > 0.f;

    // ---------------- phase A: evaluate this lane's samples ----------------
    float t_[Q], dl_[Q], d_[Q], cr_[Q], cg_[Q], cb_[Q], tau_[Q], dsig_[Q], fx_[Q], fy_[Q], fz_[Q];
    int cx_[Q], cy_[Q], cz_[Q];
    unsigned vmask = 0;
    BlockCache bc{SDG_EMPTY_KEY, -1};
    {
        int ccx = INT32_MIN, ccy = 0, ccz = 0;  // cell whose corners are loaded
        bool cvalid = false;
        int addr[8];
        float cs[8], crr[8], cgg[8], cbb[8];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int k = lane * Q + i;
            t_[i] = 0.f; dl_[i] = 0.f; d_[i] = 0.f; cr_[i] = cg_[i] = cb_[i] = 0.f; tau_[i] = 0.f; dsig_[i] = 0.f;
            fx_[i] = fy_[i] = fz_[i] = 0.f; cx_[i] = cy_[i] = cz_[i] = 0;
            if (!any || k >= N) continue;
            float sk, sn;
            bool stored_valid = true;
            if constexpr (kStoreIn) {
                const float* rec = a.rec + j.idx * RS + i * 32 + lane;
                const int64_t CS = a.n * RS;
                t_[i] = rec[0];
                d_[i] = rec[CS];
                cr_[i] = rec[2 * CS];
                cg_[i] = rec[3 * CS];
                cb_[i] = rec[4 * CS];
                stored_valid = !isnan(d_[i]);
                sk = gen.s(k);
                sn = k + 1 < N ? gen.s(k + 1) : S;
            } else {
                t_[i] = ts[k];
                sk = ss[k];
                sn = ss[k + 1];
            }
            dl_[i] = sn - sk;
            const float px = fmaf(t_[i], j.d.x, j.o.x) * g.inv_vs;
            const float py = fmaf(t_[i], j.d.y, j.o.y) * g.inv_vs;
            const float pz = fmaf(t_[i], j.d.z, j.o.z) * g.inv_vs;
            const float flx = floorf(px), fly = floorf(py), flz = floorf(pz);
            cx_[i] = (int)flx; cy_[i] = (int)fly; cz_[i] = (int)flz;
            fx_[i] = px - flx; fy_[i] = py - fly; fz_[i] = pz - flz;
            bool valid;
            if constexpr (kStoreIn) {
                valid = stored_valid;
            } else {
                if (cx_[i] != ccx || cy_[i] != ccy || cz_[i] != ccz) {
                    ccx = cx_[i]; ccy = cy_[i]; ccz = cz_[i];
                    cvalid = cell_addresses(g, ccx, ccy, ccz, bc, addr);
                    if (cvalid) load_corners<BF16>(g, addr, cs, crr, cgg, cbb);
                }
                valid = cvalid;
                if (valid) {
                    float w[8];
                    trilinear_weights(fx_[i], fy_[i], fz_[i], w);
                    float dd = 0.f, r = 0.f, gg = 0.f, bb = 0.f;
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        dd = fmaf(w[e], cs[e], dd);
                        r = fmaf(w[e], crr[e], r);
                        gg = fmaf(w[e], cgg[e], gg);
                        bb = fmaf(w[e], cbb[e], bb);
                    }
                    d_[i] = dd; cr_[i] = r; cg_[i] = gg; cb_[i] = bb;
                }
            }
            if (valid) {
                vmask |= 1u << i;
                // sigma = Psi_beta(-d) / beta, the Laplace CDF transform (Sec. 3.5.1)
                const float e = __expf(-fabsf(d_[i]) * g.inv_beta);
                const float sig = d_[i] >= 0.f ? 0.5f * g.inv_beta * e : g.inv_beta * (1.f - 0.5f * e);
                tau_[i] = sig * dl_[i];
                dsig_[i] = -0.5f * g.inv_beta * g.inv_beta * e * dl_[i];  // delta * dsigma/dd
            }
            if constexpr (kStoreOut) {
                float* rec = a.rec + j.idx * RS + i * 32 + lane;
                const int64_t CS = a.n * RS;
                rec[0] = t_[i];
                rec[CS] = valid ? d_[i] : __int_as_float(0x7fc00000);
                rec[2 * CS] = cr_[i];
                rec[3 * CS] = cg_[i];
                rec[4 * CS] = cb_[i];
            }
        }
    }

    // ---------------- phase B: transmittance and weights (Eq. 15) ----------------
    float lane_tau = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) lane_tau += tau_[i];
    const float incl = warp_incl_scan(lane_tau, lane);
    const float excl = incl - lane_tau;
    const float total = __shfl_sync(kFull, incl, 31);
    const float TN = __expf(-total);
    float w_[Q], Tn_[Q];
    {
        float T = __expf(-excl);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const float ea = -expm1f(-tau_[i]);  // 1 - exp(-tau), accurate for small tau
            w_[i] = T * ea;
            T = T - w_[i];
            Tn_[i] = T;  // T_{k+1}
        }
    }

    // semantic logits: per run of same-cell samples, corner weights W_e = sum_i w_i r_e(f_i)
    float sem_acc[SEMCAP > 0 ? SEMCAP : 1];
    if constexpr (SEM) {
#pragma unroll
        for (int c = 0; c < SEMCAP; ++c) sem_acc[c] = 0.f;
    }
    // run iteration helper: same cell and valid
    auto same_cell = [&](int i0, int i1) { return cx_[i0] == cx_[i1] && cy_[i0] == cy_[i1] && cz_[i0] == cz_[i1]; };

    if constexpr (SEM && (kFwdOut || MODE == PASS_TRAIN)) {
        if (any) {
            float W[8];
            int addr[8];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const bool v = (vmask >> i) & 1u;
                const bool start = v && (i == 0 || !((vmask >> (i - 1)) & 1u) || !same_cell(i - 1, i));
                const bool end = v && (i == Q - 1 || !((vmask >> (i + 1)) & 1u) || !same_cell(i, i + 1));
                if (start) {
#pragma unroll
                    for (int e = 0; e < 8; ++e) W[e] = 0.f;
                    cell_addresses(g, cx_[i], cy_[i], cz_[i], bc, addr);
                }
                if (v) {
                    float r[8];
                    trilinear_weights(fx_[i], fy_[i], fz_[i], r);
#pragma unroll
                    for (int e = 0; e < 8; ++e) W[e] = fmaf(w_[i], r[e], W[e]);
                }
                if (end) {
#pragma unroll
                    for (int c4 = 0; c4 < SEMCAP / 4; ++c4) {
                        if (4 * c4 < ns) {
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                float sv[4];
                                sem_load4(g, addr[e], 4 * c4, sv);
#pragma unroll
                                for (int q = 0; q < 4; ++q) sem_acc[4 * c4 + q] = fmaf(W[e], sv[q], sem_acc[4 * c4 + q]);
                            }
                        }
                    }
                }
            }
        }
    }

    // ---------------- forward outputs (Eq. 12-13 integrands) ----------------
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f, O = 0.f;
    if constexpr (MODE != PASS_BWD && MODE != PASS_BWD_STORE) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            C0 = fmaf(w_[i], cr_[i], C0);
            C1 = fmaf(w_[i], cg_[i], C1);
            C2 = fmaf(w_[i], cb_[i], C2);
            D = fmaf(w_[i], t_[i], D);
            O += w_[i];
        }
        C0 = warp_sum(C0) + TN * a.bg[0];
        C1 = warp_sum(C1) + TN * a.bg[1];
        C2 = warp_sum(C2) + TN * a.bg[2];
        D = warp_sum(D);
        O = warp_sum(O);
        if constexpr (SEM) {
#pragma unroll
            for (int c = 0; c < SEMCAP; ++c)
                if (c < ns) sem_acc[c] = warp_sum(sem_acc[c]);
        }
    }
    if constexpr (kFwdOut) {
        if (lane == 0) {
            a.out_rgb[3 * j.idx] = C0;
            a.out_rgb[3 * j.idx + 1] = C1;
            a.out_rgb[3 * j.idx + 2] = C2;
            a.out_depth[j.idx] = D;
            a.out_opac[j.idx] = O;
        }
        if constexpr (SEM) {
            if (a.out_sem) {
#pragma unroll
                for (int c = 0; c < SEMCAP; ++c)
                    if (c < ns && c == lane) a.out_sem[j.idx * ns + c] = sem_acc[c];
            }
        }
    }
    if constexpr (!kBwd) return;

    // ---------------- gradient seeds ----------------
    float gC0, gC1, gC2, gD, gO;
    float gS[SEMCAP > 0 ? SEMCAP : 1];
    if constexpr (MODE == PASS_TRAIN) {
        // L1 colour + lambda_d L1 depth (+ lambda_s squared L2 logits), mean over rays
        const float e0 = C0 - a.t_rgb[3 * j.idx], e1 = C1 - a.t_rgb[3 * j.idx + 1], e2 = C2 - a.t_rgb[3 * j.idx + 2];
        const float ed = D - a.t_depth[j.idx];
        const float third = a.inv_n * (1.0f / 3.0f);
        gC0 = sgnf(e0) * third; gC1 = sgnf(e1) * third; gC2 = sgnf(e2) * third;
        gD = a.lam_d * sgnf(ed) * a.inv_n;
        gO = 0.f;
        float L = (fabsf(e0) + fabsf(e1) + fabsf(e2)) * third + a.lam_d * fabsf(ed) * a.inv_n;
        if constexpr (SEM) {
#pragma unroll
            for (int c = 0; c < SEMCAP; ++c) {
                gS[c] = 0.f;
                if (c < ns && a.t_sem) {
                    const float es = sem_acc[c] - a.t_sem[j.idx * ns + c];
                    gS[c] = 2.f * a.lam_s * es * a.inv_n;
                    L += a.lam_s * es * es * a.inv_n;
                }
            }
        }
        if (lane == 0 && a.loss) a.loss[j.idx] = L;
    } else {
        gC0 = a.g_rgb[3 * j.idx]; gC1 = a.g_rgb[3 * j.idx + 1]; gC2 = a.g_rgb[3 * j.idx + 2];
        gD = a.g_depth ? a.g_depth[j.idx] : 0.f;
        gO = a.g_opac ? a.g_opac[j.idx] : 0.f;
        if constexpr (SEM) {
#pragma unroll
            for (int c = 0; c < SEMCAP; ++c) gS[c] = (c < ns && a.g_sem) ? a.g_sem[j.idx * ns + c] : 0.f;
        }
    }
    if (!any) return;

    // v_k = g_rgb . c_k + g_depth t_k + g_opac + g_sem . s_k
    float v_[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) v_[i] = fmaf(gC0, cr_[i], fmaf(gC1, cg_[i], fmaf(gC2, cb_[i], fmaf(gD, t_[i], gO))));
    bool sem_grad = false;
    if constexpr (SEM) {
        bool need = false;
#pragma unroll
        for (int c = 0; c < SEMCAP; ++c) need |= gS[c] != 0.f;
        sem_grad = __any_sync(kFull, need);
        if (sem_grad) {
            // per run: dot_e = g_sem . theta_s(corner e), then v_i += sum_e r_e(f_i) dot_e
            int addr[8];
            float dot[8];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const bool v = (vmask >> i) & 1u;
                const bool start = v && (i == 0 || !((vmask >> (i - 1)) & 1u) || !same_cell(i - 1, i));
                if (start) {
                    cell_addresses(g, cx_[i], cy_[i], cz_[i], bc, addr);
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        dot[e] = 0.f;
#pragma unroll
                        for (int c4 = 0; c4 < SEMCAP / 4; ++c4)
                            if (4 * c4 < ns) {
                                float sv[4];
                                sem_load4(g, addr[e], 4 * c4, sv);
#pragma unroll
                                for (int q = 0; q < 4; ++q) dot[e] = fmaf(gS[4 * c4 + q], sv[q], dot[e]);
                            }
                    }
                }
                if (v) {
                    float r[8];
                    trilinear_weights(fx_[i], fy_[i], fz_[i], r);
                    float acc = 0.f;
#pragma unroll
                    for (int e = 0; e < 8; ++e) acc = fmaf(r[e], dot[e], acc);
                    v_[i] += acc;
                }
            }
        }
    }

    // ---------------- reverse scan: R_k = sum_{j>k} w_j v_j ----------------
    float lane_wv = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) lane_wv = fmaf(w_[i], v_[i], lane_wv);
    float R = warp_excl_suffix(lane_wv, lane);
    const float ubg = TN * (gC0 * a.bg[0] + gC1 * a.bg[1] + gC2 * a.bg[2]);
    float dd_[Q];
#pragma unroll
    for (int i = Q - 1; i >= 0; --i) {
        const float dtau = Tn_[i] * v_[i] - R - ubg;
        R = fmaf(w_[i], v_[i], R);
        dd_[i] = ((vmask >> i) & 1u) ? dsig_[i] * dtau : 0.f;
    }

    // ---------------- scatter to voxels (runs of same-cell samples) ----------------
    {
        int addr[8];
        float aS[8], aR[8], aG[8], aB[8], aW[8];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const bool v = (vmask >> i) & 1u;
            const bool start = v && (i == 0 || !((vmask >> (i - 1)) & 1u) || !same_cell(i - 1, i));
            const bool end = v && (i == Q - 1 || !((vmask >> (i + 1)) & 1u) || !same_cell(i, i + 1));
            if (start) {
#pragma unroll
                for (int e = 0; e < 8; ++e) aS[e] = aR[e] = aG[e] = aB[e] = aW[e] = 0.f;
                cell_addresses(g, cx_[i], cy_[i], cz_[i], bc, addr);
            }
            if (v) {
                float r[8];
                trilinear_weights(fx_[i], fy_[i], fz_[i], r);
                const float wr = w_[i] * gC0, wg = w_[i] * gC1, wb = w_[i] * gC2;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    aS[e] = fmaf(r[e], dd_[i], aS[e]);
                    aR[e] = fmaf(r[e], wr, aR[e]);
                    aG[e] = fmaf(r[e], wg, aG[e]);
                    aB[e] = fmaf(r[e], wb, aB[e]);
                    if constexpr (SEM) aW[e] = fmaf(r[e], w_[i], aW[e]);
                }
            }
            if (end) {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    if constexpr (!BF16) {
                        red_add_v4(g.ggeo + addr[e], aS[e], aR[e], aG[e], aB[e]);
                    } else {
                        atomicAdd(g.gsdf + addr[e], aS[e]);
                        red_add_v4(g.grgb + addr[e], aR[e], aG[e], aB[e], 0.f);
                    }
                    if (SEM && sem_grad) {
#pragma unroll
                        for (int c4 = 0; c4 < SEMCAP / 4; ++c4)
                            if (4 * c4 < ns)
                                red_add_v4(reinterpret_cast<float4*>(g.gsem + (int64_t)addr[e] * ns) + c4,
                                           aW[e] * gS[4 * c4], aW[e] * gS[4 * c4 + 1], aW[e] * gS[4 * c4 + 2],
                                           aW[e] * gS[4 * c4 + 3]);
                    }
                }
            }
        }
    }
}

}  // namespace sdg
