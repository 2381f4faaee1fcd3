// Per-ray warp program of the renderer: empty-space-skipping traversal,
// stratified sampling in allocated space, trilinear fetch, Laplace density,
// compositing and its backward.  Paper: arXiv 2305.13220, Sec. 3.5.1
// (Eq. 12-15) and Sec. 3.5.2 (Eq. 17, trilinear interpolation).
//
// Work decomposition (one warp = one ray), chosen so that control flow stays
// uniform across the warp:
//  * traversal: a pass of its own (k_walk, one thread per ray) walks the ray
//    through the dense block-index grid (block-level Amanatides-Woo) and
//    writes the allocated cells it crosses -- t range, block index, grid cell
//    -- with their exact sequential skip-space offsets; lane m of the render
//    warp loads record m.  A ray crossing more than kWalkCap allocated cells,
//    and every ray of the passes that run without the traversal pass (the
//    serving loop, the allocation-free pass), is walked in-warp instead: the
//    clipped range is cut into 32 equal pieces, lane j walks piece j and
//    records its cells in shared memory (up to kSegs; a piece with more is
//    re-walked when one of its samples is placed), and a sequential shuffle
//    prefix of the pieces' allocated lengths gives the offsets P_j.
//  * sampling: lane l owns samples l*Q .. l*Q+Q-1.  It draws s_k itself and
//    finds its cell in the ray's walk records (lane m holds record m) by a
//    binary search over their skip-space offsets for its first sample and a
//    forward scan for the others (or, walking in-warp, by a binary search over
//    P and the piece's list), so every lane runs the same instructions.
//  * fetch: a lane first places all its samples, then evaluates them in
//    order; a sample in a new cell loads its 8 corner voxels (one 16-byte
//    load each in the FP32 layout), a sample in the cell of the lane's
//    previous sample reuses the values already in registers (about half of
//    the samples at 128 per ray), which halves the corner gathers.
//  * compositing: transmittance is a warp scan of the lanes' optical depths;
//    the backward keeps per-sample state in registers, takes the suffix sum
//    as a reverse warp scan, and sums each run of same-cell samples of a lane
//    in registers before one vector atomic per corner.
#pragma once

#include "common.cuh"

namespace sdg {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kWarpsPerBlock = 8;
constexpr int kSegs = 8;  // allocated cells recorded per lane piece

// PASS_TRAIN_BETA is PASS_TRAIN that also returns dL/dbeta per ray (the Laplace scale as a parameter).
enum PassMode {
    PASS_FWD = 0,
    PASS_FWD_STORE = 1,
    PASS_BWD = 2,
    PASS_BWD_STORE = 3,
    PASS_TRAIN = 4,
    PASS_TRAIN_BETA = 5,
    PASS_TRAIN_NRM = 6,  // PASS_TRAIN plus the normal loss of Eq. 14 on the rendered normal sum_k w_k grad f(x_k)
    PASS_FWD_TRACE = 7   // PASS_FWD that also writes where every sample was placed (debug export)
};

// Allocated block cells of a ray kept in the walk records: up to kWalkCap a ray is rendered by the records kernel
// (lane m holds record m), up to kWalkSlot by the kernel over the mid list (lane m holds records m and m + 32), a
// ray crossing more takes the in-warp traversal.
constexpr int kWalkCap = 32;
constexpr int kWalkSlot = 2 * kWalkCap;

// Output of k_walk, indexed by processing slot: hdr[slot] = {number of records (-1: more than kWalkSlot),
// bits of S}; record m of the slot at [slot * kWalkSlot + m]: s0 = skip-space offset of the cell (sequential FP32
// sum of the lengths before it, so the offsets are monotone and S = s0 + len of the last), and
// rec = {bits of t_in, bits of len, block index, dense-grid cell}.
// Slots of rays with kWalkCap + 1 .. kWalkSlot records are appended to mid[0, *n_mid), those of rays crossing
// more than kWalkSlot allocated cells to over[0, *n_over) (each in no particular order): the records kernel skips
// both, the mid-list kernel and the in-warp kernels render them.
struct WalkBufs {
    int2* hdr;
    float* s0;
    int4* rec;
    int* over;
    int* n_over;
    int* mid;
    int* n_mid;
};

// Store-mode record channels per sample: t, sdf (NaN if invalid), r, g, b, block index (int bits).
constexpr int kRecChannels = 6;

struct PassArgs {
    int N;  // samples per ray
    uint32_t seed;
    int strat;
    float bg[3];
    int64_t n;  // rays in this launch
    int64_t over_hint, mid_hint;  // host side: expected lengths of the overflow and mid lists (launch sizing only)
    int* over_out;  // nullable, pinned host memory [2]: k_render_rest stores the two lists' lengths there
    float *out_rgb, *out_depth, *out_opac, *out_sem;
    float* rec;    // store mode: [kRecChannels][n][32*Q]
    float* rec_S;  // store mode: [n]
    const float *g_rgb, *g_depth, *g_opac, *g_sem;
    const float *t_rgb, *t_depth, *t_sem;
    float lam_d, lam_s, inv_n;
    float* loss;
    const int* perm;  // optional processing order: warp slot i runs ray perm[i] (NULL: ray i)
    float* beta_part;  // PASS_TRAIN_BETA: dL/dbeta of each ray [n]
    const float* t_normal;  // PASS_TRAIN_NRM: target normals [n][3] (world frame)
    float lam_n;
    WalkBufs walk;  // records of the traversal pass (hdr NULL: every warp walks its ray itself)
    // PASS_FWD_TRACE outputs, per ray [n] or per sample [n][N]: walk records used (-1: the warp walked the ray),
    // S, t_k, the voxel coordinates of the sample's cell base corner [n][N][3], its own block index, validity;
    // tr_seg [n][kWalkCap][2] (nullable): t_in and length of each walk record
    int* tr_ncell;
    float* tr_S;
    float* tr_t;
    int* tr_cell;
    int* tr_blk;
    unsigned char* tr_valid;
    float* tr_seg;
};

struct RayJob {
    float3 o, d;
    float tn, tf;
    uint32_t ray_id;
    int64_t idx;   // row of this ray in per-ray arrays
    int64_t slot;  // processing slot (row of the walk records)
};

// Per-warp shared memory: the allocated cells of each lane piece (m-major so a
// lane's writes of one slot are bank-conflict free) and the piece prefixes.
struct WarpSmem {
    float tin[kSegs][32];
    float len[kSegs][32];
    int blk[kSegs][32];
    int cell[kSegs][32];  // dense block-index grid cell of the record's block
    float P[33];
    int cnt[32];
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
// ray_h = pcg_hash(ray_id + pcg_hash(seed)) is per ray; u_k = pcg_hash(k + ray_h) >> 8, times 2^-24.
__device__ __forceinline__ float sample_u(uint32_t ray_h, int k) {
    return (float)(pcg_hash((uint32_t)k + ray_h) >> 8) * 5.9604644775390625e-8f;
}

struct SampleGen {
    float s_over_n, s_max;
    uint32_t ray_h;
    int strat;
    __device__ __forceinline__ float s(int k) const {
        float u = strat ? sample_u(ray_h, k) : 0.5f;
        return fminf(((float)k + u) * s_over_n, s_max);
    }
};

// Pinhole intrinsics {fx, fy, cx, cy} and row-major 3x4 camera-to-world pose, passed to kernels by value.
struct Cam6 {
    float K[4];
    float T[12];
};

// Pinhole camera ray of pixel (u, v) (centre at +0.5): d = normalize(R ((u + 0.5 - cx)/fx, (v + 0.5 - cy)/fy, 1)),
// o = t, with K = {fx, fy, cx, cy} and T the row-major 3x4 camera-to-world pose.  Every product is an explicit
// fused multiply-add, so the serving kernel and the trace export form the same rays.
__device__ __forceinline__ void pinhole_ray(const float K[4], const float T[12], int u, int v, float3& o, float3& d) {
    const float xc = ((float)u + 0.5f - K[2]) / K[0];
    const float yc = ((float)v + 0.5f - K[3]) / K[1];
    const float dx = fmaf(T[0], xc, fmaf(T[1], yc, T[2]));
    const float dy = fmaf(T[4], xc, fmaf(T[5], yc, T[6]));
    const float dz = fmaf(T[8], xc, fmaf(T[9], yc, T[10]));
    const float inv = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    o = make_float3(T[3], T[7], T[11]);
    d = make_float3(dx * inv, dy * inv, dz * inv);
}

// ---------------------------------------------------------------------------
// Traversal
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool clip_to_grid(const GridDev& g, const float3& o, const float3& d, float& t0,
                                             float& t1) {
    if (g.n_blocks == 0) return false;
    const float oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        // products rounded on their own (no contraction into the subtraction below), so that every kernel that
        // walks a ray gets the same bits
        const float lo = __fmul_rn((float)g.bmin[a], g.L), hi = __fmul_rn((float)(g.bmin[a] + g.bdim[a]), g.L);
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


// Cell of the dense block-index grid holding block (bx, by, bz), -1 if it lies outside the AABB.
__device__ __forceinline__ int dense_cell(const GridDev& g, int bx, int by, int bz) {
    const unsigned x = (unsigned)(bx - g.bmin[0]), y = (unsigned)(by - g.bmin[1]), z = (unsigned)(bz - g.bmin[2]);
    if (x >= (unsigned)g.bdim[0] || y >= (unsigned)g.bdim[1] || z >= (unsigned)g.bdim[2]) return -1;
    return (int)((z * (unsigned)g.bdim[1] + y) * (unsigned)g.bdim[0] + x);  // < 2^31 cells
}

// Index of the block at block coordinates (bx, by, bz), -1 if it is not allocated (or outside the AABB).
__device__ __forceinline__ int block_at(const GridDev& g, int bx, int by, int bz) {
    const int c = dense_cell(g, bx, by, bz);
    return c < 0 || !sdg_in_range(g.status, c, g.dense_cells, SDG_CHECK_DENSE) ? -1 : __ldg(g.dense + c);
}

// Calls f(a, b, cell, blk) for every allocated block cell the ray crosses inside [ta, tb), in order of
// increasing t, with [a, b) its stretch of the ray and cell its index in the dense block-index grid; the walk
// stops early when f returns false.  Block-level Amanatides-Woo: the exit time of a cell is the smallest of its
// three face-plane times, each formed as one fused multiply-add and a product (the same bits in every kernel).
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
    // index steps of the dense grid (x fastest)
    const int stx = sx, sty = sy * g.bdim[0], stz = sz * (int)((unsigned)g.bdim[0] * (unsigned)g.bdim[1]);
    float tcur = ta;
    const int maxit = g.bdim[0] + g.bdim[1] + g.bdim[2] + 3;
    int cidx = (cz * g.bdim[1] + cy) * g.bdim[0] + cx;
    // the next cell's block index is loaded before the current cell is handed to f, so the loads of successive
    // cells overlap instead of each waiting for the previous one
    int blk = sdg_in_range(g.status, cidx, g.dense_cells, SDG_CHECK_DENSE) ? __ldg(g.dense + cidx) : -1;
    for (int it = 0; it < maxit; ++it) {
        const float tx = sx ? fmaf((float)(g.bmin[0] + cx + (sx > 0)), g.L, -o.x) * invd.x : INF;
        const float ty = sy ? fmaf((float)(g.bmin[1] + cy + (sy > 0)), g.L, -o.y) * invd.y : INF;
        const float tz = sz ? fmaf((float)(g.bmin[2] + cz + (sz > 0)), g.L, -o.z) * invd.z : INF;
        const float te = fminf(tx, fminf(ty, tz));
        const float b = fminf(te, tb);
        const bool mx = tx == te, my = ty == te, mz = tz == te;
        const int nx = cx + (mx ? sx : 0), ny = cy + (my ? sy : 0), nz = cz + (mz ? sz : 0);
        const bool more = te < tb && (unsigned)nx < (unsigned)g.bdim[0] && (unsigned)ny < (unsigned)g.bdim[1] &&
                          (unsigned)nz < (unsigned)g.bdim[2];
        const int nidx = cidx + (mx ? stx : 0) + (my ? sty : 0) + (mz ? stz : 0);
        const int nblk =
            more && sdg_in_range(g.status, nidx, g.dense_cells, SDG_CHECK_DENSE) ? __ldg(g.dense + nidx) : -1;
        if (b > tcur && blk >= 0)
            if (!f(tcur, b, cidx, blk)) break;
        if (!more) break;
        cx = nx;
        cy = ny;
        cz = nz;
        cidx = nidx;
        blk = nblk;
        tcur = fmaxf(te, ta);
    }
}

// The same walk for a thread that walks a whole ray alone (the traversal pass): D cells' block-index loads are
// kept in flight, so the walk advances about one cell per D load latencies instead of one per latency.  The
// cells, their stretches and the order in which f sees them are exactly those of walk_cells.
template <int D, class F>
__device__ __forceinline__ void walk_cells_pipelined(const GridDev& g, const float3& o, const float3& d,
                                                     const float3& invd, float ta, float tb, F&& f) {
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
    const int stx = sx, sty = sy * g.bdim[0], stz = sz * (int)((unsigned)g.bdim[0] * (unsigned)g.bdim[1]);
    float tcur = ta;
    int cidx = (cz * g.bdim[1] + cy) * g.bdim[0] + cx;
    int left = g.bdim[0] + g.bdim[1] + g.bdim[2] + 3;  // bounds the walk, as walk_cells' iteration limit
    bool alive = true;
    // ring of D cells between their load and their use: stretch [a, b), dense-grid cell (-1: empty slot), block
    float ra[D], rb[D];
    int rc[D], rblk[D];
    auto produce = [&](int k) {
        ra[k] = 0.f;
        rb[k] = 0.f;
        rc[k] = -1;
        rblk[k] = -1;
        if (!alive) return;
        const float tx = sx ? fmaf((float)(g.bmin[0] + cx + (sx > 0)), g.L, -o.x) * invd.x : INF;
        const float ty = sy ? fmaf((float)(g.bmin[1] + cy + (sy > 0)), g.L, -o.y) * invd.y : INF;
        const float tz = sz ? fmaf((float)(g.bmin[2] + cz + (sz > 0)), g.L, -o.z) * invd.z : INF;
        const float te = fminf(tx, fminf(ty, tz));
        ra[k] = tcur;
        rb[k] = fminf(te, tb);
        rc[k] = cidx;
        rblk[k] = sdg_in_range(g.status, cidx, g.dense_cells, SDG_CHECK_DENSE) ? __ldg(g.dense + cidx)
                                                                                 : -1;  // used D cells later
        const bool mx = tx == te, my = ty == te, mz = tz == te;
        const int nx = cx + (mx ? sx : 0), ny = cy + (my ? sy : 0), nz = cz + (mz ? sz : 0);
        alive = te < tb && (unsigned)nx < (unsigned)g.bdim[0] && (unsigned)ny < (unsigned)g.bdim[1] &&
                (unsigned)nz < (unsigned)g.bdim[2] && --left > 0;
        if (alive) {
            cidx += (mx ? stx : 0) + (my ? sty : 0) + (mz ? stz : 0);
            cx = nx;
            cy = ny;
            cz = nz;
            tcur = fmaxf(te, ta);
        }
    };
#pragma unroll
    for (int k = 0; k < D; ++k) produce(k);
    bool pending = true;
    while (pending) {
        pending = false;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            if (rc[k] >= 0 && rb[k] > ra[k] && rblk[k] >= 0)
                if (!f(ra[k], rb[k], rc[k], rblk[k])) return;
            produce(k);
            pending |= rc[k] >= 0;
        }
    }
}

// The traversal pass for one ray: clips (o, d) over [t0, t1] to the grid and walks it, writing the allocated cells
// it crosses as records of slot `slot` of w with their sequential skip-space offsets, and the slot's header
// {record count (-1: more than kWalkCap, the slot appended to the overflow list), bits of S}.
__device__ __forceinline__ void walk_ray_records(const GridDev& g, const float3& o, const float3& d, float t0,
                                                 float t1, const WalkBufs& w, int64_t slot) {
    int cnt = 0;
    float S = 0.f;
    if (clip_to_grid(g, o, d, t0, t1)) {
        const float3 invd = make_float3(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
        float* s0 = w.s0 + slot * kWalkSlot;
        int4* rec = w.rec + slot * kWalkSlot;
        walk_cells_pipelined<8>(g, o, d, invd, t0, t1, [&](float x0, float x1, int cell, int blk) {
            if (cnt == kWalkSlot) {
                cnt = -1;  // more cells than records: the render warp walks this ray itself
                return false;
            }
            const float len = x1 - x0;
            s0[cnt] = S;
            rec[cnt] = make_int4(__float_as_int(x0), __float_as_int(len), blk, cell);
            S += len;
            ++cnt;
            return true;
        });
    }
    w.hdr[slot] = make_int2(cnt, __float_as_int(S));
    if (cnt < 0) w.over[atomicAdd(w.n_over, 1)] = (int)slot;
    else if (cnt > kWalkCap) w.mid[atomicAdd(w.n_mid, 1)] = (int)slot;
}

struct Pieces {
    float t0, dt, S;
    float3 invd;
};

__device__ __forceinline__ float piece_start(const Pieces& pc, int j) { return fmaf((float)j, pc.dt, pc.t0); }
__device__ __forceinline__ float piece_end(const Pieces& pc, float t1, int j) {
    return j == 31 ? t1 : fmaf((float)(j + 1), pc.dt, pc.t0);
}

// One traversal walk per lane: records the lane piece's allocated cells and
// returns S, the ray's total allocated length (0 if it sees no block).
__device__ __forceinline__ float walk_pieces(const GridDev& g, const RayJob& j, WarpSmem& sm, int lane, Pieces& pc,
                                             float& t1_out) {
    float t0 = j.tn, t1 = j.tf;
    float S_j = 0.f;
    int cnt = 0;
    pc.invd = make_float3(1.0f / j.d.x, 1.0f / j.d.y, 1.0f / j.d.z);
    pc.t0 = 0.f;
    pc.dt = 0.f;
    const bool hit = clip_to_grid(g, j.o, j.d, t0, t1);
    if (hit) {
        pc.t0 = t0;
        pc.dt = (t1 - t0) * (1.0f / 32.0f);
        const float ta = piece_start(pc, lane), tb = piece_end(pc, t1, lane);
        walk_cells(g, j.o, j.d, pc.invd, ta, tb, [&](float x0, float x1, int cell, int blk) {
            if (cnt < kSegs) {
                sm.tin[cnt][lane] = x0;
                sm.len[cnt][lane] = x1 - x0;
                sm.blk[cnt][lane] = blk;
                sm.cell[cnt][lane] = cell;
            }
            ++cnt;
            S_j += x1 - x0;
            return true;
        });
    }
    t1_out = t1;
    // sequential prefix: P_{j+1} = fl(P_j + S_j) exactly, so the pieces tile [0, S) monotonically
    float P = 0.f;
#pragma unroll
    for (int i = 0; i < 31; ++i) {
        float v = __shfl_sync(kFull, S_j, i);
        if (i < lane) P += v;
    }
    const float S = __shfl_sync(kFull, P + S_j, 31);
    sm.P[lane] = P;
    sm.cnt[lane] = cnt;
    if (lane == 0) sm.P[32] = S;
    __syncwarp();
    pc.S = S;
    return S;
}

// t, block index and dense-grid cell of skip-space position s (0 <= s < S), from the lane pieces' records.
__device__ __forceinline__ float locate(const GridDev& g, const RayJob& j, const WarpSmem& sm, const Pieces& pc,
                                        float t1, float s, int& blk, int& cell) {
    int jp = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1)
        if (sm.P[jp + step] <= s) jp += step;
    float local = s - sm.P[jp];
    const int cnt = sm.cnt[jp];
    if (cnt <= kSegs) {
        int m = 0;
        for (; m < cnt - 1; ++m) {
            const float l = sm.len[m][jp];
            if (local < l) break;
            local -= l;
        }
        blk = sm.blk[m][jp];
        cell = sm.cell[m][jp];
        return sm.tin[m][jp] + fminf(local, sm.len[m][jp]);
    }
    // the piece had more allocated cells than were recorded: walk it again
    float ta = piece_start(pc, jp), tb = piece_end(pc, t1, jp);
    float best_a = ta, best_len = 0.f;
    int best_cell = -1, best_blk = -1;
    walk_cells(g, j.o, j.d, pc.invd, ta, tb, [&](float x0, float x1, int c, int kb) {
        best_a = x0;
        best_len = x1 - x0;
        best_cell = c;
        best_blk = kb;
        if (local < best_len) return false;
        local -= best_len;
        return true;
    });
    cell = best_cell;
    blk = best_blk;
    return best_a + fminf(local, best_len);
}

// ---------------------------------------------------------------------------
// Traversal as its own pass: one thread walks a whole ray
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Voxel stencil of a cell (Eq. 17): the 8 grid points around x
// ---------------------------------------------------------------------------
// Cell packed as lx | ly << 3 | lz << 6 (local coordinates of its base corner).  Its 8 corners are the
// voxels (lx + ex, ly + ey, lz + ez), e = ex | ey << 1 | ez << 2; a corner whose coordinate wraps past 7 on an
// axis lives in the neighbour block on that side, read from the block's neighbour row
// {self, +x, +y, +xy | +z, +xz, +yz, +xyz}.  Writes their voxel addresses; false if a corner's block is absent.
__device__ __forceinline__ bool corner_addresses(const GridDev& g, int blk, int lcell, int addr[8]) {
    const bool ox = (lcell & 7) == 7, oy = (lcell & 56) == 56, oz = lcell >= 448;
    if (!sdg_in_range(g.status, blk, g.n_blocks, SDG_CHECK_BLOCK)) return false;
    const int4 n0 = __ldg(g.nbr + 2 * blk), n1 = __ldg(g.nbr + 2 * blk + 1);
    const int b1 = ox ? n0.y : blk;
    const int b2 = oy ? n0.z : blk;
    const int b3 = ox ? (oy ? n0.w : n0.y) : b2;
    const int b4 = oz ? n1.x : blk;
    const int b5 = ox ? (oz ? n1.y : n0.y) : b4;
    const int b6 = oy ? (oz ? n1.z : n0.z) : b4;
    const int b7 = ox ? (oy ? (oz ? n1.w : n0.w) : (oz ? n1.y : n0.y)) : b6;
    // local index of the +1 corner on each axis: one step (+1, +8, +64), or, past the block's last voxel, the
    // first voxel of the neighbour block on that side (-7, -56, -448)
    const int dx = ox ? -7 : 1, dy = oy ? -56 : 8, dz = oz ? -448 : 64;
    const int l1 = lcell + dx, l2 = lcell + dy, l3 = l1 + dy;
    addr[0] = blk * 512 + lcell;
    addr[1] = b1 * 512 + l1;
    addr[2] = b2 * 512 + l2;
    addr[3] = b3 * 512 + l3;
    addr[4] = b4 * 512 + (lcell + dz);
    addr[5] = b5 * 512 + (l1 + dz);
    addr[6] = b6 * 512 + (l2 + dz);
    addr[7] = b7 * 512 + (l3 + dz);
    const bool all = (b1 | b2 | b3 | b4 | b5 | b6 | b7) >= 0;
#ifdef SDG_CHECKED
    if (all)  // every address the fetch and the scatter will use
        for (int e = 0; e < 8; ++e)
            if (!sdg_in_range(g.status, addr[e], g.n_blocks * 512, SDG_CHECK_VOXEL)) return false;
#endif
    return all;
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

// grad f = sum_e grad_x r_e theta_e (Eq. 17): the derivative of a trilinear weight along an axis swaps that axis's
// factor (f or 1 - f) for +-1/vs.
__device__ __forceinline__ void sdf_gradient(float fx, float fy, float fz, float inv_vs, const float th[8], float& gx,
                                             float& gy, float& gz) {
    const float gxm = 1.f - fx, gym = 1.f - fy, gzm = 1.f - fz;
    // differences along x at the four (y, z) corner pairs, and likewise for y and z
    const float dx00 = th[1] - th[0], dx10 = th[3] - th[2], dx01 = th[5] - th[4], dx11 = th[7] - th[6];
    const float dy00 = th[2] - th[0], dy10 = th[3] - th[1], dy01 = th[6] - th[4], dy11 = th[7] - th[5];
    const float dz00 = th[4] - th[0], dz10 = th[5] - th[1], dz01 = th[6] - th[2], dz11 = th[7] - th[3];
    gx = inv_vs * (gzm * (gym * dx00 + fy * dx10) + fz * (gym * dx01 + fy * dx11));
    gy = inv_vs * (gzm * (gxm * dy00 + fx * dy10) + fz * (gxm * dy01 + fx * dy11));
    gz = inv_vs * (gym * (gxm * dz00 + fx * dz10) + fy * (gxm * dz01 + fx * dz11));
}

// q . grad_x r_e for the 8 corners e (q already scaled by 1/vs): corner e = ex | ey << 1 | ez << 2.
__device__ __forceinline__ void dot_weight_gradients(float fx, float fy, float fz, float qx, float qy, float qz,
                                                     float out[8]) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const bool ex = e & 1, ey = (e >> 1) & 1, ez = (e >> 2) & 1;
        const float ax = ex ? fx : 1.f - fx, ay = ey ? fy : 1.f - fy, az = ez ? fz : 1.f - fz;
        out[e] = (ex ? qx : -qx) * ay * az + ax * (ey ? qy : -qy) * az + ax * ay * (ez ? qz : -qz);
    }
}

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

// a[i] for a register array and a run-time i (selects, no local memory)
template <int Q, class T>
__device__ __forceinline__ T pick(const T (&a)[Q], int i) {
    T r = a[0];
#pragma unroll
    for (int k = 1; k < Q; ++k) r = i == k ? a[k] : r;
    return r;
}

// ---------------------------------------------------------------------------
// The per-ray program
// ---------------------------------------------------------------------------
// INWARP: the warp walks its ray itself (walk_pieces); otherwise the ray's cells come from the traversal pass's
// records, RPL per lane: RPL = 1 renders rays with at most kWalkCap records (others are left to the mid-list and
// in-warp kernels), RPL = 2 those of the mid list.  NSC: semantic channels the program is unrolled for (0: no
// logits; else a multiple of 4 >= the grid's n_sem).
template <int MODE, bool BF16, int NSC, int Q, bool INWARP, int RPL = 1>
__device__ __forceinline__ void ray_program(const GridDev& g, const PassArgs& a, const RayJob& j, WarpSmem& sm,
                                            int lane) {
    static_assert(RPL == 1 || RPL == 2, "one or two records per lane");
    constexpr bool kStoreIn = MODE == PASS_BWD_STORE;
    constexpr bool kStoreOut = MODE == PASS_FWD_STORE;
    constexpr bool kTrain = MODE == PASS_TRAIN || MODE == PASS_TRAIN_BETA || MODE == PASS_TRAIN_NRM;
    constexpr bool kBeta = MODE == PASS_TRAIN_BETA;
    constexpr bool kNrm = MODE == PASS_TRAIN_NRM;
    constexpr bool kBwd = MODE == PASS_BWD || MODE == PASS_BWD_STORE || kTrain;
    constexpr bool kTrace = MODE == PASS_FWD_TRACE;
    constexpr bool kFwdOut = MODE == PASS_FWD || MODE == PASS_FWD_STORE || kTrace;
    constexpr bool SEM = NSC > 0;
    constexpr int SEMCAP = NSC;
    static_assert(NSC % 4 == 0 && NSC <= 32, "semantic channels: a multiple of 4, at most 32");
    const int N = a.N;
    const int ns = SEM ? g.n_sem : 0;
    const int64_t RS = 32 * Q;  // record stride per ray

    SampleGen gen;
    gen.ray_h = pcg_hash(j.ray_id + pcg_hash(a.seed));
    gen.strat = a.strat;
    Pieces pc;
    float t1 = 0.f;
    float S;
    // walk records of this ray (lane m holds record m, and m + 32 when RPL = 2), when the traversal ran as its own
    // pass
    bool by_rec = false;
    int n_rec = 0;
    float my_s0 = 0.f, my_s0b = 0.f;
    int4 my_rec = make_int4(0, 0, -1, -1), my_recb = make_int4(0, 0, -1, -1);
    if constexpr (kStoreIn) {
        S = a.rec_S[j.idx];
    } else {
        if constexpr (!INWARP) {
            const int2 h = __ldg(a.walk.hdr + j.slot);
            if (h.x < 0 || (RPL == 1 && h.x > kWalkCap)) return;  // warp-uniform: the mid-list or in-warp kernels
            by_rec = true;
            n_rec = h.x;
            S = __int_as_float(h.y);
            if (lane < n_rec) {
                my_s0 = __ldg(a.walk.s0 + j.slot * kWalkSlot + lane);
                my_rec = __ldg(a.walk.rec + j.slot * kWalkSlot + lane);
            }
            if constexpr (RPL == 2) {
                if (lane + kWalkCap < n_rec) {
                    my_s0b = __ldg(a.walk.s0 + j.slot * kWalkSlot + kWalkCap + lane);
                    my_recb = __ldg(a.walk.rec + j.slot * kWalkSlot + kWalkCap + lane);
                }
            }
        } else {
            S = walk_pieces(g, j, sm, lane, pc, t1);
        }
        if constexpr (kTrace) {
            // the export keeps SDG_TRACE_CELLS = kWalkCap records: -1 for a ray with more
            if (lane == 0) {
                a.tr_S[j.idx] = S;
                a.tr_ncell[j.idx] = by_rec && n_rec <= kWalkCap ? n_rec : -1;
            }
            if (a.tr_seg && by_rec && n_rec <= kWalkCap && lane < n_rec) {
                a.tr_seg[(j.idx * kWalkCap + lane) * 2] = __int_as_float(my_rec.x);
                a.tr_seg[(j.idx * kWalkCap + lane) * 2 + 1] = __int_as_float(my_rec.y);
            }
        }
    }
    if constexpr (kStoreOut) {
        if (lane == 0) a.rec_S[j.idx] = S;
    }
    const bool any = S > 0.f;
    gen.s_over_n = S / (float)N;
    gen.s_max = __int_as_float(__float_as_int(S) - 1);  // largest float below S (S > 0)

    // ---------------- phase A: place, then evaluate this lane's samples ----------------
    float s_[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int k = lane * Q + i;
        s_[i] = (any && k < N) ? gen.s(k) : 0.f;
    }
    const float s_after = __shfl_down_sync(kFull, s_[0], 1);  // first sample of the next lane

    float t_[Q] = {}, dl_[Q], d_[Q], cr_[Q], cg_[Q], cb_[Q], tau_[Q], dsig_[Q];
    int ba_[Q];  // base voxel of the sample's cell: block * 512 + local cell index (-1: no block)
    float bq_[kBeta ? Q : 1];
    float gnx_[kNrm ? Q : 1], gny_[kNrm ? Q : 1], gnz_[kNrm ? Q : 1];  // grad f at the samples (Eq. 17)
    unsigned vmask = 0;
    // fractional position of sample i in its cell, recomputed from t_[i] wherever it is needed (the same
    // operations give the same bits), so no per-sample fractions stay in registers
    auto cell_frac_t = [&](float t, float& fx, float& fy, float& fz) {
        const float px = fmaf(t, j.d.x, j.o.x) * g.inv_vs;
        const float py = fmaf(t, j.d.y, j.o.y) * g.inv_vs;
        const float pz = fmaf(t, j.d.z, j.o.z) * g.inv_vs;
        fx = px - floorf(px);
        fy = py - floorf(py);
        fz = pz - floorf(pz);
    };
    auto cell_frac = [&](int i, float& fx, float& fy, float& fz) { cell_frac_t(t_[i], fx, fy, fz); };

    unsigned smask = 0;  // stored mode: samples whose record is valid
    int rm = 0, r_blk = -1, r_cell = -1;  // the lane's current walk record and its fields
    float r_s0 = 0.f, r_tin = 0.f, r_len = 0.f;
    // place sample i: its s, t, cell and block; false if the lane has no sample i
    auto place = [&](int i) -> bool {
        const int k = lane * Q + i;
        t_[i] = 0.f; dl_[i] = 0.f; d_[i] = 0.f; cr_[i] = cg_[i] = cb_[i] = 0.f; tau_[i] = 0.f; dsig_[i] = 0.f;
        if constexpr (kBeta) bq_[i] = 0.f;
        if constexpr (kNrm) gnx_[i] = gny_[i] = gnz_[i] = 0.f;
        ba_[i] = -1;
        if (!any) {  // warp-uniform
            if constexpr (kTrace) {
                if (k < N) {
                    const int64_t q = j.idx * N + k;
                    a.tr_t[q] = 0.f;
                    a.tr_cell[3 * q] = a.tr_cell[3 * q + 1] = a.tr_cell[3 * q + 2] = 0;
                    a.tr_blk[q] = -1;
                    a.tr_valid[q] = 0;
                }
            }
            return false;
        }
        int blk = -1, cell = -1;
        float t_rec = 0.f;
        if constexpr (!kStoreIn && !INWARP) {
            // every lane takes part in the record search (it shuffles), with or without a sample i: a binary
            // search for the lane's first sample, then (its samples are consecutive) a forward scan one record at
            // a time, the record's fields fetched again only when some lane moved
            const float sq = k < N ? s_[i] : 0.f;
            bool moved = i == 0;
            if constexpr (RPL == 1) {
                if (i == 0) {
                    rm = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const float v = __shfl_sync(kFull, my_s0, rm + step);
                        if (rm + step < n_rec && v <= sq) rm += step;
                    }
                } else {
                    for (int it = 0; it < kWalkCap; ++it) {
                        const float v = __shfl_sync(kFull, my_s0, rm + 1 < kWalkCap ? rm + 1 : kWalkCap - 1);
                        const bool adv = rm + 1 < n_rec && v <= sq;
                        if (!__any_sync(kFull, adv)) break;
                        if (adv) {
                            ++rm;
                            moved = true;
                        }
                    }
                }
                if (__any_sync(kFull, moved)) {
                    r_s0 = __shfl_sync(kFull, my_s0, rm);
                    r_tin = __int_as_float(__shfl_sync(kFull, my_rec.x, rm));
                    r_len = __int_as_float(__shfl_sync(kFull, my_rec.y, rm));
                    r_blk = __shfl_sync(kFull, my_rec.z, rm);
                    r_cell = __shfl_sync(kFull, my_rec.w, rm);
                }
            } else {
                // record r lives in lane r % 32, in its first (r < 32) or second register set: both shuffled, the
                // caller's half selected
                auto s0_of = [&](int r) {
                    const float lo = __shfl_sync(kFull, my_s0, r & 31), hi = __shfl_sync(kFull, my_s0b, r & 31);
                    return r < kWalkCap ? lo : hi;
                };
                if (i == 0) {
                    rm = 0;
#pragma unroll
                    for (int step = 32; step > 0; step >>= 1) {
                        const float v = s0_of(rm + step < kWalkSlot ? rm + step : kWalkSlot - 1);
                        if (rm + step < n_rec && v <= sq) rm += step;
                    }
                } else {
                    for (int it = 0; it < kWalkSlot; ++it) {
                        const float v = s0_of(rm + 1 < kWalkSlot ? rm + 1 : kWalkSlot - 1);
                        const bool adv = rm + 1 < n_rec && v <= sq;
                        if (!__any_sync(kFull, adv)) break;
                        if (adv) {
                            ++rm;
                            moved = true;
                        }
                    }
                }
                if (__any_sync(kFull, moved)) {
                    const bool hi = rm >= kWalkCap;
                    const int src = rm & 31;
                    r_s0 = s0_of(rm);
                    const int x0 = __shfl_sync(kFull, my_rec.x, src), x1 = __shfl_sync(kFull, my_recb.x, src);
                    const int y0 = __shfl_sync(kFull, my_rec.y, src), y1 = __shfl_sync(kFull, my_recb.y, src);
                    const int z0 = __shfl_sync(kFull, my_rec.z, src), z1 = __shfl_sync(kFull, my_recb.z, src);
                    const int w0 = __shfl_sync(kFull, my_rec.w, src), w1 = __shfl_sync(kFull, my_recb.w, src);
                    r_tin = __int_as_float(hi ? x1 : x0);
                    r_len = __int_as_float(hi ? y1 : y0);
                    r_blk = hi ? z1 : z0;
                    r_cell = hi ? w1 : w0;
                }
            }
            blk = r_blk;
            cell = r_cell;
            t_rec = r_tin + fminf(sq - r_s0, r_len);
        }
        if (k >= N) return false;
        float sn;
        if (k + 1 >= N) sn = S;
        else if (i + 1 < Q) sn = s_[i + 1 < Q ? i + 1 : i];
        else sn = s_after;
        dl_[i] = sn - s_[i];
        if constexpr (kStoreIn) {
            const float* rec = a.rec + j.idx * RS + i * 32 + lane;
            const int64_t CS = a.n * RS;
            t_[i] = rec[0];
            d_[i] = rec[CS];
            cr_[i] = rec[2 * CS];
            cg_[i] = rec[3 * CS];
            cb_[i] = rec[4 * CS];
            blk = __float_as_int(rec[5 * CS]);
            if (!isnan(d_[i])) smask |= 1u << i;
        } else {
            if constexpr (INWARP) t_[i] = locate(g, j, sm, pc, t1, s_[i], blk, cell);
            else t_[i] = t_rec;
        }
        const float px = fmaf(t_[i], j.d.x, j.o.x) * g.inv_vs;
        const float py = fmaf(t_[i], j.d.y, j.o.y) * g.inv_vs;
        const float pz = fmaf(t_[i], j.d.z, j.o.z) * g.inv_vs;
        const float flx = floorf(px), fly = floorf(py), flz = floorf(pz);
        const int cx = (int)flx, cy = (int)fly, cz = (int)flz;
        const int lc = (cx & 7) | ((cy & 7) << 3) | ((cz & 7) << 6);
        if constexpr (!kStoreIn) {
            // the sample's own block: the traversal cell's, unless rounding put it across a block face
            const int own = dense_cell(g, cx >> 3, cy >> 3, cz >> 3);
            if (own != cell)
                blk = own < 0 || !sdg_in_range(g.status, own, g.dense_cells, SDG_CHECK_DENSE) ? -1
                                                                                          : __ldg(g.dense + own);
        }
        ba_[i] = blk >= 0 ? blk * 512 + lc : -1;
        if constexpr (kTrace) {
            const int64_t q = j.idx * N + k;
            a.tr_t[q] = t_[i];
            a.tr_cell[3 * q] = cx;
            a.tr_cell[3 * q + 1] = cy;
            a.tr_cell[3 * q + 2] = cz;
            a.tr_blk[q] = blk;
        }
        return true;
    };
    // evaluate sample i: corner fetch into cs/crr/cgg/cbb (or, with reuse, the corners already there when the
    // previous sample is in the same cell), trilinear interpolation, density
    auto evaluate = [&](int i, bool reuse, float (&cs)[8], float (&crr)[8], float (&cgg)[8], float (&cbb)[8]) {
        bool valid;
        if constexpr (kStoreIn) {
            valid = (smask >> i) & 1u;
        } else {
            // a sample in the previous sample's cell reuses its corner values
            const bool same =
                reuse && i > 0 && ((vmask >> (i - 1)) & 1u) && ba_[i] == ba_[i - 1];
            if (same) {
                valid = true;
            } else {
                int addr[8];
                valid = ba_[i] >= 0 && corner_addresses(g, ba_[i] >> 9, ba_[i] & 511, addr);
                if (valid) load_corners<BF16>(g, addr, cs, crr, cgg, cbb);
            }
            if (valid) {
                float w[8], fx, fy, fz;
                cell_frac(i, fx, fy, fz);
                trilinear_weights(fx, fy, fz, w);
                float dd = 0.f, r = 0.f, gg = 0.f, bb = 0.f;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    dd = fmaf(w[e], cs[e], dd);
                    r = fmaf(w[e], crr[e], r);
                    gg = fmaf(w[e], cgg[e], gg);
                    bb = fmaf(w[e], cbb[e], bb);
                }
                d_[i] = dd; cr_[i] = r; cg_[i] = gg; cb_[i] = bb;
                if constexpr (kNrm) sdf_gradient(fx, fy, fz, g.inv_vs, cs, gnx_[i], gny_[i], gnz_[i]);
            }
        }
        if constexpr (kTrace) a.tr_valid[j.idx * N + lane * Q + i] = valid ? 1 : 0;
        if (valid) {
            vmask |= 1u << i;
            // sigma = Psi_beta(-d) / beta, the Laplace CDF transform (Sec. 3.5.1)
            const float e = __expf(-fabsf(d_[i]) * g.inv_beta);
            const float sig = d_[i] >= 0.f ? 0.5f * g.inv_beta * e : g.inv_beta * (1.f - 0.5f * e);
            tau_[i] = sig * dl_[i];
            dsig_[i] = -0.5f * g.inv_beta * g.inv_beta * e * dl_[i];  // delta * dsigma/dd
            // sigma = Psi(-d/beta)/beta gives dsigma/dbeta = -sigma/beta - (d/beta) dsigma/dd, so
            // delta dsigma/dbeta = -(tau + d * dsig) / beta: keep tau + d * dsig for the backward
            if constexpr (kBeta) bq_[i] = fmaf(d_[i], dsig_[i], tau_[i]);
        }
        if constexpr (kStoreOut) {
            float* rec = a.rec + j.idx * RS + i * 32 + lane;
            const int64_t CS = a.n * RS;
            rec[0] = t_[i];
            rec[CS] = valid ? d_[i] : __int_as_float(0x7fc00000);
            rec[2 * CS] = cr_[i];
            rec[3 * CS] = cg_[i];
            rec[4 * CS] = cb_[i];
            rec[5 * CS] = __int_as_float(ba_[i] >= 0 ? ba_[i] >> 9 : -1);
        }
    };
    // The fused training and the forward modes place all samples first and then reuse a cell's corners for the
    // lane's next sample in it (about half of the samples); the separate backward passes keep the single
    // place-and-fetch loop, where holding the corners costs more registers than the loads it saves.
    if constexpr (kTrain || kFwdOut) {
        unsigned pmask = 0;  // samples placed
#pragma unroll
        for (int i = 0; i < Q; ++i)
            if (place(i)) pmask |= 1u << i;
        float cs[8], crr[8], cgg[8], cbb[8];  // corner values of the last loaded cell
#pragma unroll
        for (int i = 0; i < Q; ++i)
            if ((pmask >> i) & 1u) evaluate(i, true, cs, crr, cgg, cbb);
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            float cs[8], crr[8], cgg[8], cbb[8];
            if (place(i)) evaluate(i, false, cs, crr, cgg, cbb);
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

    // runs: consecutive valid samples of a lane in the same cell share their 8 corners
    auto same_cell = [&](int i0, int i1) { return ba_[i0] == ba_[i1]; };
    auto run_start = [&](int i) {
        return ((vmask >> i) & 1u) && (i == 0 || !((vmask >> (i - 1)) & 1u) || !same_cell(i - 1, i));
    };
    auto run_end = [&](int i) {
        return ((vmask >> i) & 1u) && (i == Q - 1 || !((vmask >> (i + 1)) & 1u) || !same_cell(i, i + 1));
    };
    // The semantic phases run their sample loop rolled (one copy of the channel loops instead of Q), taking the
    // lane's sample i out of the per-sample registers with pick() and its run boundaries from these masks.
    unsigned rs_mask = 0, re_mask = 0;
    if constexpr (SEM) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            rs_mask |= (run_start(i) ? 1u : 0u) << i;
            re_mask |= (run_end(i) ? 1u : 0u) << i;
        }
    }

    // semantic logits: per run, corner weights W_e = sum_i w_i r_e(f_i)
    float sem_acc[SEMCAP > 0 ? SEMCAP : 1];
    if constexpr (SEM) {
#pragma unroll
        for (int c = 0; c < SEMCAP; ++c) sem_acc[c] = 0.f;
    }
    if constexpr (SEM && (kFwdOut || kTrain)) {
        if (any) {
            float W[8];
            int addr[8];
#pragma unroll 1
            for (int i = 0; i < Q; ++i) {
                const bool v = (vmask >> i) & 1u;
                if ((rs_mask >> i) & 1u) {
#pragma unroll
                    for (int e = 0; e < 8; ++e) W[e] = 0.f;
                    const int bai = pick(ba_, i);
                    corner_addresses(g, bai >> 9, bai & 511, addr);
                }
                if (v) {
                    float r[8];
                    float fx, fy, fz;
                    cell_frac_t(pick(t_, i), fx, fy, fz);
                    trilinear_weights(fx, fy, fz, r);
                    const float wi = pick(w_, i);
#pragma unroll
                    for (int e = 0; e < 8; ++e) W[e] = fmaf(wi, r[e], W[e]);
                }
                if ((re_mask >> i) & 1u) {
#pragma unroll
                    for (int c4 = 0; c4 < SEMCAP / 4; ++c4) {
                        if (4 * c4 < ns) {
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                float sv[4];
                                sem_load4(g, addr[e], 4 * c4, sv);
#pragma unroll
                                for (int q = 0; q < 4; ++q)
                                    sem_acc[4 * c4 + q] = fmaf(W[e], sv[q], sem_acc[4 * c4 + q]);
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
    float Nx = 0.f, Ny = 0.f, Nz = 0.f;  // rendered normal sum_k w_k grad f(x_k) (Eq. 14)
    if constexpr (kNrm) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            Nx = fmaf(w_[i], gnx_[i], Nx);
            Ny = fmaf(w_[i], gny_[i], Ny);
            Nz = fmaf(w_[i], gnz_[i], Nz);
        }
        Nx = warp_sum(Nx);
        Ny = warp_sum(Ny);
        Nz = warp_sum(Nz);
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
    float gNx = 0.f, gNy = 0.f, gNz = 0.f;  // normal seeds (PASS_TRAIN_NRM)
    float gS[SEMCAP > 0 ? SEMCAP : 1];
    if constexpr (kTrain) {
        // L1 colour + lambda_d L1 depth (+ lambda_s squared L2 logits), mean over rays
        const float e0 = C0 - a.t_rgb[3 * j.idx], e1 = C1 - a.t_rgb[3 * j.idx + 1], e2 = C2 - a.t_rgb[3 * j.idx + 2];
        const float ed = D - a.t_depth[j.idx];
        const float third = a.inv_n * (1.0f / 3.0f);
        gC0 = sgnf(e0) * third; gC1 = sgnf(e1) * third; gC2 = sgnf(e2) * third;
        gD = a.lam_d * sgnf(ed) * a.inv_n;
        gO = 0.f;
        float L = (fabsf(e0) + fabsf(e1) + fabsf(e2)) * third + a.lam_d * fabsf(ed) * a.inv_n;
        if constexpr (kNrm) {
            // L1 normal loss (Eq. 14): lambda_n |N - N^|_1 / (3n)
            const float nth = a.lam_n * third;
            const float n0 = Nx - a.t_normal[3 * j.idx], n1 = Ny - a.t_normal[3 * j.idx + 1],
                        n2 = Nz - a.t_normal[3 * j.idx + 2];
            gNx = sgnf(n0) * nth;
            gNy = sgnf(n1) * nth;
            gNz = sgnf(n2) * nth;
            L += (fabsf(n0) + fabsf(n1) + fabsf(n2)) * nth;
        }
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
    if (!any) {
        if constexpr (kBeta)
            if (lane == 0) a.beta_part[j.idx] = 0.f;
        return;
    }

    // v_k = g_rgb . c_k + g_depth t_k + g_opac + g_sem . s_k
    float v_[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) v_[i] = fmaf(gC0, cr_[i], fmaf(gC1, cg_[i], fmaf(gC2, cb_[i], fmaf(gD, t_[i], gO))));
    if constexpr (kNrm) {
#pragma unroll
        for (int i = 0; i < Q; ++i) v_[i] = fmaf(gNx, gnx_[i], fmaf(gNy, gny_[i], fmaf(gNz, gnz_[i], v_[i])));
    }
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
#pragma unroll 1
            for (int i = 0; i < Q; ++i) {
                if ((rs_mask >> i) & 1u) {
                    const int bai = pick(ba_, i);
                    corner_addresses(g, bai >> 9, bai & 511, addr);
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
                if ((vmask >> i) & 1u) {
                    float r[8];
                    float fx, fy, fz;
                    cell_frac_t(pick(t_, i), fx, fy, fz);
                    trilinear_weights(fx, fy, fz, r);
                    float acc = 0.f;
#pragma unroll
                    for (int e = 0; e < 8; ++e) acc = fmaf(r[e], dot[e], acc);
#pragma unroll
                    for (int k = 0; k < Q; ++k)
                        if (k == i) v_[k] += acc;
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
    float bsum = 0.f;  // sum_k dL/dtau_k (tau_k + d_k dsig_k)
#pragma unroll
    for (int i = Q - 1; i >= 0; --i) {
        const float dtau = Tn_[i] * v_[i] - R - ubg;
        R = fmaf(w_[i], v_[i], R);
        dd_[i] = ((vmask >> i) & 1u) ? dsig_[i] * dtau : 0.f;
        if constexpr (kBeta) bsum = fmaf(dtau, bq_[i], bsum);
    }
    if constexpr (kBeta) {
        bsum = warp_sum(bsum);
        if (lane == 0) a.beta_part[j.idx] = -bsum * g.inv_beta;
    }

    // ---------------- scatter to voxels (runs of same-cell samples) ----------------
    // Per run and corner e only aS_e = sum_i r_e(f_i) dd_i and aW_e = sum_i r_e(f_i) w_i are accumulated:
    // the colour (and logit) gradients of a corner are the ray's seeds times aW_e.
    // Semantic records kernels first sum (aS, aW) per distinct voxel of the ray in a per-warp table in shared
    // memory (kTabSlots keys, open addressing), then issue one set of vector atomics per voxel: a ray's runs reach
    // most voxels more than once (about 400 corner contributions onto about 200 voxels at 128 samples), and a
    // voxel's logit gradient is the ray's seed times its summed aW, so the 5-8 vector atomics of a corner are
    // issued once per voxel instead of once per run (render kernels 5.70 -> 5.58 ms per 2^18-ray precision step).
    // A key that finds no slot within 32 probes is scattered straight to memory.
    constexpr bool kTab = SEM && !INWARP && RPL == 1;
    constexpr int kTabSlots = 512;
    __shared__ __align__(16) int tab_key[kTab ? kWarpsPerBlock : 1][kTab ? kTabSlots : 1];
    // the two sums in arrays of their own, so that a slot's atomics fall in 32 banks rather than the 16 even ones of
    // an interleaved pair (5.57 -> 5.53 ms)
    // With BF16 colour the SDF gradient has an array of its own: a run's SDF seeds go straight to it with scalar
    // atomics and the table keeps only the weights, one shared-memory atomic less per corner (5.53 -> 5.34 ms)
    constexpr bool kTabS = kTab && !BF16;
    __shared__ __align__(16) float tab_s[kTabS ? kWarpsPerBlock : 1][kTabS ? kTabSlots : 1];
    __shared__ __align__(16) float tab_w[kTab ? kWarpsPerBlock : 1][kTab ? kTabSlots : 1];
    const int wib = kTab ? (threadIdx.x >> 5) : 0;
    if constexpr (kTab) {
        int4* k4 = reinterpret_cast<int4*>(tab_key[wib]);
        float4* s4 = reinterpret_cast<float4*>(tab_s[wib]);
        float4* w4 = reinterpret_cast<float4*>(tab_w[wib]);
#pragma unroll
        for (int u = 0; u < kTabSlots / 128; ++u) {
            k4[lane + 32 * u] = make_int4(-1, -1, -1, -1);
            if constexpr (kTabS) s4[lane + 32 * u] = make_float4(0.f, 0.f, 0.f, 0.f);
            w4[lane + 32 * u] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncwarp();
    }
    // the gradients of one voxel from sums (as, aw) over runs (sdf false: its SDF seed already sent)
    auto scatter_voxel = [&](int ad, float as_, float aw_, bool sdf = true) {
        if constexpr (!BF16) {
            red_add_v4(g.ggeo + ad, as_, gC0 * aw_, gC1 * aw_, gC2 * aw_);
        } else {
            if (sdf) atomicAdd(g.gsdf + ad, as_);
            red_add_v4(g.grgb + ad, gC0 * aw_, gC1 * aw_, gC2 * aw_, 0.f);
        }
        if (SEM && sem_grad) {
#pragma unroll
            for (int c4 = 0; c4 < SEMCAP / 4; ++c4)
                if (4 * c4 < ns)
                    red_add_v4(reinterpret_cast<float4*>(g.gsem + (int64_t)ad * ns) + c4, aw_ * gS[4 * c4],
                               aw_ * gS[4 * c4 + 1], aw_ * gS[4 * c4 + 2], aw_ * gS[4 * c4 + 3]);
        }
    };
    {
        int addr[8];
        float aS[8], aW[8];
        // sample i of the lane (a compile-time constant in the unrolled loop, where pick() is a[i])
        auto scatter_sample = [&](int i) {
            const bool v = (vmask >> i) & 1u;
            if (SEM ? ((rs_mask >> i) & 1u) != 0 : run_start(i)) {
#pragma unroll
                for (int e = 0; e < 8; ++e) aS[e] = aW[e] = 0.f;
                const int bai = pick(ba_, i);
                corner_addresses(g, bai >> 9, bai & 511, addr);
            }
            if (v) {
                float r[8];
                float fx, fy, fz;
                cell_frac_t(pick(t_, i), fx, fy, fz);
                trilinear_weights(fx, fy, fz, r);
                const float ddi = pick(dd_, i), wi = pick(w_, i);
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    aS[e] = fmaf(r[e], ddi, aS[e]);
                    aW[e] = fmaf(r[e], wi, aW[e]);
                }
                if constexpr (kNrm) {
                    // the rendered normal's grad f part: w_i g_N . grad_x r_e(x_i) onto each corner's SDF
                    const float sc = wi * g.inv_vs;
                    float q[8];
                    dot_weight_gradients(fx, fy, fz, sc * gNx, sc * gNy, sc * gNz, q);
#pragma unroll
                    for (int e = 0; e < 8; ++e) aS[e] += q[e];
                }
            }
            if (SEM ? ((re_mask >> i) & 1u) != 0 : run_end(i)) {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    if constexpr (kTab) {
                        const int key = addr[e];
                        if constexpr (!kTabS) atomicAdd(g.gsdf + key, aS[e]);
                        unsigned h = ((unsigned)key * 2654435761u) >> 23;  // 9 bits: kTabSlots = 512
                        bool done = false;
                        for (int probe = 0; probe < 32; ++probe) {
                            const int old = atomicCAS(&tab_key[wib][h], -1, key);
                            if (old == -1 || old == key) {
                                if constexpr (kTabS) atomicAdd(&tab_s[wib][h], aS[e]);
                                atomicAdd(&tab_w[wib][h], aW[e]);
                                done = true;
                                break;
                            }
                            h = (h + 1) & (kTabSlots - 1);
                        }
                        if (!done) scatter_voxel(key, aS[e], aW[e], kTabS);  // a crowded table: straight to memory
                    } else {
                        scatter_voxel(addr[e], aS[e], aW[e]);
                    }
                }
            }
        };
        if constexpr (SEM) {
#pragma unroll 1
            for (int i = 0; i < Q; ++i) scatter_sample(i);
            if constexpr (kTab) {
                __syncwarp();
#pragma unroll 1
                for (int u = lane; u < kTabSlots; u += 32) {
                    const int key = tab_key[wib][u];
                    if (key >= 0) scatter_voxel(key, kTabS ? tab_s[wib][u] : 0.f, tab_w[wib][u], kTabS);
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) scatter_sample(i);
        }
    }
}

// ---------------------------------------------------------------------------
// Launch entry of the render kernels (defined in render_kernels.cuh, instantiated in the render_inst_*.cu files)
// ---------------------------------------------------------------------------
// Semantic channel capacities the kernels are instantiated for: a grid with at most kSemCapSmall logits per voxel
// runs the program unrolled for kSemCapSmall channels (less code than for 32, and no spills at 128 registers),
// one with more (24-32) the program unrolled for 32.
constexpr int kSemCapSmall = 20;
inline int sem_cap(int n_sem) { return n_sem == 0 ? 0 : n_sem <= kSemCapSmall ? kSemCapSmall : 32; }

template <int MODE, bool BF16, int NSC>
int launch_q(const GridDev& gd, const float* rays, uint32_t id0, const PassArgs& a, int Q, cudaStream_t s);

// launch_q for a grid's layout: FP32 or BF16 colour, and the semantic capacity its n_sem needs.
template <int MODE>
int launch_layout(bool bf16, int n_sem, const GridDev& gd, const float* rays, uint32_t id0, const PassArgs& a,
                  int Q, cudaStream_t s) {
    const int cap = sem_cap(n_sem);
    if (cap == 0) return bf16 ? launch_q<MODE, true, 0>(gd, rays, id0, a, Q, s)
                              : launch_q<MODE, false, 0>(gd, rays, id0, a, Q, s);
    if (cap == kSemCapSmall) return bf16 ? launch_q<MODE, true, kSemCapSmall>(gd, rays, id0, a, Q, s)
                                         : launch_q<MODE, false, kSemCapSmall>(gd, rays, id0, a, Q, s);
    return bf16 ? launch_q<MODE, true, 32>(gd, rays, id0, a, Q, s) : launch_q<MODE, false, 32>(gd, rays, id0, a, Q, s);
}

}  // namespace sdg
