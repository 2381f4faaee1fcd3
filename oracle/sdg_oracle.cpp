// CPU reference ("oracle") for the sparse-dense SDF volume renderer.
//
// TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
// benchmark's CPU-baseline / reference arm load this library.  It is plain,
// slow and single-threaded on purpose, written step by step from the paper
// (arXiv 2305.13220, "Fast Monocular Scene Reconstruction with Global-Sparse
// Local-Dense Grids"), and shares no source with the CUDA library.
//
// Precision: every step runs in FP64, except block activation (Eq. 7-8),
// which runs in FP32 with a fixed operation order and no fused multiply-add
// (build with -ffp-contract=off), because the block set it produces must be
// bit-identical to what any FP32 implementation of the same order gives.
//
// Data layout conventions (these are interface, not code):
//   * grid point (voxel) v in Z^3 sits at world position v * voxel_size;
//   * block key b = floor(v / 8) per axis; local index v - 8b in [0,8)^3,
//     stored at linear position lz*64 + ly*8 + lx inside the block;
//   * block indices are assigned in ascending (z, y, x) key order per
//     activation batch;
//   * a ray record is 8 floats: ox, oy, oz, tnear, dx, dy, dz, tfar.
//
// Parity pins for every function live in tests/test_oracle_*.py.  Nothing
// here is "parity unpinned".
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <set>
#include <vector>

namespace {

struct BKey {
    int32_t x, y, z;
};
// Ascending (z, y, x) order: the order in which an activation batch assigns indices.
bool operator<(const BKey& a, const BKey& b) {
    if (a.z != b.z) return a.z < b.z;
    if (a.y != b.y) return a.y < b.y;
    return a.x < b.x;
}

int64_t floordiv(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
    return q;
}

// ---------------------------------------------------------------------------
// Grid: block map + dense 8^3 voxel arrays per block (Sec. 3.2, "Sparse-Dense
// Data Structure").  The block map is an ordered map: exact, collision-free.
// ---------------------------------------------------------------------------
struct Grid {
    double vs = 0.01;
    double beta = 0.005;
    int n_sem = 0;
    std::map<BKey, int64_t> index;
    std::vector<BKey> keys;
    std::vector<double> sdf;  // [N][512]
    std::vector<double> rgb;  // [N][512][3]
    std::vector<double> sem;  // [N][512][n_sem]
    int64_t lo[3] = {0, 0, 0}, hi[3] = {-1, -1, -1};  // inclusive block AABB
};

// Voxel v -> linear storage index, or false if its block is not allocated.
bool voxel_index(const Grid& g, int64_t vx, int64_t vy, int64_t vz, int64_t* lin, int64_t* blk) {
    BKey k{(int32_t)floordiv(vx, 8), (int32_t)floordiv(vy, 8), (int32_t)floordiv(vz, 8)};
    auto it = g.index.find(k);
    if (it == g.index.end()) return false;
    int64_t lx = vx - 8 * (int64_t)k.x, ly = vy - 8 * (int64_t)k.y, lz = vz - 8 * (int64_t)k.z;
    *lin = it->second * 512 + lz * 64 + ly * 8 + lx;
    if (blk) *blk = it->second;
    return true;
}

// ---------------------------------------------------------------------------
// Trilinear interpolation, Sec. 3.5.2 (f = sum_i r(x, x_i) theta(x_i) over the
// 8 grid points around x).  A sample whose 8 grid points are not all in
// allocated blocks is invalid.
// ---------------------------------------------------------------------------
struct Stencil {
    bool valid;
    int64_t lin[8];
    int64_t blk[8];
    double r[8];
    double f[3];
};

// Stencil of the cell whose base corner is voxel c: f = x / vs - c per axis (in [0, 1) when c = floor(x / vs)).
Stencil stencil_in_cell(const Grid& g, const double x[3], const int64_t c[3]) {
    Stencil s;
    for (int a = 0; a < 3; ++a) s.f[a] = x[a] / g.vs - (double)c[a];
    s.valid = true;
    for (int e = 0; e < 8; ++e) {
        int ex = e & 1, ey = (e >> 1) & 1, ez = (e >> 2) & 1;
        if (!voxel_index(g, c[0] + ex, c[1] + ey, c[2] + ez, &s.lin[e], &s.blk[e])) {
            s.valid = false;
            s.lin[e] = -1;
            s.blk[e] = -1;
        }
        s.r[e] = (ex ? s.f[0] : 1.0 - s.f[0]) * (ey ? s.f[1] : 1.0 - s.f[1]) * (ez ? s.f[2] : 1.0 - s.f[2]);
    }
    return s;
}

Stencil stencil_at(const Grid& g, const double x[3]) {
    int64_t c[3];
    for (int a = 0; a < 3; ++a) c[a] = (int64_t)std::floor(x[a] / g.vs);
    return stencil_in_cell(g, x, c);
}

// ---------------------------------------------------------------------------
// SDF -> density, Sec. 3.5.1: alpha(x) = l(f(x)), the Laplace-CDF transform of
// VolSDF: sigma(d) = (1/beta) * Psi_beta(-d), Psi_beta the CDF of Laplace(0,beta).
// ---------------------------------------------------------------------------
double laplace_cdf(double s, double beta) {
    return s <= 0 ? 0.5 * std::exp(s / beta) : 1.0 - 0.5 * std::exp(-s / beta);
}
double density(double d, double beta) { return laplace_cdf(-d, beta) / beta; }
double density_deriv(double d, double beta) {  // d sigma / d d = -(1/beta) * pdf(-d)
    return -std::exp(-std::fabs(d) / beta) / (2.0 * beta * beta);
}
// d sigma / d beta, differentiating the two branches of sigma directly:
//   d >= 0: sigma = exp(-d/beta) / (2 beta)        -> sigma (d - beta) / beta^2
//   d <  0: sigma = (1 - exp(d/beta) / 2) / beta   -> -sigma / beta + d exp(d/beta) / (2 beta^3)
double density_dbeta(double d, double beta) {
    const double s = density(d, beta);
    if (d >= 0.0) return s * (d - beta) / (beta * beta);
    return -s / beta + d * std::exp(d / beta) / (2.0 * beta * beta * beta);
}

// ---------------------------------------------------------------------------
// Counter-based uniform numbers for stratified sampling: the PCG integer hash
// of Jarzynski & Olano, "Hash Functions for GPU Rendering" (JCGT 2020), nested
// over (seed, ray, k); u = top 24 bits * 2^-24, exact in FP32 and FP64.
// ---------------------------------------------------------------------------
uint32_t pcg_hash(uint32_t v) {
    uint32_t state = v * 747796405u + 2891336453u;
    uint32_t word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
    return (word >> 22u) ^ word;
}
uint32_t sample_hash(uint32_t seed, uint32_t ray, uint32_t k) {
    return pcg_hash(k + pcg_hash(ray + pcg_hash(seed)));
}
double sample_u(uint32_t seed, uint32_t ray, uint32_t k) {
    return (double)(sample_hash(seed, ray, k) >> 8) * (1.0 / 16777216.0);
}

// ---------------------------------------------------------------------------
// Empty-space skipping (Sec. 3.5.1: samples only where blocks are allocated).
// Brute force: every block-boundary plane crossing of the ray inside the
// grid's AABB splits it into segments; a segment is kept if the block holding
// its midpoint is allocated; touching kept segments are merged.
// ---------------------------------------------------------------------------
struct Interval {
    double t_in, t_out;
};

bool clip_to_aabb(const Grid& g, const double o[3], const double d[3], double* t0, double* t1) {
    if (g.keys.empty()) return false;
    const double L = 8.0 * g.vs;
    for (int a = 0; a < 3; ++a) {
        double lo = g.lo[a] * L, hi = (g.hi[a] + 1) * L;
        if (d[a] == 0.0) {
            if (o[a] < lo || o[a] > hi) return false;
            continue;
        }
        double ta = (lo - o[a]) / d[a], tb = (hi - o[a]) / d[a];
        *t0 = std::max(*t0, std::min(ta, tb));
        *t1 = std::min(*t1, std::max(ta, tb));
    }
    return *t0 < *t1;
}

std::vector<Interval> traverse(const Grid& g, const double o[3], const double d[3], double tn, double tf) {
    std::vector<Interval> out;
    double t0 = tn, t1 = tf;
    if (!clip_to_aabb(g, o, d, &t0, &t1)) return out;
    const double L = 8.0 * g.vs;
    std::vector<double> ts{t0, t1};
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) continue;
        double xa = o[a] + t0 * d[a], xb = o[a] + t1 * d[a];
        int64_t m0 = (int64_t)std::ceil(std::min(xa, xb) / L);
        int64_t m1 = (int64_t)std::floor(std::max(xa, xb) / L);
        for (int64_t m = m0; m <= m1; ++m) {
            double t = (m * L - o[a]) / d[a];
            if (t > t0 && t < t1) ts.push_back(t);
        }
    }
    std::sort(ts.begin(), ts.end());
    for (size_t i = 0; i + 1 < ts.size(); ++i) {
        double ta = ts[i], tb = ts[i + 1];
        if (!(tb > ta)) continue;
        double tm = 0.5 * (ta + tb);
        BKey k;
        k.x = (int32_t)std::floor((o[0] + tm * d[0]) / L);
        k.y = (int32_t)std::floor((o[1] + tm * d[1]) / L);
        k.z = (int32_t)std::floor((o[2] + tm * d[2]) / L);
        if (g.index.find(k) == g.index.end()) continue;
        if (!out.empty() && out.back().t_out == ta)
            out.back().t_out = tb;
        else
            out.push_back({ta, tb});
    }
    return out;
}

// ---------------------------------------------------------------------------
// One ray, forward: samples, interpolation, density, compositing (Eq. 12-15).
// ---------------------------------------------------------------------------
struct Sample {
    double s, t, delta;
    bool valid;
    Stencil st;
    double d, c[3];
    double gf[3];  // grad f at the sample (Eq. 17), for the rendered normal of Eq. 14
    std::vector<double> sem;
    double sigma, tau, T, w;
};

struct RayResult {
    std::vector<Sample> smp;
    std::vector<Interval> iv;
    double S = 0.0, TN = 1.0;
    double C[3] = {0, 0, 0}, D = 0.0, O = 0.0;
    double Nrm[3] = {0, 0, 0};  // rendered normal sum_k w_k grad f(x_k) (Eq. 14)
    std::vector<double> sem;
    int n_valid = 0;
    bool degenerate = false;
};

// Trilinear weight r(x, x_i) of stencil corner e and its gradient in x (Sec. 3.5.2): r is a product over the
// axes of f_a (far corner) or 1 - f_a (near corner), f = x/vs - floor(x/vs); its derivative along axis a replaces
// that axis's factor by +1/vs (far corner) or -1/vs (near corner).
void corner_weight_grad(const Stencil& s, double vs, int e, double* r, double dr[3]) {
    const int bit[3] = {e & 1, (e >> 1) & 1, (e >> 2) & 1};
    double fac[3], dfac[3];
    for (int a = 0; a < 3; ++a) {
        fac[a] = bit[a] ? s.f[a] : 1.0 - s.f[a];
        dfac[a] = (bit[a] ? 1.0 : -1.0) / vs;
    }
    *r = fac[0] * fac[1] * fac[2];
    dr[0] = dfac[0] * fac[1] * fac[2];
    dr[1] = fac[0] * dfac[1] * fac[2];
    dr[2] = fac[0] * fac[1] * dfac[2];
}

bool valid_at(const Grid& g, const double x[3]) { return stencil_at(g, x).valid; }

// Samples fixed by the caller instead of found by traversal (the comparison of a ray whose FP32 placement differs
// from the FP64 one only by rounding, at an interval joint or a block face): the allocated length S, and for every
// sample its ray parameter t_k and the base corner of its trilinear cell.  Everything else -- s_k and delta_k from
// S, the stencil's validity and weights, density, compositing, backward -- is computed here as for any ray.
struct Given {
    double S;
    const float* t;       // [N]
    const int32_t* cell;  // [N][3]
};

RayResult render_ray(const Grid& g, const float* ray, int N, uint32_t seed, uint32_t ray_id, int stratified,
                     const double bg[3], const Given* gv = nullptr) {
    RayResult R;
    R.sem.assign(g.n_sem, 0.0);
    double o[3] = {ray[0], ray[1], ray[2]}, d[3] = {ray[4], ray[5], ray[6]};
    if (gv) {
        R.S = gv->S;
    } else {
        R.iv = traverse(g, o, d, ray[3], ray[7]);
        for (auto& v : R.iv) R.S += v.t_out - v.t_in;
    }
    if (!(R.S > 0.0)) {
        for (int c = 0; c < 3; ++c) R.C[c] = bg[c];
        return R;
    }
    // interval starts in skip-space
    std::vector<double> s_start(R.iv.size());
    double acc = 0.0;
    for (size_t i = 0; i < R.iv.size(); ++i) {
        s_start[i] = acc;
        acc += R.iv[i].t_out - R.iv[i].t_in;
    }
    R.smp.resize(N);
    for (int k = 0; k < N; ++k) {
        double u = stratified ? sample_u(seed, ray_id, (uint32_t)k) : 0.5;
        R.smp[k].s = ((double)k + u) * R.S / (double)N;
    }
    for (int k = 0; k < N; ++k) {
        Sample& sm = R.smp[k];
        sm.delta = (k + 1 < N ? R.smp[k + 1].s : R.S) - sm.s;
        if (gv) {
            sm.t = gv->t[k];
        } else {
            size_t i = 0;
            while (i + 1 < R.iv.size() && sm.s >= s_start[i + 1]) ++i;
            sm.t = R.iv[i].t_in + (sm.s - s_start[i]);
        }
        double x[3] = {o[0] + sm.t * d[0], o[1] + sm.t * d[1], o[2] + sm.t * d[2]};
        if (gv) {
            const int64_t c[3] = {gv->cell[3 * k], gv->cell[3 * k + 1], gv->cell[3 * k + 2]};
            sm.st = stencil_in_cell(g, x, c);
        } else {
            sm.st = stencil_at(g, x);
        }
        sm.valid = sm.st.valid;
        sm.d = 0.0;
        sm.c[0] = sm.c[1] = sm.c[2] = 0.0;
        sm.gf[0] = sm.gf[1] = sm.gf[2] = 0.0;
        sm.sem.assign(g.n_sem, 0.0);
        if (sm.valid) {
            for (int e = 0; e < 8; ++e) {
                int64_t li = sm.st.lin[e];
                double r, dr[3];
                corner_weight_grad(sm.st, g.vs, e, &r, dr);
                for (int a = 0; a < 3; ++a) sm.gf[a] += dr[a] * g.sdf[li];
                sm.d += sm.st.r[e] * g.sdf[li];
                for (int c = 0; c < 3; ++c) sm.c[c] += sm.st.r[e] * g.rgb[li * 3 + c];
                for (int c = 0; c < g.n_sem; ++c) sm.sem[c] += sm.st.r[e] * g.sem[li * g.n_sem + c];
            }
            R.n_valid++;
        }
        sm.sigma = sm.valid ? density(sm.d, g.beta) : 0.0;
        sm.tau = sm.sigma * sm.delta;
        // degeneracy: a sample next to a skip-space joint, or whose validity flips under a tiny nudge
        if (gv) continue;
        for (size_t j = 1; j < R.iv.size(); ++j)
            if (std::fabs(sm.s - s_start[j]) < 1e-5) R.degenerate = true;
        const double eg = 5e-4 * g.vs;
        for (int a = 0; a < 3 && !R.degenerate; ++a)
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                double y[3] = {x[0], x[1], x[2]};
                y[a] += sgn * eg;
                if (valid_at(g, y) != sm.valid) R.degenerate = true;
            }
    }
    double cum = 0.0;
    for (int k = 0; k < N; ++k) {
        Sample& sm = R.smp[k];
        sm.T = std::exp(-cum);
        sm.w = sm.T * (1.0 - std::exp(-sm.tau));
        cum += sm.tau;
        for (int c = 0; c < 3; ++c) R.C[c] += sm.w * sm.c[c];
        for (int a = 0; a < 3; ++a) R.Nrm[a] += sm.w * sm.gf[a];
        R.D += sm.w * sm.t;
        R.O += sm.w;
        for (int c = 0; c < g.n_sem; ++c) R.sem[c] += sm.w * sm.sem[c];
    }
    R.TN = std::exp(-cum);
    for (int c = 0; c < 3; ++c) R.C[c] += R.TN * bg[c];
    return R;
}

}  // namespace

extern "C" {

// ----------------------------- activation ----------------------------------
// Eq. 8 with phi = 1: x = R * Pi^-1(p, D(p)) + t, in FP32 with this exact order:
//   xc = ((u + 0.5f) - cx) * (1/fx) * d ; yc likewise ; zc = d
//   x_i = ((R_i0*xc + R_i1*yc) + R_i2*zc) + t_i
// Pixels with a non-finite or non-positive depth are marked invalid.
int64_t orc_unproject(const float* depth, int H, int W, const float* K, const float* T, float* xyz,
                      uint8_t* valid) {
    const float ifx = 1.0f / K[0], ify = 1.0f / K[1];
    int64_t nv = 0;
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u) {
            int64_t i = (int64_t)v * W + u;
            float d = depth[i];
            bool ok = std::isfinite(d) && d > 0.0f;
            valid[i] = ok ? 1 : 0;
            float xc = (((float)u + 0.5f) - K[2]) * ifx * d;
            float yc = (((float)v + 0.5f) - K[3]) * ify * d;
            float zc = d;
            for (int a = 0; a < 3; ++a) {
                float p0 = T[a * 4 + 0] * xc;
                float p1 = T[a * 4 + 1] * yc;
                float p2 = T[a * 4 + 2] * zc;
                xyz[i * 3 + a] = ((p0 + p1) + p2) + T[a * 4 + 3];
            }
            nv += ok;
        }
    return nv;
}

void* orc_keyset_new() { return new std::set<BKey>(); }
void orc_keyset_free(void* ks) { delete (std::set<BKey>*)ks; }

// Eq. 7: union over points of the blocks touched by the voxel cube v + [-r, r]^3,
// v = floor(x * (1/vs)) in FP32.  The blocks touched along one axis are the
// integers floor((v-r)/8) .. floor((v+r)/8), so the union is a product of three
// ranges.  r = 8R reproduces the block dilation Dilate_R of the supplement exactly.
void orc_keyset_add_points(void* ks, const float* xyz, const uint8_t* valid, int64_t n, float vs, int r) {
    auto* S = (std::set<BKey>*)ks;
    const float inv = 1.0f / vs;
    for (int64_t i = 0; i < n; ++i) {
        if (valid && !valid[i]) continue;
        int64_t v[3];
        bool ok = true;
        for (int a = 0; a < 3; ++a) {
            float q = xyz[i * 3 + a] * inv;
            if (!std::isfinite(q) || std::fabs(q) > 8.0e6f) ok = false;
            v[a] = ok ? (int64_t)std::floor(q) : 0;
        }
        if (!ok) continue;
        int64_t b0[3], b1[3];
        for (int a = 0; a < 3; ++a) {
            b0[a] = floordiv(v[a] - r, 8);
            b1[a] = floordiv(v[a] + r, 8);
        }
        for (int64_t z = b0[2]; z <= b1[2]; ++z)
            for (int64_t y = b0[1]; y <= b1[1]; ++y)
                for (int64_t x = b0[0]; x <= b1[0]; ++x) S->insert(BKey{(int32_t)x, (int32_t)y, (int32_t)z});
    }
}

int64_t orc_keyset_size(void* ks) { return (int64_t)((std::set<BKey>*)ks)->size(); }

void orc_keyset_get(void* ks, int32_t* out) {
    int64_t i = 0;
    for (const BKey& k : *(std::set<BKey>*)ks) {
        out[i * 3 + 0] = k.x;
        out[i * 3 + 1] = k.y;
        out[i * 3 + 2] = k.z;
        ++i;
    }
}

// ------------------------------- grid --------------------------------------
void* orc_grid_new(double vs, double beta, int n_sem) {
    Grid* g = new Grid();
    g->vs = vs;
    g->beta = beta;
    g->n_sem = n_sem;
    return g;
}
void orc_grid_free(void* g) { delete (Grid*)g; }

// Blocks keys[i] get index i; the voxel arrays are copied.
int orc_grid_set(void* gp, const int32_t* keys, int64_t N, const double* sdf, const double* rgb, const double* sem) {
    Grid* g = (Grid*)gp;
    g->index.clear();
    g->keys.resize(N);
    for (int a = 0; a < 3; ++a) {
        g->lo[a] = INT64_MAX;
        g->hi[a] = INT64_MIN;
    }
    for (int64_t i = 0; i < N; ++i) {
        BKey k{keys[i * 3], keys[i * 3 + 1], keys[i * 3 + 2]};
        if (!g->index.emplace(k, i).second) return -1;  // duplicate key
        g->keys[i] = k;
        int32_t c[3] = {k.x, k.y, k.z};
        for (int a = 0; a < 3; ++a) {
            g->lo[a] = std::min<int64_t>(g->lo[a], c[a]);
            g->hi[a] = std::max<int64_t>(g->hi[a], c[a]);
        }
    }
    g->sdf.assign(sdf, sdf + N * 512);
    g->rgb.assign(rgb, rgb + N * 512 * 3);
    if (g->n_sem) g->sem.assign(sem, sem + N * 512 * g->n_sem);
    return 0;
}

void orc_grid_lookup(void* gp, const int32_t* keys, int64_t n, int32_t* idx) {
    Grid* g = (Grid*)gp;
    for (int64_t i = 0; i < n; ++i) {
        auto it = g->index.find(BKey{keys[i * 3], keys[i * 3 + 1], keys[i * 3 + 2]});
        idx[i] = it == g->index.end() ? -1 : (int32_t)it->second;
    }
}

// Allocated intervals of one ray (merged), at most cap of them; returns the count.
int orc_traverse(void* gp, const float* ray, double* t_in, double* t_out, int cap) {
    Grid* g = (Grid*)gp;
    double o[3] = {ray[0], ray[1], ray[2]}, d[3] = {ray[4], ray[5], ray[6]};
    auto iv = traverse(*g, o, d, ray[3], ray[7]);
    int n = (int)iv.size();
    for (int i = 0; i < n && i < cap; ++i) {
        t_in[i] = iv[i].t_in;
        t_out[i] = iv[i].t_out;
    }
    return n;
}

uint32_t orc_sample_hash(uint32_t seed, uint32_t ray, uint32_t k) { return sample_hash(seed, ray, k); }
double orc_sample_u(uint32_t seed, uint32_t ray, uint32_t k) { return sample_u(seed, ray, k); }
double orc_density(double d, double beta) { return density(d, beta); }
double orc_density_deriv(double d, double beta) { return density_deriv(d, beta); }

// Trilinear query of all channels at points x (n,3): sdf (n), rgb (n,3), valid (n).
void orc_query(void* gp, const double* x, int64_t n, double* sdf, double* rgb, uint8_t* valid) {
    Grid* g = (Grid*)gp;
    for (int64_t i = 0; i < n; ++i) {
        Stencil s = stencil_at(*g, x + 3 * i);
        valid[i] = s.valid;
        double dd = 0, c[3] = {0, 0, 0};
        if (s.valid)
            for (int e = 0; e < 8; ++e) {
                dd += s.r[e] * g->sdf[s.lin[e]];
                for (int a = 0; a < 3; ++a) c[a] += s.r[e] * g->rgb[s.lin[e] * 3 + a];
            }
        sdf[i] = dd;
        for (int a = 0; a < 3; ++a) rgb[i * 3 + a] = c[a];
    }
}

// SDF and its gradient at points x (n,3) in one pass (Eq. 16-17):
//   f(x) = sum_i r(x, x_i) theta_d(x_i),  grad_x f(x) = sum_i grad_x r(x, x_i) theta_d(x_i).
// Invalid points (a grid point unallocated) get valid = 0 and zeros.
void orc_query_grad(void* gp, const double* x, int64_t n, double* sdf, double* grad, uint8_t* valid) {
    Grid* g = (Grid*)gp;
    for (int64_t i = 0; i < n; ++i) {
        Stencil s = stencil_at(*g, x + 3 * i);
        valid[i] = s.valid;
        double f = 0.0, gr[3] = {0.0, 0.0, 0.0};
        if (s.valid)
            for (int e = 0; e < 8; ++e) {
                double r, dr[3];
                corner_weight_grad(s, g->vs, e, &r, dr);
                const double th = g->sdf[s.lin[e]];
                f += r * th;
                for (int a = 0; a < 3; ++a) gr[a] += dr[a] * th;
            }
        sdf[i] = f;
        for (int a = 0; a < 3; ++a) grad[3 * i + a] = gr[a];
    }
}

// CRF losses (Sec. 3.5.3, Eq. 22: "L_prop = D_f(x_prop || Q(x_prop))"), read as the divergence between each
// property at surface points x_i and its CRF message-passed value, the latter a fixed target:
//   prop 0 (labels):  (lambda/n) sum_i KL(Q_i || softmax(s(x_i))),  s the trilinear logits;
//                     dL/ds_i = (lambda/n) (softmax(s_i) - Q_i)   (Q_i sums to one)
//   prop 1 (colour):  (lambda/n) sum_i |c(x_i) - t_i|^2;           dL/dc_i = 2 (lambda/n) (c_i - t_i)
//   prop 2 (normal):  (lambda/n) sum_i |grad f(x_i) - t_i|^2;      dL/dgrad f_i = 2 (lambda/n) (grad f_i - t_i)
// each scattered onto the stored values through the trilinear weights (through their x-gradients for the
// normal).  Invalid points contribute 0.  Gradients are ADDED to g [N][512][channels]; returns L.
double orc_crf_loss(void* gp, int prop, const double* x, int64_t n, const double* target, double lambda,
                    double* g_out, double* terms) {
    Grid* g = (Grid*)gp;
    const int ns = g->n_sem;
    const int ch = prop == 0 ? ns : 3;
    double L = 0.0;
    const double k = lambda / (double)n;
    for (int64_t i = 0; i < n; ++i) {
        Stencil st = stencil_at(*g, x + 3 * i);
        double term = 0.0;
        if (st.valid) {
            const double* t = target + (int64_t)ch * i;
            std::vector<double> gp_(ch, 0.0);  // dL/d(property at x_i)
            if (prop == 0) {
                std::vector<double> s(ns, 0.0);
                for (int e = 0; e < 8; ++e)
                    for (int c = 0; c < ns; ++c) s[c] += st.r[e] * g->sem[st.lin[e] * ns + c];
                double mx = -1e300;
                for (int c = 0; c < ns; ++c) mx = std::max(mx, s[c]);
                double z = 0.0;
                for (int c = 0; c < ns; ++c) z += std::exp(s[c] - mx);
                for (int c = 0; c < ns; ++c) {
                    const double logp = s[c] - mx - std::log(z);
                    if (t[c] > 0.0) term += k * t[c] * (std::log(t[c]) - logp);
                    gp_[c] = k * (std::exp(logp) - t[c]);
                }
            } else if (prop == 1) {
                for (int c = 0; c < 3; ++c) {
                    double v = 0.0;
                    for (int e = 0; e < 8; ++e) v += st.r[e] * g->rgb[st.lin[e] * 3 + c];
                    term += k * (v - t[c]) * (v - t[c]);
                    gp_[c] = 2.0 * k * (v - t[c]);
                }
            } else {
                double gf[3] = {0.0, 0.0, 0.0};
                for (int e = 0; e < 8; ++e) {
                    double r, dr[3];
                    corner_weight_grad(st, g->vs, e, &r, dr);
                    for (int a = 0; a < 3; ++a) gf[a] += dr[a] * g->sdf[st.lin[e]];
                }
                for (int a = 0; a < 3; ++a) {
                    term += k * (gf[a] - t[a]) * (gf[a] - t[a]);
                    gp_[a] = 2.0 * k * (gf[a] - t[a]);
                }
            }
            for (int e = 0; e < 8; ++e) {
                if (prop == 2) {
                    double r, dr[3];
                    corner_weight_grad(st, g->vs, e, &r, dr);
                    g_out[st.lin[e]] += gp_[0] * dr[0] + gp_[1] * dr[1] + gp_[2] * dr[2];
                } else {
                    for (int c = 0; c < ch; ++c) g_out[st.lin[e] * ch + c] += st.r[e] * gp_[c];
                }
            }
        }
        if (terms) terms[i] = term;
        L += term;
    }
    return L;
}

// Eikonal regularisation (Sec. 3.5.3): L = (lambda / n) * sum over the n points of (|grad f(x)| - 1)^2, invalid
// points contributing 0.  Its gradient with respect to the stored SDF values,
//   dL/dtheta_d(x_i) = (lambda / n) * 2 (|grad f| - 1) * (grad f / |grad f|) . grad_x r(x, x_i),
// is added into g_sdf [N*512].  Where |grad f| < 1e-4 (a flat, e.g. truncated, region) the direction of grad f is
// undefined and the gradient is taken as 0.  Per-point terms go to terms (n) if given.
double orc_eikonal(void* gp, const double* x, int64_t n, double lambda, double* g_sdf, double* terms) {
    Grid* g = (Grid*)gp;
    double L = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double f, gr[3];
        uint8_t ok;
        orc_query_grad(gp, x + 3 * i, 1, &f, gr, &ok);
        double term = 0.0;
        if (ok) {
            const double norm = std::sqrt(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
            term = lambda / (double)n * (norm - 1.0) * (norm - 1.0);
            if (norm >= 1e-4) {
                const double c = lambda / (double)n * 2.0 * (norm - 1.0) / norm;
                Stencil s = stencil_at(*g, x + 3 * i);
                for (int e = 0; e < 8; ++e) {
                    double r, dr[3];
                    corner_weight_grad(s, g->vs, e, &r, dr);
                    g_sdf[s.lin[e]] += c * (gr[0] * dr[0] + gr[1] * dr[1] + gr[2] * dr[2]);
                }
            }
        }
        if (terms) terms[i] = term;
        L += term;
    }
    return L;
}

// Samples of ray i when the caller fixes them (g_S non-NULL): S = g_S[i], t_k = g_t[i][k], cells g_cell[i][k][3].
bool given_of(const double* g_S, const float* g_t, const int32_t* g_cell, int64_t i, int N, Given* gv) {
    if (!g_S) return false;
    gv->S = g_S[i];
    gv->t = g_t + i * N;
    gv->cell = g_cell + i * N * 3;
    return true;
}

// Forward render of n rays (ray i uses hash id ray_id0 + i).  diag[i] = {S, n_valid, degenerate, T_N}.
// g_S, g_t, g_cell: NULL, or the samples of every ray fixed by the caller (see Given).
void orc_render(void* gp, const float* rays, int64_t n, int N, uint32_t seed, uint32_t ray_id0, int stratified,
                const double* bg, double* rgb, double* depth, double* opac, double* sem, double* diag,
                double* normal, const double* g_S, const float* g_t, const int32_t* g_cell) {
    Grid* g = (Grid*)gp;
    for (int64_t i = 0; i < n; ++i) {
        Given gv;
        const bool given = given_of(g_S, g_t, g_cell, i, N, &gv);
        RayResult R = render_ray(*g, rays + 8 * i, N, seed, ray_id0 + (uint32_t)i, stratified, bg,
                                 given ? &gv : nullptr);
        for (int c = 0; c < 3; ++c) rgb[i * 3 + c] = R.C[c];
        if (normal)
            for (int a = 0; a < 3; ++a) normal[i * 3 + a] = R.Nrm[a];
        depth[i] = R.D;
        opac[i] = R.O;
        if (sem)
            for (int c = 0; c < g->n_sem; ++c) sem[i * g->n_sem + c] = R.sem[c];
        if (diag) {
            diag[i * 4 + 0] = R.S;
            diag[i * 4 + 1] = R.n_valid;
            diag[i * 4 + 2] = R.degenerate ? 1.0 : 0.0;
            diag[i * 4 + 3] = R.TN;
        }
    }
}

// Per-sample trace of one ray: out[k] = {s, t, delta, valid, d, sigma, T, w}.
int orc_trace(void* gp, const float* ray, int N, uint32_t seed, uint32_t ray_id, int stratified, double* out) {
    Grid* g = (Grid*)gp;
    double bg[3] = {0, 0, 0};
    RayResult R = render_ray(*g, ray, N, seed, ray_id, stratified, bg);
    for (int k = 0; k < (int)R.smp.size(); ++k) {
        const Sample& s = R.smp[k];
        double row[8] = {s.s, s.t, s.delta, s.valid ? 1.0 : 0.0, s.d, s.sigma, s.T, s.w};
        std::memcpy(out + 8 * k, row, sizeof(row));
    }
    return (int)R.smp.size();
}

// Backward: accumulates dL/dtheta (+=) for
//   L = sum_i g_rgb_i.C_i + g_depth_i D_i + g_opac_i O_i + g_sem_i.Sem_i (+ g_normal_i . N_i)
// with N_i = sum_k w_k grad f(x_k) the rendered normal of Eq. 14 (its grad f part adds
// w_k g_normal . grad_x r(x_k, x_e) to the SDF of each corner e),
// and, if grad_beta is given, dL/dbeta per ray (grad_beta[i] = sum_k dL/dtau_k delta_k dsigma_k/dbeta, the
// Laplace scale beta as a parameter as in VolSDF).
// Derivation of Eq. 15 w.r.t. tau_k = sigma_k delta_k (T_k = exp(-sum_{j<k} tau_j)):
//   dL/dtau_k = T_{k+1} v_k - sum_{j>k} w_j v_j - T_N (g_rgb . bg),
//   v_k = g_rgb.c_k + g_depth t_k + g_opac + g_sem.s_k (+ g_normal . grad f(x_k))
//   dL/dd_k   = delta_k sigma'(d_k) dL/dtau_k ;  dL/dc_k = w_k g_rgb ;  dL/ds_k = w_k g_sem
// and the trilinear weights r_e scatter each onto the 8 grid points (Sec. 3.5.2).
void orc_render_backward(void* gp, const float* rays, int64_t n, int N, uint32_t seed, uint32_t ray_id0,
                         int stratified, const double* bg, const double* g_rgb, const double* g_depth,
                         const double* g_opac, const double* g_sem, double* grad_sdf, double* grad_rgb,
                         double* grad_sem, double* grad_beta, const double* g_normal, const double* g_S,
                         const float* g_t, const int32_t* g_cell) {
    Grid* g = (Grid*)gp;
    const int ns = g->n_sem;
    for (int64_t i = 0; i < n; ++i) {
        if (grad_beta) grad_beta[i] = 0.0;
        Given gv;
        const bool given = given_of(g_S, g_t, g_cell, i, N, &gv);
        RayResult R = render_ray(*g, rays + 8 * i, N, seed, ray_id0 + (uint32_t)i, stratified, bg,
                                 given ? &gv : nullptr);
        if (R.smp.empty()) continue;
        const double* gc = g_rgb + 3 * i;
        double gd = g_depth ? g_depth[i] : 0.0, go = g_opac ? g_opac[i] : 0.0;
        const double* gs = (ns && g_sem) ? g_sem + (int64_t)ns * i : nullptr;
        std::vector<double> v(N);
        for (int k = 0; k < N; ++k) {
            const Sample& s = R.smp[k];
            double vk = gd * s.t + go;
            for (int c = 0; c < 3; ++c) vk += gc[c] * s.c[c];
            if (g_normal)
                for (int a = 0; a < 3; ++a) vk += g_normal[3 * i + a] * s.gf[a];
            if (gs)
                for (int c = 0; c < ns; ++c) vk += gs[c] * s.sem[c];
            v[k] = vk;
        }
        double ubg = gc[0] * bg[0] + gc[1] * bg[1] + gc[2] * bg[2];
        double suffix = 0.0;  // sum_{j>k} w_j v_j
        for (int k = N - 1; k >= 0; --k) {
            const Sample& s = R.smp[k];
            double dtau = s.T * std::exp(-s.tau) * v[k] - suffix - R.TN * ubg;
            suffix += s.w * v[k];
            if (!s.valid) continue;
            double dd = s.delta * density_deriv(s.d, g->beta) * dtau;
            if (grad_beta) grad_beta[i] += s.delta * density_dbeta(s.d, g->beta) * dtau;
            for (int e = 0; e < 8; ++e) {
                int64_t li = s.st.lin[e];
                double r = s.st.r[e];
                grad_sdf[li] += r * dd;
                if (g_normal) {
                    double rr, dr[3];
                    corner_weight_grad(s.st, g->vs, e, &rr, dr);
                    const double* gn = g_normal + 3 * i;
                    grad_sdf[li] += s.w * (gn[0] * dr[0] + gn[1] * dr[1] + gn[2] * dr[2]);
                }
                for (int c = 0; c < 3; ++c) grad_rgb[li * 3 + c] += r * s.w * gc[c];
                if (gs)
                    for (int c = 0; c < ns; ++c) grad_sem[li * ns + c] += r * s.w * gs[c];
            }
        }
    }
}

// Distinct voxels and blocks read by each ray's valid-sample stencils (algorithmic byte count).
void orc_count_touched(void* gp, const float* rays, int64_t n, int N, uint32_t seed, uint32_t ray_id0,
                       int stratified, int64_t* voxels, int64_t* blocks) {
    Grid* g = (Grid*)gp;
    double bg[3] = {0, 0, 0};
    for (int64_t i = 0; i < n; ++i) {
        RayResult R = render_ray(*g, rays + 8 * i, N, seed, ray_id0 + (uint32_t)i, stratified, bg);
        std::set<int64_t> vx, bl;
        for (const Sample& s : R.smp)
            if (s.valid)
                for (int e = 0; e < 8; ++e) {
                    vx.insert(s.st.lin[e]);
                    bl.insert(s.st.blk[e]);
                }
        voxels[i] = (int64_t)vx.size();
        blocks[i] = (int64_t)bl.size();
    }
}

// Rendering losses (Eq. 12-13 as configured): L1 colour (mean over rays and channels), lam_d * L1 depth
// (mean over rays, scale a = 1, shift b = 0), lam_s * squared L2 of semantic logits (mean over rays).
// Writes the gradient seeds and returns the loss.  sign(0) = 0.
double orc_loss(int64_t n, int n_sem, const double* rgb, const double* depth, const double* sem, const double* t_rgb,
                const double* t_depth, const double* t_sem, double lam_d, double lam_s, double* g_rgb,
                double* g_depth, double* g_sem) {
    double L = 0.0;
    auto sgn = [](double x) { return (double)((x > 0) - (x < 0)); };
    for (int64_t i = 0; i < n; ++i) {
        for (int c = 0; c < 3; ++c) {
            double e = rgb[i * 3 + c] - t_rgb[i * 3 + c];
            L += std::fabs(e) / (3.0 * n);
            g_rgb[i * 3 + c] = sgn(e) / (3.0 * n);
        }
        double e = depth[i] - t_depth[i];
        L += lam_d * std::fabs(e) / n;
        g_depth[i] = lam_d * sgn(e) / n;
        for (int c = 0; c < n_sem; ++c) {
            double es = sem[i * n_sem + c] - t_sem[i * n_sem + c];
            L += lam_s * es * es / n;
            g_sem[i * n_sem + c] = 2.0 * lam_s * es / n;
        }
    }
    return L;
}

// Normal loss (Eq. 14), L1 per component like the colour loss: L = (lambda / (3n)) sum_i |N_i - N^_i|_1 between
// the rendered normals N and the target normals N^ (both world frame, N unnormalised), with
// dL/dN = lambda sign(N - N^) / (3n), sign(0) = 0.  Returns L.
double orc_loss_normal(int64_t n, const double* N, const double* Nt, double lambda, double* g_normal) {
    double L = 0.0;
    for (int64_t i = 0; i < 3 * n; ++i) {
        const double e = N[i] - Nt[i];
        L += lambda * std::fabs(e) / (3.0 * n);
        g_normal[i] = lambda * (double)((e > 0.0) - (e < 0.0)) / (3.0 * n);
    }
    return L;
}

// Scale- and shift-invariant depth loss (Eq. 13, MiDaS-style alignment): (a, b) = argmin sum_i (a t_i + b - D_i)^2
// over the batch (t = target depth, D = rendered depth), solved by the 2x2 normal equations; where the targets do
// not vary the scale is undetermined and a = 1, b = mean(D - t).  L = (lambda / n) sum_i (D_i - a t_i - b)^2.
// At the optimum dL/da = dL/db = 0, so dL/dD_i is the partial derivative 2 lambda (D_i - a t_i - b) / n
// (written to g_depth).  Returns L; ab receives (a, b).
double orc_depth_ssi(int64_t n, const double* D, const double* t, double lambda, double* g_depth, double* ab) {
    double st = 0, sd = 0, stt = 0, std_ = 0;
    for (int64_t i = 0; i < n; ++i) {
        st += t[i];
        sd += D[i];
        stt += t[i] * t[i];
        std_ += t[i] * D[i];
    }
    const double nn = (double)n;
    const double det = nn * stt - st * st;
    double a, b;
    if (n > 0 && det > 1e-12 * nn * stt) {
        a = (nn * std_ - st * sd) / det;
        b = (sd - a * st) / nn;
    } else {
        a = 1.0;
        b = n > 0 ? (sd - st) / nn : 0.0;
    }
    double L = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double r = D[i] - a * t[i] - b;
        L += lambda * r * r / nn;
        g_depth[i] = 2.0 * lambda * r / nn;
    }
    ab[0] = a;
    ab[1] = b;
    return L;
}

// Adam (Kingma & Ba) with bias correction, step = 1, 2, ...; the gradient is zeroed afterwards.
void orc_adam(double* theta, double* grad, double* m, double* v, int64_t n, double lr, double b1, double b2,
              double eps, int step) {
    double c1 = 1.0 - std::pow(b1, step), c2 = 1.0 - std::pow(b2, step);
    for (int64_t i = 0; i < n; ++i) {
        double gi = grad[i];
        m[i] = b1 * m[i] + (1.0 - b1) * gi;
        v[i] = b2 * v[i] + (1.0 - b2) * gi * gi;
        double mh = m[i] / c1, vh = v[i] / c2;
        theta[i] -= lr * mh / (std::sqrt(vh) + eps);
        grad[i] = 0.0;
    }
}

// RMSProp as the paper states for refinement (Sec. 3.5.4): v = a v + (1-a) g^2, theta -= lr g / (sqrt(v) + eps).
void orc_rmsprop(double* theta, double* grad, double* v, int64_t n, double lr, double alpha, double eps) {
    for (int64_t i = 0; i < n; ++i) {
        double gi = grad[i];
        v[i] = alpha * v[i] + (1.0 - alpha) * gi * gi;
        theta[i] -= lr * gi / (std::sqrt(v[i]) + eps);
        grad[i] = 0.0;
    }
}

// ------------------------------ fusion -------------------------------------
// Volumetric fusion of depth, colour and semantic frames into the allocated
// voxels (Sec. 3.4.2, Eq. 9-11; the supplement's truncation psi).  Voxel v of
// block b sits at x = (8b + l) * vs.  Its association with frame i (camera to
// world R_i, t_i; pinhole fx, fy, cx, cy) is decided in FP32 with this order
// and no fused multiply-add, so that any FP32 implementation of the same
// order takes the same integer decisions:
//   x_a = (float)(8 b_a + l_a) * vs                       per axis a
//   e_a = x_a - t_a;  c_j = (R_0j e_0 + R_1j e_1) + R_2j e_2   (c = R^T (x - t))
//   kept only if c_2 > 0;  r = 1 / c_2;  pu = fx * (c_0 * r) + cx,  pv = fy * (c_1 * r) + cy
//   pixel (floor(pu), floor(pv)) inside the image, its depth D finite and > 0
//   o = D - c_2 (the SDF seen from view i, positive in front of the surface)
//   kept only if o >= -mu (farther behind the observed surface is occlusion)
//   psi = min(o, mu)
// The least-squares problems of Eq. 9-11 have the averages over the kept
// associations as solutions: theta_d = mean psi, theta_c = mean pixel colour,
// s* = mean pixel logits and theta_s = s* / |s*|.  weight = number of kept
// associations; a voxel with none keeps zeros.  Sums run in FP64.
void orc_fuse(const int32_t* keys, int64_t N, float vs, int F, int H, int W, const float* depth, const float* rgb,
              const float* sem, int n_sem, const float* K, const float* T, float mu, double* sdf, double* col,
              double* logit, double* weight) {
    for (int64_t b = 0; b < N; ++b)
        for (int l = 0; l < 512; ++l) {
            const int lc[3] = {l & 7, (l >> 3) & 7, l >> 6};
            float x[3];
            for (int a = 0; a < 3; ++a) x[a] = (float)(8 * keys[3 * b + a] + lc[a]) * vs;
            double n = 0.0, sd = 0.0, sc[3] = {0.0, 0.0, 0.0};
            std::vector<double> ss(n_sem > 0 ? n_sem : 1, 0.0);
            for (int i = 0; i < F; ++i) {
                const float* R = T + 12 * i;
                const float* k = K + 4 * i;
                float e[3];
                for (int a = 0; a < 3; ++a) e[a] = x[a] - R[a * 4 + 3];
                float c[3];
                for (int j = 0; j < 3; ++j) {
                    float p0 = R[0 * 4 + j] * e[0];
                    float p1 = R[1 * 4 + j] * e[1];
                    float p2 = R[2 * 4 + j] * e[2];
                    c[j] = (p0 + p1) + p2;
                }
                if (!(c[2] > 0.0f)) continue;
                const float r = 1.0f / c[2];
                float pu = k[0] * (c[0] * r) + k[2];
                float pv = k[1] * (c[1] * r) + k[3];
                float fu = std::floor(pu), fv = std::floor(pv);
                if (!(fu >= 0.0f && fu < (float)W && fv >= 0.0f && fv < (float)H)) continue;
                const int64_t pix = (int64_t)i * H * W + (int64_t)fv * W + (int64_t)fu;
                float D = depth[pix];
                if (!(std::isfinite(D) && D > 0.0f)) continue;
                float o = D - c[2];
                if (!(o >= -mu)) continue;
                float psi = std::min(o, mu);
                n += 1.0;
                sd += (double)psi;
                if (rgb)
                    for (int q = 0; q < 3; ++q) sc[q] += (double)rgb[3 * pix + q];
                if (sem)
                    for (int q = 0; q < n_sem; ++q) ss[q] += (double)sem[(int64_t)n_sem * pix + q];
            }
            const int64_t vi = b * 512 + l;
            weight[vi] = n;
            sdf[vi] = n > 0 ? sd / n : 0.0;
            for (int q = 0; q < 3; ++q) col[3 * vi + q] = n > 0 ? sc[q] / n : 0.0;
            if (sem && n_sem > 0) {
                double nn = 0.0;
                for (int q = 0; q < n_sem; ++q) nn += (ss[q] / n) * (ss[q] / n);
                nn = std::sqrt(nn);
                for (int q = 0; q < n_sem; ++q)
                    logit[(int64_t)n_sem * vi + q] = (n > 0 && nn > 0.0) ? (ss[q] / n) / nn : 0.0;
            }
        }
}

// ------------------------ permutohedral lattice ------------------------------
// Gaussian message passing of the continuous CRF (Sec. 3.5.3, Eq. 19-22) through the permutohedral lattice
// (Adams, Baek and Davis, Eurographics 2010), written from its definition:
//  * elevation: a d-dimensional (already scaled) feature p goes to x = s sum_i p_i u_i on the hyperplane
//    H_d = {x in R^(d+1): sum x = 0}, u_i = (1, .., 1, -i, 0, .., 0) / sqrt(i (i + 1)) (i ones), an orthonormal
//    basis of H_d, s = (d + 1) sqrt(2/3);
//  * enclosing simplex (an integer decision, taken in FP32 in a fixed order like the activation's quantisation):
//    the nearest remainder-0 lattice point r (coordinates multiples of d + 1, sum 0) found by
//    rounding each coordinate and then moving the coordinates with the most extreme residuals by d + 1 until the
//    sum is 0; the residual x - r ranked in decreasing order gives the simplex vertices r + c_j, j = 0..d, with
//    c_j = j on the coordinates of rank < d + 1 - j and j - (d + 1) on the others;
//  * barycentric weights (real-valued, FP64): the affine combination of the d + 1 vertices equal to the point
//    elevated in FP64, by a dense linear solve;
//  * splat: every point adds weight x value to its d + 1 vertices;
//  * blur: along each of the d + 1 lattice directions o_k (d on coordinate k, -1 on the others), in order,
//    v <- (v[- o_k] + 2 v + v[+ o_k]) / 4 over the splatted lattice points (absent neighbours are 0);
//  * slice: every point reads the barycentric combination of its vertices.
// The filter output is slice(blur(splat(v))); the normalised filter divides it by the same filter of ones.

struct LatticeSimplex {
    std::vector<std::vector<int64_t>> vert;  // d + 1 vertices, d + 1 coordinates each
    std::vector<double> bary;                // d + 1 weights
};

// Solves the n x n system A y = b (row-major A) by Gaussian elimination with partial pivoting, in FP64.
std::vector<double> solve_dense(std::vector<double> A, std::vector<double> b, int n) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)piv * n + c])) piv = r;
        if (piv != c) {
            for (int k = 0; k < n; ++k) std::swap(A[(size_t)c * n + k], A[(size_t)piv * n + k]);
            std::swap(b[c], b[piv]);
        }
        for (int r = c + 1; r < n; ++r) {
            const double f = A[(size_t)r * n + c] / A[(size_t)c * n + c];
            if (f == 0.0) continue;
            for (int k = c; k < n; ++k) A[(size_t)r * n + k] -= f * A[(size_t)c * n + k];
            b[r] -= f * b[c];
        }
    }
    std::vector<double> y(n);
    for (int r = n - 1; r >= 0; --r) {
        double acc = b[r];
        for (int k = r + 1; k < n; ++k) acc -= A[(size_t)r * n + k] * y[k];
        y[r] = acc / A[(size_t)r * n + r];
    }
    return y;
}

LatticeSimplex lattice_simplex(const double* pd, int d) {
    const int d1 = d + 1;
    // (1) Which simplex: an integer decision, taken in FP32 with this exact order (no fused multiply-add), so
    // that any FP32 evaluation of the same order finds the same lattice points.  Elevation first.
    std::vector<float> x(d1, 0.0f);
    const float sc = (float)d1 * std::sqrt(2.0f / 3.0f);
    for (int i = 1; i <= d; ++i) {
        const float f = (sc * (float)pd[i - 1]) / std::sqrt((float)(i * (i + 1)));
        for (int k = 0; k < i; ++k) x[k] += f;
        x[i] -= (float)i * f;
    }
    // The nearest remainder-0 point: each coordinate rounded to the nearest multiple of d + 1 (half away from
    // zero); if the rounded coordinates do not sum to 0, the |excess| coordinates whose residual x - r points
    // the other way the most are moved by d + 1 towards x.  Residual order: decreasing, ties by coordinate index.
    std::vector<int64_t> r(d1);
    int64_t excess = 0;  // sum of r / (d + 1)
    std::vector<float> res(d1);
    for (int k = 0; k < d1; ++k) {
        const int64_t q = (int64_t)std::llround(x[k] / (float)d1);
        r[k] = q * d1;
        excess += q;
        res[k] = x[k] - (float)r[k];
    }
    std::vector<int> order(d1);
    for (int k = 0; k < d1; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return res[a] > res[b]; });
    // Moving a coordinate down by d + 1 raises its residual by d + 1, above every other residual (all lie within
    // (d + 1) / 2 of 0), so it goes to the front of the order; moving one up sends it to the back.  Their
    // relative order is kept.
    std::vector<int> final_order;
    if (excess > 0) {  // too high: lower the coordinates with the smallest residuals
        for (int m = d1 - (int)excess; m < d1; ++m) {
            r[order[m]] -= d1;
            final_order.push_back(order[m]);
        }
        for (int m = 0; m < d1 - (int)excess; ++m) final_order.push_back(order[m]);
    } else if (excess < 0) {  // too low: raise the coordinates with the largest residuals
        for (int m = (int)(-excess); m < d1; ++m) final_order.push_back(order[m]);
        for (int m = 0; m < (int)(-excess); ++m) {
            r[order[m]] += d1;
            final_order.push_back(order[m]);
        }
    } else {
        final_order = order;
    }
    std::vector<int> rank(d1);
    for (int m = 0; m < d1; ++m) rank[final_order[m]] = m;
    // (2) The simplex's vertices, from the definition: v_j = r + c_j, where the canonical offset c_j is j on
    // the d + 1 - j coordinates of highest residual rank and j - (d + 1) on the others.
    LatticeSimplex S;
    S.vert.assign(d1, std::vector<int64_t>(d1));
    for (int j = 0; j < d1; ++j)
        for (int k = 0; k < d1; ++k) S.vert[j][k] = r[k] + (rank[k] < d1 - j ? j : j - d1);
    // (3) Barycentric weights, in FP64: the affine combination of the vertices that reproduces the elevated
    // point (elevated again in FP64): sum_j b_j v_j = x, sum_j b_j = 1 (d coordinates + the affine row; the last
    // coordinate follows, since every point involved sums to 0).
    std::vector<double> xe(d1, 0.0);
    const double scd = (double)d1 * std::sqrt(2.0 / 3.0);
    for (int i = 1; i <= d; ++i) {
        const double f = scd * pd[i - 1] / std::sqrt((double)i * (double)(i + 1));
        for (int k = 0; k < i; ++k) xe[k] += f;
        xe[i] -= (double)i * f;
    }
    std::vector<double> A((size_t)d1 * d1), rhs(d1);
    for (int k = 0; k < d; ++k) {
        for (int j = 0; j < d1; ++j) A[(size_t)k * d1 + j] = (double)S.vert[j][k];
        rhs[k] = xe[k];
    }
    for (int j = 0; j < d1; ++j) A[(size_t)d * d1 + j] = 1.0;
    rhs[d] = 1.0;
    S.bary = solve_dense(A, rhs, d1);
    return S;
}

// The simplex of one feature: vert [(d+1) x (d+1)] and bary [d+1].
void orc_lattice_simplex(const double* p, int d, int64_t* vert, double* bary) {
    LatticeSimplex S = lattice_simplex(p, d);
    for (int j = 0; j <= d; ++j) {
        bary[j] = S.bary[j];
        for (int k = 0; k <= d; ++k) vert[j * (d + 1) + k] = S.vert[j][k];
    }
}

// out [n][c] = slice(blur(splat(val))) at features pos [n][d]; normalised by the filter of ones if normalize.
// Returns the number of lattice points.
int64_t orc_lattice_filter(int64_t n, int d, const double* pos, int c, const double* val, double* out,
                           int normalize) {
    const int d1 = d + 1;
    const int cc = c + 1;  // channels + the homogeneous one
    std::map<std::vector<int64_t>, int64_t> index;
    std::vector<LatticeSimplex> simp(n);
    std::vector<std::vector<int64_t>> vid(n, std::vector<int64_t>(d1));
    std::vector<std::vector<int64_t>> keys;
    for (int64_t i = 0; i < n; ++i) {
        simp[i] = lattice_simplex(pos + (int64_t)d * i, d);
        for (int j = 0; j < d1; ++j) {
            auto it = index.find(simp[i].vert[j]);
            if (it == index.end()) {
                it = index.emplace(simp[i].vert[j], (int64_t)keys.size()).first;
                keys.push_back(simp[i].vert[j]);
            }
            vid[i][j] = it->second;
        }
    }
    const int64_t M = (int64_t)keys.size();
    std::vector<double> v((size_t)M * cc, 0.0), w((size_t)M * cc, 0.0);
    for (int64_t i = 0; i < n; ++i)
        for (int j = 0; j < d1; ++j) {
            const double b = simp[i].bary[j];
            for (int q = 0; q < c; ++q) v[(size_t)vid[i][j] * cc + q] += b * val[(int64_t)c * i + q];
            v[(size_t)vid[i][j] * cc + c] += b;
        }
    for (int dir = 0; dir < d1; ++dir) {
        for (int64_t m = 0; m < M; ++m) {
            std::vector<int64_t> kp = keys[m], km = keys[m];
            for (int k = 0; k < d1; ++k) {
                const int64_t o = k == dir ? d : -1;
                kp[k] += o;
                km[k] -= o;
            }
            auto ip = index.find(kp), im = index.find(km);
            for (int q = 0; q < cc; ++q) {
                double s2 = 2.0 * v[(size_t)m * cc + q];
                if (ip != index.end()) s2 += v[(size_t)ip->second * cc + q];
                if (im != index.end()) s2 += v[(size_t)im->second * cc + q];
                w[(size_t)m * cc + q] = 0.25 * s2;
            }
        }
        std::swap(v, w);
    }
    for (int64_t i = 0; i < n; ++i) {
        std::vector<double> o(cc, 0.0);
        for (int j = 0; j < d1; ++j)
            for (int q = 0; q < cc; ++q) o[q] += simp[i].bary[j] * v[(size_t)vid[i][j] * cc + q];
        for (int q = 0; q < c; ++q) out[(int64_t)c * i + q] = normalize ? o[q] / o[c] : o[q];
    }
    return M;
}

// One mean-field update of the label distribution with a Potts compatibility (Eq. 22; Krahenbuhl and Koltun
// 2011): with F the lattice filter above (not normalised), Qt = F(Q) - Q (the message without the node itself),
//   E_i(l) = U_i(l) + w (sum_l' Qt_i(l') - Qt_i(l)),   Q_i^+ = softmax(-E_i).
void orc_crf_meanfield(int64_t n, int d, const double* pos, int L, const double* unary, const double* Q, double w,
                       double* Qout) {
    std::vector<double> FQ((size_t)n * L);
    orc_lattice_filter(n, d, pos, L, Q, FQ.data(), 0);
    for (int64_t i = 0; i < n; ++i) {
        double tot = 0.0;
        for (int l = 0; l < L; ++l) tot += FQ[(size_t)i * L + l] - Q[i * L + l];
        std::vector<double> e(L);
        double emin = 1e300;
        for (int l = 0; l < L; ++l) {
            const double qt = FQ[(size_t)i * L + l] - Q[i * L + l];
            e[l] = unary[i * L + l] + w * (tot - qt);
            emin = std::min(emin, e[l]);
        }
        double z = 0.0;
        for (int l = 0; l < L; ++l) z += std::exp(-(e[l] - emin));
        for (int l = 0; l < L; ++l) Qout[i * L + l] = std::exp(-(e[l] - emin)) / z;
    }
}

// Pinhole rays of one H x W view (serve requests): o = t, d = normalize(R * ((u+0.5-cx)/fx, (v+0.5-cy)/fy, 1)).
void orc_view_rays(int H, int W, const double* K, const double* T, float tnear, float tfar, float* rays) {
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u) {
            double dc[3] = {((double)u + 0.5 - K[2]) / K[0], ((double)v + 0.5 - K[3]) / K[1], 1.0};
            double dw[3];
            for (int a = 0; a < 3; ++a) dw[a] = T[a * 4] * dc[0] + T[a * 4 + 1] * dc[1] + T[a * 4 + 2] * dc[2];
            double nn = std::sqrt(dw[0] * dw[0] + dw[1] * dw[1] + dw[2] * dw[2]);
            float* r = rays + 8 * ((int64_t)v * W + u);
            r[0] = (float)T[3];
            r[1] = (float)T[7];
            r[2] = (float)T[11];
            r[3] = tnear;
            r[4] = (float)(dw[0] / nn);
            r[5] = (float)(dw[1] / nn);
            r[6] = (float)(dw[2] / nn);
            r[7] = tfar;
        }
}

}  // extern "C"
