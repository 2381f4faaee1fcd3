// Permutohedral-lattice Gaussian filtering (Adams, Baek and Davis 2010) on a
// hash map of lattice points: the message passing of the continuous CRF,
// Sec. 3.5.3 (Eq. 19-22), and one Potts mean-field update built on it.
//
// A d-dimensional feature p (already divided by its standard deviations) is
// elevated onto the hyperplane sum x = 0 of R^(d+1) with the orthonormal basis
// u_i = (1, .., 1, -i, 0, ..) / sqrt(i (i + 1)) scaled by (d + 1) sqrt(2/3); its
// enclosing simplex is the nearest remainder-0 lattice point plus the
// canonical simplex ordered by the ranks of the residual.  The elevation and
// the simplex search run in FP64 with round-to-nearest intrinsics in a fixed
// order, so that the set of lattice points (which decides how the blur
// propagates) is exactly what an FP64 evaluation of the same order gives;
// splat, blur and slice run in FP32.
//
// Passes (separate kernels, so no thread ever waits for another):
//   insert:   every vertex's 64-bit coordinate fingerprint claims a slot of an
//             open-addressing table (compare-and-swap); the winner stores the
//             coordinates in the slot;
//   number:   occupied slots get dense lattice indices;
//   splat:    every point recomputes its simplex, checks its vertices' full
//             coordinates against the slot (a fingerprint collision is
//             reported, never merged silently) and adds weight x value;
//   neighbours, then per direction blur: v <- (v[-o] + 2 v + v[+o]) / 4;
//   slice:    barycentric read-back (divided by the filtered ones when asked).
#include <algorithm>

#include "internal.h"

namespace sdg {
namespace {

constexpr int kMaxD = 16;      // feature dimensions
constexpr int kMaxC = 64;      // value channels
constexpr int kThreads = 256;
constexpr unsigned long long kEmpty = ~0ull;

struct Simplex {
    int r[kMaxD + 1];     // remainder-0 vertex
    int rank[kMaxD + 1];  // rank of each coordinate's residual (0 = largest)
    float b[kMaxD + 1];   // barycentric weights of vertices 0..d
};

// Elevation, nearest remainder-0 point, ranks and barycentric weights (FP64, fixed order).
__device__ __forceinline__ bool lattice_simplex(const float* p, int d, Simplex& S) {
    const int d1 = d + 1;
    double x[kMaxD + 1];
    for (int k = 0; k < d1; ++k) x[k] = 0.0;
    const double sc = __dmul_rn((double)d1, sqrt(2.0 / 3.0));
    for (int i = 1; i <= d; ++i) {
        const double f = __ddiv_rn(__dmul_rn(sc, (double)p[i - 1]), sqrt(__dmul_rn((double)i, (double)(i + 1))));
        for (int k = 0; k < i; ++k) x[k] = __dadd_rn(x[k], f);
        x[i] = __dsub_rn(x[i], __dmul_rn((double)i, f));
    }
    long long sum = 0;
    double res[kMaxD + 1];
    for (int k = 0; k < d1; ++k) {
        const double q = __ddiv_rn(x[k], (double)d1);
        if (!(fabs(q) < 1e9)) return false;  // non-finite or out of range feature
        const long long qr = llround(q);
        S.r[k] = (int)(qr * d1);
        sum += qr;
        res[k] = __dsub_rn(x[k], (double)S.r[k]);
    }
    for (int k = 0; k < d1; ++k) {
        int rk = 0;
        for (int m = 0; m < d1; ++m)
            if (res[m] > res[k] || (res[m] == res[k] && m < k)) ++rk;
        S.rank[k] = rk;
    }
    for (int k = 0; k < d1; ++k) {
        S.rank[k] += (int)sum;
        if (S.rank[k] >= d1) {
            S.rank[k] -= d1;
            S.r[k] -= d1;
        } else if (S.rank[k] < 0) {
            S.rank[k] += d1;
            S.r[k] += d1;
        }
    }
    double b[kMaxD + 2];
    for (int k = 0; k <= d1; ++k) b[k] = 0.0;
    for (int k = 0; k < d1; ++k) {
        const double v = __ddiv_rn(__dsub_rn(x[k], (double)S.r[k]), (double)d1);
        b[d - S.rank[k]] = __dadd_rn(b[d - S.rank[k]], v);
        b[d1 - S.rank[k]] = __dsub_rn(b[d1 - S.rank[k]], v);
    }
    b[0] = __dadd_rn(b[0], __dadd_rn(1.0, b[d1]));
    for (int j = 0; j < d1; ++j) S.b[j] = (float)b[j];
    return true;
}

__device__ __forceinline__ int vertex_coord(const Simplex& S, int d, int j, int k) {
    return S.r[k] + (S.rank[k] < d + 1 - j ? j : j - (d + 1));
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long h) {
    h ^= h >> 33;
    h *= 0xff51afd7ed558ccdull;
    h ^= h >> 33;
    h *= 0xc4ceb9fe1a85ec53ull;
    h ^= h >> 33;
    return h;
}

// Fingerprint of a lattice point from its first d coordinates (the last one is minus their sum).
__device__ __forceinline__ unsigned long long fingerprint(const int* c, int d) {
    unsigned long long h = 0x9e3779b97f4a7c15ull;
    for (int k = 0; k < d; ++k) h = mix64(h ^ (unsigned long long)(unsigned)c[k] ^ ((unsigned long long)k << 40));
    return h == kEmpty ? kEmpty - 1 : h;
}

struct Table {
    unsigned long long* fp;  // [cap]
    int* idx;                // [cap] lattice index of the slot
    int* skey;               // [cap][d] coordinates written by the slot's owner
    unsigned mask;
};

__device__ __forceinline__ int table_find(const Table& t, unsigned long long f) {
    unsigned s = (unsigned)f & t.mask;
    for (unsigned p = 0; p <= t.mask; ++p) {
        const unsigned long long v = t.fp[s];
        if (v == f) return (int)s;
        if (v == kEmpty) return -1;
        s = (s + 1) & t.mask;
    }
    return -1;
}

__global__ void k_lat_insert(const float* __restrict__ pos, int64_t n, int d, Table t, int* status) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        Simplex S;
        if (!lattice_simplex(pos + (int64_t)d * i, d, S)) {
            atomicOr(status, 2);
            continue;
        }
        for (int j = 0; j <= d; ++j) {
            int c[kMaxD + 1];
            for (int k = 0; k <= d; ++k) c[k] = vertex_coord(S, d, j, k);
            const unsigned long long f = fingerprint(c, d);
            unsigned s = (unsigned)f & t.mask;
            bool done = false;
            for (unsigned p = 0; p <= t.mask && !done; ++p) {
                const unsigned long long old = atomicCAS(t.fp + s, kEmpty, f);
                if (old == kEmpty) {
                    for (int k = 0; k < d; ++k) t.skey[(int64_t)s * d + k] = c[k];
                    done = true;
                } else if (old == f) {
                    done = true;
                } else {
                    s = (s + 1) & t.mask;
                }
            }
            if (!done) atomicOr(status, 1);  // table full (cannot happen at the capacity the host reserves)
        }
    }
}

__global__ void k_lat_number(Table t, int* count, int* keys, int d) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s <= (int64_t)t.mask;
         s += (int64_t)gridDim.x * blockDim.x) {
        if (t.fp[s] == kEmpty) continue;
        const int m = atomicAdd(count, 1);
        t.idx[s] = m;
        for (int k = 0; k < d; ++k) keys[(int64_t)m * d + k] = t.skey[s * d + k];
    }
}

// Splat: every point's simplex again (bit-identical), its vertices' lattice indices and weights kept for the
// slice; a vertex whose coordinates differ from its slot's is a fingerprint collision.
__global__ void k_lat_splat(const float* __restrict__ pos, const float* __restrict__ val, int64_t n, int d, int c,
                            Table t, const int* __restrict__ keys, float* __restrict__ lat, int* __restrict__ vidx,
                            float* __restrict__ vbary, int* status) {
    const int cc = c + 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        Simplex S;
        if (!lattice_simplex(pos + (int64_t)d * i, d, S)) {
            for (int j = 0; j <= d; ++j) {
                vidx[i * (d + 1) + j] = -1;
                vbary[i * (d + 1) + j] = 0.f;
            }
            continue;
        }
        for (int j = 0; j <= d; ++j) {
            int cv[kMaxD + 1];
            for (int k = 0; k <= d; ++k) cv[k] = vertex_coord(S, d, j, k);
            const int s = table_find(t, fingerprint(cv, d));
            int m = s >= 0 ? t.idx[s] : -1;
            if (m >= 0)
                for (int k = 0; k < d; ++k)
                    if (keys[(int64_t)m * d + k] != cv[k]) m = -1;
            if (m < 0) {
                atomicOr(status, 4);
                vidx[i * (d + 1) + j] = -1;
                vbary[i * (d + 1) + j] = 0.f;
                continue;
            }
            vidx[i * (d + 1) + j] = m;
            vbary[i * (d + 1) + j] = S.b[j];
            float* dst = lat + (int64_t)m * cc;
            for (int q = 0; q < c; ++q) atomicAdd(dst + q, S.b[j] * val[(int64_t)c * i + q]);
            atomicAdd(dst + c, S.b[j]);
        }
    }
}

// Neighbours of every lattice point along direction dir: key +- o, o = d on coordinate dir and -1 elsewhere.
__global__ void k_lat_neighbours(const int* __restrict__ keys, int M, int d, Table t, int* __restrict__ nb) {
    const int d1 = d + 1;
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M; m += (int64_t)gridDim.x * blockDim.x) {
        int c[kMaxD + 1];
        int last = 0;
        for (int k = 0; k < d; ++k) {
            c[k] = keys[m * d + k];
            last -= c[k];
        }
        c[d] = last;
        for (int dir = 0; dir < d1; ++dir) {
            for (int sgn = 0; sgn < 2; ++sgn) {
                int e[kMaxD + 1];
                for (int k = 0; k < d1; ++k) {
                    const int o = k == dir ? d : -1;
                    e[k] = sgn ? c[k] - o : c[k] + o;
                }
                const int s = table_find(t, fingerprint(e, d));
                int r = s >= 0 ? t.idx[s] : -1;
                if (r >= 0)
                    for (int k = 0; k < d; ++k)
                        if (keys[(int64_t)r * d + k] != e[k]) r = -1;
                nb[(m * d1 + dir) * 2 + sgn] = r;
            }
        }
    }
}

__global__ void k_lat_blur(const float* __restrict__ src, float* __restrict__ dst, const int* __restrict__ nb,
                           int M, int d, int dir, int cc) {
    const int d1 = d + 1;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)M * cc;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = e / cc;
        const int q = (int)(e - m * cc);
        const int np = nb[(m * d1 + dir) * 2], nm = nb[(m * d1 + dir) * 2 + 1];
        float s2 = 2.f * src[e];
        if (np >= 0) s2 += src[(int64_t)np * cc + q];
        if (nm >= 0) s2 += src[(int64_t)nm * cc + q];
        dst[e] = 0.25f * s2;
    }
}

__global__ void k_lat_slice(const float* __restrict__ lat, const int* __restrict__ vidx,
                            const float* __restrict__ vbary, int64_t n, int d, int c, int normalize,
                            float* __restrict__ out) {
    const int cc = c + 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float acc[kMaxC + 1];
        for (int q = 0; q < cc; ++q) acc[q] = 0.f;
        for (int j = 0; j <= d; ++j) {
            const int m = vidx[i * (d + 1) + j];
            if (m < 0) continue;
            const float b = vbary[i * (d + 1) + j];
            for (int q = 0; q < cc; ++q) acc[q] = fmaf(b, lat[(int64_t)m * cc + q], acc[q]);
        }
        for (int q = 0; q < c; ++q) out[(int64_t)c * i + q] = normalize ? acc[q] / acc[c] : acc[q];
    }
}

// Potts mean-field update: E = U + w (sum_l' Qt - Qt), Qt = F(Q) - Q; Q+ = softmax(-E).
__global__ void k_meanfield(const float* __restrict__ FQ, const float* __restrict__ U, const float* __restrict__ Q,
                            int64_t n, int L, float w, float* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float tot = 0.f;
        for (int l = 0; l < L; ++l) tot += FQ[i * L + l] - Q[i * L + l];
        float emin = 3.0e38f;
        for (int l = 0; l < L; ++l) {
            const float e = U[i * L + l] + w * (tot - (FQ[i * L + l] - Q[i * L + l]));
            emin = fminf(emin, e);
        }
        float z = 0.f;
        for (int l = 0; l < L; ++l) z += __expf(-(U[i * L + l] + w * (tot - (FQ[i * L + l] - Q[i * L + l])) - emin));
        const float iz = 1.f / z;
        for (int l = 0; l < L; ++l)
            out[i * L + l] = __expf(-(U[i * L + l] + w * (tot - (FQ[i * L + l] - Q[i * L + l])) - emin)) * iz;
    }
}

int blocks_for(int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, 148 * 32));
}

template <class T>
int grow(T** p, int64_t* cap, int64_t want, cudaStream_t s) {
    if (*cap >= want) return SDG_OK;
    if (*p) {
        SDG_CUDA_TRY(cudaStreamSynchronize(s));
        cudaFree(*p);
    }
    *p = nullptr;
    *cap = 0;
    SDG_CUDA_TRY(cudaMalloc((void**)p, sizeof(T) * (size_t)want));
    *cap = want;
    return SDG_OK;
}

uint64_t pow2_at_least(uint64_t v) {
    uint64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

}  // namespace

// Runs the lattice filter; out may alias nothing else.  n_lattice (host, may be NULL) synchronises.
int lattice_filter(sdg_grid g, int64_t n, int d, const float* pos, int c, const float* val, float* out,
                   int normalize, int64_t* n_lattice) {
    LatticeScratch& L = g->lat;
    cudaStream_t s = g->stream;
    const int d1 = d + 1, cc = c + 1;
    const int64_t nv = n * d1;  // vertex references; at most this many lattice points
    const uint64_t cap = pow2_at_least((uint64_t)std::max<int64_t>(2 * nv, 1024));
    int rc;
    if ((rc = grow(&L.fp, &L.cap_fp, (int64_t)cap, s)) || (rc = grow(&L.idx, &L.cap_idx, (int64_t)cap, s)) ||
        (rc = grow(&L.skey, &L.cap_skey, (int64_t)cap * d, s)) || (rc = grow(&L.keys, &L.cap_keys, nv * d, s)) ||
        (rc = grow(&L.vidx, &L.cap_vidx, nv, s)) || (rc = grow(&L.vbary, &L.cap_vbary, nv, s)) ||
        (rc = grow(&L.val0, &L.cap_val0, nv * cc, s)) || (rc = grow(&L.val1, &L.cap_val1, nv * cc, s)) ||
        (rc = grow(&L.nb, &L.cap_nb, nv * d1 * 2, s)) || (rc = grow(&L.counters, &L.cap_counters, (int64_t)2, s)))
        return rc;
    SDG_CUDA_TRY(cudaMemsetAsync(L.fp, 0xFF, sizeof(unsigned long long) * cap, s));
    SDG_CUDA_TRY(cudaMemsetAsync(L.counters, 0, 2 * sizeof(int), s));
    Table t{L.fp, L.idx, L.skey, (unsigned)(cap - 1)};
    int* count = L.counters;
    int* status = L.counters + 1;
    k_lat_insert<<<blocks_for(n), kThreads, 0, s>>>(pos, n, d, t, status);
    SDG_LAUNCH_CHECK("lattice insert");
    k_lat_number<<<blocks_for((int64_t)cap), kThreads, 0, s>>>(t, count, L.keys, d);
    SDG_LAUNCH_CHECK("lattice numbering");
    int h[2];
    SDG_CUDA_TRY(cudaMemcpyAsync(h, L.counters, sizeof(h), cudaMemcpyDeviceToHost, s));
    SDG_CUDA_TRY(cudaStreamSynchronize(s));  // the lattice size sizes the blur launches
    const int M = h[0];
    if (h[1] & 2) return fail(SDG_ERR_ARG, "lattice filter: non-finite or out-of-range features");
    if (h[1] & 1) return fail(SDG_ERR_CAPACITY, "lattice filter: lattice table full");
    SDG_CUDA_TRY(cudaMemsetAsync(L.val0, 0, sizeof(float) * (size_t)M * cc, s));
    k_lat_splat<<<blocks_for(n), kThreads, 0, s>>>(pos, val, n, d, c, t, L.keys, L.val0, L.vidx, L.vbary, status);
    SDG_LAUNCH_CHECK("lattice splat");
    k_lat_neighbours<<<blocks_for(M), kThreads, 0, s>>>(L.keys, M, d, t, L.nb);
    SDG_LAUNCH_CHECK("lattice neighbours");
    float* a = L.val0;
    float* b = L.val1;
    for (int dir = 0; dir < d1; ++dir) {
        k_lat_blur<<<blocks_for((int64_t)M * cc), kThreads, 0, s>>>(a, b, L.nb, M, d, dir, cc);
        SDG_LAUNCH_CHECK("lattice blur");
        std::swap(a, b);
    }
    k_lat_slice<<<blocks_for(n), kThreads, 0, s>>>(a, L.vidx, L.vbary, n, d, c, normalize, out);
    SDG_LAUNCH_CHECK("lattice slice");
    SDG_CUDA_TRY(cudaMemcpyAsync(h, L.counters, sizeof(h), cudaMemcpyDeviceToHost, s));
    SDG_CUDA_TRY(cudaStreamSynchronize(s));
    if (h[1] & 4) return fail(SDG_ERR_CUDA, "lattice filter: coordinate fingerprint collision");
    if (n_lattice) *n_lattice = M;
    return SDG_OK;
}

}  // namespace sdg

using namespace sdg;

extern "C" int sdg_lattice_filter(sdg_grid g, int64_t n, int32_t d, const float* pos, int32_t c, const float* val,
                                  float* out, int32_t normalize, int64_t* n_lattice) {
    if (!g || n < 0 || d < 1 || d > kMaxD || c < 1 || c > kMaxC || (n > 0 && (!pos || !val || !out)))
        return fail(SDG_ERR_ARG, "sdg_lattice_filter: bad argument (1 <= d <= 16, 1 <= c <= 64)");
    if (n * (d + 1) > ((int64_t)1 << 30)) return fail(SDG_ERR_ARG, "sdg_lattice_filter: at most 2^30 vertices");
    int rc = use_device(g);
    if (rc) return rc;
    if (n == 0) {
        if (n_lattice) *n_lattice = 0;
        return SDG_OK;
    }
    return lattice_filter(g, n, d, pos, c, val, out, normalize, n_lattice);
}

extern "C" int sdg_crf_meanfield(sdg_grid g, int64_t n, int32_t d, const float* pos, int32_t L, const float* unary,
                                 const float* q, float w, float* q_out) {
    if (!g || n < 0 || d < 1 || d > kMaxD || L < 1 || L > kMaxC || (n > 0 && (!pos || !unary || !q || !q_out)))
        return fail(SDG_ERR_ARG, "sdg_crf_meanfield: bad argument (1 <= d <= 16, 1 <= L <= 64)");
    if (n * (d + 1) > ((int64_t)1 << 30)) return fail(SDG_ERR_ARG, "sdg_crf_meanfield: at most 2^30 vertices");
    int rc = use_device(g);
    if (rc) return rc;
    if (n == 0) return SDG_OK;
    LatticeScratch& S = g->lat;
    if ((rc = grow(&S.fq, &S.cap_fq, n * L, g->stream))) return rc;
    if ((rc = lattice_filter(g, n, d, pos, L, q, S.fq, 0, nullptr))) return rc;
    k_meanfield<<<blocks_for(n), kThreads, 0, g->stream>>>(S.fq, unary, q, n, L, w, q_out);
    SDG_LAUNCH_CHECK("mean field");
    return SDG_OK;
}
