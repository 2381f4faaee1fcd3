// Permutohedral-lattice Gaussian filtering (Adams, Baek and Davis 2010) on a
// hash map of lattice points: the message passing of the continuous CRF,
// Sec. 3.5.3 (Eq. 19-22), and one Potts mean-field update built on it.
//
// A d-dimensional feature p (already divided by its standard deviations) is
// elevated onto the hyperplane sum x = 0 of R^(d+1) with the orthonormal basis
// u_i = (1, .., 1, -i, 0, ..) / sqrt(i (i + 1)) scaled by (d + 1) sqrt(2/3); its
// enclosing simplex is the nearest remainder-0 lattice point plus the
// canonical simplex ordered by the ranks of the residual.  The elevation and
// the simplex search run in FP32 with round-to-nearest intrinsics in a fixed
// order, so that the set of lattice points (which decides how the blur
// propagates) is exactly what any evaluation of the same order gives.
// Lattice values are rows of float4 groups (channels + the homogeneous one,
// padded to a multiple of 4): splat, blur and slice move 16-byte groups.
//
// Passes (separate kernels, so no thread ever waits for another):
//   insert:   every point's simplex (kept for the splat); every vertex's 64-bit
//             coordinate fingerprint claims a slot of an open-addressing table
//             (compare-and-swap); the winner stores the coordinates in the slot;
//   number:   occupied slots get dense lattice indices;
//   splat:    every point's stored simplex: its vertices' full coordinates
//             are checked against their slots (a fingerprint collision is
//             reported, never merged silently), then weight x value is added;
//   neighbours (both fingerprints formed incrementally from the point's),
//             then per direction blur: v <- (v[-o] + 2 v + v[+o]) / 4;
//   slice:    barycentric read-back (divided by the filtered ones when asked).
#include <algorithm>
#include <climits>

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

// Elevation, nearest remainder-0 point, ranks and barycentric weights: an integer decision, taken in FP32 with
// round-to-nearest intrinsics in a fixed order (no contraction), so any FP32 evaluation of the same order finds
// the same lattice points.
__device__ __forceinline__ bool lattice_simplex(const float* p, int d, Simplex& S) {
    const int d1 = d + 1;
    const float fd1 = (float)d1;
    float x[kMaxD + 1];
    for (int k = 0; k < d1; ++k) x[k] = 0.f;
    const float sc = __fmul_rn(fd1, __fsqrt_rn(__fdiv_rn(2.0f, 3.0f)));
    for (int i = 1; i <= d; ++i) {
        const float f = __fdiv_rn(__fmul_rn(sc, p[i - 1]), __fsqrt_rn((float)(i * (i + 1))));
        for (int k = 0; k < i; ++k) x[k] = __fadd_rn(x[k], f);
        x[i] = __fsub_rn(x[i], __fmul_rn((float)i, f));
    }
    int sum = 0;
    float res[kMaxD + 1];
    for (int k = 0; k < d1; ++k) {
        const float q = __fdiv_rn(x[k], fd1);
        if (!(fabsf(q) < 5e7f)) return false;  // non-finite, or coordinates beyond the int32 lattice keys
        const int qr = (int)roundf(q);  // half away from zero, exact in float for |q| < 5e7; 32-bit conversion
        S.r[k] = qr * d1;
        sum += qr;
        res[k] = __fsub_rn(x[k], (float)S.r[k]);
    }
    for (int k = 0; k < d1; ++k) {
        int rk = 0;
        for (int m = 0; m < d1; ++m)
            if (res[m] > res[k] || (res[m] == res[k] && m < k)) ++rk;
        S.rank[k] = rk;
    }
    for (int k = 0; k < d1; ++k) {
        S.rank[k] += sum;
        if (S.rank[k] >= d1) {
            S.rank[k] -= d1;
            S.r[k] -= d1;
        } else if (S.rank[k] < 0) {
            S.rank[k] += d1;
            S.r[k] += d1;
        }
    }
    float b[kMaxD + 2];
    for (int k = 0; k <= d1; ++k) b[k] = 0.f;
    for (int k = 0; k < d1; ++k) {
        const float v = __fdiv_rn(__fsub_rn(x[k], (float)S.r[k]), fd1);
        b[d - S.rank[k]] = __fadd_rn(b[d - S.rank[k]], v);
        b[d1 - S.rank[k]] = __fsub_rn(b[d1 - S.rank[k]], v);
    }
    b[0] = __fadd_rn(b[0], __fadd_rn(1.0f, b[d1]));
    for (int j = 0; j < d1; ++j) S.b[j] = b[j];
    return true;
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long h) {
    h ^= h >> 33;
    h *= 0xff51afd7ed558ccdull;
    h ^= h >> 33;
    h *= 0xc4ceb9fe1a85ec53ull;
    h ^= h >> 33;
    return h;
}

// Fingerprint of a lattice point from its first d coordinates (the last one is minus their sum): the linear
// form sum_k c_k P_k mod 2^64 with odd multipliers P_k, then one mixing round.  The linear form of a neighbour
// key + o is the key's plus sum_k o_k P_k, so neighbour fingerprints cost O(1).
__device__ __forceinline__ unsigned long long lin_mult(int k) {
    return mix64(0x9e3779b97f4a7c15ull * (k + 1)) | 1ull;
}

__device__ __forceinline__ unsigned long long finish(unsigned long long lin) {
    const unsigned long long h = mix64(lin ^ 0x2545f4914f6cdd1dull);
    return h == kEmpty ? kEmpty - 1 : h;
}

// A second, independent 32-bit fingerprint (other multipliers, other mixing) kept in each slot: a neighbour
// lookup accepts a slot only when both fingerprints match (a false match needs a 96-bit coincidence).
__device__ __forceinline__ unsigned long long lin_mult2(int k) {
    return mix64(0xd1b54a32d192ed03ull * (k + 7)) | 1ull;
}

__device__ __forceinline__ unsigned finish2(unsigned long long lin) {
    return (unsigned)(mix64(lin + 0x632be59bd9b4e019ull) >> 32);
}

struct Table {
    unsigned long long* fp;  // [cap]
    unsigned* fp2;           // [cap] second fingerprint, written by the slot's owner
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

// Simplex of every point (remainder-0 vertex, ranks, weights); sr[i][0] = INT_MIN marks an invalid feature.
__global__ void k_lat_simplex(const float* __restrict__ pos, int64_t n, int d, int* __restrict__ sr,
                              signed char* __restrict__ srank, float* __restrict__ vbary, int* status) {
    const int d1 = d + 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        Simplex S;
        if (!lattice_simplex(pos + (int64_t)d * i, d, S)) {
            atomicOr(status, 2);
            sr[i * d1] = INT_MIN;
            continue;
        }
        for (int k = 0; k < d1; ++k) {
            sr[i * d1 + k] = S.r[k];
            srank[i * d1 + k] = (signed char)S.rank[k];
            vbary[i * d1 + k] = S.b[k];
        }
    }
}

__device__ __forceinline__ int stored_vertex_coord(const int* sr, const signed char* srank, int64_t i, int d, int j,
                                                   int k) {
    const int d1 = d + 1;
    return sr[i * d1 + k] + (srank[i * d1 + k] < d1 - j ? j : j - d1);
}

// Insert, one thread per (point, vertex): the vertex's 64-bit coordinate fingerprint claims a slot
// (compare-and-swap); the winner writes the coordinates.  vslot receives the slot (-1: invalid feature).
__global__ void __launch_bounds__(256) k_lat_insert(int64_t n, int d, Table t, const int* __restrict__ sr,
                                                    const signed char* __restrict__ srank, int* __restrict__ vslot,
                                                    int* status) {
    __shared__ unsigned long long P[kMaxD], P2[kMaxD];
    if (threadIdx.x < kMaxD) {
        P[threadIdx.x] = lin_mult(threadIdx.x);
        P2[threadIdx.x] = lin_mult2(threadIdx.x);
    }
    __syncthreads();
    const int d1 = d + 1;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * d1; e += (int64_t)gridDim.x * blockDim.x) {
        int j;
        const int64_t i = sdg_divmod(e, d1, j);
        if (sr[i * d1] == INT_MIN) {
            vslot[e] = -1;
            continue;
        }
        int c[kMaxD + 1];
        unsigned long long lin = 0, lin2 = 0;
        for (int k = 0; k < d; ++k) {
            c[k] = stored_vertex_coord(sr, srank, i, d, j, k);
            lin += (unsigned long long)(long long)c[k] * P[k];
            lin2 += (unsigned long long)(long long)c[k] * P2[k];
        }
        const unsigned long long f = finish(lin);
        unsigned s = (unsigned)f & t.mask;
        bool done = false;
        for (unsigned p = 0; p <= t.mask && !done; ++p) {
            const unsigned long long old = atomicCAS(t.fp + s, kEmpty, f);
            if (old == kEmpty) {
                for (int k = 0; k < d; ++k) t.skey[(int64_t)s * d + k] = c[k];
                t.fp2[s] = finish2(lin2);
                done = true;
            } else if (old == f) {
                done = true;
            } else {
                s = (s + 1) & t.mask;
            }
        }
        vslot[e] = done ? (int)s : -1;
        if (!done) atomicOr(status, 1);  // table full (cannot happen at the capacity the host reserves)
    }
}

// Dense lattice indices for the occupied slots: one counter update per block and sweep (warp ballots, then a
// prefix over the block's warps).
__global__ void __launch_bounds__(256) k_lat_number(Table t, int* count, int* keys, int d) {
    __shared__ int wcount[8];
    __shared__ int wbase[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t total = (int64_t)t.mask + 1;  // a multiple of 256: every block runs the loop the same number of times
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s - threadIdx.x < total; s += stride) {
        const bool occ = s < total && t.fp[s] != kEmpty;
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, occ);
        if (lane == 0) wcount[warp] = __popc(bal);
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int w = 0; w < 8; ++w) {
                wbase[w] = tot;
                tot += wcount[w];
            }
            const int b0 = tot ? atomicAdd(count, tot) : 0;
            for (int w = 0; w < 8; ++w) wbase[w] += b0;
        }
        __syncthreads();
        if (occ) {
            const int m = wbase[warp] + __popc(bal & ((1u << lane) - 1u));
            t.idx[s] = m;
            for (int k = 0; k < d; ++k) keys[(int64_t)m * d + k] = t.skey[s * d + k];
        }
        __syncthreads();
    }
}

// Splat, one thread per (point, float4 group of channels): each vertex of the stored simplex, its coordinates
// checked against its slot's (a fingerprint collision is reported, never merged silently), then a 16-byte
// vector atomic.  Group g holds channels 4g..4g+3; channel c is the homogeneous weight, the rest is padding.
// The thread of group 0 records the vertices' lattice indices for the slice.
__global__ void __launch_bounds__(256, 8) k_lat_splat(const float* __restrict__ val, int64_t n, int d, int c, int g4, Table t,
                            const int* __restrict__ keys, const int* __restrict__ sr,
                            const signed char* __restrict__ srank, const int* __restrict__ vslot,
                            const float* __restrict__ vbary, float4* __restrict__ lat, int* __restrict__ vidx,
                            int* status) {
    const int d1 = d + 1;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * g4; e += (int64_t)gridDim.x * blockDim.x) {
        int g;
        const int64_t i = sdg_divmod(e, g4, g);
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = 4 * g + u;
            v[u] = q < c ? val[(int64_t)c * i + q] : (q == c ? 1.f : 0.f);
        }
        for (int j = 0; j < d1; ++j) {
            const int s = vslot[i * d1 + j];
            int m = s >= 0 ? t.idx[s] : -1;
            if (m >= 0)
                for (int k = 0; k < d; ++k)
                    if (keys[(int64_t)m * d + k] != stored_vertex_coord(sr, srank, i, d, j, k)) m = -1;
            if (g == 0) vidx[i * d1 + j] = m;
            if (m < 0) {
                if (s >= 0 && g == 0) atomicOr(status, 4);
                continue;
            }
            const float b = vbary[i * d1 + j];
            atomicAdd(lat + (int64_t)m * g4 + g, make_float4(b * v[0], b * v[1], b * v[2], b * v[3]));
        }
    }
}

// Neighbours of every lattice point: key +- o along each direction dir (o = d on coordinate dir, -1 elsewhere),
// one thread per (point, direction) and both signs.  Both fingerprints of a neighbour key are formed
// incrementally from the point's linear forms (multiplier tables in shared memory); a slot is accepted when both
// match.
__global__ void __launch_bounds__(256, 8) k_lat_neighbours(const int* __restrict__ keys, int M, int d, Table t,
                                                        int* __restrict__ nb) {
    __shared__ unsigned long long P[kMaxD], P2[kMaxD];
    if (threadIdx.x < kMaxD) {
        P[threadIdx.x] = lin_mult(threadIdx.x);
        P2[threadIdx.x] = lin_mult2(threadIdx.x);
    }
    __syncthreads();
    const int d1 = d + 1;
    unsigned long long sum_p = 0, sum_p2 = 0;  // sum_k<d of the multipliers
    for (int k = 0; k < d; ++k) {
        sum_p += P[k];
        sum_p2 += P2[k];
    }
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)M * d1;
         e += (int64_t)gridDim.x * blockDim.x) {
        int dir;
        const int64_t m = sdg_divmod(e, d1, dir);
        unsigned long long lin = 0, lin2 = 0;
        for (int k = 0; k < d; ++k) {
            const unsigned long long ck = (unsigned long long)(long long)keys[m * d + k];
            lin += ck * P[k];
            lin2 += ck * P2[k];
        }
        // sum_k<d o_k P_k: d on coordinate dir (when dir < d), -1 on the others
        const unsigned long long step = dir < d ? (unsigned long long)(d + 1) * P[dir] - sum_p : 0ull - sum_p;
        const unsigned long long step2 = dir < d ? (unsigned long long)(d + 1) * P2[dir] - sum_p2 : 0ull - sum_p2;
        const int sp = table_find(t, finish(lin + step)), sm = table_find(t, finish(lin - step));
        nb[e * 2] = (sp >= 0 && t.fp2[sp] == finish2(lin2 + step2)) ? t.idx[sp] : -1;
        nb[e * 2 + 1] = (sm >= 0 && t.fp2[sm] == finish2(lin2 - step2)) ? t.idx[sm] : -1;
    }
}

// One blur pass along direction dir, one thread per (lattice point, float4 group).
__global__ void k_lat_blur(const float4* __restrict__ src, float4* __restrict__ dst, const int* __restrict__ nb,
                           int M, int d, int dir, int g4) {
    const int d1 = d + 1;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)M * g4;
         e += (int64_t)gridDim.x * blockDim.x) {
        int g;
        const int64_t m = sdg_divmod(e, g4, g);
        const int2 pr = *reinterpret_cast<const int2*>(nb + (m * d1 + dir) * 2);
        const float4 a = src[e];
        float4 r = make_float4(2.f * a.x, 2.f * a.y, 2.f * a.z, 2.f * a.w);
        if (pr.x >= 0) {
            const float4 p = src[(int64_t)pr.x * g4 + g];
            r.x += p.x;
            r.y += p.y;
            r.z += p.z;
            r.w += p.w;
        }
        if (pr.y >= 0) {
            const float4 p = src[(int64_t)pr.y * g4 + g];
            r.x += p.x;
            r.y += p.y;
            r.z += p.z;
            r.w += p.w;
        }
        dst[e] = make_float4(0.25f * r.x, 0.25f * r.y, 0.25f * r.z, 0.25f * r.w);
    }
}

// Slice, one thread per (point, float4 group); normalising divides by the homogeneous channel c, read from its
// own group.
__global__ void k_lat_slice(const float4* __restrict__ lat, const int* __restrict__ vidx,
                            const float* __restrict__ vbary, int64_t n, int d, int c, int g4, int normalize,
                            float* __restrict__ out) {
    const int d1 = d + 1;
    const int gh = c >> 2, uh = c & 3;  // group and lane of the homogeneous channel
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * g4; e += (int64_t)gridDim.x * blockDim.x) {
        int g;
        const int64_t i = sdg_divmod(e, g4, g);
        if (4 * g >= c) continue;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        float hom = 0.f;
        for (int j = 0; j < d1; ++j) {
            const int m = vidx[i * d1 + j];
            if (m < 0) continue;
            const float b = vbary[i * d1 + j];
            const float4 v = lat[(int64_t)m * g4 + g];
            acc.x = fmaf(b, v.x, acc.x);
            acc.y = fmaf(b, v.y, acc.y);
            acc.z = fmaf(b, v.z, acc.z);
            acc.w = fmaf(b, v.w, acc.w);
            if (normalize) {
                const float4 h = lat[(int64_t)m * g4 + gh];
                hom = fmaf(b, uh == 0 ? h.x : uh == 1 ? h.y : uh == 2 ? h.z : h.w, hom);
            }
        }
        const float a4[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = 4 * g + u;
            if (q < c) out[(int64_t)c * i + q] = normalize ? a4[u] / hom : a4[u];
        }
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
    const int d1 = d + 1, g4 = (c + 1 + 3) / 4, cc = 4 * g4;  // rows of float4 groups
    const int64_t nv = n * d1;  // vertex references; at most this many lattice points
    const uint64_t cap = pow2_at_least((uint64_t)std::max<int64_t>(nv + nv / 4, 1024));  // load <= 0.8
    int rc;
    if ((rc = grow(&L.fp, &L.cap_fp, (int64_t)cap, s)) || (rc = grow(&L.idx, &L.cap_idx, (int64_t)cap, s)) ||
        (rc = grow(&L.fp2, &L.cap_fp2, (int64_t)cap, s)) ||
        (rc = grow(&L.skey, &L.cap_skey, (int64_t)cap * d, s)) || (rc = grow(&L.keys, &L.cap_keys, nv * d, s)) ||
        (rc = grow(&L.vidx, &L.cap_vidx, nv, s)) || (rc = grow(&L.vbary, &L.cap_vbary, nv, s)) ||
        (rc = grow(&L.val0, &L.cap_val0, nv * cc, s)) || (rc = grow(&L.val1, &L.cap_val1, nv * cc, s)) ||
        (rc = grow(&L.nb, &L.cap_nb, nv * d1 * 2, s)) || (rc = grow(&L.counters, &L.cap_counters, (int64_t)2, s)) ||
        (rc = grow(&L.sr, &L.cap_sr, nv, s)) || (rc = grow(&L.srank, &L.cap_srank, nv, s)) ||
        (rc = grow(&L.vslot, &L.cap_vslot, nv, s)))
        return rc;
    SDG_CUDA_TRY(cudaMemsetAsync(L.fp, 0xFF, sizeof(unsigned long long) * cap, s));
    SDG_CUDA_TRY(cudaMemsetAsync(L.counters, 0, 2 * sizeof(int), s));
    Table t{L.fp, L.fp2, L.idx, L.skey, (unsigned)(cap - 1)};
    int* count = L.counters;
    int* status = L.counters + 1;
    k_lat_simplex<<<blocks_for(n), kThreads, 0, s>>>(pos, n, d, L.sr, L.srank, L.vbary, status);
    SDG_LAUNCH_CHECK("lattice simplex");
    k_lat_insert<<<blocks_for(nv), kThreads, 0, s>>>(n, d, t, L.sr, L.srank, L.vslot, status);
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
    k_lat_splat<<<blocks_for(n * g4), kThreads, 0, s>>>(val, n, d, c, g4, t, L.keys, L.sr, L.srank, L.vslot,
                                                        L.vbary, reinterpret_cast<float4*>(L.val0), L.vidx, status);
    SDG_LAUNCH_CHECK("lattice splat");
    k_lat_neighbours<<<blocks_for((int64_t)M * d1), kThreads, 0, s>>>(L.keys, M, d, t, L.nb);
    SDG_LAUNCH_CHECK("lattice neighbours");
    float* a = L.val0;
    float* b = L.val1;
    for (int dir = 0; dir < d1; ++dir) {
        k_lat_blur<<<blocks_for((int64_t)M * g4), kThreads, 0, s>>>(reinterpret_cast<const float4*>(a),
                                                                     reinterpret_cast<float4*>(b), L.nb, M, d, dir,
                                                                     g4);
        SDG_LAUNCH_CHECK("lattice blur");
        std::swap(a, b);
    }
    k_lat_slice<<<blocks_for(n * g4), kThreads, 0, s>>>(reinterpret_cast<const float4*>(a), L.vidx, L.vbary, n, d,
                                                        c, g4, normalize, out);
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
