// Shared device/host definitions of libsdg: block-key packing, the
// open-addressing block hash map, the device-side grid descriptor and error
// plumbing.  Paper: arXiv 2305.13220, Sec. 3.2 ("Sparse-Dense Data Structure").
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "sdg.h"

// ---------------------------------------------------------------------------
// Error plumbing (host)
// ---------------------------------------------------------------------------
namespace sdg {

void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

}  // namespace sdg

#define SDG_CUDA_TRY(expr)                                         \
    do {                                                           \
        cudaError_t _e = (expr);                                   \
        if (_e != cudaSuccess) return ::sdg::cuda_fail(_e, #expr); \
    } while (0)

#define SDG_LAUNCH_CHECK(what)                                    \
    do {                                                          \
        cudaError_t _e = cudaGetLastError();                      \
        if (_e != cudaSuccess) return ::sdg::cuda_fail(_e, what); \
    } while (0)

// ---------------------------------------------------------------------------
// Block keys: int3 in [-2^20, 2^20)^3 packed into 63 bits, x lowest.  The
// packed order is the (z, y, x) lexicographic order, which defines the index
// assignment of an activation batch.  All-ones is the empty-slot marker (never
// a valid key: bit 63 of a packed key is 0).
// ---------------------------------------------------------------------------
#define SDG_KEY_BIAS (1 << 20)
#define SDG_EMPTY_KEY 0xFFFFFFFFFFFFFFFFull

// q = e / div and r = e - q div for 0 <= e, in 32-bit unsigned arithmetic whenever e fits (every practical
// size; a 64-bit division is a long instruction sequence), else in 64 bits.
__device__ __forceinline__ int64_t sdg_divmod(int64_t e, int div, int& r) {
    if (e <= 0xFFFFFFFFll) {
        const unsigned q = (unsigned)e / (unsigned)div;
        r = (int)((unsigned)e - q * (unsigned)div);
        return (int64_t)q;
    }
    const int64_t q = e / div;
    r = (int)(e - q * div);
    return q;
}

__host__ __device__ __forceinline__ uint64_t sdg_pack_key(int x, int y, int z) {
    return (uint64_t)(uint32_t)(x + SDG_KEY_BIAS) | ((uint64_t)(uint32_t)(y + SDG_KEY_BIAS) << 21) |
           ((uint64_t)(uint32_t)(z + SDG_KEY_BIAS) << 42);
}
__host__ __device__ __forceinline__ int3 sdg_unpack_key(uint64_t k) {
    return make_int3((int)(k & 0x1FFFFF) - SDG_KEY_BIAS, (int)((k >> 21) & 0x1FFFFF) - SDG_KEY_BIAS,
                     (int)((k >> 42) & 0x1FFFFF) - SDG_KEY_BIAS);
}

// Slot hash: the 64-bit finaliser of MurmurHash3 (Appleby, public domain).
__host__ __device__ __forceinline__ uint32_t sdg_slot_hash(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return (uint32_t)k;
}

// A slot is 16 bytes {key, value}: one vector load answers a probe.
// Linear probing; capacity is a power of two >= 2 * max_blocks, so the load
// factor stays <= 0.5 and every probe sequence ends at an empty slot.  The
// loop is still bounded by the capacity.
__device__ __forceinline__ int32_t sdg_table_find(const ulonglong2* __restrict__ t, uint32_t mask, uint64_t key) {
    uint32_t h = sdg_slot_hash(key) & mask;
#pragma unroll 1
    for (uint32_t p = 0; p <= mask; ++p) {
        ulonglong2 s = __ldg(t + h);
        if (s.x == key) return (int32_t)s.y;
        if (s.x == SDG_EMPTY_KEY) return -1;
        h = (h + 1) & mask;
    }
    return -1;
}

// Same lookup through L2 only (no L1 copy), for kernels that read a table an
// earlier kernel of the same stream has just written.
__device__ __forceinline__ int32_t sdg_table_find_rw(const ulonglong2* t, uint32_t mask, uint64_t key) {
    uint32_t h = sdg_slot_hash(key) & mask;
#pragma unroll 1
    for (uint32_t p = 0; p <= mask; ++p) {
        ulonglong2 s = __ldcg(t + h);
        if (s.x == key) return (int32_t)s.y;
        if (s.x == SDG_EMPTY_KEY) return -1;
        h = (h + 1) & mask;
    }
    return -1;
}

// Insert-if-absent.  Returns 1 if this call inserted the key, 0 if it was
// present, -1 if the probe limit (the capacity) was reached.
__device__ __forceinline__ int sdg_table_insert(ulonglong2* t, uint32_t mask, uint64_t key, uint64_t value) {
    uint32_t h = sdg_slot_hash(key) & mask;
#pragma unroll 1
    for (uint32_t p = 0; p <= mask; ++p) {
        unsigned long long* kp = reinterpret_cast<unsigned long long*>(&t[h].x);
        unsigned long long cur = *reinterpret_cast<volatile unsigned long long*>(kp);
        if (cur == key) return 0;
        if (cur == SDG_EMPTY_KEY) {
            unsigned long long old = atomicCAS(kp, SDG_EMPTY_KEY, (unsigned long long)key);
            if (old == SDG_EMPTY_KEY) {
                t[h].y = value;
                return 1;
            }
            if (old == key) return 0;
        }
        h = (h + 1) & mask;
    }
    return -1;
}

// ---------------------------------------------------------------------------
// Device-side view of a grid, passed to kernels by value.
// ---------------------------------------------------------------------------
struct GridDev {
    const ulonglong2* table;  // hash slots
    const int4* nbr;          // [N][2] int4: block index of +{0,x,y,xy,z,xz,yz,xyz} neighbours, -1 if absent
    const int32_t* dense;     // block index of every cell of the block AABB (-1: not allocated), x fastest
    const int4* keys;         // [N] {x, y, z, 0}
    uint32_t mask;
    int32_t n_sem;
    int32_t bmin[3];  // AABB origin (block units)
    int32_t bdim[3];  // AABB size (blocks); all zero when the grid is empty
    float vs, inv_vs, L, inv_L;
    float beta, inv_beta;
    int64_t n_blocks;
    // SDG_F32 layout
    const float4* geo;  // {sdf, r, g, b}
    float4* ggeo;
    // SDG_BF16 layout
    const float* sdf;
    const uint2* rgbh;  // 4 x bf16
    float* gsdf;
    float4* grgb;
    // semantics (either layout)
    const __nv_bfloat16* sem;  // [N*512][n_sem]
    float* gsem;               // [N*512][n_sem]
    // bounds-checked build only: cells of the dense block-index grid, and the device status word that records the
    // first index found out of range
    int64_t dense_cells;
    unsigned long long* status;
};

// ---------------------------------------------------------------------------
// Bounds-checked build (compile with -DSDG_CHECKED).  Every block index, voxel address, dense-grid cell and ray
// index a kernel derives is checked before it is used; the first one out of range is recorded in a device
// status word -- code << 48 | the index's low 48 bits -- with no trap, and the access it guards is skipped (the
// stencil counts as invalid, the cell as unallocated, the ray as absent).  In the normal build every check is the
// constant true and compiles to nothing.
// ---------------------------------------------------------------------------
// (codes SDG_CHECK_BLOCK, _VOXEL, _DENSE, _RAY: include/sdg.h)
#ifdef SDG_CHECKED
__device__ __forceinline__ bool sdg_in_range(unsigned long long* status, long long i, long long n, unsigned code) {
    if (i >= 0 && i < n) return true;
    if (status) atomicCAS(status, 0ull, ((unsigned long long)code << 48) | ((unsigned long long)i & 0xFFFFFFFFFFFFull));
    return false;
}
#else
__device__ __forceinline__ constexpr bool sdg_in_range(unsigned long long*, long long, long long, unsigned) {
    return true;
}
#endif

// Status word bits written by kernels (never a trap).
#define SDG_STATUS_TABLE_FULL 1u
#define SDG_STATUS_BAD_INPUT 2u

__device__ __forceinline__ float sdg_bf16_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float sdg_bf16_hi(uint32_t u) { return __uint_as_float(u & 0xFFFF0000u); }
