// Deterministic reduction shared by the loss entry points.
#pragma once

#include <cstdint>

namespace sdg {

// Sum of x[0, n) into out[0] (with ACC added to it), the same bits whatever the scheduling: block b sums the b-th
// of kSumBlocks contiguous slices in a fixed per-thread strided order and a fixed tree, and the block that
// finishes last (a ticket in scratch[kSumBlocks]) adds the blocks' partials in block order and resets the ticket.
// scratch: kSumBlocks + 1 words, the ticket 0 between calls; calls on one scratch run one after the other (one
// stream).  Internal linkage: each translation unit has its own copy.
template <bool ACC = false>
static __global__ void __launch_bounds__(512) k_sum(const float* __restrict__ x, int64_t n, float* out,
                                                    float* scratch) {
    __shared__ float s[512];
    __shared__ bool last;
    const int t = threadIdx.x;
    const int64_t chunk = (n + kSumBlocks - 1) / kSumBlocks;
    const int64_t lo = (int64_t)blockIdx.x * chunk, hi = lo + chunk < n ? lo + chunk : n;
    float acc = 0.f;
    for (int64_t i = lo + t; i < hi; i += 512) acc += x[i];
    s[t] = acc;
    __syncthreads();
    for (int w = 256; w > 0; w >>= 1) {
        if (t < w) s[t] += s[t + w];
        __syncthreads();
    }
    unsigned* ticket = reinterpret_cast<unsigned*>(scratch + kSumBlocks);
    if (t == 0) {
        scratch[blockIdx.x] = s[0];
        __threadfence();
        last = atomicAdd(ticket, 1u) == (unsigned)kSumBlocks - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    s[t] = t < kSumBlocks ? reinterpret_cast<volatile float*>(scratch)[t] : 0.f;
    __syncthreads();
    for (int w = 256; w > 0; w >>= 1) {
        if (t < w) s[t] += s[t + w];
        __syncthreads();
    }
    if (t == 0) {
        out[0] = ACC ? out[0] + s[0] : s[0];
        *ticket = 0u;
    }
}

template <bool ACC = false>
static inline void launch_sum(const float* x, int64_t n, float* out, float* scratch, cudaStream_t st) {
    k_sum<ACC><<<kSumBlocks, 512, 0, st>>>(x, n, out, scratch);
}

}  // namespace sdg
