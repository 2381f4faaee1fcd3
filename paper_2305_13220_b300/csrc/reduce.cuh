// Deterministic reduction shared by the loss entry points.
#pragma once

#include <cstdint>

namespace sdg {

// Sum of x[0, n) by one block of 1024 threads: a fixed per-thread strided order, then a fixed tree, so the
// result does not depend on scheduling.  Internal linkage: each translation unit has its own copy.
// With ACC the sum is added to out[0] instead of replacing it.
template <bool ACC = false>
static __global__ void __launch_bounds__(1024) k_sum(const float* __restrict__ x, int64_t n, float* out) {
    __shared__ float s[1024];
    float acc = 0.f;
    for (int64_t i = threadIdx.x; i < n; i += 1024) acc += x[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = ACC ? out[0] + s[0] : s[0];
}

}  // namespace sdg
