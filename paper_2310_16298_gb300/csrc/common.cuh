// Shared definitions for the library's kernels and host runtime.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace stx {

constexpr int kMaxRadius = 4;
constexpr int kBcDirichlet = 0;
constexpr int kBcPeriodic = 1;

// Dense gather-orientation coefficient tensor C^g passed by value as a kernel
// parameter (it lives in the constant bank, so every unrolled use is an
// immediate-like operand of the FMA).
template <typename T, int NC>
struct Coeffs {
    T c[NC];
};

constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

__host__ __device__ inline int64_t wrap_index(int64_t i, int64_t n) {
    int64_t m = i % n;
    return m < 0 ? m + n : m;
}

}  // namespace stx
