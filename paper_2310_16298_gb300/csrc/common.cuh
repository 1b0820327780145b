// Shared definitions for the library's kernels and host runtime.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

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

// Launch with programmatic stream serialization: the kernel may start while
// the stream's previous kernel drains, so it must call griddepcontrol.wait
// before it touches memory that kernel writes (the tensor-core and boundary
// kernels do; their sweeps run back to back: about 2.5 us saved per sweep).
template <typename... P, typename... A>
cudaError_t launch_dependent(void (*fn)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, std::forward<A>(args)...);
}

__host__ __device__ inline int64_t wrap_index(int64_t i, int64_t n) {
    int64_t m = i % n;
    return m < 0 ? m + n : m;
}

}  // namespace stx
