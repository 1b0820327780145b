// Helpers shared by the matrixized kernels (2D and 3D).
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <string.h>

#include <mutex>

#include "ptx.cuh"

namespace stx {
namespace mxu {

constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

// Bounded mbarrier wait that also gives up once another role has failed.
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    const long long t0 = clock64();
    while (!ptx::mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > kWaitCycles) {
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

// TF32 high part by integer rounding (nearest, ties away from zero): the low
// 13 mantissa bits are cleared after adding half of their weight.
__device__ __forceinline__ uint32_t tf32_hi_bits(float x) {
    return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
}


inline PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}


// Round to TF32 on the host (nearest, ties to even); finite inputs.
inline float tf32_round(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    u += 0xFFFu + ((u >> 13) & 1u);
    u &= ~0x1FFFu;
    float y;
    memcpy(&y, &u, 4);
    return y;
}


}  // namespace mxu
}  // namespace stx
