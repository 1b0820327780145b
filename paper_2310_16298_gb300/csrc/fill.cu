// Device-side synthetic fields: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014)
// element i of a seed's stream, mapped to uniform[lo, hi) exactly as the host
// generator does (u = (x >> 11) * 2^-53; v = lo + (hi - lo) * u in FP64 with
// round-to-nearest, no fused multiply-add; then rounded to the storage type).
// Used by the serving loop for requests that name a seeded input instead of
// sending one.
#include "common.cuh"
#include "kernels.h"

namespace stx {

namespace {

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <typename T>
__global__ void fill_uniform_kernel(T* __restrict__ out, int64_t count, uint64_t seed, int64_t offset, double lo,
                                    double hi) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const double u = (double)(splitmix64_at(seed, (uint64_t)(offset + i)) >> 11) * 0x1.0p-53;
        const double v = (lo == 0.0 && hi == 1.0) ? u : __dadd_rn(lo, __dmul_rn(hi - lo, u));
        out[i] = (T)v;
    }
}

}  // namespace

cudaError_t fill_uniform(void* out, bool f64, int64_t count, uint64_t seed, int64_t offset, double lo, double hi,
                         cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int threads = 256;
    const int64_t want = (count + threads - 1) / threads;
    const int blocks = (int)(want < 4096 ? want : 4096);
    if (f64) fill_uniform_kernel<double><<<blocks, threads, 0, s>>>((double*)out, count, seed, offset, lo, hi);
    else fill_uniform_kernel<float><<<blocks, threads, 0, s>>>((float*)out, count, seed, offset, lo, hi);
    return cudaGetLastError();
}

}  // namespace stx
