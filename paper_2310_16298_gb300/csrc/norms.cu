// FP64 error-norm reduction of a GPU result against a reference grid:
//   {sum (g - o)^2, sum o^2, max |g - o|, max |o|}
// The relative L2 and relative max errors reported beside every result are
// formed from these four numbers on the host.  Two launches: a grid-stride
// pass writes one partial quadruple per block into device scratch, then one
// block folds the partials in a fixed order (deterministic result).
#include "common.cuh"
#include "kernels.h"

namespace stx {

namespace {

constexpr int kNormBlocks = 4 * 152;
constexpr int kNormThreads = 256;

__device__ __forceinline__ void block_reduce4(double& s0, double& s1, double& m0, double& m1,
                                              double* sh) {
    for (int off = 16; off > 0; off >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, off);
        s1 += __shfl_down_sync(0xffffffffu, s1, off);
        m0 = fmax(m0, __shfl_down_sync(0xffffffffu, m0, off));
        m1 = fmax(m1, __shfl_down_sync(0xffffffffu, m1, off));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sh[warp * 4 + 0] = s0;
        sh[warp * 4 + 1] = s1;
        sh[warp * 4 + 2] = m0;
        sh[warp * 4 + 3] = m1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        s0 = s1 = m0 = m1 = 0.0;
        for (int w = 0; w < nw; ++w) {
            s0 += sh[w * 4 + 0];
            s1 += sh[w * 4 + 1];
            m0 = fmax(m0, sh[w * 4 + 2]);
            m1 = fmax(m1, sh[w * 4 + 3]);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kNormThreads)
norms_partial_kernel(const T* __restrict__ got, const double* __restrict__ ref, int64_t count,
                     double* __restrict__ partials) {
    __shared__ double sh[4 * (kNormThreads / 32)];
    double s0 = 0.0, s1 = 0.0, m0 = 0.0, m1 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double o = ref[i];
        const double d = (double)got[i] - o;
        s0 = fma(d, d, s0);
        s1 = fma(o, o, s1);
        m0 = fmax(m0, fabs(d));
        m1 = fmax(m1, fabs(o));
    }
    block_reduce4(s0, s1, m0, m1, sh);
    if (threadIdx.x == 0) {
        partials[blockIdx.x * 4 + 0] = s0;
        partials[blockIdx.x * 4 + 1] = s1;
        partials[blockIdx.x * 4 + 2] = m0;
        partials[blockIdx.x * 4 + 3] = m1;
    }
}

__global__ void __launch_bounds__(kNormThreads)
norms_final_kernel(const double* __restrict__ partials, int nparts, double* __restrict__ out4) {
    __shared__ double sh[4 * (kNormThreads / 32)];
    double s0 = 0.0, s1 = 0.0, m0 = 0.0, m1 = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        s0 += partials[i * 4 + 0];
        s1 += partials[i * 4 + 1];
        m0 = fmax(m0, partials[i * 4 + 2]);
        m1 = fmax(m1, partials[i * 4 + 3]);
    }
    block_reduce4(s0, s1, m0, m1, sh);
    if (threadIdx.x == 0) {
        out4[0] = s0;
        out4[1] = s1;
        out4[2] = m0;
        out4[3] = m1;
    }
}

}  // namespace

size_t norms_partials_bytes() { return (size_t)kNormBlocks * 4 * sizeof(double); }

cudaError_t error_norms(const void* got, bool got_f64, const double* ref, int64_t count,
                        double* partials, double* out4, cudaStream_t s) {
    if (got_f64)
        norms_partial_kernel<double><<<kNormBlocks, kNormThreads, 0, s>>>((const double*)got, ref, count, partials);
    else
        norms_partial_kernel<float><<<kNormBlocks, kNormThreads, 0, s>>>((const float*)got, ref, count, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    norms_final_kernel<<<1, kNormThreads, 0, s>>>(partials, kNormBlocks, out4);
    return cudaGetLastError();
}

}  // namespace stx
