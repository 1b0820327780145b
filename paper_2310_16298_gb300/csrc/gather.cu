// CUDA-core gather kernels: the baseline form of the stencil,
//   B[x] = sum_o C^g[o] * A[x + o - r]                       (Eq. (stencil-2d9p))
// evaluated point by point with FMAs.  One launch advances the field by `tb`
// time steps (temporal blocking): a block stages its output tile plus a halo
// of width r*tb in shared memory, performs tb sub-steps there (the valid
// region shrinks by r per sub-step; with a zero Dirichlet boundary, points
// outside the domain are reset to 0 after every sub-step), and writes the
// tile once.  Each thread computes a strip of RS outputs along the slowest
// axis, reusing every loaded shared-memory row for all outputs it feeds.
#include "common.cuh"
#include "kernels.h"

namespace stx {

namespace {

constexpr int kBX = 32;   // threads along the contiguous axis (one warp)
constexpr int kRS = 8;    // outputs per thread along the strip axis

// Asynchronous global->shared copy of one element (Ampere-style cp.async):
// many copies stay in flight per thread, so the tile load runs at HBM rate.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Address of a tile element after the boundary rule, or nullptr for a zero.
template <typename T>
__device__ __forceinline__ const T* src2(const T* __restrict__ a, int64_t y, int64_t x, int64_t ny,
                                         int64_t nx, int bc) {
    if (y < 0 || y >= ny || x < 0 || x >= nx) {
        if (bc == kBcDirichlet) return nullptr;
        y = wrap_index(y, ny);
        x = wrap_index(x, nx);
    }
    return a + y * nx + x;
}

template <typename T>
__device__ __forceinline__ const T* src3(const T* __restrict__ a, int64_t z, int64_t y, int64_t x,
                                         int64_t nz, int64_t ny, int64_t nx, int bc) {
    if (z < 0 || z >= nz || y < 0 || y >= ny || x < 0 || x >= nx) {
        if (bc == kBcDirichlet) return nullptr;
        z = wrap_index(z, nz);
        y = wrap_index(y, ny);
        x = wrap_index(x, nx);
    }
    return a + (z * ny + y) * nx + x;
}

// ---------------------------------------------------------------------------
// 2D.  Block = (32, BY) threads; output tile TY x TX.  Strips run along y.
// ---------------------------------------------------------------------------
// One output tile (origin y0, x0) advanced by tb steps; shared by the
// single-problem and the batched kernels.
template <typename T, int R, bool STAR, int BY, int TX, int TY>
__device__ __forceinline__ void gather2d_tile(const T* __restrict__ in, T* __restrict__ out, int64_t ny,
                                              int64_t nx, int bc, int tb, const Coeffs<T, ipow(2 * R + 1, 2)>& cf,
                                              int64_t y0, int64_t x0, T* smem) {
    constexpr int W = 2 * R + 1;
    const int H = R * tb;
    const int SX = TX + 2 * H;
    const int SY = TY + 2 * H;
    // buf[0] | buf[1] (tb > 1 only) | kRS slack rows read (never used) by ragged strips
    T* buf[2] = {smem, smem + SY * SX};
    const int rows_alloc = (tb > 1 ? 2 * SY : SY) + kRS;
    const int tx = threadIdx.x, ty = threadIdx.y;

    const bool interior = (y0 - H >= 0) && (y0 + TY + H <= ny) && (x0 - H >= 0) && (x0 + TX + H <= nx);
    for (int sy = ty; sy < rows_alloc; sy += BY) {
        const int64_t gy = y0 - H + sy;
        for (int sx = tx; sx < SX; sx += kBX) {
            const int64_t gx = x0 - H + sx;
            T* d = smem + sy * SX + sx;
            const T* g = nullptr;
            if (sy < SY) g = interior ? in + gy * nx + gx : src2(in, gy, gx, ny, nx, bc);
            if (g) cp_async_elem(d, g);
            else *d = T(0);
        }
    }
    cp_async_wait_all();
    __syncthreads();

    for (int t = 1; t <= tb; ++t) {
        const T* src = buf[(t - 1) & 1];
        T* dst = buf[t & 1];
        const bool last = (t == tb);
        const int lo = R * t;
        const int Ht = SY - 2 * lo, Wt = SX - 2 * lo;
        const int nstrips = (Ht + kRS - 1) / kRS;
        for (int strip = ty; strip < nstrips; strip += BY) {
            const int sy0 = lo + strip * kRS;
            for (int c = tx; c < Wt; c += kBX) {
                const int sx = lo + c;
                T acc[kRS];
#pragma unroll
                for (int j = 0; j < kRS; ++j) acc[j] = T(0);
                const T* base = src + (sy0 - R) * SX + (sx - R);
#pragma unroll
                for (int yi = 0; yi < kRS + 2 * R; ++yi) {
                    T v[W];
#pragma unroll
                    for (int b = 0; b < W; ++b) v[b] = base[yi * SX + b];
#pragma unroll
                    for (int j = 0; j < kRS; ++j) {
                        const int a = yi - j;
                        if (a >= 0 && a < W) {
#pragma unroll
                            for (int b = 0; b < W; ++b) {
                                if (!STAR || a == R || b == R) acc[j] = fma(cf.c[a * W + b], v[b], acc[j]);
                            }
                        }
                    }
                }
                const int64_t gx = x0 - H + sx;
#pragma unroll
                for (int j = 0; j < kRS; ++j) {
                    const int sy = sy0 + j;
                    if (sy < SY - lo) {
                        const int64_t gy = y0 - H + sy;
                        if (last) {
                            if (gy < ny && gx < nx) out[gy * nx + gx] = acc[j];
                        } else {
                            const bool outside = (bc == kBcDirichlet) && (gy < 0 || gy >= ny || gx < 0 || gx >= nx);
                            dst[sy * SX + sx] = outside ? T(0) : acc[j];
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
}

template <typename T, int R, bool STAR, int BY, int TX, int TY>
__global__ void __launch_bounds__(kBX * BY)
gather2d_kernel(const T* __restrict__ in, T* __restrict__ out, int64_t ny, int64_t nx, int bc,
                int tb, Coeffs<T, ipow(2 * R + 1, 2)> cf) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    gather2d_tile<T, R, STAR, BY, TX, TY>(in, out, ny, nx, bc, tb, cf, (int64_t)blockIdx.y * TY,
                                          (int64_t)blockIdx.x * TX, reinterpret_cast<T*>(smem_raw));
}

// Persistent batched sweep: the tiles of many independent problems, each
// advanced by its own depth, processed by one grid-stride launch.  Problem
// p owns tiles [tile0[p], tile0[p+1]); its coefficients sit at coef + p*NC.
template <typename T, int R, bool STAR, int BY, int TX, int TY>
__global__ void __launch_bounds__(kBX * BY)
gather2d_batch_kernel(const BatchProblem* __restrict__ probs, int nprob, int total_tiles,
                      const T* __restrict__ coef) {
    constexpr int NC = ipow(2 * R + 1, 2);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) {
        int lo = 0, hi = nprob - 1;  // last problem whose first tile <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (probs[mid].tile0 <= t) lo = mid;
            else hi = mid - 1;
        }
        const BatchProblem P = probs[lo];
        const int local = t - P.tile0;
        Coeffs<T, NC> cf;
#pragma unroll
        for (int i = 0; i < NC; ++i) cf.c[i] = coef[(size_t)P.coef_index * NC + i];
        gather2d_tile<T, R, STAR, BY, TX, TY>((const T*)P.src, (T*)P.dst, P.ny, P.nx, P.bc, P.depth, cf,
                                              (int64_t)(local / P.tiles_x) * TY, (int64_t)(local % P.tiles_x) * TX,
                                              reinterpret_cast<T*>(smem_raw));
    }
}

// ---------------------------------------------------------------------------
// 3D.  Block = (32, BY) threads covering (y, x); strips run along z.
// Output tile TZ x TY x TX.
// ---------------------------------------------------------------------------
template <typename T, int R, bool STAR, int BY, int TX, int TY, int TZ>
__global__ void __launch_bounds__(kBX * BY)
gather3d_kernel(const T* __restrict__ in, T* __restrict__ out, int64_t nz, int64_t ny, int64_t nx,
                int bc, int tb, Coeffs<T, ipow(2 * R + 1, 3)> cf) {
    constexpr int W = 2 * R + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* smem = reinterpret_cast<T*>(smem_raw);
    const int H = R * tb;
    const int SX = TX + 2 * H, SY = TY + 2 * H, SZ = TZ + 2 * H;
    const int plane = SY * SX;
    // buf[0] | buf[1] (tb > 1 only) | kRS slack planes read (never used) by ragged strips
    const int planes_alloc = (tb > 1 ? 2 * SZ : SZ) + kRS;
    T* buf[2] = {smem, smem + SZ * plane};
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t z0 = (int64_t)blockIdx.z * TZ, y0 = (int64_t)blockIdx.y * TY,
                  x0 = (int64_t)blockIdx.x * TX;
    const bool interior = (z0 - H >= 0) && (z0 + TZ + H <= nz) && (y0 - H >= 0) &&
                          (y0 + TY + H <= ny) && (x0 - H >= 0) && (x0 + TX + H <= nx);
    for (int sz = 0; sz < planes_alloc; ++sz) {
        const int64_t gz = z0 - H + sz;
        for (int sy = ty; sy < SY; sy += BY) {
            const int64_t gy = y0 - H + sy;
            for (int sx = tx; sx < SX; sx += kBX) {
                const int64_t gx = x0 - H + sx;
                T* d = smem + sz * plane + sy * SX + sx;
                const T* g = nullptr;
                if (sz < SZ) g = interior ? in + (gz * ny + gy) * nx + gx : src3(in, gz, gy, gx, nz, ny, nx, bc);
                if (g) cp_async_elem(d, g);
                else *d = T(0);
            }
        }
    }
    cp_async_wait_all();
    __syncthreads();

    for (int t = 1; t <= tb; ++t) {
        const T* src = buf[(t - 1) & 1];
        T* dst = buf[t & 1];
        const bool last = (t == tb);
        const int lo = R * t;
        const int Dt = SZ - 2 * lo, Ht = SY - 2 * lo, Wt = SX - 2 * lo;
        const int nstrips = (Dt + kRS - 1) / kRS;
        for (int strip = 0; strip < nstrips; ++strip) {
            const int sz0 = lo + strip * kRS;
            for (int cy = ty; cy < Ht; cy += BY) {
                const int sy = lo + cy;
                for (int cx = tx; cx < Wt; cx += kBX) {
                    const int sx = lo + cx;
                    T acc[kRS];
#pragma unroll
                    for (int j = 0; j < kRS; ++j) acc[j] = T(0);
                    const T* base = src + (sz0 - R) * plane + (sy - R) * SX + (sx - R);
#pragma unroll
                    for (int zi = 0; zi < kRS + 2 * R; ++zi) {
#pragma unroll
                        for (int a1 = 0; a1 < W; ++a1) {
                            T v[W];
#pragma unroll
                            for (int b = 0; b < W; ++b) v[b] = base[zi * plane + a1 * SX + b];
#pragma unroll
                            for (int j = 0; j < kRS; ++j) {
                                const int a0 = zi - j;
                                if (a0 >= 0 && a0 < W) {
#pragma unroll
                                    for (int b = 0; b < W; ++b) {
                                        const bool on_axis = (a1 == R && b == R) || (a0 == R && b == R) ||
                                                             (a0 == R && a1 == R);
                                        if (!STAR || on_axis)
                                            acc[j] = fma(cf.c[(a0 * W + a1) * W + b], v[b], acc[j]);
                                    }
                                }
                            }
                        }
                    }
                    const int64_t gy = y0 - H + sy, gx = x0 - H + sx;
#pragma unroll
                    for (int j = 0; j < kRS; ++j) {
                        const int sz = sz0 + j;
                        if (sz < SZ - lo) {
                            const int64_t gz = z0 - H + sz;
                            if (last) {
                                if (gz < nz && gy < ny && gx < nx) out[(gz * ny + gy) * nx + gx] = acc[j];
                            } else {
                                const bool outside = (bc == kBcDirichlet) &&
                                                     (gz < 0 || gz >= nz || gy < 0 || gy >= ny || gx < 0 || gx >= nx);
                                dst[sz * plane + sy * SX + sx] = outside ? T(0) : acc[j];
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
}

// Tile shapes.
constexpr int k2BY = 8, k2TX = 128, k2TY = 64;
constexpr int k3BY = 8, k3TX = 32, k3TY = 16, k3TZ = 8;
// Tile shapes of the batched kernel (rows x columns), chosen per batch by the
// autotuner: the single-grid shape, and a smaller one that wastes less of the
// ragged edge tiles of small problems.
constexpr int kBatchShapes = 2;
constexpr int kBatchTY[kBatchShapes] = {64, 32};
constexpr int kBatchTX[kBatchShapes] = {128, 64};

template <typename T>
size_t gather_smem_bytes_t(int ndim, int r, int tb) {
    const int H = r * tb;
    const int nb = tb > 1 ? 2 : 1;
    if (ndim == 2) return (size_t)(nb * (k2TY + 2 * H) + kRS) * (k2TX + 2 * H) * sizeof(T);
    return (size_t)(nb * (k3TZ + 2 * H) + kRS) * (k3TY + 2 * H) * (k3TX + 2 * H) * sizeof(T);
}

template <typename T, int R, bool STAR>
cudaError_t launch2d(const GatherProblem& p, const void* in, void* out, int tb, cudaStream_t s) {
    constexpr int NC = ipow(2 * R + 1, 2);
    Coeffs<T, NC> cf;
    for (int i = 0; i < NC; ++i) cf.c[i] = (T)p.cg[i];
    const size_t smem = gather_smem_bytes_t<T>(2, R, tb);
    auto kern = gather2d_kernel<T, R, STAR, k2BY, k2TX, k2TY>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((p.n[1] + k2TX - 1) / k2TX), (unsigned)((p.n[0] + k2TY - 1) / k2TY));
    kern<<<grid, dim3(kBX, k2BY), smem, s>>>((const T*)in, (T*)out, p.n[0], p.n[1], p.bc, tb, cf);
    return cudaGetLastError();
}

template <typename T, int R, bool STAR>
cudaError_t launch3d(const GatherProblem& p, const void* in, void* out, int tb, cudaStream_t s) {
    constexpr int NC = ipow(2 * R + 1, 3);
    Coeffs<T, NC> cf;
    for (int i = 0; i < NC; ++i) cf.c[i] = (T)p.cg[i];
    const size_t smem = gather_smem_bytes_t<T>(3, R, tb);
    auto kern = gather3d_kernel<T, R, STAR, k3BY, k3TX, k3TY, k3TZ>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((p.n[2] + k3TX - 1) / k3TX), (unsigned)((p.n[1] + k3TY - 1) / k3TY),
              (unsigned)((p.n[0] + k3TZ - 1) / k3TZ));
    kern<<<grid, dim3(kBX, k3BY), smem, s>>>((const T*)in, (T*)out, p.n[0], p.n[1], p.n[2], p.bc, tb, cf);
    return cudaGetLastError();
}

template <typename T, bool STAR>
cudaError_t dispatch_r(const GatherProblem& p, const void* in, void* out, int tb, cudaStream_t s) {
    if (p.ndim == 2) {
        switch (p.r) {
            case 1: return launch2d<T, 1, STAR>(p, in, out, tb, s);
            case 2: return launch2d<T, 2, STAR>(p, in, out, tb, s);
            case 3: return launch2d<T, 3, STAR>(p, in, out, tb, s);
            case 4: return launch2d<T, 4, STAR>(p, in, out, tb, s);
        }
    } else {
        switch (p.r) {
            case 1: return launch3d<T, 1, STAR>(p, in, out, tb, s);
            case 2: return launch3d<T, 2, STAR>(p, in, out, tb, s);
            case 3: return launch3d<T, 3, STAR>(p, in, out, tb, s);
            case 4: return launch3d<T, 4, STAR>(p, in, out, tb, s);
        }
    }
    return cudaErrorInvalidValue;
}

template <typename T>
size_t batch_smem_bytes_t(int r, int tb, int shape) {
    const int H = r * tb;
    const int nb = tb > 1 ? 2 : 1;
    return (size_t)(nb * (kBatchTY[shape] + 2 * H) + kRS) * (kBatchTX[shape] + 2 * H) * sizeof(T);
}

template <typename T, int R, bool STAR, int S>
cudaError_t launch_batch(const BatchProblem* probs, int nprob, int total_tiles, const void* coef, int max_tb,
                         int grid, cudaStream_t s) {
    const size_t smem = batch_smem_bytes_t<T>(R, max_tb, S);
    auto kern = gather2d_batch_kernel<T, R, STAR, k2BY, kBatchTX[S], kBatchTY[S]>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (grid <= 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kBX * k2BY, smem);
        grid = sms * (per > 0 ? per : 1);
    }
    if (grid > total_tiles) grid = total_tiles;
    if (grid <= 0) return cudaSuccess;
    kern<<<grid, dim3(kBX, k2BY), smem, s>>>(probs, nprob, total_tiles, (const T*)coef);
    return cudaGetLastError();
}

template <typename T, bool STAR, int S>
cudaError_t dispatch_batch_r(int r, const BatchProblem* probs, int nprob, int total_tiles, const void* coef,
                             int max_tb, int grid, cudaStream_t s) {
    switch (r) {
        case 1: return launch_batch<T, 1, STAR, S>(probs, nprob, total_tiles, coef, max_tb, grid, s);
        case 2: return launch_batch<T, 2, STAR, S>(probs, nprob, total_tiles, coef, max_tb, grid, s);
        case 3: return launch_batch<T, 3, STAR, S>(probs, nprob, total_tiles, coef, max_tb, grid, s);
    }
    return cudaErrorInvalidValue;
}

template <typename T, bool STAR>
cudaError_t dispatch_batch(int r, const BatchProblem* probs, int nprob, int total_tiles, const void* coef,
                           int max_tb, int shape, cudaStream_t s) {
    if (shape == 1) return dispatch_batch_r<T, STAR, 1>(r, probs, nprob, total_tiles, coef, max_tb, 0, s);
    return dispatch_batch_r<T, STAR, 0>(r, probs, nprob, total_tiles, coef, max_tb, 0, s);
}

}  // namespace

cudaError_t gather_batch_sweep(bool f64, bool star, int r, const BatchProblem* d_probs, int nprob, int total_tiles,
                               const void* d_coef, int max_tb, int shape, cudaStream_t s) {
    if (shape < 0 || shape >= kBatchShapes) return cudaErrorInvalidValue;
    if (f64) return star ? dispatch_batch<double, true>(r, d_probs, nprob, total_tiles, d_coef, max_tb, shape, s)
                         : dispatch_batch<double, false>(r, d_probs, nprob, total_tiles, d_coef, max_tb, shape, s);
    return star ? dispatch_batch<float, true>(r, d_probs, nprob, total_tiles, d_coef, max_tb, shape, s)
                : dispatch_batch<float, false>(r, d_probs, nprob, total_tiles, d_coef, max_tb, shape, s);
}

int gather_batch_shapes() { return kBatchShapes; }

void gather_batch_tile_shape(int shape, int* ty, int* tx) {
    *ty = kBatchTY[shape];
    *tx = kBatchTX[shape];
}

size_t gather_batch_smem_bytes(bool f64, int r, int tb, int shape) {
    return f64 ? batch_smem_bytes_t<double>(r, tb, shape) : batch_smem_bytes_t<float>(r, tb, shape);
}

size_t gather_smem_bytes(const GatherProblem& p, int tb) {
    return p.f64 ? gather_smem_bytes_t<double>(p.ndim, p.r, tb) : gather_smem_bytes_t<float>(p.ndim, p.r, tb);
}

cudaError_t gather_sweep(const GatherProblem& p, const void* in, void* out, int tb, cudaStream_t s) {
    if (p.f64) return p.star ? dispatch_r<double, true>(p, in, out, tb, s) : dispatch_r<double, false>(p, in, out, tb, s);
    return p.star ? dispatch_r<float, true>(p, in, out, tb, s) : dispatch_r<float, false>(p, in, out, tb, s);
}

}  // namespace stx
