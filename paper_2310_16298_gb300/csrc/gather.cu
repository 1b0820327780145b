// CUDA-core gather kernels: the baseline form of the stencil,
//   B[x] = sum_o C^g[o] * A[x + o - r]                       (Eq. (stencil-2d9p))
// evaluated point by point with FMAs.  One launch advances the field by `tb`
// time steps (temporal blocking): a block stages its output tile plus a halo
// of width r*tb in shared memory, performs tb sub-steps there (the valid
// region shrinks by r per sub-step; with a zero Dirichlet boundary, points
// outside the domain are reset to 0 after every sub-step), and writes the
// tile once.  Each thread computes a strip of RS outputs along the slowest
// axis, reusing every loaded shared-memory row for all outputs it feeds.
//
// Single grids run persistent kernels that stage their tiles with TMA:
//  * 2D: each CTA walks its tiles through a ring of NST shared-memory stages
//    (four for FP32, two for FP64), the next tiles' halo blocks loading (one
//    cp.async.bulk.tensor each, zero fill outside the grid = the Dirichlet
//    halo) while the current one computes.
//  * 3D (one step per launch): a work unit is a column of output planes; the
//    CTA streams its input planes through a ring of 2r+2 plane buffers, each
//    loaded by TMA while the planes before it are used, so every input plane
//    is read from global memory once per unit instead of once per 3D tile.
// With a periodic boundary, tiles (3D: planes of units) whose halo crosses
// the grid's edge are staged by TMA like the others; then only their cells
// outside the grid are overwritten with wrapped values (`wrap_halo_block`).
// Waits are bounded; a timeout sets the plan's host-visible error word.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "kernels.h"
#include "mxutil.cuh"
#include "ptx.cuh"

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
                                         int64_t nx, int64_t ldx, int bc) {
    if (y < 0 || y >= ny || x < 0 || x >= nx) {
        if (bc == kBcDirichlet) return nullptr;
        y = wrap_index(y, ny);
        x = wrap_index(x, nx);
    }
    return a + y * ldx + x;
}

template <typename T>
__device__ __forceinline__ const T* src3(const T* __restrict__ a, int64_t z, int64_t y, int64_t x,
                                         int64_t nz, int64_t ny, int64_t nx, int64_t ldx, int bc) {
    if (z < 0 || z >= nz || y < 0 || y >= ny || x < 0 || x >= nx) {
        if (bc == kBcDirichlet) return nullptr;
        z = wrap_index(z, nz);
        y = wrap_index(y, ny);
        x = wrap_index(x, nx);
    }
    return a + (z * ny + y) * ldx + x;
}

// ---------------------------------------------------------------------------
// 2D.  Block = (32, BY) threads; output tile TY x TX.  Strips run along y.
// ---------------------------------------------------------------------------
// One output tile (origin y0, x0) advanced by tb steps; shared by the
// single-problem and the batched kernels.
template <typename T, int R, bool STAR, int BY, int TX, int TY>
__device__ __forceinline__ void gather2d_tile(const T* __restrict__ in, T* __restrict__ out, int64_t ny,
                                              int64_t nx, int64_t ldx, int bc, int tb, const Coeffs<T, ipow(2 * R + 1, 2)>& cf,
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
            if (sy < SY) g = interior ? in + gy * ldx + gx : src2(in, gy, gx, ny, nx, ldx, bc);
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
                            if (gy < ny && gx < nx) out[gy * ldx + gx] = acc[j];
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
gather2d_kernel(const T* __restrict__ in, T* __restrict__ out, int64_t ny, int64_t nx, int64_t ldx, int bc,
                int tb, Coeffs<T, ipow(2 * R + 1, 2)> cf) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    gather2d_tile<T, R, STAR, BY, TX, TY>(in, out, ny, nx, ldx, bc, tb, cf, (int64_t)blockIdx.y * TY,
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
        gather2d_tile<T, R, STAR, BY, TX, TY>((const T*)P.src, (T*)P.dst, P.ny, P.nx, P.nx, P.bc, P.depth, cf,
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
                int64_t ldx, int bc, int tb, Coeffs<T, ipow(2 * R + 1, 3)> cf) {
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
                if (sz < SZ) g = interior ? in + (gz * ny + gy) * ldx + gx : src3(in, gz, gy, gx, nz, ny, nx, ldx, bc);
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
                                if (gz < nz && gy < ny && gx < nx) out[(gz * ny + gy) * ldx + gx] = acc[j];
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

// ---------------------------------------------------------------------------
// TMA-staged persistent kernels (single grids).
// ---------------------------------------------------------------------------
constexpr long long kGatherWait = 4000000000LL;   // ~2 s of SM clock per wait

__host__ __device__ constexpr int round_up(int v, int a) { return (v + a - 1) / a * a; }

// Bounded wait on an mbarrier phase; false when the limit ran out.
__device__ __forceinline__ bool gwait(uint64_t* bar, uint32_t parity) {
    return ptx::mbar_wait(bar, parity, kGatherWait);
}

// 2D tile: TY x TX outputs per tile, threads (32, kBYT), NST stages in the
// TMA ring (NST - 1 tiles in flight ahead of the one being computed).
// FP32: 32 x 128, the last sub-step register-blocked (each thread kVR rows x
// 4 columns: 256 threads cover the tile once), four stages (about 96 KB, two
// CTAs per SM: six tiles in flight per SM); FP64: 64 x 32, one strip of kRS
// rows per thread row, two stages.
template <typename T>
struct Tile2 {
    static constexpr int TY = sizeof(T) == 4 ? 32 : 64;
    static constexpr int TX = sizeof(T) == 4 ? 128 : 32;
    static constexpr int NST = sizeof(T) == 4 ? 4 : 2;
    static constexpr int AL = 16 / (int)sizeof(T);   // TMA x granule (16 bytes)
};
constexpr int kVR = 4;   // FP32 last sub-step: rows per thread
constexpr int kBYT = 8;

struct G2Args {
    const void* in;
    void* out;
    unsigned int* err;   // host-mapped error word (may be null)
    int64_t ldx;         // row stride of the grids (elements)
    int ny, nx, bc, tb;
    int tiles_x, tiles_total;
};

// Shared-memory layout of the 2D kernel for depth tb: NST stages (TMA ring)
// and, for tb > 1, a work buffer for the sub-step ping-pong; kRS slack rows
// after each buffer are read (never used) by ragged strips.
template <typename T>
struct Layout2 {
    int H, HX, SY, SX, buf;   // halo rows, halo columns, rows, columns, elements per buffer
    __host__ __device__ Layout2(int r, int tb) {
        H = r * tb;
        HX = round_up(H, Tile2<T>::AL);
        SY = Tile2<T>::TY + 2 * H;
        SX = Tile2<T>::TX + 2 * HX;
        buf = round_up((SY + kRS) * SX, 128 / (int)sizeof(T));
    }
    __host__ __device__ int buffers(int tb) const { return Tile2<T>::NST + (tb > 1 ? 1 : 0); }
    __host__ __device__ size_t bytes(int tb) const { return (size_t)buffers(tb) * buf * sizeof(T) + 64 + 128; }
};

// One sub-step of depth t of the 2D tile: src -> dst (or -> the output grid
// on the last sub-step).  The buffer's element (sy, sx) is grid point
// (y0 - H + sy, x0 - HX + sx).
template <typename T, int R, bool STAR>
__device__ __forceinline__ void substep2(const T* src, T* dst, T* __restrict__ out, const Layout2<T>& L, int t,
                                         bool last, int64_t ny, int64_t nx, int64_t ldx, int bc, int64_t y0, int64_t x0,
                                         const Coeffs<T, ipow(2 * R + 1, 2)>& cf) {
    constexpr int W = 2 * R + 1;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int lo = R * t;                  // rows of the valid region skipped at the top
    const int lox = L.HX - L.H + R * t;    // columns skipped at the left
    const int Ht = L.SY - 2 * lo, Wt = L.SX - 2 * lox;
    const int nstrips = (Ht + kRS - 1) / kRS;
    for (int strip = ty; strip < nstrips; strip += kBYT) {
        const int sy0 = lo + strip * kRS;
        for (int c = tx; c < Wt; c += kBX) {
            const int sx = lox + c;
            T acc[kRS];
#pragma unroll
            for (int j = 0; j < kRS; ++j) acc[j] = T(0);
            const T* base = src + (sy0 - R) * L.SX + (sx - R);
#pragma unroll
            for (int yi = 0; yi < kRS + 2 * R; ++yi) {
                T v[W];
#pragma unroll
                for (int b = 0; b < W; ++b) v[b] = base[yi * L.SX + b];
#pragma unroll
                for (int j = 0; j < kRS; ++j) {
                    const int a = yi - j;
                    if (a >= 0 && a < W) {
#pragma unroll
                        for (int b = 0; b < W; ++b)
                            if (!STAR || a == R || b == R) acc[j] = fma(cf.c[a * W + b], v[b], acc[j]);
                    }
                }
            }
            const int64_t gx = x0 - L.HX + sx;
#pragma unroll
            for (int j = 0; j < kRS; ++j) {
                const int sy = sy0 + j;
                if (sy < L.SY - lo) {
                    const int64_t gy = y0 - L.H + sy;
                    if (last) {
                        if (gy < ny && gx < nx) out[gy * ldx + gx] = acc[j];
                    } else {
                        const bool outside = (bc == kBcDirichlet) && (gy < 0 || gy >= ny || gx < 0 || gx >= nx);
                        dst[sy * L.SX + sx] = outside ? T(0) : acc[j];
                    }
                }
            }
        }
    }
}

// Last sub-step of the 2D FP32 tile, register-blocked: a thread computes kRS
// rows x 4 adjacent columns.  Each input row it needs is read as three 16-byte
// shared-memory loads (columns x-4 .. x+7, enough for r <= 4), and every
// weight is applied to four columns at once, so a update costs its P FMAs and
// about one shared-memory load instruction (the scalar form spends about
// 7.5 loads and the index arithmetic around them).  Rows of 4 outputs go out
// as 16-byte stores.  The last sub-step's valid region starts at the aligned
// column HX and is TX wide, so the column groups are aligned.
template <int R, bool STAR>
__device__ __forceinline__ void last_substep2_f32(const float* src, float* __restrict__ out, const Layout2<float>& L,
                                                  int64_t ny, int64_t nx, int64_t ldx, int64_t y0, int64_t x0,
                                                  const Coeffs<float, ipow(2 * R + 1, 2)>& cf) {
    static_assert(R <= 4, "three 16-byte loads cover x-4 .. x+7");
    constexpr int W = 2 * R + 1;
    constexpr int kRS = kVR;   // rows per thread here
    static_assert(Tile2<float>::TY % kRS == 0, "whole strips");
    const int ncg = Tile2<float>::TX / 4;
    const int nstrips = Tile2<float>::TY / kRS;
    const int tid = threadIdx.y * kBX + threadIdx.x;
    for (int item = tid; item < nstrips * ncg; item += kBX * kBYT) {
        const int strip = item / ncg, cgi = item - strip * ncg;   // a warp: consecutive column groups
        const int sy0 = L.H + strip * kRS;
        const int sx = L.HX + 4 * cgi;
        float acc[kRS][4];
#pragma unroll
        for (int j = 0; j < kRS; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[j][q] = 0.0f;
        const float* base = src + (sy0 - R) * L.SX + (sx - 4);
#pragma unroll
        for (int yi = 0; yi < kRS + 2 * R; ++yi) {
            float v[12];   // v[k] = column sx - 4 + k of input row sy0 - R + yi
#pragma unroll
            for (int k4 = 0; k4 < 3; ++k4) {
                const float4 u = *reinterpret_cast<const float4*>(base + yi * L.SX + 4 * k4);
                v[4 * k4] = u.x;
                v[4 * k4 + 1] = u.y;
                v[4 * k4 + 2] = u.z;
                v[4 * k4 + 3] = u.w;
            }
#pragma unroll
            for (int j = 0; j < kRS; ++j) {
                const int a = yi - j;
                if (a >= 0 && a < W) {
#pragma unroll
                    for (int b = 0; b < W; ++b)
                        if (!STAR || a == R || b == R) {
                            const float w = cf.c[a * W + b];
#pragma unroll
                            for (int q = 0; q < 4; ++q) acc[j][q] = fmaf(w, v[4 + q + b - R], acc[j][q]);
                        }
                }
            }
        }
        const int64_t gx = x0 + 4 * cgi;
#pragma unroll
        for (int j = 0; j < kRS; ++j) {
            const int64_t gy = y0 + strip * kRS + j;
            if (gy < ny) {
                float* o = out + gy * ldx + gx;
                if (gx + 3 < nx) {
                    *reinterpret_cast<float4*>(o) = make_float4(acc[j][0], acc[j][1], acc[j][2], acc[j][3]);
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (gx + q < nx) o[q] = acc[j][q];
                }
            }
        }
    }
}

// i mod n; one add or subtract for the usual halo offsets (|i| < 2n).
__device__ __forceinline__ int wrap_fast(int i, int n) {
    if (i >= 0 && i < n) return i;
    if (i < 0 && i >= -n) return i + n;
    if (i >= n && i < 2 * n) return i - n;
    const int m = i % n;
    return m < 0 ? m + n : m;
}

// Periodic boundary, a staged block (SY rows x SX columns, cell (0, 0) =
// grid point (gy0, gx0) of the plane `in`) that crosses the grid's edge: TMA
// filled the cells outside the grid with zeros; the CTA overwrites exactly
// those cells with their wrapped values: the rows outside the grid in full,
// then the columns outside it in the other rows.  Four loads per thread are
// in flight at a time.  The 2D kernel calls it out of line (inlined, it
// raised the register pressure of the whole kernel); in the 3D kernel, whose
// budget is 64 registers, a call cost more spills than the inlined copy.
template <typename T>
__device__ __forceinline__ void wrap_halo_block_inl(T* buf, int SY, int SX, const T* __restrict__ in, int64_t ldx,
                                                    int ny, int nx, int gy0, int gx0) {
    const int top = min(SY, max(0, -gy0));          // rows [0, top) lie above the grid
    const int bot = max(top, min(SY, ny - gy0));     // rows [bot, SY) lie below it
    const int cl = min(SX, max(0, -gx0));           // columns [0, cl) left of it
    const int cr = max(cl, min(SX, nx - gx0));      // columns [cr, SX) right of it
    const int ncx = cl + (SX - cr);                 // outside columns per inside row
    const int n_rows = (top + (SY - bot)) * SX;     // cells of the outside rows
    const int n_all = n_rows + (bot - top) * ncx;
    const int nthr = blockDim.x * blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int i0 = tid; i0 < n_all; i0 += 4 * nthr) {
        T v[4];
        int off[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * nthr;
            off[u] = -1;
            v[u] = T(0);
            if (i < n_all) {
                int sy, sx;
                if (i < n_rows) {
                    const int rr = i / SX;
                    sy = rr < top ? rr : bot + (rr - top);
                    sx = i - rr * SX;
                } else {
                    const int j = i - n_rows, rr = j / ncx, c = j - rr * ncx;
                    sy = top + rr;
                    sx = c < cl ? c : cr + (c - cl);
                }
                off[u] = sy * SX + sx;
                v[u] = in[(int64_t)wrap_fast(gy0 + sy, ny) * ldx + wrap_fast(gx0 + sx, nx)];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (off[u] >= 0) buf[off[u]] = v[u];
    }
}

template <typename T>
__device__ __noinline__ void wrap_halo_block(T* buf, int SY, int SX, const T* __restrict__ in, int64_t ldx, int ny,
                                             int nx, int gy0, int gx0) {
    wrap_halo_block_inl<T>(buf, SY, SX, in, ldx, ny, nx, gy0, gx0);
}

// Register budgets of the persistent kernels: left alone, the compiler keeps
// the coefficients and unrolled sums in registers and one CTA fills an SM.
// (2D: two CTAs of four-stage rings fill the shared memory; r = 4 stars get
// the registers of one CTA, which at two spill some 600 bytes.)
template <typename T, int NDIM>
constexpr int min_ctas() { return sizeof(T) == 4 ? (NDIM == 2 ? 2 : 4) : 2; }

template <typename T, int R, bool STAR>
__global__ void __launch_bounds__(kBX * kBYT, (STAR && R >= 4) ? 1 : min_ctas<T, 2>())
gather2d_tma_kernel(const __grid_constant__ CUtensorMap tin, const G2Args a, const Coeffs<T, ipow(2 * R + 1, 2)> cf) {
    constexpr int TY = Tile2<T>::TY, TX = Tile2<T>::TX;
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char* smem_raw = (unsigned char*)(((uintptr_t)smem_dyn + 127) & ~(uintptr_t)127);
    const Layout2<T> L(R, a.tb);
    constexpr int NST = Tile2<T>::NST;
    T* const stage0 = reinterpret_cast<T*>(smem_raw);
    T* work = stage0 + NST * L.buf;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + (size_t)L.buffers(a.tb) * L.buf * sizeof(T));
    volatile int* abort_flag = reinterpret_cast<volatile int*>(full + NST);
    const int tid = threadIdx.y * kBX + threadIdx.x;
    const T* in = (const T*)a.in;
    T* out = (T*)a.out;
    const uint32_t box_bytes = (uint32_t)(L.SY * L.SX * sizeof(T));
    if (tid == 0) {
        for (int i = 0; i < NST; ++i) ptx::mbar_init(&full[i], 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    __syncthreads();
    // Every tile is staged by TMA; with a periodic boundary, a tile whose
    // staged block crosses the grid's edge then gets its outside cells wrapped.
    auto edge = [&](int t) {
        if (a.bc != kBcPeriodic) return false;
        const int y0 = (t / a.tiles_x) * TY, x0 = (t % a.tiles_x) * TX;
        return !(y0 - L.H >= 0 && y0 + TY + L.H <= a.ny && x0 - L.HX >= 0 && x0 + TX + L.HX <= a.nx);
    };
    // Thread 0 tracks the ring: bit s of `inflight` = a load into stage s not
    // yet waited for, bit s of `phase` = parity of stage s's next completion.
    uint32_t inflight = 0, phase = 0;
    auto issue = [&](int t, int s) {
        if (t >= a.tiles_total) return;
        const int y0 = (t / a.tiles_x) * TY, x0 = (t % a.tiles_x) * TX;
        ptx::mbar_arrive_expect_tx(&full[s], box_bytes);
        ptx::tma_load_2d(stage0 + s * L.buf, &tin, x0 - L.HX, y0 - L.H, &full[s]);
        inflight |= 1u << s;
    };
    const int first = blockIdx.x;
    if (tid == 0)
        for (int i = 0; i < NST - 1; ++i) issue(first + i * (int)gridDim.x, i);
    int k = 0;
    for (int t = first; t < a.tiles_total; t += gridDim.x, ++k) {
        const int s = k % NST;
        T* st_buf = stage0 + s * L.buf;
        // the stage computed at iteration k - 1 is free (barrier at its end);
        // its generic-proxy writes (halo wrap, sub-steps) are ordered
        // before the TMA write that refills it
        if (tid == 0) {
            ptx::fence_proxy_async_smem();
            issue(t + (NST - 1) * (int)gridDim.x, (k + NST - 1) % NST);
        }
        const int64_t y0 = (int64_t)(t / a.tiles_x) * TY, x0 = (int64_t)(t % a.tiles_x) * TX;
        {
            const uint32_t par = (phase >> s) & 1u;   // every thread tracks the parities
            if (!gwait(&full[s], par)) *abort_flag = 1;
            phase ^= 1u << s;
            if (tid == 0) inflight &= ~(1u << s);
        }
        if (edge(t)) {
            __syncthreads();   // every thread has seen the load land (or the abort)
            if (!*abort_flag)
                wrap_halo_block<T>(st_buf, L.SY, L.SX, in, a.ldx, a.ny, a.nx, (int)y0 - L.H, (int)x0 - L.HX);
        }
        __syncthreads();
        if (*abort_flag) break;
        T* src = st_buf;
        for (int st = 1; st <= a.tb; ++st) {
            T* dst = (st & 1) ? work : st_buf;   // sub-steps alternate between the work buffer and the stage
            if constexpr (sizeof(T) == 4) {
                if (st == a.tb)
                    last_substep2_f32<R, STAR>(src, out, L, a.ny, a.nx, a.ldx, y0, x0, cf);
                else
                    substep2<T, R, STAR>(src, dst, out, L, st, false, a.ny, a.nx, a.ldx, a.bc, y0, x0, cf);
            } else {
                substep2<T, R, STAR>(src, dst, out, L, st, st == a.tb, a.ny, a.nx, a.ldx, a.bc, y0, x0, cf);
            }
            src = dst;
            __syncthreads();   // sub-step st is complete (and, after the last, the stage is free)
        }
    }
    if (*abort_flag) {
        // let the loads still in flight land before the CTA gives up its shared memory
        if (tid == 0) {
            for (int s2 = 0; s2 < NST; ++s2)
                if ((inflight >> s2) & 1u) ptx::mbar_wait(&full[s2], (phase >> s2) & 1u, kGatherWait / 8);
            if (a.err) atomicOr(a.err, 2u);
        }
    }
}

// 3D streaming kernel: a work unit is TZC output planes of a TY x TX column;
// its TZC + 2R input planes stream through NPL = 2R + 2 plane buffers.
template <typename T>
struct Tile3 {
    static constexpr int TY = 32;
    static constexpr int TX = 64;
    static constexpr int TZC = 64;
    static constexpr int AL = 16 / (int)sizeof(T);
};
constexpr int kThreads3 = 256;   // (TY / kRS) strips x TX columns

struct G3Args {
    const void* in;
    void* out;
    unsigned int* err;
    int64_t ldx;         // row stride of the grids (elements); planes are ny rows
    int nz, ny, nx, bc;
    int tiles_x, tiles_y, chunks, units;
};

template <typename T, int R>
struct Layout3 {
    static constexpr int NPL = 2 * R + 2;
    static constexpr int HX = round_up(R, Tile3<T>::AL);
    static constexpr int SY = Tile3<T>::TY + 2 * R;
    static constexpr int SX = Tile3<T>::TX + 2 * HX;
    static constexpr int PLANE = round_up(SY * SX, 128 / (int)sizeof(T));
    static constexpr size_t bytes() { return (size_t)NPL * PLANE * sizeof(T) + 8 * NPL + 16 + 128; }
};

template <typename T, int R, bool STAR>
__global__ void __launch_bounds__(kThreads3, min_ctas<T, 3>())
gather3d_stream_kernel(const __grid_constant__ CUtensorMap tin, const G3Args a, const Coeffs<T, ipow(2 * R + 1, 3)> cf) {
    using L = Layout3<T, R>;
    constexpr int W = 2 * R + 1, TY = Tile3<T>::TY, TX = Tile3<T>::TX, TZC = Tile3<T>::TZC, NPL = L::NPL;
    static_assert(TX * (TY / kRS) == kThreads3, "one strip per thread");
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char* smem_raw = (unsigned char*)(((uintptr_t)smem_dyn + 127) & ~(uintptr_t)127);
    T* planes = reinterpret_cast<T*>(smem_raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + (size_t)NPL * L::PLANE * sizeof(T));
    volatile int* abort_flag = reinterpret_cast<volatile int*>(full + NPL);
    const int tid = threadIdx.x;
    const T* in = (const T*)a.in;
    T* out = (T*)a.out;
    constexpr uint32_t box_bytes = (uint32_t)(L::SY * L::SX * sizeof(T));
    if (tid == 0) {
        for (int b = 0; b < NPL; ++b) ptx::mbar_init(&full[b], 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    __syncthreads();
    int uses[NPL];   // TMA loads into each plane buffer so far (mbarrier phases)
#pragma unroll
    for (int b = 0; b < NPL; ++b) uses[b] = 0;
    const int col = tid % TX;            // output column of this thread
    const int sy0 = (tid / TX) * kRS;    // first output row of its strip
    unsigned int in_flight = 0;          // buffers with a TMA load nobody waited for yet (bit mask)
    for (int u = blockIdx.x; u < a.units && !*abort_flag; u += gridDim.x) {
        const int tx_ = u % a.tiles_x, ty_ = (u / a.tiles_x) % a.tiles_y, tz_ = u / (a.tiles_x * a.tiles_y);
        const int x0 = tx_ * TX, y0 = ty_ * TY, z0 = tz_ * TZC;
        const int nout = min(TZC, a.nz - z0);
        // with a periodic boundary, an edge unit's planes (staged by TMA like
        // the others, from the wrapped plane index) get their cells outside
        // the grid in y and x wrapped once they have landed
        const bool edge = a.bc == kBcPeriodic &&
                          !(y0 - R >= 0 && y0 + TY + R <= a.ny && x0 - L::HX >= 0 && x0 + TX + L::HX <= a.nx);
        // input plane i of the unit is grid plane z0 - R + i, held in buffer i % NPL
        auto load = [&](int i) {
            const int b = i % NPL;
            int gz = z0 - R + i;
            if (a.bc == kBcPeriodic) gz = (int)wrap_index(gz, a.nz);
            if (tid == 0) {
                ptx::fence_proxy_async_smem();   // after the fix-ups of the plane it replaces
                ptx::mbar_arrive_expect_tx(&full[b], box_bytes);
                ptx::tma_load_3d(planes + b * L::PLANE, &tin, x0 - L::HX, y0 - R, gz, &full[b]);
            }
            in_flight |= 1u << b;
        };
        auto ready = [&](int i) {   // input plane i is in its buffer
            const int b = i % NPL;
            if (!gwait(&full[b], (uint32_t)(uses[b] & 1))) *abort_flag = 1;
            ++uses[b];
            in_flight &= ~(1u << b);
        };
        auto wrap_plane = [&](int i) {
            int gz = z0 - R + i;
            gz = (int)wrap_index(gz, a.nz);
            wrap_halo_block_inl<T>(planes + (i % NPL) * L::PLANE, L::SY, L::SX, in + (int64_t)gz * a.ny * a.ldx,
                                   a.ldx, a.ny, a.nx, y0 - R, x0 - L::HX);
        };
        const int nin = nout + 2 * R;
        for (int i = 0; i < NPL && i < nin; ++i) load(i);
        for (int o = 0; o < nout; ++o) {
            const int i_lo = o == 0 ? 0 : o + 2 * R;   // planes that land now
            for (int i = i_lo; i <= o + 2 * R; ++i) ready(i);
            if (edge) {
                __syncthreads();   // every thread has seen the planes land (or the abort)
                if (*abort_flag) break;
                for (int i = i_lo; i <= o + 2 * R; ++i) wrap_plane(i);
            }
            __syncthreads();
            if (*abort_flag) break;
            // output plane z0 + o from input planes o .. o + 2R
            T acc[kRS];
#pragma unroll
            for (int j = 0; j < kRS; ++j) acc[j] = T(0);
            const int sx = L::HX + col;
#pragma unroll
            for (int dz = 0; dz < W; ++dz) {
                const T* pl = planes + ((o + dz) % NPL) * L::PLANE;
                if (STAR && dz != R) {
                    const T w = cf.c[(dz * W + R) * W + R];
#pragma unroll
                    for (int j = 0; j < kRS; ++j) acc[j] = fma(w, pl[(sy0 + R + j) * L::SX + sx], acc[j]);
                } else {
                    const T* base = pl + sy0 * L::SX + (sx - R);
#pragma unroll
                    for (int yi = 0; yi < kRS + 2 * R; ++yi) {
                        T v[W];
#pragma unroll
                        for (int b = 0; b < W; ++b) v[b] = base[yi * L::SX + b];
#pragma unroll
                        for (int j = 0; j < kRS; ++j) {
                            const int a1 = yi - j;
                            if (a1 >= 0 && a1 < W) {
#pragma unroll
                                for (int b = 0; b < W; ++b)
                                    if (!STAR || a1 == R || b == R)
                                        acc[j] = fma(cf.c[(dz * W + a1) * W + b], v[b], acc[j]);
                            }
                        }
                    }
                }
            }
            const int64_t gz = z0 + o, gx = x0 + col;
            if (gx < a.nx) {
#pragma unroll
                for (int j = 0; j < kRS; ++j) {
                    const int64_t gy = y0 + sy0 + j;
                    if (gy < a.ny) out[(gz * a.ny + gy) * a.ldx + gx] = acc[j];
                }
            }
            __syncthreads();   // input plane o is no longer needed: its buffer takes plane o + NPL
            if (o + NPL < nin) load(o + NPL);
        }
        // planes loaded but not needed (short last chunk) are waited for before reuse
        for (int b = 0; b < NPL; ++b)
            if (in_flight & (1u << b)) {
                if (!gwait(&full[b], (uint32_t)(uses[b] & 1))) *abort_flag = 1;
                ++uses[b];
            }
        in_flight = 0;
        __syncthreads();
    }
    if (*abort_flag) {
        if (tid == 0) {
            for (int b = 0; b < NPL; ++b)
                if (in_flight & (1u << b)) ptx::mbar_wait(&full[b], (uint32_t)(uses[b] & 1), kGatherWait / 8);
            if (a.err) atomicOr(a.err, 2u);
        }
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
cudaError_t launch2d_tiles(const GatherProblem& p, const void* in, void* out, int tb, cudaStream_t s) {
    constexpr int NC = ipow(2 * R + 1, 2);
    Coeffs<T, NC> cf;
    for (int i = 0; i < NC; ++i) cf.c[i] = (T)p.cg[i];
    const size_t smem = gather_smem_bytes_t<T>(2, R, tb);
    auto kern = gather2d_kernel<T, R, STAR, k2BY, k2TX, k2TY>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((p.n[1] + k2TX - 1) / k2TX), (unsigned)((p.n[0] + k2TY - 1) / k2TY));
    kern<<<grid, dim3(kBX, k2BY), smem, s>>>((const T*)in, (T*)out, p.n[0], p.n[1], p.ldx, p.bc, tb, cf);
    return cudaGetLastError();
}

template <typename T, int R, bool STAR>
cudaError_t launch3d_tiles(const GatherProblem& p, const void* in, void* out, int tb, cudaStream_t s) {
    constexpr int NC = ipow(2 * R + 1, 3);
    Coeffs<T, NC> cf;
    for (int i = 0; i < NC; ++i) cf.c[i] = (T)p.cg[i];
    const size_t smem = gather_smem_bytes_t<T>(3, R, tb);
    auto kern = gather3d_kernel<T, R, STAR, k3BY, k3TX, k3TY, k3TZ>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((p.n[2] + k3TX - 1) / k3TX), (unsigned)((p.n[1] + k3TY - 1) / k3TY),
              (unsigned)((p.n[0] + k3TZ - 1) / k3TZ));
    kern<<<grid, dim3(kBX, k3BY), smem, s>>>((const T*)in, (T*)out, p.n[0], p.n[1], p.n[2], p.ldx, p.bc, tb, cf);
    return cudaGetLastError();
}

int max_smem_optin() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

int sm_count() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v;
}

// TMA tiled view of a C-order grid: dims (innermost first) and element type;
// false when the driver entry point is missing or the encoder rejects it.
template <typename T>
bool encode_grid_map(CUtensorMap* map, const void* base, int rank, const cuuint64_t* dims, int64_t ldx,
                     const cuuint32_t* box) {
    auto enc = mxu::get_encode();
    if (!enc) return false;
    cuuint64_t strides[2];   // rows of ldx elements; planes of dims[1] rows
    strides[0] = (cuuint64_t)ldx * sizeof(T);
    if (rank == 3) strides[1] = strides[0] * dims[1];
    cuuint32_t es[3] = {1, 1, 1};
    return enc(map, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, rank,
               const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The TMA kernels need 16-byte aligned grid bases and rows.
template <typename T>
bool tma_layout_ok(const GatherProblem& p, const void* in) {
    return ((uintptr_t)in & 15u) == 0 && (p.ldx * (int64_t)sizeof(T)) % 16 == 0;
}

template <typename T, int R, bool STAR>
cudaError_t launch2d(const GatherProblem& p, const void* in, void* out, int tb, cudaStream_t s) {
    const Layout2<T> L(R, tb);
    const size_t smem = L.bytes(tb);
    if (!tma_layout_ok<T>(p, in) || smem > (size_t)max_smem_optin() || L.SX > 256 || L.SY > 256)
        return launch2d_tiles<T, R, STAR>(p, in, out, tb, s);
    constexpr int NC = ipow(2 * R + 1, 2);
    Coeffs<T, NC> cf;
    for (int i = 0; i < NC; ++i) cf.c[i] = (T)p.cg[i];
    G2Args a;
    a.in = in;
    a.out = out;
    a.err = p.err;
    a.ldx = p.ldx;
    a.ny = (int)p.n[0];
    a.nx = (int)p.n[1];
    a.bc = p.bc;
    a.tb = tb;
    a.tiles_x = (a.nx + Tile2<T>::TX - 1) / Tile2<T>::TX;
    a.tiles_total = a.tiles_x * ((a.ny + Tile2<T>::TY - 1) / Tile2<T>::TY);
    alignas(64) CUtensorMap tin;
    const cuuint64_t dims[2] = {(cuuint64_t)a.nx, (cuuint64_t)a.ny};
    const cuuint32_t box[2] = {(cuuint32_t)L.SX, (cuuint32_t)L.SY};
    if (!encode_grid_map<T>(&tin, in, 2, dims, p.ldx, box)) return cudaErrorInvalidValue;
    auto kern = gather2d_tma_kernel<T, R, STAR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kBX * kBYT, smem);
    if (e != cudaSuccess) return e;
    int grid = sm_count() * (per > 0 ? per : 1);
    if (grid > a.tiles_total) grid = a.tiles_total;
    kern<<<grid, dim3(kBX, kBYT), smem, s>>>(tin, a, cf);
    return cudaGetLastError();
}

template <typename T, int R, bool STAR>
cudaError_t launch3d(const GatherProblem& p, const void* in, void* out, int tb, cudaStream_t s) {
    using L = Layout3<T, R>;
    const size_t smem = L::bytes();
    if (tb != 1 || !tma_layout_ok<T>(p, in) || smem > (size_t)max_smem_optin() || L::SX > 256 || L::SY > 256)
        return launch3d_tiles<T, R, STAR>(p, in, out, tb, s);
    constexpr int NC = ipow(2 * R + 1, 3);
    Coeffs<T, NC> cf;
    for (int i = 0; i < NC; ++i) cf.c[i] = (T)p.cg[i];
    G3Args a;
    a.in = in;
    a.out = out;
    a.err = p.err;
    a.ldx = p.ldx;
    a.nz = (int)p.n[0];
    a.ny = (int)p.n[1];
    a.nx = (int)p.n[2];
    a.bc = p.bc;
    a.tiles_x = (a.nx + Tile3<T>::TX - 1) / Tile3<T>::TX;
    a.tiles_y = (a.ny + Tile3<T>::TY - 1) / Tile3<T>::TY;
    a.chunks = (a.nz + Tile3<T>::TZC - 1) / Tile3<T>::TZC;
    a.units = a.tiles_x * a.tiles_y * a.chunks;
    alignas(64) CUtensorMap tin;
    const cuuint64_t dims[3] = {(cuuint64_t)a.nx, (cuuint64_t)a.ny, (cuuint64_t)a.nz};
    const cuuint32_t box[3] = {(cuuint32_t)L::SX, (cuuint32_t)L::SY, 1};
    if (!encode_grid_map<T>(&tin, in, 3, dims, p.ldx, box)) return cudaErrorInvalidValue;
    auto kern = gather3d_stream_kernel<T, R, STAR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kThreads3, smem);
    if (e != cudaSuccess) return e;
    int grid = sm_count() * (per > 0 ? per : 1);
    if (grid > a.units) grid = a.units;
    kern<<<grid, kThreads3, smem, s>>>(tin, a, cf);
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
