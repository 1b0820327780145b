// Periodic boundary terms of the matrixized sweeps.
//
// The tensor-core kernels load their tiles through TMA, which fills rows and
// columns outside the grid with zeros: on their own they compute the sweep of
// Eq. (stencil-2d9p) with a zero halo in x and y (the 3D kernel wraps whole
// planes in z itself, by loading plane (z + dz) mod nz).  Under the periodic
// boundary, each output point within r of an x or y face misses the terms
// whose neighbour lies across that face.  This kernel adds them afterwards,
//   out[z][y][x] += sum over (dz, dy, dx) with y + dy or x + dx outside the
//                   grid of  C[dz][dy][dx] * in[(z+dz) mod nz][(y+dy) mod ny][(x+dx) mod nx],
// in FP32, which is the rest of the periodic sum (the sum is linear in the
// neighbours, so splitting it into the in-grid and the wrapped terms changes
// only the rounding order).  Only the boundary strips are touched: rows within
// r of a y face in full, the 2r edge columns of every other row.
//
// Kept out of the tensor-core kernels: wrap-around fix-ups inside their split
// warps (which turn staged rows into operand parts) put global-memory
// latency on the critical path of every edge tile, and slowed the 2D sweep by
// up to a half and the 3D sweep up to fourfold; here the boundary costs one
// short launch over about 2 r (nx + ny) nz points, one thread per point.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string.h>

#include <vector>

#include "common.cuh"
#include "mx.h"
#include "ptx.cuh"

namespace stx {

namespace {

constexpr int kMaxEdgeTerms = 120;   // 2D r = 4: (2r+1)^2 - 1 = 80; 3D r = 2 box: (2r+1)^3 - (2r+1) = 120

struct EdgeTerm {
    int8_t dz, dy, dx, pad;
    float w;
};

// The nonzero weights with a nonzero y or x offset, twice: tx sorted by x
// offset, ty by y offset.  firstx[d + r] (firsty[d + r]) = index of the first
// term of tx (ty) with x (y) offset >= d, d = -r .. r + 1, so the terms whose
// neighbour leaves the grid across one face are a prefix or a suffix.  Passed
// by value (kernel parameter space, read through the constant cache).
struct EdgeTable {
    int n;
    int firstx[2 * 4 + 2];
    int firsty[2 * 4 + 2];
    EdgeTerm tx[kMaxEdgeTerms];
    EdgeTerm ty[kMaxEdgeTerms];
};

// i mod n for -n <= i < 2n: a plan's extents are at least 2r + 1, so a
// neighbour offset (|d| <= r) wraps at most once.
__device__ __forceinline__ int wrap1(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// One thread per boundary point of plane blockIdx.y.  Per plane, points
// 0 .. fr*nx-1 lie on the full rows (within r of a y face), the rest on the
// ec edge columns of the other rows.  A point visits exactly the terms whose
// neighbour lies outside the grid, as up to four segments of the term lists:
// dy < -y (a prefix of ty), dy >= ny - y (a suffix of ty), and, near an x
// face, dx < -x or dx >= nx - x (of tx; those whose y + dy also leaves the
// grid were taken with ty).  Eight terms at a time: a chunk's loads are all
// issued before the first is used.  The point's own output value is loaded
// first.  One copy of the chunk code serves all segments (the kernel is short
// lived, so its instruction footprint is part of its latency).
__global__ void __launch_bounds__(128) periodic_edges_kernel(const float* __restrict__ in, float* __restrict__ out,
                                                             int nz, int ny, int nx, int64_t ldx, int r,
                                                             const __grid_constant__ EdgeTable tab) {
    constexpr int C = 8;
    const int fr = ny <= 2 * r ? ny : 2 * r;   // full rows per plane
    const int ec = nx <= 2 * r ? nx : 2 * r;   // edge columns per other row
    const int na = fr * nx;
    const int per_plane = na + (ny - fr) * ec;
    const int z = blockIdx.y;
    // launched as a programmatic dependent of the tensor-core kernel: let the
    // next sweep's kernel start its set-up, then wait until the tensor-core
    // grid has completed and its writes are visible
    ptx::launch_dependents();
    ptx::grid_dependency_wait();
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < per_plane; p += gridDim.x * blockDim.x) {
        int y, x;
        if (p < na) {
            const int f = p / nx;
            x = p - f * nx;
            y = ny <= 2 * r ? f : (f < r ? f : ny - 2 * r + f);
        } else {
            const int q = p - na;
            const int b = q / ec;
            const int c = q - b * ec;
            y = r + b;
            x = nx <= 2 * r ? c : (c < r ? c : nx - 2 * r + c);
        }
        float* o = out + ((int64_t)z * ny + y) * ldx + x;
        const float o0 = *o;
        const bool y_edge = y < r || y >= ny - r;
        const bool x_edge = x < r || x >= nx - r;
        float acc = 0.0f;
        for (int sg = 0; sg < 4; ++sg) {
            const bool by_x = sg >= 2;
            if (by_x ? !x_edge : !y_edge) continue;
            const int u = by_x ? x : y, nu = by_x ? nx : ny;
            const int* first = by_x ? tab.firstx : tab.firsty;
            const int t0 = (sg & 1) ? first[min(nu - u, r + 1) + r] : 0;
            const int t1 = (sg & 1) ? tab.n : first[max(-u, -r) + r];
            const EdgeTerm* terms = by_x ? tab.tx : tab.ty;
            for (int c = t0; c < t1; c += C) {
                float v[C];
#pragma unroll
                for (int k = 0; k < C; ++k) {
                    const EdgeTerm e = terms[min(c + k, kMaxEdgeTerms - 1)];
                    const int yy = y + e.dy;
                    // x segments skip the terms the y segments took
                    const bool use = c + k < t1 && !(by_x && y_edge && (yy < 0 || yy >= ny));
                    const int64_t off = ((int64_t)wrap1(z + e.dz, nz) * ny + wrap1(yy, ny)) * ldx + wrap1(x + e.dx, nx);
                    v[k] = use ? __ldg(in + off) : 0.0f;
                }
#pragma unroll
                for (int k = 0; k < C; ++k) acc = fmaf(terms[min(c + k, kMaxEdgeTerms - 1)].w, v[k], acc);
            }
        }
        *o = o0 + acc;
    }
}

static_assert(sizeof(EdgeTable) <= 4096, "kernel parameter size");

}  // namespace

stencil_status mx_edges_build(const MxRequest& q, MxPlan* p) {
    p->n_edge_terms = 0;
    p->edge_table.clear();
    if (q.bc != kBcPeriodic) return STENCIL_OK;
    if (q.r > 4) return STENCIL_EUNSUPPORTED;
    const int W = 2 * q.r + 1;
    const int WZ = q.ndim == 3 ? W : 1;
    EdgeTable tab;
    memset(&tab, 0, sizeof(tab));
    for (int c = 0; c < W; ++c)   // tx: sorted by x offset
        for (int a = 0; a < WZ; ++a)
            for (int b = 0; b < W; ++b) {
                const double w = q.cg[((size_t)a * W + b) * W + c];
                const int dz = q.ndim == 3 ? a - q.r : 0, dy = b - q.r, dx = c - q.r;
                // terms with dy = dx = 0 never leave the grid in x or y
                if (w == 0.0 || (dy == 0 && dx == 0)) continue;
                if (tab.n == kMaxEdgeTerms) return STENCIL_EUNSUPPORTED;
                tab.tx[tab.n++] = {(int8_t)dz, (int8_t)dy, (int8_t)dx, 0, (float)w};
            }
    if (tab.n == 0) return STENCIL_OK;
    // ty: the same terms sorted by y offset (stable)
    int k = 0;
    for (int dy = -q.r; dy <= q.r; ++dy)
        for (int t = 0; t < tab.n; ++t)
            if (tab.tx[t].dy == dy) tab.ty[k++] = tab.tx[t];
    for (int d = -q.r; d <= q.r + 1; ++d) {
        int kx = 0, ky = 0;
        while (kx < tab.n && tab.tx[kx].dx < d) ++kx;
        while (ky < tab.n && tab.ty[ky].dy < d) ++ky;
        tab.firstx[d + q.r] = kx;
        tab.firsty[d + q.r] = ky;
    }
    p->n_edge_terms = tab.n;
    p->edge_table.assign((const unsigned char*)&tab, (const unsigned char*)&tab + sizeof(tab));
    return STENCIL_OK;
}

cudaError_t mx_periodic_edges(const MxPlan& p, const void* src, void* dst, cudaStream_t s) {
    if (p.bc != kBcPeriodic || p.n_edge_terms == 0) return cudaSuccess;
    if (p.edge_table.size() != sizeof(EdgeTable)) return cudaErrorInvalidValue;
    const int nz = p.ndim == 3 ? (int)p.n[0] : 1;
    const int ny = (int)p.n[p.ndim - 2], nx = (int)p.n[p.ndim - 1];
    const int fr = ny <= 2 * p.r ? ny : 2 * p.r;
    const int ec = nx <= 2 * p.r ? nx : 2 * p.r;
    const int64_t per_plane = (int64_t)fr * nx + (int64_t)(ny - fr) * ec;
    if (per_plane > INT32_MAX || nz > 65535) return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // enough blocks to fill the GPU, each thread at most a few points
    const int64_t want = (per_plane + 127) / 128;
    const int64_t cap = ((int64_t)sms * 16 + nz - 1) / nz;
    const dim3 grid((unsigned)(want < cap ? want : (cap > 0 ? cap : 1)), (unsigned)nz);
    EdgeTable tab;
    memcpy(&tab, p.edge_table.data(), sizeof(tab));
    // programmatic dependent: the launch is processed while the tensor-core
    // kernel drains (about 2 us per sweep)
    return launch_dependent(periodic_edges_kernel, grid, dim3(128), 0, s, (const float*)src, (float*)dst, nz, ny, nx,
                            p.ldx, p.r, tab);
}

}  // namespace stx
