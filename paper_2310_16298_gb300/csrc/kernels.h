// Internal interface between the host runtime (api.cu) and the kernel files.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace stx {

// A single-grid problem as the gather kernels see it.
struct GatherProblem {
    int ndim;          // 2 or 3
    int64_t n[3];      // interior extents, slowest first
    int r;             // order (radius)
    bool star;         // only on-axis coefficients are nonzero
    bool f64;          // storage/compute type FP64 (else FP32)
    int bc;            // kBcDirichlet | kBcPeriodic
    const double* cg;  // host: dense C^g, (2r+1)^ndim, gather orientation
    int64_t ldx = 0;   // row stride of the grids (elements); planes are n[ndim-2] rows
    unsigned int* err = nullptr;  // device view of the plan's host-mapped error word (bounded waits)
};

// Advance `in` by `tb` time steps into `out` (distinct buffers).
cudaError_t gather_sweep(const GatherProblem& p, const void* in, void* out, int tb, cudaStream_t s);
size_t gather_smem_bytes(const GatherProblem& p, int tb);

// One problem of a batched launch (2D).
struct BatchProblem {
    const void* src;  // input grid of this launch
    void* dst;        // output grid of this launch
    int ny, nx;       // interior extents
    int depth;        // time steps this launch advances the problem (>= 1)
    int bc;           // kBcDirichlet | kBcPeriodic
    int tiles_x;      // output tiles along x
    int tile0;        // index of the problem's first tile in the launch
    int coef_index;   // row of the coefficient table
    int pad;
};

// Advance every listed problem by its depth in one persistent launch with
// batch tile shape `shape` (0 .. gather_batch_shapes()-1).
// d_probs: device array sorted by tile0; d_coef: (2r+1)^2 entries per row.
cudaError_t gather_batch_sweep(bool f64, bool star, int r, const BatchProblem* d_probs, int nprob, int total_tiles,
                               const void* d_coef, int max_tb, int shape, cudaStream_t s);
int gather_batch_shapes();
// Output tile (rows, columns) and shared memory of a batch tile shape.
void gather_batch_tile_shape(int shape, int* ty, int* tx);
size_t gather_batch_smem_bytes(bool f64, int r, int tb, int shape);

// Uniform[lo, hi) SplitMix64 field (elements offset .. offset+count-1 of the
// seed's stream), rounded to the storage type.
cudaError_t fill_uniform(void* out, bool f64, int64_t count, uint64_t seed, int64_t offset, double lo, double hi,
                         cudaStream_t s);

// FP64 error norms: out4 (device) = {sum d^2, sum ref^2, max|d|, max|ref|}.
// `partials` is device scratch of norms_partials_bytes() bytes.
size_t norms_partials_bytes();
cudaError_t error_norms(const void* got, bool got_f64, const double* ref, int64_t count,
                        double* partials, double* out4, cudaStream_t s);

}  // namespace stx
