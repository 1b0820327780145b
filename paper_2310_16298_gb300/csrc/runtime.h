// Internal runtime structures shared by the host-side translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/stencil.h"
#include "common.cuh"
#include "kernels.h"
#include "mx.h"

// A plan (opaque to callers): the validated problem, the chosen kernel and
// the device memory the plan owns.
struct stencil_plan_s {
    int ndim = 0;
    int64_t n[3] = {1, 1, 1};
    int r = 0;
    bool star = false;
    bool f64 = false;
    int bc = stx::kBcDirichlet;
    std::vector<double> cg;
    int impl = STENCIL_IMPL_GATHER;
    int prec = STENCIL_PREC_NATIVE;
    int tb = 1;
    int device = 0;
    int64_t points = 0;
    size_t grid_bytes = 0;
    void* scratch = nullptr;
    int64_t pitch = 0;              // row stride of the caller's grids (elements)
    int64_t ldx = 0;                // row stride of the grids the kernels see (elements)
    bool repack = false;            // caller rows are not 16-byte multiples: the kernels run on
                                    // padded copies (pad, scratch) of row stride ldx
    void* pad = nullptr;            // first padded grid (repack only)
    size_t pad_bytes = 0;           // bytes of one padded grid
    cudaStream_t stream = nullptr;  // for stencil_submit
    stx::MxPlan* mx = nullptr;
    uint64_t id = 0;                // unique per plan (tickets refer to plans by id)
    unsigned int host_error = 0;    // error bits raised on the host (stencil_plan_raise_error)
    void* staging = nullptr;        // device grid of stencil_apply_host (allocated on first use)
    unsigned int* err_host = nullptr;  // host-mapped error word of the gather kernels' bounded waits
    unsigned int* err_dev = nullptr;
};


namespace stx {

// Record a failure message for stencil_last_error() and return `st`.
stencil_status fail(stencil_status st, const std::string& msg);
stencil_status cuda_fail(cudaError_t e, const char* what);
const std::string& last_error_string();

GatherProblem gather_problem(const stencil_plan_s* p);
cudaError_t run_sweep(const stencil_plan_s* p, const void* src, void* dst, int tb, cudaStream_t s);
// Advance d_in by `steps` into d_out on stream s, ping-ponging through `scratch`.
stencil_status time_loop(const stencil_plan_s* p, const void* d_in, void* d_out, int64_t steps, cudaStream_t s,
                         void* scratch);

// Error bits of a plan: a kernel that gave up a bounded wait (the host-mapped
// word of the matrixized kernels) or bits raised on the host.  Sticky until
// the plan is destroyed.
unsigned int plan_error_bits(const stencil_plan_s* p);
// STENCIL_OK, or STENCIL_ECUDA with a message naming `where`, when the plan's
// error bits are set.
stencil_status plan_error_status(const stencil_plan_s* p, const char* where);

}  // namespace stx
