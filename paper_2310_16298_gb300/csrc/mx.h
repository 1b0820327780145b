// Internal interface of the matrixized (outer-product) kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/stencil.h"

namespace stx {

struct MxRequest {
    int ndim = 2;
    int64_t n[3] = {1, 1, 1};
    int r = 1;
    bool star = false;
    bool f64 = false;
    int bc = 0;
    const double* cg = nullptr;  // host, dense C^g
    int prec = STENCIL_PREC_TF32X3;
    int tb = 0;                   // 0 = library choice
    int cover = 0;                // stencil_cover (stars only)
    int64_t ldx = 0;              // row stride of the grids the kernels see (elements)
    int unit_planes = 0;          // 3D: output planes per work unit (0 = library choice)
};

struct MxPlan {
    int ndim = 2;
    int64_t n[3] = {1, 1, 1};
    int64_t ldx = 0;      // row stride of the grids the kernels read and write (elements)
    int r = 1;
    int bc = 0;
    int prec = STENCIL_PREC_TF32X3;
    int tb = 1;
    int nb = 16;          // output columns per MMA block
    int n_lines = 0;      // lines on the tensor cores
    int n_scalar = 0;     // weights applied on CUDA cores
    int cover = STENCIL_COVER_PARALLEL;   // line cover the plan runs
    int unit_planes = 0;  // 3D: output planes per work unit (0 = library choice)
    size_t operand_bytes = 0;
    void* d_operands = nullptr;  // banded line operands (device), kernel-specific layout
    void* d_scalars = nullptr;   // scalar-term table (device)
    void* tmap_storage = nullptr;
    int n_edge_terms = 0;                    // periodic boundary terms of the edge kernel
    std::vector<unsigned char> edge_table;   // its parameter block (edges.cu)
};

bool mx_supported(const MxRequest& q, std::string* why);

// 3D kernels (mx3d.cu); the mx_* entry points dispatch to them for ndim == 3.
bool mx3d_supported(const MxRequest& q, std::string* why);
stencil_status mx3d_plan_build(const MxRequest& q, MxPlan* p, std::string* why);
void mx3d_plan_free(MxPlan* p);
cudaError_t mx3d_sweep(const MxPlan& p, const void* src, void* dst, int tb, cudaStream_t s);
unsigned int mx3d_device_error(const MxPlan& p);
stencil_status mx_plan_build(const MxRequest& q, MxPlan* p, std::string* why);
cudaError_t mx2d_sweep(const MxPlan& p, const void* src, void* dst, int tb, cudaStream_t s);

// Periodic boundary (edges.cu): the tensor-core kernels see a zero halo in x
// and y; mx_periodic_edges adds the wrapped terms of the points within r of an
// x or y face to dst (a no-op for other plans).  mx_edges_build makes the
// table of nonzero weights with a nonzero y or x offset that it passes.
stencil_status mx_edges_build(const MxRequest& q, MxPlan* p);
cudaError_t mx_periodic_edges(const MxPlan& p, const void* src, void* dst, cudaStream_t s);
void mx_plan_free(MxPlan* p);
cudaError_t mx_sweep(const MxPlan& p, const void* src, void* dst, int tb, cudaStream_t s);
// Nonzero when a kernel of this plan gave up a bounded wait (bit 0: operand
// staging, bit 1: tensor-core completion).
unsigned int mx_device_error(const MxPlan& p);

}  // namespace stx
