// Matrixized outer-product kernels (tcgen05).  Placeholder until the kernels land.
#include "mx.h"

namespace stx {

bool mx_supported(const MxRequest&, std::string* why) {
    if (why) *why = "no matrixized kernel built yet";
    return false;
}

stencil_status mx_plan_build(const MxRequest&, MxPlan*, std::string* why) {
    if (why) *why = "no matrixized kernel built yet";
    return STENCIL_EUNSUPPORTED;
}

void mx_plan_free(MxPlan*) {}

cudaError_t mx_sweep(const MxPlan&, const void*, void*, int, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace stx
