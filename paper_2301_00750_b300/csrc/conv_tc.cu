// Tensor-core (tcgen05) implicit-GEMM convolution.
#include "conv_tc.cuh"

namespace tc {

bool tc_plan_conv(TcConvPlan &plan, const ConvArgs &, bool) {
    plan.enabled = false;
    return false;
}

cudaError_t launch_conv_tc(const TcConvPlan &, const ConvArgs &, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace tc

int tc_prepare_tensor_core_path(tc_stream *) { return 0; }
