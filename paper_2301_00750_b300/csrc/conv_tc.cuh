// Tensor-core (tcgen05) implicit-GEMM convolution: plan and launch interface.
#pragma once

#include "common.cuh"

struct tc_stream;

namespace tc {

// A planned launch of the tensor-core conv for one layer.  Planning encodes the TMA
// descriptors of the input activations and the packed weights; launches reuse them.
struct TcConvPlan {
    bool enabled = false;
};

// Returns false (plan disabled) when the layer is not eligible.
bool tc_plan_conv(TcConvPlan &plan, const ConvArgs &a, bool tma_in);
cudaError_t launch_conv_tc(const TcConvPlan &plan, const ConvArgs &a, cudaStream_t st);

}  // namespace tc

// Plans the tensor-core convs of a BF16 stream (no-op when not available).
int tc_prepare_tensor_core_path(tc_stream *s);
