// Tensor-core (tcgen05) implicit-GEMM 3x3 convolution: plan and launch interface.
#pragma once

#include <cuda.h>

#include <string>
#include <vector>

#include "common.cuh"

namespace tc {

// A planned tensor-core conv for one layer.  Planning packs the weights to bfloat16, half
// or e4m3 [9][cout][nch * kc] on the device and encodes the TMA descriptors of the input
// activations (covering all n_in images of the buffer) and of the weights.
struct TcConvPlan {
    bool enabled = false;
    bool head = false;  // flow-head plan (float flow output, see tc_plan_head)
    bool f8 = false;    // e4m3 operands (kind::f8f6f4) instead of bf16
    bool f16 = false;   // IEEE half operands and outputs instead of bf16 (kind::f16, same rate)
    CUtensorMap tmA;  // 64-byte aligned type
    CUtensorMap tmB;
    // stride-1 3x3 layers whose last 128-byte channel step holds at most 64 bytes: that step
    // (the tail) is taken as 64-byte rows with the 64-byte swizzle, through these maps
    CUtensorMap tmA2;
    CUtensorMap tmB2;
    bool tail = false;
    int bn = 0, nch = 0, stride = 1, h = 0, w = 0, ho = 0, wo = 0, n_in = 0, cout = 0;
    int kc = 0, rb = 0;  // channels and bytes of one K step (rb = 32, 64 or 128: the swizzle span)
    int taps = 9;        // 9: 3x3 conv; 1: pointwise 1x1 conv
    const void *in_base = nullptr;  // start of the buffer the A descriptor covers
    size_t img_bytes = 0;           // bytes between consecutive images of that buffer
    void *wpk = nullptr;            // packed weights (owned by the plan)
    size_t wpk_bytes = 0;
    float *wscale = nullptr;        // e4m3: per-output-channel weight scales (owned)
    int *err = nullptr;             // device error word shared by the stream (not owned)
    void release();
};

// Plans the conv described by `a` (a.in = first image of a buffer holding n_in images of
// a.h x a.w pixels with pixel stride a.in_cs channels; channels [0, a.cin) of each pixel are
// read).  wk_simt: float weights [9 * a.cin][a.cout] (k = tap * cin + c), already in the
// buffer's channel order.  Returns false with `why` when the layer is not eligible (then
// the caller uses the CUDA-core kernel).
// f8: e4m3 operands; wk_simt then holds the weights with the input activations' scales
// already folded in (w[o][c] * s_in[c]); the epilogue multiplies by the per-output-channel
// weight scale and quantizes with a.q_out.
// taps = 1 plans a pointwise 1x1 conv (stride 1; wk_simt then holds [a.cin][a.cout]).
// f16: half operands (weights packed to half, activations read and written as half)
// instead of bfloat16; ignored with f8.
bool tc_plan_conv(TcConvPlan &plan, const ConvArgs &a, int n_in, const std::vector<float> &wk_simt, int *err,
                  std::string &why, bool f8 = false, int taps = 9, bool f16 = false);

// Plans the flow head (cout <= 16, no activation; in practice 2) on the tensor cores: the
// weights are zero-padded to 16 outputs for the MMA.
bool tc_plan_head(TcConvPlan &plan, const ConvArgs &a, int n_in, const std::vector<float> &wk_simt, int *err,
                  std::string &why, bool f8 = false, int taps = 9, bool f16 = false);

// Launches a planned head: flow[i] = up[i] (if up) + bias + conv(a.in)[i][0..1], float (n, ho, wo, 2).
cudaError_t launch_conv_tc_head(const TcConvPlan &plan, const ConvArgs &a, const float *up, float *flow,
                                cudaStream_t st);

// Launches a planned conv for a.n images starting at a.in (which must lie inside the
// planned buffer, on an image boundary), writing the plan's 16-bit type (bfloat16 or half)
// or e4m3 to a.out with a.out_cs stride.
cudaError_t launch_conv_tc(const TcConvPlan &plan, const ConvArgs &a, cudaStream_t st);

// The same for a bf16 plan writing float32 to a.out (pixel stride a.out_cs floats, a
// multiple of 4, 16-byte aligned), added to what is there when accumulate is set.
cudaError_t launch_conv_tc_f32(const TcConvPlan &plan, const ConvArgs &a, bool accumulate, cudaStream_t st);

}  // namespace tc
