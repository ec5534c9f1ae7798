// Refinement network with depthwise-separable convs ("-sepref", Sec. 3.2): the depthwise
// dilated 3x3 conv and the CUDA-core pointwise 1x1 conv (the tensor-core pointwise conv is
// the one-tap mode of the tcgen05 conv).  NHWC activations of type T (float or bf16).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace tc {

struct DwArgs {
    const void *in;     // T input: channels [0, nin) of each pixel, pixel stride in_cs
    int in_cs, nin;
    const float *flow;  // optional (n, h, w, 2) float: channels nin and nin + 1
    int n, h, w;
    const float *dw;    // [9][cp] taps (row-major ky, kx) by channel; 0 for padding channels
    const float *db;    // [cp]
    int dil;
    void *out;          // T output: channels [0, cp) (cp a multiple of 8), pixel stride out_cs
    int out_cs, cp;
};

struct PwArgs {
    const void *in;     // T input: channels [0, cin), pixel stride in_cs
    int in_cs, cin;
    const float *w;     // [cin][cout]
    const float *b;     // [cout]
    int cout, leaky;    // cout a multiple of 8 (or 2 with flow)
    void *out;          // T output, pixel stride out_cs
    int out_cs;
    float *flow;        // cout = 2: flow[p] += (out0, out1) (float (npx, 2)) instead of out
    size_t npx;
};

template <typename T> cudaError_t launch_depthwise(const DwArgs &a, cudaStream_t st);
template <typename T> cudaError_t launch_pointwise(const PwArgs &a, cudaStream_t st);

}  // namespace tc
