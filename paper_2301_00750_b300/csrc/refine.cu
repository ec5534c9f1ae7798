// Depthwise dilated 3x3 conv and CUDA-core pointwise 1x1 conv of the refinement network
// (Sec. 3.2, "-sepref": the refinement's convs replaced by depthwise-separable ones).
#include "common.cuh"
#include "refine.cuh"

namespace tc {

namespace {

template <typename T>
__device__ __forceinline__ void load8(const T *p, float (&v)[8]) {
    const float4 a = ld4(p), b = ld4(p + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

template <typename T>
__device__ __forceinline__ void store8(T *p, const float (&v)[8]) {
    st4(p, make_float4(v[0], v[1], v[2], v[3]));
    st4(p + 4, make_float4(v[4], v[5], v[6], v[7]));
}

// One thread per (pixel, group of 8 channels): out[c] = db[c] + sum over the 9 taps of
// dw[tap][c] in[c](y + (ky - 1) dil, x + (kx - 1) dil), taps off the map contribute 0.
template <typename T>
__global__ void __launch_bounds__(256) depthwise_kernel(const DwArgs a) {
    const int groups = a.cp >> 3;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t hw = (size_t)a.h * a.w;
    if (i >= (size_t)a.n * hw * groups) return;
    const int g = (int)(i % groups);
    const size_t px = i / groups;
    const int img = (int)(px / hw);
    const int r = (int)(px - (size_t)img * hw);
    const int y = r / a.w, x = r - y * a.w;
    const int c0 = 8 * g;
    const T *in = static_cast<const T *>(a.in);
    float acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = __ldg(a.db + c0 + j);
    const bool vec = c0 + 8 <= a.nin && a.in_cs % 8 == 0;
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
        const int sy = y + (ky - 1) * a.dil;
        if (sy < 0 || sy >= a.h) continue;
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
            const int sx = x + (kx - 1) * a.dil;
            if (sx < 0 || sx >= a.w) continue;
            const size_t sp = ((size_t)img * a.h + sy) * a.w + sx;
            float v[8];
            if (vec) {
                load8(in + sp * a.in_cs + c0, v);
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int c = c0 + j;
                    v[j] = c < a.nin ? to_f(in[sp * a.in_cs + c])
                                     : (a.flow && c < a.nin + 2 ? __ldg(a.flow + sp * 2 + (c - a.nin)) : 0.f);
                }
            }
            const float *wt = a.dw + (ky * 3 + kx) * a.cp + c0;
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] = fmaf(__ldg(wt + j), v[j], acc[j]);
        }
    }
    store8(static_cast<T *>(a.out) + px * a.out_cs + c0, acc);
}

// One thread per pixel: out[o] = b[o] + sum_c w[c][o] in[c], LeakyReLU 0.1 if leaky, in
// chunks of 8 outputs; with flow (cout = 2) the two outputs are added to the flow.
template <typename T>
__global__ void __launch_bounds__(256) pointwise_kernel(const PwArgs a) {
    const size_t px = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (px >= a.npx) return;
    const T *in = static_cast<const T *>(a.in) + px * a.in_cs;
    if (a.flow) {
        float o0 = __ldg(a.b), o1 = __ldg(a.b + 1);
        for (int c = 0; c < a.cin; ++c) {
            const float v = to_f(in[c]);
            o0 = fmaf(__ldg(a.w + 2 * c), v, o0);
            o1 = fmaf(__ldg(a.w + 2 * c + 1), v, o1);
        }
        float2 *f = reinterpret_cast<float2 *>(a.flow) + px;
        const float2 old = *f;
        *f = make_float2(old.x + o0, old.y + o1);
        return;
    }
    T *out = static_cast<T *>(a.out) + px * a.out_cs;
    for (int o0 = 0; o0 < a.cout; o0 += 8) {
        float acc[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] = __ldg(a.b + o0 + j);
        for (int c = 0; c < a.cin; ++c) {
            const float v = to_f(in[c]);
            const float *wr = a.w + (size_t)c * a.cout + o0;
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] = fmaf(__ldg(wr + j), v, acc[j]);
        }
        if (a.leaky)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] = acc[j] >= 0.f ? acc[j] : 0.1f * acc[j];
#pragma unroll
        for (int j = 0; j < 8; ++j) out[o0 + j] = from_f<T>(acc[j]);
    }
}

}  // namespace

template <typename T>
cudaError_t launch_depthwise(const DwArgs &a, cudaStream_t st) {
    const size_t n = (size_t)a.n * a.h * a.w * (a.cp / 8);
    depthwise_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pointwise(const PwArgs &a, cudaStream_t st) {
    pointwise_kernel<T><<<(unsigned)((a.npx + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_depthwise<float>(const DwArgs &, cudaStream_t);
template cudaError_t launch_depthwise<__nv_bfloat16>(const DwArgs &, cudaStream_t);
template cudaError_t launch_pointwise<float>(const PwArgs &, cudaStream_t);
template cudaError_t launch_pointwise<__nv_bfloat16>(const PwArgs &, cudaStream_t);

}  // namespace tc
