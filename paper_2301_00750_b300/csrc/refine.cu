// Depthwise dilated 3x3 conv and CUDA-core pointwise 1x1 conv of the refinement network
// (Sec. 3.2, "-sepref": the refinement's convs replaced by depthwise-separable ones).
#include "common.cuh"
#include "refine.cuh"

namespace tc {

namespace {

constexpr int DW_THREADS = 128;  // threads per block: channel groups x pixel lanes
constexpr int DW_PIX = 8;        // pixels per thread, one lane count apart along the row

// 8 consecutive activations as raw bits (one 16-byte load for bf16 and half, two for float) and
// their float values.
template <typename T> struct Raw8;
template <> struct Raw8<__nv_bfloat16> {
    uint4 u;
    __device__ __forceinline__ void load(const __nv_bfloat16 *p) { u = __ldg(reinterpret_cast<const uint4 *>(p)); }
    __device__ __forceinline__ void get(float (&v)[8]) const {
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 f = __bfloat1622float2(h[k]);
            v[2 * k] = f.x;
            v[2 * k + 1] = f.y;
        }
    }
};
template <> struct Raw8<__half> {
    uint4 u;
    __device__ __forceinline__ void load(const __half *p) { u = __ldg(reinterpret_cast<const uint4 *>(p)); }
    __device__ __forceinline__ void get(float (&v)[8]) const {
        const __half2 *h = reinterpret_cast<const __half2 *>(&u);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 f = __half22float2(h[k]);
            v[2 * k] = f.x;
            v[2 * k + 1] = f.y;
        }
    }
};
template <> struct Raw8<float> {
    float4 a, b;
    __device__ __forceinline__ void load(const float *p) {
        a = __ldg(reinterpret_cast<const float4 *>(p));
        b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
    }
    __device__ __forceinline__ void get(float (&v)[8]) const {
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    }
};

template <typename T>
__device__ __forceinline__ void store8(T *p, const float (&v)[8]) {
    st4(p, make_float4(v[0], v[1], v[2], v[3]));
    st4(p + 4, make_float4(v[4], v[5], v[6], v[7]));
}

// Block (groups of 8 channels) x L lanes (L = blockDim.y) covers L x DW_PIX consecutive
// pixels of one row: thread (g, l) keeps the 9 x 8 taps and the biases of channel group g
// in registers and computes pixels x0 + l + L j, j < DW_PIX:
// out[c] = db[c] + sum over the taps of dw[tap][c] in[c](y + (ky - 1) dil, x + (kx - 1) dil),
// taps off the map contribute 0.  The nine loads of a pixel are issued together; away from
// the border they share one base pointer, at the border their addresses are clamped and
// the taps off the map get weight 0.  Channels at or beyond nin come from the flow (the
// first two) or are 0.
template <typename T>
__global__ void __launch_bounds__(DW_THREADS, 4) depthwise_kernel(const DwArgs a) {
    const int g = threadIdx.x, lane = threadIdx.y, lanes = blockDim.y;
    const int c0 = 8 * g;
    const int y = blockIdx.y, img = blockIdx.z;
    const int x0 = blockIdx.x * (lanes * DW_PIX);
    const T *in = static_cast<const T *>(a.in);
    float wt[9][8], bias[8];
#pragma unroll
    for (int t = 0; t < 9; ++t)
#pragma unroll
        for (int j = 0; j < 8; ++j) wt[t][j] = __ldg(a.dw + t * a.cp + c0 + j);
#pragma unroll
    for (int j = 0; j < 8; ++j) bias[j] = __ldg(a.db + c0 + j);
    const bool vec = c0 + 8 <= a.nin && a.in_cs % 8 == 0;
    const size_t row0 = (size_t)img * a.h;
    int rows[3];
    bool vy[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int sy = y + (k - 1) * a.dil;
        vy[k] = sy >= 0 && sy < a.h;
        rows[k] = min(max(sy, 0), a.h - 1);
    }
#pragma unroll 1
    for (int p = 0; p < DW_PIX; ++p) {
        const int x = x0 + lane + lanes * p;
        if (x >= a.w) break;
        float acc[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] = bias[j];
        int cols[3];
        bool vx[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int sx = x + (k - 1) * a.dil;
            vx[k] = sx >= 0 && sx < a.w;
            cols[k] = min(max(sx, 0), a.w - 1);
        }
        const bool inner = vx[0] && vx[2] && vy[0] && vy[2];
        if (vec && inner) {
            const T *cp = in + ((row0 + y) * a.w + x) * a.in_cs + c0;
            const ptrdiff_t dx = (ptrdiff_t)a.dil * a.in_cs, dy = (ptrdiff_t)a.dil * a.w * a.in_cs;
            Raw8<T> raw[9];
#pragma unroll
            for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) raw[ky * 3 + kx].load(cp + (ky - 1) * dy + (kx - 1) * dx);
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                float v[8];
                raw[t].get(v);
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[j] = fmaf(wt[t][j], v[j], acc[j]);
            }
        } else if (vec) {
            Raw8<T> raw[9];
#pragma unroll
            for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                for (int kx = 0; kx < 3; ++kx)
                    raw[ky * 3 + kx].load(in + ((row0 + rows[ky]) * a.w + cols[kx]) * a.in_cs + c0);
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                float v[8];
                raw[t].get(v);
                const bool ok = vy[t / 3] && vx[t % 3];
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[j] = fmaf(ok ? wt[t][j] : 0.f, v[j], acc[j]);
            }
        } else {
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                if (!(vy[t / 3] && vx[t % 3])) continue;
                const size_t sp = (row0 + rows[t / 3]) * a.w + cols[t % 3];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int c = c0 + j;
                    const float v = c < a.nin ? to_f(in[sp * a.in_cs + c])
                                              : (a.flow && c < a.nin + 2 ? __ldg(a.flow + sp * 2 + (c - a.nin)) : 0.f);
                    acc[j] = fmaf(wt[t][j], v, acc[j]);
                }
            }
        }
        store8(static_cast<T *>(a.out) + ((row0 + y) * a.w + x) * a.out_cs + c0, acc);
    }
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
    const int groups = a.cp / 8;
    if (a.cp % 8 != 0 || groups < 1 || groups > DW_THREADS || a.dil < 1) return cudaErrorInvalidValue;
    const int lanes = DW_THREADS / groups;
    const dim3 block(groups, lanes);
    const dim3 grid((a.w + lanes * DW_PIX - 1) / (lanes * DW_PIX), a.h, a.n);
    depthwise_kernel<T><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pointwise(const PwArgs &a, cudaStream_t st) {
    pointwise_kernel<T><<<(unsigned)((a.npx + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_depthwise<float>(const DwArgs &, cudaStream_t);
template cudaError_t launch_depthwise<__nv_bfloat16>(const DwArgs &, cudaStream_t);
template cudaError_t launch_depthwise<__half>(const DwArgs &, cudaStream_t);
template cudaError_t launch_pointwise<float>(const PwArgs &, cudaStream_t);
template cudaError_t launch_pointwise<__nv_bfloat16>(const PwArgs &, cudaStream_t);
template cudaError_t launch_pointwise<__half>(const PwArgs &, cudaStream_t);

}  // namespace tc
