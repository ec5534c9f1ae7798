// Internal declarations shared by the CUDA translation units of the library.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tc {

// Programmatic dependent launch: a kernel launched by launch_pdl may be scheduled as soon as
// the previous kernel of the stream exits, without a full stream-order round trip.  It calls
// pdl_wait() before it reads or writes any memory an earlier kernel touches (it returns once
// the earlier grids have completed and their writes are visible; without a programmatic
// launch it returns at once).  Most kernels trigger their dependents only implicitly, at
// exit: an explicit trigger at the start of every kernel let the next kernel's CTAs compete
// with the last wave (945 vs 954 frames/s).  The tensor-core kernels trigger early where
// their grid leaves half of the SMs free and no other stream shares the GPU (pdl_trigger).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Lets the next kernel of the stream launch before this one exits (once every CTA of this
// grid has executed it or exited); that kernel still waits for this one in pdl_wait().
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// Activation storage types: float (TC_FP32), bfloat16 (TC_BF16) and IEEE half (TC_FP16).
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
template <typename T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }

// E4M3 activations hold the value divided by a per-tensor scale; the kernels here move the
// scaled codes (warps interpolate them, copies copy them) and the scale is applied where the
// arithmetic needs it (tensor-core epilogues, the first conv's output, the up-flow channels).
__device__ __forceinline__ float to_f(__nv_fp8_e4m3 v) { return float(v); }
template <> __device__ __forceinline__ __nv_fp8_e4m3 from_f<__nv_fp8_e4m3>(float v) { return __nv_fp8_e4m3(v); }

// Loads 4 consecutive activations (16-byte aligned for float, 8-byte for bf16) as float4.
__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float4 ld4(const __nv_bfloat16 *p) {
    uint2 u = *reinterpret_cast<const uint2 *>(p);
    __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162 *>(&u.x);
    __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162 *>(&u.y);
    float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
}
__device__ __forceinline__ float4 ld4(const __half *p) {
    uint2 u = *reinterpret_cast<const uint2 *>(p);
    const float2 fa = __half22float2(*reinterpret_cast<__half2 *>(&u.x));
    const float2 fb = __half22float2(*reinterpret_cast<__half2 *>(&u.y));
    return make_float4(fa.x, fa.y, fb.x, fb.y);
}
__device__ __forceinline__ float4 ld4(const __nv_fp8_e4m3 *p) {
    const __nv_fp8x4_e4m3 q = *reinterpret_cast<const __nv_fp8x4_e4m3 *>(p);
    return float4(q);
}
__device__ __forceinline__ void st4(__nv_fp8_e4m3 *p, float4 v) {
    *reinterpret_cast<__nv_fp8x4_e4m3 *>(p) = __nv_fp8x4_e4m3(v);
}
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ void st4(__nv_bfloat16 *p, float4 v) {
    __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
    uint2 u;
    u.x = *reinterpret_cast<uint32_t *>(&a);
    u.y = *reinterpret_cast<uint32_t *>(&b);
    *reinterpret_cast<uint2 *>(p) = u;
}

__device__ __forceinline__ void st4(__half *p, float4 v) {
    __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
    uint2 u;
    u.x = *reinterpret_cast<uint32_t *>(&a);
    u.y = *reinterpret_cast<uint32_t *>(&b);
    *reinterpret_cast<uint2 *>(p) = u;
}

__device__ __forceinline__ float lrelu(float v) { return v >= 0.f ? v : 0.1f * v; }

// ---------------------------------------------------------------------------------------
// Launch parameter blocks
// ---------------------------------------------------------------------------------------

// Implicit-GEMM 3x3 convolution over NHWC activations.  Input and output buffers are
// dense [n][h][w][cs] with the layer's channels at a fixed offset (already applied to the
// pointers).  wk is [9 * cin][cout] (k = tap * cin + c, tap = ky * 3 + kx).
struct ConvArgs {
    const void *in;
    int in_cs;
    int n, h, w, cin, stride;
    int ho, wo;
    const float *wk;
    const float *bias;
    int cout;
    void *out;
    int out_cs;
    int leaky;
    float q_out;  // e4m3 outputs: 1 / output activation scale (unused otherwise)
    int accumulate;  // CUDA-core kernel only: add to the output instead of overwriting it
    // persistent tensor-core kernel only: walk the tiles from the last to the first, so a layer
    // first reads the rows its producer wrote last (still in L2); alternate layers of a chain
    int rev;
    // persistent tensor-core kernel only: the launch overlaps another stream's kernels (the
    // pipelined mode), so its tiles keep the rows TMEM allows instead of being cut down to
    // cover every SM: fewer CTAs, each fuller, leave SMs to the other stream
    int overlap;
};

// First pyramid conv: planar float image (3, H, W), edge-replicated to (Hp, Wp) and
// zero-padded by one, stride 2.  wk is [27][cout] (k = c * 9 + tap).
struct ConvFirstArgs {
    const float *img;
    int H, W, Hp, Wp;
    const float *wk;
    const float *bias;
    int cout;
    void *out;  // [Hp/2][Wp/2][cout]
    float q_out;  // outputs are multiplied by q_out before storing (1 / scale for e4m3, else 1)
    // cout == 16: the weights [27][16] and bias by value (the kernel reads them from the
    // parameter bank as FMA operands); set by set_first16
    float w16[27 * 16];
    float b16[16];
};

// Flow head: conv5 (cin -> 2, no activation) plus the residual up-flow.
struct HeadArgs {
    const void *in;  // [n][h][w][cs], offset applied
    int in_cs, cin, n, h, w;
    const float *wk;   // [9 * cin][2]
    const float *bias; // [2]
    const float *up;   // [n][h][w][2] or NULL
    float *flow;       // [n][h][w][2]
};

// Cost volume over a batch of directions; self/other pointers are per batch entry.
struct CorrArgs {
    const void *fs[2];
    const void *fo[2];
    int fs_cs, fo_cs;
    int n, h, w, c, r;
    void *out;        // [n][h][w][out_cs], correlation at channel 0
    int out_cs;
    void *self_copy;  // same buffer at channel offset D (or NULL)
    // CUDA-core kernel only: when set, batch entry b reads fs[0] + b * fs_img and
    // fo[0] + b * fo_img (elements) instead of the per-entry pointers (any n)
    size_t fs_img, fo_img;
    // Lane pairs (batched streams, pair_lanes > 0; with fs_img and fo_img set): entry b is
    // direction b & 1 of lane q = b >> 1, and the feature maps are two slots of pair_lanes
    // images (slot 0: the lanes' current frames, slot 1: their previous ones).  self =
    // fs[0] + (q + (b & 1) pair_lanes) fs_img; other = fo[0] + (q + (1 - (b & 1))
    // pair_lanes) fo_img when pair_other (both from the slots), else fo[0] + b fo_img.
    int pair_lanes;
    int pair_other;
};

struct WarpArgs {
    const void *f[2];  // per batch entry, [h][w][f_cs]
    int f_cs;
    const float *flow;  // [n][h][w][2], or NULL when `coarse` is given
    int n, h, w, c;
    void *out;          // [n][h][w][out_cs]
    int out_cs;
    // Optional fused x2 upsampling: the flow at (x, y) is the upsampled coarse flow
    // [n][h/2][w/2][2]; it is also written to up_out [n][h][w][2] and, in the activation
    // type, to act [n][h][w][act_cs] (the up-flow channels of the estimator input).
    const float *coarse;
    float *up_out;
    void *act;
    int act_cs;
    float act_q;  // the up-flow is multiplied by act_q before the activation store (1 unless e4m3)
    size_t f_img;  // when set, batch entry b reads f[0] + b * f_img (elements; any n)
    // Lane pairs (batched streams, pair_lanes > 0; with f_img set): entry b is direction
    // b & 1 of lane q = b >> 1 and reads the other frame's features, f[0] + (q + (1 - (b & 1))
    // pair_lanes) f_img (slot 0: the lanes' current frames, slot 1: their previous ones).
    int pair_lanes;
};

struct UpArgs {
    const float *flow;  // [n][h][w][2]
    int n, h, w, s;
    float *out;         // [n][s h][s w][2]
    void *act;          // optional copy into an activation buffer [n][s h][s w][act_cs]
    int act_cs;
};

// The state a stream keeps of a frame (its I, P and O, read back by the next frame's
// bilinear taps) is interleaved per pixel: A = (I0, I1, I2, P0) and B = (P1, P2, O0, O1) as
// 16-byte words and C = O2, so a tap is three loads instead of nine.
struct ConsistArgs {
    const float *It, *Pt;                 // planar (3, H, W) frame t, or NULL: its I, P from tA, tB
    const float4 *tA, *tB;                // frame t in the kept-state layout (when It is NULL)
    // frame t - 1 in the kept-state layout: I, P from pA and pB.xy, O from oB.zw and pC
    // (oB == pB when they are one frame's state)
    const float4 *pA, *pB, *oB;
    const float *pC;
    const float *Fb, *Ff;                 // (fh, fw, 2): F_{t->t-1}, F_{t-1->t}
    int H, W, fh, fw, scale;
    float k1, alpha, lambda, c1, c2;
    int fb_check;
    int first;
    float *O, *wc;
    uint8_t *mask;
    // the state kept of frame t (kA NULL: none): I, P into kA and kB.xy when keep_io, O into
    // kB.zw and kC when keep_o
    float4 *kA, *kB;
    float *kC;
    int keep_io, keep_o;
    float *Pcopy;  // planar copy of P_t (the solver's input), or NULL
    // next-frame term (next != 0): frame t+1 and the flows F_{t->t+1}, F_{t+1->t} (fh, fw, 2)
    int next;
    const float *In, *Pn, *Fn, *Fnb;
    float k2;
};

// Host launchers (return cudaGetLastError()).
template <typename T> cudaError_t launch_conv_simt(const ConvArgs &a, cudaStream_t st);
template <typename T> cudaError_t launch_conv_first(const ConvFirstArgs &a, cudaStream_t st);
template <typename T> cudaError_t launch_head(const HeadArgs &a, cudaStream_t st);
template <typename T> cudaError_t launch_corr(const CorrArgs &a, cudaStream_t st);
template <typename T> cudaError_t launch_warp(const WarpArgs &a, cudaStream_t st);
template <typename T> cudaError_t launch_up(const UpArgs &a, cudaStream_t st);
cudaError_t launch_consistency(const ConsistArgs &a, cudaStream_t st);
// Device entry addresses of the two kernels whose arguments change every frame (used to
// find their nodes in a captured CUDA graph).
template <typename T> const void *conv_first_kernel_fn();
const void *consistency_kernel_fn(bool next);
cudaError_t launch_downscale2(const float *src, int c, int h, int w, float *dst, cudaStream_t st);
const void *downscale2_kernel_fn();
cudaError_t launch_flow_out(const float *flow, int fh, int fw, int scale, int H, int W,
                            float *out, cudaStream_t st);
// Planar (3, hw) I, P, O -> the kept-state layout (A, B, C of ConsistArgs).
cudaError_t launch_pack_state(const float *I, const float *P, const float *O, size_t hw, float4 *A, float4 *B,
                              float *C, cudaStream_t st);
// Planar I, P of a frame into the I, P part of a kept state (A, B.xy): the inputs a stream
// with one frame of latency keeps.  A kernel, so that a captured graph can retarget it.
cudaError_t launch_keep_inputs(const float *I, const float *P, size_t hw, float4 *A, float4 *B, cudaStream_t st);
const void *keep_inputs_kernel_fn();
// The solver's result: planar src copied to O (and wsrc to wc, when wc is not NULL), and
// into the O part of a kept state (B.zw, C).
cudaError_t launch_solver_out(const float *src, float *O, const float *wsrc, float *wc, size_t hw, float4 *B,
                              float *C, cudaStream_t st);
const void *solver_out_kernel_fn();

// Interleaved RGB8 (hw pixels x 3 bytes) -> planar float (3, hw) as q / 255, and back as
// floor(255 clamp(v, 0, 1) + 0.5).
cudaError_t launch_unpack_rgb8(const uint8_t *src, size_t hw, float *dst, cudaStream_t st);
cudaError_t launch_pack_rgb8(const float *src, size_t hw, uint8_t *dst, cudaStream_t st);
template <typename T>
cudaError_t launch_amax(const T *base, size_t npix, int cs, int nc, unsigned *slot, cudaStream_t st);
template <typename T> cudaError_t launch_to_act(const float *in, size_t n, T *out, cudaStream_t st);
template <typename T> cudaError_t launch_from_act(const T *in, size_t n, float *out, cudaStream_t st);

}  // namespace tc

namespace tc {

// Value at integer position (X, Y) of the s-times bilinear upsampling (half-pixel centres,
// sample position clamped at 0 and at the last row/column) of a (fh, fw, 2) flow field,
// multiplied by s.  s = 1 reads the field directly.  s must be a power of two, so every
// coordinate and interpolation weight below is exact in float32 (the products by 1/s are
// the quotients by s), and fh * fw must fit an int.
__device__ __forceinline__ float2 upsampled_flow_at(const float *F, int fh, int fw, int s,
                                                    int X, int Y) {
    const float2 *f = reinterpret_cast<const float2 *>(F);
    if (s == 1) return f[Y * fw + X];
    const float fs = (float)s;
    const float rs = __int_as_float((127 - (__ffs(s) - 1)) << 23);  // 2^-k for s = 2^k
    float sy = (Y + 0.5f) * rs - 0.5f, sx = (X + 0.5f) * rs - 0.5f;
    sy = fmaxf(sy, 0.f);
    sx = fmaxf(sx, 0.f);
    int y0 = min((int)sy, fh - 1), x0 = min((int)sx, fw - 1);
    const int y1 = y0 < fh - 1 ? y0 + 1 : y0, x1 = x0 < fw - 1 ? x0 + 1 : x0;
    const float ly = sy - y0, lx = sx - x0;
    const float2 a = f[y0 * fw + x0], b = f[y0 * fw + x1];
    const float2 c = f[y1 * fw + x0], d = f[y1 * fw + x1];
    float u = (1.f - ly) * ((1.f - lx) * a.x + lx * b.x) + ly * ((1.f - lx) * c.x + lx * d.x);
    float v = (1.f - ly) * ((1.f - lx) * a.y + lx * b.y) + ly * ((1.f - lx) * c.y + lx * d.y);
    return make_float2(fs * u, fs * v);
}

}  // namespace tc
