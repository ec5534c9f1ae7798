// Fused consistency step (Sec. 3.1, Eqs. 2-7, causal or with the next frame): final flow
// upsampling, backward warp of I_{t-1}, P_{t-1}, O_{t-1} (and of I_{t+1}, P_{t+1}),
// forward-backward non-occlusion masks, photometric weights, local/global blend, warped
// input and consistency weight, plus the copies of I_t, P_t, O_t that the stream keeps for
// the next frame.  One pass over the frame, one thread per pixel, float32 throughout.
#include "common.cuh"

namespace tc {

// Bilinear interpolation weights and clamped tap positions for the sample x + u.  The
// integer part floor(u) and the fraction u - floor(u) are exact in float32, so the taps and
// weights equal those of the exact sample position.
struct Taps {
    int xa, xb, ya, yb;
    float w00, w01, w10, w11;
    float ax, ay;  // the fractions along x and y
};

__device__ __forceinline__ Taps clamp_taps(int x, int y, float u, float v, int W, int H) {
    const float fu = floorf(u), fv = floorf(v);
    const float ax = u - fu, ay = v - fv;
    const int x0 = x + (int)fu, y0 = y + (int)fv;
    Taps t;
    t.xa = min(max(x0, 0), W - 1);
    t.xb = min(max(x0 + 1, 0), W - 1);
    t.ya = min(max(y0, 0), H - 1);
    t.yb = min(max(y0 + 1, 0), H - 1);
    t.w00 = (1.f - ax) * (1.f - ay);
    t.w01 = ax * (1.f - ay);
    t.w10 = (1.f - ax) * ay;
    t.w11 = ax * ay;
    t.ax = ax;
    t.ay = ay;
    return t;
}

// (H * W fits an int: the offsets of the taps are 32-bit.)
__device__ __forceinline__ float gather(const float *p, int W, const Taps &t) {
    float acc = t.w00 * __ldg(p + (t.ya * W + t.xa));
    acc += t.w01 * __ldg(p + (t.ya * W + t.xb));
    acc += t.w10 * __ldg(p + (t.yb * W + t.xa));
    acc += t.w11 * __ldg(p + (t.yb * W + t.xb));
    return acc;
}

// Weights on the low-resolution cells base, base + 1, base + 2 of one axis (base = the
// first cell of tap a) of the bilinear combination (1 - f) up(Xa) + f up(Xb) of the
// s-times upsampled field along that axis, s = 2^k >= 2 (1/s = rs).  Xb is Xa or Xa + 1, so
// the first cell of Xb is base or base + 1.  Returns base; `third` says whether cell
// base + 2 carries weight.
__device__ __forceinline__ int axis_weights(int Xa, int Xb, float f, float rs, int n, float &c0, float &c1,
                                            float &c2, bool &third) {
    const float sa = fmaxf((Xa + 0.5f) * rs - 0.5f, 0.f), sb = fmaxf((Xb + 0.5f) * rs - 0.5f, 0.f);
    const int a0 = min((int)sa, n - 1), b0 = min((int)sb, n - 1);
    const float la = sa - a0, lb = sb - b0;
    const float wa = 1.f - f;
    third = b0 != a0;
    c0 = wa * (1.f - la);
    c1 = wa * la;
    c2 = 0.f;
    if (third) {
        c1 += f * (1.f - lb);
        c2 = f * lb;
    } else {
        c0 += f * (1.f - lb);
        c1 += f * lb;
    }
    return a0;
}

// The opposite flow G (fh, fw, 2 at 1/s resolution, s = 2^k >= 2), upsampled and sampled
// bilinearly at the taps t: the four upsampled values lie on one 3 x 3 block of G's cells
// (cells past the last row/column clamp to it, as the upsampling does), so the tap weights
// and the upsampling weights fold into one weight per cell of that block.
__device__ __forceinline__ float2 fb_flow_at_taps(const float *G, const ConsistArgs &a, const Taps &t) {
    const float2 *g = reinterpret_cast<const float2 *>(G);
    const float rs = __int_as_float((127 - (__ffs(a.scale) - 1)) << 23);  // 2^-k
    float cx[3], cy[3];
    bool tx, ty;
    const int x0 = axis_weights(t.xa, t.xb, t.ax, rs, a.fw, cx[0], cx[1], cx[2], tx);
    const int y0 = axis_weights(t.ya, t.yb, t.ay, rs, a.fh, cy[0], cy[1], cy[2], ty);
    const int xc1 = min(x0 + 1, a.fw - 1), xc2 = min(x0 + 2, a.fw - 1);
    float su = 0.f, sv = 0.f;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        if (r == 2 && !ty) break;
        const int row = min(y0 + r, a.fh - 1) * a.fw;
        const float2 p0 = g[row + x0], p1 = g[row + xc1];
        float ru = cx[0] * p0.x + cx[1] * p1.x, rv = cx[0] * p0.y + cx[1] * p1.y;
        if (tx) {
            const float2 p2 = g[row + xc2];
            ru += cx[2] * p2.x;
            rv += cx[2] * p2.y;
        }
        su += cy[r] * ru;
        sv += cy[r] * rv;
    }
    const float fs = (float)a.scale;
    return make_float2(fs * su, fs * sv);
}

// The warp of a neighbouring frame along F at (x, y): taps, and whether it is valid (in
// bounds and, with fb_check, not occluded by the forward-backward test against the
// opposite flow G sampled at the taps).
__device__ __forceinline__ bool warp_sample(const float *F, const float *G, const ConsistArgs &a, int x, int y,
                                            Taps &t) {
    const float2 f = upsampled_flow_at(F, a.fh, a.fw, a.scale, x, y);
    // Keep the sample position finite and far outside the frame for absurd flows.
    const float u = fminf(fmaxf(f.x, -1e6f), 1e6f), v = fminf(fmaxf(f.y, -1e6f), 1e6f);
    // In bounds: 0 <= x + u <= W - 1 and 0 <= y + v <= H - 1, compared exactly.
    const bool inb = u >= (float)(-x) && u <= (float)(a.W - 1 - x) && v >= (float)(-y) &&
                     v <= (float)(a.H - 1 - y);
    t = clamp_taps(x, y, u, v, a.W, a.H);
    bool occ = false;
    if (a.fb_check) {
        float fu, fv;
        if (a.scale > 1) {
            const float2 f = fb_flow_at_taps(G, a, t);
            fu = f.x;
            fv = f.y;
        } else {
            const float2 *g = reinterpret_cast<const float2 *>(G);
            const float2 f00 = g[t.ya * a.fw + t.xa], f01 = g[t.ya * a.fw + t.xb];
            const float2 f10 = g[t.yb * a.fw + t.xa], f11 = g[t.yb * a.fw + t.xb];
            fu = t.w00 * f00.x;
            fu += t.w01 * f01.x;
            fu += t.w10 * f10.x;
            fu += t.w11 * f11.x;
            fv = t.w00 * f00.y;
            fv += t.w01 * f01.y;
            fv += t.w10 * f10.y;
            fv += t.w11 * f11.y;
        }
        const float su = u + fu, sv = v + fv;
        const float lhs = su * su + sv * sv;
        const float rhs = a.c1 * ((u * u + v * v) + (fu * fu + fv * fv)) + a.c2;
        occ = lhs > rhs;
    }
    return inb && !occ;
}

// NEXT = false: causal form (w_n = 0).  NEXT = true: frame t+1 warped along F_{t->t+1}
// enters L_t and A^I_t with the weight w_n (Eqs. 2, 3, 6); the mask gets bit 1 for it.
// Both forms are bound by the latency of their dependent loads (flow, then taps), so
// occupancy comes first: the causal form runs at 40 registers (six blocks, 48 warps per
// SM), the one with the next frame at 48 (five blocks).
template <bool NEXT>
__global__ void __launch_bounds__(256, NEXT ? 5 : 6) consistency_kernel(ConsistArgs a) {
    pdl_wait();
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= a.W || y >= a.H) return;
    const size_t hw = (size_t)a.H * a.W;
    const size_t i = (size_t)y * a.W + x;
    float It[3], Pt[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        It[c] = __ldcs(a.It + c * hw + i);  // read once: streaming
        Pt[c] = __ldcs(a.Pt + c * hw + i);
    }
    if (!NEXT && a.first) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            a.O[c * hw + i] = Pt[c];
            if (a.sI) a.sI[c * hw + i] = It[c];
            if (a.sP) a.sP[c * hw + i] = Pt[c];
            if (a.sO) a.sO[c * hw + i] = Pt[c];
        }
        if (a.wc) a.wc[i] = 0.f;
        if (a.mask) a.mask[i] = 0;
        return;
    }
    Taps t;
    const bool m = warp_sample(a.Fb, a.Ff, a, x, y, t);
    float gI[3], gP[3], gO[3], d = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        gI[c] = gather(a.Ip + c * hw, a.W, t);
        gP[c] = gather(a.Pp + c * hw, a.W, t);
        gO[c] = gather(a.Op + c * hw, a.W, t);
        const float e = It[c] - gI[c];
        d += e * e;
    }
    float wp = 0.f;
    if (m) wp = fminf(a.k1, expf(-a.alpha * d));
    float dI = 0.f;
    bool mn = false;
    if constexpr (NEXT) {
        Taps tn;
        mn = warp_sample(a.Fn, a.Fnb, a, x, y, tn);
        float gIn[3], gPn[3], dn = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            gIn[c] = gather(a.In + c * hw, a.W, tn);
            gPn[c] = gather(a.Pn + c * hw, a.W, tn);
            const float e = It[c] - gIn[c];
            dn += e * e;
        }
        float wn = 0.f;
        if (mn) wn = fminf(a.k2, expf(-a.alpha * dn));
        const float wl = 1.f - (wp + wn);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float L = wl * Pt[c] + wp * gP[c] + wn * gPn[c];
            const float A = wp * gO[c] + (1.f - wp) * L;
            const float AI = wl * It[c] + wp * gI[c] + wn * gIn[c];
            const float e = It[c] - AI;
            dI += e * e;
            __stcs(a.O + c * hw + i, A);  // written once: streaming
            if (a.sI) __stcs(a.sI + c * hw + i, It[c]);
            if (a.sP) __stcs(a.sP + c * hw + i, Pt[c]);
            if (a.sO) __stcs(a.sO + c * hw + i, A);
        }
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float L = (1.f - wp) * Pt[c] + wp * gP[c];
            const float A = wp * gO[c] + (1.f - wp) * L;
            const float AI = (1.f - wp) * It[c] + wp * gI[c];
            const float e = It[c] - AI;
            dI += e * e;
            __stcs(a.O + c * hw + i, A);  // written once: streaming
            if (a.sI) __stcs(a.sI + c * hw + i, It[c]);
            if (a.sP) __stcs(a.sP + c * hw + i, Pt[c]);
            if (a.sO) __stcs(a.sO + c * hw + i, A);
        }
    }
    if (a.wc) __stcs(a.wc + i, a.lambda * expf(-a.alpha * dI));
    if (a.mask) a.mask[i] = (m ? 1 : 0) | (mn ? 2 : 0);
}

const void *consistency_kernel_fn(bool next) {
    return next ? reinterpret_cast<const void *>(consistency_kernel<true>)
                : reinterpret_cast<const void *>(consistency_kernel<false>);
}

cudaError_t launch_consistency(const ConsistArgs &a, cudaStream_t st) {
    dim3 grid((a.W + 31) / 32, (a.H + 7) / 8);
    if (a.next) return launch_pdl(consistency_kernel<true>, grid, dim3(256), 0, st, a);
    return launch_pdl(consistency_kernel<false>, grid, dim3(256), 0, st, a);
}

// (c, h, w) -> (c, ceil(h/2), ceil(w/2)): the mean of each 2 x 2 block, the last row and
// column replicated when h or w is odd (the half-size flow input of the fast preset).
__global__ void downscale2_kernel(const float *src, int c, int h, int w, float *dst) {
    const int hn = (h + 1) / 2, wn = (w + 1) / 2;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)c * hn * wn) return;
    const int ch = (int)(i / ((size_t)hn * wn));
    const int r = (int)(i - (size_t)ch * hn * wn);
    const int y = r / wn, x = r - y * wn;
    const int y0 = 2 * y, y1 = min(2 * y + 1, h - 1), x0 = 2 * x, x1 = min(2 * x + 1, w - 1);
    const float *p = src + (size_t)ch * h * w;
    const float a = __ldg(p + (size_t)y0 * w + x0), b = __ldg(p + (size_t)y0 * w + x1);
    const float cc = __ldg(p + (size_t)y1 * w + x0), d = __ldg(p + (size_t)y1 * w + x1);
    dst[i] = 0.25f * ((a + b) + (cc + d));
}

const void *downscale2_kernel_fn() { return reinterpret_cast<const void *>(downscale2_kernel); }

cudaError_t launch_downscale2(const float *src, int c, int h, int w, float *dst, cudaStream_t st) {
    const size_t n = (size_t)c * ((h + 1) / 2) * ((w + 1) / 2);
    downscale2_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, c, h, w, dst);
    return cudaGetLastError();
}

// 8-bit video frames: interleaved RGB8 (H, W, 3) <-> planar float (3, H, W).  A code q stands
// for q / 255 (an IEEE division, so host and device agree bit for bit); an output value v
// is stored as floor(255 clamp(v, 0, 1) + 0.5), with the multiply and the add rounded
// separately (no contraction), so the host can reproduce it exactly in float32.
__global__ void unpack_rgb8_kernel(const uint8_t *__restrict__ src, size_t hw, float *__restrict__ dst) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= hw) return;
    const uint8_t *p = src + 3 * i;
#pragma unroll
    for (int c = 0; c < 3; ++c) dst[c * hw + i] = __fdiv_rn((float)p[c], 255.f);
}

__global__ void pack_rgb8_kernel(const float *__restrict__ src, size_t hw, uint8_t *__restrict__ dst) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= hw) return;
    uint8_t *p = dst + 3 * i;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float v = fminf(fmaxf(src[c * hw + i], 0.f), 1.f);  // NaN -> 0
        p[c] = (uint8_t)(int)floorf(__fadd_rn(__fmul_rn(v, 255.f), 0.5f));
    }
}

cudaError_t launch_unpack_rgb8(const uint8_t *src, size_t hw, float *dst, cudaStream_t st) {
    unpack_rgb8_kernel<<<(unsigned)((hw + 255) / 256), 256, 0, st>>>(src, hw, dst);
    return cudaGetLastError();
}

cudaError_t launch_pack_rgb8(const float *src, size_t hw, uint8_t *dst, cudaStream_t st) {
    pack_rgb8_kernel<<<(unsigned)((hw + 255) / 256), 256, 0, st>>>(src, hw, dst);
    return cudaGetLastError();
}

// Full-resolution flow, cropped to (H, W), planar (2, H, W), from a (fh, fw, 2) field.
__global__ void flow_out_kernel(const float *F, int fh, int fw, int s, int H, int W, float *out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)H * W) return;
    const int y = (int)(i / W), x = (int)(i - (size_t)y * W);
    const float2 v = upsampled_flow_at(F, fh, fw, s, x, y);
    out[i] = v.x;
    out[(size_t)H * W + i] = v.y;
}

cudaError_t launch_flow_out(const float *flow, int fh, int fw, int scale, int H, int W,
                            float *out, cudaStream_t st) {
    const size_t n = (size_t)H * W;
    flow_out_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(flow, fh, fw, scale, H, W, out);
    return cudaGetLastError();
}

}  // namespace tc
