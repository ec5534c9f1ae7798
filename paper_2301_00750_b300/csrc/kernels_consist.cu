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

// Frame t - 1's I, P, O at the taps t, from the kept-state layout (see ConsistArgs): I, P from
// pA and pB.xy, O from oB.zw and pC.  When oB is pB (one frame's state) one 16-byte load of B
// serves both; otherwise (one frame of latency, where I, P and O of frame t - 1 sit in
// different slots) B's halves are loaded from their own slots, 8 bytes each.  The sum of each
// tap's weight times its value runs in the order of gather() above.
template <bool SPLIT>
__device__ __forceinline__ void gather_state(const ConsistArgs &a, const Taps &t, float (&gI)[3], float (&gP)[3],
                                             float (&gO)[3]) {
    const int o[4] = {t.ya * a.W + t.xa, t.ya * a.W + t.xb, t.yb * a.W + t.xa, t.yb * a.W + t.xb};
    const float w[4] = {t.w00, t.w01, t.w10, t.w11};
    float4 A[4], B[4];
    float C[4];
    if constexpr (!SPLIT) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            A[k] = __ldg(a.pA + o[k]);
            B[k] = __ldg(a.pB + o[k]);
            C[k] = __ldg(a.pC + o[k]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            A[k] = __ldg(a.pA + o[k]);
            const float2 ip = __ldg(reinterpret_cast<const float2 *>(a.pB + o[k]));
            const float2 op = __ldg(reinterpret_cast<const float2 *>(a.oB + o[k]) + 1);
            B[k] = make_float4(ip.x, ip.y, op.x, op.y);
            C[k] = __ldg(a.pC + o[k]);
        }
    }
    float v[9];
#define TC_TAPSUM(dst, f)                         \
    do {                                          \
        float acc_ = w[0] * (f(0));               \
        acc_ += w[1] * (f(1));                    \
        acc_ += w[2] * (f(2));                    \
        acc_ += w[3] * (f(3));                    \
        dst = acc_;                               \
    } while (0)
#define TC_AX(k) A[k].x
#define TC_AY(k) A[k].y
#define TC_AZ(k) A[k].z
#define TC_AW(k) A[k].w
#define TC_BX(k) B[k].x
#define TC_BY(k) B[k].y
#define TC_BZ(k) B[k].z
#define TC_BW(k) B[k].w
#define TC_C(k) C[k]
    TC_TAPSUM(v[0], TC_AX);
    TC_TAPSUM(v[1], TC_AY);
    TC_TAPSUM(v[2], TC_AZ);
    TC_TAPSUM(v[3], TC_AW);
    TC_TAPSUM(v[4], TC_BX);
    TC_TAPSUM(v[5], TC_BY);
    TC_TAPSUM(v[6], TC_BZ);
    TC_TAPSUM(v[7], TC_BW);
    TC_TAPSUM(v[8], TC_C);
#undef TC_TAPSUM
#undef TC_AX
#undef TC_AY
#undef TC_AZ
#undef TC_AW
#undef TC_BX
#undef TC_BY
#undef TC_BZ
#undef TC_BW
#undef TC_C
    gI[0] = v[0]; gI[1] = v[1]; gI[2] = v[2];
    gP[0] = v[3]; gP[1] = v[4]; gP[2] = v[5];
    gO[0] = v[6]; gO[1] = v[7]; gO[2] = v[8];
}

// Frame t's I, P (planar inputs, or its kept state when It is NULL).
__device__ __forceinline__ void frame_inputs(const ConsistArgs &a, size_t i, size_t hw, float (&It)[3],
                                             float (&Pt)[3]) {
    if (a.It) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            It[c] = __ldcs(a.It + c * hw + i);  // read once: streaming
            Pt[c] = __ldcs(a.Pt + c * hw + i);
        }
    } else {
        const float4 A = a.tA[i], B = a.tB[i];
        It[0] = A.x; It[1] = A.y; It[2] = A.z;
        Pt[0] = A.w; Pt[1] = B.x; Pt[2] = B.y;
    }
}

// The state kept of frame t (written once: streaming stores), and the planar P_t copy.
__device__ __forceinline__ void keep_state(const ConsistArgs &a, size_t i, size_t hw, const float (&It)[3],
                                           const float (&Pt)[3], const float (&Ot)[3]) {
    if (a.Pcopy)
#pragma unroll
        for (int c = 0; c < 3; ++c) __stcs(a.Pcopy + c * hw + i, Pt[c]);
    if (!a.kA) return;
    if (a.keep_io && a.keep_o) {
        __stcs(a.kA + i, make_float4(It[0], It[1], It[2], Pt[0]));
        __stcs(a.kB + i, make_float4(Pt[1], Pt[2], Ot[0], Ot[1]));
        __stcs(a.kC + i, Ot[2]);
    } else if (a.keep_io) {
        __stcs(a.kA + i, make_float4(It[0], It[1], It[2], Pt[0]));
        __stcs(reinterpret_cast<float2 *>(a.kB + i), make_float2(Pt[1], Pt[2]));
    } else if (a.keep_o) {
        __stcs(reinterpret_cast<float2 *>(a.kB + i) + 1, make_float2(Ot[0], Ot[1]));
        __stcs(a.kC + i, Ot[2]);
    }
}

// NEXT = false: causal form (w_n = 0).  NEXT = true: frame t+1 warped along F_{t->t+1}
// enters L_t and A^I_t with the weight w_n (Eqs. 2, 3, 6); the mask gets bit 1 for it.
// GEN: the causal form for frame t from the kept state and frame t - 1's state split over
// two slots (the last frame of a stream with one frame of latency, tc_flush); without it
// (causal streams, lanes and the stage op) frame t is planar and frame t - 1 one slot.
// Both forms are bound by the latency of their dependent loads (flow, then taps), so
// occupancy matters: five blocks (40 warps) per SM and 48 registers, which the twelve tap
// loads of the interleaved state need without spilling (at six blocks they spilled: 57.5 vs
// 55.4 us for the causal pass at 1080p; the planar state's 36 scalar tap loads: 61.6 us).
template <bool NEXT, bool GEN = false>
__global__ void __launch_bounds__(256, 5) consistency_kernel(ConsistArgs a) {
    constexpr bool RT = NEXT || GEN;  // frame t's source and frame t - 1's slots chosen at run time
    pdl_wait();
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= a.W || y >= a.H) return;
    const size_t hw = (size_t)a.H * a.W;
    const size_t i = (size_t)y * a.W + x;
    float It[3], Pt[3];
    // frame t's inputs first: their loads overlap everything up to the blend
    if (!RT) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            It[c] = __ldcs(a.It + c * hw + i);  // read once: streaming
            Pt[c] = __ldcs(a.Pt + c * hw + i);
        }
    } else {
        frame_inputs(a, i, hw, It, Pt);
    }
    if (!NEXT && a.first) {
#pragma unroll
        for (int c = 0; c < 3; ++c) a.O[c * hw + i] = Pt[c];
        keep_state(a, i, hw, It, Pt, Pt);
        if (a.wc) a.wc[i] = 0.f;
        if (a.mask) a.mask[i] = 0;
        return;
    }
    Taps t;
    const bool m = warp_sample(a.Fb, a.Ff, a, x, y, t);
    float gI[3], gP[3], gO[3], d = 0.f;
    if (RT && a.oB != a.pB)
        gather_state<true>(a, t, gI, gP, gO);
    else
        gather_state<false>(a, t, gI, gP, gO);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float e = It[c] - gI[c];
        d += e * e;
    }
    float wp = 0.f;
    if (m) wp = fminf(a.k1, expf(-a.alpha * d));
    float dI = 0.f;
    bool mn = false;
    float Ot[3];
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
            Ot[c] = A;
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
            Ot[c] = A;
        }
    }
    keep_state(a, i, hw, It, Pt, Ot);
    if (a.wc) __stcs(a.wc + i, a.lambda * expf(-a.alpha * dI));
    if (a.mask) a.mask[i] = (m ? 1 : 0) | (mn ? 2 : 0);
}

// Planar (3, hw) I, P, O -> kept-state layout.
__global__ void pack_state_kernel(const float *I, const float *P, const float *O, size_t hw, float4 *A, float4 *B,
                                  float *C) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= hw) return;
    A[i] = make_float4(I[i], I[hw + i], I[2 * hw + i], P[i]);
    B[i] = make_float4(P[hw + i], P[2 * hw + i], O[i], O[hw + i]);
    C[i] = O[2 * hw + i];
}

cudaError_t launch_pack_state(const float *I, const float *P, const float *O, size_t hw, float4 *A, float4 *B,
                              float *C, cudaStream_t st) {
    pack_state_kernel<<<(unsigned)((hw + 255) / 256), 256, 0, st>>>(I, P, O, hw, A, B, C);
    return cudaGetLastError();
}

// A frame's planar I, P -> the I, P part of a kept state (the O part is left as it is).
__global__ void keep_inputs_kernel(const float *I, const float *P, size_t hw, float4 *A, float4 *B) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= hw) return;
    A[i] = make_float4(I[i], I[hw + i], I[2 * hw + i], P[i]);
    reinterpret_cast<float2 *>(B + i)[0] = make_float2(P[hw + i], P[2 * hw + i]);
}

cudaError_t launch_keep_inputs(const float *I, const float *P, size_t hw, float4 *A, float4 *B, cudaStream_t st) {
    keep_inputs_kernel<<<(unsigned)((hw + 255) / 256), 256, 0, st>>>(I, P, hw, A, B);
    return cudaGetLastError();
}

const void *keep_inputs_kernel_fn() { return reinterpret_cast<const void *>(keep_inputs_kernel); }

// The solver's result to the caller (O, and w_c when wc is not NULL) and into the O part of
// the kept state.
__global__ void solver_out_kernel(const float *src, float *O, const float *wsrc, float *wc, size_t hw, float4 *B,
                                  float *C) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= hw) return;
    const float o0 = src[i], o1 = src[hw + i], o2 = src[2 * hw + i];
    O[i] = o0;
    O[hw + i] = o1;
    O[2 * hw + i] = o2;
    if (wc) wc[i] = wsrc[i];
    reinterpret_cast<float2 *>(B + i)[1] = make_float2(o0, o1);
    C[i] = o2;
}

cudaError_t launch_solver_out(const float *src, float *O, const float *wsrc, float *wc, size_t hw, float4 *B,
                              float *C, cudaStream_t st) {
    solver_out_kernel<<<(unsigned)((hw + 255) / 256), 256, 0, st>>>(src, O, wsrc, wc, hw, B, C);
    return cudaGetLastError();
}

const void *solver_out_kernel_fn() { return reinterpret_cast<const void *>(solver_out_kernel); }

const void *consistency_kernel_fn(bool next) {
    return next ? reinterpret_cast<const void *>(consistency_kernel<true>)
                : reinterpret_cast<const void *>(consistency_kernel<false>);
}

cudaError_t launch_consistency(const ConsistArgs &a, cudaStream_t st) {
    dim3 grid((a.W + 31) / 32, (a.H + 7) / 8);
    if (a.next) return launch_pdl(consistency_kernel<true>, grid, dim3(256), 0, st, a);
    if (!a.It || a.oB != a.pB) return launch_pdl(consistency_kernel<false, true>, grid, dim3(256), 0, st, a);
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
