// SIMT kernels of the lite flow network (Sec. 3.2): implicit-GEMM 3x3 convolution, the
// first (3-channel, stride-2) pyramid conv, the flow head with its residual, the
// shared-memory-tiled correlation, the bilinear feature warp and flow upsampling.
// Activations are NHWC in float (TC_FP32), bfloat16 (TC_BF16) or half (TC_FP16); every accumulation is
// float32.
#include "common.cuh"

namespace tc {

// =====================================================================================
// Implicit-GEMM 3x3 convolution on CUDA cores.
//   M = n * ho * wo output pixels, N = cout, K = 9 * cin (k = tap * cin + c).
//   Block tile 256 pixels x 32 channels, K step 16, 256 threads each owning 8 pixels x 4
//   channels.  A (activations) is gathered straight from the NHWC input with the conv's
//   zero padding; B (weights, [K][cout]) is read row-wise.  Two shared-memory buffers,
//   register prefetch of the next K step.  Requires cin % 4 == 0 and cout % 4 == 0.
// =====================================================================================
constexpr int SB_M = 256, SB_N = 32, SB_K = 16;

template <typename T>
__global__ void __launch_bounds__(256) conv_simt_kernel(ConvArgs a) {
    __shared__ __align__(16) float As[2][SB_K][SB_M];
    __shared__ __align__(16) float Bs[2][SB_K][SB_N];
    const int tid = threadIdx.x;
    const int HWo = a.ho * a.wo;
    const int M = a.n * HWo;
    const int K = 9 * a.cin;
    const int m0 = blockIdx.x * SB_M, n0 = blockIdx.y * SB_N;
    const T *in = static_cast<const T *>(a.in);

    // A-load assignment: pixels (tid & 63) + 64 j, k-quad kq.
    const int kq = tid >> 6;
    int pbase[4], piy[4], pix[4];
    bool pval[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int m = m0 + (tid & 63) + 64 * j;
        pval[j] = m < M;
        const int mm = pval[j] ? m : 0;
        const int img = mm / HWo, rem = mm - img * HWo;
        const int oy = rem / a.wo, ox = rem - oy * a.wo;
        pbase[j] = img * a.h * a.w;
        piy[j] = oy * a.stride - 1;
        pix[j] = ox * a.stride - 1;
    }
    float4 ra[4], rb;

    auto load = [&](int k0) {
        const int k = k0 + kq * 4;
        const int tap = k / a.cin, c = k - tap * a.cin;
        const int ky = tap / 3, kx = tap - ky * 3;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            ra[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            const int iy = piy[j] + ky, ix = pix[j] + kx;
            if (pval[j] && k < K && iy >= 0 && iy < a.h && ix >= 0 && ix < a.w)
                ra[j] = ld4(in + (size_t)(pbase[j] + iy * a.w + ix) * a.in_cs + c);
        }
        rb = make_float4(0.f, 0.f, 0.f, 0.f);
        if (tid < 128) {
            const int kb = k0 + (tid >> 3), nb = n0 + (tid & 7) * 4;
            if (kb < K && nb < a.cout) rb = *reinterpret_cast<const float4 *>(a.wk + (size_t)kb * a.cout + nb);
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int col = (tid & 63) + 64 * j;
            As[buf][kq * 4 + 0][col] = ra[j].x;
            As[buf][kq * 4 + 1][col] = ra[j].y;
            As[buf][kq * 4 + 2][col] = ra[j].z;
            As[buf][kq * 4 + 3][col] = ra[j].w;
        }
        if (tid < 128) *reinterpret_cast<float4 *>(&Bs[buf][tid >> 3][(tid & 7) * 4]) = rb;
    };

    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

    const int tm = tid >> 3, tn = tid & 7;
    const int nk = (K + SB_K - 1) / SB_K;
    load(0);
    store(0);
    __syncthreads();
    for (int kt = 0; kt < nk; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < nk) load((kt + 1) * SB_K);
#pragma unroll
        for (int kk = 0; kk < SB_K; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][tm * 8]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][tm * 8 + 4]);
            const float4 b = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tn * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (kt + 1 < nk) store(buf ^ 1);
        __syncthreads();
    }

    const int nb = n0 + tn * 4;
    if (nb >= a.cout) return;
    const float4 bias = *reinterpret_cast<const float4 *>(a.bias + nb);
    T *out = static_cast<T *>(a.out);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int m = m0 + tm * 8 + i;
        if (m >= M) continue;
        float4 v = make_float4(acc[i][0] + bias.x, acc[i][1] + bias.y, acc[i][2] + bias.z, acc[i][3] + bias.w);
        if (a.leaky) v = make_float4(lrelu(v.x), lrelu(v.y), lrelu(v.z), lrelu(v.w));
        if (a.accumulate) {
            const float4 o = ld4(out + (size_t)m * a.out_cs + nb);
            v = make_float4(v.x + o.x, v.y + o.y, v.z + o.z, v.w + o.w);
        }
        st4(out + (size_t)m * a.out_cs + nb, v);
    }
}

template <typename T>
cudaError_t launch_conv_simt(const ConvArgs &a, cudaStream_t st) {
    const int M = a.n * a.ho * a.wo;
    dim3 grid((M + SB_M - 1) / SB_M, (a.cout + SB_N - 1) / SB_N);
    conv_simt_kernel<T><<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// =====================================================================================
// First pyramid conv: 3 -> cout channels, stride 2, reading the planar float image with
// edge replication up to (Hp, Wp) (the padding to a multiple of 2^L) and zeros beyond.
// One thread per output pixel; weights [27][cout] in shared memory (cout == 16: in the
// kernel parameters).  cout % 4 == 0, <= 64.
// =====================================================================================
template <typename T>
__global__ void __launch_bounds__(256) conv_first_kernel(ConvFirstArgs a) {
    __shared__ __align__(16) float ws[27 * 64];
    __shared__ __align__(16) float bs[64];
    if (a.cout != 16) {
        for (int i = threadIdx.x; i < 27 * a.cout; i += blockDim.x) ws[i] = a.wk[i];
        for (int i = threadIdx.x; i < a.cout; i += blockDim.x) bs[i] = a.bias[i];
        __syncthreads();
    }
    pdl_wait();  // the weights above are constant; the image and the output follow the previous kernel
    const int ho = a.Hp / 2, wo = a.Wp / 2;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ho * wo) return;
    const int oy = idx / wo, ox = idx - oy * wo;
    const size_t plane = (size_t)a.H * a.W;
    float v[27];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
                const int iy = 2 * oy + ky - 1, ix = 2 * ox + kx - 1;
                float val = 0.f;
                if (iy >= 0 && iy < a.Hp && ix >= 0 && ix < a.Wp)
                    val = a.img[c * plane + (size_t)min(iy, a.H - 1) * a.W + min(ix, a.W - 1)];
                v[c * 9 + ky * 3 + kx] = val;
            }
    T *out = static_cast<T *>(a.out) + (size_t)idx * a.cout;
    if (a.cout == 16) {
        // weights straight from the parameter bank: 432 FMAs, no weight loads
        float acc[16];
#pragma unroll
        for (int o = 0; o < 16; ++o) acc[o] = a.b16[o];
#pragma unroll
        for (int k = 0; k < 27; ++k)
#pragma unroll
            for (int o = 0; o < 16; ++o) acc[o] = fmaf(a.w16[k * 16 + o], v[k], acc[o]);
#pragma unroll
        for (int o = 0; o < 16; o += 4)
            st4(out + o, make_float4(lrelu(acc[o]) * a.q_out, lrelu(acc[o + 1]) * a.q_out,
                                     lrelu(acc[o + 2]) * a.q_out, lrelu(acc[o + 3]) * a.q_out));
        return;
    }
    for (int o = 0; o < a.cout; o += 4) {
        float4 acc = *reinterpret_cast<const float4 *>(&bs[o]);
#pragma unroll
        for (int k = 0; k < 27; ++k) {
            const float4 w = *reinterpret_cast<const float4 *>(&ws[k * a.cout + o]);
            acc.x = fmaf(w.x, v[k], acc.x);
            acc.y = fmaf(w.y, v[k], acc.y);
            acc.z = fmaf(w.z, v[k], acc.z);
            acc.w = fmaf(w.w, v[k], acc.w);
        }
        st4(out + o, make_float4(lrelu(acc.x) * a.q_out, lrelu(acc.y) * a.q_out, lrelu(acc.z) * a.q_out,
                                 lrelu(acc.w) * a.q_out));
    }
}

template <typename T>
const void *conv_first_kernel_fn() {
    return reinterpret_cast<const void *>(conv_first_kernel<T>);
}

template <typename T>
cudaError_t launch_conv_first(const ConvFirstArgs &a, cudaStream_t st) {
    const int n = (a.Hp / 2) * (a.Wp / 2);
    return launch_pdl(conv_first_kernel<T>, dim3((n + 255) / 256), dim3(256), 0, st, a);
}

// =====================================================================================
// Flow head: r = conv5(cat(x3, x4)) (2 outputs, no activation), flow = up + r.
// One thread per pixel; weights [9 * cin][2] in dynamic shared memory.  cin % 4 == 0.
// =====================================================================================
template <typename T>
__global__ void __launch_bounds__(256) head_kernel(HeadArgs a) {
    extern __shared__ __align__(16) float hw[];
    const int nw = 9 * a.cin * 2;
    for (int i = threadIdx.x; i < nw; i += blockDim.x) hw[i] = a.wk[i];
    __syncthreads();
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int hwp = a.h * a.w;
    if (idx >= a.n * hwp) return;
    const int img = idx / hwp, rem = idx - img * hwp;
    const int y = rem / a.w, x = rem - y * a.w;
    const T *in = static_cast<const T *>(a.in);
    float u = a.bias[0], v = a.bias[1];
    for (int tap = 0; tap < 9; ++tap) {
        const int iy = y + tap / 3 - 1, ix = x + tap % 3 - 1;
        if (iy < 0 || iy >= a.h || ix < 0 || ix >= a.w) continue;
        const T *p = in + ((size_t)img * hwp + iy * a.w + ix) * a.in_cs;
        const float *wt = hw + tap * a.cin * 2;
        for (int c = 0; c < a.cin; c += 4) {
            const float4 f = ld4(p + c);
            const float4 w0 = *reinterpret_cast<const float4 *>(wt + 2 * c);
            const float4 w1 = *reinterpret_cast<const float4 *>(wt + 2 * c + 4);
            u = fmaf(f.x, w0.x, u); v = fmaf(f.x, w0.y, v);
            u = fmaf(f.y, w0.z, u); v = fmaf(f.y, w0.w, v);
            u = fmaf(f.z, w1.x, u); v = fmaf(f.z, w1.y, v);
            u = fmaf(f.w, w1.z, u); v = fmaf(f.w, w1.w, v);
        }
    }
    float2 up = make_float2(0.f, 0.f);
    if (a.up) up = reinterpret_cast<const float2 *>(a.up)[idx];
    reinterpret_cast<float2 *>(a.flow)[idx] = make_float2(up.x + u, up.y + v);
}

template <typename T>
cudaError_t launch_head(const HeadArgs &a, cudaStream_t st) {
    const int n = a.n * a.h * a.w;
    const size_t smem = sizeof(float) * 9 * a.cin * 2;
    head_kernel<T><<<(n + 255) / 256, 256, smem, st>>>(a);
    return cudaGetLastError();
}

// =====================================================================================
// Correlation (cost volume).  A block owns a 16x16 tile of output pixels of one batch
// entry.  For each chunk of 16 channels it stages the (16+2R)^2 halo of the other
// feature map in shared memory once and reuses it for all (2R+1)^2 displacements; the
// pixel's own features sit in registers.  Also copies the self features into the
// estimator input (x0) when self_copy is set.
// =====================================================================================
constexpr int CT = 16, CK = 16, CPS = CK + 4;  // tile, channel chunk, padded pixel stride

template <typename T, int R>
__global__ void __launch_bounds__(256) corr_kernel(CorrArgs a) {
    constexpr int HX = CT + 2 * R, ND = (2 * R + 1) * (2 * R + 1);
    __shared__ __align__(16) float tile[HX * HX * CPS];
    const int b = blockIdx.z;
    const int tx = threadIdx.x & (CT - 1), ty = threadIdx.x / CT;
    const int x0 = blockIdx.x * CT, y0 = blockIdx.y * CT;
    const int x = x0 + tx, y = y0 + ty;
    const bool valid = x < a.w && y < a.h;
    // (selects, not a.fs[b]: a runtime index into the parameter array would copy the
    // arguments to local memory)
    const int lq = b >> 1, ld = b & 1;  // lane pairs: lane and direction of entry b
    const T *fs = a.pair_lanes ? static_cast<const T *>(a.fs[0]) + (size_t)(lq + ld * a.pair_lanes) * a.fs_img
                  : a.fs_img   ? static_cast<const T *>(a.fs[0]) + b * a.fs_img
                               : static_cast<const T *>(b ? a.fs[1] : a.fs[0]);
    const T *fo = a.pair_lanes && a.pair_other
                      ? static_cast<const T *>(a.fo[0]) + (size_t)(lq + (1 - ld) * a.pair_lanes) * a.fo_img
                  : a.fo_img ? static_cast<const T *>(a.fo[0]) + b * a.fo_img
                             : static_cast<const T *>(b ? a.fo[1] : a.fo[0]);
    float acc[ND];
#pragma unroll
    for (int k = 0; k < ND; ++k) acc[k] = 0.f;

    for (int c0 = 0; c0 < a.c; c0 += CK) {
        __syncthreads();
        for (int i = threadIdx.x; i < HX * HX * (CK / 4); i += blockDim.x) {
            const int q = i % (CK / 4), p = i / (CK / 4);
            const int gy = y0 + p / HX - R, gx = x0 + p % HX - R;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gy >= 0 && gy < a.h && gx >= 0 && gx < a.w && c0 + q * 4 < a.c)
                v = ld4(fo + ((size_t)gy * a.w + gx) * a.fo_cs + c0 + q * 4);
            *reinterpret_cast<float4 *>(&tile[p * CPS + q * 4]) = v;
        }
        __syncthreads();
        float s[CK];
#pragma unroll
        for (int q = 0; q < CK / 4; ++q) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (valid && c0 + q * 4 < a.c) {
                v = ld4(fs + ((size_t)y * a.w + x) * a.fs_cs + c0 + q * 4);
                if (a.self_copy) {
                    // channel offset D is odd in general: element stores, not a vector store
                    T *dst = static_cast<T *>(a.self_copy) + (((size_t)b * a.h + y) * a.w + x) * a.out_cs + c0 + q * 4;
                    dst[0] = from_f<T>(v.x);
                    dst[1] = from_f<T>(v.y);
                    dst[2] = from_f<T>(v.z);
                    dst[3] = from_f<T>(v.w);
                }
            }
            s[4 * q] = v.x; s[4 * q + 1] = v.y; s[4 * q + 2] = v.z; s[4 * q + 3] = v.w;
        }
#pragma unroll
        for (int dy = 0; dy <= 2 * R; ++dy) {
#pragma unroll
            for (int dx = 0; dx <= 2 * R; ++dx) {
                const float *t = &tile[((ty + dy) * HX + tx + dx) * CPS];
                float sum = 0.f;
#pragma unroll
                for (int q = 0; q < CK / 4; ++q) {
                    const float4 v = *reinterpret_cast<const float4 *>(t + 4 * q);
                    sum = fmaf(s[4 * q], v.x, sum);
                    sum = fmaf(s[4 * q + 1], v.y, sum);
                    sum = fmaf(s[4 * q + 2], v.z, sum);
                    sum = fmaf(s[4 * q + 3], v.w, sum);
                }
                acc[dy * (2 * R + 1) + dx] += sum;
            }
        }
    }
    if (!valid) return;
    T *out = static_cast<T *>(a.out) + (((size_t)b * a.h + y) * a.w + x) * a.out_cs;
    const float inv = 1.f / (float)a.c;
#pragma unroll
    for (int k = 0; k < ND; ++k) out[k] = from_f<T>(lrelu(acc[k] * inv));
}

template <typename T>
cudaError_t launch_corr(const CorrArgs &a, cudaStream_t st) {
    dim3 grid((a.w + CT - 1) / CT, (a.h + CT - 1) / CT, a.n);
    switch (a.r) {
        case 1: corr_kernel<T, 1><<<grid, CT * CT, 0, st>>>(a); break;
        case 2: corr_kernel<T, 2><<<grid, CT * CT, 0, st>>>(a); break;
        case 3: corr_kernel<T, 3><<<grid, CT * CT, 0, st>>>(a); break;
        case 4: corr_kernel<T, 4><<<grid, CT * CT, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// =====================================================================================
// Bilinear feature warp, zeros off the map: out(x) = sum of on-map taps of f at x + flow.
// One thread per (pixel, 4Q channels).  With `coarse` set, the flow is the x2 upsampling of
// the coarser level's flow, computed here (and stored once per pixel) instead of by a
// separate pass.  The integer part of the sample position and the
// interpolation weights are taken from the flow alone (floor(u), u - floor(u)), which is
// exact in float32.
// =====================================================================================
template <typename T, int Q>
__global__ void __launch_bounds__(256) warp_kernel(WarpArgs a, int ng, uint32_t ng_magic) {
    // one thread per (pixel, group of Q quads of channels); block row y, image b; the
    // pixel is i / ng by a multiply-high (exact for i < 2^21, 2 <= ng <= 64; ng = 1 has
    // no 32-bit multiplier)
    pdl_wait();
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (uint32_t)(a.w * ng)) return;
    const int x = ng == 1 ? (int)i : (int)__umulhi(i, ng_magic), g = (int)i - x * ng;
    const int y = blockIdx.y, b = blockIdx.z;
    const size_t p = ((size_t)b * a.h + y) * a.w + x;
    float2 fl;
    if (a.coarse) {
        const int ch = a.h / 2, cw = a.w / 2;
        fl = upsampled_flow_at(a.coarse + (size_t)b * ch * cw * 2, ch, cw, 2, x, y);
        if (g == 0) {
            reinterpret_cast<float2 *>(a.up_out)[p] = fl;
            if (a.act) {
                T *dst = static_cast<T *>(a.act) + p * a.act_cs;
                dst[0] = from_f<T>(fl.x * a.act_q);
                dst[1] = from_f<T>(fl.y * a.act_q);
            }
        }
    } else {
        fl = reinterpret_cast<const float2 *>(a.flow)[p];
    }
    const float u = fminf(fmaxf(fl.x, -1e6f), 1e6f), v = fminf(fmaxf(fl.y, -1e6f), 1e6f);
    const float fu = floorf(u), fv = floorf(v);
    const float ax = u - fu, ay = v - fv;
    const int xa = x + (int)fu, ya = y + (int)fv;
    const T *f = a.pair_lanes ? static_cast<const T *>(a.f[0]) + (size_t)((b >> 1) + (1 - (b & 1)) * a.pair_lanes) * a.f_img
                 : a.f_img    ? static_cast<const T *>(a.f[0]) + b * a.f_img
                              : static_cast<const T *>(b ? a.f[1] : a.f[0]);  // no runtime index into the arguments
    float4 acc[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
            const int xx = xa + dx, yy = ya + dy;
            if (xx < 0 || xx >= a.w || yy < 0 || yy >= a.h) continue;
            const float wgt = (dx ? ax : 1.f - ax) * (dy ? ay : 1.f - ay);
            const T *t = f + ((size_t)yy * a.w + xx) * a.f_cs + g * (4 * Q);
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                const float4 tv = ld4(t + 4 * j);
                acc[j].x = fmaf(wgt, tv.x, acc[j].x);
                acc[j].y = fmaf(wgt, tv.y, acc[j].y);
                acc[j].z = fmaf(wgt, tv.z, acc[j].z);
                acc[j].w = fmaf(wgt, tv.w, acc[j].w);
            }
        }
    }
    T *o = static_cast<T *>(a.out) + p * a.out_cs + g * (4 * Q);
#pragma unroll
    for (int j = 0; j < Q; ++j) st4(o + 4 * j, acc[j]);
}

template <typename T>
cudaError_t launch_warp(const WarpArgs &a, cudaStream_t st) {
    // Q quads of channels per thread (2 where c / 4 is even), so the flow sample and its
    // taps are computed once for 4Q channels (Q = 4: 40 registers, fewer warps; slower)
    const int nq = a.c / 4, q = nq % 2 == 0 ? 2 : 1, ng = nq / q;
    if (ng > 64 || (size_t)a.w * ng >= (1u << 21)) return cudaErrorInvalidValue;
    const uint32_t magic = ng > 1 ? (uint32_t)((0x100000000ull + (unsigned)ng - 1) / (unsigned)ng) : 0u;
    const dim3 grid((unsigned)((a.w * ng + 255) / 256), (unsigned)a.h, (unsigned)a.n);
    if (q == 2) return launch_pdl(warp_kernel<T, 2>, grid, dim3(256), 0, st, a, ng, magic);
    return launch_pdl(warp_kernel<T, 1>, grid, dim3(256), 0, st, a, ng, magic);
}

// =====================================================================================
// Flow upsampling by s (values times s), optionally also written into an activation
// buffer (the up-flow channels of the estimator input).
// =====================================================================================
template <typename T>
__global__ void __launch_bounds__(256) up_kernel(UpArgs a) {
    const int H = a.h * a.s, W = a.w * a.s;
    const size_t total = (size_t)a.n * H * W;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int b = (int)(i / ((size_t)H * W));
    const int rem = (int)(i - (size_t)b * H * W);
    const int Y = rem / W, X = rem - Y * W;
    const float2 v = upsampled_flow_at(a.flow + (size_t)b * a.h * a.w * 2, a.h, a.w, a.s, X, Y);
    reinterpret_cast<float2 *>(a.out)[i] = v;
    if (a.act) {
        T *p = static_cast<T *>(a.act) + i * a.act_cs;
        p[0] = from_f<T>(v.x);
        p[1] = from_f<T>(v.y);
    }
}

template <typename T>
cudaError_t launch_up(const UpArgs &a, cudaStream_t st) {
    const size_t total = (size_t)a.n * a.h * a.s * a.w * a.s;
    up_kernel<T><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

// =====================================================================================
// Element conversions between float and the activation type (used by the stage ops).
// =====================================================================================
template <typename T>
__global__ void to_act_kernel(const float *in, size_t n, T *out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = from_f<T>(in[i]);
}
template <typename T>
__global__ void from_act_kernel(const T *in, size_t n, float *out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = to_f(in[i]);
}
template <typename T>
cudaError_t launch_to_act(const float *in, size_t n, T *out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    to_act_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, n, out);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_from_act(const T *in, size_t n, float *out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    from_act_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, n, out);
    return cudaGetLastError();
}

#define TC_INST(T)                                                                      \
    template cudaError_t launch_conv_simt<T>(const ConvArgs &, cudaStream_t);           \
    template cudaError_t launch_conv_first<T>(const ConvFirstArgs &, cudaStream_t);     \
    template const void *conv_first_kernel_fn<T>();                                     \
    template cudaError_t launch_head<T>(const HeadArgs &, cudaStream_t);                \
    template cudaError_t launch_corr<T>(const CorrArgs &, cudaStream_t);                \
    template cudaError_t launch_warp<T>(const WarpArgs &, cudaStream_t);                \
    template cudaError_t launch_up<T>(const UpArgs &, cudaStream_t);                    \
    template cudaError_t launch_to_act<T>(const float *, size_t, T *, cudaStream_t);    \
    template cudaError_t launch_from_act<T>(const T *, size_t, float *, cudaStream_t);
TC_INST(float)
TC_INST(__nv_bfloat16)
TC_INST(__half)
#undef TC_INST

// =====================================================================================
// amax of a channel window of an NHWC activation buffer, folded into *slot with an atomic
// max on the float's bit pattern (values are >= 0, so their bit patterns order like them).
// =====================================================================================
template <typename T>
__global__ void __launch_bounds__(256) amax_kernel(const T *base, size_t npix, int cs, int nc, unsigned *slot) {
    float m = 0.f;
    const size_t n = npix * (size_t)nc;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t p = i / nc;
        const int c = (int)(i - p * nc);
        m = fmaxf(m, fabsf(to_f(base[p * cs + c])));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(slot, __float_as_uint(m));
}

template <typename T>
cudaError_t launch_amax(const T *base, size_t npix, int cs, int nc, unsigned *slot, cudaStream_t st) {
    const size_t n = npix * (size_t)nc;
    if (n == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((n + 255) / 256 < 1184 ? (n + 255) / 256 : 1184);
    amax_kernel<T><<<blocks, 256, 0, st>>>(base, npix, cs, nc, slot);
    return cudaGetLastError();
}
template cudaError_t launch_amax<float>(const float *, size_t, int, int, unsigned *, cudaStream_t);
template cudaError_t launch_amax<__nv_bfloat16>(const __nv_bfloat16 *, size_t, int, int, unsigned *, cudaStream_t);
template cudaError_t launch_amax<__half>(const __half *, size_t, int, int, unsigned *, cudaStream_t);

// E4M3 activations: only the kernels an E4M3 stream runs outside the tensor cores.
template cudaError_t launch_conv_first<__nv_fp8_e4m3>(const ConvFirstArgs &, cudaStream_t);
template const void *conv_first_kernel_fn<__nv_fp8_e4m3>();
template cudaError_t launch_warp<__nv_fp8_e4m3>(const WarpArgs &, cudaStream_t);
template cudaError_t launch_to_act<__nv_fp8_e4m3>(const float *, size_t, __nv_fp8_e4m3 *, cudaStream_t);
template cudaError_t launch_from_act<__nv_fp8_e4m3>(const __nv_fp8_e4m3 *, size_t, float *, cudaStream_t);

}  // namespace tc
