// Kernels of the training step (forward is shared with inference): backward passes of the
// 3x3 convolution (data and weight gradients), of the correlation, of the bilinear feature
// warp and of the x2 flow upsampling; the multi-scale end-point-error loss (Eq. 10 per
// level); the ground-truth flow pyramid; weight packing from the float32 master copy; and
// the AdamW update.  Gradients are float32 throughout; saved activations are float or
// bfloat16 (the forward's activation type T).
#include "train_kernels.cuh"

namespace tc {
namespace train {

namespace {

__device__ __forceinline__ float lrelu_grad(float y) { return y > 0.f ? 1.f : 0.1f; }

inline unsigned blocks_for(size_t n, int threads = 256) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

// ---------------------------------------------------------------------------- packing

// Master weights [cout][cin][3][3] -> forward layout [9][cin_p][cout] (k = tap cin_p + c),
// zero for c >= cin.  With round_bf16 the values are rounded to bfloat16 (the BF16 path's
// operands).
__global__ void pack_fwd_kernel(const float *w, int cout, int cin, int cin_p, int round_bf16, float *wk) {
    const size_t n = (size_t)9 * cin_p * cout;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int o = (int)(i % cout);
    const size_t k = i / cout;
    const int c = (int)(k % cin_p), tap = (int)(k / cin_p);
    float v = 0.f;
    if (c < cin) v = w[((size_t)o * cin + c) * 9 + tap];
    if (round_bf16) v = __bfloat162float(__float2bfloat16_rn(v));
    wk[i] = v;
}

// Master weights -> data-gradient layout [9][cout_p][cin_p] of the flipped, transposed
// kernel: the data gradient of a stride-1 conv is the stride-1 conv of the output gradient
// with W'[o'=c][c'=o][tap] = W[o][c][8 - tap].
__global__ void pack_dgrad_kernel(const float *w, int cout, int cin, int cout_p, int cin_p, float *wk) {
    const size_t n = (size_t)9 * cout_p * cin_p;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % cin_p);
    const size_t k = i / cin_p;
    const int o = (int)(k % cout_p), tap = (int)(k / cout_p);
    float v = 0.f;
    if (c < cin && o < cout) v = w[((size_t)o * cin + c) * 9 + (8 - tap)];
    wk[i] = v;
}

cudaError_t pack_fwd(const float *w, int cout, int cin, int cin_p, bool round_bf16, float *wk, cudaStream_t st) {
    const size_t n = (size_t)9 * cin_p * cout;
    pack_fwd_kernel<<<blocks_for(n), 256, 0, st>>>(w, cout, cin, cin_p, round_bf16 ? 1 : 0, wk);
    return cudaGetLastError();
}

cudaError_t pack_dgrad(const float *w, int cout, int cin, int cout_p, int cin_p, float *wk, cudaStream_t st) {
    const size_t n = (size_t)9 * cout_p * cin_p;
    pack_dgrad_kernel<<<blocks_for(n), 256, 0, st>>>(w, cout, cin, cout_p, cin_p, wk);
    return cudaGetLastError();
}

// Master weights -> the tensor-core packing [9][bn][cinp] (bfloat16, K-major rows):
//   mode 0 (forward): row o, channel c = W[o][c][tap] for o < cout, c < cin;
//   mode 1 (data gradient, output channels [lo, lo + n) of the layer's input): row o,
//   channel c = W[c][lo + o][8 - tap] for o < n, c < cout.
// Zero elsewhere.
__global__ void pack_tc_kernel(const float *w, int cout, int cin, int mode, int lo, int n, int bn, int cinp,
                               __nv_bfloat16 *out) {
    const size_t total = (size_t)9 * bn * cinp;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int c = (int)(i % cinp);
    const size_t r = i / cinp;
    const int o = (int)(r % bn), tap = (int)(r / bn);
    float v = 0.f;
    if (mode == 0) {
        if (o < cout && c < cin) v = w[((size_t)o * cin + c) * 9 + tap];
    } else {
        if (o < n && c < cout) v = w[((size_t)c * cin + lo + o) * 9 + (8 - tap)];
    }
    out[i] = __float2bfloat16_rn(v);
}

cudaError_t pack_tc(const float *w, int cout, int cin, int mode, int lo, int n, int bn, int cinp, void *out,
                    cudaStream_t st) {
    const size_t total = (size_t)9 * bn * cinp;
    pack_tc_kernel<<<blocks_for(total), 256, 0, st>>>(w, cout, cin, mode, lo, n, bn, cinp,
                                                     static_cast<__nv_bfloat16 *>(out));
    return cudaGetLastError();
}

// dz = dy LeakyReLU'(y) written as float (dz, may be NULL) and bfloat16 (dzh, may be NULL),
// and, for a stride-2 conv, bfloat16 into the zeroed dilated map dzh_dil (hd x wd).
template <typename T>
__global__ void lrelu_bwd2_kernel(const float *dy, int dy_cs, const T *y, int y_cs, int leaky, size_t npix, int nc,
                                  float *dz, __nv_bfloat16 *dzh, __nv_bfloat16 *dzh_dil, int ho, int wo, int hd, int wd) {
    const size_t total = npix * nc;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const size_t p = i / nc;
    const int c = (int)(i - p * nc);
    float g = dy[p * dy_cs + c];
    if (leaky) g *= lrelu_grad(to_f(y[p * y_cs + c]));
    if (dz) dz[i] = g;
    const __nv_bfloat16 gh = __float2bfloat16_rn(g);
    if (dzh) dzh[i] = gh;
    if (dzh_dil) {
        const size_t hw = (size_t)ho * wo;
        const size_t b = p / hw, r = p - b * hw;
        const int oy = (int)(r / wo), ox = (int)(r - (size_t)oy * wo);
        dzh_dil[((b * hd + 2 * oy) * (size_t)wd + 2 * ox) * nc + c] = gh;
    }
}

template <typename T>
cudaError_t lrelu_bwd2(const float *dy, int dy_cs, const T *y, int y_cs, bool leaky, size_t npix, int nc, float *dz,
                       void *dzh, void *dzh_dil, int ho, int wo, int hd, int wd, cudaStream_t st) {
    const size_t total = npix * nc;
    if (total == 0) return cudaSuccess;
    lrelu_bwd2_kernel<T><<<blocks_for(total), 256, 0, st>>>(dy, dy_cs, y, y_cs, leaky ? 1 : 0, npix, nc, dz,
                                                           static_cast<__nv_bfloat16 *>(dzh),
                                                           static_cast<__nv_bfloat16 *>(dzh_dil), ho, wo, hd, wd);
    return cudaGetLastError();
}

// Planar images [n][3][h][w] (two batches, a then b) -> NHWC [2n][h][w][4] with a zero 4th
// channel, in the activation type.
template <typename T>
__global__ void pack_images_kernel(const float *a, const float *b, int n, int h, int w, T *out) {
    const size_t hw = (size_t)h * w, total = 2 * (size_t)n * hw;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const size_t img = i / hw, p = i - img * hw;
    const float *src = img < (size_t)n ? a + img * 3 * hw : b + (img - n) * 3 * hw;
    st4(out + 4 * i, make_float4(src[p], src[hw + p], src[2 * hw + p], 0.f));
}

template <typename T>
cudaError_t pack_images(const float *a, const float *b, int n, int h, int w, T *out, cudaStream_t st) {
    pack_images_kernel<T><<<blocks_for(2 * (size_t)n * h * w), 256, 0, st>>>(a, b, n, h, w, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------ LeakyReLU grad

// dz = dy * LeakyReLU'(y) over a channel window: dy, y are [npix][*_cs] with the window at
// the pointers; dz is dense [npix][nc].  With dil set, dz is written dilated for the data
// gradient of a stride-2 conv: pixel (b, oy, ox) of an (ho, wo) map goes to (b, 2oy, 2ox) of
// a zeroed (hd, wd) map (dz_dil, [n][hd][wd][nc]; hd, wd = the conv's input size).
template <typename T>
__global__ void lrelu_bwd_kernel(const float *dy, int dy_cs, const T *y, int y_cs, int leaky, size_t npix, int nc,
                                 float *dz, float *dz_dil, int ho, int wo, int hd, int wd) {
    const size_t total = npix * nc;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const size_t p = i / nc;
    const int c = (int)(i - p * nc);
    float g = dy[p * dy_cs + c];
    if (leaky) g *= lrelu_grad(to_f(y[p * y_cs + c]));
    if (dz) dz[i] = g;
    if (dz_dil) {
        const size_t hw = (size_t)ho * wo;
        const size_t b = p / hw, r = p - b * hw;
        const int oy = (int)(r / wo), ox = (int)(r - (size_t)oy * wo);
        dz_dil[((b * hd + 2 * oy) * (size_t)wd + 2 * ox) * nc + c] = g;
    }
}

template <typename T>
cudaError_t lrelu_bwd(const float *dy, int dy_cs, const T *y, int y_cs, bool leaky, size_t npix, int nc, float *dz,
                      float *dz_dil, int ho, int wo, int hd, int wd, cudaStream_t st) {
    const size_t total = npix * nc;
    if (total == 0) return cudaSuccess;
    lrelu_bwd_kernel<T><<<blocks_for(total), 256, 0, st>>>(dy, dy_cs, y, y_cs, leaky ? 1 : 0, npix, nc, dz, dz_dil,
                                                          ho, wo, hd, wd);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- weight grad

// dW[o][c][tap] += sum over output pixels p of dz[p][o] x(p, tap)[c], the input pixel under
// tap (ky, kx) of output pixel (oy, ox) being (s oy + ky - 1, s ox + kx - 1) (zero off the
// map).  Block: one tap, 32 output x 32 input channels, a chunk of WG_P output pixels staged
// through shared memory in steps of 32; each of the 256 threads owns 2 x 2 outputs.
// Partial sums of the chunk are added to dW with atomics (split over pixel chunks).
constexpr int WG_T = 32, WG_S = 32, WG_P = 2048;

// Output pixels per chunk: at least WG_P, and enough that 9 x chunks fits the grid's z.
inline size_t wgrad_chunk(size_t P) {
    size_t c = WG_P;
    while ((P + c - 1) / c * 9 > 65535) c *= 2;
    return c;
}

template <typename T>
__global__ void __launch_bounds__(256) wgrad_kernel(WgradArgs<T> a, size_t ppc) {
    __shared__ float zs[WG_S][WG_T + 1];
    __shared__ float xs[WG_S][WG_T + 1];
    const int tap = blockIdx.z % 9, chunk = blockIdx.z / 9;
    const int ky = tap / 3, kx = tap % 3;
    const int o0 = blockIdx.x * WG_T, c0 = blockIdx.y * WG_T;
    const int tid = threadIdx.x;
    const int to = (tid >> 4) * 2, tcn = (tid & 15) * 2;
    const size_t P = (size_t)a.n * a.ho * a.wo;
    const size_t p_begin = (size_t)chunk * ppc;
    const size_t p_end = p_begin + ppc < P ? p_begin + ppc : P;
    float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    const int hwo = a.ho * a.wo;
    for (size_t p0 = p_begin; p0 < p_end; p0 += WG_S) {
        // stage dz[p0 .. p0+32)[o0 .. o0+32) and x(p, tap)[c0 .. c0+32)
        for (int i = tid; i < WG_S * WG_T; i += 256) {
            const int pp = i / WG_T, k = i % WG_T;
            const size_t p = p0 + pp;
            float zv = 0.f, xv = 0.f;
            if (p < p_end) {
                if (o0 + k < a.cout) zv = a.dz[p * a.dz_cs + o0 + k];
                if (c0 + k < a.cin) {
                    const int b = (int)(p / hwo), r = (int)(p - (size_t)b * hwo);
                    const int oy = r / a.wo, ox = r - oy * a.wo;
                    const int iy = oy * a.stride + ky - 1, ix = ox * a.stride + kx - 1;
                    if (iy >= 0 && iy < a.h && ix >= 0 && ix < a.w)
                        xv = to_f(a.x[(((size_t)b * a.h + iy) * a.w + ix) * a.x_cs + c0 + k]);
                }
            }
            zs[pp][k] = zv;
            xs[pp][k] = xv;
        }
        __syncthreads();
#pragma unroll 8
        for (int pp = 0; pp < WG_S; ++pp) {
            const float z0 = zs[pp][to], z1 = zs[pp][to + 1];
            const float x0 = xs[pp][tcn], x1 = xs[pp][tcn + 1];
            acc[0][0] = fmaf(z0, x0, acc[0][0]);
            acc[0][1] = fmaf(z0, x1, acc[0][1]);
            acc[1][0] = fmaf(z1, x0, acc[1][0]);
            acc[1][1] = fmaf(z1, x1, acc[1][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int o = o0 + to + i, c = c0 + tcn + j;
            if (o < a.cout && c < a.cin) atomicAdd(&a.dw[((size_t)o * a.cin + c) * 9 + tap], acc[i][j]);
        }
}

// db[o] += sum over pixels of dz[p][o]: one block per (channel group of 32, pixel chunk).
__global__ void __launch_bounds__(256) bgrad_kernel(const float *dz, int dz_cs, size_t P, int cout, float *db,
                                                    size_t ppc) {
    __shared__ float part[8][32];
    const int o = blockIdx.x * 32 + (threadIdx.x & 31);
    const int lane_row = threadIdx.x >> 5;
    const size_t p_begin = (size_t)blockIdx.y * ppc;
    const size_t p_end = p_begin + ppc < P ? p_begin + ppc : P;
    float s = 0.f;
    if (o < cout)
        for (size_t p = p_begin + lane_row; p < p_end; p += 8) s += dz[p * dz_cs + o];
    part[lane_row][threadIdx.x & 31] = s;
    __syncthreads();
    if (lane_row == 0 && o < cout) {
        float t = 0.f;
        for (int r = 0; r < 8; ++r) t += part[r][threadIdx.x & 31];
        atomicAdd(&db[o], t);
    }
}

template <typename T>
cudaError_t wgrad(const WgradArgs<T> &a, float *db, cudaStream_t st) {
    const size_t P = (size_t)a.n * a.ho * a.wo;
    if (P == 0) return cudaSuccess;
    const size_t ppc = wgrad_chunk(P);
    const unsigned chunks = (unsigned)((P + ppc - 1) / ppc);
    dim3 grid((a.cout + WG_T - 1) / WG_T, (a.cin + WG_T - 1) / WG_T, 9 * chunks);
    wgrad_kernel<T><<<grid, 256, 0, st>>>(a, ppc);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !db) return e;
    dim3 g2((a.cout + 31) / 32, chunks);
    bgrad_kernel<<<g2, 256, 0, st>>>(a.dz, a.dz_cs, P, a.cout, db, ppc);
    return cudaGetLastError();
}

// Channel-major, zero-bordered ("CP") copies for the tensor-core weight gradient: pixel
// (b, y, x) of an n_img x h x w map sits at q = (b (h + 2) + y + 1) wp + x + 1.
//   x_to_cp: three copies shifted by kx - 1 columns: out_kx[c][q] = x at column
//   (q's column + kx - 2), zero off the map and for c >= cin (rows up to n).
//   dz_to_cp: out[o][q] = dz of output pixel (y / s, x / s) when s divides y and x
//   (s = stride), zero elsewhere; dz dense [n_img][ho][wo][cout] float.
template <typename T>
__global__ void x_to_cp_kernel(const T *x, int x_cs, int n_img, int h, int w, int cin, int wp, int n, int vec,
                               __nv_bfloat16 *o0, __nv_bfloat16 *o1, __nv_bfloat16 *o2) {
    const long long P = (long long)n_img * (h + 2) * wp;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * 3) return;
    const int kx = (int)(i / P);
    const long long q = i - (long long)kx * P;
    const int xx = (int)(q % wp);
    const long long r = q / wp;
    const int yy = (int)(r % (h + 2)), b = (int)(r / (h + 2));
    const int iy = yy - 1, ix = xx + kx - 2;
    __nv_bfloat16 *out = (kx == 0 ? o0 : (kx == 1 ? o1 : o2)) + q;
    const bool in = iy >= 0 && iy < h && ix >= 0 && ix < w;
    const T *src = x + (((size_t)b * h + (in ? iy : 0)) * w + (in ? ix : 0)) * x_cs;
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
    if (vec) {
        // bf16 input with 16-byte aligned pixels: 8 channels per load; channels past the
        // pixel stride read as zero (channels in [cin, x_cs) are zero in the buffers)
        for (int c0 = 0; c0 < n; c0 += 8) {
            uint4 u = make_uint4(0, 0, 0, 0);
            if (in && c0 < x_cs) u = *reinterpret_cast<const uint4 *>(src + c0);
            const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&u);
#pragma unroll
            for (int k = 0; k < 8; ++k) out[(size_t)(c0 + k) * P] = c0 + k < cin ? e[k] : zero;
        }
    } else {
        for (int c = 0; c < n; ++c) out[(size_t)c * P] = __float2bfloat16_rn((in && c < cin) ? to_f(src[c]) : 0.f);
    }
    // the row of ones (bias gradient through the center tap)
    if (kx == 1 && cin < n) out[(size_t)cin * P] = __float2bfloat16_rn(in ? 1.f : 0.f);
}

// dz_to_cp also sums each channel over the pixels it moves (the bias gradient): per-thread
// partial sums for its 4-channel groups, reduced over the block in shared memory, one
// atomic add per block and channel into db.
__global__ void __launch_bounds__(256) dz_to_cp_kernel(const float *dz, int dz_cs, int n_img, int h, int w, int ho,
                                                       int wo, int stride, int cout, int wp, __nv_bfloat16 *out,
                                                       float *db) {
    extern __shared__ float bsum[];  // [cout]
    for (int o = threadIdx.x; o < cout; o += blockDim.x) bsum[o] = 0.f;
    __syncthreads();
    const long long P = (long long)n_img * (h + 2) * wp;
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool in = false;
    const float *src = dz;
    if (q < P) {
        const int xx = (int)(q % wp);
        const long long r = q / wp;
        const int yy = (int)(r % (h + 2)), b = (int)(r / (h + 2));
        const int iy = yy - 1, ix = xx - 1;
        in = iy >= 0 && iy < h && ix >= 0 && ix < w && iy % stride == 0 && ix % stride == 0;
        const int oy = iy / stride, ox = ix / stride;
        in = in && oy < ho && ox < wo;
        src = dz + (((size_t)b * ho + (in ? oy : 0)) * wo + (in ? ox : 0)) * dz_cs;
        if ((cout & 3) == 0 && (dz_cs & 3) == 0) {
            for (int o = 0; o < cout; o += 4) {
                const float4 v = in ? *reinterpret_cast<const float4 *>(src + o) : make_float4(0.f, 0.f, 0.f, 0.f);
                out[(size_t)o * P + q] = __float2bfloat16_rn(v.x);
                out[(size_t)(o + 1) * P + q] = __float2bfloat16_rn(v.y);
                out[(size_t)(o + 2) * P + q] = __float2bfloat16_rn(v.z);
                out[(size_t)(o + 3) * P + q] = __float2bfloat16_rn(v.w);
            }
        } else {
            for (int o = 0; o < cout; ++o) out[(size_t)o * P + q] = __float2bfloat16_rn(in ? src[o] : 0.f);
        }
    }
    if (db) {
        // warp-level sums per channel (lanes are consecutive pixels), then shared, then global
        const unsigned full = 0xffffffffu;
        for (int o = 0; o < cout; ++o) {
            float v = in ? src[o] : 0.f;
#pragma unroll
            for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(full, v, m);
            if ((threadIdx.x & 31) == 0 && v != 0.f) atomicAdd(&bsum[o], v);
        }
        __syncthreads();
        for (int o = threadIdx.x; o < cout; o += blockDim.x)
            if (bsum[o] != 0.f) atomicAdd(&db[o], bsum[o]);
    }
}

template <typename T>
cudaError_t x_to_cp(const T *x, int x_cs, int n_img, int h, int w, int cin, int wp, int n, void *const out[3],
                    cudaStream_t st) {
    const long long P = (long long)n_img * (h + 2) * wp;
    const int vec = sizeof(T) == 2 && x_cs % 8 == 0 && reinterpret_cast<uintptr_t>(x) % 16 == 0 && n % 8 == 0;
    x_to_cp_kernel<T><<<blocks_for((size_t)P * 3), 256, 0, st>>>(x, x_cs, n_img, h, w, cin, wp, n, vec,
                                                                static_cast<__nv_bfloat16 *>(out[0]),
                                                                static_cast<__nv_bfloat16 *>(out[1]),
                                                                static_cast<__nv_bfloat16 *>(out[2]));
    return cudaGetLastError();
}

cudaError_t dz_to_cp(const float *dz, int dz_cs, int n_img, int h, int w, int ho, int wo, int stride, int cout, int wp,
                     void *out, float *db, cudaStream_t st) {
    const long long P = (long long)n_img * (h + 2) * wp;
    dz_to_cp_kernel<<<blocks_for((size_t)P), 256, (size_t)cout * sizeof(float), st>>>(
        dz, dz_cs, n_img, h, w, ho, wo, stride, cout, wp, static_cast<__nv_bfloat16 *>(out), db);
    return cudaGetLastError();
}

cudaError_t bgrad(const float *dz, int dz_cs, size_t P, int cout, float *db, cudaStream_t st) {
    if (P == 0) return cudaSuccess;
    const size_t ppc = wgrad_chunk(P);
    const unsigned chunks = (unsigned)((P + ppc - 1) / ppc);
    dim3 g2((cout + 31) / 32, chunks);
    bgrad_kernel<<<g2, 256, 0, st>>>(dz, dz_cs, P, cout, db, ppc);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------- head dgrad

// Data gradient of the flow head (2 outputs, no activation): dx[p][c] (+)= sum over taps and
// o of W[o][c][tap] dflow[p - (tap offset)][o].  One thread per (pixel, 4 channels).
__global__ void head_dgrad_kernel(const float *dflow, const float *w, int cin, int n, int h, int w_, float *dx,
                                  int dx_cs, int accumulate) {
    const int nq = (cin + 3) / 4;
    const size_t total = (size_t)n * h * w_ * nq;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int q = (int)(i % nq);
    const size_t p = i / nq;
    const int hw = h * w_;
    const int b = (int)(p / hw), r = (int)(p - (size_t)b * hw);
    const int y = r / w_, x = r - y * w_;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int tap = 0; tap < 9; ++tap) {
        // output pixel (y - (ky - 1), x - (kx - 1)) reads this pixel through tap (ky, kx)
        const int oy = y - (tap / 3 - 1), ox = x - (tap % 3 - 1);
        if (oy < 0 || oy >= h || ox < 0 || ox >= w_) continue;
        const float2 g = reinterpret_cast<const float2 *>(dflow)[((size_t)b * h + oy) * w_ + ox];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = q * 4 + j;
            if (c < cin) acc[j] += w[((size_t)0 * cin + c) * 9 + tap] * g.x + w[((size_t)1 * cin + c) * 9 + tap] * g.y;
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = q * 4 + j;
        if (c >= cin) continue;
        float *d = dx + p * dx_cs + c;
        *d = accumulate ? *d + acc[j] : acc[j];
    }
}

cudaError_t head_dgrad(const float *dflow, const float *w, int cin, int n, int h, int w_, float *dx, int dx_cs,
                       bool accumulate, cudaStream_t st) {
    const size_t total = (size_t)n * h * w_ * ((cin + 3) / 4);
    head_dgrad_kernel<<<blocks_for(total), 256, 0, st>>>(dflow, w, cin, n, h, w_, dx, dx_cs, accumulate ? 1 : 0);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------ correlation

// Backward of cost[p][k] = LeakyReLU((1/C) sum_c fs[p][c] fo[p + d_k][c]) (zero where
// p + d_k is off the map).  dpre = dcost LeakyReLU'(cost) is formed on the fly from the
// saved cost volume.
//   dfs[p][c] (+)= (1/C) sum_k dpre[p][k] fo[p + d_k][c]
//   dfo[q][c] (+)= (1/C) sum_k dpre[q - d_k][k] fs[q - d_k][c]
// One thread per (pixel, 4 channels), both gathers (no atomics).
template <typename T>
__global__ void corr_bwd_kernel(CorrBwdArgs<T> a) {
    const int nq = a.c / 4;
    const size_t total = (size_t)a.n * a.h * a.w * nq;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int q = (int)(i % nq);
    const size_t p = i / nq;
    const int hw = a.h * a.w;
    const int b = (int)(p / hw), r = (int)(p - (size_t)b * hw);
    const int y = r / a.w, x = r - y * a.w;
    const int n1 = 2 * a.r + 1;
    const float inv = 1.f / (float)a.c;
    float4 gs = make_float4(0.f, 0.f, 0.f, 0.f), go = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = 0; k < n1 * n1; ++k) {
        const int dy = k / n1 - a.r, dx = k % n1 - a.r;
        // self side: this pixel's displacement k
        {
            const int yy = y + dy, xx = x + dx;
            if (yy >= 0 && yy < a.h && xx >= 0 && xx < a.w) {
                const size_t pc = p * a.cost_cs + k;
                const float g = a.dcost[p * a.dcost_cs + k] * lrelu_grad(to_f(a.cost[pc])) * inv;
                const float4 o = ld4(a.fo + (((size_t)b * a.h + yy) * a.w + xx) * a.fo_cs + q * 4);
                gs.x = fmaf(g, o.x, gs.x); gs.y = fmaf(g, o.y, gs.y);
                gs.z = fmaf(g, o.z, gs.z); gs.w = fmaf(g, o.w, gs.w);
            }
        }
        // other side: pixel q - d_k reads this pixel through displacement k
        {
            const int yy = y - dy, xx = x - dx;
            if (yy >= 0 && yy < a.h && xx >= 0 && xx < a.w) {
                const size_t ps = ((size_t)b * a.h + yy) * a.w + xx;
                const float g = a.dcost[ps * a.dcost_cs + k] * lrelu_grad(to_f(a.cost[ps * a.cost_cs + k])) * inv;
                const float4 s = ld4(a.fs + ps * a.fs_cs + q * 4);
                go.x = fmaf(g, s.x, go.x); go.y = fmaf(g, s.y, go.y);
                go.z = fmaf(g, s.z, go.z); go.w = fmaf(g, s.w, go.w);
            }
        }
    }
    if (a.dfs) {
        float *d = a.dfs + p * a.dfs_cs + q * 4;
        if (a.accumulate) { d[0] += gs.x; d[1] += gs.y; d[2] += gs.z; d[3] += gs.w; }
        else { d[0] = gs.x; d[1] = gs.y; d[2] = gs.z; d[3] = gs.w; }
    }
    if (a.dfo) {
        float *d = a.dfo + p * a.dfo_cs + q * 4;
        if (a.accumulate) { d[0] += go.x; d[1] += go.y; d[2] += go.z; d[3] += go.w; }
        else { d[0] = go.x; d[1] = go.y; d[2] = go.z; d[3] = go.w; }
    }
}

template <typename T>
cudaError_t corr_bwd(const CorrBwdArgs<T> &a, cudaStream_t st) {
    const size_t total = (size_t)a.n * a.h * a.w * (a.c / 4);
    if (total == 0) return cudaSuccess;
    corr_bwd_kernel<T><<<blocks_for(total), 256, 0, st>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------- warp

// Backward of out[p][c] = sum over on-map taps t of w_t(p) f[tap_t(p)][c] (bilinear at
// p + flow(p), zeros off the map):
//   df[tap_t(p)][c] += w_t(p) dout[p][c]                        (scatter, float atomics)
//   dflow[p] (+)= sum_c dout[p][c] (d out[p][c] / d flow(p))    (per pixel)
// One thread per pixel, looping over the channels.
template <typename T>
__global__ void warp_bwd_kernel(WarpBwdArgs<T> a) {
    const size_t total = (size_t)a.n * a.h * a.w;
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= total) return;
    const int hw = a.h * a.w;
    const int b = (int)(p / hw), r = (int)(p - (size_t)b * hw);
    const int y = r / a.w, x = r - y * a.w;
    const float2 fl = reinterpret_cast<const float2 *>(a.flow)[p];
    const float u = fminf(fmaxf(fl.x, -1e6f), 1e6f), v = fminf(fmaxf(fl.y, -1e6f), 1e6f);
    const float fu = floorf(u), fv = floorf(v);
    const float ax = u - fu, ay = v - fv;
    const int xa = x + (int)fu, ya = y + (int)fv;
    bool ok[4];
    size_t idx[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int xx = xa + (t & 1), yy = ya + (t >> 1);
        ok[t] = xx >= 0 && xx < a.w && yy >= 0 && yy < a.h;
        idx[t] = ok[t] ? (((size_t)b * a.h + yy) * a.w + xx) : 0;
    }
    const float wt[4] = {(1.f - ax) * (1.f - ay), ax * (1.f - ay), (1.f - ax) * ay, ax * ay};
    // d w_t / d u and d w_t / d v
    const float wu[4] = {-(1.f - ay), (1.f - ay), -ay, ay};
    const float wv[4] = {-(1.f - ax), -ax, (1.f - ax), ax};
    float gu = 0.f, gv = 0.f;
    const float *dout = a.dout + p * a.dout_cs;
    for (int c = 0; c < a.c; ++c) {
        const float g = dout[c];
        if (g == 0.f) continue;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if (!ok[t]) continue;
            if (a.df) atomicAdd(a.df + idx[t] * a.df_cs + c, wt[t] * g);
            if (a.dflow) {
                const float fv_ = to_f(a.f[idx[t] * a.f_cs + c]);
                gu = fmaf(wu[t] * g, fv_, gu);
                gv = fmaf(wv[t] * g, fv_, gv);
            }
        }
    }
    if (a.dflow) {
        float2 *d = reinterpret_cast<float2 *>(a.dflow) + p;
        if (a.accumulate) {
            d->x += gu;
            d->y += gv;
        } else {
            *d = make_float2(gu, gv);
        }
    }
}

template <typename T>
cudaError_t warp_bwd(const WarpBwdArgs<T> &a, cudaStream_t st) {
    const size_t total = (size_t)a.n * a.h * a.w;
    if (total == 0) return cudaSuccess;
    warp_bwd_kernel<T><<<blocks_for(total), 256, 0, st>>>(a);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------- upsampling x s

// Backward of the bilinear flow upsampling by s (values times s, half-pixel centres, sample
// position clamped at 0 and at the last row/column): each fine pixel scatters s times its
// gradient to the four coarse taps it read (float atomics into dcoarse [n][h][w][2]).
__global__ void up_bwd_kernel(const float *dfine, int n, int h, int w, int s, float *dcoarse) {
    const int H = h * s, W = w * s;
    const size_t total = (size_t)n * H * W;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int b = (int)(i / ((size_t)H * W));
    const int rem = (int)(i - (size_t)b * H * W);
    const int Y = rem / W, X = rem - Y * W;
    const float fs = (float)s;
    float sy = (Y + 0.5f) / fs - 0.5f, sx = (X + 0.5f) / fs - 0.5f;
    sy = fmaxf(sy, 0.f);
    sx = fmaxf(sx, 0.f);
    const int y0 = min((int)sy, h - 1), x0 = min((int)sx, w - 1);
    const int y1 = y0 < h - 1 ? y0 + 1 : y0, x1 = x0 < w - 1 ? x0 + 1 : x0;
    const float ly = sy - y0, lx = sx - x0;
    const float2 g = reinterpret_cast<const float2 *>(dfine)[i];
    const float gx = fs * g.x, gy = fs * g.y;
    float *base = dcoarse + (size_t)b * h * w * 2;
    const float wts[4] = {(1.f - ly) * (1.f - lx), (1.f - ly) * lx, ly * (1.f - lx), ly * lx};
    const int ys[4] = {y0, y0, y1, y1}, xs[4] = {x0, x1, x0, x1};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        float *d = base + ((size_t)ys[t] * w + xs[t]) * 2;
        atomicAdd(d, wts[t] * gx);
        atomicAdd(d + 1, wts[t] * gy);
    }
}

cudaError_t up_bwd(const float *dfine, int n, int h, int w, int s, float *dcoarse, cudaStream_t st) {
    const size_t total = (size_t)n * h * s * w * s;
    if (total == 0) return cudaSuccess;
    up_bwd_kernel<<<blocks_for(total), 256, 0, st>>>(dfine, n, h, w, s, dcoarse);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- window add / copy

// dst[p][k] (+)= src[p][k] for k < nc over npix pixels (channel windows at the pointers).
__global__ void window_add_kernel(const float *src, int src_cs, size_t npix, int nc, float *dst, int dst_cs,
                                  int accumulate) {
    const size_t total = npix * nc;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const size_t p = i / nc;
    const int k = (int)(i - p * nc);
    float *d = dst + p * dst_cs + k;
    const float v = src[p * src_cs + k];
    *d = accumulate ? *d + v : v;
}

cudaError_t window_add(const float *src, int src_cs, size_t npix, int nc, float *dst, int dst_cs, bool accumulate,
                       cudaStream_t st) {
    const size_t total = npix * nc;
    if (total == 0) return cudaSuccess;
    window_add_kernel<<<blocks_for(total), 256, 0, st>>>(src, src_cs, npix, nc, dst, dst_cs, accumulate ? 1 : 0);
    return cudaGetLastError();
}

// Copies a float flow window [npix][2] into an activation window (the up-flow channels).
template <typename T>
__global__ void flow_to_act_kernel(const float *flow, size_t npix, T *act, int act_cs) {
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    const float2 f = reinterpret_cast<const float2 *>(flow)[p];
    act[p * act_cs] = from_f<T>(f.x);
    act[p * act_cs + 1] = from_f<T>(f.y);
}

template <typename T>
cudaError_t flow_to_act(const float *flow, size_t npix, T *act, int act_cs, cudaStream_t st) {
    if (npix == 0) return cudaSuccess;
    flow_to_act_kernel<T><<<blocks_for(npix), 256, 0, st>>>(flow, npix, act, act_cs);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------- the loss

// Ground-truth flow of level l: the mean of the 2^l x 2^l block of the full-resolution flow
// (planar [n][2][H][W]) divided by 2^l (flows are in pixels of their level), NHWC output.
__global__ void gt_level_kernel(const float *gt, int n, int H, int W, int l, float *out) {
    const int s = 1 << l, h = H >> l, w = W >> l;
    const size_t total = (size_t)n * h * w;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int b = (int)(i / ((size_t)h * w));
    const int r = (int)(i - (size_t)b * h * w);
    const int y = r / w, x = r - y * w;
    const size_t HW = (size_t)H * W;
    const float *gu = gt + (size_t)b * 2 * HW, *gv = gu + HW;
    float su = 0.f, sv = 0.f;
    for (int dy = 0; dy < s; ++dy)
        for (int dx = 0; dx < s; ++dx) {
            const size_t q = (size_t)(y * s + dy) * W + x * s + dx;
            su += gu[q];
            sv += gv[q];
        }
    const float k = 1.f / ((float)s * s * s);
    reinterpret_cast<float2 *>(out)[i] = make_float2(su * k, sv * k);
}

cudaError_t gt_level(const float *gt, int n, int H, int W, int l, float *out, cudaStream_t st) {
    const size_t total = (size_t)n * (H >> l) * (W >> l);
    gt_level_kernel<<<blocks_for(total), 256, 0, st>>>(gt, n, H, W, l, out);
    return cudaGetLastError();
}

// Mean end-point error of one level (Eq. 10) and its gradient:
//   loss += (1/N) sum_p |f(p) - g(p)|,   dflow[p] (+)= (1/N) (f - g) / |f - g|  (0 where equal)
// with N = npix.  The loss is accumulated in double on the device.
__global__ void __launch_bounds__(256) epe_kernel(const float *flow, const float *gt, size_t npix, double *loss,
                                                  float *dflow, int accumulate) {
    __shared__ double part[8];
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0;
    if (i < npix) {
        const float2 f = reinterpret_cast<const float2 *>(flow)[i];
        const float2 g = reinterpret_cast<const float2 *>(gt)[i];
        const float du = f.x - g.x, dv = f.y - g.y;
        const float nrm = sqrtf(du * du + dv * dv);
        e = nrm;
        if (dflow) {
            const float k = nrm > 0.f ? 1.f / (nrm * (float)npix) : 0.f;
            float2 *d = reinterpret_cast<float2 *>(dflow) + i;
            if (accumulate) {
                d->x += du * k;
                d->y += dv * k;
            } else {
                *d = make_float2(du * k, dv * k);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += part[k];
        atomicAdd(loss, t / (double)npix);
    }
}

cudaError_t epe(const float *flow, const float *gt, size_t npix, double *loss, float *dflow, bool accumulate,
                cudaStream_t st) {
    if (npix == 0) return cudaSuccess;
    epe_kernel<<<blocks_for(npix), 256, 0, st>>>(flow, gt, npix, loss, dflow, accumulate ? 1 : 0);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ AdamW

// Decoupled weight decay (AdamW): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
// p -= lr (m / (1 - b1^t) / (sqrt(v / (1 - b2^t)) + eps) + wd p).  Biases (mask 0) take no
// decay.
__global__ void adamw_kernel(float *p, const float *g, float *m, float *v, const uint8_t *decay, size_t n,
                             AdamW h, float bc1, float bc2) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = h.beta1 * m[i] + (1.f - h.beta1) * gi;
    const float vi = h.beta2 * v[i] + (1.f - h.beta2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float upd = (mi / bc1) / (sqrtf(vi / bc2) + h.eps) + (decay[i] ? h.weight_decay * p[i] : 0.f);
    p[i] -= h.lr * upd;
}

cudaError_t adamw(float *p, const float *g, float *m, float *v, const uint8_t *decay, size_t n, const AdamW &h,
                  long long step, cudaStream_t st) {
    const float bc1 = 1.f - powf(h.beta1, (float)step), bc2 = 1.f - powf(h.beta2, (float)step);
    adamw_kernel<<<blocks_for(n), 256, 0, st>>>(p, g, m, v, decay, n, h, bc1, bc2);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ brute-force flow

// Integer-displacement flow: for each pixel of a the displacement d in [-r, r]^2 minimising
// the sum over a 3x3 patch and all channels of (a(x+p) - b(x+p+d))^2, border-clamped; ties
// go to the smaller |d|^2, then to the smaller index k = (dy+r)(2r+1) + (dx+r).  Planar
// float images (c, h, w); writes k per pixel.  One thread per pixel.
__global__ void bruteforce_kernel(const float *a, const float *b, int c, int h, int w, int r, int *kout) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)h * w) return;
    const int y = (int)(i / w), x = (int)(i - (size_t)y * w);
    const int n1 = 2 * r + 1;
    const size_t hw = (size_t)h * w;
    float best = INFINITY;
    int bestk = 0, bestn = 1 << 30;
    for (int k = 0; k < n1 * n1; ++k) {
        const int dy = k / n1 - r, dx = k % n1 - r;
        float s = 0.f;
        for (int py = -1; py <= 1; ++py)
            for (int px = -1; px <= 1; ++px) {
                const int ay = min(max(y + py, 0), h - 1), ax = min(max(x + px, 0), w - 1);
                const int by = min(max(y + py + dy, 0), h - 1), bx = min(max(x + px + dx, 0), w - 1);
                for (int ch = 0; ch < c; ++ch) {
                    const float e = a[ch * hw + (size_t)ay * w + ax] - b[ch * hw + (size_t)by * w + bx];
                    s = fmaf(e, e, s);
                }
            }
        const int nn = dx * dx + dy * dy;
        if (s < best || (s == best && nn < bestn)) {
            best = s;
            bestk = k;
            bestn = nn;
        }
    }
    kout[i] = bestk;
}

cudaError_t bruteforce(const float *a, const float *b, int c, int h, int w, int r, int *kout, cudaStream_t st) {
    bruteforce_kernel<<<blocks_for((size_t)h * w), 256, 0, st>>>(a, b, c, h, w, r, kout);
    return cudaGetLastError();
}

#define TC_TRAIN_INST(T)                                                                                         \
    template cudaError_t lrelu_bwd<T>(const float *, int, const T *, int, bool, size_t, int, float *, float *, int, \
                                      int, int, int, cudaStream_t);                                                \
    template cudaError_t wgrad<T>(const WgradArgs<T> &, float *, cudaStream_t);                                    \
    template cudaError_t corr_bwd<T>(const CorrBwdArgs<T> &, cudaStream_t);                                        \
    template cudaError_t warp_bwd<T>(const WarpBwdArgs<T> &, cudaStream_t);                                        \
    template cudaError_t flow_to_act<T>(const float *, size_t, T *, int, cudaStream_t);                          \
    template cudaError_t pack_images<T>(const float *, const float *, int, int, int, T *, cudaStream_t);          \
    template cudaError_t lrelu_bwd2<T>(const float *, int, const T *, int, bool, size_t, int, float *, void *,   \
                                       void *, int, int, int, int, cudaStream_t);                                \
    template cudaError_t x_to_cp<T>(const T *, int, int, int, int, int, int, int, void *const[3], cudaStream_t);
TC_TRAIN_INST(float)
TC_TRAIN_INST(__nv_bfloat16)
#undef TC_TRAIN_INST

}  // namespace train
}  // namespace tc
