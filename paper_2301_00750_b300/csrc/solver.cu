// Screened-Poisson solver of Sec. 3.1 (Eq. 1) by SGD with momentum (Eq. 8):
//   O^{j+1} = O^j - eta (Lg (O^j - P) + wc (O^j - A)) + kappa (O^j - O^{j-1}),
// from O^0 = O^{-1} = A; Lg is the 4-neighbour graph Laplacian with Neumann boundary.
// With b = Lg P + wc A (computed once) the gradient is Lg O + wc O - b.
//
// The iterations are blocked in time: a CTA loads a 32 x 32 tile of O^j, O^{j-1}, b and wc
// with a halo of T pixels into shared memory, runs T iterations there (the valid region
// shrinks by one pixel per iteration, so the tile stays exact), and writes the tile's
// O^{j+T}, O^{j+T-1}.  One pass moves T iterations for (1 + 2T/32)^2 of the tile's
// traffic; the working set (three 1080p images and the weights) also fits the 126 MB L2.
#include "solver.cuh"

namespace tc {

namespace {

constexpr int TS = 32;                    // output tile
constexpr int TMAX = 8;                   // iterations per pass
constexpr int RS = TS + 2 * TMAX;         // region side (48)
constexpr int RP = RS * RS;               // region pixels

// b = Lg P + wc A per channel (planar (c, h, w)).
__global__ void poisson_rhs_kernel(const float *P, const float *A, const float *wc, int c, int h, int w, float *b) {
    const size_t hw = (size_t)h * w;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)c * hw) return;
    const size_t ch = i / hw, p = i - ch * hw;
    const int y = (int)(p / w), x = (int)(p - (size_t)y * w);
    const float *Pc = P + ch * hw;
    const float v = Pc[p];
    float lap = 0.f;
    if (y > 0) lap += v - Pc[p - w];
    if (y < h - 1) lap += v - Pc[p + w];
    if (x > 0) lap += v - Pc[p - 1];
    if (x < w - 1) lap += v - Pc[p + 1];
    b[i] = lap + wc[p] * A[i];
}

// T (<= TMAX) iterations on one tile; cur / prev in, cur_out / prev_out written for the
// tile (cur_out2, if set, receives a second copy of the final iterate).
template <int C>
__global__ void __launch_bounds__(256) poisson_block_kernel(const float *cur, const float *prev, const float *b,
                                                            const float *wc, int h, int w, int T, float eta,
                                                            float kappa, float *cur_out, float *prev_out,
                                                            float *cur_out2) {
    extern __shared__ float sm[];
    float *sc = sm;               // [C][RP] current iterate
    float *sp = sc + C * RP;      // [C][RP] previous iterate (overwritten by the next)
    float *sb = sp + C * RP;      // [C][RP] right-hand side
    float *sw = sb + C * RP;      // [RP] weights
    const size_t hw = (size_t)h * w;
    const int ty0 = blockIdx.y * TS - T, tx0 = blockIdx.x * TS - T;  // region origin
    const int rs = TS + 2 * T;
    for (int k = threadIdx.x; k < rs * rs; k += blockDim.x) {
        const int r = k / rs, q = k - r * rs;
        const int gy = ty0 + r, gx = tx0 + q;
        const bool in = gy >= 0 && gy < h && gx >= 0 && gx < w;
        const size_t g = in ? (size_t)gy * w + gx : 0;
#pragma unroll
        for (int ch = 0; ch < C; ++ch) {
            sc[ch * RP + k] = in ? cur[ch * hw + g] : 0.f;
            sp[ch * RP + k] = in ? prev[ch * hw + g] : 0.f;
            sb[ch * RP + k] = in ? b[ch * hw + g] : 0.f;
        }
        sw[k] = in ? wc[g] : 0.f;
    }
    __syncthreads();
    float *pc = sc, *pp = sp;
    for (int it = 0; it < T; ++it) {
        // pixels of the region's inner (rs - 2) ring can read all four neighbours; those
        // nearer the edge of the region are outside the valid tile by the end anyway
        for (int k = threadIdx.x; k < rs * rs; k += blockDim.x) {
            const int r = k / rs, q = k - r * rs;
            const int gy = ty0 + r, gx = tx0 + q;
            if (r == 0 || q == 0 || r == rs - 1 || q == rs - 1) continue;
            if (gy < 0 || gy >= h || gx < 0 || gx >= w) continue;
            const bool up = gy > 0, dn = gy < h - 1, lf = gx > 0, rt = gx < w - 1;
            const float deg = (float)(up + dn + lf + rt);
            const float wk = sw[k];
#pragma unroll
            for (int ch = 0; ch < C; ++ch) {
                const float *xc = pc + ch * RP;
                const float x = xc[k];
                float nb = 0.f;
                if (up) nb += xc[k - rs];
                if (dn) nb += xc[k + rs];
                if (lf) nb += xc[k - 1];
                if (rt) nb += xc[k + 1];
                const float grad = (deg * x - nb) + wk * x - sb[ch * RP + k];
                const float xp = pp[ch * RP + k];
                pp[ch * RP + k] = x - eta * grad + kappa * (x - xp);  // the next iterate
            }
        }
        __syncthreads();
        float *t = pc;
        pc = pp;
        pp = t;
    }
    for (int k = threadIdx.x; k < TS * TS; k += blockDim.x) {
        const int r = T + k / TS, q = T + k % TS;
        const int gy = ty0 + r, gx = tx0 + q;
        if (gy >= h || gx >= w) continue;
        const int s = r * rs + q;
        const size_t g = (size_t)gy * w + gx;
#pragma unroll
        for (int ch = 0; ch < C; ++ch) {
            cur_out[ch * hw + g] = pc[ch * RP + s];
            prev_out[ch * hw + g] = pp[ch * RP + s];
            if (cur_out2) cur_out2[ch * hw + g] = pc[ch * RP + s];
        }
    }
}

__global__ void copy_out_kernel(const float *src, float *dst, size_t n, const float *wsrc, float *wdst, size_t nw) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i];
    if (wdst)
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += stride) wdst[i] = wsrc[i];
}

}  // namespace

cudaError_t launch_copy_out(const float *src, float *dst, size_t n, const float *wsrc, float *wdst, size_t nw,
                            cudaStream_t st) {
    copy_out_kernel<<<4 * 148, 256, 0, st>>>(src, dst, n, wsrc, wdst, nw);
    return cudaGetLastError();
}

const void *copy_out_kernel_fn() { return reinterpret_cast<const void *>(copy_out_kernel); }

size_t poisson_smem_bytes(int c) { return ((size_t)3 * c + 1) * RP * sizeof(float); }

cudaError_t launch_poisson(const PoissonArgs &a, cudaStream_t st) {
    if (a.c != 3 && a.c != 1) return cudaErrorInvalidValue;
    const size_t n = (size_t)a.c * a.h * a.w;
    poisson_rhs_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a.P, a.A, a.wc, a.c, a.h, a.w, a.b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || a.iters <= 0) return e;
    const size_t smem = poisson_smem_bytes(a.c);
    static bool attr3 = false, attr1 = false;
    if (a.c == 3 && !attr3) {
        if ((e = cudaFuncSetAttribute(poisson_block_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;
        attr3 = true;
    }
    if (a.c == 1 && !attr1) {
        if ((e = cudaFuncSetAttribute(poisson_block_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;
        attr1 = true;
    }
    dim3 grid((a.w + TS - 1) / TS, (a.h + TS - 1) / TS);
    // ping-pong through (bufA, bufB) pairs: pass k reads (cur, prev) and writes the other pair
    const float *cur = a.A, *prev = a.A;
    float *pair[2][2] = {{a.s0, a.s1}, {a.s2, a.s3}};
    int done = 0, k = 0;
    while (done < a.iters) {
        const int T = a.iters - done < TMAX ? a.iters - done : TMAX;
        const bool last = done + T == a.iters;
        float *co = last ? a.O : pair[k & 1][0];
        float *po = pair[k & 1][1];
        if (a.c == 3)
            poisson_block_kernel<3><<<grid, 256, smem, st>>>(cur, prev, a.b, a.wc, a.h, a.w, T, a.eta, a.kappa, co, po,
                                                             last ? a.O2 : nullptr);
        else
            poisson_block_kernel<1><<<grid, 256, smem, st>>>(cur, prev, a.b, a.wc, a.h, a.w, T, a.eta, a.kappa, co, po,
                                                             last ? a.O2 : nullptr);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        cur = co;
        prev = po;
        done += T;
        k += 1;
    }
    return cudaSuccess;
}

}  // namespace tc
