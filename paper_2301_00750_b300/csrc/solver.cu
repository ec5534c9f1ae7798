// Screened-Poisson solver of Sec. 3.1 (Eq. 1) by SGD with momentum (Eq. 8):
//   O^{j+1} = O^j - eta (Lg (O^j - P) + wc (O^j - A)) + kappa (O^j - O^{j-1}),
// from O^0 = O^{-1} = A; Lg is the 4-neighbour graph Laplacian with Neumann boundary.
// With b = Lg P + wc A (computed once) the gradient is Lg O + wc O - b, and one step is
//   O^{j+1} = c0 O^j + eta (sum of the in-frame neighbours of O^j) + eta b - kappa O^{j-1},
//   c0 = 1 + kappa - eta (deg + wc),  deg = number of in-frame neighbours.
//
// The iterations are blocked in time and held in registers.  A CTA owns one channel of a
// region of RW x RH pixels (RW = 32 CW: a warp spans the region's width, CW columns per
// lane; the NW warps stack R rows each).  Every thread keeps O^j, O^{j-1}, c0 and eta b of
// its R x CW pixels in registers for T <= HALO iterations; left/right neighbours come from
// the adjacent lane by shuffle (or the thread's own registers), up/down neighbours from its
// own registers except at the warp's first and last row, which the warps exchange through
// shared memory once per iteration.  Cells of the region outside the frame stay 0, so the
// neighbour sum of an in-frame pixel is over its in-frame neighbours.  Cells on the region's
// outer ring read values from outside the region that are wrong, and the error moves in by
// one pixel per iteration, so after T <= HALO iterations the pixels at least HALO from the
// region's edge are exact: those form the output tile of (RW - 2 HALO) x (RH - 2 HALO).
// Passes of T iterations ping-pong (O^j, O^{j-1}) through global memory (L2-resident at
// 1080p).
#include "solver.cuh"

#include <stdint.h>

namespace tc {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// The pass-invariant coefficients, once per solve: eb = eta b, b = Lg P + wc A, per channel
// (planar (c, h, w)), and c0 = 1 + kappa - eta (deg + wc) per pixel ((h, w)).
__global__ void poisson_rhs_kernel(const float *P, const float *A, const float *wc, int c, int h, int w, float eta,
                                   float kappa, float *eb, float *c0) {
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
    const float b = lap + wc[p] * A[i];
    eb[i] = eta * b;
    if (ch == 0) {
        const int deg = (y > 0) + (y < h - 1) + (x > 0) + (x < w - 1);
        c0[p] = 1.f + kappa - eta * ((float)deg + wc[p]);
    }
}

// Region of a CTA: RW x RH pixels; HALO = iterations per pass = the margin around the output
// tile of OW x OH pixels.
template <int CW, int R, int NW, int HALO>
struct Geo {
    static constexpr int RW = 32 * CW, RH = NW * R;
    static constexpr int OW = RW - 2 * HALO, OH = RH - 2 * HALO;
    static constexpr int XCH = 2 * 2 * NW * RW;  // exchange rows: [parity][top, bottom][warp][RW]
};

// CW consecutive floats at p (aligned to CW floats) into v, and back.
template <int CW>
__device__ __forceinline__ void ld_row(const float *__restrict__ p, float (&v)[CW]) {
    if constexpr (CW == 2) {
        const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
        v[0] = t.x;
        v[1] = t.y;
    } else {
#pragma unroll
        for (int j = 0; j < CW; ++j) v[j] = __ldg(p + j);
    }
}

template <int CW>
__device__ __forceinline__ void st_row(float *p, const float (&v)[CW]) {
    if constexpr (CW == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    } else {
#pragma unroll
        for (int j = 0; j < CW; ++j) p[j] = v[j];
    }
}

// One iteration: the next iterate (in place of the previous one, pv) from the current cu.
template <int CW, int R, int NW, bool EDGE>
__device__ __forceinline__ void step(const float (&cu)[R][CW], float (&pv)[R][CW], const float (&c0)[R][CW],
                                     const float (&eb)[R][CW], unsigned mask, float eta, float kappa, float *buf,
                                     int lane, int wp) {
    constexpr int RW = 32 * CW;
    float *top = buf, *bot = buf + NW * RW;
#pragma unroll
    for (int j = 0; j < CW; ++j) {
        top[wp * RW + lane * CW + j] = cu[0][j];
        bot[wp * RW + lane * CW + j] = cu[R - 1][j];
    }
    __syncthreads();
    float upr[CW], dnr[CW];
#pragma unroll
    for (int j = 0; j < CW; ++j) {
        upr[j] = wp > 0 ? bot[(wp - 1) * RW + lane * CW + j] : 0.f;
        dnr[j] = wp < NW - 1 ? top[(wp + 1) * RW + lane * CW + j] : 0.f;
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const float lin = __shfl_up_sync(FULL, cu[i][CW - 1], 1);
        const float rin = __shfl_down_sync(FULL, cu[i][0], 1);
#pragma unroll
        for (int j = 0; j < CW; ++j) {
            const float up = i > 0 ? cu[i - 1][j] : upr[j];
            const float dn = i < R - 1 ? cu[i + 1][j] : dnr[j];
            const float lf = j > 0 ? cu[i][j - 1] : lin;
            const float rt = j < CW - 1 ? cu[i][j + 1] : rin;
            float v = fmaf(c0[i][j], cu[i][j], fmaf(eta, (up + dn) + (lf + rt), fmaf(-kappa, pv[i][j], eb[i][j])));
            if (EDGE && !((mask >> (i * CW + j)) & 1u)) v = 0.f;
            pv[i][j] = v;
        }
    }
}

struct SolveArgs {
    const float *cur, *prev, *eb, *c0;  // eb = eta b per channel, c0 per pixel
    int h, w, T, tiles_x;
    float eta, kappa;
    float *cur_out, *prev_out, *cur_out2;
    int vec_ok;  // width and every buffer aligned to CW floats
};

template <int CW, int R, int NW, int HALO, bool EDGE>
__device__ __forceinline__ void region(const SolveArgs &s, size_t off, int oy, int ox, float *xch) {
    using G = Geo<CW, R, NW, HALO>;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int cx = ox + lane * CW, ry = oy + wp * R;
    const float *cur = s.cur + off, *prev = s.prev + off, *ebp = s.eb + off;
    float x[R][CW], p[R][CW], c0[R][CW], eb[R][CW];
    unsigned mask = 0;
    // Interior regions load and store rows of CW floats when the host found the frame width
    // and every buffer CW-aligned (HALO and OW are multiples of CW, so then is every row of
    // a thread).
    const bool vec = !EDGE && HALO % CW == 0 && s.vec_ok;
    if (vec) {
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const size_t g = (size_t)(ry + i) * s.w + cx;
            ld_row<CW>(cur + g, x[i]);
            ld_row<CW>(prev + g, p[i]);
            ld_row<CW>(ebp + g, eb[i]);
            ld_row<CW>(s.c0 + g, c0[i]);
        }
    } else {
#pragma unroll
        for (int i = 0; i < R; ++i) {
#pragma unroll
            for (int j = 0; j < CW; ++j) {
                const int gy = ry + i, gx = cx + j;
                const bool in = !EDGE || (gy >= 0 && gy < s.h && gx >= 0 && gx < s.w);
                x[i][j] = p[i][j] = c0[i][j] = eb[i][j] = 0.f;
                if (in) {
                    const size_t g = (size_t)gy * s.w + gx;
                    x[i][j] = __ldg(cur + g);
                    p[i][j] = __ldg(prev + g);
                    eb[i][j] = __ldg(ebp + g);
                    c0[i][j] = __ldg(s.c0 + g);
                    mask |= 1u << (i * CW + j);
                }
            }
        }
    }
    int t = 0;
    for (; t + 1 < s.T; t += 2) {
        step<CW, R, NW, EDGE>(x, p, c0, eb, mask, s.eta, s.kappa, xch, lane, wp);
        step<CW, R, NW, EDGE>(p, x, c0, eb, mask, s.eta, s.kappa, xch + G::XCH / 2, lane, wp);
    }
    if (t < s.T) step<CW, R, NW, EDGE>(x, p, c0, eb, mask, s.eta, s.kappa, xch, lane, wp);
    const bool odd = s.T & 1;  // the last iterate is in p when T is odd
    float *co = s.cur_out + off, *po = s.prev_out + off, *c2 = s.cur_out2 ? s.cur_out2 + off : nullptr;
    if (vec) {
        // a thread's CW columns are all inside the output tile or all outside
        const int q = lane * CW;
        if (q < HALO || q >= G::RW - HALO) return;
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int r = wp * R + i;
            if (r < HALO || r >= G::RH - HALO) continue;
            const size_t g = (size_t)(ry + i) * s.w + cx;
            st_row<CW>(co + g, odd ? p[i] : x[i]);
            st_row<CW>(po + g, odd ? x[i] : p[i]);
            if (c2) st_row<CW>(c2 + g, odd ? p[i] : x[i]);
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int r = wp * R + i, gy = ry + i;
        if (r < HALO || r >= G::RH - HALO || gy >= s.h) continue;
#pragma unroll
        for (int j = 0; j < CW; ++j) {
            const int q = lane * CW + j, gx = cx + j;
            if (q < HALO || q >= G::RW - HALO || gx >= s.w) continue;
            const size_t g = (size_t)gy * s.w + gx;
            co[g] = odd ? p[i][j] : x[i][j];
            po[g] = odd ? x[i][j] : p[i][j];
            if (c2) c2[g] = odd ? p[i][j] : x[i][j];
        }
    }
}

// T (<= HALO) iterations on one region per CTA: blockIdx.x = tile, blockIdx.y = channel.
template <int CW, int R, int NW, int HALO, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) poisson_solve_kernel(const SolveArgs s) {
    using G = Geo<CW, R, NW, HALO>;
    static_assert(R * CW <= 32, "one mask bit per pixel of a thread");
    __shared__ float xch[G::XCH];
    const size_t off = (size_t)blockIdx.y * s.h * s.w;
    const int ty = blockIdx.x / s.tiles_x, tx = blockIdx.x - ty * s.tiles_x;
    const int oy = ty * G::OH - HALO, ox = tx * G::OW - HALO;
    if (oy >= 0 && ox >= 0 && oy + G::RH <= s.h && ox + G::RW <= s.w)
        region<CW, R, NW, HALO, false>(s, off, oy, ox, xch);
    else
        region<CW, R, NW, HALO, true>(s, off, oy, ox, xch);
}

// Region shape: 64 x 64 pixels (2 columns per lane, 8 warps of 8 rows), 8 iterations per
// pass, 48 x 48 output; two CTAs per SM.
constexpr int CW = 2, RR = 8, NWARP = 8, TPASS = 8, MINB = 2;

}  // namespace

cudaError_t launch_poisson(const PoissonArgs &a, cudaStream_t st) {
    if (a.c < 1 || a.c > 3) return cudaErrorInvalidValue;
    const size_t n = (size_t)a.c * a.h * a.w;
    poisson_rhs_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a.P, a.A, a.wc, a.c, a.h, a.w, a.eta, a.kappa,
                                                                   a.b, a.c0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || a.iters <= 0) return e;
    using G = Geo<CW, RR, NWARP, TPASS>;
    SolveArgs s{};
    s.eb = a.b;
    s.c0 = a.c0;
    s.h = a.h;
    s.w = a.w;
    s.tiles_x = (a.w + G::OW - 1) / G::OW;
    s.eta = a.eta;
    s.kappa = a.kappa;
    auto al = [](const void *q) { return reinterpret_cast<uintptr_t>(q) % (CW * sizeof(float)) == 0; };
    s.vec_ok = a.w % CW == 0 && al(a.A) && al(a.c0) && al(a.b) && al(a.s0) && al(a.s1) && al(a.s2) && al(a.s3) &&
               al(a.O) && (a.O2 == nullptr || al(a.O2));
    const dim3 grid(s.tiles_x * ((a.h + G::OH - 1) / G::OH), a.c);
    // ping-pong through (s0, s1), (s2, s3): pass k reads (cur, prev) and writes the other pair
    s.cur = a.A;
    s.prev = a.A;
    float *pair[2][2] = {{a.s0, a.s1}, {a.s2, a.s3}};
    int done = 0, k = 0;
    while (done < a.iters) {
        s.T = a.iters - done < TPASS ? a.iters - done : TPASS;
        const bool last = done + s.T == a.iters;
        s.cur_out = last ? a.O : pair[k & 1][0];
        s.prev_out = pair[k & 1][1];
        s.cur_out2 = last ? a.O2 : nullptr;
        poisson_solve_kernel<CW, RR, NWARP, TPASS, MINB><<<grid, NWARP * 32, 0, st>>>(s);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        s.cur = s.cur_out;
        s.prev = s.prev_out;
        done += s.T;
        k += 1;
    }
    return cudaSuccess;
}

}  // namespace tc
