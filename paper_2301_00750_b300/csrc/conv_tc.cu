// Implicit-GEMM 3x3 convolution on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// GEMM view: M = output pixels, N = cout, K = 9 taps x input channels, taken in K steps of
// one swizzle span: 64 bf16 (128 e4m3) channels with the 128-byte swizzle, or 32 / 16 bf16
// channels with the 64- / 32-byte swizzle for layers that have no more input channels than
// that (the 16- and 32-channel pyramid levels), so no step multiplies zero padding
// wider than the layer.  The descriptions below use the 128-byte case.  Stride-1 layers use
// conv_tc_halo_kernel (below), which loads each activation tile once per kernel row and
// reuses it for the three horizontal taps; the description here is of the per-tap kernel,
// which serves the stride-2 layers.  One CTA computes a
// tile of 128 consecutive output pixels of one row (M = 128) and all cout (N = BN, a
// multiple of 16 up to 128):
//   * warp 0, lane 0 (producer): for every (tap, 64-channel chunk) step, one TMA tiled load
//     of the shifted activation tile [128 px][64 ch] (zero padding and ragged edges come
//     from the TMA out-of-bounds fill; stride-2 convs address the input through a
//     (channel, parity, x/2, y, image) view) and one of the weight tile [BN][64 ch], both
//     with the 128-byte swizzle, into a ring of STAGES shared-memory slots;
//   * warp 1, lane 0 (MMA issuer): four tcgen05.mma (kind::f16, BF16 x BF16 -> FP32,
//     128 x BN x 16 each) per step into a TMEM accumulator; tcgen05.commit frees the slot;
//   * all four warps (epilogue): tcgen05.ld of their 32 accumulator rows, bias, LeakyReLU,
//     bfloat16 rounding, 16-byte stores into the NHWC output.
// Every mbarrier wait is bounded by a 2 s timer: on timeout the CTA records a code in the
// stream's device error word, stops issuing work, drains what it issued and frees its TMEM.
#include <cudaTypedefs.h>
#include <cuda_fp8.h>

#include <atomic>
#include <cstring>
#include <mutex>

#include "../../include/tc_stream.h"
#include "conv_tc.cuh"
#include "tc_ptx.cuh"

namespace tc {

namespace {

using namespace ptx;

constexpr int BM = 128;                    // output pixels per CTA (MMA M)
constexpr int BK = 64;                     // bf16 channels of the widest K step (128 B); e4m3 steps hold 128

enum : int { ERR_PRODUCER = 1, ERR_MMA = 2, ERR_EPILOGUE = 3, ERR_DRAIN = 4 };

__host__ __device__ constexpr int stages_for(int bn) { return bn >= 96 ? 3 : 4; }
__host__ __device__ constexpr int tmem_cols_for(int bn) { return bn <= 32 ? 32 : (bn <= 64 ? 64 : 128); }
// Ring slots of the per-tap kernel hold one K step of rb bytes per row (A: BM rows, B: bn
// rows), each rounded up to the 1024-byte swizzle atom.
__host__ __device__ constexpr uint32_t a_slot_for(int rb) { return (uint32_t)((BM * rb + 1023) / 1024 * 1024); }
__host__ __device__ constexpr uint32_t b_slot_for(int bn, int rb) { return (uint32_t)((bn * rb + 1023) / 1024 * 1024); }
__host__ __device__ constexpr size_t smem_bytes_for(int bn, int rb) {
    return (size_t)stages_for(bn) * (a_slot_for(rb) + b_slot_for(bn, rb)) + 1024 + 256;
}

struct TcLaunch {
    int nch;      // K steps of the input channels (kc channels, rb bytes each)
    int kc, rb;   // channels per step; bytes per step (32, 64 or 128: the TMA/MMA swizzle span)
    int stride;   // 1 or 2
    int ho, wo;
    int img_off;  // first input image in the A descriptor
    void *out;        // bf16 or e4m3 NHWC output (channel offset applied)
    int out_cs;
    const float *bias;
    int leaky;
    int *err;
    float *flow;      // flow-head mode: (n, ho, wo, 2) float output
    const float *up;  // flow-head mode: residual base flow, same layout, or NULL
    const float *wscale;  // e4m3: per-output-channel weight scale (activation scales folded in)
    float q_out;          // e4m3: 1 / output activation scale
    int out_f32;          // bf16 operands only: write float32 (out_cs in floats) instead of bf16
    int accumulate;       // with out_f32: add to the output instead of overwriting it
    int taps;             // 9: 3x3 conv; 1: pointwise 1x1 conv (the centre tap only)
    int tail;             // halo kernel: the last channel step is a 64-byte tail
    int f16;              // 16-bit operands and outputs are IEEE half instead of bfloat16
    int stall;            // halo kernel, test hook: the producer issues no loads (see tc_test_stall_next_convs)
};

// Epilogue shared by the conv kernels: thread r of the CTA owns accumulator row r, i.e.
// output pixel (img, y, x0 + r).
template <int BN, bool HEAD, bool F8>
__device__ __forceinline__ void conv_epilogue(uint32_t tmem, const TcLaunch &p, int warp, int lane, int x0, int y,
                                              int img) {
    if (HEAD) {
        const int x = x0 + warp * 32 + lane;
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16), r);
        if (x < p.wo) {
            const size_t pix = (size_t)(img * p.ho + y) * p.wo + x;
            float2 up = make_float2(0.f, 0.f);
            if (p.up) up = reinterpret_cast<const float2 *>(p.up)[pix];
            const float s0 = F8 ? __ldg(p.wscale) : 1.f, s1 = F8 ? __ldg(p.wscale + 1) : 1.f;
            reinterpret_cast<float2 *>(p.flow)[pix] =
                make_float2(up.x + (__uint_as_float(r[0]) * s0 + __ldg(p.bias)),
                            up.y + (__uint_as_float(r[1]) * s1 + __ldg(p.bias + 1)));
        }
    } else {
        const int row = warp * 32 + lane;
        const int x = x0 + row;
        const size_t pix = (size_t)(img * p.ho + y) * p.wo + x;
        const bool vec_params = ((reinterpret_cast<uintptr_t>(p.bias) |
                                  (F8 ? reinterpret_cast<uintptr_t>(p.wscale) : 0)) & 15) == 0;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t r[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
            if (x < p.wo) {
                // bias (and e4m3 weight scales) of the 16 columns: four 16-byte loads where
                // the arrays allow it, else 16 scalar ones
                float bv[16], sv[16];
                if (vec_params) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 b4 = __ldg(reinterpret_cast<const float4 *>(p.bias + c0) + q);
                        bv[4 * q] = b4.x; bv[4 * q + 1] = b4.y; bv[4 * q + 2] = b4.z; bv[4 * q + 3] = b4.w;
                        if (F8) {
                            const float4 s4 = __ldg(reinterpret_cast<const float4 *>(p.wscale + c0) + q);
                            sv[4 * q] = s4.x; sv[4 * q + 1] = s4.y; sv[4 * q + 2] = s4.z; sv[4 * q + 3] = s4.w;
                        }
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        bv[j] = __ldg(p.bias + c0 + j);
                        if (F8) sv[j] = __ldg(p.wscale + c0 + j);
                    }
                }
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float a = __uint_as_float(r[j]);
                    v[j] = (F8 ? a * sv[j] : a) + bv[j];
                    if (p.leaky) v[j] = v[j] >= 0.f ? v[j] : 0.1f * v[j];
                }
                if (!F8 && p.out_f32) {
                    float4 *dst = reinterpret_cast<float4 *>(static_cast<float *>(p.out) + pix * p.out_cs + c0);
#pragma unroll
                    for (int q4 = 0; q4 < 4; ++q4) {
                        float4 o = make_float4(v[4 * q4], v[4 * q4 + 1], v[4 * q4 + 2], v[4 * q4 + 3]);
                        if (p.accumulate) {
                            const float4 e = dst[q4];
                            o.x += e.x; o.y += e.y; o.z += e.z; o.w += e.w;
                        }
                        dst[q4] = o;
                    }
                } else if (F8) {
                    uint4 q;
                    q.x = pack_e4m3x4(v[0] * p.q_out, v[1] * p.q_out, v[2] * p.q_out, v[3] * p.q_out);
                    q.y = pack_e4m3x4(v[4] * p.q_out, v[5] * p.q_out, v[6] * p.q_out, v[7] * p.q_out);
                    q.z = pack_e4m3x4(v[8] * p.q_out, v[9] * p.q_out, v[10] * p.q_out, v[11] * p.q_out);
                    q.w = pack_e4m3x4(v[12] * p.q_out, v[13] * p.q_out, v[14] * p.q_out, v[15] * p.q_out);
                    *reinterpret_cast<uint4 *>(static_cast<uint8_t *>(p.out) + pix * p.out_cs + c0) = q;
                } else {
                    uint16_t *dst = static_cast<uint16_t *>(p.out) + pix * p.out_cs;  // bf16 or half
                    uint4 lo, hi;
                    lo.x = pack16x2(p.f16, v[0], v[1]);
                    lo.y = pack16x2(p.f16, v[2], v[3]);
                    lo.z = pack16x2(p.f16, v[4], v[5]);
                    lo.w = pack16x2(p.f16, v[6], v[7]);
                    hi.x = pack16x2(p.f16, v[8], v[9]);
                    hi.y = pack16x2(p.f16, v[10], v[11]);
                    hi.z = pack16x2(p.f16, v[12], v[13]);
                    hi.w = pack16x2(p.f16, v[14], v[15]);
                    *reinterpret_cast<uint4 *>(dst + c0) = lo;
                    *reinterpret_cast<uint4 *>(dst + c0 + 8) = hi;
                }
            }
        }
    }
}

// HEAD = true: the flow head (cout = 2, zero-padded to BN = 16 for the MMA); the epilogue
// writes float32 flow = up + (acc[0], acc[1]) + bias without activation.
template <int BN, bool HEAD, bool F8>
__global__ void __launch_bounds__(128, 1)
conv_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcLaunch p) {
    constexpr int STAGES = stages_for(BN);
    constexpr uint32_t TMEM_COLS = tmem_cols_for(BN);
    const uint32_t A_BYTES = a_slot_for(p.rb), B_BYTES = b_slot_for(BN, p.rb);
    const uint32_t stage_tx = (uint32_t)(BM + BN) * (uint32_t)p.rb;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;
    uint8_t *sB = smem + STAGES * A_BYTES;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + STAGES * (A_BYTES + B_BYTES));
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 1);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES), accum = smem_u32(bars + 2 * STAGES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x0 = blockIdx.x * BM, y = blockIdx.y, img = blockIdx.z;
    const int nk = p.taps * p.nch;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(accum, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    pdl_wait();  // every global access below follows the previous kernel

    if (threadIdx.x == 0) {
        // ---- producer
        int issued = 0;
        for (int ks = 0; ks < nk; ++ks) {
            const int s = ks % STAGES;
            const uint32_t ph = (uint32_t)(ks / STAGES) & 1u;
            if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, p.err, ERR_PRODUCER)) break;
            const int tap = ks / p.nch, ch = ks - tap * p.nch;
            const int ky = p.taps == 9 ? tap / 3 : 1, kx = p.taps == 9 ? tap - (tap / 3) * 3 : 1;
            const uint32_t fb = full0 + 8 * s;
            mbar_expect_tx(fb, stage_tx);
            const uint32_t dA = smem_u32(sA + s * A_BYTES), dB = smem_u32(sB + s * B_BYTES);
            if (p.stride == 1) {
                tma_load_4d(&tmA, fb, dA, ch * p.kc, x0 + kx - 1, y + ky - 1, img + p.img_off);
            } else {
                const int dx = kx - 1;
                tma_load_5d(&tmA, fb, dA, ch * p.kc, dx != 0 ? 1 : 0, x0 + (dx < 0 ? -1 : 0), 2 * y + ky - 1,
                            img + p.img_off);
            }
            tma_load_3d(&tmB, fb, dB, ch * p.kc, 0, tap);
            issued = ks + 1;
        }
        if (issued < nk) {
            // Error path: let the loads already issued land before the CTA exits.
            for (int ks = issued - STAGES < 0 ? 0 : issued - STAGES; ks < issued; ++ks) {
                unsigned long long t0 = global_ns();
                while (!mbar_try(full0 + 8 * (ks % STAGES), (uint32_t)(ks / STAGES) & 1u))
                    if (global_ns() - t0 > WAIT_NS) {
                        atomicCAS(p.err, 0, ERR_DRAIN);
                        break;
                    }
            }
        }
    } else if (threadIdx.x == 32) {
        // ---- MMA issuer
        const uint32_t idesc = F8 ? idesc_e4m3(BM, BN) : (p.f16 ? idesc_f16(BM, BN) : idesc_bf16(BM, BN));
        for (int ks = 0; ks < nk; ++ks) {
            const int s = ks % STAGES;
            if (!mbar_wait(full0 + 8 * s, (uint32_t)(ks / STAGES) & 1u, p.err, ERR_MMA)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t da = sw_desc(smem_u32(sA + s * A_BYTES), (uint32_t)p.rb);
            const uint64_t db = sw_desc(smem_u32(sB + s * B_BYTES), (uint32_t)p.rb);
            for (int kk = 0; kk < p.rb / 32; ++kk)
                umma<F8>(tmem, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc, (ks | kk) != 0 ? 1u : 0u);
            umma_commit(empty0 + 8 * s);
        }
        umma_commit(accum);  // arrives when every MMA issued above has completed
    }

    // ---- epilogue (all 128 threads; thread r owns accumulator row r = pixel x0 + r)
    // Lane 0 of each warp polls the accumulator barrier (lane 0 of warps 0 and 1 arrive here
    // after their producer / MMA loops); the other lanes block in the shuffle meanwhile.
    int ok = 1;
    if (lane == 0) ok = mbar_wait(accum, 0, p.err, ERR_EPILOGUE) && *(volatile int *)p.err == 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) conv_epilogue<BN, HEAD, F8>(tmem, p, warp, lane, x0, y, img);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// Stride-1 variant that fetches each activation tile once per (kernel row ky, channel
// step): a TMA load of the 130-pixel halo row [x0 - 1, x0 + 129) x 64 channels, reused by
// the three horizontal taps through descriptors whose start is shifted by kx rows of the
// 128-byte-swizzled tile.  Activation halos and weight tiles travel in two separate rings
// (2 halo slots, SB weight slots), so a halo stays resident while its three taps run.
constexpr uint32_t HALO_ROWS = BM + 2;
constexpr uint32_t HALO_SLOT = 17408;             // rounded up to the 1024-byte swizzle atom
constexpr int HALO_SA = 2;
__host__ __device__ constexpr int halo_sb(int bn) { return bn >= 96 ? 3 : 4; }
__host__ __device__ constexpr size_t halo_smem_for(int bn) {
    return (size_t)HALO_SA * HALO_SLOT + (size_t)halo_sb(bn) * bn * BK * 2 + 1024 + 256;
}

template <int BN, bool HEAD, bool F8>
__global__ void __launch_bounds__(128, 1)
conv_tc_halo_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmB2, const TcLaunch p) {
    constexpr int SB = halo_sb(BN);
    constexpr uint32_t B_BYTES = BN * BK * 2;
    constexpr uint32_t TMEM_COLS = tmem_cols_for(BN);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;
    uint8_t *sB = smem + HALO_SA * HALO_SLOT;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sB + SB * B_BYTES);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * HALO_SA + 2 * SB + 1);
    const uint32_t fullA = smem_u32(bars), emptyA = fullA + 8 * HALO_SA;
    const uint32_t fullB = emptyA + 8 * HALO_SA, emptyB = fullB + 8 * SB;
    const uint32_t accum = emptyB + 8 * SB;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x0 = blockIdx.x * BM, y = blockIdx.y, img = blockIdx.z;
    const int ng = 3 * p.nch;  // (ky, channel step) groups
    const uint32_t halo_tx = HALO_ROWS * (uint32_t)p.rb, b_tx = (uint32_t)BN * (uint32_t)p.rb;

    if (threadIdx.x == 0) {
        for (int s = 0; s < HALO_SA; ++s) {
            mbar_init(fullA + 8 * s, 1);
            mbar_init(emptyA + 8 * s, 1);
        }
        for (int s = 0; s < SB; ++s) {
            mbar_init(fullB + 8 * s, 1);
            mbar_init(emptyB + 8 * s, 1);
        }
        mbar_init(accum, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    pdl_wait();  // every global access below follows the previous kernel

    if (threadIdx.x == 0) {
        // ---- producer
        int ga = 0, gb = 0;  // halo loads and weight loads issued
        bool fine = !p.stall;  // stalled (test hook): nothing is issued, so the MMA warp's waits run out
        for (int g = 0; g < ng && fine; ++g) {
            const int ky = g / p.nch, ch = g - ky * p.nch;
            const int sa = g % HALO_SA;
            if (!mbar_wait(emptyA + 8 * sa, ((uint32_t)(g / HALO_SA) & 1u) ^ 1u, p.err, ERR_PRODUCER)) break;
            const bool tl = p.tail && ch == p.nch - 1;  // the 32-channel tail step
            mbar_expect_tx(fullA + 8 * sa, tl ? HALO_ROWS * 64u : halo_tx);
            tma_load_4d(tl ? &tmA2 : &tmA, fullA + 8 * sa, smem_u32(sA + sa * HALO_SLOT), ch * p.kc, x0 - 1,
                        y + ky - 1, img + p.img_off);
            ga = g + 1;
            for (int kx = 0; kx < 3; ++kx) {
                const int kb = 3 * g + kx, sb = kb % SB;
                if (!mbar_wait(emptyB + 8 * sb, ((uint32_t)(kb / SB) & 1u) ^ 1u, p.err, ERR_PRODUCER)) {
                    fine = false;
                    break;
                }
                mbar_expect_tx(fullB + 8 * sb, tl ? (uint32_t)BN * 64u : b_tx);
                tma_load_3d(tl ? &tmB2 : &tmB, fullB + 8 * sb, smem_u32(sB + sb * B_BYTES), ch * p.kc, 0, ky * 3 + kx);
                gb = kb + 1;
            }
        }
        if (ga < ng || gb < 3 * ng) {
            // Error path: let the loads already issued land before the CTA exits (none when
            // stalled).
            const unsigned long long t0 = global_ns();
            for (int g = ga - HALO_SA < 0 ? 0 : ga - HALO_SA; g < ga; ++g)
                while (!mbar_try(fullA + 8 * (g % HALO_SA), (uint32_t)(g / HALO_SA) & 1u))
                    if (global_ns() - t0 > WAIT_NS) { atomicCAS(p.err, 0, ERR_DRAIN); break; }
            for (int kb = gb - SB < 0 ? 0 : gb - SB; kb < gb; ++kb)
                while (!mbar_try(fullB + 8 * (kb % SB), (uint32_t)(kb / SB) & 1u))
                    if (global_ns() - t0 > WAIT_NS) { atomicCAS(p.err, 0, ERR_DRAIN); break; }
        }
    } else if (threadIdx.x == 32) {
        // ---- MMA issuer
        const uint32_t idesc = F8 ? idesc_e4m3(BM, BN) : (p.f16 ? idesc_f16(BM, BN) : idesc_bf16(BM, BN));
        bool fine = true;
        for (int g = 0; g < ng && fine; ++g) {
            const int sa = g % HALO_SA;
            if (!mbar_wait(fullA + 8 * sa, (uint32_t)(g / HALO_SA) & 1u, p.err, ERR_MMA)) break;
            const uint32_t a0 = smem_u32(sA + sa * HALO_SLOT);
            const int ch = g % p.nch;
            const uint32_t rb = p.tail && ch == p.nch - 1 ? 64u : (uint32_t)p.rb;  // bytes of this K step
            for (int kx = 0; kx < 3; ++kx) {
                const int kb = 3 * g + kx, sb = kb % SB;
                if (!mbar_wait(fullB + 8 * sb, (uint32_t)(kb / SB) & 1u, p.err, ERR_MMA)) {
                    fine = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint64_t da = sw_desc(a0 + rb * (uint32_t)kx, rb);
                const uint64_t db = sw_desc(smem_u32(sB + sb * B_BYTES), rb);
                for (int kk = 0; kk < (int)rb / 32; ++kk)
                    umma<F8>(tmem, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc,
                              (g | kx | kk) != 0 ? 1u : 0u);
                umma_commit(emptyB + 8 * sb);
            }
            if (fine) umma_commit(emptyA + 8 * sa);  // the halo's three taps are done
        }
        umma_commit(accum);
    }

    int ok = 1;
    if (lane == 0) ok = mbar_wait(accum, 0, p.err, ERR_EPILOGUE) && *(volatile int *)p.err == 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) conv_epilogue<BN, HEAD, F8>(tmem, p, warp, lane, x0, y, img);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// Multi-row stride-1 variant for narrow layers (at most 32 outputs) whose input channels
// fit one or two K steps (the launcher takes it for one): there the per-CTA
// set-up (TMEM allocation, barriers, pipeline fill) outweighs the few MMAs of one row.  A
// CTA computes ROWS output rows of one 128-pixel column tile:
//   * warp 4, lane 0 (producer): the 9 x nch weight tiles once, then the halo units
//     (input row, channel step) of the ROWS + 2 input rows [x0 - 1, x0 + 129) in order
//     through a ring of RING x nch slots; each input row is loaded once for the three
//     output rows that read it;
//   * warp 5, lane 0 (MMA issuer): for output row r the nine taps of every channel step
//     from input rows r, r + 1, r + 2 into TMEM accumulator r % 2; then it frees the units
//     of input row r (their last reader) and signals the accumulator;
//   * warps 0-3 (epilogue): drain accumulator r % 2 into output row y0 + r while the MMAs of
//     row r + 1 run, then hand the accumulator back.
// Every wait is bounded as in the kernels above.
constexpr int ROWS = 4;
constexpr int RING = 4;  // input rows held at once
__host__ __device__ constexpr uint32_t halo_slot_for(int rb) { return (uint32_t)((HALO_ROWS * rb + 1023) / 1024 * 1024); }
__host__ __device__ constexpr uint32_t wtile_for(int bn, int rb) { return (uint32_t)((bn * rb + 1023) / 1024 * 1024); }
__host__ __device__ constexpr size_t rows_smem_for(int bn, int rb, int nch) {
    return (size_t)RING * nch * halo_slot_for(rb) + 9 * (size_t)nch * wtile_for(bn, rb) + 1024 + 256;
}

template <int BN, bool HEAD, bool F8, int NCH>
__global__ void __launch_bounds__(192, 1)
conv_tc_rows_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcLaunch p) {
    constexpr uint32_t ACC_COLS = tmem_cols_for(BN);
    constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    constexpr int nch = NCH, ru = RING * NCH;  // channel steps (p.nch), ring units
    const uint32_t hslot = halo_slot_for(p.rb), wtile = wtile_for(BN, p.rb);
    uint8_t *sA = smem;
    uint8_t *sW = smem + ru * hslot;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sW + 9 * nch * wtile);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * ru + 5);
    const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * ru, wfull = empty0 + 8 * ru;
    const uint32_t accf0 = wfull + 8, acce0 = accf0 + 16;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x0 = blockIdx.x * BM, y0 = blockIdx.y * ROWS, img = blockIdx.z;
    const int nrows = p.ho - y0 < ROWS ? p.ho - y0 : ROWS;
    const int nunits = (nrows + 2) * nch;  // input rows y0 - 1 .. y0 + nrows, every channel step

    if (threadIdx.x == 0) {
        for (int s = 0; s < ru; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(wfull, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf0 + 8 * b, 1);
            mbar_init(acce0 + 8 * b, 4);  // one arrival per epilogue warp
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    pdl_wait();  // every global access below follows the previous kernel

    if (warp == 4 && lane == 0) {
        // ---- producer
        mbar_expect_tx(wfull, 9u * (uint32_t)nch * BN * (uint32_t)p.rb);
        for (int t = 0; t < 9; ++t)
            for (int ch = 0; ch < nch; ++ch)
                tma_load_3d(&tmB, wfull, smem_u32(sW + (t * nch + ch) * wtile), ch * p.kc, 0, t);
        int issued = 0;
        for (int u = 0; u < nunits; ++u) {
            const int s = u % ru, i = u / nch, ch = u - i * nch;
            if (!mbar_wait(empty0 + 8 * s, ((uint32_t)(u / ru) & 1u) ^ 1u, p.err, ERR_PRODUCER)) break;
            mbar_expect_tx(full0 + 8 * s, HALO_ROWS * (uint32_t)p.rb);
            tma_load_4d(&tmA, full0 + 8 * s, smem_u32(sA + s * hslot), ch * p.kc, x0 - 1, y0 - 1 + i,
                        img + p.img_off);
            issued = u + 1;
        }
        if (issued < nunits) {
            // Error path: let the loads already issued land before the CTA exits.
            const unsigned long long t0 = global_ns();
            while (!mbar_try(wfull, 0))
                if (global_ns() - t0 > WAIT_NS) { atomicCAS(p.err, 0, ERR_DRAIN); break; }
            for (int u = issued - ru < 0 ? 0 : issued - ru; u < issued; ++u)
                while (!mbar_try(full0 + 8 * (u % ru), (uint32_t)(u / ru) & 1u))
                    if (global_ns() - t0 > WAIT_NS) { atomicCAS(p.err, 0, ERR_DRAIN); break; }
        }
    } else if (warp == 5 && lane == 0) {
        // ---- MMA issuer
        const uint32_t idesc = F8 ? idesc_e4m3(BM, BN) : (p.f16 ? idesc_f16(BM, BN) : idesc_bf16(BM, BN));
        bool fine = mbar_wait(wfull, 0, p.err, ERR_MMA);
        for (int r = 0; r < nrows && fine; ++r) {
            const int b = r & 1;
            // accumulator b was last drained for row r - 2
            if (r >= 2 && !mbar_wait(acce0 + 8 * b, (uint32_t)((r >> 1) - 1) & 1u, p.err, ERR_MMA)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t acc = tmem + (uint32_t)b * ACC_COLS;
            for (int ky = 0; ky < 3 && fine; ++ky) {
                for (int ch = 0; ch < nch; ++ch) {
                    const int u = (r + ky) * nch + ch, s = u % ru;
                    if (!mbar_wait(full0 + 8 * s, (uint32_t)(u / ru) & 1u, p.err, ERR_MMA)) {
                        fine = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a0 = smem_u32(sA + s * hslot);
                    for (int kx = 0; kx < 3; ++kx) {
                        const uint64_t da = sw_desc(a0 + (uint32_t)p.rb * (uint32_t)kx, (uint32_t)p.rb);
                        const uint64_t db = sw_desc(smem_u32(sW + ((ky * 3 + kx) * nch + ch) * wtile), (uint32_t)p.rb);
                        for (int kk = 0; kk < p.rb / 32; ++kk)
                            umma<F8>(acc, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc,
                                     (ky | ch | kx | kk) != 0 ? 1u : 0u);
                    }
                }
            }
            if (!fine) break;
            for (int ch = 0; ch < nch; ++ch) umma_commit(empty0 + 8 * ((r * nch + ch) % ru));  // input row r is done
            umma_commit(accf0 + 8 * b);
        }
    } else if (warp < 4) {
        // ---- epilogue (thread r of warps 0-3 owns accumulator row r = pixel x0 + r)
        for (int r = 0; r < nrows; ++r) {
            const int b = r & 1;
            int ok = 1;
            if (lane == 0) ok = mbar_wait(accf0 + 8 * b, (uint32_t)(r >> 1) & 1u, p.err, ERR_EPILOGUE) &&
                                *(volatile int *)p.err == 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            conv_epilogue<BN, HEAD, F8>(tmem + (uint32_t)b * ACC_COLS, p, warp, lane, x0, y0 + r, img);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(acce0 + 8 * b);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// Test hook: stride-1 conv launches still to stall (tc_test_stall_next_convs).
std::atomic<int> g_stall_next{0};

// 1 if this launch takes one of the armed stalls: never while st is being captured into a
// graph, so no graph ever bakes a stall in.
int take_stall(cudaStream_t st) {
    if (g_stall_next.load() <= 0) return 0;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (cs != cudaStreamCaptureStatusNone) return 0;
    int k = g_stall_next.load();
    while (k > 0 && !g_stall_next.compare_exchange_weak(k, k - 1)) {
    }
    return k > 0 ? 1 : 0;
}

template <int BN, bool HEAD = false, bool F8 = false>
cudaError_t launch_bn(const TcConvPlan &plan, const TcLaunch &lp, int n_img, cudaStream_t st) {
    dim3 grid((plan.wo + BM - 1) / BM, plan.ho, n_img);
    if constexpr (BN <= 32 && !HEAD) {
        // the multi-row form pays off where the grid stays large: measured on the 16- and
        // 32-channel pyramid levels (4 rows per CTA beat 8 and 2); the flow heads (two K
        // steps, one CTA per SM) and the coarse levels lose with ROWS times fewer CTAs
        if (plan.stride == 1 && plan.taps == 9 && plan.nch == 1) {
            const size_t smem = rows_smem_for(BN, plan.rb, 1);
            static size_t attr_bytes = 0;
            if (attr_bytes < smem) {
                cudaError_t e = cudaFuncSetAttribute(conv_tc_rows_kernel<BN, HEAD, F8, 1>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
                attr_bytes = smem;
            }
            const dim3 rgrid((plan.wo + BM - 1) / BM, (plan.ho + ROWS - 1) / ROWS, n_img);
            return launch_pdl(conv_tc_rows_kernel<BN, HEAD, F8, 1>, rgrid, dim3(192), smem, st, plan.tmA, plan.tmB, lp);
        }
    }
    if (plan.stride == 1 && plan.taps == 9) {
        static bool attr_set = false;
        const size_t smem = halo_smem_for(BN);
        if (!attr_set) {
            cudaError_t e = cudaFuncSetAttribute(conv_tc_halo_kernel<BN, HEAD, F8>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            attr_set = true;
        }
        TcLaunch lt = lp;
        lt.tail = plan.tail ? 1 : 0;
        lt.stall = take_stall(st);
        return launch_pdl(conv_tc_halo_kernel<BN, HEAD, F8>, grid, dim3(128), smem, st, plan.tmA, plan.tmB,
                          plan.tail ? plan.tmA2 : plan.tmA, plan.tail ? plan.tmB2 : plan.tmB, lt);
    } else {
        static size_t attr_bytes = 0;
        const size_t smem = smem_bytes_for(BN, plan.rb);
        if (attr_bytes < smem) {
            cudaError_t e =
                cudaFuncSetAttribute(conv_tc_kernel<BN, HEAD, F8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            attr_bytes = smem;
        }
        return launch_pdl(conv_tc_kernel<BN, HEAD, F8>, grid, dim3(128), smem, st, plan.tmA, plan.tmB, lp);
    }
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
        else
            cudaGetLastError();
    });
    return fn;
}

void TcConvPlan::release() {
    if (wpk) cudaFree(wpk);
    if (wscale) cudaFree(wscale);
    wpk = nullptr;
    wscale = nullptr;
    wpk_bytes = 0;
    enabled = false;
}

bool tc_plan_conv(TcConvPlan &plan, const ConvArgs &a, int n_in, const std::vector<float> &wk_simt, int *err,
                  std::string &why, bool f8, int taps, bool f16) {
    if (f8) f16 = false;
    plan.enabled = false;
    plan.head = false;
    if (taps != 9 && (taps != 1 || a.stride != 1)) { why = "taps must be 9, or 1 at stride 1"; return false; }
    const int bn = a.cout;
    const int align = f8 ? 16 : 8;  // 16-byte TMA strides and vector stores
    if (bn < 16 || bn > 128 || bn % 16 != 0) { why = "cout must be a multiple of 16 in [16, 128]"; return false; }
    if (a.cin % align != 0 || a.in_cs % align != 0 || a.out_cs % align != 0) {
        why = "channel counts must be multiples of 16 bytes";
        return false;
    }
    if (reinterpret_cast<uintptr_t>(a.in) % 16 != 0) { why = "input not 16-byte aligned"; return false; }
    if (a.stride != 1 && (a.stride != 2 || a.w % 2 != 0)) { why = "stride must be 1, or 2 with even width"; return false; }
    if (a.ho != (a.h - 1) / a.stride + 1 || a.wo != (a.w - 1) / a.stride + 1) { why = "output size mismatch"; return false; }
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) { why = "cuTensorMapEncodeTiled unavailable"; return false; }
    const cuuint64_t esz = f8 ? 1 : 2;
    // K step: the narrowest swizzle span (32, 64 or 128 bytes) that holds the input
    // channels, so layers with 16 or 32 channels do not multiply zero padding
    const int rb = a.cin * (int)esz <= 32 ? 32 : (a.cin * (int)esz <= 64 ? 64 : 128);
    const int kc = rb / (int)esz;
    const int nch = (a.cin + kc - 1) / kc, cinp = nch * kc;
    const CUtensorMapSwizzle swz = rb == 32 ? CU_TENSOR_MAP_SWIZZLE_32B
                                            : (rb == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B);
    // Packed weights [taps][cout][cinp] (zero beyond cin): bfloat16 or half, or e4m3 with
    // one scale per output channel (amax / 448 over its taps x cin weights).
    std::vector<uint8_t> pk((size_t)taps * bn * cinp * esz, 0);
    std::vector<float> ws(bn, 1.f);
    if (f8) {
        for (int o = 0; o < bn; ++o) {
            float amax = 0.f;
            for (size_t k = 0; k < (size_t)taps * a.cin; ++k) amax = fmaxf(amax, fabsf(wk_simt[k * bn + o]));
            ws[o] = amax > 0.f ? amax / 448.f : 1.f;
        }
    }
    for (int tap = 0; tap < taps; ++tap)
        for (int c = 0; c < a.cin; ++c)
            for (int o = 0; o < bn; ++o) {
                const float v = wk_simt[((size_t)tap * a.cin + c) * bn + o];
                const size_t idx = ((size_t)tap * bn + o) * cinp + c;
                if (f8) {
                    pk[idx] = (uint8_t)__nv_cvt_float_to_fp8(v / ws[o], __NV_SATFINITE, __NV_E4M3);
                } else if (f16) {
                    const __half b = __float2half_rn(v);
                    memcpy(&pk[2 * idx], &b, 2);
                } else {
                    const __nv_bfloat16 b = __float2bfloat16_rn(v);
                    memcpy(&pk[2 * idx], &b, 2);
                }
            }
    void *wdev = nullptr;
    float *sdev = nullptr;
    if (cudaMalloc(&wdev, pk.size()) != cudaSuccess || (f8 && cudaMalloc(&sdev, bn * sizeof(float)) != cudaSuccess)) {
        cudaGetLastError();
        if (wdev) cudaFree(wdev);
        why = "weight allocation failed";
        return false;
    }
    if (cudaMemcpy(wdev, pk.data(), pk.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        (f8 && cudaMemcpy(sdev, ws.data(), bn * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)) {
        cudaGetLastError();
        cudaFree(wdev);
        if (sdev) cudaFree(sdev);
        why = "weight upload failed";
        return false;
    }
    const CUtensorMapDataType dt = f8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                      : (f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
    const cuuint32_t ones[5] = {1, 1, 1, 1, 1};
    CUresult r;
    if (a.stride == 1) {
        const cuuint64_t dims[4] = {(cuuint64_t)a.cin, (cuuint64_t)a.w, (cuuint64_t)a.h, (cuuint64_t)n_in};
        const cuuint64_t strides[3] = {a.in_cs * esz, (cuuint64_t)a.w * a.in_cs * esz, (cuuint64_t)a.h * a.w * a.in_cs * esz};
        // the 3x3 stride-1 kernel loads halo rows; the pointwise one tiles of BM pixels
        const cuuint32_t box[4] = {(cuuint32_t)kc, taps == 9 ? HALO_ROWS : (cuuint32_t)BM, 1, 1};
        r = enc(&plan.tmA, dt, 4, const_cast<void *>(a.in), dims, strides, box, ones, CU_TENSOR_MAP_INTERLEAVE_NONE,
                swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        const cuuint64_t dims[5] = {(cuuint64_t)a.cin, 2, (cuuint64_t)(a.w / 2), (cuuint64_t)a.h, (cuuint64_t)n_in};
        const cuuint64_t strides[4] = {a.in_cs * esz, 2 * a.in_cs * esz, (cuuint64_t)a.w * a.in_cs * esz,
                                       (cuuint64_t)a.h * a.w * a.in_cs * esz};
        const cuuint32_t box[5] = {(cuuint32_t)kc, 1, BM, 1, 1};
        r = enc(&plan.tmA, dt, 5, const_cast<void *>(a.in), dims, strides, box, ones, CU_TENSOR_MAP_INTERLEAVE_NONE,
                swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (r == CUDA_SUCCESS) {
        const cuuint64_t dims[3] = {(cuuint64_t)cinp, (cuuint64_t)bn, (cuuint64_t)taps};
        const cuuint64_t strides[2] = {(cuuint64_t)cinp * esz, (cuuint64_t)bn * cinp * esz};
        const cuuint32_t box[3] = {(cuuint32_t)kc, (cuuint32_t)bn, 1};
        r = enc(&plan.tmB, dt, 3, wdev, dims, strides, box, ones, CU_TENSOR_MAP_INTERLEAVE_NONE,
                swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    // A stride-1 3x3 layer whose last 128-byte channel step holds at most 64 bytes of
    // channels (32 bf16, 64 e4m3) takes that step as 64-byte rows with the 64-byte swizzle:
    // the same tensors, boxes of 64 bytes.
    plan.tail = taps == 9 && a.stride == 1 && rb == 128 && nch >= 2 && (a.cin - (nch - 1) * kc) * (int)esz <= 64;
    const cuuint32_t tail_ch = (cuuint32_t)(64 / esz);
    if (r == CUDA_SUCCESS && plan.tail) {
        const cuuint64_t dims[4] = {(cuuint64_t)a.cin, (cuuint64_t)a.w, (cuuint64_t)a.h, (cuuint64_t)n_in};
        const cuuint64_t strides[3] = {a.in_cs * esz, (cuuint64_t)a.w * a.in_cs * esz, (cuuint64_t)a.h * a.w * a.in_cs * esz};
        const cuuint32_t box[4] = {tail_ch, HALO_ROWS, 1, 1};
        r = enc(&plan.tmA2, dt, 4, const_cast<void *>(a.in), dims, strides, box, ones, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r == CUDA_SUCCESS) {
            const cuuint64_t wdims[3] = {(cuuint64_t)cinp, (cuuint64_t)bn, (cuuint64_t)taps};
            const cuuint64_t wstrides[2] = {(cuuint64_t)cinp * esz, (cuuint64_t)bn * cinp * esz};
            const cuuint32_t wbox[3] = {tail_ch, (cuuint32_t)bn, 1};
            r = enc(&plan.tmB2, dt, 3, wdev, wdims, wstrides, wbox, ones, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        }
    }
    if (r != CUDA_SUCCESS) {
        cudaFree(wdev);
        if (sdev) cudaFree(sdev);
        why = "tensor map encoding failed (" + std::to_string((int)r) + ")";
        return false;
    }
    plan.bn = bn;
    plan.cout = bn;
    plan.taps = taps;
    plan.nch = nch;
    plan.kc = kc;
    plan.rb = rb;
    plan.f8 = f8;
    plan.f16 = f16;
    plan.stride = a.stride;
    plan.h = a.h;
    plan.w = a.w;
    plan.ho = a.ho;
    plan.wo = a.wo;
    plan.n_in = n_in;
    plan.in_base = a.in;
    plan.img_bytes = (size_t)a.h * a.w * a.in_cs * esz;
    plan.wpk = wdev;
    plan.wscale = sdev;
    plan.wpk_bytes = pk.size() + (f8 ? bn * sizeof(float) : 0);
    plan.err = err;
    plan.enabled = true;
    return true;
}

bool tc_plan_head(TcConvPlan &plan, const ConvArgs &a, int n_in, const std::vector<float> &wk_simt, int *err,
                  std::string &why, bool f8, int taps, bool f16) {
    if (a.cout > 16) { why = "head has more than 16 outputs"; return false; }
    std::vector<float> wk16((size_t)taps * a.cin * 16, 0.f);
    for (size_t k = 0; k < (size_t)taps * a.cin; ++k)
        for (int o = 0; o < a.cout; ++o) wk16[k * 16 + o] = wk_simt[k * a.cout + o];
    ConvArgs a16 = a;
    a16.cout = 16;
    a16.out_cs = 16;  // not used by the head epilogue
    if (!tc_plan_conv(plan, a16, n_in, wk16, err, why, f8, taps, f16)) return false;
    plan.head = true;
    plan.cout = a.cout;
    return true;
}

static bool image_offset(const TcConvPlan &plan, const ConvArgs &a, int *img_off) {
    const ptrdiff_t off = static_cast<const char *>(a.in) - static_cast<const char *>(plan.in_base);
    if (off < 0 || off % (ptrdiff_t)plan.img_bytes != 0) return false;
    *img_off = (int)(off / (ptrdiff_t)plan.img_bytes);
    return *img_off + a.n <= plan.n_in && a.n >= 1;
}

cudaError_t launch_conv_tc_head(const TcConvPlan &plan, const ConvArgs &a, const float *up, float *flow,
                                cudaStream_t st) {
    int img_off = 0;
    if (!plan.enabled || !plan.head || !image_offset(plan, a, &img_off)) return cudaErrorInvalidValue;
    TcLaunch lp{plan.nch, plan.kc, plan.rb, plan.stride, plan.ho, plan.wo, img_off, nullptr, 0, a.bias, 0, plan.err,
                flow, up, plan.wscale, 1.f, 0, 0, plan.taps, 0, plan.f16 ? 1 : 0};
    return plan.f8 ? launch_bn<16, true, true>(plan, lp, a.n, st) : launch_bn<16, true, false>(plan, lp, a.n, st);
}

template <bool F8>
static cudaError_t launch_any_bn(const TcConvPlan &plan, const TcLaunch &lp, int n, cudaStream_t st) {
    switch (plan.bn) {
        case 16: return launch_bn<16, false, F8>(plan, lp, n, st);
        case 32: return launch_bn<32, false, F8>(plan, lp, n, st);
        case 48: return launch_bn<48, false, F8>(plan, lp, n, st);
        case 64: return launch_bn<64, false, F8>(plan, lp, n, st);
        case 80: return launch_bn<80, false, F8>(plan, lp, n, st);
        case 96: return launch_bn<96, false, F8>(plan, lp, n, st);
        case 112: return launch_bn<112, false, F8>(plan, lp, n, st);
        case 128: return launch_bn<128, false, F8>(plan, lp, n, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_conv_tc(const TcConvPlan &plan, const ConvArgs &a, cudaStream_t st) {
    int img_off = 0;
    if (!plan.enabled || plan.head || !image_offset(plan, a, &img_off)) return cudaErrorInvalidValue;
    if (reinterpret_cast<uintptr_t>(a.out) % 16 != 0 || a.out_cs % (plan.f8 ? 16 : 8) != 0) return cudaErrorInvalidValue;
    TcLaunch lp{plan.nch, plan.kc, plan.rb, plan.stride, plan.ho, plan.wo, img_off, a.out, a.out_cs, a.bias, a.leaky,
                plan.err, nullptr, nullptr, plan.wscale, a.q_out, 0, 0, plan.taps, 0, plan.f16 ? 1 : 0};
    return plan.f8 ? launch_any_bn<true>(plan, lp, a.n, st) : launch_any_bn<false>(plan, lp, a.n, st);
}

cudaError_t launch_conv_tc_f32(const TcConvPlan &plan, const ConvArgs &a, bool accumulate, cudaStream_t st) {
    int img_off = 0;
    if (!plan.enabled || plan.head || plan.f8 || !image_offset(plan, a, &img_off)) return cudaErrorInvalidValue;
    if (reinterpret_cast<uintptr_t>(a.out) % 16 != 0 || a.out_cs % 4 != 0) return cudaErrorInvalidValue;
    TcLaunch lp{plan.nch, plan.kc, plan.rb, plan.stride, plan.ho, plan.wo, img_off, a.out, a.out_cs, a.bias, a.leaky,
                plan.err, nullptr, nullptr, plan.wscale, 1.f, 1, accumulate ? 1 : 0, plan.taps, 0, plan.f16 ? 1 : 0};
    return launch_any_bn<false>(plan, lp, a.n, st);
}

}  // namespace tc

extern "C" void tc_test_stall_next_convs(int count) { tc::g_stall_next.store(count > 0 ? count : 0); }
