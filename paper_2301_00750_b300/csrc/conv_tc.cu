// Implicit-GEMM 3x3 convolution on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// GEMM view: M = output pixels, N = cout, K = 9 taps x input channels, taken in K steps of
// one swizzle span: 64 bf16 (128 e4m3) channels with the 128-byte swizzle, or 32 / 16 bf16
// channels with the 64- / 32-byte swizzle for layers that have no more input channels than
// that (the 16- and 32-channel pyramid levels), so no step multiplies zero padding
// wider than the layer.  The descriptions below use the 128-byte case.  Stride-1 3x3 layers
// run conv_tc_tiles_kernel (below), a persistent kernel that reuses each loaded halo row for
// the three horizontal taps and up to three output rows and each loaded kernel row of
// weights for several output rows; the description here is of the per-tap kernel, which
// serves the stride-2 layers and the pointwise (1x1) convs.  One CTA computes a
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
#include <type_traits>

#include "../../include/tc_stream.h"
#include "conv_tc.cuh"
#include "tc_ptx.cuh"

namespace tc {

namespace {

using namespace ptx;

constexpr int BM = 128;                    // output pixels per CTA (MMA M)

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
    int stall;            // stride-1 kernels, test hook: the producer issues no loads (see tc_test_stall_next_convs)
    // persistent tile kernel (conv_tc_tiles_kernel): its tiling, chosen by the launcher
    int R;                // output rows per tile (1..TILE_RMAX), each a 128-pixel accumulator
    int acc_cols;         // TMEM columns per accumulator (two sets of R accumulators)
    int tmem_cols;        // TMEM columns allocated (a power of two >= 2 * R * acc_cols)
    int sa, sb;           // halo ring units (a channel step's R + 2 rows each); weight ring slots, a
                          // kernel row each (0: resident weights)
    int ntx, nrg, ntiles; // tiles: 126-pixel column tiles x groups of R rows x images
    int tailunit;         // halo unit 1 holds the 64-byte tail step (two channel steps per tile)
    int rev;              // tiles in reverse order (tile ts is ntiles - 1 - ts)
    int overlap;          // launcher only: keep the full rows per tile (see ConvArgs::overlap)
    int trigger;          // let the next kernel of the stream launch once every CTA holds its TMEM
};

// Epilogue shared by the conv kernels: thread r of the CTA owns accumulator row r, i.e.
// output pixel (img, y, x0 + r), stored for r < tw; columns [c_lo, c_hi) (multiples of 16);
// bias and e4m3 weight scales from global or shared memory.
template <int BN, bool HEAD, bool F8>
__device__ __forceinline__ void conv_epilogue(uint32_t tmem, const TcLaunch &p, int warp, int lane, int x0, int y,
                                              int img, int tw, const float *bias, const float *wscale, int c_lo,
                                              int c_hi) {
    if (HEAD) {
        const int x = x0 + warp * 32 + lane;
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16), r);
        if (warp * 32 + lane < tw && x < p.wo) {
            const size_t pix = (size_t)(img * p.ho + y) * p.wo + x;
            float2 up = make_float2(0.f, 0.f);
            if (p.up) up = reinterpret_cast<const float2 *>(p.up)[pix];
            const float s0 = F8 ? wscale[0] : 1.f, s1 = F8 ? wscale[1] : 1.f;
            reinterpret_cast<float2 *>(p.flow)[pix] =
                make_float2(up.x + (__uint_as_float(r[0]) * s0 + bias[0]), up.y + (__uint_as_float(r[1]) * s1 + bias[1]));
        }
    } else {
        const int row = warp * 32 + lane;
        const int x = x0 + row;
        const size_t pix = (size_t)(img * p.ho + y) * p.wo + x;
        const bool vec_params = ((reinterpret_cast<uintptr_t>(bias) |
                                  (F8 ? reinterpret_cast<uintptr_t>(wscale) : 0)) & 15) == 0;
#pragma unroll 1
        for (int c0 = c_lo; c0 < c_hi; c0 += 16) {
            uint32_t r[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
            if (row < tw && x < p.wo) {
                // bias (and e4m3 weight scales) of the 16 columns: four 16-byte loads where
                // the arrays allow it, else 16 scalar ones
                float bv[16], sv[16];
                if (vec_params) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 b4 = reinterpret_cast<const float4 *>(bias + c0)[q];
                        bv[4 * q] = b4.x; bv[4 * q + 1] = b4.y; bv[4 * q + 2] = b4.z; bv[4 * q + 3] = b4.w;
                        if (F8) {
                            const float4 s4 = reinterpret_cast<const float4 *>(wscale + c0)[q];
                            sv[4 * q] = s4.x; sv[4 * q + 1] = s4.y; sv[4 * q + 2] = s4.z; sv[4 * q + 3] = s4.w;
                        }
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        bv[j] = bias[c0 + j];
                        if (F8) sv[j] = wscale[c0 + j];
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
    if (p.trigger) pdl_trigger();
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
    if (ok) conv_epilogue<BN, HEAD, F8>(tmem, p, warp, lane, x0, y, img, BM, p.bias, p.wscale, 0, BN);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// Persistent stride-1 3x3 conv.  A tile is R output rows of TW = 126 consecutive pixels; the
// grid holds one CTA per SM and each CTA walks the tiles blockIdx.x, blockIdx.x + gridDim.x,
// ...  A halo row is the 128 input pixels [x0 - 1, x0 + 127) of one channel step, so the
// MMA's M = 128 rows read halo rows m + kx for output m: outputs 126 and 127 read the two
// rows past the slot and are discarded (no tile count changes at the pyramid sizes used, and
// a slot is exactly 128 x 128 bytes).  Per tile and channel step c the R + 2 halo rows form
// one unit of a ring (one barrier), and the weights of each kernel row (c, ky, kx = 0..2, one
// TMA box of three taps) are multiplied into all R row accumulators while resident, so an
// output row costs (R + 2) / R halo rows and 1 / R of the layer's weights.  Layers whose
// packed weights fit beside the ring keep them resident for the whole kernel (loaded once
// per CTA, before the previous kernel has finished); wider layers stream them through a
// second ring, a kernel row per slot, in the order the MMAs consume them.
//   * warp 8, lane 0 (halo producer): per tile and channel step, the unit of halo rows
//     0 .. R + 1;
//   * warp 9, lane 0 (weight producer): the resident weights once, or per tile, channel step
//     and kernel row the three taps of that row;
//   * warps 10 and 11, lane 0 (MMA issuers): issuer j owns the output rows r = j, j + 2, ...
//     of every tile.  Per channel step it waits for the halo unit, per kernel row for the
//     weight slot; it issues the K steps of its rows for the three taps (halo row r + ky
//     shifted by kx pixels: a row offset of the swizzled slot) and releases the weight slot,
//     then the halo unit after ky = 2.  Every release barrier counts both issuers.  A thread
//     issues MMAs only as fast as its instruction stream allows (a barrier wait or a commit
//     costs ~100-160 cycles of issue), so two issuers overlap one's synchronisation with the
//     other's MMAs; each accumulator still receives its MMAs in the same order;
//   * warps 0-7 (epilogue): warp w drains TMEM lanes 32 (w % 4) .. of rows r = w / 4,
//     w / 4 + 2, ... of the finished set, then returns the set to the issuers.  The two sets
//     let the epilogue of tile j run under the MMAs of tile j + 1.
// Every wait is bounded as in the kernel above; on an error each role stops, the producers
// wait for their loads in flight and the issuers for their MMAs before TMEM is freed.
constexpr int TW = BM - 2;  // output pixels per tile
constexpr int TILE_RMAX = 8;
constexpr int TILE_EPI_WARPS = 8;
constexpr int TILE_ISSUERS = 2;
constexpr int TILE_THREADS = 32 * (TILE_EPI_WARPS + 2 + TILE_ISSUERS);
__host__ __device__ constexpr uint32_t round1k(uint32_t b) { return (b + 1023u) / 1024u * 1024u; }
__host__ __device__ constexpr int tile_issuers(int r) { return r >= 2 ? TILE_ISSUERS : 1; }

// Waits for the last loads issued into a ring to land (error path of the producers).
__device__ __forceinline__ void drain_ring(uint32_t full0, int slots, uint32_t issued, int *err) {
    const unsigned long long t0 = global_ns();
    for (uint32_t u = issued > (uint32_t)slots ? issued - (uint32_t)slots : 0; u < issued; ++u)
        while (!mbar_try(full0 + 8 * (u % (uint32_t)slots), (u / (uint32_t)slots) & 1u))
            if (global_ns() - t0 > WAIT_NS) { atomicCAS(err, 0, ERR_DRAIN); return; }
}

// The K steps of one tap into an issuer's accumulators: its m-th row reads halo slot
// descriptor dA[m] advanced by the kx shift.  NK = 4, 2 or 1 (128-, 64- or 32-byte channel
// steps); f0 = 0 for the first MMA of a tile (clears the accumulators).
template <bool F8, int M, int NK>
__device__ __forceinline__ void tap_mmas(uint32_t acc0, uint32_t acc_step, const uint64_t (&dA)[M], uint32_t ashift,
                                         uint64_t db, uint32_t idesc, int nmine, uint32_t f0) {
#pragma unroll
    for (int kk = 0; kk < NK; ++kk)
#pragma unroll
        for (int m = 0; m < M; ++m)
            if (m < nmine)
                umma<F8>(acc0 + (uint32_t)m * acc_step, dA[m] + (uint64_t)(ashift + 2 * kk), db + (uint64_t)(2 * kk),
                         idesc, kk == 0 ? f0 : 1u);
}

template <int BN, bool HEAD, bool F8, int R>
__global__ void __launch_bounds__(TILE_THREADS, 1)
conv_tc_tiles_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmB2,
                     const TcLaunch p) {
    constexpr int NI = tile_issuers(R);  // MMA issuers
    constexpr int MR = R / NI;           // accumulator rows per issuer
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int nch = p.nch, UA = p.sa, SB = p.sb;
    const bool resident = SB == 0;
    // a kernel row of weights (three taps): bytes in a full channel step and in the 64-byte tail step
    const uint32_t ufull = round1k(3u * BN * (uint32_t)p.rb), utail = round1k(3u * BN * 64u);
    const uint32_t wbytes = resident ? 3u * (uint32_t)(nch - p.tail) * ufull + (p.tail ? 3u * utail : 0u)
                                     : (uint32_t)SB * ufull;
    // halo units: (R + 2) slots of a channel step; with p.tailunit (two steps per tile, the
    // second a 64-byte tail) unit 0 always holds the full step and unit 1 the tail step, in
    // slots of their own widths
    const uint32_t aslot = (uint32_t)BM * (uint32_t)p.rb, aunit = (uint32_t)(R + 2) * aslot;
    const uint32_t aslot_t = p.tailunit ? (uint32_t)BM * 64u : aslot;
    auto unit_base = [&](uint32_t u) -> uint32_t { return p.tailunit ? (u ? aunit : 0u) : u * aunit; };
    const uint32_t abytes = p.tailunit ? aunit + (uint32_t)(R + 2) * aslot_t : (uint32_t)UA * aunit;
    uint8_t *sW = smem;
    uint8_t *sA = smem + wbytes;
    // 256 bytes after the halo ring: the two rows past a slot that outputs 126, 127 read
    uint64_t *bars = reinterpret_cast<uint64_t *>(sA + abytes + 256);
    // bias and e4m3 weight scales, staged once for the epilogue (512 bytes after the barriers)
    float *sbias = reinterpret_cast<float *>(reinterpret_cast<uint8_t *>(bars) + 512), *sscale = sbias + 128;
    const uint32_t fullA = smem_u32(bars), emptyA = fullA + 8 * UA;
    const uint32_t fullB = emptyA + 8 * UA, emptyB = fullB + 8 * SB;
    const uint32_t wfull = emptyB + 8 * SB, accf0 = wfull + 8, acce0 = accf0 + 16, done0 = acce0 + 16;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * UA + 2 * SB + 7);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < UA; ++s) {
            mbar_init(fullA + 8 * s, 1);
            mbar_init(emptyA + 8 * s, NI);
        }
        for (int s = 0; s < SB; ++s) {
            mbar_init(fullB + 8 * s, 1);
            mbar_init(emptyB + 8 * s, NI);
        }
        mbar_init(wfull, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf0 + 8 * b, NI);
            mbar_init(acce0 + 8 * b, TILE_EPI_WARPS);
            mbar_init(done0 + 8 * b, 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)p.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    if (p.trigger) pdl_trigger();

    // offset of the resident kernel row (c, ky): full steps first, the tail step last
    auto woff = [&](int c, int ky) -> uint32_t {
        return (uint32_t)(c * 3) * ufull + (uint32_t)ky * (p.tail && c == nch - 1 ? utail : ufull);
    };

    if (warp == TILE_EPI_WARPS && lane == 0) {
        // ---- halo producer
        pdl_wait();  // the activations follow the previous kernel
        bool fine = !p.stall;  // stalled (test hook): nothing is issued, so the issuers' waits run out
        uint32_t ua = 0, u = 0, q = 0;  // units issued; unit and phase of the next one
        for (int ts = blockIdx.x; ts < p.ntiles && fine; ts += gridDim.x) {
            const int tt = p.rev ? p.ntiles - 1 - ts : ts;
            const int xt = tt % p.ntx, rg = (tt / p.ntx) % p.nrg, img = tt / (p.ntx * p.nrg);
            const int x0 = xt * TW, y0 = rg * R;
            const int nrows = p.ho - y0 < R ? p.ho - y0 : R;
            for (int c = 0; c < nch; ++c) {
                const bool tl = p.tail && c == nch - 1;
                if (!mbar_wait(emptyA + 8 * u, q ^ 1u, p.err, ERR_PRODUCER)) {
                    fine = false;
                    break;
                }
                mbar_expect_tx(fullA + 8 * u, (uint32_t)(nrows + 2) * BM * (tl ? 64u : (uint32_t)p.rb));
                const uint32_t dst = smem_u32(sA + unit_base(u)), pitch = p.tailunit && u ? aslot_t : aslot;
                for (int i = 0; i < nrows + 2; ++i)
                    tma_load_4d(tl ? &tmA2 : &tmA, fullA + 8 * u, dst + (uint32_t)i * pitch, c * p.kc, x0 - 1,
                                y0 - 1 + i, img + p.img_off);
                ++ua;
                if (++u == (uint32_t)UA) { u = 0; q ^= 1u; }
            }
        }
        if (!fine) drain_ring(fullA, UA, ua, p.err);  // let the loads already issued land
    } else if (warp == TILE_EPI_WARPS + 1 && lane == 0) {
        // ---- weight producer
        bool fine = !p.stall;
        if (resident) {
            // the packed weights are constant: loaded before the previous kernel has finished
            if (fine) {
                mbar_expect_tx(wfull, (uint32_t)(9 * (nch - p.tail) * BN * p.rb + (p.tail ? 9 * BN * 64 : 0)));
                for (int c = 0; c < nch; ++c) {
                    const bool tl = p.tail && c == nch - 1;
                    for (int ky = 0; ky < 3; ++ky)
                        tma_load_3d(tl ? &tmB2 : &tmB, wfull, smem_u32(sW + woff(c, ky)), c * p.kc, 0, 3 * ky);
                }
                const unsigned long long t0 = global_ns();
                while (!mbar_try(wfull, 0))  // before this thread may leave
                    if (global_ns() - t0 > WAIT_NS) { atomicCAS(p.err, 0, ERR_DRAIN); break; }
            }
        } else {
            uint32_t ub = 0, s = 0, q = 0;
            for (int ts = blockIdx.x; ts < p.ntiles && fine; ts += gridDim.x) {
                for (int c = 0; c < nch && fine; ++c) {
                    const bool tl = p.tail && c == nch - 1;
                    const uint32_t tx = 3u * BN * (tl ? 64u : (uint32_t)p.rb);
                    for (int ky = 0; ky < 3; ++ky) {
                        if (!mbar_wait(emptyB + 8 * s, q ^ 1u, p.err, ERR_PRODUCER)) {
                            fine = false;
                            break;
                        }
                        mbar_expect_tx(fullB + 8 * s, tx);
                        tma_load_3d(tl ? &tmB2 : &tmB, fullB + 8 * s, smem_u32(sW + s * ufull), c * p.kc, 0, 3 * ky);
                        ++ub;
                        if (++s == (uint32_t)SB) { s = 0; q ^= 1u; }
                    }
                }
            }
            if (!fine) drain_ring(fullB, SB, ub, p.err);
        }
    } else if (warp >= TILE_EPI_WARPS + 2 && warp < TILE_EPI_WARPS + 2 + NI && lane == 0) {
        // ---- MMA issuer j
        const int j = warp - (TILE_EPI_WARPS + 2);
        const uint32_t idesc = F8 ? idesc_e4m3(BM, BN) : (p.f16 ? idesc_f16(BM, BN) : idesc_bf16(BM, BN));
        const uint32_t acc_step = (uint32_t)p.acc_cols, unit16 = ufull >> 4;
        bool fine = !resident || mbar_wait(wfull, 0, p.err, ERR_MMA);
        uint32_t ua = 0, qa = 0;  // halo ring: unit and phase of the next step
        uint32_t sb = 0, qb = 0;  // weight ring
        int k = 0;
        for (int ts = blockIdx.x; ts < p.ntiles && fine; ts += gridDim.x, ++k) {
            const int b = k & 1, use = k >> 1;
            if (use >= 1) {
                if (!mbar_wait(acce0 + 8 * b, (uint32_t)(use - 1) & 1u, p.err, ERR_MMA)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");  // the epilogue's TMEM reads are done
            }
            const int y0 = (((p.rev ? p.ntiles - 1 - ts : ts) / p.ntx) % p.nrg) * R;
            const int nrows = p.ho - y0 < R ? p.ho - y0 : R;
            const int nmine = (nrows - j + NI - 1) / NI;  // rows j, j + NI, ... below nrows
            const uint32_t acc0 = tmem + (uint32_t)(b * R + j) * acc_step;
            for (int c = 0; c < nch && fine; ++c) {
                const bool tl = p.tail && c == nch - 1;
                const uint32_t rbc = tl ? 64u : (uint32_t)p.rb;
                if (!mbar_wait(fullA + 8 * ua, qa, p.err, ERR_MMA)) { fine = false; break; }
                const uint64_t dA0 = sw_desc(smem_u32(sA + unit_base(ua)), rbc), dW0 = sw_desc(smem_u32(sW), rbc);
                const uint32_t sh = rbc >> 4;                    // one pixel row of a halo slot, 16-byte units
                const uint32_t slot16 = (p.tailunit && ua ? aslot_t : aslot) >> 4;
                const uint32_t tap16 = (uint32_t)BN * rbc >> 4;  // one tap of a weight row
                for (int ky = 0; ky < 3 && fine; ++ky) {
                    uint64_t dB;
                    if (resident) {
                        dB = dW0 + (uint64_t)(woff(c, ky) >> 4);
                    } else {
                        if (!mbar_wait(fullB + 8 * sb, qb, p.err, ERR_MMA)) { fine = false; break; }
                        dB = dW0 + (uint64_t)(sb * unit16);
                    }
                    // this issuer's rows r = j + m NI read halo row r + ky of the unit
                    uint64_t dA[MR];
#pragma unroll
                    for (int m = 0; m < MR; ++m) dA[m] = dA0 + (uint64_t)((uint32_t)(j + m * NI + ky) * slot16);
                    for (int kx = 0; kx < 3; ++kx) {
                        const uint32_t f = (c | ky | kx) != 0 ? 1u : 0u;
                        const uint64_t db = dB + (uint64_t)(kx * tap16);
                        if (rbc == 128u)
                            tap_mmas<F8, MR, 4>(acc0, NI * acc_step, dA, sh * (uint32_t)kx, db, idesc, nmine, f);
                        else if (rbc == 64u)
                            tap_mmas<F8, MR, 2>(acc0, NI * acc_step, dA, sh * (uint32_t)kx, db, idesc, nmine, f);
                        else
                            tap_mmas<F8, MR, 1>(acc0, NI * acc_step, dA, sh * (uint32_t)kx, db, idesc, nmine, f);
                    }
                    if (!resident) {
                        umma_commit(emptyB + 8 * sb);
                        if (++sb == (uint32_t)SB) { sb = 0; qb ^= 1u; }
                    }
                }
                if (!fine) break;
                umma_commit(emptyA + 8 * ua);  // the step's halo rows are read
                if (++ua == (uint32_t)UA) { ua = 0; qa ^= 1u; }
            }
            if (fine) umma_commit(accf0 + 8 * b);
        }
        // every MMA this issuer issued has completed once its `done` fires
        umma_commit(done0 + 8 * j);
        const unsigned long long t0 = global_ns();
        while (!mbar_try(done0 + 8 * j, 0))
            if (global_ns() - t0 > WAIT_NS) { atomicCAS(p.err, 0, ERR_DRAIN); break; }
    } else if (warp < TILE_EPI_WARPS) {
        // ---- epilogue
        for (int i = threadIdx.x; i < BN; i += 32 * TILE_EPI_WARPS) {
            if (i < (HEAD ? 2 : BN)) sbias[i] = p.bias[i];  // a flow head's bias has its 2 outputs only
            if (F8) sscale[i] = p.wscale[i];
        }
        asm volatile("bar.sync 1, %0;" ::"n"(32 * TILE_EPI_WARPS) : "memory");  // the epilogue warps only
        pdl_wait();  // the outputs may still be read by the previous kernel
        const int q = warp & 3, g = warp >> 2;
        // one-row tiles: the two warp groups take half of the columns each; else alternate rows
        constexpr bool COLS = !HEAD && BN >= 32 && R == 1;
        constexpr int CH = (BN / 2 + 15) / 16 * 16;
        int k = 0;
        for (int ts = blockIdx.x; ts < p.ntiles; ts += gridDim.x, ++k) {
            const int b = k & 1, use = k >> 1;
            // the issuers hand a set over only when all of their MMAs were issued
            int ok = 1;
            if (lane == 0) ok = mbar_wait(accf0 + 8 * b, (uint32_t)use & 1u, p.err, ERR_EPILOGUE);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int tt = p.rev ? p.ntiles - 1 - ts : ts;
            const int xt = tt % p.ntx, rg = (tt / p.ntx) % p.nrg, img = tt / (p.ntx * p.nrg);
            const int y0 = rg * R, nrows = p.ho - y0 < R ? p.ho - y0 : R;
            const uint32_t acc0 = tmem + (uint32_t)(b * R) * (uint32_t)p.acc_cols;
            if (COLS) {
                conv_epilogue<BN, HEAD, F8>(acc0, p, q, lane, xt * TW, y0, img, TW, sbias, sscale, g ? CH : 0,
                                            g ? BN : CH);
            } else {
                for (int r = g; r < nrows; r += TILE_EPI_WARPS / 4)
                    conv_epilogue<BN, HEAD, F8>(acc0 + (uint32_t)r * (uint32_t)p.acc_cols, p, q, lane, xt * TW, y0 + r,
                                                img, TW, sbias, sscale, 0, BN);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(acce0 + 8 * b);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)p.tmem_cols)
                     : "memory");
    }
}

// Test hook: stride-1 3x3 conv launches still to stall (tc_test_stall_next_convs).
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

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int d = 0;
        if (cudaGetDevice(&d) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d) != cudaSuccess) {
            cudaGetLastError();
            n = 148;
        }
    }
    return n;
}

// Tiling of conv_tc_tiles_kernel for a planned stride-1 3x3 layer over n_img images:
// rows per tile, halo units (at least two, so the next channel step loads under the current
// one), resident or streamed weights.  Returns the dynamic shared memory it needs.
// overlap: the launch shares the GPU with another stream's kernels; the rows per tile are
// not cut down to cover the SMs (measured at 1080p: sequential 1201 vs 1269 frames/s, so
// off there; pipelined 1633 vs 1575).
constexpr int kOverlapGrid = 120;

size_t plan_tiles(const TcConvPlan &plan, int bn, int n_img, TcLaunch &lp, int *grid, bool overlap) {
    constexpr uint32_t SMEM_MAX = 232448;                  // opt-in maximum per CTA
    const uint32_t budget = SMEM_MAX - 1024 - 256 - 1536;   // alignment slack, slot overrun guard, barriers and epilogue parameters
    const int acc = tmem_cols_for(bn);
    const uint32_t aslot = (uint32_t)BM * (uint32_t)plan.rb;
    const uint32_t ufull = round1k(3u * (uint32_t)bn * (uint32_t)plan.rb), utail = round1k(3u * (uint32_t)bn * 64u);
    const int tail = plan.tail ? 1 : 0;
    const uint32_t wres = 3u * (uint32_t)(plan.nch - tail) * ufull + (tail ? 3u * utail : 0u);
    const int ntx = (plan.wo + TW - 1) / TW;
    const int nsm = sm_count();
    // rows per tile: as many as two accumulator sets of TMEM hold, fewer where the tiles
    // would not cover the SMs or two halo units would not fit beside the weights
    int R = 512 / (2 * acc);
    if (R > TILE_RMAX) R = TILE_RMAX;
    while (!overlap && R > 1 && (long)ntx * ((plan.ho + R - 1) / R) * n_img < nsm) R /= 2;
    // one-step layers with narrow K steps (the 16- and 32-channel pyramid levels) get few
    // tiles per CTA, too few to overlap one tile's loads, MMAs and epilogue with the next; in
    // a launch alone on the GPU, rows such that two CTAs share each SM let one CTA's latency
    // hide under the other's work (sequential 1264 vs 1252 frames/s; with overlapped launches
    // it cost 0.5%, and on E4M3 layers, whose 128-byte step holds up to 128 channels, 4%)
    if (!overlap && plan.nch == 1 && plan.rb <= 64 && R >= 2 && 2 * R * acc > 256) R /= 2;
    // two channel steps, the second a 64-byte tail: the two halo units alternate between
    // them, so unit 1 takes tail-width slots
    const bool split = tail && plan.nch == 2 && plan.rb == 128;
    int SB = 0;
    uint32_t wbytes = 0, aunit = 0, a2 = 0;  // a2: bytes of two halo units
    for (;; R /= 2) {
        aunit = (uint32_t)(R + 2) * aslot;
        a2 = split ? aunit + (uint32_t)(R + 2) * BM * 64u : 2 * aunit;
        if (wres + a2 <= budget) { SB = 0; wbytes = wres; break; }
        if (3 * ufull + a2 <= budget) { SB = 3; wbytes = 3 * ufull; break; }
        if (2 * ufull + a2 <= budget) { SB = 2; wbytes = 2 * ufull; break; }
        if (R == 1) return 0;  // no tiling fits
    }
    // two halo units: the next channel step loads under the current one (deeper rings
    // measured no faster, and the smaller footprint leaves room for other streams' CTAs)
    const int UA = 2;
    lp.tailunit = split ? 1 : 0;
    lp.R = R;
    lp.acc_cols = acc;
    int cols = 32;
    while (cols < 2 * R * acc) cols *= 2;
    lp.tmem_cols = cols;
    lp.sa = UA;
    lp.sb = SB;
    lp.tail = tail;
    lp.ntx = ntx;
    lp.nrg = (plan.ho + R - 1) / R;
    lp.ntiles = ntx * lp.nrg * n_img;
    const size_t smem = 1024 + wbytes + (size_t)a2 + 256 + 1536;
    // resident CTAs per SM: TMEM columns and the SM's 228 KB of shared memory (1 KB of it
    // reserved per CTA)
    int per_sm = 512 / cols;
    const int by_smem = (int)(233472 / (smem + 1024));
    if (by_smem < per_sm) per_sm = by_smem;
    *grid = lp.ntiles < nsm * per_sm ? lp.ntiles : nsm * per_sm;
    // overlapped launches also leave SMs to the other streams' kernels: a persistent grid of at
    // most kOverlapGrid CTAs (its tiles are spread over fewer SMs, so none starts late behind
    // another stream's CTAs and holds up the launch's end)
    if (overlap && *grid > kOverlapGrid) *grid = kOverlapGrid;
    return smem;
}

// Early launch of the next kernel (griddepcontrol.launch_dependents once a CTA holds its TMEM)
// for a launch alone on the GPU whose CTAs leave at least half of the SMs free: the next
// kernel's CTAs then set up (barriers, TMEM, their constant weights) on those SMs while this
// one runs, and wait in griddepcontrol.wait for its results.  Every CTA of this launch holds
// its TMEM before any CTA of the next one starts, so the waiting CTAs only wait on work that
// is running.  Launches that fill the GPU, and those of pipelined mode (whose streams share
// the GPU), trigger at exit.  Measured at 1080p in default mode: about 1272 -> 1285-1288
// frames/s with this rule; an early trigger in every persistent launch, 1279.5 against 1287.5
// (in pipelined mode, 4% slower).  A server's batches run in default mode, several at once,
// and keep the rule (8-bit serving capacity 1759.5 vs 1743.5 frames/s).
inline int early_trigger(const TcLaunch &lp, long ctas) { return !lp.overlap && 2 * ctas <= sm_count() ? 1 : 0; }

template <int BN, bool HEAD, bool F8, int R>
cudaError_t launch_tiles(const TcConvPlan &plan, const TcLaunch &lt, int grid, size_t smem, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(conv_tc_tiles_kernel<BN, HEAD, F8, R>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    return launch_pdl(conv_tc_tiles_kernel<BN, HEAD, F8, R>, dim3(grid), dim3(TILE_THREADS), smem, st, plan.tmA, plan.tmB,
                      plan.tail ? plan.tmA2 : plan.tmA, plan.tail ? plan.tmB2 : plan.tmB, lt);
}

template <int BN, bool HEAD = false, bool F8 = false>
cudaError_t launch_bn(const TcConvPlan &plan, const TcLaunch &lp, int n_img, cudaStream_t st) {
    if (plan.stride == 1 && plan.taps == 9) {
        TcLaunch lt = lp;
        int g = 0;
        const size_t smem = plan_tiles(plan, BN, n_img, lt, &g, lp.overlap != 0);
        if (smem == 0 || lt.sa < 2) return cudaErrorInvalidConfiguration;
        lt.stall = take_stall(st);
        lt.trigger = early_trigger(lt, g);
        constexpr int ACC = tmem_cols_for(BN);
        switch (lt.R) {
            case 1: return launch_tiles<BN, HEAD, F8, 1>(plan, lt, g, smem, st);
            case 2: return launch_tiles<BN, HEAD, F8, 2>(plan, lt, g, smem, st);
            case 4: if constexpr (ACC <= 64) return launch_tiles<BN, HEAD, F8, 4>(plan, lt, g, smem, st); break;
            case 8: if constexpr (ACC <= 32) return launch_tiles<BN, HEAD, F8, 8>(plan, lt, g, smem, st); break;
            default: break;
        }
        return cudaErrorInvalidConfiguration;
    }
    const dim3 grid((plan.wo + BM - 1) / BM, plan.ho, n_img);
    TcLaunch l1 = lp;
    l1.trigger = early_trigger(lp, (long)grid.x * grid.y * grid.z);
    static size_t attr_bytes = 0;
    const size_t smem = smem_bytes_for(BN, plan.rb);
    if (attr_bytes < smem) {
        cudaError_t e =
            cudaFuncSetAttribute(conv_tc_kernel<BN, HEAD, F8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_bytes = smem;
    }
    return launch_pdl(conv_tc_kernel<BN, HEAD, F8>, grid, dim3(128), smem, st, plan.tmA, plan.tmB, l1);
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
        // halo rows of the 3x3 kernel and pixel tiles of the pointwise one: BM pixels
        const cuuint32_t box[4] = {(cuuint32_t)kc, (cuuint32_t)BM, 1, 1};
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
        // the stride-1 3x3 kernel loads a kernel row (three taps) at a time, the others one tap
        const cuuint32_t box[3] = {(cuuint32_t)kc, (cuuint32_t)bn, taps == 9 && a.stride == 1 ? 3u : 1u};
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
        const cuuint32_t box[4] = {tail_ch, (cuuint32_t)BM, 1, 1};
        r = enc(&plan.tmA2, dt, 4, const_cast<void *>(a.in), dims, strides, box, ones, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r == CUDA_SUCCESS) {
            const cuuint64_t wdims[3] = {(cuuint64_t)cinp, (cuuint64_t)bn, (cuuint64_t)taps};
            const cuuint64_t wstrides[2] = {(cuuint64_t)cinp * esz, (cuuint64_t)bn * cinp * esz};
            const cuuint32_t wbox[3] = {tail_ch, (cuuint32_t)bn, 3};
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
    lp.overlap = a.overlap;
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
    lp.rev = a.rev;
    lp.overlap = a.overlap;
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
