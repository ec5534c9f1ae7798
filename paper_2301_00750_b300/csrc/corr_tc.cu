// Correlation cost volume (Sec. 3.2) on the 5th-generation tensor cores.
//
// For a block of 16 x 8 output pixels the products f_self(x) . f_other(q) are a dense GEMM
// D[m][n] = sum_c A[m][c] B[n][c] with M = 128 block pixels and N = the (16+2R) x (8+2R)
// halo positions q around the block; the cost volume of pixel m at displacement d is the
// entry D[m][q = m + d] (81 of the 384 columns of its row for R = 4).  One TMA load brings
// the block's self features [8][16][64 ch] and one the halo of the other map
// [8+2R][16+2R][64 ch] (zero outside the map, which gives the zero product the definition
// asks for), 128-byte swizzled; one lane issues tcgen05.mma kind::f16 (BF16 x BF16 or
// F16 x F16 -> FP32) for the two halves of N into TMEM; the four warps then read, per
// displacement row dy, the two halo rows their 32 pixels need (tcgen05.ld), pick each
// pixel's 2R+1 entries through a per-thread shared-memory slice, scale by 1/C, apply
// LeakyReLU, and store the (2R+1)^2 values in the features' type.  The self features of
// the pixel are copied into the estimator input in the same pass.  Waits are bounded like
// those of the convolution kernel.
#include <mutex>

#include "corr_tc.cuh"
#include "tc_ptx.cuh"

namespace tc {

namespace {

using namespace ptx;

constexpr int BX = 16, BY = 8;  // output pixel block: M = 128 rows, row m = py * 16 + px
constexpr int BK = 64;          // channels per TMA step (128 B of bf16)
constexpr int MAX_NCH = 2;      // channels <= 128
constexpr int TILE_CORR_EPI = 8;  // epilogue warps: two halves of the displacements per pixel

enum : int { ERR_CORR_MMA = 5, ERR_CORR_EPILOGUE = 6, ERR_CORR_DRAIN = 7, ERR_CORR_PRODUCER = 8 };

struct CorrTcLaunch {
    int h, w, nch;
    int img_s[2], img_o[2];
    void *out;    // bf16 or e4m3 cost volume
    int out_cs;
    int vec_out;  // out and out_cs allow 16-byte stores
    const void *fs[2];
    int c;
    void *self_copy;
    float scale;  // dot product -> cost: 1/C (bf16), s_f^2 / C (e4m3 features with scale s_f)
    float q_out;  // e4m3: 1 / scale of the stored cost volume
    int *err;
    int rb;       // bytes of channels per step (128, or 64: 32 bf16 channels with the 64-byte swizzle)
    int f16;      // 16-bit features and cost volume are IEEE half instead of bfloat16
    // Lane pairs (pair_lanes > 0, any number of entries): entry z is direction d = z & 1 of
    // lane q = z >> 1; self image s0 + q + d pair_lanes, other image o0 + q oq + d od; the
    // self copy reads fs[0] + (q + d pair_lanes) fs_img_bytes.
    int pair_lanes, s0, o0, oq, od;
    size_t fs_img_bytes;
    int nb;       // batch entries (blocks run over nbx x nby x nb)
    int nstages;  // operand stages in shared memory
    int tma_self; // the self copy is a TMA store of the block's self operand (tmC), not per thread
    int trigger;  // let the next kernel of the stream launch once every CTA holds its TMEM
};

template <int R>
struct Geo {
    static constexpr int HX = BX + 2 * R, HY = BY + 2 * R, NPOS = HX * HY;
    static constexpr int NP = (NPOS + 31) / 32 * 32, NH = NP / 2;
    static constexpr uint32_t TMEM_COLS = NP <= 256 ? 256 : 512;
    // epilogue: per displacement row dy a warp reads the two halo rows of its two pixel rows
    static constexpr int WIN = (2 * HX + 15) / 16 * 16;  // columns loaded (tcgen05.ld x16 granularity)
    // per-thread staging slice: a whole number of 16-byte units, odd, so the 16-byte stores
    // of 8 consecutive threads hit distinct banks
    static constexpr int SSTRIDE = (WIN / 4) % 2 ? WIN : WIN + 4;
    static constexpr size_t SLICES = (size_t)TILE_CORR_EPI * 32 * SSTRIDE * 4;
    static_assert(NH % 16 == 0 && NH <= 256, "MMA N");
    static_assert(2 * (BY / 2 - 1) + 2 * R + 2 <= HY && (HY - 2) * HX + WIN <= (int)TMEM_COLS,
                  "epilogue column window inside TMEM");
};

// Operand bytes of one block: per channel step the self block [8][16][rb] and the other
// map's halo [HY][HX][rb], each rounded to the 1024-byte swizzle atom.
__host__ __device__ constexpr uint32_t corr_a_bytes(int rb) { return (uint32_t)(BX * BY * rb + 1023) / 1024u * 1024u; }
__host__ __device__ constexpr uint32_t corr_b_bytes(int np, int rb) { return (uint32_t)(np * rb + 1023) / 1024u * 1024u; }

// Displacements k in [K0, K1) of one pixel (k = dy (2R+1) + dx): the epilogue half G of the
// CTA computes K0 = 0 .. KS or KS .. ND, split on a 16-byte boundary of the stored vector.
template <int R, bool F8, int G>
struct Half {
    static constexpr int ND = (2 * R + 1) * (2 * R + 1);
    static constexpr int VEC = F8 ? 16 : 8;
    static constexpr int KS = ND / 2 / VEC * VEC;
    static constexpr int K0 = G == 0 ? 0 : KS, K1 = G == 0 ? KS : ND;
    static constexpr int N = K1 - K0;
    static constexpr int DY0 = K0 / (2 * R + 1), DY1 = N > 0 ? (K1 - 1) / (2 * R + 1) : -1;
    static_assert(N == 0 || (DY0 <= DY1 && DY1 <= 2 * R), "displacement rows of the half");
    // whole-window staging: halo rows 2q + DY0 .. 2q + DY1 + 1 of warp quarter q
    static constexpr int WROWS = N > 0 ? DY1 - DY0 + 2 : 0;
    static constexpr int WLOAD = (WROWS * (BX + 2 * R) + 15) / 16 * 16;
    static_assert(WROWS <= 2 * R + 3, "window rows");
};

// Whole-window staging (the epilogue copies every halo row its half reads, then frees TMEM
// for the next block): slices of the larger of the two halves' windows, pitch as above.
template <int R, bool F8>
struct Whole {
    static constexpr int W0 = Half<R, F8, 0>::WLOAD, W1 = Half<R, F8, 1>::WLOAD;
    static constexpr int SSW0 = W0 > W1 ? W0 : W1;
    static constexpr int SSW = (SSW0 / 4) % 2 ? SSW0 : SSW0 + 4;
    static constexpr size_t SLICES = (size_t)TILE_CORR_EPI * 32 * SSW * 4;
};

// Whole-window staging of half G: the warp's halo rows into the thread's slice (row i of the
// window at slice + i HX), two 16-column loads per wait.
template <int R, bool F8, int G>
__device__ __forceinline__ void corr_stage_window(uint32_t ta, float *slice, int q) {
    using Gm = Geo<R>;
    using H = Half<R, F8, G>;
    static_assert((2 * 3 + H::DY0) * Gm::HX + H::WLOAD <= (int)Gm::TMEM_COLS && H::WLOAD <= Whole<R, F8>::SSW,
                  "window inside TMEM and the slice");
    if constexpr (H::N > 0) {
        const uint32_t col = (uint32_t)((2 * q + H::DY0) * Gm::HX);
#pragma unroll
        for (int c0 = 0; c0 < H::WLOAD; c0 += 32) {
            uint32_t r[32];
#pragma unroll
            for (int k = 0; k < 2; ++k)
                if (c0 + 16 * k < H::WLOAD) tmem_ld16_nowait(ta + col + (uint32_t)(c0 + 16 * k), r + 16 * k);
            tmem_wait_ld();
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (c0 + 4 * k < H::WLOAD)
                    *reinterpret_cast<float4 *>(slice + c0 + 4 * k) = make_float4(
                        __uint_as_float(r[4 * k]), __uint_as_float(r[4 * k + 1]), __uint_as_float(r[4 * k + 2]),
                        __uint_as_float(r[4 * k + 3]));
        }
    }
}

// The half's entries of the pixel from its staged window (after corr_stage_window).  16-bit
// cost volumes where 16-byte stores are allowed go through the warp: every thread packs its
// pixel's entries into its slice, then the warp writes the 32 pixels' rows chunk by chunk, so
// consecutive lanes write consecutive 16-byte chunks of one pixel (the pixels are a whole
// estimator-input row apart) instead of 32 different lines per store; else (and for e4m3)
// each thread stores its own vectors as they are computed.
template <int R, bool F8, int G>
__device__ __forceinline__ void corr_pick_store_window(const CorrTcLaunch &p, float *slice, int py, int px, bool valid,
                                                       size_t pix, float *slices, int sstride, int q, int lane, int bx,
                                                       int by, int z) {
    using H = Half<R, F8, G>;
    constexpr int HX = BX + 2 * R, W = 2 * R + 1, VEC = H::VEC;
    if constexpr (H::N > 0) {
        const int base = (py & 1) * HX + px;
        const bool f16 = p.f16 != 0;
        auto value = [&](int kk) -> float {  // entry kk of the pixel (LeakyReLU of the scaled mean)
            const int dy = kk / W, dx = kk - dy * W;
            const float v = slice[base + (dy - H::DY0) * HX + dx] * p.scale;
            return v >= 0.f ? v : 0.1f * v;
        };
        if constexpr (!F8) {
            if (p.vec_out) {
                constexpr int NV = H::N / 8;  // whole 16-byte chunks of the half
                uint32_t pk[NV * 4];
#pragma unroll
                for (int k = 0; k < NV * 8; k += 2) pk[k / 2] = pack16x2(f16, value(H::K0 + k), value(H::K0 + k + 1));
                uint16_t tail[H::N - NV * 8 > 0 ? H::N - NV * 8 : 1];
#pragma unroll
                for (int k = NV * 8; k < H::N; ++k) tail[k - NV * 8] = (uint16_t)pack16x2(f16, value(H::K0 + k), 0.f);
                __syncwarp();  // every lane has read its window
                uint4 *own = reinterpret_cast<uint4 *>(slice);
#pragma unroll
                for (int j = 0; j < NV; ++j) own[j] = make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
                __syncwarp();
                const int w0 = q * 32;  // first pixel (and slice) of this warp
                for (int j = lane; j < 32 * NV; j += 32) {
                    const int l = j / NV, part = j - l * NV, m = w0 + l;
                    const int yy = by * BY + (m >> 4), xx = bx * BX + (m & 15);
                    if (yy < p.h && xx < p.w) {
                        const size_t pp = ((size_t)z * p.h + yy) * p.w + xx;
                        const uint4 v = reinterpret_cast<const uint4 *>(slices + (size_t)(threadIdx.x - lane + l) * sstride)[part];
                        *reinterpret_cast<uint4 *>(static_cast<uint16_t *>(p.out) + pp * p.out_cs + H::K0 + 8 * part) = v;
                    }
                }
                if (valid) {
                    uint16_t *dst = static_cast<uint16_t *>(p.out) + pix * p.out_cs + H::K0 + NV * 8;
#pragma unroll
                    for (int k = NV * 8; k < H::N; ++k) dst[k - NV * 8] = tail[k - NV * 8];
                }
                return;
            }
        }
        uint8_t *dst8 = static_cast<uint8_t *>(p.out) + pix * p.out_cs * (F8 ? 1 : 2) + (size_t)H::K0 * (F8 ? 1 : 2);
#pragma unroll
        for (int k0 = H::K0; k0 < H::K1; k0 += VEC) {
            if (k0 + VEC <= H::K1 && p.vec_out) {
                float v[VEC];
#pragma unroll
                for (int j = 0; j < VEC; ++j) v[j] = value(k0 + j);
                uint4 o;
                if constexpr (F8) {
                    o.x = pack_e4m3x4(v[0] * p.q_out, v[1] * p.q_out, v[2] * p.q_out, v[3] * p.q_out);
                    o.y = pack_e4m3x4(v[4] * p.q_out, v[5] * p.q_out, v[6] * p.q_out, v[7] * p.q_out);
                    o.z = pack_e4m3x4(v[8] * p.q_out, v[9] * p.q_out, v[10] * p.q_out, v[11] * p.q_out);
                    o.w = pack_e4m3x4(v[12] * p.q_out, v[13] * p.q_out, v[14] * p.q_out, v[15] * p.q_out);
                } else {
                    o.x = pack16x2(f16, v[0], v[1]);
                    o.y = pack16x2(f16, v[2], v[3]);
                    o.z = pack16x2(f16, v[4], v[5]);
                    o.w = pack16x2(f16, v[6], v[7]);
                }
                if (valid) *reinterpret_cast<uint4 *>(dst8 + (size_t)(k0 - H::K0) * (F8 ? 1 : 2)) = o;
            } else if (valid) {
#pragma unroll
                for (int j = 0; j < VEC; ++j)
                    if (k0 + j < H::K1) {
                        const float v = value(k0 + j);
                        if constexpr (F8)
                            dst8[k0 + j - H::K0] = (uint8_t)__nv_cvt_float_to_fp8(v * p.q_out, __NV_SATFINITE, __NV_E4M3);
                        else
                            reinterpret_cast<uint16_t *>(dst8)[k0 + j - H::K0] = (uint16_t)pack16x2(f16, v, 0.f);
                    }
            }
        }
    }
}

// Store of half G's entries (scaled, LeakyReLU) of pixel pix: 16-byte vectors where the
// buffer allows, in the features' type.
template <int R, bool F8, int G>
__device__ __forceinline__ void corr_store_half(const CorrTcLaunch &p,
                                                const float (&res)[Half<R, F8, G>::N > 0 ? Half<R, F8, G>::N : 1],
                                                size_t pix) {
    using H = Half<R, F8, G>;
    if constexpr (H::N > 0) {
        if constexpr (F8) {
            uint8_t *dst = static_cast<uint8_t *>(p.out) + pix * p.out_cs + H::K0;
            if (p.vec_out) {
#pragma unroll
                for (int k = 0; k + 16 <= H::N; k += 16) {
                    uint4 v;
                    v.x = pack_e4m3x4(res[k] * p.q_out, res[k + 1] * p.q_out, res[k + 2] * p.q_out, res[k + 3] * p.q_out);
                    v.y = pack_e4m3x4(res[k + 4] * p.q_out, res[k + 5] * p.q_out, res[k + 6] * p.q_out, res[k + 7] * p.q_out);
                    v.z = pack_e4m3x4(res[k + 8] * p.q_out, res[k + 9] * p.q_out, res[k + 10] * p.q_out, res[k + 11] * p.q_out);
                    v.w = pack_e4m3x4(res[k + 12] * p.q_out, res[k + 13] * p.q_out, res[k + 14] * p.q_out, res[k + 15] * p.q_out);
                    *reinterpret_cast<uint4 *>(dst + k) = v;
                }
#pragma unroll
                for (int k = H::N / 16 * 16; k < H::N; ++k)
                    dst[k] = (uint8_t)__nv_cvt_float_to_fp8(res[k] * p.q_out, __NV_SATFINITE, __NV_E4M3);
            } else {
#pragma unroll
                for (int k = 0; k < H::N; ++k)
                    dst[k] = (uint8_t)__nv_cvt_float_to_fp8(res[k] * p.q_out, __NV_SATFINITE, __NV_E4M3);
            }
        } else {
            uint16_t *dst = static_cast<uint16_t *>(p.out) + pix * p.out_cs + H::K0;  // bf16 or half
            const bool f16 = p.f16 != 0;
            if (p.vec_out) {
#pragma unroll
                for (int k = 0; k + 8 <= H::N; k += 8) {
                    uint4 v;
                    v.x = pack16x2(f16, res[k], res[k + 1]);
                    v.y = pack16x2(f16, res[k + 2], res[k + 3]);
                    v.z = pack16x2(f16, res[k + 4], res[k + 5]);
                    v.w = pack16x2(f16, res[k + 6], res[k + 7]);
                    *reinterpret_cast<uint4 *>(dst + k) = v;
                }
#pragma unroll
                for (int k = H::N / 8 * 8; k < H::N; ++k) dst[k] = (uint16_t)pack16x2(f16, res[k], 0.f);
            } else {
#pragma unroll
                for (int k = 0; k < H::N; ++k) dst[k] = (uint16_t)pack16x2(f16, res[k], 0.f);
            }
        }
    }
}

// One epilogue half: for displacement rows DY0 .. DY1, load the warp's two halo rows from
// TMEM, stage the thread's own values in its slice, pick the pixel's 2R+1 entries, then scale,
// LeakyReLU and store the half's (k0 .. k1) cost-volume entries of the pixel.
template <int R, bool F8, int G>
__device__ __forceinline__ void corr_epilogue_half(const CorrTcLaunch &p, uint32_t ta, float *slice, int py, int px,
                                                   int q, bool valid, size_t pix) {
    using Gm = Geo<R>;
    using H = Half<R, F8, G>;
    if constexpr (H::N > 0) {
        float res[H::N > 0 ? H::N : 1];
        const int base = (py & 1) * Gm::HX + px;
#pragma unroll
        for (int dy = H::DY0; dy <= H::DY1; ++dy) {
            uint32_t r[Gm::WIN];
            const uint32_t col = (uint32_t)((2 * q + dy) * Gm::HX);
#pragma unroll
            for (int k = 0; k < Gm::WIN / 16; ++k) tmem_ld16_nowait(ta + col + (uint32_t)(16 * k), r + 16 * k);
            tmem_wait_ld();
#pragma unroll
            for (int k = 0; k < Gm::WIN / 4; ++k)
                *reinterpret_cast<float4 *>(slice + 4 * k) = make_float4(
                    __uint_as_float(r[4 * k]), __uint_as_float(r[4 * k + 1]), __uint_as_float(r[4 * k + 2]),
                    __uint_as_float(r[4 * k + 3]));
#pragma unroll
            for (int dx = 0; dx <= 2 * R; ++dx) {
                const int kk = dy * (2 * R + 1) + dx;
                if (kk >= H::K0 && kk < H::K1) {
                    const float v = slice[base + dx] * p.scale;
                    res[kk - H::K0] = v >= 0.f ? v : 0.1f * v;
                }
            }
        }
        if (valid) corr_store_half<R, F8, G>(p, res, pix);
    }
}

// Persistent correlation: one CTA per SM walks the blocks blockIdx.x, blockIdx.x + gridDim.x,
// ...; the operands of the next block load while the current one is in TMEM.
//   * warp 8, lane 0 (producer): per block, the self block and the other map's halo of every
//     channel step into an operand stage (NS stages, one barrier each);
//   * warp 9, lane 0 (MMA issuer): per block, after the epilogue has released TMEM, the MMAs
//     of both N halves over the channel steps; the commit frees the operand stage and hands
//     TMEM to the epilogue;
//   * warps 0-7 (epilogue): warp w reads TMEM lanes 32 (w % 4) .. (pixel rows 2 (w % 4) and
//     2 (w % 4) + 1 of the block) and computes half of each pixel's displacements (w / 4
//     selects the half): per displacement row it loads the two halo rows its pixels read,
//     stages its own values in a per-thread slice and picks each pixel's 2R+1 entries.  Each
//     half also copies half of the pixel's self features into the estimator input.
template <int R, bool F8, bool WHOLE>
__global__ void __launch_bounds__(32 * (TILE_CORR_EPI + 2), 1)
corr_tc_kernel(const __grid_constant__ CUtensorMap tmS, const __grid_constant__ CUtensorMap tmO,
               const __grid_constant__ CUtensorMap tmC, const CorrTcLaunch p) {
    using G = Geo<R>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t abytes = corr_a_bytes(p.rb), bbytes = corr_b_bytes(G::NP, p.rb);
    const uint32_t stage = (uint32_t)p.nch * (abytes + bbytes);
    const int NS = p.nstages;
    float *slices = reinterpret_cast<float *>(smem + (size_t)NS * stage);
    uint64_t *bars = reinterpret_cast<uint64_t *>(reinterpret_cast<uint8_t *>(slices) +
                                                  (WHOLE ? Whole<R, F8>::SLICES : G::SLICES));
    const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * NS;
    const uint32_t tfull = empty0 + 8 * NS, tempty = tfull + 8, done = tempty + 8;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * NS + 3);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nbx = (p.w + BX - 1) / BX, nby = (p.h + BY - 1) / BY;
    const int nblocks = nbx * nby * p.nb;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, p.tma_self ? 2 : 1);  // the MMAs, and the self store's reads
        }
        mbar_init(tfull, 1);
        mbar_init(tempty, TILE_CORR_EPI);
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(G::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    if (p.trigger) pdl_trigger();

    // images of block entry z in the self and other tensor maps
    auto images = [&](int z, int &img_self, int &img_other) {
        const int pq = z >> 1, pd = z & 1;
        img_self = p.pair_lanes ? p.s0 + pq + pd * p.pair_lanes : (z ? p.img_s[1] : p.img_s[0]);
        img_other = p.pair_lanes ? p.o0 + pq * p.oq + pd * p.od : (z ? p.img_o[1] : p.img_o[0]);
    };

    if (warp == TILE_CORR_EPI && lane == 0) {
        // ---- producer
        pdl_wait();  // the features follow the previous kernel
        uint32_t s = 0, ph = 0, issued = 0;
        bool fine = true;
        for (int t = blockIdx.x; t < nblocks && fine; t += gridDim.x) {
            const int bx = t % nbx, by = (t / nbx) % nby, z = t / (nbx * nby);
            int is, io;
            images(z, is, io);
            if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, p.err, ERR_CORR_PRODUCER)) {
                fine = false;
                break;
            }
            const uint32_t fb = full0 + 8 * s;
            mbar_expect_tx(fb, (uint32_t)p.nch * (uint32_t)(BX * BY + G::NPOS) * (uint32_t)p.rb);
            const uint32_t dst = smem_u32(smem + s * stage);
            for (int ch = 0; ch < p.nch; ++ch) {
                const int c0 = ch * (F8 ? p.rb : p.rb / 2);  // a step: rb bytes of e4m3 or 16-bit channels
                const uint32_t d = dst + (uint32_t)ch * (abytes + bbytes);
                tma_load_4d(&tmS, fb, d, c0, bx * BX, by * BY, is);
                tma_load_4d(&tmO, fb, d + abytes, c0, bx * BX - R, by * BY - R, io);
            }
            ++issued;
            if (++s == (uint32_t)NS) { s = 0; ph ^= 1u; }
        }
        if (!fine) {
            // Error path: let the loads already issued land before the CTA exits.
            const unsigned long long t0 = global_ns();
            for (uint32_t u = issued > (uint32_t)NS ? issued - NS : 0; u < issued; ++u)
                while (!mbar_try(full0 + 8 * (u % NS), (u / NS) & 1u))
                    if (global_ns() - t0 > WAIT_NS) { atomicCAS(p.err, 0, ERR_CORR_DRAIN); break; }
        }
    } else if (warp == TILE_CORR_EPI + 1 && lane == 0) {
        // ---- MMA issuer: D[:, 0:NH] and D[:, NH:NP] per block
        const uint32_t idesc = F8 ? idesc_e4m3(128, G::NH) : (p.f16 ? idesc_f16(128, G::NH) : idesc_bf16(128, G::NH));
        const uint32_t rb = (uint32_t)p.rb;
        uint32_t s = 0, ph = 0;
        int k = 0;
        if (p.tma_self) pdl_wait();  // the self store writes the estimator input
        for (int t = blockIdx.x; t < nblocks; t += gridDim.x, ++k) {
            if (k >= 1 && !mbar_wait(tempty, (uint32_t)(k - 1) & 1u, p.err, ERR_CORR_MMA)) break;
            if (!mbar_wait(full0 + 8 * s, ph, p.err, ERR_CORR_MMA)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t base = smem_u32(smem + s * stage);
            if (p.tma_self) {
                // the block's self features, already in the stage, into the estimator input
                const int bx = t % nbx, by = (t / nbx) % nby, z = t / (nbx * nby);
                for (int ch = 0; ch < p.nch; ++ch)
                    tma_store_4d(&tmC, base + (uint32_t)ch * (abytes + bbytes), ch * (F8 ? p.rb : p.rb / 2), bx * BX,
                                 by * BY, z);
                tma_store_commit();
            }
            for (int ch = 0; ch < p.nch; ++ch) {
                const uint32_t a = base + (uint32_t)ch * (abytes + bbytes);
                const uint64_t da = sw_desc(a, rb), db0 = sw_desc(a + abytes, rb);
                const uint64_t db1 = sw_desc(a + abytes + (uint32_t)G::NH * rb, rb);
                for (int kk = 0; kk < p.rb / 32; ++kk) {  // 32 bytes of K per MMA
                    const uint32_t acc = (ch | kk) != 0 ? 1u : 0u;
                    umma<F8>(tmem, da + (uint64_t)(kk * 2), db0 + (uint64_t)(kk * 2), idesc, acc);
                    umma<F8>(tmem + (uint32_t)G::NH, da + (uint64_t)(kk * 2), db1 + (uint64_t)(kk * 2), idesc, acc);
                }
            }
            umma_commit(empty0 + 8 * s);  // the operand stage is read
            umma_commit(tfull);           // the block is in TMEM
            if (p.tma_self) {
                tma_store_wait_read();  // the self store has read the stage as well
                mbar_arrive(empty0 + 8 * s);
            }
            if (++s == (uint32_t)NS) { s = 0; ph ^= 1u; }
        }
        if (p.tma_self) tma_store_wait_all();
        umma_commit(done);  // every MMA issued above has completed once it fires
        const unsigned long long t0 = global_ns();
        while (!mbar_try(done, 0))
            if (global_ns() - t0 > WAIT_NS) { atomicCAS(p.err, 0, ERR_CORR_DRAIN); break; }
    } else if (warp < TILE_CORR_EPI) {
        // ---- epilogue
        pdl_wait();  // the outputs may still be read by the previous kernel
        const int q = warp & 3, half = warp >> 2;
        const int m = q * 32 + lane, py = m >> 4, px = m & 15;
        float *slice = slices + (size_t)threadIdx.x * (WHOLE ? Whole<R, F8>::SSW : G::SSTRIDE);
        const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16);
        const size_t esz = F8 ? 1 : 2;
        const int nq = p.self_copy && !p.tma_self ? (int)(p.c * esz / 16) : 0;  // 16-byte units of a pixel's self features
        const int q0 = half ? nq / 2 : 0, q1 = half ? nq : nq / 2;  // this half's share of them
        int k = 0;
        for (int t = blockIdx.x; t < nblocks; t += gridDim.x, ++k) {
            const int bx = t % nbx, by = (t / nbx) % nby, z = t / (nbx * nby);
            const int y = by * BY + py, x = bx * BX + px;
            const bool valid = y < p.h && x < p.w;
            const size_t pix = ((size_t)z * p.h + y) * p.w + x;
            // the pixel's self features, copied into the estimator input below
            const uint4 *src = nullptr;
            if (valid && nq > 0) {
                const int pq = z >> 1, pd = z & 1;
                const uint8_t *fsb = p.pair_lanes ? static_cast<const uint8_t *>(p.fs[0]) +
                                                        (size_t)(pq + pd * p.pair_lanes) * p.fs_img_bytes
                                                  : static_cast<const uint8_t *>(z ? p.fs[1] : p.fs[0]);
                src = reinterpret_cast<const uint4 *>(fsb + ((size_t)y * p.w + x) * p.c * esz);
            }
            // up to four 16-byte units of them in flight under the MMAs and the staging
            uint4 sf[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (src && q0 + i < q1) sf[i] = __ldg(src + q0 + i);
            int ok = 1;
            if (lane == 0) ok = mbar_wait(tfull, (uint32_t)k & 1u, p.err, ERR_CORR_EPILOGUE);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if constexpr (WHOLE) {
                // copy the window out of TMEM, hand TMEM to the next block's MMAs, then pick
                if (half == 0) corr_stage_window<R, F8, 0>(ta, slice, q);
                else corr_stage_window<R, F8, 1>(ta, slice, q);
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(tempty);
                if (half == 0)
                    corr_pick_store_window<R, F8, 0>(p, slice, py, px, valid, pix, slices, Whole<R, F8>::SSW, q, lane, bx,
                                                     by, z);
                else
                    corr_pick_store_window<R, F8, 1>(p, slice, py, px, valid, pix, slices, Whole<R, F8>::SSW, q, lane, bx,
                                                     by, z);
            } else if (half == 0) {
                corr_epilogue_half<R, F8, 0>(p, ta, slice, py, px, q, valid, pix);
            } else {
                corr_epilogue_half<R, F8, 1>(p, ta, slice, py, px, q, valid, pix);
            }
            if (src) {
                uint4 *cp = reinterpret_cast<uint4 *>(static_cast<uint8_t *>(p.self_copy) + pix * p.out_cs * esz);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (q0 + i < q1) cp[q0 + i] = sf[i];
                for (int qq = q0 + 4; qq < q1; ++qq) cp[qq] = __ldg(src + qq);
            }
            if constexpr (!WHOLE) {
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(tempty);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G::TMEM_COLS) : "memory");
    }
}

bool encode_features(CUtensorMap *map, const void *base, int n, int cs, int h, int w, int c, int box_x, int box_y,
                     bool f8, int rb, bool f16) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t es = f8 ? 1 : 2;
    const cuuint64_t dims[4] = {(cuuint64_t)c, (cuuint64_t)w, (cuuint64_t)h, (cuuint64_t)n};
    const cuuint64_t strides[3] = {(cuuint64_t)cs * es, (cuuint64_t)w * cs * es, (cuuint64_t)h * w * cs * es};
    const cuuint32_t box[4] = {(cuuint32_t)(rb / es), (cuuint32_t)box_x, (cuuint32_t)box_y, 1};
    const cuuint32_t ones[4] = {1, 1, 1, 1};
    const CUtensorMapDataType dt = f8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                      : (f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
    return enc(map, dt, 4, const_cast<void *>(base), dims, strides, box, ones,
               CU_TENSOR_MAP_INTERLEAVE_NONE, rb == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int corr_sm_count() {
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

template <int R, bool F8, bool WHOLE>
cudaError_t launch_rw(const CorrTcPlan &plan, const CorrTcLaunch &lp, const CUtensorMap &tmC, int grid, size_t smem,
                      cudaStream_t st) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e =
            cudaFuncSetAttribute(corr_tc_kernel<R, F8, WHOLE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    return launch_pdl(corr_tc_kernel<R, F8, WHOLE>, dim3(grid), dim3(32 * (TILE_CORR_EPI + 2)), smem, st, plan.tmS,
                      plan.tmO, tmC, lp);
}

// Whole-window staging where its slices fit beside one operand stage (the narrow levels),
// else staging per displacement row; as many operand stages as fit, up to four.
template <int R, bool F8>
cudaError_t launch_r(const CorrTcPlan &plan, const CorrTcLaunch &lp0, int nb, cudaStream_t st) {
    using G = Geo<R>;
    CorrTcLaunch lp = lp0;
    lp.nb = nb;
    const size_t budget = 232448 - 1024 - 256;
    const size_t stage = (size_t)plan.nch * (corr_a_bytes(plan.rb) + corr_b_bytes(G::NP, plan.rb));
    const bool whole = stage + Whole<R, F8>::SLICES <= budget;
    const size_t slices = whole ? Whole<R, F8>::SLICES : G::SLICES;
    int ns = stage + slices <= budget ? (int)((budget - slices) / stage) : 0;
    if (ns > 4) ns = 4;
    if (ns < 1) return cudaErrorInvalidConfiguration;
    lp.nstages = ns;
    const long nblocks = (long)((plan.w + BX - 1) / BX) * ((plan.h + BY - 1) / BY) * nb;
    const int nsm = corr_sm_count();
    const int grid = nblocks < nsm ? (int)nblocks : nsm;
    // a launch alone on the GPU whose CTAs leave half of the SMs free lets the next kernel
    // set up on them while it runs (as the convolutions do; every CTA holds its TMEM first)
    lp.trigger = lp.trigger && 2 * grid <= nsm ? 1 : 0;
    const size_t smem = 1024 + (size_t)ns * stage + slices + 256;
    // the self copy as a TMA store of each block's self operand: a map over the destination
    // (channels [0, c) of nb images at pixel stride out_cs), boxed and swizzled like the self
    // map; the per-thread copy where the encoding fails
    CUtensorMap tmC = plan.tmS;
    lp.tma_self = 0;
    if (lp.self_copy && encode_features(&tmC, lp.self_copy, nb, lp.out_cs, plan.h, plan.w, plan.c, BX, BY, plan.f8,
                                        plan.rb, plan.f16))
        lp.tma_self = 1;
    return whole ? launch_rw<R, F8, true>(plan, lp, tmC, grid, smem, st)
                 : launch_rw<R, F8, false>(plan, lp, tmC, grid, smem, st);
}

}  // namespace

bool tc_plan_corr(CorrTcPlan &plan, const void *self, int n_self, int self_cs, const void *other, int n_other,
                  int other_cs, int h, int w, int c, int r, int *err, std::string &why, bool f8, bool f16) {
    plan.enabled = false;
    if (f8) f16 = false;
    const int al = f8 ? 16 : 8;  // 16-byte strides
    if (c % al != 0 || c < al || c > BK * MAX_NCH) { why = "channels must be a multiple of 16 bytes, up to 128"; return false; }
    if (r < 1 || r > 4) { why = "radius must be 1..4"; return false; }
    if (self_cs % al != 0 || other_cs % al != 0) { why = "pixel strides must be multiples of 16 bytes"; return false; }
    if (reinterpret_cast<uintptr_t>(self) % 16 || reinterpret_cast<uintptr_t>(other) % 16) { why = "misaligned"; return false; }
    // BF16 features of at most 32 channels: 64-byte steps, so no step multiplies zero padding
    const int rb = !f8 && c <= 32 ? 64 : 128;
    if (!encode_features(&plan.tmS, self, n_self, self_cs, h, w, c, BX, BY, f8, rb, f16) ||
        !encode_features(&plan.tmO, other, n_other, other_cs, h, w, c, BX + 2 * r, BY + 2 * r, f8, rb, f16)) {
        why = "tensor map encoding failed";
        return false;
    }
    plan.h = h;
    plan.w = w;
    plan.c = c;
    plan.r = r;
    plan.rb = rb;
    plan.nch = f8 ? 1 : (c + rb / 2 - 1) / (rb / 2);
    plan.f8 = f8;
    plan.f16 = f16;
    plan.err = err;
    plan.enabled = true;
    return true;
}

static cudaError_t launch_plan(const CorrTcPlan &plan, const CorrTcLaunch &lp, int nb, cudaStream_t st) {
    if (plan.f8) {
        switch (plan.r) {
            case 1: return launch_r<1, true>(plan, lp, nb, st);
            case 2: return launch_r<2, true>(plan, lp, nb, st);
            case 3: return launch_r<3, true>(plan, lp, nb, st);
            case 4: return launch_r<4, true>(plan, lp, nb, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (plan.r) {
        case 1: return launch_r<1, false>(plan, lp, nb, st);
        case 2: return launch_r<2, false>(plan, lp, nb, st);
        case 3: return launch_r<3, false>(plan, lp, nb, st);
        case 4: return launch_r<4, false>(plan, lp, nb, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_corr_tc_pairs(const CorrTcPlan &plan, int lanes, int pair_lanes, int s0, int o0, int oq, int od,
                                 void *out, int out_cs, const void *fs0, size_t fs_img_bytes, void *self_copy,
                                 cudaStream_t st) {
    if (!plan.enabled || plan.f8 || lanes < 1 || pair_lanes < 1 || 2 * lanes > 65535) return cudaErrorInvalidValue;
    const int esz = 2;
    if (self_copy && ((out_cs * esz) % 16 != 0 || reinterpret_cast<uintptr_t>(self_copy) % 16 != 0 || !fs0 ||
                      reinterpret_cast<uintptr_t>(fs0) % 16 != 0 || fs_img_bytes % 16 != 0))
        return cudaErrorInvalidValue;
    CorrTcLaunch lp{};
    lp.h = plan.h;
    lp.w = plan.w;
    lp.nch = plan.nch;
    lp.rb = plan.rb;
    lp.out = out;
    lp.out_cs = out_cs;
    lp.vec_out = ((out_cs * esz) % 16 == 0 && reinterpret_cast<uintptr_t>(out) % 16 == 0) ? 1 : 0;
    lp.c = plan.c;
    lp.fs[0] = lp.fs[1] = fs0;
    lp.self_copy = self_copy;
    lp.scale = 1.f / (float)plan.c;
    lp.q_out = 1.f;
    lp.err = plan.err;
    lp.f16 = plan.f16 ? 1 : 0;
    lp.pair_lanes = pair_lanes;
    lp.s0 = s0;
    lp.o0 = o0;
    lp.oq = oq;
    lp.od = od;
    lp.fs_img_bytes = fs_img_bytes;
    return launch_plan(plan, lp, 2 * lanes, st);
}

cudaError_t launch_corr_tc(const CorrTcPlan &plan, int nb, const int img_self[2], const int img_other[2], void *out,
                           int out_cs, const void *const fs[2], void *self_copy, cudaStream_t st, float feat_scale,
                           float q_out, bool alone) {
    if (!plan.enabled || nb < 1 || nb > 2) return cudaErrorInvalidValue;
    const int esz = plan.f8 ? 1 : 2;
    if (self_copy && ((out_cs * esz) % 16 != 0 || reinterpret_cast<uintptr_t>(self_copy) % 16 != 0 || !fs ||
                      reinterpret_cast<uintptr_t>(fs[0]) % 16 || reinterpret_cast<uintptr_t>(fs[nb - 1]) % 16))
        return cudaErrorInvalidValue;
    CorrTcLaunch lp{};
    lp.h = plan.h;
    lp.w = plan.w;
    lp.nch = plan.nch;
    lp.rb = plan.rb;
    for (int b = 0; b < 2; ++b) {
        lp.img_s[b] = img_self[b < nb ? b : 0];
        lp.img_o[b] = img_other[b < nb ? b : 0];
        lp.fs[b] = fs ? fs[b < nb ? b : 0] : nullptr;
    }
    lp.out = out;
    lp.out_cs = out_cs;
    lp.vec_out = ((out_cs * esz) % 16 == 0 && reinterpret_cast<uintptr_t>(out) % 16 == 0) ? 1 : 0;
    lp.c = plan.c;
    lp.self_copy = self_copy;
    lp.trigger = alone ? 1 : 0;
    lp.scale = feat_scale * feat_scale / (float)plan.c;
    lp.q_out = q_out;
    lp.err = plan.err;
    lp.f16 = plan.f16 ? 1 : 0;
    return launch_plan(plan, lp, nb, st);
}

}  // namespace tc
