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
constexpr uint32_t A_BYTES = BX * BY * BK * 2;


enum : int { ERR_CORR_MMA = 5, ERR_CORR_EPILOGUE = 6, ERR_CORR_DRAIN = 7 };

template <int R>
struct Geo {
    static constexpr int HX = BX + 2 * R, HY = BY + 2 * R, NPOS = HX * HY;
    static constexpr int NP = (NPOS + 31) / 32 * 32, NH = NP / 2;
    static constexpr uint32_t B_BYTES = (uint32_t)NP * BK * 2;
    static constexpr int ND = (2 * R + 1) * (2 * R + 1);
    static constexpr uint32_t TMEM_COLS = NP <= 256 ? 256 : 512;
    // epilogue: every thread stages the WROWS halo rows its warp reads (2 pixel rows + 2R)
    static constexpr int WROWS = 2 + 2 * R, WCOLS = WROWS * HX;         // 240 for R = 4
    static constexpr int WLOAD = (WCOLS + 15) / 16 * 16;                // tcgen05.ld x16 granularity
    // slice pitch: a whole number of 16-byte units, odd, so the 16-byte stores of 8
    // consecutive threads hit distinct banks
    static constexpr int SSTRIDE = (WLOAD / 4) % 2 ? WLOAD : WLOAD + 4;
    static constexpr size_t OPERANDS = (size_t)MAX_NCH * (A_BYTES + B_BYTES);
    static constexpr size_t SLICES = (size_t)128 * SSTRIDE * 4;
    static constexpr size_t SMEM = (OPERANDS > SLICES ? OPERANDS : SLICES) + 1024 + 256;
    static_assert(NH % 16 == 0 && NH <= 256, "MMA N");
    static_assert(2 * (BY / 2 - 1) * HX + WLOAD <= (int)TMEM_COLS, "epilogue column window inside TMEM");
};

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
};

template <int R, bool F8>
__global__ void __launch_bounds__(128, 1)
corr_tc_kernel(const __grid_constant__ CUtensorMap tmS, const __grid_constant__ CUtensorMap tmO, const CorrTcLaunch p) {
    using G = Geo<R>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;
    uint8_t *sB = smem + MAX_NCH * A_BYTES;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + MAX_NCH * (A_BYTES + G::B_BYTES));
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + MAX_NCH + 1);
    const uint32_t full0 = smem_u32(bars), accum = smem_u32(bars + MAX_NCH);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.z, x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    // images of this entry in the self and other tensor maps (selects, not a runtime index
    // into the argument arrays)
    const int pq = b >> 1, pd = b & 1;
    const int img_self = p.pair_lanes ? p.s0 + pq + pd * p.pair_lanes : (b ? p.img_s[1] : p.img_s[0]);
    const int img_other = p.pair_lanes ? p.o0 + pq * p.oq + pd * p.od : (b ? p.img_o[1] : p.img_o[0]);

    if (threadIdx.x == 0) {
        for (int ch = 0; ch < MAX_NCH; ++ch) mbar_init(full0 + 8 * ch, 1);
        mbar_init(accum, 1);
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
    pdl_wait();  // every global access below follows the previous kernel

    if (threadIdx.x == 0) {
        // ---- producer: every channel step at once (the whole block fits in shared memory)
        for (int ch = 0; ch < p.nch; ++ch) {
            const uint32_t fb = full0 + 8 * ch;
            mbar_expect_tx(fb, (uint32_t)(BX * BY + G::NPOS) * (uint32_t)p.rb);
            const int c0 = ch * (F8 ? p.rb : p.rb / 2);  // a step: rb bytes of e4m3 or bf16 channels
            tma_load_4d(&tmS, fb, smem_u32(sA + ch * A_BYTES), c0, x0, y0, img_self);
            tma_load_4d(&tmO, fb, smem_u32(sB + ch * G::B_BYTES), c0, x0 - R, y0 - R, img_other);
        }
    } else if (threadIdx.x == 32) {
        // ---- MMA issuer: D[:, 0:NH] and D[:, NH:NP]
        const uint32_t idesc = F8 ? idesc_e4m3(128, G::NH) : (p.f16 ? idesc_f16(128, G::NH) : idesc_bf16(128, G::NH));
        bool ok = true;
        for (int ch = 0; ch < p.nch && ok; ++ch) {
            if (!mbar_wait(full0 + 8 * ch, 0, p.err, ERR_CORR_MMA)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t rb = (uint32_t)p.rb;
            const uint64_t da = sw_desc(smem_u32(sA + ch * A_BYTES), rb);
            const uint64_t db0 = sw_desc(smem_u32(sB + ch * G::B_BYTES), rb);
            const uint64_t db1 = sw_desc(smem_u32(sB + ch * G::B_BYTES + (uint32_t)G::NH * rb), rb);
#pragma unroll
            for (int kk = 0; kk < p.rb / 32; ++kk) {  // 32 bytes of K per MMA
                const uint32_t acc = (ch | kk) != 0 ? 1u : 0u;
                umma<F8>(tmem, da + (uint64_t)(kk * 2), db0 + (uint64_t)(kk * 2), idesc, acc);
                umma<F8>(tmem + (uint32_t)G::NH, da + (uint64_t)(kk * 2), db1 + (uint64_t)(kk * 2), idesc, acc);
            }
        }
        umma_commit(accum);
        if (!ok) {
            // Error path: let every issued load land before the CTA exits.
            for (int ch = 0; ch < p.nch; ++ch) {
                const unsigned long long t0 = global_ns();
                while (!mbar_try(full0 + 8 * ch, 0))
                    if (global_ns() - t0 > WAIT_NS) {
                        atomicCAS(p.err, 0, ERR_CORR_DRAIN);
                        break;
                    }
            }
        }
    }

    int ok = 1;
    if (lane == 0) ok = mbar_wait(accum, 0, p.err, ERR_CORR_EPILOGUE) && *(volatile int *)p.err == 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        // The MMAs have completed, so the operand buffers are free: reuse them as per-thread
        // slices.  Warp w's pixel rows 2w, 2w + 1 read halo rows 2w .. 2w + 2R + 1: those
        // WCOLS contiguous TMEM columns are staged once, then each pixel picks its (2R+1)^2
        // entries (row dy + (py & 1), columns px + dx of the staged window).
        float *slice = reinterpret_cast<float *>(smem) + threadIdx.x * G::SSTRIDE;
        const int py = threadIdx.x >> 4, px = threadIdx.x & 15;
        const int y = y0 + py, x = x0 + px;
        const bool valid = y < p.h && x < p.w;
        const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(2 * warp * G::HX);
        // up to four 16-column loads in flight per wait; 16-byte shared stores
#pragma unroll
        for (int c0 = 0; c0 < G::WLOAD; c0 += 64) {
            constexpr int MAXK = 4;
            uint32_t r[16 * MAXK];
#pragma unroll
            for (int k = 0; k < MAXK; ++k)
                if (c0 + 16 * k < G::WLOAD) tmem_ld16_nowait(ta + (uint32_t)(c0 + 16 * k), r + 16 * k);
            tmem_wait_ld();
#pragma unroll
            for (int k = 0; k < MAXK; ++k)
                if (c0 + 16 * k < G::WLOAD) {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        *reinterpret_cast<float4 *>(slice + c0 + 16 * k + 4 * q) =
                            make_float4(__uint_as_float(r[16 * k + 4 * q]), __uint_as_float(r[16 * k + 4 * q + 1]),
                                        __uint_as_float(r[16 * k + 4 * q + 2]), __uint_as_float(r[16 * k + 4 * q + 3]));
                }
        }
        const int base = (py & 1) * G::HX + px;
        float res[G::ND];
#pragma unroll
        for (int j = 0; j <= 2 * R; ++j) {
#pragma unroll
            for (int i = 0; i <= 2 * R; ++i) {
                const float v = slice[base + j * G::HX + i] * p.scale;
                res[j * (2 * R + 1) + i] = v >= 0.f ? v : 0.1f * v;
            }
        }
        if (valid) {
            const size_t pix = ((size_t)b * p.h + y) * p.w + x;
            if (F8) {
                uint8_t *dst = static_cast<uint8_t *>(p.out) + pix * p.out_cs;
                if (p.vec_out) {
#pragma unroll
                    for (int k = 0; k + 16 <= G::ND; k += 16) {
                        uint4 v;
                        v.x = pack_e4m3x4(res[k] * p.q_out, res[k + 1] * p.q_out, res[k + 2] * p.q_out, res[k + 3] * p.q_out);
                        v.y = pack_e4m3x4(res[k + 4] * p.q_out, res[k + 5] * p.q_out, res[k + 6] * p.q_out, res[k + 7] * p.q_out);
                        v.z = pack_e4m3x4(res[k + 8] * p.q_out, res[k + 9] * p.q_out, res[k + 10] * p.q_out, res[k + 11] * p.q_out);
                        v.w = pack_e4m3x4(res[k + 12] * p.q_out, res[k + 13] * p.q_out, res[k + 14] * p.q_out, res[k + 15] * p.q_out);
                        *reinterpret_cast<uint4 *>(dst + k) = v;
                    }
#pragma unroll
                    for (int k = G::ND / 16 * 16; k < G::ND; ++k)
                        dst[k] = (uint8_t)__nv_cvt_float_to_fp8(res[k] * p.q_out, __NV_SATFINITE, __NV_E4M3);
                } else {
#pragma unroll
                    for (int k = 0; k < G::ND; ++k)
                        dst[k] = (uint8_t)__nv_cvt_float_to_fp8(res[k] * p.q_out, __NV_SATFINITE, __NV_E4M3);
                }
            } else {
                uint16_t *dst = static_cast<uint16_t *>(p.out) + pix * p.out_cs;  // bf16 or half
                const bool f16 = p.f16 != 0;
                if (p.vec_out) {
#pragma unroll
                    for (int k = 0; k + 8 <= G::ND; k += 8) {
                        uint4 v;
                        v.x = pack16x2(f16, res[k], res[k + 1]);
                        v.y = pack16x2(f16, res[k + 2], res[k + 3]);
                        v.z = pack16x2(f16, res[k + 4], res[k + 5]);
                        v.w = pack16x2(f16, res[k + 6], res[k + 7]);
                        *reinterpret_cast<uint4 *>(dst + k) = v;
                    }
#pragma unroll
                    for (int k = G::ND / 8 * 8; k < G::ND; ++k) dst[k] = (uint16_t)pack16x2(f16, res[k], 0.f);
                } else {
#pragma unroll
                    for (int k = 0; k < G::ND; ++k) dst[k] = (uint16_t)pack16x2(f16, res[k], 0.f);
                }
            }
            if (p.self_copy) {
                const size_t esz = F8 ? 1 : 2;
                const uint8_t *fsb = p.pair_lanes ? static_cast<const uint8_t *>(p.fs[0]) +
                                                        (size_t)(pq + pd * p.pair_lanes) * p.fs_img_bytes
                                                  : static_cast<const uint8_t *>(b ? p.fs[1] : p.fs[0]);
                const uint4 *src = reinterpret_cast<const uint4 *>(fsb + ((size_t)y * p.w + x) * p.c * esz);
                uint4 *cp = reinterpret_cast<uint4 *>(static_cast<uint8_t *>(p.self_copy) + pix * p.out_cs * esz);
                for (int q = 0; q < (int)(p.c * esz / 16); ++q) cp[q] = __ldg(src + q);
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

template <int R, bool F8>
cudaError_t launch_r(const CorrTcPlan &plan, const CorrTcLaunch &lp, int nb, cudaStream_t st) {
    using G = Geo<R>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e =
            cudaFuncSetAttribute(corr_tc_kernel<R, F8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid((plan.w + BX - 1) / BX, (plan.h + BY - 1) / BY, nb);
    return launch_pdl(corr_tc_kernel<R, F8>, grid, dim3(128), G::SMEM, st, plan.tmS, plan.tmO, lp);
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
                           float q_out) {
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
    lp.scale = feat_scale * feat_scale / (float)plan.c;
    lp.q_out = q_out;
    lp.err = plan.err;
    lp.f16 = plan.f16 ? 1 : 0;
    return launch_plan(plan, lp, nb, st);
}

}  // namespace tc
