// Implicit-GEMM 3x3 convolution on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// GEMM view: M = output pixels, N = cout, K = 9 taps x input channels.  One CTA computes a
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

#include <cstring>
#include <mutex>

#include "conv_tc.cuh"

namespace tc {

namespace {

constexpr int BM = 128;                    // output pixels per CTA (MMA M)
constexpr int BK = 64;                     // input channels per step (128 B of bf16)
constexpr uint32_t A_BYTES = BM * BK * 2;  // 16 KB
constexpr unsigned long long WAIT_NS = 2000000000ull;

enum : int { ERR_PRODUCER = 1, ERR_MMA = 2, ERR_EPILOGUE = 3, ERR_DRAIN = 4 };

__host__ __device__ constexpr int stages_for(int bn) { return bn >= 96 ? 3 : 4; }
__host__ __device__ constexpr int tmem_cols_for(int bn) { return bn <= 32 ? 32 : (bn <= 64 ? 64 : 128); }
__host__ __device__ constexpr size_t smem_bytes_for(int bn) {
    return (size_t)stages_for(bn) * (A_BYTES + (size_t)bn * BK * 2) + 1024 + 256;
}

struct TcLaunch {
    int nch;      // 64-channel steps of the input
    int stride;   // 1 or 2
    int ho, wo;
    int img_off;  // first input image in the A descriptor
    __nv_bfloat16 *out;
    int out_cs;
    const float *bias;
    int leaky;
    int *err;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase of `bar` with the given parity; gives up after WAIT_NS or as soon as
// another role of this CTA (or another CTA) has recorded an error.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, int *err, int code) {
    unsigned long long t0 = 0;
    for (uint32_t i = 0;; ++i) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 63) == 63) {
            if (*(volatile int *)err != 0) return false;
            const unsigned long long t = global_ns();
            if (t0 == 0) t0 = t;
            else if (t - t0 > WAIT_NS) {
                atomicCAS(err, 0, code);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void tma_load_3d(const CUtensorMap *map, uint32_t bar, uint32_t dst, int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(const CUtensorMap *map, uint32_t bar, uint32_t dst, int c0, int c1, int c2,
                                            int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_5d(const CUtensorMap *map, uint32_t bar, uint32_t dst, int c0, int c1, int c2,
                                            int c3, int c4) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand in the 128-byte swizzled layout written
// by TMA (rows of 128 B, 8-row groups 1024 B apart), version 1 (tcgen05).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;            // leading-dimension byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;  // stride-dimension byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;            // descriptor version
    d |= (uint64_t)2 << 61;            // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: D f32, A and B bf16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(dtmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&v);
}

template <int BN>
__global__ void __launch_bounds__(128, 1)
conv_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcLaunch p) {
    constexpr int STAGES = stages_for(BN);
    constexpr uint32_t B_BYTES = BN * BK * 2;
    constexpr uint32_t STAGE_TX = A_BYTES + B_BYTES;
    constexpr uint32_t TMEM_COLS = tmem_cols_for(BN);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;
    uint8_t *sB = smem + STAGES * A_BYTES;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + STAGES * (A_BYTES + B_BYTES));
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 1);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES), accum = smem_u32(bars + 2 * STAGES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x0 = blockIdx.x * BM, y = blockIdx.y, img = blockIdx.z;
    const int nk = 9 * p.nch;

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

    if (threadIdx.x == 0) {
        // ---- producer
        int issued = 0;
        for (int ks = 0; ks < nk; ++ks) {
            const int s = ks % STAGES;
            const uint32_t ph = (uint32_t)(ks / STAGES) & 1u;
            if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, p.err, ERR_PRODUCER)) break;
            const int tap = ks / p.nch, ch = ks - tap * p.nch;
            const int ky = tap / 3, kx = tap - ky * 3;
            const uint32_t fb = full0 + 8 * s;
            mbar_expect_tx(fb, STAGE_TX);
            const uint32_t dA = smem_u32(sA + s * A_BYTES), dB = smem_u32(sB + s * B_BYTES);
            if (p.stride == 1) {
                tma_load_4d(&tmA, fb, dA, ch * BK, x0 + kx - 1, y + ky - 1, img + p.img_off);
            } else {
                const int dx = kx - 1;
                tma_load_5d(&tmA, fb, dA, ch * BK, dx != 0 ? 1 : 0, x0 + (dx < 0 ? -1 : 0), 2 * y + ky - 1,
                            img + p.img_off);
            }
            tma_load_3d(&tmB, fb, dB, ch * BK, 0, tap);
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
        constexpr uint32_t idesc = idesc_bf16(BM, BN);
        for (int ks = 0; ks < nk; ++ks) {
            const int s = ks % STAGES;
            if (!mbar_wait(full0 + 8 * s, (uint32_t)(ks / STAGES) & 1u, p.err, ERR_MMA)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t da = sw128_desc(smem_u32(sA + s * A_BYTES));
            const uint64_t db = sw128_desc(smem_u32(sB + s * B_BYTES));
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
                umma_bf16(tmem, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc, (ks | kk) != 0 ? 1u : 0u);
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
    if (ok) {
        const int row = warp * 32 + lane;
        const int x = x0 + row;
        __nv_bfloat16 *dst = p.out + ((size_t)(img * p.ho + y) * p.wo + x) * p.out_cs;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t r[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
            if (x < p.wo) {
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    v[j] = __uint_as_float(r[j]) + __ldg(p.bias + c0 + j);
                    if (p.leaky) v[j] = v[j] >= 0.f ? v[j] : 0.1f * v[j];
                }
                uint4 lo, hi;
                lo.x = pack_bf16x2(v[0], v[1]);
                lo.y = pack_bf16x2(v[2], v[3]);
                lo.z = pack_bf16x2(v[4], v[5]);
                lo.w = pack_bf16x2(v[6], v[7]);
                hi.x = pack_bf16x2(v[8], v[9]);
                hi.y = pack_bf16x2(v[10], v[11]);
                hi.z = pack_bf16x2(v[12], v[13]);
                hi.w = pack_bf16x2(v[14], v[15]);
                *reinterpret_cast<uint4 *>(dst + c0) = lo;
                *reinterpret_cast<uint4 *>(dst + c0 + 8) = hi;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

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

template <int BN>
cudaError_t launch_bn(const TcConvPlan &plan, const TcLaunch &lp, int n_img, cudaStream_t st) {
    static bool attr_set = false;
    const size_t smem = smem_bytes_for(BN);
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(conv_tc_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid((plan.wo + BM - 1) / BM, plan.ho, n_img);
    conv_tc_kernel<BN><<<grid, 128, smem, st>>>(plan.tmA, plan.tmB, lp);
    return cudaGetLastError();
}

}  // namespace

void TcConvPlan::release() {
    if (wpk) cudaFree(wpk);
    wpk = nullptr;
    enabled = false;
}

bool tc_plan_conv(TcConvPlan &plan, const ConvArgs &a, int n_in, const std::vector<float> &wk_simt, int *err,
                  std::string &why) {
    plan.enabled = false;
    const int bn = a.cout;
    if (bn < 16 || bn > 128 || bn % 16 != 0) { why = "cout must be a multiple of 16 in [16, 128]"; return false; }
    if (a.cin % 8 != 0 || a.in_cs % 8 != 0 || a.out_cs % 8 != 0) { why = "channel counts must be multiples of 8"; return false; }
    if (reinterpret_cast<uintptr_t>(a.in) % 16 != 0) { why = "input not 16-byte aligned"; return false; }
    if (a.stride != 1 && (a.stride != 2 || a.w % 2 != 0)) { why = "stride must be 1, or 2 with even width"; return false; }
    if (a.ho != (a.h - 1) / a.stride + 1 || a.wo != (a.w - 1) / a.stride + 1) { why = "output size mismatch"; return false; }
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) { why = "cuTensorMapEncodeTiled unavailable"; return false; }
    const int nch = (a.cin + BK - 1) / BK, cinp = nch * BK;
    // Packed weights [9][cout][cinp] in bfloat16 (zero beyond cin).
    std::vector<__nv_bfloat16> pk((size_t)9 * bn * cinp, __float2bfloat16_rn(0.f));
    for (int tap = 0; tap < 9; ++tap)
        for (int c = 0; c < a.cin; ++c)
            for (int o = 0; o < bn; ++o)
                pk[((size_t)tap * bn + o) * cinp + c] = __float2bfloat16_rn(wk_simt[((size_t)tap * a.cin + c) * bn + o]);
    __nv_bfloat16 *wdev = nullptr;
    if (cudaMalloc(&wdev, pk.size() * 2) != cudaSuccess) { cudaGetLastError(); why = "weight allocation failed"; return false; }
    if (cudaMemcpy(wdev, pk.data(), pk.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(wdev);
        why = "weight upload failed";
        return false;
    }
    const cuuint32_t ones[5] = {1, 1, 1, 1, 1};
    CUresult r;
    const cuuint64_t esz = 2;
    if (a.stride == 1) {
        const cuuint64_t dims[4] = {(cuuint64_t)a.cin, (cuuint64_t)a.w, (cuuint64_t)a.h, (cuuint64_t)n_in};
        const cuuint64_t strides[3] = {a.in_cs * esz, (cuuint64_t)a.w * a.in_cs * esz, (cuuint64_t)a.h * a.w * a.in_cs * esz};
        const cuuint32_t box[4] = {BK, BM, 1, 1};
        r = enc(&plan.tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(a.in), dims, strides, box, ones,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        const cuuint64_t dims[5] = {(cuuint64_t)a.cin, 2, (cuuint64_t)(a.w / 2), (cuuint64_t)a.h, (cuuint64_t)n_in};
        const cuuint64_t strides[4] = {a.in_cs * esz, 2 * a.in_cs * esz, (cuuint64_t)a.w * a.in_cs * esz,
                                       (cuuint64_t)a.h * a.w * a.in_cs * esz};
        const cuuint32_t box[5] = {BK, 1, BM, 1, 1};
        r = enc(&plan.tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(a.in), dims, strides, box, ones,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (r == CUDA_SUCCESS) {
        const cuuint64_t dims[3] = {(cuuint64_t)cinp, (cuuint64_t)bn, 9};
        const cuuint64_t strides[2] = {(cuuint64_t)cinp * esz, (cuuint64_t)bn * cinp * esz};
        const cuuint32_t box[3] = {BK, (cuuint32_t)bn, 1};
        r = enc(&plan.tmB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, wdev, dims, strides, box, ones,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (r != CUDA_SUCCESS) {
        cudaFree(wdev);
        why = "tensor map encoding failed (" + std::to_string((int)r) + ")";
        return false;
    }
    plan.bn = bn;
    plan.cout = bn;
    plan.nch = nch;
    plan.stride = a.stride;
    plan.h = a.h;
    plan.w = a.w;
    plan.ho = a.ho;
    plan.wo = a.wo;
    plan.n_in = n_in;
    plan.in_base = a.in;
    plan.img_bytes = (size_t)a.h * a.w * a.in_cs * esz;
    plan.wpk = wdev;
    plan.err = err;
    plan.enabled = true;
    return true;
}

cudaError_t launch_conv_tc(const TcConvPlan &plan, const ConvArgs &a, cudaStream_t st) {
    if (!plan.enabled) return cudaErrorInvalidValue;
    const ptrdiff_t off = static_cast<const char *>(a.in) - static_cast<const char *>(plan.in_base);
    if (off < 0 || off % (ptrdiff_t)plan.img_bytes != 0) return cudaErrorInvalidValue;
    const int img_off = (int)(off / (ptrdiff_t)plan.img_bytes);
    if (img_off + a.n > plan.n_in || a.n < 1) return cudaErrorInvalidValue;
    if (reinterpret_cast<uintptr_t>(a.out) % 16 != 0 || a.out_cs % 8 != 0) return cudaErrorInvalidValue;
    TcLaunch lp{plan.nch, plan.stride, plan.ho, plan.wo, img_off, static_cast<__nv_bfloat16 *>(a.out), a.out_cs,
                a.bias, a.leaky, plan.err};
    switch (plan.bn) {
        case 16: return launch_bn<16>(plan, lp, a.n, st);
        case 32: return launch_bn<32>(plan, lp, a.n, st);
        case 48: return launch_bn<48>(plan, lp, a.n, st);
        case 64: return launch_bn<64>(plan, lp, a.n, st);
        case 80: return launch_bn<80>(plan, lp, a.n, st);
        case 96: return launch_bn<96>(plan, lp, a.n, st);
        case 112: return launch_bn<112>(plan, lp, a.n, st);
        case 128: return launch_bn<128>(plan, lp, a.n, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tc
