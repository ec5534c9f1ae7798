// Weight gradient of the 3x3 convolutions on the tensor cores (tcgen05), for the BF16
// trainer.  For each tap the gradient is a GEMM with the pixels as K:
//   D_tap[o][c] = sum_q dz[o][q] x[c][q + shift(tap)]
// over operands stored channel-major with a zero border (see wgrad_tc.cuh), so that both
// operand tiles are K-major rows of 64 pixels (128 bytes, 128-byte swizzle) read straight by
// TMA, and the tap shift is a coordinate offset.  A CTA owns one tap and one chunk of the
// pixel range: lane 0 of warp 0 loads [128 x 64] dz and [n x 64] x tiles into a ring of
// stages, lane 0 of warp 1 issues tcgen05.mma (128 x n x 16, BF16 -> FP32) into TMEM, and
// the four warps write the CTA's partial [128][n] tile; a second kernel sums the partial
// tiles of the chunks into dW.  Waits are bounded as in the convolution kernels.
#include <cudaTypedefs.h>

#include "tc_ptx.cuh"
#include "wgrad_tc.cuh"

namespace tc {

namespace {

using namespace ptx;

constexpr int WG_M = 128;           // MMA rows (output channels; rows past cout are not used)
constexpr int WG_K = 64;            // pixels per K step (128 bytes of bf16)
constexpr int WG_STAGES = 4;
constexpr uint32_t A_FULL = WG_M * WG_K * 2;   // 16 KB: what one MMA reads of A

// Shared memory of a plan: STAGES A tiles of am rows (cout rounded up to 8) and B tiles of n
// rows, each 128-byte rows; the MMA reads 128 rows of A, so the region after the last A tile
// stays inside the allocation (rows past cout read whatever is there and only feed
// accumulator rows that are never stored).
inline size_t wg_smem(int am, int n) {
    const size_t a = (size_t)am * WG_K * 2, b = (size_t)n * WG_K * 2;
    size_t bytes = WG_STAGES * (a + b);
    const size_t last_a_end = (WG_STAGES - 1) * a + A_FULL;
    if (last_a_end > bytes) bytes = last_a_end;
    return bytes + 1024 + 256;
}

enum : int { ERR_WG_PRODUCER = 11, ERR_WG_MMA = 12, ERR_WG_EPILOGUE = 13, ERR_WG_DRAIN = 14 };

struct WgLaunch {
    int n, am, cout, wp, nsteps, spc;
    float *partial;
    int *err;
};

__global__ void __launch_bounds__(128, 1)
wgrad_tc_kernel(const __grid_constant__ CUtensorMap tmDZ, const __grid_constant__ CUtensorMap tmX0,
                const __grid_constant__ CUtensorMap tmX1, const __grid_constant__ CUtensorMap tmX2, const WgLaunch p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t a_bytes = (uint32_t)p.am * WG_K * 2, b_bytes = (uint32_t)p.n * WG_K * 2;
    uint8_t *sA = smem;
    uint8_t *sB = smem + WG_STAGES * a_bytes;
    size_t bar_off = (size_t)WG_STAGES * (a_bytes + b_bytes);
    if ((WG_STAGES - 1) * (size_t)a_bytes + A_FULL > bar_off) bar_off = (WG_STAGES - 1) * (size_t)a_bytes + A_FULL;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + bar_off);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * WG_STAGES + 1);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + WG_STAGES), accum = smem_u32(bars + 2 * WG_STAGES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tap = blockIdx.x, chunk = blockIdx.y;
    const int ky = tap / 3, kx = tap - 3 * ky;
    const CUtensorMap *tmX = kx == 0 ? &tmX0 : (kx == 1 ? &tmX1 : &tmX2);
    const int k0 = chunk * p.spc, k1 = k0 + p.spc < p.nsteps ? k0 + p.spc : p.nsteps;
    const uint32_t tmem_cols = p.n <= 32 ? 32 : (p.n <= 64 ? 64 : (p.n <= 128 ? 128 : 256));

    if (threadIdx.x == 0) {
        for (int s = 0; s < WG_STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(accum, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const int shift = (ky - 1) * p.wp;  // a multiple of 8 pixels: 16-byte aligned TMA x

    if (threadIdx.x == 0) {
        int issued = 0;
        for (int k = k0; k < k1; ++k) {
            const int i = k - k0, s = i % WG_STAGES;
            if (!mbar_wait(empty0 + 8 * s, ((uint32_t)(i / WG_STAGES) & 1u) ^ 1u, p.err, ERR_WG_PRODUCER)) break;
            mbar_expect_tx(full0 + 8 * s, a_bytes + b_bytes);
            tma_load_2d(&tmDZ, full0 + 8 * s, smem_u32(sA + s * a_bytes), k * WG_K, 0);
            tma_load_2d(tmX, full0 + 8 * s, smem_u32(sB + s * b_bytes), k * WG_K + shift, 0);
            issued = i + 1;
        }
        if (issued < k1 - k0) {
            const unsigned long long t0 = global_ns();
            for (int i = issued - WG_STAGES < 0 ? 0 : issued - WG_STAGES; i < issued; ++i)
                while (!mbar_try(full0 + 8 * (i % WG_STAGES), (uint32_t)(i / WG_STAGES) & 1u))
                    if (global_ns() - t0 > WAIT_NS) { atomicCAS(p.err, 0, ERR_WG_DRAIN); break; }
        }
    } else if (threadIdx.x == 32) {
        const uint32_t idesc = idesc_bf16(WG_M, p.n);
        for (int k = k0; k < k1; ++k) {
            const int i = k - k0, s = i % WG_STAGES;
            if (!mbar_wait(full0 + 8 * s, (uint32_t)(i / WG_STAGES) & 1u, p.err, ERR_WG_MMA)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t da = sw128_desc(smem_u32(sA + s * a_bytes));
            const uint64_t db = sw128_desc(smem_u32(sB + s * b_bytes));
#pragma unroll
            for (int kk = 0; kk < WG_K / 16; ++kk)
                umma_bf16(tmem, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc, (i | kk) != 0 ? 1u : 0u);
            umma_commit(empty0 + 8 * s);
        }
        umma_commit(accum);
    }

    int ok = 1;
    if (lane == 0) ok = mbar_wait(accum, 0, p.err, ERR_WG_EPILOGUE) && *(volatile int *)p.err == 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok && warp * 32 < p.cout) {
        // row o = threadIdx.x (o < cout): its n accumulator columns (zero for an empty chunk)
        float *dst = p.partial + (((size_t)chunk * 9 + tap) * p.cout + threadIdx.x) * p.n;
        const bool mine = (int)threadIdx.x < p.cout, any = k1 > k0;
        for (int c0 = 0; c0 < p.n; c0 += 16) {
            uint32_t r[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
            if (!mine) continue;
            float4 *d4 = reinterpret_cast<float4 *>(dst + c0);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                d4[q] = any ? make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                          __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]))
                            : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
    }
}

// dw[o][c][tap] += sum over chunks of partial[chunk][tap][o][c]; with db, also
// db[o] += sum over chunks of partial[chunk][4][o][cin] (the center tap against the row of
// ones that the x operand carries at channel cin: the bias gradient).
__global__ void wgrad_reduce_kernel(const float *partial, int chunks, int n, int cout, int cin, float *dw, float *db) {
    const size_t total = (size_t)cout * cin * 9;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < total) {
        const int tap = (int)(i % 9);
        const size_t r = i / 9;
        const int c = (int)(r % cin), o = (int)(r / cin);
        float s = 0.f;
        for (int ch = 0; ch < chunks; ++ch) s += partial[(((size_t)ch * 9 + tap) * cout + o) * n + c];
        dw[i] += s;
    } else if (db && i < total + (size_t)cout) {
        const int o = (int)(i - total);
        float s = 0.f;
        for (int ch = 0; ch < chunks; ++ch) s += partial[(((size_t)ch * 9 + 4) * cout + o) * n + cin];
        db[o] += s;
    }
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 encode_fn();

// Pixel chunks per tap: about 64 K steps each, at least enough for two CTAs per SM.
static int wg_chunks(long long nsteps) {
    long long chunks = (nsteps + 63) / 64;
    const long long min_chunks = (2 * 148 + 8) / 9;
    if (chunks < min_chunks) chunks = min_chunks;
    if (chunks > nsteps) chunks = nsteps;
    if (chunks < 1) chunks = 1;
    if (chunks > 65535) chunks = 65535;
    return (int)chunks;
}

size_t wgrad_tc_partial_floats(long long P, int n, int cout) {
    const long long nsteps = (P + WG_K - 1) / WG_K;
    return (size_t)wg_chunks(nsteps) * 9 * cout * n;
}

bool wgrad_tc_plan(WgradTcPlan &plan, const void *dz_cp, const void *const x_cp[3], int cout, int cin, int n, int wp,
                   long long P, float *partial, int *err, std::string &why) {
    plan.enabled = false;
    if (cout < 1 || cout > WG_M) { why = "cout must lie in [1, 128]"; return false; }
    if (n % 16 != 0 || n < 16 || n > 256 || cin >= n) {
        why = "channels plus the row of ones must fit a multiple of 16 <= 256";
        return false;
    }
    if (wp % 8 != 0 || P % 8 != 0) { why = "row pitch and pixel count must be multiples of 8"; return false; }
    if (reinterpret_cast<uintptr_t>(dz_cp) % 16 != 0) { why = "misaligned dz"; return false; }
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) { why = "cuTensorMapEncodeTiled unavailable"; return false; }
    const cuuint32_t ones[2] = {1, 1};
    {
        const cuuint64_t dims[2] = {(cuuint64_t)P, (cuuint64_t)cout};
        const cuuint64_t strides[1] = {(cuuint64_t)P * 2};
        const cuuint32_t box[2] = {WG_K, (cuuint32_t)((cout + 7) / 8 * 8)};
        if (enc(&plan.tmDZ, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(dz_cp), dims, strides, box, ones,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
            why = "tensor map encoding failed (dz)";
            return false;
        }
    }
    for (int k = 0; k < 3; ++k) {
        if (reinterpret_cast<uintptr_t>(x_cp[k]) % 16 != 0) { why = "misaligned x"; return false; }
        const cuuint64_t dims[2] = {(cuuint64_t)P, (cuuint64_t)n};
        const cuuint64_t strides[1] = {(cuuint64_t)P * 2};
        const cuuint32_t box[2] = {WG_K, (cuuint32_t)n};
        if (enc(&plan.tmX[k], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(x_cp[k]), dims, strides, box, ones,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
            why = "tensor map encoding failed (x)";
            return false;
        }
    }
    plan.cout = cout;
    plan.cin = cin;
    plan.n = n;
    plan.wp = wp;
    plan.P = P;
    plan.nsteps = (int)((P + WG_K - 1) / WG_K);
    plan.chunks = wg_chunks(plan.nsteps);
    plan.spc = (plan.nsteps + plan.chunks - 1) / plan.chunks;
    plan.partial = partial;
    plan.err = err;
    plan.enabled = true;
    return true;
}

cudaError_t wgrad_tc_launch(const WgradTcPlan &plan, float *dw, float *db, cudaStream_t st) {
    if (!plan.enabled) return cudaErrorInvalidValue;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(wgrad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)wg_smem(WG_M, 256));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int am = (plan.cout + 7) / 8 * 8;
    WgLaunch lp{plan.n, am, plan.cout, plan.wp, plan.nsteps, plan.spc, plan.partial, plan.err};
    dim3 grid(9, plan.chunks);
    wgrad_tc_kernel<<<grid, 128, wg_smem(am, plan.n), st>>>(plan.tmDZ, plan.tmX[0], plan.tmX[1], plan.tmX[2], lp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t total = (size_t)plan.cout * plan.cin * 9 + (db ? plan.cout : 0);
    wgrad_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(plan.partial, plan.chunks, plan.n, plan.cout,
                                                                        plan.cin, dw, db);
    return cudaGetLastError();
}

}  // namespace tc
