// BF16 cost volume for callers that cannot allocate device memory.
//
// tc_op_correlation(TC_BF16, ...) stages bfloat16 copies of its two feature maps and of the
// cost volume in temporary device buffers that it allocates and frees on every call.  Some
// hosts cannot allow that: an application whose memory pool has reserved the device memory
// up front and hands the library only pre-allocated buffers, or a real-time loop that
// cannot afford cudaMalloc/cudaFree (both may synchronise the whole device and take an
// unbounded time).  tc_op_correlation_bf16_noalloc runs the same kernels -- the tensor-core
// correlation where the channel count allows it, else the CUDA-core one -- with its staging
// buffers and its device error word in one fixed array of TC_NOALLOC_SCRATCH_BYTES of device
// memory, defined below at file scope.  Every GPU that loads the library holds that array
// until the process exits.
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/tc_stream.h"
#include "common.cuh"
#include "corr_tc.cuh"

#include "engine_internal.h"

// Staging area shared by every call on a device.  In host code this name is only a
// host-side stand-in for the symbol, never a device address: the device address comes
// from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[TC_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
// The last 256 bytes of the array hold the device error word of the tensor-core kernel.
constexpr size_t kErrBytes = 256;
std::mutex g_mu;
unsigned char *g_scratch_ptr[kMaxDevices] = {nullptr};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Device address of the staging array on the current device, looked up once per device
// (on the first call made with that device current).  That lookup is not made while
// cuda_stream is being captured into a graph: the call is refused instead.
tc_status scratch_address(cudaStream_t s, unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return tc_record_error(TC_ERR_CUDA, std::string("tc_op_correlation_bf16_noalloc: cudaGetDevice: ") +
                                                cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return tc_record_error(TC_ERR_UNSUPPORTED, "tc_op_correlation_bf16_noalloc: device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        e = cudaStreamIsCapturing(s, &cs);
        if (e != cudaSuccess)
            return tc_record_error(TC_ERR_CUDA, std::string("tc_op_correlation_bf16_noalloc: cudaStreamIsCapturing: ") +
                                                    cudaGetErrorString(e));
        if (cs != cudaStreamCaptureStatusNone)
            return tc_record_error(TC_ERR_UNSUPPORTED,
                                   "tc_op_correlation_bf16_noalloc: the first call on a device sets up the staging "
                                   "array and must come before any stream capture");
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            return tc_record_error(TC_ERR_CUDA, std::string("tc_op_correlation_bf16_noalloc: cudaGetSymbolAddress: ") +
                                                    cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_ptr[dev];
    return TC_OK;
}

tc_status launch_failed(cudaError_t e) {
    return tc_record_error(TC_ERR_CUDA, std::string("tc_op_correlation_bf16_noalloc: ") + cudaGetErrorString(e));
}

}  // namespace

extern "C" tc_status tc_op_correlation_bf16_noalloc(const float *f1, const float *f2, int n, int h, int w, int c,
                                                    int r, float *out, void *cuda_stream) {
    if (!f1 || !f2 || !out || n < 1 || h < 1 || w < 1 || c < 4 || c % 4 != 0 || r < 1 || r > 4)
        return tc_record_error(TC_ERR_INVALID_ARG, "tc_op_correlation_bf16_noalloc: bad argument");
    const size_t D = (size_t)(2 * r + 1) * (2 * r + 1);
    const size_t nf = (size_t)n * h * w * c, no = (size_t)n * h * w * D;
    const size_t bytes_f = align256(nf * sizeof(__nv_bfloat16));
    const size_t need = 2 * bytes_f + align256(no * sizeof(__nv_bfloat16)) + kErrBytes;
    if (need > TC_NOALLOC_SCRATCH_BYTES) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "tc_op_correlation_bf16_noalloc: needs %zu bytes of staging, more than the fixed %zu "
                 "(use tc_op_correlation, or a smaller n*h*w*(2c + (2r+1)^2))",
                 need, (size_t)TC_NOALLOC_SCRATCH_BYTES);
        return tc_record_error(TC_ERR_INVALID_ARG, msg);
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    unsigned char *base = nullptr;
    tc_status st = scratch_address(s, &base);
    if (st != TC_OK) return st;
    // Staging regions: bf16 f1, bf16 f2, bf16 cost volume, and the error word at the end.
    // Every staged byte read below is written earlier in the same call; the error word is
    // cleared here, since the array keeps the last call's contents.
    __nv_bfloat16 *a = reinterpret_cast<__nv_bfloat16 *>(base);
    __nv_bfloat16 *b = reinterpret_cast<__nv_bfloat16 *>(base + bytes_f);
    __nv_bfloat16 *o = reinterpret_cast<__nv_bfloat16 *>(base + 2 * bytes_f);
    int *err = reinterpret_cast<int *>(base + TC_NOALLOC_SCRATCH_BYTES - kErrBytes);
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = tc::launch_to_act<__nv_bfloat16>(f1, nf, a, s);
    if (e == cudaSuccess) e = tc::launch_to_act<__nv_bfloat16>(f2, nf, b, s);
    if (e != cudaSuccess) return launch_failed(e);
    // The tensor-core plan only encodes tensor maps on the host (no allocation); it is taken
    // exactly when tc_op_correlation(TC_BF16) takes it (c a multiple of 8 up to 128).
    tc::CorrTcPlan plan;
    std::string why;
    const bool use_tc = tc::tc_plan_corr(plan, a, n, c, b, n, c, h, w, c, r, err, why);
    const size_t img = (size_t)h * w * c;
    for (int i = 0; i < n && e == cudaSuccess; i += 2) {
        const int nb = n - i < 2 ? n - i : 2;
        if (use_tc) {
            const int imgs[2] = {i, i + nb - 1};
            e = tc::launch_corr_tc(plan, nb, imgs, imgs, o + (size_t)i * h * w * D, (int)D, nullptr, nullptr, s);
        } else {
            tc::CorrArgs ca{{a + i * img, a + (i + nb - 1) * img}, {b + i * img, b + (i + nb - 1) * img}, c, c, nb, h,
                            w, c, r, o + (size_t)i * h * w * D, (int)D, nullptr};
            e = tc::launch_corr<__nv_bfloat16>(ca, s);
        }
    }
    if (e == cudaSuccess) e = tc::launch_from_act<__nv_bfloat16>(o, no, out, s);
    if (e != cudaSuccess) return launch_failed(e);
    // Like tc_op_correlation: wait, then report a tensor-core wait that gave up.
    int code = 0;
    e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&code, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return launch_failed(e);
    if (code != 0)
        return tc_record_error(TC_ERR_TIMEOUT, "tc_op_correlation_bf16_noalloc: tensor-core kernel gave up waiting");
    tc_set_last_op_tensor_cores(use_tc ? 1 : 0);
    return TC_OK;
}
