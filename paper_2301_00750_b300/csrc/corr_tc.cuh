// Tensor-core (tcgen05) correlation cost volume: plan and launch interface.
#pragma once

#include <cuda.h>

#include <string>

#include "common.cuh"

namespace tc {

// A planned tensor-core correlation over bfloat16 (or half, or e4m3) NHWC feature buffers.
// tmS covers the "self" buffer, tmO the "other" buffer (they may be the same buffer); both
// hold n_img images of h x w pixels with c channels at pixel stride cs.
struct CorrTcPlan {
    bool enabled = false;
    CUtensorMap tmS;
    CUtensorMap tmO;
    int h = 0, w = 0, c = 0, r = 0, nch = 0;
    int rb = 128;     // bytes of channels per step: 128, or 64 for BF16 features of <= 32 channels
    bool f8 = false;  // e4m3 features (kind::f8f6f4)
    bool f16 = false; // IEEE half features and cost volume instead of bfloat16
    int *err = nullptr;  // device error word (not owned)
};

// Plans the correlation between channels [0, c) of `self` (n_self images, pixel stride
// self_cs) and of `other` (n_other images, pixel stride other_cs).  Returns false with `why`
// when not eligible (c % 8 != 0, c > 128, r > 4, misaligned buffers).
bool tc_plan_corr(CorrTcPlan &plan, const void *self, int n_self, int self_cs, const void *other, int n_other,
                  int other_cs, int h, int w, int c, int r, int *err, std::string &why, bool f8 = false,
                  bool f16 = false);

// Launches the planned correlation for nb <= 2 batch entries: entry b correlates image
// img_self[b] of the self buffer with image img_other[b] of the other buffer and writes
// LeakyReLU(mean over channels) for the (2r+1)^2 displacements, in the features' type, to
// out + ((b h + y) w + x) out_cs + k.  If self_copy is set, it also copies the c self
// features of pixel (b, y, x) (read from fs[b], [h][w][c]) to self_copy + ((b h + y) w + x)
// out_cs.
// For e4m3 features stored with scale feat_scale, the cost is feat_scale^2 / c times the
// integer-grid dot product, stored e4m3 after multiplying by q_out (1 / its scale).
// alone: no other stream's kernels share the GPU (a small launch then lets the next kernel
// of the stream set up early).
cudaError_t launch_corr_tc(const CorrTcPlan &plan, int nb, const int img_self[2], const int img_other[2], void *out,
                           int out_cs, const void *const fs[2], void *self_copy, cudaStream_t st,
                           float feat_scale = 1.f, float q_out = 1.f, bool alone = false);

// Lane pairs (batched streams): 2 lanes entries, entry z = direction d = z & 1 of lane
// q = z >> 1, correlates image s0 + q + d pair_lanes of the self buffer with image
// o0 + q oq + d od of the other buffer and writes to out + ((z h + y) w + x) out_cs; the
// self copy (if set) reads fs0 + (q + d pair_lanes) fs_img_bytes.  16-bit features only.
cudaError_t launch_corr_tc_pairs(const CorrTcPlan &plan, int lanes, int pair_lanes, int s0, int o0, int oq, int od,
                                 void *out, int out_cs, const void *fs0, size_t fs_img_bytes, void *self_copy,
                                 cudaStream_t st);

}  // namespace tc
