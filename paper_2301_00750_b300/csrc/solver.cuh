// Screened-Poisson solver (Eq. 1 by the SGD-momentum iteration of Eq. 8): launch interface.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace tc {

// Planar float images (c, h, w), 1 <= c <= 3; wc (h, w).  b and s0..s3 are scratch of
// c * h * w floats each, c0 of h * w floats (none may alias the others or the inputs); O
// receives the last iterate, O2 (may be NULL) a second copy of it.  iters = 0 computes the
// coefficients only.
struct PoissonArgs {
    const float *P, *A, *wc;
    int c, h, w, iters;
    float eta, kappa;
    float *b, *s0, *s1, *s2, *s3;
    float *O, *O2;
    float *c0;
};

cudaError_t launch_poisson(const PoissonArgs &a, cudaStream_t st);

// dst[i] = src[i] for i < n and wdst[i] = wsrc[i] for i < nw (wdst may be NULL): the
// solver's output and weights copied to the caller's buffers (tag 0), or the caller's
// inputs copied into the stream's state (tag 1).  A kernel, so that a captured frame graph
// can retarget it; the tag tells the two apart in the graph.
cudaError_t launch_copy_out(const float *src, float *dst, size_t n, const float *wsrc, float *wdst, size_t nw,
                            cudaStream_t st, int tag = 0);
const void *copy_out_kernel_fn(int tag);

}  // namespace tc
