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

}  // namespace tc
