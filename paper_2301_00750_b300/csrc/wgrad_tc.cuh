// Weight gradient of a 3x3 conv on the tensor cores: plan and launch interface.
#pragma once

#include <cuda.h>

#include <string>

#include "common.cuh"

namespace tc {

// dW[o][c][tap] = sum over pixels q of dz[o][q] x[c][q + shift(tap)], as nine GEMMs with
// M = cout (<= 128), N = the padded input channels (<= 256), K = pixels, over operands in a
// channel-major, zero-bordered layout ("CP"):
//   q runs over n images x (h + 2) rows x wp columns (wp = w + 2 rounded up to 8), image
//   pixel (y, x) at row y + 1, column x + 1, zero elsewhere;
//   dz_cp [cout][P]: the output gradient after the activation, at input resolution (for a
//   stride-2 conv, the gradient of output pixel (oy, ox) sits at (2 oy, 2 ox), zero
//   between);
//   x_cp[kx] [n_ch][P]: the conv input shifted by kx - 1 columns (kx = 0, 1, 2), so the
//   tap (ky, kx) reads x_cp[kx] at q + (ky - 1) wp, a multiple of 8 elements (16 bytes);
//   channel cin of x_cp[1] is 1 at the image pixels (and 0 on the border), so the center
//   tap's column cin is the bias gradient.
struct WgradTcPlan {
    bool enabled = false;
    CUtensorMap tmDZ;
    CUtensorMap tmX[3];
    int cout = 0, cin = 0, n = 0, wp = 0, nsteps = 0, chunks = 0, spc = 0;
    long long P = 0;
    float *partial = nullptr;  // [chunks][9][cout][n] (not owned)
    int *err = nullptr;
};

// Plans the nine GEMMs of one layer over the CP buffers (bf16).  n = channels of x_cp (a
// multiple of 16, > cin, <= 256).  partial must hold wgrad_tc_partial_floats(...) floats.
bool wgrad_tc_plan(WgradTcPlan &plan, const void *dz_cp, const void *const x_cp[3], int cout, int cin, int n, int wp,
                   long long P, float *partial, int *err, std::string &why);
size_t wgrad_tc_partial_floats(long long P, int n, int cout);

// Runs the GEMMs and adds the result to dw [cout][cin][3][3] and (if db) the bias gradient
// to db [cout] (float).
cudaError_t wgrad_tc_launch(const WgradTcPlan &plan, float *dw, float *db, cudaStream_t st);

}  // namespace tc
