// Training-step kernels: launch parameter blocks and host launchers.
#pragma once

#include "common.cuh"

namespace tc {
namespace train {

// Weight gradient of a 3x3 conv (pad 1, stride 1 or 2): x [n][h][w][x_cs] (window at the
// pointer, cin channels), dz [n * ho * wo][dz_cs] (cout channels: the gradient after the
// activation), dw [cout][cin][3][3] accumulated.
template <typename T>
struct WgradArgs {
    const T *x;
    int x_cs;
    int n, h, w, cin, stride, ho, wo;
    const float *dz;
    int dz_cs;
    int cout;
    float *dw;
};

// Correlation backward; all maps [n][h][w][*_cs] with their windows at the pointers.
template <typename T>
struct CorrBwdArgs {
    const T *fs;   // self features (c channels)
    int fs_cs;
    const T *fo;   // other features
    int fo_cs;
    const T *cost; // saved cost volume (after LeakyReLU), (2r+1)^2 channels
    int cost_cs;
    const float *dcost;
    int dcost_cs;
    int n, h, w, c, r;
    float *dfs;    // may be NULL
    int dfs_cs;
    float *dfo;    // may be NULL
    int dfo_cs;
    int accumulate;
};

// Feature-warp backward: f [n][h][w][f_cs], flow [n][h][w][2], dout [n][h][w][dout_cs].
template <typename T>
struct WarpBwdArgs {
    const T *f;
    int f_cs;
    const float *flow;
    const float *dout;
    int dout_cs;
    int n, h, w, c;
    float *df;     // scatter target (accumulated with atomics), may be NULL
    int df_cs;
    float *dflow;  // may be NULL
    int accumulate;
};

struct AdamW {
    float lr, beta1, beta2, eps, weight_decay;
};

cudaError_t pack_fwd(const float *w, int cout, int cin, int cin_p, bool round_bf16, float *wk, cudaStream_t st);
cudaError_t pack_dgrad(const float *w, int cout, int cin, int cout_p, int cin_p, float *wk, cudaStream_t st);
template <typename T>
cudaError_t pack_images(const float *a, const float *b, int n, int h, int w, T *out, cudaStream_t st);
template <typename T>
cudaError_t lrelu_bwd(const float *dy, int dy_cs, const T *y, int y_cs, bool leaky, size_t npix, int nc, float *dz,
                      float *dz_dil, int ho, int wo, int hd, int wd, cudaStream_t st);
template <typename T> cudaError_t wgrad(const WgradArgs<T> &a, float *db, cudaStream_t st);
cudaError_t pack_tc(const float *w, int cout, int cin, int mode, int lo, int n, int bn, int cinp, void *out,
                    cudaStream_t st);
template <typename T>
cudaError_t x_to_cp(const T *x, int x_cs, int n_img, int h, int w, int cin, int wp, int n, void *const out[3],
                    cudaStream_t st);
cudaError_t dz_to_cp(const float *dz, int dz_cs, int n_img, int h, int w, int ho, int wo, int stride, int cout, int wp,
                     void *out, float *db, cudaStream_t st);
cudaError_t bgrad(const float *dz, int dz_cs, size_t P, int cout, float *db, cudaStream_t st);
template <typename T>
cudaError_t lrelu_bwd2(const float *dy, int dy_cs, const T *y, int y_cs, bool leaky, size_t npix, int nc, float *dz,
                       void *dzh, void *dzh_dil, int ho, int wo, int hd, int wd, cudaStream_t st);
cudaError_t head_dgrad(const float *dflow, const float *w, int cin, int n, int h, int w_, float *dx, int dx_cs,
                       bool accumulate, cudaStream_t st);
template <typename T> cudaError_t corr_bwd(const CorrBwdArgs<T> &a, cudaStream_t st);
template <typename T> cudaError_t warp_bwd(const WarpBwdArgs<T> &a, cudaStream_t st);
cudaError_t up_bwd(const float *dfine, int n, int h, int w, int s, float *dcoarse, cudaStream_t st);
cudaError_t window_add(const float *src, int src_cs, size_t npix, int nc, float *dst, int dst_cs, bool accumulate,
                       cudaStream_t st);
template <typename T> cudaError_t flow_to_act(const float *flow, size_t npix, T *act, int act_cs, cudaStream_t st);
cudaError_t gt_level(const float *gt, int n, int H, int W, int l, float *out, cudaStream_t st);
cudaError_t epe(const float *flow, const float *gt, size_t npix, double *loss, float *dflow, bool accumulate,
                cudaStream_t st);
cudaError_t adamw(float *p, const float *g, float *m, float *v, const uint8_t *decay, size_t n, const AdamW &h,
                  long long step, cudaStream_t st);
cudaError_t bruteforce(const float *a, const float *b, int c, int h, int w, int r, int *kout, cudaStream_t st);

}  // namespace train
}  // namespace tc
