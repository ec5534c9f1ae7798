/* tc_train.h -- C ABI of the in-project training of the lite flow network (Sec. 3.2), the
 * backward passes of its stages, and the brute-force flow used as fallback and as the yardstick of learned flows.
 *
 * The paper trains its flow network with a multi-scale loss of equal level weights and
 * AdamW (Sec. 3.2 "Training"; supplement "Training Settings"), on datasets this library
 * does not have; here the same network trains on synthetic pairs with known flow.  One
 * training step for a batch of pairs (a, b) with ground-truth flow F = F_{a->b}
 * (a(x) ~ b(x + F(x))) runs, as explicit kernel launches on the caller's CUDA stream:
 *   forward   the feature pyramids of a and b, the coarse-to-fine estimators for a -> b
 *             (the same layers as tc_process_frame; level flows kept);
 *   loss      sum over estimator levels l = L..2 of the mean end-point error (Eq. 10,
 *             the supplement's EPE loss) between flow^l and the ground truth of level l
 *             (the mean of F over each 2^l x 2^l block, divided by 2^l: flows are in
 *             pixels of their level, so the supplement's x20 scaling is not needed), equal
 *             weights;
 *   backward  data and weight gradients of every conv, the correlation, the feature warp
 *             and the flow upsampling (float32 gradients);
 *   update    AdamW on the float32 master weights (decoupled weight decay on conv weights,
 *             none on biases).
 * TC_BF16 stores the forward activations as bfloat16 and rounds the conv weights to
 * bfloat16 in the forward (the master weights stay float32); TC_FP32 is float32
 * throughout.  All device pointers; errors as in tc_stream.h.
 */
#ifndef TC_TRAIN_H
#define TC_TRAIN_H

#include "tc_stream.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tc_trainer tc_trainer;

typedef struct {
    int batch;                 /* pairs per step, >= 1 */
    int height, width;         /* pair size: multiples of 2^levels of the network */
    tc_precision precision;    /* TC_FP32 or TC_BF16 */
    const char *weights_path;  /* initial weights: TCW1 file (tc_stream.h), or NULL and */
    const void *weights_blob;  /*   the same bytes in memory (copied) */
    size_t weights_bytes;
    float lr, beta1, beta2, eps, weight_decay;  /* AdamW */
} tc_trainer_desc;

/* Defaults for the optimiser fields: lr 1e-4, betas (0.9, 0.99), eps 1e-8, weight decay
 * 4e-4 (Sec. 3.2 "Training": beta2 0.99 and decay 0.0004 as printed; the printed beta1 =
 * 0.09 is read as 0.9). */
TC_API void tc_trainer_default_desc(tc_trainer_desc *d);

/* Creates a trainer: parses the weights, allocates every activation, gradient and
 * optimiser buffer for the batch.  Errors: TC_ERR_INVALID_ARG (sizes, precision),
 * TC_ERR_IO (weights), TC_ERR_UNSUPPORTED (a TCW2 file with a refinement network: the
 * trainer trains the network without it), TC_ERR_OOM, TC_ERR_CUDA. */
TC_API tc_status tc_trainer_create(const tc_trainer_desc *desc, void *cuda_stream, tc_trainer **out);

/* What tc_trainer_run does. */
typedef enum {
    TC_TRAIN_FORWARD = 0,   /* forward and loss only */
    TC_TRAIN_BACKWARD = 1,  /* + gradients (kept until the next run; tc_trainer_get_grads) */
    TC_TRAIN_STEP = 2       /* + AdamW update of the master weights */
} tc_train_mode;

/* One run over a batch.  I_a, I_b: device (batch, 3, height, width) float32 planar, values
 * in [0, 1]; flow_gt: device (batch, 2, height, width) float32 planar (u then v), the flow
 * F_{a->b}.  loss_out: optional HOST double receiving the loss; if given the call waits for
 * the stream, otherwise it returns without waiting (tc_trainer_loss reads it later). */
TC_API tc_status tc_trainer_run(tc_trainer *t, const float *I_a, const float *I_b, const float *flow_gt,
                                tc_train_mode mode, double *loss_out);

/* Loss of the last run (waits for the stream). */
TC_API tc_status tc_trainer_loss(tc_trainer *t, double *loss_out);

/* Number of float32 master parameters: every layer in weight-file order, weights
 * (cout, cin, 3, 3) then bias (cout). */
TC_API size_t tc_trainer_num_params(const tc_trainer *t);

/* Host copies of the master weights, of the gradients of the last BACKWARD/STEP run, and
 * a host write of the master weights (resets nothing else).  n must equal
 * tc_trainer_num_params.  Wait for the stream. */
TC_API tc_status tc_trainer_get_params(tc_trainer *t, float *host, size_t n);
TC_API tc_status tc_trainer_get_grads(tc_trainer *t, float *host, size_t n);
TC_API tc_status tc_trainer_set_params(tc_trainer *t, const float *host, size_t n);

/* Flow of estimator level l (2 <= l <= levels) from the last run: device
 * (batch, h >> l, w >> l, 2) float32 (u, v interleaved), in pixels of level l. */
TC_API tc_status tc_trainer_level_flow(tc_trainer *t, int level, float *out);

/* Completed AdamW steps. */
TC_API long long tc_trainer_steps(const tc_trainer *t);

/* Checkpoint: "TCK1", the step count, the network header, the master weights and both
 * AdamW moments, little-endian.  tc_trainer_load requires the same network and restores
 * all three and the step count.  Errors: TC_ERR_IO. */
TC_API tc_status tc_trainer_save(tc_trainer *t, const char *path);
TC_API tc_status tc_trainer_load(tc_trainer *t, const char *path);

/* Writes the current master weights as a TCW1 weight file for tc_create_stream. */
TC_API tc_status tc_trainer_export_weights(tc_trainer *t, const char *path);

TC_API const char *tc_trainer_last_error(const tc_trainer *t);
TC_API tc_status tc_trainer_destroy(tc_trainer *t);

/* ---- stage backward passes (float32, device buffers, enqueued on cuda_stream; they
 * allocate temporary device memory and wait for completion) ---------------------------- */

/* 3x3 conv of tc_op_conv3x3 (pad 1, stride 1 or 2, bias, optional LeakyReLU 0.1): given
 * its input x (n, h, w, cin), DEVICE weights w_oihw (cout, cin, 3, 3), its output y (n, ho,
 * wo, cout) and the output gradient dy (same shape), writes dx (n, h, w, cin; may be NULL),
 * dw (cout, cin, 3, 3) and db (cout) (device; may be NULL).  cin, cout >= 1. */
TC_API tc_status tc_op_conv3x3_backward(const float *x, int n, int h, int w, int cin, const float *w_oihw,
                                        int cout, int stride, int leaky, const float *y, const float *dy, float *dx,
                                        float *dw, float *db, void *cuda_stream);

/* Correlation of tc_op_correlation: given f1, f2 (n, h, w, c), its output cost (n, h, w,
 * (2r+1)^2) and dcost, writes df1, df2 (n, h, w, c; either may be NULL).  c % 4 == 0. */
TC_API tc_status tc_op_correlation_backward(const float *f1, const float *f2, int n, int h, int w, int c, int r,
                                            const float *cost, const float *dcost, float *df1, float *df2,
                                            void *cuda_stream);

/* Feature warp of tc_op_warp_features: given f (n, h, w, c), flow (n, h, w, 2) and dout
 * (n, h, w, c), writes df (n, h, w, c) and dflow (n, h, w, 2) (either may be NULL).  The
 * bilinear weights are differentiated inside a cell (a flow with an integer component sits
 * on a kink; the right-hand derivative is returned).  c % 4 == 0. */
TC_API tc_status tc_op_warp_features_backward(const float *f, const float *flow, int n, int h, int w, int c,
                                              const float *dout, float *df, float *dflow, void *cuda_stream);

/* Flow upsampling of tc_op_upsample_flow: given dfine (n, s h, s w, 2), writes dcoarse
 * (n, h, w, 2). */
TC_API tc_status tc_op_upsample_flow_backward(const float *dfine, int n, int h, int w, int s, float *dcoarse,
                                              void *cuda_stream);

/* Brute-force integer flow (the training fallback and the yardstick of learned flows): for
 * every pixel of a the displacement d in [-r, r]^2 minimising the sum over a 3x3 patch and
 * the c channels of (a(x+p) - b(x+p+d))^2, border-clamped, ties to the smaller |d|^2 then
 * the smaller index; writes k = (dy+r)(2r+1) + (dx+r) per pixel to k_out (h, w) int32.
 * a, b: device planar (c, h, w) float32.  1 <= r <= 32. */
TC_API tc_status tc_op_bruteforce_flow(const float *a, const float *b, int c, int h, int w, int r, int *k_out,
                                       void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* TC_TRAIN_H */
