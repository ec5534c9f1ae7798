/*
 * tc_stream.h -- C ABI of the per-frame hot path of "Interactive Control over Temporal
 * Consistency while Stylizing Video Streams" (arXiv 2301.00750), for NVIDIA B300 (sm_103a).
 *
 * For each new frame I_t of a video stream and its per-frame stylised version P_t, the
 * library computes the temporally consistent output O_t (Sec. 3.1, problem statement):
 *   1. the lite optical-flow network (Sec. 3.2): feature pyramid, correlation cost volume,
 *      bilinear feature warping and coarse-to-fine flow estimators, run in both directions
 *      between frames t and t-1;
 *   2. backward warping of I_{t-1}, P_{t-1}, O_{t-1} along F_{t->t-1} (the warping function
 *      Gamma of Sec. 3.1), a forward-backward non-occlusion mask (the mask used with the
 *      warping error, Eq. 9), the photometric weight w_p (Eq. 3, clamped to [0, k1]), the
 *      local and global consistency images L_t, G_t (Eqs. 2, 4), their adaptive blend A_t
 *      (Eq. 5), the warped input A^I_t (Eq. 6) and the consistency weight w_c (Eq. 7).
 *   O_t := A_t (causal form: no next frame, w_n = 0; the screened-Poisson solve of Eq. 1 is
 *   not part of this path).  The first frame of a stream returns O_1 = P_1.
 *
 * Conventions
 *   - Images are planar CHW float32, 3 channels (RGB), values nominally in [0, 1].
 *   - Flows are float32 displacements in pixels, F_{a->b}(x) with I_a(x) ~ I_b(x + F(x)).
 *   - "device" pointers are CUDA device (or managed) memory on the stream's device;
 *     "host" pointers are CPU memory (pinned memory gives asynchronous copies).
 *   - cuda_stream is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *   - Every call returns a tc_status and never aborts the process.  After a CUDA error a
 *     stream is poisoned: later calls return TC_ERR_STATE.  tc_last_error() describes the
 *     last failure of a stream (or of the last stream-less call when passed NULL).
 *   - One stream object must not be used from two host threads at once; distinct stream
 *     objects are independent and may run concurrently.
 *
 * Precision: TC_FP32 runs every stage in float32.  TC_BF16 runs the convolutions and the
 * correlation with bfloat16 operands and float32 accumulation; flow coordinates, feature
 * warp interpolation weights, the mask thresholds and the consistency step stay float32.
 * TC_FP16 is TC_BF16 with IEEE half (11 significant bits instead of 8) for the weights and
 * the stored activations: the same tensor-core kernels and rate, about a quarter of
 * TC_BF16's deviation from the float32 flows.  Activations must stay below 65504 in
 * magnitude (the network's are O(10)); tiny ones lose relative precision below 6.1e-5.
 * TC_FP8_E4M3 stores every network activation as e4m3 with one float scale per activation
 * segment (see tc_set_fp8_scales) and every weight as e4m3 with one scale per output
 * channel; the products accumulate in float32 on the tensor cores.  The flows, the
 * residual base flow and the consistency step stay float32.  The paper runs in float32
 * (Sec. 4); this precision has no counterpart there.
 */
#ifndef TC_STREAM_H
#define TC_STREAM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TC_API __attribute__((visibility("default")))
#else
#define TC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tc_stream tc_stream;   /* opaque, owned by the library */

typedef enum {
    TC_OK = 0,
    TC_ERR_INVALID_ARG = 1,   /* a NULL pointer, a bad size, a value out of range */
    TC_ERR_OOM = 2,           /* device or host allocation failed */
    TC_ERR_CUDA = 3,          /* a CUDA runtime call or kernel launch failed */
    TC_ERR_BUSY = 4,          /* resource in use (reserved) */
    TC_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up */
    TC_ERR_STATE = 6,         /* the stream is poisoned by an earlier CUDA error */
    TC_ERR_IO = 7,            /* the weight file could not be read or parsed */
    TC_ERR_UNSUPPORTED = 8    /* the request is valid but not built in this library */
} tc_status;

typedef enum { TC_FP32 = 0, TC_BF16 = 1, TC_FP8_E4M3 = 2, TC_FP16 = 3 } tc_precision;

/* Consistency controls (Sec. 3.1 "Consistency Control Modes", values of Sec. 4.2).
 *   k1      upper clamp of w_p (Eq. 3); the global/local proportion of A_t.  [0, 1]
 *   k2      upper clamp of w_n (Eq. 3), the weight of the next frame; used only by streams
 *           with one frame of latency (tc_set_latency), where k1 + k2 < 1 is required;
 *           the causal path has w_n = 0.  [0, 1]
 *   alpha   sharpness of the photometric weights (Eqs. 3, 7).  >= 0
 *   lambda  scale of the consistency weight w_c (Eq. 7).  >= 0
 *   fb_check, fb_c1, fb_c2: forward-backward occlusion test
 *           |Fb + Ff~|^2 > c1 (|Fb|^2 + |Ff~|^2) + c2 marks a pixel occluded (mask 0).
 *   solver_iters, eta, kappa: the screened-Poisson solve of Eq. 1 by the SGD-momentum
 *           iteration of Eq. 8 (Sec. 3.1 "Optimization Solver"): solver_iters = 0 (default)
 *           returns O_t = A_t (the causal blend); solver_iters > 0 (the paper uses 150)
 *           runs that many iterations from O = A_t with step eta (> 0, paper 0.15) and
 *           momentum kappa (in [0, 1), paper 0.2), and O_t (also the next frame's O_{t-1})
 *           is the last iterate.  The gradient is Lg (O - P_t) + w_c (O - A_t), Lg the
 *           4-neighbour graph Laplacian with Neumann boundary; w_c of Eq. 7 weighs the
 *           pull toward A_t, so lambda now matters (the iteration is stable for
 *           eta (8 + lambda) < 2 (1 + kappa)). */
typedef struct {
    float k1, k2, alpha, lambda;
    int fb_check;
    float fb_c1, fb_c2;
    int solver_iters;
    float eta, kappa;
} tc_consistency;

/* Stream description.
 *   width, height   frame size in pixels, each >= 2^levels of the network.
 *   precision       TC_FP32, TC_BF16, TC_FP16 or TC_FP8_E4M3 (the latter processes frames
 *                   only after tc_set_fp8_scales).
 *   weights_path    path of a 'TCW1' weight file, or NULL to use weights_blob.
 *   weights_blob    host pointer to the same bytes as such a file (copied at creation).
 * The weight file fixes the number of pyramid levels, the channel counts and the
 * correlation radius.  Its layout, little-endian: "TCW1"; int32 levels, radius,
 * chans[levels], decoder[4] (128,96,64,32), n_layers; per layer int32 cout, cin, stride,
 * leaky, float32 w[cout][cin][3][3], float32 b[cout].  Layer order: pyramid levels 1..L
 * (three convs each), then the estimators at levels L..2 (five convs each; conv4 reads
 * cat(x3, x2), conv5 reads cat(x4, x3)).  Magic "TCW2" adds a refinement network after
 * the level-2 estimator (Sec. 3.2 "-sepref"): int32 n_ref; per layer int32 cin, cout,
 * dilation, leaky, float32 dw[cin][3][3], db[cin], pw[cout][cin], pb[cout]; each layer is a
 * depthwise 3x3 conv with that dilation (zero padding, bias, no activation) and a pointwise
 * 1x1 conv (bias, LeakyReLU if leaky); the first reads cat(flow, x4, x3) of the level-2
 * estimator (cin = 2 + decoder[3] + decoder[2]), the last has cout = 2, no activation, and
 * is added to the level-2 flow.  Refinement networks run in TC_FP32, TC_BF16 and TC_FP16
 * streams.
 *   flow_downscale  0 or 1: the flow network runs on the frames as given.  2: it runs on the
 *                   frames downscaled by 2 (the mean of each 2 x 2 block, the last row and
 *                   column replicated for odd sizes) and its final flow is upsampled x8
 *                   (values x8) to the frame; everything else stays at full resolution.
 *                   With solver_iters = 50 this is the paper's fast preset (Sec. 4, Table 3:
 *                   flow on half-sized inputs, 50 iterations instead of 150).  The size
 *                   rule then applies to ceil(width / 2) and ceil(height / 2). */
typedef struct {
    int width, height;
    tc_precision precision;
    const char *weights_path;
    const void *weights_blob;
    size_t weights_bytes;
    int flow_downscale;
} tc_stream_desc;

/* Fills *p with the paper's final setting (Sec. 4.2: k1 = 0.3, k2 = 0.5, alpha = 6.5e3,
 * lambda = 2.0), the forward-backward test on with c1 = 0.01, c2 = 0.5, solver off. */
TC_API void tc_default_consistency(tc_consistency *p);

/* Creates a stream (Sec. 3.1: per-stream state I_{t-1}, P_{t-1}, O_{t-1} and the cached
 * feature pyramid of frame t-1 live on the device).  Allocates all device memory the
 * stream needs.  Errors: TC_ERR_INVALID_ARG (sizes, precision), TC_ERR_IO (weights),
 * TC_ERR_OOM, TC_ERR_CUDA.  On error *out is NULL. */
TC_API tc_status tc_create_stream(const tc_stream_desc *desc, void *cuda_stream, tc_stream **out);

/* Sets the consistency controls; they apply from the next tc_process_frame call.
 * Errors: TC_ERR_INVALID_ARG (k1 or k2 outside [0,1], k1 + k2 >= 1 on a stream with one
 * frame of latency, alpha or lambda negative, NaN, solver settings out of range). */
TC_API tc_status tc_set_consistency(tc_stream *s, const tc_consistency *p);

/* Processes the next frame.  I_t, P_t: device (3, H, W) float32, read only.  O_t: device
 * (3, H, W) float32, written.  wc_opt: device (H, W) float32 consistency weight w_c, or
 * NULL.  mask_opt: device (H, W) uint8 non-occlusion mask M (1 = usable), or NULL.
 * Work is enqueued on the stream's CUDA stream and the call returns without waiting; the
 * library copies what it keeps, so the caller may reuse I_t and P_t once that work has
 * completed.  On the first frame O_t = P_t, w_c = 0 and M = 0.
 * With one frame of latency (tc_set_latency(s, 1)) the frame given is frame t+1 and the
 * outputs are those of frame t, blended with both neighbours (Eqs. 2-7 with w_n); the
 * mask then has bit 0 for the previous frame's warp and bit 1 for the next frame's.  The
 * first call of a sequence writes no output; tc_last_output_frame tells which frame a
 * call wrote, and tc_flush returns the last frame. */
TC_API tc_status tc_process_frame(tc_stream *s, const float *I_t, const float *P_t, float *O_t,
                           float *wc_opt, uint8_t *mask_opt);

/* As tc_process_frame with HOST buffers: copies I_t, P_t to the device, runs the frame and
 * copies O_t (and the optional outputs) back, then waits for the stream.  The same
 * layouts as above; host pointers.  Pinned host memory makes the copies faster.  P_t is
 * uploaded on a second, library-owned stream while the flow network runs (only the
 * consistency pass reads it), so its copy overlaps the frame's kernels. */
TC_API tc_status tc_process_frame_host(tc_stream *s, const float *I_t, const float *P_t, float *O_t,
                                float *wc_opt, uint8_t *mask_opt);

/* Pipelined form of tc_process_frame_host for a stream of frames: enqueues the upload of
 * I_t, P_t, the frame, and the download of its outputs into O_t (and wc_opt, mask_opt),
 * then returns without waiting.  The next call's upload and this call's download run on
 * two library-owned copy streams while the neighbouring frames' kernels run (device staging
 * has two slots, four in pipelined mode, where the call works too: see tc_set_pipelined),
 * so the copies and the kernels overlap.  The host buffers
 * must stay valid, the inputs unmodified and the outputs unread, until tc_synchronize
 * returns; the copies overlap only from page-locked memory.  Same layouts and the same
 * one-frame-of-latency behaviour as tc_process_frame_host (the first call of a latency-1
 * sequence writes nothing; the last frame comes from tc_flush).  Errors as
 * tc_process_frame; device-side failures are reported by tc_synchronize. */
TC_API tc_status tc_process_frame_host_async(tc_stream *s, const float *I_t, const float *P_t, float *O_t,
                                             float *wc_opt, uint8_t *mask_opt);

/* tc_process_frame_host_async for 8-bit video frames, the form decoders produce and displays
 * take (Sec. 3.1: the method reads frames I_t, P_t and returns O_t; the paper fixes no pixel
 * format, this one moves a quarter of the float32 bytes over the host link).
 * I_t, P_t: HOST (H, W, 3) interleaved RGB, one byte per channel, row-major; code q stands
 * for the value q / 255 (IEEE float32 division).  O_t: HOST (H, W, 3) interleaved RGB bytes,
 * O quantised as floor(255 clamp(O, 0, 1) + 0.5) in float32 (product and sum rounded
 * separately).  wc_opt, mask_opt: HOST (H, W) float w_c and uint8 mask, or NULL.  Between
 * the conversions the frame is the one tc_process_frame computes from the decoded values,
 * so O_t equals the quantised float32 output of tc_process_frame_host_async given the
 * decoded frames.  Ordering, buffer lifetimes (valid and unmodified until tc_synchronize),
 * one frame of latency and errors as tc_process_frame_host_async, whose device staging
 * slots this call shares (the two may be interleaved in one sequence). */
TC_API tc_status tc_process_frame_host_rgb8_async(tc_stream *s, const uint8_t *I_t, const uint8_t *P_t,
                                                  uint8_t *O_t, float *wc_opt, uint8_t *mask_opt);

/* Pipelined mode (enable != 0) for sequences whose frames are all resident before they are
 * given: tc_process_frame then enqueues frame t on library-owned streams without ordering it
 * on the caller's stream, so the next frame's feature pyramid and two frames' flow
 * estimations run at the same time (the flow network estimates each frame pair on its own;
 * the stream keeps four pyramid slots and two sets of estimator and refinement buffers).  The inputs must be
 * valid when tc_process_frame is called and stay unmodified until the frame is done; the
 * outputs are valid after tc_join (the caller's stream then waits for every frame given)
 * or tc_synchronize.  tc_get_flows joins first; tc_flush runs after the frames given.
 * tc_process_frame_host_async and tc_process_frame_host_rgb8_async work in this mode too
 * (four device staging slots; each call's upload is fenced to the frame's pyramid and blend
 * streams and its download to the blend); tc_process_frame_host and amax recording do not.
 * Only before the first frame of a sequence; results equal those of the default mode bit
 * for bit.
 * Errors: TC_ERR_STATE (after the first frame of a sequence, or while recording amax). */
TC_API tc_status tc_set_pipelined(tc_stream *s, int enable);

/* Pipelined mode: makes the caller's stream wait for every frame given so far (no-op
 * otherwise). */
TC_API tc_status tc_join(tc_stream *s);

/* One frame of latency (Sec. 1, Sec. 3.1: the local term of Eq. 2 also warps the next
 * frame).  frames = 1: each tc_process_frame call with frame t+1 returns frame t, with w_n
 * of Eq. 3 (clamped to k2) and the next frame in L_t (Eq. 2) and A^I_t (Eq. 6); the flows
 * of the pair (t+1, t) computed for the call give F_{t->t+1} and F_{t+1->t}.  frames = 0
 * (default): the causal path (w_n = 0).  Only before the first frame of a sequence (a new
 * stream, or after tc_flush).  Errors: TC_ERR_INVALID_ARG (frames not 0 or 1; k1 + k2 >= 1
 * for frames = 1), TC_ERR_STATE (frames already processed), TC_ERR_OOM. */
TC_API tc_status tc_set_latency(tc_stream *s, int frames);

/* Streams with one frame of latency: writes the outputs of the last frame given (the
 * causal blend, as no next frame exists; O = P for a sequence of one frame) into O_t
 * (device (3, H, W) float32) and the optional wc_opt, mask_opt, and ends the sequence: the
 * next tc_process_frame starts a new one.  Enqueued on the stream's CUDA stream.
 * Errors: TC_ERR_STATE (no latency, or no frame pending), TC_ERR_INVALID_ARG (NULL O_t). */
TC_API tc_status tc_flush(tc_stream *s, float *O_t, float *wc_opt, uint8_t *mask_opt);

/* Index, within its sequence (0 = first frame), of the frame whose outputs the last
 * tc_process_frame / tc_flush call wrote; -1 if that call wrote none (the first call with
 * one frame of latency) or for s == NULL. */
TC_API long long tc_last_output_frame(const tc_stream *s);

/* CUDA graphs (on by default): from the third frame on, a stream replays one captured graph
 * per slot parity -- every launch of the frame in one cudaGraphLaunch -- after updating the
 * two kernel nodes that read the caller's buffers (in pipelined mode: three graphs per
 * frame, its pyramid's, its flow estimation's and its blend's).  enable = 0 returns to one
 * launch per kernel.  Waits for the stream.  Per-stage profiling always runs without graphs. */
TC_API tc_status tc_set_graphs(tc_stream *s, int enable);

/* ---- E4M3 calibration --------------------------------------------------------------
 * An activation segment is one group of channels that shares an e4m3 scale: for each
 * pyramid level l = 1..L the outputs of its three convs (index 3(l-1) + j, j = 0, 1, 2);
 * for each estimator level l = L..2 the six input groups of its decoder, cost volume,
 * up-sampled flow, x1, x2, x3, x4 (index 3L + 6(L-l) + k, k = 0..5).
 * tc_activation_segments(s) = 3L + 6(L-1); 0 for s == NULL. */
TC_API int tc_activation_segments(const tc_stream *s);

/* TC_FP32 / TC_BF16 / TC_FP16 streams: enable != 0 clears the record and from then on folds the
 * largest |value| of every activation segment of every processed frame into it (frames run
 * without graphs while recording).  enable = 0 stops recording and keeps the record.
 * Errors: TC_ERR_INVALID_ARG for a TC_FP8_E4M3 stream. */
TC_API tc_status tc_set_amax_recording(tc_stream *s, int enable);

/* Copies the record into amax[0 .. tc_activation_segments(s)) (host floats; n is the
 * array's length).  Waits for the stream. */
TC_API tc_status tc_get_amax(tc_stream *s, float *amax, int n);

/* TC_FP8_E4M3 streams: sets the scale of every activation segment (host array of exactly
 * tc_activation_segments(s) floats; an activation x is stored as e4m3(x / scale), so
 * amax / 448 uses the whole e4m3 range; 0 means "always zero" and is taken as 1).  Folds
 * the scales into the e4m3 weights and plans every layer and correlation on the tensor
 * cores; may be called again to re-calibrate.  Waits for the stream and drops its captured
 * graphs.  Errors: TC_ERR_INVALID_ARG (not e4m3, wrong n, negative or non-finite scale),
 * TC_ERR_UNSUPPORTED (a layer the e4m3 tensor-core kernels cannot take: every layer needs
 * cin and cout multiples of 16, cout <= 128). */
TC_API tc_status tc_set_fp8_scales(tc_stream *s, const float *scales, int n);

/* Static E4M3 activation scales from a calibration record (the reading of the supplement's
 * 8-bit linear quantisation used here): scales[i] = margin * amax[i] / 448, so the largest
 * calibrated |activation| of segment i, times margin, maps to the largest finite e4m3 value;
 * a segment whose amax is 0 gets scale 0 (tc_set_fp8_scales takes it as 1).  amax and
 * scales are host arrays of n floats (they may be the same array); margin > 0 and finite.
 * Pure host arithmetic: needs no device and no stream.  Errors: TC_ERR_INVALID_ARG (NULL
 * array, n < 1, margin not positive and finite, an amax negative or not finite). */
TC_API tc_status tc_fp8_scales_from_amax(const float *amax, int n, float margin, float *scales);

/* Writes the flows of the last processed frame at full resolution: Fb = F_{t->t-1} and
 * Ff = F_{t-1->t}, each device (2, H, W) float32 (planar u then v).  Either may be NULL.
 * Errors: TC_ERR_STATE before the second frame. */
TC_API tc_status tc_get_flows(tc_stream *s, float *Fb, float *Ff);

/* Waits for the stream's enqueued work (the copies of tc_process_frame_host_async
 * included) and reports device-side failures: TC_ERR_TIMEOUT
 * (and a poisoned stream) if a tensor-core kernel gave up on a bounded wait, TC_ERR_CUDA on
 * a CUDA error.  tc_process_frame_host performs the same check. */
TC_API tc_status tc_synchronize(tc_stream *s);

/* Number of convolution layers of s that run on the tensor cores (tcgen05), flow heads
 * included; 0 for TC_FP32 (and for TC_FP8_E4M3 before tc_set_fp8_scales). */
TC_API int tc_tensor_core_layers(const tc_stream *s);

/* Number of pyramid levels of s whose correlation runs on the tensor cores; 0 for TC_FP32. */
TC_API int tc_tensor_core_correlation_levels(const tc_stream *s);

/* Destroys a stream and frees its device memory (waits for its pending work). */
TC_API tc_status tc_destroy(tc_stream *s);

/* Human-readable description of the last error of s (s may be NULL for stream-less calls).
 * The string is owned by the library and valid until the next call on s. */
TC_API const char *tc_last_error(const tc_stream *s);

/* Number of kernel launches enqueued by the last tc_process_frame on s (for accounting). */
TC_API int tc_last_launch_count(const tc_stream *s);

/* Per-stage timing.  With profiling on, the library records a CUDA event pair around every
 * kernel it launches for s and adds the elapsed device time to the stage's total.
 * Categories (index into the arrays of tc_get_profile): */
enum {
    TC_PROF_PYRAMID_CONV = 0,    /* feature pyramid convolutions (Sec. 3.2) */
    TC_PROF_ESTIMATOR_CONV = 1,  /* estimator convolutions conv1..conv4 */
    TC_PROF_HEAD = 2,            /* flow head conv5 + residual */
    TC_PROF_CORRELATION = 3,     /* cost volume */
    TC_PROF_WARP = 4,            /* bilinear feature warp */
    TC_PROF_UPSAMPLE = 5,        /* x2 flow upsampling */
    TC_PROF_CONSISTENCY = 6,     /* fused warp + mask + blend (Eqs. 2-7) */
    TC_PROF_OTHER = 7,
    TC_PROF_SOLVER = 8,          /* screened-Poisson iterations (Eq. 8) and their output copy */
    TC_PROF_REFINE = 9,          /* the refinement network (TCW2 weights) */
    TC_PROF_CATEGORIES = 10
};

/* Turns per-stage timing on (enable != 0) or off and resets the totals. */
TC_API tc_status tc_set_profiling(tc_stream *s, int enable);

/* Waits for the recorded events and writes the per-category totals since the last
 * tc_set_profiling: ms[k] milliseconds and launches[k] (may be NULL) launch counts, for
 * k < n (n <= TC_PROF_CATEGORIES).  Host arrays. */
TC_API tc_status tc_get_profile(tc_stream *s, double *ms, long long *launches, int n);

/* ------------------------------------------------------------------------------------
 * Single-stage entry points.  Each runs one stage of the path on caller-owned device
 * buffers, enqueued on cuda_stream, and returns without waiting.  Feature maps are NHWC
 * float32 (n, h, w, c) contiguous; flows are (n, h, w, 2) float32 (u, v interleaved).
 * `precision` selects the arithmetic: TC_FP32, or TC_BF16 / TC_FP16 (inputs rounded to
 * bfloat16 / half on load, float32 accumulation, outputs rounded to the same type and
 * returned as float32).  These allocate temporary device
 * memory for reformatted weights where noted and free it before returning.
 * ---------------------------------------------------------------------------------- */

/* 3x3 convolution, zero padding 1, stride 1 or 2, bias, optional LeakyReLU(0.1)
 * (Sec. 3.2 pyramid and estimator layers).  in (n, h, w, cin); w_oihw, bias: HOST float32
 * (cout, cin, 3, 3) and (cout); out (n, (h-1)/stride+1, (w-1)/stride+1, cout).
 * Allocates temporary device memory for the weights, waits for completion.  cin, cout >= 1.
 * With TC_BF16 or TC_FP16 eligible layers run on the tensor cores (see
 * tc_op_last_used_tensor_cores).
 * TC_FP8_E4M3 (tensor cores only; cout <= 128, else TC_ERR_UNSUPPORTED): the input is
 * rounded to e4m3 as given (activation scale 1), each output channel's weights to e4m3
 * after dividing by s_o = max |w[o]| / 448, the products accumulate in float32, and
 * out = e4m3(LeakyReLU(s_o acc + bias)) (scale 1), returned as float32. */
TC_API tc_status tc_op_conv3x3(tc_precision precision, const float *in, int n, int h, int w, int cin,
                        const float *w_oihw, const float *bias, int cout, int stride, int leaky,
                        float *out, void *cuda_stream);

/* 1 if the last successful tc_op_conv3x3 or tc_op_correlation in this process ran on the
 * tensor cores, else 0.  TC_BF16 / TC_FP16 convs with cin a multiple of 8 and cout a
 * multiple of 16 up to 128, and TC_BF16 / TC_FP16 correlations with c a multiple of 8 up to
 * 128, do; TC_FP8_E4M3 ones always do. */
TC_API int tc_op_last_used_tensor_cores(void);

/* Cost volume (Sec. 3.2): out[n][y][x][k] = LeakyReLU((1/c) sum_ch f1[n][y][x][ch] *
 * f2[n][y+dy][x+dx][ch]), zero off the map, k = (dy+r)(2r+1) + (dx+r).  f1, f2
 * (n, h, w, c); out (n, h, w, (2r+1)^2).  1 <= r <= 4, c a multiple of 4.  TC_FP8_E4M3
 * (tensor cores only; c a multiple of 16 up to 128, else TC_ERR_UNSUPPORTED): f1, f2 rounded
 * to e4m3 as given, float32 accumulation, out = e4m3(LeakyReLU(sum / c)) (scale 1). */
TC_API tc_status tc_op_correlation(tc_precision precision, const float *f1, const float *f2, int n,
                            int h, int w, int c, int r, float *out, void *cuda_stream);

/* Bilinear backward warp of features with zeros off the map (Sec. 3.2 feature warping):
 * out[n][y][x] = sum of the bilinear taps of f[n] at (x + u, y + v) that lie on the map.
 * f (n, h, w, c), flow (n, h, w, 2), out (n, h, w, c).  c a multiple of 4.  TC_FP8_E4M3:
 * f rounded to e4m3 as given, float32 interpolation, out rounded to e4m3 (scale 1). */
TC_API tc_status tc_op_warp_features(tc_precision precision, const float *f, const float *flow, int n,
                              int h, int w, int c, float *out, void *cuda_stream);

/* Flow upsampling by s in {2, 4}: bilinear, half-pixel centres (sample positions clamped
 * at 0 and at the last row/column), values multiplied by s.  flow (n, h, w, 2) ->
 * out (n, s h, s w, 2).  h * w at most INT_MAX. */
TC_API tc_status tc_op_upsample_flow(const float *flow, int n, int h, int w, int s, float *out,
                              void *cuda_stream);

/* One layer of the refinement network with depthwise-separable convs (Sec. 3.2 "-sepref";
 * TCW2 weight files) on its own: out = LeakyReLU_if_leaky(pb + pw * (db + dw (*) in)), with
 * dw (*) the depthwise 3x3 conv of dilation dil (zero padding) and pw * the pointwise 1x1
 * conv.  in: device (n, h, w, cin) float32 NHWC, cin a multiple of 8 (<= 256); dw (cin, 3, 3),
 * db (cin), pw (cout, cin), pb (cout): host float32; cout a multiple of 8 (<= 256) written to
 * out (n, h, w, cout), or cout = 2 (the refinement's last layer, no activation) written as
 * float pairs.  precision TC_FP32 (CUDA cores) or TC_BF16 / TC_FP16 (activations rounded
 * to bfloat16 / half, pointwise conv on the tensor cores when eligible).  Allocates temporaries and waits. */
TC_API tc_status tc_op_sepconv(tc_precision precision, const float *in, int n, int h, int w, int cin,
                               const float *dw, const float *db, const float *pw, const float *pb, int cout,
                               int dil, int leaky, float *out, void *cuda_stream);

/* The flow input of flow_downscale = 2 alone: (c, h, w) -> (c, ceil(h/2), ceil(w/2)), each
 * output the mean of a 2 x 2 block of src, the last row and column replicated when h or w
 * is odd.  Device float32 planar buffers; enqueued on cuda_stream. */
TC_API tc_status tc_op_downscale2(const float *src, int c, int h, int w, float *dst, void *cuda_stream);

/* The consistency step alone (Sec. 3.1, Eqs. 2-7 with w_n = 0, O_t := A_t) on images of
 * h x w pixels.  It, Pt, Ip, Pp, Op: device (3, h, w) float32 (I_t, P_t, I_{t-1},
 * P_{t-1}, O_{t-1}).  Fb, Ff: device (fh, fw, 2) float32 flows at 1/scale resolution,
 * scale in {1, 2, 4, ...} (1 = full resolution, fh = h, fw = w); they are upsampled on
 * the fly as by tc_op_upsample_flow and read on the h x w crop.  Requires fh * scale >= h,
 * fw * scale >= w, and h * w and fh * fw at most INT_MAX.  O: device (3, h, w); wc_opt
 * (h, w) float32 or NULL; mask_opt (h, w) uint8 or NULL.  Ip, Pp, Op are first packed into
 * the interleaved per-pixel layout a stream keeps of its previous frame (temporary device
 * memory), and the call waits for completion. */
TC_API tc_status tc_op_consistency(const float *It, const float *Pt, const float *Ip, const float *Pp,
                            const float *Op, const float *Fb, const float *Ff, int h, int w,
                            int fh, int fw, int scale, const tc_consistency *p, float *O,
                            float *wc_opt, uint8_t *mask_opt, void *cuda_stream);

/* The consistency step with both temporal neighbours (Sec. 3.1, Eqs. 2-7 with w_n clamped
 * to k2): as tc_op_consistency, plus In, Pn: device (3, h, w) float32 (I_{t+1}, P_{t+1})
 * and Fn = F_{t->t+1}, Fnb = F_{t+1->t}: device (fh, fw, 2) float32 at the same 1/scale
 * resolution; Fn warps the next frame and Fnb is its forward-backward test.  mask_opt
 * receives bit 0 for M_p and bit 1 for M_n.  Errors: TC_ERR_INVALID_ARG as
 * tc_op_consistency, and k1 + k2 >= 1. */
TC_API tc_status tc_op_consistency_next(const float *It, const float *Pt, const float *Ip, const float *Pp,
                                        const float *Op, const float *Fb, const float *Ff, const float *In,
                                        const float *Pn, const float *Fn, const float *Fnb, int h, int w,
                                        int fh, int fw, int scale, const tc_consistency *p, float *O,
                                        float *wc_opt, uint8_t *mask_opt, void *cuda_stream);

/* The screened-Poisson solve of tc_consistency.solver_iters on its own: from O = A, `iters`
 * iterations of O <- O - eta (Lg (O - P) + wc (O - A)) + kappa (O - O_prev) (Eq. 1, Eq. 8,
 * Lg the 4-neighbour graph Laplacian, Neumann boundary).  P, A, O: device (c, h, w)
 * float32 planar, c = 1 or 3; wc: device (h, w).  Allocates temporary device memory and
 * waits for completion. */
TC_API tc_status tc_op_poisson_solve(const float *P, const float *A, const float *wc, int c, int h, int w,
                                     int iters, float eta, float kappa, float *O, void *cuda_stream);

/* Device bytes held by s (its buffers, packed weights and host-entry staging; the solver's
 * buffers, about 7 x 3 x H x W floats, once solver_iters was first set > 0; the kept flows
 * of one frame of latency, H x W / 4 floats, once tc_set_latency(s, 1) was called). */
TC_API size_t tc_stream_device_bytes(const tc_stream *s);

/* ------------------------------------------------------------------------------------
 * Multi-stream server.  Many concurrent streams (each with its own state on the device, as
 * Sec. 3.1 requires: I_{t-1}, P_{t-1}, O_{t-1} and the cached pyramid) of mixed
 * resolutions share one GPU.  Streams of one resolution are lanes of a shared batch
 * (tc_create_batch) of batch_lanes lanes; admission reserves a batch's device memory
 * against an HBM budget when a stream finds no free lane of its size.  Frames are
 * submitted with host buffers and run, in order per stream, by a pool of worker threads:
 * a free worker takes the batch with the oldest queued frame and runs the next frame of
 * every lane of it that has one as one batched step (their pyramids and flow estimations
 * in shared launches, replayed as CUDA graphs); frames that arrive meanwhile join the next
 * step (continuous batching), and different batches run at the same time on their own CUDA
 * streams.  A stream's results are the same whichever other streams share its steps.
 * ---------------------------------------------------------------------------------- */
typedef struct tc_server tc_server;

typedef struct {
    tc_precision precision;          /* TC_FP32, TC_BF16 or TC_FP16 for every stream */
    const char *weights_path;        /* TCW1 file, or NULL and weights_blob (copied) */
    const void *weights_blob;
    size_t weights_bytes;
    size_t hbm_budget_bytes;         /* device bytes the streams may hold together; 0 = unlimited */
    int workers;                     /* batched steps in flight at once, 1..64 */
    int max_streams;                 /* stream slots, >= 1 */
    int batch_lanes;                 /* streams per shared batch, 0..64 (0 or 1: a batch per stream) */
} tc_server_desc;

typedef struct {
    int stream_id;
    long long frame;                 /* index of the frame within its stream (0-based) */
    unsigned long long tag;          /* as passed to tc_server_submit */
    tc_status status;                /* TC_OK, TC_ERR_STATE if cancelled, or the frame's error */
    double queued_us, gpu_us, total_us;  /* submit -> start, start -> done, submit -> done */
    int batch;                       /* frames run by the step that ran this one */
} tc_completion;

/* Creates a server and its worker threads on the current device. */
TC_API tc_status tc_server_create(const tc_server_desc *desc, tc_server **out);

/* Device bytes a batch of width x height (batch_lanes lanes and its float and 8-bit staging)
 * holds: the admission charge of a stream that finds no free lane of its size. */
TC_API size_t tc_server_stream_bytes(const tc_server *srv, int width, int height);

/* Device bytes currently reserved by admitted streams. */
TC_API size_t tc_server_bytes_in_use(const tc_server *srv);

/* Admits a stream: TC_OK and *stream_id > 0, or TC_ERR_BUSY when every slot is taken or the
 * stream would exceed the HBM budget (nothing is allocated then; retry after a close). */
TC_API tc_status tc_server_open(tc_server *srv, int width, int height, int *stream_id);

/* Consistency controls of one stream, applied from its next frame to run.  Served streams
 * run the causal path: solver_iters must be 0 (TC_ERR_UNSUPPORTED otherwise; the admission
 * charge does not cover the solver's buffers). */
TC_API tc_status tc_server_set_consistency(tc_server *srv, int stream_id, const tc_consistency *p);

/* Queues the next frame of a stream.  I_host, P_host: host (3, H, W) float32; O_host: host
 * output, written before the frame's completion is reported.  The caller keeps all three
 * alive and unchanged until then (pinned memory makes the copies faster). */
TC_API tc_status tc_server_submit(tc_server *srv, int stream_id, const float *I_host, const float *P_host,
                                 float *O_host, unsigned long long tag);

/* tc_server_submit for 8-bit frames: I_host, P_host, O_host are host (H, W, 3) interleaved
 * RGB bytes, decoded and quantised on the device exactly as tc_process_frame_host_rgb8_async
 * does (Sec. 3.1 fixes no pixel format; this one moves a quarter of the bytes over the host
 * link).  A stream may mix both forms of submission.  Same lifetimes and errors. */
TC_API tc_status tc_server_submit_rgb8(tc_server *srv, int stream_id, const uint8_t *I_host, const uint8_t *P_host,
                                      uint8_t *O_host, unsigned long long tag);

/* Copies up to max finished frames into out, waiting up to timeout_ms for the first one;
 * returns how many. */
TC_API int tc_server_poll(tc_server *srv, tc_completion *out, int max, int timeout_ms);

/* Drops the stream's queued frames (each reported with status TC_ERR_STATE). */
TC_API tc_status tc_server_cancel(tc_server *srv, int stream_id);

/* Waits for the stream's queued frames, then frees its slot and device memory. */
TC_API tc_status tc_server_close(tc_server *srv, int stream_id);

/* Cancels every queued frame, stops the workers and frees everything. */
TC_API tc_status tc_server_destroy(tc_server *srv);

/* Per-frame latency in pipelined mode (tc_set_pipelined), where frames overlap and the
 * caller's stream sees no per-frame order: enable != 0 starts a record (cleared) of, for
 * every frame given from now on, the device time from the moment its feature pyramid may
 * start (its own stream past the waits for the frames it depends on) to the end of its
 * blend.  Two timing events per frame; 0 stops recording. */
TC_API tc_status tc_set_frame_timing(tc_stream *s, int enable);

/* Waits for the last recorded frame, then copies the first min(n, recorded) latencies (ms,
 * host floats) to ms and the number recorded to *count. */
TC_API tc_status tc_get_frame_times(tc_stream *s, float *ms, int n, int *count);

/* ------------------------------------------------------------------------------------
 * Batches: `lanes` independent streams of one size whose networks run in shared launches.
 * The serving problem of Sec. 3.1 (many streams, each with its own per-frame state) at a
 * load where several streams have a frame ready at once: their feature pyramids and flow
 * estimations run as one launch per layer over every lane's images (both directions of
 * every lane in the estimators) instead of one launch per stream.  Each lane is a causal
 * stream of its own (O_1 = P_1, then Eqs. 2-7 with w_n = 0 and O_t := A_t): its own frame
 * count, state (I, P, O of its previous frame) and consistency controls; a lane's results
 * are those of a tc_create_stream stream given the same frames, bit for bit, whichever other
 * lanes run in the same step.  TC_FP32, TC_BF16 or TC_FP16; no solver, one frame of
 * latency, fast preset or refinement network (TC_ERR_UNSUPPORTED), and the stream-only
 * calls (tc_process_frame*, tc_get_flows, tc_set_pipelined, ...) answer TC_ERR_STATE.
 * ---------------------------------------------------------------------------------- */

/* Creates a batch of 1 <= lanes <= 64 lanes (desc as for tc_create_stream; flow_downscale
 * 0 or 1).  Every lane starts at its first frame with the default controls.  Device memory:
 * about `lanes` times a stream's, without the host-entry staging. */
TC_API tc_status tc_create_batch(const tc_stream_desc *desc, int lanes, void *cuda_stream, tc_stream **out);

/* One frame for each of n distinct lanes (lanes[k] in [0, lanes)): device planar (3, H, W)
 * float32 I_t[k], P_t[k] in, O_t[k] out (caller-owned, as tc_process_frame), w_c and mask
 * optional (wc_opt / mask_opt NULL, or arrays whose entries may be NULL).  The pyramids and
 * flow estimations of lanes min(lanes) .. max(lanes) run in shared launches (the range's
 * launches are captured into a CUDA graph on its second use and replayed from then on);
 * lanes inside that range without a frame in this step are computed too, but keep their
 * state.  Enqueued on the batch's CUDA stream; returns without waiting. */
TC_API tc_status tc_process_lanes(tc_stream *s, int n, const int *lanes, const float *const *I_t,
                                  const float *const *P_t, float *const *O_t, float *const *wc_opt,
                                  uint8_t *const *mask_opt);

/* Consistency controls of one lane (tc_set_consistency on a batch sets every lane's).
 * solver_iters must be 0. */
TC_API tc_status tc_set_lane_consistency(tc_stream *s, int lane, const tc_consistency *p);

/* The lane's next frame is a first frame (a new stream takes the lane); its controls go
 * back to the defaults. */
TC_API tc_status tc_reset_lane(tc_stream *s, int lane);

/* The lane's flows of its last frame pair, as tc_get_flows (device (2, H, W) float32 each,
 * NULL to skip); TC_ERR_STATE before its second frame. */
TC_API tc_status tc_get_lane_flows(tc_stream *s, int lane, float *Fb, float *Ff);

/* ------------------------------------------------------------------------------------
 * Failure injection, for tests of the error paths only (process-wide; not for use in
 * production).  Neither faults nor hangs the device: the failures are made on the host, or
 * are a kernel that issues no work and whose bounded waits then run out.
 * ---------------------------------------------------------------------------------- */

/* The next `count` stride-1 tensor-core convolution launches made eagerly (not while the
 * launching stream is being captured into a CUDA graph; a stream with graphs replays its
 * captured launches from the third frame on, see tc_set_graphs) issue none of their loads:
 * every CTA's MMA issuer waits for operands that never arrive until the wait limit (2 s),
 * records a code in the stream's device error word, and the CTA frees its tensor memory
 * and exits.  The stream then reports TC_ERR_TIMEOUT at tc_synchronize and is poisoned
 * (later calls: TC_ERR_STATE).  count <= 0 disarms. */
TC_API void tc_test_stall_next_convs(int count);

/* The nth stream device allocation from now (nth >= 1; allocations of tc_create_stream and
 * of the host-buffer entry points) fails as an out-of-memory cudaMalloc would, so the call
 * returns TC_ERR_OOM after freeing what it had allocated.  nth <= 0 disarms. */
TC_API void tc_test_fail_device_allocation(long long nth);

/* ------------------------------------------------------------------------------------
 * Allocation-free variant.  The paper has no counterpart: this entry point exists for hosts
 * that cannot let the library allocate device memory -- an application whose memory pool
 * has reserved the device memory up front and passes only pre-allocated buffers, or a
 * real-time loop that cannot afford cudaMalloc/cudaFree (both may synchronise the device).
 * ---------------------------------------------------------------------------------- */

/* Size of the fixed device staging array behind tc_op_correlation_bf16_noalloc.  Every GPU
 * that loads the library holds it until the process exits. */
#define TC_NOALLOC_SCRATCH_BYTES (16u << 20)

/* Same result as tc_op_correlation(TC_BF16, f1, f2, n, h, w, c, r, out, cuda_stream) -- the
 * bfloat16 cost volume returned as float32, bit for bit: the same kernels run (the
 * tensor-core correlation when c is a multiple of 8 up to 128, else the CUDA-core one, as
 * tc_op_last_used_tensor_cores then reports) -- but it allocates nothing: the bfloat16
 * copies of f1, f2 and of the cost volume, and the tensor-core kernel's error word, live in
 * a fixed array of TC_NOALLOC_SCRATCH_BYTES in device memory instead of temporary buffers.
 * Same arguments, layouts and limits as tc_op_correlation (device NHWC float32 inputs,
 * output (n, h, w, (2r+1)^2) float32).
 *   - Sizes: requires 2 * align256(2 n h w c) + align256(2 n h w (2r+1)^2) + 256 <=
 *     TC_NOALLOC_SCRATCH_BYTES, else TC_ERR_INVALID_ARG with the needed size in
 *     tc_last_error(NULL).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call before any
 *     stream capture (a first call on a capturing stream returns TC_ERR_UNSUPPORTED).
 *   - Every call on a device shares the one array, which keeps the last call's contents
 *     (each call writes every staged byte it reads and clears the error word first).  Calls
 *     whose work overlaps on the GPU (other streams, other host threads) race on it: order
 *     them on one stream or synchronise between them.
 *   - Enqueued on cuda_stream; like tc_op_correlation it waits for completion, and returns
 *     TC_ERR_TIMEOUT if a bounded tensor-core wait gave up. */
TC_API tc_status tc_op_correlation_bf16_noalloc(const float *f1, const float *f2, int n, int h, int w, int c,
                                               int r, float *out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* TC_STREAM_H */
