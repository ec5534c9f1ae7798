/*
 * FP64 CPU oracle for the per-frame hot path of "Interactive Control over Temporal
 * Consistency while Stylizing Video Streams" (arXiv 2301.00750).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct statement of
 * what the hot path computes.  Only the tests, the smoke check and the benchmark's CPU
 * baseline use it; the product library never links, loads or calls it, and it shares no
 * code, header or table with the CUDA path.
 *
 * Layout: every array is planar (C, H, W), row-major, double precision.
 * Flow fields are (2, H, W): component 0 = horizontal displacement u, 1 = vertical v, in
 * pixels, with the convention I_a(x) ~ I_b(x + F_{a->b}(x)).
 *
 * Every function is pinned by a CPU test against something other than itself (library
 * routines on tiny inputs, closed forms, invariants); none is "parity unpinned".
 *
 * Readings of points the paper leaves open (each is listed in the design notes):
 *  - warping function Gamma (Sec. 3.1, named only): bilinear, pixel centres on integer
 *    coordinates; for images the taps are clamped to the border, for network features the
 *    out-of-range taps contribute zero.
 *  - network (Sec. 3.2): PWC-style pyramid of 3x3 convs (first of each level stride 2),
 *    LeakyReLU(0.1) after every conv but the flow head, correlation averaged over channels
 *    followed by LeakyReLU, "light" estimators (dense links only in the last two layers) at
 *    every level but the finest, coarse-to-fine residual flow, bilinear x2 upsampling with
 *    half-pixel centres (values x2), final x4 upsampling.
 *  - occlusion mask: forward-backward consistency test (the non-occlusion mask used with
 *    the warping error of Eq. 9), multiplied into the photometric weight of Eq. 3.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_API __attribute__((visibility("default")))

static inline double lrelu(double v) { return v >= 0.0 ? v : 0.1 * v; }

/* 3x3 convolution, zero padding 1, stride s, bias, optional LeakyReLU(0.1).
 * out[o][y][x] = b[o] + sum_c sum_ky sum_kx w[o][c][ky][kx] * in[c][s*y+ky-1][s*x+kx-1]
 * (Sec. 3.2: the pyramid and estimators are plain conv layers).  ho = (h-1)/s + 1. */
ORC_API void orc_conv3x3(const double *in, int cin, int h, int w, const double *wt,
                         const double *bias, int cout, int stride, int leaky, double *out)
{
    const int ho = (h - 1) / stride + 1, wo = (w - 1) / stride + 1;
#pragma omp parallel for collapse(2) schedule(static)
    for (int o = 0; o < cout; ++o) {
        for (int y = 0; y < ho; ++y) {
            double *row = out + ((size_t)o * ho + y) * wo;
            for (int x = 0; x < wo; ++x) row[x] = bias ? bias[o] : 0.0;
            for (int c = 0; c < cin; ++c) {
                for (int ky = 0; ky < 3; ++ky) {
                    const int iy = stride * y + ky - 1;
                    if (iy < 0 || iy >= h) continue;
                    const double *irow = in + ((size_t)c * h + iy) * w;
                    for (int kx = 0; kx < 3; ++kx) {
                        const double wv = wt[(((size_t)o * cin + c) * 3 + ky) * 3 + kx];
                        int xlo = 0, xhi = wo;
                        while (xlo < wo && stride * xlo + kx - 1 < 0) ++xlo;
                        while (xhi > xlo && stride * (xhi - 1) + kx - 1 >= w) --xhi;
                        for (int x = xlo; x < xhi; ++x) row[x] += wv * irow[stride * x + kx - 1];
                    }
                }
            }
            if (leaky)
                for (int x = 0; x < wo; ++x) row[x] = lrelu(row[x]);
        }
    }
}

/* Bilinear sample of channel plane p (h x w) at (sx, sy); taps outside contribute zero
 * when zero_outside, else they are clamped to the border. */
static double bilinear(const double *p, int h, int w, double sx, double sy, int zero_outside)
{
    const double fx = floor(sx), fy = floor(sy);
    const double ax = sx - fx, ay = sy - fy;
    const long x0 = (long)fx, y0 = (long)fy;
    double acc = 0.0;
    for (int dy = 0; dy < 2; ++dy) {
        for (int dx = 0; dx < 2; ++dx) {
            long xx = x0 + dx, yy = y0 + dy;
            const double wgt = (dx ? ax : 1.0 - ax) * (dy ? ay : 1.0 - ay);
            if (zero_outside) {
                if (xx < 0 || xx >= w || yy < 0 || yy >= h) continue;
            } else {
                if (xx < 0) xx = 0;
                if (xx > w - 1) xx = w - 1;
                if (yy < 0) yy = 0;
                if (yy > h - 1) yy = h - 1;
            }
            acc += wgt * p[(size_t)yy * w + xx];
        }
    }
    return acc;
}

/* Backward warp Gamma_F(J)(x) = J(x + F(x)) by bilinear interpolation (Sec. 3.1, Eq. 2-4).
 * zero_outside = 1: feature warping inside the flow network (taps off the map are 0);
 * zero_outside = 0: image warping (taps clamped to the border).
 * If in_bounds is non-NULL it receives 1 where 0 <= x+u <= w-1 and 0 <= y+v <= h-1. */
ORC_API void orc_warp(const double *src, int c, int h, int w, const double *flow,
                      int zero_outside, double *out, unsigned char *in_bounds)
{
    const size_t hw = (size_t)h * w;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
            const size_t i = (size_t)y * w + x;
            const double sx = x + flow[i], sy = y + flow[hw + i];
            for (int k = 0; k < c; ++k)
                out[k * hw + i] = bilinear(src + k * hw, h, w, sx, sy, zero_outside);
            if (in_bounds)
                in_bounds[i] = (sx >= 0.0 && sx <= w - 1 && sy >= 0.0 && sy <= h - 1) ? 1 : 0;
        }
    }
}

/* Cost volume (Sec. 3.2 "correlation"): for displacement d = (dx, dy) in [-r, r]^2 and
 * channel index k = (dy + r)(2r + 1) + (dx + r),
 *   out[k][y][x] = LeakyReLU( (1/c) sum_ch f1[ch][y][x] * f2[ch][y+dy][x+dx] ),
 * with the product taken as zero where (x+dx, y+dy) is off the map. */
ORC_API void orc_correlation(const double *f1, const double *f2, int c, int h, int w, int r,
                             double *out)
{
    const int n = 2 * r + 1;
    const size_t hw = (size_t)h * w;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < n * n; ++k) {
        for (int y = 0; y < h; ++y) {
            const int dy = k / n - r, dx = k % n - r;
            for (int x = 0; x < w; ++x) {
                double s = 0.0;
                const int yy = y + dy, xx = x + dx;
                if (yy >= 0 && yy < h && xx >= 0 && xx < w)
                    for (int ch = 0; ch < c; ++ch)
                        s += f1[ch * hw + (size_t)y * w + x] * f2[ch * hw + (size_t)yy * w + xx];
                out[k * hw + (size_t)y * w + x] = lrelu(s / c);
            }
        }
    }
}

/* Source coordinate of output index d for an s-times upsampling with half-pixel centres,
 * clamped at 0 (the bilinear "align_corners = false" convention). */
static void up_src(int d, int s, int n, int *i0, int *i1, double *lam)
{
    double src = (d + 0.5) / s - 0.5;
    if (src < 0.0) src = 0.0;
    int a = (int)src;
    if (a > n - 1) a = n - 1;
    *i0 = a;
    *i1 = a < n - 1 ? a + 1 : a;
    *lam = src - a;
}

/* Flow upsampling by an integer factor s (Sec. 3.2 coarse-to-fine): bilinear resampling of
 * each component from (h, w) to (s h, s w) with half-pixel centres, values multiplied by s
 * so that the flow stays in pixels of the finer grid. */
ORC_API void orc_upsample_flow(const double *flow, int h, int w, int s, double *out)
{
    const int H = s * h, W = s * w;
    for (int k = 0; k < 2; ++k) {
        const double *p = flow + (size_t)k * h * w;
        double *q = out + (size_t)k * H * W;
        for (int Y = 0; Y < H; ++Y) {
            int y0, y1; double ly;
            up_src(Y, s, h, &y0, &y1, &ly);
            for (int X = 0; X < W; ++X) {
                int x0, x1; double lx;
                up_src(X, s, w, &x0, &x1, &lx);
                const double v = (1 - ly) * ((1 - lx) * p[y0 * w + x0] + lx * p[y0 * w + x1])
                               + ly * ((1 - lx) * p[y1 * w + x0] + lx * p[y1 * w + x1]);
                q[(size_t)Y * W + X] = s * v;
            }
        }
    }
}

/* Edge-replicate padding of a (c, h, w) image to (c, hp, wp), hp >= h, wp >= w. */
ORC_API void orc_pad_replicate(const double *img, int c, int h, int w, int hp, int wp, double *out)
{
    for (int k = 0; k < c; ++k)
        for (int y = 0; y < hp; ++y)
            for (int x = 0; x < wp; ++x)
                out[((size_t)k * hp + y) * wp + x] =
                    img[((size_t)k * h + (y < h ? y : h - 1)) * w + (x < w ? x : w - 1)];
}

/* One layer of the network as passed from the host. */
typedef struct {
    int cin, cout, stride, leaky;
    const double *w;   /* (cout, cin, 3, 3) */
    const double *b;   /* (cout) */
} orc_layer;

/* Feature pyramid (Sec. 3.2, kept from PWC-Net): level l = 1..L has three 3x3 convs, the
 * first with stride 2, all followed by LeakyReLU.  feat[l-1] receives level l at
 * (chans[l-1], h >> l, w >> l).  layers[3(l-1) + j] is conv j of level l. */
ORC_API void orc_pyramid(const double *img, int h, int w, int levels, const orc_layer *layers,
                         double **feat)
{
    const double *cur = img;
    int ch = h, cw = w;
    for (int l = 1; l <= levels; ++l) {
        const orc_layer *La = &layers[3 * (l - 1)];
        const int nh = (ch - 1) / 2 + 1, nw = (cw - 1) / 2 + 1;
        double *t0 = malloc(sizeof(double) * La[0].cout * nh * nw);
        double *t1 = malloc(sizeof(double) * La[1].cout * nh * nw);
        orc_conv3x3(cur, La[0].cin, ch, cw, La[0].w, La[0].b, La[0].cout, 2, La[0].leaky, t0);
        orc_conv3x3(t0, La[1].cin, nh, nw, La[1].w, La[1].b, La[1].cout, 1, La[1].leaky, t1);
        orc_conv3x3(t1, La[2].cin, nh, nw, La[2].w, La[2].b, La[2].cout, 1, La[2].leaky, feat[l - 1]);
        free(t0);
        free(t1);
        cur = feat[l - 1];
        ch = nh;
        cw = nw;
    }
}

/* One depthwise-separable layer of the refinement network (Sec. 3.2 "-sepref"):
 * a depthwise 3x3 conv with dilation dil (per channel, zero padding, bias, no activation)
 * followed by a pointwise 1x1 conv (bias, LeakyReLU 0.1 if leaky). */
typedef struct {
    int cin, cout, dil, leaky;
    const double *dw;  /* (cin, 3, 3) */
    const double *db;  /* (cin) */
    const double *pw;  /* (cout, cin) */
    const double *pb;  /* (cout) */
} orc_sep_layer;

/* Depthwise 3x3 conv with dilation dil: out[c](y, x) = db[c] + sum over ky, kx of
 * dw[c][ky][kx] x[c](y + (ky - 1) dil, x + (kx - 1) dil), taps off the map are 0. */
ORC_API void orc_depthwise3x3(const double *x, int c, int h, int w, const double *dw, const double *db, int dil,
                              double *out)
{
    const size_t hw = (size_t)h * w;
#pragma omp parallel for schedule(static)
    for (int ch = 0; ch < c; ++ch)
        for (int y = 0; y < h; ++y)
            for (int xx = 0; xx < w; ++xx) {
                double acc = db ? db[ch] : 0.0;
                for (int ky = 0; ky < 3; ++ky) {
                    const int sy = y + (ky - 1) * dil;
                    if (sy < 0 || sy >= h) continue;
                    for (int kx = 0; kx < 3; ++kx) {
                        const int sx = xx + (kx - 1) * dil;
                        if (sx < 0 || sx >= w) continue;
                        acc += dw[ch * 9 + ky * 3 + kx] * x[ch * hw + (size_t)sy * w + sx];
                    }
                }
                out[ch * hw + (size_t)y * w + xx] = acc;
            }
}

/* Pointwise 1x1 conv: out[o] = pb[o] + sum_c pw[o][c] x[c], LeakyReLU 0.1 if leaky. */
ORC_API void orc_pointwise(const double *x, int cin, int h, int w, const double *pw, const double *pb, int cout,
                           int leaky, double *out)
{
    const size_t hw = (size_t)h * w;
#pragma omp parallel for schedule(static)
    for (int o = 0; o < cout; ++o)
        for (size_t i = 0; i < hw; ++i) {
            double acc = pb ? pb[o] : 0.0;
            for (int c = 0; c < cin; ++c) acc += pw[(size_t)o * cin + c] * x[c * hw + i];
            out[o * hw + i] = leaky && acc < 0.0 ? 0.1 * acc : acc;
        }
}

/* Refinement of the finest flow (Sec. 3.2, "-sepref": the refinement network with
 * depthwise-separable convs): the input is cat(flow, x4, x3) of the level-2 estimator (the
 * flow head's input, after the flow), the layers run in order, and the last layer's two
 * outputs are added to the flow: out = flow + ref(cat(flow, x4, x3)). */
ORC_API void orc_refine(const double *flow, const double *x4, int c4, const double *x3, int c3, int h, int w,
                        const orc_sep_layer *ref, int n, double *out)
{
    const size_t hw = (size_t)h * w;
    int c = 2 + c4 + c3;
    double *cur = malloc(sizeof(double) * c * hw);
    memcpy(cur, flow, sizeof(double) * 2 * hw);
    memcpy(cur + 2 * hw, x4, sizeof(double) * c4 * hw);
    memcpy(cur + (size_t)(2 + c4) * hw, x3, sizeof(double) * c3 * hw);
    for (int k = 0; k < n; ++k) {
        double *d = malloc(sizeof(double) * ref[k].cin * hw);
        double *p = malloc(sizeof(double) * ref[k].cout * hw);
        orc_depthwise3x3(cur, ref[k].cin, h, w, ref[k].dw, ref[k].db, ref[k].dil, d);
        orc_pointwise(d, ref[k].cin, h, w, ref[k].pw, ref[k].pb, ref[k].cout, ref[k].leaky, p);
        free(d);
        free(cur);
        cur = p;
        c = ref[k].cout;
    }
    for (size_t i = 0; i < 2 * hw; ++i) out[i] = flow[i] + cur[i];
    free(cur);
}

/* Concatenate planar blocks along the channel axis. */
static void cat2(const double *a, int ca, const double *b, int cb, size_t hw, double *out)
{
    memcpy(out, a, sizeof(double) * ca * hw);
    memcpy(out + (size_t)ca * hw, b, sizeof(double) * cb * hw);
}

/* Coarse-to-fine flow for one direction (Sec. 3.2, PWC-style "light" estimators at levels
 * L..2).  At level l:
 *   up   = 2x upsampled flow of level l+1 (zeros at the coarsest level),
 *   f2w  = feature map of the other frame warped by up (zeros off the map),
 *   cv   = correlation(f_self, f2w, r),
 *   x0   = cat(cv, f_self, up);  x1 = conv1(x0); x2 = conv2(x1); x3 = conv3(x2);
 *   x4   = conv4(cat(x3, x2));   res = conv5(cat(x4, x3))   (no activation on conv5),
 *   flow = up + res.
 * With a refinement network (n_ref > 0) the flow of level 2 is refined by orc_refine from
 * that level's flow, x4 and x3.  The flow of level 2 is upsampled 4x to the padded input
 * resolution into flow_out (2, h, w).  est[5 (L - l) + j] is conv j+1 of the estimator at
 * level l.  If level_flows is non-NULL, level_flows[l-2] receives flow of level l,
 * (2, h>>l, w>>l) (the refined one at level 2). */
ORC_API void orc_flow2(double *const *feat_self, double *const *feat_other, const int *chans,
                       int h, int w, int levels, int r, const orc_layer *est, double *flow_out,
                       double **level_flows, const orc_sep_layer *ref, int n_ref)
{
    const int nd = (2 * r + 1) * (2 * r + 1);
    double *prev = NULL;
    int ph = 0, pw = 0;
    for (int l = levels; l >= 2; --l) {
        const int lh = h >> l, lw = w >> l, cl = chans[l - 1];
        const size_t hw = (size_t)lh * lw;
        const orc_layer *E = &est[5 * (levels - l)];
        double *up = calloc(2 * hw, sizeof(double));
        double *f2w = malloc(sizeof(double) * cl * hw);
        if (prev) {
            orc_upsample_flow(prev, ph, pw, 2, up);
            orc_warp(feat_other[l - 1], cl, lh, lw, up, 1, f2w, NULL);
        } else {
            memcpy(f2w, feat_other[l - 1], sizeof(double) * cl * hw);
        }
        const int c0 = nd + cl + 2;
        double *x0 = malloc(sizeof(double) * c0 * hw);
        orc_correlation(feat_self[l - 1], f2w, cl, lh, lw, r, x0);
        memcpy(x0 + (size_t)nd * hw, feat_self[l - 1], sizeof(double) * cl * hw);
        memcpy(x0 + (size_t)(nd + cl) * hw, up, sizeof(double) * 2 * hw);
        double *x1 = malloc(sizeof(double) * E[0].cout * hw);
        double *x2 = malloc(sizeof(double) * E[1].cout * hw);
        double *x3 = malloc(sizeof(double) * E[2].cout * hw);
        double *x32 = malloc(sizeof(double) * (E[2].cout + E[1].cout) * hw);
        double *x4 = malloc(sizeof(double) * E[3].cout * hw);
        double *x43 = malloc(sizeof(double) * (E[3].cout + E[2].cout) * hw);
        double *res = malloc(sizeof(double) * 2 * hw);
        orc_conv3x3(x0, E[0].cin, lh, lw, E[0].w, E[0].b, E[0].cout, 1, E[0].leaky, x1);
        orc_conv3x3(x1, E[1].cin, lh, lw, E[1].w, E[1].b, E[1].cout, 1, E[1].leaky, x2);
        orc_conv3x3(x2, E[2].cin, lh, lw, E[2].w, E[2].b, E[2].cout, 1, E[2].leaky, x3);
        cat2(x3, E[2].cout, x2, E[1].cout, hw, x32);
        orc_conv3x3(x32, E[3].cin, lh, lw, E[3].w, E[3].b, E[3].cout, 1, E[3].leaky, x4);
        cat2(x4, E[3].cout, x3, E[2].cout, hw, x43);
        orc_conv3x3(x43, E[4].cin, lh, lw, E[4].w, E[4].b, E[4].cout, 1, E[4].leaky, res);
        double *flow = malloc(sizeof(double) * 2 * hw);
        for (size_t i = 0; i < 2 * hw; ++i) flow[i] = up[i] + res[i];
        if (l == 2 && n_ref > 0) {
            double *refined = malloc(sizeof(double) * 2 * hw);
            orc_refine(flow, x4, E[3].cout, x3, E[2].cout, lh, lw, ref, n_ref, refined);
            free(flow);
            flow = refined;
        }
        if (level_flows) memcpy(level_flows[l - 2], flow, sizeof(double) * 2 * hw);
        free(up); free(f2w); free(x0); free(x1); free(x2); free(x3); free(x32);
        free(x4); free(x43); free(res); free(prev);
        prev = flow;
        ph = lh;
        pw = lw;
    }
    orc_upsample_flow(prev, ph, pw, 4, flow_out);
    free(prev);
}

/* orc_flow2 without a refinement network. */
ORC_API void orc_flow(double *const *feat_self, double *const *feat_other, const int *chans,
                      int h, int w, int levels, int r, const orc_layer *est, double *flow_out,
                      double **level_flows)
{
    orc_flow2(feat_self, feat_other, chans, h, w, levels, r, est, flow_out, level_flows, NULL, 0);
}

/* Consistency step of Sec. 3.1 in its causal form (no next frame, no solver), per pixel:
 *   Gamma = backward warp along Fb = F_{t->t-1} (bilinear, border clamp),
 *   M     = in_bounds and, if fb_check, not occluded by the forward-backward test
 *           |Fb + Ff~|^2 > c1 (|Fb|^2 + |Ff~|^2) + c2,  Ff~ = Gamma(Ff), Ff = F_{t-1->t},
 *   d     = sum_c (I_t - Gamma I_{t-1})^2,          w_p = M min(k1, exp(-alpha d))   (Eq. 3)
 *   L     = (1 - w_p) P_t + w_p Gamma P_{t-1}                                       (Eq. 2, w_n = 0)
 *   G     = Gamma O_{t-1}                                                           (Eq. 4)
 *   A     = w_p G + (1 - w_p) L                                                     (Eq. 5)
 *   A^I   = (1 - w_p) I_t + w_p Gamma I_{t-1}                                       (Eq. 6, w_n = 0)
 *   w_c   = lambda exp(-alpha sum_c (I_t - A^I)^2)                                  (Eq. 7)
 *   O_t   = A.
 * band[i] = 1 marks pixels whose occlusion decision lies within
 * 1e-6 (1 + |Fb|^2 + |Ff~|^2) of its threshold (FP32 rounding can flip those).
 * Images are (3, h, w); flows (2, h, w).  wp_out, band may be NULL. */
ORC_API void orc_consistency(int h, int w, const double *It, const double *Pt, const double *Ip,
                             const double *Pp, const double *Op, const double *Fb,
                             const double *Ff, double k1, double alpha, double lambda,
                             int fb_check, double c1, double c2, double *O, double *wc,
                             unsigned char *mask, unsigned char *band, double *wp_out)
{
    const size_t hw = (size_t)h * w;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
            const size_t i = (size_t)y * w + x;
            const double u = Fb[i], v = Fb[hw + i];
            const double sx = x + u, sy = y + v;
            const int inb = sx >= 0.0 && sx <= w - 1 && sy >= 0.0 && sy <= h - 1;
            int occ = 0, near = 0;
            if (fb_check) {
                const double fu = bilinear(Ff, h, w, sx, sy, 0);
                const double fv = bilinear(Ff + hw, h, w, sx, sy, 0);
                const double su = u + fu, sv = v + fv;
                const double nb = u * u + v * v, nf = fu * fu + fv * fv;
                const double lhs = su * su + sv * sv;
                const double rhs = c1 * (nb + nf) + c2;
                occ = lhs > rhs;
                near = fabs(lhs - rhs) <= 1e-6 * (1.0 + nb + nf);
            }
            const int m = inb && !occ;
            double gI[3], gP[3], gO[3], d = 0.0;
            for (int c = 0; c < 3; ++c) {
                gI[c] = bilinear(Ip + c * hw, h, w, sx, sy, 0);
                gP[c] = bilinear(Pp + c * hw, h, w, sx, sy, 0);
                gO[c] = bilinear(Op + c * hw, h, w, sx, sy, 0);
                const double e = It[c * hw + i] - gI[c];
                d += e * e;
            }
            double wp = 0.0;
            if (m) {
                wp = exp(-alpha * d);
                if (wp > k1) wp = k1;
            }
            double dI = 0.0;
            for (int c = 0; c < 3; ++c) {
                const double Lc = (1.0 - wp) * Pt[c * hw + i] + wp * gP[c];
                const double Ac = wp * gO[c] + (1.0 - wp) * Lc;
                const double AIc = (1.0 - wp) * It[c * hw + i] + wp * gI[c];
                const double e = It[c * hw + i] - AIc;
                dI += e * e;
                O[c * hw + i] = Ac;
            }
            if (wc) wc[i] = lambda * exp(-alpha * dI);
            if (mask) mask[i] = (unsigned char)m;
            if (band) band[i] = (unsigned char)near;
            if (wp_out) wp_out[i] = wp;
        }
    }
}

/* Validity of the warp of one neighbouring frame at pixel (x, y) along F (Sec. 3.1 with the
 * non-occlusion mask of reading R6): in bounds and, if fb_check, not occluded by the
 * forward-backward test against the opposite flow G sampled at x + F(x).  *near is set when
 * the occlusion decision lies within 1e-6 (1 + |F|^2 + |G~|^2) of its threshold. */
static int warp_valid(const double *F, const double *G, int h, int w, int x, int y, int fb_check,
                      double c1, double c2, int *near)
{
    const size_t hw = (size_t)h * w, i = (size_t)y * w + x;
    const double u = F[i], v = F[hw + i];
    const double sx = x + u, sy = y + v;
    const int inb = sx >= 0.0 && sx <= w - 1 && sy >= 0.0 && sy <= h - 1;
    int occ = 0;
    *near = 0;
    if (fb_check) {
        const double gu = bilinear(G, h, w, sx, sy, 0);
        const double gv = bilinear(G + hw, h, w, sx, sy, 0);
        const double su = u + gu, sv = v + gv;
        const double nf = u * u + v * v, ng = gu * gu + gv * gv;
        const double lhs = su * su + sv * sv, rhs = c1 * (nf + ng) + c2;
        occ = lhs > rhs;
        *near = fabs(lhs - rhs) <= 1e-6 * (1.0 + nf + ng);
    }
    return inb && !occ;
}

/* Consistency step of Sec. 3.1 with both temporal neighbours (one frame of latency), per
 * pixel of frame t:
 *   Gamma_p = backward warp along Fb = F_{t->t-1}, mask M_p from the test against
 *             Ff = F_{t-1->t};  Gamma_n = warp along Fn = F_{t->t+1}, mask M_n from the
 *             test against Fnb = F_{t+1->t} (bilinear, border clamp);
 *   w_p = M_p min(k1, exp(-alpha |I_t - Gamma_p I_{t-1}|^2)),
 *   w_n = M_n min(k2, exp(-alpha |I_t - Gamma_n I_{t+1}|^2))                         (Eq. 3)
 *   L   = (1 - (w_p + w_n)) P_t + w_p Gamma_p P_{t-1} + w_n Gamma_n P_{t+1}             (Eq. 2)
 *   G   = Gamma_p O_{t-1}                                                            (Eq. 4)
 *   A   = w_p G + (1 - w_p) L                                                        (Eq. 5)
 *   A^I = (1 - (w_p + w_n)) I_t + w_p Gamma_p I_{t-1} + w_n Gamma_n I_{t+1}             (Eq. 6)
 *   w_c = lambda exp(-alpha |I_t - A^I|^2)                                           (Eq. 7)
 * O = A; mask = M_p | M_n << 1; band bit 0 / bit 1 mark the decisions of M_p / M_n that
 * lie within FP32 rounding of their threshold.  Images (3, h, w), flows (2, h, w);
 * band, wp_out, wn_out may be NULL. */
ORC_API void orc_consistency_next(int h, int w, const double *It, const double *Pt, const double *Ip,
                                  const double *Pp, const double *Op, const double *Fb, const double *Ff,
                                  const double *In, const double *Pn, const double *Fn, const double *Fnb,
                                  double k1, double k2, double alpha, double lambda, int fb_check,
                                  double c1, double c2, double *O, double *wc, unsigned char *mask,
                                  unsigned char *band, double *wp_out, double *wn_out)
{
    const size_t hw = (size_t)h * w;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
            const size_t i = (size_t)y * w + x;
            int near_p, near_n;
            const int mp = warp_valid(Fb, Ff, h, w, x, y, fb_check, c1, c2, &near_p);
            const int mn = warp_valid(Fn, Fnb, h, w, x, y, fb_check, c1, c2, &near_n);
            const double px = x + Fb[i], py = y + Fb[hw + i];
            const double nx = x + Fn[i], ny = y + Fn[hw + i];
            double gIp[3], gPp[3], gOp[3], gIn[3], gPn[3], dp = 0.0, dn = 0.0;
            for (int c = 0; c < 3; ++c) {
                gIp[c] = bilinear(Ip + c * hw, h, w, px, py, 0);
                gPp[c] = bilinear(Pp + c * hw, h, w, px, py, 0);
                gOp[c] = bilinear(Op + c * hw, h, w, px, py, 0);
                gIn[c] = bilinear(In + c * hw, h, w, nx, ny, 0);
                gPn[c] = bilinear(Pn + c * hw, h, w, nx, ny, 0);
                const double ep = It[c * hw + i] - gIp[c], en = It[c * hw + i] - gIn[c];
                dp += ep * ep;
                dn += en * en;
            }
            double wp = 0.0, wn = 0.0;
            if (mp) {
                wp = exp(-alpha * dp);
                if (wp > k1) wp = k1;
            }
            if (mn) {
                wn = exp(-alpha * dn);
                if (wn > k2) wn = k2;
            }
            double dI = 0.0;
            for (int c = 0; c < 3; ++c) {
                const double Lc = (1.0 - (wp + wn)) * Pt[c * hw + i] + wp * gPp[c] + wn * gPn[c];
                const double Ac = wp * gOp[c] + (1.0 - wp) * Lc;
                const double AIc = (1.0 - (wp + wn)) * It[c * hw + i] + wp * gIp[c] + wn * gIn[c];
                const double e = It[c * hw + i] - AIc;
                dI += e * e;
                O[c * hw + i] = Ac;
            }
            if (wc) wc[i] = lambda * exp(-alpha * dI);
            if (mask) mask[i] = (unsigned char)(mp | (mn << 1));
            if (band) band[i] = (unsigned char)(near_p | (near_n << 1));
            if (wp_out) wp_out[i] = wp;
            if (wn_out) wn_out[i] = wn;
        }
    }
}

/* Integer-displacement flow by brute force: for each pixel the displacement d in [-r, r]^2
 * minimising the sum over a 3x3 patch and all channels of (a(x+p) - b(x+p+d))^2, with
 * border clamping; ties go to the smallest |d|^2 and then the smallest index
 * k = (dy + r)(2r + 1) + (dx + r).  Writes the index k per pixel. */
ORC_API void orc_bruteforce_flow(const double *a, const double *b, int c, int h, int w, int r,
                                 int *kout)
{
    const int n = 2 * r + 1;
    const size_t hw = (size_t)h * w;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
            double best = INFINITY;
            int bestk = 0, bestn = 1 << 30;
            for (int k = 0; k < n * n; ++k) {
                const int dy = k / n - r, dx = k % n - r;
                double s = 0.0;
                for (int py = -1; py <= 1; ++py) {
                    for (int px = -1; px <= 1; ++px) {
                        int ay = y + py, ax = x + px, by = ay + dy, bx = ax + dx;
                        ay = ay < 0 ? 0 : (ay >= h ? h - 1 : ay);
                        ax = ax < 0 ? 0 : (ax >= w ? w - 1 : ax);
                        by = by < 0 ? 0 : (by >= h ? h - 1 : by);
                        bx = bx < 0 ? 0 : (bx >= w ? w - 1 : bx);
                        for (int ch = 0; ch < c; ++ch) {
                            const double e = a[ch * hw + (size_t)ay * w + ax] - b[ch * hw + (size_t)by * w + bx];
                            s += e * e;
                        }
                    }
                }
                const int nn = dx * dx + dy * dy;
                if (s < best || (s == best && nn < bestn)) {
                    best = s;
                    bestk = k;
                    bestn = nn;
                }
            }
            kout[(size_t)y * w + x] = bestk;
        }
    }
}

/* Gradient of the screened-Poisson energy of Eq. 1 for one channel (h, w), read as
 *   E(O) = 1/2 sum over 4-neighbour pixel pairs (i, j) of ((O_i - O_j) - (P_i - P_j))^2
 *        + 1/2 sum_i wc_i (O_i - A_i)^2,
 * i.e. dE/dO = Lg (O - P) + wc (O - A), with Lg the graph Laplacian of the image's
 * 4-neighbour grid: (Lg x)_i = sum over the neighbours j of i that exist of (x_i - x_j)
 * (Neumann boundary: a border pixel has fewer neighbours). */
ORC_API void orc_poisson_grad(int h, int w, const double *O, const double *P, const double *A,
                              const double *wc, double *g)
{
#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
            const size_t i = (size_t)y * w + x;
            const double d = O[i] - P[i];
            double lap = 0.0;
            const int ny[4] = {y - 1, y + 1, y, y}, nx[4] = {x, x, x - 1, x + 1};
            for (int k = 0; k < 4; ++k) {
                if (ny[k] < 0 || ny[k] >= h || nx[k] < 0 || nx[k] >= w) continue;
                const size_t j = (size_t)ny[k] * w + nx[k];
                lap += d - (O[j] - P[j]);
            }
            g[i] = lap + wc[i] * (O[i] - A[i]);
        }
    }
}

/* The solver of Sec. 3.1 ("Optimization Solver", Eq. 8): SGD with momentum,
 *   O^{j+1} = O^j - eta grad E(O^j) + kappa (O^j - O^{j-1}),
 * started from O^0 = O^{-1} = A, for `iters` iterations, each of the c channels of the
 * planar (c, h, w) images on its own with the same per-pixel wc (h, w).  O_out (c, h, w). */
ORC_API void orc_poisson_solve(int c, int h, int w, const double *P, const double *A, const double *wc,
                               double eta, double kappa, int iters, double *O_out)
{
    const size_t hw = (size_t)h * w;
    double *cur = malloc(sizeof(double) * hw), *prev = malloc(sizeof(double) * hw);
    double *next = malloc(sizeof(double) * hw), *g = malloc(sizeof(double) * hw);
    for (int ch = 0; ch < c; ++ch) {
        const double *Pc = P + ch * hw, *Ac = A + ch * hw;
        memcpy(cur, Ac, sizeof(double) * hw);
        memcpy(prev, Ac, sizeof(double) * hw);
        for (int j = 0; j < iters; ++j) {
            orc_poisson_grad(h, w, cur, Pc, Ac, wc, g);
            for (size_t i = 0; i < hw; ++i) next[i] = cur[i] - eta * g[i] + kappa * (cur[i] - prev[i]);
            double *t = prev;
            prev = cur;
            cur = next;
            next = t;
        }
        memcpy(O_out + ch * hw, cur, sizeof(double) * hw);
    }
    free(cur);
    free(prev);
    free(next);
    free(g);
}
