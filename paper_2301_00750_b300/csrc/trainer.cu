// In-project training of the lite flow network (Sec. 3.2 "Training"): forward with every
// activation kept, multi-scale end-point-error loss, explicit backward schedule, AdamW.
// One trainer owns all of its device buffers; a run is a fixed sequence of kernel launches
// on the caller's stream.
//
// Layouts (NHWC, B pairs; the pyramid batch is 2B images, a's first):
//   img   [2B][H][W][4] (RGB + a zero channel)
//   pyr   per level l and conv j: [2B][h][w][c_l]
//   x0    per estimator level: [B][h][w][x0p] = [cost volume D | f_self c | up-flow 2 | 0 pad]
//         (the weight file's cat order, so no permutation)
//   x1    [B][h][w][dec0]
//   xd    [B][h][w][dec3 + dec2 + dec1] = [x4 | x3 | x2]: conv4 reads the window [x3 | x2]
//         and the head the window [x4 | x3], both in the file's cat order
//   up, flow, gt: [B][h][w][2] float
// Gradients are float buffers of the same shapes.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/tc_train.h"
#include "common.cuh"
#include "engine_internal.h"
#include "conv_tc.cuh"
#include "train_kernels.cuh"
#include "wgrad_tc.cuh"

using namespace tc;

namespace {

int round_up(int v, int m) { return (v + m - 1) / m * m; }

struct Layer {
    int cout, cin, stride, leaky;
    size_t w_off, b_off;   // into the flat parameter vector
    int cin_p;             // forward packing (input channel stride of the layer's input)
    float *wk = nullptr;   // forward packed [9][cin_p][cout]
    float *bk = nullptr;   // bias copy (the flat parameter vector does not keep it 16-byte aligned)
    int dg_cout_p = 0, dg_cin_p = 0;
    float *wkT = nullptr;  // data-gradient packed [9][cout][cin_p] (flipped, transposed)
    // forward input and output (fixed buffers; windows at the pointers)
    const void *in = nullptr;
    int in_cs = 0, n = 0, h = 0, w = 0;
    void *out = nullptr;
    int out_cs = 0;
    // BF16 trainer: forward and data-gradient convs on the tensor cores (weights packed from
    // the master copy every step); the data gradient in slices of <= 128 output channels
    bool tc = false;
    TcConvPlan fplan;
    TcConvPlan dplan[2];
    int dlo[2] = {0, 0}, dn[2] = {0, 0}, ndp = 0;
    WgradTcPlan wplan;  // weight gradient on the tensor cores (over the CP scratch buffers)
};

struct Level {
    int h, w, c;
    void *pyr[3] = {nullptr, nullptr, nullptr};  // T
    float *dpyr = nullptr;                        // gradient of pyr[2]
    // estimator (l >= 2)
    int x0p = 0, xdc = 0;
    void *x0 = nullptr, *x1 = nullptr, *xd = nullptr, *f2w = nullptr;  // T
    float *up = nullptr, *flow = nullptr, *gt = nullptr;
    float *dx0 = nullptr, *dx1 = nullptr, *dxd = nullptr, *df2w = nullptr, *dup = nullptr, *dflow = nullptr;
};

}  // namespace

struct tc_trainer {
    int B = 0, H = 0, W = 0, L = 0, R = 0, D = 0;
    tc_precision prec = TC_FP32;
    HostNet net;
    cudaStream_t st = nullptr;
    train::AdamW hp{};
    long long steps = 0;
    std::vector<Layer> layers;
    size_t n_params = 0;
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    uint8_t *decay = nullptr;
    float *zeros = nullptr;  // bias of the data-gradient convs
    void *img = nullptr;     // T
    std::vector<Level> lv;
    float *dz = nullptr, *dz_dil = nullptr, *dtmp0 = nullptr, *dtmp1 = nullptr;
    void *dzh = nullptr, *dzh_dil = nullptr;  // bfloat16 copies of dz (tensor-core data gradients)
    void *dz_cp = nullptr, *x_cp[3] = {nullptr, nullptr, nullptr};  // weight-gradient operands (bf16)
    float *wg_partial = nullptr;
    int *dev_err = nullptr;                   // device error word of the tensor-core kernels
    double *loss_dev = nullptr;
    std::vector<void *> allocs;
    std::string err;
    bool poisoned = false;
};

namespace {

tc_status tfail(tc_trainer *t, tc_status code, const std::string &msg) {
    if (t) {
        t->err = msg;
        if (code == TC_ERR_CUDA) t->poisoned = true;
        return code;
    }
    return tc_record_error(code, msg);
}

#define TT_TRY(t, expr, what)                                                                         \
    do {                                                                                              \
        cudaError_t _e = (expr);                                                                      \
        if (_e != cudaSuccess) return tfail(t, TC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(_e)); \
    } while (0)

template <typename P>
tc_status talloc(tc_trainer *t, P **p, size_t bytes) {
    void *q = nullptr;
    if (cudaMalloc(&q, bytes ? bytes : 16) != cudaSuccess) {
        cudaGetLastError();
        return tfail(t, TC_ERR_OOM, "trainer: cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    t->allocs.push_back(q);
    *p = static_cast<P *>(q);
    TT_TRY(t, cudaMemset(q, 0, bytes ? bytes : 16), "memset");
    return TC_OK;
}

void free_trainer(tc_trainer *t) {
    for (auto &ly : t->layers) {
        ly.fplan.release();
        ly.dplan[0].release();
        ly.dplan[1].release();
    }
    for (void *p : t->allocs) cudaFree(p);
    t->allocs.clear();
}

bool read_blob(const tc_trainer_desc *d, std::vector<uint8_t> &blob, std::string &err) {
    if (d->weights_path) {
        FILE *f = fopen(d->weights_path, "rb");
        if (!f) { err = std::string("cannot open weights file ") + d->weights_path; return false; }
        fseek(f, 0, SEEK_END);
        const long n = ftell(f);
        fseek(f, 0, SEEK_SET);
        blob.resize(n > 0 ? (size_t)n : 0);
        const size_t got = n > 0 ? fread(blob.data(), 1, (size_t)n, f) : 0;
        fclose(f);
        if (got != blob.size()) { err = "short read of the weights file"; return false; }
        return true;
    }
    if (d->weights_blob && d->weights_bytes) {
        blob.assign((const uint8_t *)d->weights_blob, (const uint8_t *)d->weights_blob + d->weights_bytes);
        return true;
    }
    err = "tc_trainer_create: no weights given";
    return false;
}

template <typename T>
tc_status build(tc_trainer *t) {
    const int L = t->L, B = t->B;
    const size_t es = sizeof(T);
    tc_status r;
    // parameters in file order
    for (const auto &HL : t->net.layers) {
        Layer ly;
        ly.cout = HL.cout;
        ly.cin = HL.cin;
        ly.stride = HL.stride;
        ly.leaky = HL.leaky;
        ly.w_off = t->n_params;
        t->n_params += HL.w.size();
        ly.b_off = t->n_params;
        t->n_params += HL.b.size();
        t->layers.push_back(ly);
    }
    const size_t np = t->n_params;
    if ((r = talloc(t, &t->params, np * 4)) != TC_OK) return r;
    if ((r = talloc(t, &t->grads, np * 4)) != TC_OK) return r;
    if ((r = talloc(t, &t->m, np * 4)) != TC_OK) return r;
    if ((r = talloc(t, &t->v, np * 4)) != TC_OK) return r;
    if ((r = talloc(t, &t->decay, np)) != TC_OK) return r;
    if ((r = talloc(t, &t->loss_dev, sizeof(double))) != TC_OK) return r;
    std::vector<float> hostp(np);
    std::vector<uint8_t> hostd(np, 0);
    for (size_t i = 0; i < t->layers.size(); ++i) {
        const HostLayer &HL = t->net.layers[i];
        memcpy(&hostp[t->layers[i].w_off], HL.w.data(), HL.w.size() * 4);
        memcpy(&hostp[t->layers[i].b_off], HL.b.data(), HL.b.size() * 4);
        memset(&hostd[t->layers[i].w_off], 1, HL.w.size());
    }
    TT_TRY(t, cudaMemcpy(t->params, hostp.data(), np * 4, cudaMemcpyHostToDevice), "parameter upload");
    TT_TRY(t, cudaMemcpy(t->decay, hostd.data(), np, cudaMemcpyHostToDevice), "parameter upload");

    // levels
    t->lv.resize(L);
    int max_c = 4;
    for (int l = 1; l <= L; ++l) {
        Level &V = t->lv[l - 1];
        V.h = t->H >> l;
        V.w = t->W >> l;
        V.c = t->net.chans[l - 1];
        max_c = std::max(max_c, V.c);
    }
    if ((r = talloc(t, &t->img, (size_t)2 * B * t->H * t->W * 4 * es)) != TC_OK) return r;
    const int dec0 = t->net.dec[0], dec1 = t->net.dec[1], dec2 = t->net.dec[2], dec3 = t->net.dec[3];
    size_t max_dz = 0, max_dil = 0, max_tmp = 0;
    for (int l = 1; l <= L; ++l) {
        Level &V = t->lv[l - 1];
        const size_t px2 = (size_t)2 * B * V.h * V.w, px = (size_t)B * V.h * V.w;
        for (int j = 0; j < 3; ++j)
            if ((r = talloc(t, &V.pyr[j], px2 * V.c * es)) != TC_OK) return r;
        if ((r = talloc(t, &V.dpyr, px2 * V.c * 4)) != TC_OK) return r;
        max_dz = std::max(max_dz, px2 * V.c);
        max_tmp = std::max(max_tmp, px2 * V.c);
        if (l > 1) max_dil = std::max(max_dil, (size_t)2 * B * t->lv[l - 2].h * t->lv[l - 2].w * V.c);
        if (l < 2) continue;
        V.x0p = round_up(t->D + V.c + 2, 16);  // 16: tensor-core K steps and 16-byte pixel strides
        V.xdc = dec3 + dec2 + dec1;
        if ((r = talloc(t, &V.x0, px * V.x0p * es)) != TC_OK) return r;
        if ((r = talloc(t, &V.x1, px * dec0 * es)) != TC_OK) return r;
        if ((r = talloc(t, &V.xd, px * V.xdc * es)) != TC_OK) return r;
        if ((r = talloc(t, &V.f2w, px * V.c * es)) != TC_OK) return r;
        if ((r = talloc(t, &V.up, px * 2 * 4)) != TC_OK) return r;
        if ((r = talloc(t, &V.flow, px * 2 * 4)) != TC_OK) return r;
        if ((r = talloc(t, &V.gt, px * 2 * 4)) != TC_OK) return r;
        if ((r = talloc(t, &V.dx0, px * V.x0p * 4)) != TC_OK) return r;
        if ((r = talloc(t, &V.dx1, px * dec0 * 4)) != TC_OK) return r;
        if ((r = talloc(t, &V.dxd, px * V.xdc * 4)) != TC_OK) return r;
        if ((r = talloc(t, &V.df2w, px * V.c * 4)) != TC_OK) return r;
        if ((r = talloc(t, &V.dup, px * 2 * 4)) != TC_OK) return r;
        if ((r = talloc(t, &V.dflow, px * 2 * 4)) != TC_OK) return r;
        max_dz = std::max(max_dz, px * (size_t)std::max(dec0, std::max(dec1, dec2)));
    }
    if ((r = talloc(t, &t->dz, max_dz * 4)) != TC_OK) return r;
    if ((r = talloc(t, &t->dz_dil, std::max<size_t>(max_dil, 1) * 4)) != TC_OK) return r;
    if ((r = talloc(t, &t->dtmp0, max_tmp * 4)) != TC_OK) return r;
    if ((r = talloc(t, &t->dtmp1, max_tmp * 4)) != TC_OK) return r;
    int max_w = 4;
    for (auto &ly : t->layers) max_w = std::max(max_w, round_up(std::max(ly.cin, ly.cout), 4));
    if ((r = talloc(t, &t->zeros, (size_t)max_w * 4)) != TC_OK) return r;

    // packed weights: the forward input channel stride of each layer, and the data-gradient
    // form of every layer whose input needs a gradient (all but the first conv)
    for (int l = 1; l <= L; ++l) {
        const Level &V = t->lv[l - 1];
        for (int j = 0; j < 3; ++j) {
            Layer &ly = t->layers[3 * (l - 1) + j];
            ly.cin_p = (l == 1 && j == 0) ? 4 : ly.cin;
            if (!(l == 1 && j == 0)) {
                ly.dg_cout_p = ly.cout;
                ly.dg_cin_p = ly.cin;
            }
            (void)V;
        }
    }
    for (int l = L; l >= 2; --l) {
        const Level &V = t->lv[l - 1];
        Layer *E = &t->layers[3 * L + 5 * (L - l)];
        E[0].cin_p = V.x0p;
        for (int j = 1; j < 5; ++j) E[j].cin_p = E[j].cin;
        E[0].dg_cout_p = E[0].cout;
        E[0].dg_cin_p = V.x0p;
        for (int j = 1; j < 4; ++j) {
            E[j].dg_cout_p = E[j].cout;
            E[j].dg_cin_p = E[j].cin;
        }
    }
    for (auto &ly : t->layers) {
        if ((r = talloc(t, &ly.wk, (size_t)9 * ly.cin_p * ly.cout * 4)) != TC_OK) return r;
        if ((r = talloc(t, &ly.bk, (size_t)round_up(ly.cout, 4) * 4)) != TC_OK) return r;
        if (ly.dg_cout_p)
            if ((r = talloc(t, &ly.wkT, (size_t)9 * ly.dg_cout_p * ly.dg_cin_p * 4)) != TC_OK) return r;
    }
    // forward I/O of every layer
    {
        const int dec0 = t->net.dec[0], dec2 = t->net.dec[2], dec3 = t->net.dec[3];
        auto set = [](Layer &ly, const void *in, int in_cs, int n, int h, int w, void *out, int out_cs) {
            ly.in = in; ly.in_cs = in_cs; ly.n = n; ly.h = h; ly.w = w; ly.out = out; ly.out_cs = out_cs;
        };
        for (int l = 1; l <= L; ++l) {
            Level &V = t->lv[l - 1];
            Layer *P = &t->layers[3 * (l - 1)];
            if (l == 1)
                set(P[0], t->img, 4, 2 * B, t->H, t->W, V.pyr[0], V.c);
            else
                set(P[0], t->lv[l - 2].pyr[2], t->lv[l - 2].c, 2 * B, t->lv[l - 2].h, t->lv[l - 2].w, V.pyr[0], V.c);
            set(P[1], V.pyr[0], V.c, 2 * B, V.h, V.w, V.pyr[1], V.c);
            set(P[2], V.pyr[1], V.c, 2 * B, V.h, V.w, V.pyr[2], V.c);
        }
        for (int l = L; l >= 2; --l) {
            Level &V = t->lv[l - 1];
            Layer *E = &t->layers[3 * L + 5 * (L - l)];
            T *xd = static_cast<T *>(V.xd);
            set(E[0], V.x0, V.x0p, B, V.h, V.w, V.x1, dec0);
            set(E[1], V.x1, dec0, B, V.h, V.w, xd + dec3 + dec2, V.xdc);
            set(E[2], xd + dec3 + dec2, V.xdc, B, V.h, V.w, xd + dec3, V.xdc);
            set(E[3], xd + dec3, V.xdc, B, V.h, V.w, xd, V.xdc);
            set(E[4], xd, V.xdc, B, V.h, V.w, V.flow, 2);
        }
    }
    if (t->prec == TC_BF16) {
        if ((r = talloc(t, &t->dev_err, sizeof(int))) != TC_OK) return r;
        if ((r = talloc(t, &t->dzh, max_dz * 2)) != TC_OK) return r;
        if ((r = talloc(t, &t->dzh_dil, std::max<size_t>(max_dil, 1) * 2)) != TC_OK) return r;
        const int L5 = 3 * L;
        for (size_t k = 1; k < t->layers.size(); ++k) {
            Layer &ly = t->layers[k];
            const bool head = k >= (size_t)L5 && (k - L5) % 5 == 4;
            const int ho = (ly.h - 1) / ly.stride + 1, wo = (ly.w - 1) / ly.stride + 1;
            std::string why;
            ConvArgs a{ly.in, ly.in_cs, ly.n, ly.h, ly.w, ly.cin_p, ly.stride, ho, wo, nullptr, nullptr, ly.cout,
                       ly.out, ly.out_cs, ly.leaky, 1.f, 0};
            bool ok;
            if (head) {
                a.out = nullptr;
                ok = tc_plan_head(ly.fplan, a, ly.n, std::vector<float>((size_t)9 * ly.cin_p * ly.cout, 0.f),
                                  t->dev_err, why);
            } else {
                ok = tc_plan_conv(ly.fplan, a, ly.n, std::vector<float>((size_t)9 * ly.cin_p * ly.cout, 0.f),
                                  t->dev_err, why);
            }
            if (!ok) return tfail(t, TC_ERR_UNSUPPORTED, "trainer: layer not eligible for the tensor cores: " + why);
            if (head) {
                ly.tc = true;
                continue;
            }
            if (!ly.dg_cout_p) continue;
            // data gradient: stride-1 conv of dz (or of its dilation for stride 2) with the
            // flipped, transposed kernel, in slices of <= 128 output channels
            const int N = ly.dg_cin_p;
            ly.ndp = N > 128 ? 2 : 1;
            ly.dlo[0] = 0;
            ly.dn[0] = N > 128 ? 128 : N;
            ly.dlo[1] = 128;
            ly.dn[1] = N - 128;
            for (int q = 0; q < ly.ndp; ++q) {
                if (ly.dn[q] % 16 != 0) return tfail(t, TC_ERR_UNSUPPORTED, "trainer: data-gradient slice not a multiple of 16");
                ConvArgs d{ly.stride == 2 ? t->dzh_dil : t->dzh, ly.cout, ly.n, ly.h, ly.w, ly.cout, 1, ly.h, ly.w,
                           nullptr, nullptr, ly.dn[q], nullptr, ly.dn[q], 0, 1.f, 0};
                if (!tc_plan_conv(ly.dplan[q], d, ly.n, std::vector<float>((size_t)9 * ly.cout * ly.dn[q], 0.f),
                                  t->dev_err, why))
                    return tfail(t, TC_ERR_UNSUPPORTED, "trainer: data gradient not eligible for the tensor cores: " + why);
            }
            ly.tc = true;
        }
        t->layers[0].tc = false;
        // weight gradients: CP scratch sized for the largest layer
        size_t max_dz_cp = 0, max_x_cp = 0, max_part = 0;
        for (auto &ly : t->layers) {
            const int wp = round_up(ly.w + 2, 8), n = round_up(ly.cin + 1, 16);
            const long long P = (long long)ly.n * (ly.h + 2) * wp;
            max_dz_cp = std::max(max_dz_cp, (size_t)ly.cout * (size_t)P);
            max_x_cp = std::max(max_x_cp, (size_t)n * (size_t)P);
            max_part = std::max(max_part, wgrad_tc_partial_floats(P, n, ly.cout));
        }
        if ((r = talloc(t, &t->dz_cp, max_dz_cp * 2)) != TC_OK) return r;
        for (int k = 0; k < 3; ++k)
            if ((r = talloc(t, &t->x_cp[k], max_x_cp * 2)) != TC_OK) return r;
        if ((r = talloc(t, &t->wg_partial, max_part * 4)) != TC_OK) return r;
        for (auto &ly : t->layers) {
            const int wp = round_up(ly.w + 2, 8), n = round_up(ly.cin + 1, 16);  // + the row of ones
            const long long P = (long long)ly.n * (ly.h + 2) * wp;
            std::string why;
            const void *xs[3] = {t->x_cp[0], t->x_cp[1], t->x_cp[2]};
            if (!wgrad_tc_plan(ly.wplan, t->dz_cp, xs, ly.cout, ly.cin, n, wp, P, t->wg_partial, t->dev_err, why))
                return tfail(t, TC_ERR_UNSUPPORTED, "trainer: weight gradient not eligible for the tensor cores: " + why);
        }
    }
    return TC_OK;
}

// Weight and bias gradients on the tensor cores from the float dz [n ho wo][cout] of a layer
// whose input is x (window of x_cs channels).
template <typename T>
tc_status wgrad_tc(tc_trainer *t, const Layer &ly, const void *x, int x_cs, const float *dz, int dz_cs) {
    const int ho = (ly.h - 1) / ly.stride + 1, wo = (ly.w - 1) / ly.stride + 1;
    const WgradTcPlan &W = ly.wplan;
    TT_TRY(t, train::dz_to_cp(dz, dz_cs, ly.n, ly.h, ly.w, ho, wo, ly.stride, ly.cout, W.wp, t->dz_cp, nullptr,
                              t->st),
           "weight gradient operands");
    TT_TRY(t, train::x_to_cp<T>(static_cast<const T *>(x), x_cs, ly.n, ly.h, ly.w, ly.cin, W.wp, W.n, t->x_cp, t->st),
           "weight gradient operands");
    TT_TRY(t, wgrad_tc_launch(W, t->grads + ly.w_off, t->grads + ly.b_off, t->st), "weight gradient (tensor cores)");
    return TC_OK;
}

// --------------------------------------------------------------------------- forward

template <typename T>
tc_status conv_fwd(tc_trainer *t, const Layer &ly) {
    const int ho = (ly.h - 1) / ly.stride + 1, wo = (ly.w - 1) / ly.stride + 1;
    ConvArgs a{ly.in, ly.in_cs, ly.n, ly.h, ly.w, ly.cin_p, ly.stride, ho, wo, ly.wk, ly.bk, ly.cout, ly.out,
               ly.out_cs, ly.leaky, 1.f, 0};
    if (ly.tc)
        TT_TRY(t, launch_conv_tc(ly.fplan, a, t->st), "conv forward (tensor cores)");
    else
        TT_TRY(t, launch_conv_simt<T>(a, t->st), "conv forward");
    return TC_OK;
}

template <typename T>
tc_status forward(tc_trainer *t, const float *Ia, const float *Ib, const float *gt, bool want_grad) {
    const int L = t->L, B = t->B, D = t->D;
    const bool bf = t->prec == TC_BF16;
    tc_status r;
    for (auto &ly : t->layers) {
        TT_TRY(t, cudaMemcpyAsync(ly.bk, t->params + ly.b_off, (size_t)ly.cout * 4, cudaMemcpyDeviceToDevice, t->st),
               "bias copy");
        const float *w = t->params + ly.w_off;
        if (ly.tc) {
            const TcConvPlan &f = ly.fplan;
            TT_TRY(t, train::pack_tc(w, ly.cout, ly.cin, 0, 0, 0, f.bn, f.nch * f.kc, f.wpk, t->st), "pack");
            if (want_grad)
                for (int q = 0; q < ly.ndp; ++q) {
                    const TcConvPlan &d = ly.dplan[q];
                    TT_TRY(t, train::pack_tc(w, ly.cout, ly.cin, 1, ly.dlo[q], std::min(ly.dn[q], ly.cin - ly.dlo[q]),
                                             d.bn, d.nch * d.kc, d.wpk, t->st),
                           "pack");
                }
            if (ly.cout == 2) TT_TRY(t, train::pack_fwd(w, ly.cout, ly.cin, ly.cin_p, bf, ly.wk, t->st), "pack");
        } else {
            TT_TRY(t, train::pack_fwd(w, ly.cout, ly.cin, ly.cin_p, bf, ly.wk, t->st), "pack");
            if (want_grad && ly.wkT)
                TT_TRY(t, train::pack_dgrad(w, ly.cout, ly.cin, ly.dg_cout_p, ly.dg_cin_p, ly.wkT, t->st), "pack");
        }
    }
    T *img = static_cast<T *>(t->img);
    TT_TRY(t, train::pack_images<T>(Ia, Ib, B, t->H, t->W, img, t->st), "pack images");
    // pyramids of a and b (2B images)
    for (int l = 1; l <= L; ++l) {
        Level &V = t->lv[l - 1];
        const Layer *P = &t->layers[3 * (l - 1)];
        const void *in = l == 1 ? (const void *)img : t->lv[l - 2].pyr[2];
        const int in_cs = l == 1 ? 4 : t->lv[l - 2].c;
        const int ih = l == 1 ? t->H : t->lv[l - 2].h, iw = l == 1 ? t->W : t->lv[l - 2].w;
        (void)in; (void)in_cs; (void)ih; (void)iw;
        for (int j = 0; j < 3; ++j)
            if ((r = conv_fwd<T>(t, P[j])) != TC_OK) return r;
    }
    const int dec1 = t->net.dec[1], dec2 = t->net.dec[2], dec3 = t->net.dec[3];
    // estimators a -> b, coarse to fine
    for (int l = L; l >= 2; --l) {
        Level &V = t->lv[l - 1];
        const Layer *E = &t->layers[3 * L + 5 * (L - l)];
        const size_t img_el = (size_t)V.h * V.w * V.c;
        const T *fa = static_cast<const T *>(V.pyr[2]);
        const T *fb = fa + (size_t)B * img_el;
        T *x0 = static_cast<T *>(V.x0);
        const T *fo = fb;
        if (l < L) {
            const Level &C = t->lv[l];
            UpArgs u{C.flow, B, C.h, C.w, 2, V.up, x0 + D + V.c, V.x0p};
            TT_TRY(t, launch_up<T>(u, t->st), "upsample");
            WarpArgs wa{{fb, fb}, V.c, V.up, B, V.h, V.w, V.c, V.f2w, V.c, nullptr, nullptr, nullptr, 0, 1.f, img_el};
            TT_TRY(t, launch_warp<T>(wa, t->st), "warp");
            fo = static_cast<const T *>(V.f2w);
        }
        CorrArgs ca{{fa, fa}, {fo, fo}, V.c, V.c, B, V.h, V.w, V.c, t->R, x0, V.x0p, x0 + D, img_el, img_el};
        TT_TRY(t, launch_corr<T>(ca, t->st), "correlation");
        T *x1 = static_cast<T *>(V.x1);
        T *xd = static_cast<T *>(V.xd);
        (void)x1; (void)dec1; (void)dec2; (void)dec3;
        for (int j = 0; j < 4; ++j)
            if ((r = conv_fwd<T>(t, E[j])) != TC_OK) return r;
        if (E[4].tc) {
            ConvArgs a5{xd, V.xdc, B, V.h, V.w, E[4].cin_p, 1, V.h, V.w, nullptr, E[4].bk, 2, nullptr, 2, 0, 1.f, 0};
            TT_TRY(t, launch_conv_tc_head(E[4].fplan, a5, l < L ? V.up : nullptr, V.flow, t->st),
                   "flow head (tensor cores)");
        } else {
            HeadArgs ha{xd, V.xdc, E[4].cin_p, B, V.h, V.w, E[4].wk, E[4].bk, l < L ? V.up : nullptr, V.flow};
            TT_TRY(t, launch_head<T>(ha, t->st), "flow head");
        }
    }
    // loss: sum over levels of the mean EPE against the block-averaged ground truth
    TT_TRY(t, cudaMemsetAsync(t->loss_dev, 0, sizeof(double), t->st), "memset");
    for (int l = 2; l <= L; ++l) {
        Level &V = t->lv[l - 1];
        TT_TRY(t, train::gt_level(gt, B, t->H, t->W, l, V.gt, t->st), "gt pyramid");
        if (want_grad) TT_TRY(t, cudaMemsetAsync(V.dflow, 0, (size_t)B * V.h * V.w * 2 * 4, t->st), "memset");
        TT_TRY(t, train::epe(V.flow, V.gt, (size_t)B * V.h * V.w, t->loss_dev, want_grad ? V.dflow : nullptr, true,
                             t->st),
               "loss");
    }
    return TC_OK;
}

// -------------------------------------------------------------------------- backward

// Gradients of a conv given dy (window of a float buffer): dz = dy LeakyReLU'(y), the
// weight and bias gradients, and (if dx) the data gradient added into dx.
template <typename T>
tc_status conv_bwd(tc_trainer *t, const Layer &ly, const void *x, int x_cs, int n, int h, int w, const T *y, int y_cs,
                   const float *dy, int dy_cs, float *dx, int dx_cs, bool dx_accumulate) {
    const int ho = (h - 1) / ly.stride + 1, wo = (w - 1) / ly.stride + 1;
    const size_t npix = (size_t)n * ho * wo;
    const bool dil = dx && ly.stride == 2;
    if (ly.wplan.enabled && (dx ? (ly.tc && ly.ndp > 0) : true)) {
        if (dil) TT_TRY(t, cudaMemsetAsync(t->dzh_dil, 0, (size_t)n * h * w * ly.cout * 2, t->st), "memset");
        TT_TRY(t, train::lrelu_bwd2<T>(dy, dy_cs, y, y_cs, ly.leaky != 0, npix, ly.cout, t->dz, dil ? nullptr : t->dzh,
                                       dil ? t->dzh_dil : nullptr, ho, wo, h, w, t->st),
               "activation backward");
        tc_status rr = wgrad_tc<T>(t, ly, x, x_cs, t->dz, ly.cout);
        if (rr != TC_OK) return rr;
        for (int q = 0; q < ly.ndp; ++q) {
            ConvArgs a{dil ? t->dzh_dil : t->dzh, ly.cout, n, h, w, ly.cout, 1, h, w, nullptr, t->zeros, ly.dn[q],
                       dx + ly.dlo[q], dx_cs, 0, 1.f, 0};
            TT_TRY(t, launch_conv_tc_f32(ly.dplan[q], a, dx_accumulate, t->st), "data gradient (tensor cores)");
        }
        return TC_OK;
    }
    if (dil) TT_TRY(t, cudaMemsetAsync(t->dz_dil, 0, (size_t)n * h * w * ly.cout * 4, t->st), "memset");
    TT_TRY(t, train::lrelu_bwd<T>(dy, dy_cs, y, y_cs, ly.leaky != 0, npix, ly.cout, t->dz, dil ? t->dz_dil : nullptr,
                                  ho, wo, h, w, t->st),
           "activation backward");
    train::WgradArgs<T> wa{static_cast<const T *>(x), x_cs, n, h, w, ly.cin, ly.stride, ho, wo, t->dz, ly.cout,
                           ly.cout, t->grads + ly.w_off};
    TT_TRY(t, train::wgrad<T>(wa, t->grads + ly.b_off, t->st), "weight gradient");
    if (dx) {
        // data gradient: the stride-1 conv of dz (dilated for stride 2) with the flipped,
        // transposed kernel
        ConvArgs a{dil ? (const void *)t->dz_dil : (const void *)t->dz, ly.cout, n, h, w, ly.dg_cout_p, 1, h, w,
                   ly.wkT, t->zeros, ly.dg_cin_p, dx, dx_cs, 0, 1.f, dx_accumulate ? 1 : 0};
        TT_TRY(t, launch_conv_simt<float>(a, t->st), "data gradient");
    }
    return TC_OK;
}

template <typename T>
tc_status backward(tc_trainer *t) {
    const int L = t->L, B = t->B, D = t->D;
    const int dec0 = t->net.dec[0], dec2 = t->net.dec[2], dec3 = t->net.dec[3];
    tc_status r;
    TT_TRY(t, cudaMemsetAsync(t->grads, 0, t->n_params * 4, t->st), "memset");
    for (int l = 1; l <= L; ++l) {
        Level &V = t->lv[l - 1];
        TT_TRY(t, cudaMemsetAsync(V.dpyr, 0, (size_t)2 * B * V.h * V.w * V.c * 4, t->st), "memset");
        if (l >= 2) TT_TRY(t, cudaMemsetAsync(V.dup, 0, (size_t)B * V.h * V.w * 2 * 4, t->st), "memset");
    }
    // estimators, fine to coarse (the reverse of the forward)
    for (int l = 2; l <= L; ++l) {
        Level &V = t->lv[l - 1];
        const Layer *E = &t->layers[3 * L + 5 * (L - l)];
        const size_t px = (size_t)B * V.h * V.w;
        const size_t img_el = (size_t)V.h * V.w * V.c;
        const T *x0 = static_cast<const T *>(V.x0);
        const T *x1 = static_cast<const T *>(V.x1);
        const T *xd = static_cast<const T *>(V.xd);
        TT_TRY(t, cudaMemsetAsync(V.dxd, 0, px * V.xdc * 4, t->st), "memset");
        // head: flow = up + conv5([x4 | x3])
        {
            if (E[4].tc) {
                if ((r = wgrad_tc<T>(t, E[4], xd, V.xdc, V.dflow, 2)) != TC_OK) return r;
            } else {
                train::WgradArgs<T> wa{xd, V.xdc, B, V.h, V.w, E[4].cin, 1, V.h, V.w, V.dflow, 2, 2,
                                       t->grads + E[4].w_off};
                TT_TRY(t, train::wgrad<T>(wa, t->grads + E[4].b_off, t->st), "head weight gradient");
            }
            TT_TRY(t, train::head_dgrad(V.dflow, t->params + E[4].w_off, E[4].cin, B, V.h, V.w, V.dxd, V.xdc, true,
                                        t->st),
                   "head data gradient");
            if (l < L) TT_TRY(t, train::window_add(V.dflow, 2, px, 2, V.dup, 2, true, t->st), "residual");
        }
        // conv4: [x3 | x2] -> x4
        if ((r = conv_bwd<T>(t, E[3], xd + dec3, V.xdc, B, V.h, V.w, xd, V.xdc, V.dxd, V.xdc, V.dxd + dec3, V.xdc,
                             true)) != TC_OK)
            return r;
        // conv3: x2 -> x3
        if ((r = conv_bwd<T>(t, E[2], xd + dec3 + dec2, V.xdc, B, V.h, V.w, xd + dec3, V.xdc, V.dxd + dec3, V.xdc,
                             V.dxd + dec3 + dec2, V.xdc, true)) != TC_OK)
            return r;
        // conv2: x1 -> x2
        if ((r = conv_bwd<T>(t, E[1], x1, dec0, B, V.h, V.w, xd + dec3 + dec2, V.xdc, V.dxd + dec3 + dec2, V.xdc,
                             V.dx1, dec0, false)) != TC_OK)
            return r;
        // conv1: x0 -> x1
        if ((r = conv_bwd<T>(t, E[0], x0, V.x0p, B, V.h, V.w, x1, dec0, V.dx1, dec0, V.dx0, V.x0p, false)) != TC_OK)
            return r;
        // x0 = [cost | f_self | up]
        float *dpa = V.dpyr, *dpb = V.dpyr + (size_t)B * img_el;
        TT_TRY(t, train::window_add(V.dx0 + D, V.x0p, px, V.c, dpa, V.c, true, t->st), "x0 split");
        if (l < L) TT_TRY(t, train::window_add(V.dx0 + D + V.c, V.x0p, px, 2, V.dup, 2, true, t->st), "x0 split");
        const T *fa = static_cast<const T *>(V.pyr[2]);
        const T *fb = fa + (size_t)B * img_el;
        const T *fo = l < L ? static_cast<const T *>(V.f2w) : fb;
        if (l < L) TT_TRY(t, cudaMemsetAsync(V.df2w, 0, px * V.c * 4, t->st), "memset");
        train::CorrBwdArgs<T> cb{fa, V.c, fo, V.c, x0, V.x0p, V.dx0, V.x0p, B, V.h, V.w, V.c, t->R,
                                 dpa, V.c, l < L ? V.df2w : dpb, V.c, 1};
        TT_TRY(t, train::corr_bwd<T>(cb, t->st), "correlation backward");
        if (l < L) {
            train::WarpBwdArgs<T> wb{fb, V.c, V.up, V.df2w, V.c, B, V.h, V.w, V.c, dpb, V.c, V.dup, 1};
            TT_TRY(t, train::warp_bwd<T>(wb, t->st), "warp backward");
            const Level &C = t->lv[l];
            TT_TRY(t, train::up_bwd(V.dup, B, C.h, C.w, 2, C.dflow, t->st), "upsample backward");
        }
    }
    // pyramids, coarse to fine
    for (int l = L; l >= 1; --l) {
        Level &V = t->lv[l - 1];
        const Layer *P = &t->layers[3 * (l - 1)];
        const T *p0 = static_cast<const T *>(V.pyr[0]);
        const T *p1 = static_cast<const T *>(V.pyr[1]);
        const T *p2 = static_cast<const T *>(V.pyr[2]);
        if ((r = conv_bwd<T>(t, P[2], p1, V.c, 2 * B, V.h, V.w, p2, V.c, V.dpyr, V.c, t->dtmp1, V.c, false)) != TC_OK)
            return r;
        if ((r = conv_bwd<T>(t, P[1], p0, V.c, 2 * B, V.h, V.w, p1, V.c, t->dtmp1, V.c, t->dtmp0, V.c, false)) != TC_OK)
            return r;
        const void *in = l == 1 ? t->img : t->lv[l - 2].pyr[2];
        const int in_cs = l == 1 ? 4 : t->lv[l - 2].c;
        const int ih = l == 1 ? t->H : t->lv[l - 2].h, iw = l == 1 ? t->W : t->lv[l - 2].w;
        float *dprev = l == 1 ? nullptr : t->lv[l - 2].dpyr;
        if ((r = conv_bwd<T>(t, P[0], in, in_cs, 2 * B, ih, iw, p0, V.c, t->dtmp0, V.c, dprev, in_cs, true)) != TC_OK)
            return r;
    }
    return TC_OK;
}

template <typename T>
tc_status run(tc_trainer *t, const float *Ia, const float *Ib, const float *gt, tc_train_mode mode) {
    tc_status r;
    if ((r = forward<T>(t, Ia, Ib, gt, mode != TC_TRAIN_FORWARD)) != TC_OK) return r;
    if (mode == TC_TRAIN_FORWARD) return TC_OK;
    if ((r = backward<T>(t)) != TC_OK) return r;
    if (mode == TC_TRAIN_STEP) {
        t->steps += 1;
        TT_TRY(t, train::adamw(t->params, t->grads, t->m, t->v, t->decay, t->n_params, t->hp, t->steps, t->st),
               "AdamW");
    }
    return TC_OK;
}

tc_status check(tc_trainer *t, const char *what) {
    if (!t) return tc_record_error(TC_ERR_INVALID_ARG, std::string(what) + ": NULL trainer");
    if (t->poisoned) return tfail(t, TC_ERR_STATE, std::string(what) + ": trainer poisoned by an earlier CUDA error: " + t->err);
    return TC_OK;
}

}  // namespace

extern "C" void tc_trainer_default_desc(tc_trainer_desc *d) {
    if (!d) return;
    memset(d, 0, sizeof(*d));
    d->batch = 32;
    d->height = d->width = 256;
    d->precision = TC_BF16;
    d->lr = 1e-4f;
    d->beta1 = 0.9f;
    d->beta2 = 0.99f;
    d->eps = 1e-8f;
    d->weight_decay = 4e-4f;
}

extern "C" tc_status tc_trainer_create(const tc_trainer_desc *d, void *cuda_stream, tc_trainer **out) {
    if (out) *out = nullptr;
    if (!d || !out) return tc_record_error(TC_ERR_INVALID_ARG, "tc_trainer_create: NULL argument");
    if (d->precision != TC_FP32 && d->precision != TC_BF16)
        return tc_record_error(TC_ERR_INVALID_ARG, "tc_trainer_create: precision must be TC_FP32 or TC_BF16");
    if (d->batch < 1 || d->batch > 4096)
        return tc_record_error(TC_ERR_INVALID_ARG, "tc_trainer_create: batch must lie in [1, 4096]");
    if (!(d->lr > 0.f) || !(d->beta1 >= 0.f && d->beta1 < 1.f) || !(d->beta2 >= 0.f && d->beta2 < 1.f) ||
        !(d->eps > 0.f) || !(d->weight_decay >= 0.f))
        return tc_record_error(TC_ERR_INVALID_ARG, "tc_trainer_create: bad optimiser settings");
    std::unique_ptr<tc_trainer> t(new (std::nothrow) tc_trainer());
    if (!t) return tc_record_error(TC_ERR_OOM, "tc_trainer_create: host allocation failed");
    std::vector<uint8_t> blob;
    std::string err;
    if (!read_blob(d, blob, err)) return tc_record_error(d->weights_path ? TC_ERR_IO : TC_ERR_INVALID_ARG, err);
    if (!parse_weights(blob.data(), blob.size(), t->net, err)) return tc_record_error(TC_ERR_IO, err);
    if (!t->net.ref.empty())
        return tc_record_error(TC_ERR_UNSUPPORTED, "tc_trainer_create: the trainer has no refinement network");
    t->L = t->net.levels;
    t->R = t->net.radius;
    t->D = (2 * t->R + 1) * (2 * t->R + 1);
    const int m = 1 << t->L;
    if (d->height < m || d->width < m || d->height % m || d->width % m || d->height > 8192 || d->width > 8192)
        return tc_record_error(TC_ERR_INVALID_ARG,
                               "tc_trainer_create: height and width must be multiples of 2^levels, <= 8192");
    t->B = d->batch;
    t->H = d->height;
    t->W = d->width;
    t->prec = d->precision;
    t->st = static_cast<cudaStream_t>(cuda_stream);
    t->hp = train::AdamW{d->lr, d->beta1, d->beta2, d->eps, d->weight_decay};
    tc_status r = t->prec == TC_FP32 ? build<float>(t.get()) : build<__nv_bfloat16>(t.get());
    if (r != TC_OK) {
        const std::string msg = t->err;
        free_trainer(t.get());
        return tc_record_error(r, msg);
    }
    *out = t.release();
    return TC_OK;
}

extern "C" tc_status tc_trainer_run(tc_trainer *t, const float *Ia, const float *Ib, const float *gt,
                                    tc_train_mode mode, double *loss_out) {
    tc_status r = check(t, "tc_trainer_run");
    if (r != TC_OK) return r;
    if (!Ia || !Ib || !gt || (mode != TC_TRAIN_FORWARD && mode != TC_TRAIN_BACKWARD && mode != TC_TRAIN_STEP))
        return tfail(t, TC_ERR_INVALID_ARG, "tc_trainer_run: bad argument");
    r = t->prec == TC_FP32 ? run<float>(t, Ia, Ib, gt, mode) : run<__nv_bfloat16>(t, Ia, Ib, gt, mode);
    if (r != TC_OK) return r;
    if (loss_out) return tc_trainer_loss(t, loss_out);
    return TC_OK;
}

extern "C" tc_status tc_trainer_loss(tc_trainer *t, double *loss_out) {
    tc_status r = check(t, "tc_trainer_loss");
    if (r != TC_OK) return r;
    if (!loss_out) return tfail(t, TC_ERR_INVALID_ARG, "tc_trainer_loss: NULL");
    TT_TRY(t, cudaStreamSynchronize(t->st), "stream synchronize");
    TT_TRY(t, cudaMemcpy(loss_out, t->loss_dev, sizeof(double), cudaMemcpyDeviceToHost), "loss read");
    return TC_OK;
}

extern "C" size_t tc_trainer_num_params(const tc_trainer *t) { return t ? t->n_params : 0; }

static tc_status copy_params(tc_trainer *t, float *host, const float *dev, size_t n, const char *what) {
    tc_status r = check(t, what);
    if (r != TC_OK) return r;
    if (!host || n != t->n_params) return tfail(t, TC_ERR_INVALID_ARG, std::string(what) + ": need num_params floats");
    TT_TRY(t, cudaStreamSynchronize(t->st), "stream synchronize");
    TT_TRY(t, cudaMemcpy(host, dev, n * 4, cudaMemcpyDeviceToHost), what);
    return TC_OK;
}

extern "C" tc_status tc_trainer_get_params(tc_trainer *t, float *host, size_t n) {
    return copy_params(t, host, t ? t->params : nullptr, n, "tc_trainer_get_params");
}

extern "C" tc_status tc_trainer_get_grads(tc_trainer *t, float *host, size_t n) {
    return copy_params(t, host, t ? t->grads : nullptr, n, "tc_trainer_get_grads");
}

extern "C" tc_status tc_trainer_set_params(tc_trainer *t, const float *host, size_t n) {
    tc_status r = check(t, "tc_trainer_set_params");
    if (r != TC_OK) return r;
    if (!host || n != t->n_params) return tfail(t, TC_ERR_INVALID_ARG, "tc_trainer_set_params: need num_params floats");
    TT_TRY(t, cudaStreamSynchronize(t->st), "stream synchronize");
    TT_TRY(t, cudaMemcpy(t->params, host, n * 4, cudaMemcpyHostToDevice), "tc_trainer_set_params");
    return TC_OK;
}

extern "C" tc_status tc_trainer_level_flow(tc_trainer *t, int level, float *out) {
    tc_status r = check(t, "tc_trainer_level_flow");
    if (r != TC_OK) return r;
    if (!out || level < 2 || level > t->L) return tfail(t, TC_ERR_INVALID_ARG, "tc_trainer_level_flow: bad level");
    const Level &V = t->lv[level - 1];
    TT_TRY(t, cudaMemcpyAsync(out, V.flow, (size_t)t->B * V.h * V.w * 2 * 4, cudaMemcpyDeviceToDevice, t->st),
           "level flow copy");
    return TC_OK;
}

extern "C" long long tc_trainer_steps(const tc_trainer *t) { return t ? t->steps : 0; }

// ------------------------------------------------------------------ files

static void put(std::vector<uint8_t> &b, const void *p, size_t n) {
    b.insert(b.end(), (const uint8_t *)p, (const uint8_t *)p + n);
}

static std::vector<uint8_t> net_header(const tc_trainer *t) {
    std::vector<uint8_t> b;
    const int32_t lv = t->L, rad = t->R;
    put(b, &lv, 4);
    put(b, &rad, 4);
    put(b, t->net.chans.data(), 4 * t->L);
    put(b, t->net.dec, 16);
    const int32_t nl = (int32_t)t->layers.size();
    put(b, &nl, 4);
    return b;
}

static bool write_file(const char *path, const std::vector<uint8_t> &b) {
    FILE *f = fopen(path, "wb");
    if (!f) return false;
    const bool ok = fwrite(b.data(), 1, b.size(), f) == b.size();
    return fclose(f) == 0 && ok;
}

extern "C" tc_status tc_trainer_export_weights(tc_trainer *t, const char *path) {
    tc_status r = check(t, "tc_trainer_export_weights");
    if (r != TC_OK) return r;
    if (!path) return tfail(t, TC_ERR_INVALID_ARG, "tc_trainer_export_weights: NULL path");
    std::vector<float> p(t->n_params);
    if ((r = tc_trainer_get_params(t, p.data(), p.size())) != TC_OK) return r;
    std::vector<uint8_t> b;
    put(b, "TCW1", 4);
    const std::vector<uint8_t> hdr = net_header(t);
    b.insert(b.end(), hdr.begin(), hdr.end());
    for (const auto &ly : t->layers) {
        const int32_t h4[4] = {ly.cout, ly.cin, ly.stride, ly.leaky};
        put(b, h4, 16);
        put(b, &p[ly.w_off], (size_t)ly.cout * ly.cin * 9 * 4);
        put(b, &p[ly.b_off], (size_t)ly.cout * 4);
    }
    if (!write_file(path, b)) return tfail(t, TC_ERR_IO, std::string("cannot write ") + path);
    return TC_OK;
}

extern "C" tc_status tc_trainer_save(tc_trainer *t, const char *path) {
    tc_status r = check(t, "tc_trainer_save");
    if (r != TC_OK) return r;
    if (!path) return tfail(t, TC_ERR_INVALID_ARG, "tc_trainer_save: NULL path");
    const size_t n = t->n_params;
    std::vector<float> p(n), m(n), v(n);
    TT_TRY(t, cudaStreamSynchronize(t->st), "stream synchronize");
    TT_TRY(t, cudaMemcpy(p.data(), t->params, n * 4, cudaMemcpyDeviceToHost), "checkpoint read");
    TT_TRY(t, cudaMemcpy(m.data(), t->m, n * 4, cudaMemcpyDeviceToHost), "checkpoint read");
    TT_TRY(t, cudaMemcpy(v.data(), t->v, n * 4, cudaMemcpyDeviceToHost), "checkpoint read");
    std::vector<uint8_t> b;
    put(b, "TCK1", 4);
    const int64_t steps = t->steps, np = (int64_t)n;
    put(b, &steps, 8);
    const std::vector<uint8_t> hdr = net_header(t);
    b.insert(b.end(), hdr.begin(), hdr.end());
    put(b, &np, 8);
    put(b, p.data(), n * 4);
    put(b, m.data(), n * 4);
    put(b, v.data(), n * 4);
    if (!write_file(path, b)) return tfail(t, TC_ERR_IO, std::string("cannot write ") + path);
    return TC_OK;
}

extern "C" tc_status tc_trainer_load(tc_trainer *t, const char *path) {
    tc_status r = check(t, "tc_trainer_load");
    if (r != TC_OK) return r;
    if (!path) return tfail(t, TC_ERR_INVALID_ARG, "tc_trainer_load: NULL path");
    FILE *f = fopen(path, "rb");
    if (!f) return tfail(t, TC_ERR_IO, std::string("cannot open ") + path);
    std::vector<uint8_t> b;
    uint8_t buf[1 << 16];
    size_t k;
    while ((k = fread(buf, 1, sizeof buf, f)) > 0) b.insert(b.end(), buf, buf + k);
    fclose(f);
    const std::vector<uint8_t> hdr = net_header(t);
    const size_t n = t->n_params;
    const size_t want = 4 + 8 + hdr.size() + 8 + 3 * n * 4;
    if (b.size() != want || memcmp(b.data(), "TCK1", 4) != 0 || memcmp(b.data() + 12, hdr.data(), hdr.size()) != 0)
        return tfail(t, TC_ERR_IO, "tc_trainer_load: not a checkpoint of this network");
    int64_t steps, np;
    memcpy(&steps, b.data() + 4, 8);
    memcpy(&np, b.data() + 12 + hdr.size(), 8);
    if (np != (int64_t)n || steps < 0) return tfail(t, TC_ERR_IO, "tc_trainer_load: parameter count mismatch");
    const uint8_t *base = b.data() + 12 + hdr.size() + 8;
    TT_TRY(t, cudaStreamSynchronize(t->st), "stream synchronize");
    TT_TRY(t, cudaMemcpy(t->params, base, n * 4, cudaMemcpyHostToDevice), "checkpoint write");
    TT_TRY(t, cudaMemcpy(t->m, base + n * 4, n * 4, cudaMemcpyHostToDevice), "checkpoint write");
    TT_TRY(t, cudaMemcpy(t->v, base + 2 * n * 4, n * 4, cudaMemcpyHostToDevice), "checkpoint write");
    t->steps = steps;
    return TC_OK;
}

extern "C" const char *tc_trainer_last_error(const tc_trainer *t) { return t ? t->err.c_str() : tc_last_error(nullptr); }

extern "C" tc_status tc_trainer_destroy(tc_trainer *t) {
    if (!t) return TC_OK;
    cudaStreamSynchronize(t->st);
    free_trainer(t);
    delete t;
    return TC_OK;
}

// ------------------------------------------------------------------ stage backward ops

namespace {
struct Tmp {
    std::vector<void *> ps;
    ~Tmp() {
        for (void *p : ps) cudaFree(p);
    }
    cudaError_t get(float **p, size_t n) {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, (n ? n : 4) * sizeof(float));
        if (e == cudaSuccess) {
            ps.push_back(q);
            *p = static_cast<float *>(q);
        }
        return e;
    }
};
}  // namespace

#define OPB_TRY(expr, what)                                                                                  \
    do {                                                                                                     \
        cudaError_t _e = (expr);                                                                             \
        if (_e != cudaSuccess) return tc_record_error(TC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(_e)); \
    } while (0)

extern "C" tc_status tc_op_conv3x3_backward(const float *x, int n, int h, int w, int cin, const float *w_oihw,
                                            int cout, int stride, int leaky, const float *y, const float *dy,
                                            float *dx, float *dw, float *db, void *cuda_stream) {
    if (!x || !w_oihw || !y || !dy || n < 1 || h < 1 || w < 1 || cin < 1 || cout < 1 || (stride != 1 && stride != 2))
        return tc_record_error(TC_ERR_INVALID_ARG, "tc_op_conv3x3_backward: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int ho = (h - 1) / stride + 1, wo = (w - 1) / stride + 1;
    const int cout_p = round_up(cout, 4), cin_p = round_up(cin, 4);
    const size_t npix = (size_t)n * ho * wo;
    Tmp tmp;
    float *dz, *dzd = nullptr, *wkT, *zeros, *dxp, *dwt, *dbt;
    OPB_TRY(tmp.get(&dz, npix * cout_p), "tc_op_conv3x3_backward alloc");
    OPB_TRY(cudaMemsetAsync(dz, 0, npix * cout_p * 4, st), "memset");
    // dz with cout_p channels (zero pad): activation backward into a cout-wide window
    float *dz1;
    OPB_TRY(tmp.get(&dz1, npix * cout), "alloc");
    OPB_TRY(train::lrelu_bwd<float>(dy, cout, y, cout, leaky != 0, npix, cout, dz1, nullptr, ho, wo, h, w, st),
            "activation backward");
    OPB_TRY(train::window_add(dz1, cout, npix, cout, dz, cout_p, false, st), "pad");
    OPB_TRY(tmp.get(&dwt, (size_t)cout * cin * 9), "alloc");
    OPB_TRY(tmp.get(&dbt, (size_t)cout), "alloc");
    OPB_TRY(cudaMemsetAsync(dwt, 0, (size_t)cout * cin * 9 * 4, st), "memset");
    OPB_TRY(cudaMemsetAsync(dbt, 0, (size_t)cout * 4, st), "memset");
    train::WgradArgs<float> wa{x, cin, n, h, w, cin, stride, ho, wo, dz, cout_p, cout, dwt};
    OPB_TRY(train::wgrad<float>(wa, dbt, st), "weight gradient");
    if (dw) OPB_TRY(cudaMemcpyAsync(dw, dwt, (size_t)cout * cin * 9 * 4, cudaMemcpyDeviceToDevice, st), "copy");
    if (db) OPB_TRY(cudaMemcpyAsync(db, dbt, (size_t)cout * 4, cudaMemcpyDeviceToDevice, st), "copy");
    if (dx) {
        OPB_TRY(tmp.get(&wkT, (size_t)9 * cout_p * cin_p), "alloc");
        OPB_TRY(tmp.get(&zeros, (size_t)cin_p), "alloc");
        OPB_TRY(tmp.get(&dxp, (size_t)n * h * w * cin_p), "alloc");
        OPB_TRY(cudaMemsetAsync(zeros, 0, (size_t)cin_p * 4, st), "memset");
        OPB_TRY(train::pack_dgrad(w_oihw, cout, cin, cout_p, cin_p, wkT, st), "pack");
        const float *src = dz;
        if (stride == 2) {
            OPB_TRY(tmp.get(&dzd, (size_t)n * h * w * cout_p), "alloc");
            OPB_TRY(cudaMemsetAsync(dzd, 0, (size_t)n * h * w * cout_p * 4, st), "memset");
            OPB_TRY(train::lrelu_bwd<float>(dz, cout_p, dz, cout_p, false, npix, cout_p, nullptr, dzd, ho, wo, h, w,
                                            st),
                    "dilate");
            src = dzd;
        }
        ConvArgs a{src, cout_p, n, h, w, cout_p, 1, h, w, wkT, zeros, cin_p, dxp, cin_p, 0, 1.f, 0};
        OPB_TRY(launch_conv_simt<float>(a, st), "data gradient");
        OPB_TRY(train::window_add(dxp, cin_p, (size_t)n * h * w, cin, dx, cin, false, st), "copy");
    }
    OPB_TRY(cudaStreamSynchronize(st), "tc_op_conv3x3_backward sync");
    return TC_OK;
}

extern "C" tc_status tc_op_correlation_backward(const float *f1, const float *f2, int n, int h, int w, int c, int r,
                                                const float *cost, const float *dcost, float *df1, float *df2,
                                                void *cuda_stream) {
    if (!f1 || !f2 || !cost || !dcost || n < 1 || h < 1 || w < 1 || c < 4 || c % 4 != 0 || r < 1 || r > 4)
        return tc_record_error(TC_ERR_INVALID_ARG, "tc_op_correlation_backward: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int D = (2 * r + 1) * (2 * r + 1);
    train::CorrBwdArgs<float> a{f1, c, f2, c, cost, D, dcost, D, n, h, w, c, r, df1, c, df2, c, 0};
    OPB_TRY(train::corr_bwd<float>(a, st), "correlation backward");
    OPB_TRY(cudaStreamSynchronize(st), "tc_op_correlation_backward sync");
    return TC_OK;
}

extern "C" tc_status tc_op_warp_features_backward(const float *f, const float *flow, int n, int h, int w, int c,
                                                  const float *dout, float *df, float *dflow, void *cuda_stream) {
    if (!f || !flow || !dout || n < 1 || h < 1 || w < 1 || c < 4 || c % 4 != 0)
        return tc_record_error(TC_ERR_INVALID_ARG, "tc_op_warp_features_backward: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (df) OPB_TRY(cudaMemsetAsync(df, 0, (size_t)n * h * w * c * 4, st), "memset");
    train::WarpBwdArgs<float> a{f, c, flow, dout, c, n, h, w, c, df, c, dflow, 0};
    OPB_TRY(train::warp_bwd<float>(a, st), "warp backward");
    OPB_TRY(cudaStreamSynchronize(st), "tc_op_warp_features_backward sync");
    return TC_OK;
}

extern "C" tc_status tc_op_upsample_flow_backward(const float *dfine, int n, int h, int w, int s, float *dcoarse,
                                                  void *cuda_stream) {
    if (!dfine || !dcoarse || n < 1 || h < 1 || w < 1 || (s != 2 && s != 4))
        return tc_record_error(TC_ERR_INVALID_ARG, "tc_op_upsample_flow_backward: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    OPB_TRY(cudaMemsetAsync(dcoarse, 0, (size_t)n * h * w * 2 * 4, st), "memset");
    OPB_TRY(train::up_bwd(dfine, n, h, w, s, dcoarse, st), "upsample backward");
    OPB_TRY(cudaStreamSynchronize(st), "tc_op_upsample_flow_backward sync");
    return TC_OK;
}

extern "C" tc_status tc_op_bruteforce_flow(const float *a, const float *b, int c, int h, int w, int r, int *k_out,
                                           void *cuda_stream) {
    if (!a || !b || !k_out || c < 1 || h < 1 || w < 1 || r < 1 || r > 32)
        return tc_record_error(TC_ERR_INVALID_ARG, "tc_op_bruteforce_flow: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    OPB_TRY(train::bruteforce(a, b, c, h, w, r, k_out, st), "brute-force flow");
    return TC_OK;
}
