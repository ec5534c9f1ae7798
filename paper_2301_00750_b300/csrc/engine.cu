// Stream engine and C ABI (see include/tc_stream.h): per-stream device state, weight
// loading, the per-frame launch sequence of the flow network and the consistency step,
// and the single-stage entry points.
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/tc_stream.h"
#include "common.cuh"
#include "conv_tc.cuh"
#include "engine_internal.h"
#include "solver.cuh"
#include "refine.cuh"
#include "corr_tc.cuh"

namespace tc {

// ------------------------------------------------------------------------------- weights

bool parse_weights(const uint8_t *p, size_t n, HostNet &net, std::string &err) {
    size_t off = 0;
    auto rd = [&](void *dst, size_t k) -> bool {
        if (off + k > n) return false;
        memcpy(dst, p + off, k);
        off += k;
        return true;
    };
    char magic[4];
    if (!rd(magic, 4) || (memcmp(magic, "TCW1", 4) != 0 && memcmp(magic, "TCW2", 4) != 0)) {
        err = "weights: bad magic (want TCW1 or TCW2)";
        return false;
    }
    const bool v2 = memcmp(magic, "TCW2", 4) == 0;
    int32_t lv, rad;
    if (!rd(&lv, 4) || !rd(&rad, 4)) { err = "weights: truncated header"; return false; }
    if (lv < 2 || lv > 7 || rad < 1 || rad > 4) { err = "weights: levels must be 2..7 and radius 1..4"; return false; }
    net.levels = lv;
    net.radius = rad;
    net.chans.resize(lv);
    if (!rd(net.chans.data(), 4 * lv) || !rd(net.dec, 16)) { err = "weights: truncated header"; return false; }
    int32_t nl;
    if (!rd(&nl, 4)) { err = "weights: truncated header"; return false; }
    const int want = 3 * lv + 5 * (lv - 1);
    if (nl != want) { err = "weights: layer count does not match the level count"; return false; }
    const int D = (2 * rad + 1) * (2 * rad + 1);
    for (int i = 0; i < nl; ++i) {
        HostLayer L;
        int32_t h4[4];
        if (!rd(h4, 16)) { err = "weights: truncated layer header"; return false; }
        L.cout = h4[0]; L.cin = h4[1]; L.stride = h4[2]; L.leaky = h4[3];
        if (L.cout < 1 || L.cin < 1 || L.cout > 4096 || L.cin > 4096) { err = "weights: bad layer shape"; return false; }
        L.w.resize((size_t)L.cout * L.cin * 9);
        L.b.resize(L.cout);
        if (!rd(L.w.data(), 4 * L.w.size()) || !rd(L.b.data(), 4 * L.b.size())) { err = "weights: truncated layer data"; return false; }
        net.layers.push_back(std::move(L));
    }
    // Shape checks against the architecture (Sec. 3.2).
    int prev = 3;
    for (int l = 0; l < lv; ++l) {
        const int c = net.chans[l];
        const HostLayer *P = &net.layers[3 * l];
        if (c % 4 != 0 || c > 256) { err = "weights: pyramid channels must be multiples of 4, <= 256"; return false; }
        if (P[0].cin != prev || P[0].cout != c || P[0].stride != 2 || P[1].cin != c || P[1].cout != c ||
            P[2].cin != c || P[2].cout != c || P[1].stride != 1 || P[2].stride != 1) {
            err = "weights: pyramid layer shapes do not match the channel list"; return false;
        }
        prev = c;
    }
    if (net.chans[0] > 64) { err = "weights: first pyramid level must have <= 64 channels"; return false; }
    for (int k = 0; k < 4; ++k)
        if (net.dec[k] % 4 != 0 || net.dec[k] <= 0) { err = "weights: decoder widths must be multiples of 4"; return false; }
    for (int l = lv; l >= 2; --l) {
        const HostLayer *E = &net.layers[3 * lv + 5 * (lv - l)];
        const int c0 = D + net.chans[l - 1] + 2;
        if (E[0].cin != c0 || E[0].cout != net.dec[0] || E[1].cin != net.dec[0] || E[1].cout != net.dec[1] ||
            E[2].cin != net.dec[1] || E[2].cout != net.dec[2] || E[3].cin != net.dec[2] + net.dec[1] ||
            E[3].cout != net.dec[3] || E[4].cin != net.dec[3] + net.dec[2] || E[4].cout != 2) {
            err = "weights: estimator layer shapes do not match the architecture"; return false;
        }
        for (int j = 0; j < 5; ++j)
            if (E[j].stride != 1) { err = "weights: estimator convs must have stride 1"; return false; }
    }
    net.ref.clear();
    if (v2) {
        // the refinement section: reads cat(flow, x4, x3) of the level-2 estimator
        int32_t nr;
        if (!rd(&nr, 4) || nr < 1 || nr > 16) { err = "weights: refinement layer count must be 1..16"; return false; }
        int cin = 2 + net.dec[3] + net.dec[2];
        for (int k = 0; k < nr; ++k) {
            HostSep R;
            int32_t h4[4];
            if (!rd(h4, 16)) { err = "weights: truncated refinement header"; return false; }
            R.cin = h4[0]; R.cout = h4[1]; R.dil = h4[2]; R.leaky = h4[3];
            const bool last = k == nr - 1;
            if (R.cin != cin || R.dil < 1 || R.dil > 64 || (last ? (R.cout != 2 || R.leaky) : (R.cout % 8 != 0 || R.cout > 256))) {
                err = "weights: refinement layer shapes (cin chain from 2 + x4 + x3, cout multiple of 8 up to 256, "
                      "the last 2 outputs without activation, dilation 1..64)";
                return false;
            }
            R.dw.resize((size_t)R.cin * 9);
            R.db.resize(R.cin);
            R.pw.resize((size_t)R.cout * R.cin);
            R.pb.resize(R.cout);
            if (!rd(R.dw.data(), 4 * R.dw.size()) || !rd(R.db.data(), 4 * R.db.size()) ||
                !rd(R.pw.data(), 4 * R.pw.size()) || !rd(R.pb.data(), 4 * R.pb.size())) {
                err = "weights: truncated refinement data";
                return false;
            }
            cin = R.cout;
            net.ref.push_back(std::move(R));
        }
    }
    return true;
}

// 16-bit tensor-core precisions: bfloat16 (TC_BF16) or IEEE half (TC_FP16) operands.
static inline bool is16(tc_precision p) { return p == TC_BF16 || p == TC_FP16; }

// The value a float weight takes as an operand of precision p: rounded to bfloat16 or half
// for the 16-bit paths; unchanged otherwise (float, and e4m3, which quantises per channel
// when it plans its layers).
static inline float operand_value(float v, tc_precision p) {
    if (p == TC_BF16) return __bfloat162float(__float2bfloat16_rn(v));
    if (p == TC_FP16) return __half2float(__float2half_rn(v));
    return v;
}

// [9 * cin_pad][cout] layout for the SIMT conv; input channel ci of the buffer maps to
// channel perm[ci] of the file's layer (-1 = zero padding).  The weights take their operand
// values for precision p (see operand_value).
static std::vector<float> simt_weights(const HostLayer &L, const std::vector<int> &perm, tc_precision p) {
    const int cp = (int)perm.size();
    std::vector<float> out((size_t)9 * cp * L.cout, 0.f);
    for (int tap = 0; tap < 9; ++tap)
        for (int ci = 0; ci < cp; ++ci) {
            const int c = perm[ci];
            if (c < 0) continue;
            for (int o = 0; o < L.cout; ++o) {
                float v = L.w[(((size_t)o * L.cin + c) * 3 + tap / 3) * 3 + tap % 3];
                out[((size_t)tap * cp + ci) * L.cout + o] = operand_value(v, p);
            }
        }
    return out;
}

static std::vector<int> iota_perm(int n, int pad_to) {
    std::vector<int> p(pad_to, -1);
    for (int i = 0; i < n; ++i) p[i] = i;
    return p;
}

static inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Feature pyramids kept per stream: frame t's lives in slot t % 2 (t % NPYR in pipelined
// mode), and the flow estimation of frame t reads the slots of t and t - 1.  With four
// slots, the pyramids of the next frames never overwrite one that a flow estimation still in
// flight reads (pipelined mode runs two of them and the next pyramid at the same time).
constexpr int NPYR = 4;
// Estimator buffer sets (decoder activations, warped features, flows): pipelined mode
// estimates frame t with set t % 2, so two frames' flow estimations can run at once.
constexpr int NSET = 2;
// A pipelined frame's flow estimation depends on t through its buffer set (t % 2) and the
// pyramid slots (t % 4): one captured graph per t % NGRAPH.
constexpr int NGRAPH = 4;

size_t stream_device_bytes(const HostNet &net, int width, int height, tc_precision prec, int fs, int lanes) {
    // a single stream (lanes = 0) keeps NPYR pyramid slots and NSET estimator sets; a batch
    // of `lanes` lanes keeps two slots (current, previous) and one set per lane
    const size_t npyr = lanes ? 2 * (size_t)lanes : NPYR, nest = lanes ? 2 * (size_t)lanes : 2 * NSET;
    const size_t nl = lanes ? (size_t)lanes : 1;
    const int L = net.levels, D = (2 * net.radius + 1) * (2 * net.radius + 1), m = 1 << L;
    const bool f8 = prec == TC_FP8_E4M3;
    const size_t es = prec == TC_FP32 ? 4 : (f8 ? 1 : 2);
    const int wn = (width + fs - 1) / fs, hn = (height + fs - 1) / fs;  // the flow network's input
    const size_t Hp = (size_t)round_up(hn, m), Wp = (size_t)round_up(wn, m);
    const bool bf = prec != TC_FP32;
    auto al = [](size_t b) { return (b + 511) & ~(size_t)511; };  // allocation granularity
    // packed tensor-core weights (bf16, or e4m3 plus one float scale per output channel)
    auto tcw = [&](int cin, int cout) {
        return !bf ? 0 : f8 ? al((size_t)9 * cout * round_up(cin, 128)) + al((size_t)cout * 4)
                            : al((size_t)9 * cout * round_up(cin, 64) * 2);
    };
    size_t total = al(sizeof(int)) + al(sizeof(unsigned) * (3 * L + 6 * (L - 1)));  // error word, amax slots
    int prev = 3;
    for (int l = 1; l <= L; ++l) {
        const size_t h = Hp >> l, w = Wp >> l, px = h * w;
        const int c = net.chans[l - 1];
        total += al(npyr * px * c * es) + 2 * al(nl * px * c * es);
        total += al((size_t)9 * prev * c * 4) + al((size_t)c * 4) + 2 * (al((size_t)9 * c * c * 4) + al((size_t)c * 4));
        if (l > 1) total += tcw(prev, c);
        total += 2 * tcw(c, c);
        prev = c;
        if (l < 2) continue;
        const int x0p = round_up(c + D + 2, f8 ? 16 : 8);
        const int ctot = x0p + net.dec[0] + net.dec[1] + net.dec[2] + net.dec[3];
        total += al(nest * px * ctot * es) + al(nest * px * c * es) + 2 * al(nest * px * 2 * 4);
        const int cin[5] = {x0p, net.dec[0], net.dec[1], net.dec[1] + net.dec[2], net.dec[2] + net.dec[3]};
        const int cout[5] = {net.dec[0], net.dec[1], net.dec[2], net.dec[3], 2};
        for (int j = 0; j < 5; ++j) {
            total += al((size_t)9 * cin[j] * cout[j] * 4) + al((size_t)cout[j] * 4);
            total += j < 4 ? tcw(cin[j], cout[j]) : tcw(cin[j], 16);
        }
    }
    const size_t img = al((size_t)3 * height * width * 4), plane = (size_t)height * width;
    // kept state, 2 slots: two 16-byte words and one float per pixel (per lane)
    const size_t px_all = (size_t)height * width * (lanes ? nl : 1);
    const size_t kept = 2 * (2 * al(px_all * 16) + al(px_all * 4));
    if (lanes) return total + kept;
    total += kept;
    total += 3 * img + al(plane * 4) + al(plane);            // host-entry staging
    if (fs > 1) total += al((size_t)3 * hn * wn * 4);        // the downscaled frame
    if (!net.ref.empty()) {                                  // refinement buffers and weights
        const size_t px2 = (Hp >> 2) * (Wp >> 2);
        int dcs = 0, pcs = 8;
        for (size_t k = 0; k < net.ref.size(); ++k) {
            dcs = std::max(dcs, round_up(net.ref[k].cin, 8));
            if (k + 1 < net.ref.size()) pcs = std::max(pcs, round_up(net.ref[k].cout, 8));
            const size_t cp = round_up(net.ref[k].cin, 8);
            total += al(9 * cp * 4) + al(cp * 4) + al(cp * net.ref[k].cout * 4) + al(net.ref[k].cout * 4);
            if (bf) total += al(cp * std::max(16, net.ref[k].cout) * 2);
        }
        total += al(NSET * 2 * px2 * dcs * es) + al(NSET * 2 * px2 * pcs * es);
    }
    return total;
}

}  // namespace tc

using namespace tc;

// ------------------------------------------------------------------------------- stream

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct LevelBufs {
    int h = 0, w = 0, c = 0;
    void *pyr = nullptr;   // [NPYR slots][h][w][c]
    void *tmpA = nullptr;  // [h][w][c]
    void *tmpB = nullptr;
    // estimator (l >= 2)
    int x0p = 0, ctot = 0;
    int off_x1 = 0, off_x2 = 0, off_x3 = 0, off_x4 = 0;
    void *dec = nullptr;   // [NSET sets][2 dirs][h][w][ctot]
    void *f2w = nullptr;   // [NSET][2][h][w][c]
    float *flow = nullptr; // [NSET][2][h][w][2]
    float *up = nullptr;   // [NSET][2][h][w][2]
    // device weights of the estimator
    float *wk[4] = {nullptr, nullptr, nullptr, nullptr};
    float *bias[4] = {nullptr, nullptr, nullptr, nullptr};
    float *head_w = nullptr, *head_b = nullptr;
    TcConvPlan tcplan[4];
    TcConvPlan headplan;
    // activation scales (e4m3 streams; 1 otherwise): pyramid conv a/b/c outputs, and the
    // estimator segments cost volume, up-flow, x1..x4.  q = 1 / s.
    float s_pyr[3] = {1.f, 1.f, 1.f}, q_pyr[3] = {1.f, 1.f, 1.f};
    float s_est[6] = {1.f, 1.f, 1.f, 1.f, 1.f, 1.f}, q_est[6] = {1.f, 1.f, 1.f, 1.f, 1.f, 1.f};
    CorrTcPlan corrplan;   // BF16: self = pyramid slots, other = pyramid (coarsest) or f2w
};

// Buffer set `set` of a level's estimator buffers.
template <typename T> static T *dec_of(const LevelBufs &B, int set) {
    return static_cast<T *>(B.dec) + (size_t)set * 2 * B.h * B.w * B.ctot;
}
template <typename T> static T *f2w_of(const LevelBufs &B, int set) {
    return static_cast<T *>(B.f2w) + (size_t)set * 2 * B.h * B.w * B.c;
}
static float *flow_of(const LevelBufs &B, int set) { return B.flow + (size_t)set * B.h * B.w * 4; }
static float *up_of(const LevelBufs &B, int set) { return B.up + (size_t)set * B.h * B.w * 4; }

}  // namespace

struct tc_stream {
    int W = 0, H = 0, Wp = 0, Hp = 0;
    // the flow network's input: the frame (fs = 1) or its 2x2 means (fs = 2, the fast
    // preset), Wn x Hn = ceil(W / fs) x ceil(H / fs), padded to Wp x Hp
    int fs = 1, Wn = 0, Hn = 0;
    float *xs = nullptr;
    tc_precision prec = TC_FP32;
    cudaStream_t st = nullptr;
    HostNet net;
    int L = 0, R = 0, D = 0;
    tc_consistency params{};
    std::vector<void *> allocs;
    std::vector<LevelBufs> lv;  // index l-1
    // pyramid weights per level (3 convs)
    std::vector<float *> pyr_w, pyr_b;
    std::vector<float> first_w, first_b;  // host copy of the first conv ([27][cout], cout)
    TcConvPlan pyr_plan[8][3];
    // kept state ring: [2 slots] of the interleaved layout of ConsistArgs, (H, W) pixels per
    // lane: kA = (I0, I1, I2, P0), kB = (P1, P2, O0, O1), kC = O2
    float4 *kA[2] = {nullptr, nullptr}, *kB[2] = {nullptr, nullptr};
    float *kC[2] = {nullptr, nullptr};
    // staging for the host entry point
    float *hI = nullptr, *hP = nullptr, *hO = nullptr, *hwc = nullptr;
    uint8_t *hmask = nullptr;
    long long t = 0;
    bool poisoned = false;
    int *dev_err = nullptr;     // device error word of the tensor-core kernels (0 = ok)
    int tc_layers = 0;          // convolution layers planned on the tensor cores
    int tc_corr_levels = 0;     // pyramid levels whose correlation runs on the tensor cores
    size_t dev_bytes = 0;       // device bytes allocated by the stream itself
    // Tensor-core layers with what planning them needs (planned at creation for BF16, when
    // the activation scales arrive for E4M3).
    struct LayerRec {
        TcConvPlan *plan;
        ConvArgs a;
        int n_in;
        std::vector<float> wk;      // [9 * cin][cout] in buffer channel order
        std::vector<int> in_seg;    // activation segment of each input channel (-1: zero pad)
        bool head;
    };
    std::vector<LayerRec> recs;
    bool fp8_ready = false;
    // amax of every activation segment (FP32 / BF16 streams, for E4M3 calibration)
    bool rec_amax = false;
    unsigned *amax_dev = nullptr;
    int launches = 0;
    std::string err;
    // per-stage timing (tc_set_profiling): events around every launch, folded lazily
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int> ev_cat;       // category of pending pair k (events 2k, 2k+1)
    double prof_ms[TC_PROF_CATEGORIES] = {0};
    long long prof_n[TC_PROF_CATEGORIES] = {0};
    // CUDA graphs of a whole frame, one per t % NGRAPH (the pointers of every launch depend
    // only on the state parity and the pyramid slots, except the caller's buffers read by the
    // first pyramid conv and the consistency pass, whose nodes are updated before each replay).
    bool graphs = true;
    cudaStream_t gst = nullptr;               // library stream the graphs are captured on and replayed on
    // tc_process_frame_host uploads P_t on cst while the flow network runs and records ev_p
    // after it; the pass that reads P_t waits on ev_p (in the host calls' graphs: an external
    // event node on a side branch).  Device calls have P_t already and wait for nothing.
    cudaStream_t cst = nullptr;
    cudaEvent_t ev_p = nullptr;
    bool p_pending = false;  // this frame's P_t arrives through the upload on cst
    bool capturing = false;  // frame_launches is being captured into a graph
    // tc_process_frame_host_async: device staging per slot (call parity), the download
    // stream, and per slot: inputs uploaded, frame done, outputs downloaded
    // (two slots in the default mode, four in pipelined mode, where the inputs of the next
    // frames' pyramids and of the frames still blending are alive at once)
    static constexpr int NSLOT = 4;
    float *aI[NSLOT] = {}, *aP[NSLOT] = {}, *aO[NSLOT] = {}, *awc[NSLOT] = {};
    uint8_t *amask[NSLOT] = {};
    uint8_t *a8I[NSLOT] = {}, *a8P[NSLOT] = {}, *a8O[NSLOT] = {};  // tc_process_frame_host_rgb8_async: 8-bit staging
    cudaStream_t dst = nullptr;
    cudaEvent_t a_in[NSLOT] = {}, a_done[NSLOT] = {}, a_out[NSLOT] = {};
    long long a_n = 0;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;  // capture: the wait on ev_p as a side branch
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;  // fence gst to the caller's stream
    struct FrameGraph {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaGraphNode_t n_first = nullptr, n_cons = nullptr, n_copy = nullptr, n_in = nullptr;
        cudaKernelNodeParams p_first{}, p_cons{}, p_copy{}, p_in{};
        int launches = 0;
    } fg[2][2];  // [host entry point][t % 2]: only host calls' graphs wait for the P_t upload
    // pipelined mode (tc_set_pipelined): the pyramid of frame t runs on pst, its flow
    // estimation on the stream of its buffer set, its blend on bst; see process_pipelined
    bool pipelined = false;
    int last_blend = -1;  // event ring index of the last frame's blend
    int last_set = 0;     // estimator buffer set of the last frame given
    cudaStream_t pst = nullptr, bst = nullptr;  // pyramid, blend
    cudaStream_t estx[NSET - 1] = {};           // estimation of sets 1.. (set 0: gst)
    static constexpr int NEV = 8;  // event rings, indexed by t % NEV
    cudaEvent_t ev_pyrs[NEV] = {}, ev_ests[NEV] = {}, ev_blends[NEV] = {};  // pyramid / estimation / blend of frame t done
    FrameGraph pg_pyr[NPYR], pg_est[NGRAPH], pg_blend[NGRAPH];
    // screened-Poisson solver (allocated when first enabled): A_t, w_c, right-hand side and
    // four iterate planes, each (3, H, W) float (w_c (H, W))
    // solver: A_t and w_c from the blend, its result, the planar P_t copy, coefficients, scratch
    float *sv_A = nullptr, *sv_wc = nullptr, *sv_O = nullptr, *sv_P = nullptr, *sv_b = nullptr, *sv_c0 = nullptr,
          *sv_s[4] = {nullptr, nullptr, nullptr, nullptr};
    // one frame of latency (tc_set_latency): frame t is blended when frame t+1 arrives, with
    // the final flows of the pair (t, t-1) kept from the previous call ((2, h_2, w_2, 2) float)
    int latency = 0;
    float *Fprev = nullptr;
    long long last_out = -1;  // index in its sequence of the frame the last call wrote
    // refinement network (TCW2): per layer the depthwise taps and bias and the pointwise
    // weights in buffer channel order, its tensor-core plan (BF16) or none (CUDA cores);
    // refD holds the depthwise outputs, refP the pointwise ones, both for the two flow
    // directions at level 2, one copy per estimator buffer set
    struct RefLayer {
        int cin_p = 0, nin = 0, cout = 0, dil = 1, leaky = 1;
        float *dw = nullptr, *db = nullptr, *pw = nullptr, *pb = nullptr;
        TcConvPlan plan;
    };
    std::vector<RefLayer> ref;
    void *refD = nullptr, *refP = nullptr;
    int refD_cs = 0, refP_cs = 0;
    // batch (tc_create_batch): `lanes` independent causal streams of one size whose feature
    // pyramids and flow estimations run in shared launches (the lanes are the images of
    // every buffer); per lane its frame count, its state slot and its consistency controls.
    // The pyramid buffers hold two slots of `lanes` images: slot 0 the current frames, slot
    // 1 every lane's previous frame (copied from slot 0 after each step of the lane).
    bool batch = false;
    int lanes = 1;
    int npyr = NPYR;       // images of a level's pyramid buffer
    int n_est = 2 * NSET;  // images of a level's estimator buffers
    std::vector<long long> lane_t;
    std::vector<int> lane_cur;  // state slot the lane's next frame writes
    std::vector<tc_consistency> lane_params;
    // the shared launches of lanes [lo, lo + n), key lo * 4096 + n: uses so far, and the
    // graph captured on the second use
    std::map<int, int> range_uses;
    std::map<int, FrameGraph> range_graphs;
    // per-frame latency in pipelined mode (tc_set_frame_timing): a timing event when a
    // frame's pyramid may start (its stream past its waits) and one when its blend ends
    bool frame_timing = false;
    std::vector<cudaEvent_t> ft_start, ft_done;
    size_t ft_n = 0;
};

static std::mutex g_err_mu;
static std::string g_err;
static int g_last_op_tc = 0;  // 1 if the last tc_op_conv3x3 ran on the tensor cores

static tc_status fail(tc_stream *s, tc_status code, const std::string &msg) {
    if (s) {
        s->err = msg;
        if (code == TC_ERR_CUDA) s->poisoned = true;
    } else {
        std::lock_guard<std::mutex> lk(g_err_mu);
        g_err = msg;
    }
    return code;
}

tc_status tc_record_error(tc_status code, const std::string &msg) { return fail(nullptr, code, msg); }

static tc_status cuda_fail(tc_stream *s, cudaError_t e, const char *what) {
    return fail(s, TC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define TC_TRY(stream, expr, what)                                  \
    do {                                                            \
        cudaError_t _e = (expr);                                    \
        if (_e != cudaSuccess) return cuda_fail(stream, _e, what);  \
    } while (0)

// Test hook (tc_test_fail_device_allocation): the stream device allocation that brings
// this countdown from 1 to 0 fails as an out-of-memory cudaMalloc would.
static std::atomic<long long> g_alloc_fail_countdown{0};

static tc_status dalloc(tc_stream *s, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    bool inject = false;
    if (g_alloc_fail_countdown.load() > 0) inject = g_alloc_fail_countdown.fetch_sub(1) == 1;
    cudaError_t e = inject ? cudaErrorMemoryAllocation : cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(s, TC_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    s->allocs.push_back(*p);
    s->dev_bytes += bytes;
    return TC_OK;
}

template <typename P>
static tc_status dalloc_t(tc_stream *s, P **p, size_t bytes) {
    void *v = nullptr;
    tc_status r = dalloc(s, &v, bytes);
    *p = static_cast<P *>(v);
    return r;
}

static tc_status upload(tc_stream *s, float **dst, const std::vector<float> &v) {
    tc_status r = dalloc_t(s, dst, v.size() * sizeof(float));
    if (r != TC_OK) return r;
    TC_TRY(s, cudaMemcpy(*dst, v.data(), v.size() * sizeof(float), cudaMemcpyHostToDevice), "weight upload");
    return TC_OK;
}

static void free_all(tc_stream *s) {
    for (cudaEvent_t e : s->ft_start) cudaEventDestroy(e);
    for (cudaEvent_t e : s->ft_done) cudaEventDestroy(e);
    s->ft_start.clear();
    s->ft_done.clear();
    for (auto &B : s->lv) {
        for (auto &pl : B.tcplan) pl.release();
        B.headplan.release();
    }
    for (auto &lvl : s->pyr_plan)
        for (auto &pl : lvl) pl.release();
    for (auto &R : s->ref) R.plan.release();
    for (void *p : s->allocs) cudaFree(p);
    s->allocs.clear();
}

extern "C" void tc_default_consistency(tc_consistency *p) {
    if (!p) return;
    p->k1 = 0.3f;
    p->k2 = 0.5f;
    p->alpha = 6.5e3f;
    p->lambda = 2.0f;
    p->fb_check = 1;
    p->fb_c1 = 0.01f;
    p->fb_c2 = 0.5f;
    p->solver_iters = 0;
    p->eta = 0.15f;
    p->kappa = 0.2f;
}

static bool valid_params(const tc_consistency *p, std::string &why) {
    auto finite = [](float v) { return std::isfinite(v); };
    if (!finite(p->k1) || !finite(p->alpha) || !finite(p->lambda) || !finite(p->fb_c1) || !finite(p->fb_c2)) {
        why = "consistency parameters must be finite";
        return false;
    }
    if (p->k1 < 0.f || p->k1 > 1.f) { why = "k1 must lie in [0, 1]"; return false; }
    if (p->alpha < 0.f || p->lambda < 0.f) { why = "alpha and lambda must be >= 0"; return false; }
    if (!finite(p->k2) || p->k2 < 0.f || p->k2 > 1.f) { why = "k2 must lie in [0, 1]"; return false; }
    if (p->solver_iters < 0 || p->solver_iters > 10000) { why = "solver_iters must lie in [0, 10000]"; return false; }
    if (p->solver_iters > 0 && (!finite(p->eta) || !finite(p->kappa) || p->eta <= 0.f || p->kappa < 0.f ||
                                p->kappa >= 1.f)) {
        why = "the solver needs eta > 0 and 0 <= kappa < 1";
        return false;
    }
    return true;
}

static void release_graphs(tc_stream *s);

extern "C" tc_status tc_set_consistency(tc_stream *s, const tc_consistency *p) {
    if (!s || !p) return fail(s, TC_ERR_INVALID_ARG, "tc_set_consistency: NULL argument");
    std::string why;
    if (!valid_params(p, why)) return fail(s, TC_ERR_INVALID_ARG, why);
    if (s->batch) {
        // a batch: every lane's controls (tc_set_lane_consistency sets one lane's)
        if (p->solver_iters != 0) return fail(s, TC_ERR_UNSUPPORTED, "tc_set_consistency: a batch runs without the solver");
        for (auto &lp : s->lane_params) lp = *p;
        s->params = *p;
        return TC_OK;
    }
    if (s->latency && !(p->k1 + p->k2 < 1.f))
        return fail(s, TC_ERR_INVALID_ARG, "with the next-frame term k1 + k2 must be < 1");
    if (p->solver_iters > 0 && !s->sv_A) {
        const size_t img = (size_t)3 * s->H * s->W * sizeof(float), plane = (size_t)s->H * s->W * sizeof(float);
        tc_status r;
        if ((r = dalloc_t(s, &s->sv_A, img)) != TC_OK || (r = dalloc_t(s, &s->sv_wc, plane)) != TC_OK ||
            (r = dalloc_t(s, &s->sv_O, img)) != TC_OK || (r = dalloc_t(s, &s->sv_P, img)) != TC_OK ||
            (r = dalloc_t(s, &s->sv_b, img)) != TC_OK || (r = dalloc_t(s, &s->sv_c0, plane)) != TC_OK)
            return r;
        for (int k = 0; k < 4; ++k)
            if ((r = dalloc_t(s, &s->sv_s[k], img)) != TC_OK) return r;
    }
    // the solver's launches are part of a captured frame: a change of its settings needs a
    // new capture (the consistency controls are updated per frame without one)
    if (p->solver_iters != s->params.solver_iters ||
        (p->solver_iters > 0 && (p->eta != s->params.eta || p->kappa != s->params.kappa))) {
        if (s->st) cudaStreamSynchronize(s->st);
        release_graphs(s);
    }
    s->params = *p;
    return TC_OK;
}

// Activation segments: the outputs of pyramid conv a/b/c of level l, and the estimator
// input segments of level l (cost volume, up-flow, x1, x2, x3, x4).  E4M3 scales and amax
// records are indexed this way.
static int seg_pyr(const tc_stream *s, int l, int j) { return 3 * (l - 1) + j; }
static int seg_est(const tc_stream *s, int l, int k) { return 3 * s->L + 6 * (s->L - l) + k; }
static int n_segments(const tc_stream *s) { return 3 * s->L + 6 * (s->L - 1); }

// Records a tensor-core layer; BF16 layers are planned at once (layers that are not
// eligible keep the CUDA-core kernel), and so are FP16 layers; E4M3 layers when the scales
// are set.
static void add_layer(tc_stream *s, TcConvPlan &plan, const ConvArgs &a, int n_in, std::vector<float> wk,
                      std::vector<int> in_seg, bool head) {
    if (s->prec == TC_FP32) return;
    if (is16(s->prec)) {
        std::string why;
        const bool f16 = s->prec == TC_FP16;
        const bool ok = head ? tc_plan_head(plan, a, n_in, wk, s->dev_err, why, false, 9, f16)
                             : tc_plan_conv(plan, a, n_in, wk, s->dev_err, why, false, 9, f16);
        if (ok) s->tc_layers += 1;
        return;
    }
    s->recs.push_back(tc_stream::LayerRec{&plan, a, n_in, std::move(wk), std::move(in_seg), head});
}

// Refinement layers of a TCW2 net: weights in buffer channel order (the first layer's
// input is [x3 | x4 | flow | zero pad] in the buffers, cat(flow, x4, x3) in the file),
// the two activation buffers, and for BF16 a pointwise tensor-core plan per layer.
template <typename T>
static tc_status build_refine(tc_stream *s) {
    const HostNet &net = s->net;
    if (s->prec == TC_FP8_E4M3)
        return fail(s, TC_ERR_UNSUPPORTED, "the refinement network runs in TC_FP32, TC_BF16 or TC_FP16 streams");
    const LevelBufs &B = s->lv[1];
    const size_t px = (size_t)B.h * B.w;
    const int c3 = net.dec[2], c4 = net.dec[3];
    auto ru8 = [](int v) { return (v + 7) / 8 * 8; };
    const int nl = (int)net.ref.size();
    s->ref.resize(nl);
    int dcs = 0, pcs = 8;
    for (int k = 0; k < nl; ++k) {
        dcs = std::max(dcs, ru8(net.ref[k].cin));
        if (k < nl - 1) pcs = std::max(pcs, ru8(net.ref[k].cout));
    }
    s->refD_cs = dcs;
    s->refP_cs = pcs;
    tc_status r;
    if ((r = dalloc(s, &s->refD, NSET * 2 * px * dcs * sizeof(T))) != TC_OK) return r;
    if ((r = dalloc(s, &s->refP, NSET * 2 * px * pcs * sizeof(T))) != TC_OK) return r;
    TC_TRY(s, cudaMemset(s->refD, 0, NSET * 2 * px * dcs * sizeof(T)), "memset");
    TC_TRY(s, cudaMemset(s->refP, 0, NSET * 2 * px * pcs * sizeof(T)), "memset");
    for (int k = 0; k < nl; ++k) {
        const HostSep &H = net.ref[k];
        tc_stream::RefLayer &R = s->ref[k];
        R.cin_p = ru8(H.cin);
        R.nin = k == 0 ? c3 + c4 : H.cin;
        R.cout = H.cout;
        R.dil = H.dil;
        R.leaky = H.leaky;
        // buffer channel g -> file channel (-1: zero padding)
        std::vector<int> src(R.cin_p, -1);
        for (int g = 0; g < H.cin; ++g) {
            if (k > 0) src[g] = g;
            else if (g < c3) src[g] = 2 + c4 + g;            // x3
            else if (g < c3 + c4) src[g] = 2 + (g - c3);     // x4
            else src[g] = g - c3 - c4;                       // flow u, v
        }
        std::vector<float> dw((size_t)9 * R.cin_p, 0.f), db(R.cin_p, 0.f), pw((size_t)R.cin_p * H.cout, 0.f);
        for (int g = 0; g < R.cin_p; ++g) {
            if (src[g] < 0) continue;
            for (int t = 0; t < 9; ++t) dw[(size_t)t * R.cin_p + g] = H.dw[(size_t)src[g] * 9 + t];
            db[g] = H.db[src[g]];
            for (int o = 0; o < H.cout; ++o) pw[(size_t)g * H.cout + o] = H.pw[(size_t)o * H.cin + src[g]];
        }
        if ((r = upload(s, &R.dw, dw)) != TC_OK || (r = upload(s, &R.db, db)) != TC_OK ||
            (r = upload(s, &R.pw, pw)) != TC_OK || (r = upload(s, &R.pb, H.pb)) != TC_OK)
            return r;
        if (is16(s->prec)) {
            const bool last = k == nl - 1;
            const bool f16 = s->prec == TC_FP16;
            ConvArgs a{s->refD, dcs, 1, B.h, B.w, R.cin_p, 1, B.h, B.w, nullptr, nullptr, last ? 2 : H.cout,
                       last ? nullptr : s->refP, last ? 16 : pcs, H.leaky};
            std::string why;
            const bool ok = last ? tc_plan_head(R.plan, a, 2 * NSET, pw, s->dev_err, why, false, 1, f16)
                                 : tc_plan_conv(R.plan, a, 2 * NSET, pw, s->dev_err, why, false, 1, f16);
            if (ok) s->tc_layers += 1;
        }
    }
    return TC_OK;
}

template <typename T>
static tc_status build_stream(tc_stream *s) {
    const HostNet &net = s->net;
    const bool bf = s->prec != TC_FP32;
    const size_t es = sizeof(T);
    const int L = s->L, D = s->D;
    const int cal = es == 1 ? 16 : 8;  // channel-offset alignment: 16 bytes
    s->lv.resize(L);
    s->pyr_w.assign(3 * L, nullptr);
    s->pyr_b.assign(3 * L, nullptr);
    tc_status r;
    if ((r = dalloc_t(s, &s->dev_err, sizeof(int))) != TC_OK) return r;
    TC_TRY(s, cudaMemset(s->dev_err, 0, sizeof(int)), "memset");
    if ((r = dalloc_t(s, &s->amax_dev, sizeof(unsigned) * n_segments(s))) != TC_OK) return r;
    TC_TRY(s, cudaMemset(s->amax_dev, 0, sizeof(unsigned) * n_segments(s)), "memset");
    for (int l = 1; l <= L; ++l) {
        LevelBufs &B = s->lv[l - 1];
        B.h = s->Hp >> l;
        B.w = s->Wp >> l;
        B.c = net.chans[l - 1];
        const size_t px = (size_t)B.h * B.w;
        if ((r = dalloc(s, &B.pyr, s->npyr * px * B.c * es)) != TC_OK) return r;
        if ((r = dalloc(s, &B.tmpA, s->lanes * px * B.c * es)) != TC_OK) return r;
        if ((r = dalloc(s, &B.tmpB, s->lanes * px * B.c * es)) != TC_OK) return r;
        for (int j = 0; j < 3; ++j) {
            const HostLayer &HL = net.layers[3 * (l - 1) + j];
            std::vector<float> wk;
            if (l == 1 && j == 0) {
                // [27][cout], k = c * 9 + tap
                wk.assign(27 * HL.cout, 0.f);
                for (int o = 0; o < HL.cout; ++o)
                    for (int k = 0; k < 27; ++k) {
                        float v = HL.w[(size_t)o * 27 + k];
                        // the first conv reads the float image: its weights take the 16-bit
                        // operand values (bfloat16 also for e4m3 streams)
                        if (bf) v = operand_value(v, s->prec == TC_FP16 ? TC_FP16 : TC_BF16);
                        wk[(size_t)k * HL.cout + o] = v;
                    }
            } else {
                wk = simt_weights(HL, iota_perm(HL.cin, HL.cin), s->prec);
            }
            if ((r = upload(s, &s->pyr_w[3 * (l - 1) + j], wk)) != TC_OK) return r;
            if ((r = upload(s, &s->pyr_b[3 * (l - 1) + j], HL.b)) != TC_OK) return r;
            if (l == 1 && j == 0) {
                s->first_w = wk;
                s->first_b = HL.b;
                continue;
            }
            // Same arguments as run_pyramid builds; the first conv of a level reads any
            // slot of the previous level's pyramid buffer.
            if (j == 0) {
                LevelBufs &P = s->lv[l - 2];
                ConvArgs a{P.pyr, P.c, 1, P.h, P.w, P.c, 2, B.h, B.w, nullptr, nullptr, B.c, B.tmpA, B.c, 1};
                add_layer(s, s->pyr_plan[l - 1][0], a, s->npyr, wk, std::vector<int>(P.c, seg_pyr(s, l - 1, 2)), false);
            } else {
                ConvArgs a{j == 1 ? B.tmpA : B.tmpB, B.c, 1, B.h, B.w, B.c, 1, B.h, B.w, nullptr, nullptr, B.c,
                           B.tmpB, B.c, 1};
                add_layer(s, s->pyr_plan[l - 1][j], a, s->lanes, wk, std::vector<int>(B.c, seg_pyr(s, l, j - 1)), false);
            }
        }
        if (l < 2) continue;
        // Estimator buffers: x0 = [self c | corr D | up 2 | zero pad] then x1..x4 (the file's
        // order cat(corr, self, up) is restored by permuting conv1's input channels).
        B.x0p = round_up(B.c + D + 2, cal);
        B.off_x1 = B.x0p;
        B.off_x2 = B.off_x1 + net.dec[0];
        B.off_x3 = B.off_x2 + net.dec[1];
        B.off_x4 = B.off_x3 + net.dec[2];
        B.ctot = B.off_x4 + net.dec[3];
        const size_t ne = (size_t)s->n_est;
        if ((r = dalloc(s, &B.dec, ne * px * B.ctot * es)) != TC_OK) return r;
        TC_TRY(s, cudaMemset(B.dec, 0, ne * px * B.ctot * es), "memset");
        if ((r = dalloc(s, &B.f2w, ne * px * B.c * es)) != TC_OK) return r;
        if ((r = dalloc_t(s, &B.flow, ne * px * 2 * sizeof(float))) != TC_OK) return r;
        if ((r = dalloc_t(s, &B.up, ne * px * 2 * sizeof(float))) != TC_OK) return r;
        TC_TRY(s, cudaMemset(B.up, 0, ne * px * 2 * sizeof(float)), "memset");
        const HostLayer *E = &net.layers[3 * L + 5 * (L - l)];
        // conv1 reads x0 (padded to x0p), conv2 x1, conv3 x2, conv4 [x2 | x3], head [x3 | x4].
        std::vector<int> p1(B.x0p, -1), g1(B.x0p, -1);
        for (int i = 0; i < B.c; ++i) { p1[i] = D + i; g1[i] = seg_pyr(s, l, 2); }            // self
        for (int i = 0; i < D; ++i) { p1[B.c + i] = i; g1[B.c + i] = seg_est(s, l, 0); }       // corr
        for (int i = 0; i < 2; ++i) { p1[B.c + D + i] = D + B.c + i; g1[B.c + D + i] = seg_est(s, l, 1); }  // up
        std::vector<int> p4(net.dec[1] + net.dec[2]), g4(net.dec[1] + net.dec[2]);
        for (int i = 0; i < net.dec[1]; ++i) { p4[i] = net.dec[2] + i; g4[i] = seg_est(s, l, 3); }   // x2
        for (int i = 0; i < net.dec[2]; ++i) { p4[net.dec[1] + i] = i; g4[net.dec[1] + i] = seg_est(s, l, 4); }  // x3
        std::vector<int> p5(net.dec[2] + net.dec[3]), g5(net.dec[2] + net.dec[3]);
        for (int i = 0; i < net.dec[2]; ++i) { p5[i] = net.dec[3] + i; g5[i] = seg_est(s, l, 4); }   // x3
        for (int i = 0; i < net.dec[3]; ++i) { p5[net.dec[2] + i] = i; g5[net.dec[2] + i] = seg_est(s, l, 5); }  // x4
        const std::vector<int> perms[4] = {p1, iota_perm(E[1].cin, E[1].cin), iota_perm(E[2].cin, E[2].cin), p4};
        const std::vector<int> segs[4] = {g1, std::vector<int>(E[1].cin, seg_est(s, l, 2)),
                                          std::vector<int>(E[2].cin, seg_est(s, l, 3)), g4};
        const int in_off[4] = {0, B.off_x1, B.off_x2, B.off_x2};
        const int cin[4] = {B.x0p, net.dec[0], net.dec[1], net.dec[1] + net.dec[2]};
        for (int j = 0; j < 4; ++j) {
            std::vector<float> wk = simt_weights(E[j], perms[j], s->prec);
            if ((r = upload(s, &B.wk[j], wk)) != TC_OK) return r;
            if ((r = upload(s, &B.bias[j], E[j].b)) != TC_OK) return r;
            T *dec = static_cast<T *>(B.dec);
            ConvArgs a{dec + in_off[j], B.ctot, 2, B.h, B.w, cin[j], 1, B.h, B.w, nullptr, nullptr, net.dec[j],
                       dec + B.off_x1, B.ctot, 1};
            add_layer(s, B.tcplan[j], a, s->n_est, wk, segs[j], false);
        }
        std::vector<float> wk5 = simt_weights(E[4], p5, s->prec);
        if ((r = upload(s, &B.head_w, wk5)) != TC_OK) return r;
        if ((r = upload(s, &B.head_b, E[4].b)) != TC_OK) return r;
        if (is16(s->prec)) {
            std::string why;
            // level L correlates the two pyramid slots; finer levels correlate with f2w
            const void *other = l == L ? B.pyr : B.f2w;
            if (tc_plan_corr(B.corrplan, B.pyr, s->npyr, B.c, other, l == L ? s->npyr : s->n_est, B.c, B.h, B.w, B.c,
                             s->R, s->dev_err, why, false, s->prec == TC_FP16))
                s->tc_corr_levels += 1;
        }
        {
            T *dec = static_cast<T *>(B.dec);
            ConvArgs a{dec + B.off_x3, B.ctot, 2, B.h, B.w, net.dec[2] + net.dec[3], 1, B.h, B.w, nullptr, nullptr, 2,
                       nullptr, 2, 0};
            add_layer(s, B.headplan, a, s->n_est, wk5, g5, true);
        }
    }
    if (!net.ref.empty() && (r = build_refine<T>(s)) != TC_OK) return r;
    const size_t npx = (size_t)s->H * s->W * s->lanes;
    for (int k = 0; k < 2; ++k) {
        if ((r = dalloc_t(s, &s->kA[k], npx * sizeof(float4))) != TC_OK) return r;
        if ((r = dalloc_t(s, &s->kB[k], npx * sizeof(float4))) != TC_OK) return r;
        if ((r = dalloc_t(s, &s->kC[k], npx * sizeof(float))) != TC_OK) return r;
    }
    if (s->fs == 2 && (r = dalloc_t(s, &s->xs, (size_t)3 * s->Hn * s->Wn * sizeof(float))) != TC_OK) return r;
    return TC_OK;
}

// A stream (lanes = 0) or a batch of `lanes` lanes (tc_create_batch).
static tc_status create_impl(const tc_stream_desc *desc, void *cuda_stream, tc_stream **out, int lanes) {
    if (out) *out = nullptr;
    if (!desc || !out) return fail(nullptr, TC_ERR_INVALID_ARG, "tc_create_stream: NULL argument");
    if (desc->precision != TC_FP32 && desc->precision != TC_BF16 && desc->precision != TC_FP8_E4M3 &&
        desc->precision != TC_FP16)
        return fail(nullptr, TC_ERR_INVALID_ARG,
                    "tc_create_stream: precision must be TC_FP32, TC_BF16, TC_FP16 or TC_FP8_E4M3");
    std::unique_ptr<tc_stream> s(new (std::nothrow) tc_stream());
    if (!s) return fail(nullptr, TC_ERR_OOM, "tc_create_stream: host allocation failed");
    std::vector<uint8_t> blob;
    if (desc->weights_path) {
        FILE *f = fopen(desc->weights_path, "rb");
        if (!f) return fail(nullptr, TC_ERR_IO, std::string("cannot open weights file ") + desc->weights_path);
        fseek(f, 0, SEEK_END);
        long n = ftell(f);
        fseek(f, 0, SEEK_SET);
        blob.resize(n > 0 ? (size_t)n : 0);
        size_t got = n > 0 ? fread(blob.data(), 1, (size_t)n, f) : 0;
        fclose(f);
        if (got != blob.size()) return fail(nullptr, TC_ERR_IO, "short read of the weights file");
    } else if (desc->weights_blob && desc->weights_bytes) {
        blob.assign((const uint8_t *)desc->weights_blob, (const uint8_t *)desc->weights_blob + desc->weights_bytes);
    } else {
        return fail(nullptr, TC_ERR_INVALID_ARG, "tc_create_stream: no weights given");
    }
    std::string err;
    if (!parse_weights(blob.data(), blob.size(), s->net, err)) return fail(nullptr, TC_ERR_IO, err);
    if (lanes) {
        if (desc->precision == TC_FP8_E4M3)
            return fail(nullptr, TC_ERR_UNSUPPORTED, "tc_create_batch: a batch runs in TC_FP32, TC_BF16 or TC_FP16");
        if (desc->flow_downscale == 2 || !s->net.ref.empty())
            return fail(nullptr, TC_ERR_UNSUPPORTED,
                        "tc_create_batch: a batch runs the causal path without the fast preset or the refinement");
        s->batch = true;
        s->lanes = lanes;
        s->npyr = 2 * lanes;
        s->n_est = 2 * lanes;
        s->lane_t.assign(lanes, 0);
        s->lane_cur.assign(lanes, 0);
        s->lane_params.resize(lanes);
        for (auto &lp : s->lane_params) tc_default_consistency(&lp);
    }
    s->L = s->net.levels;
    s->R = s->net.radius;
    s->D = (2 * s->R + 1) * (2 * s->R + 1);
    const int m = 1 << s->L;
    if (desc->flow_downscale < 0 || desc->flow_downscale > 2)
        return fail(nullptr, TC_ERR_INVALID_ARG, "tc_create_stream: flow_downscale must be 0, 1 or 2");
    const int fs = desc->flow_downscale == 2 ? 2 : 1;
    if (desc->width > 16384 || desc->height > 16384 || (desc->width + fs - 1) / fs < m ||
        (desc->height + fs - 1) / fs < m)
        return fail(nullptr, TC_ERR_INVALID_ARG,
                    "tc_create_stream: width and height must be <= 16384 and, divided by flow_downscale, >= 2^levels");
    s->W = desc->width;
    s->H = desc->height;
    s->fs = fs;
    s->Wn = (s->W + fs - 1) / fs;
    s->Hn = (s->H + fs - 1) / fs;
    s->Wp = round_up(s->Wn, m);
    s->Hp = round_up(s->Hn, m);
    s->prec = desc->precision;
    s->st = static_cast<cudaStream_t>(cuda_stream);
    tc_default_consistency(&s->params);
    tc_status r = s->prec == TC_FP32   ? build_stream<float>(s.get())
                  : s->prec == TC_BF16 ? build_stream<__nv_bfloat16>(s.get())
                  : s->prec == TC_FP16 ? build_stream<__half>(s.get())
                                       : build_stream<__nv_fp8_e4m3>(s.get());
    if (r != TC_OK) {
        std::string msg = s->err;
        free_all(s.get());
        return fail(nullptr, r, msg);
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_all(s.get());
        return fail(nullptr, TC_ERR_CUDA, std::string("tc_create_stream: ") + cudaGetErrorString(e));
    }
    *out = s.release();
    return TC_OK;
}

extern "C" tc_status tc_create_stream(const tc_stream_desc *desc, void *cuda_stream, tc_stream **out) {
    return create_impl(desc, cuda_stream, out, 0);
}

extern "C" tc_status tc_create_batch(const tc_stream_desc *desc, int lanes, void *cuda_stream, tc_stream **out) {
    if (lanes < 1 || lanes > 64) {
        if (out) *out = nullptr;
        return fail(nullptr, TC_ERR_INVALID_ARG, "tc_create_batch: lanes must lie in [1, 64]");
    }
    return create_impl(desc, cuda_stream, out, lanes);
}

// Folds the pending profiling events of s into its per-category totals.
static tc_status prof_flush(tc_stream *s) {
    const size_t n = s->ev_cat.size();
    if (n == 0) return TC_OK;
    TC_TRY(s, cudaEventSynchronize(s->ev_pool[2 * n - 1]), "profiling event synchronize");
    for (size_t k = 0; k < n; ++k) {
        float ms = 0.f;
        TC_TRY(s, cudaEventElapsedTime(&ms, s->ev_pool[2 * k], s->ev_pool[2 * k + 1]), "profiling elapsed time");
        s->prof_ms[s->ev_cat[k]] += ms;
        s->prof_n[s->ev_cat[k]] += 1;
    }
    s->ev_cat.clear();
    return TC_OK;
}

static tc_status prof_begin(tc_stream *s, int cat) {
    const size_t k = s->ev_cat.size();
    while (s->ev_pool.size() < 2 * (k + 1)) {
        cudaEvent_t e;
        TC_TRY(s, cudaEventCreate(&e), "cudaEventCreate");
        s->ev_pool.push_back(e);
    }
    s->ev_cat.push_back(cat);
    TC_TRY(s, cudaEventRecord(s->ev_pool[2 * k], s->st), "cudaEventRecord");
    return TC_OK;
}

static tc_status prof_end(tc_stream *s) {
    TC_TRY(s, cudaEventRecord(s->ev_pool[2 * (s->ev_cat.size() - 1) + 1], s->st), "cudaEventRecord");
    return TC_OK;
}

#define TC_LAUNCH_CAT(s, cat, expr)                                               \
    do {                                                                          \
        if ((s)->prof) {                                                          \
            tc_status _r = prof_begin(s, cat);                                    \
            if (_r != TC_OK) return _r;                                           \
        }                                                                         \
        cudaError_t _e = (expr);                                                  \
        ++(s)->launches;                                                          \
        if (_e != cudaSuccess) return cuda_fail(s, _e, "kernel launch");          \
        if ((s)->prof) {                                                          \
            tc_status _r = prof_end(s);                                           \
            if (_r != TC_OK) return _r;                                           \
        }                                                                         \
    } while (0)
#define TC_LAUNCH(s, expr) TC_LAUNCH_CAT(s, TC_PROF_OTHER, expr)

template <typename T>
static tc_status conv_layer(tc_stream *s, const ConvArgs &a, const TcConvPlan *plan, int cat) {
    if (plan && plan->enabled) {
        ConvArgs b = a;
        b.overlap = s->pipelined ? 1 : 0;  // pipelined mode: the launches overlap the other streams'
        TC_LAUNCH_CAT(s, cat, launch_conv_tc(*plan, b, s->st));
    } else if constexpr (sizeof(T) == 1) {
        return fail(s, TC_ERR_UNSUPPORTED, "e4m3 layer without a tensor-core plan");
    } else {
        TC_LAUNCH_CAT(s, cat, launch_conv_simt<T>(a, s->st));
    }
    return TC_OK;
}

// The first conv's arguments for input image img (the 16-output form carries its weights).
static ConvFirstArgs first_args(const tc_stream *s, const float *img) {
    const LevelBufs &B = s->lv[0];
    ConvFirstArgs f{img, s->Hn, s->Wn, s->Hp, s->Wp, s->pyr_w[0], s->pyr_b[0], B.c, B.tmpA, B.q_pyr[0], {}, {}};
    if (B.c == 16 && s->first_w.size() == 27 * 16 && s->first_b.size() == 16) {
        memcpy(f.w16, s->first_w.data(), sizeof f.w16);
        memcpy(f.b16, s->first_b.data(), sizeof f.b16);
    }
    return f;
}

// The pyramid slot of frame t (see NPYR).
static inline int pyr_slot(const tc_stream *s, long long t) { return (int)(t % (s->pipelined ? NPYR : 2)); }
// The estimator buffer set of frame t.
static inline int est_set(const tc_stream *s, long long t) { return s->pipelined ? (int)(t % NSET) : 0; }

template <typename T>
static tc_status run_pyramid(tc_stream *s, const float *img, int slot) {
    tc_status r;
    for (int l = 1; l <= s->L; ++l) {
        LevelBufs &B = s->lv[l - 1];
        const size_t px = (size_t)B.h * B.w;
        T *dst = static_cast<T *>(B.pyr) + (size_t)slot * px * B.c;
        if (l == 1) {
            if (s->fs == 2) {
                TC_LAUNCH_CAT(s, TC_PROF_PYRAMID_CONV, launch_downscale2(img, 3, s->H, s->W, s->xs, s->st));
                img = s->xs;
            }
            const ConvFirstArgs f = first_args(s, img);
            TC_LAUNCH_CAT(s, TC_PROF_PYRAMID_CONV, launch_conv_first<T>(f, s->st));
        } else {
            LevelBufs &P = s->lv[l - 2];
            const T *src = static_cast<const T *>(P.pyr) + (size_t)slot * P.h * P.w * P.c;
            ConvArgs a{src, P.c, 1, P.h, P.w, P.c, 2, B.h, B.w, s->pyr_w[3 * (l - 1)], s->pyr_b[3 * (l - 1)],
                       B.c, B.tmpA, B.c, 1, B.q_pyr[0]};
            if ((r = conv_layer<T>(s, a, &s->pyr_plan[l - 1][0], TC_PROF_PYRAMID_CONV)) != TC_OK) return r;
        }
        ConvArgs b{B.tmpA, B.c, 1, B.h, B.w, B.c, 1, B.h, B.w, s->pyr_w[3 * (l - 1) + 1], s->pyr_b[3 * (l - 1) + 1],
                   B.c, B.tmpB, B.c, 1, B.q_pyr[1]};
        b.rev = 1;  // reads the rows conv a wrote last first
        if ((r = conv_layer<T>(s, b, &s->pyr_plan[l - 1][1], TC_PROF_PYRAMID_CONV)) != TC_OK) return r;
        ConvArgs c{B.tmpB, B.c, 1, B.h, B.w, B.c, 1, B.h, B.w, s->pyr_w[3 * (l - 1) + 2], s->pyr_b[3 * (l - 1) + 2],
                   B.c, dst, B.c, 1, B.q_pyr[2]};
        if ((r = conv_layer<T>(s, c, &s->pyr_plan[l - 1][2], TC_PROF_PYRAMID_CONV)) != TC_OK) return r;
    }
    return TC_OK;
}

// The refinement of the level-2 flows of both directions (Sec. 3.2 "-sepref"): each layer a
// depthwise dilated 3x3 conv (CUDA cores) and a pointwise conv (tensor cores for BF16); the
// first reads [x3 | x4 | flow] (the buffer order of cat(flow, x4, x3)), the last adds its
// two outputs to the flow in place.
template <typename T>
static tc_status run_refine(tc_stream *s, int set) {
    if constexpr (sizeof(T) == 1) {
        return fail(s, TC_ERR_UNSUPPORTED, "the refinement network runs in TC_FP32, TC_BF16 or TC_FP16 streams");
    } else {
    LevelBufs &B = s->lv[1];
    T *dec = dec_of<T>(B, set);
    float *flow = flow_of(B, set);
    const size_t px = (size_t)B.h * B.w;
    T *refD = static_cast<T *>(s->refD) + (size_t)set * 2 * px * s->refD_cs;
    T *refP = static_cast<T *>(s->refP) + (size_t)set * 2 * px * s->refP_cs;
    const int nl = (int)s->ref.size();
    for (int k = 0; k < nl; ++k) {
        tc_stream::RefLayer &R = s->ref[k];
        DwArgs d{};
        d.in = k == 0 ? static_cast<const void *>(dec + B.off_x3) : static_cast<const void *>(refP);
        d.in_cs = k == 0 ? B.ctot : s->refP_cs;
        d.nin = R.nin;
        d.flow = k == 0 ? flow : nullptr;
        d.n = 2; d.h = B.h; d.w = B.w;
        d.dw = R.dw; d.db = R.db; d.dil = R.dil;
        d.out = refD; d.out_cs = s->refD_cs; d.cp = R.cin_p;
        TC_LAUNCH_CAT(s, TC_PROF_REFINE, launch_depthwise<T>(d, s->st));
        const bool last = k == nl - 1;
        if (R.plan.enabled) {
            ConvArgs a{refD, s->refD_cs, 2, B.h, B.w, R.cin_p, 1, B.h, B.w, nullptr, R.pb, last ? 2 : R.cout,
                       last ? nullptr : refP, last ? 16 : s->refP_cs, R.leaky};
            if (last)
                TC_LAUNCH_CAT(s, TC_PROF_REFINE, launch_conv_tc_head(R.plan, a, flow, flow, s->st));
            else
                TC_LAUNCH_CAT(s, TC_PROF_REFINE, launch_conv_tc(R.plan, a, s->st));
        } else {
            PwArgs pa{};
            pa.in = refD; pa.in_cs = s->refD_cs; pa.cin = R.cin_p;
            pa.w = R.pw; pa.b = R.pb; pa.cout = R.cout; pa.leaky = R.leaky;
            pa.out = last ? nullptr : refP; pa.out_cs = s->refP_cs;
            pa.flow = last ? flow : nullptr;
            pa.npx = 2 * px;
            TC_LAUNCH_CAT(s, TC_PROF_REFINE, launch_pointwise<T>(pa, s->st));
        }
    }
    return TC_OK;
    }
}

// Both directions at once (batch entry 0: self = frame t, other = t-1, giving F_{t->t-1};
// entry 1: self = t-1, other = t, giving F_{t-1->t}).
template <typename T>
static tc_status run_estimators(tc_stream *s, int pcur, int pprev, int set) {
    tc_status r;
    const HostNet &net = s->net;
    for (int l = s->L; l >= 2; --l) {
        LevelBufs &B = s->lv[l - 1];
        const size_t px = (size_t)B.h * B.w;
        const T *pyr = static_cast<const T *>(B.pyr);
        const T *self_p[2] = {pyr + (size_t)pcur * px * B.c, pyr + (size_t)pprev * px * B.c};
        const T *other_p[2] = {self_p[1], self_p[0]};
        T *dec = dec_of<T>(B, set);
        T *f2w = f2w_of<T>(B, set);
        float *flow = flow_of(B, set), *up = up_of(B, set);
        const void *fo[2] = {other_p[0], other_p[1]};
        int fo_cs = B.c;
        if (l < s->L) {
            LevelBufs &C = s->lv[l];
            // x2 upsampling of the coarser flow fused into the feature warp; the up-flow also
            // lands in B.up (residual base) and in the estimator input.
            WarpArgs wa{{other_p[0], other_p[1]}, B.c, nullptr, 2, B.h, B.w, B.c, f2w, B.c,
                        flow_of(C, set), up, dec + B.c + s->D, B.ctot, B.q_est[1]};
            TC_LAUNCH_CAT(s, TC_PROF_WARP, launch_warp<T>(wa, s->st));
            fo[0] = f2w;
            fo[1] = f2w + px * B.c;
        }
        if (B.corrplan.enabled) {
            const int img_s[2] = {pcur, pprev};
            const int img_o[2] = {l < s->L ? 2 * set : pprev, l < s->L ? 2 * set + 1 : pcur};
            const void *fs[2] = {self_p[0], self_p[1]};
            TC_LAUNCH_CAT(s, TC_PROF_CORRELATION,
                          launch_corr_tc(B.corrplan, 2, img_s, img_o, dec + B.c, B.ctot, fs, dec, s->st, B.s_pyr[2],
                                         B.q_est[0], !s->pipelined));
        } else if constexpr (sizeof(T) == 1) {
            return fail(s, TC_ERR_UNSUPPORTED, "e4m3 correlation without a tensor-core plan");
        } else {
            CorrArgs ca{{self_p[0], self_p[1]}, {fo[0], fo[1]}, B.c, fo_cs, 2, B.h, B.w, B.c, s->R, dec + B.c, B.ctot,
                        dec};
            TC_LAUNCH_CAT(s, TC_PROF_CORRELATION, launch_corr<T>(ca, s->st));
        }
        ConvArgs c1{dec, B.ctot, 2, B.h, B.w, B.x0p, 1, B.h, B.w, B.wk[0], B.bias[0], net.dec[0], dec + B.off_x1, B.ctot, 1, B.q_est[2]};
        if ((r = conv_layer<T>(s, c1, &B.tcplan[0], TC_PROF_ESTIMATOR_CONV)) != TC_OK) return r;
        ConvArgs c2{dec + B.off_x1, B.ctot, 2, B.h, B.w, net.dec[0], 1, B.h, B.w, B.wk[1], B.bias[1], net.dec[1], dec + B.off_x2, B.ctot, 1, B.q_est[3]};
        c2.rev = 1;  // conv2 and conv4 walk their tiles backwards (see ConvArgs::rev)
        if ((r = conv_layer<T>(s, c2, &B.tcplan[1], TC_PROF_ESTIMATOR_CONV)) != TC_OK) return r;
        ConvArgs c3{dec + B.off_x2, B.ctot, 2, B.h, B.w, net.dec[1], 1, B.h, B.w, B.wk[2], B.bias[2], net.dec[2], dec + B.off_x3, B.ctot, 1, B.q_est[4]};
        if ((r = conv_layer<T>(s, c3, &B.tcplan[2], TC_PROF_ESTIMATOR_CONV)) != TC_OK) return r;
        ConvArgs c4{dec + B.off_x2, B.ctot, 2, B.h, B.w, net.dec[1] + net.dec[2], 1, B.h, B.w, B.wk[3], B.bias[3], net.dec[3], dec + B.off_x4, B.ctot, 1, B.q_est[5]};
        c4.rev = 1;
        if ((r = conv_layer<T>(s, c4, &B.tcplan[3], TC_PROF_ESTIMATOR_CONV)) != TC_OK) return r;
        if (B.headplan.enabled) {
            ConvArgs a5{dec + B.off_x3, B.ctot, 2, B.h, B.w, net.dec[2] + net.dec[3], 1, B.h, B.w, B.head_w, B.head_b,
                        2, nullptr, 2, 0};
            a5.overlap = s->pipelined ? 1 : 0;
            TC_LAUNCH_CAT(s, TC_PROF_HEAD, launch_conv_tc_head(B.headplan, a5, l < s->L ? up : nullptr, flow, s->st));
        } else if constexpr (sizeof(T) == 1) {
            return fail(s, TC_ERR_UNSUPPORTED, "e4m3 flow head without a tensor-core plan");
        } else {
            HeadArgs ha{dec + B.off_x3, B.ctot, net.dec[2] + net.dec[3], 2, B.h, B.w, B.head_w, B.head_b,
                        l < s->L ? up : nullptr, flow};
            TC_LAUNCH_CAT(s, TC_PROF_HEAD, launch_head<T>(ha, s->st));
        }
    }
    return s->ref.empty() ? TC_OK : run_refine<T>(s, set);
}

static tc_status check_stream(tc_stream *s, const char *fn) {
    if (!s) return fail(nullptr, TC_ERR_INVALID_ARG, std::string(fn) + ": NULL stream");
    if (s->poisoned) return fail(s, TC_ERR_STATE, std::string(fn) + ": stream is poisoned by an earlier CUDA error: " + s->err);
    return TC_OK;
}

// The entry points of a single stream refuse a batch.
static tc_status single_only(tc_stream *s, const char *fn) {
    tc_status r = check_stream(s, fn);
    if (r != TC_OK) return r;
    if (s->batch) return fail(s, TC_ERR_STATE, std::string(fn) + ": not available on a batch (tc_create_batch)");
    return TC_OK;
}

// Arguments of the consistency pass of a call at slot parity cur.  Causal streams blend the
// frame just given.  Streams with one frame of latency blend the frame before it (its I, P
// are in the state slot 1 - cur, those of the frame before that in slot cur), with the
// frame just given as the next frame unless flush (no next frame).
static ConsistArgs consist_args(tc_stream *s, const float *I, const float *P, float *O, float *wc, uint8_t *mask,
                                int cur, bool flush = false) {
    ConsistArgs ca{};
    const int prev = cur ^ 1;
    const bool lat = s->latency != 0;
    const long long n = s->t;  // frames given before this call
    // latency: frame t's I, P are the previous call's inputs, kept in slot prev
    ca.It = lat ? nullptr : I;
    ca.Pt = lat ? nullptr : P;
    ca.tA = lat ? s->kA[prev] : nullptr;
    ca.tB = lat ? s->kB[prev] : nullptr;
    ca.H = s->H; ca.W = s->W;
    ca.k1 = s->params.k1; ca.alpha = s->params.alpha; ca.lambda = s->params.lambda;
    ca.c1 = s->params.fb_c1; ca.c2 = s->params.fb_c2; ca.fb_check = s->params.fb_check;
    ca.k2 = s->params.k2;
    ca.O = O; ca.wc = wc; ca.mask = mask;
    // the state kept in slot cur: O_t, and I_t, P_t in the causal form (with latency the
    // caller's inputs are kept after this pass)
    ca.kA = s->kA[cur]; ca.kB = s->kB[cur]; ca.kC = s->kC[cur];
    ca.keep_io = lat ? 0 : 1;
    ca.keep_o = 1;
    const bool first = lat ? n == 1 : n == 0;
    if (!first && s->params.solver_iters > 0) {
        // A_t and w_c go to the solver's buffers, P_t as its planar input; the solver writes
        // O_t and the kept O
        ca.O = s->sv_A;
        ca.wc = s->sv_wc;
        ca.keep_o = 0;
        ca.Pcopy = s->sv_P;
    }
    if (first) {
        ca.first = 1;
        ca.Fb = ca.Ff = nullptr;
        ca.fh = ca.fw = 1; ca.scale = 1;
        return ca;
    }
    LevelBufs &B2 = s->lv[1];
    const size_t half = (size_t)B2.h * B2.w * 2;
    float *flow2 = flow_of(B2, est_set(s, s->t));
    ca.first = 0;
    // frame t - 1: its I, P in slot cur with latency (prev otherwise), its O in slot prev
    ca.pA = lat ? s->kA[cur] : s->kA[prev];
    ca.pB = lat ? s->kB[cur] : s->kB[prev];
    ca.oB = s->kB[prev];
    ca.pC = s->kC[prev];
    ca.fh = B2.h; ca.fw = B2.w; ca.scale = 4 * s->fs;
    if (!lat) {
        ca.Fb = flow2;
        ca.Ff = flow2 + half;
        return ca;
    }
    // the pair (t, t-1) from the previous call; the pair (t+1, t) just computed
    ca.Fb = s->Fprev;
    ca.Ff = s->Fprev + half;
    if (!flush) {
        ca.next = 1;
        ca.In = I;
        ca.Pn = P;
        ca.Fn = flow2 + half;  // F_{t->t+1}
        ca.Fnb = flow2;        // F_{t+1->t}
    }
    return ca;
}

// The solver after the consistency pass (A_t, w_c and the planar P_t in its buffers), then
// its result to the caller (O_t, w_c) and into the kept state of slot cur.
static tc_status solver_launches(tc_stream *s, float *O, float *wc, int cur) {
    PoissonArgs pa{s->sv_P, s->sv_A, s->sv_wc, 3, s->H, s->W, s->params.solver_iters, s->params.eta, s->params.kappa,
                   s->sv_b, s->sv_s[0], s->sv_s[1], s->sv_s[2], s->sv_s[3], s->sv_O, nullptr, s->sv_c0};
    TC_LAUNCH_CAT(s, TC_PROF_SOLVER, launch_poisson(pa, s->st));
    const size_t hw = (size_t)s->H * s->W;
    TC_LAUNCH_CAT(s, TC_PROF_SOLVER, launch_solver_out(s->sv_O, O, s->sv_wc, wc, hw, s->kB[cur], s->kC[cur], s->st));
    return TC_OK;
}

// The flow estimation of a frame (from the second frame on; with the refinement).
template <typename T>
static tc_status est_launches(tc_stream *s) {
    if (s->t == 0) return TC_OK;
    return run_estimators<T>(s, pyr_slot(s, s->t), pyr_slot(s, s->t - 1), est_set(s, s->t));
}

// The launches of a frame after its flow estimation: the blend, and the solver or the state
// copies.  upload: P_t arrives by the host entry point's upload (waited for before the first
// read of P_t).
template <typename T>
static tc_status blend_launches(tc_stream *s, const float *I, const float *P, float *O, float *wc, uint8_t *mask,
                                int cur, bool upload) {
    tc_status r;
    // everything from here on may read P_t
    if (upload) TC_TRY(s, cudaStreamWaitEvent(s->st, s->capturing ? s->ev_join : s->ev_p, 0), "cudaStreamWaitEvent");
    if (!s->latency) {
        const ConsistArgs ca = consist_args(s, I, P, O, wc, mask, cur);
        TC_LAUNCH_CAT(s, TC_PROF_CONSISTENCY, launch_consistency(ca, s->st));
        // Eq. 1 by Eq. 8 from A_t; P_t is read from the planar copy written above
        if (s->t > 0 && s->params.solver_iters > 0 && (r = solver_launches(s, O, wc, cur)) != TC_OK) return r;
        return TC_OK;
    }
    // one frame of latency: frame t = (frames given before) - 1 is blended now
    if (s->t > 0) {
        const ConsistArgs ca = consist_args(s, I, P, O, wc, mask, cur);
        TC_LAUNCH_CAT(s, TC_PROF_CONSISTENCY, launch_consistency(ca, s->st));
        if (s->t > 1 && s->params.solver_iters > 0 && (r = solver_launches(s, O, wc, cur)) != TC_OK) return r;
    }
    TC_LAUNCH_CAT(s, TC_PROF_CONSISTENCY,
                  launch_keep_inputs(I, P, (size_t)s->H * s->W, s->kA[cur], s->kB[cur], s->st));
    if (s->t > 0) {
        LevelBufs &B2 = s->lv[1];
        TC_TRY(s, cudaMemcpyAsync(s->Fprev, flow_of(B2, est_set(s, s->t)), (size_t)B2.h * B2.w * 4 * sizeof(float),
                                  cudaMemcpyDeviceToDevice, s->st),
               "flow copy");
    }
    return TC_OK;
}

// Every launch of one frame, in order.
template <typename T>
static tc_status frame_launches(tc_stream *s, const float *I, const float *P, float *O, float *wc, uint8_t *mask,
                                int cur) {
    tc_status r;
    const bool upload = s->p_pending;  // P_t is being uploaded on cst (host entry point)
    if (upload && s->capturing) {
        // the wait for P_t (an external event node) on a branch forked at the frame's start
        // and joined before the pass that reads P_t, off the chain of kernels
        TC_TRY(s, cudaEventRecord(s->ev_fork, s->st), "cudaEventRecord");
        TC_TRY(s, cudaStreamWaitEvent(s->cst, s->ev_fork, 0), "cudaStreamWaitEvent");
        TC_TRY(s, cudaStreamWaitEvent(s->cst, s->ev_p, cudaEventWaitExternal), "cudaStreamWaitEvent");
        TC_TRY(s, cudaEventRecord(s->ev_join, s->cst), "cudaEventRecord");
    }
    if ((r = run_pyramid<T>(s, I, pyr_slot(s, s->t))) != TC_OK) return r;
    if ((r = est_launches<T>(s)) != TC_OK) return r;
    return blend_launches<T>(s, I, P, O, wc, mask, cur, upload);
}

// Captures the launches made by `launches` on stream cs into graph G and finds the kernel
// nodes whose arguments change from frame to frame: the first pyramid conv (or the 2x2
// downscale) when need_first, the consistency pass and the copies when need_rest.
template <typename T, typename F>
static tc_status capture_into(tc_stream *s, cudaStream_t cs, tc_stream::FrameGraph &G, F &&launches, bool need_first,
                              bool need_rest) {
    // Capture on a library-owned stream (capture is not allowed on the legacy default stream
    // a caller may pass); the launch helpers use s->st, so point it there meanwhile.
    cudaStream_t caller = s->st;
    const int launches0 = s->launches;
    TC_TRY(s, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    s->st = cs;
    s->capturing = true;
    const tc_status r = launches();
    s->capturing = false;
    s->st = caller;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (r != TC_OK) {
        if (g) cudaGraphDestroy(g);
        return r;
    }
    if (e != cudaSuccess) return cuda_fail(s, e, "cudaStreamEndCapture");
    size_t n = 0;
    TC_TRY(s, cudaGraphGetNodes(g, nullptr, &n), "cudaGraphGetNodes");
    std::vector<cudaGraphNode_t> nodes(n);
    TC_TRY(s, cudaGraphGetNodes(g, nodes.data(), &n), "cudaGraphGetNodes");
    for (cudaGraphNode_t node : nodes) {
        cudaGraphNodeType ty;
        TC_TRY(s, cudaGraphNodeGetType(node, &ty), "cudaGraphNodeGetType");
        if (ty != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp{};
        TC_TRY(s, cudaGraphKernelNodeGetParams(node, &kp), "cudaGraphKernelNodeGetParams");
        if (s->fs == 1 && kp.func == conv_first_kernel_fn<T>()) { G.n_first = node; G.p_first = kp; }
        if (s->fs == 2 && kp.func == downscale2_kernel_fn()) { G.n_first = node; G.p_first = kp; }
        if (kp.func == consistency_kernel_fn(s->latency != 0)) { G.n_cons = node; G.p_cons = kp; }
        if (kp.func == solver_out_kernel_fn()) { G.n_copy = node; G.p_copy = kp; }
        if (kp.func == keep_inputs_kernel_fn()) { G.n_in = node; G.p_in = kp; }
    }
    if ((need_first && !G.n_first) ||
        (need_rest && (!G.n_cons || (s->params.solver_iters > 0 && !G.n_copy) || (s->latency && !G.n_in)))) {
        cudaGraphDestroy(g);
        return fail(s, TC_ERR_STATE, "frame graph: per-frame kernel nodes not found");
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
    if (ei != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(s, ei, "cudaGraphInstantiate");
    }
    G.g = g;
    G.exec = ex;
    G.launches = s->launches - launches0;
    return TC_OK;
}

// Points the graph's node that reads the caller's I_t (the first pyramid conv, or the 2x2
// downscale) at this frame's I_t.
template <typename T>
static tc_status update_first_node(tc_stream *s, tc_stream::FrameGraph &G, const float *I) {
    ConvFirstArgs f = first_args(s, I);
    int c3 = 3, hh = s->H, ww = s->W;
    float *xs = s->xs;
    void *fa[1] = {&f};
    void *da[5] = {&I, &c3, &hh, &ww, &xs};
    cudaKernelNodeParams pf = G.p_first;
    pf.kernelParams = s->fs == 2 ? da : fa;
    pf.extra = nullptr;
    TC_TRY(s, cudaGraphExecKernelNodeSetParams(G.exec, G.n_first, &pf), "graph node update");
    return TC_OK;
}

// Points the consistency pass and the copies of the graph at this frame's buffers and
// consistency controls.
static tc_status update_rest_nodes(tc_stream *s, tc_stream::FrameGraph &G, const float *I, const float *P, float *O,
                                   float *wc, uint8_t *mask, int cur) {
    ConsistArgs ca = consist_args(s, I, P, O, wc, mask, cur);
    void *cargs[1] = {&ca};
    cudaKernelNodeParams pc = G.p_cons;
    pc.kernelParams = cargs;
    pc.extra = nullptr;
    TC_TRY(s, cudaGraphExecKernelNodeSetParams(G.exec, G.n_cons, &pc), "graph node update");
    if (G.n_copy) {
        // the solver's result: retarget it to this frame's O_t, w_c and kept-state slot
        size_t hw = (size_t)s->H * s->W;
        const float *src = s->sv_O, *wsrc = s->sv_wc;
        float4 *kb = s->kB[cur];
        float *kc = s->kC[cur];
        void *ka[7] = {&src, &O, &wsrc, &wc, &hw, &kb, &kc};
        cudaKernelNodeParams pk = G.p_copy;
        pk.kernelParams = ka;
        pk.extra = nullptr;
        TC_TRY(s, cudaGraphExecKernelNodeSetParams(G.exec, G.n_copy, &pk), "graph node update");
    }
    if (G.n_in) {
        // the copy of this frame's inputs into the kept state (one frame of latency)
        size_t hw = (size_t)s->H * s->W;
        float4 *da = s->kA[cur], *db = s->kB[cur];
        void *ka[5] = {&I, &P, &hw, &da, &db};
        cudaKernelNodeParams pk = G.p_in;
        pk.kernelParams = ka;
        pk.extra = nullptr;
        TC_TRY(s, cudaGraphExecKernelNodeSetParams(G.exec, G.n_in, &pk), "graph node update");
    }
    return TC_OK;
}

static void release_graphs(tc_stream *s);

// Folds the amax of every activation segment of the frame just launched into amax_dev.
template <typename T>
static tc_status record_amax(tc_stream *s, int cur) {
    if constexpr (sizeof(T) == 1) {
        return fail(s, TC_ERR_INVALID_ARG, "amax recording needs a TC_FP32, TC_BF16 or TC_FP16 stream");
    } else {
        for (int l = 1; l <= s->L; ++l) {
            LevelBufs &B = s->lv[l - 1];
            const size_t px = (size_t)B.h * B.w;
            const T *pyr = static_cast<const T *>(B.pyr) + (size_t)pyr_slot(s, s->t) * px * B.c;
            TC_LAUNCH(s, launch_amax<T>(static_cast<const T *>(B.tmpA), px, B.c, B.c, s->amax_dev + seg_pyr(s, l, 0), s->st));
            TC_LAUNCH(s, launch_amax<T>(static_cast<const T *>(B.tmpB), px, B.c, B.c, s->amax_dev + seg_pyr(s, l, 1), s->st));
            TC_LAUNCH(s, launch_amax<T>(pyr, px, B.c, B.c, s->amax_dev + seg_pyr(s, l, 2), s->st));
            if (l < 2 || s->t == 0) continue;
            const T *dec = static_cast<const T *>(B.dec);
            const int off[6] = {B.c, B.c + s->D, B.off_x1, B.off_x2, B.off_x3, B.off_x4};
            const int nc[6] = {s->D, 2, s->net.dec[0], s->net.dec[1], s->net.dec[2], s->net.dec[3]};
            for (int k = 0; k < 6; ++k)
                TC_LAUNCH(s, launch_amax<T>(dec + off[k], 2 * px, B.ctot, nc[k], s->amax_dev + seg_est(s, l, k), s->st));
        }
        return TC_OK;
    }
}

template <typename T>
static tc_status process_pipelined(tc_stream *s, const float *I, const float *P, float *O, float *wc, uint8_t *mask);

template <typename T>
static tc_status process(tc_stream *s, const float *I, const float *P, float *O, float *wc, uint8_t *mask) {
    tc_status r;
    s->launches = 0;
    if (s->ev_cat.size() > 4096 && (r = prof_flush(s)) != TC_OK) return r;
    if (s->pipelined) return process_pipelined<T>(s, I, P, O, wc, mask);
    const int cur = (int)(s->t & 1);
    // The first two frames run eagerly (the first has no flow; the second sets every kernel
    // attribute); later frames replay the graph of their t % 2 (state parity and pyramid
    // slot), one set for host calls and one for device calls.  Profiling runs eagerly.
    const long long out = s->latency ? s->t - 1 : s->t;
    if (!s->graphs || s->prof || s->t < 2 || s->rec_amax) {
        if ((r = frame_launches<T>(s, I, P, O, wc, mask, cur)) != TC_OK) return r;
        if (s->rec_amax && (r = record_amax<T>(s, cur)) != TC_OK) return r;
        s->t += 1;
        s->last_out = out;
        return TC_OK;
    }
    tc_stream::FrameGraph &G = s->fg[s->p_pending ? 1 : 0][cur];
    if (!s->gst) {
        TC_TRY(s, cudaStreamCreateWithFlags(&s->gst, cudaStreamNonBlocking), "cudaStreamCreate");
        TC_TRY(s, cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming), "cudaEventCreate");
        TC_TRY(s, cudaEventCreateWithFlags(&s->ev_out, cudaEventDisableTiming), "cudaEventCreate");
    }
    if (!G.exec) {
        r = capture_into<T>(s, s->gst, G, [&] { return frame_launches<T>(s, I, P, O, wc, mask, cur); }, true, true);
        if (r != TC_OK) return r;
    } else {
        if ((r = update_first_node<T>(s, G, I)) != TC_OK) return r;
        if ((r = update_rest_nodes(s, G, I, P, O, wc, mask, cur)) != TC_OK) return r;
    }
    // caller's stream -> library stream -> caller's stream
    TC_TRY(s, cudaEventRecord(s->ev_in, s->st), "cudaEventRecord");
    TC_TRY(s, cudaStreamWaitEvent(s->gst, s->ev_in, 0), "cudaStreamWaitEvent");
    TC_TRY(s, cudaGraphLaunch(G.exec, s->gst), "cudaGraphLaunch");
    TC_TRY(s, cudaEventRecord(s->ev_out, s->gst), "cudaEventRecord");
    TC_TRY(s, cudaStreamWaitEvent(s->st, s->ev_out, 0), "cudaStreamWaitEvent");
    s->launches = G.launches;
    s->last_set = 0;
    s->t += 1;
    s->last_out = out;
    return TC_OK;
}

// Pipelined mode: frame t's pyramid runs on pst, its flow estimation on the stream of its
// buffer set (t % NSET: gst, estx[...]), its blend on bst, with no ordering on the caller's stream (the inputs
// are valid when the call is made; tc_join or tc_synchronize make the results visible).
//   * pyramid t writes slot t % NPYR, last read by the flow estimations of frames t - NPYR
//     and t - NPYR + 1, and waits for both;
//   * the flow estimation of frame t waits for pyramid t (pyramid t - 1 came before it on
//     pst) and for the blend that last read its buffer set's flows (frame t - NSET), and
//     follows frame t - NSET's estimation on its stream;
//   * the blend of frame t waits for its flow estimation and follows frame t - 1's blend.
// So the next frame's pyramid and NSET frames' flow estimations run at the same time.
// The library streams and event rings of the pipelined mode, created on first use.
static tc_status ensure_pipeline_streams(tc_stream *s) {
    constexpr int NEV = tc_stream::NEV;
    if (!s->gst) {
        TC_TRY(s, cudaStreamCreateWithFlags(&s->gst, cudaStreamNonBlocking), "cudaStreamCreate");
        TC_TRY(s, cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming), "cudaEventCreate");
        TC_TRY(s, cudaEventCreateWithFlags(&s->ev_out, cudaEventDisableTiming), "cudaEventCreate");
    }
    if (!s->pst) {
        TC_TRY(s, cudaStreamCreateWithFlags(&s->pst, cudaStreamNonBlocking), "cudaStreamCreate");
        for (cudaStream_t &q : s->estx) TC_TRY(s, cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking), "cudaStreamCreate");
        TC_TRY(s, cudaStreamCreateWithFlags(&s->bst, cudaStreamNonBlocking), "cudaStreamCreate");
        for (int j = 0; j < NEV; ++j) {
            TC_TRY(s, cudaEventCreateWithFlags(&s->ev_pyrs[j], cudaEventDisableTiming), "cudaEventCreate");
            TC_TRY(s, cudaEventCreateWithFlags(&s->ev_ests[j], cudaEventDisableTiming), "cudaEventCreate");
            TC_TRY(s, cudaEventCreateWithFlags(&s->ev_blends[j], cudaEventDisableTiming), "cudaEventCreate");
        }
    }
    return TC_OK;
}

template <typename T>
static tc_status process_pipelined(tc_stream *s, const float *I, const float *P, float *O, float *wc, uint8_t *mask) {
    constexpr int NEV = tc_stream::NEV;
    tc_status r;
    const long long t = s->t;
    const int cur = (int)(t & 1), ps = pyr_slot(s, t), set = est_set(s, t), e = (int)(t % NEV);
    const int nsets = NSET;
    const long long out = s->latency ? t - 1 : t;
    if ((r = ensure_pipeline_streams(s)) != TC_OK) return r;
    cudaStream_t es = set == 0 ? s->gst : s->estx[set - 1];
    // pyramid t: after everything before the sequence, or after the estimations that read
    // its slot last (frames t - NPYR and t - NPYR + 1)
    if (t == 0) {
        if (s->last_blend >= 0)
            TC_TRY(s, cudaStreamWaitEvent(s->pst, s->ev_blends[s->last_blend], 0), "cudaStreamWaitEvent");
    } else {
        for (int j = NPYR - 1; j <= NPYR; ++j)
            if (t - j >= 0) TC_TRY(s, cudaStreamWaitEvent(s->pst, s->ev_ests[(t - j) % NEV], 0), "cudaStreamWaitEvent");
    }
    // estimation t: after the blend that last read this buffer set's flows
    if (t >= nsets) TC_TRY(s, cudaStreamWaitEvent(es, s->ev_blends[(t - nsets) % NEV], 0), "cudaStreamWaitEvent");
    if (s->frame_timing) {
        if (s->ft_n == s->ft_start.size()) {
            cudaEvent_t a = nullptr, b = nullptr;
            TC_TRY(s, cudaEventCreate(&a), "cudaEventCreate");
            TC_TRY(s, cudaEventCreate(&b), "cudaEventCreate");
            s->ft_start.push_back(a);
            s->ft_done.push_back(b);
        }
        TC_TRY(s, cudaEventRecord(s->ft_start[s->ft_n], s->pst), "cudaEventRecord");
    }
    cudaStream_t caller = s->st;
    if (!s->graphs || s->prof || t < 2) {
        s->st = s->pst;
        r = run_pyramid<T>(s, I, ps);
        s->st = caller;
        if (r != TC_OK) return r;
        TC_TRY(s, cudaEventRecord(s->ev_pyrs[e], s->pst), "cudaEventRecord");
        TC_TRY(s, cudaStreamWaitEvent(es, s->ev_pyrs[e], 0), "cudaStreamWaitEvent");
        s->st = es;
        r = est_launches<T>(s);
        s->st = caller;
        if (r != TC_OK) return r;
        TC_TRY(s, cudaEventRecord(s->ev_ests[e], es), "cudaEventRecord");
        TC_TRY(s, cudaStreamWaitEvent(s->bst, s->ev_ests[e], 0), "cudaStreamWaitEvent");
        s->st = s->bst;
        r = blend_launches<T>(s, I, P, O, wc, mask, cur, false);
        s->st = caller;
        if (r != TC_OK) return r;
    } else {
        tc_stream::FrameGraph &Gp = s->pg_pyr[ps], &Ge = s->pg_est[t % NGRAPH], &Gb = s->pg_blend[t % NGRAPH];
        if (!Gp.exec) {
            r = capture_into<T>(s, s->pst, Gp, [&] { return run_pyramid<T>(s, I, ps); }, true, false);
            if (r != TC_OK) return r;
        } else if ((r = update_first_node<T>(s, Gp, I)) != TC_OK) {
            return r;
        }
        if (!Ge.exec) {
            r = capture_into<T>(s, es, Ge, [&] { return est_launches<T>(s); }, false, false);
            if (r != TC_OK) return r;
        }
        if (!Gb.exec) {
            r = capture_into<T>(s, s->bst, Gb, [&] { return blend_launches<T>(s, I, P, O, wc, mask, cur, false); },
                                false, true);
            if (r != TC_OK) return r;
        } else if ((r = update_rest_nodes(s, Gb, I, P, O, wc, mask, cur)) != TC_OK) {
            return r;
        }
        TC_TRY(s, cudaGraphLaunch(Gp.exec, s->pst), "cudaGraphLaunch");
        TC_TRY(s, cudaEventRecord(s->ev_pyrs[e], s->pst), "cudaEventRecord");
        TC_TRY(s, cudaStreamWaitEvent(es, s->ev_pyrs[e], 0), "cudaStreamWaitEvent");
        TC_TRY(s, cudaGraphLaunch(Ge.exec, es), "cudaGraphLaunch");
        TC_TRY(s, cudaEventRecord(s->ev_ests[e], es), "cudaEventRecord");
        TC_TRY(s, cudaStreamWaitEvent(s->bst, s->ev_ests[e], 0), "cudaStreamWaitEvent");
        TC_TRY(s, cudaGraphLaunch(Gb.exec, s->bst), "cudaGraphLaunch");
        s->launches = Gp.launches + Ge.launches + Gb.launches;
    }
    TC_TRY(s, cudaEventRecord(s->ev_blends[e], s->bst), "cudaEventRecord");
    if (s->frame_timing) TC_TRY(s, cudaEventRecord(s->ft_done[s->ft_n++], s->bst), "cudaEventRecord");
    s->last_blend = e;
    s->last_set = set;
    s->t += 1;
    s->last_out = out;
    return TC_OK;
}

// Pipelined mode: makes the caller's stream wait for every frame given so far (the last
// blend follows every earlier blend, each after its frame's estimation and pyramid).
static tc_status join_caller(tc_stream *s) {
    if (s->pipelined && s->last_blend >= 0)
        TC_TRY(s, cudaStreamWaitEvent(s->st, s->ev_blends[s->last_blend], 0), "cudaStreamWaitEvent");
    return TC_OK;
}

static void release_graph(tc_stream::FrameGraph &G) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.g) cudaGraphDestroy(G.g);
    G = tc_stream::FrameGraph{};
}

static void release_graphs(tc_stream *s) {
    for (auto &GG : s->fg)
        for (auto &G : GG) release_graph(G);
    for (auto &G : s->pg_pyr) release_graph(G);
    for (auto &G : s->pg_est) release_graph(G);
    for (auto &G : s->pg_blend) release_graph(G);
    for (auto &kv : s->range_graphs) release_graph(kv.second);
    s->range_graphs.clear();
    s->range_uses.clear();
}

static void release_graph_stream(tc_stream *s) {
    std::vector<cudaStream_t *> qs = {&s->pst, &s->bst};
    for (cudaStream_t &q : s->estx) qs.push_back(&q);
    for (cudaStream_t *q : qs)
        if (*q) {
            cudaStreamSynchronize(*q);
            cudaStreamDestroy(*q);
            *q = nullptr;
        }
    for (int j = 0; j < tc_stream::NEV; ++j) {
        if (s->ev_pyrs[j]) cudaEventDestroy(s->ev_pyrs[j]);
        if (s->ev_ests[j]) cudaEventDestroy(s->ev_ests[j]);
        if (s->ev_blends[j]) cudaEventDestroy(s->ev_blends[j]);
        s->ev_pyrs[j] = s->ev_ests[j] = s->ev_blends[j] = nullptr;
    }
    s->last_blend = -1;
    if (s->gst) {
        cudaStreamSynchronize(s->gst);
        cudaStreamDestroy(s->gst);
    }
    if (s->ev_in) cudaEventDestroy(s->ev_in);
    if (s->ev_out) cudaEventDestroy(s->ev_out);
    s->gst = nullptr;
    s->ev_in = s->ev_out = nullptr;
}

extern "C" int tc_activation_segments(const tc_stream *s) { return s ? n_segments(s) : 0; }

extern "C" tc_status tc_set_amax_recording(tc_stream *s, int enable) {
    tc_status r = single_only(s, "tc_set_amax_recording");
    if (r != TC_OK) return r;
    if (s->pipelined) return fail(s, TC_ERR_STATE, "tc_set_amax_recording: not available in pipelined mode");
    if (s->prec == TC_FP8_E4M3) return fail(s, TC_ERR_INVALID_ARG, "amax recording needs a TC_FP32, TC_BF16 or TC_FP16 stream");
    TC_TRY(s, cudaMemsetAsync(s->amax_dev, 0, sizeof(unsigned) * n_segments(s), s->st), "memset");
    s->rec_amax = enable != 0;
    return TC_OK;
}

extern "C" tc_status tc_get_amax(tc_stream *s, float *amax, int n) {
    tc_status r = check_stream(s, "tc_get_amax");
    if (r != TC_OK) return r;
    if (!amax || n < n_segments(s)) return fail(s, TC_ERR_INVALID_ARG, "tc_get_amax: need tc_activation_segments() floats");
    std::vector<unsigned> bits(n_segments(s));
    TC_TRY(s, cudaStreamSynchronize(s->st), "stream synchronize");
    TC_TRY(s, cudaMemcpy(bits.data(), s->amax_dev, bits.size() * sizeof(unsigned), cudaMemcpyDeviceToHost), "amax read");
    for (size_t i = 0; i < bits.size(); ++i) memcpy(&amax[i], &bits[i], sizeof(float));
    return TC_OK;
}

extern "C" tc_status tc_fp8_scales_from_amax(const float *amax, int n, float margin, float *scales) {
    if (!amax || !scales || n < 1) return fail(nullptr, TC_ERR_INVALID_ARG, "tc_fp8_scales_from_amax: NULL array or n < 1");
    if (!std::isfinite(margin) || margin <= 0.f)
        return fail(nullptr, TC_ERR_INVALID_ARG, "tc_fp8_scales_from_amax: margin must be positive and finite");
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(amax[i]) || amax[i] < 0.f)
            return fail(nullptr, TC_ERR_INVALID_ARG, "tc_fp8_scales_from_amax: amax must be finite and >= 0");
    // 448: the largest finite e4m3 value (4 exponent bits, bias 7, 3 mantissa bits)
    for (int i = 0; i < n; ++i) scales[i] = margin * amax[i] / 448.f;
    return TC_OK;
}

extern "C" tc_status tc_set_fp8_scales(tc_stream *s, const float *scales, int n) {
    tc_status r = single_only(s, "tc_set_fp8_scales");
    if (r != TC_OK) return r;
    if (s->prec != TC_FP8_E4M3) return fail(s, TC_ERR_INVALID_ARG, "tc_set_fp8_scales: not a TC_FP8_E4M3 stream");
    if (!scales || n != n_segments(s)) return fail(s, TC_ERR_INVALID_ARG, "tc_set_fp8_scales: need tc_activation_segments() scales");
    std::vector<float> sc(scales, scales + n);
    for (float &v : sc) {
        if (!std::isfinite(v) || v < 0.f) return fail(s, TC_ERR_INVALID_ARG, "tc_set_fp8_scales: scales must be finite and >= 0");
        if (v == 0.f) v = 1.f;  // a segment that is always zero
    }
    TC_TRY(s, cudaStreamSynchronize(s->st), "stream synchronize");
    release_graphs(s);
    for (auto &rec : s->recs) rec.plan->release();
    for (auto &B : s->lv) B.corrplan.enabled = false;
    s->tc_layers = 0;
    s->tc_corr_levels = 0;
    s->fp8_ready = false;
    for (int l = 1; l <= s->L; ++l) {
        LevelBufs &B = s->lv[l - 1];
        for (int j = 0; j < 3; ++j) {
            B.s_pyr[j] = sc[seg_pyr(s, l, j)];
            B.q_pyr[j] = 1.f / B.s_pyr[j];
        }
        if (l < 2) continue;
        for (int k = 0; k < 6; ++k) {
            B.s_est[k] = sc[seg_est(s, l, k)];
            B.q_est[k] = 1.f / B.s_est[k];
        }
    }
    // Fold each input channel's activation scale into the weights: the MMA then sees the
    // stored e4m3 codes, and each output channel needs only its weight scale.
    for (auto &rec : s->recs) {
        std::vector<float> wk = rec.wk;
        const int cin = rec.a.cin, cout = rec.head ? 2 : rec.a.cout;
        for (int tap = 0; tap < 9; ++tap)
            for (int c = 0; c < cin; ++c) {
                const float f = rec.in_seg[c] >= 0 ? sc[rec.in_seg[c]] : 0.f;
                for (int o = 0; o < cout; ++o) wk[((size_t)tap * cin + c) * cout + o] *= f;
            }
        std::string why;
        const bool ok = rec.head ? tc_plan_head(*rec.plan, rec.a, rec.n_in, wk, s->dev_err, why, true)
                                 : tc_plan_conv(*rec.plan, rec.a, rec.n_in, wk, s->dev_err, why, true);
        if (!ok) return fail(s, TC_ERR_UNSUPPORTED, "e4m3 layer not eligible for the tensor cores: " + why);
        s->tc_layers += 1;
    }
    for (int l = 2; l <= s->L; ++l) {
        LevelBufs &B = s->lv[l - 1];
        std::string why;
        const void *other = l == s->L ? B.pyr : B.f2w;
        if (!tc_plan_corr(B.corrplan, B.pyr, s->npyr, B.c, other, l == s->L ? s->npyr : s->n_est, B.c, B.h, B.w, B.c,
                          s->R, s->dev_err, why, true))
            return fail(s, TC_ERR_UNSUPPORTED, "e4m3 correlation not eligible for the tensor cores: " + why);
        s->tc_corr_levels += 1;
    }
    s->fp8_ready = true;
    return TC_OK;
}

extern "C" tc_status tc_set_graphs(tc_stream *s, int enable) {
    tc_status r = check_stream(s, "tc_set_graphs");
    if (r != TC_OK) return r;
    TC_TRY(s, cudaStreamSynchronize(s->st), "stream synchronize");
    release_graphs(s);
    s->graphs = enable != 0;
    return TC_OK;
}

// ------------------------------------------------------------------------------- batch

// The first pyramid conv of one lane: its frame I -> the lane's image of the level-1
// scratch buffer.
template <typename T>
static tc_status lane_first(tc_stream *s, int lane, const float *I) {
    const LevelBufs &B = s->lv[0];
    ConvFirstArgs f = first_args(s, I);
    f.out = static_cast<T *>(B.tmpA) + (size_t)lane * B.h * B.w * B.c;
    TC_LAUNCH_CAT(s, TC_PROF_PYRAMID_CONV, launch_conv_first<T>(f, s->st));
    return TC_OK;
}

// The shared launches of lanes [lo, lo + n): the feature pyramids of their current frames
// (after each lane's first conv) into pyramid slot 0, then both flow directions of every
// lane, entry 2q + d of the estimator buffers being direction d of lane lo + q (d = 0: the
// current frame against the previous one, F_{t->t-1}; d = 1: F_{t-1->t}).  Every launch
// covers all 2n (pyramid: n) images; the warp and the correlation find each entry's frames
// in the two pyramid slots (lane pairs).
template <typename T>
static tc_status lanes_network(tc_stream *s, int lo, int n) {
    tc_status r;
    const HostNet &net = s->net;
    const int NL = s->lanes;
    for (int l = 1; l <= s->L; ++l) {
        LevelBufs &B = s->lv[l - 1];
        const size_t img = (size_t)B.h * B.w * B.c;
        T *tA = static_cast<T *>(B.tmpA) + lo * img, *tB = static_cast<T *>(B.tmpB) + lo * img;
        T *cur = static_cast<T *>(B.pyr) + lo * img;
        if (l > 1) {
            LevelBufs &P = s->lv[l - 2];
            const T *src = static_cast<const T *>(P.pyr) + (size_t)lo * P.h * P.w * P.c;
            ConvArgs a{src, P.c, n, P.h, P.w, P.c, 2, B.h, B.w, s->pyr_w[3 * (l - 1)], s->pyr_b[3 * (l - 1)],
                       B.c, tA, B.c, 1, 1.f};
            if ((r = conv_layer<T>(s, a, &s->pyr_plan[l - 1][0], TC_PROF_PYRAMID_CONV)) != TC_OK) return r;
        }
        ConvArgs b{tA, B.c, n, B.h, B.w, B.c, 1, B.h, B.w, s->pyr_w[3 * (l - 1) + 1], s->pyr_b[3 * (l - 1) + 1],
                   B.c, tB, B.c, 1, 1.f};
        b.rev = 1;
        if ((r = conv_layer<T>(s, b, &s->pyr_plan[l - 1][1], TC_PROF_PYRAMID_CONV)) != TC_OK) return r;
        ConvArgs c{tB, B.c, n, B.h, B.w, B.c, 1, B.h, B.w, s->pyr_w[3 * (l - 1) + 2], s->pyr_b[3 * (l - 1) + 2],
                   B.c, cur, B.c, 1, 1.f};
        if ((r = conv_layer<T>(s, c, &s->pyr_plan[l - 1][2], TC_PROF_PYRAMID_CONV)) != TC_OK) return r;
    }
    const int ne = 2 * n;
    for (int l = s->L; l >= 2; --l) {
        LevelBufs &B = s->lv[l - 1];
        const size_t px = (size_t)B.h * B.w, img = px * B.c;
        const T *pyr0 = static_cast<const T *>(B.pyr) + lo * img;  // slot 0, lane lo (slot 1: + NL images)
        T *dec = static_cast<T *>(B.dec) + (size_t)2 * lo * px * B.ctot;
        T *f2w = static_cast<T *>(B.f2w) + (size_t)2 * lo * img;
        float *flow = B.flow + (size_t)2 * lo * px * 2, *up = B.up + (size_t)2 * lo * px * 2;
        if (l < s->L) {
            const LevelBufs &C = s->lv[l];
            const float *cflow = C.flow + (size_t)2 * lo * C.h * C.w * 2;
            WarpArgs wa{{pyr0, pyr0}, B.c, nullptr, ne, B.h, B.w, B.c, f2w, B.c, cflow, up, dec + B.c + s->D, B.ctot,
                        1.f, img, NL};
            TC_LAUNCH_CAT(s, TC_PROF_WARP, launch_warp<T>(wa, s->st));
        }
        if (B.corrplan.enabled) {
            // self: image d NL + lo + q of the pyramid; other: the pyramid's other slot at
            // the coarsest level, else entry 2 (lo + q) + d of the warped features
            const bool top = l == s->L;
            TC_LAUNCH_CAT(s, TC_PROF_CORRELATION,
                          launch_corr_tc_pairs(B.corrplan, n, NL, lo, top ? lo + NL : 2 * lo, top ? 1 : 2,
                                               top ? -NL : 1, dec + B.c, B.ctot, pyr0, img * sizeof(T), dec, s->st));
        } else {
            const T *fo0 = l == s->L ? pyr0 : f2w;
            CorrArgs ca{{pyr0, pyr0}, {fo0, fo0}, B.c, B.c, ne, B.h, B.w, B.c, s->R, dec + B.c, B.ctot, dec, img, img,
                        NL, l == s->L ? 1 : 0};
            TC_LAUNCH_CAT(s, TC_PROF_CORRELATION, launch_corr<T>(ca, s->st));
        }
        ConvArgs c1{dec, B.ctot, ne, B.h, B.w, B.x0p, 1, B.h, B.w, B.wk[0], B.bias[0], net.dec[0], dec + B.off_x1, B.ctot, 1, 1.f};
        if ((r = conv_layer<T>(s, c1, &B.tcplan[0], TC_PROF_ESTIMATOR_CONV)) != TC_OK) return r;
        ConvArgs c2{dec + B.off_x1, B.ctot, ne, B.h, B.w, net.dec[0], 1, B.h, B.w, B.wk[1], B.bias[1], net.dec[1], dec + B.off_x2, B.ctot, 1, 1.f};
        c2.rev = 1;
        if ((r = conv_layer<T>(s, c2, &B.tcplan[1], TC_PROF_ESTIMATOR_CONV)) != TC_OK) return r;
        ConvArgs c3{dec + B.off_x2, B.ctot, ne, B.h, B.w, net.dec[1], 1, B.h, B.w, B.wk[2], B.bias[2], net.dec[2], dec + B.off_x3, B.ctot, 1, 1.f};
        if ((r = conv_layer<T>(s, c3, &B.tcplan[2], TC_PROF_ESTIMATOR_CONV)) != TC_OK) return r;
        ConvArgs c4{dec + B.off_x2, B.ctot, ne, B.h, B.w, net.dec[1] + net.dec[2], 1, B.h, B.w, B.wk[3], B.bias[3], net.dec[3], dec + B.off_x4, B.ctot, 1, 1.f};
        c4.rev = 1;
        if ((r = conv_layer<T>(s, c4, &B.tcplan[3], TC_PROF_ESTIMATOR_CONV)) != TC_OK) return r;
        if (B.headplan.enabled) {
            ConvArgs a5{dec + B.off_x3, B.ctot, ne, B.h, B.w, net.dec[2] + net.dec[3], 1, B.h, B.w, B.head_w, B.head_b,
                        2, nullptr, 2, 0};
            a5.overlap = s->pipelined ? 1 : 0;
            TC_LAUNCH_CAT(s, TC_PROF_HEAD, launch_conv_tc_head(B.headplan, a5, l < s->L ? up : nullptr, flow, s->st));
        } else {
            HeadArgs ha{dec + B.off_x3, B.ctot, net.dec[2] + net.dec[3], ne, B.h, B.w, B.head_w, B.head_b,
                        l < s->L ? up : nullptr, flow};
            TC_LAUNCH_CAT(s, TC_PROF_HEAD, launch_head<T>(ha, s->st));
        }
    }
    return TC_OK;
}

// The causal consistency pass of one lane (its own controls and state slots; a lane's
// first frame returns P), then its current pyramid becomes its previous one.
template <typename T>
static tc_status lane_blend(tc_stream *s, int lane, const float *I, const float *P, float *O, float *wc,
                            uint8_t *mask) {
    const tc_consistency &pr = s->lane_params[lane];
    const int cur = s->lane_cur[lane], prev = cur ^ 1;
    const size_t off = (size_t)s->H * s->W * lane;  // the lane's pixels in the kept state
    ConsistArgs ca{};
    ca.It = I; ca.Pt = P;
    ca.H = s->H; ca.W = s->W;
    ca.k1 = pr.k1; ca.alpha = pr.alpha; ca.lambda = pr.lambda;
    ca.c1 = pr.fb_c1; ca.c2 = pr.fb_c2; ca.fb_check = pr.fb_check; ca.k2 = pr.k2;
    ca.O = O; ca.wc = wc; ca.mask = mask;
    ca.kA = s->kA[cur] + off; ca.kB = s->kB[cur] + off; ca.kC = s->kC[cur] + off;
    ca.keep_io = ca.keep_o = 1;
    if (s->lane_t[lane] == 0) {
        ca.first = 1;
        ca.fh = ca.fw = 1; ca.scale = 1;
    } else {
        const LevelBufs &B2 = s->lv[1];
        const size_t fimg = (size_t)B2.h * B2.w * 2;
        ca.pA = s->kA[prev] + off; ca.pB = ca.oB = s->kB[prev] + off; ca.pC = s->kC[prev] + off;
        ca.Fb = B2.flow + (size_t)2 * lane * fimg;
        ca.Ff = ca.Fb + fimg;
        ca.fh = B2.h; ca.fw = B2.w; ca.scale = 4;
    }
    TC_LAUNCH_CAT(s, TC_PROF_CONSISTENCY, launch_consistency(ca, s->st));
    for (int l = 1; l <= s->L; ++l) {
        const LevelBufs &B = s->lv[l - 1];
        const size_t bytes = (size_t)B.h * B.w * B.c * sizeof(T);
        char *base = static_cast<char *>(B.pyr);
        TC_TRY(s, cudaMemcpyAsync(base + (size_t)(s->lanes + lane) * bytes, base + (size_t)lane * bytes, bytes,
                                  cudaMemcpyDeviceToDevice, s->st),
               "pyramid copy");
    }
    return TC_OK;
}

template <typename T>
static tc_status process_lanes(tc_stream *s, int n, const int *lanes, const float *const *I, const float *const *P,
                               float *const *O, float *const *wc, uint8_t *const *mask) {
    tc_status r;
    s->launches = 0;
    int lo = lanes[0], hi = lanes[0];
    for (int k = 1; k < n; ++k) {
        lo = std::min(lo, lanes[k]);
        hi = std::max(hi, lanes[k]);
    }
    const int nr = hi - lo + 1;
    for (int k = 0; k < n; ++k)
        if ((r = lane_first<T>(s, lanes[k], I[k])) != TC_OK) return r;
    // The shared launches: eager on a range's first use (which also sets every kernel's
    // attributes), then captured once and replayed as one graph.
    const int key = lo * 4096 + nr;
    int &uses = s->range_uses[key];
    if (s->graphs && !s->prof && uses >= 1) {
        tc_stream::FrameGraph &G = s->range_graphs[key];
        if (!G.exec) {
            if (!s->gst) TC_TRY(s, cudaStreamCreateWithFlags(&s->gst, cudaStreamNonBlocking), "cudaStreamCreate");
            const int before = s->launches;
            r = capture_into<T>(s, s->gst, G, [&] { return lanes_network<T>(s, lo, nr); }, false, false);
            if (r != TC_OK) return r;
            s->launches = before;
        }
        TC_TRY(s, cudaGraphLaunch(G.exec, s->st), "cudaGraphLaunch");
        s->launches += G.launches;
    } else if ((r = lanes_network<T>(s, lo, nr)) != TC_OK) {
        return r;
    }
    uses += 1;
    for (int k = 0; k < n; ++k)
        if ((r = lane_blend<T>(s, lanes[k], I[k], P[k], O[k], wc ? wc[k] : nullptr, mask ? mask[k] : nullptr)) != TC_OK)
            return r;
    for (int k = 0; k < n; ++k) {
        s->lane_t[lanes[k]] += 1;
        s->lane_cur[lanes[k]] ^= 1;
    }
    return TC_OK;
}

extern "C" tc_status tc_process_lanes(tc_stream *s, int n, const int *lanes, const float *const *I_t,
                                      const float *const *P_t, float *const *O_t, float *const *wc_opt,
                                      uint8_t *const *mask_opt) {
    tc_status r = check_stream(s, "tc_process_lanes");
    if (r != TC_OK) return r;
    if (!s->batch) return fail(s, TC_ERR_STATE, "tc_process_lanes: not a batch (tc_create_batch)");
    if (n < 1 || n > s->lanes || !lanes || !I_t || !P_t || !O_t)
        return fail(s, TC_ERR_INVALID_ARG, "tc_process_lanes: n must lie in [1, lanes] with non-NULL arrays");
    std::vector<char> seen(s->lanes, 0);
    for (int k = 0; k < n; ++k) {
        if (lanes[k] < 0 || lanes[k] >= s->lanes || seen[lanes[k]])
            return fail(s, TC_ERR_INVALID_ARG, "tc_process_lanes: lanes must be distinct and in [0, lanes)");
        seen[lanes[k]] = 1;
        if (!I_t[k] || !P_t[k] || !O_t[k]) return fail(s, TC_ERR_INVALID_ARG, "tc_process_lanes: NULL image pointer");
    }
    if (s->prec == TC_FP32) return process_lanes<float>(s, n, lanes, I_t, P_t, O_t, wc_opt, mask_opt);
    if (s->prec == TC_BF16) return process_lanes<__nv_bfloat16>(s, n, lanes, I_t, P_t, O_t, wc_opt, mask_opt);
    return process_lanes<__half>(s, n, lanes, I_t, P_t, O_t, wc_opt, mask_opt);
}

extern "C" tc_status tc_set_lane_consistency(tc_stream *s, int lane, const tc_consistency *p) {
    tc_status r = check_stream(s, "tc_set_lane_consistency");
    if (r != TC_OK) return r;
    if (!s->batch) return fail(s, TC_ERR_STATE, "tc_set_lane_consistency: not a batch (tc_create_batch)");
    if (lane < 0 || lane >= s->lanes || !p) return fail(s, TC_ERR_INVALID_ARG, "tc_set_lane_consistency: bad lane");
    if (p->solver_iters != 0) return fail(s, TC_ERR_UNSUPPORTED, "tc_set_lane_consistency: a batch runs without the solver");
    std::string why;
    if (!valid_params(p, why)) return fail(s, TC_ERR_INVALID_ARG, why);
    s->lane_params[lane] = *p;
    return TC_OK;
}

extern "C" tc_status tc_reset_lane(tc_stream *s, int lane) {
    tc_status r = check_stream(s, "tc_reset_lane");
    if (r != TC_OK) return r;
    if (!s->batch) return fail(s, TC_ERR_STATE, "tc_reset_lane: not a batch (tc_create_batch)");
    if (lane < 0 || lane >= s->lanes) return fail(s, TC_ERR_INVALID_ARG, "tc_reset_lane: bad lane");
    s->lane_t[lane] = 0;
    s->lane_cur[lane] = 0;
    tc_default_consistency(&s->lane_params[lane]);
    return TC_OK;
}

extern "C" tc_status tc_get_lane_flows(tc_stream *s, int lane, float *Fb, float *Ff) {
    tc_status r = check_stream(s, "tc_get_lane_flows");
    if (r != TC_OK) return r;
    if (!s->batch) return fail(s, TC_ERR_STATE, "tc_get_lane_flows: not a batch (tc_create_batch)");
    if (lane < 0 || lane >= s->lanes) return fail(s, TC_ERR_INVALID_ARG, "tc_get_lane_flows: bad lane");
    if (s->lane_t[lane] < 2) return fail(s, TC_ERR_STATE, "tc_get_lane_flows: the lane has no flows yet");
    const LevelBufs &B2 = s->lv[1];
    const size_t fimg = (size_t)B2.h * B2.w * 2;
    const float *fb = B2.flow + (size_t)2 * lane * fimg;
    if (Fb) TC_LAUNCH(s, launch_flow_out(fb, B2.h, B2.w, 4, s->H, s->W, Fb, s->st));
    if (Ff) TC_LAUNCH(s, launch_flow_out(fb + fimg, B2.h, B2.w, 4, s->H, s->W, Ff, s->st));
    return TC_OK;
}

extern "C" tc_status tc_process_frame(tc_stream *s, const float *I_t, const float *P_t, float *O_t,
                                      float *wc_opt, uint8_t *mask_opt) {
    tc_status r = single_only(s, "tc_process_frame");
    if (r != TC_OK) return r;
    if (!I_t || !P_t || !O_t) return fail(s, TC_ERR_INVALID_ARG, "tc_process_frame: NULL image pointer");
    if (s->prec == TC_FP32) return process<float>(s, I_t, P_t, O_t, wc_opt, mask_opt);
    if (s->prec == TC_BF16) return process<__nv_bfloat16>(s, I_t, P_t, O_t, wc_opt, mask_opt);
    if (s->prec == TC_FP16) return process<__half>(s, I_t, P_t, O_t, wc_opt, mask_opt);
    if (!s->fp8_ready)
        return fail(s, TC_ERR_STATE, "tc_process_frame: an e4m3 stream needs tc_set_fp8_scales before its first frame");
    return process<__nv_fp8_e4m3>(s, I_t, P_t, O_t, wc_opt, mask_opt);
}

// Reads the stream's device error word (after the stream has been synchronised).
static tc_status check_device_error(tc_stream *s) {
    if (!s->dev_err) return TC_OK;
    int e = 0;
    TC_TRY(s, cudaMemcpy(&e, s->dev_err, sizeof(int), cudaMemcpyDeviceToHost), "error word read");
    if (e != 0) {
        s->poisoned = true;
        return fail(s, TC_ERR_TIMEOUT, "a tensor-core kernel gave up waiting (code " + std::to_string(e) +
                                            "); the frame's results are invalid");
    }
    return TC_OK;
}

extern "C" tc_status tc_synchronize(tc_stream *s) {
    tc_status r = check_stream(s, "tc_synchronize");
    if (r != TC_OK) return r;
    TC_TRY(s, cudaStreamSynchronize(s->st), "stream synchronize");
    for (cudaStream_t q : {s->pst, s->bst})
        if (q) TC_TRY(s, cudaStreamSynchronize(q), "pipeline stream synchronize");
    for (cudaStream_t q : s->estx)
        if (q) TC_TRY(s, cudaStreamSynchronize(q), "pipeline stream synchronize");
    if (s->gst) TC_TRY(s, cudaStreamSynchronize(s->gst), "library stream synchronize");
    if (s->cst) TC_TRY(s, cudaStreamSynchronize(s->cst), "upload stream synchronize");
    if (s->dst) TC_TRY(s, cudaStreamSynchronize(s->dst), "download stream synchronize");
    return check_device_error(s);
}

// tc_process_frame_host_async and its 8-bit form.  Slot k of the device staging holds one
// call's inputs and outputs: two slots used in turn in the default mode, four in pipelined
// mode.  Copies run on two library streams: uploads on cst (with the 8-bit decode), downloads
// on dst.  Default mode: the frame runs on the stream's CUDA stream after the upload.
// Pipelined mode: the frame's pyramid (pst) and blend (bst) wait for the upload, and the
// blend also for the download that last read the slot's outputs; the slot's next upload waits
// for the blend (its last reader).  Either way the download follows the frame's last step.
static tc_status host_async(tc_stream *s, const void *I_t, const void *P_t, void *O_t, float *wc_opt,
                            uint8_t *mask_opt, bool rgb8, const char *fn) {
    tc_status r = single_only(s, fn);
    if (r != TC_OK) return r;
    if (!I_t || !P_t || !O_t) return fail(s, TC_ERR_INVALID_ARG, std::string(fn) + ": NULL image pointer");
    const size_t plane = (size_t)s->H * s->W, img = 3 * plane * sizeof(float), img8 = 3 * plane;
    const int nslot = s->pipelined ? tc_stream::NSLOT : 2;
    for (int k = 0; k < nslot; ++k) {
        if (!s->aI[k]) {
            if ((r = dalloc_t(s, &s->aI[k], img)) != TC_OK) return r;
            if ((r = dalloc_t(s, &s->aP[k], img)) != TC_OK) return r;
            if ((r = dalloc_t(s, &s->aO[k], img)) != TC_OK) return r;
            if ((r = dalloc_t(s, &s->awc[k], plane * sizeof(float))) != TC_OK) return r;
            if ((r = dalloc_t(s, &s->amask[k], plane)) != TC_OK) return r;
            TC_TRY(s, cudaEventCreateWithFlags(&s->a_in[k], cudaEventDisableTiming), "cudaEventCreate");
            TC_TRY(s, cudaEventCreateWithFlags(&s->a_done[k], cudaEventDisableTiming), "cudaEventCreate");
            TC_TRY(s, cudaEventCreateWithFlags(&s->a_out[k], cudaEventDisableTiming), "cudaEventCreate");
        }
        if (rgb8 && !s->a8I[k]) {
            if ((r = dalloc_t(s, &s->a8I[k], img8)) != TC_OK) return r;
            if ((r = dalloc_t(s, &s->a8P[k], img8)) != TC_OK) return r;
            if ((r = dalloc_t(s, &s->a8O[k], img8)) != TC_OK) return r;
        }
    }
    if (!s->cst) TC_TRY(s, cudaStreamCreateWithFlags(&s->cst, cudaStreamNonBlocking), "cudaStreamCreate");
    if (!s->dst) TC_TRY(s, cudaStreamCreateWithFlags(&s->dst, cudaStreamNonBlocking), "cudaStreamCreate");
    if (s->pipelined && (r = ensure_pipeline_streams(s)) != TC_OK) return r;
    const int k = (int)(s->a_n % nslot);
    // Slot k was last used nslot calls ago: a_done[k] marks the end of that frame's last step
    // (the last reader of aI[k], aP[k]), a_out[k] the end of its download (the last reader of
    // aO[k], awc[k], amask[k]).  A wait on an event not yet recorded returns at once.
    TC_TRY(s, cudaStreamWaitEvent(s->cst, s->a_done[k], 0), "cudaStreamWaitEvent");
    if (rgb8) {
        TC_TRY(s, cudaMemcpyAsync(s->a8I[k], I_t, img8, cudaMemcpyHostToDevice, s->cst), "H2D I_t");
        TC_TRY(s, cudaMemcpyAsync(s->a8P[k], P_t, img8, cudaMemcpyHostToDevice, s->cst), "H2D P_t");
        cudaStream_t st = s->st;
        s->st = s->cst;
        TC_LAUNCH(s, launch_unpack_rgb8(s->a8I[k], plane, s->aI[k], s->cst));
        TC_LAUNCH(s, launch_unpack_rgb8(s->a8P[k], plane, s->aP[k], s->cst));
        s->st = st;
    } else {
        TC_TRY(s, cudaMemcpyAsync(s->aI[k], I_t, img, cudaMemcpyHostToDevice, s->cst), "H2D I_t");
        TC_TRY(s, cudaMemcpyAsync(s->aP[k], P_t, img, cudaMemcpyHostToDevice, s->cst), "H2D P_t");
    }
    TC_TRY(s, cudaEventRecord(s->a_in[k], s->cst), "cudaEventRecord");
    // the streams that read the slot: the frame's stream, or the pyramid and blend streams
    cudaStream_t last = s->pipelined ? s->bst : s->st;
    if (s->pipelined) {
        TC_TRY(s, cudaStreamWaitEvent(s->pst, s->a_in[k], 0), "cudaStreamWaitEvent");
        TC_TRY(s, cudaStreamWaitEvent(s->bst, s->a_in[k], 0), "cudaStreamWaitEvent");
        TC_TRY(s, cudaStreamWaitEvent(s->bst, s->a_out[k], 0), "cudaStreamWaitEvent");
    } else {
        TC_TRY(s, cudaStreamWaitEvent(s->st, s->a_in[k], 0), "cudaStreamWaitEvent");
        TC_TRY(s, cudaStreamWaitEvent(s->st, s->a_out[k], 0), "cudaStreamWaitEvent");
    }
    r = tc_process_frame(s, s->aI[k], s->aP[k], s->aO[k], wc_opt ? s->awc[k] : nullptr,
                         mask_opt ? s->amask[k] : nullptr);
    if (r != TC_OK) return r;
    const bool wrote = s->last_out >= 0;  // one frame of latency: the first call of a sequence writes nothing
    if (rgb8 && wrote) {
        cudaStream_t st = s->st;
        s->st = last;
        TC_LAUNCH(s, launch_pack_rgb8(s->aO[k], plane, s->a8O[k], last));
        s->st = st;
    }
    TC_TRY(s, cudaEventRecord(s->a_done[k], last), "cudaEventRecord");
    TC_TRY(s, cudaStreamWaitEvent(s->dst, s->a_done[k], 0), "cudaStreamWaitEvent");
    if (wrote) {
        if (rgb8)
            TC_TRY(s, cudaMemcpyAsync(O_t, s->a8O[k], img8, cudaMemcpyDeviceToHost, s->dst), "D2H O_t");
        else
            TC_TRY(s, cudaMemcpyAsync(O_t, s->aO[k], img, cudaMemcpyDeviceToHost, s->dst), "D2H O_t");
        if (wc_opt)
            TC_TRY(s, cudaMemcpyAsync(wc_opt, s->awc[k], plane * sizeof(float), cudaMemcpyDeviceToHost, s->dst),
                   "D2H w_c");
        if (mask_opt) TC_TRY(s, cudaMemcpyAsync(mask_opt, s->amask[k], plane, cudaMemcpyDeviceToHost, s->dst), "D2H mask");
    }
    TC_TRY(s, cudaEventRecord(s->a_out[k], s->dst), "cudaEventRecord");
    s->a_n += 1;
    return TC_OK;
}

extern "C" tc_status tc_process_frame_host_async(tc_stream *s, const float *I_t, const float *P_t, float *O_t,
                                                 float *wc_opt, uint8_t *mask_opt) {
    return host_async(s, I_t, P_t, O_t, wc_opt, mask_opt, false, "tc_process_frame_host_async");
}

extern "C" tc_status tc_process_frame_host_rgb8_async(tc_stream *s, const uint8_t *I_t, const uint8_t *P_t,
                                                      uint8_t *O_t, float *wc_opt, uint8_t *mask_opt) {
    return host_async(s, I_t, P_t, O_t, wc_opt, mask_opt, true, "tc_process_frame_host_rgb8_async");
}

extern "C" tc_status tc_process_frame_host(tc_stream *s, const float *I_t, const float *P_t, float *O_t,
                                           float *wc_opt, uint8_t *mask_opt) {
    tc_status r = single_only(s, "tc_process_frame_host");
    if (r != TC_OK) return r;
    if (s->pipelined) return fail(s, TC_ERR_STATE, "tc_process_frame_host: not available in pipelined mode");
    if (!I_t || !P_t || !O_t) return fail(s, TC_ERR_INVALID_ARG, "tc_process_frame_host: NULL image pointer");
    const size_t img = (size_t)3 * s->H * s->W * sizeof(float), plane = (size_t)s->H * s->W;
    if (!s->hI) {
        if ((r = dalloc_t(s, &s->hI, img)) != TC_OK) return r;
        if ((r = dalloc_t(s, &s->hP, img)) != TC_OK) return r;
        if ((r = dalloc_t(s, &s->hO, img)) != TC_OK) return r;
        if ((r = dalloc_t(s, &s->hwc, plane * sizeof(float))) != TC_OK) return r;
        if ((r = dalloc_t(s, &s->hmask, plane)) != TC_OK) return r;
    }
    if (!s->cst) TC_TRY(s, cudaStreamCreateWithFlags(&s->cst, cudaStreamNonBlocking), "cudaStreamCreate");
    if (!s->ev_p) {
        TC_TRY(s, cudaEventCreateWithFlags(&s->ev_p, cudaEventDisableTiming), "cudaEventCreate");
        TC_TRY(s, cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming), "cudaEventCreate");
        TC_TRY(s, cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming), "cudaEventCreate");
    }
    // I_t first on the frame's stream; P_t, read only by the consistency pass at the end of
    // the frame, on the copy stream while the flow network runs (the previous call has
    // finished with hP: it waited for its stream)
    TC_TRY(s, cudaMemcpyAsync(s->hI, I_t, img, cudaMemcpyHostToDevice, s->st), "H2D I_t");
    TC_TRY(s, cudaMemcpyAsync(s->hP, P_t, img, cudaMemcpyHostToDevice, s->cst), "H2D P_t");
    TC_TRY(s, cudaEventRecord(s->ev_p, s->cst), "cudaEventRecord");
    s->p_pending = true;
    r = tc_process_frame(s, s->hI, s->hP, s->hO, wc_opt ? s->hwc : nullptr, mask_opt ? s->hmask : nullptr);
    s->p_pending = false;
    if (r != TC_OK) {
        cudaStreamSynchronize(s->cst);  // the upload into hP ends before any later call reuses it
        return r;
    }
    if (s->last_out < 0) {  // one frame of latency: the first call writes nothing
        TC_TRY(s, cudaStreamSynchronize(s->st), "stream synchronize");
        return check_device_error(s);
    }
    TC_TRY(s, cudaMemcpyAsync(O_t, s->hO, img, cudaMemcpyDeviceToHost, s->st), "D2H O_t");
    if (wc_opt) TC_TRY(s, cudaMemcpyAsync(wc_opt, s->hwc, plane * sizeof(float), cudaMemcpyDeviceToHost, s->st), "D2H w_c");
    if (mask_opt) TC_TRY(s, cudaMemcpyAsync(mask_opt, s->hmask, plane, cudaMemcpyDeviceToHost, s->st), "D2H mask");
    TC_TRY(s, cudaStreamSynchronize(s->st), "stream synchronize");
    return check_device_error(s);
}

extern "C" tc_status tc_set_latency(tc_stream *s, int frames) {
    tc_status r = single_only(s, "tc_set_latency");
    if (r != TC_OK) return r;
    if (frames != 0 && frames != 1) return fail(s, TC_ERR_INVALID_ARG, "tc_set_latency: frames must be 0 or 1");
    if (s->t != 0) return fail(s, TC_ERR_STATE, "tc_set_latency: only before the first frame of a sequence");
    if (frames == 1 && !(s->params.k1 + s->params.k2 < 1.f))
        return fail(s, TC_ERR_INVALID_ARG, "with the next-frame term k1 + k2 must be < 1");
    if (frames == 1 && !s->Fprev) {
        const LevelBufs &B2 = s->lv[1];
        if ((r = dalloc_t(s, &s->Fprev, (size_t)B2.h * B2.w * 4 * sizeof(float))) != TC_OK) return r;
    }
    if (frames != s->latency) {
        TC_TRY(s, cudaStreamSynchronize(s->st), "stream synchronize");
        release_graphs(s);
    }
    s->latency = frames;
    s->last_out = -1;
    return TC_OK;
}

extern "C" tc_status tc_set_pipelined(tc_stream *s, int enable) {
    tc_status r = single_only(s, "tc_set_pipelined");
    if (r != TC_OK) return r;
    if (s->t != 0) return fail(s, TC_ERR_STATE, "tc_set_pipelined: only before the first frame of a sequence");
    if (enable && s->rec_amax) return fail(s, TC_ERR_STATE, "tc_set_pipelined: not while recording amax");
    if ((enable != 0) != s->pipelined) {
        if ((r = tc_synchronize(s)) != TC_OK) return r;
        release_graphs(s);
        s->pipelined = enable != 0;
    }
    return TC_OK;
}

extern "C" tc_status tc_join(tc_stream *s) {
    tc_status r = check_stream(s, "tc_join");
    if (r != TC_OK) return r;
    return join_caller(s);
}

extern "C" tc_status tc_set_frame_timing(tc_stream *s, int enable) {
    tc_status r = single_only(s, "tc_set_frame_timing");
    if (r != TC_OK) return r;
    s->frame_timing = enable != 0;
    s->ft_n = 0;
    return TC_OK;
}

extern "C" tc_status tc_get_frame_times(tc_stream *s, float *ms, int n, int *count) {
    tc_status r = single_only(s, "tc_get_frame_times");
    if (r != TC_OK) return r;
    if (!count || (n > 0 && !ms)) return fail(s, TC_ERR_INVALID_ARG, "tc_get_frame_times: NULL argument");
    const int k = (int)std::min<size_t>(s->ft_n, n > 0 ? (size_t)n : 0);
    if (s->ft_n > 0) TC_TRY(s, cudaEventSynchronize(s->ft_done[s->ft_n - 1]), "cudaEventSynchronize");
    for (int i = 0; i < k; ++i)
        TC_TRY(s, cudaEventElapsedTime(&ms[i], s->ft_start[i], s->ft_done[i]), "cudaEventElapsedTime");
    *count = (int)s->ft_n;
    return TC_OK;
}

extern "C" tc_status tc_flush(tc_stream *s, float *O_t, float *wc_opt, uint8_t *mask_opt) {
    tc_status r = single_only(s, "tc_flush");
    if (r != TC_OK) return r;
    if (!s->latency) return fail(s, TC_ERR_STATE, "tc_flush: the stream has no frame of latency");
    if (s->t == 0) return fail(s, TC_ERR_STATE, "tc_flush: no frame pending");
    if (!O_t) return fail(s, TC_ERR_INVALID_ARG, "tc_flush: NULL image pointer");
    s->launches = 0;
    const int cur = (int)(s->t & 1);
    // the last frame has no next frame: the causal blend with the kept flows (pipelined
    // mode: on the library stream, after the frames given)
    cudaStream_t caller = s->st;
    if (s->pipelined && s->bst) s->st = s->bst;
    const ConsistArgs ca = consist_args(s, nullptr, nullptr, O_t, wc_opt, mask_opt, cur, true);
    r = TC_OK;
    const cudaError_t ce = launch_consistency(ca, s->st);
    ++s->launches;
    if (ce != cudaSuccess) r = cuda_fail(s, ce, "tc_flush launch");
    if (r == TC_OK && s->t > 1 && s->params.solver_iters > 0) r = solver_launches(s, O_t, wc_opt, cur);
    if (r == TC_OK && s->pipelined && s->bst && s->last_blend >= 0) {
        const cudaError_t ee = cudaEventRecord(s->ev_blends[s->last_blend], s->bst);
        if (ee != cudaSuccess) r = cuda_fail(s, ee, "cudaEventRecord");
    }
    s->st = caller;
    if (r != TC_OK) return r;
    s->last_out = s->t - 1;
    s->t = 0;
    return TC_OK;
}

extern "C" long long tc_last_output_frame(const tc_stream *s) { return s ? s->last_out : -1; }

extern "C" tc_status tc_get_flows(tc_stream *s, float *Fb, float *Ff) {
    tc_status r = single_only(s, "tc_get_flows");
    if (r != TC_OK) return r;
    if (s->t < 2) return fail(s, TC_ERR_STATE, "tc_get_flows: no flow before the second frame");
    if ((r = join_caller(s)) != TC_OK) return r;
    LevelBufs &B2 = s->lv[1];
    float *flow2 = flow_of(B2, s->last_set);
    if (Fb) TC_LAUNCH(s, launch_flow_out(flow2, B2.h, B2.w, 4 * s->fs, s->H, s->W, Fb, s->st));
    if (Ff)
        TC_LAUNCH(s, launch_flow_out(flow2 + (size_t)B2.h * B2.w * 2, B2.h, B2.w, 4 * s->fs, s->H, s->W, Ff, s->st));
    return TC_OK;
}

extern "C" tc_status tc_destroy(tc_stream *s) {
    if (!s) return fail(nullptr, TC_ERR_INVALID_ARG, "tc_destroy: NULL stream");
    if (s->st) cudaStreamSynchronize(s->st);
    else cudaDeviceSynchronize();
    for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
    release_graphs(s);
    release_graph_stream(s);
    if (s->cst) {
        cudaStreamSynchronize(s->cst);
        cudaStreamDestroy(s->cst);
    }
    if (s->ev_p) cudaEventDestroy(s->ev_p);  // after the graphs that wait on it
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    if (s->ev_join) cudaEventDestroy(s->ev_join);
    if (s->dst) {
        cudaStreamSynchronize(s->dst);
        cudaStreamDestroy(s->dst);
    }
    for (int k = 0; k < 2; ++k) {
        if (s->a_in[k]) cudaEventDestroy(s->a_in[k]);
        if (s->a_done[k]) cudaEventDestroy(s->a_done[k]);
        if (s->a_out[k]) cudaEventDestroy(s->a_out[k]);
    }
    free_all(s);
    delete s;
    return TC_OK;
}

extern "C" tc_status tc_set_profiling(tc_stream *s, int enable) {
    tc_status r = check_stream(s, "tc_set_profiling");
    if (r != TC_OK) return r;
    if ((r = prof_flush(s)) != TC_OK) return r;
    s->prof = enable != 0;
    for (int k = 0; k < TC_PROF_CATEGORIES; ++k) {
        s->prof_ms[k] = 0.0;
        s->prof_n[k] = 0;
    }
    return TC_OK;
}

extern "C" tc_status tc_get_profile(tc_stream *s, double *ms, long long *launches, int n) {
    tc_status r = check_stream(s, "tc_get_profile");
    if (r != TC_OK) return r;
    if (!ms || n < 1) return fail(s, TC_ERR_INVALID_ARG, "tc_get_profile: bad argument");
    if ((r = prof_flush(s)) != TC_OK) return r;
    for (int k = 0; k < n && k < TC_PROF_CATEGORIES; ++k) {
        ms[k] = s->prof_ms[k];
        if (launches) launches[k] = s->prof_n[k];
    }
    return TC_OK;
}

extern "C" const char *tc_last_error(const tc_stream *s) {
    if (s) return s->err.c_str();
    std::lock_guard<std::mutex> lk(g_err_mu);
    return g_err.c_str();
}

extern "C" int tc_last_launch_count(const tc_stream *s) { return s ? s->launches : 0; }

extern "C" int tc_tensor_core_layers(const tc_stream *s) { return s ? s->tc_layers : 0; }

extern "C" int tc_tensor_core_correlation_levels(const tc_stream *s) { return s ? s->tc_corr_levels : 0; }

extern "C" size_t tc_stream_device_bytes(const tc_stream *s) {
    if (!s) return 0;
    size_t b = s->dev_bytes;
    for (const auto &B : s->lv) {
        for (const auto &pl : B.tcplan) b += pl.wpk_bytes;
        b += B.headplan.wpk_bytes;
    }
    for (const auto &lvl : s->pyr_plan)
        for (const auto &pl : lvl) b += pl.wpk_bytes;
    for (const auto &R : s->ref) b += R.plan.wpk_bytes;
    return b;
}

// ------------------------------------------------------------------------------- stage ops

namespace {
struct TmpAlloc {
    std::vector<void *> ps;
    ~TmpAlloc() {
        for (void *p : ps) cudaFree(p);
    }
    cudaError_t get(void **p, size_t bytes) {
        cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
        if (e == cudaSuccess) ps.push_back(*p);
        return e;
    }
};
}  // namespace

#define OP_TRY(expr, what)                                               \
    do {                                                                 \
        cudaError_t _e = (expr);                                         \
        if (_e != cudaSuccess) return cuda_fail(nullptr, _e, what);      \
    } while (0)

template <typename T>
static tc_status op_conv(const float *in, int n, int h, int w, int cin, const float *w_oihw, const float *bias,
                         int cout, int stride, int leaky, float *out, cudaStream_t st) {
    HostLayer L;
    L.cout = cout; L.cin = cin; L.stride = stride; L.leaky = leaky;
    L.w.assign(w_oihw, w_oihw + (size_t)cout * cin * 9);
    L.b.assign(bias, bias + cout);
    const bool bf = sizeof(T) == 2;      // bfloat16 or half operands
    constexpr bool f16 = std::is_same<T, __half>::value;
    constexpr bool f8 = sizeof(T) == 1;  // e4m3 activations with scale 1; tensor cores only
    const int cin_p = round_up(cin, f8 ? 16 : (bf ? 8 : 4)), cout_p = round_up(cout, f8 ? 16 : 4);
    const int ho = (h - 1) / stride + 1, wo = (w - 1) / stride + 1;
    std::vector<float> wk =
        simt_weights(L, iota_perm(cin, cin_p), !bf ? TC_FP32 : (f16 ? TC_FP16 : TC_BF16));
    // pad cout to a multiple of 4 (16 for e4m3)
    std::vector<float> wkp((size_t)9 * cin_p * cout_p, 0.f), bp(cout_p, 0.f);
    for (size_t k = 0; k < (size_t)9 * cin_p; ++k)
        for (int o = 0; o < cout; ++o) wkp[k * cout_p + o] = wk[k * cout + o];
    for (int o = 0; o < cout; ++o) bp[o] = bias[o];
    TmpAlloc tmp;
    float *dw, *db;
    T *din, *dout;
    OP_TRY(tmp.get((void **)&dw, wkp.size() * 4), "tc_op_conv3x3 alloc");
    OP_TRY(tmp.get((void **)&db, bp.size() * 4), "tc_op_conv3x3 alloc");
    OP_TRY(cudaMemcpyAsync(dw, wkp.data(), wkp.size() * 4, cudaMemcpyHostToDevice, st), "tc_op_conv3x3 copy");
    OP_TRY(cudaMemcpyAsync(db, bp.data(), bp.size() * 4, cudaMemcpyHostToDevice, st), "tc_op_conv3x3 copy");
    const size_t nin = (size_t)n * h * w * cin_p, nout = (size_t)n * ho * wo * cout_p;
    OP_TRY(tmp.get((void **)&din, nin * sizeof(T)), "tc_op_conv3x3 alloc");
    OP_TRY(tmp.get((void **)&dout, nout * sizeof(T)), "tc_op_conv3x3 alloc");
    // Repack the input to cin_p channels in the activation type.
    std::vector<float> dummy;
    if (cin_p == cin) {
        OP_TRY(launch_to_act<T>(in, nin, din, st), "tc_op_conv3x3 convert");
    } else {
        float *tmpf;
        OP_TRY(tmp.get((void **)&tmpf, nin * 4), "tc_op_conv3x3 alloc");
        OP_TRY(cudaMemsetAsync(tmpf, 0, nin * 4, st), "tc_op_conv3x3 memset");
        OP_TRY(cudaMemcpy2DAsync(tmpf, cin_p * 4, in, cin * 4, cin * 4, (size_t)n * h * w, cudaMemcpyDeviceToDevice, st),
               "tc_op_conv3x3 repack");
        OP_TRY(launch_to_act<T>(tmpf, nin, din, st), "tc_op_conv3x3 convert");
    }
    ConvArgs a{din, cin_p, n, h, w, cin_p, stride, ho, wo, dw, db, cout_p, dout, cout_p, leaky, 1.f};
    TcConvPlan plan;
    int *derr = nullptr;
    OP_TRY(tmp.get((void **)&derr, sizeof(int)), "tc_op_conv3x3 alloc");
    OP_TRY(cudaMemsetAsync(derr, 0, sizeof(int), st), "tc_op_conv3x3 memset");
    std::string why;
    const bool use_tc = (bf || f8) && tc_plan_conv(plan, a, n, wkp, derr, why, f8, 9, f16);
    if (use_tc) {
        cudaError_t e = launch_conv_tc(plan, a, st);
        if (e != cudaSuccess) {
            plan.release();
            return cuda_fail(nullptr, e, "tc_op_conv3x3 tensor-core launch");
        }
    } else if constexpr (f8) {
        return fail(nullptr, TC_ERR_UNSUPPORTED, "tc_op_conv3x3: e4m3 runs on the tensor cores only: " + why);
    } else {
        OP_TRY(launch_conv_simt<T>(a, st), "tc_op_conv3x3 launch");
    }
    float *outp;
    if (cout_p == cout) {
        OP_TRY(launch_from_act<T>(dout, nout, out, st), "tc_op_conv3x3 convert");
    } else {
        OP_TRY(tmp.get((void **)&outp, nout * 4), "tc_op_conv3x3 alloc");
        OP_TRY(launch_from_act<T>(dout, nout, outp, st), "tc_op_conv3x3 convert");
        OP_TRY(cudaMemcpy2DAsync(out, cout * 4, outp, cout_p * 4, cout * 4, (size_t)n * ho * wo, cudaMemcpyDeviceToDevice, st),
               "tc_op_conv3x3 repack");
    }
    cudaError_t se = cudaStreamSynchronize(st);
    plan.release();
    if (se != cudaSuccess) return cuda_fail(nullptr, se, "tc_op_conv3x3 sync");
    int e = 0;
    OP_TRY(cudaMemcpy(&e, derr, sizeof(int), cudaMemcpyDeviceToHost), "tc_op_conv3x3 error word");
    if (e != 0) return fail(nullptr, TC_ERR_TIMEOUT, "tc_op_conv3x3: tensor-core kernel gave up waiting");
    g_last_op_tc = use_tc ? 1 : 0;
    return TC_OK;
}

extern "C" int tc_op_last_used_tensor_cores(void) { return g_last_op_tc; }

extern "C" void tc_test_fail_device_allocation(long long nth) { g_alloc_fail_countdown.store(nth > 0 ? nth : 0); }

void tc_set_last_op_tensor_cores(int used) { g_last_op_tc = used ? 1 : 0; }

extern "C" tc_status tc_op_conv3x3(tc_precision precision, const float *in, int n, int h, int w, int cin,
                                   const float *w_oihw, const float *bias, int cout, int stride, int leaky,
                                   float *out, void *cuda_stream) {
    if (!in || !w_oihw || !bias || !out || n < 1 || h < 1 || w < 1 || cin < 1 || cout < 1 ||
        (stride != 1 && stride != 2))
        return fail(nullptr, TC_ERR_INVALID_ARG, "tc_op_conv3x3: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (precision == TC_FP32) return op_conv<float>(in, n, h, w, cin, w_oihw, bias, cout, stride, leaky, out, st);
    if (precision == TC_BF16) return op_conv<__nv_bfloat16>(in, n, h, w, cin, w_oihw, bias, cout, stride, leaky, out, st);
    if (precision == TC_FP16) return op_conv<__half>(in, n, h, w, cin, w_oihw, bias, cout, stride, leaky, out, st);
    if (precision == TC_FP8_E4M3)
        return op_conv<__nv_fp8_e4m3>(in, n, h, w, cin, w_oihw, bias, cout, stride, leaky, out, st);
    return fail(nullptr, TC_ERR_INVALID_ARG, "tc_op_conv3x3: precision");
}

// One depthwise-separable layer on its own (see tc_op_sepconv).
template <typename T>
static tc_status op_sepconv(const float *in, int n, int h, int w, int cin, const float *dw, const float *db,
                            const float *pw, const float *pb, int cout, int dil, int leaky, float *out,
                            cudaStream_t st) {
    const bool bf = sizeof(T) == 2;
    const bool head = cout == 2;
    const size_t npx = (size_t)n * h * w;
    // weights in the engine's layout: depthwise [9][cin], pointwise [cin][cout]
    std::vector<float> dwk((size_t)9 * cin), pwk((size_t)cin * cout);
    for (int c = 0; c < cin; ++c)
        for (int t = 0; t < 9; ++t) dwk[(size_t)t * cin + c] = dw[(size_t)c * 9 + t];
    for (int c = 0; c < cin; ++c)
        for (int o = 0; o < cout; ++o) pwk[(size_t)c * cout + o] = pw[(size_t)o * cin + c];
    TmpAlloc tmp;
    float *ddw, *ddb, *dpw, *dpb, *flow = nullptr;
    T *x, *d, *o = nullptr;
    OP_TRY(tmp.get((void **)&ddw, dwk.size() * 4), "tc_op_sepconv alloc");
    OP_TRY(tmp.get((void **)&ddb, (size_t)cin * 4), "tc_op_sepconv alloc");
    OP_TRY(tmp.get((void **)&dpw, pwk.size() * 4), "tc_op_sepconv alloc");
    OP_TRY(tmp.get((void **)&dpb, (size_t)cout * 4), "tc_op_sepconv alloc");
    OP_TRY(tmp.get((void **)&x, npx * cin * sizeof(T)), "tc_op_sepconv alloc");
    OP_TRY(tmp.get((void **)&d, npx * cin * sizeof(T)), "tc_op_sepconv alloc");
    if (head) {
        OP_TRY(tmp.get((void **)&flow, npx * 2 * 4), "tc_op_sepconv alloc");
        OP_TRY(cudaMemsetAsync(flow, 0, npx * 2 * 4, st), "tc_op_sepconv memset");
    } else {
        OP_TRY(tmp.get((void **)&o, npx * cout * sizeof(T)), "tc_op_sepconv alloc");
    }
    OP_TRY(cudaMemcpyAsync(ddw, dwk.data(), dwk.size() * 4, cudaMemcpyHostToDevice, st), "tc_op_sepconv copy");
    OP_TRY(cudaMemcpyAsync(ddb, db, (size_t)cin * 4, cudaMemcpyHostToDevice, st), "tc_op_sepconv copy");
    OP_TRY(cudaMemcpyAsync(dpw, pwk.data(), pwk.size() * 4, cudaMemcpyHostToDevice, st), "tc_op_sepconv copy");
    OP_TRY(cudaMemcpyAsync(dpb, pb, (size_t)cout * 4, cudaMemcpyHostToDevice, st), "tc_op_sepconv copy");
    OP_TRY(launch_to_act<T>(in, npx * cin, x, st), "tc_op_sepconv convert");
    DwArgs da{x, cin, cin, nullptr, n, h, w, ddw, ddb, dil, d, cin, cin};
    OP_TRY(launch_depthwise<T>(da, st), "tc_op_sepconv depthwise launch");
    TcConvPlan plan;
    int *derr = nullptr;
    OP_TRY(tmp.get((void **)&derr, sizeof(int)), "tc_op_sepconv alloc");
    OP_TRY(cudaMemsetAsync(derr, 0, sizeof(int), st), "tc_op_sepconv memset");
    ConvArgs a{d, cin, n, h, w, cin, 1, h, w, nullptr, dpb, cout, o, head ? 16 : cout, leaky};
    std::string why;
    constexpr bool f16 = std::is_same<T, __half>::value;
    const bool use_tc = bf && (head ? tc_plan_head(plan, a, n, pwk, derr, why, false, 1, f16)
                                    : tc_plan_conv(plan, a, n, pwk, derr, why, false, 1, f16));
    if (use_tc) {
        const cudaError_t e = head ? launch_conv_tc_head(plan, a, flow, flow, st) : launch_conv_tc(plan, a, st);
        if (e != cudaSuccess) {
            plan.release();
            return fail(nullptr, TC_ERR_CUDA, std::string("tc_op_sepconv tensor-core launch: ") + cudaGetErrorString(e));
        }
    } else {
        PwArgs pa{d, cin, cin, dpw, dpb, cout, leaky, o, cout, flow, npx};
        OP_TRY(launch_pointwise<T>(pa, st), "tc_op_sepconv pointwise launch");
    }
    if (head)
        OP_TRY(cudaMemcpyAsync(out, flow, npx * 2 * 4, cudaMemcpyDeviceToDevice, st), "tc_op_sepconv copy");
    else
        OP_TRY(launch_from_act<T>(o, npx * cout, out, st), "tc_op_sepconv convert");
    const cudaError_t se = cudaStreamSynchronize(st);
    plan.release();
    OP_TRY(se, "tc_op_sepconv sync");
    int e = 0;
    OP_TRY(cudaMemcpy(&e, derr, sizeof(int), cudaMemcpyDeviceToHost), "tc_op_sepconv error word");
    if (e != 0) return fail(nullptr, TC_ERR_TIMEOUT, "tc_op_sepconv: tensor-core kernel gave up waiting");
    g_last_op_tc = use_tc ? 1 : 0;
    return TC_OK;
}

extern "C" tc_status tc_op_sepconv(tc_precision precision, const float *in, int n, int h, int w, int cin,
                                   const float *dw, const float *db, const float *pw, const float *pb, int cout,
                                   int dil, int leaky, float *out, void *cuda_stream) {
    if (!in || !dw || !db || !pw || !pb || !out || n < 1 || h < 1 || w < 1 || cin < 8 || cin % 8 != 0 ||
        cin > 256 || (cout != 2 && (cout < 8 || cout % 8 != 0 || cout > 256)) || dil < 1 || dil > 64)
        return fail(nullptr, TC_ERR_INVALID_ARG, "tc_op_sepconv: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (precision == TC_FP32) return op_sepconv<float>(in, n, h, w, cin, dw, db, pw, pb, cout, dil, leaky, out, st);
    if (precision == TC_BF16)
        return op_sepconv<__nv_bfloat16>(in, n, h, w, cin, dw, db, pw, pb, cout, dil, leaky, out, st);
    if (precision == TC_FP16) return op_sepconv<__half>(in, n, h, w, cin, dw, db, pw, pb, cout, dil, leaky, out, st);
    return fail(nullptr, TC_ERR_INVALID_ARG, "tc_op_sepconv: precision must be TC_FP32, TC_BF16 or TC_FP16");
}

template <typename T>
static tc_status op_corr(const float *f1, const float *f2, int n, int h, int w, int c, int r, float *out,
                         cudaStream_t st) {
    const int D = (2 * r + 1) * (2 * r + 1);
    const size_t nf = (size_t)n * h * w * c, no = (size_t)n * h * w * D;
    TmpAlloc tmp;
    T *a, *b, *o;
    OP_TRY(tmp.get((void **)&a, nf * sizeof(T)), "tc_op_correlation alloc");
    OP_TRY(tmp.get((void **)&b, nf * sizeof(T)), "tc_op_correlation alloc");
    OP_TRY(tmp.get((void **)&o, no * sizeof(T)), "tc_op_correlation alloc");
    OP_TRY(launch_to_act<T>(f1, nf, a, st), "tc_op_correlation convert");
    OP_TRY(launch_to_act<T>(f2, nf, b, st), "tc_op_correlation convert");
    const size_t img = (size_t)h * w * c;
    CorrTcPlan plan;
    int *derr = nullptr;
    OP_TRY(tmp.get((void **)&derr, sizeof(int)), "tc_op_correlation alloc");
    OP_TRY(cudaMemsetAsync(derr, 0, sizeof(int), st), "tc_op_correlation memset");
    std::string why;
    constexpr bool f8 = sizeof(T) == 1;  // e4m3 features and cost volume with scale 1
    const bool use_tc = (sizeof(T) == 2 || f8) &&
                        tc_plan_corr(plan, a, n, c, b, n, c, h, w, c, r, derr, why, f8, std::is_same<T, __half>::value);
    if (f8 && !use_tc)
        return fail(nullptr, TC_ERR_UNSUPPORTED, "tc_op_correlation: e4m3 runs on the tensor cores only: " + why);
    for (int i = 0; i < n; i += 2) {
        const int nb = n - i < 2 ? n - i : 2;
        if (use_tc) {
            const int imgs[2] = {i, i + nb - 1};
            OP_TRY(launch_corr_tc(plan, nb, imgs, imgs, o + (size_t)i * h * w * D, D, nullptr, nullptr, st),
                   "tc_op_correlation tensor-core launch");
        } else if constexpr (!f8) {
            CorrArgs ca{{a + i * img, a + (i + nb - 1) * img}, {b + i * img, b + (i + nb - 1) * img}, c, c, nb, h, w, c,
                        r, o + (size_t)i * h * w * D, D, nullptr};
            OP_TRY(launch_corr<T>(ca, st), "tc_op_correlation launch");
        }
    }
    OP_TRY(launch_from_act<T>(o, no, out, st), "tc_op_correlation convert");
    OP_TRY(cudaStreamSynchronize(st), "tc_op_correlation sync");
    int e = 0;
    OP_TRY(cudaMemcpy(&e, derr, sizeof(int), cudaMemcpyDeviceToHost), "tc_op_correlation error word");
    if (e != 0) return fail(nullptr, TC_ERR_TIMEOUT, "tc_op_correlation: tensor-core kernel gave up waiting");
    g_last_op_tc = use_tc ? 1 : 0;
    return TC_OK;
}

extern "C" tc_status tc_op_correlation(tc_precision precision, const float *f1, const float *f2, int n, int h,
                                       int w, int c, int r, float *out, void *cuda_stream) {
    if (!f1 || !f2 || !out || n < 1 || h < 1 || w < 1 || c < 4 || c % 4 != 0 || r < 1 || r > 4)
        return fail(nullptr, TC_ERR_INVALID_ARG, "tc_op_correlation: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (precision == TC_FP32) return op_corr<float>(f1, f2, n, h, w, c, r, out, st);
    if (precision == TC_BF16) return op_corr<__nv_bfloat16>(f1, f2, n, h, w, c, r, out, st);
    if (precision == TC_FP16) return op_corr<__half>(f1, f2, n, h, w, c, r, out, st);
    if (precision == TC_FP8_E4M3) return op_corr<__nv_fp8_e4m3>(f1, f2, n, h, w, c, r, out, st);
    return fail(nullptr, TC_ERR_INVALID_ARG, "tc_op_correlation: precision");
}

template <typename T>
static tc_status op_warp(const float *f, const float *flow, int n, int h, int w, int c, float *out, cudaStream_t st) {
    const size_t nf = (size_t)n * h * w * c;
    TmpAlloc tmp;
    T *a, *o;
    OP_TRY(tmp.get((void **)&a, nf * sizeof(T)), "tc_op_warp_features alloc");
    OP_TRY(tmp.get((void **)&o, nf * sizeof(T)), "tc_op_warp_features alloc");
    OP_TRY(launch_to_act<T>(f, nf, a, st), "tc_op_warp_features convert");
    const size_t img = (size_t)h * w * c;
    for (int i = 0; i < n; i += 2) {
        const int nb = n - i < 2 ? n - i : 2;
        WarpArgs wa{{a + i * img, a + (i + nb - 1) * img}, c, flow + (size_t)i * h * w * 2, nb, h, w, c, o + i * img, c,
                    nullptr, nullptr, nullptr, 0, 1.f};
        OP_TRY(launch_warp<T>(wa, st), "tc_op_warp_features launch");
    }
    OP_TRY(launch_from_act<T>(o, nf, out, st), "tc_op_warp_features convert");
    OP_TRY(cudaStreamSynchronize(st), "tc_op_warp_features sync");
    return TC_OK;
}

extern "C" tc_status tc_op_warp_features(tc_precision precision, const float *f, const float *flow, int n, int h,
                                         int w, int c, float *out, void *cuda_stream) {
    if (!f || !flow || !out || n < 1 || h < 1 || w < 1 || c < 4 || c % 4 != 0)
        return fail(nullptr, TC_ERR_INVALID_ARG, "tc_op_warp_features: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (precision == TC_FP32) return op_warp<float>(f, flow, n, h, w, c, out, st);
    if (precision == TC_BF16) return op_warp<__nv_bfloat16>(f, flow, n, h, w, c, out, st);
    if (precision == TC_FP16) return op_warp<__half>(f, flow, n, h, w, c, out, st);
    if (precision == TC_FP8_E4M3) return op_warp<__nv_fp8_e4m3>(f, flow, n, h, w, c, out, st);
    return fail(nullptr, TC_ERR_INVALID_ARG, "tc_op_warp_features: precision");
}

extern "C" tc_status tc_op_upsample_flow(const float *flow, int n, int h, int w, int s, float *out, void *cuda_stream) {
    if (!flow || !out || n < 1 || h < 1 || w < 1 || (s != 2 && s != 4) || (size_t)h * w > (size_t)INT_MAX)
        return fail(nullptr, TC_ERR_INVALID_ARG, "tc_op_upsample_flow: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    UpArgs u{flow, n, h, w, s, out, nullptr, 0};
    OP_TRY(launch_up<float>(u, st), "tc_op_upsample_flow launch");
    return TC_OK;
}

extern "C" tc_status tc_op_poisson_solve(const float *P, const float *A, const float *wc, int c, int h, int w,
                                         int iters, float eta, float kappa, float *O, void *cuda_stream) {
    if (!P || !A || !wc || !O || (c != 1 && c != 3) || h < 1 || w < 1 || iters < 0 || iters > 100000 ||
        !std::isfinite(eta) || !std::isfinite(kappa))
        return fail(nullptr, TC_ERR_INVALID_ARG, "tc_op_poisson_solve: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const size_t n = (size_t)c * h * w;
    TmpAlloc tmp;
    float *b, *s0, *s1, *s2, *s3, *c0;
    OP_TRY(tmp.get((void **)&b, n * 4), "tc_op_poisson_solve alloc");
    OP_TRY(tmp.get((void **)&c0, (size_t)h * w * 4), "tc_op_poisson_solve alloc");
    OP_TRY(tmp.get((void **)&s0, n * 4), "tc_op_poisson_solve alloc");
    OP_TRY(tmp.get((void **)&s1, n * 4), "tc_op_poisson_solve alloc");
    OP_TRY(tmp.get((void **)&s2, n * 4), "tc_op_poisson_solve alloc");
    OP_TRY(tmp.get((void **)&s3, n * 4), "tc_op_poisson_solve alloc");
    if (iters == 0) {
        OP_TRY(cudaMemcpyAsync(O, A, n * 4, cudaMemcpyDeviceToDevice, st), "tc_op_poisson_solve copy");
    } else {
        PoissonArgs pa{P, A, wc, c, h, w, iters, eta, kappa, b, s0, s1, s2, s3, O, nullptr, c0};
        OP_TRY(launch_poisson(pa, st), "tc_op_poisson_solve launch");
    }
    OP_TRY(cudaStreamSynchronize(st), "tc_op_poisson_solve sync");
    return TC_OK;
}

extern "C" tc_status tc_op_consistency(const float *It, const float *Pt, const float *Ip, const float *Pp,
                                       const float *Op, const float *Fb, const float *Ff, int h, int w, int fh,
                                       int fw, int scale, const tc_consistency *p, float *O, float *wc_opt,
                                       uint8_t *mask_opt, void *cuda_stream) {
    if (!It || !Pt || !Ip || !Pp || !Op || !Fb || !Ff || !p || !O || h < 1 || w < 1 || fh < 1 || fw < 1 ||
        scale < 1 || (scale & (scale - 1)) != 0 || (size_t)fh * scale < (size_t)h || (size_t)fw * scale < (size_t)w ||
        (size_t)h * w > (size_t)INT_MAX || (size_t)fh * fw > (size_t)INT_MAX)
        return fail(nullptr, TC_ERR_INVALID_ARG, "tc_op_consistency: bad argument");
    std::string why;
    if (!valid_params(p, why)) return fail(nullptr, TC_ERR_INVALID_ARG, why);
    ConsistArgs ca{};
    const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    TmpAlloc tmp;
    const size_t hw = (size_t)h * w;
    float4 *A, *B;
    float *C;
    // frame t - 1 into the layout a stream keeps (the pass reads it there)
    OP_TRY(tmp.get((void **)&A, hw * sizeof(float4)), "tc_op_consistency alloc");
    OP_TRY(tmp.get((void **)&B, hw * sizeof(float4)), "tc_op_consistency alloc");
    OP_TRY(tmp.get((void **)&C, hw * sizeof(float)), "tc_op_consistency alloc");
    OP_TRY(launch_pack_state(Ip, Pp, Op, hw, A, B, C, st), "tc_op_consistency pack");
    ca.It = It; ca.Pt = Pt; ca.pA = A; ca.pB = ca.oB = B; ca.pC = C; ca.Fb = Fb; ca.Ff = Ff;
    ca.H = h; ca.W = w; ca.fh = fh; ca.fw = fw; ca.scale = scale;
    ca.k1 = p->k1; ca.alpha = p->alpha; ca.lambda = p->lambda; ca.c1 = p->fb_c1; ca.c2 = p->fb_c2;
    ca.fb_check = p->fb_check; ca.first = 0;
    ca.O = O; ca.wc = wc_opt; ca.mask = mask_opt;
    OP_TRY(launch_consistency(ca, st), "tc_op_consistency launch");
    OP_TRY(cudaStreamSynchronize(st), "tc_op_consistency synchronize");  // before the temporaries go
    return TC_OK;
}

extern "C" tc_status tc_op_downscale2(const float *src, int c, int h, int w, float *dst, void *cuda_stream) {
    if (!src || !dst || c < 1 || h < 1 || w < 1) return fail(nullptr, TC_ERR_INVALID_ARG, "tc_op_downscale2: bad argument");
    OP_TRY(launch_downscale2(src, c, h, w, dst, static_cast<cudaStream_t>(cuda_stream)), "tc_op_downscale2 launch");
    return TC_OK;
}

extern "C" tc_status tc_op_consistency_next(const float *It, const float *Pt, const float *Ip, const float *Pp,
                                            const float *Op, const float *Fb, const float *Ff, const float *In,
                                            const float *Pn, const float *Fn, const float *Fnb, int h, int w,
                                            int fh, int fw, int scale, const tc_consistency *p, float *O,
                                            float *wc_opt, uint8_t *mask_opt, void *cuda_stream) {
    if (!It || !Pt || !Ip || !Pp || !Op || !Fb || !Ff || !In || !Pn || !Fn || !Fnb || !p || !O || h < 1 || w < 1 ||
        fh < 1 || fw < 1 || scale < 1 || (scale & (scale - 1)) != 0 || (size_t)fh * scale < (size_t)h ||
        (size_t)fw * scale < (size_t)w || (size_t)h * w > (size_t)INT_MAX || (size_t)fh * fw > (size_t)INT_MAX)
        return fail(nullptr, TC_ERR_INVALID_ARG, "tc_op_consistency_next: bad argument");
    std::string why;
    if (!valid_params(p, why)) return fail(nullptr, TC_ERR_INVALID_ARG, why);
    if (!(p->k1 + p->k2 < 1.f)) return fail(nullptr, TC_ERR_INVALID_ARG, "with the next-frame term k1 + k2 must be < 1");
    ConsistArgs ca{};
    const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    TmpAlloc tmp;
    const size_t hw = (size_t)h * w;
    float4 *A, *B;
    float *C;
    OP_TRY(tmp.get((void **)&A, hw * sizeof(float4)), "tc_op_consistency_next alloc");
    OP_TRY(tmp.get((void **)&B, hw * sizeof(float4)), "tc_op_consistency_next alloc");
    OP_TRY(tmp.get((void **)&C, hw * sizeof(float)), "tc_op_consistency_next alloc");
    OP_TRY(launch_pack_state(Ip, Pp, Op, hw, A, B, C, st), "tc_op_consistency_next pack");
    ca.It = It; ca.Pt = Pt; ca.pA = A; ca.pB = ca.oB = B; ca.pC = C; ca.Fb = Fb; ca.Ff = Ff;
    ca.In = In; ca.Pn = Pn; ca.Fn = Fn; ca.Fnb = Fnb; ca.next = 1; ca.k2 = p->k2;
    ca.H = h; ca.W = w; ca.fh = fh; ca.fw = fw; ca.scale = scale;
    ca.k1 = p->k1; ca.alpha = p->alpha; ca.lambda = p->lambda; ca.c1 = p->fb_c1; ca.c2 = p->fb_c2;
    ca.fb_check = p->fb_check; ca.first = 0;
    ca.O = O; ca.wc = wc_opt; ca.mask = mask_opt;
    OP_TRY(launch_consistency(ca, st), "tc_op_consistency_next launch");
    OP_TRY(cudaStreamSynchronize(st), "tc_op_consistency_next synchronize");  // before the temporaries go
    return TC_OK;
}
