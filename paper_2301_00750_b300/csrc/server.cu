// Multi-stream server: many concurrent video streams (Sec. 3.1: one state per stream, O(1)
// in the stream length) of mixed resolutions on one GPU.
//
//   * Groups: streams of the same resolution share a batch (tc_create_batch) of
//     desc.batch_lanes lanes, one lane per stream; a group is created (device memory
//     reserved against the HBM budget) when a stream finds no free lane of its size, and
//     destroyed when its last stream closes.  tc_server_open answers TC_ERR_BUSY when the
//     slots or the budget are used up, and succeeds again once streams have closed.
//   * Continuous batching: a pool of worker threads takes, whenever a worker is free, the
//     group holding the oldest submitted frame among idle groups, and runs the oldest queued
//     frame of every lane of that group that has one as one batched step: uploads to the
//     group's device staging, tc_process_lanes (the pyramids and flow estimations of those
//     lanes in shared launches, one CUDA graph per lane range), downloads.  Lanes far apart
//     run as separate runs of the step so that idle lanes between them are not computed.
//     Frames that arrive while a group is on the GPU join its next step; different groups
//     run at the same time on their own CUDA streams; a stream's frames stay in order.
//   * Completions carry the time spent queued, on the GPU and in total (submit to done), and
//     how many frames their step ran.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/tc_stream.h"
#include "common.cuh"
#include "engine_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    const void *I;  // float32 planar, or RGB8 interleaved when rgb8
    const void *P;
    void *O;
    unsigned long long tag;
    long long frame;
    double t_submit;
    bool rgb8 = false;
};

struct Group;

struct Slot {
    int id = 0, W = 0, H = 0;
    Group *g = nullptr;
    int lane = -1;
    std::deque<Request> q;
    bool busy = false, closing = false;
    long long next_frame = 0;
    tc_consistency params{};
    bool params_dirty = true;  // applied by the worker before the lane's next frame
    bool reset = true;         // the lane starts a new stream at its next frame
};

struct Group {
    int W = 0, H = 0, lanes = 0;
    size_t bytes = 0;
    tc_stream *b = nullptr;  // NULL while being created
    cudaStream_t cs = nullptr;
    float *stage = nullptr;  // device staging [3][lanes][3][H][W]: I, P, O
    uint8_t *stage8 = nullptr;  // 8-bit frames: [3][lanes][H][W][3] RGB8 I, P, O
    std::vector<Slot *> lane_slot;  // NULL = free lane
    bool busy = false;
    int open_slots() const {
        int n = 0;
        for (Slot *s : lane_slot) n += s != nullptr;
        return n;
    }
};

}  // namespace

struct tc_server {
    tc_server_desc desc{};
    std::vector<uint8_t> blob;
    tc::HostNet net;
    int device = 0;
    int lanes = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::map<int, Slot *> slots;
    std::vector<Group *> groups;
    int next_id = 1;
    size_t bytes_used = 0;
    std::deque<tc_completion> done;
    std::vector<std::thread> workers;
    bool stop = false;
    Clock::time_point t0 = Clock::now();

    double now_us() const { return std::chrono::duration<double, std::micro>(Clock::now() - t0).count(); }

    size_t group_bytes(int W, int H) const {
        const size_t img = (size_t)3 * W * H * sizeof(float), img8 = (size_t)3 * W * H;
        return tc::stream_device_bytes(net, W, H, desc.precision, 1, lanes) + ((3 * lanes * img + 511) & ~(size_t)511) +
               ((3 * lanes * img8 + 511) & ~(size_t)511);
    }

    // The idle group holding the oldest queued frame (FIFO across groups).
    Group *pick_ready() {
        Group *best = nullptr;
        double best_t = 0;
        for (Group *g : groups) {
            if (!g->b || g->busy) continue;
            for (Slot *s : g->lane_slot)
                if (s && !s->q.empty() && (!best || s->q.front().t_submit < best_t)) {
                    best = g;
                    best_t = s->q.front().t_submit;
                }
        }
        return best;
    }

    void worker() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            Group *g = nullptr;
            cv_work.wait(lk, [&] { return stop || (g = pick_ready()) != nullptr; });
            if (!g) break;  // stopping and nothing runnable
            struct Item {
                Slot *s;
                Request rq;
                bool reset, dirty;
                tc_consistency prm;
            };
            std::vector<Item> items;
            for (int l = 0; l < g->lanes; ++l) {
                Slot *s = g->lane_slot[l];
                if (!s || s->q.empty()) continue;
                items.push_back(Item{s, s->q.front(), s->reset, s->params_dirty, s->params});
                s->q.pop_front();
                s->busy = true;
                s->reset = false;
                s->params_dirty = false;
            }
            g->busy = true;
            lk.unlock();
            const double t_start = now_us();
            const tc_status st = run_step(g, items);
            const double t_end = now_us();
            lk.lock();
            g->busy = false;
            for (const Item &it : items) {
                it.s->busy = false;
                tc_completion c{};
                c.stream_id = it.s->id;
                c.frame = it.rq.frame;
                c.tag = it.rq.tag;
                c.status = st;
                c.queued_us = t_start - it.rq.t_submit;
                c.gpu_us = t_end - t_start;
                c.total_us = t_end - it.rq.t_submit;
                c.batch = (int)items.size();
                done.push_back(c);
            }
            cv_done.notify_all();
            cv_work.notify_all();
        }
    }

    // One batched step of a group (no lock held): every item's lane gets its frame.
    template <typename Item>
    tc_status run_step(Group *g, const std::vector<Item> &items) {
        const size_t img = (size_t)3 * g->W * g->H, plane = (size_t)g->W * g->H;
        float *dI = g->stage, *dP = g->stage + g->lanes * img, *dO = g->stage + 2 * g->lanes * img;
        uint8_t *bI = g->stage8, *bP = g->stage8 + g->lanes * img, *bO = g->stage8 + 2 * g->lanes * img;
        tc_status st = TC_OK;
        for (const Item &it : items) {
            const int l = it.s->lane;
            if (st == TC_OK && it.reset) st = tc_reset_lane(g->b, l);
            if (st == TC_OK && it.dirty) st = tc_set_lane_consistency(g->b, l, &it.prm);
            if (st != TC_OK) continue;
            cudaError_t e;
            if (it.rq.rgb8) {
                // 8-bit frames: upload the codes, decode them into the lane's float staging
                e = cudaMemcpyAsync(bI + l * img, it.rq.I, img, cudaMemcpyHostToDevice, g->cs);
                if (e == cudaSuccess) e = cudaMemcpyAsync(bP + l * img, it.rq.P, img, cudaMemcpyHostToDevice, g->cs);
                if (e == cudaSuccess) e = tc::launch_unpack_rgb8(bI + l * img, plane, dI + l * img, g->cs);
                if (e == cudaSuccess) e = tc::launch_unpack_rgb8(bP + l * img, plane, dP + l * img, g->cs);
            } else {
                e = cudaMemcpyAsync(dI + l * img, it.rq.I, img * sizeof(float), cudaMemcpyHostToDevice, g->cs);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(dP + l * img, it.rq.P, img * sizeof(float), cudaMemcpyHostToDevice, g->cs);
            }
            if (e != cudaSuccess) {
                cudaGetLastError();
                st = tc_record_error(TC_ERR_CUDA, "server: upload failed");
            }
        }
        // Lanes in ascending order, split into runs that skip more than one idle lane: each
        // run is one tc_process_lanes call, whose shared launches cover lanes lo .. hi.
        std::vector<int> ls;
        for (const Item &it : items) ls.push_back(it.s->lane);
        std::sort(ls.begin(), ls.end());
        size_t k0 = 0;
        while (st == TC_OK && k0 < ls.size()) {
            size_t k1 = k0 + 1;
            while (k1 < ls.size() && ls[k1] - ls[k1 - 1] <= 2) ++k1;
            std::vector<const float *> I, P;
            std::vector<float *> O;
            for (size_t k = k0; k < k1; ++k) {
                I.push_back(dI + ls[k] * img);
                P.push_back(dP + ls[k] * img);
                O.push_back(dO + ls[k] * img);
            }
            st = tc_process_lanes(g->b, (int)(k1 - k0), ls.data() + k0, I.data(), P.data(), O.data(), nullptr, nullptr);
            k0 = k1;
        }
        for (const Item &it : items) {
            if (st != TC_OK) break;
            const int l = it.s->lane;
            cudaError_t e;
            if (it.rq.rgb8) {
                e = tc::launch_pack_rgb8(dO + l * img, plane, bO + l * img, g->cs);
                if (e == cudaSuccess) e = cudaMemcpyAsync(it.rq.O, bO + l * img, img, cudaMemcpyDeviceToHost, g->cs);
            } else {
                e = cudaMemcpyAsync(it.rq.O, dO + l * img, img * sizeof(float), cudaMemcpyDeviceToHost, g->cs);
            }
            if (e != cudaSuccess) {
                cudaGetLastError();
                st = tc_record_error(TC_ERR_CUDA, "server: download failed");
            }
        }
        const tc_status ss = tc_synchronize(g->b);
        return st != TC_OK ? st : ss;
    }
};

static tc_status srv_fail(tc_status code, const std::string &msg) { return tc_record_error(code, msg); }

static void destroy_group(Group *g) {
    if (g->b) tc_destroy(g->b);
    if (g->stage) cudaFree(g->stage);
    if (g->stage8) cudaFree(g->stage8);
    if (g->cs) cudaStreamDestroy(g->cs);
    delete g;
}

extern "C" tc_status tc_server_create(const tc_server_desc *desc, tc_server **out) {
    if (out) *out = nullptr;
    if (!desc || !out) return srv_fail(TC_ERR_INVALID_ARG, "tc_server_create: NULL argument");
    if (desc->precision != TC_FP32 && desc->precision != TC_BF16 && desc->precision != TC_FP16)
        return srv_fail(TC_ERR_INVALID_ARG, "tc_server_create: precision must be TC_FP32, TC_BF16 or TC_FP16");
    if (desc->workers < 1 || desc->workers > 64 || desc->max_streams < 1 || desc->batch_lanes < 0 ||
        desc->batch_lanes > 64)
        return srv_fail(TC_ERR_INVALID_ARG,
                        "tc_server_create: workers must lie in [1, 64], max_streams >= 1, batch_lanes in [0, 64]");
    tc_server *srv = new (std::nothrow) tc_server();
    if (!srv) return srv_fail(TC_ERR_OOM, "tc_server_create: host allocation failed");
    srv->desc = *desc;
    srv->lanes = desc->batch_lanes > 1 ? desc->batch_lanes : 1;
    if (desc->weights_path) {
        FILE *f = fopen(desc->weights_path, "rb");
        if (!f) {
            delete srv;
            return srv_fail(TC_ERR_IO, std::string("cannot open weights file ") + desc->weights_path);
        }
        fseek(f, 0, SEEK_END);
        const long n = ftell(f);
        fseek(f, 0, SEEK_SET);
        srv->blob.resize(n > 0 ? (size_t)n : 0);
        const size_t got = n > 0 ? fread(srv->blob.data(), 1, (size_t)n, f) : 0;
        fclose(f);
        if (got != srv->blob.size()) {
            delete srv;
            return srv_fail(TC_ERR_IO, "short read of the weights file");
        }
    } else if (desc->weights_blob && desc->weights_bytes) {
        const uint8_t *b = static_cast<const uint8_t *>(desc->weights_blob);
        srv->blob.assign(b, b + desc->weights_bytes);
    } else {
        delete srv;
        return srv_fail(TC_ERR_INVALID_ARG, "tc_server_create: no weights given");
    }
    std::string err;
    if (!tc::parse_weights(srv->blob.data(), srv->blob.size(), srv->net, err)) {
        delete srv;
        return srv_fail(TC_ERR_IO, err);
    }
    if (!srv->net.ref.empty()) {
        delete srv;
        return srv_fail(TC_ERR_UNSUPPORTED, "tc_server_create: served streams run without the refinement network");
    }
    srv->desc.weights_path = nullptr;
    srv->desc.weights_blob = nullptr;
    if (cudaGetDevice(&srv->device) != cudaSuccess) {
        cudaGetLastError();
        srv->device = 0;
    }
    for (int i = 0; i < desc->workers; ++i) srv->workers.emplace_back([srv] { srv->worker(); });
    *out = srv;
    return TC_OK;
}

extern "C" size_t tc_server_stream_bytes(const tc_server *srv, int width, int height) {
    if (!srv || width < 1 || height < 1) return 0;
    return srv->group_bytes(width, height);
}

extern "C" tc_status tc_server_open(tc_server *srv, int width, int height, int *stream_id) {
    if (!srv || !stream_id) return srv_fail(TC_ERR_INVALID_ARG, "tc_server_open: NULL argument");
    *stream_id = 0;
    const int m = 1 << srv->net.levels;
    if (width < m || height < m || width > 16384 || height > 16384)
        return srv_fail(TC_ERR_INVALID_ARG, "tc_server_open: width and height must lie in [2^levels, 16384]");
    Slot *sl = nullptr;
    Group *fresh = nullptr;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if ((int)srv->slots.size() >= srv->desc.max_streams)
            return srv_fail(TC_ERR_BUSY, "tc_server_open: all stream slots are in use");
        Group *g = nullptr;
        int lane = -1;
        for (Group *c : srv->groups) {
            if (c->W != width || c->H != height || !c->b) continue;  // (a group being created is skipped)
            for (int l = 0; l < c->lanes && lane < 0; ++l)
                if (!c->lane_slot[l]) lane = l;
            if (lane >= 0) {
                g = c;
                break;
            }
        }
        if (!g) {
            const size_t need = srv->group_bytes(width, height);
            if (srv->desc.hbm_budget_bytes && srv->bytes_used + need > srv->desc.hbm_budget_bytes)
                return srv_fail(TC_ERR_BUSY, "tc_server_open: the stream would exceed the HBM budget (" +
                                                 std::to_string(srv->bytes_used + need) + " > " +
                                                 std::to_string(srv->desc.hbm_budget_bytes) + " bytes)");
            g = fresh = new Group();
            g->W = width;
            g->H = height;
            g->lanes = srv->lanes;
            g->bytes = need;
            g->lane_slot.assign(g->lanes, nullptr);
            srv->groups.push_back(g);
            srv->bytes_used += need;
            lane = 0;
        }
        sl = new Slot();
        sl->id = srv->next_id++;
        sl->W = width;
        sl->H = height;
        sl->g = g;
        sl->lane = lane;
        tc_default_consistency(&sl->params);
        g->lane_slot[lane] = sl;
        srv->slots[sl->id] = sl;
    }
    if (fresh) {
        // Create the batch outside the lock (allocation and weight upload take time); until
        // then the group is not picked (b == NULL).
        tc_status st = TC_OK;
        cudaSetDevice(srv->device);
        if (cudaStreamCreateWithFlags(&fresh->cs, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            st = srv_fail(TC_ERR_CUDA, "tc_server_open: cudaStreamCreate failed");
        }
        const size_t img = (size_t)3 * width * height * sizeof(float);
        if (st == TC_OK && cudaMalloc(&fresh->stage, 3 * fresh->lanes * img) != cudaSuccess) {
            cudaGetLastError();
            fresh->stage = nullptr;
            st = srv_fail(TC_ERR_OOM, "tc_server_open: staging allocation failed");
        }
        if (st == TC_OK && cudaMalloc(&fresh->stage8, 3 * fresh->lanes * (img / sizeof(float))) != cudaSuccess) {
            cudaGetLastError();
            fresh->stage8 = nullptr;
            st = srv_fail(TC_ERR_OOM, "tc_server_open: staging allocation failed");
        }
        tc_stream *b = nullptr;
        if (st == TC_OK) {
            tc_stream_desc d{};
            d.width = width;
            d.height = height;
            d.precision = srv->desc.precision;
            d.weights_blob = srv->blob.data();
            d.weights_bytes = srv->blob.size();
            st = tc_create_batch(&d, fresh->lanes, fresh->cs, &b);
        }
        std::lock_guard<std::mutex> lk(srv->mu);
        if (st != TC_OK) {
            // no other stream joins a group being created, so only this slot goes with it
            srv->slots.erase(sl->id);
            delete sl;
            srv->groups.erase(std::find(srv->groups.begin(), srv->groups.end(), fresh));
            srv->bytes_used -= fresh->bytes;
            destroy_group(fresh);
            return st;
        }
        fresh->b = b;
    }
    std::lock_guard<std::mutex> lk(srv->mu);
    *stream_id = sl->id;
    srv->cv_work.notify_all();
    return TC_OK;
}

extern "C" tc_status tc_server_set_consistency(tc_server *srv, int stream_id, const tc_consistency *p) {
    if (!srv || !p) return srv_fail(TC_ERR_INVALID_ARG, "tc_server_set_consistency: NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->slots.find(stream_id);
    if (it == srv->slots.end()) return srv_fail(TC_ERR_INVALID_ARG, "tc_server_set_consistency: unknown stream");
    if (p->solver_iters != 0)
        // the admission charge covers the causal path; the solver's buffers are not budgeted
        return srv_fail(TC_ERR_UNSUPPORTED, "tc_server_set_consistency: served streams run without the solver");
    it->second->params = *p;
    it->second->params_dirty = true;
    return TC_OK;
}

static tc_status submit(tc_server *srv, int stream_id, const void *I_host, const void *P_host, void *O_host,
                        unsigned long long tag, bool rgb8, const char *fn) {
    if (!srv || !I_host || !P_host || !O_host) return srv_fail(TC_ERR_INVALID_ARG, std::string(fn) + ": NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->slots.find(stream_id);
    if (it == srv->slots.end() || !it->second->g->b)
        return srv_fail(TC_ERR_INVALID_ARG, std::string(fn) + ": unknown stream");
    Slot *sl = it->second;
    if (sl->closing) return srv_fail(TC_ERR_STATE, std::string(fn) + ": stream is closing");
    sl->q.push_back(Request{I_host, P_host, O_host, tag, sl->next_frame++, srv->now_us(), rgb8});
    srv->cv_work.notify_one();
    return TC_OK;
}

extern "C" tc_status tc_server_submit(tc_server *srv, int stream_id, const float *I_host, const float *P_host,
                                      float *O_host, unsigned long long tag) {
    return submit(srv, stream_id, I_host, P_host, O_host, tag, false, "tc_server_submit");
}

extern "C" tc_status tc_server_submit_rgb8(tc_server *srv, int stream_id, const uint8_t *I_host, const uint8_t *P_host,
                                           uint8_t *O_host, unsigned long long tag) {
    return submit(srv, stream_id, I_host, P_host, O_host, tag, true, "tc_server_submit_rgb8");
}

extern "C" int tc_server_poll(tc_server *srv, tc_completion *out, int max, int timeout_ms) {
    if (!srv || !out || max < 1) return 0;
    std::unique_lock<std::mutex> lk(srv->mu);
    if (srv->done.empty() && timeout_ms > 0)
        srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return !srv->done.empty(); });
    int n = 0;
    while (n < max && !srv->done.empty()) {
        out[n++] = srv->done.front();
        srv->done.pop_front();
    }
    return n;
}

// Drops the frames of `sl` still queued; each becomes a completion with TC_ERR_STATE.
static void cancel_locked(tc_server *srv, Slot *sl) {
    const double t = srv->now_us();
    for (const Request &rq : sl->q) {
        tc_completion c{};
        c.stream_id = sl->id;
        c.frame = rq.frame;
        c.tag = rq.tag;
        c.status = TC_ERR_STATE;
        c.queued_us = c.total_us = t - rq.t_submit;
        srv->done.push_back(c);
    }
    sl->q.clear();
    srv->cv_done.notify_all();
}

extern "C" tc_status tc_server_cancel(tc_server *srv, int stream_id) {
    if (!srv) return srv_fail(TC_ERR_INVALID_ARG, "tc_server_cancel: NULL server");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->slots.find(stream_id);
    if (it == srv->slots.end()) return srv_fail(TC_ERR_INVALID_ARG, "tc_server_cancel: unknown stream");
    cancel_locked(srv, it->second);
    return TC_OK;
}

extern "C" tc_status tc_server_close(tc_server *srv, int stream_id) {
    if (!srv) return srv_fail(TC_ERR_INVALID_ARG, "tc_server_close: NULL server");
    Group *dead = nullptr;
    {
        std::unique_lock<std::mutex> lk(srv->mu);
        auto it = srv->slots.find(stream_id);
        if (it == srv->slots.end() || !it->second->g->b)
            return srv_fail(TC_ERR_INVALID_ARG, "tc_server_close: unknown stream");
        Slot *sl = it->second;
        sl->closing = true;
        srv->cv_done.wait(lk, [&] { return sl->q.empty() && !sl->busy; });
        Group *g = sl->g;
        srv->slots.erase(sl->id);
        g->lane_slot[sl->lane] = nullptr;
        delete sl;
        if (g->open_slots() == 0) {
            // the group's last stream: free its memory (no step of it can be running: every
            // lane's frames are done)
            srv->cv_done.wait(lk, [&] { return !g->busy; });
            srv->groups.erase(std::find(srv->groups.begin(), srv->groups.end(), g));
            srv->bytes_used -= g->bytes;
            dead = g;
        }
        srv->cv_work.notify_all();
    }
    if (dead) destroy_group(dead);
    return TC_OK;
}

extern "C" size_t tc_server_bytes_in_use(const tc_server *srv) {
    if (!srv) return 0;
    std::lock_guard<std::mutex> lk(const_cast<tc_server *>(srv)->mu);
    return srv->bytes_used;
}

extern "C" tc_status tc_server_destroy(tc_server *srv) {
    if (!srv) return srv_fail(TC_ERR_INVALID_ARG, "tc_server_destroy: NULL server");
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        for (auto &kv : srv->slots) cancel_locked(srv, kv.second);
        srv->stop = true;
        srv->cv_work.notify_all();
    }
    for (auto &t : srv->workers) t.join();
    for (auto &kv : srv->slots) delete kv.second;
    for (Group *g : srv->groups) destroy_group(g);
    delete srv;
    return TC_OK;
}
