// Multi-stream server: many concurrent video streams (Sec. 3.1: one state per stream, O(1)
// in the stream length) of mixed resolutions on one GPU.
//
//   * Admission: tc_server_open reserves a stream slot and the device memory the stream will
//     hold (computed from the same buffer sizes the stream allocates); it answers
//     TC_ERR_BUSY when the slots or the HBM budget are used up, and succeeds again once a
//     stream has been closed.
//   * Continuous batching: a pool of worker threads takes, whenever a worker is free, the
//     oldest submitted frame of any stream whose previous frame has finished, and runs it
//     through tc_process_frame_host on that stream's own CUDA stream (one CUDA-graph replay
//     per frame from its third frame on).  Frames that arrive while others are on the GPU
//     start as soon as a worker frees up, and the work of different streams overlaps on the
//     device; a stream's own frames stay in order.
//   * Completions carry the time spent queued, on the GPU and in total (submit to done).
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/tc_stream.h"
#include "engine_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    const float *I;
    const float *P;
    float *O;
    unsigned long long tag;
    long long frame;
    double t_submit;
};

struct Slot {
    int id = 0, W = 0, H = 0;
    size_t bytes = 0;
    tc_stream *s = nullptr;      // NULL while the stream is being created
    cudaStream_t cs = nullptr;
    std::deque<Request> q;
    bool busy = false, closing = false;
    long long next_frame = 0;
    tc_consistency params{};
    bool params_dirty = false;
};

}  // namespace

struct tc_server {
    tc_server_desc desc{};
    std::vector<uint8_t> blob;
    tc::HostNet net;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::map<int, Slot *> slots;
    int next_id = 1;
    size_t bytes_used = 0;
    std::deque<tc_completion> done;
    std::vector<std::thread> workers;
    bool stop = false;
    Clock::time_point t0 = Clock::now();

    double now_us() const { return std::chrono::duration<double, std::micro>(Clock::now() - t0).count(); }

    // Oldest pending frame among the streams that are idle (FIFO across streams).
    Slot *pick_ready() {
        Slot *best = nullptr;
        for (auto &kv : slots) {
            Slot *sl = kv.second;
            if (!sl->s || sl->busy || sl->q.empty()) continue;
            if (!best || sl->q.front().t_submit < best->q.front().t_submit) best = sl;
        }
        return best;
    }

    void worker() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            Slot *sl = nullptr;
            cv_work.wait(lk, [&] { return stop || (sl = pick_ready()) != nullptr; });
            if (!sl) break;  // stopping and nothing runnable
            Request rq = sl->q.front();
            sl->q.pop_front();
            sl->busy = true;
            const bool dirty = sl->params_dirty;
            const tc_consistency prm = sl->params;
            sl->params_dirty = false;
            lk.unlock();
            const double t_start = now_us();
            tc_status st = TC_OK;
            if (dirty) st = tc_set_consistency(sl->s, &prm);
            if (st == TC_OK) st = tc_process_frame_host(sl->s, rq.I, rq.P, rq.O, nullptr, nullptr);
            const double t_end = now_us();
            lk.lock();
            sl->busy = false;
            tc_completion c{};
            c.stream_id = sl->id;
            c.frame = rq.frame;
            c.tag = rq.tag;
            c.status = st;
            c.queued_us = t_start - rq.t_submit;
            c.gpu_us = t_end - t_start;
            c.total_us = t_end - rq.t_submit;
            done.push_back(c);
            cv_done.notify_all();
            cv_work.notify_all();
        }
    }
};

static tc_status srv_fail(tc_status code, const std::string &msg) { return tc_record_error(code, msg); }

extern "C" tc_status tc_server_create(const tc_server_desc *desc, tc_server **out) {
    if (out) *out = nullptr;
    if (!desc || !out) return srv_fail(TC_ERR_INVALID_ARG, "tc_server_create: NULL argument");
    if (desc->precision != TC_FP32 && desc->precision != TC_BF16 && desc->precision != TC_FP16)
        return srv_fail(TC_ERR_INVALID_ARG, "tc_server_create: precision must be TC_FP32, TC_BF16 or TC_FP16");
    if (desc->workers < 1 || desc->workers > 64 || desc->max_streams < 1)
        return srv_fail(TC_ERR_INVALID_ARG, "tc_server_create: workers must lie in [1, 64], max_streams >= 1");
    tc_server *srv = new (std::nothrow) tc_server();
    if (!srv) return srv_fail(TC_ERR_OOM, "tc_server_create: host allocation failed");
    srv->desc = *desc;
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
    return tc::stream_device_bytes(srv->net, width, height, srv->desc.precision);
}

extern "C" tc_status tc_server_open(tc_server *srv, int width, int height, int *stream_id) {
    if (!srv || !stream_id) return srv_fail(TC_ERR_INVALID_ARG, "tc_server_open: NULL argument");
    *stream_id = 0;
    const int m = 1 << srv->net.levels;
    if (width < m || height < m || width > 16384 || height > 16384)
        return srv_fail(TC_ERR_INVALID_ARG, "tc_server_open: width and height must lie in [2^levels, 16384]");
    const size_t need = tc::stream_device_bytes(srv->net, width, height, srv->desc.precision);
    Slot *sl = nullptr;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if ((int)srv->slots.size() >= srv->desc.max_streams)
            return srv_fail(TC_ERR_BUSY, "tc_server_open: all stream slots are in use");
        if (srv->desc.hbm_budget_bytes && srv->bytes_used + need > srv->desc.hbm_budget_bytes)
            return srv_fail(TC_ERR_BUSY, "tc_server_open: the stream would exceed the HBM budget (" +
                                             std::to_string(srv->bytes_used + need) + " > " +
                                             std::to_string(srv->desc.hbm_budget_bytes) + " bytes)");
        sl = new Slot();
        sl->id = srv->next_id++;
        sl->W = width;
        sl->H = height;
        sl->bytes = need;
        tc_default_consistency(&sl->params);
        srv->slots[sl->id] = sl;
        srv->bytes_used += need;
    }
    // Create the stream outside the lock (allocation and weight upload take time).
    tc_status st = TC_OK;
    cudaSetDevice(srv->device);
    if (cudaStreamCreateWithFlags(&sl->cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        st = srv_fail(TC_ERR_CUDA, "tc_server_open: cudaStreamCreate failed");
    }
    tc_stream *s = nullptr;
    if (st == TC_OK) {
        tc_stream_desc d{};
        d.width = width;
        d.height = height;
        d.precision = srv->desc.precision;
        d.weights_blob = srv->blob.data();
        d.weights_bytes = srv->blob.size();
        st = tc_create_stream(&d, sl->cs, &s);
    }
    std::lock_guard<std::mutex> lk(srv->mu);
    if (st != TC_OK) {
        srv->slots.erase(sl->id);
        srv->bytes_used -= need;
        if (sl->cs) cudaStreamDestroy(sl->cs);
        delete sl;
        return st;
    }
    sl->s = s;
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

extern "C" tc_status tc_server_submit(tc_server *srv, int stream_id, const float *I_host, const float *P_host,
                                      float *O_host, unsigned long long tag) {
    if (!srv || !I_host || !P_host || !O_host) return srv_fail(TC_ERR_INVALID_ARG, "tc_server_submit: NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->slots.find(stream_id);
    if (it == srv->slots.end() || !it->second->s)
        return srv_fail(TC_ERR_INVALID_ARG, "tc_server_submit: unknown stream");
    Slot *sl = it->second;
    if (sl->closing) return srv_fail(TC_ERR_STATE, "tc_server_submit: stream is closing");
    sl->q.push_back(Request{I_host, P_host, O_host, tag, sl->next_frame++, srv->now_us()});
    srv->cv_work.notify_one();
    return TC_OK;
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
    Slot *sl = nullptr;
    {
        std::unique_lock<std::mutex> lk(srv->mu);
        auto it = srv->slots.find(stream_id);
        if (it == srv->slots.end() || !it->second->s) return srv_fail(TC_ERR_INVALID_ARG, "tc_server_close: unknown stream");
        sl = it->second;
        sl->closing = true;
        srv->cv_done.wait(lk, [&] { return sl->q.empty() && !sl->busy; });
        srv->slots.erase(it);
        srv->bytes_used -= sl->bytes;
    }
    tc_status st = tc_destroy(sl->s);
    cudaStreamDestroy(sl->cs);
    delete sl;
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->cv_work.notify_all();
    return st;
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
    for (auto &kv : srv->slots) {
        if (kv.second->s) tc_destroy(kv.second->s);
        if (kv.second->cs) cudaStreamDestroy(kv.second->cs);
        delete kv.second;
    }
    delete srv;
    return TC_OK;
}
