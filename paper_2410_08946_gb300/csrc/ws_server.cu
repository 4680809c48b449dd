// ws_server.cu -- the request loop of libws (ws_server_create / ws_submit /
// ws_poll / ws_cancel / ws_server_destroy): continuous batching of
// partitioning requests over several lanes (context + stream each), with
// admission by a device-memory budget and resident staging buffers.
//
// Scheduling: one host thread.  A lane is free when its previous batch has
// completed (signalled by a host function enqueued on the lane's stream).
// For a free lane the scheduler takes the oldest queued request and every
// later queued request with the same dtype, connectivity, dimensionality and
// NL, up to max_batch and the lane's memory share, and enqueues them as one
// ws_segment_batch: host inputs are copied into the lane's staging buffers,
// outputs are copied back after the batch, all on the lane's stream.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ws_internal.h"

namespace {

enum ReqState { Q_QUEUED, Q_RUNNING, Q_DONE };

struct Req {
    ws_request r;
    size_t N = 0;
    size_t est = 0;  // device bytes the request needs in a lane (admission estimate)
    ReqState state = Q_QUEUED;
    ws_status result = WS_OK;
};

struct Lane {
    ws_context *ctx = nullptr;
    cudaStream_t stream = nullptr;
    bool busy = false;
    bool finished = false;  // set by the host function at the end of the batch
    std::vector<uint64_t> ids;
    uint8_t *grad_stage = nullptr;
    size_t grad_cap = 0;
    int32_t *out_stage = nullptr;
    size_t out_cap = 0;  // int32 elements
    int32_t *cnt_stage = nullptr;
    size_t cnt_cap = 0;
};

size_t pixels_of(const ws_shape &s)
{
    int64_t n = s.dims[0] * s.dims[1] * (s.ndim == 3 ? s.dims[2] : 1);
    return n > 0 ? (size_t)n : 0;
}

// Device bytes a request occupies in a lane, an upper bound whose sum over a
// batch bounds the batch: workspace (per-pixel and per-tile arrays, region
// table and graph, as the context sizes them) plus staging of host inputs and
// outputs (with their growth margin).
size_t estimate(const ws_request &r, size_t N)
{
    const int64_t W = r.shape.dims[0], H = r.shape.dims[1], D = r.shape.ndim == 3 ? r.shape.dims[2] : 1;
    // tiles: at least 32 x 16 (x 16) pixels each, so this counts them from above
    const size_t tiles = (size_t)((W + 31) / 32) * (size_t)((H + 15) / 16) * (size_t)((D + 15) / 16);
    size_t b = ws::workspace_bound(N, tiles, 2, r.connectivity, r.NL, true);
    if (r.on_host) b += (N * (r.dtype == WS_U8 ? 1 : 2) + 256 + N * 4 * (size_t)r.NL) * 3 / 2;
    return b;
}

bool compatible(const ws_request &a, const ws_request &b)
{
    return a.dtype == b.dtype && a.connectivity == b.connectivity && a.shape.ndim == b.shape.ndim && a.NL == b.NL &&
           a.on_host == b.on_host;
}

}  // namespace

struct ws_server {
    int device = 0;
    size_t lane_budget = 0;  // 0 = unbounded
    int max_batch = 64;
    std::vector<Lane> lanes;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Req> reqs;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread th;
};

namespace {

struct LaneDone {
    ws_server *s;
    int lane;
};

void CUDART_CB lane_done(void *arg)
{
    LaneDone *d = (LaneDone *)arg;
    {
        std::lock_guard<std::mutex> lk(d->s->mu);
        d->s->lanes[d->lane].finished = true;
    }
    d->s->cv_work.notify_one();
    delete d;
}

template <typename P> bool grow(P **p, size_t &cap, size_t need)
{
    if (need <= cap) return true;
    size_t n = need + need / 2;
    if (*p) cudaFree(*p);
    *p = nullptr;
    cap = 0;
    if (cudaMalloc((void **)p, n * sizeof(P)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cap = n;
    return true;
}

// Enqueues one batch on a lane (called without the server lock held).
ws_status launch_batch(ws_server *s, int li, std::vector<Req *> &batch)
{
    Lane &L = s->lanes[li];
    const ws_request &h = batch[0]->r;
    const bool host = h.on_host != 0;
    const size_t b = h.dtype == WS_U8 ? 1 : 2;
    size_t gtot = 0, otot = 0;
    for (Req *q : batch) {
        gtot += (q->N * b + 255) & ~(size_t)255;
        otot += q->N * (size_t)h.NL;
    }
    if (host && (!grow(&L.grad_stage, L.grad_cap, gtot) || !grow(&L.out_stage, L.out_cap, otot) ||
                 !grow(&L.cnt_stage, L.cnt_cap, (size_t)h.NL * batch.size())))
        return WS_ERR_OOM;
    std::vector<ws_item> items(batch.size());
    size_t go = 0, oo = 0;
    for (size_t i = 0; i < batch.size(); i++) {
        const ws_request &r = batch[i]->r;
        items[i].shape = r.shape;
        if (host) {
            cudaMemcpyAsync(L.grad_stage + go, r.grad, batch[i]->N * b, cudaMemcpyHostToDevice, L.stream);
            items[i].grad_d = L.grad_stage + go;
            items[i].levels_d = L.out_stage + oo;
            items[i].counts_d = L.cnt_stage + (size_t)h.NL * i;
            go += (batch[i]->N * b + 255) & ~(size_t)255;
            oo += batch[i]->N * (size_t)h.NL;
        } else {
            items[i].grad_d = r.grad;
            items[i].levels_d = r.levels;
            items[i].counts_d = r.counts;
        }
    }
    ws_status st = ws_segment_batch(L.ctx, (int)batch.size(), items.data(), h.dtype, h.connectivity, h.NL,
                                    (ws_stream_t)L.stream);
    if (st == WS_ERR_OOM) {
        // the batch fits the lane's share (admission), but arrays kept from
        // earlier batches may not leave room for it: start from an empty
        // workspace once
        cudaStreamSynchronize(L.stream);
        ws::release_workspace(L.ctx);
        st = ws_segment_batch(L.ctx, (int)batch.size(), items.data(), h.dtype, h.connectivity, h.NL,
                              (ws_stream_t)L.stream);
    }
    if (st != WS_OK) return st;
    if (host) {
        for (size_t i = 0; i < batch.size(); i++) {
            const ws_request &r = batch[i]->r;
            cudaMemcpyAsync(r.levels, items[i].levels_d, batch[i]->N * (size_t)h.NL * 4, cudaMemcpyDeviceToHost,
                            L.stream);
            if (r.counts)
                cudaMemcpyAsync(r.counts, items[i].counts_d, (size_t)h.NL * 4, cudaMemcpyDeviceToHost, L.stream);
        }
    }
    LaneDone *d = new LaneDone{s, li};
    cudaError_t e = cudaLaunchHostFunc(L.stream, lane_done, d);
    if (e != cudaSuccess) {
        delete d;
        cudaGetLastError();
        return WS_ERR_CUDA;
    }
    return WS_OK;
}

void scheduler(ws_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // completions
        for (size_t li = 0; li < s->lanes.size(); li++) {
            Lane &L = s->lanes[li];
            if (!L.busy || !L.finished) continue;
            lk.unlock();
            ws_status st = ws_context_check(L.ctx, (ws_stream_t)L.stream);  // the stream is already idle
            lk.lock();
            for (uint64_t id : L.ids) {
                auto it = s->reqs.find(id);
                if (it == s->reqs.end()) continue;
                it->second.state = Q_DONE;
                it->second.result = st;
            }
            L.ids.clear();
            L.busy = false;
            L.finished = false;
            s->cv_done.notify_all();
        }
        // dispatch queued requests to free lanes
        for (size_t li = 0; li < s->lanes.size() && !s->queue.empty(); li++) {
            Lane &L = s->lanes[li];
            if (L.busy) continue;
            std::vector<Req *> batch;
            std::vector<uint64_t> ids;
            size_t bytes = 0;
            const ws_request head = s->reqs[s->queue.front()].r;
            for (auto it = s->queue.begin(); it != s->queue.end() && (int)batch.size() < s->max_batch;) {
                Req &q = s->reqs[*it];
                if (!compatible(head, q.r) ||
                    (s->lane_budget && !batch.empty() && bytes + q.est > s->lane_budget)) {
                    ++it;
                    continue;
                }
                bytes += q.est;
                q.state = Q_RUNNING;
                batch.push_back(&q);
                ids.push_back(*it);
                it = s->queue.erase(it);
            }
            L.busy = true;
            L.finished = false;
            L.ids = ids;
            lk.unlock();
            ws_status st = launch_batch(s, (int)li, batch);
            lk.lock();
            if (st != WS_OK) {  // nothing of the batch will complete: fail its requests now
                for (uint64_t id : ids) {
                    auto it = s->reqs.find(id);
                    if (it == s->reqs.end()) continue;
                    it->second.state = Q_DONE;
                    it->second.result = st;
                }
                cudaStreamSynchronize(L.stream);
                L.ids.clear();
                L.busy = false;
                s->cv_done.notify_all();
            }
        }
        bool any_busy = false;
        for (auto &L : s->lanes) any_busy |= L.busy;
        if (s->stop && !any_busy) break;
        bool any_finished = false;
        for (auto &L : s->lanes) any_finished |= (L.busy && L.finished);
        if (any_finished) continue;
        bool free_lane = false;
        for (auto &L : s->lanes) free_lane |= !L.busy;
        if (!s->queue.empty() && free_lane) continue;
        s->cv_work.wait(lk);
    }
}

}  // namespace

extern "C" {

void ws_server_destroy(ws_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (uint64_t id : s->queue) {
            auto it = s->reqs.find(id);
            if (it != s->reqs.end()) {
                it->second.state = Q_DONE;
                it->second.result = WS_ERR_CANCELLED;
            }
        }
        s->queue.clear();
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
    if (s->th.joinable()) s->th.join();
    cudaSetDevice(s->device);
    for (auto &L : s->lanes) {
        if (L.stream) cudaStreamSynchronize(L.stream);
        if (L.ctx) ws_context_destroy(L.ctx);
        if (L.stream) cudaStreamDestroy(L.stream);
        if (L.grad_stage) cudaFree(L.grad_stage);
        if (L.out_stage) cudaFree(L.out_stage);
        if (L.cnt_stage) cudaFree(L.cnt_stage);
    }
    delete s;
}

ws_status ws_server_create(ws_server **out, int device, size_t budget_bytes, int n_lanes, int max_batch)
{
    if (!out || n_lanes < 1 || n_lanes > 64 || max_batch < 1) return WS_ERR_INVALID;
    *out = nullptr;
    ws_server *s = new (std::nothrow) ws_server();
    if (!s) return WS_ERR_OOM;
    s->device = device;
    s->max_batch = max_batch;
    s->lane_budget = budget_bytes ? budget_bytes / (size_t)n_lanes : 0;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return WS_ERR_CUDA;
    }
    s->lanes.resize((size_t)n_lanes);
    for (auto &L : s->lanes) {
        ws_status st = ws_context_create(&L.ctx, device, s->lane_budget);
        if (st == WS_OK && cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) != cudaSuccess)
            st = WS_ERR_CUDA;
        if (st != WS_OK) {
            ws_server_destroy(s);
            return st;
        }
    }
    s->th = std::thread(scheduler, s);
    *out = s;
    return WS_OK;
}

ws_status ws_submit(ws_server *s, const ws_request *r, uint64_t *ticket)
{
    if (!s || !r || !ticket || !r->grad || !r->levels || r->NL < 1 || r->NL > ws::kMaxLevels) return WS_ERR_INVALID;
    if (r->dtype != WS_U8 && r->dtype != WS_U16) return WS_ERR_INVALID;
    if (r->shape.ndim != 2 && r->shape.ndim != 3) return WS_ERR_INVALID;
    const size_t N = pixels_of(r->shape);
    if (N == 0 || N >= ((size_t)1 << 31)) return WS_ERR_INVALID;
    const bool ok2 = r->shape.ndim == 2 && (r->connectivity == 4 || r->connectivity == 8);
    const bool ok3 = r->shape.ndim == 3 && r->connectivity == 6;
    if (!ok2 && !ok3) return WS_ERR_INVALID;
    Req q;
    q.r = *r;
    q.N = N;
    q.est = estimate(*r, N);
    if (s->lane_budget && q.est > s->lane_budget) return WS_ERR_OOM;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return WS_ERR_CANCELLED;
        const uint64_t id = s->next_id++;
        s->reqs.emplace(id, q);
        s->queue.push_back(id);
        *ticket = id;
    }
    s->cv_work.notify_one();
    return WS_OK;
}

ws_status ws_poll(ws_server *s, uint64_t ticket, int64_t timeout_us)
{
    if (!s) return WS_ERR_INVALID;
    std::unique_lock<std::mutex> lk(s->mu);
    auto done = [&]() {
        auto it = s->reqs.find(ticket);
        return it == s->reqs.end() || it->second.state == Q_DONE;
    };
    if (timeout_us < 0)
        s->cv_done.wait(lk, done);
    else if (timeout_us > 0)
        s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return WS_ERR_INVALID;
    if (it->second.state != Q_DONE) return WS_ERR_NOT_READY;
    const ws_status st = it->second.result;
    s->reqs.erase(it);
    return st;
}

ws_status ws_cancel(ws_server *s, uint64_t ticket)
{
    if (!s) return WS_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return WS_ERR_INVALID;
    if (it->second.state != Q_QUEUED) return it->second.state == Q_DONE ? WS_OK : WS_ERR_NOT_READY;
    for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
        if (*q == ticket) {
            s->queue.erase(q);
            break;
        }
    it->second.state = Q_DONE;
    it->second.result = WS_ERR_CANCELLED;
    s->cv_done.notify_all();
    return WS_OK;
}

}  // extern "C"
