// Serving loop of wt_gb300 (see include/wt_gb300.h, "serving").
//
// Requests are copied to host memory at submit, admitted in arrival order
// while their device footprint (text + bit vectors + Z + workspace of a solo
// build) fits in the remaining HBM budget, and packed into batches whenever a
// stream is idle: up to max_batch admitted requests per launch, one batched
// build per (kind, storage type) present.  Several streams run batches at
// the same time, so requests arriving while others are on the GPU start as
// soon as a stream and memory are free.  Results stay on the device until
// released.  Latency is measured from submit to the host callback that
// follows the batch on its stream.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "wt_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    uint64_t ticket = 0;
    wt_kind kind = WT_TREE;
    wt_symtype type = WT_U8;
    uint64_t n = 0, sigma = 0;
    uint32_t L = 0;
    std::unique_ptr<uint8_t[]> host;  // text copy (freed once on the device)
    const void *src = nullptr;        // host.get(), or the caller's page-locked text
    void *d_text = nullptr;
    uint64_t *d_bv = nullptr;
    uint64_t *d_zeros = nullptr;
    size_t reserved = 0;              // bytes charged to the budget
    size_t ws_alone = 0;
    Clock::time_point t_submit, t_done;
    bool done = false;
    wt_status status = WT_OK;
};

struct Batch;

struct Slot {
    cudaStream_t stream = nullptr;
    uint32_t *h_status = nullptr;     // pinned: device status of each build of the batch
    bool busy = false;
};

struct Batch {
    struct wt_server *srv = nullptr;
    int slot = -1;
    std::vector<std::shared_ptr<Req>> reqs;
    void *d_ws = nullptr;
    size_t ws_bytes = 0;
    wt_status status = WT_OK;
};

}  // namespace

struct wt_server {
    wt_server_config cfg{};
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<std::shared_ptr<Req>> pending;   // submitted, not admitted
    std::deque<std::shared_ptr<Req>> admitted;  // memory reserved, not launched
    std::map<uint64_t, std::shared_ptr<Req>> all;
    std::vector<Slot> slots;
    std::vector<Batch *> finished;              // batches whose callback ran
    size_t in_use = 0;
    uint64_t next_ticket = 1;
    uint64_t submitted = 0, completed = 0, rejected = 0, in_flight = 0;
    uint64_t symbols_done = 0;
    std::vector<double> latencies;
    Clock::time_point t_create;
    bool stop = false;
    std::thread sched;
};

namespace {

size_t footprint(const Req &r)
{
    const uint64_t W = (r.n + 63) / 64;
    size_t b = r.n * (size_t)r.type + r.L * W * 8 + (r.kind == WT_MATRIX ? r.L * 8 + 8 : 0);
    return b + r.ws_alone + 4096;
}

void CUDART_CB on_batch_done(void *p)
{
    Batch *b = static_cast<Batch *>(p);
    wt_server *s = b->srv;
    std::lock_guard<std::mutex> lk(s->mu);
    s->finished.push_back(b);
    s->cv_sched.notify_all();
}

// Launches one batch on its slot's stream.  Called without the lock held.
void launch_batch(wt_server *s, Batch *b)
{
    cudaStream_t st = s->slots[b->slot].stream;
    wt_status status = WT_OK;
    for (auto &r : b->reqs) {
        if (r->n == 0 || r->L == 0) continue;
        if (cudaMallocAsync(&r->d_text, r->n * (size_t)r->type, st) != cudaSuccess ||
            cudaMallocAsync(reinterpret_cast<void **>(&r->d_bv), r->L * ((r->n + 63) / 64) * 8, st) !=
                cudaSuccess) {
            status = WT_ERR_OUT_OF_MEMORY;
            break;
        }
        if (r->kind == WT_MATRIX &&
            cudaMallocAsync(reinterpret_cast<void **>(&r->d_zeros), r->L * 8, st) != cudaSuccess) {
            status = WT_ERR_OUT_OF_MEMORY;
            break;
        }
        if (cudaMemcpyAsync(r->d_text, r->src, r->n * (size_t)r->type, cudaMemcpyHostToDevice, st) !=
            cudaSuccess) {
            status = WT_ERR_CUDA;
            break;
        }
    }
    // one batched build per (kind, type)
    uint32_t *hs = s->slots[b->slot].h_status;
    int nbuild = 0;
    for (int k = 0; k < 8; ++k) hs[k] = 0;
    for (int kind = 0; kind < 2 && status == WT_OK; ++kind) {
        for (int w : {1, 2, 4}) {
            std::vector<wt_text_desc> d;
            for (auto &r : b->reqs)
                if ((int)r->kind == kind && (int)r->type == w && r->n > 0 && r->L > 0)
                    d.push_back(wt_text_desc{r->d_text, r->n, r->sigma, r->d_bv, r->d_zeros});
            if (d.empty()) continue;
            size_t ws = 0;
            status = wt_batched_workspace_size((wt_kind)kind, (wt_symtype)w, d.data(), (uint32_t)d.size(), &ws);
            if (status != WT_OK) break;
            void *p = nullptr;
            if (cudaMallocAsync(&p, ws, st) != cudaSuccess) { status = WT_ERR_OUT_OF_MEMORY; break; }
            status = wt_build_batched((wt_kind)kind, (wt_symtype)w, d.data(), (uint32_t)d.size(), p, ws, st);
            // device-detected errors: the status word sits at the start of the workspace
            if (status == WT_OK && cudaMemcpyAsync(hs + nbuild++, p, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                                   st) != cudaSuccess)
                status = WT_ERR_CUDA;
            cudaFreeAsync(p, st);
            if (status != WT_OK) break;
        }
    }
    b->status = status;
    if (cudaLaunchHostFunc(st, on_batch_done, b) != cudaSuccess) {
        b->status = WT_ERR_CUDA;
        on_batch_done(b);
    }
}

void finish_batch(wt_server *s, Batch *b)   // lock held
{
    const auto now = Clock::now();
    const uint32_t *hs = s->slots[b->slot].h_status;
    for (int k = 0; k < 8 && b->status == WT_OK; ++k)
        if (hs[k] != 0) b->status = static_cast<wt_status>(hs[k]);
    for (auto &r : b->reqs) {
        r->done = true;
        r->status = b->status;
        r->t_done = now;
        r->host.reset();
        r->src = nullptr;
        // the workspace share of the reservation is returned now
        s->in_use -= r->ws_alone;
        r->reserved -= r->ws_alone;
        s->completed++;
        s->in_flight--;
        s->symbols_done += r->n;
        s->latencies.push_back(std::chrono::duration<double, std::micro>(now - r->t_submit).count());
    }
    s->slots[b->slot].busy = false;
    delete b;
    s->cv_done.notify_all();
}

void scheduler(wt_server *s)
{
    cudaSetDevice(s->cfg.device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        for (Batch *b : s->finished) finish_batch(s, b);
        s->finished.clear();
        if (s->stop) {
            // destroy: requests not on a stream yet are dropped (pending ones might
            // never be admitted: finished results keep their memory charged until
            // released); batches already launched run to their callbacks
            for (auto &r : s->admitted) s->in_use -= r->reserved;
            s->admitted.clear();
            s->pending.clear();
            bool idle = true;
            for (auto &sl : s->slots) idle &= !sl.busy;
            if (idle) break;
            s->cv_sched.wait(lk);
            continue;
        }
        // admission in arrival order
        while (!s->pending.empty()) {
            auto &r = s->pending.front();
            if (s->in_use + r->reserved > s->cfg.hbm_budget_bytes) break;
            s->in_use += r->reserved;
            s->admitted.push_back(r);
            s->pending.pop_front();
        }
        // continuous batching onto idle streams
        bool launched = false;
        for (size_t k = 0; k < s->slots.size() && !s->admitted.empty(); ++k) {
            if (s->slots[k].busy) continue;
            Batch *b = new Batch();
            b->srv = s;
            b->slot = (int)k;
            while (!s->admitted.empty() && b->reqs.size() < s->cfg.max_batch) {
                b->reqs.push_back(s->admitted.front());
                s->admitted.pop_front();
            }
            s->slots[k].busy = true;
            lk.unlock();
            launch_batch(s, b);
            lk.lock();
            launched = true;
        }
        // (stop is set under the lock: if nothing was launched, the lock was held
        // since the check above and the next wake-up sees it)
        if (!launched) s->cv_sched.wait(lk);
    }
}

}  // namespace

extern "C" {

wt_status wt_server_create(const wt_server_config *cfg, wt_server **out)
{
    if (cfg == nullptr || out == nullptr || cfg->max_batch == 0 || cfg->streams == 0) return WT_ERR_INVALID_ARG;
    if (cudaSetDevice(cfg->device) != cudaSuccess) return WT_ERR_CUDA;
    wt_server *s = new wt_server();
    s->cfg = *cfg;
    if (s->cfg.max_pending == 0) s->cfg.max_pending = 1u << 20;
    s->slots.resize(cfg->streams);
    for (auto &sl : s->slots)
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaHostAlloc(reinterpret_cast<void **>(&sl.h_status), 8 * sizeof(uint32_t), cudaHostAllocDefault) !=
                cudaSuccess) {
            for (auto &x : s->slots) {
                if (x.stream) cudaStreamDestroy(x.stream);
                if (x.h_status) cudaFreeHost(x.h_status);
            }
            delete s;
            return WT_ERR_CUDA;
        }
    s->t_create = Clock::now();
    s->sched = std::thread(scheduler, s);
    *out = s;
    return WT_OK;
}

}  // extern "C"

namespace {

// Queues a request; `borrowed`: the text is the caller's page-locked buffer,
// read by the device copy of the batch, and must stay unchanged until the
// request is done.
wt_status submit_impl(wt_server *s, const wt_request *req, uint64_t *ticket, bool borrowed)
{
    if (s == nullptr || req == nullptr || ticket == nullptr) return WT_ERR_INVALID_ARG;
    if (req->kind != WT_TREE && req->kind != WT_MATRIX) return WT_ERR_INVALID_ARG;
    if (req->n > 0 && req->h_text == nullptr) return WT_ERR_INVALID_ARG;
    if (borrowed && req->n > 0) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, req->h_text) != cudaSuccess || at.type != cudaMemoryTypeHost) {
            cudaGetLastError();
            return WT_ERR_INVALID_ARG;
        }
    }
    auto r = std::make_shared<Req>();
    r->kind = req->kind;
    r->type = req->type;
    r->n = req->n;
    r->sigma = req->sigma;
    r->L = wt_levels(req->sigma);
    wt_status st = wt_workspace_size(req->kind, req->type, req->n, req->sigma, &r->ws_alone);
    if (st != WT_OK) return st;
    r->reserved = footprint(*r);
    std::unique_lock<std::mutex> lk(s->mu);
    if (r->reserved > s->cfg.hbm_budget_bytes || s->pending.size() >= s->cfg.max_pending || s->stop) {
        s->rejected++;
        return WT_ERR_BUSY;
    }
    lk.unlock();
    if (borrowed) {
        r->src = req->h_text;
    } else if (req->n) {
        const size_t bytes = req->n * (size_t)req->type;
        r->host.reset(new (std::nothrow) uint8_t[bytes]);     // no value-initialisation
        if (!r->host) return WT_ERR_OUT_OF_MEMORY;
        std::memcpy(r->host.get(), req->h_text, bytes);
        r->src = r->host.get();
    }
    lk.lock();
    r->ticket = s->next_ticket++;
    r->t_submit = Clock::now();
    s->all[r->ticket] = r;
    s->pending.push_back(r);
    s->submitted++;
    s->in_flight++;
    *ticket = r->ticket;
    s->cv_sched.notify_all();
    return WT_OK;
}

}  // namespace

extern "C" {

wt_status wt_server_submit(wt_server *s, const wt_request *req, uint64_t *ticket)
{
    return submit_impl(s, req, ticket, false);
}

wt_status wt_server_submit_pinned(wt_server *s, const wt_request *req, uint64_t *ticket)
{
    return submit_impl(s, req, ticket, true);
}

wt_status wt_server_wait(wt_server *s, uint64_t ticket, int64_t timeout_us, wt_result *res)
{
    if (s == nullptr) return WT_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return WT_ERR_NOT_FOUND;
    std::shared_ptr<Req> r = it->second;
    if (timeout_us < 0) {
        s->cv_done.wait(lk, [&] { return r->done; });
    } else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return r->done; })) {
        return WT_ERR_TIMEOUT;
    }
    if (res) {
        res->d_bv = r->d_bv;
        res->d_zeros = r->d_zeros;
        res->levels = r->L;
        res->words_per_level = (r->n + 63) / 64;
        res->n = r->n;
        res->status = r->status;
        res->latency_us = std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count();
    }
    return r->status;
}

wt_status wt_server_read(wt_server *s, uint64_t ticket, uint64_t *h_bv, uint64_t *h_zeros)
{
    if (s == nullptr) return WT_ERR_INVALID_ARG;
    std::shared_ptr<Req> r;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->all.find(ticket);
        if (it == s->all.end()) return WT_ERR_NOT_FOUND;
        r = it->second;
        if (!r->done) return WT_ERR_BUSY;
    }
    const size_t bytes = (size_t)r->L * ((r->n + 63) / 64) * 8;
    if (bytes && (h_bv == nullptr || r->d_bv == nullptr)) return WT_ERR_INVALID_ARG;
    cudaSetDevice(s->cfg.device);
    if (bytes && cudaMemcpy(h_bv, r->d_bv, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return WT_ERR_CUDA;
    if (h_zeros && r->kind == WT_MATRIX) {
        if (r->d_zeros) {
            if (cudaMemcpy(h_zeros, r->d_zeros, r->L * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return WT_ERR_CUDA;
        } else {
            for (uint32_t l = 0; l < r->L; ++l) h_zeros[l] = 0;
        }
    }
    return WT_OK;
}

wt_status wt_server_release(wt_server *s, uint64_t ticket)
{
    if (s == nullptr) return WT_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return WT_ERR_NOT_FOUND;
    std::shared_ptr<Req> r = it->second;
    if (!r->done) return WT_ERR_BUSY;
    s->all.erase(it);
    s->in_use -= r->reserved;
    cudaStream_t st = s->slots[0].stream;
    lk.unlock();
    if (r->d_text) cudaFreeAsync(r->d_text, st);
    if (r->d_bv) cudaFreeAsync(r->d_bv, st);
    if (r->d_zeros) cudaFreeAsync(r->d_zeros, st);
    lk.lock();
    s->cv_sched.notify_all();
    return WT_OK;
}

wt_status wt_server_get_stats(wt_server *s, wt_server_stats *st)
{
    if (s == nullptr || st == nullptr) return WT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    st->submitted = s->submitted;
    st->completed = s->completed;
    st->rejected = s->rejected;
    st->in_flight = s->in_flight;
    std::vector<double> v = s->latencies;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) { return v.empty() ? 0.0 : v[std::min(v.size() - 1, (size_t)(q * (v.size() - 1) + 0.5))]; };
    st->p50_us = pct(0.50);
    st->p99_us = pct(0.99);
    double secs = std::chrono::duration<double>(Clock::now() - s->t_create).count();
    st->symbols_per_s = secs > 0 ? s->symbols_done / secs : 0.0;
    st->hbm_in_use = s->in_use;
    return WT_OK;
}

void wt_server_destroy(wt_server *s)
{
    if (s == nullptr) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_sched.notify_all();
    }
    if (s->sched.joinable()) s->sched.join();
    for (auto &kv : s->all) {
        auto &r = kv.second;
        if (r->d_text) cudaFreeAsync(r->d_text, s->slots[0].stream);
        if (r->d_bv) cudaFreeAsync(r->d_bv, s->slots[0].stream);
        if (r->d_zeros) cudaFreeAsync(r->d_zeros, s->slots[0].stream);
    }
    for (auto &sl : s->slots) {
        cudaStreamSynchronize(sl.stream);
        cudaStreamDestroy(sl.stream);
        cudaFreeHost(sl.h_status);
    }
    delete s;
}

}  // extern "C"
