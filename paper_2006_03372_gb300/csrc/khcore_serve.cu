// khcore_serve.cu — a request server for (k,h)-core decompositions with
// continuous batching (host code only; the device work is the batch path of
// khcore_api.cu).
//
// Requests (a graph and its h) wait in a FIFO queue. Each of `slots` worker
// threads owns a CUDA stream; a free worker takes every queued request that
// still fits the device-memory budget (up to max_batch), packs them into one
// batch context, decomposes them together and publishes the results. Workers
// run concurrently, so a request that arrives while others are on the GPU is
// admitted as soon as a slot and enough budget are free, and its work overlaps
// with theirs on the device. A request's core indices do not depend on which
// other requests share its batch (each graph peels with its own level).
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/khcore.h"
#include "khcore_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id = 0;
    int32_t n = 0;
    int32_t h = 1;
    std::vector<int32_t> rp, col;
    size_t bytes = 0;
    std::vector<int32_t> core;
    khcore_status status = KHCORE_OK;
    std::string err;
    bool done = false;
    Clock::time_point submitted, started, finished;
};

}  // namespace

struct khcore_server {
    size_t budget = 0;
    size_t in_use = 0;
    int32_t slots = 1;
    int32_t max_batch = 256;
    int device = 0;
    uint64_t next_id = 1;
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, Request *> table;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<std::thread> workers;
    bool stop = false;
    int64_t batches = 0, completed = 0;
    std::string err;
};

namespace {

// Device bytes a request can need inside a batch context: CSR, per-vertex
// peel state and frontier lists (about 64 B per vertex), and the BFS bitsets
// (3 arrays of W 64-bit words per vertex, W <= 16).
size_t request_bytes(int32_t n, int64_t m) { return (size_t)n * (64 + 3 * 8 * 16) + (size_t)m * 4 + 4096; }

// One batch context over the group; blocks: one thread block per graph (all
// graphs small) instead of grid-wide rounds.
void run_group(khcore_server *s, std::vector<Request *> &batch, cudaStream_t stream, bool blocks)
{
    const int32_t G = (int32_t)batch.size();
    std::vector<int64_t> v_off(G + 1, 0), e_off(G + 1, 0);
    for (int32_t g = 0; g < G; g++) {
        v_off[g + 1] = v_off[g] + batch[g]->n;
        e_off[g + 1] = e_off[g] + (int64_t)batch[g]->col.size();
    }
    std::vector<int32_t> rp((size_t)(v_off[G] + G)), col((size_t)e_off[G]), h(G), core((size_t)v_off[G]);
    for (int32_t g = 0; g < G; g++) {
        std::memcpy(rp.data() + v_off[g] + g, batch[g]->rp.data(), sizeof(int32_t) * batch[g]->rp.size());
        if (!batch[g]->col.empty())
            std::memcpy(col.data() + e_off[g], batch[g]->col.data(), sizeof(int32_t) * batch[g]->col.size());
        h[g] = batch[g]->h;
    }
    khcore_ctx *ctx = nullptr;
    khcore_status st = khcore_batch_create(G, v_off.data(), e_off.data(), rp.data(), col.empty() ? nullptr : col.data(),
                                           KHCORE_FLAG_TRUST_INPUT, stream, &ctx);
    std::string msg;
    // small graphs: one block each (no grid barrier, so concurrent groups
    // interleave freely); large graphs: each alone on the grid-wide path, its
    // rounds in one persistent launch (host-driven rounds, one sync per
    // round, left the larger requests far behind the offered load)
    if (st == KHCORE_OK) st = khcore_set_graph_blocks(ctx, blocks ? 1 : 0);
    if (st == KHCORE_OK) {
        st = khcore_batch_decompose(ctx, h.data(), core.data(), nullptr, nullptr);
        if (st != KHCORE_OK) msg = khcore_last_error(ctx);
    } else {
        msg = khcore_last_error(nullptr);
    }
    khcore_destroy(ctx);
    const auto now = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    for (int32_t g = 0; g < G; g++) {
        Request *r = batch[g];
        r->status = st;
        r->err = msg;
        if (st == KHCORE_OK) r->core.assign(core.begin() + v_off[g], core.begin() + v_off[g + 1]);
        r->finished = now;
        r->done = true;
        s->in_use -= r->bytes;
        s->completed++;
    }
    s->batches++;
    s->cv_done.notify_all();
    s->cv_work.notify_all();  // budget freed
}

bool is_small(const Request *r) { return r->n <= khc::kBlockGraphsMaxN; }

// A worker takes either every queued small request that fits the budget (up
// to max_batch, in arrival order), decomposed together in one launch of one
// thread block per graph, or, when no small request waits, the oldest large
// request, decomposed alone on the grid-wide path. Each is published as soon
// as its own work is done, so a large request never holds small ones back and
// several large ones run at once on different slots.
void worker_main(khcore_server *s)
{
    cudaSetDevice(s->device);
    cudaStream_t stream = nullptr;
    if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) return;
    for (;;) {
        std::vector<Request *> batch;
        bool small = false;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            auto admissible = [&](const Request *r) { return s->in_use + r->bytes <= s->budget; };
            auto any_work = [&] {
                for (const Request *r : s->queue)
                    if (admissible(r)) return true;
                return false;
            };
            s->cv_work.wait(lk, [&] { return s->stop || any_work(); });
            if (s->stop) break;  // queued requests are dropped by khcore_server_destroy
            for (auto it = s->queue.begin(); it != s->queue.end() && (int32_t)batch.size() < s->max_batch;) {
                Request *r = *it;
                if (is_small(r) && admissible(r)) {
                    s->in_use += r->bytes;
                    r->started = Clock::now();
                    batch.push_back(r);
                    it = s->queue.erase(it);
                } else {
                    ++it;
                }
            }
            small = !batch.empty();
            if (!small) {
                for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
                    Request *r = *it;
                    if (!admissible(r)) continue;
                    s->in_use += r->bytes;
                    r->started = Clock::now();
                    batch.push_back(r);
                    s->queue.erase(it);
                    break;
                }
            }
        }
        if (!batch.empty()) run_group(s, batch, stream, small);
    }
    cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

khcore_status khcore_server_create(size_t device_bytes_budget, int32_t slots, int32_t max_batch, khcore_server **out)
{
    if (!out) return KHCORE_EINVAL;
    *out = nullptr;
    if (device_bytes_budget == 0 || slots < 1 || slots > 64 || max_batch < 1) return KHCORE_EINVAL;
    khcore_server *s = new (std::nothrow) khcore_server();
    if (!s) return KHCORE_ENOMEM;
    s->budget = device_bytes_budget;
    s->slots = slots;
    s->max_batch = max_batch;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        (void)cudaGetLastError();
        delete s;
        return KHCORE_ECUDA;
    }
    try {
        for (int32_t i = 0; i < slots; i++) s->workers.emplace_back(worker_main, s);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv_work.notify_all();
        for (auto &t : s->workers) t.join();
        delete s;
        return KHCORE_ENOMEM;
    }
    *out = s;
    return KHCORE_OK;
}

khcore_status khcore_server_submit(khcore_server *s, int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t h,
                                   uint64_t *ticket)
{
    if (!s || !ticket || n < 0 || !row_ptr || h < 1) return KHCORE_EINVAL;
    const int64_t m = row_ptr[n];
    if (m < 0 || (m > 0 && !col)) return KHCORE_EINVAL;
    Request *r = new (std::nothrow) Request();
    if (!r) return KHCORE_ENOMEM;
    r->n = n;
    r->h = h;
    r->rp.assign(row_ptr, row_ptr + n + 1);
    r->col.assign(col ? col : row_ptr, col ? col + m : row_ptr);
    r->bytes = request_bytes(n, m);
    r->submitted = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (r->bytes > s->budget) {
        delete r;
        return KHCORE_ENOMEM;  // can never be admitted
    }
    r->id = s->next_id++;
    s->table[r->id] = r;
    s->queue.push_back(r);
    *ticket = r->id;
    s->cv_work.notify_one();
    return KHCORE_OK;
}

khcore_status khcore_server_wait(khcore_server *s, uint64_t ticket, int32_t *core_out, double timeout_s,
                                 double *latency_ms)
{
    if (!s) return KHCORE_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->table.find(ticket);
    if (it == s->table.end()) return KHCORE_EINVAL;
    Request *r = it->second;
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    if (!s->cv_done.wait_until(lk, deadline, [&] { return r->done; })) return KHCORE_ETIMEOUT;
    const khcore_status st = r->status;
    if (st == KHCORE_OK && core_out && r->n) std::memcpy(core_out, r->core.data(), sizeof(int32_t) * (size_t)r->n);
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->finished - r->submitted).count();
    if (st != KHCORE_OK) s->err = r->err;
    s->table.erase(it);
    delete r;
    return st;
}

khcore_status khcore_server_poll(khcore_server *s, uint64_t ticket, int32_t *done)
{
    if (!s || !done) return KHCORE_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->table.find(ticket);
    if (it == s->table.end()) return KHCORE_EINVAL;
    *done = it->second->done ? 1 : 0;
    return KHCORE_OK;
}

khcore_status khcore_server_stats(khcore_server *s, int64_t *queued, int64_t *completed, int64_t *batches,
                                  size_t *bytes_in_use)
{
    if (!s) return KHCORE_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (queued) *queued = (int64_t)s->queue.size();
    if (completed) *completed = s->completed;
    if (batches) *batches = s->batches;
    if (bytes_in_use) *bytes_in_use = s->in_use;
    return KHCORE_OK;
}

size_t khcore_request_bytes(int32_t n, int64_t m) { return request_bytes(n, m); }

const char *khcore_server_last_error(khcore_server *s)
{
    if (!s) return "";
    std::lock_guard<std::mutex> lk(s->mu);
    return s->err.c_str();
}

void khcore_server_destroy(khcore_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    for (auto &kv : s->table) delete kv.second;
    delete s;
}

}  // extern "C"
