// khcore_api.cu — the C ABI declared in include/khcore.h: context life cycle,
// CSR validation, and the host side of the level-synchronous peeler for one
// graph or a batch of disjoint graphs.
#include <algorithm>
#include <climits>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/khcore.h"
#include "khcore_internal.cuh"

using namespace khc;

struct khcore_ctx {
    int32_t n = 0;
    int64_t m = 0;
    int32_t G = 1;                // graphs held (1 for khcore_create)
    std::vector<int64_t> v_off;   // [G+1] vertex offsets of the graphs
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool failed = false;
    std::string err;

    // graph (device)
    int32_t *row_ptr = nullptr, *col = nullptr;
    int32_t *classes = nullptr;  // light | medium | heavy lists, back to back
    int32_t n_light = 0, n_medium = 0, n_heavy = 0;
    int32_t *gid = nullptr;      // [n] graph of each vertex (G > 1 only)

    // per-graph peel parameters (device)
    int32_t *kg = nullptr, *ming = nullptr, *hg = nullptr, *gcls = nullptr;
    int32_t *cls_off = nullptr, *nAc = nullptr;  // [G] capacity each (ncls <= G)
    int32_t *nDc = nullptr, *inner = nullptr, *clsh = nullptr;  // [G] capacity each
    int32_t *cls_src = nullptr;                  // [n] vertices grouped by h-class
    int32_t *dcls = nullptr;                     // [n] deleted vertices grouped by h-class (per round)
    int32_t *dcount = nullptr;                   // [n] deleted vertices within h (outer-shell update)
    int32_t *comb = nullptr;                     // [n] round source list: inner vertices, then deleted ones
    int32_t *slack = nullptr;                    // [n] lazy mode: deg - slack is a lower bound
    int32_t *cand = nullptr;                     // [n] lazy mode: exact-recompute list (class regions)
    int32_t *wsum = nullptr;                     // [n] lazy mode: ball bounds of the deleted set, zero between rounds
    int32_t *mind = nullptr, *minub = nullptr, *ncand = nullptr;  // [G]
    bool lazy = true;                            // bounds instead of recomputing every inner vertex

    // peel state (device)
    uint32_t *alive = nullptr;
    int32_t *deg = nullptr, *core = nullptr, *rnd = nullptr, *src = nullptr;
    uint32_t *vis = nullptr;
    PeelState *st = nullptr;
    PeelState *st_host = nullptr;  // pinned mirror
    int32_t *nAc_host = nullptr;   // pinned mirror of nAc, inner, nDc, ncand (4 x G)

    // BFS buffers, sized for W_alloc words per vertex
    int W_req = 0;   // 0 = automatic
    int W_av = 0;    // the all-vertex pass's W chosen by khcore_autotune (0 = none)
    int Wr_req = 0;  // W of the peel rounds, 0 = automatic
    int W_alloc = 0;
    uint64_t *V = nullptr, *F[2] = {nullptr, nullptr};
    uint32_t *flag[2] = {nullptr, nullptr};  // frontier bitmaps
    uint64_t *Fx = nullptr;                    // third frontier array of the persistent kernel's ring
    uint32_t *flagx = nullptr, *tflag = nullptr;  // its flag bitmap; vertices already in the touched list
    int32_t *Q[3] = {nullptr, nullptr, nullptr};
    int2 *I[3] = {nullptr, nullptr, nullptr};
    int32_t *T = nullptr;
    LevelCtl *ctl = nullptr;
    int32_t *cnt = nullptr;
    unsigned long long *edges = nullptr;  // device counter of plain-BFS-equivalent edges
    unsigned long long *alg = nullptr;    // device counter of algorithmic bytes of the BFS levels
    int32_t push_alpha = 4;               // push when frontier degree sum * alpha < alive CSR entries
    int32_t round_loop = 0;               // 0: one persistent launch per decomposition, 1: host-driven rounds
    int32_t graph_blocks = 0;             // 0: auto, 1: one thread block per graph, -1: never
    int32_t *voff_d = nullptr;            // [G+1] vertex offsets (int32) for the per-block path
    int32_t *order_d = nullptr;           // [G] graph order of the per-block path
    int32_t *bnext = nullptr;             // per-block path work counter
    BlockStats *bstats = nullptr;
    unsigned long long wait_limit_ns = 10ull * 1000 * 1000 * 1000;  // one grid-barrier wait
    bool dirty = false;                   // a launch stopped midway: BFS buffers need clearing
    int32_t *cls_size = nullptr;          // [G] initial class sizes (device)
    GridSync *gs = nullptr;
    PersistStats *pstats = nullptr;
    int32_t update_mode = 0;              // 0: BFS recompute; 1: the paper's per-deletion update (Algorithms 3/4)
    // tuning knobs (khcore_autotune picks them)
    int32_t light_max = kLightMax;        // pull degree classes
    int32_t medium_max = kMediumMax;
    int32_t block = kBlock;               // threads per block of the per-phase BFS kernels
    int32_t block_graph_max = kBlockGraphsMaxN;  // batches: graphs decomposed by one thread block
    int32_t init_alpha = 16;              // push alpha of the all-vertex pass (0: push_alpha)
    int32_t round_blocks = 0;             // round kernel blocks per SM (0: by h)
    int32_t persist_sms = 0;              // SMs the round kernel's grid covers (0: all)
    int32_t concurrent = 1;               // batches: larger graphs decomposed at once
    int32_t *class_counts = nullptr;      // [6] scratch of the class builder
    // the sampling variant (Algorithms 5 and 6): sample bytes, select at the
    // start and now, exact h-degrees at the start, the per-batch mask of the
    // sources that count every vertex; sampling = 0 off, 1 select pass, 2 rounds
    uint8_t *s_in = nullptr;
    int32_t *s_sel0 = nullptr, *s_sel = nullptr, *s_d0 = nullptr;
    uint64_t *s_full = nullptr;
    int sampling = 0;
    bool sampling_req = false;
    UpdBufs upd{};                        // its slots, allocated on first use
    bool upd_ready = false;

    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev_init = nullptr;

    // profiling: an event pair around every BFS level launch
    bool profiling = false;
    std::vector<cudaEvent_t> tev;
    LevelTimer timer{nullptr, 0, 0};
    double level_ms = 0.0;
    int64_t level_launches = 0;

    // degree classes of the all-vertex pass when tuned apart from the rounds'
    // (khcore_autotune); nullptr: the same lists
    int32_t *classes_av = nullptr;
    int32_t n_light_av = 0, n_medium_av = 0, n_heavy_av = 0;

    GraphView view(bool all_vertex = false) const
    {
        const bool av = all_vertex && classes_av;
        GraphView g;
        g.n = n;
        g.m = m;
        g.row_ptr = row_ptr;
        g.col = col;
        const int32_t *cl = av ? classes_av : classes;
        const int32_t nl = av ? n_light_av : n_light, nm = av ? n_medium_av : n_medium;
        g.light = cl;
        g.medium = cl + nl;
        g.heavy = cl + nl + nm;
        g.n_light = nl;
        g.n_medium = nm;
        g.n_heavy = av ? n_heavy_av : n_heavy;
        return g;
    }
};

namespace {

thread_local std::string g_create_err;

khcore_status fail(khcore_ctx *c, khcore_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) {
        c->err = buf;
        if (s == KHCORE_ECUDA) c->failed = true;
    } else {
        g_create_err = buf;
    }
    return s;
}

#define CU(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            if (e_ == cudaErrorMemoryAllocation) {                                      \
                (void)cudaGetLastError();                                               \
                return fail(c, KHCORE_ENOMEM, "%s: %s", #call, cudaGetErrorString(e_)); \
            }                                                                           \
            return fail(c, KHCORE_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));      \
        }                                                                               \
    } while (0)

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Allocation-failure injection for tests, entirely on the host: when the
// environment variable KHCORE_FAIL_ALLOC_AT holds N > 0 as a context is
// created, the N-th device allocation the calling thread makes from then on
// (the context's own buffers first, then the BFS rows its first decomposition
// allocates) fails as if the device were out of memory, without calling
// cudaMalloc. Unset or 0: no injection.
thread_local int64_t g_fail_alloc_at = 0;
thread_local int64_t g_allocs_seen = 0;

void arm_alloc_injection()
{
    const char *e = getenv("KHCORE_FAIL_ALLOC_AT");
    g_fail_alloc_at = e ? atoll(e) : 0;
    g_allocs_seen = 0;
}

template <class T>
cudaError_t dev_alloc(T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    if (g_fail_alloc_at > 0 && ++g_allocs_seen == g_fail_alloc_at) return cudaErrorMemoryAllocation;
    return cudaMalloc((void **)p, count * sizeof(T));
}

// Copy `count` elements from a host or device pointer into a host vector.
template <class T>
cudaError_t fetch(std::vector<T> &dst, const T *src, size_t count)
{
    dst.resize(count);
    if (count == 0) return cudaSuccess;
    if (is_device_ptr(src)) return cudaMemcpy(dst.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost);
    std::memcpy(dst.data(), src, count * sizeof(T));
    return cudaSuccess;
}

// Validates an undirected simple CSR; on success `sorted` holds col with every
// row sorted (the library does not depend on row order, but validation does).
bool validate_csr(int32_t n, const std::vector<int32_t> &rp, const std::vector<int32_t> &col,
                  std::vector<int32_t> &sorted, std::string &msg)
{
    char buf[256];
    if (rp[0] != 0) {
        msg = "row_ptr[0] must be 0";
        return false;
    }
    for (int32_t v = 0; v < n; v++)
        if (!csr_row_ok(rp[v], rp[v + 1], rp[n])) {
            snprintf(buf, sizeof buf, "row_ptr is not a CSR offset array at vertex %d (it decreases or leaves [0, %d])",
                     v, rp[n]);
            msg = buf;
            return false;
        }
    sorted = col;
    for (int32_t v = 0; v < n; v++) {
        auto b = sorted.begin() + rp[v], e = sorted.begin() + rp[v + 1];
        if (!std::is_sorted(b, e)) std::sort(b, e);
        for (auto it = b; it != e; ++it) {
            const int32_t u = *it;
            if (u < 0 || u >= n) {
                snprintf(buf, sizeof buf, "neighbour id %d of vertex %d outside [0, %d)", u, v, n);
                msg = buf;
                return false;
            }
            if (u == v) {
                snprintf(buf, sizeof buf, "self-loop at vertex %d", v);
                msg = buf;
                return false;
            }
            if (it != b && *(it - 1) == u) {
                snprintf(buf, sizeof buf, "duplicate edge %d-%d", v, u);
                msg = buf;
                return false;
            }
        }
    }
    for (int32_t v = 0; v < n; v++)
        for (int32_t e = rp[v]; e < rp[v + 1]; e++) {
            const int32_t u = sorted[e];
            if (!std::binary_search(sorted.begin() + rp[u], sorted.begin() + rp[u + 1], v)) {
                snprintf(buf, sizeof buf, "edge %d-%d has no reverse entry (graph must be undirected)", v, u);
                msg = buf;
                return false;
            }
        }
    return true;
}

// W of the all-vertex h-degree pass: the widest batch (1024 sources) amortises
// the CSR scan of every level best; small graphs take the smallest W whose
// batch holds every vertex.
int auto_words(int32_t n)
{
    int W = 1;
    while (W < 16 && 64 * W < n) W *= 2;
    return W;
}

// W of the peel rounds: their source sets (the affected vertices closer than
// h to the deleted set) are usually small, and a narrow row keeps the level
// kernels at two resident blocks per SM and 32/W edges per warp step in the
// push direction.
int auto_round_words(int32_t n) { return std::min(auto_words(n), 4); }

khcore_status ensure_bfs(khcore_ctx *c, int W)
{
    if (c->W_alloc >= W) return KHCORE_OK;  // rows of any narrower W fit the same arrays
    cudaFree(c->V);
    cudaFree(c->F[0]);
    cudaFree(c->F[1]);
    cudaFree(c->Fx);
    cudaFree(c->cnt);
    c->V = c->F[0] = c->F[1] = c->Fx = nullptr;
    c->cnt = nullptr;
    c->W_alloc = 0;
    const size_t words = (size_t)std::max(c->n, 1) * W;
    CU(dev_alloc(&c->V, words));
    CU(dev_alloc(&c->F[0], words));
    CU(dev_alloc(&c->F[1], words));
    CU(dev_alloc(&c->Fx, words));
    CU(dev_alloc(&c->cnt, (size_t)64 * W));
    CU(cudaMemsetAsync(c->V, 0, words * sizeof(uint64_t), c->stream));
    CU(cudaMemsetAsync(c->F[0], 0, words * sizeof(uint64_t), c->stream));
    CU(cudaMemsetAsync(c->F[1], 0, words * sizeof(uint64_t), c->stream));
    CU(cudaMemsetAsync(c->Fx, 0, words * sizeof(uint64_t), c->stream));
    CU(cudaMemsetAsync(c->cnt, 0, (size_t)64 * W * sizeof(int32_t), c->stream));
    c->W_alloc = W;
    return KHCORE_OK;
}

int bfs_grid(khcore_ctx *c, int W) { return c->sm_count * max_blocks_per_sm_bfs(W, c->block); }

// After a launch that stopped midway (a timed-out barrier) the BFS buffers may
// hold rows of an unfinished batch: restore the all-zero state.
khcore_status clear_if_dirty(khcore_ctx *c)
{
    if (!c->dirty || c->W_alloc == 0) return KHCORE_OK;
    const size_t words = (size_t)std::max(c->n, 1) * c->W_alloc;
    const size_t nflag = (((size_t)c->n + 31) / 32) * 4;  // bytes of one flag bitmap
    CU(cudaMemsetAsync(c->V, 0, words * sizeof(uint64_t), c->stream));
    CU(cudaMemsetAsync(c->F[0], 0, words * sizeof(uint64_t), c->stream));
    CU(cudaMemsetAsync(c->F[1], 0, words * sizeof(uint64_t), c->stream));
    CU(cudaMemsetAsync(c->Fx, 0, words * sizeof(uint64_t), c->stream));
    CU(cudaMemsetAsync(c->flag[0], 0, nflag, c->stream));
    CU(cudaMemsetAsync(c->flag[1], 0, nflag, c->stream));
    CU(cudaMemsetAsync(c->flagx, 0, nflag, c->stream));
    CU(cudaMemsetAsync(c->tflag, 0, nflag, c->stream));
    CU(cudaMemsetAsync(c->cnt, 0, (size_t)64 * c->W_alloc * sizeof(int32_t), c->stream));
    CU(cudaMemsetAsync(c->dcount, 0, sizeof(int32_t) * (size_t)std::max(c->n, 1), c->stream));
    CU(cudaMemsetAsync(c->wsum, 0, sizeof(int32_t) * (size_t)std::max(c->n, 1), c->stream));
    c->dirty = false;
    return KHCORE_OK;
}

// Sum the timed level launches recorded so far (waits for the last one).
khcore_status flush_timer(khcore_ctx *c)
{
    if (!c->profiling || c->timer.used == 0) return KHCORE_OK;
    CU(cudaEventSynchronize(c->timer.ev[2 * c->timer.used - 1]));
    for (int i = 0; i < c->timer.used; i++) {
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, c->timer.ev[2 * i], c->timer.ev[2 * i + 1]));
        c->level_ms += ms;
    }
    c->level_launches += c->timer.used;
    c->timer.used = 0;
    return KHCORE_OK;
}

// h-degrees of the sources src[0..ns) in G[alive], in batches of 64*W.
// n_b / m_b: alive rows and their CSR entries (direction choice and
// algorithmic bytes).
// rowcnt (nullable): row counts of the sources at list positions >= row_first.
// wsum (nullable, lazy mode with src = the deleted set): ball bounds of the
// sources for the vertices they reach within h-1 (dev_weight_pass).
khcore_status hdeg_sources(khcore_ctx *c, int W, int32_t h, const int32_t *src, int32_t ns, int64_t n_b,
                           int64_t m_b, khcore_stats *stt, int32_t *rowcnt = nullptr, int32_t row_first = 0,
                           int32_t *wsum = nullptr, bool all_vertex = false)
{
    const GraphView g = c->view(all_vertex);
    BfsBufs b;
    b.V = c->V;
    b.F[0] = c->F[0];
    b.F[1] = c->F[1];
    b.flag[0] = c->flag[0];
    b.flag[1] = c->flag[1];
    for (int k = 0; k < 3; k++) {
        b.Q[k] = c->Q[k];
        b.I[k] = c->I[k];
    }
    b.T = c->T;
    b.ctl = c->ctl;
    b.cnt = c->cnt;
    b.edges = c->edges;
    b.Fx = nullptr;  // the per-phase kernels use two-slot levels
    b.flagx = nullptr;
    b.tflag = nullptr;
    b.rowcnt = rowcnt;
    b.row_first = 0;
    b.row_sign = 1;
    b.newcnt = nullptr;
    b.alg_bytes = c->alg;
    b.slev = nullptr;
    b.cum = nullptr;
    b.hcnt = 0;
    b.boff = 0;
    b.wsum = wsum;
    b.wdeg = c->deg;
    // sampling variant: 1 = the pass that counts the sampled vertices of every
    // ball (select at the start), 2 = the rounds (estimates)
    b.in_s = c->sampling ? c->s_in : nullptr;
    b.fullmask = c->sampling ? c->s_full : nullptr;
    b.sel0 = c->sampling == 2 ? c->s_sel0 : nullptr;
    b.sel = c->sampling == 1 ? c->s_sel0 : (c->sampling == 2 ? c->s_sel : nullptr);
    b.d0 = c->sampling == 2 ? c->s_d0 : nullptr;
    BfsTuning tune;
    // the all-vertex pass may have a push alpha of its own (khcore_autotune)
    tune.alpha = (all_vertex && c->init_alpha) ? c->init_alpha : c->push_alpha;
    tune.n_alive = (int32_t)n_b;
    tune.m_alive = (unsigned long long)m_b;
    const int32_t S = 64 * W;
    const int grid = bfs_grid(c, W);
    for (int32_t off = 0; off < ns; off += S) {
        const int32_t cur = std::min(S, ns - off);
        b.row_first = std::max(0, row_first - off);
        if (c->profiling && c->timer.used + h > c->timer.cap) {
            khcore_status s = flush_timer(c);
            if (s != KHCORE_OK) return s;
        }
        // a batch of at most 64 sources runs on one-word rows (a quarter of
        // the row traffic of W = 4; the row arrays are all zero between
        // batches in either layout)
        const int Wb = (W > 1 && cur <= 64) ? 1 : W;
        CU(run_bfs_batch(Wb, g, c->alive, b, src + off, cur, h, c->deg, tune, Wb == W ? grid : bfs_grid(c, Wb),
                         c->block, c->stream, stt ? &stt->kernel_launches : nullptr, c->profiling ? &c->timer : nullptr));
        if (stt) {
            stt->source_batches++;
        }
    }
    return KHCORE_OK;
}

khcore_status check_ctx(khcore_ctx *c)
{
    if (!c) return KHCORE_EINVAL;
    if (c->failed) return KHCORE_ECUDA;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return fail(c, KHCORE_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    return KHCORE_OK;
}

khcore_status write_out(khcore_ctx *c, int32_t *dst, const int32_t *src_dev)
{
    if (!dst || c->n == 0) return KHCORE_OK;
    const size_t bytes = (size_t)c->n * sizeof(int32_t);
    CU(cudaMemcpyAsync(dst, src_dev, bytes, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       c->stream));
    return KHCORE_OK;
}

// h > n-1 behaves as n-1 (no distance exceeds it).
int32_t effective_h(int64_t n, int32_t h) { return (int32_t)std::min<int64_t>(h, std::max<int64_t>(n - 1, 1)); }

// Upload a validated global CSR and set up every device buffer.
khcore_status setup_ctx(khcore_ctx *c, const std::vector<int32_t> &rp, const std::vector<int32_t> &col,
                        const std::vector<int32_t> *gid_host, void *stream)
{
    const int32_t n = c->n;
    const int64_t m = c->m;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) return fail(nullptr, KHCORE_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return fail(nullptr, KHCORE_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
        c->own_stream = true;
    }
    // degree classes of the pull direction
    std::vector<int32_t> classes;
    classes.reserve(n);
    for (int pass = 0; pass < 3; pass++)
        for (int32_t v = 0; v < n; v++) {
            const int32_t d = rp[v + 1] - rp[v];
            const int cls = d <= kLightMax ? 0 : (d <= kMediumMax ? 1 : 2);
            if (cls == pass) classes.push_back(v);
        }
    for (int32_t v = 0; v < n; v++) {
        const int32_t d = rp[v + 1] - rp[v];
        if (d <= kLightMax) c->n_light++;
        else if (d <= kMediumMax) c->n_medium++;
        else c->n_heavy++;
    }
    const size_t nw = ((size_t)n + 31) / 32;
    const size_t nflag = (((size_t)n + 31) / 32) * 4;  // bytes of one frontier flag bitmap
    khcore_status st = KHCORE_OK;
    auto A = [&](cudaError_t e2) {
        if (e2 != cudaSuccess && st == KHCORE_OK) {
            (void)cudaGetLastError();
            st = fail(nullptr, e2 == cudaErrorMemoryAllocation ? KHCORE_ENOMEM : KHCORE_ECUDA, "device allocation: %s",
                      cudaGetErrorString(e2));
        }
    };
    A(dev_alloc(&c->row_ptr, (size_t)n + 1));
    A(dev_alloc(&c->col, (size_t)m));
    A(dev_alloc(&c->classes, (size_t)n));
    A(dev_alloc(&c->alive, nw));
    A(dev_alloc(&c->deg, (size_t)n));
    A(dev_alloc(&c->core, (size_t)n));
    A(dev_alloc(&c->rnd, (size_t)n));
    A(dev_alloc(&c->src, (size_t)n));
    A(dev_alloc(&c->cls_src, (size_t)n));
    A(dev_alloc(&c->vis, nw));
    A(dev_alloc(&c->st, 1));
    A(dev_alloc(&c->edges, 1));
    A(dev_alloc(&c->alg, 1));
    A(dev_alloc(&c->flag[0], nflag / 4));
    A(dev_alloc(&c->flag[1], nflag / 4));
    A(dev_alloc(&c->flagx, nflag / 4));
    A(dev_alloc(&c->tflag, nflag / 4));
    for (int k = 0; k < 3; k++) {
        A(dev_alloc(&c->Q[k], (size_t)n));
        // push items: every frontier row in chunks of at least 8 entries
        A(dev_alloc(&c->I[k], (size_t)n + (size_t)m / 8 + 1));
    }
    A(dev_alloc(&c->T, (size_t)n));
    A(dev_alloc(&c->ctl, 1));
    A(dev_alloc(&c->kg, (size_t)c->G));
    A(dev_alloc(&c->ming, (size_t)c->G));
    A(dev_alloc(&c->hg, (size_t)c->G));
    A(dev_alloc(&c->gcls, (size_t)c->G));
    A(dev_alloc(&c->cls_off, (size_t)c->G));
    A(dev_alloc(&c->nAc, (size_t)c->G));
    A(dev_alloc(&c->nDc, (size_t)c->G));
    A(dev_alloc(&c->inner, (size_t)c->G));
    A(dev_alloc(&c->clsh, (size_t)c->G));
    A(dev_alloc(&c->dcls, (size_t)n));
    A(dev_alloc(&c->dcount, (size_t)n));
    A(dev_alloc(&c->comb, (size_t)n));
    A(dev_alloc(&c->slack, (size_t)n));
    A(dev_alloc(&c->cand, (size_t)n));
    A(dev_alloc(&c->wsum, (size_t)n));
    A(dev_alloc(&c->mind, (size_t)c->G));
    A(dev_alloc(&c->minub, (size_t)c->G));
    A(dev_alloc(&c->ncand, (size_t)c->G));
    A(dev_alloc(&c->cls_size, (size_t)c->G));
    A(dev_alloc(&c->gs, 1));
    A(dev_alloc(&c->pstats, 1));
    if (c->G > 1) A(dev_alloc(&c->gid, (size_t)n));
    A(dev_alloc(&c->voff_d, (size_t)c->G + 1));
    A(dev_alloc(&c->order_d, (size_t)c->G));
    A(dev_alloc(&c->bnext, 1));
    A(dev_alloc(&c->bstats, 1));
    if (st != KHCORE_OK) return st;
    {
        std::vector<int32_t> vo(c->v_off.begin(), c->v_off.end());
        e = cudaMemcpy(c->voff_d, vo.data(), sizeof(int32_t) * vo.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(nullptr, KHCORE_ECUDA, "offset upload: %s", cudaGetErrorString(e));
    }
    e = cudaMallocHost((void **)&c->st_host, sizeof(PeelState));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->nAc_host, 4 * sizeof(int32_t) * (size_t)c->G);
    if (e == cudaSuccess && n) e = cudaMemsetAsync(c->dcount, 0, sizeof(int32_t) * (size_t)n, c->stream);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev_init);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->row_ptr, rp.data(), ((size_t)n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice,
                            c->stream);
    if (e == cudaSuccess && m)
        e = cudaMemcpyAsync(c->col, col.data(), (size_t)m * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && n)
        e = cudaMemcpyAsync(c->classes, classes.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice,
                            c->stream);
    if (e == cudaSuccess && gid_host && n && c->gid)  // one graph needs no graph ids
        e = cudaMemcpyAsync(c->gid, gid_host->data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->flag[0], 0, nflag, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->flag[1], 0, nflag, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->flagx, 0, nflag, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->tflag, 0, nflag, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(nullptr, KHCORE_ECUDA, "graph upload: %s", cudaGetErrorString(e));
    return KHCORE_OK;
}

// Outputs and statistics common to both round loops. persistent: the level
// time is the whole launch (one kernel).
khcore_status finish_decompose(khcore_ctx *c, int32_t G, int32_t *core_out, int32_t *round_out, khcore_stats *stats,
                               khcore_stats stt, bool persistent)
{
    khcore_status s;
    CU(cudaEventRecord(c->ev1, c->stream));
    if ((s = write_out(c, core_out, c->core)) != KHCORE_OK) return s;
    if ((s = write_out(c, round_out, c->rnd)) != KHCORE_OK) return s;
    unsigned long long edges = 0, alg = 0;
    std::vector<int32_t> kg(G);
    CU(cudaMemcpyAsync(&edges, c->edges, sizeof edges, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(&alg, c->alg, sizeof alg, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(kg.data(), c->kg, sizeof(int32_t) * G, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    float ms = 0.f, ms_init = 0.f;
    CU(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    CU(cudaEventElapsedTime(&ms_init, c->ev0, c->ev_init));
    stt.device_ms = ms;
    stt.init_ms = ms_init;
    stt.round_ms = ms - ms_init;
    stt.edges_traversed = (int64_t)edges;
    stt.round_bytes = (double)alg - stt.level_bytes;  // every level after the initial pass
    stt.k_max = *std::max_element(kg.begin(), kg.end());
    if (persistent) {
        if ((s = flush_timer(c)) != KHCORE_OK) return s;  // the initial pass's level launches
        stt.level_ms = c->level_ms;
        stt.level_launches = c->level_launches;
    } else {
        if ((s = flush_timer(c)) != KHCORE_OK) return s;
        stt.level_ms = c->level_ms;
        stt.level_launches = c->level_launches;
    }
    if (!c->profiling) {
        stt.level_ms = 0;
        stt.level_launches = 0;
    }
    if (stats) *stats = stt;
    return KHCORE_OK;
}

// Slots of the paper's per-deletion update: kUpdSlots deleted vertices per
// wave, balls of at most kUpdCap members (and the graph's n), bitmaps of
// kUpdWords words (|N_v^{h-1}| <= 256).
constexpr int32_t kUpdSlots = 64;
constexpr int32_t kUpdCap = 1 << 16;
constexpr int32_t kUpdWords = 4;
constexpr int32_t kUpdMaxH = 255;  // distances are stored in one byte

khcore_status ensure_upd(khcore_ctx *c)
{
    if (c->upd_ready) return KHCORE_OK;
    UpdBufs &u = c->upd;
    const size_t n = (size_t)std::max(c->n, 1);
    u.nblk = kUpdSlots;
    u.cap = (int32_t)std::min<size_t>(kUpdCap, n);
    u.wc = kUpdWords;
    u.vis_words = (int64_t)((n + 31) / 32);
    CU(dev_alloc(&u.vis, (size_t)u.nblk * (size_t)u.vis_words));
    CU(dev_alloc(&u.list, (size_t)u.nblk * u.cap));
    CU(dev_alloc(&u.dist, (size_t)u.nblk * u.cap));
    CU(dev_alloc(&u.reach, (size_t)u.nblk * 2 * u.cap * u.wc));
    CU(dev_alloc(&u.meta, (size_t)u.nblk * 4));
    CU(dev_alloc(&u.owner, n));
    CU(dev_alloc(&u.lab, n));
    CU(dev_alloc(&u.done, (size_t)u.nblk));
    CU(dev_alloc(&u.flag, 2));
    CU(dev_alloc(&u.cand[0], n));
    CU(dev_alloc(&u.cand[1], n));
    CU(cudaMemsetAsync(u.vis, 0, sizeof(uint32_t) * (size_t)u.nblk * (size_t)u.vis_words, c->stream));
    CU(launch_fill_i32(u.owner, INT_MAX, (int64_t)n, c->stream));
    c->upd_ready = true;
    return KHCORE_OK;
}

// The deleted vertices cand[0..nd) of G[c->alive], all still alive, updated
// one after the other by the paper's exact update (waves of pairwise
// disjoint closed balls) and deleted. st (nullable) gets the alive counts.
// *fit = false (nothing changed) when some ball is over the slots' limits or
// nd exceeds the slots of one wave; the caller then uses the BFS recompute.
khcore_status update_deleted(khcore_ctx *c, int32_t h, int32_t nd, PeelState *st, bool *fit, int64_t *launches)
{
    *fit = false;
    if (h > kUpdMaxH || nd > kUpdSlots) return KHCORE_OK;
    khcore_status s;
    if ((s = ensure_upd(c)) != KHCORE_OK) return s;
    UpdBufs &u = c->upd;
    const GraphView g = c->view();
    int cur = 0;
    int32_t nrem = nd, hflag[2] = {0, 0};
    for (int wave = 0; nrem > 0; wave++) {
        const int32_t ncur = std::min(nrem, u.nblk);
        if (wave == 0) CU(cudaMemsetAsync(u.flag, 0, sizeof(int32_t) * 2, c->stream));
        CU(launch_ball_claim(g, c->alive, u, u.cand[cur], ncur, h, c->stream));
        if (wave == 0) {
            // every ball is as large as it will get in this round: check once
            CU(cudaMemcpyAsync(hflag, u.flag, sizeof hflag, cudaMemcpyDeviceToHost, c->stream));
            CU(cudaStreamSynchronize(c->stream));
            if (hflag[0]) {
                CU(launch_ball_reset(u, u.cand[cur], ncur, c->stream));
                if (launches) *launches += 2;
                return KHCORE_OK;
            }
        }
        CU(launch_ball_apply(g, c->alive, u, u.cand[cur], ncur, h, c->deg, st, c->stream));
        CU(launch_ball_reset(u, u.cand[cur], ncur, c->stream));
        CU(launch_wave_next(u, u.cand[cur], nrem, ncur, u.cand[cur ^ 1], c->stream));
        CU(cudaMemcpyAsync(hflag, u.flag, sizeof hflag, cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
        if (launches) *launches += 4;
        if (hflag[1] >= nrem) return fail(c, KHCORE_EINTERNAL, "update wave made no progress (%d left)", nrem);
        nrem = hflag[1];
        cur ^= 1;
    }
    *fit = true;
    return KHCORE_OK;
}

khcore_status decompose(khcore_ctx *c, const std::vector<int32_t> &h_in, int32_t *core_out, int32_t *round_out,
                        khcore_stats *stats);

// Graph gi of a batch context decomposed alone on the grid-wide path: a
// context of its own over a copy of its CSR (local ids), the same stream and
// settings; core indices and rounds go straight into c->core / c->rnd.
// A context of its own over a copy of graph gi's CSR (local ids), on `stream`
// (NULL: c's stream) and with c's settings. Only reads c's graph, so several
// threads may make sub-contexts of one context at once (each on its own
// stream); failures are reported through the return value only.
khcore_status make_sub(khcore_ctx *c, int32_t gi, khcore_ctx **out, cudaStream_t stream = nullptr)
{
    *out = nullptr;
    cudaStream_t st = stream ? stream : c->stream;
    const int64_t v0 = c->v_off[gi];
    const int32_t ng = (int32_t)(c->v_off[gi + 1] - v0);
    std::vector<int32_t> rp((size_t)ng + 1);
    if (cudaMemcpyAsync(rp.data(), c->row_ptr + v0, sizeof(int32_t) * rp.size(), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return KHCORE_ECUDA;
    const int32_t e0 = rp[0];
    for (auto &x : rp) x -= e0;
    std::vector<int32_t> col((size_t)rp[ng]);
    if (!col.empty()) {
        if (cudaMemcpyAsync(col.data(), c->col + e0, sizeof(int32_t) * col.size(), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return KHCORE_ECUDA;
    }
    for (auto &x : col) x -= (int32_t)v0;
    khcore_ctx *sub = nullptr;
    khcore_status s = khcore_create(ng, rp.data(), col.empty() ? nullptr : col.data(), KHCORE_FLAG_TRUST_INPUT,
                                    st, &sub);
    if (s != KHCORE_OK) return s;
    sub->W_req = c->W_req;
    sub->W_av = c->W_av;
    sub->Wr_req = c->Wr_req;
    sub->push_alpha = c->push_alpha;
    sub->lazy = c->lazy;
    sub->update_mode = c->update_mode;
    sub->block = c->block;
    sub->init_alpha = c->init_alpha;
    sub->round_blocks = c->round_blocks;
    sub->round_loop = c->round_loop;
    sub->wait_limit_ns = c->wait_limit_ns;
    *out = sub;
    return KHCORE_OK;
}

// Graph gi of a batch context decomposed alone on the grid-wide path;
// core indices and rounds go straight into c->core / c->rnd.
khcore_status decompose_alone(khcore_ctx *c, int32_t gi, int32_t h, khcore_stats *sst)
{
    khcore_ctx *sub = nullptr;
    khcore_status s = make_sub(c, gi, &sub);
    if (s != KHCORE_OK) return fail(c, s, "graph %d alone: %s", gi, khcore_last_error(nullptr));
    const int64_t v0 = c->v_off[gi];
    s = decompose(sub, std::vector<int32_t>{h}, c->core + v0, c->rnd + v0, sst);
    if (s != KHCORE_OK) {
        const std::string msg = sub->err;
        if (s == KHCORE_ETIMEOUT) c->dirty = true;
        khcore_destroy(sub);
        return fail(c, s, "graph %d alone: %s", gi, msg.c_str());
    }
    khcore_destroy(sub);
    return KHCORE_OK;
}

// The decomposition driver. h_in[g] is the hop bound of graph g (g < c->G).
khcore_status decompose(khcore_ctx *c, const std::vector<int32_t> &h_in, int32_t *core_out, int32_t *round_out,
                        khcore_stats *stats)
{
    khcore_stats stt;
    std::memset(&stt, 0, sizeof stt);
    const int32_t G = c->G;
    // effective h per graph, h-classes (graphs with equal h), class regions
    std::vector<int32_t> hg(G), gcls(G);
    std::map<int32_t, int32_t> cls_of_h;
    int32_t hmax = 1;
    for (int32_t g = 0; g < G; g++) {
        hg[g] = effective_h(c->v_off[g + 1] - c->v_off[g], h_in[g]);
        hmax = std::max(hmax, hg[g]);
    }
    for (int32_t g = 0; g < G; g++) cls_of_h.emplace(hg[g], 0);
    std::vector<int32_t> cls_h;
    for (auto &kv : cls_of_h) {
        kv.second = (int32_t)cls_h.size();
        cls_h.push_back(kv.first);
    }
    const int32_t ncls = (int32_t)cls_h.size();
    std::vector<int64_t> cls_size(ncls, 0);
    for (int32_t g = 0; g < G; g++) {
        gcls[g] = cls_of_h[hg[g]];
        cls_size[gcls[g]] += c->v_off[g + 1] - c->v_off[g];
    }
    std::vector<int32_t> cls_off(ncls), cls_src((size_t)c->n);
    {
        int64_t o = 0;
        for (int32_t k = 0; k < ncls; k++) {
            cls_off[k] = (int32_t)o;
            o += cls_size[k];
        }
        std::vector<int64_t> fill(cls_off.begin(), cls_off.end());
        for (int32_t g = 0; g < G; g++)
            for (int64_t v = c->v_off[g]; v < c->v_off[g + 1]; v++) cls_src[fill[gcls[g]]++] = (int32_t)v;
    }
    stt.h = G == 1 ? hg[0] : hmax;
    if (c->n == 0) {
        if (stats) *stats = stt;
        return KHCORE_OK;
    }
    const int W = c->W_req ? c->W_req : (c->W_av ? c->W_av : auto_words(c->n));
    const int Wr = c->Wr_req ? c->Wr_req : (c->W_req ? c->W_req : auto_round_words(c->n));
    stt.words_per_vertex = W;
    stt.round_words = Wr;
    khcore_status s;
    if ((s = ensure_bfs(c, std::max(W, Wr))) != KHCORE_OK) return s;
    if ((s = clear_if_dirty(c)) != KHCORE_OK) return s;
    const GraphView g = c->view();
    const int grid = bfs_grid(c, Wr);

    PeelView pv;
    pv.G = G;
    pv.ncls = ncls;
    pv.gid = c->G > 1 ? c->gid : nullptr;
    pv.kg = c->kg;
    pv.ming = c->ming;
    pv.hg = c->hg;
    pv.cls = c->gcls;
    pv.cls_off = c->cls_off;
    pv.nAc = c->nAc;
    pv.nDc = c->nDc;
    // the paper's per-deletion update (one graph): exact h-degrees after every
    // round (no bounds), host-driven rounds
    const bool sampled = c->sampling_req && G == 1;
    const bool paper_update = c->update_mode == 1 && G == 1 && !(c->graph_blocks > 0) && !sampled;
    const bool lazy = c->lazy && !paper_update && !sampled;
    pv.slack = lazy ? c->slack : nullptr;
    pv.mind = lazy ? c->mind : nullptr;
    pv.minub = lazy ? c->minub : nullptr;
    pv.ncand = lazy ? c->ncand : nullptr;

    CU(cudaEventRecord(c->ev0, c->stream));
    PeelState init;
    std::memset(&init, 0, sizeof init);
    init.alive = c->n;
    init.m_alive = (unsigned long long)c->m;
    *c->st_host = init;
    c->level_ms = 0.0;
    c->level_launches = 0;
    c->timer.used = 0;
    std::vector<int32_t> ming_init(G, INT_MAX);
    CU(cudaMemcpyAsync(c->st, c->st_host, sizeof(PeelState), cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemsetAsync(c->kg, 0, sizeof(int32_t) * G, c->stream));
    CU(cudaMemcpyAsync(c->ming, ming_init.data(), sizeof(int32_t) * G, cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(c->mind, ming_init.data(), sizeof(int32_t) * G, cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(c->minub, ming_init.data(), sizeof(int32_t) * G, cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemsetAsync(c->ncand, 0, sizeof(int32_t) * G, c->stream));
    CU(cudaMemsetAsync(c->slack, 0, sizeof(int32_t) * (size_t)c->n, c->stream));
    CU(cudaMemsetAsync(c->wsum, 0, sizeof(int32_t) * (size_t)c->n, c->stream));
    CU(cudaMemcpyAsync(c->hg, hg.data(), sizeof(int32_t) * G, cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(c->gcls, gcls.data(), sizeof(int32_t) * G, cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(c->cls_off, cls_off.data(), sizeof(int32_t) * ncls, cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(c->clsh, cls_h.data(), sizeof(int32_t) * ncls, cudaMemcpyHostToDevice, c->stream));
    std::vector<int32_t> cls_size32(cls_size.begin(), cls_size.end());
    CU(cudaMemcpyAsync(c->cls_size, cls_size32.data(), sizeof(int32_t) * ncls, cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemsetAsync(c->inner, 0, sizeof(int32_t) * ncls, c->stream));
    CU(cudaMemcpyAsync(c->cls_src, cls_src.data(), sizeof(int32_t) * c->n, cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemsetAsync(c->edges, 0, sizeof(unsigned long long), c->stream));
    CU(cudaMemsetAsync(c->alg, 0, sizeof(unsigned long long), c->stream));
    CU(launch_alive_init(c->alive, c->n, c->stream));
    stt.kernel_launches += 1;
    // the host vectors above must outlive the async copies
    CU(cudaStreamSynchronize(c->stream));

    // Batches (mode 0 with G >= 2, or mode 1): graphs of at most
    // kBlockGraphsMaxN vertices (mode 1: all graphs) are decomposed whole by
    // one thread block each, in one launch with no grid-wide barrier
    // (khcore_block.cu); each larger graph then runs alone on the grid-wide
    // path, in a context of its own over a copy of its CSR.
    const bool all_blocks = c->graph_blocks > 0;
    if (all_blocks || (c->graph_blocks == 0 && G >= 2)) {
        std::vector<int32_t> small, large;
        for (int32_t gi = 0; gi < G; gi++)
            (all_blocks || c->v_off[gi + 1] - c->v_off[gi] <= c->block_graph_max ? small : large).push_back(gi);
        std::stable_sort(small.begin(), small.end(), [&](int32_t x, int32_t y) {
            return c->v_off[x + 1] - c->v_off[x] > c->v_off[y + 1] - c->v_off[y];
        });
        CU(cudaEventRecord(c->ev_init, c->stream));
        stt.words_per_vertex = 1;
        if (!small.empty()) {
            const int32_t ns = (int32_t)small.size();
            CU(cudaMemcpyAsync(c->order_d, small.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, c->stream));
            CU(cudaMemsetAsync(c->bnext, 0, sizeof(int32_t), c->stream));
            CU(cudaMemsetAsync(c->bstats, 0, sizeof(BlockStats), c->stream));
            BlockLaunch L;
            L.rp = c->row_ptr;
            L.col = c->col;
            L.voff = c->voff_d;
            L.hg = c->hg;
            L.order = c->order_d;
            L.count = ns;
            L.next = c->bnext;
            L.alive = c->alive;
            L.deg = c->deg;
            L.core = c->core;
            L.rnd = c->rnd;
            L.kg = c->kg;
            L.V = c->V;
            L.F0 = c->F[0];
            L.F1 = c->F[1];
            L.live0 = c->src;
            L.live1 = c->comb;
            L.qa = c->Q[0];
            L.qb = c->Q[1];
            L.tl = c->T;
            L.al = c->Q[2];
            L.dl = c->dcls;
            L.sl = c->cand;
            L.mark = c->slack;  // zero here (cleared above) and left zero
            L.dcount = c->dcount;
            L.edges = c->edges;
            L.bs = c->bstats;
            const int bgrid = std::min(ns, c->sm_count * max_blocks_per_sm_block_decompose());
            CU(launch_decompose_blocks(L, bgrid, c->stream));
            BlockStats bsh;
            CU(cudaMemcpyAsync(&bsh, c->bstats, sizeof bsh, cudaMemcpyDeviceToHost, c->stream));
            CU(cudaStreamSynchronize(c->stream));
            stt.kernel_launches += 1;
            stt.rounds = (int32_t)bsh.rounds;
            stt.source_batches += bsh.batches;
            stt.affected_total += bsh.affected;
            stt.recomputed_total += bsh.recomputed;
        }
        stt.deleted_total += c->n;
        khcore_stats sub_sum;
        std::memset(&sub_sum, 0, sizeof sub_sum);
        std::vector<int32_t> kg_large(large.size(), 0);
        auto add_stats = [&](const khcore_stats &sst) {
            stt.rounds = std::max(stt.rounds, sst.rounds);
            stt.source_batches += sst.source_batches;
            stt.kernel_launches += sst.kernel_launches;
            stt.affected_total += sst.affected_total;
            stt.recomputed_total += sst.recomputed_total;
            sub_sum.edges_traversed += sst.edges_traversed;
            sub_sum.level_bytes += sst.level_bytes;
            sub_sum.round_bytes += sst.round_bytes;
        };
        const int K = (int)std::min<size_t>(std::max(c->concurrent, 1), large.size());
        if (K <= 1) {
            for (size_t i = 0; i < large.size(); i++) {
                khcore_stats sst;
                if ((s = decompose_alone(c, large[i], h_in[large[i]], &sst)) != KHCORE_OK) return s;
                kg_large[i] = sst.k_max;
                add_stats(sst);
            }
        } else {
            // K larger graphs at a time, each in a context of its own on its
            // own stream, its round kernel on sm_count / K SMs: one graph's
            // rounds are latency-bound and leave most of the GPU idle
            std::atomic<size_t> next{0};
            std::mutex mu;
            khcore_status first = KHCORE_OK;
            std::string first_msg;
            auto worker = [&]() {
                cudaSetDevice(c->device);
                cudaStream_t st = nullptr;
                if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
                    std::lock_guard<std::mutex> lk(mu);
                    if (first == KHCORE_OK) {
                        first = KHCORE_ECUDA;
                        first_msg = "cudaStreamCreate failed";
                    }
                    return;
                }
                for (;;) {
                    {
                        std::lock_guard<std::mutex> lk(mu);
                        if (first != KHCORE_OK) break;
                    }
                    const size_t i = next++;
                    if (i >= large.size()) break;
                    const int32_t gi = large[i];
                    khcore_ctx *sub = nullptr;
                    khcore_status ws = make_sub(c, gi, &sub, st);
                    khcore_stats sst;
                    std::memset(&sst, 0, sizeof sst);
                    std::string msg;
                    if (ws == KHCORE_OK) {
                        sub->persist_sms = std::max(1, c->sm_count / K);
                        const int64_t v0 = c->v_off[gi];
                        ws = decompose(sub, std::vector<int32_t>{h_in[gi]}, c->core + v0, c->rnd + v0, &sst);
                        if (ws != KHCORE_OK) msg = sub->err;
                    } else {
                        msg = khcore_last_error(nullptr);
                    }
                    khcore_destroy(sub);
                    std::lock_guard<std::mutex> lk(mu);
                    if (ws != KHCORE_OK) {
                        if (first == KHCORE_OK) {
                            first = ws;
                            char buf[64];
                            snprintf(buf, sizeof buf, "graph %d: ", gi);
                            first_msg = buf + msg;
                        }
                        break;
                    }
                    kg_large[i] = sst.k_max;
                    add_stats(sst);
                }
                cudaStreamDestroy(st);
            };
            std::vector<std::thread> pool;
            for (int t = 0; t < K; t++) pool.emplace_back(worker);
            for (auto &t : pool) t.join();
            if (first != KHCORE_OK) {
                if (first == KHCORE_ETIMEOUT) c->dirty = true;
                return fail(c, first, "%s", first_msg.c_str());
            }
        }
        for (size_t i = 0; i < large.size(); i++)
            CU(cudaMemcpyAsync(c->kg + large[i], &kg_large[i], sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
        if ((s = finish_decompose(c, G, core_out, round_out, stats, stt, true)) != KHCORE_OK) return s;
        if (stats) {
            stats->edges_traversed += sub_sum.edges_traversed;
            stats->level_bytes += sub_sum.level_bytes;
            stats->round_bytes += sub_sum.round_bytes;
        }
        return KHCORE_OK;
    }

    // initial h-degrees, class by class
    for (int32_t k = 0; k < ncls; k++)
        if ((s = hdeg_sources(c, W, cls_h[k], c->cls_src + cls_off[k], (int32_t)cls_size[k], c->n, c->m, &stt,
                              nullptr, 0, nullptr, true)) !=
            KHCORE_OK)
            return s;

    CU(cudaEventRecord(c->ev_init, c->stream));
    unsigned long long init_alg = 0;
    CU(cudaMemcpyAsync(&init_alg, c->alg, sizeof init_alg, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    stt.level_bytes = (double)init_alg;  // the initial pass
    if (sampled) {
        // Algorithm 5: select = |N_v^h cap S| of every vertex (d0 = the exact
        // h-degrees just computed), then the estimates start at d0
        CU(cudaMemcpyAsync(c->s_d0, c->deg, sizeof(int32_t) * (size_t)c->n, cudaMemcpyDeviceToDevice, c->stream));
        c->sampling = 1;
        s = hdeg_sources(c, W, cls_h[0], c->cls_src, c->n, c->n, c->m, &stt, nullptr, 0, nullptr, true);
        c->sampling = 2;
        if (s != KHCORE_OK) {
            c->sampling = 0;
            return s;
        }
        CU(launch_sample_init(c->s_sel0, c->s_d0, c->s_sel, c->n, c->stream));
        stt.kernel_launches++;
    }
    struct SamplingOff {  // the context leaves sampling mode on every return
        khcore_ctx *c;
        ~SamplingOff() { c->sampling = 0; }
    } sampling_off{c};
    // resident blocks per SM of the round kernel (W = 4): one while the
    // rounds are latency-bound (h <= 2), two for the larger BFS levels of h >= 3
    const int minb = c->round_blocks ? c->round_blocks : (hmax >= 3 ? 2 : 1);
    const int pgrid = (c->round_loop == 0 && !paper_update && !sampled)
                          ? (c->persist_sms ? std::min(c->persist_sms, c->sm_count) : c->sm_count) *
                                max_blocks_per_sm_persist(Wr, minb)
                          : 0;
    if (pgrid > 0) {
        // the whole decomposition in one cooperative launch
        PersistLaunch L;
        L.g = g;
        L.alive = c->alive;
        L.deg = c->deg;
        L.core = c->core;
        L.rnd = c->rnd;
        L.p = pv;
        L.st = c->st;
        L.b.V = c->V;
        L.b.F[0] = c->F[0];
        L.b.F[1] = c->F[1];
        L.b.flag[0] = c->flag[0];
        L.b.flag[1] = c->flag[1];
        for (int k = 0; k < 3; k++) {
            L.b.Q[k] = c->Q[k];
            L.b.I[k] = c->I[k];
            L.aq[k] = c->Q[k];  // the affected-BFS ring reuses the BFS frontier lists
        }
        L.b.T = c->T;
        L.b.ctl = c->ctl;
        L.b.cnt = c->cnt;
        L.b.edges = c->edges;
        L.b.Fx = c->Fx;
        L.b.flagx = c->flagx;
        L.b.tflag = c->tflag;
        L.b.rowcnt = nullptr;
        L.b.row_first = 0;
        L.b.row_sign = 1;
        L.b.newcnt = nullptr;
        L.b.alg_bytes = c->alg;
        L.b.slev = nullptr;
        L.b.cum = nullptr;
        L.b.hcnt = 0;
        L.b.boff = 0;
        L.b.wsum = nullptr;
        L.b.wdeg = c->deg;
        L.b.in_s = nullptr;
        L.b.fullmask = nullptr;
        L.b.sel0 = nullptr;
        L.b.sel = nullptr;
        L.b.d0 = nullptr;
        L.wsum = lazy ? c->wsum : nullptr;
        L.vis = c->vis;
        L.A = c->src;
        L.dcls = c->dcls;
        L.cls_src = c->cls_src;
        L.cls_h = c->clsh;
        L.cls_size = c->cls_size;
        L.cls_off = c->cls_off;
        L.inner = c->inner;
        L.dcount = c->dcount;
        L.comb = c->comb;
        L.cand = c->cand;
        L.ncls = ncls;
        L.hmax = hmax;
        L.alpha = c->push_alpha;
        L.gs = c->gs;
        L.ps = c->pstats;
        L.timeout_ns = c->wait_limit_ns;
        CU(cudaMemsetAsync(c->gs, 0, sizeof(GridSync), c->stream));
        CU(cudaMemsetAsync(c->pstats, 0, sizeof(PersistStats), c->stream));
        CU(launch_decompose_persist(Wr, L, pgrid, c->stream, minb));
        GridSync gsh;
        PersistStats psh;
        CU(cudaMemcpyAsync(&gsh, c->gs, sizeof gsh, cudaMemcpyDeviceToHost, c->stream));
        CU(cudaMemcpyAsync(&psh, c->pstats, sizeof psh, cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
        if (gsh.err) {
            c->dirty = true;
            return fail(c, KHCORE_ETIMEOUT, "a grid-barrier wait exceeded %.3f s; the decomposition stopped",
                        (double)c->wait_limit_ns * 1e-9);
        }
        stt.kernel_launches += 1;
        stt.rounds = (int32_t)psh.rounds;
        stt.source_batches += psh.source_batches;
        stt.recomputed_total += psh.recomputed_total;
        stt.deleted_total += psh.deleted_total;
        stt.affected_total += psh.affected_total;
        for (int k = 0; k < 5; k++) stt.phase_ms[k] = (double)psh.phase_ns[k] * 1e-6;
        stt.grid_barriers = (int64_t)gsh.passed;
        stt.round_blocks = minb;
        return finish_decompose(c, G, core_out, round_out, stats, stt, true);
    }


    // KHCORE_TRACE=1 prints one line per peel round to stderr (tracing aid)
    const char *trace_env = getenv("KHCORE_TRACE");
    const bool trace = trace_env && trace_env[0] == '1';
    int32_t round = 0;
    for (;;) {
        // one round: levels, peel sets D, affected sets A, recompute deg[A];
        // the affected-BFS frontier lists reuse the BFS frontier lists Q[0..2]
        CU(launch_min_alive_deg(g, c->alive, c->deg, pv, grid, c->stream));
        if (lazy) {
            // exact recompute of the vertices whose bounds leave their fate open
            CU(launch_refine_select(g, c->alive, c->deg, pv, c->cand, grid, c->stream));
            CU(cudaMemcpyAsync(c->nAc_host + 3 * G, c->ncand, sizeof(int32_t) * ncls, cudaMemcpyDeviceToHost,
                               c->stream));
            CU(cudaStreamSynchronize(c->stream));
            stt.kernel_launches++;
            for (int32_t k = 0; k < ncls; k++) {
                const int32_t nc = c->nAc_host[3 * G + k];
                if (nc <= 0) continue;
                if ((s = hdeg_sources(c, Wr, cls_h[k], c->cand + cls_off[k], nc, c->st_host->alive,
                                      (int64_t)c->st_host->m_alive, &stt)) != KHCORE_OK)
                    return s;
                stt.recomputed_total += nc;
                CU(launch_min_over_list(c->cand + cls_off[k], nc, c->deg, pv, c->stream));
                stt.kernel_launches++;
            }
        }
        CU(launch_set_level(pv, c->st, c->stream));
        if (paper_update) {
            // D marked (core, round) but kept alive; then deleted one after
            // the other by the paper's update, unless a ball is over the
            // slots' limits (then the BFS recompute below handles the round)
            CU(launch_peel_mark(c->n, c->alive, c->deg, c->kg, c->st, c->core, c->rnd, c->upd_ready ? c->upd.cand[0]
                                                                                                     : c->comb,
                                grid, c->stream));
            CU(cudaMemcpyAsync(c->st_host, c->st, sizeof(PeelState), cudaMemcpyDeviceToHost, c->stream));
            CU(cudaStreamSynchronize(c->stream));
            stt.kernel_launches += 3;
            const int32_t nd = c->st_host->nD;
            if (nd <= 0) return fail(c, KHCORE_EINTERNAL, "round %d deleted no vertex", round);
            bool fit = false;
            if (c->upd_ready) {
                if ((s = update_deleted(c, hg[0], nd, c->st, &fit, &stt.kernel_launches)) != KHCORE_OK) return s;
            } else if (nd <= kUpdSlots && hg[0] <= kUpdMaxH) {
                // first use: allocate the slots, then list D again into them
                if ((s = ensure_upd(c)) != KHCORE_OK) return s;
                CU(cudaMemcpyAsync(c->upd.cand[0], c->comb, sizeof(int32_t) * nd, cudaMemcpyDeviceToDevice,
                                   c->stream));
                if ((s = update_deleted(c, hg[0], nd, c->st, &fit, &stt.kernel_launches)) != KHCORE_OK) return s;
            }
            if (fit) {
                CU(cudaMemcpyAsync(c->st_host, c->st, sizeof(PeelState), cudaMemcpyDeviceToHost, c->stream));
                CU(cudaStreamSynchronize(c->stream));
                stt.deleted_total += nd;
                round++;
                if (c->st_host->alive == 0) break;
                c->st_host->round = round;
                CU(cudaMemcpyAsync(&c->st->round, &c->st_host->round, sizeof(int32_t), cudaMemcpyHostToDevice,
                                   c->stream));
                continue;
            }
            // over the limits: the compaction below selects the same D
            CU(cudaMemsetAsync(&c->st->nD, 0, sizeof(int32_t), c->stream));
        }
        CU(launch_peel_compact(g, c->alive, c->deg, pv, c->st, c->core, c->rnd, c->vis, c->Q[0], c->dcls, grid,
                               c->stream));
        stt.kernel_launches += 3;
        for (int lvl = 0; lvl < hmax; lvl++) {
            CU(launch_snapshot_inner(pv, c->clsh, lvl, c->inner, c->stream));
            CU(launch_affected_level(g, c->alive, lvl, c->Q, c->vis, pv, c->st, c->src, lvl == hmax - 1, grid,
                                     c->stream));
            stt.kernel_launches += 2;
        }
        CU(launch_sum_classes(pv, c->st, c->stream));
        stt.kernel_launches++;
        CU(cudaMemcpyAsync(c->st_host, c->st, sizeof(PeelState), cudaMemcpyDeviceToHost, c->stream));
        CU(cudaMemcpyAsync(c->nAc_host, c->nAc, sizeof(int32_t) * ncls, cudaMemcpyDeviceToHost, c->stream));
        CU(cudaMemcpyAsync(c->nAc_host + G, c->inner, sizeof(int32_t) * ncls, cudaMemcpyDeviceToHost, c->stream));
        CU(cudaMemcpyAsync(c->nAc_host + 2 * G, c->nDc, sizeof(int32_t) * ncls, cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
        const PeelState ps = *c->st_host;
        if (ps.nD <= 0)
            return fail(c, KHCORE_EINTERNAL, "round %d deleted no vertex with %d alive", round, ps.alive);
        stt.deleted_total += ps.nD;
        stt.affected_total += ps.nA;
        if (trace) {
            float tms = 0.f;
            cudaEventRecord(c->ev1, c->stream);
            cudaEventSynchronize(c->ev1);
            cudaEventElapsedTime(&tms, c->ev0, c->ev1);
            fprintf(stderr, "khcore round %d: |D|=%d |A|=%d alive=%d m_alive=%llu t=%.1f ms\n", round, ps.nD, ps.nA,
                    ps.alive, (unsigned long long)ps.m_alive, tms);
        }
        round++;
        if (ps.alive == 0) break;
        // Affected vertices closer than h to D get their h-degree recomputed;
        // those exactly h away lose exactly the deleted vertices within h
        // (Observation 2 with s = h), counted by a BFS from D (row counts),
        // or 1 when a single vertex went.
        for (int32_t k = 0; k < ncls; k++) {
            const int32_t na = c->nAc_host[k];
            // sampling: every affected vertex is recounted (its estimate
            // depends on which sampled vertices it still reaches)
            const int32_t ni = sampled ? na : std::min(c->nAc_host[G + k], na);
            const int32_t nd = c->nAc_host[2 * G + k];
            if (na == 0) continue;
            const bool single = (ps.nD == 1);  // every affected vertex loses exactly that one
            if (lazy) {
                // row counts of the deleted set; bounds for the inner vertices
                if (!single && (s = hdeg_sources(c, Wr, cls_h[k], c->dcls + cls_off[k], nd, ps.alive,
                                                 (int64_t)ps.m_alive, &stt, c->dcount, 0, c->wsum)) != KHCORE_OK)
                    return s;
                CU(launch_apply_lazy(c->src + cls_off[k], ni, na, single ? nullptr : c->dcount, c->deg, c->slack,
                                     ni + nd, c->wsum, c->dcls + cls_off[k], c->row_ptr, cls_h[k], c->stream));
                stt.kernel_launches++;
                continue;
            }
            const bool count_d = na > ni && !single;
            // one source list: the inner vertices (their h-degrees) and, after
            // them, the deleted vertices (row counts on the outer shell)
            const int32_t total = ni + (count_d ? nd : 0);
            if (total > 0) {
                CU(launch_concat(c->comb, c->src + cls_off[k], ni, c->dcls + cls_off[k], count_d ? nd : 0, c->stream));
                if ((s = hdeg_sources(c, Wr, cls_h[k], c->comb, total, ps.alive, (int64_t)ps.m_alive, &stt,
                                      count_d ? c->dcount : nullptr, ni)) != KHCORE_OK)
                    return s;
            }
            stt.recomputed_total += ni;
            if (na > ni) {
                CU(launch_apply_dcount(c->src + cls_off[k], ni, na, single ? nullptr : c->dcount, c->deg, c->stream));
                stt.kernel_launches += 2;
            }
        }
        // advance the device-side round counter
        c->st_host->round = round;
        CU(cudaMemcpyAsync(&c->st->round, &c->st_host->round, sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    }
    stt.rounds = round;
    return finish_decompose(c, G, core_out, round_out, stats, stt, false);
}

khcore_status create_common(int32_t G, const std::vector<int64_t> &v_off, std::vector<int32_t> &rp,
                            std::vector<int32_t> &cl, const std::vector<int32_t> *gid, void *stream,
                            khcore_ctx **out)
{
    arm_alloc_injection();
    khcore_ctx *c = new (std::nothrow) khcore_ctx();
    if (!c) return fail(nullptr, KHCORE_ENOMEM, "host allocation failed");
    c->n = (int32_t)v_off[G];
    c->m = rp[c->n];
    c->G = G;
    c->v_off = v_off;
    khcore_status st = setup_ctx(c, rp, cl, gid, stream);
    if (st != KHCORE_OK) {
        khcore_destroy(c);
        return st;
    }
    *out = c;
    return KHCORE_OK;
}

}  // namespace

namespace khc {

// Failure message for khcore_last_error(NULL), for the entry points that take
// no context.
khcore_status set_thread_error(khcore_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_create_err = buf;
    return s;
}

}  // namespace khc

extern "C" {

const char *khcore_status_string(khcore_status s)
{
    switch (s) {
    case KHCORE_OK: return "KHCORE_OK";
    case KHCORE_EINVAL: return "KHCORE_EINVAL";
    case KHCORE_ENOMEM: return "KHCORE_ENOMEM";
    case KHCORE_ECUDA: return "KHCORE_ECUDA";
    case KHCORE_ETIMEOUT: return "KHCORE_ETIMEOUT";
    case KHCORE_EBUSY: return "KHCORE_EBUSY";
    case KHCORE_EINTERNAL: return "KHCORE_EINTERNAL";
    }
    return "KHCORE_UNKNOWN";
}

const char *khcore_last_error(const khcore_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

int32_t khcore_num_vertices(const khcore_ctx *ctx) { return ctx ? ctx->n : 0; }
int64_t khcore_num_entries(const khcore_ctx *ctx) { return ctx ? ctx->m : 0; }
int32_t khcore_num_graphs(const khcore_ctx *ctx) { return ctx ? ctx->G : 0; }

void khcore_destroy(khcore_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream && !c->failed) cudaStreamSynchronize(c->stream);
    void *bufs[] = {c->row_ptr, c->col, c->classes, c->gid, c->kg, c->ming, c->hg, c->gcls, c->cls_off, c->nAc,
                    c->nDc, c->inner, c->clsh, c->dcls, c->dcount, c->comb, c->slack, c->wsum, c->cand, c->voff_d, c->order_d, c->bnext, c->bstats, c->mind, c->minub, c->ncand, c->cls_size, c->gs, c->pstats,
                    c->cls_src, c->alive, c->deg, c->core, c->rnd, c->src, c->vis, c->st, c->V, c->F[0], c->F[1],
                    c->Fx, c->flagx, c->tflag, c->flag[0], c->flag[1], c->Q[0], c->Q[1], c->Q[2], c->I[0], c->I[1], c->I[2], c->T, c->ctl,
                    c->cnt, c->edges, c->alg};
    for (void *p : bufs) cudaFree(p);
    void *sbufs[] = {c->s_in, c->s_sel0, c->s_sel, c->s_d0, c->s_full, c->class_counts, c->classes_av};
    for (void *p : sbufs) cudaFree(p);
    void *ubufs[] = {c->upd.vis, c->upd.list, c->upd.dist, c->upd.reach, c->upd.meta, c->upd.owner, c->upd.lab,
                     c->upd.done, c->upd.flag, c->upd.cand[0], c->upd.cand[1]};
    for (void *p : ubufs) cudaFree(p);
    for (cudaEvent_t e : c->tev) cudaEventDestroy(e);
    if (c->st_host) cudaFreeHost(c->st_host);
    if (c->nAc_host) cudaFreeHost(c->nAc_host);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->ev_init) cudaEventDestroy(c->ev_init);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    (void)cudaGetLastError();
    delete c;
}

khcore_status khcore_create(int32_t n, const int32_t *row_ptr, const int32_t *col, uint32_t flags, void *stream,
                            khcore_ctx **out)
{
    if (!out) return fail(nullptr, KHCORE_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 0) return fail(nullptr, KHCORE_EINVAL, "n must be >= 0 (got %d)", n);
    if (!row_ptr) return fail(nullptr, KHCORE_EINVAL, "row_ptr is NULL");

    std::vector<int32_t> rp, cl, sorted;
    if (fetch(rp, row_ptr, (size_t)n + 1) != cudaSuccess) return fail(nullptr, KHCORE_ECUDA, "cannot read row_ptr");
    const int64_t m = rp[n];
    if (m < 0) return fail(nullptr, KHCORE_EINVAL, "row_ptr[n] is negative");
    if (m > 0 && !col) return fail(nullptr, KHCORE_EINVAL, "col is NULL but row_ptr[n] = %lld", (long long)m);
    if (fetch(cl, col, (size_t)m) != cudaSuccess) return fail(nullptr, KHCORE_ECUDA, "cannot read col");
    if (!(flags & KHCORE_FLAG_TRUST_INPUT)) {
        std::string msg;
        if (!validate_csr(n, rp, cl, sorted, msg)) return fail(nullptr, KHCORE_EINVAL, "invalid CSR: %s", msg.c_str());
    } else {
        sorted.swap(cl);
    }
    std::vector<int64_t> v_off = {0, n};
    return create_common(1, v_off, rp, sorted, nullptr, stream, out);
}

khcore_status khcore_batch_create(int32_t G, const int64_t *v_off, const int64_t *e_off, const int32_t *row_ptr_local,
                                  const int32_t *col_local, uint32_t flags, void *stream, khcore_ctx **out)
{
    if (!out) return fail(nullptr, KHCORE_EINVAL, "out is NULL");
    *out = nullptr;
    if (G < 1) return fail(nullptr, KHCORE_EINVAL, "G must be >= 1 (got %d)", G);
    if (!v_off || !e_off || !row_ptr_local) return fail(nullptr, KHCORE_EINVAL, "NULL offset or row_ptr array");
    std::vector<int64_t> vo, eo;
    if (fetch(vo, v_off, (size_t)G + 1) != cudaSuccess || fetch(eo, e_off, (size_t)G + 1) != cudaSuccess)
        return fail(nullptr, KHCORE_ECUDA, "cannot read offsets");
    if (vo[0] != 0 || eo[0] != 0) return fail(nullptr, KHCORE_EINVAL, "v_off[0] and e_off[0] must be 0");
    for (int32_t g = 0; g < G; g++)
        if (vo[g + 1] < vo[g] || eo[g + 1] < eo[g])
            return fail(nullptr, KHCORE_EINVAL, "offsets decrease at graph %d", g);
    if (vo[G] > INT32_MAX || eo[G] > INT32_MAX)
        return fail(nullptr, KHCORE_EINVAL, "batch too large for int32 ids (%lld vertices, %lld entries)",
                    (long long)vo[G], (long long)eo[G]);
    const int32_t n = (int32_t)vo[G];
    const int64_t m = eo[G];
    std::vector<int32_t> rpl, cll;
    if (fetch(rpl, row_ptr_local, (size_t)n + G) != cudaSuccess)
        return fail(nullptr, KHCORE_ECUDA, "cannot read row_ptr");
    if (m > 0 && !col_local) return fail(nullptr, KHCORE_EINVAL, "col_local is NULL");
    if (fetch(cll, col_local, (size_t)m) != cudaSuccess) return fail(nullptr, KHCORE_ECUDA, "cannot read col");
    // the union graph: global ids, one CSR; each graph validated on its own
    std::vector<int32_t> rp((size_t)n + 1), cl((size_t)m), gid((size_t)n);
    for (int32_t g = 0; g < G; g++) {
        const int32_t ng = (int32_t)(vo[g + 1] - vo[g]);
        const int64_t mg = eo[g + 1] - eo[g];
        const int32_t *lrp = rpl.data() + vo[g] + g;
        if (lrp[ng] != mg)
            return fail(nullptr, KHCORE_EINVAL, "graph %d: row_ptr[n_g] = %d but e_off gives %lld entries", g,
                        lrp[ng], (long long)mg);
        std::vector<int32_t> lr(lrp, lrp + ng + 1), lc(cll.begin() + eo[g], cll.begin() + eo[g + 1]), ls;
        if (!(flags & KHCORE_FLAG_TRUST_INPUT)) {
            std::string msg;
            if (!validate_csr(ng, lr, lc, ls, msg))
                return fail(nullptr, KHCORE_EINVAL, "graph %d: invalid CSR: %s", g, msg.c_str());
        } else {
            ls.swap(lc);
        }
        for (int32_t i = 0; i < ng; i++) {
            rp[vo[g] + i] = (int32_t)(eo[g] + lr[i]);
            gid[vo[g] + i] = g;
        }
        for (int64_t k = 0; k < mg; k++) cl[eo[g] + k] = (int32_t)(vo[g] + ls[k]);
    }
    rp[n] = (int32_t)m;
    return create_common(G, vo, rp, cl, &gid, stream, out);
}

khcore_status khcore_set_words(khcore_ctx *c, int32_t words)
{
    if (!c) return KHCORE_EINVAL;
    if (words != 0 && words != 1 && words != 2 && words != 4 && words != 8 && words != 16)
        return fail(c, KHCORE_EINVAL, "words must be 0, 1, 2, 4, 8 or 16 (got %d)", words);
    c->W_req = words;
    return KHCORE_OK;
}

khcore_status khcore_set_round_words(khcore_ctx *c, int32_t words)
{
    if (!c) return KHCORE_EINVAL;
    if (words != 0 && words != 1 && words != 2 && words != 4 && words != 8 && words != 16)
        return fail(c, KHCORE_EINVAL, "words must be 0, 1, 2, 4, 8 or 16 (got %d)", words);
    c->Wr_req = words;
    return KHCORE_OK;
}

khcore_status khcore_set_push_alpha(khcore_ctx *c, int32_t alpha)
{
    if (!c) return KHCORE_EINVAL;
    if (alpha < 0) return fail(c, KHCORE_EINVAL, "alpha must be >= 0 (got %d)", alpha);
    c->push_alpha = alpha;
    c->init_alpha = 0;  // the all-vertex pass follows
    return KHCORE_OK;
}

khcore_status khcore_set_lazy(khcore_ctx *c, int32_t on)
{
    if (!c) return KHCORE_EINVAL;
    c->lazy = on != 0;
    return KHCORE_OK;
}

namespace {

// Rebuild a degree-class list (the rounds' when all_vertex is false, else the
// all-vertex pass's own).
khcore_status build_classes(khcore_ctx *c, int32_t light_max, int32_t medium_max, bool all_vertex)
{
    if (!c->class_counts) CU(dev_alloc(&c->class_counts, 6));
    if (all_vertex && !c->classes_av) CU(dev_alloc(&c->classes_av, (size_t)std::max(c->n, 1)));
    int32_t *dst = all_vertex ? c->classes_av : c->classes;
    int32_t cnt[3] = {0, 0, 0};
    CU(launch_degree_classes(c->row_ptr, c->n, light_max, medium_max, dst, c->class_counts, c->stream));
    CU(cudaMemcpyAsync(cnt, c->class_counts, sizeof cnt, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (all_vertex) {
        c->n_light_av = cnt[0];
        c->n_medium_av = cnt[1];
        c->n_heavy_av = cnt[2];
    } else {
        c->n_light = cnt[0];
        c->n_medium = cnt[1];
        c->n_heavy = cnt[2];
        c->light_max = light_max;
        c->medium_max = medium_max;
    }
    return KHCORE_OK;
}

}  // namespace

khcore_status khcore_set_degree_classes(khcore_ctx *c, int32_t light_max, int32_t medium_max)
{
    khcore_status s;
    if ((s = check_ctx(c)) != KHCORE_OK) return s;
    if (light_max < 0 || medium_max < light_max)
        return fail(c, KHCORE_EINVAL, "degree classes need 0 <= light_max <= medium_max (got %d, %d)", light_max,
                    medium_max);
    if ((s = build_classes(c, light_max, medium_max, false)) != KHCORE_OK) return s;
    cudaFree(c->classes_av);  // every BFS of the context uses these lists now
    c->classes_av = nullptr;
    return KHCORE_OK;
}

khcore_status khcore_set_block_size(khcore_ctx *c, int32_t threads)
{
    if (!c || (threads != 128 && threads != 256 && threads != 512)) return KHCORE_EINVAL;
    c->block = threads;
    return KHCORE_OK;
}

khcore_status khcore_set_round_blocks(khcore_ctx *c, int32_t blocks)
{
    if (!c || blocks < 0 || blocks > 2) return KHCORE_EINVAL;
    c->round_blocks = blocks;
    return KHCORE_OK;
}

khcore_status khcore_set_round_sms(khcore_ctx *c, int32_t sms)
{
    if (!c || sms < 0 || sms > c->sm_count) return KHCORE_EINVAL;
    c->persist_sms = sms;
    return KHCORE_OK;
}

khcore_status khcore_set_concurrent_graphs(khcore_ctx *c, int32_t k)
{
    if (!c || k < 1 || k > 64) return KHCORE_EINVAL;
    c->concurrent = k;
    return KHCORE_OK;
}

khcore_status khcore_set_block_graph_max(khcore_ctx *c, int32_t nmax)
{
    if (!c || nmax < 0) return KHCORE_EINVAL;
    c->block_graph_max = nmax;
    return KHCORE_OK;
}

namespace {

// One line of the tuning cache: {"key": "...", "words": W, ...}.
bool cache_lookup(const char *path, const std::string &key, khcore_tuning *t)
{
    FILE *f = path ? fopen(path, "r") : nullptr;
    if (!f) return false;
    char line[1024];
    bool found = false;
    const std::string want = "\"key\": \"" + key + "\"";
    while (fgets(line, sizeof line, f)) {
        if (!strstr(line, want.c_str())) continue;
        khcore_tuning r;
        std::memset(&r, 0, sizeof r);
        auto num = [&](const char *name, int32_t *dst) {
            const std::string tag = std::string("\"") + name + "\": ";
            const char *p = strstr(line, tag.c_str());
            return p && sscanf(p + tag.size(), "%d", dst) == 1;
        };
        if (num("words", &r.words) && num("block", &r.block) && num("light_max", &r.light_max) &&
            num("medium_max", &r.medium_max) && num("push_alpha", &r.push_alpha) &&
            num("block_graph_max", &r.block_graph_max)) {
            *t = r;  // the last matching line wins
            found = true;
        }
    }
    fclose(f);
    return found;
}

void cache_store(const char *path, const std::string &key, const khcore_tuning &t)
{
    FILE *f = path ? fopen(path, "a") : nullptr;
    if (!f) return;
    fprintf(f,
            "{\"key\": \"%s\", \"words\": %d, \"block\": %d, \"light_max\": %d, \"medium_max\": %d, "
            "\"push_alpha\": %d, \"block_graph_max\": %d, \"trial_ms\": %.3f}\n",
            key.c_str(), t.words, t.block, t.light_max, t.medium_max, t.push_alpha, t.block_graph_max, t.trial_ms);
    fclose(f);
}

int ilog2(int64_t x)
{
    int l = 0;
    while (x > 1) {
        x >>= 1;
        l++;
    }
    return l;
}

}  // namespace

khcore_status khcore_autotune(khcore_ctx *c, int32_t h, const char *cache_path, khcore_tuning *out)
{
    khcore_status s;
    if ((s = check_ctx(c)) != KHCORE_OK) return s;
    if (h < 1) return fail(c, KHCORE_EINVAL, "h must be >= 1 (got %d)", h);
    khcore_tuning t;
    std::memset(&t, 0, sizeof t);
    t.words = c->W_req ? c->W_req : (c->W_av ? c->W_av : auto_words(c->n));
    t.block = c->block;
    t.light_max = c->light_max;
    t.medium_max = c->medium_max;
    t.push_alpha = c->init_alpha ? c->init_alpha : c->push_alpha;
    t.block_graph_max = c->block_graph_max;
    if (c->n == 0) {
        if (out) *out = t;
        return KHCORE_OK;
    }
    // cache key: the GPU, the graph's size classes and h
    cudaDeviceProp prop;
    CU(cudaGetDeviceProperties(&prop, c->device));
    std::vector<int32_t> rp;
    CU(fetch(rp, c->row_ptr, (size_t)c->n + 1));
    int64_t dmax = 0;
    for (int32_t v = 0; v < c->n; v++) dmax = std::max<int64_t>(dmax, rp[v + 1] - rp[v]);
    const int32_t he = effective_h(c->n, h);
    char kb[512];
    snprintf(kb, sizeof kb, "%s|G:%d|n:2^%d|m:2^%d|dmax:2^%d|h:%d", prop.name, c->G, ilog2(c->n), ilog2(c->m + 1),
             ilog2(dmax + 1), he);
    const std::string key = kb;
    khcore_tuning cached;
    if (cache_lookup(cache_path, key, &cached)) {
        t = cached;
        t.from_cache = 1;
    } else if (c->G == 1) {
        // The all-vertex pass decides the one-graph knobs: time it on the
        // first S vertices as sources (4 batches of the widest W), knob by
        // knob, keeping the best value of each before tuning the next. The
        // h-degrees of every trial must agree (results do not depend on the
        // knobs).
        const int32_t S = std::min<int32_t>(c->n, 4096);
        if ((s = ensure_bfs(c, 16)) != KHCORE_OK) return s;
        if ((s = clear_if_dirty(c)) != KHCORE_OK) return s;
        CU(launch_alive_init(c->alive, c->n, c->stream));
        CU(launch_iota(c->comb, S, c->stream));
        std::vector<int32_t> ref, got;
        cudaEvent_t e0, e1;
        CU(cudaEventCreate(&e0));
        CU(cudaEventCreate(&e1));
        auto trial = [&](const khcore_tuning &k, float *ms) -> khcore_status {
            khcore_status st;
            if ((st = build_classes(c, k.light_max, k.medium_max, true)) != KHCORE_OK) return st;
            c->block = k.block;
            c->init_alpha = k.push_alpha;
            float best = 1e30f;
            for (int rep = 0; rep < 2; rep++) {
                CU(cudaEventRecord(e0, c->stream));
                if ((st = hdeg_sources(c, k.words, he, c->comb, S, c->n, c->m, nullptr, nullptr, 0, nullptr, true)) !=
                    KHCORE_OK)
                    return st;
                CU(cudaEventRecord(e1, c->stream));
                CU(cudaEventSynchronize(e1));
                float m = 0.f;
                CU(cudaEventElapsedTime(&m, e0, e1));
                best = std::min(best, m);
            }
            got.resize(S);
            CU(cudaMemcpy(got.data(), c->deg, sizeof(int32_t) * S, cudaMemcpyDeviceToHost));
            if (ref.empty()) ref = got;
            else if (got != ref) return fail(c, KHCORE_EINTERNAL, "autotune: h-degrees differ between settings");
            *ms = best;
            t.trials++;
            t.trial_ms += best;
            return KHCORE_OK;
        };
        const int32_t cand_words[] = {4, 8, 16}, cand_block[] = {128, 256, 512};
        const int32_t cand_light[] = {16, 32, 64}, cand_medium[] = {256, 1024, 4096}, cand_alpha[] = {4, 16, 64};
        struct Knob {
            int32_t khcore_tuning::*field;
            const int32_t *cand;
            int count;
        } knobs[] = {{&khcore_tuning::words, cand_words, 3},       {&khcore_tuning::block, cand_block, 3},
                     {&khcore_tuning::light_max, cand_light, 3},   {&khcore_tuning::medium_max, cand_medium, 3},
                     {&khcore_tuning::push_alpha, cand_alpha, 3}};
        khcore_status st = KHCORE_OK;
        for (const Knob &kn : knobs) {
            int32_t best_v = t.*kn.field;
            float best_ms = 1e30f;
            for (int i = 0; i < kn.count && st == KHCORE_OK; i++) {
                khcore_tuning k = t;
                k.*kn.field = kn.cand[i];
                if (k.light_max > k.medium_max) continue;
                float ms = 0.f;
                if ((st = trial(k, &ms)) == KHCORE_OK && ms < best_ms) {
                    best_ms = ms;
                    best_v = kn.cand[i];
                }
            }
            t.*kn.field = best_v;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (st != KHCORE_OK) return st;
        cache_store(cache_path, key, t);
    } else {
        // Batches: the largest graph size that one thread block decomposes
        // faster than the whole grid, from up to 8 graphs of 512 to 32768
        // vertices timed both ways (each alone in a context of its own)
        std::vector<int32_t> mid;
        for (int32_t gi = 0; gi < c->G; gi++) {
            const int64_t ng = c->v_off[gi + 1] - c->v_off[gi];
            if (ng >= 512 && ng <= 32768) mid.push_back(gi);
        }
        std::sort(mid.begin(), mid.end(), [&](int32_t a, int32_t b) {
            return c->v_off[a + 1] - c->v_off[a] < c->v_off[b + 1] - c->v_off[b];
        });
        std::vector<int32_t> pick;
        for (int i = 0; i < 8 && !mid.empty(); i++) pick.push_back(mid[(size_t)i * (mid.size() - 1) / 7]);
        pick.erase(std::unique(pick.begin(), pick.end()), pick.end());
        int32_t cut = 0;
        for (int32_t gi : pick) {
            double ms[2] = {0, 0};
            for (int mode = 0; mode < 2; mode++) {
                khcore_ctx *sub = nullptr;
                if ((s = make_sub(c, gi, &sub)) != KHCORE_OK)
                    return fail(c, s, "autotune, graph %d: %s", gi, khcore_last_error(nullptr));
                sub->graph_blocks = mode == 0 ? 1 : 0;  // 1: one thread block; 0: the grid-wide path
                khcore_stats st;
                for (int rep = 0; rep < 2 && s == KHCORE_OK; rep++)
                    s = decompose(sub, std::vector<int32_t>{h}, nullptr, nullptr, &st);
                if (s != KHCORE_OK) {
                    const std::string msg = sub->err;
                    khcore_destroy(sub);
                    return fail(c, s, "autotune, graph %d: %s", gi, msg.c_str());
                }
                ms[mode] = st.device_ms;
                t.trials++;
                t.trial_ms += st.device_ms;
                khcore_destroy(sub);
            }
            const int32_t ng = (int32_t)(c->v_off[gi + 1] - c->v_off[gi]);
            if (ms[0] <= ms[1]) cut = std::max(cut, ng);
        }
        if (!pick.empty()) t.block_graph_max = cut;
        cache_store(cache_path, key, t);
    }
    // apply: the all-vertex pass takes the tuned classes, the rounds keep theirs
    if ((s = build_classes(c, t.light_max, t.medium_max, true)) != KHCORE_OK) return s;
    c->W_av = t.words;  // the all-vertex pass only; the rounds keep their W
    c->block = t.block;
    c->init_alpha = t.push_alpha;
    c->block_graph_max = t.block_graph_max;
    if (out) *out = t;
    return KHCORE_OK;
}

khcore_status khcore_set_update(khcore_ctx *c, int32_t mode)
{
    if (!c || (mode != 0 && mode != 1)) return KHCORE_EINVAL;
    c->update_mode = mode;
    return KHCORE_OK;
}

khcore_status khcore_bitmap_update(khcore_ctx *c, int32_t h, const uint8_t *alive_in, int32_t v, int32_t *deg_inout,
                                   int64_t *ball_out)
{
    khcore_status s;
    if ((s = check_ctx(c)) != KHCORE_OK) return s;
    if (c->G != 1) return fail(c, KHCORE_EINVAL, "khcore_bitmap_update takes a one-graph context");
    if (h < 1) return fail(c, KHCORE_EINVAL, "h must be >= 1 (got %d)", h);
    if (v < 0 || v >= c->n) return fail(c, KHCORE_EINVAL, "vertex %d outside [0, %d)", v, c->n);
    if (!alive_in || !deg_inout) return fail(c, KHCORE_EINVAL, "alive and deg must not be NULL");
    const int32_t he = effective_h(c->n, h);
    if (he > kUpdMaxH) return fail(c, KHCORE_EINVAL, "h = %d above the update's limit %d", he, kUpdMaxH);
    std::vector<uint8_t> al;
    CU(fetch(al, alive_in, (size_t)c->n));
    if (!al[v]) return fail(c, KHCORE_EINVAL, "vertex %d is not alive", v);
    if ((s = ensure_upd(c)) != KHCORE_OK) return s;
    uint8_t *bytes = nullptr;
    CU(dev_alloc(&bytes, (size_t)c->n));
    cudaError_t e = cudaMemcpyAsync(bytes, al.data(), (size_t)c->n, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_alive_from_bytes(c->alive, bytes, c->n, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->deg, deg_inout, sizeof(int32_t) * (size_t)c->n,
                            is_device_ptr(deg_inout) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->upd.cand[0], &v, sizeof v, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(bytes);
    CU(e);
    bool fit = false;
    if ((s = update_deleted(c, he, 1, nullptr, &fit, nullptr)) != KHCORE_OK) return s;
    if (!fit)
        return fail(c, KHCORE_EINVAL,
                    "the ball of vertex %d is over the update's limits (%d members, %d bitmap words per member)", v,
                    c->upd.cap, c->upd.wc);
    int32_t meta[4];
    CU(cudaMemcpyAsync(meta, c->upd.meta, sizeof meta, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(deg_inout, c->deg, sizeof(int32_t) * (size_t)c->n,
                       is_device_ptr(deg_inout) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (ball_out) *ball_out = meta[0];
    return KHCORE_OK;
}

khcore_status khcore_set_round_loop(khcore_ctx *c, int32_t mode)
{
    if (!c) return KHCORE_EINVAL;
    if (mode != 0 && mode != 1) return fail(c, KHCORE_EINVAL, "mode must be 0 (device) or 1 (host), got %d", mode);
    c->round_loop = mode;
    return KHCORE_OK;
}

khcore_status khcore_set_graph_blocks(khcore_ctx *c, int32_t mode)
{
    if (!c) return KHCORE_EINVAL;
    if (mode < -1 || mode > 1) return fail(c, KHCORE_EINVAL, "mode must be -1, 0 or 1, got %d", mode);
    c->graph_blocks = mode;
    return KHCORE_OK;
}

khcore_status khcore_set_wait_limit(khcore_ctx *c, uint64_t ns)
{
    if (!c) return KHCORE_EINVAL;
    c->wait_limit_ns = ns;
    return KHCORE_OK;
}

khcore_status khcore_set_profiling(khcore_ctx *c, int32_t on)
{
    if (!c) return KHCORE_EINVAL;
    if (on && c->tev.empty()) {
        const int cap = 1024;  // event pairs between two summations
        c->tev.resize(2 * cap, nullptr);
        for (auto &e : c->tev) {
            cudaError_t err = cudaEventCreate(&e);
            if (err != cudaSuccess) return fail(c, KHCORE_ECUDA, "cudaEventCreate: %s", cudaGetErrorString(err));
        }
        c->timer.ev = c->tev.data();
        c->timer.cap = cap;
    }
    c->profiling = on != 0;
    c->timer.used = 0;
    return KHCORE_OK;
}

khcore_status khcore_hdegrees_ex(khcore_ctx *c, int32_t h, int32_t *deg_out, khcore_stats *stats)
{
    khcore_status s = check_ctx(c);
    if (s != KHCORE_OK) return s;
    if (h < 1) return fail(c, KHCORE_EINVAL, "h must be >= 1 (got %d)", h);
    if (!deg_out && c->n) return fail(c, KHCORE_EINVAL, "deg_out is NULL");
    khcore_stats stt;
    std::memset(&stt, 0, sizeof stt);
    if (c->n == 0) {
        if (stats) *stats = stt;
        return KHCORE_OK;
    }
    const int W = c->W_req ? c->W_req : (c->W_av ? c->W_av : auto_words(c->n));
    if ((s = ensure_bfs(c, W)) != KHCORE_OK) return s;
    if ((s = clear_if_dirty(c)) != KHCORE_OK) return s;
    int32_t hmax = 1;
    for (int32_t g = 0; g < c->G; g++) hmax = std::max(hmax, effective_h(c->v_off[g + 1] - c->v_off[g], h));
    stt.h = hmax;
    stt.words_per_vertex = W;
    c->level_ms = 0.0;
    c->level_launches = 0;
    c->timer.used = 0;
    CU(cudaMemsetAsync(c->edges, 0, sizeof(unsigned long long), c->stream));
    CU(cudaMemsetAsync(c->alg, 0, sizeof(unsigned long long), c->stream));
    CU(cudaEventRecord(c->ev0, c->stream));
    CU(launch_alive_init(c->alive, c->n, c->stream));
    CU(launch_iota(c->src, c->n, c->stream));
    stt.kernel_launches += 2;
    // graphs are disjoint: one BFS over the union gives every graph's h-degrees
    if ((s = hdeg_sources(c, W, hmax, c->src, c->n, c->n, c->m, &stt, nullptr, 0, nullptr, true)) != KHCORE_OK)
        return s;
    CU(cudaEventRecord(c->ev1, c->stream));
    if ((s = write_out(c, deg_out, c->deg)) != KHCORE_OK) return s;
    unsigned long long edges = 0, alg = 0;
    CU(cudaMemcpyAsync(&edges, c->edges, sizeof edges, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(&alg, c->alg, sizeof alg, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (stats) {
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
        if ((s = flush_timer(c)) != KHCORE_OK) return s;
        stt.device_ms = ms;
        stt.init_ms = ms;
        stt.edges_traversed = (int64_t)edges;
        stt.level_bytes = (double)alg;
        stt.level_ms = c->level_ms;
        stt.level_launches = c->level_launches;
        *stats = stt;
    } else if ((s = flush_timer(c)) != KHCORE_OK) {
        return s;
    }
    return KHCORE_OK;
}

khcore_status khcore_hdegrees(khcore_ctx *c, int32_t h, int32_t *deg_out)
{
    return khcore_hdegrees_ex(c, h, deg_out, nullptr);
}

khcore_status khcore_hdegrees_of(khcore_ctx *c, int32_t h, int32_t count, const int32_t *verts, int32_t *deg_out)
{
    khcore_status s = check_ctx(c);
    if (s != KHCORE_OK) return s;
    if (h < 1) return fail(c, KHCORE_EINVAL, "h must be >= 1 (got %d)", h);
    if (count < 0 || count > c->n) return fail(c, KHCORE_EINVAL, "count %d outside [0, %d]", count, c->n);
    if (count == 0) return KHCORE_OK;
    if (!verts || !deg_out) return fail(c, KHCORE_EINVAL, "verts or deg_out is NULL");
    std::vector<int32_t> vs;
    if (fetch(vs, verts, (size_t)count) != cudaSuccess) return fail(c, KHCORE_ECUDA, "cannot read verts");
    {
        std::vector<uint8_t> seen((size_t)c->n, 0);
        for (int32_t i = 0; i < count; i++) {
            if (vs[i] < 0 || vs[i] >= c->n) return fail(c, KHCORE_EINVAL, "vertex %d outside [0, %d)", vs[i], c->n);
            if (seen[vs[i]]++) return fail(c, KHCORE_EINVAL, "vertex %d listed twice", vs[i]);
        }
    }
    const int W = c->W_req ? c->W_req : (c->W_av ? c->W_av : auto_words(c->n));
    if ((s = ensure_bfs(c, W)) != KHCORE_OK) return s;
    if ((s = clear_if_dirty(c)) != KHCORE_OK) return s;
    int32_t hmax = 1;
    for (int32_t g = 0; g < c->G; g++) hmax = std::max(hmax, effective_h(c->v_off[g + 1] - c->v_off[g], h));
    CU(launch_alive_init(c->alive, c->n, c->stream));
    CU(cudaMemcpyAsync(c->src, vs.data(), sizeof(int32_t) * (size_t)count, cudaMemcpyHostToDevice, c->stream));
    if ((s = hdeg_sources(c, W, hmax, c->src, count, c->n, c->m, nullptr, nullptr, 0, nullptr, true)) != KHCORE_OK)
        return s;
    // gather deg[verts[i]] into deg_out[i] on the host side of the copy
    std::vector<int32_t> all((size_t)c->n);
    CU(cudaMemcpyAsync(all.data(), c->deg, sizeof(int32_t) * (size_t)c->n, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    std::vector<int32_t> outv((size_t)count);
    for (int32_t i = 0; i < count; i++) outv[i] = all[vs[i]];
    if (is_device_ptr(deg_out)) {
        CU(cudaMemcpy(deg_out, outv.data(), sizeof(int32_t) * (size_t)count, cudaMemcpyHostToDevice));
    } else {
        std::memcpy(deg_out, outv.data(), sizeof(int32_t) * (size_t)count);
    }
    return KHCORE_OK;
}

khcore_status khcore_decompose_ex(khcore_ctx *c, int32_t h, int32_t *core_out, int32_t *round_out,
                                  khcore_stats *stats)
{
    khcore_status s = check_ctx(c);
    if (s != KHCORE_OK) return s;
    if (h < 1) return fail(c, KHCORE_EINVAL, "h must be >= 1 (got %d)", h);
    if (!core_out && c->n) return fail(c, KHCORE_EINVAL, "core_out is NULL");
    return decompose(c, std::vector<int32_t>((size_t)c->G, h), core_out, round_out, stats);
}

khcore_status khcore_decompose(khcore_ctx *c, int32_t h, int32_t *core_out)
{
    return khcore_decompose_ex(c, h, core_out, nullptr, nullptr);
}

khcore_status khcore_decompose_sampled(khcore_ctx *c, int32_t h, const uint8_t *in_s, int32_t *core_out,
                                      int32_t *round_out, khcore_stats *stats)
{
    khcore_status s;
    if ((s = check_ctx(c)) != KHCORE_OK) return s;
    if (h < 1) return fail(c, KHCORE_EINVAL, "h must be >= 1 (got %d)", h);
    if (c->G != 1) return fail(c, KHCORE_EINVAL, "khcore_decompose_sampled takes a one-graph context");
    if (!in_s && c->n > 0) return fail(c, KHCORE_EINVAL, "in_s must not be NULL");
    const size_t n = (size_t)std::max(c->n, 1);
    if (!c->s_in) {
        CU(dev_alloc(&c->s_in, n));
        CU(dev_alloc(&c->s_sel0, n));
        CU(dev_alloc(&c->s_sel, n));
        CU(dev_alloc(&c->s_d0, n));
        CU(dev_alloc(&c->s_full, 16));
        CU(cudaMemsetAsync(c->s_full, 0, 16 * sizeof(uint64_t), c->stream));
    }
    if (c->n > 0)
        CU(cudaMemcpyAsync(c->s_in, in_s, (size_t)c->n,
                           is_device_ptr(in_s) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    c->sampling_req = true;
    s = decompose(c, std::vector<int32_t>{h}, core_out, round_out, stats);
    c->sampling_req = false;
    return s;
}

khcore_status khcore_batch_decompose(khcore_ctx *c, const int32_t *h, int32_t *core_out, int32_t *round_out,
                                     khcore_stats *stats)
{
    khcore_status s = check_ctx(c);
    if (s != KHCORE_OK) return s;
    if (!h) return fail(c, KHCORE_EINVAL, "h is NULL");
    if (!core_out && c->n) return fail(c, KHCORE_EINVAL, "core_out is NULL");
    std::vector<int32_t> hv;
    if (fetch(hv, h, (size_t)c->G) != cudaSuccess) return fail(c, KHCORE_ECUDA, "cannot read h");
    for (int32_t g = 0; g < c->G; g++)
        if (hv[g] < 1) return fail(c, KHCORE_EINVAL, "h[%d] must be >= 1 (got %d)", g, hv[g]);
    return decompose(c, hv, core_out, round_out, stats);
}

}  // extern "C"
