// khcore_persist.cuh — the whole decomposition in one cooperative launch.
//
// The host-driven path launches every phase of every round and waits for the
// round's counts before planning the recompute; on graphs that need tens of
// thousands of rounds that launch-and-wait cost dominates. Here one persistent
// kernel (grid = every block that can be resident, launched cooperatively so
// that all blocks run at once) steps through the same phases, separated by
// grid barriers, after the initial h-degrees. Per round, in the default lazy
// mode: level minimum -> bound check -> exact recompute of the candidates ->
// set level -> peel set -> one BFS from the deleted set that updates the
// bounds (its last batch's end runs beside the next round's minimum). In the
// eager mode: level minimum -> set level -> peel set -> affected BFS ->
// recompute / outer-shell update. The decisions between phases (batch plans,
// push or pull, the end of the loop) read device counters after a barrier,
// so every block takes the same path. Small serial steps (resetting counters,
// snapshots, statistics) run in the barrier itself, on the block that arrives
// last, while every other block waits.
//
// Every barrier wait has a time limit: a block that waits longer sets an
// error flag and leaves; every block checks the flag after each barrier and
// returns, so a stuck barrier ends the launch with KHCORE_ETIMEOUT instead of
// hanging the GPU.
#pragma once

#include "khcore_device.cuh"

namespace khc {

namespace {

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned atom_add_acq_rel_gpu(unsigned *p, unsigned x)
{
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(x) : "memory");
    return old;
}

__device__ __forceinline__ void red_add_release_gpu(unsigned *p, unsigned x)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(x) : "memory");
}

// Grid barrier; serial() runs on one thread of the last block to arrive,
// before any block is released. Returns false once any wait has timed out.
// Each block's thread 0 arrives with an acquire-release add on the counter
// (after the block's __syncthreads, so it publishes the block's writes and,
// when it is last, sees every other block's); the last one runs serial(),
// resets the counter and releases the generation word, which the others poll
// with acquire loads. No full fences: a probe of back-to-back barriers on the
// GB300 measured 2.24 us per barrier this way against 2.88 us with
// __threadfence around plain atomics (152 blocks of 512 threads).
template <class F>
__device__ __forceinline__ bool grid_sync(GridSync *gs, unsigned long long timeout_ns, F serial)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned g0 = ld_acquire_gpu(&gs->gen);
        const unsigned arrived = atom_add_acq_rel_gpu(&gs->count, 1u);
        if (arrived == gridDim.x - 1) {
            serial();
            gs->passed++;
            gs->count = 0;
            red_add_release_gpu(&gs->gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (ld_acquire_gpu(&gs->gen) == g0) {
                if (global_ns() - t0 > timeout_ns) {
                    atomicExch(&gs->err, 1);
                    break;
                }
                __nanosleep(32);
            }
        }
        s_ok = *((volatile int *)&gs->err) == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

struct Nop {
    __device__ void operator()() const {}
};

struct PersistArgs {
    GraphView g;
    uint32_t *alive;
    int32_t *deg, *core, *rnd;
    PeelView p;
    PeelState *st;
    BfsBufs b;
    uint32_t *vis;       // affected-BFS visited bits
    int32_t *A;          // affected vertices, class regions
    int32_t *aq[3];      // affected-BFS frontier ring (slot 0 starts as the deleted set)
    int32_t *dcls;       // deleted vertices, class regions
    int32_t *cls_src;    // every vertex, class regions (initial pass)
    const int32_t *cls_h, *cls_size, *cls_off;  // per class
    int32_t *inner;      // per class: affected vertices closer than h
    int32_t *dcount;     // per vertex: deleted vertices within h
    int32_t *comb;       // round source list: inner vertices, then deleted ones
    int32_t *cand;       // lazy mode: exact-recompute list (class regions)
    int32_t *wsum;       // lazy mode: ball bounds of the deleted set
    int32_t ncls, hmax, alpha;
    GridSync *gs;
    PersistStats *ps;
    unsigned long long timeout_ns;
};

// What one BFS batch of the persistent kernel produces besides the column
// counts.
struct BatchOpt {
    int32_t *rowcnt = nullptr;  // row counts (see BfsBufs::rowcnt), or nullptr
    int32_t row_first = 0;
    int32_t row_sign = 1;       // -1: the row counts are taken off rowcnt
    bool weights = false;       // lazy mode, seeded at the deleted set: ball bounds into wsum
    bool lazy_end = false;      // lazy mode, seeded at the deleted set: slack update of T (in the
                                // last level's weight pass), no degree writes at the end
    bool min_fold = false;      // fold the sources' h-degrees into their graph's exact minimum
    bool pre_reset = false;     // the caller's last barrier already reset the ring for the first batch
    bool defer_end = false;     // return after the last level; the caller runs the end (DeferredEnd)
};

// The end of a batch that the caller runs later, beside other work (the
// deleted set's last batch: in the next round's minimum scan).
struct DeferredEnd {
    bool pending = false;
    bool one_word = false;  // the batch's row layout: 1 word, else W
    const int32_t *src = nullptr;
    int32_t ns = 0, h = 0;
};

// The level ring's reset for a batch of ns sources, in a barrier's serial step.
__device__ __forceinline__ void reset_ring(LevelCtl *ctl, int32_t ns)
{
    for (int k = 0; k < 3; k++) {
        ctl->q[k] = 0;
        ctl->qi[k] = 0;
        ctl->fe[k] = 0;
    }
    ctl->t = ns;
}

// One batch of the multi-source BFS (sources src[0..ns), h levels), every
// block taking part, with fused levels (dev_level<W, LAST, true>): a barrier
// to reset the level ring, one phase per level, one to finish (h + 2
// barriers; one more before level h-2 for the h-2 ball weights when h >= 3).
// With o.defer_end it returns after the last level and the caller runs the
// end later (h + 1). Returns false on timeout.
template <int W>
__device__ bool bfs_batch(const PersistArgs &a, const int32_t *src, int32_t ns, int32_t h, const BatchOpt &o)
{
    BfsBufs b = a.b;
    b.rowcnt = o.rowcnt;
    b.row_first = o.row_first;
    b.row_sign = o.row_sign;
    b.wsum = o.weights ? a.wsum : nullptr;
    b.wdeg = a.deg;
    b.newcnt = o.lazy_end ? reinterpret_cast<unsigned long long *>(&a.ps->affected_total) : nullptr;
    LevelCtl *ctl = b.ctl;
    // reset the level ring (unless the caller's barrier did) and place the
    // sources (level 0)
    if (!o.pre_reset && !grid_sync(a.gs, a.timeout_ns, [&] { reset_ring(ctl, ns); })) return false;
    {
        const int lane = threadIdx.x & 31;
        for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < ns; i0 += (int64_t)gridDim.x * blockDim.x) {
            const int64_t i = i0 + threadIdx.x;  // block-uniform loop
            unsigned long long d = 0;
            int32_t s = -1;
            if (i < ns) {
                s = src[i];
                d = (unsigned long long)(a.g.row_ptr[s + 1] - a.g.row_ptr[s]);
                const int word = (int)(i >> 6);
                const uint64_t bit = 1ull << (i & 63);
                b.V[(size_t)s * W + word] = bit;     // V rows are zero between batches
                b.F[0][(size_t)s * W + word] = bit;  // so are F rows
                flag_set(b.flag[0], s);
                flag_set(b.tflag, s);
                b.T[i] = s;
            }
            Acc acc0{0, 0, 0};
            append_frontier<W>(i < ns, s, (int32_t)d, b, 0, acc0, a.g.row_ptr);  // Q[0] and level-0 push items
            const unsigned long long ws = warp_sum(acc0.fe);
            if (lane == 0 && ws) {
                atomicAdd(&ctl->fe[0], ws);
                atomicAdd(b.edges, ws);  // every source scans its own row
            }
        }
    }
    BfsTuning tune;
    tune.alpha = a.alpha;
    for (int lvl = 0; lvl < h; lvl++) {
        // the slot this level appends to was cleared by the previous level
        if (!grid_sync(a.gs, a.timeout_ns, [&] {
                a.ps->level_steps++;
                const int sl = (lvl + 1) % 3;
                ctl->q[sl] = 0;
                ctl->qi[sl] = 0;
                ctl->fe[sl] = 0;
            }))
            return false;
        tune.m_alive = *((volatile unsigned long long *)&a.st->m_alive);
        tune.n_alive = *((volatile int32_t *)&a.st->alive);
        if (b.wsum && h >= 3 && lvl == h - 2) {
            // V holds every source within h-2 now; the next level adds more
            dev_weight_pass<W>(b, src, a.g.row_ptr, a.alive, false);
            if (!grid_sync(a.gs, a.timeout_ns, Nop{})) return false;
        }
        if (lvl == h - 1) {
            // the last level writes neither V nor T, so the weights of the
            // sources within h-1 are taken in the same phase
            if (b.wsum && h >= 2)
                dev_weight_pass<W>(b, src, a.g.row_ptr, a.alive, true, o.lazy_end ? a.p.slack : nullptr, a.deg);
            dev_level<W, true, true>(a.g, a.alive, b, lvl, tune);
        } else {
            dev_level<W, false, true>(a.g, a.alive, b, lvl, tune);
        }
    }
    if (o.defer_end) return true;
    if (!grid_sync(a.gs, a.timeout_ns, [&] {
            if (o.lazy_end) a.ps->affected_total += ctl->t - ns;  // the vertices within h-1
        }))
        return false;
    // the lazy mode's deleted-set batch writes no degrees (its row counts
    // came off them during the levels)
    dev_end_fused<W>(b, src, ns, h, o.lazy_end ? nullptr : a.deg, o.min_fold ? &a.p : nullptr);
    return true;
}

// h-degrees (or row counts) of src[0..ns) in batches of 64*W sources.
// defer: the last batch's end is left to the caller, described in *def.
template <int W>
__device__ __forceinline__ bool bfs_sources(const PersistArgs &a, const int32_t *src, int32_t ns, int32_t h,
                                            BatchOpt o, DeferredEnd *def = nullptr, bool defer = false)
{
    constexpr int32_t S = 64 * W;
    const int32_t row_first = o.row_first;
    for (int32_t off = 0; off < ns; off += S) {
        const int32_t cur = ns - off < S ? ns - off : S;
        o.row_first = row_first > off ? row_first - off : 0;
        if (off > 0) o.pre_reset = false;  // only the first batch can be pre-reset
        o.defer_end = def && defer && off + cur == ns;
        // a batch of at most 64 sources runs on one-word rows: a quarter of
        // the row traffic of W = 4 for the same result (the row arrays are
        // all zero between batches in either layout)
        const bool one = W > 1 && cur <= 64;
        const bool ok = one ? bfs_batch<1>(a, src + off, cur, h, o) : bfs_batch<W>(a, src + off, cur, h, o);
        if (!ok) return false;
        if (blockIdx.x == 0 && threadIdx.x == 0) a.ps->source_batches++;
        if (o.defer_end) {
            def->pending = true;
            def->one_word = one || W == 1;
            def->src = src + off;
            def->ns = cur;
            def->h = h;
        }
    }
    return true;
}

// Contexts with at most this many graphs update the levels on one thread
// inside a barrier (one barrier less per round).
constexpr int32_t kSerialLevelMaxGraphs = 64;

// MINB: resident blocks of 512 threads per SM. One (up to 128 registers per
// thread, no spills, half the blocks at every grid barrier) measured 4 %
// faster than two (64 registers) on the 1e6-vertex Chung-Lu graph at h = 2,
// where the rounds are latency-bound; two measured 14 % faster at h = 3 and 7 %
// on the R-MAT graph at h = 4, where the rounds' BFS levels are larger.
template <int W, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_decompose(PersistArgs a)
{
    // phase clock of block 0: called right after a barrier, so the phase
    // before it is complete on every block
    unsigned long long t_last = (blockIdx.x == 0 && threadIdx.x == 0) ? global_ns() : 0;
    auto mark = [&](int ph) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            const unsigned long long t = global_ns();
            a.ps->phase_ns[ph] += t - t_last;
            t_last = t;
        }
    };
    // the initial h-degrees are in deg already (computed by the per-phase
    // kernels at the widest W); the rounds follow
    const bool serial_level = a.p.G <= kSerialLevelMaxGraphs;
    const bool lazy = a.p.slack != nullptr;
    DeferredEnd def;  // the deleted set's last batch (lazy mode, one class)
    for (bool first = true;; first = false) {
        // level of every graph: k_g <- max(k_g, min alive h-degree); the
        // barrier closing the previous round advances the round counter
        if (!grid_sync(a.gs, a.timeout_ns, [&] {
                if (!first) a.st->round++;
                a.st->lvl_set = 0;
                if (def.pending) a.ps->affected_total += a.b.ctl->t - def.ns;  // the vertices within h-1
            }))
            return;
        mark(4);
        if (def.pending) {
            // the end of the previous round's last batch, beside the scan:
            // it clears BFS rows, the scan reads alive, deg and slack
            BfsBufs bd = a.b;
            bd.wsum = a.wsum;
            if (def.one_word)
                dev_end_fused<1>(bd, def.src, def.ns, def.h, nullptr, nullptr);
            else
                dev_end_fused<W>(bd, def.src, def.ns, def.h, nullptr, nullptr);
            def.pending = false;
        }
        dev_min_alive_deg(a.g.n, a.alive, a.deg, a.p);
        if (lazy) {
            // lazy mode: exact recompute of the vertices whose bounds leave
            // their fate at the coming level open; when there are none, the
            // level step runs in the serial step of the barrier after the
            // selection
            if (!grid_sync(a.gs, a.timeout_ns, Nop{})) return;
            dev_refine_select(a.g.n, a.alive, a.deg, a.p, a.cand);
            // one class: the same serial step resets the BFS ring for the first
            // batch of candidates (one barrier less)
            if (!grid_sync(a.gs, a.timeout_ns, [&] {
                    int32_t tot = 0;
                    for (int32_t c = 0; c < a.ncls; c++) tot += a.p.ncand[c];
                    if (tot == 0 && serial_level) {
                        dev_set_level_serial(a.p, a.st);
                        a.st->lvl_set = 1;
                    } else if (a.ncls == 1) {
                        reset_ring(a.b.ctl, tot < 64 * W ? tot : 64 * W);
                    }
                }))
                return;
            mark(0);
            if (!*((volatile int32_t *)&a.st->lvl_set)) {
                for (int32_t c = 0; c < a.ncls; c++) {
                    const int32_t nc = *((volatile int32_t *)&a.p.ncand[c]);
                    if (nc <= 0) continue;
                    BatchOpt o;
                    o.min_fold = true;
                    o.pre_reset = a.ncls == 1;
                    if (!bfs_sources<W>(a, a.cand + a.cls_off[c], nc, a.cls_h[c], o)) return;
                    if (blockIdx.x == 0 && threadIdx.x == 0) a.ps->recomputed_total += nc;
                }
                if (!grid_sync(a.gs, a.timeout_ns, [&] {
                        if (serial_level) dev_set_level_serial(a.p, a.st);
                    }))
                    return;
            }
            mark(1);
        } else {
            // few graphs: the level step runs inside the barrier
            if (!grid_sync(a.gs, a.timeout_ns, [&] {
                    if (serial_level) dev_set_level_serial(a.p, a.st);
                }))
                return;
            mark(0);
        }
        if (!serial_level) {
            dev_set_level(a.p, a.st);
            if (!grid_sync(a.gs, a.timeout_ns, Nop{})) return;
        }
        // peel set D
        // (lazy mode: no affected-set BFS, so neither its bits nor its list)
        dev_peel_compact(a.g.n, a.g.row_ptr, a.alive, a.deg, a.p, a.st, a.core, a.rnd, lazy ? nullptr : a.vis,
                         lazy ? nullptr : a.aq[0], a.dcls);
        if (lazy) {
            // One BFS seeded at the deleted set of each class does what the
            // affected-set BFS and the update did: every alive vertex it
            // reaches loses, on the spot, the deleted vertices that reach it
            // through survivors (row counts taken off deg); those within h-1
            // also widen their slack at the end of the batch (reading of
            // Observation 2: what they lose besides lies within h-1 of the
            // deleted set).
            // one class: the statistics barrier also resets the BFS ring for
            // the first batch seeded at the deleted set
            if (!grid_sync(a.gs, a.timeout_ns, [&] {
                    a.ps->rounds++;
                    a.ps->deleted_total += a.st->nD;
                    if (a.ncls == 1) reset_ring(a.b.ctl, a.st->nD < 64 * W ? a.st->nD : 64 * W);
                }))
                return;
            mark(2);
            if (*((volatile int32_t *)&a.st->alive) == 0) break;
            for (int32_t c = 0; c < a.ncls; c++) {
                const int32_t nd = *((volatile int32_t *)&a.p.nDc[c]);
                if (nd <= 0) continue;
                BatchOpt o;
                o.pre_reset = a.ncls == 1;
                o.rowcnt = a.deg;
                o.row_sign = -1;
                o.weights = true;
                o.lazy_end = true;
                if (!bfs_sources<W>(a, a.dcls + a.cls_off[c], nd, a.cls_h[c], o, &def, a.ncls == 1))
                    return;
            }
            continue;
        }
        // affected set A: BFS from D through survivors; snapshot the per-class
        // counts before the level that reaches distance h of each class
        for (int lvl = 0; lvl < a.hmax; lvl++) {
            if (!grid_sync(a.gs, a.timeout_ns, [&] {
                    for (int32_t c = 0; c < a.p.ncls; c++)
                        if (a.cls_h[c] == lvl + 1) a.inner[c] = a.p.nAc[c];
                }))
                return;
            mark(lvl == 0 ? 2 : 3);
            dev_affected_push(a.g, a.alive, lvl, a.aq[0], a.aq[1], a.aq[2], a.vis, a.p, a.st, a.A, lvl == a.hmax - 1);
        }
        if (!grid_sync(a.gs, a.timeout_ns, [&] {
                int32_t s = 0;
                for (int32_t c = 0; c < a.p.ncls; c++) s += a.p.nAc[c];
                a.st->nA = s;
                a.ps->rounds++;
                a.ps->deleted_total += a.st->nD;
                a.ps->affected_total += s;
            }))
            return;
        mark(3);
        const int32_t alive_left = *((volatile int32_t *)&a.st->alive);
        if (alive_left == 0) break;
        const bool single = *((volatile int32_t *)&a.st->nD) == 1;
        // recompute the inner part of A; update the outer shell by counting
        for (int32_t c = 0; c < a.ncls; c++) {
            const int32_t na = *((volatile int32_t *)&a.p.nAc[c]);
            int32_t ni = *((volatile int32_t *)&a.inner[c]);
            ni = ni < na ? ni : na;
            const int32_t nd = *((volatile int32_t *)&a.p.nDc[c]);
            if (na == 0) continue;
            int32_t *Ac = a.A + a.cls_off[c];
            const bool count_d = na > ni && !single;
            const int32_t total = ni + (count_d ? nd : 0);
            if (total > 0) {
                // one source list: inner vertices, then the deleted vertices
                // whose row counts update the outer shell (the barrier keeps
                // the previous class's batch from still reading the list)
                if (!grid_sync(a.gs, a.timeout_ns, Nop{})) return;
                dev_concat(a.comb, Ac, ni, a.dcls + a.cls_off[c], count_d ? nd : 0);
                BatchOpt o;
                o.rowcnt = count_d ? a.dcount : nullptr;
                o.row_first = ni;
                if (!bfs_sources<W>(a, a.comb, total, a.cls_h[c], o)) return;
            }
            if (blockIdx.x == 0 && threadIdx.x == 0) a.ps->recomputed_total += ni;
            if (na > ni) {
                if (!grid_sync(a.gs, a.timeout_ns, Nop{})) return;
                dev_apply_dcount(Ac, ni, na, single ? nullptr : a.dcount, a.deg);
            }
        }
    }
}

}  // namespace

// Per-W entry points, one translation unit each (khcore_persist_w*.cu).
template <int W, int MINB>
cudaError_t persist_launch_w(const PersistLaunch &L, int grid, cudaStream_t s)
{
    PersistArgs a;
    a.g = L.g;
    a.alive = L.alive;
    a.deg = L.deg;
    a.core = L.core;
    a.rnd = L.rnd;
    a.p = L.p;
    a.st = L.st;
    a.b = L.b;
    a.vis = L.vis;
    a.A = L.A;
    for (int k = 0; k < 3; k++) a.aq[k] = L.aq[k];
    a.dcls = L.dcls;
    a.cls_src = L.cls_src;
    a.cls_h = L.cls_h;
    a.cls_size = L.cls_size;
    a.cls_off = L.cls_off;
    a.inner = L.inner;
    a.dcount = L.dcount;
    a.comb = L.comb;
    a.cand = L.cand;
    a.wsum = L.wsum;
    a.ncls = L.ncls;
    a.hmax = L.hmax;
    a.alpha = L.alpha;
    a.gs = L.gs;
    a.ps = L.ps;
    a.timeout_ns = L.timeout_ns;
    void *args[] = {&a};
    return cudaLaunchCooperativeKernel((const void *)k_decompose<W, MINB>, grid, kBlock, args, 0, s);
}

template <int W, int MINB>
int persist_occupancy_w()
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_decompose<W, MINB>, kBlock, 0) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return nb;
}

cudaError_t persist_launch_1(const PersistLaunch &L, int grid, cudaStream_t s);
cudaError_t persist_launch_2(const PersistLaunch &L, int grid, cudaStream_t s);
cudaError_t persist_launch_4(const PersistLaunch &L, int grid, cudaStream_t s);
cudaError_t persist_launch_8(const PersistLaunch &L, int grid, cudaStream_t s);
cudaError_t persist_launch_16(const PersistLaunch &L, int grid, cudaStream_t s);
cudaError_t persist_launch_4x2(const PersistLaunch &L, int grid, cudaStream_t s);
int persist_occupancy_1();
int persist_occupancy_2();
int persist_occupancy_4();
int persist_occupancy_8();
int persist_occupancy_16();
int persist_occupancy_4x2();

}  // namespace khc
