// khcore_device.cuh — device code of the (k,h)-core hot path, shared by the
// per-phase kernels (khcore_bfs.cu, khcore_peel.cu) and the persistent
// decomposition kernel (khcore_persist.cu).
//
// Multi-source h-bounded BFS: the h-hop degree d_v^h of Sec. II for a batch
// of 64*W sources at once. Each vertex holds W 64-bit words per state array;
// bit b of word j stands for source 64*j+b of the batch (the paper packs 64
// set members per 64-bit word in its Reach bitmaps, Sec. IV-B; here the
// members are BFS sources). A level turns the frontier F (sources that
// reached a vertex at exactly the current distance) into the next one, in one
// of two directions chosen on the device from the frontier's degree sum:
//   pull  every alive y: new(y) = OR_{x in N(y), x in frontier} F(x), minus V(y);
//   push  every frontier x, every alive neighbour y: F'(y) |= F(x) & ~V(y)
//         with atomicOr, whose returned old value tells which bits are new.
// The number of newly reached vertices per source is a column count over the
// new words, kept per lane in byte-sliced (SWAR) counters.
//
// Peel rounds (Algorithm 1 / 2 made level-synchronous), for one graph or a
// batch of disjoint graphs that peel side by side with their own level k and
// hop bound h: level min, peel-set compaction, affected-set BFS.
//
// Loads of data that change during a decomposition (alive bits, frontier
// flags and rows, levels) are plain loads, never the non-coherent read-only
// path, so that the persistent kernel sees every phase's writes after a grid
// barrier. Only the CSR and per-graph constants use __ldg.
#pragma once

#include <climits>
#include <cstdint>

#include "khcore_internal.cuh"

namespace khc {
namespace {


constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ bool is_alive(const uint32_t *alive, int32_t y)
{
    return (alive[y >> 5] >> (y & 31)) & 1u;
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Kernel parameters indexed with a runtime value would be copied to local
// memory; pick array members with selects instead.
template <class T>
__device__ __forceinline__ T pick2(const T (&a)[2], int i)
{
    return i ? a[1] : a[0];
}
template <class T>
__device__ __forceinline__ T pick3(const T (&a)[3], int i)
{
    return i == 0 ? a[0] : (i == 1 ? a[1] : a[2]);
}

// Whole warp calls; lanes with pred append val to list (warp-aggregated).
__device__ __forceinline__ void warp_append(bool pred, int32_t val, int32_t *list, int32_t *counter)
{
    const unsigned m = __ballot_sync(kFull, pred);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    int32_t base = 0;
    if (lane == leader) base = atomicAdd(counter, __popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (pred) list[base + __popc(m & lanemask_lt())] = val;
}

// Frontier flags, one bit per vertex (n/8 bytes: the pull direction tests a
// flag for every CSR entry it scans, and a bitmap keeps those tests in L1).
__device__ __forceinline__ bool flag_test(const uint32_t *f, int32_t y) { return (f[y >> 5] >> (y & 31)) & 1u; }
__device__ __forceinline__ void flag_set(uint32_t *f, int32_t y) { atomicOr(&f[y >> 5], 1u << (y & 31)); }
__device__ __forceinline__ void flag_clear(uint32_t *f, int32_t y) { atomicAnd(&f[y >> 5], ~(1u << (y & 31))); }
// Test-and-set: true for the one caller that set the bit.
__device__ __forceinline__ bool flag_claim(uint32_t *f, int32_t y)
{
    const uint32_t bit = 1u << (y & 31);
    return (atomicOr(&f[y >> 5], bit) & bit) == 0;
}

// Byte-sliced column counters: byte k of a[t] counts bit 8k+t of the words
// added. Each add contributes at most 1 per byte, so a flush every 255 adds
// keeps the bytes exact.
struct Swar {
    uint64_t a[8];
    int n;
    __device__ __forceinline__ void reset()
    {
#pragma unroll
        for (int t = 0; t < 8; t++) a[t] = 0;
        n = 0;
    }
    __device__ __forceinline__ void add(uint64_t w)
    {
#pragma unroll
        for (int t = 0; t < 8; t++) a[t] += (w >> t) & 0x0101010101010101ull;
    }
};

// Whole warp calls. Lanes with the same word index j = lane % W are summed
// (16-bit lanes cannot overflow: at most 32 * 255), then lane j adds its 64
// column counts to cnt_s[64*j + bit].
template <int W>
__device__ __forceinline__ void swar_flush(Swar &s, int32_t *cnt_s)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int t = 0; t < 8; t++) {
        uint64_t lo = s.a[t] & 0x00FF00FF00FF00FFull;         // bytes 0,2,4,6
        uint64_t hi = (s.a[t] >> 8) & 0x00FF00FF00FF00FFull;  // bytes 1,3,5,7
#pragma unroll
        for (int off = W; off < 32; off <<= 1) {
            lo += __shfl_xor_sync(kFull, lo, off);
            hi += __shfl_xor_sync(kFull, hi, off);
        }
        if (lane < W) {
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint32_t c0 = (uint32_t)(lo >> (16 * k)) & 0xffffu;  // byte 2k   -> bit 16k+t
                const uint32_t c1 = (uint32_t)(hi >> (16 * k)) & 0xffffu;  // byte 2k+1 -> bit 16k+8+t
                if (c0) atomicAdd(&cnt_s[lane * 64 + 16 * k + t], (int32_t)c0);
                if (c1) atomicAdd(&cnt_s[lane * 64 + 16 * k + 8 + t], (int32_t)c1);
            }
        }
        s.a[t] = 0;
    }
    s.n = 0;
}

template <int W>
__device__ __forceinline__ void swar_step(Swar &s, uint64_t w, int32_t *cnt_s)
{
    s.add(w);
    if (++s.n == 255) swar_flush<W>(s, cnt_s);
}

// Bits of word j that stand for row-counted sources (batch positions >=
// row_first).
__device__ __forceinline__ uint64_t row_mask(int j, int32_t row_first)
{
    const int32_t lo = 64 * j;
    if (row_first <= lo) return ~0ull;
    if (row_first >= lo + 64) return 0ull;
    return ~0ull << (row_first - lo);
}

// Bits of word j that a vertex y may count for (see BfsBufs::slev): source
// positions below cum[hcnt - slev[y]]; every bit when no eligibility is set.
// With sampling (b.in_s), an unsampled vertex counts only for the sources
// of b.fullmask.
__device__ __forceinline__ uint64_t elig_mask(const BfsBufs &b, int j, int32_t y)
{
    if (y < 0) return ~0ull;
    uint64_t m = ~0ull;
    if (b.slev) {
        const int32_t lim = b.cum[b.hcnt - b.slev[y]] - b.boff - 64 * j;
        m = lim <= 0 ? 0ull : (lim >= 64 ? ~0ull : (1ull << lim) - 1ull);
    }
    if (b.in_s && !b.in_s[y]) m &= b.fullmask[j];
    return m;
}

// Per-thread accumulators flushed once at the end of a level kernel.
struct Acc {
    unsigned long long scanned;  // plain-BFS-equivalent CSR entries
    unsigned long long fe;       // degree sum of vertices appended to the next frontier
    unsigned long long newv;     // vertices first reached at the last level (when b.newcnt is set)
    unsigned long long gathered; // pull: frontier rows OR-ed in (one per flagged CSR entry)
    unsigned long long rows;     // pull: vertices with a frontier neighbour (own rows read / written)
};

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v)
{
#pragma unroll
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    return v;
}

__device__ __forceinline__ bool use_push(const LevelCtl *ctl, int slot, BfsTuning tune)
{
    return tune.alpha > 0 &&
           (unsigned long long)ctl->fe[slot] * (unsigned long long)tune.alpha < tune.m_alive;
}

// Append y (already claimed in the next frontier) to Q, and its CSR row as
// push work items of push_chunk(W) entries. Whole warp calls; pred marks the
// lanes that append.
template <int W>
__device__ __forceinline__ void append_frontier(bool pred, int32_t y, int32_t deg, const BfsBufs &b, int nslot,
                                                Acc &acc, const int32_t *rp)
{
    constexpr int C = push_chunk(W);
    warp_append(pred, y, pick3(b.Q, nslot), &b.ctl->q[nslot]);
    int32_t nch = pred ? (deg + C - 1) / C : 0;
    // warp-wide exclusive prefix of the item counts, one atomic per warp
    const int lane = threadIdx.x & 31;
    int32_t incl = nch;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int32_t t = __shfl_up_sync(kFull, incl, off);
        if (lane >= off) incl += t;
    }
    const int32_t total = __shfl_sync(kFull, incl, 31);
    if (total) {
        int32_t base = 0;
        if (lane == 0) base = atomicAdd(&b.ctl->qi[nslot], total);
        base = __shfl_sync(kFull, base, 0) + incl - nch;
        if (nch) {
            int2 *items = pick3(b.I, nslot);
            const int32_t e0 = rp[y];
            for (int32_t k = 0; k < nch; k++) items[base + k] = make_int2(y, e0 + k * C);
        }
    }
    if (pred) acc.fe += (unsigned long long)deg;
}

// Fused push levels before the last: append y to the next frontier list Q
// (claimed) with its CSR row as push work items (row [e0, e0 + dy)), and to
// T (first), with the three list counters taken in one atomic round trip
// per warp. Whole warp calls.
template <int W>
__device__ __forceinline__ void append_next_and_touched(bool claimed, bool first, int32_t y, int32_t e0, int32_t dy,
                                                        const BfsBufs &b, int nslot, Acc &acc)
{
    constexpr int C = push_chunk(W);
    const int lane = threadIdx.x & 31;
    const unsigned mq = __ballot_sync(kFull, claimed), mt = __ballot_sync(kFull, first);
    if (!(mq | mt)) return;  // warp-uniform
    const int32_t nch = claimed ? (dy + C - 1) / C : 0;
    int32_t incl = nch;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int32_t t = __shfl_up_sync(kFull, incl, off);
        if (lane >= off) incl += t;
    }
    const int32_t total = __shfl_sync(kFull, incl, 31);
    int32_t bq = 0, bi = 0, bt = 0;
    if (lane == 0) {  // independent atomics: issued back to back
        if (mq) bq = atomicAdd(&b.ctl->q[nslot], __popc(mq));
        if (total) bi = atomicAdd(&b.ctl->qi[nslot], total);
        if (mt) bt = atomicAdd(&b.ctl->t, __popc(mt));
    }
    bq = __shfl_sync(kFull, bq, 0);
    bi = __shfl_sync(kFull, bi, 0);
    bt = __shfl_sync(kFull, bt, 0);
    const unsigned lt = lanemask_lt();
    if (claimed) pick3(b.Q, nslot)[bq + __popc(mq & lt)] = y;
    if (first) b.T[bt + __popc(mt & lt)] = y;
    if (nch) {
        int2 *items = pick3(b.I, nslot);
        const int32_t base = bi + incl - nch;
        for (int32_t k = 0; k < nch; k++) items[base + k] = make_int2(y, e0 + k * C);
    }
    if (claimed) acc.fe += (unsigned long long)dy;
}

// OR the W words of frontier row x into a.
template <int W>
__device__ __forceinline__ void or_row(uint64_t (&a)[W], const uint64_t *F, int32_t x)
{
    if constexpr (W == 1) {
        a[0] |= F[x];
    } else {
        const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(F + (size_t)x * W);
#pragma unroll
        for (int k = 0; k < W / 2; k++) {
            const ulonglong2 v = p[k];
            a[2 * k] |= v.x;
            a[2 * k + 1] |= v.y;
        }
    }
}

// Edges e = first, first+stride, ... < e1: OR the rows of flagged neighbours
// into a. Two edges per step so that each lane keeps two independent
// col -> flag -> row chains in flight.
template <int W>
__device__ __forceinline__ void gather_edges(uint64_t (&a)[W], const int32_t *col,
                                             const uint32_t *flc, const uint64_t *Fc,
                                             int32_t first, int32_t e1, int32_t stride,
                                             unsigned long long &gathered)
{
    int32_t e = first;
    for (; e + stride < e1; e += 2 * stride) {
        const int32_t x0 = __ldg(&col[e]);
        const int32_t x1 = __ldg(&col[e + stride]);
        const bool f0 = flag_test(flc, x0);
        const bool f1 = flag_test(flc, x1);
        if (f0) or_row<W>(a, Fc, x0);
        if (f1) or_row<W>(a, Fc, x1);
        gathered += (unsigned)f0 + (unsigned)f1;
    }
    if (e < e1) {
        const int32_t x0 = __ldg(&col[e]);
        if (flag_test(flc, x0)) {
            or_row<W>(a, Fc, x0);
            gathered++;
        }
    }
}

// OR a across the G lanes of each aligned lane group (G a power of two <= 32).
template <int W, int G>
__device__ __forceinline__ void group_or(uint64_t (&a)[W])
{
#pragma unroll
    for (int off = 1; off < G; off <<= 1) {
#pragma unroll
        for (int k = 0; k < W; k++) a[k] |= __shfl_xor_sync(kFull, a[k], off);
    }
}

// a[i] without dynamic register indexing.
template <int W>
__device__ __forceinline__ uint64_t select_word(const uint64_t (&a)[W], int i)
{
    uint64_t r = 0;
#pragma unroll
    for (int k = 0; k < W; k++)
        if (k == i) r = a[k];
    return r;
}

// ---------------------------------------------------------------------------
// level 0: sources. One block of up to 1024 threads; resets the level ring.
// ---------------------------------------------------------------------------
template <int W>
__device__ __forceinline__ void dev_seed(const int32_t *src, int32_t ns, BfsBufs b, const int32_t *rp)
{
    __shared__ unsigned long long s_fe;
    const int i = threadIdx.x;
    if (i == 0) {
        for (int k = 0; k < 3; k++) {
            b.ctl->q[k] = 0;
            b.ctl->qi[k] = 0;
            b.ctl->fe[k] = 0;
        }
        b.ctl->t = 0;
        s_fe = 0;
    }
    __syncthreads();
    unsigned long long d = 0;
    int32_t s = -1;
    if (i < ns) {
        s = src[i];
        d = (unsigned long long)(rp[s + 1] - rp[s]);
        const int word = i >> 6;
        const uint64_t bit = 1ull << (i & 63);
        b.V[(size_t)s * W + word] = bit;  // V(s) is zero between batches
        b.F[0][(size_t)s * W + word] = bit;  // F rows are zero between batches
        flag_set(b.flag[0], s);
        b.T[i] = s;
        // sampling: sources without a rate count every vertex they reach
        if (b.in_s && b.sel0 && b.sel0[s] == 0)
            atomicOr(reinterpret_cast<unsigned long long *>(&b.fullmask[word]), (unsigned long long)bit);
    }
    Acc dummy{0, 0, 0, 0, 0};
    append_frontier<W>(i < ns, s, (int32_t)d, b, 0, dummy, rp);  // Q[0] and the level-0 push items
    const unsigned long long ws = warp_sum(d);
    if ((i & 31) == 0 && ws) atomicAdd(&s_fe, ws);
    __syncthreads();
    if (i == 0) {
        b.ctl->t = ns;
        b.ctl->fe[0] = s_fe;
        if (s_fe) atomicAdd(b.edges, s_fe);  // every source scans its own row
    }
}


// Non-last levels: store the new words of vertex y (lanes gi < W of its
// group hold word gi), mark it in the next frontier, append it to Q (and T
// on its first visit). Whole warp calls.
template <int W, int G>
__device__ __forceinline__ void finish_vertex(bool act, int32_t y, int32_t dy, uint64_t nw, uint64_t v, int gi,
                                              int grp, uint64_t *V, uint64_t *Fn,
                                              uint32_t *fln, const BfsBufs &b, int nslot, Acc &acc,
                                              const int32_t *rp)
{
    const unsigned gmask = (G == 32) ? kFull : ((1u << G) - 1u);
    const unsigned any = __ballot_sync(kFull, nw != 0);
    const unsigned vany = __ballot_sync(kFull, v != 0);
    const bool gany = ((any >> (grp * G)) & gmask) != 0;
    const bool gv = ((vany >> (grp * G)) & gmask) != 0;
    if (act && gany && gi < W) {
        Fn[(size_t)y * W + gi] = nw;
        if (nw) V[(size_t)y * W + gi] = v | nw;
        acc.scanned += (unsigned long long)__popcll(nw) * (unsigned long long)dy;
    }
    const bool lead = act && gany && gi == 0;
    if (lead) flag_set(fln, y);
    append_frontier<W>(lead, y, dy, b, nslot, acc, rp);
    if (b.tflag && lead && !gv) flag_set(b.tflag, y);  // first visit (fused levels keep T by tflag)
    warp_append(lead && !gv, y, b.T, &b.ctl->t);
}

// Pull over a vertex list with G lanes per vertex (32/G vertices per warp).
template <int W, int G, bool LAST>
__device__ __forceinline__ void pull_groups(const int32_t *list, int32_t count, int64_t warp,
                                            int64_t nwarps, const GraphView &g, const uint32_t *alive,
                                            uint64_t *V, const uint64_t *Fc,
                                            const uint32_t *flc, uint64_t *Fn,
                                            uint32_t *fln, const BfsBufs &b, int nslot, Swar &sw,
                                            int32_t *cnt_s, Acc &acc)
{
    static_assert(G >= W && 32 % G == 0, "group");
    constexpr int VPW = 32 / G;
    const int lane = threadIdx.x & 31;
    const int gi = lane % G;
    const int grp = lane / G;
    const int32_t *rp = g.row_ptr;
    for (int64_t base = warp * VPW; base < count; base += nwarps * VPW) {  // warp-uniform
        const int64_t idx = base + grp;
        int32_t y = -1, dy = 0;
        bool act = false;
        uint64_t a[W];
#pragma unroll
        for (int k = 0; k < W; k++) a[k] = 0;
        if (idx < count) {
            y = list[idx];
            if (is_alive(alive, y)) {
                act = true;
                const int32_t e0 = rp[y], e1 = rp[y + 1];
                dy = e1 - e0;
                gather_edges<W>(a, g.col, flc, Fc, e0 + gi, e1, G, acc.gathered);
            }
        }
        // no frontier neighbour for any vertex of this warp (most warps at the
        // last level): nothing to combine, count or store
        bool mine = false;
#pragma unroll
        for (int k = 0; k < W; k++) mine |= a[k] != 0;
        if (!__any_sync(kFull, mine)) continue;  // warp-uniform
        group_or<W, G>(a);
        // a vertex none of whose neighbours is in the frontier has nothing to
        // do: its own rows are not touched (most vertices at the last level);
        // a is the same on every lane of the group here
        bool any_a = false;
#pragma unroll
        for (int k = 0; k < W; k++) any_a |= a[k] != 0;
        uint64_t nw = 0, v = 0;
        if (act && any_a && gi < W) {
            v = V[(size_t)y * W + gi];
            nw = select_word<W>(a, gi) & ~v;
        }
        if (act && any_a && gi == 0) acc.rows++;
        swar_step<W>(sw, nw & elig_mask(b, gi, act ? y : -1), cnt_s);
        if (b.rowcnt) {  // uniform
            int32_t rc = __popcll(nw & row_mask(gi, b.row_first));
#pragma unroll
            for (int off = 1; off < G; off <<= 1) rc += __shfl_xor_sync(kFull, rc, off);
            if (act && gi == 0 && rc) atomicAdd(&b.rowcnt[y], b.row_sign * rc);
        }
        if (LAST && b.newcnt) {  // uniform
            const unsigned gm = (G == 32) ? kFull : ((1u << G) - 1u);
            const unsigned nb = __ballot_sync(kFull, nw != 0), vb = __ballot_sync(kFull, v != 0);
            if (act && gi == 0 && ((nb >> (grp * G)) & gm) && !((vb >> (grp * G)) & gm)) acc.newv++;
        }
        if (!LAST) finish_vertex<W, G>(act, y, dy, nw, v, gi, grp, V, Fn, fln, b, nslot, acc, rp);
    }
}

// ---------------------------------------------------------------------------
// One level (lvl = 0-based distance of the frontier being expanded).
// LAST: the expansion reaching distance h; only counts (pull) or counts and
// records the rows to clear (push).
// ---------------------------------------------------------------------------
// FUSED (persistent kernel): one grid phase per level instead of two (level,
// then post). The frontier arrays and flags rotate over three slots (F[0],
// F[1], Fx and flag[0], flag[1], flagx, indexed like the lists Q), so the
// rows of the frontier the previous level expanded (slot (lvl+2)%3) are
// cleared here: nothing else reads or writes that slot during this level.
// The push direction writes the bits it discovers into V at once (atomicOr)
// and enters first-visited vertices into T (claimed in tflag), so V and T
// are complete at every barrier and no fold is needed. The last level writes
// neither V nor T.
template <class T>
__device__ __forceinline__ T *ring3(T *a0, T *a1, T *a2, int i)
{
    return i == 0 ? a0 : (i == 1 ? a1 : a2);
}

// Clear the frontier rows and flags of the vertices listed in ring slot
// `slot` (fused levels). W lanes per vertex.
// rot shifts the work to other warps than those starting at warp 0, so that
// its chain of loads runs beside the phase's other work instead of after it.
template <int W>
__device__ __forceinline__ void clear_slot(const BfsBufs &b, int slot, int32_t nq, int64_t rot)
{
    const int lane = threadIdx.x & 31;
    const int j = lane % W, grp = lane / W;
    constexpr int VPW = 32 / W;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t warp = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) + rot % nwarps;
    if (warp >= nwarps) warp -= nwarps;
    const int32_t *Qs = pick3(b.Q, slot);
    uint64_t *Fs = ring3(b.F[0], b.F[1], b.Fx, slot);
    uint32_t *fls = ring3(b.flag[0], b.flag[1], b.flagx, slot);
    for (int64_t base = warp * VPW; base < nq; base += nwarps * VPW) {
        const int64_t idx = base + grp;
        if (idx < nq) {
            const int32_t x = Qs[idx];
            Fs[(size_t)x * W + j] = 0;
            if (j == 0) flag_clear(fls, x);
        }
    }
}

// Fused push levels: frontier degree sum up to which the atomic on V is not
// preceded by a load of V.
constexpr unsigned long long kProbeEdges = 1ull << 15;

template <int W, bool LAST, bool FUSED = false>
__device__ __forceinline__ void dev_level(GraphView g, const uint32_t *alive, BfsBufs b,
                                                  int lvl, BfsTuning tune)
{
    static_assert(W == 1 || W == 2 || W == 4 || W == 8 || W == 16, "W");
    __shared__ int32_t cnt_s[64 * W];
    __shared__ uint64_t red[kBlock / 32][W];

    const int cslot = lvl % 3, nslot = (lvl + 1) % 3;
    const int cb = lvl & 1, nb_ = cb ^ 1;
    const uint64_t *Fc = FUSED ? ring3(b.F[0], b.F[1], b.Fx, cslot) : pick2(b.F, cb);
    const uint32_t *flc = FUSED ? ring3(b.flag[0], b.flag[1], b.flagx, cslot) : pick2(b.flag, cb);
    uint64_t *Fn = FUSED ? ring3(b.F[0], b.F[1], b.Fx, nslot) : pick2(b.F, nb_);
    uint32_t *fln = FUSED ? ring3(b.flag[0], b.flag[1], b.flagx, nslot) : pick2(b.flag, nb_);
    uint64_t *V = b.V;
    // the frontier's list lengths, loaded together (one round trip)
    const unsigned long long fe_c = b.ctl->fe[cslot];
    const int32_t nq_c = b.ctl->q[cslot];
    const int32_t ni = b.ctl->qi[cslot];
    const int32_t nq_old = (FUSED && lvl > 0) ? b.ctl->q[(lvl + 2) % 3] : 0;
    const bool push = tune.alpha > 0 && fe_c * (unsigned long long)tune.alpha < tune.m_alive;

    // on the upper half of the warps: the push work items start at warp 0
    if (FUSED && lvl > 0)
        clear_slot<W>(b, (lvl + 2) % 3, nq_old, ((int64_t)gridDim.x * blockDim.x >> 5) / 2);
    for (int i = threadIdx.x; i < 64 * W; i += blockDim.x) cnt_s[i] = 0;
    // Algorithmic bytes of this level. Pull: 4 n_b (row offsets) + 4 m_b
    // (column ids) over the n_b alive rows and their m_b entries, 8 W per
    // frontier entry gathered (the neighbour's frontier row), and 16 W per
    // vertex with a frontier neighbour (its visited row read, its
    // next-frontier row written), the last two counted as the level runs.
    // Push: the frontier rows it reads
    // (8 W per frontier vertex) and, per frontier entry, the column id, the
    // neighbour's visited row and its next-frontier row (4 + 16 W).
    if (blockIdx.x == 0 && threadIdx.x == 0 && b.alg_bytes) {
        const unsigned long long nb = (unsigned long long)tune.n_alive;
        const unsigned long long bytes =
            push ? fe_c * (4ull + 16ull * W) + (unsigned long long)nq_c * 8ull * W
                 : 4ull * nb + 4ull * tune.m_alive;
        atomicAdd(b.alg_bytes, bytes);
    }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int j = lane % W;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t *rp = g.row_ptr;
    const int32_t *col = g.col;
    Swar sw;
    sw.reset();
    Acc acc{0, 0, 0, 0, 0};

    if (push) {
        // ---------------- push: frontier vertices scatter to neighbours ----
        constexpr int SLOTS = 32 / W;
        const int slot = lane / W;
        const int grp = slot;
        const unsigned gmask = (1u << W) - 1u;
        constexpr int C = push_chunk(W);
        const int2 *Ic = pick3(b.I, cslot);
        // one edge of the expansion: y = col[e] gets fx & ~V(y) (per-phase
        // levels, and the last fused level, which writes neither V nor T)
        auto edge = [&](int32_t e, int32_t e1, uint64_t fx) {
            int32_t y = -1;
            uint64_t nbits = 0, fresh = 0, v = 0;
            if (e < e1) {
                y = __ldg(&col[e]);
                if (is_alive(alive, y)) {
                    v = V[(size_t)y * W + j];
                    nbits = fx & ~v;
                    if (nbits) {
                        const unsigned long long old =
                            atomicOr(reinterpret_cast<unsigned long long *>(&Fn[(size_t)y * W + j]),
                                     (unsigned long long)nbits);
                        fresh = nbits & ~(uint64_t)old;
                        if (b.rowcnt) {
                            const uint64_t rf = fresh & row_mask(j, b.row_first);
                            if (rf) atomicAdd(&b.rowcnt[y], b.row_sign * __popcll(rf));
                        }
                    }
                }
            }
            swar_step<W>(sw, fresh & elig_mask(b, j, y), cnt_s);
            const unsigned any = __ballot_sync(kFull, nbits != 0);
            const bool lead = (j == 0) && (((any >> (grp * W)) & gmask) != 0);
            bool claimed = false;
            int32_t dy = 0;
            if (lead) {
                claimed = flag_claim(fln, y);
                dy = rp[y + 1] - rp[y];
            }
            append_frontier<W>(claimed, y, (FUSED && LAST) ? 0 : dy, b, nslot, acc, rp);
            if constexpr (FUSED && LAST) {
                const unsigned vany = __ballot_sync(kFull, v != 0);
                const bool gv = ((vany >> (grp * W)) & gmask) != 0;
                if (b.newcnt && claimed && !gv) acc.newv++;
            }
        };
        // Fused levels before the last: V itself takes the atomicOr (its old
        // value says which bits are new), the new bits go on into the next
        // frontier row without a return value, and the frontier and
        // touched-list claims, and then the three list appends, each take one
        // round trip. Same result as edge: every bit is new for exactly one
        // writer. A small frontier skips the load of V before the atomic (one
        // round trip less); a large one keeps it, so that the atomics on
        // much-visited rows stay few.
        const bool probe = fe_c > kProbeEdges;
        auto edge_fused = [&](int32_t e, int32_t e1, uint64_t fx) {
            int32_t y = -1;
            uint64_t fresh = 0;
            if (e < e1) {
                y = __ldg(&col[e]);
                uint64_t nb = is_alive(alive, y) ? fx : 0;
                if (probe && nb) nb &= ~V[(size_t)y * W + j];
                if (nb) {
                    const unsigned long long old = atomicOr(
                        reinterpret_cast<unsigned long long *>(&V[(size_t)y * W + j]), (unsigned long long)nb);
                    fresh = nb & ~(uint64_t)old;
                    if (fresh) {
                        atomicOr(reinterpret_cast<unsigned long long *>(&Fn[(size_t)y * W + j]),
                                 (unsigned long long)fresh);
                        if (b.rowcnt) {
                            const uint64_t rf = fresh & row_mask(j, b.row_first);
                            if (rf) atomicAdd(&b.rowcnt[y], b.row_sign * __popcll(rf));
                        }
                    }
                }
            }
            swar_step<W>(sw, fresh & elig_mask(b, j, y), cnt_s);
            const unsigned fany = __ballot_sync(kFull, fresh != 0);
            const bool lead = (j == 0) && (((fany >> (grp * W)) & gmask) != 0);
            bool claimed = false, first = false;
            int32_t e0 = 0, dy = 0;
            if (lead) {
                const uint32_t bit = 1u << (y & 31);
                const uint32_t of = atomicOr(&fln[y >> 5], bit);
                const uint32_t ot = atomicOr(&b.tflag[y >> 5], bit);
                e0 = rp[y];
                dy = rp[y + 1] - e0;
                claimed = (of & bit) == 0;
                first = (ot & bit) == 0;
            }
            append_next_and_touched<W>(claimed, first, y, e0, dy, b, nslot, acc);
            // the plain-BFS edges of the sources that reach y now
            const int32_t dyg = __shfl_sync(kFull, dy, lane & ~(W - 1));
            if (fresh) acc.scanned += (unsigned long long)__popcll(fresh) * (unsigned long long)dyg;
        };
        // The last fused level with one-word rows (a small frontier): the
        // next-frontier row takes the atomicOr beside the load of V (the last
        // level writes no V), a bit is new when neither had it, and the one
        // writer that finds the row empty lists y for the clearing at the
        // batch's end; no frontier flag is claimed.
        auto edge_last1 = [&](int32_t e, int32_t e1, uint64_t fx) {
            int32_t y = -1;
            uint64_t fresh = 0;
            bool listed = false, seen = false;
            if (e < e1) {
                y = __ldg(&col[e]);
                if (fx && is_alive(alive, y)) {
                    const uint64_t v = V[y];
                    const unsigned long long old =
                        atomicOr(reinterpret_cast<unsigned long long *>(&Fn[y]), (unsigned long long)fx);
                    fresh = fx & ~(uint64_t)old & ~v;
                    listed = old == 0;
                    seen = v != 0;
                    if (b.rowcnt) {
                        const uint64_t rf = fresh & row_mask(0, b.row_first);
                        if (rf) atomicAdd(&b.rowcnt[y], b.row_sign * __popcll(rf));
                    }
                }
            }
            swar_step<W>(sw, fresh & elig_mask(b, 0, y), cnt_s);
            warp_append(listed, y, pick3(b.Q, nslot), &b.ctl->q[nslot]);
            if (b.newcnt && listed && !seen) acc.newv++;
        };
        // work items: up to C entries of one frontier row each, one warp per item
        for (int64_t it = warp; it < ni; it += nwarps) {  // warp-uniform
            const int2 item = Ic[it];
            const int32_t x = item.x;
            const int32_t rend = rp[x + 1];
            const int32_t e1 = item.y + C < rend ? item.y + C : rend;
            const uint64_t fx = Fc[(size_t)x * W + j];
            for (int32_t eb = item.y; eb < e1; eb += SLOTS) {
                if constexpr (FUSED && !LAST) {
                    edge_fused(eb + slot, e1, fx);
                } else if constexpr (FUSED && LAST && W == 1) {
                    if (probe)
                        edge(eb + slot, e1, fx);
                    else
                        edge_last1(eb + slot, e1, fx);
                } else {
                    edge(eb + slot, e1, fx);
                }
            }
        }
    } else {
        // ---------------- pull: every alive vertex gathers its neighbours ----
        // A group of G lanes takes one vertex; each lane walks its own share
        // of the edges (two independent chains per lane), ORs whole frontier
        // rows into a[0..W-1], and the group ORs the lanes together. Lane
        // gi < W of the group then finishes word gi.
        // light (deg <= kLightMax): G = max(8, W) lanes per vertex
        pull_groups<W, (W > 8 ? W : 8), LAST>(g.light, g.n_light, warp, nwarps, g, alive, V, Fc, flc, Fn, fln,
                                              b, nslot, sw, cnt_s, acc);
        // medium (deg <= kMediumMax): one warp per vertex
        pull_groups<W, 32, LAST>(g.medium, g.n_medium, warp, nwarps, g, alive, V, Fc, flc, Fn, fln, b, nslot,
                                 sw, cnt_s, acc);
        // heavy: one block per vertex
        {
            const int wid = threadIdx.x >> 5;
            const int nwarp_blk = blockDim.x >> 5;
            for (int64_t i = blockIdx.x; i < g.n_heavy; i += gridDim.x) {
                const int32_t y = g.heavy[i];
                const bool act = is_alive(alive, y);  // block-uniform
                const int32_t e0 = rp[y], e1 = rp[y + 1];
                if (act) {
                    uint64_t a[W];
#pragma unroll
                    for (int k = 0; k < W; k++) a[k] = 0;
                    gather_edges<W>(a, col, flc, Fc, e0 + (int32_t)threadIdx.x, e1, (int32_t)blockDim.x,
                                    acc.gathered);
                    group_or<W, 32>(a);
                    if (lane < W) red[wid][lane] = select_word<W>(a, lane);
                }
                __syncthreads();
                if (wid == 0) {
                    uint64_t nw = 0, v = 0;
                    if (act && lane < W) {
                        uint64_t m = 0;
                        for (int w = 0; w < nwarp_blk; w++) m |= red[w][lane];
                        v = V[(size_t)y * W + j];
                        nw = m & ~v;
                    }
                    if (act && lane == 0) acc.rows++;
                    swar_step<W>(sw, nw & elig_mask(b, lane, act ? y : -1), cnt_s);
                    if (b.rowcnt) {
                        int32_t rc = __popcll(nw & row_mask(lane, b.row_first));
#pragma unroll
                        for (int off = 1; off < 32; off <<= 1) rc += __shfl_xor_sync(kFull, rc, off);
                        if (act && lane == 0 && rc) atomicAdd(&b.rowcnt[y], b.row_sign * rc);
                    }
                    if (LAST && b.newcnt) {
                        const unsigned nb = __ballot_sync(kFull, nw != 0), vb = __ballot_sync(kFull, v != 0);
                        if (act && lane == 0 && nb && !vb) acc.newv++;
                    }
                    if (!LAST) finish_vertex<W, 32>(act, y, e1 - e0, nw, v, lane, 0, V, Fn, fln, b, nslot, acc, rp);
                }
                __syncthreads();
            }
        }
    }

    swar_flush<W>(sw, cnt_s);
    const unsigned long long sc = warp_sum(acc.scanned);
    const unsigned long long fe = warp_sum(acc.fe);
    const unsigned long long nv = warp_sum(acc.newv);
    const unsigned long long gb = warp_sum(8ull * W * (acc.gathered + 2ull * acc.rows));
    if (lane == 0) {
        if (sc) atomicAdd(b.edges, sc);
        if (fe) atomicAdd(&b.ctl->fe[nslot], fe);
        if (nv) atomicAdd(b.newcnt, nv);
        if (gb && b.alg_bytes) atomicAdd(b.alg_bytes, gb);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 64 * W; i += blockDim.x) {
        const int32_t c = cnt_s[i];
        if (c) atomicAdd(&b.cnt[i], c);
    }
}

// ---------------------------------------------------------------------------
// After level lvl: (push) fold the next frontier into V; clear the rows of the
// expanded frontier (and, at the last level, of the next one); reset the ring
// slot two levels ahead.
// ---------------------------------------------------------------------------
template <int W, bool LAST>
__device__ __forceinline__ void dev_post(GraphView g, BfsBufs b, int lvl, BfsTuning tune)
{
    const int cslot = lvl % 3, nslot = (lvl + 1) % 3, oslot = (lvl + 2) % 3;
    const int cb = lvl & 1, nb_ = cb ^ 1;
    const bool push = use_push(b.ctl, cslot, tune);
    const int lane = threadIdx.x & 31;
    const int j = lane % W;
    const int grp = lane / W;
    constexpr int VPW = 32 / W;
    const unsigned gmask = (1u << W) - 1u;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t *rp = g.row_ptr;
    unsigned long long scanned = 0;

    if (blockIdx.x == 0 && threadIdx.x == 0) {
        b.ctl->q[oslot] = 0;
        b.ctl->qi[oslot] = 0;
        b.ctl->fe[oslot] = 0;
    }
    const int32_t nq = b.ctl->q[cslot];
    const int32_t nn = b.ctl->q[nslot];
    const int32_t *Qc = pick3(b.Q, cslot);
    const int32_t *Qn = pick3(b.Q, nslot);
    uint64_t *Fc = pick2(b.F, cb);
    uint64_t *Fn = pick2(b.F, nb_);
    uint32_t *flc = pick2(b.flag, cb);
    uint32_t *fln = pick2(b.flag, nb_);

    // clear the expanded frontier's rows
    for (int64_t base = warp * VPW; base < nq; base += nwarps * VPW) {
        const int64_t idx = base + grp;
        if (idx < nq) {
            const int32_t x = Qc[idx];
            Fc[(size_t)x * W + j] = 0;
            if (j == 0) flag_clear(flc, x);
        }
    }
    if (push) {
        for (int64_t base = warp * VPW; base < nn; base += nwarps * VPW) {
            const int64_t idx = base + grp;
            int32_t y = -1;
            uint64_t f = 0, v = 0;
            if (idx < nn) {
                y = Qn[idx];
                f = Fn[(size_t)y * W + j];
                if (LAST) {
                    Fn[(size_t)y * W + j] = 0;
                    if (j == 0) flag_clear(fln, y);
                } else {
                    v = b.V[(size_t)y * W + j];
                    if (f) b.V[(size_t)y * W + j] = v | f;
                    scanned += (unsigned long long)__popcll(f) * (unsigned long long)(rp[y + 1] - rp[y]);
                }
            }
            if (!LAST) {
                const unsigned vany = __ballot_sync(kFull, v != 0);
                const bool gv = ((vany >> (grp * W)) & gmask) != 0;
                warp_append(idx < nn && j == 0 && !gv, y, b.T, &b.ctl->t);
            }
        }
    }
    scanned = warp_sum(scanned);
    if (lane == 0 && scanned) atomicAdd(b.edges, scanned);
}

// Lazy-mode bound on what an alive u loses besides the deleted vertices it
// reaches through survivors. Every such lost vertex lies, on some shortest
// path from u, beyond the first deleted vertex d on it: within h - s hops of
// d, where s = dist(u, d) through survivors, 1 <= s <= h-1 (Observation 2).
// So the loss is at most the sum over deleted d within h-1 of u of the size
// of d's (h-s)-ball: at most d's h-degree bound wdeg[d], and at most its row
// length when h - s = 1. Called after the level that completes the sources
// within `radius` hops: radius h-1 adds min(row length, wdeg) per source bit,
// radius h-2 adds the rest, wdeg - min(row length, wdeg), for the sources
// already that close. One thread per vertex of T; plain adds (each vertex is
// once in T), saturating at INT_MAX. Threads are taken from the last one
// down, away from the warps that take a level's first work items when the
// pass shares a phase with the level.
template <int W>
//
// slack (lazy mode's batch seeded at the deleted set, last radius; else
// nullptr): wsum[u] is then final, and u widens its slack by
// min(|T|, wsum[u]) (Observation 2: what it loses besides the sources it still
// reaches lies within h-1 of them), capped at deg[u] read during the level
// (any value at least the final one keeps deg - slack a lower bound). The
// last level writes no T, so |T| is final too.
__device__ __forceinline__ void dev_weight_pass(const BfsBufs &b, const int32_t *src, const int32_t *rp,
                                                const uint32_t *alive, bool last_radius, int32_t *slack = nullptr,
                                                const int32_t *deg = nullptr)
{
    const int32_t nt = b.ctl->t;
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = nthr - 1 - ((int64_t)blockIdx.x * blockDim.x + threadIdx.x); i < nt; i += nthr) {
        const int32_t u = b.T[i];
        if (!is_alive(alive, u)) continue;
        const int32_t w0 = b.wsum[u];
        const int32_t s0 = slack ? slack[u] : 0;
        const int32_t du = slack ? deg[u] : 0;
        long long sum = 0;
#pragma unroll 1
        for (int j = 0; j < W; j++) {
            uint64_t w = b.V[(size_t)u * W + j];
            while (w) {
                const int p = __ffsll((long long)w) - 1;
                w &= w - 1;
                const int32_t d = src[j * 64 + p];
                const int32_t wd = b.wdeg[d];
                const int32_t r1 = min(rp[d + 1] - rp[d], wd);
                sum += last_radius ? r1 : wd - r1;
            }
        }
        const int32_t ws = (int32_t)min((long long)w0 + sum, (long long)INT_MAX);
        if (sum) b.wsum[u] = ws;
        if (slack) {
            const long long sl = (long long)s0 + min(nt, ws);
            slack[u] = (int32_t)(sl < du ? sl : du);
        }
    }
}

// End of batch: zero the V rows in T, write the h-degrees of the sources.
template <int W>
__device__ __forceinline__ void dev_end(BfsBufs b, const int32_t *src, int32_t ns,
                                                int32_t *deg)
{
    const int lane = threadIdx.x & 31;
    const int j = lane % W;
    const int grp = lane / W;
    constexpr int VPW = 32 / W;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t warp = tid >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t nt = b.ctl->t;
    for (int64_t base = warp * VPW; base < nt; base += nwarps * VPW) {
        const int64_t idx = base + grp;
        if (idx < nt) b.V[(size_t)b.T[idx] * W + j] = 0;
    }
    if (tid < ns) {
        const int32_t s = src[tid], c = b.cnt[tid];
        if (b.sel) {
            b.sel[s] = c;
            if (b.sel0) {
                const int32_t s0 = b.sel0[s];
                deg[s] = s0 > 0 ? (c > 0 ? (int32_t)((long long)c * b.d0[s] / s0) : 0) : c;
            }
        } else {
            deg[s] = c;
        }
        b.cnt[tid] = 0;
    }
    if (b.fullmask && tid < W) b.fullmask[tid] = 0;
}


// End of a batch run with fused levels: zero the V rows and tflag of T (and
// wsum, when set), the frontier rows and flags of the last level's slot and
// of the slot its push direction wrote, and the per-source counts. Per source
// position i < ns: when deg is set, deg[src[i]] = its count; when p.ming is
// set too, the count also goes into its graph's exact minimum (the refine
// step of the lazy mode). Nothing here reads what a phase running beside it
// writes, other than these rows (the lazy mode's batch seeded at the deleted
// set ends inside the next round's minimum scan; its slack update ran in the
// weight pass of its last level).
template <int W>
__device__ __forceinline__ void dev_end_fused(const BfsBufs &b, const int32_t *src, int32_t ns, int32_t h,
                                              int32_t *deg, const PeelView *pmin)
{
    const int lane = threadIdx.x & 31;
    const int j = lane % W;
    const int grp = lane / W;
    constexpr int VPW = 32 / W;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t warp = tid >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t nt = b.ctl->t;
    const int32_t nq1 = b.ctl->q[(h - 1) % 3], nq2 = b.ctl->q[h % 3];
    for (int64_t base = warp * VPW; base < nt; base += nwarps * VPW) {
        const int64_t idx = base + grp;
        if (idx < nt) {
            const int32_t u = b.T[idx];
            b.V[(size_t)u * W + j] = 0;
            if (j == 0) {
                flag_clear(b.tflag, u);
                if (b.wsum) b.wsum[u] = 0;
            }
        }
    }
    // the other pieces start at other warps (their load chains run side by
    // side): the two slots at a third and two thirds of the grid, the
    // sources from the last thread down
    clear_slot<W>(b, (h - 1) % 3, nq1, nwarps / 3);
    clear_slot<W>(b, h % 3, nq2, 2 * nwarps / 3);
    const int64_t si = (int64_t)gridDim.x * blockDim.x - 1 - tid;
    if (si < ns) {
        const int32_t c = b.cnt[si];
        b.cnt[si] = 0;
        if (deg) deg[src[si]] = c;
        if (pmin) atomicMin(&pmin->ming[pmin->gid ? __ldg(&pmin->gid[src[si]]) : 0], c);
    }
}

// ===========================================================================
// Peel rounds
// ===========================================================================



__device__ __forceinline__ int32_t graph_of(const PeelView &p, int32_t v) { return p.gid ? __ldg(&p.gid[v]) : 0; }

__device__ __forceinline__ void dev_iota(int32_t *dst, int32_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (int32_t)i;
}

__device__ __forceinline__ void dev_alive_init(uint32_t *alive, int32_t n)
{
    const int32_t nw = (n + 31) >> 5;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x) {
        const int32_t rem = n - (int32_t)w * 32;
        alive[w] = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
    }
}

// Whole warp calls: atomicMin of m into arr[g] per graph, one atomic per warp
// when the warp's contributing lanes share a graph (lanes with g < 0 skip).
__device__ __forceinline__ void warp_min_by_graph(int32_t m, int32_t g, int32_t *arr)
{
    const unsigned act = __ballot_sync(kFull, g >= 0);
    if (!act) return;
    const int lane = threadIdx.x & 31;
    const int32_t g0 = __shfl_sync(kFull, g, __ffs(act) - 1);
    if (__all_sync(kFull, g < 0 || g == g0)) {
        int32_t r = g >= 0 ? m : INT_MAX;
#pragma unroll
        for (int off = 16; off; off >>= 1) r = min(r, __shfl_xor_sync(kFull, r, off));
        if (lane == 0) atomicMin(&arr[g0], r);
    } else if (g >= 0) {
        atomicMin(&arr[g], m);
    }
}

// Per-graph minimum over alive vertices: exact h-degrees into p.ming; in the
// lazy mode, vertices with slack give their lower bound deg - slack to p.mind
// (and their upper bound deg to p.minub). One graph: every thread keeps its
// own minima, reduced over the block, one atomic per block and quantity.
// Whole blocks call.
__device__ __forceinline__ void dev_min_alive_deg(int32_t n, const uint32_t *alive,
                                                          const int32_t *deg, PeelView p)
{
    const int lane = threadIdx.x & 31;
    const int32_t nw = (n + 31) >> 5;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    if (p.G == 1) {
        __shared__ int32_t red[3][32];
        int32_t me = INT_MAX, ml = INT_MAX, mu = INT_MAX;
        // U words per warp step, the alive words and the degrees and slacks
        // loaded together whatever the alive bits (one round trip per step;
        // the scan is latency-bound: a handful of words per warp)
        constexpr int U = 8;
        for (int64_t w0 = warp * U; w0 < nw; w0 += nwarps * U) {
            uint32_t aw[U];
            int32_t d[U], sl[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int32_t v = (int32_t)(w0 + u) * 32 + lane;
                const bool in = w0 + u < nw && v < n;
                aw[u] = (w0 + u < nw) ? alive[w0 + u] : 0u;
                d[u] = in ? deg[v] : INT_MAX;
                sl[u] = (in && p.slack) ? p.slack[v] : 0;
            }
#pragma unroll
            for (int u = 0; u < U; u++)
                if (!((aw[u] >> lane) & 1u)) d[u] = INT_MAX;
#pragma unroll
            for (int u = 0; u < U; u++) {
                if (d[u] == INT_MAX) continue;
                if (sl[u] == 0) {
                    me = min(me, d[u]);
                } else {
                    ml = min(ml, d[u] - sl[u]);
                    mu = min(mu, d[u]);
                }
            }
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            me = min(me, __shfl_xor_sync(kFull, me, off));
            ml = min(ml, __shfl_xor_sync(kFull, ml, off));
            mu = min(mu, __shfl_xor_sync(kFull, mu, off));
        }
        const int wid = threadIdx.x >> 5;
        if (lane == 0) {
            red[0][wid] = me;
            red[1][wid] = ml;
            red[2][wid] = mu;
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            const int nwb = blockDim.x >> 5;
            me = lane < nwb ? red[0][lane] : INT_MAX;
            ml = lane < nwb ? red[1][lane] : INT_MAX;
            mu = lane < nwb ? red[2][lane] : INT_MAX;
#pragma unroll
            for (int off = 16; off; off >>= 1) {
                me = min(me, __shfl_xor_sync(kFull, me, off));
                ml = min(ml, __shfl_xor_sync(kFull, ml, off));
                mu = min(mu, __shfl_xor_sync(kFull, mu, off));
            }
            if (lane == 0) {
                if (me != INT_MAX) atomicMin(&p.ming[0], me);
                if (p.slack && ml != INT_MAX) atomicMin(&p.mind[0], ml);
                if (p.slack && mu != INT_MAX) atomicMin(&p.minub[0], mu);
            }
        }
        __syncthreads();
        return;
    }
    for (int64_t w = warp; w < nw; w += nwarps) {
        const int32_t v = (int32_t)w * 32 + lane;
        const uint32_t aw = alive[w];
        if (!aw) continue;  // warp-uniform
        const bool a = v < n && ((aw >> lane) & 1u);
        const int32_t gv = a ? graph_of(p, v) : -1;
        const int32_t sl = (a && p.slack) ? p.slack[v] : 0;
        const int32_t d = a ? deg[v] : INT_MAX;
        warp_min_by_graph(d, (a && sl == 0) ? gv : -1, p.ming);
        if (p.slack) {
            warp_min_by_graph(d - sl, (a && sl > 0) ? gv : -1, p.mind);
            warp_min_by_graph(d, (a && sl > 0) ? gv : -1, p.minub);
        }
    }
}

// Lazy mode: the coming level is max(k_g, true min of graph g) <= T_g =
// max(k_g, min(exact min, smallest upper bound with slack)). An alive vertex
// whose lower bound deg - slack is at most T_g might be peeled at that level
// or be the minimum; it is listed (class region of cand, p.ncand) for an
// exact recompute and its slack dropped. Every other vertex with slack has a
// true h-degree above T_g, so it is neither peeled nor the minimum.
__device__ __forceinline__ void dev_refine_select(int32_t n, const uint32_t *alive, const int32_t *deg, PeelView p,
                                                  int32_t *cand)
{
    const int lane = threadIdx.x & 31;
    const int32_t nw = (n + 31) >> 5;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    if (p.G == 1) {
        // one graph: the threshold is one number, and no vertex is picked at
        // all unless the least lower bound reaches it
        const int32_t T = max(p.kg[0], min(p.ming[0], p.minub[0]));
        if (p.mind[0] > T) return;
        int32_t *cand0 = cand + __ldg(&p.cls_off[0]);
        // U words per warp step: alive words, slacks and degrees loaded
        // together, one list atomic per step
        constexpr int U = 8;
        const unsigned lt = lanemask_lt();
        for (int64_t w0 = warp * U; w0 < nw; w0 += nwarps * U) {
            uint32_t aw[U];
            int32_t d[U], sl[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int32_t v = (int32_t)(w0 + u) * 32 + lane;
                const bool in = w0 + u < nw && v < n;
                aw[u] = (w0 + u < nw) ? alive[w0 + u] : 0u;
                sl[u] = in ? p.slack[v] : 0;
                d[u] = in ? deg[v] : 0;
            }
            unsigned m[U];
            int32_t tot = 0;
#pragma unroll
            for (int u = 0; u < U; u++) {
                const bool pick = ((aw[u] >> lane) & 1u) && sl[u] > 0 && d[u] - sl[u] <= T;
                m[u] = __ballot_sync(kFull, pick);
                tot += __popc(m[u]);
            }
            if (tot == 0) continue;  // warp-uniform
            int32_t base = 0;
            if (lane == 0) base = atomicAdd(&p.ncand[0], tot);
            base = __shfl_sync(kFull, base, 0);
#pragma unroll
            for (int u = 0; u < U; u++) {
                if ((m[u] >> lane) & 1u) {
                    const int32_t v = (int32_t)(w0 + u) * 32 + lane;
                    p.slack[v] = 0;
                    cand0[base + __popc(m[u] & lt)] = v;
                }
                base += __popc(m[u]);
            }
        }
        return;
    }
    for (int64_t w = warp; w < nw; w += nwarps) {
        const uint32_t aw = alive[w];
        if (!aw) continue;  // warp-uniform
        const int32_t v = (int32_t)w * 32 + lane;
        bool pick = false;
        int32_t cv = -1;
        if (v < n && ((aw >> lane) & 1u)) {
            const int32_t sl = p.slack[v];
            if (sl > 0) {
                const int32_t g = graph_of(p, v);
                const int32_t T = max(p.kg[g], min(p.ming[g], p.minub[g]));
                if (p.mind[g] <= T) {
                    if (deg[v] - sl <= T) {
                        pick = true;
                        cv = __ldg(&p.cls[g]);
                        p.slack[v] = 0;
                    }
                }
            }
        }
        const unsigned m = __ballot_sync(kFull, pick);
        if (!m) continue;
        const int32_t c0 = __shfl_sync(kFull, cv, __ffs(m) - 1);
        if (__all_sync(kFull, !pick || cv == c0)) {
            warp_append(pick, v, cand + __ldg(&p.cls_off[c0]), &p.ncand[c0]);
        } else if (pick) {
            cand[__ldg(&p.cls_off[cv]) + atomicAdd(&p.ncand[cv], 1)] = v;
        }
    }
}

// After the exact recompute of the listed vertices: fold their h-degrees into
// the per-graph exact minimum.
__device__ __forceinline__ void dev_min_over_list(const int32_t *list, int32_t count, const int32_t *deg, PeelView p)
{
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < count; i0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + threadIdx.x;  // block-uniform loop
        int32_t v = -1, d = INT_MAX, g = -1;
        if (i < count) {
            v = list[i];
            d = deg[v];
            g = graph_of(p, v);
        }
        warp_min_by_graph(d, g, p.ming);
    }
}

// k_g <- max(k_g, min alive deg of g) (Algorithm 1 moves a vertex to
// B[max{k, d}], so the level never falls); reset the per-round counters.
__device__ __forceinline__ void set_level_part(PeelView p, PeelState *st, int32_t i0, int32_t step, bool leader)
{
    for (int32_t g = i0; g < p.G; g += step) {
        const int32_t m = p.ming[g];
        if (m != INT_MAX && m > p.kg[g]) p.kg[g] = m;
        p.ming[g] = INT_MAX;
        if (p.mind) p.mind[g] = INT_MAX;
        if (p.minub) p.minub[g] = INT_MAX;
    }
    if (leader) {
        st->nD = 0;
        st->nA = 0;
        st->aq[0] = st->aq[1] = st->aq[2] = 0;
    }
    for (int32_t c = i0; c < p.ncls; c += step) {
        p.nAc[c] = 0;
        p.nDc[c] = 0;
        if (p.ncand) p.ncand[c] = 0;
    }
}

__device__ __forceinline__ void dev_set_level(PeelView p, PeelState *st)
{
    set_level_part(p, st, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x,
                   blockIdx.x == 0 && threadIdx.x == 0);
}

// The same on one thread (few graphs: run inside a grid barrier's serial step).
__device__ __forceinline__ void dev_set_level_serial(PeelView p, PeelState *st) { set_level_part(p, st, 0, 1, true); }

// D = {alive v : deg[v] <= k_g(v)}: core[v] = k, rnd[v] = round, clear the
// alive bit, append v to dlist (st->aq[0]; skipped when dlist is null) and to
// its class region of dcls.
// vis is rewritten whole: exactly the bits of D. A warp owns one 32-vertex
// word of each bitset.
__device__ __forceinline__ void dev_peel_compact(int32_t n, const int32_t *rp,
                                                         uint32_t *alive, const int32_t *deg,
                                                         PeelView p, PeelState *st, int32_t *core,
                                                         int32_t *rnd, uint32_t *vis,
                                                         int32_t *dlist, int32_t *dcls)
{
    const int lane = threadIdx.x & 31;
    const int32_t nw = (n + 31) >> 5;
    const int32_t r = st->round;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // one word of the alive bitset whose deleted lanes are `del` (mask != 0)
    auto peel_word = [&](int64_t w, uint32_t aw, unsigned mask, bool del, int32_t y, int32_t k, int32_t gy) {
        unsigned long long dsum = 0;
        if (del) {
            core[y] = k;
            if (rnd) rnd[y] = r;
            dsum = (unsigned long long)(rp[y + 1] - rp[y]);
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) dsum += __shfl_xor_sync(kFull, dsum, off);
        int32_t base = 0;
        if (lane == 0) {
            alive[w] = aw & ~mask;
            if (vis) vis[w] = mask;  // every word of vis is written: it starts the round's affected BFS
            if (dlist) base = atomicAdd(&st->aq[0], __popc(mask));
            atomicAdd(&st->nD, __popc(mask));
            atomicSub(&st->alive, __popc(mask));
            atomicAdd(&st->m_alive, 0ull - dsum);
        }
        if (dlist) {  // uniform
            base = __shfl_sync(kFull, base, 0);
            if (del) dlist[base + __popc(mask & lanemask_lt())] = y;
        }
        // class regions of the deleted-source lists
        const int32_t cy = del ? __ldg(&p.cls[gy]) : -1;
        const int32_t c0 = __shfl_sync(kFull, cy, __ffs(mask) - 1);
        if (__all_sync(kFull, !del || cy == c0)) {
            warp_append(del, y, dcls + __ldg(&p.cls_off[c0]), &p.nDc[c0]);
        } else if (del) {
            dcls[__ldg(&p.cls_off[cy]) + atomicAdd(&p.nDc[cy], 1)] = y;
        }
    };
    if (p.G == 1 && !vis && !dlist) {
        // one graph, neither affected-set bits nor list to write (lazy mode):
        // U words per warp step, alive words and degrees loaded together,
        // one set of counter atomics and one class-list atomic per step
        const int32_t k = p.kg[0];
        const int32_t c0 = __ldg(&p.cls[0]);
        int32_t *dc = dcls + __ldg(&p.cls_off[c0]);
        const unsigned lt = lanemask_lt();
        constexpr int U = 8;
        for (int64_t w0 = warp * U; w0 < nw; w0 += nwarps * U) {
            uint32_t aw[U];
            int32_t d[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int32_t y = (int32_t)(w0 + u) * 32 + lane;
                aw[u] = (w0 + u < nw) ? alive[w0 + u] : 0u;
                d[u] = (w0 + u < nw && y < n) ? deg[y] : INT_MAX;
            }
            unsigned m[U];
            int32_t tot = 0;
#pragma unroll
            for (int u = 0; u < U; u++) {
                m[u] = __ballot_sync(kFull, ((aw[u] >> lane) & 1u) && d[u] <= k);
                tot += __popc(m[u]);
            }
            if (tot == 0) continue;  // warp-uniform
            int32_t base = 0;
            if (lane == 0) base = atomicAdd(&p.nDc[c0], tot);
            unsigned long long dsum = 0;
#pragma unroll
            for (int u = 0; u < U; u++) {
                if ((m[u] >> lane) & 1u) {
                    const int32_t y = (int32_t)(w0 + u) * 32 + lane;
                    core[y] = k;
                    if (rnd) rnd[y] = r;
                    dsum += (unsigned long long)(rp[y + 1] - rp[y]);
                }
            }
#pragma unroll
            for (int off = 16; off; off >>= 1) dsum += __shfl_xor_sync(kFull, dsum, off);
            if (lane == 0) {
#pragma unroll
                for (int u = 0; u < U; u++)
                    if (m[u]) alive[w0 + u] = aw[u] & ~m[u];
                atomicAdd(&st->nD, tot);
                atomicSub(&st->alive, tot);
                atomicAdd(&st->m_alive, 0ull - dsum);
            }
            base = __shfl_sync(kFull, base, 0);
#pragma unroll
            for (int u = 0; u < U; u++) {
                if ((m[u] >> lane) & 1u) dc[base + __popc(m[u] & lt)] = (int32_t)(w0 + u) * 32 + lane;
                base += __popc(m[u]);
            }
        }
        return;
    }
    for (int64_t w = warp; w < nw; w += nwarps) {
        const uint32_t aw = alive[w];
        if (!aw) {  // warp-uniform
            if (lane == 0 && vis) vis[w] = 0;
            continue;
        }
        const int32_t y = (int32_t)w * 32 + lane;
        bool del = false;
        int32_t k = 0, gy = 0;
        if (y < n && ((aw >> lane) & 1u)) {
            gy = graph_of(p, y);
            k = p.kg[gy];
            del = deg[y] <= k;
        }
        const unsigned mask = __ballot_sync(kFull, del);
        if (!mask) {  // warp-uniform
            if (lane == 0 && vis) vis[w] = 0;
            continue;
        }
        peel_word(w, aw, mask, del, y, k, gy);
    }
}

// One level of the affected-set BFS, push direction (lvl = distance of the
// frontier from D). Frontier = ring slot lvl%3; every alive neighbour not yet
// visited is claimed in vis and appended to the next frontier and to the
// source list of its graph's h-class. A frontier vertex x expands only while
// lvl < h_g(x). Frontier vertices with more than kAffHeavy CSR entries are
// expanded by a whole block.
constexpr int kAffHeavy = 1024;

__device__ __forceinline__ void dev_affected_push(GraphView g, const uint32_t *alive, int lvl,
                                                          int32_t *aq0, int32_t *aq1, int32_t *aq2,
                                                          uint32_t *vis, PeelView p, PeelState *st,
                                                          int32_t *A, int last)
{
    const int cs = lvl % 3, ns = (lvl + 1) % 3, os = (lvl + 2) % 3;
    const int32_t *fr = cs == 0 ? aq0 : (cs == 1 ? aq1 : aq2);
    int32_t *nx = ns == 0 ? aq0 : (ns == 1 ? aq1 : aq2);
    const int32_t nf = st->aq[cs];
    if (blockIdx.x == 0 && threadIdx.x == 0) st->aq[os] = 0;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t *rp = g.row_ptr;
    const int32_t *col = g.col;

    // all neighbours of x belong to x's graph, so its class and h apply
    auto visit = [&](int32_t e, int32_t e1, int32_t cls) {
        bool hit = false;
        int32_t y = -1;
        if (e < e1) {
            y = __ldg(&col[e]);
            if (is_alive(alive, y)) {
                const uint32_t bit = 1u << (y & 31);
                if (!(vis[y >> 5] & bit)) hit = !(atomicOr(&vis[y >> 5], bit) & bit);
            }
        }
        if (!last) warp_append(hit, y, nx, &st->aq[ns]);
        warp_append(hit, y, A + __ldg(&p.cls_off[cls]), &p.nAc[cls]);
    };
    for (int64_t i = warp; i < nf; i += nwarps) {  // warp-uniform
        const int32_t x = fr[i];
        const int32_t e0 = rp[x], e1 = rp[x + 1];
        if (e1 - e0 > kAffHeavy) continue;
        const int32_t gx = graph_of(p, x);
        if (__ldg(&p.hg[gx]) <= lvl) continue;
        const int32_t cls = __ldg(&p.cls[gx]);
        for (int32_t eb = e0; eb < e1; eb += 32) visit(eb + lane, e1, cls);
    }
    for (int64_t i = blockIdx.x; i < nf; i += gridDim.x) {  // block-uniform
        const int32_t x = fr[i];
        const int32_t e0 = rp[x], e1 = rp[x + 1];
        if (e1 - e0 <= kAffHeavy) continue;
        const int32_t gx = graph_of(p, x);
        if (__ldg(&p.hg[gx]) <= lvl) continue;
        const int32_t cls = __ldg(&p.cls[gx]);
        for (int32_t eb = e0; eb < e1; eb += blockDim.x) visit(eb + (int32_t)threadIdx.x, e1, cls);
    }
}

__device__ __forceinline__ void dev_apply_dcount(const int32_t *list, int32_t inner, int32_t total,
                               int32_t *dcount, int32_t *deg)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = list[i];
        if (i >= inner) deg[u] -= dcount ? dcount[u] : 1;
        if (dcount) dcount[u] = 0;
    }
}

// Lazy mode update of the affected list[0..total): every vertex loses the
// deleted vertices it reaches within h hops through survivors (dcount, or 1
// when dcount is null: a single deleted vertex d1[0]) for sure; those closer
// than h (index < inner) may lose more, which widens their slack. What more
// they lose lies within h-1 of the deleted set (Observation 2): at most
// `extra` (the inner count plus the deleted count), and at most the ball
// bound of dev_weight_pass (wsum; for a single deleted vertex, its h-degree
// bound, or its row length when h = 2). Resets dcount and wsum.
__device__ __forceinline__ void dev_apply_lazy(const int32_t *list, int32_t inner, int32_t total, int32_t *dcount,
                                               int32_t *deg, int32_t *slack, int32_t extra, int32_t *wsum,
                                               const int32_t *d1, const int32_t *rp, int32_t h)
{
    if (!dcount && d1) {
        const int32_t d = d1[0];
        const int32_t wd = h == 2 ? min(deg[d], rp[d + 1] - rp[d]) : deg[d];
        extra = min(extra, wd);
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = list[i];
        const int32_t d = deg[u] - (dcount ? dcount[u] : 1);
        deg[u] = d;
        if (i < inner) {
            int32_t ex = extra;
            if (dcount && wsum) ex = min(ex, wsum[u]);
            const long long sl = (long long)slack[u] + ex;
            slack[u] = (int32_t)(sl < d ? sl : d);
        }
        if (dcount) dcount[u] = 0;
        if (wsum) wsum[u] = 0;
    }
}

__device__ __forceinline__ void dev_concat(int32_t *dst, const int32_t *a, int32_t na, const int32_t *b, int32_t nb)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)na + nb;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = i < na ? a[i] : b[i - na];
}

__device__ __forceinline__ void dev_snapshot_inner(PeelView p, const int32_t *cls_h, int lvl, int32_t *inner)
{
    for (int32_t c = threadIdx.x; c < p.ncls; c += blockDim.x)
        if (cls_h[c] == lvl + 1) inner[c] = p.nAc[c];
}

// nA = sum over classes of the per-class counts (for the host).
__device__ __forceinline__ void dev_sum_classes(PeelView p, PeelState *st)
{
    int32_t s = 0;
    for (int32_t c = 0; c < p.ncls; c++) s += p.nAc[c];
    st->nA = s;
}


}  // namespace
}  // namespace khc
