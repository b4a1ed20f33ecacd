// khcore_peel.cu — sm_103a kernels of the peel rounds (Algorithm 1 / 2 made
// level-synchronous), for one graph or for a batch of disjoint graphs that
// peel side by side, each with its own level k and hop bound h.
//
//  * level:    k_g <- max(k_g, min over alive vertices of graph g of d^h)
//  * peel set: D = {alive v : d^h(v) <= k_g(v)}; core(v) = k_g(v); ballot
//              compaction, alive bits cleared
//  * affected: alive vertices within h_g hops of D through survivors
//              (Observation 1: no other h-degree can change), appended to
//              the source list of their graph's h-class
#include <climits>
#include <cstdint>

#include "khcore_internal.cuh"

namespace khc {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ bool is_alive(const uint32_t *alive, int32_t y)
{
    return (__ldg(&alive[y >> 5]) >> (y & 31)) & 1u;
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int32_t graph_of(const PeelView &p, int32_t v) { return p.gid ? __ldg(&p.gid[v]) : 0; }

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

__global__ void k_iota(int32_t *dst, int32_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (int32_t)i;
}

__global__ void k_alive_init(uint32_t *alive, int32_t n)
{
    const int32_t nw = (n + 31) >> 5;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x) {
        const int32_t rem = n - (int32_t)w * 32;
        alive[w] = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
    }
}

// Per-graph minimum of deg over alive vertices, into p.ming (atomicMin). A
// warp whose 32 vertices belong to one graph reduces first.
__global__ void __launch_bounds__(kBlock) k_min_alive_deg(int32_t n, const uint32_t *__restrict__ alive,
                                                          const int32_t *__restrict__ deg, PeelView p)
{
    const int lane = threadIdx.x & 31;
    const int32_t nw = (n + 31) >> 5;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = warp; w < nw; w += nwarps) {
        const int32_t v = (int32_t)w * 32 + lane;
        const uint32_t aw = __ldg(&alive[w]);
        if (!aw) continue;  // warp-uniform
        const bool a = v < n && ((aw >> lane) & 1u);
        int32_t m = a ? deg[v] : INT_MAX;
        const int32_t gv = a ? graph_of(p, v) : -1;
        const int32_t g0 = __shfl_sync(kFull, gv, __ffs(aw) - 1);
        const bool uniform = __all_sync(kFull, !a || gv == g0);
        if (uniform) {
#pragma unroll
            for (int off = 16; off; off >>= 1) m = min(m, __shfl_xor_sync(kFull, m, off));
            if (lane == 0) atomicMin(&p.ming[g0], m);
        } else if (a) {
            atomicMin(&p.ming[gv], m);
        }
    }
}

// k_g <- max(k_g, min alive deg of g) (Algorithm 1 moves a vertex to
// B[max{k, d}], so the level never falls); reset the per-round counters.
__global__ void k_set_level(PeelView p, PeelState *st)
{
    for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < p.G; g += gridDim.x * blockDim.x) {
        const int32_t m = p.ming[g];
        if (m != INT_MAX && m > p.kg[g]) p.kg[g] = m;
        p.ming[g] = INT_MAX;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->nD = 0;
        st->nA = 0;
        st->aq[0] = st->aq[1] = st->aq[2] = 0;
    }
    for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < p.ncls; c += gridDim.x * blockDim.x) {
        p.nAc[c] = 0;
        p.nDc[c] = 0;
    }
}

// D = {alive v : deg[v] <= k_g(v)}: core[v] = k, rnd[v] = round, clear the
// alive bit, append v to dlist (st->aq[0]) and to its class region of dcls.
// vis is rewritten whole: exactly the bits of D. A warp owns one 32-vertex
// word of each bitset.
__global__ void __launch_bounds__(kBlock) k_peel_compact(int32_t n, const int32_t *__restrict__ rp,
                                                         uint32_t *__restrict__ alive, const int32_t *__restrict__ deg,
                                                         PeelView p, PeelState *st, int32_t *__restrict__ core,
                                                         int32_t *__restrict__ rnd, uint32_t *__restrict__ vis,
                                                         int32_t *__restrict__ dlist, int32_t *__restrict__ dcls)
{
    const int lane = threadIdx.x & 31;
    const int32_t nw = (n + 31) >> 5;
    const int32_t r = st->round;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = warp; w < nw; w += nwarps) {
        const uint32_t aw = alive[w];
        if (!aw) {  // warp-uniform
            if (lane == 0) vis[w] = 0;
            continue;
        }
        const int32_t y = (int32_t)w * 32 + lane;
        bool del = false;
        int32_t k = 0, gy = 0;
        if (y < n && ((aw >> lane) & 1u)) {
            gy = graph_of(p, y);
            k = __ldg(&p.kg[gy]);
            del = deg[y] <= k;
        }
        const unsigned mask = __ballot_sync(kFull, del);
        if (!mask) {  // warp-uniform
            if (lane == 0) vis[w] = 0;
            continue;
        }
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
            vis[w] = mask;  // every word of vis is written: it starts the round's affected BFS
            base = atomicAdd(&st->aq[0], __popc(mask));
            atomicAdd(&st->nD, __popc(mask));
            atomicSub(&st->alive, __popc(mask));
            atomicAdd(&st->m_alive, 0ull - dsum);
        }
        base = __shfl_sync(kFull, base, 0);
        if (del) dlist[base + __popc(mask & lanemask_lt())] = y;
        // class regions of the deleted-source lists
        const int32_t cy = del ? __ldg(&p.cls[gy]) : -1;
        const int32_t c0 = __shfl_sync(kFull, cy, __ffs(mask) - 1);
        if (__all_sync(kFull, !del || cy == c0)) {
            warp_append(del, y, dcls + __ldg(&p.cls_off[c0]), &p.nDc[c0]);
        } else if (del) {
            dcls[__ldg(&p.cls_off[cy]) + atomicAdd(&p.nDc[cy], 1)] = y;
        }
    }
}

// One level of the affected-set BFS, push direction (lvl = distance of the
// frontier from D). Frontier = ring slot lvl%3; every alive neighbour not yet
// visited is claimed in vis and appended to the next frontier and to the
// source list of its graph's h-class. A frontier vertex x expands only while
// lvl < h_g(x). Frontier vertices with more than kAffHeavy CSR entries are
// expanded by a whole block.
constexpr int kAffHeavy = 1024;

__global__ void __launch_bounds__(kBlock) k_affected_push(GraphView g, const uint32_t *__restrict__ alive, int lvl,
                                                          int32_t *aq0, int32_t *aq1, int32_t *aq2,
                                                          uint32_t *__restrict__ vis, PeelView p, PeelState *st,
                                                          int32_t *__restrict__ A, int last)
{
    const int cs = lvl % 3, ns = (lvl + 1) % 3, os = (lvl + 2) % 3;
    const int32_t *__restrict__ fr = cs == 0 ? aq0 : (cs == 1 ? aq1 : aq2);
    int32_t *__restrict__ nx = ns == 0 ? aq0 : (ns == 1 ? aq1 : aq2);
    const int32_t nf = st->aq[cs];
    if (blockIdx.x == 0 && threadIdx.x == 0) st->aq[os] = 0;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t *__restrict__ rp = g.row_ptr;
    const int32_t *__restrict__ col = g.col;

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

__global__ void k_apply_dcount(const int32_t *__restrict__ list, int32_t inner, int32_t total,
                               int32_t *__restrict__ dcount, int32_t *__restrict__ deg)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = list[i];
        if (i >= inner) deg[u] -= dcount ? dcount[u] : 1;
        if (dcount) dcount[u] = 0;
    }
}

__global__ void k_snapshot_inner(PeelView p, const int32_t *__restrict__ cls_h, int lvl, int32_t *__restrict__ inner)
{
    for (int32_t c = threadIdx.x; c < p.ncls; c += blockDim.x)
        if (cls_h[c] == lvl + 1) inner[c] = p.nAc[c];
}

// nA = sum over classes of the per-class counts (for the host).
__global__ void k_sum_classes(PeelView p, PeelState *st)
{
    int32_t s = 0;
    for (int32_t c = 0; c < p.ncls; c++) s += p.nAc[c];
    st->nA = s;
}

}  // namespace

cudaError_t launch_iota(int32_t *dst, int32_t n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int grid = (int)((n + 1023) / 1024 < 4096 ? (n + 1023) / 1024 : 4096);
    k_iota<<<grid, 1024, 0, s>>>(dst, n);
    return cudaGetLastError();
}

cudaError_t launch_alive_init(uint32_t *alive, int32_t n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int32_t nw = (n + 31) >> 5;
    const int grid = (nw + 1023) / 1024 < 4096 ? (nw + 1023) / 1024 : 4096;
    k_alive_init<<<grid, 1024, 0, s>>>(alive, n);
    return cudaGetLastError();
}

cudaError_t launch_min_alive_deg(const GraphView &g, const uint32_t *alive, const int32_t *deg, const PeelView &p,
                                 int grid, cudaStream_t s)
{
    k_min_alive_deg<<<grid, kBlock, 0, s>>>(g.n, alive, deg, p);
    return cudaGetLastError();
}

cudaError_t launch_set_level(const PeelView &p, PeelState *st, cudaStream_t s)
{
    const int blocks = (p.G + 255) / 256 < 1024 ? (p.G + 255) / 256 : 1024;
    k_set_level<<<blocks < 1 ? 1 : blocks, 256, 0, s>>>(p, st);
    return cudaGetLastError();
}

cudaError_t launch_peel_compact(const GraphView &g, uint32_t *alive, const int32_t *deg, const PeelView &p,
                                PeelState *st, int32_t *core, int32_t *rnd, uint32_t *vis, int32_t *dlist,
                                int32_t *dcls, int grid, cudaStream_t s)
{
    k_peel_compact<<<grid, kBlock, 0, s>>>(g.n, g.row_ptr, alive, deg, p, st, core, rnd, vis, dlist, dcls);
    return cudaGetLastError();
}

cudaError_t launch_apply_dcount(const int32_t *list, int32_t inner, int32_t total, int32_t *dcount, int32_t *deg,
                                cudaStream_t s)
{
    if (total <= 0) return cudaSuccess;
    const int blocks = (total + 511) / 512 < 2048 ? (total + 511) / 512 : 2048;
    k_apply_dcount<<<blocks, 512, 0, s>>>(list, inner, total, dcount, deg);
    return cudaGetLastError();
}

cudaError_t launch_affected_level(const GraphView &g, const uint32_t *alive, int lvl, int32_t *const aq[3],
                                  uint32_t *vis, const PeelView &p, PeelState *st, int32_t *A, int last, int grid,
                                  cudaStream_t s)
{
    k_affected_push<<<grid, kBlock, 0, s>>>(g, alive, lvl, aq[0], aq[1], aq[2], vis, p, st, A, last);
    return cudaGetLastError();
}

cudaError_t launch_snapshot_inner(const PeelView &p, const int32_t *cls_h, int lvl, int32_t *inner, cudaStream_t s)
{
    k_snapshot_inner<<<1, 256, 0, s>>>(p, cls_h, lvl, inner);
    return cudaGetLastError();
}

cudaError_t launch_sum_classes(const PeelView &p, PeelState *st, cudaStream_t s)
{
    k_sum_classes<<<1, 1, 0, s>>>(p, st);
    return cudaGetLastError();
}

}  // namespace khc
