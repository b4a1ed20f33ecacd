// khcore_block.cu — whole decompositions of small graphs, one thread block per
// graph.
//
// In a batch of many small graphs the grid-wide round loop makes every graph
// wait at every grid barrier of the batch's slowest graph, and every level
// scans the whole union. Here each block takes graphs from a work list
// (largest first) and runs the complete peel of one graph at a time: the
// initial h-degrees, then rounds of level / peel set / affected set /
// recompute, with __syncthreads between phases and no grid-wide barrier, no
// spin wait and no host round trip. Graphs are vertex-disjoint, so the blocks
// share the union-indexed arrays without conflict: each touches only its own
// graph's vertex range (the alive bitset, whose words straddle graphs, is
// cleared with atomics).
//
// Per round the steps are those of the grid path (Algorithm 1 deleting a
// whole level set at once): k <- max(k, min alive h-degree); D = alive with
// h-degree <= k; A = alive within h of D through survivors; the part of A
// closer than h to D is recomputed by BFS, and the rest loses exactly the
// members of D within h (Observation 2), counted by the same BFS seeded at D.
#include "khcore_device.cuh"

namespace khc {

namespace {

constexpr int kBB = 512;  // threads per block
constexpr int kGrp = 8;   // lanes per frontier vertex in the push steps

struct BlockShared {
    int32_t cnt[64];
    int32_t nq[2];
    int32_t nt;
    int32_t nlist[3];
    int32_t red[kBB / 32];
    unsigned long long scanned;
};

__device__ __forceinline__ bool bit_alive(const uint32_t *alive, int32_t y)
{
    return (alive[y >> 5] >> (y & 31)) & 1u;
}

// Block-wide minimum of v (every thread calls; result to all threads).
__device__ __forceinline__ int32_t block_min(int32_t v, BlockShared &sh)
{
#pragma unroll
    for (int off = 16; off; off >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, off));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh.red[threadIdx.x >> 5] = v;
    __syncthreads();
    int32_t r = INT_MAX;
    for (int i = 0; i < kBB / 32; i++) r = min(r, sh.red[i]);
    return r;
}

// Multi-source h-bounded BFS over G[alive] from src[0..ns), ns <= 64, one
// bit per source in 64-bit rows V (visited) and F0/F1 (frontier), all zero
// on entry and on exit. Sources at positions < ndeg are alive: their
// h-degree (vertices reached, itself excluded) goes to deg. The others are
// deleted vertices: each alive y they reach gets dcount[y] += how many reach
// it. qa, qb, tl: list space of at least n_g entries each.
__device__ void block_bfs(const BlockLaunch &a, const int32_t *src, int ns, int ndeg, int h, int32_t *qa,
                          int32_t *qb, int32_t *tl, BlockShared &sh)
{
    const int tid = threadIdx.x;
    if (tid < 64) sh.cnt[tid] = 0;
    if (tid == 0) {
        sh.nq[0] = ns;
        sh.nq[1] = 0;
        sh.nt = ns;
    }
    if (tid < ns) {
        const int32_t s = src[tid];
        const uint64_t bit = 1ull << tid;
        a.V[s] = bit;
        a.F0[s] = bit;
        qa[tid] = s;
        tl[tid] = s;
    }
    __syncthreads();
    uint64_t *Fc = a.F0, *Fn = a.F1;
    int32_t *qc = qa, *qn = qb;
    int cur = 0;
    unsigned long long scanned = 0;
    const int grp = tid / kGrp, lane = tid % kGrp;
    for (int lvl = 0; lvl < h; lvl++) {
        const int nq = sh.nq[cur];
        // push the frontier rows to the alive neighbours
        for (int i = grp; i < nq; i += kBB / kGrp) {
            const int32_t x = qc[i];
            const uint64_t fx = Fc[x];
            const int32_t e0 = a.rp[x], e1 = a.rp[x + 1];
            if (lane == 0) scanned += (unsigned long long)__popcll(fx) * (unsigned long long)(e1 - e0);
            for (int32_t e = e0 + lane; e < e1; e += kGrp) {
                const int32_t y = a.col[e];
                if (!bit_alive(a.alive, y)) continue;
                const uint64_t nb = fx & ~a.V[y];
                if (nb && atomicOr((unsigned long long *)&Fn[y], (unsigned long long)nb) == 0ull)
                    qn[atomicAdd(&sh.nq[cur ^ 1], 1)] = y;
            }
        }
        __syncthreads();
        // visited |= new; record first visits; clear the expanded rows
        const int nn = sh.nq[cur ^ 1];
        for (int i = tid; i < nq; i += kBB) Fc[qc[i]] = 0;
        for (int i = tid; i < nn; i += kBB) {
            const int32_t y = qn[i];
            const uint64_t v = a.V[y];
            a.V[y] = v | Fn[y];
            if (v == 0) tl[atomicAdd(&sh.nt, 1)] = y;
        }
        __syncthreads();
        if (tid == 0) sh.nq[cur] = 0;
        uint64_t *tf = Fc;
        Fc = Fn;
        Fn = tf;
        int32_t *tq = qc;
        qc = qn;
        qn = tq;
        cur ^= 1;
        __syncthreads();
    }
    // clear the last frontier rows; count and clear the visited rows
    {
        const int nq = sh.nq[cur];
        for (int i = tid; i < nq; i += kBB) Fc[qc[i]] = 0;
    }
    const int nt = sh.nt;
    const uint64_t dmask = ndeg >= 64 ? ~0ull : ((1ull << ndeg) - 1ull);
    for (int i = tid; i < nt; i += kBB) {
        const int32_t y = tl[i];
        const uint64_t v = a.V[y];
        a.V[y] = 0;
        uint64_t w = v & dmask;
        while (w) {
            const int b = __ffsll((long long)w) - 1;
            w &= w - 1;
            atomicAdd(&sh.cnt[b], 1);
        }
        const uint64_t r = v & ~dmask;
        if (r && bit_alive(a.alive, y)) a.dcount[y] += __popcll(r);  // y is once in tl
    }
    if (lane == 0 && scanned) atomicAdd(&sh.scanned, scanned);
    __syncthreads();
    if (tid < ndeg && tid < ns) a.deg[src[tid]] = sh.cnt[tid] - 1;
    __syncthreads();
}

// Complete decomposition of graph gi (vertex range [v0, v1)).
__device__ void block_graph(const BlockLaunch &a, int32_t gi, BlockShared &sh)
{
    const int tid = threadIdx.x;
    const int32_t v0 = a.voff[gi], v1 = a.voff[gi + 1], ng = v1 - v0;
    const int32_t h = a.hg[gi];
    if (ng == 0) {  // block-uniform
        if (tid == 0) a.kg[gi] = 0;
        return;
    }
    // list space: the graph's own range of every union-sized list
    int32_t *live[2] = {a.live0 + v0, a.live1 + v0};
    int32_t *qa = a.qa + v0, *qb = a.qb + v0, *tl = a.tl + v0;
    int32_t *al = a.al + v0, *dl = a.dl + v0, *sl = a.sl + v0;
    for (int32_t i = tid; i < ng; i += kBB) live[0][i] = v0 + i;
    __syncthreads();
    // initial h-degrees, 64 sources per batch
    long long batches = 0, affected = 0, recomputed = 0;
    for (int32_t b = 0; b < ng; b += 64) {
        block_bfs(a, live[0] + b, min(64, ng - b), 64, h, qa, qb, tl, sh);
        batches++;
    }
    int32_t k = 0, round = 0, nlive = ng, cl = 0;
    for (;;) {
        // level: k <- max(k, min alive h-degree)
        int32_t m = INT_MAX;
        for (int32_t i = tid; i < nlive; i += kBB) m = min(m, a.deg[live[cl][i]]);
        m = block_min(m, sh);
        if (m > k) k = m;
        // peel set D, survivors to the other live list
        if (tid == 0) {
            sh.nlist[0] = 0;
            sh.nlist[1] = 0;
        }
        __syncthreads();
        for (int32_t i = tid; i < nlive; i += kBB) {
            const int32_t v = live[cl][i];
            if (a.deg[v] <= k) {
                dl[atomicAdd(&sh.nlist[0], 1)] = v;
                a.core[v] = k;
                a.rnd[v] = round;
                atomicAnd(&a.alive[v >> 5], ~(1u << (v & 31)));
            } else {
                live[cl ^ 1][atomicAdd(&sh.nlist[1], 1)] = v;
            }
        }
        __syncthreads();
        const int32_t nd = sh.nlist[0];
        nlive = sh.nlist[1];
        cl ^= 1;
        round++;
        if (nlive == 0) break;
        // affected set: BFS from D through survivors, marks = distance
        if (tid == 0) sh.nlist[2] = 0;
        __syncthreads();
        int32_t fb = 0, fe = nd, ni = 0;
        for (int lvl = 0; lvl < h; lvl++) {
            const int32_t *fr = lvl == 0 ? dl : al;
            for (int32_t i = fb + tid / kGrp; i < fe; i += kBB / kGrp) {
                const int32_t x = fr[i];
                const int32_t e0 = a.rp[x], e1 = a.rp[x + 1];
                for (int32_t e = e0 + tid % kGrp; e < e1; e += kGrp) {
                    const int32_t y = a.col[e];
                    if (bit_alive(a.alive, y) && atomicCAS(&a.mark[y], 0, lvl + 1) == 0)
                        al[atomicAdd(&sh.nlist[2], 1)] = y;
                }
            }
            __syncthreads();
            fb = lvl == 0 ? 0 : fe;
            fe = sh.nlist[2];
            if (lvl == h - 2) ni = fe;
            __syncthreads();
        }
        const int32_t na = sh.nlist[2];
        affected += na;
        recomputed += ni;
        // recompute the inner part (h-degrees) and count D on the outer part
        const bool count_d = na > ni && nd > 1;
        const int32_t total = ni + (count_d ? nd : 0);
        for (int32_t i = tid; i < total; i += kBB) sl[i] = i < ni ? al[i] : dl[i - ni];
        __syncthreads();
        for (int32_t b = 0; b < total; b += 64) {
            const int ns = min(64, total - b);
            block_bfs(a, sl + b, ns, max(0, min(ns, ni - b)), h, qa, qb, tl, sh);
            batches++;
        }
        for (int32_t i = tid; i < na; i += kBB) {
            const int32_t u = al[i];
            if (i >= ni) a.deg[u] -= count_d ? a.dcount[u] : 1;
            a.dcount[u] = 0;
            a.mark[u] = 0;
        }
        __syncthreads();
    }
    if (tid == 0) {
        a.kg[gi] = k;
        atomicMax(&a.bs->rounds, (long long)round);
        atomicAdd((unsigned long long *)&a.bs->batches, (unsigned long long)batches);
        atomicAdd((unsigned long long *)&a.bs->affected, (unsigned long long)affected);
        atomicAdd((unsigned long long *)&a.bs->recomputed, (unsigned long long)recomputed);
    }
}

__global__ void __launch_bounds__(kBB) k_decompose_blocks(BlockLaunch a)
{
    __shared__ BlockShared sh;
    __shared__ int32_t s_next;
    if (threadIdx.x == 0) sh.scanned = 0;
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(a.next, 1);
        __syncthreads();
        const int32_t i = s_next;
        __syncthreads();
        if (i >= a.count) break;
        block_graph(a, a.order[i], sh);
    }
    __syncthreads();
    if (threadIdx.x == 0 && sh.scanned) atomicAdd(a.edges, sh.scanned);
}

}  // namespace

cudaError_t launch_decompose_blocks(const BlockLaunch &L, int grid, cudaStream_t s)
{
    if (L.count <= 0) return cudaSuccess;
    k_decompose_blocks<<<grid, kBB, 0, s>>>(L);
    return cudaGetLastError();
}

int block_decompose_threads() { return kBB; }

int max_blocks_per_sm_block_decompose()
{
    int nb = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_decompose_blocks, kBB, 0) != cudaSuccess || nb < 1)
        nb = 1;
    return nb;
}

}  // namespace khc
