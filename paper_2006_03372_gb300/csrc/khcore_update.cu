// khcore_update.cu — the paper's exact h-degree update after deleting one
// vertex (Sec. IV-A, Observation 2, Theorem 1 and Algorithm 3, with the
// bitmaps of Sec. IV-B, Algorithm 4), on the GPU, one thread block per deleted
// vertex.
//
// For a deleted vertex v of G[alive]:
//   R = N_v^h: the other vertices within h of v, found by a BFS from v; they
//       are labelled in BFS order, so the d = |N_v^{h-1}| members closer than
//       h take the first labels (bit i of a 64-bit word array stands for
//       member i, as in the paper's Reach bitmaps).
//   Reach(u_i) starts as {u_i} for i < d and empty otherwise; then h rounds
//       of Reach_q(u_i) |= Reach_p(u_j) over the edges (u_i, u_j) of the
//       subgraph induced by R (v excluded), the two buffers alternating.
//   A member u at distance s from v loses v and every member u_j with
//       dist(v, u_j) <= h - s whose bit its Reach misses (Observation 2: the
//       lost vertices lie in N_v^{h-s}; Theorem 1: the shortest paths that
//       keep them lie inside G(N_v^h)).
//
// Several deleted vertices are updated at once only when their closed balls
// N_v^h + v are pairwise disjoint: then none of them changes another's ball
// or the subgraph it induces, so the updates commute and the result is that
// of deleting them one after the other. Each wave: every candidate's block
// builds its ball and claims its members (atomicMin of the candidate's
// position on owner[]); a block that owns its whole ball is a winner and
// applies the update; the others retry in the next wave with the graph the
// winners left. The candidate at the lowest position always wins, so every
// wave makes progress.
#include <climits>

#include "khcore_device.cuh"

namespace khc {

namespace {

constexpr int kUB = 512;  // threads per block

// Number of members with dist <= t (dist[0..size) is non-decreasing).
__device__ __forceinline__ int32_t members_within(const uint8_t *dist, int32_t size, int32_t t)
{
    int32_t lo = 0, hi = size;
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if ((int32_t)dist[mid] <= t) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Bits of word k (members 64k .. 64k+63) that stand for the first a members.
__device__ __forceinline__ uint64_t first_bits(int32_t a, int k)
{
    const int32_t lo = 64 * k;
    if (a >= lo + 64) return ~0ull;
    if (a <= lo) return 0ull;
    return (1ull << (a - lo)) - 1ull;
}

// Block b builds the ball of cand[b] in G[alive] (BFS, h levels) into its
// slot: list (BFS order), dist; meta = {size or -1 on overflow, d, listed}.
// Without overflow it claims the ball and the centre on owner[].
__global__ void __launch_bounds__(kUB) k_ball_claim(GraphView g, const uint32_t *alive, UpdBufs u,
                                                    const int32_t *cand, int32_t h)
{
    const int32_t b = blockIdx.x;
    const int32_t v = cand[b];
    uint32_t *vis = u.vis + (size_t)b * u.vis_words;
    int32_t *list = u.list + (size_t)b * u.cap;
    uint8_t *dist = u.dist + (size_t)b * u.cap;
    __shared__ int32_t s_n;
    __shared__ int s_ovf;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwb = blockDim.x >> 5;
    if (tid == 0) {
        s_n = 0;
        s_ovf = 0;
        atomicOr(&vis[v >> 5], 1u << (v & 31));
    }
    __syncthreads();
    int32_t lo = 0, hi = 0, d = -1;
    for (int l = 0; l < h; l++) {
        const int32_t nf = l == 0 ? 1 : hi - lo;
        for (int32_t f = wid; f < nf; f += nwb) {
            const int32_t x = l == 0 ? v : list[lo + f];
            const int32_t e0 = g.row_ptr[x], e1 = g.row_ptr[x + 1];
            for (int32_t eb = e0; eb < e1; eb += 32) {
                const int32_t e = eb + lane;
                bool fresh = false;
                int32_t y = -1;
                if (e < e1) {
                    y = __ldg(&g.col[e]);
                    if (is_alive(alive, y)) {
                        const uint32_t m = 1u << (y & 31);
                        fresh = !(atomicOr(&vis[y >> 5], m) & m);
                    }
                }
                const unsigned bal = __ballot_sync(kFull, fresh);
                if (!bal) continue;
                const int leader = __ffs(bal) - 1;
                int32_t base = 0;
                if (lane == leader) base = atomicAdd(&s_n, __popc(bal));
                base = __shfl_sync(kFull, base, leader);
                if (fresh) {
                    const int32_t pos = base + __popc(bal & lanemask_lt());
                    if (pos < u.cap) {
                        list[pos] = y;
                        dist[pos] = (uint8_t)(l + 1);
                    } else {
                        s_ovf = 1;  // not listed: unmark it, so the reset finds a clean slot
                        atomicAnd(&vis[y >> 5], ~(1u << (y & 31)));
                    }
                }
            }
        }
        __syncthreads();
        if (s_ovf) break;
        lo = hi;
        hi = s_n;
        if (l == h - 2) d = hi;  // members at distance 1 .. h-1
        __syncthreads();
        if (hi == lo) break;  // the ball is complete
    }
    const int32_t listed = min(s_n, u.cap);
    if (d < 0) d = h == 1 ? 0 : listed;
    const bool ovf = s_ovf || d > 64 * u.wc;
    if (tid == 0) {
        u.meta[4 * b + 0] = ovf ? -1 : listed;
        u.meta[4 * b + 1] = d;
        u.meta[4 * b + 2] = listed;
        if (ovf) atomicOr(&u.flag[0], 1);
        else atomicMin(&u.owner[v], b);
    }
    if (!ovf)
        for (int32_t i = tid; i < listed; i += blockDim.x) atomicMin(&u.owner[list[i]], b);
}

// Blocks that own their whole closed ball apply the update (Algorithm 3 with
// the bitmaps of Algorithm 4) and delete their vertex; done[b] tells which.
__global__ void __launch_bounds__(kUB) k_ball_apply(GraphView g, uint32_t *alive, UpdBufs u, const int32_t *cand,
                                                    int32_t h, int32_t *deg, PeelState *st)
{
    const int32_t b = blockIdx.x;
    const int32_t v = cand[b];
    const int32_t size = u.meta[4 * b + 0];
    const int32_t d = u.meta[4 * b + 1];
    const int32_t *list = u.list + (size_t)b * u.cap;
    const uint8_t *dist = u.dist + (size_t)b * u.cap;
    const int wc = u.wc;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwb = blockDim.x >> 5;
    __shared__ int s_lose;
    if (tid == 0) s_lose = size < 0 || u.owner[v] != b;
    __syncthreads();
    for (int32_t i = tid; i < size; i += blockDim.x)
        if (u.owner[list[i]] != b) s_lose = 1;
    __syncthreads();
    if (s_lose) {
        if (tid == 0) u.done[b] = 0;
        return;
    }
    if (tid == 0) u.done[b] = 1;
    uint64_t *R[2];
    R[0] = u.reach + (size_t)b * 2 * u.cap * wc;
    R[1] = R[0] + (size_t)u.cap * wc;
    for (int32_t i = tid; i < size; i += blockDim.x) {
        u.lab[list[i]] = i;
        for (int k = 0; k < wc; k++) {
            const uint64_t w = (i < d && k == (i >> 6)) ? (1ull << (i & 63)) : 0ull;
            R[0][(size_t)i * wc + k] = w;
            R[1][(size_t)i * wc + k] = w;
        }
    }
    __syncthreads();
    // the DP over the subgraph induced by R: one warp per member, lanes over
    // its row; a neighbour is a member iff this block owns it (and it is not v)
    int p = 1, q = 0;
    for (int hop = 1; hop <= h; hop++) {
        q = p;
        p = 1 - p;
        const uint64_t *Rp = R[p];
        uint64_t *Rq = R[q];
        for (int32_t i = wid; i < size; i += nwb) {
            const int32_t x = list[i];
            uint64_t acc[4] = {0, 0, 0, 0};
            for (int32_t e = g.row_ptr[x] + lane; e < g.row_ptr[x + 1]; e += 32) {
                const int32_t w = __ldg(&g.col[e]);
                if (w == v || u.owner[w] != b) continue;
                const int32_t j = u.lab[w];
                for (int k = 0; k < wc; k++) acc[k] |= Rp[(size_t)j * wc + k];
            }
            for (int k = 0; k < wc; k++) {
#pragma unroll
                for (int off = 16; off; off >>= 1) acc[k] |= __shfl_xor_sync(kFull, acc[k], off);
            }
            if (lane == 0)
                for (int k = 0; k < wc; k++) Rq[(size_t)i * wc + k] |= acc[k];
        }
        __syncthreads();
    }
    // the update: u_i at distance s loses v and the members within h - s of v
    // that its Reach misses
    const uint64_t *Rf = R[q];
    for (int32_t i = tid; i < size; i += blockDim.x) {
        const int32_t s = dist[i];
        const int32_t lim = members_within(dist, size, h - s);
        int32_t miss = 0;
        for (int k = 0; k < wc; k++) miss += __popcll(first_bits(lim, k) & ~Rf[(size_t)i * wc + k]);
        deg[list[i]] -= 1 + miss;
    }
    if (tid == 0) {
        atomicAnd(&alive[v >> 5], ~(1u << (v & 31)));
        if (st) {
            atomicSub(&st->alive, 1);
            atomicAdd(&st->m_alive, 0ull - (unsigned long long)(g.row_ptr[v + 1] - g.row_ptr[v]));
        }
    }
}

// Every block releases what it claimed and clears its visited bits.
__global__ void __launch_bounds__(kUB) k_ball_reset(UpdBufs u, const int32_t *cand)
{
    const int32_t b = blockIdx.x;
    const int32_t v = cand[b];
    const int32_t listed = u.meta[4 * b + 2];
    uint32_t *vis = u.vis + (size_t)b * u.vis_words;
    const int32_t *list = u.list + (size_t)b * u.cap;
    for (int32_t i = threadIdx.x; i < listed; i += blockDim.x) {
        const int32_t y = list[i];
        u.owner[y] = INT_MAX;
        atomicAnd(&vis[y >> 5], ~(1u << (y & 31)));
    }
    if (threadIdx.x == 0) {
        u.owner[v] = INT_MAX;
        atomicAnd(&vis[v >> 5], ~(1u << (v & 31)));
    }
}

// The next wave's list: the losers among the first ncur candidates, then the
// candidates that did not fit this wave, in order. One block.
__global__ void __launch_bounds__(1024) k_wave_next(UpdBufs u, const int32_t *cand, int32_t nrem, int32_t ncur,
                                                    int32_t *out)
{
    __shared__ int32_t wsum[32];
    __shared__ int32_t s_base;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) s_base = 0;
    __syncthreads();
    for (int32_t c0 = 0; c0 < nrem; c0 += blockDim.x) {
        const int32_t i = c0 + tid;
        const bool keep = i < nrem && (i >= ncur || u.done[i] == 0);
        const unsigned bal = __ballot_sync(kFull, keep);
        if (lane == 0) wsum[wid] = __popc(bal);
        __syncthreads();
        int32_t before = 0, total = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            if (w < wid) before += wsum[w];
            total += wsum[w];
        }
        if (keep) out[s_base + before + __popc(bal & lanemask_lt())] = cand[i];
        __syncthreads();
        if (tid == 0) s_base += total;
        __syncthreads();
    }
    if (tid == 0) u.flag[1] = s_base;
}

// D = {alive v : deg[v] <= k} of a one-graph context, without deleting them:
// core and round written, v appended to cand (st->nD counts them).
__global__ void __launch_bounds__(kBlock) k_peel_mark(int32_t n, const uint32_t *alive, const int32_t *deg,
                                                      const int32_t *kg, PeelState *st, int32_t *core, int32_t *rnd,
                                                      int32_t *cand)
{
    const int lane = threadIdx.x & 31;
    const int32_t nw = (n + 31) >> 5;
    const int32_t k = kg[0], r = st->round;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = warp; w < nw; w += nwarps) {
        const uint32_t aw = alive[w];
        if (!aw) continue;  // warp-uniform
        const int32_t y = (int32_t)w * 32 + lane;
        const bool del = y < n && ((aw >> lane) & 1u) && deg[y] <= k;
        if (del) {
            core[y] = k;
            if (rnd) rnd[y] = r;
        }
        warp_append(del, y, cand, &st->nD);
    }
}

__global__ void k_alive_from_bytes(uint32_t *alive, const uint8_t *bytes, int32_t n)
{
    const int32_t nw = (n + 31) >> 5;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x) {
        uint32_t m = 0;
        for (int t = 0; t < 32; t++) {
            const int64_t y = w * 32 + t;
            if (y < n && bytes[y]) m |= 1u << t;
        }
        alive[w] = m;
    }
}

__global__ void k_fill_i32(int32_t *p, int32_t val, int64_t count)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = val;
}

}  // namespace

cudaError_t launch_fill_i32(int32_t *p, int32_t val, int64_t count, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    const int64_t blocks = (count + 255) / 256;
    k_fill_i32<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(p, val, count);
    return cudaGetLastError();
}

cudaError_t launch_ball_claim(const GraphView &g, const uint32_t *alive, const UpdBufs &u, const int32_t *cand,
                              int32_t ncur, int32_t h, cudaStream_t s)
{
    if (ncur <= 0) return cudaSuccess;
    k_ball_claim<<<ncur, kUB, 0, s>>>(g, alive, u, cand, h);
    return cudaGetLastError();
}

cudaError_t launch_ball_apply(const GraphView &g, uint32_t *alive, const UpdBufs &u, const int32_t *cand,
                              int32_t ncur, int32_t h, int32_t *deg, PeelState *st, cudaStream_t s)
{
    if (ncur <= 0) return cudaSuccess;
    k_ball_apply<<<ncur, kUB, 0, s>>>(g, alive, u, cand, h, deg, st);
    return cudaGetLastError();
}

cudaError_t launch_ball_reset(const UpdBufs &u, const int32_t *cand, int32_t ncur, cudaStream_t s)
{
    if (ncur <= 0) return cudaSuccess;
    k_ball_reset<<<ncur, kUB, 0, s>>>(u, cand);
    return cudaGetLastError();
}

cudaError_t launch_wave_next(const UpdBufs &u, const int32_t *cand, int32_t nrem, int32_t ncur, int32_t *out,
                             cudaStream_t s)
{
    k_wave_next<<<1, 1024, 0, s>>>(u, cand, nrem, ncur, out);
    return cudaGetLastError();
}

cudaError_t launch_peel_mark(int32_t n, const uint32_t *alive, const int32_t *deg, const int32_t *kg, PeelState *st,
                             int32_t *core, int32_t *rnd, int32_t *cand, int grid, cudaStream_t s)
{
    k_peel_mark<<<grid, kBlock, 0, s>>>(n, alive, deg, kg, st, core, rnd, cand);
    return cudaGetLastError();
}

cudaError_t launch_alive_from_bytes(uint32_t *alive, const uint8_t *bytes, int32_t n, cudaStream_t s)
{
    const int32_t nw = (n + 31) >> 5;
    k_alive_from_bytes<<<(nw + 255) / 256 > 0 ? (nw + 255) / 256 : 1, 256, 0, s>>>(alive, bytes, n);
    return cudaGetLastError();
}

}  // namespace khc
