// khcore_kernels.cu — sm_103a kernels of the (k,h)-core hot path.
//
//  * Multi-source h-bounded BFS (the h-hop degree d_v^h of Sec. II for a
//    batch of 64*W sources at once). Each vertex holds W 64-bit words per
//    state array; bit b of word j stands for source 64*j+b of the batch, the
//    same packing of 64 set members per word that the paper uses for its
//    Reach bitmaps (Sec. IV-B), here applied to BFS sources. A level is a
//    pull step: new(y) = OR over alive neighbours x in the frontier of F(x),
//    minus V(y). The number of newly reached vertices per source is a
//    column count over the new words, kept in byte-sliced (SWAR) counters
//    per lane and reduced once per 255 words.
//  * Level min-reduction, ballot compaction of the peel set D (Algorithm 1/2:
//    delete the vertices of minimum h-degree, core index = level), the
//    affected-set BFS (alive vertices within h hops of D, Observation 1) and
//    its compaction into the next source list.
#include <climits>
#include <cstdint>

#include "khcore_internal.cuh"

namespace khc {

namespace {

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
            lo += __shfl_xor_sync(0xffffffffu, lo, off);
            hi += __shfl_xor_sync(0xffffffffu, hi, off);
        }
        if (lane < W) {
#pragma unroll
            for (int k = 0; k < 4; k++) {
                uint32_t c0 = (uint32_t)(lo >> (16 * k)) & 0xffffu;  // byte 2k   -> bit 16k+t
                uint32_t c1 = (uint32_t)(hi >> (16 * k)) & 0xffffu;  // byte 2k+1 -> bit 16k+8+t
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

// ---------------------------------------------------------------------------
// MS-BFS kernels
// ---------------------------------------------------------------------------

// Level 0: V(s) and F0(s) get the source's own bit; flag0(s) = 1.
// flag0 must be all zero before the launch. One thread per source.
template <int W>
__global__ void k_seed(const int32_t *__restrict__ src, int32_t ns, uint64_t *__restrict__ V,
                       uint64_t *__restrict__ F0, uint8_t *__restrict__ flag0)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    const int32_t s = src[i];
    const int word = i >> 6;
    const uint64_t bit = 1ull << (i & 63);
    V[(size_t)s * W + word] = bit;  // V(s) is zero between batches
#pragma unroll
    for (int j = 0; j < W; j++) F0[(size_t)s * W + j] = (j == word) ? bit : 0ull;
    flag0[s] = 1;
}

// One BFS level in the pull direction over every vertex, in three degree
// classes. LAST: the level that reaches distance h; it only counts, and
// clears V for the next batch.
template <int W, bool LAST>
__global__ void __launch_bounds__(kBlock) k_pull(GraphView g, const uint32_t *__restrict__ alive,
                                                 uint64_t *__restrict__ V,
                                                 const uint64_t *__restrict__ Fc,
                                                 const uint8_t *__restrict__ flc,
                                                 uint64_t *__restrict__ Fn, uint8_t *__restrict__ fln,
                                                 int32_t *__restrict__ cnt)
{
    static_assert(W == 1 || W == 2 || W == 4 || W == 8 || W == 16, "W");
    __shared__ int32_t cnt_s[64 * W];
    __shared__ uint64_t red[kBlock / 32][W];

    for (int i = threadIdx.x; i < 64 * W; i += blockDim.x) cnt_s[i] = 0;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int j = lane % W;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t *__restrict__ rp = g.row_ptr;
    const int32_t *__restrict__ col = g.col;
    Swar sw;
    sw.reset();

    // ---- light: W lanes per vertex, 32/W vertices per warp ----
    {
        constexpr int VPW = 32 / W;
        const int grp = lane / W;
        const unsigned gmask = (W == 32) ? 0xffffffffu : ((1u << W) - 1u);
        for (int64_t base = warp * VPW; base < g.n_light; base += nwarps * VPW) {
            const int64_t idx = base + grp;
            uint64_t nw = 0, v = 0;
            int32_t y = -1;
            bool act = false;
            if (idx < g.n_light) {
                y = g.light[idx];
                if (is_alive(alive, y)) {
                    act = true;
                    uint64_t acc = 0;
                    const int32_t e1 = rp[y + 1];
                    for (int32_t e = rp[y]; e < e1; e++) {
                        const int32_t x = __ldg(&col[e]);
                        if (flc[x]) acc |= Fc[(size_t)x * W + j];
                    }
                    v = V[(size_t)y * W + j];
                    nw = acc & ~v;
                }
            }
            if (!LAST) {
                const unsigned any = __ballot_sync(0xffffffffu, nw != 0);
                const bool gany = ((any >> (grp * W)) & gmask) != 0;
                if (idx < g.n_light) {
                    if (act && gany) {
                        Fn[(size_t)y * W + j] = nw;
                        if (nw) V[(size_t)y * W + j] = v | nw;
                    }
                    if (j == 0) fln[y] = (act && gany) ? 1 : 0;
                }
            } else if (act && v) {
                V[(size_t)y * W + j] = 0;
            }
            swar_step<W>(sw, nw, cnt_s);
        }
    }

    // ---- medium: one warp per vertex, 32/W neighbour slots ----
    {
        constexpr int SLOTS = 32 / W;
        const int slot = lane / W;
        for (int64_t i = warp; i < g.n_medium; i += nwarps) {
            const int32_t y = g.medium[i];
            const bool act = is_alive(alive, y);
            uint64_t nw = 0, v = 0;
            if (act) {
                uint64_t acc = 0;
                const int32_t e1 = rp[y + 1];
                for (int32_t e = rp[y] + slot; e < e1; e += SLOTS) {
                    const int32_t x = __ldg(&col[e]);
                    if (flc[x]) acc |= Fc[(size_t)x * W + j];
                }
#pragma unroll
                for (int off = W; off < 32; off <<= 1) acc |= __shfl_xor_sync(0xffffffffu, acc, off);
                if (lane < W) {
                    v = V[(size_t)y * W + j];
                    nw = acc & ~v;
                }
            }
            if (!LAST) {
                const unsigned any = __ballot_sync(0xffffffffu, nw != 0);
                if (lane < W) {
                    if (act && any) {
                        Fn[(size_t)y * W + j] = nw;
                        if (nw) V[(size_t)y * W + j] = v | nw;
                    }
                    if (lane == 0) fln[y] = (act && any) ? 1 : 0;
                }
            } else if (lane < W && act && v) {
                V[(size_t)y * W + j] = 0;
            }
            swar_step<W>(sw, nw, cnt_s);
        }
    }

    // ---- heavy: one block per vertex, kBlock/W neighbour slots ----
    {
        const int slot = threadIdx.x / W;
        const int slots = blockDim.x / W;
        const int wid = threadIdx.x >> 5;
        const int nwarp_blk = blockDim.x >> 5;
        for (int64_t i = blockIdx.x; i < g.n_heavy; i += gridDim.x) {
            const int32_t y = g.heavy[i];
            const bool act = is_alive(alive, y);
            uint64_t nw = 0, v = 0;
            if (act) {
                uint64_t acc = 0;
                const int32_t e1 = rp[y + 1];
                for (int32_t e = rp[y] + slot; e < e1; e += slots) {
                    const int32_t x = __ldg(&col[e]);
                    if (flc[x]) acc |= Fc[(size_t)x * W + j];
                }
#pragma unroll
                for (int off = W; off < 32; off <<= 1) acc |= __shfl_xor_sync(0xffffffffu, acc, off);
                if (lane < W) red[wid][lane] = acc;
            }
            __syncthreads();
            if (act && wid == 0) {
                uint64_t acc = 0;
                if (lane < W) {
                    for (int w = 0; w < nwarp_blk; w++) acc |= red[w][lane];
                    v = V[(size_t)y * W + j];
                    nw = acc & ~v;
                }
            }
            if (wid == 0) {
                if (!LAST) {
                    const unsigned any = __ballot_sync(0xffffffffu, nw != 0);
                    if (lane < W) {
                        if (act && any) {
                            Fn[(size_t)y * W + j] = nw;
                            if (nw) V[(size_t)y * W + j] = v | nw;
                        }
                        if (lane == 0) fln[y] = (act && any) ? 1 : 0;
                    }
                } else if (lane < W && act && v) {
                    V[(size_t)y * W + j] = 0;
                }
            }
            swar_step<W>(sw, nw, cnt_s);
            __syncthreads();
        }
    }

    swar_flush<W>(sw, cnt_s);
    __syncthreads();
    for (int i = threadIdx.x; i < 64 * W; i += blockDim.x) {
        const int32_t c = cnt_s[i];
        if (c) atomicAdd(&cnt[i], c);
    }
}

// deg[src[i]] = cnt[i]; cnt[i] = 0.
__global__ void k_finish(const int32_t *__restrict__ src, int32_t ns, int32_t *__restrict__ cnt,
                         int32_t *__restrict__ deg)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    deg[src[i]] = cnt[i];
    cnt[i] = 0;
}

template <int W>
cudaError_t bfs_batch_t(const GraphView &g, const uint32_t *alive, const BfsBufs &b,
                        const int32_t *src, int32_t ns, int32_t h, int32_t *deg, int grid,
                        cudaStream_t s, int64_t *launches)
{
    cudaError_t e = cudaMemsetAsync(b.flag[0], 0, (size_t)g.n, s);
    if (e != cudaSuccess) return e;
    const int tb = ns < 1024 ? ((ns + 31) / 32) * 32 : 1024;
    k_seed<W><<<(ns + tb - 1) / tb, tb, 0, s>>>(src, ns, b.V, b.F[0], b.flag[0]);
    int64_t l = 1;
    for (int lvl = 0; lvl < h; lvl++) {
        const int c = lvl & 1, nx = c ^ 1;
        if (lvl == h - 1)
            k_pull<W, true><<<grid, kBlock, 0, s>>>(g, alive, b.V, b.F[c], b.flag[c], b.F[nx],
                                                    b.flag[nx], b.cnt);
        else
            k_pull<W, false><<<grid, kBlock, 0, s>>>(g, alive, b.V, b.F[c], b.flag[c], b.F[nx],
                                                     b.flag[nx], b.cnt);
        l++;
    }
    k_finish<<<(ns + tb - 1) / tb, tb, 0, s>>>(src, ns, b.cnt, deg);
    l++;
    if (launches) *launches += l;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Peel kernels
// ---------------------------------------------------------------------------

__global__ void k_iota(int32_t *dst, int32_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (int32_t)i;
}

__global__ void k_alive_init(uint32_t *alive, int32_t n)
{
    const int32_t nw = (n + 31) >> 5;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw;
         w += (int64_t)gridDim.x * blockDim.x) {
        const int32_t rem = n - (int32_t)w * 32;
        alive[w] = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
    }
}

// min over alive vertices of deg, into st->min_deg (atomicMin).
__global__ void __launch_bounds__(kBlock) k_min_alive_deg(int32_t n, const uint32_t *__restrict__ alive,
                                                          const int32_t *__restrict__ deg,
                                                          PeelState *st)
{
    __shared__ int32_t s_min[kBlock / 32];
    int32_t m = INT_MAX;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        if (is_alive(alive, (int32_t)v)) m = min(m, deg[v]);
#pragma unroll
    for (int off = 16; off; off >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) s_min[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? s_min[threadIdx.x] : INT_MAX;
#pragma unroll
        for (int off = 16; off; off >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, off));
        if (threadIdx.x == 0 && m != INT_MAX) atomicMin(&st->min_deg, m);
    }
}

// k <- max(k, min alive deg) (Algorithm 1 moves a vertex to B[max(k, d)]);
// reset the per-round counters.
__global__ void k_set_level(PeelState *st)
{
    if (st->min_deg != INT_MAX && st->min_deg > st->k) st->k = st->min_deg;
    st->min_deg = INT_MAX;
    st->nD = 0;
    st->nA = 0;
}

// D = {alive v : deg[v] <= k}: core[v] = k, rnd[v] = round, clear alive bit,
// set v's bit in the level-0 frontier of the affected BFS. A warp owns one
// 32-vertex word of each bitset.
__global__ void __launch_bounds__(kBlock) k_peel_compact(int32_t n, uint32_t *__restrict__ alive,
                                                         const int32_t *__restrict__ deg,
                                                         PeelState *st, int32_t *__restrict__ core,
                                                         int32_t *__restrict__ rnd,
                                                         uint32_t *__restrict__ fr0)
{
    const int lane = threadIdx.x & 31;
    const int32_t nw = (n + 31) >> 5;
    const int32_t k = st->k;
    const int32_t r = st->round;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = warp; w < nw; w += nwarps) {
        const int32_t y = (int32_t)w * 32 + lane;
        const uint32_t aw = alive[w];
        const bool del = y < n && ((aw >> lane) & 1u) && deg[y] <= k;
        const unsigned mask = __ballot_sync(0xffffffffu, del);
        if (del) {
            core[y] = k;
            if (rnd) rnd[y] = r;
        }
        if (lane == 0 && mask) {
            alive[w] = aw & ~mask;
            fr0[w] = mask;
            atomicAdd(&st->nD, __popc(mask));
            atomicSub(&st->alive, __popc(mask));
        }
    }
}

// One level of the affected-set BFS, pull direction: an alive vertex not yet
// visited joins the next frontier if any neighbour is in the current one.
// fr_next must be zero before the launch.
__global__ void __launch_bounds__(kBlock) k_affected_level(GraphView g, const uint32_t *__restrict__ alive,
                                                           const uint32_t *__restrict__ fc,
                                                           uint32_t *__restrict__ fn,
                                                           uint32_t *__restrict__ vis)
{
    const int lane = threadIdx.x & 31;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    const int64_t warp = tid >> 5;
    const int64_t nwarps = nthr >> 5;
    const int32_t *__restrict__ rp = g.row_ptr;
    const int32_t *__restrict__ col = g.col;
    // light vertices: one thread each
    for (int64_t i = tid; i < g.n_light; i += nthr) {
        const int32_t y = g.light[i];
        if (!is_alive(alive, y) || ((vis[y >> 5] >> (y & 31)) & 1u)) continue;
        bool hit = false;
        for (int32_t e = rp[y]; e < rp[y + 1] && !hit; e++) {
            const int32_t x = __ldg(&col[e]);
            hit = (fc[x >> 5] >> (x & 31)) & 1u;
        }
        if (hit) {
            atomicOr(&fn[y >> 5], 1u << (y & 31));
            atomicOr(&vis[y >> 5], 1u << (y & 31));
        }
    }
    // medium and heavy vertices: one warp each, early exit on the first hit
    const int64_t nmh = (int64_t)g.n_medium + g.n_heavy;
    for (int64_t i = warp; i < nmh; i += nwarps) {
        const int32_t y = i < g.n_medium ? g.medium[i] : g.heavy[i - g.n_medium];
        if (!is_alive(alive, y) || ((vis[y >> 5] >> (y & 31)) & 1u)) continue;  // warp-uniform
        bool hit = false;
        const int32_t e1 = rp[y + 1];
        for (int32_t e0 = rp[y]; e0 < e1; e0 += 32) {
            const int32_t e = e0 + lane;
            bool h1 = false;
            if (e < e1) {
                const int32_t x = __ldg(&col[e]);
                h1 = (fc[x >> 5] >> (x & 31)) & 1u;
            }
            if (__any_sync(0xffffffffu, h1)) {
                hit = true;
                break;
            }
        }
        if (hit && lane == 0) {
            atomicOr(&fn[y >> 5], 1u << (y & 31));
            atomicOr(&vis[y >> 5], 1u << (y & 31));
        }
    }
}

// list <- alive vertices with a vis bit (warp-aggregated append).
__global__ void __launch_bounds__(kBlock) k_compact_affected(int32_t n, const uint32_t *__restrict__ alive,
                                                             const uint32_t *__restrict__ vis,
                                                             PeelState *st, int32_t *__restrict__ list)
{
    const int lane = threadIdx.x & 31;
    const int32_t nw = (n + 31) >> 5;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = warp; w < nw; w += nwarps) {
        const uint32_t bits = alive[w] & vis[w];
        if (!bits) continue;  // warp-uniform
        int32_t base = 0;
        if (lane == 0) base = atomicAdd(&st->nA, __popc(bits));
        base = __shfl_sync(0xffffffffu, base, 0);
        if ((bits >> lane) & 1u) list[base + __popc(bits & lanemask_lt())] = (int32_t)w * 32 + lane;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

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

cudaError_t run_bfs_batch(int W, const GraphView &g, const uint32_t *alive, const BfsBufs &b,
                          const int32_t *src, int32_t ns, int32_t h, int32_t *deg, int grid,
                          cudaStream_t s, int64_t *launches)
{
    if (ns <= 0) return cudaSuccess;
    switch (W) {
    case 1: return bfs_batch_t<1>(g, alive, b, src, ns, h, deg, grid, s, launches);
    case 2: return bfs_batch_t<2>(g, alive, b, src, ns, h, deg, grid, s, launches);
    case 4: return bfs_batch_t<4>(g, alive, b, src, ns, h, deg, grid, s, launches);
    case 8: return bfs_batch_t<8>(g, alive, b, src, ns, h, deg, grid, s, launches);
    case 16: return bfs_batch_t<16>(g, alive, b, src, ns, h, deg, grid, s, launches);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_min_alive_deg(const GraphView &g, const uint32_t *alive, const int32_t *deg,
                                 PeelState *st, int grid, cudaStream_t s)
{
    k_min_alive_deg<<<grid, kBlock, 0, s>>>(g.n, alive, deg, st);
    return cudaGetLastError();
}

cudaError_t launch_set_level(PeelState *st, cudaStream_t s)
{
    k_set_level<<<1, 1, 0, s>>>(st);
    return cudaGetLastError();
}

cudaError_t launch_peel_compact(const GraphView &g, uint32_t *alive, const int32_t *deg,
                                PeelState *st, int32_t *core, int32_t *rnd, uint32_t *fr0,
                                int grid, cudaStream_t s)
{
    k_peel_compact<<<grid, kBlock, 0, s>>>(g.n, alive, deg, st, core, rnd, fr0);
    return cudaGetLastError();
}

cudaError_t launch_affected_level(const GraphView &g, const uint32_t *alive, const uint32_t *fr_cur,
                                  uint32_t *fr_next, uint32_t *vis, int grid, cudaStream_t s)
{
    k_affected_level<<<grid, kBlock, 0, s>>>(g, alive, fr_cur, fr_next, vis);
    return cudaGetLastError();
}

cudaError_t launch_compact_affected(const GraphView &g, const uint32_t *alive, const uint32_t *vis,
                                    PeelState *st, int32_t *list, int grid, cudaStream_t s)
{
    k_compact_affected<<<grid, kBlock, 0, s>>>(g.n, alive, vis, st, list);
    return cudaGetLastError();
}

int max_blocks_per_sm_bfs(int W)
{
    int nb = 1;
    cudaError_t e = cudaSuccess;
    switch (W) {
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pull<1, false>, kBlock, 0); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pull<2, false>, kBlock, 0); break;
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pull<4, false>, kBlock, 0); break;
    case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pull<8, false>, kBlock, 0); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pull<16, false>, kBlock, 0); break;
    }
    if (e != cudaSuccess || nb < 1) nb = 1;
    return nb;
}

}  // namespace khc
