// khcore_peel.cu — sm_103a kernels of the peel rounds.
//
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
__global__ void __launch_bounds__(kBlock) k_peel_compact(int32_t n, const int32_t *__restrict__ rp,
                                                         uint32_t *__restrict__ alive,
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
        unsigned long long dsum = 0;
        if (del) {
            core[y] = k;
            if (rnd) rnd[y] = r;
            dsum = (unsigned long long)(rp[y + 1] - rp[y]);
        }
        if (mask) {
#pragma unroll
            for (int off = 16; off; off >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, off);
        }
        if (lane == 0 && mask) {
            alive[w] = aw & ~mask;
            fr0[w] = mask;
            atomicAdd(&st->nD, __popc(mask));
            atomicSub(&st->alive, __popc(mask));
            if (dsum) atomicAdd(&st->m_alive, 0ull - dsum);
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
    k_peel_compact<<<grid, kBlock, 0, s>>>(g.n, g.row_ptr, alive, deg, st, core, rnd, fr0);
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

}  // namespace khc
