// khcore_bfs.cu — per-phase kernels of the multi-source h-bounded BFS (one
// launch per phase, host-driven) and their launcher. The device code lives in
// khcore_device.cuh.
#include "khcore_device.cuh"

namespace khc {

namespace {

template <int W>
__global__ void k_seed(const int32_t *src, int32_t ns, BfsBufs b, const int32_t *rp)
{
    dev_seed<W>(src, ns, b, rp);
}

template <int W, bool LAST>
__global__ void __launch_bounds__(kBlock, (W >= 8 ? 1 : 2)) k_level(GraphView g, const uint32_t *alive, BfsBufs b, int lvl,
                                                  BfsTuning tune)
{
    dev_level<W, LAST>(g, alive, b, lvl, tune);
}

template <int W, bool LAST>
__global__ void __launch_bounds__(kBlock) k_post(GraphView g, BfsBufs b, int lvl, BfsTuning tune)
{
    dev_post<W, LAST>(g, b, lvl, tune);
}

template <int W>
__global__ void __launch_bounds__(kBlock) k_end(BfsBufs b, const int32_t *src, int32_t ns, int32_t *deg)
{
    dev_end<W>(b, src, ns, deg);
}

template <int W>
__global__ void __launch_bounds__(kBlock) k_weight_pass(BfsBufs b, const int32_t *src, const int32_t *rp,
                                                        const uint32_t *alive, int last_radius)
{
    dev_weight_pass<W>(b, src, rp, alive, last_radius != 0);
}

template <int W>
cudaError_t bfs_batch_t(const GraphView &g, const uint32_t *alive, const BfsBufs &b, const int32_t *src,
                        int32_t ns, int32_t h, int32_t *deg, BfsTuning tune, int grid, int block, cudaStream_t s,
                        int64_t *launches, LevelTimer *timer)
{
    const int tb = ((ns + 31) / 32) * 32;
    k_seed<W><<<1, tb, 0, s>>>(src, ns, b, g.row_ptr);
    int64_t l = 1;
    for (int lvl = 0; lvl < h; lvl++) {
        const bool timed = timer && timer->used < timer->cap;
        if (timed) cudaEventRecord(timer->ev[2 * timer->used], s);
        if (lvl == h - 1)
            k_level<W, true><<<grid, block, 0, s>>>(g, alive, b, lvl, tune);
        else
            k_level<W, false><<<grid, block, 0, s>>>(g, alive, b, lvl, tune);
        if (timed) {
            cudaEventRecord(timer->ev[2 * timer->used + 1], s);
            timer->used++;
        }
        if (lvl == h - 1)
            k_post<W, true><<<grid, block, 0, s>>>(g, b, lvl, tune);
        else
            k_post<W, false><<<grid, block, 0, s>>>(g, b, lvl, tune);
        l += 2;
        if (b.wsum && (lvl == h - 2 || lvl == h - 3)) {
            k_weight_pass<W><<<grid, block, 0, s>>>(b, src, g.row_ptr, alive, lvl == h - 2);
            l++;
        }
    }
    k_end<W><<<grid, block, 0, s>>>(b, src, ns, deg);
    l++;
    if (launches) *launches += l;
    return cudaGetLastError();
}

}  // namespace

cudaError_t run_bfs_batch(int W, const GraphView &g, const uint32_t *alive, const BfsBufs &b, const int32_t *src,
                          int32_t ns, int32_t h, int32_t *deg, BfsTuning tune, int grid, int block, cudaStream_t s,
                          int64_t *launches, LevelTimer *timer)
{
    if (ns <= 0) return cudaSuccess;
    if (ns > 64 * W || block < 64 || block > kBlock || block % 32) return cudaErrorInvalidValue;
    switch (W) {
    case 1: return bfs_batch_t<1>(g, alive, b, src, ns, h, deg, tune, grid, block, s, launches, timer);
    case 2: return bfs_batch_t<2>(g, alive, b, src, ns, h, deg, tune, grid, block, s, launches, timer);
    case 4: return bfs_batch_t<4>(g, alive, b, src, ns, h, deg, tune, grid, block, s, launches, timer);
    case 8: return bfs_batch_t<8>(g, alive, b, src, ns, h, deg, tune, grid, block, s, launches, timer);
    case 16: return bfs_batch_t<16>(g, alive, b, src, ns, h, deg, tune, grid, block, s, launches, timer);
    default: return cudaErrorInvalidValue;
    }
}

int max_blocks_per_sm_bfs(int W, int block)
{
    int nb = 1;
    cudaError_t e = cudaSuccess;
    switch (W) {
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_level<1, false>, block, 0); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_level<2, false>, block, 0); break;
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_level<4, false>, block, 0); break;
    case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_level<8, false>, block, 0); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_level<16, false>, block, 0); break;
    }
    if (e != cudaSuccess || nb < 1) nb = 1;
    return nb;
}

}  // namespace khc
