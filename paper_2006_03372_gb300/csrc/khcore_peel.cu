// khcore_peel.cu — per-phase kernels of the peel rounds (host-driven) and
// their launchers. The device code lives in khcore_device.cuh.
#include "khcore_device.cuh"

namespace khc {

namespace {

__global__ void k_iota(int32_t *dst, int32_t n) { dev_iota(dst, n); }
__global__ void k_alive_init(uint32_t *alive, int32_t n) { dev_alive_init(alive, n); }
__global__ void __launch_bounds__(kBlock) k_min_alive_deg(int32_t n, const uint32_t *alive, const int32_t *deg,
                                                          PeelView p)
{
    dev_min_alive_deg(n, alive, deg, p);
}
__global__ void k_set_level(PeelView p, PeelState *st) { dev_set_level(p, st); }
__global__ void __launch_bounds__(kBlock) k_peel_compact(int32_t n, const int32_t *rp, uint32_t *alive,
                                                         const int32_t *deg, PeelView p, PeelState *st,
                                                         int32_t *core, int32_t *rnd, uint32_t *vis, int32_t *dlist,
                                                         int32_t *dcls)
{
    dev_peel_compact(n, rp, alive, deg, p, st, core, rnd, vis, dlist, dcls);
}
__global__ void __launch_bounds__(kBlock) k_affected_push(GraphView g, const uint32_t *alive, int lvl, int32_t *aq0,
                                                          int32_t *aq1, int32_t *aq2, uint32_t *vis, PeelView p,
                                                          PeelState *st, int32_t *A, int last)
{
    dev_affected_push(g, alive, lvl, aq0, aq1, aq2, vis, p, st, A, last);
}
__global__ void k_apply_dcount(const int32_t *list, int32_t inner, int32_t total, int32_t *dcount, int32_t *deg)
{
    dev_apply_dcount(list, inner, total, dcount, deg);
}
__global__ void k_snapshot_inner(PeelView p, const int32_t *cls_h, int lvl, int32_t *inner)
{
    dev_snapshot_inner(p, cls_h, lvl, inner);
}
__global__ void k_sum_classes(PeelView p, PeelState *st) { dev_sum_classes(p, st); }
__global__ void __launch_bounds__(kBlock) k_refine_select(int32_t n, const uint32_t *alive, const int32_t *deg,
                                                          PeelView p, int32_t *cand)
{
    dev_refine_select(n, alive, deg, p, cand);
}
__global__ void __launch_bounds__(kBlock) k_min_over_list(const int32_t *list, int32_t count, const int32_t *deg,
                                                          PeelView p)
{
    dev_min_over_list(list, count, deg, p);
}
__global__ void k_apply_lazy(const int32_t *list, int32_t inner, int32_t total, int32_t *dcount, int32_t *deg,
                             int32_t *slack, int32_t extra, int32_t *wsum, const int32_t *d1, const int32_t *rp,
                             int32_t h)
{
    dev_apply_lazy(list, inner, total, dcount, deg, slack, extra, wsum, d1, rp, h);
}
__global__ void k_concat(int32_t *dst, const int32_t *a, int32_t na, const int32_t *b, int32_t nb)
{
    dev_concat(dst, a, na, b, nb);
}
__global__ void k_class_count(const int32_t *rp, int32_t n, int32_t l, int32_t m, int32_t *counts)
{
    int32_t c[3] = {0, 0, 0};
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = rp[v + 1] - rp[v];
        c[d <= l ? 0 : (d <= m ? 1 : 2)]++;
    }
    for (int k = 0; k < 3; k++)
        if (c[k]) atomicAdd(&counts[k], c[k]);
}
__global__ void k_class_fill(const int32_t *rp, int32_t n, int32_t l, int32_t m, int32_t *counts, int32_t *classes)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = rp[v + 1] - rp[v];
        const int k = d <= l ? 0 : (d <= m ? 1 : 2);
        const int32_t base = k == 0 ? 0 : (k == 1 ? counts[0] : counts[0] + counts[1]);
        classes[base + atomicAdd(&counts[3 + k], 1)] = (int32_t)v;
    }
}
// Sampling variant: the running select count starts at select0, or at the
// exact h-degree for a vertex without a rate (select0 = 0).
__global__ void k_sample_init(const int32_t *sel0, const int32_t *d0, int32_t *sel, int32_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        sel[i] = sel0[i] > 0 ? sel0[i] : d0[i];
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

cudaError_t launch_concat(int32_t *dst, const int32_t *a, int32_t na, const int32_t *b, int32_t nb, cudaStream_t s)
{
    const int64_t t = (int64_t)na + nb;
    if (t <= 0) return cudaSuccess;
    const int blocks = (int)((t + 511) / 512 < 1024 ? (t + 511) / 512 : 1024);
    k_concat<<<blocks, 512, 0, s>>>(dst, a, na, b, nb);
    return cudaGetLastError();
}

cudaError_t launch_refine_select(const GraphView &g, const uint32_t *alive, const int32_t *deg, const PeelView &p,
                                 int32_t *cand, int grid, cudaStream_t s)
{
    k_refine_select<<<grid, kBlock, 0, s>>>(g.n, alive, deg, p, cand);
    return cudaGetLastError();
}

cudaError_t launch_min_over_list(const int32_t *list, int32_t count, const int32_t *deg, const PeelView &p,
                                 cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    const int blocks = (count + kBlock - 1) / kBlock < 1024 ? (count + kBlock - 1) / kBlock : 1024;
    k_min_over_list<<<blocks, kBlock, 0, s>>>(list, count, deg, p);
    return cudaGetLastError();
}

cudaError_t launch_apply_lazy(const int32_t *list, int32_t inner, int32_t total, int32_t *dcount, int32_t *deg,
                              int32_t *slack, int32_t extra, int32_t *wsum, const int32_t *d1, const int32_t *rp,
                              int32_t h, cudaStream_t s)
{
    if (total <= 0) return cudaSuccess;
    const int blocks = (total + 511) / 512 < 2048 ? (total + 511) / 512 : 2048;
    k_apply_lazy<<<blocks, 512, 0, s>>>(list, inner, total, dcount, deg, slack, extra, wsum, d1, rp, h);
    return cudaGetLastError();
}

cudaError_t launch_sum_classes(const PeelView &p, PeelState *st, cudaStream_t s)
{
    k_sum_classes<<<1, 1, 0, s>>>(p, st);
    return cudaGetLastError();
}

cudaError_t launch_sample_init(const int32_t *sel0, const int32_t *d0, int32_t *sel, int32_t n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_sample_init<<<(n + 255) / 256 < 2048 ? (n + 255) / 256 : 2048, 256, 0, s>>>(sel0, d0, sel, n);
    return cudaGetLastError();
}

cudaError_t launch_degree_classes(const int32_t *rp, int32_t n, int32_t light_max, int32_t medium_max,
                                  int32_t *classes, int32_t *counts, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(counts, 0, 6 * sizeof(int32_t), s);
    if (e != cudaSuccess || n <= 0) return e;
    const int blocks = (n + 255) / 256 < 2048 ? (n + 255) / 256 : 2048;
    k_class_count<<<blocks, 256, 0, s>>>(rp, n, light_max, medium_max, counts);
    k_class_fill<<<blocks, 256, 0, s>>>(rp, n, light_max, medium_max, counts, classes);
    return cudaGetLastError();
}

}  // namespace khc
