// khcore_static.cu — h-degrees of listed vertices with no device allocation:
// the multi-source BFS of khcore_hdegrees_of, its scratch carved from one
// fixed array that the library holds on every device it runs on.
//
// The paper has no counterpart. It is for callers that are not allowed to
// allocate device memory while they run: plugins of a host process that owns
// all device memory through its own pool and hands out only input and output
// buffers, and latency-bound paths where cudaMalloc's implicit device-wide
// synchronisation and unbounded latency are not acceptable.
#include <algorithm>
#include <mutex>

#include "../../include/khcore.h"
#include "khcore_device.cuh"

namespace khc {

khcore_status set_thread_error(khcore_status s, const char *fmt, ...);  // khcore_api.cu

namespace {

// A device holds this array from the first load of the library's device code
// on it (the first call here, under lazy module loading) until the process
// exits.
constexpr size_t kStaticScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kStaticW = 1;  // 64 sources per BFS batch
constexpr int kMaxDevices = 64;

// Start of the scratch: status words written by the checking kernel.
struct StaticHeader {
    int32_t err;           // bit 0: row offsets; bit 1: column id; bit 2: listed id; bit 3: repeated id
    int32_t ncls[3];       // light / medium / heavy counts
    int32_t fill[3];       // fill positions of the class lists
    int32_t pad;
    LevelCtl ctl;
    unsigned long long edges;
    unsigned long long alg_bytes;
};

inline size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// Regions of the scratch for a graph of n vertices and m CSR entries. The
// ones that must start at zero (header, seen, cnt, V, F, flag) come first, so
// one memset clears them.
struct StaticLayout {
    size_t hdr, seen, cnt, V, F0, F1, flag0, flag1, zero_end;
    size_t alive, classes, deg, Q[3], I[3], T, total;

    StaticLayout(int32_t n, int64_t m)
    {
        const size_t nn = (size_t)(n > 0 ? n : 1);
        const size_t nw = (nn + 31) / 32;
        const size_t nflag = nw * sizeof(uint32_t);  // one frontier flag bitmap
        const size_t items = nn + (size_t)m / push_chunk(kStaticW) + 1;
        size_t o = 0;
        auto take = [&](size_t bytes) {
            const size_t at = o;
            o += up256(bytes);
            return at;
        };
        hdr = take(sizeof(StaticHeader));
        seen = take(nw * sizeof(uint32_t));
        cnt = take(64 * kStaticW * sizeof(int32_t));
        V = take(nn * kStaticW * sizeof(uint64_t));
        F0 = take(nn * kStaticW * sizeof(uint64_t));
        F1 = take(nn * kStaticW * sizeof(uint64_t));
        flag0 = take(nflag);
        flag1 = take(nflag);
        zero_end = o;
        alive = take(nw * sizeof(uint32_t));
        classes = take(nn * sizeof(int32_t));
        deg = take(nn * sizeof(int32_t));
        for (int k = 0; k < 3; k++) Q[k] = take(nn * sizeof(int32_t));
        for (int k = 0; k < 3; k++) I[k] = take(items * sizeof(int2));
        T = take(nn * sizeof(int32_t));
        total = o;
    }
};

__device__ __forceinline__ int degree_class(int32_t d) { return d <= kLightMax ? 0 : (d <= kMediumMax ? 1 : 2); }

// Check the CSR and the listed ids without reading out of bounds, and count
// the degree classes. Listed ids are marked in the seen bitset to find
// repeats.
__global__ void k_static_check(int32_t n, int64_t m, const int32_t *rp, const int32_t *col, const int32_t *verts,
                               int32_t count, StaticHeader *hd, uint32_t *seen)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int32_t err = 0;
    int32_t c[3] = {0, 0, 0};
    if (t0 == 0 && (rp[0] != 0 || (int64_t)rp[n] != m)) err |= 1;
    for (int64_t v = t0; v < n; v += stride) {
        const int64_t lo = rp[v], hi = rp[v + 1];
        if (!csr_row_ok(lo, hi, m)) err |= 1;
        const int64_t d = hi - lo;
        c[degree_class(d < 0 ? 0 : (int32_t)min(d, (int64_t)INT32_MAX))]++;
    }
    for (int64_t e = t0; e < m; e += stride) {
        const int32_t x = col[e];
        if (x < 0 || x >= n) err |= 2;
    }
    for (int64_t i = t0; i < count; i += stride) {
        const int32_t v = verts[i];
        if (v < 0 || v >= n) {
            err |= 4;
        } else {
            const uint32_t bit = 1u << (v & 31);
            if (atomicOr(&seen[v >> 5], bit) & bit) err |= 8;
        }
    }
    if (err) atomicOr(&hd->err, err);
    for (int k = 0; k < 3; k++)
        if (c[k]) atomicAdd(&hd->ncls[k], c[k]);
}

// Degree-class lists of the pull direction: light, medium, heavy back to back
// (the order inside a class changes no result).
__global__ void k_static_classes(int32_t n, const int32_t *rp, StaticHeader *hd, int32_t *classes)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int k = degree_class(rp[v + 1] - rp[v]);
        const int32_t base = k == 0 ? 0 : (k == 1 ? hd->ncls[0] : hd->ncls[0] + hd->ncls[1]);
        classes[base + atomicAdd(&hd->fill[k], 1)] = (int32_t)v;
    }
}

__global__ void k_static_gather(const int32_t *verts, int32_t count, const int32_t *deg, int32_t *out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = deg[verts[i]];
}

struct DeviceSlot {
    unsigned char *scratch = nullptr;  // device address of g_static_scratch
    int grid = 0;
};
std::mutex g_slot_mu;
DeviceSlot g_slots[kMaxDevices];

// Once per device, with that device current: the device address of the
// scratch array (its host-side name is only a stand-in) and the BFS grid.
// The address is cached per device ordinal for the life of the process, which
// is why cudaDeviceReset between calls is not supported.
cudaError_t device_slot(int dev, DeviceSlot *out)
{
    std::lock_guard<std::mutex> lock(g_slot_mu);
    DeviceSlot &s = g_slots[dev];
    if (!s.scratch) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        s.grid = sms * max_blocks_per_sm_bfs(kStaticW);
        s.scratch = (unsigned char *)p;
    }
    *out = s;
    return cudaSuccess;
}

}  // namespace

}  // namespace khc

using namespace khc;

#define SCU(call)                                                                    \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess)                                                       \
            return set_thread_error(KHCORE_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

extern "C" khcore_status khcore_hdegrees_static(int32_t n, int64_t m, const int32_t *row_ptr, const int32_t *col,
                                                int32_t h, int32_t count, const int32_t *verts, int32_t *deg_out,
                                                void *stream)
{
    if (n < 0 || m < 0) return set_thread_error(KHCORE_EINVAL, "n and m must be >= 0 (got %d, %lld)", n, (long long)m);
    if (h < 1) return set_thread_error(KHCORE_EINVAL, "h must be >= 1 (got %d)", h);
    if (count < 0 || count > n) return set_thread_error(KHCORE_EINVAL, "count %d outside [0, %d]", count, n);
    if (m > INT32_MAX) return set_thread_error(KHCORE_EINVAL, "m = %lld does not fit int32 offsets", (long long)m);
    const StaticLayout L(n, m);
    if (L.total > kStaticScratchBytes)
        return set_thread_error(KHCORE_EINVAL,
                                "graph too large for the static scratch: n = %d, m = %lld need %zu bytes, the "
                                "fixed array holds %zu",
                                n, (long long)m, L.total, kStaticScratchBytes);
    if (count == 0) return KHCORE_OK;
    if (!row_ptr || !col || !verts || !deg_out) return set_thread_error(KHCORE_EINVAL, "a pointer argument is NULL");
    int dev = -1;
    SCU(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_thread_error(KHCORE_EINVAL, "device ordinal %d unsupported", dev);
    DeviceSlot slot;
    SCU(device_slot(dev, &slot));
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *base = slot.scratch;
    StaticHeader *hd = (StaticHeader *)(base + L.hdr);
    uint32_t *seen = (uint32_t *)(base + L.seen);

    // the array keeps whatever the last call left (a call that failed midway
    // included): clear everything the BFS expects to start at zero
    SCU(cudaMemsetAsync(base, 0, L.zero_end, s));
    k_static_check<<<slot.grid, kBlock, 0, s>>>(n, m, row_ptr, col, verts, count, hd, seen);
    SCU(cudaGetLastError());
    int32_t h_hdr[4] = {0, 0, 0, 0};
    SCU(cudaMemcpyAsync(h_hdr, hd, sizeof h_hdr, cudaMemcpyDeviceToHost, s));
    SCU(cudaStreamSynchronize(s));
    if (h_hdr[0] & 1) return set_thread_error(KHCORE_EINVAL, "row_ptr is not a CSR offset array ending at m");
    if (h_hdr[0] & 2) return set_thread_error(KHCORE_EINVAL, "a column id is outside [0, %d)", n);
    if (h_hdr[0] & 4) return set_thread_error(KHCORE_EINVAL, "a listed vertex is outside [0, %d)", n);
    if (h_hdr[0] & 8) return set_thread_error(KHCORE_EINVAL, "a vertex is listed twice");

    GraphView g;
    g.n = n;
    g.m = m;
    g.row_ptr = row_ptr;
    g.col = col;
    int32_t *classes = (int32_t *)(base + L.classes);
    g.light = classes;
    g.medium = classes + h_hdr[1];
    g.heavy = classes + h_hdr[1] + h_hdr[2];
    g.n_light = h_hdr[1];
    g.n_medium = h_hdr[2];
    g.n_heavy = h_hdr[3];
    k_static_classes<<<slot.grid, kBlock, 0, s>>>(n, row_ptr, hd, classes);
    SCU(cudaGetLastError());
    uint32_t *alive = (uint32_t *)(base + L.alive);
    SCU(launch_alive_init(alive, n, s));

    BfsBufs b;
    b.V = (uint64_t *)(base + L.V);
    b.F[0] = (uint64_t *)(base + L.F0);
    b.F[1] = (uint64_t *)(base + L.F1);
    b.flag[0] = (uint32_t *)(base + L.flag0);
    b.flag[1] = (uint32_t *)(base + L.flag1);
    for (int k = 0; k < 3; k++) {
        b.Q[k] = (int32_t *)(base + L.Q[k]);
        b.I[k] = (int2 *)(base + L.I[k]);
    }
    b.T = (int32_t *)(base + L.T);
    b.ctl = &hd->ctl;
    b.cnt = (int32_t *)(base + L.cnt);
    b.edges = &hd->edges;
    b.Fx = nullptr;
    b.flagx = nullptr;
    b.tflag = nullptr;
    b.rowcnt = nullptr;
    b.row_first = 0;
    b.row_sign = 1;
    b.newcnt = nullptr;
    b.alg_bytes = &hd->alg_bytes;
    b.slev = nullptr;
    b.cum = nullptr;
    b.hcnt = 0;
    b.boff = 0;
    b.wsum = nullptr;
    b.wdeg = nullptr;
    b.in_s = nullptr;
    b.fullmask = nullptr;
    b.sel0 = nullptr;
    b.sel = nullptr;
    b.d0 = nullptr;
    BfsTuning tune;
    tune.alpha = 16;
    tune.n_alive = n;
    tune.m_alive = (unsigned long long)m;
    const int32_t hh = (int32_t)std::min<int64_t>(h, std::max<int64_t>((int64_t)n - 1, 1));
    int32_t *deg = (int32_t *)(base + L.deg);
    constexpr int32_t S = 64 * kStaticW;
    for (int32_t off = 0; off < count; off += S)
        SCU(run_bfs_batch(kStaticW, g, alive, b, verts + off, std::min(S, count - off), hh, deg, tune, slot.grid, kBlock, s,
                          nullptr, nullptr));
    k_static_gather<<<(count + kBlock - 1) / kBlock, kBlock, 0, s>>>(verts, count, deg, deg_out);
    SCU(cudaGetLastError());
    SCU(cudaStreamSynchronize(s));
    return KHCORE_OK;
}
