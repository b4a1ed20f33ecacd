// khcore_internal.cuh — device data layout and kernel launchers shared by the
// translation units of the library. Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace khc {

// Threads per block of the BFS and peel kernels.
constexpr int kBlock = 512;
// Degree classes of the pull expansion: a vertex with deg <= kLightMax is
// expanded by W lanes (one 64-bit word each), deg <= kMediumMax by a warp,
// larger degrees by a whole block.
constexpr int kLightMax = 32;
constexpr int kMediumMax = 1024;

// Static CSR plus the degree-class vertex lists (built once at create time).
struct GraphView {
    int32_t n;
    int64_t m;                 // directed CSR entries
    const int32_t *row_ptr;    // [n+1]
    const int32_t *col;        // [m]
    const int32_t *light;      // vertices with deg <= kLightMax
    const int32_t *medium;     // kLightMax < deg <= kMediumMax
    const int32_t *heavy;      // deg > kMediumMax
    int32_t n_light, n_medium, n_heavy;
};

// Multi-source BFS state for one batch of 64*W sources. Vertex-major: the W
// words of vertex y are V[y*W .. y*W+W-1]; bit b of word j is source 64*j+b
// of the batch.
//   V        visited (sources within distance < current level); all zero
//            between batches
//   F[2]     frontier words of the current / next level; only meaningful
//            where the matching flag byte is 1
//   flag[2]  one byte per vertex: 1 iff the vertex is in that frontier
//   cnt      [64*W] per-source count of newly reached vertices; zero between
//            batches
struct BfsBufs {
    uint64_t *V;
    uint64_t *F[2];
    uint8_t *flag[2];
    int32_t *cnt;
};

// Round state of the peeler, device-resident.
struct PeelState {
    int32_t k;        // current level (never decreases)
    int32_t min_deg;  // scratch for the min-reduction (INT32_MAX between uses)
    int32_t nD;       // vertices deleted this round
    int32_t nA;       // affected vertices this round
    int32_t alive;    // vertices still alive
    int32_t round;    // current round
    int32_t err;      // device-side consistency error code (0 = none)
    int32_t pad;
};

// ---- launchers (khcore_kernels.cu) -----------------------------------------
// All return the cudaError_t of the launch.

cudaError_t launch_iota(int32_t *dst, int32_t n, cudaStream_t s);
cudaError_t launch_alive_init(uint32_t *alive, int32_t n, cudaStream_t s);

// One MS-BFS batch: sources src[0..ns) (ns <= 64*W), alive mask, h levels;
// on return deg[src[i]] = |{u != src[i] alive : dist <= h}| in G[alive].
// grid = number of blocks for the expansion kernels.
cudaError_t run_bfs_batch(int W, const GraphView &g, const uint32_t *alive, const BfsBufs &b,
                          const int32_t *src, int32_t ns, int32_t h, int32_t *deg,
                          int grid, cudaStream_t s, int64_t *launches);

// Peel round pieces.
cudaError_t launch_min_alive_deg(const GraphView &g, const uint32_t *alive, const int32_t *deg,
                                 PeelState *st, int grid, cudaStream_t s);
cudaError_t launch_set_level(PeelState *st, cudaStream_t s);
cudaError_t launch_peel_compact(const GraphView &g, uint32_t *alive, const int32_t *deg,
                                PeelState *st, int32_t *core, int32_t *rnd, uint32_t *fr0,
                                int grid, cudaStream_t s);
cudaError_t launch_affected_level(const GraphView &g, const uint32_t *alive, const uint32_t *fr_cur,
                                  uint32_t *fr_next, uint32_t *vis, int grid, cudaStream_t s);
cudaError_t launch_compact_affected(const GraphView &g, const uint32_t *alive, const uint32_t *vis,
                                    PeelState *st, int32_t *list, int grid, cudaStream_t s);

int max_blocks_per_sm_bfs(int W);

}  // namespace khc
