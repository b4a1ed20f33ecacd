// khcore_internal.cuh — device data layout and kernel launchers shared by the
// translation units of the library. Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace khc {

// One CSR row [lo, hi) of an array of m entries is well formed when
// 0 <= lo <= hi <= m. Taken in 64 bits, so that the difference of two int32
// offsets cannot wrap (offsets 2^31 - 1 followed by -2 would give a positive
// int32 row length). Host-side validation and the device-side check of the
// allocation-free entry point use this same predicate.
__host__ __device__ __forceinline__ bool csr_row_ok(int64_t lo, int64_t hi, int64_t m)
{
    return 0 <= lo && lo <= hi && hi <= m;
}

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

// Frontier bookkeeping of one BFS batch, device-resident. Levels use a ring
// of three slots: level l reads slot l%3, appends the next frontier to slot
// (l+1)%3, and slot (l+2)%3 is reset by the level's post kernel.
struct LevelCtl {
    int32_t q[3];                // |Q| per slot: frontier vertex lists
    int32_t qi[3];               // |I| per slot: push work items of the frontier
    unsigned long long fe[3];    // sum of CSR degrees over Q (direction choice)
    int32_t t;                   // |T|: vertices whose V row is nonzero
    int32_t pad;
};

// Push work items: a frontier vertex's CSR row is cut into chunks of
// push_chunk(W) = max(32/W, 8) entries (one warp step of 32/W edges, at
// least 8), so that a hub's edges spread over many warps and a small
// frontier keeps many warps busy with one short dependent chain each (load
// the neighbour, test it, claim its bits) instead of few warps walking long
// chunks. Item = (vertex, first entry); a frontier of total degree D makes at
// most |frontier| + D / 8 items.
__host__ __device__ constexpr int push_chunk(int W) { return (32 / W) > 8 ? 32 / W : 8; }

// Multi-source BFS state for one batch of 64*W sources. Vertex-major: the W
// words of vertex y are V[y*W .. y*W+W-1]; bit b of word j is source 64*j+b
// of the batch.
//   V        visited (distance < current level); rows zero between batches
//            except those listed in T
//   F[2]     frontier words of the current / next level; a row is nonzero
//            only while its vertex is in that level's list Q
//   flag[2]  one bit per vertex: set iff the vertex is in that frontier
//   Q[3], I[3], T   frontier lists and their push work items (ring of three),
//                   touched-row list
//   ctl      list lengths and frontier degree sums
//   cnt      [64*W] per-source count of newly reached vertices; zero between
//            batches
//   edges    plain-BFS-equivalent CSR entries scanned: sum over sources s and
//            vertices x with dist(s, x) < h of deg(x) (for GTEPS reporting)
//   rowcnt   optional [n]: when set, rowcnt[y] += number of batch sources
//            at bit position >= row_first that reach y at distance 1..h
//            (row counts, the transpose of cnt)
struct BfsBufs {
    uint64_t *V;
    uint64_t *F[2];
    uint32_t *flag[2];
    // Fused levels (persistent kernel) only: the third frontier array and
    // flag bitmap of the three-slot ring, and one bit per vertex marking the
    // vertices already in T (all zero between batches).
    uint64_t *Fx;
    uint32_t *flagx;
    uint32_t *tflag;
    int32_t *Q[3];
    int2 *I[3];
    int32_t *T;
    LevelCtl *ctl;
    int32_t *cnt;
    unsigned long long *edges;
    int32_t *rowcnt;
    int32_t row_first;
    int32_t row_sign;               // +1: rowcnt[y] += count; -1: rowcnt[y] -= count
    unsigned long long *newcnt;     // optional: += vertices first reached at the last level
    unsigned long long *alg_bytes;  // algorithmic bytes of every level run (see dev_level)
    // Optional eligibility of the column counts (the ball-restricted label BFS
    // of the paper's update, Algorithm 3): when slev is set, vertex y counts
    // for source position p (in the whole source list) only if
    // p < cum[hcnt - slev[y]]; boff is the batch's first position.
    const int32_t *slev;
    const int32_t *cum;
    int32_t hcnt;
    int32_t boff;
    // Optional (lazy mode, BFS seeded at the deleted set): when wsum is set,
    // every alive vertex the batch reaches within h-1 hops gets, in wsum, the
    // sizes bound of the sources' balls it may lose through them (see
    // dev_weight_pass); wdeg holds the sources' h-degree bounds.
    int32_t *wsum;
    const int32_t *wdeg;
    // Optional sampling (the paper's sampling variant, Algorithms 5 and 6;
    // per-phase kernels only): when in_s is set, a source counts only the
    // sampled vertices it reaches (in_s[y] != 0), except the sources whose
    // bit is set in fullmask (W words, filled by the seed from sel0: those
    // with sel0 == 0 count every vertex). At the end of the batch the count
    // of source s goes to sel[s]; when sel0 is set too, deg[s] receives the
    // estimate floor(count * d0[s] / sel0[s]) (the count itself when
    // sel0[s] == 0), otherwise deg is left alone.
    const uint8_t *in_s;
    uint64_t *fullmask;
    const int32_t *sel0;
    int32_t *sel;
    const int32_t *d0;
};

// Direction choice of one level: push when (sum of frontier degrees) * alpha
// < CSR entries of the alive graph, else pull.
struct BfsTuning {
    int32_t alpha;
    int32_t n_alive;
    unsigned long long m_alive;
};

// Optional CUDA-event timing of every BFS level launch.
struct LevelTimer {
    cudaEvent_t *ev;   // pool of 2*cap events
    int cap;
    int used;          // pairs recorded so far
};

// Round state of the peeler, device-resident.
struct PeelState {
    int32_t nD;       // vertices deleted this round
    int32_t nA;       // affected vertices this round (all classes)
    int32_t alive;    // vertices still alive
    int32_t round;    // current round
    int32_t err;      // device-side consistency error code (0 = none)
    int32_t aq[3];    // affected-BFS frontier list lengths (ring of three)
    int32_t lvl_set;  // persistent kernel: the level step of this round already ran
    unsigned long long m_alive;  // CSR entries of alive vertices
};

// Per-graph peel parameters. One context may hold several disjoint graphs
// (a batch); each peels with its own level k_g and hop bound h_g. Graphs
// with equal h form an h-class; the sources of a class are recomputed in
// BFS batches of that h.
struct PeelView {
    int32_t G;               // graphs
    int32_t ncls;            // h-classes
    const int32_t *gid;      // [n] graph of each vertex, or nullptr when G == 1
    int32_t *kg;             // [G] current level of each graph
    int32_t *ming;           // [G] min scratch (INT32_MAX between rounds)
    const int32_t *hg;       // [G] h of each graph
    const int32_t *cls;      // [G] h-class of each graph
    const int32_t *cls_off;  // [ncls] start of each class's region of the source list
    int32_t *nAc;            // [ncls] affected vertices per class this round
    int32_t *nDc;            // [ncls] deleted vertices per class this round
    // Lazy mode (slack != nullptr): deg[v] is an upper bound on v's h-degree
    // and deg[v] - slack[v] a lower bound (slack 0 = exact).
    int32_t *slack;          // [n]
    int32_t *mind;           // [G] min over alive vertices with slack of deg - slack
    int32_t *minub;          // [G] min over alive vertices with slack of deg
    int32_t *ncand;          // [ncls] vertices picked for an exact recompute this round
};

// ---- launchers (khcore_kernels.cu) -----------------------------------------
// All return the cudaError_t of the launch.

cudaError_t launch_iota(int32_t *dst, int32_t n, cudaStream_t s);
cudaError_t launch_alive_init(uint32_t *alive, int32_t n, cudaStream_t s);

// One MS-BFS batch: sources src[0..ns) (ns <= 64*W), alive mask, h levels;
// on return deg[src[i]] = |{u != src[i] alive : dist <= h}| in G[alive].
// grid = number of blocks for the level kernels.
// timer (nullable): an event pair is recorded around each level launch
// while pairs are left in the pool.
// block: threads per block of the batch's kernels (a multiple of 32, at
// most kBlock).
cudaError_t run_bfs_batch(int W, const GraphView &g, const uint32_t *alive, const BfsBufs &b,
                          const int32_t *src, int32_t ns, int32_t h, int32_t *deg, BfsTuning tune,
                          int grid, int block, cudaStream_t s, int64_t *launches, LevelTimer *timer);

// Peel round pieces (khcore_peel.cu).
cudaError_t launch_min_alive_deg(const GraphView &g, const uint32_t *alive, const int32_t *deg, const PeelView &p,
                                 int grid, cudaStream_t s);
cudaError_t launch_set_level(const PeelView &p, PeelState *st, cudaStream_t s);
// Also subtracts the CSR degree of every deleted vertex from st->m_alive,
// sets the deleted vertices' bits in vis, appends them to dlist (st->aq[0])
// and to their class region of dcls (p.nDc).
cudaError_t launch_peel_compact(const GraphView &g, uint32_t *alive, const int32_t *deg, const PeelView &p,
                                PeelState *st, int32_t *core, int32_t *rnd, uint32_t *vis, int32_t *dlist,
                                int32_t *dcls, int grid, cudaStream_t s);
// Affected vertices list[0..total): those at index >= inner lie exactly h hops
// from the deleted set, so (Observation 2) they lose exactly the deleted
// vertices within h: deg[u] -= dcount[u] (or 1 when dcount is null). Resets
// dcount[u] for every listed vertex.
cudaError_t launch_apply_dcount(const int32_t *list, int32_t inner, int32_t total, int32_t *dcount, int32_t *deg,
                                cudaStream_t s);
// Affected-set BFS, push direction. aq[3] are frontier lists (ring of three;
// slot 0 holds D after launch_peel_compact); vis is the visited bitset (D's
// bits set by the compaction); every newly reached alive vertex is appended
// to the next frontier and to its class region of A (p.nAc).
cudaError_t launch_affected_level(const GraphView &g, const uint32_t *alive, int lvl, int32_t *const aq[3],
                                  uint32_t *vis, const PeelView &p, PeelState *st, int32_t *A, int last, int grid,
                                  cudaStream_t s);
// Lazy mode (see dev_refine_select, dev_min_over_list, dev_apply_lazy).
cudaError_t launch_refine_select(const GraphView &g, const uint32_t *alive, const int32_t *deg, const PeelView &p,
                                 int32_t *cand, int grid, cudaStream_t s);
cudaError_t launch_min_over_list(const int32_t *list, int32_t count, const int32_t *deg, const PeelView &p,
                                 cudaStream_t s);
cudaError_t launch_apply_lazy(const int32_t *list, int32_t inner, int32_t total, int32_t *dcount, int32_t *deg,
                              int32_t *slack, int32_t extra, int32_t *wsum, const int32_t *d1, const int32_t *rp,
                              int32_t h, cudaStream_t s);
// Sampling variant: sel[i] = sel0[i] > 0 ? sel0[i] : d0[i].
cudaError_t launch_sample_init(const int32_t *sel0, const int32_t *d0, int32_t *sel, int32_t n, cudaStream_t s);
// dst = a[0..na) followed by b[0..nb).
cudaError_t launch_concat(int32_t *dst, const int32_t *a, int32_t na, const int32_t *b, int32_t nb, cudaStream_t s);
// st->nA = sum of p.nAc.
cudaError_t launch_sum_classes(const PeelView &p, PeelState *st, cudaStream_t s);
// Before affected-BFS level lvl: inner[c] = p.nAc[c] for every class whose
// h is lvl + 1 (the vertices found so far are those closer than h).
cudaError_t launch_snapshot_inner(const PeelView &p, const int32_t *cls_h, int lvl, int32_t *inner, cudaStream_t s);

int max_blocks_per_sm_bfs(int W, int block = kBlock);

// Degree classes of the pull direction: classes = the vertices with
// deg <= light_max, then those with deg <= medium_max, then the rest;
// counts[0..2] receives the class sizes (device pointers; counts zeroed here).
cudaError_t launch_degree_classes(const int32_t *rp, int32_t n, int32_t light_max, int32_t medium_max,
                                  int32_t *classes, int32_t *counts, cudaStream_t s);

// ---- the paper's exact update after one deletion (khcore_update.cu) ---------
// Slots of the per-deleted-vertex update (Algorithm 3 with Algorithm 4's
// bitmaps): one slot per thread block of a wave, each holding one ball.
struct UpdBufs {
    int32_t nblk;        // slots (deleted vertices per wave at most)
    int32_t cap;         // ball members per slot
    int32_t wc;          // 64-bit bitmap words per member: |N_v^{h-1}| <= 64 * wc (wc <= 4)
    int64_t vis_words;   // 32-bit words of one slot's visited bitmap ((n + 31) / 32)
    uint32_t *vis;       // [nblk * vis_words], zero between waves
    int32_t *list;       // [nblk * cap] ball members in BFS order
    uint8_t *dist;       // [nblk * cap] their distance from the slot's vertex
    uint64_t *reach;     // [nblk * 2 * cap * wc] the two Reach buffers
    int32_t *meta;       // [nblk * 4] size (-1: over the limits), d, entries listed
    int32_t *owner;      // [n] claiming slot, INT_MAX between waves
    int32_t *lab;        // [n] member label (valid where owner is the reader's slot)
    int32_t *done;       // [nblk] the slot's vertex was updated and deleted
    int32_t *flag;       // [2] any slot over the limits; candidates left after a wave
    int32_t *cand[2];    // [n] candidate lists (current, next)
};
cudaError_t launch_ball_claim(const GraphView &g, const uint32_t *alive, const UpdBufs &u, const int32_t *cand,
                              int32_t ncur, int32_t h, cudaStream_t s);
cudaError_t launch_ball_apply(const GraphView &g, uint32_t *alive, const UpdBufs &u, const int32_t *cand,
                              int32_t ncur, int32_t h, int32_t *deg, PeelState *st, cudaStream_t s);
cudaError_t launch_ball_reset(const UpdBufs &u, const int32_t *cand, int32_t ncur, cudaStream_t s);
cudaError_t launch_wave_next(const UpdBufs &u, const int32_t *cand, int32_t nrem, int32_t ncur, int32_t *out,
                             cudaStream_t s);
cudaError_t launch_peel_mark(int32_t n, const uint32_t *alive, const int32_t *deg, const int32_t *kg, PeelState *st,
                             int32_t *core, int32_t *rnd, int32_t *cand, int grid, cudaStream_t s);
cudaError_t launch_alive_from_bytes(uint32_t *alive, const uint8_t *bytes, int32_t n, cudaStream_t s);
cudaError_t launch_fill_i32(int32_t *p, int32_t val, int64_t count, cudaStream_t s);

// ---- persistent decomposition (khcore_persist.cu) ---------------------------

// Grid barrier state (zero before the launch); err = 1 after a timed-out wait.
struct GridSync {
    unsigned count;
    unsigned gen;
    int err;
    int pad;
    unsigned long long passed;  // barriers completed
};

// Statistics the persistent kernel accumulates (zero before the launch).
struct PersistStats {
    long long rounds;
    long long source_batches;
    long long recomputed_total;
    long long deleted_total;
    long long affected_total;
    long long level_steps;  // BFS level phases run
    double level_bytes;     // their algorithmic bytes (4 n_b + 4 m_b + 16 W n_b each)
    unsigned long long phase_ns[5];  // per phase, block 0's time between closing barriers
};

// Everything the persistent kernel works on (device pointers).
struct PersistLaunch {
    GraphView g;
    uint32_t *alive;
    int32_t *deg, *core, *rnd;
    PeelView p;
    PeelState *st;
    BfsBufs b;
    uint32_t *vis;
    int32_t *A;
    int32_t *aq[3];
    int32_t *dcls;
    int32_t *cls_src;
    const int32_t *cls_h, *cls_size, *cls_off;  // [ncls]
    int32_t *inner;
    int32_t *dcount;
    int32_t *comb;  // [n] round source list
    int32_t *cand;  // [n] lazy mode: vertices to recompute exactly (class regions)
    int32_t *wsum;  // [n] lazy mode: ball bounds of the deleted set (dev_weight_pass), zero between rounds
    int32_t ncls, hmax, alpha;
    GridSync *gs;
    PersistStats *ps;
    unsigned long long timeout_ns;  // limit of one barrier wait
};

// Whole decompositions of small graphs, one thread block per graph
// (khcore_block.cu). Union-indexed arrays; each block touches only the vertex
// range of the graph it works on. V, F0, F1 (one 64-bit row per vertex),
// mark and dcount are zero on entry and on exit; the list arrays (n entries
// each) are scratch.
// Batches: graphs of at most this many vertices go to the per-block path
// (above it one block per graph is slower than the grid-wide path alone).
constexpr int32_t kBlockGraphsMaxN = 1 << 12;
struct BlockStats {
    long long rounds;      // largest per-graph round count
    long long batches;     // BFS batches of 64 sources
    long long affected;    // sum of |A| over rounds and graphs
    long long recomputed;  // sum of the inner parts recomputed by BFS
};
struct BlockLaunch {
    const int32_t *rp, *col;
    const int32_t *voff;   // [G+1] vertex offsets
    const int32_t *hg;     // [G] effective h
    const int32_t *order;  // graphs to decompose, in the order they are taken
    int32_t count;         // entries of order
    int32_t *next;         // work counter, zero before the launch
    uint32_t *alive;       // all bits of the listed graphs set on entry
    int32_t *deg, *core, *rnd, *kg;
    uint64_t *V, *F0, *F1;
    int32_t *live0, *live1, *qa, *qb, *tl, *al, *dl, *sl;
    int32_t *mark, *dcount;
    unsigned long long *edges;
    BlockStats *bs;
};
cudaError_t launch_decompose_blocks(const BlockLaunch &L, int grid, cudaStream_t s);
int max_blocks_per_sm_block_decompose();
int block_decompose_threads();

// Cooperative launch of the whole decomposition; grid must not exceed
// max_blocks_per_sm_persist(W) * SMs.
// minb: 2 selects the two-blocks-per-SM variant (W = 4 only), else one.
cudaError_t launch_decompose_persist(int W, const PersistLaunch &L, int grid, cudaStream_t s, int minb);
int max_blocks_per_sm_persist(int W, int minb);

}  // namespace khc
