/*
 * khcore.h — C ABI of the GB300 (sm_103a) library for distance-generalized
 * (k,h)-core decomposition ("Scaling Up Distance-generalized Core
 * Decomposition", 2020).
 *
 * Model (Sec. II). G = (V, E) is undirected and unweighted. For h >= 1 the
 * h-hop neighbourhood N_v^h(G) is the set of vertices u != v with
 * dist_G(u, v) <= h, and the h-hop degree d_v^h(G) = |N_v^h(G)|. The
 * (k,h)-core is the largest induced subgraph in which every vertex has
 * h-hop degree >= k measured INSIDE that subgraph (Definition 2), and the
 * core index core_h(v) is the largest k whose (k,h)-core contains v. The
 * problem (end of Sec. II) is to compute core_h(v) for all v.
 *
 * Graph format. An int32 CSR over vertices 0..n-1: row_ptr has n+1 entries,
 * row_ptr[0] = 0, non-decreasing, and col has row_ptr[n] entries with
 * 0 <= col[e] < n. The graph is simple and undirected, so the CSR holds both
 * directions of every edge, no self-loops and no duplicate entries. Row order
 * does not matter.
 *
 * Pointers. Every array argument may be a host pointer (pageable or pinned)
 * or a CUDA device pointer; the library tells them apart with
 * cudaPointerGetAttributes. Output arrays are allocated by the caller.
 * The library never keeps a caller pointer past the call that received it.
 *
 * Errors. Every entry point returns a khcore_status and never throws or
 * aborts. After a failure khcore_last_error(ctx) holds a one-line message.
 * A CUDA error leaves the context failed: later calls on it return
 * KHCORE_ECUDA, and the context may only be destroyed.
 *
 * Fault injection (testing). If the environment variable KHCORE_FAIL_ALLOC_AT
 * holds N > 0 when a context is created, the N-th device allocation the
 * creating thread makes from then on fails as if the device were full (no
 * cudaMalloc is called for it): the call that made it returns KHCORE_ENOMEM
 * and releases whatever it had allocated. Unset or 0 turns this off.
 *
 * Threads and streams. A context belongs to one host thread at a time. All
 * of its device work is ordered on the stream given to khcore_create. The
 * calls return after their outputs are written (host outputs are complete;
 * device outputs are complete when the call returns, because each call
 * synchronises its stream before returning).
 */
#ifndef KHCORE_H
#define KHCORE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct khcore_ctx khcore_ctx;

typedef enum {
    KHCORE_OK = 0,
    KHCORE_EINVAL = 1,    /* bad argument or malformed graph */
    KHCORE_ENOMEM = 2,    /* device or host allocation failed */
    KHCORE_ECUDA = 3,     /* a CUDA call failed; the context is now failed */
    KHCORE_ETIMEOUT = 4,  /* a bounded device-side wait ran out */
    KHCORE_EBUSY = 5,     /* resource (slot or memory budget) not available now */
    KHCORE_EINTERNAL = 6  /* a device-side consistency check failed */
} khcore_status;

/* Flags for khcore_create. */
#define KHCORE_FLAG_TRUST_INPUT 0x1u  /* skip CSR validation (caller guarantees the format) */

/* Per-call statistics of khcore_decompose_ex. */
typedef struct {
    int32_t h;                 /* h actually used: min(h, max(n-1, 1)) */
    int32_t rounds;            /* peel rounds (level-synchronous deletions) */
    int32_t k_max;             /* largest core index */
    int32_t words_per_vertex;  /* W of the initial h-degree pass (64*W sources per batch) */
    int64_t deleted_total;     /* sum over rounds of |D| (equals n) */
    int64_t affected_total;    /* sum over rounds of |A| (vertices recomputed) */
    int64_t source_batches;    /* multi-source BFS batches run, initial pass included */
    int64_t kernel_launches;   /* kernels launched by this call */
    double device_ms;          /* device time of the call (CUDA events) */
    int64_t edges_traversed;   /* CSR entries a plain single-source h-bounded BFS
                                  would scan, summed over every source of every
                                  h-degree computation of the call */
    /* The BFS level kernels of the initial all-vertex pass: count and time
     * only while profiling is on (khcore_set_profiling): */
    int64_t level_launches;    /* level kernel launches timed */
    double level_ms;           /* their summed device time (CUDA events) */
    double level_bytes;        /* algorithmic bytes of the initial pass's levels.
                                  Per level, pull: 4*n_b + 4*m_b for the n_b
                                  alive rows and their m_b CSR entries, 8*W per
                                  frontier entry gathered and 16*W per vertex
                                  with a frontier neighbour (own visited row
                                  read, next-frontier row written); push:
                                  (4 + 16*W) per frontier CSR entry plus 8*W per
                                  frontier vertex */
    int64_t recomputed_total;  /* affected vertices whose h-degree was recomputed
                                  by BFS (those closer than h to the deleted set);
                                  the others were updated by counting */
    double init_ms;            /* device time of the initial all-vertex h-degree pass */
    double round_ms;           /* device time of the peel rounds (with the persistent
                                  round loop: the one kernel's duration) */
    double round_bytes;        /* algorithmic bytes of the BFS levels run in the
                                  rounds (same per-level formula) */
    /* Persistent round loop only (zero otherwise): time between the grid
     * barriers that close each phase, summed over rounds, as seen by block 0:
     * [0] level (minimum, bound check), [1] exact recomputes of the lazy mode,
     * [2] peel-set compaction, [3] affected-set BFS, [4] h-degree update. */
    double phase_ms[5];
    int64_t grid_barriers;     /* grid-wide barriers the persistent kernel passed */
    int32_t round_words;       /* W of the peel rounds' BFS batches */
    int32_t round_blocks;      /* resident blocks per SM of the persistent round kernel
                                  (0: the rounds were not run by it) */
} khcore_stats;

/*
 * khcore_create — copy an undirected graph to the device and set up the
 * per-graph state (alive bitset, h-degrees, core indices, BFS bitsets).
 *   n        number of vertices, n >= 0 (n = 0 is valid and gives empty results)
 *   row_ptr  int32[n+1] CSR offsets (host or device)
 *   col      int32[row_ptr[n]] neighbour ids (host or device; may be NULL if
 *            row_ptr[n] == 0)
 *   flags    KHCORE_FLAG_* bits
 *   stream   cudaStream_t to order all work on, or NULL for a stream owned by
 *            the context
 *   out      receives the new context (NULL on failure)
 * Returns KHCORE_EINVAL (with a message in khcore_last_error(NULL)) when the
 * CSR is malformed: offsets not starting at 0 or decreasing, an id outside
 * [0, n), a self-loop, a duplicate entry, or an edge present in one direction
 * only. Returns KHCORE_ENOMEM if the device cannot hold the graph.
 */
khcore_status khcore_create(int32_t n, const int32_t *row_ptr, const int32_t *col,
                            uint32_t flags, void *stream, khcore_ctx **out);

/*
 * khcore_hdegrees — d_v^h(G) for every vertex of the whole graph (Sec. II;
 * the first step of the peeling algorithms, Algorithm 1 and Algorithm 2).
 *   h        hop bound, h >= 1 (EINVAL otherwise); h > n-1 acts as n-1
 *   deg_out  int32[n], host or device; deg_out[v] = d_v^h(G)
 * Computed by a multi-source h-bounded BFS on 64-bit source bitsets.
 */
khcore_status khcore_hdegrees(khcore_ctx *ctx, int32_t h, int32_t *deg_out);

/*
 * khcore_hdegrees_ex — khcore_hdegrees with statistics (stats may be NULL):
 * device_ms (= init_ms) of the whole pass, edges_traversed (CSR entries a
 * plain single-source h-bounded BFS would scan, summed over all sources: the
 * numerator of the pass's traversed-edges rate), level_bytes (algorithmic
 * bytes of its BFS levels), source_batches, kernel_launches, and, while
 * profiling is on, level_launches / level_ms of the level kernels.
 */
khcore_status khcore_hdegrees_ex(khcore_ctx *ctx, int32_t h, int32_t *deg_out, khcore_stats *stats);

/*
 * khcore_hdegrees_of — d_v^h(G) for the listed vertices only (a subset of
 * the sources of khcore_hdegrees; same BFS, fewer batches).
 *   count    number of listed vertices, 0 <= count <= n
 *   verts    int32[count] distinct vertex ids (host or device); EINVAL on a
 *            repeated or out-of-range id
 *   deg_out  int32[count] (host or device); deg_out[i] = d^h of verts[i]
 */
khcore_status khcore_hdegrees_of(khcore_ctx *ctx, int32_t h, int32_t count, const int32_t *verts,
                                 int32_t *deg_out);

/*
 * khcore_hdegrees_static — the h-degrees of khcore_hdegrees_of without any
 * device allocation and without a context. The paper has no counterpart.
 *
 * For callers that may not allocate device memory while they run: a plugin
 * inside a host process that owns all device memory through its own pool and
 * hands it only input and output buffers, or a latency-bound path that cannot
 * take cudaMalloc's device-wide synchronisation. The BFS scratch comes from a
 * fixed 32 MiB array in the library's device image. A device holds that array
 * from the moment the library's device code is loaded on it until the process
 * exits; under CUDA's default lazy module loading that is the first call of
 * this entry point on the device, so make that first call during the caller's
 * set-up, where acquiring device memory is still allowed. This call allocates
 * nothing (no cudaMalloc, cudaFree or allocating library routine); it only
 * copies four status words to a host stack buffer and synchronises `stream`
 * once after its checks and once before returning.
 *
 *   n, m     vertices and CSR entries of the graph (m = row_ptr[n])
 *   row_ptr  int32[n+1], device: CSR offsets, row_ptr[0] = 0, non-decreasing
 *   col      int32[m], device: neighbour ids in [0, n). Self-loops, repeated
 *            entries and one-way edges are not detected here: the caller
 *            passes the same symmetric simple graph khcore_create accepts
 *   h        hop bound, h >= 1; h > n-1 acts as n-1
 *   count    number of listed vertices, 0 <= count <= n
 *   verts    int32[count], device: distinct ids in [0, n)
 *   deg_out  int32[count], device: deg_out[i] = d^h of verts[i] in G
 *   stream   cudaStream_t the work is ordered on (NULL: the legacy default
 *            stream)
 * Limit: the scratch needs about 73 n + 0.75 m bytes (exactly: 256-byte
 * aligned regions of the multi-source BFS at 64 sources per batch); larger
 * graphs are rejected with KHCORE_EINVAL and a message naming the bytes
 * needed, before any device work. Offsets that are not a CSR, ids out of
 * range and repeated listed ids are found on the device and also return
 * KHCORE_EINVAL. Messages: khcore_last_error(NULL), per host thread.
 * Set-up: the first call on a device, with that device current, looks up
 * the array's device address (cudaGetSymbolAddress) and caches it for that
 * device ordinal. Under lazy module loading (the CUDA default) that first
 * lookup is also when the device reserves the array, so make the first call
 * during set-up, where allocation is allowed. Every call reads status words
 * back and synchronises its stream, so no call can be captured into a CUDA
 * graph.
 * cudaDeviceReset between calls is not supported: it discards the device's
 * copy of the array, and the cached address would then be stale.
 * Sharing: every call on a device uses the same array, and each call clears
 * the parts that must start at zero. Calls whose device work overlaps (two
 * host threads, or two streams, on one device) race on the array and give
 * wrong results: order them, e.g. on one stream from one thread.
 */
khcore_status khcore_hdegrees_static(int32_t n, int64_t m, const int32_t *row_ptr, const int32_t *col,
                                     int32_t h, int32_t count, const int32_t *verts, int32_t *deg_out,
                                     void *stream);

/*
 * khcore_decompose — core_h(v) for every vertex (problem statement, Sec. II).
 *   h         hop bound, h >= 1 (EINVAL otherwise); h > n-1 acts as n-1
 *   core_out  int32[n], host or device
 * Peels level-synchronously: at level k every alive vertex with h-degree
 * <= k is deleted with core index k (Algorithm 1 deletes them one at a time
 * in some order; the result is the same, because h-degrees only fall as
 * vertices go). Only alive vertices within h hops of the deleted set can
 * change h-degree (Sec. IV-A, Observation 1); their h-degrees are recomputed
 * on the surviving induced subgraph.
 */
khcore_status khcore_decompose(khcore_ctx *ctx, int32_t h, int32_t *core_out);

/*
 * khcore_decompose_ex — khcore_decompose with the peel round of every vertex
 * and statistics.
 *   round_out  int32[n] or NULL; round_out[v] = the round in which v was
 *              deleted (0-based). Rounds and core indices together form a
 *              certificate that a CPU checker can verify.
 *   stats      khcore_stats* or NULL
 */
khcore_status khcore_decompose_ex(khcore_ctx *ctx, int32_t h, int32_t *core_out,
                                  int32_t *round_out, khcore_stats *stats);

/*
 * khcore_decompose_sampled — the paper's sampling variant (Sec. IV-C,
 * Algorithms 5 and 6): estimated core indices from a vertex sample S drawn by
 * the caller (the paper draws r|V| vertices uniformly; the draw is an input
 * here so that runs are reproducible).
 *   in_s      uint8[n] (host or device): 1 = the vertex is in S
 *   core_out  int32[n] (host or device): the estimated core indices
 *   round_out, stats as for khcore_decompose_ex
 * Every vertex v gets select0(v) = |N_v^h(G) cap S| and d0(v) = d_v^h(G);
 * while peeling, select(v) = |N_v^h(G[alive]) cap S| and the estimated
 * h-degree is floor(select * d0 / select0) (the paper's select / rate with
 * rate = select0 / d0, in exact integers, rounded down as its example 8 /
 * 0.45 -> 17 shows). A vertex with select0 = 0 has no rate and keeps its
 * exact h-degree. The peel is Algorithm 2's on these estimates, level by
 * level: each estimate only falls as vertices go, so the estimated cores do
 * not depend on the order of deletions inside a level. S = V gives the exact
 * core indices. Rounds are host-driven; the affected vertices of every round
 * are recounted by the multi-source BFS, counting only sampled vertices (all
 * vertices for the sources without a rate). One-graph contexts only (EINVAL
 * otherwise).
 */
khcore_status khcore_decompose_sampled(khcore_ctx *ctx, int32_t h, const uint8_t *in_s, int32_t *core_out,
                                      int32_t *round_out, khcore_stats *stats);

/*
 * khcore_batch_create — one context holding G independent graphs (batching
 * many graphs of uneven size into the same kernel launches). The graphs are
 * packed: graph g has n_g = v_off[g+1] - v_off[g] vertices and
 * m_g = e_off[g+1] - e_off[g] CSR entries;
 *   v_off, e_off     int64[G+1], v_off[0] = e_off[0] = 0, non-decreasing
 *   row_ptr_local    int32[v_off[G] + G]: graph g's own row_ptr (n_g + 1
 *                    entries, starting at 0) at offset v_off[g] + g
 *   col_local        int32[e_off[G]]: graph g's neighbour ids, local to the
 *                    graph (0 <= id < n_g), at offset e_off[g]
 * Each graph must be a valid undirected CSR (as for khcore_create; EINVAL
 * names the graph otherwise). Vertex v of graph g is vertex v_off[g] + v of
 * the context: outputs of khcore_hdegrees / khcore_decompose /
 * khcore_batch_decompose are int32[v_off[G]] in that order. The batch must
 * fit int32 ids (v_off[G], e_off[G] <= INT32_MAX).
 */
khcore_status khcore_batch_create(int32_t G, const int64_t *v_off, const int64_t *e_off,
                                  const int32_t *row_ptr_local, const int32_t *col_local,
                                  uint32_t flags, void *stream, khcore_ctx **out);

/*
 * khcore_batch_decompose — core_h(v) of every vertex of every graph of a
 * batch context, graph g with its own hop bound h[g] >= 1 (int32[G], host or
 * device). The graphs peel side by side, each with its own level k (a graph's
 * core indices are those it would get alone). round_out and stats as for
 * khcore_decompose_ex; stats->h is the largest h used.
 */
khcore_status khcore_batch_decompose(khcore_ctx *ctx, const int32_t *h, int32_t *core_out,
                                     int32_t *round_out, khcore_stats *stats);

/* Number of vertices, directed CSR entries and graphs of the context. */
int32_t khcore_num_vertices(const khcore_ctx *ctx);
int64_t khcore_num_entries(const khcore_ctx *ctx);
int32_t khcore_num_graphs(const khcore_ctx *ctx);

/*
 * khcore_set_words — choose W, the number of 64-bit source words per vertex
 * (64*W sources per BFS batch). W must be 1, 2, 4, 8 or 16 (EINVAL
 * otherwise); 0 restores the automatic choice. Results do not depend on W.
 */
khcore_status khcore_set_words(khcore_ctx *ctx, int32_t words);

/*
 * khcore_set_round_words — W of the BFS batches of the peel rounds (the
 * recompute of the affected vertices and the count from the deleted set),
 * separately from the initial all-vertex pass (khcore_set_words). Same
 * values; 0 = automatic (at most 4). Results do not depend on it.
 */
khcore_status khcore_set_round_words(khcore_ctx *ctx, int32_t words);

/*
 * khcore_set_push_alpha — direction choice of the multi-source BFS: a level
 * expands in the push direction (frontier vertices scatter to neighbours)
 * when (sum of frontier degrees) * alpha < CSR entries of the alive graph,
 * and in the pull direction (every alive vertex gathers) otherwise. Sets it
 * for every BFS of the context. Defaults: 16 for the all-vertex pass (its
 * 16-word rows make push atomics dear) and 4 in the peel rounds (1- to 4-word
 * rows; measured against 16: 20 % faster rounds on the 1e6-vertex Chung-Lu
 * graph at h = 3, 7 % on a 97k-vertex batch graph at h = 4); 0 forces pull
 * everywhere. alpha < 0 is EINVAL. Results do not depend on alpha.
 */
khcore_status khcore_set_push_alpha(khcore_ctx *ctx, int32_t alpha);

/*
 * khcore_set_lazy — (default on) keep, for every alive vertex, an upper bound
 * on its h-degree (decremented exactly by the deleted vertices it can still
 * reach) and a lower bound (the upper bound minus the most it can have lost
 * besides: the vertices within h-1 of the deleted set, Observation 2), and
 * recompute exactly only the vertices whose lower bound does not rule out
 * being peeled at the coming level. That level is at most T = max(k, least
 * exact h-degree, least upper bound), so a vertex whose lower bound exceeds T
 * is neither peeled at it nor sets it: the peeled sets, core indices and
 * rounds are identical to the eager mode (0: recompute every affected vertex
 * closer than h to the deleted set in every round).
 */
khcore_status khcore_set_lazy(khcore_ctx *ctx, int32_t on);

/*
 * Tuning knobs. None of them changes a result; each changes only how the
 * kernels cut up the work.
 *
 * khcore_set_degree_classes — degree classes of the pull direction of the
 * multi-source BFS: a vertex with at most light_max CSR entries is gathered by
 * a group of max(8, W) lanes, one with at most medium_max by a warp, a larger
 * one by a whole thread block (defaults 32 and 1024). EINVAL unless
 * 0 <= light_max <= medium_max.
 */
khcore_status khcore_set_degree_classes(khcore_ctx *ctx, int32_t light_max, int32_t medium_max);

/* khcore_set_block_size — threads per block of the per-phase BFS kernels
 * (the all-vertex pass and the host-driven rounds): 128, 256 or 512 (the
 * default); EINVAL otherwise. The persistent round kernel keeps 512. */
khcore_status khcore_set_block_size(khcore_ctx *ctx, int32_t threads);

/* khcore_set_round_blocks — resident 512-thread blocks per SM of the
 * persistent round kernel when its rows are 4 words wide (the default round
 * W): 1 (up to 128 registers per thread) or 2 (64); 0 (default) picks 1 for
 * h <= 2, where the rounds are latency-bound, and 2 for h >= 3. EINVAL
 * otherwise. */
khcore_status khcore_set_round_blocks(khcore_ctx *ctx, int32_t blocks);

/* khcore_set_round_sms — SMs the persistent round kernel's grid covers: 1 up
 * to the device's SM count, or 0 (default) for all of them. Fewer blocks make
 * each grid barrier cheaper (fewer arrivals on its counter) and each scan
 * phase longer. Batch contexts that run graphs concurrently size their
 * graphs' kernels themselves (khcore_set_concurrent_graphs). EINVAL
 * otherwise. */
khcore_status khcore_set_round_sms(khcore_ctx *ctx, int32_t sms);

/* khcore_set_concurrent_graphs — batch contexts: the graphs above the
 * per-block cut (khcore_set_block_graph_max) are decomposed k at a time
 * (1..64, default 1), each in a context of its own on its own CUDA stream and
 * host thread, its persistent round kernel on sm_count / k SMs. (On the
 * 1,024-graph batch the default measured best: 250 s for k = 1, 266 s for
 * k = 8, 410 s for k = 16 — its time sits in the largest graphs at h = 4,
 * whose rounds keep the whole GPU busy.) EINVAL otherwise. */
khcore_status khcore_set_concurrent_graphs(khcore_ctx *ctx, int32_t k);

/* khcore_set_block_graph_max — batch contexts: graphs of at most nmax
 * vertices are decomposed by one thread block each (default 4096; see
 * khcore_set_graph_blocks). EINVAL for nmax < 0. */
khcore_status khcore_set_block_graph_max(khcore_ctx *ctx, int32_t nmax);

/* The knobs khcore_autotune chose (they apply to the all-vertex pass: its
 * W, block size, degree classes and push alpha; the peel rounds keep theirs,
 * and khcore_set_degree_classes / khcore_set_push_alpha set both). */
typedef struct {
    int32_t words;            /* W of the all-vertex pass (khcore_set_words) */
    int32_t block;            /* khcore_set_block_size */
    int32_t light_max;        /* khcore_set_degree_classes */
    int32_t medium_max;
    int32_t push_alpha;       /* push alpha of the all-vertex pass only (the rounds
                                 keep khcore_set_push_alpha's) */
    int32_t block_graph_max;  /* khcore_set_block_graph_max */
    int32_t from_cache;       /* 1: read from the cache file, nothing measured */
    int32_t trials;           /* settings timed */
    double trial_ms;          /* device time of the timed trials */
} khcore_tuning;

/*
 * khcore_autotune — pick the knobs above for this context's graph, GPU and h
 * by measurement, and apply them.
 *   One-graph contexts: the multi-source BFS is timed (CUDA events) on the
 *   first min(n, 4096) vertices as sources, knob by knob (W in {4, 8, 16},
 *   block size in {128, 256, 512}, light_max in {16, 32, 64}, medium_max in
 *   {256, 1024, 4096}, the all-vertex pass's push alpha in {4, 16, 64}),
 *   each set to its fastest
 *   value before the next is tried; every trial's h-degrees must agree
 *   (KHCORE_EINTERNAL otherwise).
 *   Batch contexts: block_graph_max, from up to 8 graphs of 512 to 32,768
 *   vertices each decomposed alone on one thread block and on the whole
 *   grid: the largest size where one block was not slower.
 *   cache_path  NULL, or a file of JSON lines keyed by the GPU name, the
 *               number of graphs, log2 of n, m and the largest degree, and
 *               the effective h. A matching line is applied without any
 *               measurement (from_cache = 1); otherwise the choice is
 *               appended to the file.
 *   out         khcore_tuning* or NULL
 * The round W (khcore_set_round_words) is left to its automatic choice: the
 * rounds' BFS batches are small and latency-bound, and timing them needs
 * whole decompositions.
 */
khcore_status khcore_autotune(khcore_ctx *ctx, int32_t h, const char *cache_path, khcore_tuning *out);

/*
 * khcore_set_update — how the h-degrees are brought up to date after a
 * round's deletions (one-graph contexts, and each larger graph of a batch).
 *   0 (default)  multi-source BFS: the vertices near the deleted set are
 *                bounded (khcore_set_lazy) or recomputed, the outer shell
 *                counted (Observation 1 and 2, Sec. IV-A)
 *   1            the paper's exact update (Sec. IV-A, Algorithm 3 with the
 *                bitmaps of Sec. IV-B, Algorithm 4; driven as in Algorithm 2):
 *                each deleted vertex's ball N_v^h is updated by the Reach DP
 *                on the subgraph it induces, deleted vertices with pairwise
 *                disjoint balls at once, one thread block each (see
 *                khcore_bitmap_update). A round whose deleted set holds more
 *                than 64 vertices, or a ball over the limits of
 *                khcore_bitmap_update, falls back to the BFS recompute.
 *                Rounds are driven from the host; khcore_set_lazy does not
 *                apply.
 * Results (core indices, rounds) are identical. EINVAL for other values.
 */
khcore_status khcore_set_update(khcore_ctx *ctx, int32_t mode);

/*
 * khcore_bitmap_update — the paper's exact h-degree update after deleting one
 * vertex (Sec. IV-A, Observation 2, Theorem 1 and Algorithm 3, with the
 * bitmaps of Sec. IV-B, Algorithm 4), on the context's graph restricted to
 * the alive vertices.
 *   h          hop bound, h >= 1; h > n-1 acts as n-1; at most 255
 *   alive_in   uint8[n] (host or device): 1 = vertex present in G[alive]
 *   v          the vertex deleted; it must be alive
 *   deg_inout  int32[n] (host or device): in, the h-degrees in G[alive]; out,
 *              those of the members of N_v^h updated to G[alive] - v (every
 *              other entry unchanged)
 *   ball_out   int64* or NULL: |N_v^h| in G[alive]
 * Members are labelled in BFS order from v, so the members closer than h take
 * the first bitmap bits (Table 1 labels N_v^{h-1} first). Limits: a ball of
 * at most 65,536 members and |N_v^{h-1}| <= 256 (four 64-bit words per
 * member); over them the call returns KHCORE_EINVAL and changes nothing. The
 * context's own decomposition state is overwritten (a later decomposition
 * starts afresh).
 */
khcore_status khcore_bitmap_update(khcore_ctx *ctx, int32_t h, const uint8_t *alive_in, int32_t v, int32_t *deg_inout,
                                   int64_t *ball_out);

/*
 * khcore_set_round_loop — how the peel rounds are driven.
 *   0 (default)  the whole decomposition runs as one cooperative persistent
 *                kernel; phases are separated by grid barriers and every
 *                decision between them is taken on the device
 *   1            the host launches each phase and reads the round's counts
 *                back before planning the recompute
 * Results are identical. EINVAL for other values.
 */
khcore_status khcore_set_round_loop(khcore_ctx *ctx, int32_t mode);

/*
 * khcore_set_graph_blocks — how a context of several graphs is decomposed.
 * mode 0 (default): the graphs of at most 4,096 vertices are decomposed whole
 * by one thread block each (initial h-degrees and every round), in one launch
 * with no grid-wide barrier and no host round trip, the blocks taking graphs
 * largest first; then every larger graph runs alone on the grid-wide path
 * (its own persistent launch over a copy of its CSR). mode 1: every graph on
 * one block. mode -1: all graphs' rounds in lock-step on the grid-wide path
 * (one launch over the union). Contexts of one graph use the grid-wide path
 * unless mode is 1. Results are identical in every mode; the per-block path
 * recomputes the inner affected vertices eagerly (khcore_set_lazy and
 * khcore_set_round_loop do not apply to it). The larger graphs run several at
 * a time (khcore_set_concurrent_graphs). EINVAL for other modes.
 */
khcore_status khcore_set_graph_blocks(khcore_ctx *ctx, int32_t mode);

/*
 * khcore_set_wait_limit — time limit of one grid-barrier wait of the
 * persistent kernel, in nanoseconds (default 10 s). A wait that runs out stops
 * the decomposition with KHCORE_ETIMEOUT; the context stays usable and the
 * next call starts from a clean state.
 */
khcore_status khcore_set_wait_limit(khcore_ctx *ctx, uint64_t ns);

/*
 * khcore_set_profiling — when on (nonzero), every BFS level kernel launch is
 * bracketed by CUDA events on the context's stream and khcore_stats reports
 * their count, summed time and algorithmic bytes. Results do not change.
 */
khcore_status khcore_set_profiling(khcore_ctx *ctx, int32_t on);

/* ---------------------------------------------------------------------------
 * Serving: a request server with continuous batching.
 *
 * Requests wait in arrival order. Each of `slots` worker threads owns a CUDA
 * stream on the device current at khcore_server_create. A free worker admits
 * either every queued small request (at most 4,096 vertices) that still fits
 * the device-memory budget, at most max_batch, and decomposes them together
 * as one batch context (one thread block per graph, one launch), or, when no
 * small request waits, the oldest large request that fits, decomposed alone
 * on the grid-wide path; each finished unit is published at once. Workers run
 * concurrently, so requests that arrive while others are on the GPU are
 * admitted as slots and budget free up, a large request never holds small
 * ones back, and their work overlaps on the device. A request's core indices
 * equal those of a solo khcore_decompose.
 * ------------------------------------------------------------------------- */
typedef struct khcore_server khcore_server;

/* Device bytes a request with n vertices and m CSR entries is charged
 * against the budget: CSR, per-vertex state and frontier lists, and BFS
 * bitsets for the largest W (16). */
size_t khcore_request_bytes(int32_t n, int64_t m);

/* budget: device bytes all admitted requests may use at once (> 0);
 * slots: worker threads / streams (1..64); max_batch: requests per batch
 * (>= 1). EINVAL on bad arguments, ECUDA without a device. */
khcore_status khcore_server_create(size_t device_bytes_budget, int32_t slots, int32_t max_batch,
                                   khcore_server **out);

/* Queue one decomposition. The graph (int32 CSR, host memory, both edge
 * directions, as for khcore_create but not validated) is copied, so the
 * caller may free it on return. ticket receives the request id. ENOMEM if
 * the request alone exceeds the budget (it could never be admitted). */
khcore_status khcore_server_submit(khcore_server *srv, int32_t n, const int32_t *row_ptr,
                                   const int32_t *col, int32_t h, uint64_t *ticket);

/* done = 1 once the request has finished (EINVAL for an unknown ticket). */
khcore_status khcore_server_poll(khcore_server *srv, uint64_t ticket, int32_t *done);

/* Wait at most timeout_s seconds (ETIMEOUT after that; the request stays
 * queryable) for the request, copy its core indices to core_out (int32[n],
 * host; may be NULL) and its latency (finish minus submit, ms) to
 * latency_ms (may be NULL), and forget the ticket. Returns the request's own
 * status. */
khcore_status khcore_server_wait(khcore_server *srv, uint64_t ticket, int32_t *core_out,
                                 double timeout_s, double *latency_ms);

/* Counters: requests queued, requests completed, batches run, budget bytes
 * in use (each pointer may be NULL). */
khcore_status khcore_server_stats(khcore_server *srv, int64_t *queued, int64_t *completed,
                                  int64_t *batches, size_t *bytes_in_use);

/* Message of the last failed request returned by khcore_server_wait ("" if
 * none); valid until the next khcore_server_wait. */
const char *khcore_server_last_error(khcore_server *srv);

/* Stop the workers after their current batch; queued requests are dropped. */
void khcore_server_destroy(khcore_server *srv);

/* Release every device and host resource of the context. NULL is a no-op. */
void khcore_destroy(khcore_ctx *ctx);

/* Message of the last failure on ctx (or of the last failed khcore_create
 * when ctx is NULL); "" if none. The pointer stays valid until the next call
 * on the same context. */
const char *khcore_last_error(const khcore_ctx *ctx);

/* Static name of a status code. */
const char *khcore_status_string(khcore_status s);

#ifdef __cplusplus
}
#endif

#endif /* KHCORE_H */
