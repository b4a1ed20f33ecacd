/*
 * oracle.c — plain, slow CPU oracle for distance-generalized (k,h)-core
 * decomposition ("Scaling Up Distance-generalized Core Decomposition", 2020).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline / reference legs load this file. The product library
 * (paper_2006_03372_gb300) never calls, links or imports it, and this file
 * shares no code, header, table or helper with the CUDA path.
 *
 * Every routine here is written for being checked by eye against the paper,
 * not for speed:
 *   orc_hdegrees      the h-hop degree d_v^h(G[alive]) by one BFS per vertex
 *                     (Sec. II, definition of N_v^h and d_v^h).
 *   orc_peel          the basic peeling algorithm (Sec. III, Algorithm 1):
 *                     bucket array B, remove a vertex of the current bucket,
 *                     recompute by BFS the h-degree of every vertex of its
 *                     h-neighbourhood in G(V \ {v}), move it to B[max(k, d)].
 *   orc_bruteforce    the definition itself (Sec. II, Definition 2 and the
 *                     core index that follows it): core_h(v) is the largest
 *                     min_{w in S} d_w^h(G(S)) over all vertex sets S that
 *                     contain v. Exponential; tiny graphs only.
 *   orc_kcore_bz      classic linear-time k-core by bin sort (Batagelj and
 *                     Zaversnik, cited in Sec. II), the h = 1 special case.
 *   orc_bitmap_update the paper's exact h-degree update after one deletion
 *                     (Sec. IV-A, Algorithm 3, with the bitmaps of Sec. IV-B,
 *                     Algorithm 4): a reachability DP on the subgraph induced
 *                     by N_v^h instead of a BFS per member.
 *   orc_peel_bitmap   the paper's decomposition driving that update
 *                     (Sec. IV-A, Algorithm 2).
 *   orc_peel_sampled  the paper's sampling variant (Sec. IV-C, Algorithms 5
 *                     and 6) on a caller-drawn sample; approximate.
 *   orc_certificate   checks a claimed core index c and peel round r against
 *                     two inequalities that together imply c is exact (the
 *                     argument is written above the function).
 *   orc_certificate_all  the same check on every vertex, each BFS stopped as
 *                     soon as its inequality is decided (full-size graphs).
 *
 * Readings of the paper taken here:
 *   - k starts at 0, so isolated vertices get core index 0 (Algorithm 1 starts
 *     its bucket loop at 1 and would never empty B[0]).
 *   - After deleting v, distances are measured in the surviving induced
 *     subgraph only (Definition 2 measures d^h inside the subgraph).
 *
 * Pins: tests/test_oracle_pins.py checks every routine against brute force,
 * closed forms, SciPy's all-pairs shortest paths, networkx.core_number at
 * h = 1, the paper's worked example (Example 1, Example 2, and Table 1's
 * bitmaps for orc_bitmap_update) and invariants; orc_bitmap_update against a
 * fresh BFS after every single deletion, orc_peel_bitmap against orc_peel and
 * brute force; orc_peel_sampled against the paper's estimator example and
 * against Algorithm 1 when every vertex is sampled.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* One bounded BFS from v inside the vertices with alive[u] != 0.            */
/* dist[] must be all -1 on entry and is all -1 again on return.             */
/* If ball != NULL the visited vertices other than v are appended to it.     */
/* Returns |{u != v : dist(v,u) <= h}|.                                      */
/* ------------------------------------------------------------------------ */
static int64_t bfs_count_scan(int32_t v, int32_t h, const int32_t *row_ptr,
                              const int32_t *col, const uint8_t *alive,
                              int32_t *dist, int32_t *queue, int32_t *ball,
                              int64_t *ball_len, int64_t *scanned)
{
    int64_t head = 0, tail = 0;
    queue[tail++] = v;
    dist[v] = 0;
    while (head < tail) {
        int32_t x = queue[head++];
        if (dist[x] == h) continue;           /* do not expand past radius h */
        if (scanned) *scanned += row_ptr[x + 1] - row_ptr[x];
        for (int32_t e = row_ptr[x]; e < row_ptr[x + 1]; e++) {
            int32_t y = col[e];
            if (alive && !alive[y]) continue; /* paths stay inside G[alive] */
            if (dist[y] >= 0) continue;
            dist[y] = dist[x] + 1;
            queue[tail++] = y;
        }
    }
    for (int64_t i = 0; i < tail; i++) {
        int32_t x = queue[i];
        if (ball && x != v) ball[(*ball_len)++] = x;
        dist[x] = -1;
    }
    return tail - 1;
}

static int64_t bfs_count(int32_t v, int32_t h, const int32_t *row_ptr,
                         const int32_t *col, const uint8_t *alive,
                         int32_t *dist, int32_t *queue, int32_t *ball,
                         int64_t *ball_len)
{
    return bfs_count_scan(v, h, row_ptr, col, alive, dist, queue, ball, ball_len, NULL);
}

/* d_v^h(G[alive]) for every vertex; -1 for vertices that are not alive.
 * alive == NULL means every vertex is alive. Returns 0, or -1 on ENOMEM. */
int orc_hdegrees(int32_t n, const int32_t *row_ptr, const int32_t *col,
                 const uint8_t *alive, int32_t h, int32_t *deg_out)
{
    int ok = 0;
#pragma omp parallel
    {
        int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
        int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
        if (!dist || !queue) {
#pragma omp atomic write
            ok = -1;
        } else {
            for (int32_t i = 0; i < n; i++) dist[i] = -1;
#pragma omp for schedule(dynamic, 64)
            for (int32_t v = 0; v < n; v++) {
                if (alive && !alive[v]) { deg_out[v] = -1; continue; }
                deg_out[v] = (int32_t)bfs_count(v, h, row_ptr, col, alive, dist, queue, NULL, NULL);
            }
        }
        free(dist);
        free(queue);
    }
    return ok;
}

/* h-hop degree of a list of vertices (used for spot checks on large graphs).
 * scanned_out (nullable, one per listed vertex) receives the number of CSR
 * entries the BFS scanned, i.e. the sum of deg(x) over x with dist < h. */
int orc_hdegree_list(int32_t n, const int32_t *row_ptr, const int32_t *col,
                     const uint8_t *alive, int32_t h, int64_t count,
                     const int32_t *verts, int32_t *deg_out, int64_t *scanned_out)
{
    int ok = 0;
#pragma omp parallel
    {
        int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
        int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
        if (!dist || !queue) {
#pragma omp atomic write
            ok = -1;
        } else {
            for (int32_t i = 0; i < n; i++) dist[i] = -1;
#pragma omp for schedule(dynamic, 1)
            for (int64_t i = 0; i < count; i++) {
                int32_t v = verts[i];
                int64_t sc = 0;
                deg_out[i] = (alive && !alive[v]) ? -1
                    : (int32_t)bfs_count_scan(v, h, row_ptr, col, alive, dist, queue, NULL, NULL, &sc);
                if (scanned_out) scanned_out[i] = sc;
            }
        }
        free(dist);
        free(queue);
    }
    return ok;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (Sec. III): the basic peeling algorithm.                      */
/* Buckets B[0..n-1] are doubly linked lists of alive vertices keyed by the  */
/* bucket index; core_out[v] receives k at v's removal. order_out (nullable) */
/* receives the vertices in removal order. Returns 0, or -1 on ENOMEM.       */
/* ------------------------------------------------------------------------ */
/* orc_peel_bounded: the same algorithm, optionally starting from given
 * h-degrees (deg_init, nullable: computed here otherwise) and stopping after
 * max_removed removals (< 0: run to the end). Returns the number of vertices
 * removed, or -1 on ENOMEM. Used to time the oracle on a bounded sample. */
int64_t orc_peel_bounded(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t h,
                         const int32_t *deg_init, int64_t max_removed, int32_t *core_out, int32_t *order_out);

int orc_peel(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t h,
             int32_t *core_out, int32_t *order_out)
{
    int64_t r = orc_peel_bounded(n, row_ptr, col, h, NULL, -1, core_out, order_out);
    if (r < 0) return -1;
    return r == n ? 0 : -2;
}

int64_t orc_peel_bounded(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t h,
                         const int32_t *deg_init, int64_t max_removed, int32_t *core_out, int32_t *order_out)
{
    if (n == 0) return 0;
    size_t N = (size_t)n;
    int32_t *deg = malloc(sizeof(int32_t) * N);
    int32_t *head = malloc(sizeof(int32_t) * N);
    int32_t *next = malloc(sizeof(int32_t) * N);
    int32_t *prev = malloc(sizeof(int32_t) * N);
    int32_t *bucket = malloc(sizeof(int32_t) * N);
    uint8_t *alive = malloc(N);
    int32_t *dist = malloc(sizeof(int32_t) * N);
    int32_t *queue = malloc(sizeof(int32_t) * N);
    int32_t *ball = malloc(sizeof(int32_t) * N);
    if (!deg || !head || !next || !prev || !bucket || !alive || !dist || !queue || !ball) {
        free(deg); free(head); free(next); free(prev); free(bucket);
        free(alive); free(dist); free(queue); free(ball);
        return -1;
    }
    for (size_t i = 0; i < N; i++) { head[i] = -1; alive[i] = 1; dist[i] = -1; }

    /* lines 2-4: h-degree of every vertex, then its bucket */
    for (int32_t v = 0; v < n; v++)
        deg[v] = deg_init ? deg_init[v] : (int32_t)bfs_count(v, h, row_ptr, col, alive, dist, queue, NULL, NULL);
    for (int32_t v = n - 1; v >= 0; v--) {
        int32_t b = deg[v];
        bucket[v] = b;
        prev[v] = -1;
        next[v] = head[b];
        if (head[b] >= 0) prev[head[b]] = v;
        head[b] = v;
    }

    int64_t removed = 0;
    /* lines 5-12, with k starting at 0 (isolated vertices have d^h = 0) */
    for (int32_t k = 0; k < n; k++) {
        while (head[k] >= 0) {
            if (max_removed >= 0 && removed >= max_removed) goto done;
            /* lines 7-8: pick and remove a vertex of B[k]; its core index is k */
            int32_t v = head[k];
            head[k] = next[v];
            if (head[k] >= 0) prev[head[k]] = -1;
            core_out[v] = k;
            if (order_out) order_out[removed] = v;
            removed++;

            /* N_v^h in the current graph, before v goes */
            int64_t ball_len = 0;
            bfs_count(v, h, row_ptr, col, alive, dist, queue, ball, &ball_len);
            alive[v] = 0; /* line 12 */

            /* lines 9-11: recompute d_u^h(G(V \ {v})), move u to B[max(k, d)] */
            for (int64_t i = 0; i < ball_len; i++) {
                int32_t u = ball[i];
                int32_t d = (int32_t)bfs_count(u, h, row_ptr, col, alive, dist, queue, NULL, NULL);
                deg[u] = d;
                int32_t nb = d > k ? d : k;
                if (nb == bucket[u]) continue;
                /* unlink from the old bucket */
                if (prev[u] >= 0) next[prev[u]] = next[u]; else head[bucket[u]] = next[u];
                if (next[u] >= 0) prev[next[u]] = prev[u];
                /* push on the new one */
                bucket[u] = nb;
                prev[u] = -1;
                next[u] = head[nb];
                if (head[nb] >= 0) prev[head[nb]] = u;
                head[nb] = u;
            }
        }
    }
done:
    free(deg); free(head); free(next); free(prev); free(bucket);
    free(alive); free(dist); free(queue); free(ball);
    return removed;
}

/* ------------------------------------------------------------------------ */
/* The paper's h-degree update after deleting one vertex v (Sec. IV-A,       */
/* Observation 2 and Theorem 1, Algorithm 3; with the bitmaps of Sec. IV-B,  */
/* Algorithm 4). Works in G[alive] with v still alive; v itself is not       */
/* removed here.                                                             */
/*                                                                           */
/*   R = N_v^h(G): the other vertices within h of v, labelled u_0, u_1, ...  */
/*       by distance from v, then by vertex id (so N_v^{h-1} gets the first  */
/*       d labels, as Table 1 shows: u_0..u_2 at distance 1, u_3, u_4 at 2). */
/*   Reach(u_i) starts as {u_i} when dist(v, u_i) < h, else empty; then for  */
/*   hop = 1..h every edge (u_i, u_j) of the subgraph induced by R ORs the   */
/*   other end's set of the previous buffer into its own (two buffers,       */
/*   alternating). Bit j of u_i's bitmap stands for u_j.                     */
/*   New h-degree of u_i at distance s: the old one, minus 1 for v, minus 1  */
/*   for every u_j with dist(v, u_j) <= h - s that Reach(u_i) misses.        */
/*                                                                           */
/* deg: in: h-degrees in G[alive]; out: those of R's members in G[alive]-v   */
/* (other entries untouched). If trace != NULL and |R| <= trace_cap, the     */
/* first 64-bit word of every member's bitmap after the initialisation and   */
/* after each hop is stored at trace[t * |R| + i], t = 0..h, and labels[i] = */
/* u_i's vertex id. Returns |R|, or -1 on ENOMEM.                            */
/* ------------------------------------------------------------------------ */
static int cmp_i32(const void *a, const void *b)
{
    const int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

int64_t orc_bitmap_update(int32_t n, const int32_t *row_ptr, const int32_t *col, const uint8_t *alive,
                          int32_t h, int32_t v, int32_t *deg, uint64_t *trace, int64_t trace_cap,
                          int32_t *labels)
{
    size_t N = (size_t)n;
    int32_t *dist = malloc(sizeof(int32_t) * N);
    int32_t *lab = malloc(sizeof(int32_t) * N);   /* vertex -> label, -1 outside R */
    int32_t *queue = malloc(sizeof(int32_t) * N);
    if (!dist || !lab || !queue) { free(dist); free(lab); free(queue); return -1; }
    for (size_t i = 0; i < N; i++) { dist[i] = -1; lab[i] = -1; }

    /* R by BFS from v inside G[alive], distances dis_G(v, .) */
    int64_t head = 0, tail = 0;
    queue[tail++] = v;
    dist[v] = 0;
    while (head < tail) {
        int32_t x = queue[head++];
        if (dist[x] == h) continue;
        for (int32_t e = row_ptr[x]; e < row_ptr[x + 1]; e++) {
            int32_t y = col[e];
            if (alive && !alive[y]) continue;
            if (dist[y] >= 0) continue;
            dist[y] = dist[x] + 1;
            queue[tail++] = y;
        }
    }
    /* labels: queue[1..tail) is in nondecreasing distance; sort each level by id */
    int32_t *R = queue + 1;
    int64_t nr = tail - 1;
    for (int64_t a = 0; a < nr;) {
        int64_t b = a;
        while (b < nr && dist[R[b]] == dist[R[a]]) b++;
        qsort(R + a, (size_t)(b - a), sizeof(int32_t), cmp_i32);
        a = b;
    }
    int64_t d = 0; /* |N_v^{h-1}|: the members that start with their own bit */
    for (int64_t i = 0; i < nr; i++) {
        lab[R[i]] = (int32_t)i;
        if (dist[R[i]] < h) d++;
    }
    const int64_t W = d > 0 ? (d + 63) / 64 : 1;
    uint64_t *reach[2];
    reach[0] = calloc((size_t)(nr > 0 ? nr : 1) * (size_t)W, sizeof(uint64_t));
    reach[1] = calloc((size_t)(nr > 0 ? nr : 1) * (size_t)W, sizeof(uint64_t));
    if (!reach[0] || !reach[1]) {
        free(reach[0]); free(reach[1]); free(dist); free(lab); free(queue);
        return -1;
    }
    /* initialisation: Reach(u_i) = {u_i} for dist < h, in both buffers */
    for (int64_t i = 0; i < d; i++) {
        reach[0][i * W + i / 64] = 1ull << (i % 64);
        reach[1][i * W + i / 64] = 1ull << (i % 64);
    }
    const int keep = trace && nr <= trace_cap;
    if (keep) {
        for (int64_t i = 0; i < nr; i++) { labels[i] = R[i]; trace[i] = reach[0][i * W]; }
    }
    /* the DP over the subgraph induced by R: each CSR entry (u_i -> u_j) is
     * one direction of an edge of E(R) */
    int p = 1, q = 0;
    for (int32_t hop = 1; hop <= h; hop++) {
        q = p;
        p = 1 - p;
        for (int64_t i = 0; i < nr; i++) {
            int32_t x = R[i];
            for (int32_t e = row_ptr[x]; e < row_ptr[x + 1]; e++) {
                int32_t j = lab[col[e]];
                if (j < 0) continue; /* v itself, dead or outside R */
                for (int64_t b = 0; b < W; b++) reach[q][i * W + b] |= reach[p][(int64_t)j * W + b];
            }
        }
        if (keep)
            for (int64_t i = 0; i < nr; i++) trace[(int64_t)hop * nr + i] = reach[q][i * W];
    }
    /* the update */
    for (int64_t i = 0; i < nr; i++) {
        int32_t u = R[i];
        int32_t s = dist[u];
        int32_t nd = deg[u] - 1;
        for (int64_t j = 0; j < nr; j++) {
            if (dist[R[j]] > h - s) break; /* labels are in distance order */
            if (!((reach[q][i * W + j / 64] >> (j % 64)) & 1ull)) nd--;
        }
        deg[u] = nd;
    }
    free(reach[0]); free(reach[1]); free(dist); free(lab); free(queue);
    return nr;
}

/* ------------------------------------------------------------------------ */
/* The paper's decomposition with that update (Sec. IV-A, Algorithm 2):     */
/* h-degrees of every vertex by BFS; then repeatedly k = the least h-degree */
/* (never below the previous k), B = the alive vertices at <= k; while B is  */
/* not empty, take its smallest vertex v, core(v) = k, update the h-degrees  */
/* of N_v^h by orc_bitmap_update, add to B every member now at <= k, and     */
/* delete v. Returns 0, or -1 on ENOMEM.                                     */
/* ------------------------------------------------------------------------ */
int orc_peel_bitmap(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t h,
                    int32_t *core_out, int32_t *order_out)
{
    if (n == 0) return 0;
    size_t N = (size_t)n;
    int32_t *deg = malloc(sizeof(int32_t) * N);
    uint8_t *alive = malloc(N);
    uint8_t *inB = calloc(N, 1);
    int32_t *dist = malloc(sizeof(int32_t) * N);
    int32_t *queue = malloc(sizeof(int32_t) * N);
    if (!deg || !alive || !inB || !dist || !queue) {
        free(deg); free(alive); free(inB); free(dist); free(queue);
        return -1;
    }
    for (size_t i = 0; i < N; i++) { alive[i] = 1; dist[i] = -1; }
    for (int32_t v = 0; v < n; v++)
        deg[v] = (int32_t)bfs_count(v, h, row_ptr, col, alive, dist, queue, NULL, NULL);
    int32_t k = 0;
    int64_t removed = 0;
    while (removed < n) {
        /* k <- min alive h-degree (not below the previous k) */
        int32_t m = -1;
        for (int32_t u = 0; u < n; u++)
            if (alive[u] && (m < 0 || deg[u] < m)) m = deg[u];
        if (m > k) k = m;
        for (int32_t u = 0; u < n; u++)
            if (alive[u] && deg[u] <= k) inB[u] = 1;
        for (;;) {
            int32_t v = -1;
            for (int32_t u = 0; u < n; u++)
                if (inB[u]) { v = u; break; }
            if (v < 0) break;
            inB[v] = 0;
            core_out[v] = k;
            if (order_out) order_out[removed] = v;
            removed++;
            if (orc_bitmap_update(n, row_ptr, col, alive, h, v, deg, NULL, 0, NULL) < 0) {
                free(deg); free(alive); free(inB); free(dist); free(queue);
                return -1;
            }
            alive[v] = 0;
            for (int32_t u = 0; u < n; u++)
                if (alive[u] && !inB[u] && deg[u] <= k) inB[u] = 1;
        }
    }
    free(deg); free(alive); free(inB); free(dist); free(queue);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The paper's sampling variant (Sec. IV-C, Algorithms 5 and 6). The sample  */
/* S is an input (in_s[v] != 0: v in S), drawn by the caller.                */
/*                                                                           */
/*   select[v] = |N_v^h(G) ∩ S| and rate[v] = select[v] / d_v^h(G) at the   */
/*   start; the estimated h-degree is select[v] / rate[v], taken in exact    */
/*   integer arithmetic and rounded down: floor(select * d0 / select0) (the  */
/*   paper's example turns 8 / 0.45 into 17).                                */
/*   Peeling as in Algorithm 2 on the estimates. Deleting v (Algorithm 6):   */
/*   bitmaps only for the sampled members of N_v^{h-1}, the same DP on the   */
/*   subgraph induced by N_v^h; every member u at distance s loses          */
/*   cnt = [v in S] + |{sampled u_j, dist(v, u_j) <= h - s, not reached}|    */
/*   from select[u] (<= as in Algorithm 4, so that S = V gives Algorithm 2   */
/*   exactly).                                                               */
/*   A vertex whose initial ball holds no sampled vertex (select0 = 0) has  */
/*   no rate (Algorithm 5 divides by it): it keeps its exact h-degree,       */
/*   recomputed by BFS after every deletion within h of it (the estimate    */
/*   every full sample gives; it makes each estimate a function of the      */
/*   surviving vertex set, like select and the h-degree).                    */
/* core_out: the core estimates. Returns 0, or -1 on ENOMEM.                 */
/* ------------------------------------------------------------------------ */
static int32_t sampled_estimate(int64_t sel, int64_t sel0, int64_t d0, int32_t fallback)
{
    if (sel0 <= 0) return fallback;
    if (sel <= 0) return 0;
    return (int32_t)((sel * d0) / sel0);
}

static int64_t sampled_update(int32_t n, const int32_t *row_ptr, const int32_t *col, const uint8_t *alive,
                              const uint8_t *in_s, int32_t h, int32_t v, int64_t *sel, const int64_t *sel0,
                              const int32_t *d0, int32_t *est)
{
    size_t N = (size_t)n;
    int32_t *dist = malloc(sizeof(int32_t) * N);
    int32_t *lab = malloc(sizeof(int32_t) * N);
    int32_t *queue = malloc(sizeof(int32_t) * N);
    if (!dist || !lab || !queue) { free(dist); free(lab); free(queue); return -1; }
    for (size_t i = 0; i < N; i++) { dist[i] = -1; lab[i] = -1; }
    int64_t head = 0, tail = 0;
    queue[tail++] = v;
    dist[v] = 0;
    while (head < tail) {
        int32_t x = queue[head++];
        if (dist[x] == h) continue;
        for (int32_t e = row_ptr[x]; e < row_ptr[x + 1]; e++) {
            int32_t y = col[e];
            if (!alive[y] || dist[y] >= 0) continue;
            dist[y] = dist[x] + 1;
            queue[tail++] = y;
        }
    }
    int32_t *R = queue + 1;
    const int64_t nr = tail - 1;
    for (int64_t a = 0; a < nr;) {
        int64_t b = a;
        while (b < nr && dist[R[b]] == dist[R[a]]) b++;
        qsort(R + a, (size_t)(b - a), sizeof(int32_t), cmp_i32);
        a = b;
    }
    /* bit index: the sampled members of N_v^{h-1}, in label order */
    int32_t *bit = malloc(sizeof(int32_t) * (size_t)(nr > 0 ? nr : 1));
    if (!bit) { free(dist); free(lab); free(queue); return -1; }
    int64_t d = 0;
    for (int64_t i = 0; i < nr; i++) {
        lab[R[i]] = (int32_t)i;
        bit[i] = (dist[R[i]] < h && in_s[R[i]]) ? (int32_t)d++ : -1;
    }
    const int64_t W = d > 0 ? (d + 63) / 64 : 1;
    uint64_t *reach[2];
    reach[0] = calloc((size_t)(nr > 0 ? nr : 1) * (size_t)W, sizeof(uint64_t));
    reach[1] = calloc((size_t)(nr > 0 ? nr : 1) * (size_t)W, sizeof(uint64_t));
    if (!reach[0] || !reach[1]) {
        free(reach[0]); free(reach[1]); free(bit); free(dist); free(lab); free(queue);
        return -1;
    }
    for (int64_t i = 0; i < nr; i++)
        if (bit[i] >= 0) {
            reach[0][i * W + bit[i] / 64] = 1ull << (bit[i] % 64);
            reach[1][i * W + bit[i] / 64] = 1ull << (bit[i] % 64);
        }
    int p = 1, q = 0;
    for (int32_t hop = 1; hop <= h; hop++) {
        q = p;
        p = 1 - p;
        for (int64_t i = 0; i < nr; i++) {
            int32_t x = R[i];
            for (int32_t e = row_ptr[x]; e < row_ptr[x + 1]; e++) {
                int32_t j = lab[col[e]];
                if (j < 0) continue;
                for (int64_t b = 0; b < W; b++) reach[q][i * W + b] |= reach[p][(int64_t)j * W + b];
            }
        }
    }
    for (int64_t i = 0; i < nr; i++) {
        int32_t u = R[i];
        int32_t s = dist[u];
        int64_t cnt = in_s[v] ? 1 : 0;
        for (int64_t j = 0; j < nr; j++) {
            if (dist[R[j]] > h - s) break;
            if (bit[j] < 0) continue; /* not sampled */
            if (!((reach[q][i * W + bit[j] / 64] >> (bit[j] % 64)) & 1ull)) cnt++;
        }
        sel[u] -= cnt;
        est[u] = sampled_estimate(sel[u], sel0[u], d0[u], est[u] - 1);
    }
    free(reach[0]); free(reach[1]); free(bit); free(dist); free(lab); free(queue);
    return nr;
}

int orc_peel_sampled(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t h, const uint8_t *in_s,
                     int32_t *core_out, int32_t *est_init_out)
{
    if (n == 0) return 0;
    size_t N = (size_t)n;
    int32_t *d0 = malloc(sizeof(int32_t) * N);
    int32_t *est = malloc(sizeof(int32_t) * N);
    int64_t *sel = malloc(sizeof(int64_t) * N);
    int64_t *sel0 = malloc(sizeof(int64_t) * N);
    uint8_t *alive = malloc(N);
    uint8_t *inB = calloc(N, 1);
    int32_t *dist = malloc(sizeof(int32_t) * N);
    int32_t *queue = malloc(sizeof(int32_t) * N);
    int32_t *ball = malloc(sizeof(int32_t) * N);
    if (!d0 || !est || !sel || !sel0 || !alive || !inB || !dist || !queue || !ball) {
        free(d0); free(est); free(sel); free(sel0); free(alive); free(inB); free(dist); free(queue); free(ball);
        return -1;
    }
    for (size_t i = 0; i < N; i++) { alive[i] = 1; dist[i] = -1; }
    /* Algorithm 5, lines 1-4: exact h-degrees, the sampled counts and rates */
    for (int32_t v = 0; v < n; v++) {
        int64_t len = 0;
        d0[v] = (int32_t)bfs_count(v, h, row_ptr, col, alive, dist, queue, ball, &len);
        int64_t c = 0;
        for (int64_t i = 0; i < len; i++) c += in_s[ball[i]] ? 1 : 0;
        sel[v] = sel0[v] = c;
    }
    for (int32_t v = 0; v < n; v++) {
        est[v] = d0[v] == 0 ? 0 : sampled_estimate(sel[v], sel0[v], d0[v], d0[v]);
        if (est_init_out) est_init_out[v] = est[v];
    }
    /* lines 5-7: Algorithm 2 on the estimates */
    int32_t k = 0;
    int64_t removed = 0;
    while (removed < n) {
        int32_t m = -1;
        for (int32_t u = 0; u < n; u++)
            if (alive[u] && (m < 0 || est[u] < m)) m = est[u];
        if (m > k) k = m;
        for (int32_t u = 0; u < n; u++)
            if (alive[u] && est[u] <= k) inB[u] = 1;
        for (;;) {
            int32_t v = -1;
            for (int32_t u = 0; u < n; u++)
                if (inB[u]) { v = u; break; }
            if (v < 0) break;
            inB[v] = 0;
            core_out[v] = k;
            removed++;
            int64_t blen = 0;
            bfs_count(v, h, row_ptr, col, alive, dist, queue, ball, &blen);
            if (sampled_update(n, row_ptr, col, alive, in_s, h, v, sel, sel0, d0, est) < 0) {
                free(d0); free(est); free(sel); free(sel0); free(alive); free(inB); free(dist); free(queue);
                free(ball);
                return -1;
            }
            alive[v] = 0;
            /* members without a rate keep their exact h-degree */
            for (int64_t i = 0; i < blen; i++)
                if (sel0[ball[i]] == 0)
                    est[ball[i]] = (int32_t)bfs_count(ball[i], h, row_ptr, col, alive, dist, queue, NULL, NULL);
            for (int32_t u = 0; u < n; u++)
                if (alive[u] && !inB[u] && est[u] <= k) inB[u] = 1;
        }
    }
    free(d0); free(est); free(sel); free(sel0); free(alive); free(inB); free(dist); free(queue); free(ball);
    return 0;
}

/* The estimator alone (for the pins): floor(sel * d0 / sel0). */
int32_t orc_sampled_estimate(int64_t sel, int64_t sel0, int64_t d0) { return sampled_estimate(sel, sel0, d0, -1); }

/* ------------------------------------------------------------------------ */
/* Definition 2 by exhaustion, for n <= 24: adj[v] is v's neighbour bitmask.  */
/* For every non-empty S, mu(S) = min over w in S of d_w^h(G(S)); then        */
/* core_h(v) = max over S containing v of mu(S).                              */
/* ------------------------------------------------------------------------ */
static int popcount32(uint32_t x) { int c = 0; while (x) { x &= x - 1; c++; } return c; }

int orc_bruteforce(int32_t n, const uint32_t *adj, int32_t h, int32_t *core_out)
{
    if (n < 0 || n > 24) return -1;
    for (int32_t v = 0; v < n; v++) core_out[v] = 0;
    uint32_t full = n == 32 ? 0xffffffffu : ((1u << n) - 1u);
    for (uint32_t S = 1; S <= full && S != 0; S++) {
        int32_t mu = 1 << 30;
        for (int32_t w = 0; w < n && mu > 0; w++) {
            if (!(S >> w & 1u)) continue;
            uint32_t ball = 1u << w, frontier = 1u << w;
            for (int32_t step = 0; step < h && frontier; step++) {
                uint32_t reach = 0;
                for (int32_t x = 0; x < n; x++)
                    if (frontier >> x & 1u) reach |= adj[x];
                reach &= S & ~ball;
                ball |= reach;
                frontier = reach;
            }
            int32_t d = popcount32(ball) - 1;
            if (d < mu) mu = d;
        }
        for (int32_t v = 0; v < n; v++)
            if ((S >> v & 1u) && mu > core_out[v]) core_out[v] = mu;
        if (S == full) break;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Classic k-core (h = 1) by the Batagelj-Zaversnik bin sort.                */
/* ------------------------------------------------------------------------ */
int orc_kcore_bz(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t *core_out)
{
    if (n == 0) return 0;
    size_t N = (size_t)n;
    int32_t maxd = 0;
    int32_t *deg = malloc(sizeof(int32_t) * N);
    int32_t *vert = malloc(sizeof(int32_t) * N);
    int32_t *pos = malloc(sizeof(int32_t) * N);
    if (!deg || !vert || !pos) { free(deg); free(vert); free(pos); return -1; }
    for (int32_t v = 0; v < n; v++) {
        deg[v] = row_ptr[v + 1] - row_ptr[v];
        if (deg[v] > maxd) maxd = deg[v];
    }
    int32_t *bin = calloc((size_t)maxd + 2, sizeof(int32_t));
    if (!bin) { free(deg); free(vert); free(pos); return -1; }
    for (int32_t v = 0; v < n; v++) bin[deg[v]]++;
    int32_t start = 0;                    /* bin[d] becomes the first slot of degree d */
    for (int32_t d = 0; d <= maxd; d++) { int32_t c = bin[d]; bin[d] = start; start += c; }
    for (int32_t v = 0; v < n; v++) { pos[v] = bin[deg[v]]; vert[pos[v]] = v; bin[deg[v]]++; }
    for (int32_t d = maxd; d >= 1; d--) bin[d] = bin[d - 1];
    bin[0] = 0;
    for (int32_t i = 0; i < n; i++) {
        int32_t v = vert[i];              /* v has the smallest current degree */
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; e++) {
            int32_t u = col[e];
            if (deg[u] > deg[v]) {        /* move u to the front of its bin, then shrink it */
                int32_t du = deg[u], pu = pos[u], pw = bin[du], w = vert[pw];
                if (u != w) { pos[u] = pw; vert[pu] = w; pos[w] = pu; vert[pw] = u; }
                bin[du]++;
                deg[u]--;
            }
        }
    }
    for (int32_t v = 0; v < n; v++) core_out[v] = deg[v];
    free(deg); free(vert); free(pos); free(bin);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Certificate check for a claimed core index c[] and peel round r[].        */
/*  (0) every round holds one c value, and c never falls as r grows;         */
/*  (i)  d_v^h(G[{w : c[w] >= c[v]}]) >= c[v];                                */
/*  (ii) d_v^h(G[{w : r[w] >= r[v]}]) <= c[v].                                */
/* (i) for all v makes each {c >= k} a subgraph whose h-degrees are all >= k, */
/* so c <= core. For (ii): take the true (k+1,h)-core K and its vertex x of  */
/* smallest round; K lies inside {r >= r[x]}, so by (ii)                     */
/* c[x] >= d_x^h(G[K]) >= k+1, and by (0) every vertex of K has c >= c[x].   */
/* So c >= core. With both for every vertex, c equals the core index.        */
/* (0) is checked on every vertex; (i) and (ii) on the listed vertices.      */
/* Returns the number of failed checks (0 = pass); bad_out (nullable, one    */
/* int32 per listed vertex) gets a bitmask 1 = (i) failed, 2 = (ii) failed.  */
/* Returns -1 on ENOMEM.                                                     */
/* ------------------------------------------------------------------------ */
int64_t orc_certificate(int32_t n, const int32_t *row_ptr, const int32_t *col,
                        int32_t h, const int32_t *c, const int32_t *r,
                        int64_t count, const int32_t *verts, int32_t *bad_out)
{
    int64_t fails = 0;
    if (n == 0) return 0;
    /* (0) */
    int32_t rmax = 0;
    for (int32_t v = 0; v < n; v++) {
        if (r[v] < 0 || c[v] < 0) return -2;
        if (r[v] > rmax) rmax = r[v];
    }
    int32_t *cr = malloc(sizeof(int32_t) * ((size_t)rmax + 1));
    if (!cr) return -1;
    for (int32_t i = 0; i <= rmax; i++) cr[i] = -1;
    for (int32_t v = 0; v < n; v++) {
        if (cr[r[v]] < 0) cr[r[v]] = c[v];
        else if (cr[r[v]] != c[v]) fails++;
    }
    int32_t last = -1;
    for (int32_t i = 0; i <= rmax; i++) {
        if (cr[i] < 0) continue;
        if (cr[i] < last) fails++;
        last = cr[i];
    }
    free(cr);

    int64_t f2 = 0;
    int err = 0;
#pragma omp parallel reduction(+ : f2)
    {
        int32_t *dist = malloc(sizeof(int32_t) * (size_t)n);
        int32_t *queue = malloc(sizeof(int32_t) * (size_t)n);
        uint8_t *mask = malloc((size_t)n);
        if (!dist || !queue || !mask) {
#pragma omp atomic write
            err = 1;
        } else {
            for (int32_t i = 0; i < n; i++) dist[i] = -1;
#pragma omp for schedule(dynamic, 1)
            for (int64_t i = 0; i < count; i++) {
                int32_t v = verts[i];
                int32_t bad = 0;
                for (int32_t w = 0; w < n; w++) mask[w] = c[w] >= c[v];
                if (bfs_count(v, h, row_ptr, col, mask, dist, queue, NULL, NULL) < c[v]) bad |= 1;
                for (int32_t w = 0; w < n; w++) mask[w] = r[w] >= r[v];
                if (bfs_count(v, h, row_ptr, col, mask, dist, queue, NULL, NULL) > c[v]) bad |= 2;
                if (bad_out) bad_out[i] = bad;
                if (bad) f2++;
            }
        }
        free(dist); free(queue); free(mask);
    }
    if (err) return -1;
    return fails + f2;
}

/* ------------------------------------------------------------------------ */
/* The same certificate on EVERY vertex, fast enough for the 1e6-vertex      */
/* graphs. Conditions (0), (i) and (ii) are exactly those of                  */
/* orc_certificate; what changes is how the BFS counts are taken:             */
/*  - the vertex set of each BFS ({c >= c[v]} for (i), {r >= r[v]} for (ii))  */
/*    is tested on the fly from c[] and r[] (no n-byte mask per vertex);      */
/*  - a vertex with c[v] <= small_cap runs its own BFS, stopped as soon as    */
/*    the inequality is decided ((i) holds once c[v] other vertices are       */
/*    reached, (ii) fails once c[v] + 1 are);                                 */
/*  - the other vertices are checked 64*W at a time by a bit-parallel BFS:   */
/*    bit j of a vertex's W words stands for source j of the batch. For one  */
/*    condition the sources are sorted by key (c or r), so that a vertex u   */
/*    belongs to source j's subgraph {key >= key[s_j]} exactly for the first */
/*    acc(u) sources of the batch, acc(u) = |{j : key[s_j] <= key[u]}|; u    */
/*    carries and passes on only those bits.                                 */
/* Returns the number of failed checks (0 = pass), -1 on ENOMEM, -2 on a    */
/* negative value; bad_out (nullable, int32[n]) as for orc_certificate.     */
/* ------------------------------------------------------------------------ */

/* BFS from v to radius h inside {u : key[u] >= key[v]}; stops once `cap`    */
/* other vertices are reached. Returns min(reached, cap). dist[] all -1 on   */
/* entry and on return.                                                      */
static int64_t bfs_count_capped(int32_t v, int32_t h, const int32_t *row_ptr, const int32_t *col,
                                const int32_t *key, int64_t cap, int32_t *dist, int32_t *queue)
{
    const int32_t kv = key[v];
    int64_t head = 0, tail = 0, reached = 0;
    queue[tail++] = v;
    dist[v] = 0;
    while (head < tail && reached < cap) {
        int32_t x = queue[head++];
        if (dist[x] == h) continue;
        for (int32_t e = row_ptr[x]; e < row_ptr[x + 1] && reached < cap; e++) {
            int32_t y = col[e];
            if (key[y] < kv || dist[y] >= 0) continue; /* outside the subgraph, or seen */
            dist[y] = dist[x] + 1;
            queue[tail++] = y;
            reached++;
        }
    }
    for (int64_t i = 0; i < tail; i++) dist[queue[i]] = -1;
    return reached;
}

static const int32_t *g_sort_key; /* qsort has no context argument */
static int cmp_by_key(const void *a, const void *b)
{
    const int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    const int32_t kx = g_sort_key[x], ky = g_sort_key[y];
    if (kx != ky) return (kx > ky) - (kx < ky);
    return (x > y) - (x < y);
}

/* Bits of word k (sources 64k .. 64k+63) that stand for the first a sources. */
static uint64_t prefix_bits(int64_t a, int k)
{
    const int64_t lo = 64 * (int64_t)k;
    if (a >= lo + 64) return ~0ull;
    if (a <= lo) return 0ull;
    return (1ull << (a - lo)) - 1ull;
}

/* Adds the byte-sliced column counts sl (W words x 8 slices) into lc and
 * clears them: byte b of slice t of word k counts column 64k + 8b + t. */
static void slice_flush(uint64_t *sl, int64_t *lc, int W)
{
    for (int k = 0; k < W; k++)
        for (int t = 0; t < 8; t++) {
            uint64_t v = sl[8 * k + t];
            for (int b = 0; b < 8; b++) lc[64 * k + 8 * b + t] += (int64_t)((v >> (8 * b)) & 0xffu);
            sl[8 * k + t] = 0;
        }
}

/* One condition (cond 1: count >= c[s]; cond 2: count <= c[s]) for the
 * sources srcs[0..ns), sorted by key, 64*W per batch. */
static int bits_condition(int32_t n, const int32_t *rp, const int32_t *col, int32_t h, const int32_t *key,
                          const int32_t *c, const int32_t *srcs, int64_t ns, int cond, int W,
                          int32_t *bad_out)
{
    const int64_t B = 64 * (int64_t)W;
    const size_t words = (size_t)n * (size_t)W;
    uint64_t *V = malloc(sizeof(uint64_t) * words);
    uint64_t *F = malloc(sizeof(uint64_t) * words);
    uint64_t *N = malloc(sizeof(uint64_t) * words);
    uint8_t *fl = malloc((size_t)n), *fn = malloc((size_t)n);
    int32_t *acc = malloc(sizeof(int32_t) * (size_t)n);
    int64_t *cnt = malloc(sizeof(int64_t) * (size_t)B);
    if (!V || !F || !N || !fl || !fn || !acc || !cnt) {
        free(V); free(F); free(N); free(fl); free(fn); free(acc); free(cnt);
        return -1;
    }
    int oom = 0;
    for (int64_t b0 = 0; b0 < ns && !oom; b0 += B) {
        const int64_t nb = ns - b0 < B ? ns - b0 : B;
        const int32_t *bs = srcs + b0;
        const int32_t kmin = key[bs[0]], kmax = key[bs[nb - 1]];
#pragma omp parallel for schedule(static)
        for (int32_t u = 0; u < n; u++) {
            const int32_t ku = key[u];
            int64_t a;
            if (ku < kmin) a = 0;
            else if (ku >= kmax) a = nb;
            else { /* first batch position whose key exceeds ku */
                int64_t lo = 0, hi = nb;
                while (lo < hi) {
                    const int64_t mid = (lo + hi) / 2;
                    if (key[bs[mid]] <= ku) lo = mid + 1; else hi = mid;
                }
                a = lo;
            }
            acc[u] = (int32_t)a;
            for (int k = 0; k < W; k++) V[(size_t)u * W + k] = F[(size_t)u * W + k] = 0;
            fl[u] = 0;
        }
        for (int64_t j = 0; j < nb; j++) {
            const int32_t s = bs[j];
            V[(size_t)s * W + j / 64] |= 1ull << (j % 64);
            F[(size_t)s * W + j / 64] |= 1ull << (j % 64);
            fl[s] = 1;
        }
        for (int64_t j = 0; j < B; j++) cnt[j] = 0;
        for (int32_t lvl = 1; lvl <= h; lvl++) {
#pragma omp parallel
            {
                /* column counts: byte t of sl[8k + t'] counts bit 8t + t' of
                 * word k over the words added; flushed every 255 adds */
                int64_t *lc = calloc((size_t)B, sizeof(int64_t));
                uint64_t *sl = calloc((size_t)W * 8, sizeof(uint64_t));
                int adds = 0;
                uint64_t x[64];
                if (!lc || !sl) {
#pragma omp atomic write
                    oom = 1;
                }
#pragma omp for schedule(dynamic, 1024)
                for (int32_t u = 0; u < n; u++) {
                    fn[u] = 0;
                    if (oom) continue;
                    const int32_t a = acc[u];
                    if (a == 0) continue;
                    int any = 0;
                    for (int k = 0; k < W; k++) x[k] = 0;
                    for (int32_t e = rp[u]; e < rp[u + 1]; e++) {
                        const int32_t w = col[e];
                        if (!fl[w]) continue;
                        for (int k = 0; k < W; k++) x[k] |= F[(size_t)w * W + k];
                    }
                    for (int k = 0; k < W; k++) {
                        x[k] &= ~V[(size_t)u * W + k] & prefix_bits(a, k);
                        any |= x[k] != 0;
                    }
                    if (!any) continue;
                    fn[u] = 1;
                    for (int k = 0; k < W; k++) {
                        N[(size_t)u * W + k] = x[k];
                        V[(size_t)u * W + k] |= x[k];
                        for (int t = 0; t < 8; t++) sl[8 * k + t] += (x[k] >> t) & 0x0101010101010101ull;
                    }
                    if (++adds == 255) {
                        slice_flush(sl, lc, W);
                        adds = 0;
                    }
                }
                if (lc && sl) {
                    slice_flush(sl, lc, W);
#pragma omp critical
                    for (int64_t j = 0; j < B; j++) cnt[j] += lc[j];
                }
                free(lc);
                free(sl);
            }
            if (oom) break;
            uint64_t *t = F; F = N; N = t;
            uint8_t *tf = fl; fl = fn; fn = tf;
        }
        for (int64_t j = 0; j < nb; j++) {
            const int32_t s = bs[j];
            if (cond == 1 ? (cnt[j] < c[s]) : (cnt[j] > c[s])) bad_out[s] |= cond;
        }
    }
    free(V); free(F); free(N); free(fl); free(fn); free(acc); free(cnt);
    return oom ? -1 : 0;
}

int64_t orc_certificate_all(int32_t n, const int32_t *row_ptr, const int32_t *col,
                            int32_t h, const int32_t *c, const int32_t *r, int32_t small_cap, int32_t W,
                            int32_t *bad_out)
{
    int64_t fails = 0;
    if (n == 0) return 0;
    if (W < 1 || W > 64) return -2;
    /* (0) */
    int32_t rmax = 0;
    for (int32_t v = 0; v < n; v++) {
        if (r[v] < 0 || c[v] < 0) return -2;
        if (r[v] > rmax) rmax = r[v];
    }
    int32_t *cr = malloc(sizeof(int32_t) * ((size_t)rmax + 1));
    if (!cr) return -1;
    for (int32_t i = 0; i <= rmax; i++) cr[i] = -1;
    for (int32_t v = 0; v < n; v++) {
        if (cr[r[v]] < 0) cr[r[v]] = c[v];
        else if (cr[r[v]] != c[v]) fails++;
    }
    int32_t last = -1;
    for (int32_t i = 0; i <= rmax; i++) {
        if (cr[i] < 0) continue;
        if (cr[i] < last) fails++;
        last = cr[i];
    }
    free(cr);
    int32_t *bad_mem = NULL;
    if (!bad_out) {
        bad_mem = malloc(sizeof(int32_t) * (size_t)n);
        if (!bad_mem) return -1;
        bad_out = bad_mem;
    }
    for (int32_t v = 0; v < n; v++) bad_out[v] = 0;

    /* vertices with a small claimed core: one early-stopped BFS each */
    int64_t f2 = 0;
    int err = 0;
#pragma omp parallel reduction(+ : f2)
    {
        int32_t *dist = malloc(sizeof(int32_t) * (size_t)n);
        int32_t *queue = malloc(sizeof(int32_t) * (size_t)n);
        if (!dist || !queue) {
#pragma omp atomic write
            err = 1;
        } else {
            for (int32_t i = 0; i < n; i++) dist[i] = -1;
#pragma omp for schedule(dynamic, 256)
            for (int32_t v = 0; v < n; v++) {
                if (c[v] > small_cap) continue;
                int32_t bad = 0;
                /* (i): at least c[v] others within h in G[{c >= c[v]}] */
                if (bfs_count_capped(v, h, row_ptr, col, c, c[v], dist, queue) < c[v]) bad |= 1;
                /* (ii): at most c[v] others within h in G[{r >= r[v]}] */
                if (bfs_count_capped(v, h, row_ptr, col, r, (int64_t)c[v] + 1, dist, queue) > c[v]) bad |= 2;
                bad_out[v] = bad;
            }
        }
        free(dist); free(queue);
    }
    if (err) { free(bad_mem); return -1; }

    /* the others: bit-parallel, 64*W sources per BFS, one pass per condition */
    int64_t ns = 0;
    for (int32_t v = 0; v < n; v++) ns += c[v] > small_cap;
    if (ns > 0) {
        int32_t *srcs = malloc(sizeof(int32_t) * (size_t)ns);
        if (!srcs) { free(bad_mem); return -1; }
        for (int cond = 1; cond <= 2; cond++) {
            const int32_t *key = cond == 1 ? c : r;
            int64_t i = 0;
            for (int32_t v = 0; v < n; v++)
                if (c[v] > small_cap) srcs[i++] = v;
            g_sort_key = key;
            qsort(srcs, (size_t)ns, sizeof(int32_t), cmp_by_key);
            if (bits_condition(n, row_ptr, col, h, key, c, srcs, ns, cond, W, bad_out) < 0) {
                free(srcs);
                free(bad_mem);
                return -1;
            }
        }
        free(srcs);
    }
    /* a vertex failing both conditions counts once, as in orc_certificate */
    for (int32_t v = 0; v < n; v++) f2 += bad_out[v] != 0;
    free(bad_mem);
    return fails + f2;
}

int orc_has_openmp(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 0;
#endif
}
