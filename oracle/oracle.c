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
 *   orc_certificate   checks a claimed core index c and peel round r against
 *                     two inequalities that together imply c is exact (the
 *                     argument is written above the function).
 *
 * Readings of the paper taken here:
 *   - k starts at 0, so isolated vertices get core index 0 (Algorithm 1 starts
 *     its bucket loop at 1 and would never empty B[0]).
 *   - After deleting v, distances are measured in the surviving induced
 *     subgraph only (Definition 2 measures d^h inside the subgraph).
 *
 * Pins: tests/test_oracle_pins.py checks every routine against brute force,
 * closed forms, SciPy's all-pairs shortest paths, networkx.core_number at
 * h = 1, the paper's worked example (Example 1, Example 2) and invariants.
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

int orc_has_openmp(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 0;
#endif
}
