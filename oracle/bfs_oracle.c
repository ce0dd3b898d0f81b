/*
 * bfs_oracle.c -- the CPU oracle for breadth-first search.  TEST
 * INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
 * baseline may call it; the library's product path never does.
 *
 * What it computes (Section "Preliminaries" and Algorithm 1, Parallel Top
 * Down BFS): for a graph G=(V,E) stored as CSR and a root r, d[v] is the
 * number of hops of a shortest directed path r -> v, and d[v] = infinity when
 * no path exists.  Infinity is encoded as -1.  Algorithm 1 sets every d to
 * infinity, puts the root in the queue with d[root] = 0, and then, level by
 * level, gives every unvisited neighbour u of a frontier vertex v the
 * distance d[v]+1 and enqueues it.  Run serially with one FIFO queue, the
 * levels come out of the queue in order, which is the textbook serial BFS.
 *
 * Parents are not part of Algorithm 1; this oracle records the vertex that
 * first reached each vertex (parent[root] = root, -1 when unreached) only as
 * one valid example -- any neighbour one level closer to the root is equally
 * valid.  It also reports the number of vertices per level and the number
 * of adjacency entries scanned (sum of the out-degrees of reached vertices,
 * the top-down work behind the TEPS figure of Section "Top Down Vs. Bottom
 * Up").
 *
 * Shares no code with the GPU library.
 */
#include <stdint.h>
#include <stdlib.h>

/* Returns the number of levels (>= 1 for a valid root), or a negative value
 * on a bad argument.  level_sizes (nullable) receives up to max_levels
 * counts; *edges_scanned (nullable) receives the scanned entry count. */
int64_t oracle_bfs(int64_t n, const int64_t* off, const int32_t* col, int64_t root,
                   int32_t* dist, int32_t* parent, int64_t* level_sizes, int64_t max_levels,
                   int64_t* edges_scanned)
{
    if (n <= 0 || root < 0 || root >= n) return -1;
    for (int64_t v = 0; v < n; ++v) {
        dist[v] = -1;
        if (parent) parent[v] = -1;
    }
    int32_t* queue = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!queue) return -2;

    int64_t head = 0, tail = 0, scanned = 0, nlevels = 0;
    queue[tail++] = (int32_t)root;
    dist[root] = 0;
    if (parent) parent[root] = (int32_t)root;

    while (head < tail) {
        int32_t v = queue[head++];
        int32_t dv = dist[v];
        if (dv + 1 > nlevels) {
            nlevels = dv + 1;
        }
        if (level_sizes && dv < max_levels) level_sizes[dv] += 1;
        for (int64_t e = off[v]; e < off[v + 1]; ++e) {
            int32_t u = col[e];
            ++scanned;
            if (dist[u] == -1) {
                dist[u] = dv + 1;
                if (parent) parent[u] = v;
                queue[tail++] = u;
            }
        }
    }
    free(queue);
    if (edges_scanned) *edges_scanned = scanned;
    return nlevels;
}

/* The batched result is, by definition, one independent BFS per root:
 * dist is k rows of n, row i the distances from roots[i]. */
int64_t oracle_bfs_multi(int64_t n, const int64_t* off, const int32_t* col, const int64_t* roots,
                         int64_t k, int32_t* dist, int64_t* edges_scanned)
{
    int64_t total = 0;
    for (int64_t i = 0; i < k; ++i) {
        int64_t m = 0;
        int64_t rc = oracle_bfs(n, off, col, roots[i], dist + i * n, NULL, NULL, 0, &m);
        if (rc < 0) return rc;
        if (edges_scanned) edges_scanned[i] = m;
        total += m;
    }
    return total;
}

/* Shortest-path counts, optionally on the subgraph of entries whose weight
 * passes a filter.  Section "Top Down Vs. Bottom Up" names both as problems
 * a bottom-up level cannot serve: betweenness-type computations need every
 * shortest path, and weight-filtering BFS follows only the edges of given
 * weights, so every edge out of the frontier has to be examined.
 *
 * Definition: keep the CSR entries e with lo <= weight[e] <= hi (all of
 * them when weight is NULL).  In that subgraph hops[v] is the length of a
 * shortest root -> v path (-1 when there is none) and sigma[v] the number of
 * distinct shortest root -> v paths, a path being a sequence of kept entries
 * (a duplicated entry gives two paths); sigma[root] = 1, sigma = 0 where
 * unreached.
 *
 * Computed as the forward phase of Brandes' algorithm (U. Brandes, "A faster
 * algorithm for betweenness centrality", J. Math. Sociol. 25(2), 2001):
 * serial FIFO BFS over the kept entries; an entry a -> b reaching b for the
 * first time sets hops[b] = hops[a] + 1, and every kept entry with
 * hops[b] = hops[a] + 1 adds sigma[a] to sigma[b].  A vertex leaves the FIFO
 * only after every vertex one level closer, so its count is complete when
 * it is expanded.  Counts are summed in double.
 *
 * Returns the number of levels, or a negative value on a bad argument.
 * *edges_scanned (nullable) receives the entries of the reached vertices'
 * rows, kept or not. */
int64_t oracle_bfs_paths(int64_t n, const int64_t* off, const int32_t* col,
                         const int32_t* weight, int32_t lo, int32_t hi, int64_t root,
                         int32_t* hops, double* sigma, int64_t* edges_scanned)
{
    if (n <= 0 || root < 0 || root >= n) return -1;
    int32_t* fifo = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!fifo) return -2;
    for (int64_t x = 0; x < n; ++x) {
        hops[x] = -1;
        sigma[x] = 0.0;
    }
    int64_t first = 0, last = 0, seen = 0, depth = 0;
    hops[root] = 0;
    sigma[root] = 1.0;
    fifo[last++] = (int32_t)root;
    while (first < last) {
        const int32_t a = fifo[first++];
        const int32_t ha = hops[a];
        if (ha + 1 > depth) depth = ha + 1;
        for (int64_t k = off[a]; k < off[a + 1]; ++k) {
            ++seen;
            if (weight && (weight[k] < lo || weight[k] > hi)) continue;
            const int32_t b = col[k];
            if (hops[b] < 0) {
                hops[b] = ha + 1;
                fifo[last++] = b;
            }
            if (hops[b] == ha + 1) sigma[b] += sigma[a];
        }
    }
    free(fifo);
    if (edges_scanned) *edges_scanned = seen;
    return depth;
}
