/*
 * bfs_check.c -- a streaming certificate check of a BFS result.  TEST
 * INFRASTRUCTURE ONLY (tests, the smoke check and the benchmark's parity
 * record); the library's product path never calls it, and it shares no code
 * with the GPU library or with bfs_oracle.c.
 *
 * For a root r and a candidate distance array d (-1 = unreached,
 * Section "Preliminaries": d = infinity when no path exists), the checks
 * below hold together exactly when d is the vector of shortest-path hop
 * counts from r (the result Algorithm 1 defines):
 *
 *   C0  d[r] = 0;
 *   C1  no d is below -1;
 *   C2  every out-entry u -> v of a reached vertex u leads to a reached v;
 *   C3  along every such entry d[v] <= d[u] + 1;
 *   C4  every reached v != r has a predecessor witness: an entry u -> v
 *       with u reached and d[u] = d[v] - 1.  (So no vertex but r has
 *       d = 0: its witness would need d = -1, which is not reached.)
 *
 * Why this pins d exactly.  Along a shortest path r = x0 -> ... -> xk, C0,
 * C2 and C3 give by induction that every xi is reached with d[xi] <= i, so
 * d <= the true distance and every vertex with a path is reached.
 * Following witnesses from a reached v (C4) lowers d by one per step over
 * real entries and can only stop at r, the one reached vertex that needs
 * no witness: a path of length d[v] exists, so d >= the true distance.  A
 * reached vertex therefore has a path, and an unreached one has none (C2).
 * These are the Graph500 validation rules in directed form; on a symmetric
 * graph C2 and C3 imply their undirected versions.
 *
 * With a parent array p the tree is checked too (the GPU's parents are
 * accepted by these rules, not compared, because several are valid):
 *   P0  p[r] = r;
 *   P1  an unreached vertex has p = -1;
 *   P2  a reached v != r has as p[v] a reached vertex one level closer
 *       (d[p[v]] = d[v] - 1) whose row holds the entry p[v] -> v.
 * P2 is checked with the same marks as C4: scanning the entries u -> v of
 * reached rows with d[v] = d[u] + 1, the one whose u is p[v] marks v.
 *
 * One pass over the reached vertices' rows (C2, C3, and the witness and
 * parent marks), split over threads by row ranges of about equal
 * entry counts; one pass over the vertices for the rest.  The marks are
 * byte flags set with relaxed atomic stores (several threads may set the
 * same flag; none clears it).  Counts of each violation come back in bad[].
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum {
    BAD_ROOT_DIST = 0,      /* C0 */
    BAD_RANGE = 1,          /* C1 */
    BAD_REACH_GAP = 2,      /* C2 */
    BAD_LEVEL_SKIP = 3,     /* C3 */
    BAD_NO_WITNESS = 4,     /* C4 */
    BAD_ROOT_PARENT = 5,    /* P0 */
    BAD_UNREACHED_PARENT = 6, /* P1 */
    BAD_PARENT = 7,         /* P2 */
    BAD_KINDS = 8
};

typedef struct {
    const int64_t* off;
    const int32_t* col;
    const int32_t* dist;
    const int32_t* parent;
    uint8_t* witness;
    uint8_t* entry;
    int64_t n, root, v0, v1;
    int64_t bad[BAD_KINDS];
    int64_t scanned;   /* row pass: entries of the reached rows in [v0, v1) */
    int64_t reached;   /* vertex pass: reached vertices in [v0, v1) */
    int64_t maxd;      /* vertex pass: deepest level in [v0, v1) */
} RowTask;

static void* row_pass(void* arg)
{
    RowTask* t = (RowTask*)arg;
    for (int64_t u = t->v0; u < t->v1; ++u) {
        const int32_t du = t->dist[u];
        if (du < 0) continue;
        t->scanned += t->off[u + 1] - t->off[u];
        for (int64_t e = t->off[u]; e < t->off[u + 1]; ++e) {
            const int32_t v = t->col[e];
            const int32_t dv = t->dist[v];
            if (dv < 0) {
                t->bad[BAD_REACH_GAP] += 1;
            } else if (dv > du + 1) {
                t->bad[BAD_LEVEL_SKIP] += 1;
            } else if (dv == du + 1) {
                __atomic_store_n(&t->witness[v], (uint8_t)1, __ATOMIC_RELAXED);
                if (t->parent && t->parent[v] == (int32_t)u)
                    __atomic_store_n(&t->entry[v], (uint8_t)1, __ATOMIC_RELAXED);
            }
        }
    }
    return NULL;
}

static void* vertex_pass(void* arg)
{
    RowTask* t = (RowTask*)arg;
    const int64_t root = t->root;
    int64_t nreached = 0, maxd = -1;
    for (int64_t x = t->v0; x < t->v1; ++x) {
        const int32_t dx = t->dist[x];
        if (dx < -1) {
            t->bad[BAD_RANGE] += 1;
            continue;
        }
        if (dx < 0) {
            if (t->parent && t->parent[x] != -1) t->bad[BAD_UNREACHED_PARENT] += 1;
            continue;
        }
        nreached += 1;
        if (dx > maxd) maxd = dx;
        if (x == root) continue;
        if (!t->witness[x]) t->bad[BAD_NO_WITNESS] += 1;
        if (t->parent && !t->entry[x]) t->bad[BAD_PARENT] += 1;
    }
    t->reached = nreached;
    t->maxd = maxd;
    return NULL;
}

/* bad: int64[BAD_KINDS] counts (zeroed here).  *reached, *levels (max d + 1)
 * and *scanned (entries of the reached rows) describe d.  Returns the total
 * number of violations, or a negative value on a bad argument or when
 * memory runs out. */
int64_t oracle_check_bfs(int64_t n, const int64_t* off, const int32_t* col, int64_t root,
                         const int32_t* dist, const int32_t* parent, int32_t nthreads,
                         int64_t* bad, int64_t* reached, int64_t* levels, int64_t* scanned)
{
    if (n <= 0 || root < 0 || root >= n || !off || !dist || !bad) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    memset(bad, 0, sizeof(int64_t) * BAD_KINDS);
    uint8_t* witness = (uint8_t*)calloc((size_t)n, 1);
    uint8_t* entry = (uint8_t*)calloc((size_t)n, 1);
    RowTask* tasks = (RowTask*)calloc((size_t)nthreads, sizeof(RowTask));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!witness || !entry || !tasks || !th) {
        free(witness);
        free(entry);
        free(tasks);
        free(th);
        return -2;
    }
    /* row ranges of about equal entry counts (plus one unit per row) */
    const double total = (double)(off[n] - off[0]) + (double)n;
    int64_t v = 0;
    for (int32_t i = 0; i < nthreads; ++i) {
        RowTask* t = &tasks[i];
        t->off = off;
        t->col = col;
        t->dist = dist;
        t->parent = parent;
        t->witness = witness;
        t->entry = entry;
        t->n = n;
        t->root = root;
        t->v0 = v;
        const double goal = total * (double)(i + 1) / (double)nthreads;
        if (i == nthreads - 1) {
            v = n;
        } else {
            while (v < n && (double)(off[v] - off[0]) + (double)v < goal) ++v;
        }
        t->v1 = v;
    }
    for (int32_t i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, row_pass, &tasks[i]);
    for (int32_t i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
    int64_t m = 0;
    for (int32_t i = 0; i < nthreads; ++i) {
        for (int k = 0; k < BAD_KINDS; ++k) bad[k] += tasks[i].bad[k];
        m += tasks[i].scanned;
        memset(tasks[i].bad, 0, sizeof(tasks[i].bad));
    }
    /* vertex pass: equal vertex ranges, each vertex's own checks and marks */
    for (int32_t i = 0; i < nthreads; ++i) {
        tasks[i].v0 = n * (int64_t)i / nthreads;
        tasks[i].v1 = n * (int64_t)(i + 1) / nthreads;
    }
    for (int32_t i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, vertex_pass, &tasks[i]);
    for (int32_t i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
    int64_t nreached = 0, maxd = -1;
    for (int32_t i = 0; i < nthreads; ++i) {
        for (int k = 0; k < BAD_KINDS; ++k) bad[k] += tasks[i].bad[k];
        nreached += tasks[i].reached;
        if (tasks[i].maxd > maxd) maxd = tasks[i].maxd;
    }
    if (dist[root] != 0) bad[BAD_ROOT_DIST] += 1;
    if (parent && parent[root] != (int32_t)root) bad[BAD_ROOT_PARENT] += 1;
    if (reached) *reached = nreached;
    if (levels) *levels = maxd + 1;
    if (scanned) *scanned = m;
    free(witness);
    free(entry);
    free(tasks);
    free(th);
    int64_t sum = 0;
    for (int k = 0; k < BAD_KINDS; ++k) sum += bad[k];
    return sum;
}
