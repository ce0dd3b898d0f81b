/*
 * graphgen.c -- seeded synthetic graph generators (Kronecker/R-MAT and
 * Erdos-Renyi) producing an undirected, self-loop-free, duplicate-free CSR
 * with int64 row offsets and int32 column indices.
 *
 * This module holds input generation only; it contains none of the BFS
 * arithmetic.  Both the CPU oracle (through the tests) and the GPU library
 * (through the tests and the benchmark) consume the CSR it writes.
 *
 * Randomness is counter based: every draw is SplitMix64 (Steele, Lea and
 * Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014)
 * applied to (key + (index + 1) * golden_gamma), so edge e's bits do not
 * depend on how the work is split across threads, and a regeneration pass
 * reproduces the same edge list without storing it.
 *
 * R-MAT (Chakrabarti, Zhan and Faloutsos, SDM 2004): for each generated edge
 * and each of the `scale` bit levels, one uniform draw picks a quadrant of the
 * adjacency matrix with probabilities A, B, C, D = 1-A-B-C; no noise is added.
 * Vertex ids are then relabelled by a seeded pseudo-random permutation of
 * [0, 2^scale): a 6-round balanced Feistel network on 2*ceil(scale/2) bits,
 * cycle-walked back into range when scale is odd (Luby-Rackoff construction).
 *
 * Cleanup (the paper's input conversion, Section "Inputs"): self-loops
 * dropped, both directions added, each row sorted and deduplicated.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

#define GG_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t gg_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* draw number `idx` of the stream keyed by `key` */
static inline uint64_t gg_draw(uint64_t key, uint64_t idx)
{
    return gg_mix64(key + (idx + 1ULL) * GG_GAMMA);
}

/* stream keys: one per purpose, derived from the user seed */
static inline uint64_t gg_key(uint64_t seed, uint64_t stream)
{
    return gg_mix64(seed * 0xD1B54A32D192ED03ULL + gg_mix64(stream + 0x632BE59BD9B4E019ULL));
}

enum { GG_STREAM_EDGES = 1, GG_STREAM_PERM = 2, GG_STREAM_ROOTS = 3 };
enum { GG_KIND_RMAT = 0, GG_KIND_UNIFORM = 1 };

uint64_t gg_splitmix64_draw(uint64_t seed, uint64_t stream, uint64_t idx)
{
    return gg_draw(gg_key(seed, stream), idx);
}

/* uniform double in [0,1) from the top 53 bits */
static inline double gg_u01(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

typedef struct {
    int scale;
    int kind;
    int permute;
    int64_t nedges;
    double a, ab, abc;
    uint64_t key_edges;
    uint64_t perm_keys[6];
    int half_bits;
} gg_params;

static void gg_setup(gg_params* p, int scale, int64_t nedges, double A, double B, double C,
                     uint64_t seed, int kind, int permute)
{
    p->scale = scale;
    p->kind = kind;
    p->permute = permute;
    p->nedges = nedges;
    p->a = A;
    p->ab = A + B;
    p->abc = A + B + C;
    p->key_edges = gg_key(seed, GG_STREAM_EDGES);
    uint64_t kp = gg_key(seed, GG_STREAM_PERM);
    for (int r = 0; r < 6; ++r) p->perm_keys[r] = gg_draw(kp, (uint64_t)r);
    p->half_bits = (scale + 1) / 2;
}

/* seeded pseudo-random permutation of [0, 2^scale) */
static inline uint64_t gg_permute(const gg_params* p, uint64_t x)
{
    if (!p->permute || p->scale == 0) return x;
    const int h = p->half_bits;
    const uint64_t mask = (1ULL << h) - 1ULL;
    const uint64_t n = 1ULL << p->scale;
    do {
        uint64_t L = x >> h, R = x & mask;
        for (int r = 0; r < 6; ++r) {
            uint64_t F = gg_mix64(R ^ p->perm_keys[r]) & mask;
            uint64_t nl = R;
            R = L ^ F;
            L = nl;
        }
        x = (L << h) | R;
    } while (x >= n); /* cycle-walk: only possible when scale is odd */
    return x;
}

/* generated edge e (before cleanup), endpoints after permutation */
static inline void gg_edge(const gg_params* p, int64_t e, uint64_t* src, uint64_t* dst)
{
    uint64_t s = 0, d = 0;
    if (p->kind == GG_KIND_RMAT) {
        const uint64_t base = (uint64_t)e * (uint64_t)p->scale;
        for (int j = 0; j < p->scale; ++j) {
            double u = gg_u01(gg_draw(p->key_edges, base + (uint64_t)j));
            uint64_t bs, bd;
            if (u < p->a) { bs = 0; bd = 0; }
            else if (u < p->ab) { bs = 0; bd = 1; }
            else if (u < p->abc) { bs = 1; bd = 0; }
            else { bs = 1; bd = 1; }
            s |= bs << j;
            d |= bd << j;
        }
    } else {
        const uint64_t nmask = (p->scale >= 64) ? ~0ULL : ((1ULL << p->scale) - 1ULL);
        s = gg_draw(p->key_edges, 2ULL * (uint64_t)e) & nmask;
        d = gg_draw(p->key_edges, 2ULL * (uint64_t)e + 1ULL) & nmask;
    }
    *src = gg_permute(p, s);
    *dst = gg_permute(p, d);
}

/* Raw generated edge list (before permutation-independent cleanup), for
 * generator tests on small inputs.  src/dst are written for e in [0, nedges). */
int gg_edges_raw(int scale, int64_t nedges, double A, double B, double C, uint64_t seed,
                 int kind, int permute, int32_t* src, int32_t* dst)
{
    gg_params p;
    if (scale < 0 || scale > 31 || nedges < 0) return -1;
    gg_setup(&p, scale, nedges, A, B, C, seed, kind, permute);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < nedges; ++e) {
        uint64_t s, d;
        gg_edge(&p, e, &s, &d);
        src[e] = (int32_t)s;
        dst[e] = (int32_t)d;
    }
    return 0;
}

/* Pass 1: per-vertex count of directed entries before dedup (self-loops
 * dropped, both directions counted).  deg must hold 2^scale zeros. */
int gg_count(int scale, int64_t nedges, double A, double B, double C, uint64_t seed,
             int kind, int permute, int64_t* deg)
{
    gg_params p;
    if (scale < 0 || scale > 31 || nedges < 0) return -1;
    gg_setup(&p, scale, nedges, A, B, C, seed, kind, permute);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < nedges; ++e) {
        uint64_t s, d;
        gg_edge(&p, e, &s, &d);
        if (s == d) continue;
        __atomic_fetch_add(&deg[s], 1, __ATOMIC_RELAXED);
        __atomic_fetch_add(&deg[d], 1, __ATOMIC_RELAXED);
    }
    return 0;
}

static int gg_cmp_i32(const void* x, const void* y)
{
    int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
    return (a > b) - (a < b);
}

/* Pass 2: regenerate, scatter into rows laid out by off_tmp (the exclusive
 * prefix of pass 1's counts), sort and deduplicate each row, and compact the
 * rows in place to the front of col.  off_out (N+1 entries) receives the
 * final offsets; off_out[N] is the final number of directed entries.
 * cursor is scratch of N int64. */
int gg_fill(int scale, int64_t nedges, double A, double B, double C, uint64_t seed,
            int kind, int permute, const int64_t* off_tmp, int64_t* cursor, int32_t* col,
            int64_t* off_out)
{
    gg_params p;
    if (scale < 0 || scale > 31 || nedges < 0) return -1;
    gg_setup(&p, scale, nedges, A, B, C, seed, kind, permute);
    const int64_t n = (int64_t)1 << scale;
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v) cursor[v] = off_tmp[v];
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < nedges; ++e) {
        uint64_t s, d;
        gg_edge(&p, e, &s, &d);
        if (s == d) continue;
        int64_t ps = __atomic_fetch_add(&cursor[s], 1, __ATOMIC_RELAXED);
        int64_t pd = __atomic_fetch_add(&cursor[d], 1, __ATOMIC_RELAXED);
        col[ps] = (int32_t)d;
        col[pd] = (int32_t)s;
    }
    /* sort + dedup each row; cursor[v] becomes the deduplicated degree */
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t v = 0; v < n; ++v) {
        int64_t b = off_tmp[v], e = off_tmp[v + 1];
        int64_t len = e - b;
        if (len > 1) qsort(col + b, (size_t)len, sizeof(int32_t), gg_cmp_i32);
        int64_t w = 0;
        for (int64_t i = 0; i < len; ++i)
            if (w == 0 || col[b + i] != col[b + w - 1]) col[b + w++] = col[b + i];
        cursor[v] = w;
    }
    off_out[0] = 0;
    for (int64_t v = 0; v < n; ++v) off_out[v + 1] = off_out[v] + cursor[v];
    /* in-order compaction is safe: off_out[v] <= off_tmp[v] and
     * off_out[v+1] <= off_tmp[v+1], so row v never overwrites a later row */
    for (int64_t v = 0; v < n; ++v)
        if (cursor[v] > 0 && off_out[v] != off_tmp[v])
            memmove(col + off_out[v], col + off_tmp[v], (size_t)cursor[v] * sizeof(int32_t));
    return 0;
}

int gg_num_threads(void) { return omp_get_max_threads(); }
