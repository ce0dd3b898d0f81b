// bfs_tune.cpp -- per-graph autotuner for the degree-bin thresholds, base
// chunk sizes and resident CTAs per SM.
//
// Coordinate descent from the current setting: one knob at a time is swept
// over a short candidate list while the others stay fixed, each candidate
// timed by CUDA events over the caller's sample roots (single-source or one
// batched launch, as asked), the best kept.  Results can be cached in a JSON
// file keyed by a fingerprint of the graph (vertex and entry counts and a
// hash of sampled row offsets and columns), so a graph seen before is set up
// without timing.
#include <cuda_runtime.h>

#include <algorithm>
#include <cinttypes>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "bfs_runtime.h"

namespace bfs {
namespace {

struct Knobs {
    int32_t t_small, t_large, chunk_warp, chunk_cta, ctas;
};

uint64_t mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

bfs_status fingerprint(bfs_graph* g, uint64_t* out) {
    const int kSamples = 256;
    std::vector<int64_t> offs(kSamples);
    std::vector<int32_t> cols(kSamples);
    uint64_t h = mix((uint64_t)g->n * 0x9E3779B97F4A7C15ull ^ (uint64_t)g->nnz);
    for (int i = 0; i < kSamples; ++i) {
        const int64_t v = (int64_t)((double)i / kSamples * (double)g->n);
        cudaError_t e = cudaMemcpy(&offs[i], g->d_off + v, 8, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && g->nnz > 0) {
            const int64_t k = (int64_t)((double)i / kSamples * (double)g->nnz);
            e = cudaMemcpy(&cols[i], g->d_col + k, 4, cudaMemcpyDeviceToHost);
        } else {
            cols[i] = 0;
        }
        if (e != cudaSuccess) return cuda_fail(e, "autotune fingerprint");
        h = mix(h ^ (uint64_t)offs[i]) ^ mix((uint64_t)(uint32_t)cols[i] + (uint64_t)i);
    }
    *out = h;
    return BFS_OK;
}

bool cache_lookup(const char* path, uint64_t fp, uint32_t flags, Knobs* k) {
    if (!path) return false;
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        unsigned long long key = 0;
        unsigned fl = 0;
        Knobs c{};
        if (std::sscanf(line,
                        " {\"fingerprint\": \"%llx\", \"flags\": %u, \"t_small\": %d, \"t_large\": %d, "
                        "\"chunk_warp\": %d, \"chunk_cta\": %d, \"ctas_per_sm\": %d",
                        &key, &fl, &c.t_small, &c.t_large, &c.chunk_warp, &c.chunk_cta,
                        &c.ctas) == 7 &&
            key == fp && fl == flags) {
            *k = c;
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

void cache_store(const char* path, uint64_t fp, uint32_t flags, const Knobs& k, double ms) {
    if (!path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f,
                 "{\"fingerprint\": \"%016" PRIx64 "\", \"flags\": %u, \"t_small\": %d, \"t_large\": %d, "
                 "\"chunk_warp\": %d, \"chunk_cta\": %d, \"ctas_per_sm\": %d, \"ms\": %.4f}\n",
                 fp, flags, k.t_small, k.t_large, k.chunk_warp, k.chunk_cta, k.ctas, ms);
    std::fclose(f);
}

bfs_status apply(bfs_graph* g, const Knobs& k) {
    bfs_status st = bfs_graph_set_bins(g, k.t_small, k.t_large, k.chunk_warp, k.chunk_cta);
    if (st == BFS_OK) st = bfs_graph_set_option(g, BFS_OPT_CTAS_PER_SM, k.ctas);
    return st;
}

}  // namespace
}  // namespace bfs

using namespace bfs;

extern "C" bfs_status bfs_graph_autotune(bfs_graph* g, const int32_t* roots, int32_t nroots,
                                         uint32_t flags, const char* cache_path,
                                         bfs_tune_result* out) {
    bfs::TraceRange tr("bfs_graph_autotune", nroots);
    if (!g || !roots || nroots < 1 || nroots > 64) {
        set_error("autotune: need a graph and 1..64 sample roots");
        return BFS_ERR_INVALID_ARG;
    }
    if (flags & ~(uint32_t)BFS_TUNE_BATCHED) {
        set_error("autotune: unknown flag");
        return BFS_ERR_INVALID_ARG;
    }
    for (int i = 0; i < nroots; ++i)
        if (roots[i] < 0 || roots[i] >= g->n) {
            set_error("autotune: root out of range");
            return BFS_ERR_ROOT_RANGE;
        }
    cudaError_t e = cudaSetDevice(g->ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    uint64_t fp = 0;
    bfs_status st = fingerprint(g, &fp);
    if (st != BFS_OK) return st;
    Knobs best{g->t_small, g->t_large, g->chunk_warp, g->chunk_cta, g->min_blocks};
    if (cache_lookup(cache_path, fp, flags, &best)) {
        st = apply(g, best);
        if (st != BFS_OK) return st;
        if (out) {
            *out = bfs_tune_result{best.t_small, best.t_large, best.chunk_warp, best.chunk_cta,
                                   best.ctas, 1, 0, -1.0, fp};
        }
        return BFS_OK;
    }
    const bool batched = (flags & BFS_TUNE_BATCHED) != 0;
    cudaStream_t s = nullptr;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "autotune stream");
    void* d_out = nullptr;
    size_t out_bytes = (size_t)g->n * 4 * (batched ? (size_t)nroots : 2);
    d_out = g->ctx->mem->alloc(out_bytes);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int trials = 0;
    auto measure = [&](const Knobs& k, double* ms) -> bfs_status {
        bfs_status r = apply(g, k);
        if (r != BFS_OK) return r;
        int32_t* dist = static_cast<int32_t*>(d_out);
        int32_t* parent = batched ? nullptr : dist + g->n;
        auto once = [&]() -> bfs_status {
            if (batched) return bfs_run_batch(g, roots, nroots, dist, s, 0);
            for (int i = 0; i < nroots; ++i) {
                bfs_status q = bfs_run(g, roots[i], dist, parent, s, 0);
                if (q != BFS_OK) return q;
            }
            return BFS_OK;
        };
        if ((r = once()) != BFS_OK) return r;  // warm-up
        float best_ms = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, s);
            if ((r = once()) != BFS_OK) return r;
            cudaEventRecord(e1, s);
            cudaError_t ee = cudaEventSynchronize(e1);
            if (ee != cudaSuccess) return cuda_fail(ee, "autotune timing");
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            best_ms = std::min(best_ms, t);
        }
        bfs_run_stats rs;
        r = batched ? bfs_batch_sync(g, s, &rs) : bfs_graph_sync(g, s, &rs);
        if (r != BFS_OK) return r;
        ++trials;
        *ms = best_ms;
        return BFS_OK;
    };
    double best_ms = 0.0;
    if (!d_out) {
        st = BFS_ERR_NO_MEMORY;
        set_error("autotune: device memory exhausted (output buffers)");
    } else {
        st = measure(best, &best_ms);
    }
    const double start_ms = best_ms;
    // coordinate descent, one knob at a time
    const std::vector<int32_t> c_small = {8, 16, 32, 64, 128};
    const std::vector<int32_t> c_large = {1024, 2048, 4096, 8192, 16384};
    const std::vector<std::pair<int32_t, int32_t>> c_chunks = {{256, 1024}, {512, 2048}, {1024, 4096}};
    const std::vector<int32_t> c_ctas = {2, 3, 4};
    for (int pass = 0; pass < 2 && st == BFS_OK; ++pass) {
        for (int32_t v : c_small) {
            if (st != BFS_OK || v == best.t_small || v >= best.t_large) continue;
            Knobs k = best;
            k.t_small = v;
            double ms;
            st = measure(k, &ms);
            if (st == BFS_OK && ms < best_ms) best = k, best_ms = ms;
        }
        for (int32_t v : c_large) {
            if (st != BFS_OK || v == best.t_large || v <= best.t_small) continue;
            Knobs k = best;
            k.t_large = v;
            double ms;
            st = measure(k, &ms);
            if (st == BFS_OK && ms < best_ms) best = k, best_ms = ms;
        }
        for (auto c : c_chunks) {
            if (st != BFS_OK || (c.first == best.chunk_warp && c.second == best.chunk_cta)) continue;
            Knobs k = best;
            k.chunk_warp = c.first;
            k.chunk_cta = c.second;
            double ms;
            st = measure(k, &ms);
            if (st == BFS_OK && ms < best_ms) best = k, best_ms = ms;
        }
        for (int32_t v : c_ctas) {
            if (st != BFS_OK || v == best.ctas) continue;
            Knobs k = best;
            k.ctas = v;
            double ms;
            st = measure(k, &ms);
            if (st == BFS_OK && ms < best_ms) best = k, best_ms = ms;
        }
    }
    if (st == BFS_OK) st = apply(g, best);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    g->ctx->mem->release(d_out);
    if (st != BFS_OK) return st;
    cache_store(cache_path, fp, flags, best, best_ms);
    if (out)
        *out = bfs_tune_result{best.t_small, best.t_large, best.chunk_warp, best.chunk_cta,
                               best.ctas, 0, trials, best_ms, fp};
    (void)start_ms;
    return BFS_OK;
}
