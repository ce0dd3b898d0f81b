// bfs_lrb.cu -- the paper's own per-GPU traversal scheme, for comparison.
//
// Section "Load Balanced Traversals Per compute-node": the frontier is
// grouped by Logarithmic Radix Binning -- bin b holds the vertices whose
// degree lies in [2^(b-1), 2^b), so vertices of one bin differ in degree by
// at most 2x -- and one kernel per non-empty bin is dispatched on its own
// stream, its thread-block shape chosen from the bin's degree bound.  The
// level loop is driven by the host (the paper's host threads orchestrate the
// GPU), which joins the bin streams and reads the next frontier size after
// every level.  The visited test is the paper's own: d[u] = infinity, claimed
// with an atomic compare-and-swap whose success gates the enqueue
// (Algorithm 2 Phase 1).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "bfs_runtime.h"

namespace bfs {
namespace {

constexpr int kLrbBins = 33;  // bin 0: degree 0; bin b >= 1: [2^(b-1), 2^b)

__device__ __forceinline__ int lrb_bin(long long deg) {
    return deg <= 0 ? 0 : min(64 - __clzll((unsigned long long)deg), kLrbBins - 1);
}

__global__ void lrb_count(const int64_t* off, const int32_t* fr, long long nfr,
                          unsigned long long* counts) {
    __shared__ unsigned s[kLrbBins];
    for (int i = threadIdx.x; i < kLrbBins; i += blockDim.x) s[i] = 0;
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nfr; i += stride) {
        const int32_t v = fr[i];
        atomicAdd(&s[lrb_bin(off[v + 1] - off[v])], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kLrbBins; i += blockDim.x)
        if (s[i]) atomicAdd(&counts[i], (unsigned long long)s[i]);
}

__global__ void lrb_scatter(const int64_t* off, const int32_t* fr, long long nfr,
                            unsigned long long* cursor, int32_t* binned) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nfr; i += stride) {
        const int32_t v = fr[i];
        const int b = lrb_bin(off[v + 1] - off[v]);
        binned[atomicAdd(&cursor[b], 1ull)] = v;
    }
}

__device__ __forceinline__ void lrb_visit(bool ok, int32_t u, int level, int32_t* d,
                                          int32_t* next, unsigned long long* tail) {
    bool win = false;
    if (ok && d[u] == -1) win = atomicCAS(d + u, -1, level + 1) == -1;
    const unsigned m = __ballot_sync(0xffffffffu, win);
    if (!m) return;
    unsigned lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    const int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if ((int)(threadIdx.x & 31) == leader) base = atomicAdd(tail, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (win) next[base + __popc(m & lt)] = u;
}

// Small bins: one thread per vertex.
__global__ void lrb_thread(const int64_t* off, const int32_t* col, const int32_t* vs, long long cnt,
                           int bound, int level, int32_t* d, int32_t* next, unsigned long long* tail) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = i < cnt;
    const int32_t v = ok ? vs[i] : 0;
    const long long b = ok ? off[v] : 0, deg = ok ? off[v + 1] - b : 0;
    for (int k = 0; k < bound; ++k)  // warp-uniform trip count: the bin's degree bound
        lrb_visit(k < deg, k < deg ? col[b + k] : 0, level, d, next, tail);
}

// Medium bins: one warp per vertex.
__global__ void lrb_warp(const int64_t* off, const int32_t* col, const int32_t* vs, long long cnt,
                         int level, int32_t* d, int32_t* next, unsigned long long* tail) {
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= cnt) return;
    const int32_t v = vs[w];
    const long long b = off[v], e = off[v + 1];
    for (long long k0 = b; k0 < e; k0 += 32)
        lrb_visit(k0 + lane < e, k0 + lane < e ? col[k0 + lane] : 0, level, d, next, tail);
}

// Large bins: one thread block per vertex, blockDim from the bin's bound.
__global__ void lrb_block(const int64_t* off, const int32_t* col, const int32_t* vs, int level,
                          int32_t* d, int32_t* next, unsigned long long* tail) {
    const int32_t v = vs[blockIdx.x];
    const long long b = off[v], e = off[v + 1];
    const long long span = (e - b + blockDim.x - 1) / blockDim.x * blockDim.x;
    for (long long k = threadIdx.x; k < span; k += blockDim.x)
        lrb_visit(b + k < e, b + k < e ? col[b + k] : 0, level, d, next, tail);
}

__global__ void lrb_init(int32_t* d, long long n, int32_t root, int32_t* fr) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        d[i] = i == root ? 0 : -1;
    if (blockIdx.x == 0 && threadIdx.x == 0) fr[0] = root;
}

__global__ void lrb_output(const int32_t* d, long long n, const int32_t* new2old, int32_t* dist) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        dist[new2old ? new2old[v] : v] = d[v];
}

}  // namespace
}  // namespace bfs

using namespace bfs;

extern "C" bfs_status bfs_run_lrb(bfs_graph* g, int32_t root, int32_t* dist, void* stream,
                                  bfs_lrb_stats* stats) {
    TraceRange tr("bfs_run_lrb", root);
    if (!g || !dist) {
        set_error("lrb: null graph or dist");
        return BFS_ERR_INVALID_ARG;
    }
    if (root < 0 || root >= g->n) {
        set_error("lrb: root out of range");
        return BFS_ERR_ROOT_RANGE;
    }
    cudaError_t e = cudaSetDevice(g->ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long n = g->n;
    const int sms = g->ctx->sms;
    DeviceAllocator* m = g->ctx->mem;
    int32_t* d = static_cast<int32_t*>(m->alloc((size_t)n * 4));
    int32_t* fr[2] = {static_cast<int32_t*>(m->alloc((size_t)n * 4 + 64)),
                      static_cast<int32_t*>(m->alloc((size_t)n * 4 + 64))};
    int32_t* binned = static_cast<int32_t*>(m->alloc((size_t)n * 4 + 64));
    unsigned long long* cnt = static_cast<unsigned long long*>(m->alloc(3 * kLrbBins * 8 + 64));
    std::vector<cudaStream_t> bs(kLrbBins, nullptr);
    std::vector<cudaEvent_t> ev(kLrbBins + 1, nullptr);
    auto release = [&]() {
        for (auto x : bs)
            if (x) cudaStreamDestroy(x);
        for (auto x : ev)
            if (x) cudaEventDestroy(x);
        m->release(d);
        m->release(fr[0]);
        m->release(fr[1]);
        m->release(binned);
        m->release(cnt);
    };
    if (!d || !fr[0] || !fr[1] || !binned || !cnt) {
        release();
        set_error("lrb: device memory exhausted");
        return BFS_ERR_NO_MEMORY;
    }
    for (int b = 0; b < kLrbBins && e == cudaSuccess; ++b) {
        e = cudaStreamCreateWithFlags(&bs[b], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[b], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[kLrbBins], cudaEventDisableTiming);
    int32_t dev_root = root;
    if (e == cudaSuccess && g->relabelled)
        e = cudaMemcpy(&dev_root, g->d_old2new + root, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        release();
        return cuda_fail(e, "lrb set-up");
    }
    unsigned long long* bin_cnt = cnt;               // [33]
    unsigned long long* cursor = cnt + kLrbBins;     // [33]
    unsigned long long* tail = cnt + 2 * kLrbBins;   // next frontier size
    lrb_init<<<sms * 4, 256, 0, s>>>(d, n, dev_root, fr[0]);
    bfs_lrb_stats st{};
    long long nfr = 1;
    int cur = 0;
    for (int level = 0; nfr > 0 && e == cudaSuccess; ++level) {
        TraceRange lv("level", level);
        st.levels = level + 1;
        // bin the frontier by log2(degree)
        e = cudaMemsetAsync(cnt, 0, 3 * kLrbBins * 8, s);
        const int gb = (int)std::min<long long>(sms * 4, (nfr + 255) / 256);
        lrb_count<<<gb, 256, 0, s>>>(g->d_off, fr[cur], nfr, bin_cnt);
        unsigned long long h[kLrbBins];
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, bin_cnt, sizeof(h), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        unsigned long long start[kLrbBins], acc = 0;
        for (int b = 0; b < kLrbBins; ++b) {
            start[b] = acc;
            acc += h[b];
        }
        e = cudaMemcpyAsync(cursor, start, sizeof(start), cudaMemcpyHostToDevice, s);
        lrb_scatter<<<gb, 256, 0, s>>>(g->d_off, fr[cur], nfr, cursor, binned);
        if (e == cudaSuccess) e = cudaEventRecord(ev[kLrbBins], s);
        // one kernel per non-empty bin, each on its own stream
        for (int b = 1; b < kLrbBins && e == cudaSuccess; ++b) {
            if (h[b] == 0) continue;
            e = cudaStreamWaitEvent(bs[b], ev[kLrbBins], 0);
            const long long c = (long long)h[b];
            const int32_t* vs = binned + start[b];
            const int bound = 1 << std::min(b, 30);  // the bin's degrees are below 2^b
            if (b <= 5) {           // degree < 32: one thread per vertex
                lrb_thread<<<(unsigned)((c + 255) / 256), 256, 0, bs[b]>>>(
                    g->d_off, g->d_col, vs, c, bound, level, d, fr[cur ^ 1], tail);
            } else if (b <= 10) {   // degree < 1024: one warp per vertex
                lrb_warp<<<(unsigned)((c * 32 + 255) / 256), 256, 0, bs[b]>>>(
                    g->d_off, g->d_col, vs, c, level, d, fr[cur ^ 1], tail);
            } else {                // one block per vertex, up to 1024 threads
                const int threads = std::min(1024, 1 << std::min(b - 1, 10));
                lrb_block<<<(unsigned)c, threads, 0, bs[b]>>>(g->d_off, g->d_col, vs, level, d,
                                                             fr[cur ^ 1], tail);
            }
            st.kernels += 1;
            if (e == cudaSuccess) e = cudaEventRecord(ev[b], bs[b]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[b], 0);
        }
        if (e == cudaSuccess) e = cudaGetLastError();
        unsigned long long hn = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hn, tail, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        nfr = (long long)hn;
        cur ^= 1;
    }
    if (e == cudaSuccess) {
        lrb_output<<<sms * 4, 256, 0, s>>>(d, n, g->relabelled ? g->d_new2old : nullptr, dist);
        e = cudaStreamSynchronize(s);
    }
    release();
    if (e != cudaSuccess) return cuda_fail(e, "lrb traversal");
    if (stats) *stats = st;
    return BFS_OK;
}
