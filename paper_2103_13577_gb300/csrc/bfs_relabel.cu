// bfs_relabel.cu -- degree-ordered renumbering of an uploaded graph.
//
// Vertices are ordered by logarithmic degree bucket, heaviest first (bucket
// = floor(log2 deg) + 1, 0 for isolated vertices: the same log2 classes as
// the paper's Logarithmic Radix Binning, used here for layout), stable by
// the caller's id inside a bucket.  Hubs then get the smallest ids, so the
// visited-bitmap words, row offsets and distances that most edges touch
// sit together at the front of each array.  Results are always written in
// the caller's numbering (new2old on every dist/parent write).
//
// Steps (all on the device):
//   1. per tile of 1024 vertices, count vertices per bucket
//   2. exclusive scan of the bucket-major count table -> tile offsets
//   3. stable scatter: new2old[pos] = v, old2new[v] = pos
//   4. new offsets = exclusive scan of deg[new2old[i]]
//   5. new columns: row of new2old[i] copied with old2new applied, heavy
//      neighbours first
#include <cuda_runtime.h>

#include <cstdint>

#include "bfs_internal.h"

namespace bfs {

constexpr int kRelTile = 1024;
constexpr int kRelThreads = 256;
constexpr int kBuckets = 33;  // deg 0, [1,2), [2,4), ..., [2^31, ...)

__device__ __forceinline__ int rel_key(long long deg) {
    // ascending key = descending degree bucket
    const int bucket = deg <= 0 ? 0 : 64 - __clzll((unsigned long long)deg);  // floor(log2)+1
    return (kBuckets - 1) - min(bucket, kBuckets - 1);
}

__global__ void rel_count_kernel(const int64_t* off, long long n, long long ntiles,
                                 unsigned long long* counts) {
    __shared__ unsigned s_cnt[kBuckets];
    for (int i = threadIdx.x; i < kBuckets; i += blockDim.x) s_cnt[i] = 0;
    __syncthreads();
    const long long t = blockIdx.x;
    for (int k = threadIdx.x; k < kRelTile; k += blockDim.x) {
        const long long v = t * kRelTile + k;
        if (v < n) atomicAdd(&s_cnt[rel_key(off[v + 1] - off[v])], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kBuckets; i += blockDim.x) counts[(long long)i * ntiles + t] = s_cnt[i];
}

// Stable scatter of one tile: sub-batches of 256 vertices in order; inside a
// sub-batch, warps in order; inside a warp, lanes in order.
__global__ void rel_scatter_kernel(const int64_t* off, long long n, long long ntiles,
                                   const unsigned long long* offsets, int32_t* new2old,
                                   int32_t* old2new) {
    __shared__ unsigned long long s_base[kBuckets];
    __shared__ unsigned s_warp[kRelThreads / 32][kBuckets];
    const long long t = blockIdx.x;
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kBuckets; i += blockDim.x) s_base[i] = offsets[(long long)i * ntiles + t];
    __syncthreads();
    for (int sub = 0; sub < kRelTile; sub += kRelThreads) {
        const long long v = t * kRelTile + sub + threadIdx.x;
        const bool ok = v < n;
        const int key = ok ? rel_key(off[v + 1] - off[v]) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        unsigned lt;
        asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
        const int rank_in_warp = __popc(peers & lt);
        for (int i = threadIdx.x; i < (kRelThreads / 32) * kBuckets; i += blockDim.x)
            (&s_warp[0][0])[i] = 0;
        __syncthreads();
        if (ok && rank_in_warp == 0) s_warp[warp][key] = __popc(peers);
        __syncthreads();
        if (ok) {
            unsigned before = 0;
            for (int w = 0; w < warp; ++w) before += s_warp[w][key];
            const long long pos = (long long)s_base[key] + before + rank_in_warp;
            new2old[pos] = (int32_t)v;
            old2new[v] = (int32_t)pos;
        }
        __syncthreads();
        if (threadIdx.x < kBuckets) {
            unsigned tot = 0;
            for (int w = 0; w < kRelThreads / 32; ++w) tot += s_warp[w][threadIdx.x];
            s_base[threadIdx.x] += tot;
        }
        __syncthreads();
    }
}

__global__ void rel_newdeg_kernel(const int64_t* off, const int32_t* new2old, long long n,
                                  int64_t* out) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int32_t o = new2old[i];
        out[i] = off[o + 1] - off[o];
    }
}

// One warp per new row; columns renamed through old2new and each row
// stably partitioned into three groups by the new id of the neighbour:
// vertices of degree >= 256, of degree >= 16, and the rest (new ids are in
// decreasing degree-bucket order, so the groups are id ranges [0, h1),
// [h1, h2), [h2, n)).  A bottom-up level checks neighbours in row order, and
// the heavy neighbours first are the ones most likely in the frontier.
__global__ void rel_columns_kernel(const int64_t* off, const int32_t* col, const int32_t* new2old,
                                   const int32_t* old2new, const int64_t* new_off, long long n,
                                   const unsigned long long* key_start, long long ntiles,
                                   int32_t* new_col) {
    // key = 32 - bucket, bucket = floor(log2 deg) + 1: deg >= 256 <=> key <= 23
#ifdef BFS_NO_ROW_PARTITION
    const long long h1 = n, h2 = n;
#else
    const long long h1 = (long long)key_start[24ll * ntiles];
    const long long h2 = (long long)key_start[28ll * ntiles];
#endif
    const long long nwarps = (long long)gridDim.x * (blockDim.x / 32);
    const int lane = threadIdx.x & 31;
    unsigned lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    for (long long i = (long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); i < n;
         i += nwarps) {
        const int32_t o = new2old[i];
        const long long b = off[o], d = off[o + 1] - b, nb = new_off[i];
        long long c0 = 0, c1 = 0;
        for (long long k0 = 0; k0 < d; k0 += 32) {
            const long long k = k0 + lane;
            const int32_t x = k < d ? old2new[col[b + k]] : 0;
            c0 += __popc(__ballot_sync(0xffffffffu, k < d && x < h1));
            c1 += __popc(__ballot_sync(0xffffffffu, k < d && x >= h1 && x < h2));
        }
        long long w0 = nb, w1 = nb + c0, w2 = nb + c0 + c1;
        for (long long k0 = 0; k0 < d; k0 += 32) {
            const long long k = k0 + lane;
            const int32_t x = k < d ? old2new[col[b + k]] : 0;
            const int g = k >= d ? -1 : (x < h1 ? 0 : (x < h2 ? 1 : 2));
            const unsigned m0 = __ballot_sync(0xffffffffu, g == 0);
            const unsigned m1 = __ballot_sync(0xffffffffu, g == 1);
            const unsigned m2 = __ballot_sync(0xffffffffu, g == 2);
            if (g == 0) new_col[w0 + __popc(m0 & lt)] = x;
            if (g == 1) new_col[w1 + __popc(m1 & lt)] = x;
            if (g == 2) new_col[w2 + __popc(m2 & lt)] = x;
            w0 += __popc(m0);
            w1 += __popc(m1);
            w2 += __popc(m2);
        }
    }
}

// ---------------------------------------------------- exclusive scan (int64)
// Three passes: per-block sums, scan of the block sums in one block, then
// each block scans its segment and adds its base.  out may alias in.
constexpr int kScanThreads = 512;
constexpr int kScanPerThread = 8;
constexpr long long kScanBlock = (long long)kScanThreads * kScanPerThread;

__device__ __forceinline__ long long block_excl_scan(long long x, long long* total) {
    __shared__ long long s_w[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long incl = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < kScanThreads / 32 ? s_w[lane] : 0;
        long long wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += y;
        }
        if (lane < kScanThreads / 32) s_w[lane] = wi - w;
        if (lane == kScanThreads / 32 - 1) *total = wi;
    }
    __syncthreads();
    const long long r = s_w[warp] + incl - x;
    __syncthreads();
    return r;
}

__global__ void scan_block_sums(const int64_t* in, long long n, int64_t* sums) {
    __shared__ long long s_tot;
    const long long base = (long long)blockIdx.x * kScanBlock + (long long)threadIdx.x * kScanPerThread;
    long long acc = 0;
    for (int k = 0; k < kScanPerThread; ++k)
        if (base + k < n) acc += in[base + k];
    block_excl_scan(acc, &s_tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = s_tot;
}

__global__ void scan_sums_single(int64_t* sums, long long nblocks) {
    __shared__ long long s_tot;
    long long carry = 0;
    for (long long start = 0; start < nblocks; start += kScanThreads) {
        const long long i = start + threadIdx.x;
        const long long x = i < nblocks ? sums[i] : 0;
        const long long ex = block_excl_scan(x, &s_tot);
        if (i < nblocks) sums[i] = carry + ex;
        __syncthreads();
        carry += s_tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[nblocks] = carry;
}

__global__ void scan_apply(const int64_t* in, long long n, const int64_t* sums, int64_t* out) {
    __shared__ long long s_tot;
    const long long base = (long long)blockIdx.x * kScanBlock + (long long)threadIdx.x * kScanPerThread;
    long long v[kScanPerThread];
    long long acc = 0;
    for (int k = 0; k < kScanPerThread; ++k) {
        v[k] = base + k < n ? in[base + k] : 0;
        acc += v[k];
    }
    long long run = block_excl_scan(acc, &s_tot) + sums[blockIdx.x];
    for (int k = 0; k < kScanPerThread; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

// Exclusive scan of n int64 values; out[n] receives the total.  tmp needs
// ceil(n / 4096) + 1 int64.
cudaError_t exclusive_scan_i64(const int64_t* in, long long n, int64_t* out, int64_t* tmp,
                               cudaStream_t s) {
    const long long nb = (n + kScanBlock - 1) / kScanBlock;
    if (nb > 0) {
        scan_block_sums<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, tmp);
        scan_sums_single<<<1, kScanThreads, 0, s>>>(tmp, nb);
        scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, tmp, out);
    } else {
        cudaMemsetAsync(tmp, 0, sizeof(int64_t), s);
    }
    // out[n] = total
    return cudaMemcpyAsync(out + n, tmp + nb, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
}

// Scratch sizes (bytes) the relabel needs beyond the new graph arrays.
size_t relabel_scratch_bytes(long long n) {
    const long long ntiles = (n + kRelTile - 1) / kRelTile;
    const long long table = (long long)kBuckets * ntiles;
    const long long big = table > n ? table : n;
    return (size_t)(2 * (big + 1) * 8 + ((big + kScanBlock - 1) / kScanBlock + 2) * 8) + 1024;
}

// Builds new2old/old2new and the renumbered CSR (new_off[n+1], new_col[nnz]).
cudaError_t relabel_graph(const int64_t* off, const int32_t* col, long long n, long long nnz,
                          int sms, int32_t* new2old, int32_t* old2new, int64_t* new_off,
                          int32_t* new_col, void* scratch, cudaStream_t s) {
    const long long ntiles = (n + kRelTile - 1) / kRelTile;
    const long long table = (long long)kBuckets * ntiles;
    const long long big = table > n ? table : n;
    int64_t* a = static_cast<int64_t*>(scratch);
    int64_t* b = a + big + 1;
    int64_t* tmp = b + big + 1;
    rel_count_kernel<<<(unsigned)ntiles, kRelThreads, 0, s>>>(off, n, ntiles,
                                                               reinterpret_cast<unsigned long long*>(a));
    cudaError_t e = exclusive_scan_i64(a, table, b, tmp, s);
    if (e != cudaSuccess) return e;
    rel_scatter_kernel<<<(unsigned)ntiles, kRelThreads, 0, s>>>(
        off, n, ntiles, reinterpret_cast<const unsigned long long*>(b), new2old, old2new);
    rel_newdeg_kernel<<<sms * 4, 256, 0, s>>>(off, new2old, n, a);
    e = exclusive_scan_i64(a, n, new_off, tmp, s);
    if (e != cudaSuccess) return e;
    rel_columns_kernel<<<sms * 8, 256, 0, s>>>(off, col, new2old, old2new, new_off, n,
                                                reinterpret_cast<const unsigned long long*>(b), ntiles,
                                                new_col);
    (void)nnz;
    return cudaGetLastError();
}

}  // namespace bfs
