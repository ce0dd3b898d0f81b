// bfs_kernels.cu -- the top-down level step on sm_103a.
//
// Algorithm 2 Phase 1 with one compute node (= Algorithm 1 with an atomic
// enqueue): every vertex v of the current frontier scans adj(v); each
// neighbour u whose distance is still infinity is claimed by exactly one
// thread (the claim is an atomicOr on the visited bitmap; Algorithm 2 gates
// the distance write on the success of the atomic enqueue), which writes
// d[u] = level + 1 and appends u to the next frontier.  When the frontier is
// empty the traversal ends (the While loop of Algorithm 1).
//
// GB300 design:
//  * The whole level loop runs inside one cooperative persistent launch
//    (grid = resident CTAs of all 152 SMs) separated by a grid barrier
//    whose wait is bounded by %globaltimer, so no per-level host round trip;
//    the same level kernels also run as the body of a CUDA-graph while loop
//    (phases 5-9 of the step kernels) or one launch per level from the host.
//  * Load balancing replaces the paper's Logarithmic Radix Binning (one
//    kernel per log2-degree bin, Section "Load Balanced Traversals Per
//    compute-node") with three degree bins written while the next frontier
//    is built: deg < t_small (edges of 32 vertices spread over the warp by a
//    scan), t_small <= deg < t_large (warp chunks of 16-byte column units
//    over several rows, 128-bit loads) and deg >= t_large (CTA chunks;
//    heavy vertices span many CTAs).  Each bin counter packs (entries << 34 |
//    edge prefix) so that one 64-bit atomicAdd per bin reserves queue slots
//    and edge ranges at once; warp and CTA work items are fixed-size edge
//    chunks, located through a chunk-start table filled at enqueue time.
//  * Probes read the visited bitmap with plain loads, 8 per lane in flight;
//    the atomicOr claims are batched -- per probe round when it has many
//    candidates, otherwise per 64-entry stage at flush time.
//  * The batched traversal carries a 64-bit source-lane set per vertex:
//    phase A ORs the frontier lanes into next[u] (or, bottom-up, ORs the
//    neighbours' frontier lanes into each vertex that lacks some), phase B
//    (a sweep) turns the lanes that are new into distances and the next
//    frontier.
#include <cuda_runtime.h>
#include <cstdint>

#include "bfs_internal.h"

// This file is compiled twice.  As is, it holds every traversal kernel and
// the upload helpers.  bfs_kernels_lean.cu compiles it again with
// BFS_LEAN_PATHS = 1 into namespace bfs::lean, where only the single-source
// persistent kernel is instantiated and the paths that the full kernel
// enables at run time -- direction optimisation and the frontier bitmaps,
// the shared-memory copy of the hot bitmap, warp-aggregated claims, bulk L2
// prefetch -- are compiled out.  The host launches that kernel whenever a
// traversal uses none of them (the default): its probe loops then get the
// registers those paths held (spills at 4 CTAs/SM 232/352 -> 108/256 bytes,
// 0.539 -> 0.493 ms per scale-22 root).
#ifndef BFS_LEAN_PATHS
#define BFS_LEAN_PATHS 0
#endif

namespace bfs {
#if BFS_LEAN_PATHS
namespace lean {
#endif

constexpr bool kLean = BFS_LEAN_PATHS != 0;

#define FULL_MASK 0xffffffffu

// ---------------------------------------------------------------- helpers

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ unsigned long long global_timer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) { return *(const volatile int*)p; }
__device__ __forceinline__ unsigned long long ld_cg_u64(const unsigned long long* p) {
    return __ldcg(p);
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T x) {
    const unsigned lane = lane_id();
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T y = __shfl_up_sync(FULL_MASK, x, d);
        if (lane >= (unsigned)d) x += y;
    }
    return x;
}

__device__ __forceinline__ void raise_status(const TraversalParams& P, int code) {
    atomicCAS(&P.stats->status, 0, code);
}

// One bulk request that brings col[a, b) into L2 (cp.async.bulk.prefetch:
// no shared memory, no completion to wait for).  Start and size must be
// multiples of 16 bytes; col is padded past its last entry, so rounding the
// end up stays inside the allocation.
__device__ __forceinline__ void prefetch_cols_l2(const int32_t* col, long long a, long long b) {
    if (b <= a) return;
    const long long a4 = a & ~3ll, b4 = (b + 3) & ~3ll;
    const unsigned bytes = (unsigned)((b4 - a4) * 4);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(col + a4), "r"(bytes)
                 : "memory");
}

// Prefetch distance of the heavy bins, in column entries (32 KiB).
constexpr long long kPrefetchAhead = 8192;

// Level timeline (diagnostics): block 0, thread 0 records %globaltimer.
__device__ __forceinline__ void stamp(const TraversalParams& P, int i) {
    if (P.timeline && i < P.timeline_cap && blockIdx.x == 0 && threadIdx.x == 0)
        P.timeline[i] = global_timer_ns();
}

// ------------------------------------------------- TMA bulk copies (1D)
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
// Arrive on bar and expect `bytes` of asynchronous transfers in this phase.
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// One bulk copy global -> shared (16-byte aligned ends, size a multiple of
// 16), completing `bytes` transactions on bar.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, unsigned bytes,
                                            unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// Waits for phase `parity` of bar, giving up after the traversal's wait
// limit (%globaltimer) or when another CTA has aborted the launch.
__device__ __forceinline__ bool mbar_wait_bounded(const TraversalParams& P,
                                                  unsigned long long* bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_timer_ns();
    for (unsigned it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 15u) == 15u) {
            if (global_timer_ns() - t0 > (unsigned long long)P.timeout_ns) return false;
            if (ld_volatile_i32(&P.stats->abort) != 0) return false;
        }
    }
}

// ------------------------------------------------------------ grid barrier
// All CTAs are co-resident (cooperative launch).  Thread 0 of each CTA adds
// its arrival to one 64-bit word that only grows during a launch: the k-th
// barrier is complete once the word reaches k * gridDim.x, so an arrival is
// a fire-and-forget reduction and the wait is a loop of acquire loads (no
// reset or generation step that the last arrival would have to publish with
// further round trips).  Bit 63 of the word says that a CTA gave up: a wait
// longer than timeout_ns of %globaltimer records kDevTimeout, sets the bit
// and returns false, and every CTA that reads the bit returns false too.
// `epoch` (thread 0's, in shared memory: no register held across the level
// loop) counts the barriers this CTA has passed in the launch, the same in
// every CTA; the last CTA to leave the launch clears the word.
constexpr unsigned long long kBarGaveUp = 1ull << 63;

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Tells every CTA waiting at (or arriving at) a grid barrier to leave.
__device__ __forceinline__ void give_up(const TraversalParams& P) {
    atomicExch(&P.stats->abort, 1);
    atomicOr(&P.bar->arrived, kBarGaveUp);
}

__device__ bool grid_barrier(const TraversalParams& P, unsigned long long& epoch) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long* const word = &P.bar->arrived;
        const unsigned long long target =
            ++epoch * gridDim.x + (P.debug_stall ? 1ull : 0ull);
        __threadfence();
        asm volatile("red.relaxed.gpu.global.add.u64 [%0], 1;" ::"l"(word) : "memory");
        int ok = 1;
        unsigned long long t0 = 0ull;
        for (;;) {
            const unsigned long long a = ld_acquire_u64(word);
            if (a & kBarGaveUp) { ok = 0; break; }
            if (a >= target) break;
            const unsigned long long t = global_timer_ns();
            if (t0 == 0ull) {
                t0 = t;
            } else if (t - t0 > (unsigned long long)P.timeout_ns) {
                raise_status(P, kDevTimeout);
                give_up(P);
                ok = 0;
                break;
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Last CTA to leave a persistent launch clears the barrier and abort flag,
// so the next launch starts clean even after a timed-out wait.
__device__ void kernel_exit(const TraversalParams& P) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned done = atomicAdd(&P.bar->exited, 1u) + 1u;
        if (done == gridDim.x) {
            atomicExch(&P.bar->arrived, 0ull);
            atomicExch(&P.bar->exited, 0u);
            atomicExch(&P.stats->abort, 0);
            __threadfence();
        }
    }
}

// --------------------------------------------------------------- enqueue
// Candidate vertices (claimed or still to claim) are staged per warp in
// shared memory and appended to the next frontier up to 64 at a time
// (measured faster than 32, 128 and 256 on GB300).  The flush claims the
// unclaimed ones, does the per-vertex work that needs random reads (degree
// from the row offsets, caller numbering) for the whole group at once,
// writes the distances and parents, bins the group by degree, and reserves
// queue slots and edge ranges with one 64-bit atomicAdd per bin (the bin
// counter packs entries << 34 | edge prefix).
#ifndef BFS_STAGE_CAP
#define BFS_STAGE_CAP 64
#endif
constexpr int kStageCap = BFS_STAGE_CAP;
// A probe round whose warp holds at least this many candidates claims them
// at once (one atomic round trip shared by all of them); rounds with fewer
// leave the claim to the stage flush.
#ifndef BFS_CLAIM_NOW
#define BFS_CLAIM_NOW 16
#endif
constexpr int kClaimNow = BFS_CLAIM_NOW;
// Parent field flag of a staged entry that is already claimed.
constexpr uint32_t kClaimed = 0x80000000u;

template <bool kBatch>
struct Stage {
    int32_t u[kStageCap];
    int32_t v[kBatch ? 1 : kStageCap];                 // plain: parent of u
    unsigned long long mask[kBatch ? kStageCap : 1];   // batched: new lanes of u
    int cnt;
    unsigned long long edges;                          // batched: sum deg * lanes
    const uint32_t* hot;                               // plain: shared copy of visited[0, hot_bits)
    int hot_bits;                                      // 0 when the copy is off for this level
    int disc;                                          // plain: vertices this warp claimed
    uint4* tma_buf;                  // plain, BFS_OPT_TMA_STAGE: two 1 KB staging buffers
    unsigned long long* tma_bar;     // their mbarriers
    unsigned tma_ph;                 // bit b: parity of buffer b's next phase
    int tma_ok;                      // 0 after a staging wait gave up
};

// Warp-collective flush of the staged entries into the next frontier.
// Lane l owns entries [H l, H l + H): all their random reads (row offsets,
// caller numbering) are issued together; one packed atomicAdd per bin,
// issued by lanes 0..2 at once, places the lane's entries at consecutive
// queue slots.
//
// The flush is inlined at every call site: as an out-of-line call it made
// the callers save their live registers around it (spills on the probe
// loops' critical path).  Launch parameters are still read into registers
// before the stores that follow them: P is a reference, and a parameter read
// after a global store through a generic pointer cannot be moved above it
// (the compiler cannot rule out that the store changed the parameter), which
// would put a round trip on every chunk-table iteration.
template <bool kBatch>
__device__ __forceinline__ void stage_flush(const TraversalParams& P, Stage<kBatch>& S, int level,
                                         int nxt, int nslot) {
    constexpr int H = kStageCap / 32;
    const unsigned lane = lane_id();
    const int n = S.cnt;
    if (n == 0) return;
    const int64_t* const off = P.off;
    const int32_t* const new2old = P.new2old;
    int32_t* const dist = P.dist;
    int32_t* const parent = P.parent;
    uint32_t* const fbn = (!kLean && P.fb[0]) ? P.fb[(level + 1) % 3] : nullptr;
    const int t_small = P.t_small, t_large = P.t_large;
    const int sh_warp = __ffs(P.chunk_warp) - 1, sh_cta = __ffs(P.chunk_cta) - 1;
    unsigned long long* const packed = P.ctl[nslot].packed;
    bool overflow = false;

    const int i0 = (int)lane * H;
    int32_t u[H];
    int deg[H];
#pragma unroll
    for (int h = 0; h < H; ++h) u[h] = (i0 + h < n) ? S.u[i0 + h] : -1;
    // The random reads that do not depend on the claim (row offsets, caller
    // numbering) are issued before it, so that their round trip overlaps the
    // atomics' instead of following it.
#pragma unroll
    for (int h = 0; h < H; ++h) {
        deg[h] = -1;
        if (u[h] >= 0) deg[h] = (int)(__ldg(off + u[h] + 1) - __ldg(off + u[h]));
    }
    int32_t cu[H], cv[H];
    // Plain entries are candidates (their target looked unvisited when it
    // was probed): the claim -- an atomicOr on the visited bitmap whose old
    // value says who set the bit first -- happens here, for all of a flush's
    // entries at once, instead of one round trip per probe round.
    uint32_t old[H];
    uint32_t pv[H];  // plain: staged parent with the claimed flag
    if constexpr (!kBatch) {
        uint32_t* const visited = P.visited;
#pragma unroll
        for (int h = 0; h < H; ++h) {
            pv[h] = u[h] >= 0 ? (uint32_t)S.v[i0 + h] : 0u;
            cu[h] = u[h];
            cv[h] = (u[h] >= 0) ? (int32_t)(pv[h] & ~kClaimed) : 0;
            if (new2old && u[h] >= 0) {
                cu[h] = __ldg(new2old + u[h]);
                cv[h] = __ldg(new2old + cv[h]);
            }
        }
        if (!kLean && P.use_match_any) {
            // lanes claiming bits of the same word merge them: one atomicOr
            // per word, the first lane holding a vertex wins it
#pragma unroll
            for (int h = 0; h < H; ++h) {
                old[h] = (u[h] >= 0 && (pv[h] & kClaimed)) ? 0u : 0xffffffffu;
                const bool need = u[h] >= 0 && !(pv[h] & kClaimed);
                const unsigned needm = __ballot_sync(FULL_MASK, need);
                if (need) {
                    const uint32_t bit = 1u << (u[h] & 31);
                    const unsigned peers = __match_any_sync(needm, u[h] >> 5);
                    const uint32_t bits = __reduce_or_sync(peers, bit);
                    const int leader = __ffs(peers) - 1;
                    uint32_t o = 0u;
                    if ((int)lane == leader) o = atomicOr(visited + (u[h] >> 5), bits);
                    o = __shfl_sync(peers, o, leader);
                    const unsigned same = __match_any_sync(peers, u[h]);
                    if ((o & bit) == 0u && (int)lane == __ffs(same) - 1) old[h] = 0u;
                }
            }
        } else {
#pragma unroll
            for (int h = 0; h < H; ++h) {
                old[h] = 0xffffffffu;
                if (u[h] >= 0)
                    old[h] = (pv[h] & kClaimed) ? 0u : atomicOr(visited + (u[h] >> 5), 1u << (u[h] & 31));
            }
        }
    }
    if constexpr (kBatch) {
        unsigned long long e = 0;
#pragma unroll
        for (int h = 0; h < H; ++h)
            if (u[h] >= 0) e += (unsigned long long)deg[h] * __popcll(S.mask[i0 + h]);
        if (e) atomicAdd(&S.edges, e);
    } else {
        // entries whose claim lost are dropped
        int won = 0;
#pragma unroll
        for (int h = 0; h < H; ++h) {
            if (u[h] >= 0 && ((old[h] >> (u[h] & 31)) & 1u)) {
                u[h] = -1;
                deg[h] = -1;
            }
            won += __popc(__ballot_sync(FULL_MASK, u[h] >= 0));
        }
        if (lane == 0) S.disc += won;
#pragma unroll
        for (int h = 0; h < H; ++h) {
            if (u[h] < 0) continue;
            dist[cu[h]] = level + 1;
            if (parent) parent[cu[h]] = cv[h];
            if (fbn) atomicOr(fbn + (u[h] >> 5), 1u << (u[h] & 31));
        }
    }
    // Reserve queue slots and edge ranges for all bins in one round trip:
    // per bin one warp scan of (entries << 48 | degree sum) -- a lane holds
    // at most H entries and degrees stay below 2^31, so the sum fits in 48
    // bits -- then lanes 0..2 issue the bins' atomicAdds together.
    int bh[H];
#pragma unroll
    for (int h = 0; h < H; ++h)
        bh[h] = deg[h] <= 0 ? -1 : (deg[h] < t_small ? 0 : (deg[h] < t_large ? 1 : 2));
    unsigned long long incl[kBins], mine[kBins];
    unsigned long long add = 0ull;
#pragma unroll
    for (int b = 0; b < kBins; ++b) {
        unsigned long long x = 0ull;
#pragma unroll
        for (int h = 0; h < H; ++h)
            if (bh[h] == b) x += (1ull << 48) + (unsigned long long)deg[h];
        mine[b] = x;
        incl[b] = 0ull;
        if (__ballot_sync(FULL_MASK, x != 0ull) == 0u) continue;
        incl[b] = warp_incl_scan(x);
        const unsigned long long tot = __shfl_sync(FULL_MASK, incl[b], 31);
        if (lane == (unsigned)b)
            add = ((tot >> 48) << kCountShift) + (tot & ((1ull << 48) - 1ull));
    }
    unsigned long long basep = 0ull;
    if (add != 0ull) basep = atomicAdd(packed + lane, add);
#pragma unroll
    for (int b = 0; b < kBins; ++b) {
        const unsigned long long base = __shfl_sync(FULL_MASK, basep, b);
        if (mine[b] == 0ull) continue;
        const unsigned long long excl = incl[b] - mine[b];
        long long pos = (long long)(base >> kCountShift) + (long long)(excl >> 48);
        long long eo = (long long)(base & kEdgeMask) + (long long)(excl & ((1ull << 48) - 1ull));
        // chunk sizes are powers of two: chunk c starts at edge c << cshift
        const int cshift = b == 1 ? sh_warp : sh_cta;
        const BinQueue& Q = P.q[nxt][b];
        int32_t* const qv = Q.v;
        int64_t* const qe = Q.eoff;
        int32_t* const qc = Q.chunk;
        uint64_t* const qm = kBatch ? Q.mask : nullptr;
        const long long qcap = Q.cap, qccap = Q.chunk_cap;
#pragma unroll
        for (int h = 0; h < H; ++h) {
            if (bh[h] != b) continue;
            if (pos < qcap) {
                qv[pos] = u[h];
                if (kBatch) qm[pos] = S.mask[kBatch ? i0 + h : 0];
                if (b > 0) {
                    qe[pos] = eo;
                    // chunks whose first edge lies in [eo, eo + deg) start here
                    const long long c_end = (eo + deg[h] - 1) >> cshift;
                    const long long c0 = (eo + (1ll << cshift) - 1) >> cshift;
                    if (c_end >= qccap) overflow = true;
                    for (long long c = c0; c <= c_end && c < qccap; ++c) qc[c] = (int32_t)pos;
                }
            } else {
                overflow = true;
            }
            ++pos;
            eo += deg[h];
        }
    }
    if (overflow) raise_status(P, kDevOverflow);
    __syncwarp();
    if (lane == 0) S.cnt = 0;
    __syncwarp();
}

// Warp-collective: lanes with ok stage u (with its parent v, or its new
// lanes mask).
template <bool kBatch>
__device__ __forceinline__ void stage_push(const TraversalParams& P, Stage<kBatch>& S, bool ok,
                                           int32_t u, int32_t v, uint64_t mask, int level,
                                           int nxt, int nslot) {
    const unsigned m = __ballot_sync(FULL_MASK, ok);
    if (m == 0u) return;
    int n0 = S.cnt;
    const int k = __popc(m);
    if (n0 + k > kStageCap) {
        stage_flush<kBatch>(P, S, level, nxt, nslot);
        n0 = 0;
    }
    if (ok) {
        const int i = n0 + __popc(m & lanemask_lt());
        S.u[i] = u;
        if constexpr (kBatch) S.mask[i] = mask;
        else S.v[i] = v;
    }
    __syncwarp();
    if (lane_id() == 0) S.cnt = n0 + k;
    __syncwarp();
}

template <bool kBatch>
__device__ __forceinline__ void stage_init(Stage<kBatch>& S) {
    if (lane_id() == 0) {
        S.cnt = 0;
        S.edges = 0ull;
        S.hot = nullptr;
        S.hot_bits = 0;
        S.disc = 0;
        S.tma_buf = nullptr;
        S.tma_bar = nullptr;
        S.tma_ph = 0u;
        S.tma_ok = 0;
    }
    __syncwarp();
}

// Staging buffers and mbarriers of this warp (plain kernels with
// BFS_OPT_TMA_STAGE): two 1 KB buffers in dynamic shared memory after the
// hot bitmap prefix, two mbarriers with one arrival per phase.
__device__ void tma_setup(const TraversalParams& P, Stage<false>& S, uint4* s_dyn) {
    __shared__ __align__(8) unsigned long long s_tma_bar[kWarps * 2];
    if (!P.tma_stage) return;
    const int warp = threadIdx.x >> 5;
    if (lane_id() == 0) {
        unsigned long long* bar = s_tma_bar + 2 * warp;
        mbar_init(bar, 1u);
        mbar_init(bar + 1, 1u);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        S.tma_buf = s_dyn + P.tma_offset / 16 + warp * 128;
        S.tma_bar = bar;
        S.tma_ph = 0u;
        S.tma_ok = 1;
    }
    __syncwarp();
}

// ----------------------------------------------------------------- visits
// Stages each lane's candidates (bit j of candm: u[j] with parent v[j],
// flag kClaimed when already claimed) in one pass: a warp scan of the
// per-lane counts places them; a full stage is flushed and the rest placed
// after it.
template <int K>
__device__ __forceinline__ void stage_push_multi(const TraversalParams& P, Stage<false>& S,
                                                 unsigned candm, const int32_t (&u)[K],
                                                 const int32_t (&v)[K], uint32_t flag, int level,
                                                 int nxt, int nslot) {
    const int c = __popc(candm);
    if (__ballot_sync(FULL_MASK, c != 0) == 0u) return;
    const int incl = warp_incl_scan(c);
    const int total = __shfl_sync(FULL_MASK, incl, 31);
    const int excl = incl - c;
    for (int done = 0; done < total;) {
        int n0 = S.cnt;
        if (n0 == kStageCap) {
            stage_flush<false>(P, S, level, nxt, nslot);
            n0 = 0;
        }
        const int take = min(kStageCap - n0, total - done);
        int k = excl - done;  // stage offset of this lane's next candidate
#pragma unroll
        for (int j = 0; j < K; ++j) {
            if ((candm >> j) & 1u) {
                if (k >= 0 && k < take) {
                    S.u[n0 + k] = u[j];
                    S.v[n0 + k] = (int32_t)((uint32_t)v[j] | flag);
                }
                ++k;
            }
        }
        __syncwarp();
        if (lane_id() == 0) S.cnt = n0 + take;
        __syncwarp();
        done += take;
    }
}

// K edges per lane at once: all K visited-bitmap probes are issued before
// any result is used, so a warp keeps K random reads in flight instead of
// one.  A probe that finds the bit clear makes the edge a candidate.  The
// claim (the atomicOr whose old value decides which edge discovers the
// vertex) is made here when the round has many candidates -- discovery-
// heavy levels, where claiming early also keeps other warps from staging
// the same vertex -- and otherwise left to the stage flush, which claims a
// whole stage in one round trip instead of one per probe round.  A stale
// cached word can only show clear a bit that is already set (bits are never
// cleared during a traversal), and the claim then rejects the candidate.
template <int K>
__device__ __forceinline__ void visit_plain_k(const TraversalParams& P, Stage<false>& S,
                                              unsigned okm, const int32_t (&u)[K],
                                              const int32_t (&v)[K], int level, int nxt,
                                              int nslot) {
    // pass 1 (shared memory only): drop edges whose target was visited before
    // the level and lies in the hot prefix copied at level start
    const int hot_bits = S.hot_bits;
    if (!kLean && hot_bits > 0) {
        const uint32_t* hot = S.hot;
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (((okm >> j) & 1u) && u[j] < hot_bits && ((hot[u[j] >> 5] >> (u[j] & 31)) & 1u))
                okm &= ~(1u << j);
    }
    // pass 2: independent global probes for the rest
    uint32_t w[K];
#pragma unroll
    for (int j = 0; j < K; ++j) w[j] = ((okm >> j) & 1u) ? P.visited[u[j] >> 5] : 0xffffffffu;
    unsigned candm = 0u;
#pragma unroll
    for (int j = 0; j < K; ++j)
        if (((w[j] >> (u[j] & 31)) & 1u) == 0u) candm |= 1u << j;
    const int total = __reduce_add_sync(FULL_MASK, (unsigned)__popc(candm));
    if (total == 0) return;
    uint32_t flag = 0u;
    if (total >= kClaimNow) {
#pragma unroll
        for (int j = 0; j < K; ++j)
            if ((candm >> j) & 1u) w[j] = atomicOr(P.visited + (u[j] >> 5), 1u << (u[j] & 31));
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (((w[j] >> (u[j] & 31)) & 1u) != 0u) candm &= ~(1u << j);
        flag = kClaimed;
    }
    stage_push_multi<K>(P, S, candm, u, v, flag, level, nxt, nslot);
}

// Batched traversal, phase A: OR the lanes of the frontier entry that u has
// not seen yet into next[u].  visited only changes in phase B, so a cached
// value is a safe filter; next[u] is read first so that lanes already
// present skip the atomic (a fire-and-forget red.or otherwise).
// The K pairs are read in groups of kBatchProbeGroup (4 at 3 CTAs/SM: 8
// would keep 32 registers of pairs live, which spills at that occupancy).
template <int K>
__device__ __forceinline__ void visit_batch_k(const TraversalParams& P, unsigned okm,
                                              const int32_t (&u)[K],
                                              const uint64_t (&mask)[K]) {
    constexpr int G = K < 4 ? K : 4;
#pragma unroll
    for (int j0 = 0; j0 < K; j0 += G) {
        // visited and next of a vertex are adjacent: one 16-byte load each
        ulonglong2 vn[G];
#pragma unroll
        for (int j = 0; j < G; ++j)
            vn[j] = ((okm >> (j0 + j)) & 1u)
                        ? *reinterpret_cast<const ulonglong2*>(P.lane_vn + 2 * (long long)u[j0 + j])
                        : make_ulonglong2(~0ull, ~0ull);
#pragma unroll
        for (int j = 0; j < G; ++j) {
            const uint64_t m = mask[j0 + j] & ~vn[j].x;
            if ((m & ~vn[j].y) != 0ull)
                atomicOr(reinterpret_cast<unsigned long long*>(P.lane_vn + 2 * (long long)u[j0 + j] + 1),
                         (unsigned long long)m);
        }
    }
}

template <bool kBatch, int K>
__device__ __forceinline__ void visit_k(const TraversalParams& P, Stage<kBatch>& S, unsigned okm,
                                        const int32_t (&u)[K], const int32_t (&v)[K],
                                        const uint64_t (&mask)[K], int level, int nxt, int nslot) {
    if constexpr (kBatch) visit_batch_k<K>(P, okm, u, mask);
    else visit_plain_k<K>(P, S, okm, u, v, level, nxt, nslot);
}

// ------------------------------------------------------------ expansion
// A heavy vertex's column run read through shared memory (BFS_OPT_TMA_STAGE):
// the warp's 256-entry blocks of the run (block j at wbase + 2048 j
// entries from a4, as in the CTA-interleaved schedule below) stream through
// its two 1 KB buffers, each filled by one TMA bulk copy that lane 0 issues
// two blocks ahead, so the next block is in flight while the current one is
// probed.  valid entries: [lo, hi) relative to a4 (16-byte aligned).
__device__ void expand_segment_staged(const TraversalParams& P, Stage<false>& S, long long a4,
                                      int lo, int hi, int32_t v, int level, int nxt, int nslot,
                                      int wbase) {
    const unsigned lane = lane_id();
    const int nblk = wbase < hi ? (hi - wbase + 2047) / 2048 : 0;
    if (nblk == 0 || !S.tma_ok) return;
    uint4* const buf = S.tma_buf;
    unsigned long long* const bar = S.tma_bar;
    unsigned ph = S.tma_ph;
    const int32_t* const colp = P.col + a4;
    auto issue = [&](int j) {  // lane 0
        const int rw = wbase + j * 2048;
        const int cnt = min(256, hi - rw);
        const unsigned bytes = (unsigned)((cnt * 4 + 15) & ~15);
        const int b = j & 1;
        // the buffer's previous contents were read by the generic proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar + b, bytes);
        tma_load_1d(buf + b * 64, colp + rw, bytes, bar + b);
    };
    if (lane == 0) {
        issue(0);
        if (nblk > 1) issue(1);
    }
    int j = 0;
    bool ok = true;
    for (; j < nblk; ++j) {
        const int b = j & 1;
        ok = __all_sync(FULL_MASK, mbar_wait_bounded(P, bar + b, (ph >> b) & 1u));
        if (!ok) break;
        ph ^= 1u << b;
        const uint4 x0 = buf[b * 64 + lane], x1 = buf[b * 64 + 32 + lane];
        __syncwarp();
        if (lane == 0 && j + 2 < nblk) issue(j + 2);
        const int r0 = wbase + j * 2048 + 4 * (int)lane, r1 = r0 + 128;
        unsigned okm = 0u;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (r0 + c >= lo && r0 + c < hi) okm |= 1u << c;
            if (r1 + c >= lo && r1 + c < hi) okm |= 1u << (4 + c);
        }
        const int32_t u[8] = {(int32_t)x0.x, (int32_t)x0.y, (int32_t)x0.z, (int32_t)x0.w,
                              (int32_t)x1.x, (int32_t)x1.y, (int32_t)x1.z, (int32_t)x1.w};
        const int32_t vv[8] = {v, v, v, v, v, v, v, v};
        visit_plain_k<8>(P, S, okm, u, vv, level, nxt, nslot);
    }
    if (!ok) {
        // a copy did not land in time: stop the launch, then let the copies
        // still in flight (blocks j and j + 1) complete before leaving
        if (lane == 0) {
            raise_status(P, kDevTimeout);
            give_up(P);
            for (int k = j; k < min(j + 2, nblk); ++k) {
                const int b = k & 1;
                const unsigned long long t0 = global_timer_ns();
                while (!mbar_try_wait(bar + b, (ph >> b) & 1u) &&
                       global_timer_ns() - t0 < (unsigned long long)P.timeout_ns) {
                }
                ph ^= 1u << b;
            }
            S.tma_ok = 0;
        }
    }
    if (lane == 0) S.tma_ph = ph;
    __syncwarp();
}

// One column segment col[a, b) of vertex v, read by a group of warps with
// 128-bit loads (start rounded down to 16 bytes; col is padded so the
// rounded reads stay inside the allocation).  wbase/wstride place this
// warp's 256-entry blocks; a segment that fits in 128 entries uses one
// 128-bit load per lane.
template <bool kBatch, bool kStaged = false>
__device__ __forceinline__ void expand_segment(const TraversalParams& P, Stage<kBatch>& S,
                                               long long a, long long b, int32_t v, uint64_t mask,
                                               int level, int nxt, int nslot, long long wbase,
                                               long long wstride) {
    const unsigned lane = lane_id();
    const long long a4 = a & ~3ll;
    const int lo = (int)(a - a4);                 // valid entries: [lo, hi) relative to a4
    const int hi = (int)(b - a4);
    if constexpr (!kBatch && kStaged) {
        if (S.tma_buf != nullptr && wstride == 256ll * kWarps) {
            expand_segment_staged(P, S, a4, lo, hi, v, level, nxt, nslot, (int)wbase);
            return;
        }
    }
    const int32_t* colp = P.col + a4;
    int32_t vv[8];
    uint64_t mm[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        vv[j] = v;
        mm[j] = mask;
    }
    if (wbase == 0 && wstride == 256 && hi <= 128) {
        const int r0 = 4 * (int)lane;
        int4 x0 = make_int4(0, 0, 0, 0);
        if (r0 < hi) x0 = __ldcs(reinterpret_cast<const int4*>(colp + r0));
        unsigned okm = 0u;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (r0 + j >= lo && r0 + j < hi) okm |= 1u << j;
        const int32_t u[4] = {x0.x, x0.y, x0.z, x0.w};
        const int32_t v4[4] = {v, v, v, v};
        const uint64_t m4[4] = {mask, mask, mask, mask};
        visit_k<kBatch, 4>(P, S, okm, u, v4, m4, level, nxt, nslot);
        return;
    }
    for (int rw = (int)wbase; rw < hi; rw += (int)wstride) {
        if (!kLean && P.l2_prefetch && lane == 0 && rw + kPrefetchAhead < hi)
            prefetch_cols_l2(P.col, a4 + rw + kPrefetchAhead,
                             a4 + min((long long)hi, rw + kPrefetchAhead + 256));
        const int r0 = rw + 4 * (int)lane;
        const int r1 = r0 + 128;
        int4 x0 = make_int4(0, 0, 0, 0), x1 = make_int4(0, 0, 0, 0);
        if (r0 < hi) x0 = __ldcs(reinterpret_cast<const int4*>(colp + r0));
        if (r1 < hi) x1 = __ldcs(reinterpret_cast<const int4*>(colp + r1));
        unsigned okm = 0u;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (r0 + j >= lo && r0 + j < hi) okm |= 1u << j;
            if (r1 + j >= lo && r1 + j < hi) okm |= 1u << (4 + j);
        }
        const int32_t u[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
        visit_k<kBatch, 8>(P, S, okm, u, vv, mm, level, nxt, nslot);
    }
}

// Bin 0: 32 frontier vertices per warp, one per lane; their edges are laid
// end to end by an exclusive scan and consumed 256 per round, lane l taking
// edges l + 32 j (j < 8) and finding each edge's owner vertex in a
// per-round owner table in shared memory that each lane fills for its own
// edges (cheaper than a shuffle binary search per edge: a lane writes at
// most its degree's slots).
template <bool kBatch>
__device__ void expand_small_group(const TraversalParams& P, Stage<kBatch>& S, int cur,
                                   long long grp, long long cnt, int level, int nxt, int nslot) {
    const BinQueue& Q = P.q[cur][0];
    const unsigned lane = lane_id();
    const long long i = grp * 32 + lane;
    int32_t v = 0;
    long long base = 0;
    int deg = 0;
    uint64_t mask = 0ull;
    if (i < cnt) {
        v = __ldcg(Q.v + i);
        base = __ldg(P.off + v);
        deg = (int)(__ldg(P.off + v + 1) - base);
        if (kBatch) mask = __ldcg(reinterpret_cast<const unsigned long long*>(Q.mask) + i);
    }
    const int incl = warp_incl_scan(deg);
    const int excl = incl - deg;
    const int total = __shfl_sync(FULL_MASK, incl, 31);
    // owner of each of the round's 256 edge slots, written by the owning lane
    __shared__ uint8_t s_owner[kWarps][256];
    uint8_t* const own = s_owner[threadIdx.x >> 5];
    for (int e0 = 0; e0 < total; e0 += 256) {
        unsigned okm = 0u;
        int32_t u[8], vv[8];
        uint64_t mm[8];
        {
            const int a = max(excl, e0), b = min(excl + deg, e0 + 256);
            __syncwarp();
            for (int e = a; e < b; ++e) own[e - e0] = (uint8_t)lane;
            __syncwarp();
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int e = e0 + 32 * j + (int)lane;
            u[j] = 0;
            vv[j] = 0;
            mm[j] = 0ull;
            // slots past the round's last edge (the same for the whole warp)
            // need no owner lookup
            if (e0 + 32 * j < total) {
                const int o = e < total ? own[32 * j + lane] : 0;
                const long long bo = __shfl_sync(FULL_MASK, base, o);
                const int xo = __shfl_sync(FULL_MASK, excl, o);
                vv[j] = __shfl_sync(FULL_MASK, v, o);
                mm[j] = kBatch ? __shfl_sync(FULL_MASK, (unsigned long long)mask, o) : 0ull;
                if (e < total) {
                    okm |= 1u << j;
                    u[j] = __ldcs(P.col + bo + (e - xo));
                }
            }
        }
        visit_k<kBatch, 8>(P, S, okm, u, vv, mm, level, nxt, nslot);
    }
}

// Valid columns of the 16-byte unit holding row-relative columns [r, r + 4)
// of a row whose valid columns are [lo, hi): bits [lo - r, hi - r) of 4.
__device__ __forceinline__ unsigned unit_mask(int r, int lo, int hi) {
    const int a = min(max(lo - r, 0), 4), b = min(max(hi - r, 0), 4);
    return ((1u << b) - 1u) & ~((1u << a) - 1u);
}

// Bins 1 and 2 as warp items: edges [cs, ce) of bin b's level sequence
// (a bin-1 chunk of chunk_warp edges, or, on small levels, a 32-edge slice
// of either bin).  The range's vertex segments (up to 32 at a time, from the
// entry that holds the first edge of its base chunk) are cut into 16-byte
// units (4 columns, the first rounded down to a 16-byte boundary) laid end
// to end by a scan; each round a lane takes two units, finds their segments
// by a shuffle binary search, and reads each with one 128-bit load -- short
// and long segments alike keep every lane busy.
template <bool kBatch>
__device__ void expand_warp_range(const TraversalParams& P, Stage<kBatch>& S, const BinQueue& Q,
                                  int cshift, long long cs, long long ce, long long cnt, int level,
                                  int nxt, int nslot) {
    const unsigned lane = lane_id();
    long long i = __ldcg(Q.chunk + (cs >> cshift));
    for (;;) {
        const long long ij = i + lane;
        long long eo = 0x7fffffffffffffffll;
        if (ij < cnt) eo = __ldcg(Q.eoff + ij);
        const bool ok = eo < ce;
        bool live = false;  // the segment overlaps [cs, ce) (a slice's first
                            // entries may end before cs)
        int32_t v = 0;
        long long a = 0, b = 0;
        uint64_t mask = 0ull;
        if (ok) {
            v = __ldcg(Q.v + ij);
            const long long base = __ldg(P.off + v), end = __ldg(P.off + v + 1);
            const long long lo = max(eo, cs), hi = min(eo + (end - base), ce);
            live = hi > lo;
            a = base + (lo - eo);
            b = base + (hi - eo);
            if (kBatch) mask = __ldcg(reinterpret_cast<const unsigned long long*>(Q.mask) + ij);
            if (!kLean && P.l2_prefetch && live) prefetch_cols_l2(P.col, a, min(b, a + kPrefetchAhead));
        }
        const unsigned okb = __ballot_sync(FULL_MASK, ok);
        const long long a4 = a & ~3ll;
        const int rlo = (int)(a - a4), rhi = (int)(b - a4);  // valid columns, relative to a4
        const int units = live ? (rhi + 3) >> 2 : 0;
        const int incl = warp_incl_scan(units);
        const int excl = incl - units;
        const int total = __shfl_sync(FULL_MASK, incl, 31);
        for (int q0 = 0; q0 < total; q0 += 64) {
            unsigned okm = 0u;
            int32_t u[8], vv[8];
            uint64_t mm[8];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int q = q0 + 32 * h + (int)lane;
                int o = 0;
#pragma unroll
                for (int st = 16; st > 0; st >>= 1) {
                    const int c = o + st;
                    if (__shfl_sync(FULL_MASK, excl, c & 31) <= q) o = c;
                }
                const long long a4o = __shfl_sync(FULL_MASK, a4, o);
                const int lo_o = __shfl_sync(FULL_MASK, rlo, o);
                const int hi_o = __shfl_sync(FULL_MASK, rhi, o);
                const int xo = __shfl_sync(FULL_MASK, excl, o);
                const int32_t vo = __shfl_sync(FULL_MASK, v, o);
                const uint64_t mo = kBatch ? __shfl_sync(FULL_MASK, (unsigned long long)mask, o) : 0ull;
                const int r = 4 * (q - xo);
                int4 x = make_int4(0, 0, 0, 0);
                if (q < total) {
                    x = __ldcs(reinterpret_cast<const int4*>(P.col + a4o + r));
                    okm |= unit_mask(r, lo_o, hi_o) << (4 * h);
                }
                u[4 * h + 0] = x.x;
                u[4 * h + 1] = x.y;
                u[4 * h + 2] = x.z;
                u[4 * h + 3] = x.w;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    vv[4 * h + c] = vo;
                    mm[4 * h + c] = mo;
                }
            }
            visit_k<kBatch, 8>(P, S, okm, u, vv, mm, level, nxt, nslot);
        }
        if (__popc(okb) < 32) break;
        i += 32;
    }
}

// Bin 2: one CTA per chunk of chunk_cta edges (a heavy vertex spans many
// chunks, hence many CTAs); the CTA's warps interleave over each segment.
template <bool kBatch, bool kStaged = false>
__device__ void expand_cta_chunk(const TraversalParams& P, Stage<kBatch>& S, int cur,
                                 long long item, int k, long long cnt, long long E, int level,
                                 int nxt, int nslot) {
    __shared__ long long s_eo[kBlock], s_base[kBlock], s_end[kBlock];
    __shared__ int32_t s_v[kBlock];
    __shared__ unsigned long long s_mask[kBatch ? kBlock : 1];
    const BinQueue& Q = P.q[cur][2];
    const int warp = threadIdx.x >> 5;
    const long long cs = item * k * (long long)P.chunk_cta;
    const long long ce = min(cs + k * (long long)P.chunk_cta, E);
    long long i = __ldcg(Q.chunk + item * k);
    for (;;) {
        const long long ij = i + threadIdx.x;
        long long eo = 0x7fffffffffffffffll;
        if (ij < cnt) eo = __ldcg(Q.eoff + ij);
        const bool ok = eo < ce;
        if (ok) {
            const int32_t v = __ldcg(Q.v + ij);
            s_v[threadIdx.x] = v;
            s_eo[threadIdx.x] = eo;
            const long long base = __ldg(P.off + v), end = __ldg(P.off + v + 1);
            s_base[threadIdx.x] = base;
            s_end[threadIdx.x] = end;
            if (!kLean && P.l2_prefetch) {
                const long long a = base + (max(eo, cs) - eo);
                const long long b = base + (min(eo + (end - base), ce) - eo);
                prefetch_cols_l2(P.col, a, min(b, a + kPrefetchAhead));
            }
            if (kBatch)
                s_mask[kBatch ? threadIdx.x : 0] =
                    __ldcg(reinterpret_cast<const unsigned long long*>(Q.mask) + ij);
        }
        const int nent = __syncthreads_count(ok);
        for (int k = 0; k < nent; ++k) {
            const long long eok = s_eo[k], bk = s_base[k];
            const long long lo = max(eok, cs), hi = min(eok + (s_end[k] - bk), ce);
            expand_segment<kBatch, kStaged>(P, S, bk + (lo - eok), bk + (hi - eok), s_v[k],
                                   kBatch ? s_mask[kBatch ? k : 0] : 0ull, level, nxt, nslot,
                                   (long long)warp * 256, 256ll * kWarps);
        }
        __syncthreads();
        if (nent < kBlock) break;
        i += kBlock;
    }
}

struct LevelShape {
    long long cnt[kBins], edges[kBins];
    long long n_cta;            // CTA items (bin 2)
    long long items_w1, items_w2;  // warp items of bins 1 and 2
    long long groups_small;     // light groups (bin 0)
    int k_cta;                  // base chunks per CTA item
    int sh_w1, sh_w2;           // log2 of the edges of a warp item of bins 1 and 2
    unsigned discovered;
};

__device__ __forceinline__ int pow2_floor_clamped(long long x, int kmax) {
    if (x <= 1) return 1;
    const int p = 63 - __clzll((unsigned long long)x);
    return p >= 31 ? kmax : min(1 << p, kmax);
}

// Shape of level `level` (frontier in slot level % 3, queues level & 1).
// Counts are clamped to the queue capacities so that a recorded overflow
// can never turn into an out-of-bounds read.
__device__ __forceinline__ LevelShape read_level(const TraversalParams& P, int level) {
    LevelShape s;
    const int slot = level % 3, cur = level & 1;
#pragma unroll
    for (int b = 0; b < kBins; ++b) {
        const unsigned long long p = ld_cg_u64(&P.ctl[slot].packed[b]);
        s.cnt[b] = min((long long)(p >> kCountShift), (long long)P.q[cur][b].cap);
        s.edges[b] = (long long)(p & kEdgeMask);
    }
    s.discovered = __ldcg(&P.ctl[slot].discovered);
    // base chunks (the granularity of the chunk tables), then work items of k
    // base chunks: small levels keep k = 1 so that every CTA / warp gets work,
    // large levels aim at ~4 items per CTA (or warp) to bound per-item costs
    const int sh_cta = __ffs(P.chunk_cta) - 1, sh_warp = __ffs(P.chunk_warp) - 1;
    const long long base_cta =
        min((s.edges[2] + P.chunk_cta - 1) >> sh_cta, (long long)P.q[cur][2].chunk_cap);
    const long long base_warp =
        min((s.edges[1] + P.chunk_warp - 1) >> sh_warp, (long long)P.q[cur][1].chunk_cap);
    s.k_cta = pow2_floor_clamped(base_cta / (4ll * gridDim.x), 32);
    const int k_warp = pow2_floor_clamped(base_warp / (4ll * gridDim.x * kWarps), 16);
    s.n_cta = (base_cta + s.k_cta - 1) / s.k_cta;
    s.items_w1 = (base_warp + k_warp - 1) / k_warp;
    s.sh_w1 = sh_warp + __ffs(k_warp) - 1;
    s.items_w2 = 0;
    s.sh_w2 = sh_cta;
    s.groups_small = (s.cnt[0] + 31) / 32;
    // Small levels: bins 1 and 2 cut into 32-edge warp slices when that,
    // with the light groups, still gives no warp more than one item.  The
    // level then costs one slice's chain of dependent accesses, where a
    // CTA chunk (1024 edges on 4 warps) or a warp chunk chained a probe
    // round and several flushes of its discoveries.
    const long long f1 = min((s.edges[1] + 31) >> 5, base_warp << (sh_warp - 5));
    const long long f2 = min((s.edges[2] + 31) >> 5, base_cta << (sh_cta - 5));
    if (f1 + f2 > 0 && f1 + f2 + s.groups_small <= (long long)gridDim.x * kWarps) {
        s.n_cta = 0;
        s.items_w1 = f1;
        s.items_w2 = f2;
        s.sh_w1 = s.sh_w2 = 5;
    }
    return s;
}

// One level's expansion.  CTA chunks (bin 2) are pulled from a counter so
// heavy vertices spread over whichever CTAs are free; warp items (bin 1
// chunks, then bin 0 groups) are equal-sized by construction and dealt out
// round robin over all warps of the grid, with no atomics or CTA barriers.
// Each warp flushes its staged discoveries at the end; the CTA adds its
// discovered-vertex count with one atomic.
// Bottom-up level (Section "Top Down Vs. Bottom Up"; the paper notes its
// exchange works with either direction): every vertex not yet visited looks
// for a neighbour in the current frontier bitmap and stops at the first.
// A warp owns one 32-vertex visited word at a time, so claims need no
// atomics.  Found vertices go through the same stage as top-down winners
// (distance level + 1, parent = the frontier neighbour, next frontier).
__device__ void bottom_up_level(const TraversalParams& P, Stage<false>& S, int level, int nxt,
                                int nslot) {
    const uint32_t* F = P.fb[level % 3];
    const unsigned lane = lane_id();
    const long long words = (P.bu_limit + 31) / 32;
    const long long nwarps = (long long)gridDim.x * kWarps;
    for (long long w = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5); w < words; w += nwarps) {
        const uint32_t vis = __ldcg(P.visited + w);
        const long long v = w * 32 + lane;
        const bool unv = v < P.bu_limit && !((vis >> lane) & 1u);
        if (__ballot_sync(FULL_MASK, unv) == 0u) continue;
        bool found = false;
        int32_t par = 0;
        if (unv) {
            long long k = __ldg(P.off + v);
            const long long e = __ldg(P.off + v + 1);
            for (; k + 4 <= e && !found; k += 4) {
                const int32_t u0 = __ldg(P.col + k), u1 = __ldg(P.col + k + 1);
                const int32_t u2 = __ldg(P.col + k + 2), u3 = __ldg(P.col + k + 3);
                const uint32_t f0 = F[u0 >> 5], f1 = F[u1 >> 5], f2 = F[u2 >> 5], f3 = F[u3 >> 5];
                if ((f0 >> (u0 & 31)) & 1u) { found = true; par = u0; }
                else if ((f1 >> (u1 & 31)) & 1u) { found = true; par = u1; }
                else if ((f2 >> (u2 & 31)) & 1u) { found = true; par = u2; }
                else if ((f3 >> (u3 & 31)) & 1u) { found = true; par = u3; }
            }
            for (; k < e && !found; ++k) {
                const int32_t u0 = __ldg(P.col + k);
                if ((F[u0 >> 5] >> (u0 & 31)) & 1u) { found = true; par = u0; }
            }
        }
        // the warp is the only one looking at word w, so the flush's claim of
        // a found vertex always wins
        stage_push<false>(P, S, found, (int32_t)v, par, 0ull, level, nxt, nslot);
    }
}

// Batched bottom-up level (a multi-source BFS over lane sets): every vertex
// that lacks some lane whose frontier is non-empty ORs the frontier lane
// sets of its neighbours and stops once it has every such lane.  Rows are
// scanned two ways: a warp scans one row 32 entries per step, OR-reducing
// the lane sets across the warp (the heavy vertices -- below `heavy_end`
// in the degree order, one vertex per warp spread over the grid -- and any
// heavy row met among the light ones), and a lane scans a light row four
// entries at a time.  The lanes found go to next[v] (each vertex has one
// owner, so no atomics) and the sweep turns them into distances and the
// next frontier, as after a top-down level.  Frontier sets are read past
// L1 (the previous level's sweep wrote them).
__device__ __forceinline__ uint64_t warp_scan_row(const unsigned long long* F, const int32_t* col,
                                                  long long k, long long e, uint64_t need) {
    const unsigned lane = lane_id();
    uint64_t found = 0ull;
    for (long long kk = k; kk < e; kk += 32) {
        uint64_t f = 0ull;
        if (kk + lane < e) f = __ldcg(F + __ldg(col + kk + lane));
        const unsigned lo = __reduce_or_sync(FULL_MASK, (unsigned)f);
        const unsigned hi = __reduce_or_sync(FULL_MASK, (unsigned)(f >> 32));
        found |= ((uint64_t)hi << 32) | lo;
        if ((found & need) == need) break;
    }
    return found;
}

__device__ void bottom_up_batch_level(const TraversalParams& P, int level) {
    const unsigned lane = lane_id();
    // only lanes whose frontier is non-empty can be found at this level; a
    // lane whose traversal has ended would otherwise keep every vertex it
    // never reaches scanning its whole row
    const uint64_t live = ld_cg_u64(&P.ctl[level % 3].front_lanes);
    const unsigned long long* F = reinterpret_cast<const unsigned long long*>(P.lane_front);
    unsigned long long* const vn = reinterpret_cast<unsigned long long*>(P.lane_vn);
    const long long nwarps = (long long)gridDim.x * kWarps;
    const long long gw = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const long long heavy_end = min(P.bitmap_from, P.bu_limit);
    for (long long v = gw; v < heavy_end; v += nwarps) {
        const uint64_t need = live & ~__ldcg(vn + 2 * v);
        if (need == 0ull) continue;
        const uint64_t found =
            warp_scan_row(F, P.col, __ldg(P.off + v), __ldg(P.off + v + 1), need);
        if (lane == 0 && (found & need) != 0ull) vn[2 * v + 1] = found & need;
    }
    const long long groups = (P.bu_limit - heavy_end + 31) / 32;
    for (long long w = gw; w < groups; w += nwarps) {
        const long long v = heavy_end + w * 32 + lane;
        uint64_t need = 0ull;
        long long k = 0, e = 0;
        if (v < P.bu_limit) {
            need = live & ~__ldcg(vn + 2 * v);
            if (need != 0ull) {
                k = __ldg(P.off + v);
                e = __ldg(P.off + v + 1);
            }
        }
        const bool heavy = e - k > 32;
        if (__ballot_sync(FULL_MASK, need != 0ull) == 0u) continue;
        uint64_t found = 0ull;
        if (need != 0ull && !heavy) {
            for (; k + 4 <= e; k += 4) {
                const int32_t u0 = __ldg(P.col + k), u1 = __ldg(P.col + k + 1);
                const int32_t u2 = __ldg(P.col + k + 2), u3 = __ldg(P.col + k + 3);
                found |= __ldcg(F + u0) | __ldcg(F + u1) | __ldcg(F + u2) | __ldcg(F + u3);
                if ((found & need) == need) break;
            }
            if ((found & need) != need)
                for (; k < e; ++k) {
                    found |= __ldcg(F + __ldg(P.col + k));
                    if ((found & need) == need) break;
                }
        }
        for (unsigned hm = __ballot_sync(FULL_MASK, need != 0ull && heavy); hm != 0u; hm &= hm - 1u) {
            const int src = __ffs(hm) - 1;
            const uint64_t hf = warp_scan_row(F, P.col, __shfl_sync(FULL_MASK, k, src),
                                              __shfl_sync(FULL_MASK, e, src),
                                              __shfl_sync(FULL_MASK, need, src));
            if ((int)lane == src) found = hf;
        }
        const uint64_t nx = found & need;
        if (nx != 0ull) vn[2 * v + 1] = nx;
    }
}

// Position of the set bit of rank n (0-based) in x, which has more than n
// set bits: the largest p with fewer than n + 1 set bits below p.
__device__ __forceinline__ int nth_set_bit(uint32_t x, int n) {
    int pos = 0;
#pragma unroll
    for (int st = 16; st > 0; st >>= 1)
        if (__popc(x & ((1u << (pos + st)) - 1u)) <= n) pos += st;
    return pos;
}

// Top-down over the frontier bitmap (dense levels, "queue -> bitmap"): the
// light bin (deg < t_small, most of the vertices) is read from the frontier
// bitmap instead of its queue.  A warp takes a tile of 32 bitmap words
// (1024 consecutive vertices); its light frontier vertices, in vertex order,
// are gathered 32 at a time and their rows cut into 16-byte units as in the
// warp bin.  After the degree-ordered renumbering the light vertices are
// one id range with adjacent rows, so a tile's column reads are close to
// one stream.  The heavier bins keep their (balanced) queues.
__device__ void expand_bitmap_tile(const TraversalParams& P, Stage<false>& S, long long tile,
                                   int level, int nxt, int nslot) {
    const uint32_t* F = P.fb[level % 3];
    const unsigned lane = lane_id();
    const long long words = (P.n + 31) / 32;
    const long long w = tile * 32 + lane;
    const uint32_t word = w < words ? __ldcg(F + w) : 0u;
    const int pc = __popc(word);
    const int pincl = warp_incl_scan(pc);
    const int pexcl = pincl - pc;
    const int nfront = __shfl_sync(FULL_MASK, pincl, 31);
    for (int k0 = 0; k0 < nfront; k0 += 32) {
        const int k = k0 + (int)lane;
        int o = 0;
#pragma unroll
        for (int st = 16; st > 0; st >>= 1) {
            const int c = o + st;
            if (__shfl_sync(FULL_MASK, pexcl, c & 31) <= k) o = c;
        }
        const uint32_t ow = __shfl_sync(FULL_MASK, word, o);
        const int oex = __shfl_sync(FULL_MASK, pexcl, o);
        bool ok = k < nfront;
        int32_t v = 0;
        long long a = 0, b = 0;
        if (ok) {
            const int bit = nth_set_bit(ow, k - oex);
            v = (int32_t)((tile * 32 + o) * 32 + bit);
            a = __ldg(P.off + v);
            b = __ldg(P.off + v + 1);
            if (b - a >= P.t_small || b == a) ok = false;
        }
        // unit gather over the (up to 32) rows
        const long long a4 = a & ~3ll;
        const int rlo = (int)(a - a4), rhi = (int)(b - a4);
        const int units = ok ? (rhi + 3) >> 2 : 0;
        const int incl = warp_incl_scan(units);
        const int excl = incl - units;
        const int total = __shfl_sync(FULL_MASK, incl, 31);
        for (int q0 = 0; q0 < total; q0 += 64) {
            unsigned okm = 0u;
            int32_t u[8], vv[8];
            uint64_t mm[8];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int q = q0 + 32 * h + (int)lane;
                int oo = 0;
#pragma unroll
                for (int st = 16; st > 0; st >>= 1) {
                    const int c = oo + st;
                    if (__shfl_sync(FULL_MASK, excl, c & 31) <= q) oo = c;
                }
                const long long a4o = __shfl_sync(FULL_MASK, a4, oo);
                const int lo_o = __shfl_sync(FULL_MASK, rlo, oo);
                const int hi_o = __shfl_sync(FULL_MASK, rhi, oo);
                const int xo = __shfl_sync(FULL_MASK, excl, oo);
                const int32_t vo = __shfl_sync(FULL_MASK, v, oo);
                const int r = 4 * (q - xo);
                int4 x = make_int4(0, 0, 0, 0);
                if (q < total) {
                    x = __ldcs(reinterpret_cast<const int4*>(P.col + a4o + r));
                    okm |= unit_mask(r, lo_o, hi_o) << (4 * h);
                }
                u[4 * h + 0] = x.x;
                u[4 * h + 1] = x.y;
                u[4 * h + 2] = x.z;
                u[4 * h + 3] = x.w;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    vv[4 * h + c] = vo;
                    mm[4 * h + c] = 0ull;
                }
            }
            visit_k<false, 8>(P, S, okm, u, vv, mm, level, nxt, nslot);
        }
    }
}

// Top-down work of one level: CTA chunks of bin 2 pulled from a counter
// (heavy vertices spread over whichever CTAs are free), then warp items
// (bin 1 chunks, bin 0 groups) dealt round robin over all warps of the grid.
template <bool kBatch, bool kStaged = false>
__device__ void expand_top_down(const TraversalParams& P, Stage<kBatch>& S, const LevelShape& L,
                                int level, bool bitmap = false) {
    __shared__ long long s_item;
    const int slot = level % 3, nslot = (level + 1) % 3;
    const int cur = level & 1, nxt = cur ^ 1;
    const int warp = threadIdx.x >> 5;
    if (L.n_cta > 0) {
        for (;;) {
            if (threadIdx.x == 0) s_item = (long long)atomicAdd(&P.ctl[slot].work, 1u);
            __syncthreads();
            const long long item = s_item;
            __syncthreads();
            if (item >= L.n_cta) break;
            expand_cta_chunk<kBatch, kStaged>(P, S, cur, item, L.k_cta, L.cnt[2], L.edges[2], level, nxt,
                                     nslot);
        }
    }
    const long long nwarps = (long long)gridDim.x * kWarps;
    const long long gw = (long long)blockIdx.x * kWarps + warp;
    // bitmap mode: the light bin's groups are replaced by bitmap tiles
    // starting at the first tile that can hold a light vertex
    long long tile0 = 0, tiles = 0;
    if (!kLean && !kBatch && bitmap) {
        tile0 = P.bitmap_from / 1024;
        tiles = ((P.n + 31) / 32 + 31) / 32 - tile0;
    }
    const long long small_items = (!kLean && !kBatch && bitmap) ? tiles : L.groups_small;
    const long long w1 = L.items_w1, w12 = w1 + L.items_w2;
    const long long witems = w12 + small_items;
    const int sh_warp = __ffs(P.chunk_warp) - 1, sh_cta = __ffs(P.chunk_cta) - 1;
    for (long long it = gw; it < witems; it += nwarps) {
        if (it < w12) {
            const bool b2 = it >= w1;
            const int shw = b2 ? L.sh_w2 : L.sh_w1;
            const long long cs = (b2 ? it - w1 : it) << shw;
            const long long E = b2 ? L.edges[2] : L.edges[1];
            expand_warp_range<kBatch>(P, S, P.q[cur][b2 ? 2 : 1], b2 ? sh_cta : sh_warp, cs,
                                      min(cs + (1ll << shw), E), b2 ? L.cnt[2] : L.cnt[1], level,
                                      nxt, nslot);
        } else if constexpr (!kBatch) {
            if (!kLean && bitmap)
                expand_bitmap_tile(P, S, tile0 + (it - w12), level, nxt, nslot);
            else
                expand_small_group<kBatch>(P, S, cur, it - w12, L.cnt[0], level, nxt, nslot);
        } else {
            expand_small_group<kBatch>(P, S, cur, it - w12, L.cnt[0], level, nxt, nslot);
        }
    }
}

template <bool kBatch, bool kStaged = false>
__device__ void expand_level(const TraversalParams& P, Stage<kBatch>& S, const LevelShape& L,
                             int level, uint32_t* s_hot, int dir = 0) {
    __shared__ int s_disc;
    const int nslot = (level + 1) % 3;
    const int nxt = (level & 1) ^ 1;
    if (threadIdx.x == 0) s_disc = 0;
    if (lane_id() == 0) S.disc = 0;
    if (!kBatch) {
        // large levels: copy the hot prefix of the visited bitmap (after the
        // degree-ordered renumbering, the highest-degree vertices) into
        // shared memory; most probes of a dense level end there
        const long long ledges = L.edges[0] + L.edges[1] + L.edges[2];
        const int words = (!kLean && P.hot_words > 0 && ledges >= P.hot_min_edges)
                              ? (int)min((long long)P.hot_words, (long long)((P.n + 31) / 32)) : 0;
        if (words > 0) {
            const int w4 = words / 4;
            const uint4* src = reinterpret_cast<const uint4*>(P.visited);
            uint4* dst = reinterpret_cast<uint4*>(s_hot);
            for (int i = threadIdx.x; i < w4; i += kBlock) dst[i] = __ldcg(src + i);
            for (int i = w4 * 4 + threadIdx.x; i < words; i += kBlock) s_hot[i] = __ldcg(P.visited + i);
        }
        if (lane_id() == 0) {
            S.hot = s_hot;
            S.hot_bits = words * 32;
        }
    }
    __syncthreads();
    bool bottom_up = false;
    if (!kLean && dir == 2) {
        if constexpr (kBatch) bottom_up_batch_level(P, level);
        else bottom_up_level(P, S, level, nxt, nslot);
        bottom_up = true;
    }
    if (!bottom_up) expand_top_down<kBatch, kStaged>(P, S, L, level, dir == 1);
    stage_flush<kBatch>(P, S, level, nxt, nslot);
    if (!kBatch) {
        if (lane_id() == 0 && S.disc > 0) atomicAdd(&s_disc, S.disc);
        __syncthreads();
        if (threadIdx.x == 0 && s_disc > 0) atomicAdd(&P.ctl[nslot].discovered, (unsigned)s_disc);
    }
}

// ------------------------------------------------------------- init/seed
// Byte-uniform fill (0x00 or 0xff patterns): scalar bytes up to a 16-byte
// boundary, 16-byte stores for the body, scalar bytes for the tail.
__device__ void fill_bytes(void* ptr, long long nbytes, unsigned char value, long long tid,
                           long long nthreads) {
    unsigned char* p = static_cast<unsigned char*>(ptr);
    const long long head = min(nbytes, (long long)((16 - ((uintptr_t)p & 15)) & 15));
    for (long long i = tid; i < head; i += nthreads) p[i] = value;
    const long long nvec = (nbytes - head) / 16;
    int4* pv = reinterpret_cast<int4*>(p + head);
    const int w = (int)(value * 0x01010101u);
    const int4 v4 = make_int4(w, w, w, w);
    for (long long i = tid; i < nvec; i += nthreads) pv[i] = v4;
    for (long long i = head + nvec * 16 + tid; i < nbytes; i += nthreads) p[i] = value;
}

__device__ void fill_u64(uint64_t* p, long long n, long long tid, long long nthreads) {
    for (long long i = tid; i < n; i += nthreads) p[i] = 0ull;
}

__device__ void init_plain(const TraversalParams& P, long long tid, long long nthreads) {
    if (blockIdx.x == 0 && threadIdx.x < 3 * (int)(sizeof(LevelCtl) / 8))
        reinterpret_cast<unsigned long long*>(P.ctl)[threadIdx.x] = 0ull;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        P.stats->levels = 0;
        P.stats->reached = 0;
        P.stats->edges = 0;
        P.stats->status = 0;
        P.stats->max_level = 0;
        P.stats->bu_levels = 0;
        P.stats->graph_seen = 0;
        P.stats->graph_level = 0;
        P.stats->graph_prev_bu = 0;
        P.stats->graph_dir = 0;
    }
    const long long words = (P.n + 31) / 32;
    fill_bytes(P.visited, words * 4, 0, tid, nthreads);
    if (!kLean && P.fb[0])
        for (int f = 0; f < 3; ++f) fill_bytes(P.fb[f], words * 4, 0, tid, nthreads);
    fill_bytes(P.dist, P.n * 4, 0xff, tid, nthreads);
    if (P.parent) fill_bytes(P.parent, P.n * 4, 0xff, tid, nthreads);
}

__device__ void seed_plain(const TraversalParams& P, Stage<false>& S) {
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    const bool l0 = threadIdx.x == 0;
    const int32_t root = P.old2new ? __ldg(P.old2new + P.root_caller) : P.root_caller;
    if (l0) P.ctl[0].discovered = 1u;
    // staged with level -1 and itself as parent: the flush writes dist 0 and
    // parent = root, and queues the root in the bin of its degree
    stage_push<false>(P, S, l0, root, root, 0ull, -1, 0, 0);
    stage_flush<false>(P, S, -1, 0, 0);
}

// Per-level housekeeping of the frontier bitmaps: the bitmap the level after
// next will fill is cleared now (it held the previous level's frontier);
// bottom-up levels are counted.
__device__ void prepare_level(const TraversalParams& P, int level, int dir, long long tid,
                              long long nthreads) {
    if (kLean || !P.fb[0]) return;
    fill_bytes(P.fb[(level + 2) % 3], ((P.n + 31) / 32) * 4, 0, tid, nthreads);
    if (dir == 2 && blockIdx.x == 0 && threadIdx.x == 0) P.stats->bu_levels += 1;
}

// Books the level that is about to be expanded; block 0, thread 0 only.
__device__ void book_level(const TraversalParams& P, const LevelShape& S, int level) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    // clear the slot that the level after next will fill
    unsigned long long* z = reinterpret_cast<unsigned long long*>(P.ctl + (level + 2) % 3);
    for (int i = 0; i < (int)(sizeof(LevelCtl) / 8); ++i) z[i] = 0ull;
    if (S.discovered > 0) {
        P.stats->levels = level + 1;
        P.stats->reached += S.discovered;
    }
    P.stats->edges += S.edges[0] + S.edges[1] + S.edges[2];
}

// Direction of a batched level: bottom-up when the frontier's degree sum
// exceeds the degree sum of the vertices some lane has not reached yet plus
// 4 entries per vertex (a bottom-up level reads every vertex's lane sets),
// decided afresh each level.  Unlike the single-source rule (Beamer et al.,
// alpha 15 / beta 18) a bottom-up vertex stops only once it has every lane
// it lacks, not at its first frontier neighbour, so bottom-up pays off only
// on the levels whose frontiers cover most of the graph.
__device__ __forceinline__ int batch_direction(const TraversalParams& P, const LevelShape& L,
                                               bool prev_bu) {
    (void)prev_bu;
    if (P.dir_mode == 0) return 0;
    if (P.dir_mode == 2) return 2;
    const long long mf = L.edges[0] + L.edges[1] + L.edges[2];
    const long long full = (long long)ld_cg_u64(
        reinterpret_cast<const unsigned long long*>(&P.stats->full_edges));
    return mf > P.nnz - full + 4 * P.n ? 2 : 0;
}

// ------------------------------------------- graph-captured level loop
// End of one loop-body launch (one CTA, thread 0): carry the direction
// state to the next level and set the while node's condition -- 0 when the
// next frontier is empty (its discoveries of degree-0 vertices are booked
// first, as the device-side loop does) or the launch failed.
__device__ void graph_advance_plain(const TraversalParams& P) {
    if (threadIdx.x != 0) return;
    DevStats* st = P.stats;
    const int level = st->graph_level;
    const int slot = level % 3, nslot = (level + 1) % 3;
    long long mf = 0, nf_next = 0;
#pragma unroll
    for (int b = 0; b < kBins; ++b) {
        mf += (long long)(ld_cg_u64(&P.ctl[slot].packed[b]) & kEdgeMask);
        nf_next += (long long)(ld_cg_u64(&P.ctl[nslot].packed[b]) >> kCountShift);
    }
    st->graph_seen += mf;
    st->graph_prev_bu = st->graph_dir == 2 ? 1 : 0;
    st->graph_level = level + 1;
    unsigned go = 1u;
    if (nf_next == 0 || ld_volatile_i32(&st->status) != 0) {
        if (nf_next == 0) book_level(P, read_level(P, level + 1), level + 1);
        go = 0u;
    }
    cudaGraphSetConditional(P.graph_cond, go);
}

// Batched body end: records the level count, applies the int8 depth limit
// and sets the while node's condition for the next level.
__device__ void graph_advance_batch(const TraversalParams& P) {
    if (threadIdx.x != 0) return;
    DevStats* st = P.stats;
    const int level = st->graph_level;
    const int nslot = (level + 1) % 3;
    if (ld_cg_u64(reinterpret_cast<const unsigned long long*>(&P.ctl[nslot].new_lanes)) > 0ull)
        st->levels = level + 2;
    long long nf_next = 0;
#pragma unroll
    for (int b = 0; b < kBins; ++b)
        nf_next += (long long)(ld_cg_u64(&P.ctl[nslot].packed[b]) >> kCountShift);
    st->graph_level = level + 1;
    st->graph_prev_bu = st->graph_dir == 2 ? 1 : 0;
    unsigned go = (nf_next > 0 && ld_volatile_i32(&st->status) == 0) ? 1u : 0u;
    if (go && P.dist_int8 && level + 2 > 126) {
        raise_status(P, kDevDepth);
        go = 0u;
    }
    cudaGraphSetConditional(P.graph_cond, go);
}

// --------------------------------------------------------- plain kernels
// kStaged: heavy runs go through the TMA staging buffers (BFS_OPT_TMA_STAGE);
// a separate instantiation, so the default kernel carries none of that code.
template <int MB, bool kStaged>
__global__ void __launch_bounds__(kBlock, MB)
bfs_plain_persistent(const __grid_constant__ TraversalParams P) {
    extern __shared__ uint4 s_dyn[];
    uint32_t* s_hot = reinterpret_cast<uint32_t*>(s_dyn);
    __shared__ Stage<false> s_stage[kWarps];
    Stage<false>& S = s_stage[threadIdx.x >> 5];
    stage_init(S);
    if (kStaged) tma_setup(P, S, s_dyn);
    const long long nthreads = (long long)gridDim.x * kBlock;
    const long long tid = (long long)blockIdx.x * kBlock + threadIdx.x;
    // a failed validation launch (same stream, so its result is visible to
    // every CTA) ends the traversal before anything reads the graph
    if (P.pre_status && ld_volatile_i32(P.pre_status) != 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) raise_status(P, ld_volatile_i32(P.pre_status));
        kernel_exit(P);
        return;
    }
    stamp(P, 0);
    init_plain(P, tid, nthreads);
    __shared__ unsigned long long epoch;
    if (threadIdx.x == 0) epoch = 0ull;
    if (grid_barrier(P, epoch)) {
        stamp(P, 1);
        seed_plain(P, S);
        if (grid_barrier(P, epoch)) {
            stamp(P, 2);
            long long seen_edges = 0;  // edges of all frontiers so far (same in every CTA)
            bool prev_bu = false;
            for (int level = 0;; ++level) {
                const LevelShape L = read_level(P, level);
                book_level(P, L, level);
                const long long nf = L.cnt[0] + L.cnt[1] + L.cnt[2];
                if (nf == 0) break;
                const long long mf = L.edges[0] + L.edges[1] + L.edges[2];
                seen_edges += mf;
                const int dir = (!kLean && P.fb[0]) ? choose_direction(P.dir_mode, prev_bu, mf, P.nnz - seen_edges,
                                                           nf, P.n, P.do_alpha, P.do_beta,
                                                           P.bitmap_div)
                                        : 0;
                prepare_level(P, level, dir, tid, nthreads);
                expand_level<false, kStaged>(P, S, L, level, s_hot, dir);
                prev_bu = dir == 2;
                if (!grid_barrier(P, epoch)) break;
                stamp(P, 3 + level);
            }
        }
    }
    kernel_exit(P);
}

// Host-loop variant: one launch per phase / level, no grid barrier.
template <int MB, bool kStaged>
__global__ void __launch_bounds__(kBlock, MB)
bfs_plain_step(const __grid_constant__ TraversalParams P) {
    extern __shared__ uint4 s_dyn[];
    uint32_t* s_hot = reinterpret_cast<uint32_t*>(s_dyn);
    __shared__ Stage<false> s_stage[kWarps];
    Stage<false>& S = s_stage[threadIdx.x >> 5];
    stage_init(S);
    if (kStaged) tma_setup(P, S, s_dyn);
    const long long nthreads = (long long)gridDim.x * kBlock;
    const long long tid = (long long)blockIdx.x * kBlock + threadIdx.x;
    if (P.phase == 0) {
        init_plain(P, tid, nthreads);
    } else if (P.phase == 1) {
        seed_plain(P, S);
    } else if (P.phase == 2) {
        const LevelShape L = read_level(P, P.level);
        book_level(P, L, P.level);
        if (L.cnt[0] + L.cnt[1] + L.cnt[2] == 0) return;
        const int dir = (P.fb[0] && P.dir_override > 0) ? P.dir_override : 0;
        prepare_level(P, P.level, dir, tid, nthreads);
        expand_level<false, kStaged>(P, S, L, P.level, s_hot, dir);
    } else if (P.phase == 5) {
        // graph-captured loop body: the level and the direction state come
        // from the device (written by the previous body launch)
        const int level = ld_volatile_i32(&P.stats->graph_level);
        const LevelShape L = read_level(P, level);
        book_level(P, L, level);
        const long long nf = L.cnt[0] + L.cnt[1] + L.cnt[2];
        if (nf == 0) return;
        const long long mf = L.edges[0] + L.edges[1] + L.edges[2];
        const long long seen = *(volatile long long*)&P.stats->graph_seen + mf;
        const int dir = P.fb[0] ? choose_direction(P.dir_mode,
                                                   ld_volatile_i32(&P.stats->graph_prev_bu) != 0,
                                                   mf, P.nnz - seen, nf, P.n, P.do_alpha,
                                                   P.do_beta, P.bitmap_div)
                                : 0;
        if (blockIdx.x == 0 && threadIdx.x == 0) P.stats->graph_dir = dir;
        prepare_level(P, level, dir, tid, nthreads);
        expand_level<false, kStaged>(P, S, L, level, s_hot, dir);
    } else if (P.phase == 6) {
        graph_advance_plain(P);
    }
}

// ------------------------------------------------------- batched kernels
__device__ void init_batch(const TraversalParams& P, long long tid, long long nthreads) {
    if (blockIdx.x == 0 && threadIdx.x < 3 * (int)(sizeof(LevelCtl) / 8))
        reinterpret_cast<unsigned long long*>(P.ctl)[threadIdx.x] = 0ull;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        P.stats->levels = 0;
        P.stats->reached = 0;
        P.stats->edges = 0;
        P.stats->status = 0;
        P.stats->max_level = 0;
        P.stats->bu_levels = 0;
        P.stats->graph_level = 0;
        P.stats->graph_seen = 0;
        P.stats->graph_prev_bu = 0;
        P.stats->graph_dir = 0;
        P.stats->full_edges = 0;
    }
    fill_u64(P.lane_vn, 2 * P.n, tid, nthreads);
    if (P.dir_mode != 0) fill_u64(P.lane_front, P.n, tid, nthreads);
    // distances are not filled here: emit_batch writes every (lane, vertex)
}

// Level of lane i at vertex v, one byte per lane in a vertex-major array
// (64 bytes per vertex): a sweep's writes for one vertex stay inside its own
// two sectors.  255 means "level >= 255, written straight into dist".
__device__ __forceinline__ void record_lane_level(const TraversalParams& P, int lane_idx,
                                                  long long v, int32_t cv, int level) {
    if (level < 255) {
        P.lane_level[v * 64 + lane_idx] = (uint8_t)level;
    } else {
        P.lane_level[v * 64 + lane_idx] = 255;
        const long long idx = (long long)lane_idx * P.n + cv;
        if (P.dist_int8) reinterpret_cast<int8_t*>(P.dist)[idx] = (int8_t)level;
        else P.dist[idx] = level;
    }
}

// After the last level: dist rows in the caller's numbering, one thread per
// caller vertex (coalesced stores in every row); unreached lanes get -1.
// Caller-order rows from the per-vertex level rows.  Four consecutive
// caller vertices per thread: each lane row gets one 16-byte (int32) or
// 4-byte (int8) store covering all four, when the row starts keep that
// alignment (n a multiple of 4, dist 16-byte aligned); otherwise one store
// per value.  A level byte of 255 marks a lane whose level (>= 255) was
// written straight into dist: such values are left as they are.
__device__ __forceinline__ uint32_t level_byte(const uint4& r, int b) {
    const uint32_t w = b < 4 ? r.x : b < 8 ? r.y : b < 12 ? r.z : r.w;
    return (w >> (8 * (b & 3))) & 0xffu;
}

__device__ void emit_batch(const TraversalParams& P, long long tid, long long nthreads) {
    const bool vec = (P.n & 3) == 0 && ((uintptr_t)P.dist & 15) == 0;
    if (vec) {
        const long long groups = P.n >> 2;
        for (long long g = tid; g < groups; g += nthreads) {
            const long long c0 = g << 2;
            uint64_t vis[4];
            const uint4* lv[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const long long v = P.old2new ? __ldg(P.old2new + c0 + j) : c0 + j;
                vis[j] = __ldcg(reinterpret_cast<const unsigned long long*>(P.lane_vn) + 2 * v);
                lv[j] = reinterpret_cast<const uint4*>(P.lane_level + v * 64);
            }
#pragma unroll 1
            for (int k = 0; k < 4 && 16 * k < P.nlanes; ++k) {
                uint4 r[4];
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    r[j] = vis[j] ? __ldcg(lv[j] + k) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                for (int b = 0; b < 16; ++b) {
                    const int i = 16 * k + b;
                    if (i >= P.nlanes) break;
                    int val[4];
                    bool deep = false;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const bool hit = (vis[j] >> i) & 1ull;
                        const int lvl = (int)level_byte(r[j], b);
                        deep |= hit && lvl == 255;
                        val[j] = hit ? lvl : -1;
                    }
                    const long long idx = (long long)i * P.n + c0;
                    if (!deep) {
                        if (P.dist_int8)
                            *reinterpret_cast<uint32_t*>(reinterpret_cast<int8_t*>(P.dist) + idx) =
                                (uint32_t)(val[0] & 0xff) | ((uint32_t)(val[1] & 0xff) << 8) |
                                ((uint32_t)(val[2] & 0xff) << 16) | ((uint32_t)(val[3] & 0xff) << 24);
                        else
                            *reinterpret_cast<int4*>(P.dist + idx) =
                                make_int4(val[0], val[1], val[2], val[3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            if (((vis[j] >> i) & 1ull) && val[j] == 255) continue;
                            if (P.dist_int8) reinterpret_cast<int8_t*>(P.dist)[idx + j] = (int8_t)val[j];
                            else P.dist[idx + j] = val[j];
                        }
                    }
                }
            }
        }
        return;
    }
    for (long long c = tid; c < P.n; c += nthreads) {
        const long long v = P.old2new ? __ldg(P.old2new + c) : c;
        const uint64_t vis = __ldcg(reinterpret_cast<const unsigned long long*>(P.lane_vn) + 2 * v);
        const uint4* lv = reinterpret_cast<const uint4*>(P.lane_level + v * 64);
        for (int k = 0; k < 4 && 16 * k < P.nlanes; ++k) {
            const uint4 r = vis ? __ldcg(lv + k) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
            for (int b = 0; b < 16; ++b) {
                const int i = 16 * k + b;
                if (i >= P.nlanes) break;
                const bool hit = (vis >> i) & 1ull;
                const int lvl = (int)level_byte(r, b);
                if (hit && lvl == 255) continue;  // deep level, already written
                const int val = hit ? lvl : -1;
                const long long idx = (long long)i * P.n + c;
                if (P.dist_int8) reinterpret_cast<int8_t*>(P.dist)[idx] = (int8_t)val;
                else P.dist[idx] = val;
            }
        }
    }
}


// One warp seeds all roots: duplicates share one queue entry whose mask
// holds every lane with that root.
__device__ void seed_batch(const TraversalParams& P, Stage<true>& S) {
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    const unsigned lane = lane_id();
    for (int base = 0; base < P.nlanes; base += 32) {
        const int i = base + (int)lane;
        bool first = false;
        int32_t r = 0;
        uint64_t mask = 0ull;
        if (i < P.nlanes) {
            const int32_t cr = P.roots[i];
            first = true;
            for (int j = 0; j < P.nlanes; ++j) {
                if (P.roots[j] == cr) {
                    mask |= 1ull << j;
                    if (j < i) first = false;
                }
            }
            r = P.old2new ? __ldg(P.old2new + cr) : cr;
            record_lane_level(P, i, r, cr, 0);
            if (first) {
                P.lane_vn[2 * (long long)r] = mask;
                if (P.dir_mode != 0) P.lane_front[r] = mask;
            }
        }
        stage_push<true>(P, S, first, r, 0, mask, -1, 0, 0);
    }
    stage_flush<true>(P, S, -1, 0, 0);
    if (lane == 0) {
        P.ctl[0].front_lanes = P.nlanes >= 64 ? ~0ull : ((1ull << P.nlanes) - 1ull);
        P.stats->reached = P.nlanes;
        P.stats->edges = (long long)S.edges;
        P.stats->levels = 1;
        S.edges = 0ull;
    }
    __syncwarp();
}

// Phase B of a batched level: lanes that reached v for the first time get
// distance level + 1 and make v part of the next frontier with those lanes.
// Byte i of the result is 0xff when bit i of m (8 bits) is set: the bits
// are spread to one per byte by three shift-or-mask steps, then each 0x01
// byte is multiplied up to 0xff (no carries between bytes).
__device__ __forceinline__ unsigned long long byte_mask_of_bits(unsigned m) {
    unsigned long long x = m & 0xffu;
    x = (x | (x << 28)) & 0x0000000f0000000full;
    x = (x | (x << 14)) & 0x0003000300030003ull;
    x = (x | (x << 7)) & 0x0101010101010101ull;
    return x * 0xffull;
}

__device__ void sweep_batch(const TraversalParams& P, Stage<true>& S, int level, long long tid,
                            long long nthreads) {
    const int nslot = (level + 1) % 3, nxt = (level + 1) & 1;
    const unsigned lane = lane_id();
    long long my_pairs = 0, my_full = 0;
    unsigned long long my_front = 0ull;  // lanes with a vertex in the next frontier
    const uint64_t all_lanes = P.nlanes >= 64 ? ~0ull : ((1ull << P.nlanes) - 1ull);
    // kSweepUnroll vertices per thread and pass, their lane-set pairs loaded
    // together; the trip count is the same for every thread (the stage push
    // is warp-collective)
    constexpr int kSweepUnroll = 4;
    const long long stride = nthreads * kSweepUnroll;
    const long long nround = (P.n + stride - 1) / stride * stride;
    ulonglong2* const pairs = reinterpret_cast<ulonglong2*>(P.lane_vn);
    for (long long v0 = tid; v0 < nround; v0 += stride) {
        ulonglong2 vnu[kSweepUnroll];
#pragma unroll
        for (int x = 0; x < kSweepUnroll; ++x) {
            const long long v = v0 + x * nthreads;
            vnu[x] = v < P.n ? __ldcg(pairs + v) : make_ulonglong2(0ull, 0ull);
        }
#pragma unroll
        for (int x = 0; x < kSweepUnroll; ++x) {
            const long long v = v0 + x * nthreads;
            uint64_t fresh = 0ull;
            bool reached_before = false;  // some lane had reached v at an earlier level
            if (v < P.n) {
                const ulonglong2 vn = vnu[x];
                if (vn.y != 0ull) {
                    fresh = vn.y & ~vn.x;
                    reached_before = vn.x != 0ull;
                    pairs[v] = make_ulonglong2(vn.x | fresh, 0ull);
                    my_pairs += __popcll(fresh);
                    // bottom-up bookkeeping: edges of vertices every lane has now reached
                    if (P.dir_mode != 0 && fresh != 0ull && (vn.x | fresh) == all_lanes)
                        my_full += __ldg(P.off + v + 1) - __ldg(P.off + v);
                }
                if (P.dir_mode != 0) P.lane_front[v] = fresh;
                my_front |= fresh;
            }
            // levels: one read-modify-write of the vertex's 64-byte level row
            // (16-byte accesses, consecutive vertices' rows adjacent), bytes of
            // the new lanes set to level + 1; bytes of lanes not reached yet are
            // never read, so a first visit skips the read
            if (fresh != 0ull) {
                uint4* row = reinterpret_cast<uint4*>(P.lane_level + v * 64);
                uint4 q[4];
    #pragma unroll
                for (int k = 0; k < 4; ++k)
                    q[k] = reached_before ? __ldcg(row + k) : make_uint4(0, 0, 0, 0);
                const int lvl = level + 1 < 255 ? level + 1 : 255;
                const unsigned long long lvl8 = (unsigned long long)lvl * 0x0101010101010101ull;
                unsigned long long* w = reinterpret_cast<unsigned long long*>(q);
    #pragma unroll
                for (int g = 0; g < 8; ++g) {
                    const unsigned long long bm = byte_mask_of_bits((unsigned)(fresh >> (8 * g)) & 0xffu);
                    w[g] = (w[g] & ~bm) | (lvl8 & bm);
                }
    #pragma unroll
                for (int k = 0; k < 4; ++k) row[k] = q[k];
                if (level + 1 >= 255) {
                    // deep levels: the distance goes straight to the output
                    const int32_t cv = P.new2old ? __ldg(P.new2old + v) : (int32_t)v;
                    for (unsigned long long f = fresh; f != 0ull; f &= f - 1ull) {
                        const long long idx = (long long)(__ffsll((long long)f) - 1) * P.n + cv;
                        if (P.dist_int8) reinterpret_cast<int8_t*>(P.dist)[idx] = (int8_t)(level + 1);
                        else P.dist[idx] = level + 1;
                    }
                }
            }
            stage_push<true>(P, S, fresh != 0ull, (int32_t)(v < P.n ? v : 0), 0, fresh, level, nxt,
                             nslot);
        }
    }
    stage_flush<true>(P, S, level, nxt, nslot);
    if (P.dir_mode != 0) {
        my_full = warp_incl_scan(my_full);
        if (lane == 31 && my_full > 0)
            atomicAdd(reinterpret_cast<unsigned long long*>(&P.stats->full_edges),
                      (unsigned long long)my_full);
        const unsigned flo = __reduce_or_sync(FULL_MASK, (unsigned)my_front);
        const unsigned fhi = __reduce_or_sync(FULL_MASK, (unsigned)(my_front >> 32));
        const unsigned long long fr = ((unsigned long long)fhi << 32) | flo;
        if (lane == 0 && fr != 0ull) atomicOr(&P.ctl[nslot].front_lanes, fr);
    }
    my_pairs = warp_incl_scan(my_pairs);
    if (lane == 31 && my_pairs > 0) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&P.ctl[nslot].new_lanes),
                  (unsigned long long)my_pairs);
        atomicAdd(reinterpret_cast<unsigned long long*>(&P.stats->reached),
                  (unsigned long long)my_pairs);
    }
    if (lane == 0 && S.edges != 0ull) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&P.stats->edges), S.edges);
        S.edges = 0ull;
    }
    __syncwarp();
}

__device__ void book_batch_level(const TraversalParams& P, int level) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    unsigned long long* z = reinterpret_cast<unsigned long long*>(P.ctl + (level + 2) % 3);
    for (int i = 0; i < (int)(sizeof(LevelCtl) / 8); ++i) z[i] = 0ull;
}

template <int MB>
__global__ void __launch_bounds__(kBlock, MB)
bfs_batch_persistent(const __grid_constant__ TraversalParams P) {
    __shared__ Stage<true> s_stage[kWarps];
    Stage<true>& S = s_stage[threadIdx.x >> 5];
    stage_init(S);
    const long long nthreads = (long long)gridDim.x * kBlock;
    const long long tid = (long long)blockIdx.x * kBlock + threadIdx.x;
    stamp(P, 0);
    init_batch(P, tid, nthreads);
    __shared__ unsigned long long epoch;
    if (threadIdx.x == 0) epoch = 0ull;
    if (grid_barrier(P, epoch)) {
        stamp(P, 1);
        seed_batch(P, S);
        if (grid_barrier(P, epoch)) {
            stamp(P, 2);
            bool prev_bu = false;
            for (int level = 0;; ++level) {
                const LevelShape L = read_level(P, level);
                if (L.cnt[0] + L.cnt[1] + L.cnt[2] == 0) break;
                if (P.dist_int8 && level + 1 > 126) {
                    if (blockIdx.x == 0 && threadIdx.x == 0) raise_status(P, kDevDepth);
                    break;
                }
                book_batch_level(P, level);
                const int dir = batch_direction(P, L, prev_bu);
                if (dir == 2 && blockIdx.x == 0 && threadIdx.x == 0) P.stats->bu_levels += 1;
                expand_level<true>(P, S, L, level, nullptr, dir);
                prev_bu = dir == 2;
                if (!grid_barrier(P, epoch)) break;
                stamp(P, 3 + 2 * level);
                sweep_batch(P, S, level, tid, nthreads);
                if (!grid_barrier(P, epoch)) break;
                stamp(P, 4 + 2 * level);
                if (blockIdx.x == 0 && threadIdx.x == 0) {
                    if (__ldcg(reinterpret_cast<const unsigned long long*>(
                            &P.ctl[(level + 1) % 3].new_lanes)) > 0ull)
                        P.stats->levels = level + 2;
                }
            }
            // every sweep is complete here (the loop exits right after a barrier
            // or before any expansion of an empty level)
            if (ld_volatile_i32(&P.stats->abort) == 0) emit_batch(P, tid, nthreads);
        }
    }
    kernel_exit(P);
}

template <int MB>
__global__ void __launch_bounds__(kBlock, MB)
bfs_batch_step(const __grid_constant__ TraversalParams P) {
    __shared__ Stage<true> s_stage[kWarps];
    Stage<true>& S = s_stage[threadIdx.x >> 5];
    stage_init(S);
    const long long nthreads = (long long)gridDim.x * kBlock;
    const long long tid = (long long)blockIdx.x * kBlock + threadIdx.x;
    if (P.phase == 0) {
        init_batch(P, tid, nthreads);
    } else if (P.phase == 1) {
        seed_batch(P, S);
    } else if (P.phase == 2) {
        const LevelShape L = read_level(P, P.level);
        if (L.cnt[0] + L.cnt[1] + L.cnt[2] == 0) return;
        book_batch_level(P, P.level);
        expand_level<true>(P, S, L, P.level, nullptr);
    } else if (P.phase == 3) {
        sweep_batch(P, S, P.level, tid, nthreads);
    } else if (P.phase == 4) {
        emit_batch(P, tid, nthreads);
    } else if (P.phase == 7) {
        // graph-captured loop body: expansion of the device's current level
        const int level = ld_volatile_i32(&P.stats->graph_level);
        const LevelShape L = read_level(P, level);
        if (L.cnt[0] + L.cnt[1] + L.cnt[2] == 0) return;
        book_batch_level(P, level);
        const int dir = batch_direction(P, L, ld_volatile_i32(&P.stats->graph_prev_bu) != 0);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            P.stats->graph_dir = dir;
            if (dir == 2) P.stats->bu_levels += 1;
        }
        expand_level<true>(P, S, L, level, nullptr, dir);
    } else if (P.phase == 8) {
        sweep_batch(P, S, ld_volatile_i32(&P.stats->graph_level), tid, nthreads);
    } else if (P.phase == 9) {
        graph_advance_batch(P);
    }
}

#if BFS_LEAN_PATHS
// The lean build's one kernel family (see the top of the file).
const void* plain_persistent_fn(int mb) {
    return mb >= 4 ? (const void*)bfs_plain_persistent<4, false>
         : mb == 3 ? (const void*)bfs_plain_persistent<3, false>
                   : (const void*)bfs_plain_persistent<2, false>;
}
#else
// ------------------------------------------------------ upload helpers
// CSR validation: flags[0] |= 1 for a column out of range, |= 2 for a
// decreasing offset.
__global__ void csr_check_kernel(const int64_t* off, const int32_t* col, long long n, long long nnz,
                                 int* flags) {
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int bad = 0;
    for (long long e = tid; e < nnz; e += nthreads) {
        const int32_t c = col[e];
        if (c < 0 || (long long)c >= n) bad |= 1;
    }
    for (long long v = tid; v < n; v += nthreads)
        if (off[v + 1] < off[v]) bad |= 2;
    if (bad) atomicOr(flags, bad);
}

// Symmetry test for the bottom-up step: the multiset of edges (v, u) equals
// the multiset of reversed edges (u, v) exactly when every edge is stored in
// both directions.  Both multisets are summed through a 64-bit mixing hash
// (order independent, wrapping); unequal sums prove asymmetry, equal sums
// mean symmetric up to a 2^-64-scale collision chance.
__device__ __forceinline__ unsigned long long edge_hash(unsigned long long a, unsigned long long b) {
    unsigned long long z = (a << 32 | b) + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void symmetry_hash_kernel(const int64_t* off, const int32_t* col, long long n,
                                     unsigned long long* sums) {
    const long long nwarps = (long long)gridDim.x * (blockDim.x / 32);
    const int lane = threadIdx.x & 31;
    unsigned long long fwd = 0, rev = 0;
    for (long long v = (long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); v < n;
         v += nwarps) {
        const long long b = off[v], e = off[v + 1];
        for (long long k = b + lane; k < e; k += 32) {
            const unsigned long long u = (unsigned)col[k];
            fwd += edge_hash((unsigned long long)v, u);
            rev += edge_hash(u, (unsigned long long)v);
        }
    }
    atomicAdd(&sums[0], fwd);
    atomicAdd(&sums[1], rev);
}

// Degree histogram by bin: counts[b] vertices and edges[b] entries.
__global__ void degree_bins_kernel(const int64_t* off, long long n, int t_small, int t_large,
                                   unsigned long long* counts, unsigned long long* edges,
                                   unsigned long long* maxdeg) {
    __shared__ unsigned long long s_c[kBins], s_e[kBins], s_m;
    if (threadIdx.x < kBins) { s_c[threadIdx.x] = 0; s_e[threadIdx.x] = 0; }
    if (threadIdx.x == 0) s_m = 0;
    __syncthreads();
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    unsigned long long c[kBins] = {0, 0, 0}, e[kBins] = {0, 0, 0}, m = 0;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += nthreads) {
        const long long d = off[v + 1] - off[v];
        if (d <= 0) continue;
        const int b = d < t_small ? 0 : (d < t_large ? 1 : 2);
        c[b] += 1;
        e[b] += (unsigned long long)d;
        m = d > (long long)m ? (unsigned long long)d : m;
    }
    for (int b = 0; b < kBins; ++b) {
        atomicAdd(&s_c[b], c[b]);
        atomicAdd(&s_e[b], e[b]);
    }
    atomicMax(&s_m, m);
    __syncthreads();
    if (threadIdx.x < kBins) {
        atomicAdd(&counts[threadIdx.x], s_c[threadIdx.x]);
        atomicAdd(&edges[threadIdx.x], s_e[threadIdx.x]);
    }
    if (threadIdx.x == 0) atomicMax(maxdeg, s_m);
}

// -------------------------------------------------------- host wrappers
// Kernels are instantiated for 2, 3 and 4 resident CTAs per SM (register
// cap 128, 80 or 64; batched kernels 2 and 3: at 4 their spills cost more
// than the extra warps gain); the graph's occupancy option picks one.
const void* plain_persistent_fn(int mb, bool staged) {
    if (staged)
        return mb >= 4 ? (const void*)bfs_plain_persistent<4, true>
             : mb == 3 ? (const void*)bfs_plain_persistent<3, true>
                       : (const void*)bfs_plain_persistent<2, true>;
    return mb >= 4 ? (const void*)bfs_plain_persistent<4, false>
         : mb == 3 ? (const void*)bfs_plain_persistent<3, false>
                   : (const void*)bfs_plain_persistent<2, false>;
}
const void* plain_step_fn(int mb, bool staged) {
    if (staged)
        return mb >= 4 ? (const void*)bfs_plain_step<4, true>
             : mb == 3 ? (const void*)bfs_plain_step<3, true> : (const void*)bfs_plain_step<2, true>;
    return mb >= 4 ? (const void*)bfs_plain_step<4, false>
         : mb == 3 ? (const void*)bfs_plain_step<3, false> : (const void*)bfs_plain_step<2, false>;
}
const void* batch_persistent_fn(int mb) {
    return mb >= 3 ? (const void*)bfs_batch_persistent<3> : (const void*)bfs_batch_persistent<2>;
}
const void* batch_step_fn(int mb) {
    return mb >= 3 ? (const void*)bfs_batch_step<3> : (const void*)bfs_batch_step<2>;
}

// int8 rows from int32 distances, 16 per thread and step (16-byte loads and
// stores when both arrays are 16-byte aligned, else one at a time).
__global__ void dist_to_int8_kernel(const int32_t* __restrict__ src, int8_t* __restrict__ dst,
                                    long long count, DevStats* stats, bool vec) {
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n16 = vec ? count / 16 : 0;   // 16-byte accesses need aligned ends
    bool deep = false;
    for (long long i = tid; i < n16; i += nthreads) {
        const int4* s4 = reinterpret_cast<const int4*>(src + 16 * i);
        unsigned w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int4 x = __ldcs(s4 + k);
            const int v[4] = {x.x, x.y, x.z, x.w};
            unsigned b = 0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                int y = v[c];
                if (y > 126) { deep = true; y = -2; }
                b |= (unsigned)(uint8_t)(int8_t)y << (8 * c);
            }
            w[k] = b;
        }
        reinterpret_cast<uint4*>(dst)[i] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    for (long long i = 16 * n16 + tid; i < count; i += nthreads) {
        int y = src[i];
        if (y > 126) { deep = true; y = -2; }
        dst[i] = (int8_t)y;
    }
    if (deep && stats) atomicCAS(&stats->status, 0, (int)kDevDepth);
}

cudaError_t launch_dist_to_int8(const int32_t* src, int8_t* dst, long long count, DevStats* stats,
                                int sms, cudaStream_t s) {
    const bool vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0;
    dist_to_int8_kernel<<<sms * 4, 256, 0, s>>>(src, dst, count, stats, vec);
    return cudaGetLastError();
}

cudaError_t launch_csr_check(const int64_t* off, const int32_t* col, long long n, long long nnz,
                             int* flags, int sms, cudaStream_t s) {
    csr_check_kernel<<<sms * 4, 512, 0, s>>>(off, col, n, nnz, flags);
    return cudaGetLastError();
}

cudaError_t launch_symmetry_hash(const int64_t* off, const int32_t* col, long long n,
                                 unsigned long long* sums, int sms, cudaStream_t s) {
    symmetry_hash_kernel<<<sms * 4, 256, 0, s>>>(off, col, n, sums);
    return cudaGetLastError();
}

cudaError_t launch_degree_bins(const int64_t* off, long long n, int t_small, int t_large,
                               unsigned long long* counts, unsigned long long* edges,
                               unsigned long long* maxdeg, int sms, cudaStream_t s) {
    degree_bins_kernel<<<sms * 2, 512, 0, s>>>(off, n, t_small, t_large, counts, edges, maxdeg);
    return cudaGetLastError();
}

#endif  // BFS_LEAN_PATHS

#if BFS_LEAN_PATHS
}  // namespace lean
#endif
}  // namespace bfs
