// Internal declarations shared by the kernels of the D-RSF library.
//
// Device state layout (all in HBM, one copy per handle):
//   parent[n], rep[n]           int32   the forest and each vertex's tree root
//   off[n+1]                    int64   slack-CSR row starts (row capacity =
//                                       off[u+1] - off[u])
//   used[n]                     int32   append cursor of each row
//   col[off[n]]                 int32   neighbours; -1 = empty or deleted
//   hkey[H], hpu[H], hpv[H]             open-addressing edge index: key ->
//                                       global col positions of the edge in
//                                       the rows of min(u,v) and max(u,v),
//                                       or (POS_OVF, overflow slot)
//   ovf[ovf_cap]                uint64  edges whose row had no free slot
//   per-batch work arrays (epoch-stamped, never cleared per batch)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>

#include "../../include/drsf.h"

typedef unsigned long long u64;

#define EMPTY_KEY 0xFFFFFFFFFFFFFFFFull
#define TOMB_KEY 0xFFFFFFFFFFFFFFFEull
#define POS_OVF 0xFFFFFFFFu
#define NIL (-1)

// latched device error bits (ctl->err)
#define ERR_BATCH_ID 1   // out-of-range id in the current batch: batch skipped
#define ERR_TIMEOUT 2    // a bounded grid barrier gave up
#define ERR_CAPACITY 4   // an internal buffer would overflow (never expected)
#define ERR_ROUNDS 8     // an iteration exceeded its round bound (cyclic parent)

// grid-barrier wait limit in nanoseconds (globaltimer)
#define BARRIER_TIMEOUT_NS 2000000000ull
#define MAX_ROUNDS 40

// Device control block: latched errors, batch epoch, grid barrier state,
// per-batch counts.  Statistic fields mirror drsf_batch_stats.
struct Ctl {
    int err;
    int skip;               // current batch rejected (ERR_BATCH_ID seen)
    unsigned epoch;         // batch counter; epoch stamps compare against it
    int op;
    u64 bar[8];             // grid-barrier counters: jump, hook, orient, mark, bfs, Euler marks, detach
                            // (reset at each batch's start and before each static BFS)
    int flag[3];            // per-round "another round needed" flags
    u64 cnt[3];             // per-round list sizes (hook-and-compress)
    u64 dv[3], dp[3];       // top-down delete, per level (ring of 3): vertices appended, and
                            // rows << 32 | entries appended
    u64 dovf;               // top-down delete: tree edges listed from the overflow list
    unsigned depth_hint;    // top-down delete, kept across batches: levels the last search took, or
                            // above the level limit after one gave up (counts down once per skip)
    int det_skip;           // the batch skipped the top-down search (read by the next k_begin)
    u64 nb;                 // normalised batch edges (new / deleted keys)
    u64 ncut;               // cut vertices
    u64 naff;               // affected list
    u64 ndet;               // detached list
    u64 ncand;              // candidates
    u64 ner;                // replacement edges
    u64 npc;                // distinct pieces touched by E_r
    u64 nact;               // active vertices (path reversal)
    u64 ncore;              // core arcs of the super-forest Euler tour
    u64 ovf_count;          // overflow list length (grows until rebuild)
    long long edges;        // live undirected edges of G
    long long htomb;        // index tombstones
    long long ctomb;        // CSR tombstones (deleted entries)
    long long scanned;      // adjacency entries scanned
    long long self_loops;
    long long dropped;
    long long tree_cut;
    long long hook_rounds;
    long long rank_rounds;
    long long mark_rounds;
    long long jump_rounds;
    long long jump_visits;
    long long reversed;
    long long batch_len;
    long long overflow_total;
    const int *batch;       // the current batch (device), set by k_begin
    int td;                 // delete: the detached vertices were found top-down (else: pointer jumping)
    int need_root;          // delete, top-down: a tree's root piece is re-rooted (list its vertices)
    long long det_levels;   // top-down levels of the batch (0: not taken)
    long long det_entries;  // adjacency entries the top-down search read
};

// The edge index.
struct Index {
    u64 *key;
    uint32_t *pu;   // position of the edge in the row of min(u,v), or POS_OVF
    uint32_t *pv;   // position in the row of max(u,v), or overflow slot
    u64 mask;
};

// The slack CSR.
struct Csr {
    const long long *off;
    int *used;
    int *col;
};

__host__ __device__ __forceinline__ u64 ekey(uint32_t u, uint32_t v) {
    return u < v ? ((u64)u << 32) | v : ((u64)v << 32) | u;
}
__host__ __device__ __forceinline__ uint32_t klo(u64 k) { return (uint32_t)(k >> 32); }
__host__ __device__ __forceinline__ uint32_t khi(u64 k) { return (uint32_t)(k & 0xFFFFFFFFu); }

// 64-bit finaliser (MurmurHash3 fmix64) for the edge index.
__device__ __forceinline__ u64 hslot(u64 k, u64 mask) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k & mask;
}

// Edge index probes (open addressing, linear probing).
// Insert-if-absent.  Returns the slot when this call claimed it, -1-slot
// when the key was already present, LLONG_MIN when the table is full.
__device__ __forceinline__ long long index_claim(Index ix, u64 key) {
    u64 s = hslot(key, ix.mask);
    for (u64 p = 0; p <= ix.mask; ++p) {
        u64 cur = __ldcg(&ix.key[s]);
        if (cur == key) return -1 - (long long)s;
        if (cur == EMPTY_KEY) {
            u64 old = atomicCAS(&ix.key[s], EMPTY_KEY, key);
            if (old == EMPTY_KEY) return (long long)s;
            if (old == key) return -1 - (long long)s;
        }
        s = (s + 1) & ix.mask;
    }
    return LLONG_MIN;
}

// Pull a whole array into L2, one prefetch per 128-byte line, strided over
// the calling threads (thread tid of nthreads): for arrays that the next
// kernels gather from at random, which would otherwise pay one DRAM latency
// per dependent access.
__device__ __forceinline__ void l2_prefetch(const void *p, long long bytes, long long tid, long long nthreads) {
    const char *c = (const char *)p;
    for (long long off = tid * 128; off < bytes; off += nthreads * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(c + off));
}

// Hook-forest slots of the candidates' endpoints (read by k_boruvka): the
// kernel that writes a candidate sets up each of its endpoints once per
// batch (whoever stamps it first): its own root in comp, both per-round
// minimum slots empty.
struct HookSlots {
    unsigned *stamp;
    int *comp;
    u64 *best0, *best1;
};
__device__ __forceinline__ void hook_slot_init(const HookSlots &hs, int a, unsigned ep) {
    // one lane per endpoint among the calling lanes (the giant tree's root
    // is an endpoint of most candidates)
    const unsigned grp = __match_any_sync(__activemask(), a);
    if ((int)(threadIdx.x & 31) != __ffs(grp) - 1) return;
    if (__ldcg(&hs.stamp[a]) != ep && atomicExch(&hs.stamp[a], ep) != ep) {
        hs.comp[a] = a;
        hs.best0[a] = EMPTY_KEY;
        hs.best1[a] = EMPTY_KEY;
    }
}

// Lookup; -1 when absent.  Deleted entries (TOMB_KEY) are probed past.
__device__ __forceinline__ long long index_find(Index ix, u64 key) {
    u64 s = hslot(key, ix.mask);
    for (u64 p = 0; p <= ix.mask; ++p) {
        u64 cur = __ldcg(&ix.key[s]);
        if (cur == key) return (long long)s;
        if (cur == EMPTY_KEY) return -1;
        s = (s + 1) & ix.mask;
    }
    return -1;
}

// Warp-aggregated append: one atomicAdd per warp; returns the slot of this
// lane (or -1 when pred is false).
__device__ __forceinline__ long long agg_append(u64 *ctr, bool pred) {
    unsigned active = __activemask();
    unsigned m = __ballot_sync(active, pred);
    if (!pred) return -1;
    int lane = threadIdx.x & 31;
    int leader = __ffs(m) - 1;
    u64 base = 0;
    if (lane == leader) base = atomicAdd(ctr, (u64)__popc(m));
    base = __shfl_sync(m, base, leader);
    return (long long)(base + __popc(m & ((1u << lane) - 1u)));
}

// One slot of row r's append cursor per calling lane; lanes of a warp with
// the same row share one atomicAdd.
__device__ __forceinline__ int row_slot(int *used, int r) {
    const unsigned grp = __match_any_sync(__activemask(), r);
    const int lane = threadIdx.x & 31, ld = __ffs(grp) - 1;
    int base = 0;
    if (lane == ld) base = atomicAdd(&used[r], __popc(grp));
    base = __shfl_sync(grp, base, ld);
    return base + __popc(grp & ((1u << lane) - 1u));
}

// Pair table: piece pair (min, max) -> minimum edge key between the two
// pieces.  Probing is bounded; a pair that finds no slot returns false and
// the caller keeps the edge as a plain candidate instead.
#define PAIR_PROBES 64
// Slot of a piece pair key (claimed if absent), or -1 when the probes found
// no slot.
__device__ __forceinline__ long long pair_slot(u64 *pk, u64 mask, u64 pair) {
    u64 s = hslot(pair, mask);
    for (int p = 0; p < PAIR_PROBES; ++p) {
        u64 cur = __ldcg(&pk[s]);
        if (cur == pair) return (long long)s;
        if (cur == EMPTY_KEY) {
            u64 old = atomicCAS(&pk[s], EMPTY_KEY, pair);
            if (old == EMPTY_KEY || old == pair) return (long long)s;
        }
        s = (s + 1) & mask;
    }
    return -1;
}
__device__ __forceinline__ bool pair_min(u64 *pk, u64 *mk, u64 mask, int a, int b, u64 key) {
    u64 pair = a < b ? ((u64)(unsigned)a << 32) | (unsigned)b : ((u64)(unsigned)b << 32) | (unsigned)a;
    u64 s = hslot(pair, mask);
    for (int p = 0; p < PAIR_PROBES; ++p) {
        u64 cur = __ldcg(&pk[s]);
        if (cur == EMPTY_KEY) {
            u64 old = atomicCAS(&pk[s], EMPTY_KEY, pair);
            if (old == EMPTY_KEY || old == pair) {
                atomicMin(&mk[s], key);
                return true;
            }
        } else if (cur == pair) {
            atomicMin(&mk[s], key);
            return true;
        }
        s = (s + 1) & mask;
    }
    return false;
}

// Block-wide sum of per-thread counts added to a counter: one atomic per
// block.  Every thread of the block must call it.
__device__ __forceinline__ void block_add(long long *ctr, long long v) {
    __shared__ unsigned long long s_sum;
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&s_sum, (unsigned long long)v);
    __syncthreads();
    if (threadIdx.x == 0 && s_sum) atomicAdd((unsigned long long *)ctr, s_sum);
    __syncthreads();
}

// Block-aggregated append: one atomicAdd per block.  Every thread of the
// block must call it (the loop around it must be block-uniform); the slots
// of a block are contiguous and ordered by thread index.
__device__ __forceinline__ long long block_append(u64 *ctr, bool pred) {
    __shared__ unsigned s_w[32];
    __shared__ u64 s_base;
    unsigned m = __ballot_sync(0xffffffffu, pred);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) s_w[w] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned tot = 0;
        int nw = (blockDim.x + 31) >> 5;
        for (int k = 0; k < nw; ++k) {
            unsigned c = s_w[k];
            s_w[k] = tot;
            tot += c;
        }
        s_base = tot ? atomicAdd(ctr, (u64)tot) : 0;
    }
    __syncthreads();
    long long r = pred ? (long long)(s_base + s_w[w] + __popc(m & ((1u << lane) - 1u))) : -1;
    __syncthreads();
    return r;
}

// Block-wide exclusive scan (any blockDim multiple of 32, <= 1024);
// *total receives the block sum.  All threads must call it.
__device__ __forceinline__ long long block_excl_scan_ll(long long v, long long *total) {
    __shared__ long long s_ws[32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_ws[w] = x;
    __syncthreads();
    if (w == 0) {
        long long t = lane < nw ? s_ws[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) s_ws[lane] = t;
    }
    __syncthreads();
    long long pre = (w > 0 ? s_ws[w - 1] : 0) + x - v;
    *total = s_ws[nw - 1];
    __syncthreads();
    return pre;
}

// Block-aggregated reservation of `cnt` consecutive slots per thread (one
// atomicAdd per block); returns this thread's first slot.  Every thread of
// the block must call it.
__device__ __forceinline__ long long block_reserve(u64 *ctr, int cnt) {
    __shared__ u64 s_rb;
    long long tot;
    long long pre = block_excl_scan_ll(cnt, &tot);
    if (threadIdx.x == 0) s_rb = tot ? atomicAdd(ctr, (u64)tot) : 0;
    __syncthreads();
    long long r = (long long)s_rb + pre;
    __syncthreads();
    return r;
}

// Block-aggregated reservation for four separate slabs: thread t has
// flags f[0..3] (item k of thread t lies in input slab k); the output keeps
// slab order and, within a slab, thread order, so a compacted list keeps the
// order of its input.  One block scan of the four counts packed in 16-bit
// fields (a block has at most 1024 threads) and one atomicAdd per block.
// Returns the output slot of item k in slot[k] (-1 when its flag is 0).
__device__ __forceinline__ void block_reserve4(u64 *ctr, const bool f[4], long long slot[4]) {
    __shared__ u64 s_rb4;
    long long packed = (long long)f[0] | ((long long)f[1] << 16) | ((long long)f[2] << 32) | ((long long)f[3] << 48);
    long long tot;
    long long pre = block_excl_scan_ll(packed, &tot);
    long long t[4], p[4];
    for (int k = 0; k < 4; ++k) {
        t[k] = (tot >> (16 * k)) & 0xFFFF;
        p[k] = (pre >> (16 * k)) & 0xFFFF;
    }
    long long all = t[0] + t[1] + t[2] + t[3];
    if (threadIdx.x == 0) s_rb4 = all ? atomicAdd(ctr, (u64)all) : 0;
    __syncthreads();
    long long base = (long long)s_rb4, off = 0;
    for (int k = 0; k < 4; ++k) {
        slot[k] = f[k] ? base + off + p[k] : -1;
        off += t[k];
    }
    __syncthreads();
}

// Block-aggregated reservation of list rows together with their entry
// ranges, from one packed counter: rows in the high 32 bits, entries in the
// low 32 bits (the entries of all rows stay below 2^32, so the low half
// never carries into the high half).  Row k of each thread (f[k] set, len[k]
// entries) gets its list position pos[k] and entry offset off[k]; positions
// and offsets follow slab order, then thread order, so the offsets are the
// exclusive prefix sum of the lengths in list order.  One atomicAdd per
// block; every thread of the block must call it.
template <int K>
__device__ __forceinline__ void block_reserve_rows(u64 *ctr, const bool f[K], const int len[K], long long pos[K],
                                                   long long off[K]) {
    __shared__ u64 s_rr;
    long long pre[K], tot[K];
#pragma unroll
    for (int k = 0; k < K; ++k)
        pre[k] = block_excl_scan_ll(f[k] ? (1ll << 32) | (long long)(unsigned)len[k] : 0ll, &tot[k]);
    long long all = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) all += tot[k];
    if (threadIdx.x == 0) s_rr = all ? atomicAdd(ctr, (u64)all) : 0;
    __syncthreads();
    u64 acc = s_rr;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const u64 b = acc + (u64)pre[k];
        pos[k] = f[k] ? (long long)(b >> 32) : -1;
        off[k] = (long long)(b & 0xFFFFFFFFull);
        acc += (u64)tot[k];
    }
    __syncthreads();
}

// 64-bit minimum over a group of lanes (mask from __match_any_sync).
__device__ __forceinline__ u64 group_min_u64(unsigned grp, u64 k) {
    unsigned hi = (unsigned)(k >> 32), lo = (unsigned)k;
    unsigned hmin = __reduce_min_sync(grp, hi);
    unsigned lmin = __reduce_min_sync(grp, hi == hmin ? lo : 0xFFFFFFFFu);
    return ((u64)hmin << 32) | lmin;
}

__device__ __forceinline__ u64 globaltimer_ns() {
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ u64 ld_acquire_u64(const u64 *p) {
    u64 v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier for cooperative launches (all blocks co-resident).
// Ticket barrier on a monotonic counter owned by one kernel (always launched
// with the same block count, so the counter is a multiple of gridDim.x
// between barriers): each block takes a ticket t and waits until the counter
// reaches the end of t's group.  The wait is bounded: after
// BARRIER_TIMEOUT_NS it latches ERR_TIMEOUT and returns false, and a block
// that sees another block's timeout returns false too, so the kernel unwinds
// instead of hanging.
__device__ __forceinline__ bool grid_barrier(Ctl *ctl, u64 *bar) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const u64 nb = gridDim.x;
        __threadfence();
        u64 t = atomicAdd(bar, 1ull);
        u64 target = (t / nb + 1) * nb;
        int ok = 1;
        if (ld_acquire_u64(bar) < target) {
            u64 t0 = globaltimer_ns();
            unsigned it = 0;
            while (ld_acquire_u64(bar) < target) {
                if ((++it & 255u) == 0) {
                    if (*(volatile int *)&ctl->err & ERR_TIMEOUT) { ok = 0; break; }
                    if (globaltimer_ns() - t0 > BARRIER_TIMEOUT_NS) {
                        atomicOr(&ctl->err, ERR_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Root search with path halving on a hook forest that is not being hooked
// concurrently (halving writes keep every pointer on the path to the same
// root).  The walk is bounded: a cycle (impossible for valid input) latches
// ERR_ROUNDS instead of spinning.
__device__ __forceinline__ int find_root(int *comp, int x, Ctl *ctl) {
    for (int it = 0; it < (1 << 24); ++it) {
        int p = __ldcg(&comp[x]);
        if (p == x) return x;
        int gp = __ldcg(&comp[p]);
        if (gp == p) return p;
        comp[x] = gp;
        x = gp;
    }
    atomicOr(&ctl->err, ERR_ROUNDS);
    return x;
}

// Root of x in the hook forest without writes (for short chains read by
// many threads at once: no stores to shared entries).  Bounded; a cycle
// latches ERR_ROUNDS.
__device__ __forceinline__ int find_root_ro(const int *comp, int x, Ctl *ctl) {
    for (int it = 0; it < (1 << 24); ++it) {
        int p = __ldcg(&comp[x]);
        if (p == x) return x;
        x = p;
    }
    atomicOr(&ctl->err, ERR_ROUNDS);
    return x;
}

// Loads of data that other blocks wrote earlier in the same cooperative
// launch go to L2 (the SM's L1 may hold a stale line).
#define LD(x) __ldcg(&(x))

static inline unsigned grid_for(long long n, int block, unsigned cap) {
    long long g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > (long long)cap) g = cap;
    return (unsigned)g;
}
