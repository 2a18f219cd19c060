// Forest kernels of the D-RSF batch update (Algorithm 1):
//   - representatives by pointer jumping on the cut forest F^;
//   - replacement edges by hooking and compressing over the trees of F^
//     (Section III-B, Algorithm 2, phase 1), with minimum-key hooking so
//     that the chosen edges are the unique minimum spanning forest of the
//     tree multigraph (Boruvka);
//   - orientation of the replacement edges by an Euler tour of the
//     tree-of-trees (Algorithm 2, phase 2; Euler tour technique, Section I
//     preliminaries) rooted at the tree with the smallest root id;
//   - path reversal of every (x, rep[x]) path at once by pointer doubling
//     over the re-rooted trees, then attachment parent[x] <- y
//     (Algorithm 1; ReversePaths, Section II-C), and the representative
//     refresh.
// Iterative phases run as one cooperative launch each with a bounded grid
// barrier between rounds; no host round trip per round.
#include <climits>

#include "kernels.h"

// cores of up to this many arcs are list-ranked in one block's shared memory
#define ORIENT_SMEM_ARCS 12288
#define ORIENT_SMEM_BYTES (4 * ORIENT_SMEM_ARCS * (int)sizeof(int))
#define ORIENT_THREADS 1024
// hooking: threads per block (one block per SM) and the live candidates at
// the start of a round (after round 0) up to which block 0 finishes alone
// (the kernel comes in two block sizes: 1024 threads, one block per SM, so
// that block 0 has the threads for the tail, and 256 threads, four per SM,
// for batches whose candidates stay in the millions past round 0, where
// the grid rounds measured faster with smaller blocks)
#define HOOK_TAIL 8192
// a core of at most this many edges is oriented by one block (measured on
// R-MAT-22: faster than the grid phases for small batches' cores of tens of
// edges, slower for the 100K batches' cores of about 900 edges)
#define ORIENT_SMALL_EDGES 256
// independent items per thread and iteration in the pointer-doubling rounds
#ifndef JU
#define JU 4
#endif
// the same for the final pass of the jump (more state per item)
#define JF 2
// consecutive items per thread in the list-building vertex passes: IPT over
// a list, IPN over all n vertices (more loads in flight per thread: those
// passes are one dependent gather behind a streaming load)
#define IPT 4
#define IPN 16
// k_aff_collect keeps more per item (old root, list position): 8 items per
// thread (48 registers) measured faster than 16 (64 registers, fewer
// resident blocks): 0.036 vs 0.041 ms per pass on R-MAT scale 22
#define IPA 8
// top-down delete: after a search that gave up at its level limit, the
// deletes that skip it before it is tried again
#define DETACH_BACKOFF 8
// longest path reversed by one walking thread (longer ones: doubling marks)
#define WALK_MAX 64

// x[k] = a[i0 + k] for k < IP (IP a multiple of 4, i0 a multiple of IP, a
// 16-byte aligned): vector loads when all IP items are in range.
template <int IP>
__device__ __forceinline__ void load_vec(const int *a, long long i0, long long cnt, int (&x)[IP]) {
    if (i0 + IP <= cnt) {
#pragma unroll
        for (int j = 0; j < IP / 4; ++j) {
            const int4 q = *reinterpret_cast<const int4 *>(a + i0 + 4 * j);
            x[4 * j] = q.x;
            x[4 * j + 1] = q.y;
            x[4 * j + 2] = q.z;
            x[4 * j + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < IP; ++k) x[k] = i0 + k < cnt ? a[i0 + k] : 0;
    }
}
__device__ __forceinline__ void load_ipt(const int *a, long long i0, long long cnt, int (&x)[IPT]) {
    load_vec<IPT>(a, i0, cnt, x);
}
// a detached piece is left out of the cross-edge scan instead of its tree's
// root piece only if it has this many more vertices (the swap costs a full
// pass over the affected list)
#define HEAVY_SWAP_MIN 4096
// shared-memory piece-count table of the final jump pass
#define WT_BITS 6
#define WT_SLOTS (1 << WT_BITS)
#define WT_PROBES 8

#define GS_LOOP(i, n) \
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)(n); \
         i += (long long)gridDim.x * blockDim.x)

__device__ __forceinline__ long long gtid() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long gstride() { return (long long)gridDim.x * blockDim.x; }

// Reset the per-batch counters, advance the epoch and record the batch (the
// kernels after this one read the batch and its length from the control
// block, so their launches do not depend on them).
__global__ void k_begin(Ctl *ctl, int op, long long len, const int *batch) {
    if (threadIdx.x != 0) return;
    ctl->batch = batch;
    ctl->epoch += 1;
    ctl->skip = 0;
    ctl->op = op;
    ctl->nb = ctl->ncut = ctl->naff = ctl->ndet = ctl->ncand = ctl->ner = ctl->npc = ctl->nact = 0;
    ctl->scanned = ctl->self_loops = ctl->dropped = ctl->tree_cut = 0;
    ctl->hook_rounds = ctl->rank_rounds = ctl->mark_rounds = ctl->jump_rounds = ctl->reversed = 0;
    ctl->jump_visits = 0;
    ctl->td = ctl->need_root = 0;
    if (ctl->det_skip) {   // the last batch skipped the top-down search
        if (ctl->depth_hint > 0) ctl->depth_hint -= 1;
        ctl->det_skip = 0;
    }
    ctl->det_levels = ctl->det_entries = 0;
    ctl->batch_len = len;
    for (int i = 0; i < 3; ++i) {
        ctl->flag[i] = 0;
        ctl->cnt[i] = 0;
        ctl->dv[i] = ctl->dp[i] = 0;
    }
    ctl->dovf = 0;
    // each barrier counter serves one cooperative launch per batch; its
    // targets are multiples of that launch's grid size, so it restarts at 0
    // (launches of different grid sizes, or a wait that timed out, leave it
    // at any value)
    for (int i = 0; i < 8; ++i) ctl->bar[i] = 0;
}

// Delete: list the vertices of every tree that lost a tree edge (its old
// root was stamped by the cut), with their old root.
// Each thread takes IPN vertices per iteration, k-major (item k of thread t
// is vertex b0 + k * blockDim + t, so every load and store of a warp covers
// 32 consecutive vertices), with all IPN loads and gathers in flight before
// any is used.  A warp's listed vertices take consecutive slots (one block
// reservation of the warps' totals), in vertex order within the warp.
// With roots_only (after a top-down search of the detached vertices, when
// some tree's root piece is re-rooted) only the root pieces' vertices are
// appended (the detached ones already hold their new representative, which
// is no stamped old root); otherwise the pass runs only when the top-down
// search did not (the pointer-jumping path).
__global__ void __launch_bounds__(BLK) k_aff_collect(int n, const int *rep, const unsigned *aff_ep, int *A, int *rold,
                                                     unsigned *w, u64 *heavy, Ctl *ctl, const int *par, int *J,
                                                     int roots_only) {
    static_assert(IPA <= 32, "item masks are 32 bits");
    if (*(volatile int *)&ctl->skip) return;
    if (roots_only ? !(*(volatile int *)&ctl->td && *(volatile int *)&ctl->need_root) : *(volatile int *)&ctl->td)
        return;
    unsigned ep = ctl->epoch;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const long long step = (long long)gridDim.x * blockDim.x * IPA;
    for (long long b0 = (long long)blockIdx.x * blockDim.x * IPA; b0 < n; b0 += step) {
        const long long v0 = b0 + threadIdx.x;
        int r[IPA];
#pragma unroll
        for (int k = 0; k < IPA; ++k) {
            const long long v = v0 + (long long)k * blockDim.x;
            r[k] = v < n ? rep[v] : 0;
        }
        unsigned in = 0;
#pragma unroll
        for (int k = 0; k < IPA; ++k) {
            const long long v = v0 + (long long)k * blockDim.x;
            if (v < n && aff_ep[r[k]] == ep) in |= 1u << k;
        }
        // (the warp's ballots are recomputed below rather than kept)
        const int tot = __reduce_add_sync(0xffffffffu, __popc(in));
        long long p = block_reserve(&ctl->naff, lane == 0 ? tot : 0);
        p = __shfl_sync(0xffffffffu, p, 0);
#pragma unroll
        for (int k = 0; k < IPA; ++k) {
            const unsigned bk = __ballot_sync(0xffffffffu, (in >> k) & 1u);
            if ((in >> k) & 1u) {
                const int v = (int)(v0 + (long long)k * blockDim.x);
                A[p + __popc(bk & lt)] = v;
                if (!roots_only) {
                    rold[v] = r[k];
                    if (J) J[v] = par[v];   // seed of the asynchronous doubling
                    if (r[k] == v) {        // the old root: piece-weight and heaviest-piece slots
                        w[v] = 0;
                        heavy[v] = 0;
                    }
                }
            }
            p += __popc(bk);
        }
    }
}

// Root of v in the forest J by pointer jumping with path halving, in place:
// every J[x] only ever moves to an ancestor of x, so concurrent walks over
// shared paths stay correct and shorten each other's paths (no round
// barrier is needed).  The walk is bounded; a cycle latches ERR_ROUNDS.
__device__ __forceinline__ int find_halving(int *J, int v, Ctl *ctl) {
    int x = v;
    for (int it = 0; it < (1 << 22); ++it) {
        int p = __ldcg(&J[x]);
        int gp = __ldcg(&J[p]);
        if (p == gp) return p;
        J[x] = gp;
        x = gp;
    }
    atomicOr(&ctl->err, ERR_ROUNDS);
    return x;
}

// Adds cnt to the weight of piece p through the block's shared table
// (open addressing, WT_PROBES probes), or to w[p] when no slot is free.
__device__ __forceinline__ void piece_count(int *s_wk, unsigned *s_wc, unsigned *w, int p, unsigned cnt) {
    unsigned h = ((unsigned)p * 0x9E3779B1u) >> (32 - WT_BITS);
    for (int pr = 0; pr < WT_PROBES; ++pr) {
        int key = *(volatile int *)&s_wk[h];
        if (key == -1) key = atomicCAS(&s_wk[h], -1, p);
        if (key == -1 || key == p) {
            atomicAdd(&s_wc[h], cnt);
            return;
        }
        h = (h + 1) & (WT_SLOTS - 1);
    }
    atomicAdd(&w[p], cnt);
}

// tile[T] = row for the tiles of 32 entries whose first entry lies in the
// row of entries [st, st + d), d > 0 (rows are never empty), for the rows of
// the lanes with `on` (called by the whole warp).  A lane writes the tiles of
// a short row itself; a long row (a hub's, up to tens of thousands of tiles)
// is written by the whole warp, so no lane writes more than a few tiles of
// it in sequence.
#define FILL_OWN 4
__device__ __forceinline__ void warp_fill_tiles(int *tile, bool on, long long st, long long d, int row) {
    const int lane = threadIdx.x & 31;
    const long long t0 = (st + 31) >> 5, t1 = on ? ((st + d - 1) >> 5) + 1 : t0;   // tiles [t0, t1)
    const bool big = t1 - t0 > FILL_OWN;
    if (on && !big)
        for (long long T = t0; T < t1; ++T) tile[T] = row;
    unsigned bm = __ballot_sync(0xffffffffu, big);
    while (bm) {
        const int l = __ffs(bm) - 1;
        bm &= bm - 1;
        const long long a = __shfl_sync(0xffffffffu, t0, l), b = __shfl_sync(0xffffffffu, t1, l);
        const int r = __shfl_sync(0xffffffffu, row, l);
        for (long long T = a + lane; T < b; T += 32) tile[T] = r;
    }
}

// Append the non-empty rows (`f`, `len` > 0) of a warp's lanes to the row
// list of the scan, with their entry ranges and the tile map: positions are
// pb (rows << 32 | entries) plus offsets from one atomic per warp on the
// packed counter pc.  All 32 lanes call.
__device__ __forceinline__ void warp_list_rows(u64 *pc, u64 pb, RowList rl, Csr g, bool f, int w, int len, int p,
                                               int ro) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const unsigned fm = __ballot_sync(0xffffffffu, f);
    if (!fm) return;
    // exclusive warp scan of the row lengths
    int x = f ? len : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    const int tot = __shfl_sync(0xffffffffu, x, 31);
    const int ex = x - (f ? len : 0);
    const int fl = __ffs(fm) - 1;
    u64 base = 0;
    if (lane == fl) base = atomicAdd(pc, ((u64)__popc(fm) << 32) | (u64)(unsigned)tot);
    base = __shfl_sync(0xffffffffu, base, fl) + pb;
    const long long q = (long long)(base >> 32) + __popc(fm & lt);
    const long long eo = (long long)(base & 0xFFFFFFFFull) + ex;
    if (f) {
        rl.D[q] = w;
        rl.roff[q] = (unsigned)eo;
        rl.base[q] = (unsigned)g.off[w];
        rl.meta[q] = make_int2(p, ro);
    }
    warp_fill_tiles(rl.tile, f, eo, len, (int)q);
}

// Append one warp's detached vertices (lanes with `on`) to the vertex list
// and their non-empty rows (`len` > 0) to the row list of the scan: positions
// are the level's bases (vb vertices; pb rows << 32 | entries) plus offsets
// taken from the level's own counters (vc, and pc packed like pb), one
// atomic per warp on each.  All 32 lanes call.
__device__ __forceinline__ void warp_detach_append(u64 *vc, u64 *pc, long long vb, u64 pb, RowList rl, int *A, Csr g,
                                                   bool on, int w, int len, int p, int ro) {
    const int lane = threadIdx.x & 31;
    const unsigned m = __ballot_sync(0xffffffffu, on);
    if (!m) return;
    const int ld = __ffs(m) - 1;
    u64 a0 = 0;
    if (lane == ld) a0 = atomicAdd(vc, (u64)__popc(m));
    a0 = __shfl_sync(0xffffffffu, a0, ld);
    if (on) A[vb + (long long)a0 + __popc(m & ((1u << lane) - 1u))] = w;
    warp_list_rows(pc, pb, rl, g, on && len > 0, w, len, p, ro);
}

// Representatives by asynchronous pointer doubling in place (delete batches
// with DRSF_JUMP=async): no grid barrier between steps.  J holds a copy of
// the cut forest for the listed vertices; afterwards J[v] is the complemented
// root of every listed vertex, and k_jump<2> carries on from there.
__global__ void __launch_bounds__(BLK, 6) k_jump_async(const int *A, Ctl *ctl, int *J, int *X, int *Y) {
    if (*(volatile int *)&ctl->skip || *(volatile int *)&ctl->td) return;
    const long long cnt = (long long)ctl->naff;
    // asynchronous doubling in place (one buffer, no grid barrier
    // between steps): each warp owns a slice of the list and repeats
    // J[v] <- J[J[v]] over its open vertices until none is left.  A
    // pointer only ever moves to an ancestor, whatever mix of old and
    // new values a step reads, so every step moves an open vertex up
    // at least one level and the result is the same roots.
    // (list positions are below 2^31: at most n entries)
    const int lane = threadIdx.x & 31;
    const int nwarp = (int)(gstride() >> 5);
    const int slice = (int)((cnt + nwarp - 1) / nwarp);
    const int wlo = (int)(gtid() >> 5) * slice;
    int wlen = wlo < cnt ? (int)(wlo + slice < cnt ? slice : cnt - wlo) : 0;
    const int *in = A + wlo;
    int *out = X + wlo, *spare = Y + wlo;
    int it = 0;
    long long vis = 0;
    while (wlen > 0) {
        if (it >= MAX_ROUNDS * 64) {
            if (lane == 0) atomicOr(&ctl->err, ERR_ROUNDS);
            return;
        }
        vis += wlen;
        int nopen = 0;
        for (int b0 = 0; b0 < wlen; b0 += 32 * JU) {
            int v[JU], w0[JU], w2[JU];
            bool ok[JU], open[JU];
#pragma unroll
            for (int k = 0; k < JU; ++k) {
                const int i = b0 + k * 32 + lane;
                ok[k] = i < wlen;
                v[k] = ok[k] ? in[i] : 0;
            }
#pragma unroll
            for (int k = 0; k < JU; ++k) w0[k] = ok[k] ? LD(J[v[k]]) : -1;
#pragma unroll
            for (int k = 0; k < JU; ++k) w2[k] = (ok[k] && w0[k] >= 0) ? LD(J[w0[k]]) : 0;
#pragma unroll
            for (int k = 0; k < JU; ++k) {
                open[k] = false;
                if (!ok[k]) continue;
                int nv;
                if (w0[k] < 0) nv = w0[k];
                else if (w2[k] < 0) nv = w2[k];
                else if (w2[k] == w0[k]) nv = ~w0[k];
                else {
                    nv = w2[k];
                    open[k] = true;
                }
                J[v[k]] = nv;
            }
#pragma unroll
            for (int k = 0; k < JU; ++k) {
                const unsigned m = __ballot_sync(0xffffffffu, open[k]);
                if (open[k]) out[nopen + __popc(m & ((1u << lane) - 1u))] = v[k];
                nopen += __popc(m);
            }
        }
        wlen = nopen;
        in = out;
        int *t = out; out = spare; spare = t;
        ++it;
    }
    if (lane == 0 && vis) {
        atomicAdd((u64 *)&ctl->jump_visits, (u64)vis);
        atomicMax((unsigned long long *)&ctl->jump_rounds, (unsigned long long)it);
    }
}

// Warp-aggregated list appends of the top-down search (no block barrier):
// the calling lanes with `on` take consecutive slots of A, those with a
// non-empty row (`len` > 0) consecutive rows of the row list and their entry
// ranges, from one atomic per warp on each counter (rows in the high and
// entries in the low 32 bits of the packed row counter).  All 32 lanes call.
// Delete, top-down alternative to the pointer jumping of Algorithm 1 (same
// representatives): the detached vertices are the cut vertices and every
// descendant of one in the cut forest, and a detached vertex's piece is the
// nearest cut vertex above it.  A level-synchronous search goes down from
// the cut vertices over tree children (neighbours w of v with parent[w] ==
// v, found in v's row or, for edges held outside the rows, in the overflow
// list) and touches only the detached vertices' rows, where pointer jumping
// touches every vertex of every cut tree.  Each level's rows are appended to
// the row list of the cross-edge scan as they are found (rows and entry
// ranges from one packed counter, 32-entry tiles), so level k reads exactly
// the rows appended in level k-1 with the tile-window scan of k_scan_lb, and
// the scan afterwards reuses the list (the piece left out of every tree is
// its root piece).  Every level appends through counters of its own (a ring
// of three: level k appends to slot k+1, reads the final count of slot k
// after the barrier and clears slot k+2), so all blocks see the same level
// sizes although some append while others still read.  New representatives
// go to J1 and are committed only when the search ends within its budget
// (vertices, entries, levels); otherwise nothing is published and the
// pointer-jumping path runs.
__global__ void __launch_bounds__(BLK, 4)
    k_detach(Ctl *ctl, const int *cuts, const int *par, int *rep, Csr g, const u64 *ovf, u64 ovf_cap, RowList rl,
             int *A, int *J1, unsigned *det_ep, unsigned *det_claim, const int *rold, long long budget_v,
             long long budget_e, int max_levels, int *oc, int *op) {
    if (*(volatile int *)&ctl->skip) return;
    // Deep trees below the cuts make the search a long chain of levels
    // (one grid barrier each) where pointer doubling needs a logarithmic
    // number of steps: after a search that gave up at the level limit the
    // next DETACH_BACKOFF deletes go straight to pointer jumping, then the
    // search is tried again.  The hint is not written in this launch before
    // every block has read it (the next batch's k_begin counts it down), so
    // all blocks take the same branch.
    if (*(volatile unsigned *)&ctl->depth_hint > (unsigned)max_levels) {
        if (gtid() == 0) ctl->det_skip = 1;
        return;
    }
    const unsigned ep = ctl->epoch;
    const long long nc = (long long)ctl->ncut;
    u64 *bar = &ctl->bar[6];
    const int lane = threadIdx.x & 31;
    // level 0: the cut vertices (pieces of their own), slot 0
    for (long long b0 = gtid() & ~31ll; b0 < nc; b0 += gstride()) {
        const long long i = b0 + lane;
        const bool on = i < nc;
        int c = 0, len = 0, ro = 0;
        if (on) {
            c = cuts[i];
            ro = rold[c];
            J1[c] = c;
            __threadfence();   // J1 before the stamp that publishes it
            det_ep[c] = ep;
            len = min(g.used[c], (int)(g.off[c + 1] - g.off[c]));
        }
        warp_detach_append(&ctl->dv[0], &ctl->dp[0], 0, 0, rl, A, g, on, c, len, c, ro);
    }
    // the tree edges held outside the rows (overflow list), as (child,
    // parent): listed once, read by every level (few: edges land there
    // only when a row is full)
    {
        const long long no = (long long)min((u64)ctl->ovf_count, ovf_cap);
        for (long long b0 = gtid() & ~31ll; b0 < no; b0 += gstride()) {
            const long long i = b0 + lane;
            int cw = -1, pv = -1;
            if (i < no) {
                const u64 k = ovf[i];
                if (k != TOMB_KEY) {
                    const int a = (int)klo(k), b = (int)khi(k);
                    if (LD(par[a]) == b) cw = a, pv = b;
                    else if (LD(par[b]) == a) cw = b, pv = a;
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, cw >= 0);
            if (!m) continue;
            const int ld = __ffs(m) - 1;
            u64 q0 = 0;
            if (lane == ld) q0 = atomicAdd(&ctl->dovf, (u64)__popc(m));
            q0 = __shfl_sync(0xffffffffu, q0, ld);
            if (cw >= 0) {
                const u64 q = q0 + __popc(m & ((1u << lane) - 1u));
                oc[q] = cw;
                op[q] = pv;
            }
        }
    }
    long long vb = 0;   // vertices listed before the current level's
    u64 pb = 0;         // rows << 32 | entries listed before it
    int lvl = 0;
    bool ok = true;
    for (;; ++lvl) {
        if (!grid_barrier(ctl, bar)) return;
        // the level found in the last round (slot lvl % 3) is final
        const int sl = lvl % 3, sn = (lvl + 1) % 3;
        const long long dv = (long long)*(volatile u64 *)&ctl->dv[sl];
        const u64 dp = *(volatile u64 *)&ctl->dp[sl];
        if (gtid() == 0) ctl->dv[(lvl + 2) % 3] = ctl->dp[(lvl + 2) % 3] = 0;   // read last one level ago
        const unsigned e_lo = (unsigned)pb, r_lo = (unsigned)(pb >> 32);
        const long long vn = vb + dv;
        const u64 pn = pb + dp;
        const unsigned e_hi = (unsigned)pn, r_hi = (unsigned)(pn >> 32);
        if (dv == 0) break;   // the last level found nothing
        if (lvl >= max_levels || vn > budget_v || (long long)e_hi > budget_e) {
            ok = false;
            break;
        }
        (void)r_lo;
        // tiles covering the entries of the rows found in the last level,
        // a contiguous range of tiles per warp
        const unsigned T0 = e_lo >> 5, T1 = (e_hi + 31) >> 5;
        const unsigned NT = T1 - T0;
        const unsigned nw = (unsigned)(gstride() >> 5), wid = (unsigned)(gtid() >> 5);
        const unsigned per = (NT + nw - 1) / nw;
        for (unsigned it = 0; it < per; ++it) {
            const unsigned T = T0 + wid * per + it;
            bool child = false;
            int w = -1, p = 0, ro = 0;
            if (T < T1) {   // warp-uniform
                const unsigned t0 = T << 5;
                // (rows of earlier levels, written by other blocks: read through L2)
                const int r0 = LD(rl.tile[T]);
                const unsigned wr = (unsigned)r0 + lane;
                const bool wok = wr < r_hi;
                const unsigned wo = wok ? LD(rl.roff[wr]) : 0xFFFFFFFFu;
                const int wv = wok ? LD(rl.D[wr]) : 0;
                const unsigned wb = wok ? LD(rl.base[wr]) : 0;
                const int2 wm = wok ? __ldcg(&rl.meta[wr]) : make_int2(0, 0);
                const unsigned pos = wo - t0;
                const unsigned bit = (lane > 0 && pos < 32) ? (1u << pos) : 0u;
                const unsigned starts = __reduce_or_sync(0xffffffffu, bit);
                const int c = __popc(starts & (lane == 31 ? 0xffffffffu : ((2u << lane) - 1u)));
                const unsigned rstart = __shfl_sync(0xffffffffu, wo, c);
                const int v = __shfl_sync(0xffffffffu, wv, c);
                const unsigned rb = __shfl_sync(0xffffffffu, wb, c);
                p = __shfl_sync(0xffffffffu, wm.x, c);
                ro = __shfl_sync(0xffffffffu, wm.y, c);
                const unsigned e = t0 + lane;
                if (e >= e_lo && e < e_hi) {
                    w = __ldcs(&g.col[(size_t)(rb + (e - rstart))]);
                    child = w >= 0 && LD(par[w]) == v;
                }
            }
            int len = 0;
            if (child) {
                J1[w] = p;
                __threadfence();
                det_ep[w] = ep;
                len = min(g.used[w], (int)(g.off[w + 1] - g.off[w]));
            }
            warp_detach_append(&ctl->dv[sn], &ctl->dp[sn], vn, pn, rl, A, g, child, w, len, p, ro);
        }
        // children joined by a tree edge outside the rows: a vertex whose
        // parent is detached (published: its J1 before its stamp)
        const long long nt = (long long)*(volatile u64 *)&ctl->dovf;
        for (long long b0 = gtid() & ~31ll; b0 < nt; b0 += gstride()) {
            const long long i = b0 + lane;
            bool child = false;
            int w = -1, p = 0, ro = 0, len = 0;
            if (i < nt) {
                const int cw = LD(oc[i]), pv = LD(op[i]);
                const bool pd = LD(det_ep[pv]) == ep;
                __threadfence();
                if (pd && LD(det_claim[cw]) != ep && atomicExch(&det_claim[cw], ep) != ep) {
                    child = true;
                    w = cw;
                    p = LD(J1[pv]);
                    ro = rep[w];   // rep still holds the old roots
                }
            }
            if (child) {
                J1[w] = p;
                __threadfence();
                det_ep[w] = ep;
                len = min(g.used[w], (int)(g.off[w + 1] - g.off[w]));
            }
            warp_detach_append(&ctl->dv[sn], &ctl->dp[sn], vn, pn, rl, A, g, child, w, len, p, ro);
        }
        vb = vn;
        pb = pn;
    }
    // over budget: nothing was published (naff, ndet and rep untouched);
    // the pointer-jumping path takes over from the cut
    if (!ok) {
        if (gtid() == 0) {
            ctl->det_levels = -lvl;
            if (lvl >= max_levels) ctl->depth_hint = (unsigned)max_levels + DETACH_BACKOFF;
        }
        return;
    }
    // commit the representatives of the detached vertices
    for (long long i = gtid(); i < vb; i += gstride()) {
        const int v = A[i];
        rep[v] = LD(J1[v]);
    }
    if (gtid() == 0) {
        ctl->naff = (u64)vb;
        ctl->ndet = pb >> 32;
        ctl->det_entries = (long long)(pb & 0xFFFFFFFFull);
        rl.roff[pb >> 32] = (unsigned)pb;
        ctl->det_levels = lvl;
        ctl->depth_hint = (unsigned)lvl;
        ctl->td = 1;
    }
}

// After the orientation of a top-down delete: does some cut tree's root
// piece get a new representative (a detached piece with a smaller root id
// joined its super-tree)?  Then its vertices must be listed for the refresh
// and the path marks (k_aff_collect with roots_only).
__global__ void k_rootcheck(Ctl *ctl, const int *cuts, const int *rold, const unsigned *rep_ep) {
    if (*(volatile int *)&ctl->skip || !*(volatile int *)&ctl->td) return;
    const unsigned ep = ctl->epoch;
    const long long nc = (long long)ctl->ncut;
    for (long long i = gtid(); i < nc; i += gstride())
        if (rep_ep[rold[cuts[i]]] == ep) ctl->need_root = 1;
}

// Representatives (Algorithm 1, parallel pointer jumping) of the listed
// vertices: rep[v] = root of v in F^ (J starts as a copy of parent).
// Delete mode (1) then chooses the rows to scan for cross edges: every cross
// edge joins two pieces of one old tree, so scanning all pieces but one per
// tree finds each of them.  The piece left out is the root piece, unless a
// detached piece has HEAVY_SWAP_MIN more vertices (a cut near the root that
// detaches most of a tree): then the heaviest piece.  The listed rows get an
// exclusive prefix sum of their lengths in roff (roff[ndet] = total; rows
// and entry ranges are reserved together from one packed counter), their
// CSR start, their (piece, piece left out) and the row of every 32-entry
// tile for the load-balanced scan.
// (6 blocks of BLK threads per SM: the rounds are latency-bound)
template <int sync_rounds>
__global__ void __launch_bounds__(BLK, 6)
    k_jump(const int *A, int use_list, long long cnt_static, Ctl *ctl, const int *par, int *J, int *J1, int *rep,
           RowList rl, int mode, const int *rold, unsigned *w, u64 *heavy, Csr g, int *X, int *Y, const int *cuts) {
    int *const D = rl.D;
    unsigned *const roff = rl.roff;
    if (*(volatile int *)&ctl->skip) return;
    if (mode == 1 && *(volatile int *)&ctl->td) return;   // the top-down search found the pieces
    long long cnt = use_list ? (long long)ctl->naff : cnt_static;
    if constexpr (sync_rounds != 0) {
        // synchronous doubling J <- J o J (ping-pong).  A pointer that has
        // reached a root is stored complemented (negative): a converged
        // vertex skips the gather, and the loop ends in the first round in
        // which every listed vertex is converged (no verification round).
        // Round r reads the list of vertices still open (the full list in
        // round 0) and appends the ones still open after it to the other
        // work list (X, Y alternate); a vertex that converges writes its
        // complemented root into both buffers, so later reads of it from
        // either buffer see the root.  Round 0 reads the forest itself
        // (par); its converged vertices still write both buffers.
        int *Jc = J, *Jn = J1;
        int r = 0;
        if constexpr (sync_rounds == 2) {
            // the roots were found by k_jump_async (complemented in J)
        } else {
        if (gtid() == 0) {
            ctl->cnt[0] = (u64)cnt;
            ctl->cnt[1] = 0;
        }
        if (!grid_barrier(ctl, &ctl->bar[0])) return;
        for (;; ++r) {
            if (r >= MAX_ROUNDS) {
                if (gtid() == 0) atomicOr(&ctl->err, ERR_ROUNDS);
                return;
            }
            const long long c = (long long)*(volatile u64 *)&ctl->cnt[r % 3];
            if (c == 0) break;
            if (gtid() == 0) {
                ctl->cnt[(r + 2) % 3] = 0;
                ctl->jump_visits += c;
            }
            const int *in = r == 0 ? (use_list ? A : nullptr) : ((r & 1) ? X : Y);
            int *out = (r & 1) ? Y : X;
            // JU independent vertices per thread and iteration: their loads
            // are issued together (more loads in flight per thread)
            const long long S = gstride();
            for (long long base = (long long)blockIdx.x * blockDim.x; base < c; base += S * JU) {
                int v[JU], w0[JU], w2[JU];
                bool ok[JU], open[JU];
#pragma unroll
                for (int k = 0; k < JU; ++k) {
                    long long i = base + k * S + threadIdx.x;
                    ok[k] = i < c;
                    v[k] = ok[k] ? (in ? in[i] : (int)i) : 0;
                }
                const int *Jr = r == 0 ? par : Jc;
#pragma unroll
                for (int k = 0; k < JU; ++k) w0[k] = ok[k] ? LD(Jr[v[k]]) : -1;
#pragma unroll
                for (int k = 0; k < JU; ++k) w2[k] = (ok[k] && w0[k] >= 0) ? LD(Jr[w0[k]]) : 0;
#pragma unroll
                for (int k = 0; k < JU; ++k) {
                    open[k] = false;
                    if (!ok[k]) continue;
                    int nv;
                    if (w0[k] < 0) nv = w0[k];
                    else if (w2[k] < 0) nv = w2[k];
                    else if (w2[k] == w0[k]) nv = ~w0[k];
                    else {
                        nv = w2[k];
                        open[k] = true;
                    }
                    Jn[v[k]] = nv;
                    if (!open[k]) Jc[v[k]] = nv;
                }
                long long q[JU];
                block_reserve4(&ctl->cnt[(r + 1) % 3], open, q);
#pragma unroll
                for (int k = 0; k < JU; ++k)
                    if (open[k]) out[q[k]] = v[k];
            }
            if (!grid_barrier(ctl, &ctl->bar[0])) return;
            int *t = Jc; Jc = Jn; Jn = t;
        }
        if (gtid() == 0) ctl->jump_rounds = r;
        }
        if (mode == 0) {
            for (long long i = gtid(); i < cnt; i += gstride()) {
                int v = use_list ? A[i] : (int)i;
                rep[v] = ~LD(Jc[v]);
            }
            return;
        }
        // final pass: representatives, piece weights (vertex counts; the
        // weight slots of piece roots were zeroed at the cut) and a
        // provisional list of rows to scan: every vertex outside its tree's
        // root piece (only those read their row length).  JU vertices per
        // thread and iteration.  Piece counts go to a small open-addressing
        // table in shared memory (one global atomic per piece and block at
        // the end; a large piece spans many blocks), or straight to global
        // memory when the table has no slot.
        __shared__ int s_wk[WT_SLOTS];
        __shared__ unsigned s_wc[WT_SLOTS];
        for (int t = threadIdx.x; t < WT_SLOTS; t += blockDim.x) {
            s_wk[t] = -1;
            s_wc[t] = 0;
        }
        __syncthreads();
        const long long S = gstride();
        for (long long base = (long long)blockIdx.x * blockDim.x; base < cnt; base += S * JF) {
            int v[JF], p[JF], ro[JF], len[JF];
            bool ok[JF], scan[JF];
#pragma unroll
            for (int k = 0; k < JF; ++k) {
                long long i = base + k * S + threadIdx.x;
                ok[k] = i < cnt;
                v[k] = ok[k] ? A[i] : 0;
            }
#pragma unroll
            for (int k = 0; k < JF; ++k) {
                p[k] = ok[k] ? ~LD(Jc[v[k]]) : 0;
                ro[k] = ok[k] ? rold[v[k]] : 0;
            }
#pragma unroll
            for (int k = 0; k < JF; ++k) {
                scan[k] = false;
                len[k] = 0;
                if (!ok[k]) continue;
                // rep[v] == rold[v] already for the root piece's vertices
                if (p[k] != ro[k]) {
                    rep[v[k]] = p[k];
                    int cap = (int)(g.off[v[k] + 1] - g.off[v[k]]);
                    int used = g.used[v[k]];
                    len[k] = used < cap ? used : cap;
                    scan[k] = len[k] > 0;
                }
            }
#pragma unroll
            for (int k = 0; k < JF; ++k) {
                unsigned vm = __ballot_sync(0xffffffffu, ok[k]);
                if (ok[k]) {
                    unsigned grp = __match_any_sync(vm, p[k]);
                    if ((int)(threadIdx.x & 31) == __ffs(grp) - 1) {
                        piece_count(s_wk, s_wc, w, p[k], (unsigned)__popc(grp));
                    }
                }
            }
            long long q[JF], eo[JF];
            block_reserve_rows<JF>(&ctl->ndet, scan, len, q, eo);
#pragma unroll
            for (int k = 0; k < JF; ++k) {
                if (scan[k]) {
                    D[q[k]] = v[k];
                    roff[q[k]] = (unsigned)eo[k];
                    rl.base[q[k]] = (unsigned)g.off[v[k]];
                    rl.meta[q[k]] = make_int2(p[k], ro[k]);
                }
                warp_fill_tiles(rl.tile, scan[k], eo[k], len[k], (int)q[k]);
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < WT_SLOTS; t += blockDim.x)
            if (s_wk[t] != -1) atomicAdd(&w[s_wk[t]], s_wc[t]);
    } else {
        // J[v] may later be overwritten by another walk's halving step with
        // a non-root ancestor; rep[v] takes this thread's own result.
        for (long long i = gtid(); i < cnt; i += gstride()) {
            int v = use_list ? A[i] : (int)i;
            J[v] = par[v];
        }
        if (!grid_barrier(ctl, &ctl->bar[0])) return;
        for (long long i = gtid(); i < cnt; i += gstride()) {
            int v = use_list ? A[i] : (int)i;
            int root = find_halving(J, v, ctl);
            J[v] = root;
            rep[v] = root;
        }
        if (gtid() == 0) ctl->jump_rounds = 1;
        if (mode == 0) return;
        if (!grid_barrier(ctl, &ctl->bar[0])) return;
        for (long long i = gtid(); i < cnt; i += gstride()) {
            int v = A[i];
            atomicAdd(&w[LD(rep[v])], 1u);
        }
    }
    if (!grid_barrier(ctl, &ctl->bar[0])) return;
    // heaviest piece per cut tree: its pieces are the root piece and one
    // piece per cut vertex, so the cut list covers them all
    const long long nc = (long long)ctl->ncut;
    if (gtid() == 0) ctl->flag[0] = 0;   // set by the swap check below
    for (long long i = gtid(); i < nc; i += gstride()) {
        int c = cuts[i];
        int r = rold[c];
        u64 kc = ((u64)LD(w[c]) << 32) | (unsigned)c;
        unsigned act = __activemask();
        unsigned grp = __match_any_sync(act, r);
        unsigned hi = (unsigned)(kc >> 32), lo = (unsigned)kc;
        unsigned hmax = __reduce_max_sync(grp, hi);
        unsigned lmax = __reduce_max_sync(grp, hi == hmax ? lo : 0u);
        if ((int)(threadIdx.x & 31) == __ffs(grp) - 1) {
            atomicMax(&heavy[r], ((u64)hmax << 32) | lmax);
            // the root piece stays the piece left out unless a detached
            // piece outweighs it by HEAVY_SWAP_MIN vertices
            atomicMax(&heavy[r], ((u64)(LD(w[r]) + HEAVY_SWAP_MIN) << 32) | (unsigned)r);
        }
    }
    if (!grid_barrier(ctl, &ctl->bar[0])) return;
    // the provisional list left out each tree's root piece; where another
    // piece is heavier, rebuild the list with the exact rule (rare)
    {
        bool swap = false;
        for (long long i = gtid(); i < nc; i += gstride()) {
            int r = rold[cuts[i]];
            swap |= (int)(unsigned)LD(heavy[r]) != r;
        }
        // (the halving root search builds no provisional list: always exact)
        if (__syncthreads_or(swap || !sync_rounds) && threadIdx.x == 0) atomicOr(&ctl->flag[0], 1);
    }
    if (!grid_barrier(ctl, &ctl->bar[0])) return;
    if (*(volatile int *)&ctl->flag[0]) {
        if (gtid() == 0) ctl->ndet = 0;
        if (!grid_barrier(ctl, &ctl->bar[0])) return;
        for (long long base = (long long)blockIdx.x * blockDim.x; base < cnt; base += gstride()) {
            long long i = base + threadIdx.x;
            bool scan[1] = {false};
            int v = 0, hp = 0, pv = 0, len[1] = {0};
            if (i < cnt) {
                v = A[i];
                hp = (int)(unsigned)LD(heavy[rold[v]]);
                int cap = (int)(g.off[v + 1] - g.off[v]);
                int used = g.used[v];
                len[0] = used < cap ? used : cap;
                pv = LD(rep[v]);
                scan[0] = pv != hp && len[0] > 0;
            }
            long long q[1], eo[1];
            block_reserve_rows<1>(&ctl->ndet, scan, len, q, eo);
            if (scan[0]) {
                D[q[0]] = v;
                roff[q[0]] = (unsigned)eo[0];
                rl.base[q[0]] = (unsigned)g.off[v];
                rl.meta[q[0]] = make_int2(pv, hp);
            }
            warp_fill_tiles(rl.tile, scan[0], eo[0], len[0], (int)q[0]);
        }
        if (!grid_barrier(ctl, &ctl->bar[0])) return;
    }
    // the packed row counter becomes the row count; roff[nd] = all entries
    if (gtid() == 0) {
        const u64 pk = *(volatile u64 *)&ctl->ndet;
        ctl->ndet = pk >> 32;
        roff[pk >> 32] = (unsigned)pk;
    }
}

// Per-block table of hot indices for 64-bit minimum updates: lanes of a
// warp with the same index combine first; an index held by two or more
// lanes of a warp (one piece, such as the giant one, can be an endpoint of
// most candidates) is combined in shared memory and sent to global memory
// once per block by hm_flush; a lone index goes straight to global memory.
#define HM_SLOTS 16
#define HM_PROBES 4
struct HotMin {
    int k[HM_SLOTS];
    u64 v[HM_SLOTS];
    int rst[HM_SLOTS];
};
__device__ __forceinline__ void hm_init(HotMin &t) {
    for (int i = threadIdx.x; i < HM_SLOTS; i += blockDim.x) {
        t.k[i] = -1;
        t.v[i] = EMPTY_KEY;
        t.rst[i] = 0;
    }
    __syncthreads();
}
// slot of idx in the table (inserted when ins and absent), or -1
__device__ __forceinline__ int hm_slot(HotMin &t, int idx, bool ins) {
    unsigned h = ((unsigned)idx * 0x9E3779B1u) >> 28;
    for (int p = 0; p < HM_PROBES; ++p) {
        int key = *(volatile int *)&t.k[h];
        if (key == -1 && ins) key = atomicCAS(&t.k[h], -1, idx);
        if (key == idx || (key == -1 && ins)) return (int)h;
        if (key == -1) return -1;
        h = (h + 1) & (HM_SLOTS - 1);
    }
    return -1;
}
__device__ __forceinline__ void hm_min(HotMin &t, u64 *arr, int idx, u64 k, bool pred) {
    unsigned m = __ballot_sync(__activemask(), pred);
    if (!pred) return;
    unsigned grp = __match_any_sync(m, idx);
    u64 kmin = group_min_u64(grp, k);
    if ((int)(threadIdx.x & 31) != __ffs(grp) - 1) return;
    int sl = __popc(grp) > 1 ? hm_slot(t, idx, true) : -1;
    if (sl >= 0) atomicMin(&t.v[sl], kmin);
    else atomicMin(&arr[idx], kmin);
}
// bestn[idx] = EMPTY_KEY, once per block for the table's indices
__device__ __forceinline__ void hm_reset(HotMin &t, u64 *arr, int idx, bool pred) {
    unsigned m = __ballot_sync(__activemask(), pred);
    if (!pred) return;
    unsigned grp = __match_any_sync(m, idx);
    if ((int)(threadIdx.x & 31) != __ffs(grp) - 1) return;
    int sl = __popc(grp) > 1 ? hm_slot(t, idx, true) : -1;
    if (sl >= 0) t.rst[sl] = 1;
    else arr[idx] = EMPTY_KEY;
}
// sends the table's minima to arr (min) and its resets to rst_arr, then
// clears it; every thread of the block calls it
__device__ __forceinline__ void hm_flush(HotMin &t, u64 *arr, u64 *rst_arr) {
    __syncthreads();
    for (int i = threadIdx.x; i < HM_SLOTS; i += blockDim.x) {
        if (t.k[i] != -1) {
            if (t.v[i] != EMPTY_KEY) atomicMin(&arr[t.k[i]], t.v[i]);
            if (t.rst[i]) rst_arr[t.k[i]] = EMPTY_KEY;
        }
        t.k[i] = -1;
        t.v[i] = EMPTY_KEY;
        t.rst[i] = 0;
    }
    __syncthreads();
}

// Replacement edges by hook-and-compress over the trees of F^ (pieces).
// Each round: every component takes the minimum key among its incident
// candidates (64-bit atomicMin); a component whose minimum edge leads to
// another component hooks onto it (a mutual choice hooks the larger id under
// the smaller); each hooking edge joins E_r.  Candidates inside one
// component are dropped, the rest are compacted for the next round.  With
// distinct keys this is Boruvka's algorithm: E_r is the unique minimum
// spanning forest of the piece multigraph, |E_r| = k - l.
// Rounds r, r+1, ... of the hook-and-compress, by the whole grid (ONE
// false: grid barriers between phases) or by block 0 alone (ONE true: block
// barriers).  On the grid, a round that starts with at most HOOK_TAIL live
// candidates (after round 0 on R-MAT batches: about 2.5% of them) is handed
// to block 0: every block reads the same count after the barrier, so all
// take that branch together.  Returns -1 when a grid barrier gave up, the
// round to hand to block 0 (grid only), or 0 when done.
template <bool ONE>
__device__ __forceinline__ int hook_rounds(Ctl *ctl, HotMin &hm, int r, long long c0, u64 *ck0, int *ca0, int *cb0,
                                           u64 *ck1, int *ca1, int *cb1, int *comp, u64 *best0, u64 *best1, u64 *er,
                                           long long er_cap) {
    const long long T = ONE ? (long long)threadIdx.x : gtid();
    const long long S = ONE ? (long long)blockDim.x : gstride();
    const long long B0 = ONE ? 0 : (long long)blockIdx.x * blockDim.x;
    for (;; ++r) {
        if (r >= MAX_ROUNDS) {
            if (T == 0) atomicOr(&ctl->err, ERR_ROUNDS);
            return 0;
        }
        u64 *ck = (r & 1) ? ck1 : ck0, *ckn = (r & 1) ? ck0 : ck1;
        int *ca = (r & 1) ? ca1 : ca0, *can = (r & 1) ? ca0 : ca1;
        int *cb = (r & 1) ? cb1 : cb0, *cbn = (r & 1) ? cb0 : cb1;
        u64 *best = (r & 1) ? best1 : best0, *bestn = (r & 1) ? best0 : best1;
        const long long c = r == 0 ? c0 : (long long)*(volatile u64 *)&ctl->cnt[r % 3];
        if (!ONE && r > 0 && c <= HOOK_TAIL) return r;
        if (T == 0) {
            ctl->cnt[(r + 2) % 3] = 0;
            ctl->flag[(r + 1) % 3] = 0;
        }
        // phase A: roots of both ends, per-component minimum key
        for (long long i = T; i < c; i += S) {
            int a = LD(ca[i]), b = LD(cb[i]);
            if (r > 0) {   // every endpoint is its own root in round 0
                a = find_root_ro(comp, a, ctl);
                b = find_root_ro(comp, b, ctl);
                ca[i] = a;
                cb[i] = b;
            }
            u64 k = LD(ck[i]);
            hm_min(hm, best, a, k, a != b);
            hm_min(hm, best, b, k, a != b);
        }
        hm_flush(hm, best, bestn);
        if (!ONE && !grid_barrier(ctl, &ctl->bar[1])) return -1;
        // phase B: hook along minimum edges, keep the rest (block-uniform
        // loop: list appends are reserved once per block)
        bool hooked = false;
        for (long long b0 = B0; b0 < c; b0 += S) {
            const long long i = b0 + threadIdx.x;
            int a = 0, b = 0;
            bool alive = false, hook = false, keep = false;
            u64 k = 0;
            if (i < c) {
                a = LD(ca[i]);
                b = LD(cb[i]);
                alive = a != b;
                k = LD(ck[i]);
            }
            if (alive) {
                bool ba = __ldcg(&best[a]) == k, bb = __ldcg(&best[b]) == k;
                if (ba && bb) comp[a > b ? a : b] = a > b ? b : a;
                else if (ba) comp[a] = b;
                else if (bb) comp[b] = a;
                hook = ba || bb;
                keep = !hook;
            }
            hm_reset(hm, bestn, a, alive);
            hm_reset(hm, bestn, b, alive);
            hooked |= hook;
            long long pe = block_append(&ctl->ner, hook);
            if (hook) {
                if (pe < er_cap) er[pe] = k;
                else atomicOr(&ctl->err, ERR_CAPACITY);
            }
            long long pk = block_append(&ctl->cnt[(r + 1) % 3], keep);
            if (keep) {
                ckn[pk] = k;
                can[pk] = a;
                cbn[pk] = b;
            }
        }
        hm_flush(hm, best, bestn);
        const int any = __syncthreads_or(hooked);
        if (ONE) {
            if (!any) break;
        } else {
            if (any && threadIdx.x == 0) atomicOr(&ctl->flag[r % 3], 1);
            if (!grid_barrier(ctl, &ctl->bar[1])) return -1;
            if (!*(volatile int *)&ctl->flag[r % 3]) break;
        }
    }
    if (T == 0) ctl->hook_rounds = r;
    return 0;
}

template <int HT>
__global__ void __launch_bounds__(HT, 1024 / HT) k_boruvka(Ctl *ctl, u64 *ck0, int *ca0, int *cb0, u64 *ck1,
                                                          int *ca1, int *cb1, HookSlots hs, u64 *er,
                                                          long long er_cap, int init) {
    if (*(volatile int *)&ctl->skip) return;
    __shared__ HotMin hm;
    const unsigned ep = ctl->epoch;
    const long long c0 = (long long)ctl->ncand;
    if (gtid() == 0) {
        ctl->cnt[1] = ctl->cnt[2] = 0;
        ctl->flag[0] = ctl->flag[1] = ctl->flag[2] = 0;
    }
    hm_init(hm);
    if (init) {
        // set up each candidate endpoint once (the first lane to stamp it);
        // with init == 0 the kernel that wrote the candidates did it and
        // round 0 starts at once
        for (long long i = gtid(); i < c0; i += gstride()) {
            hook_slot_init(hs, ca0[i], ep);
            hook_slot_init(hs, cb0[i], ep);
        }
        if (!grid_barrier(ctl, &ctl->bar[1])) return;
    } else {
        __syncthreads();
    }
    const int r = hook_rounds<false>(ctl, hm, 0, c0, ck0, ca0, cb0, ck1, ca1, cb1, hs.comp, hs.best0, hs.best1, er,
                                     er_cap);
    if (r > 0 && blockIdx.x == 0)
        hook_rounds<true>(ctl, hm, r, c0, ck0, ca0, cb0, ck1, ca1, cb1, hs.comp, hs.best0, hs.best1, er, er_cap);
}

// Orientation of replacement edge i: down = its lower-id endpoint's piece
// p0 is the parent of the other piece p1.  The child piece P of edge {x, y}
// (x in P) gets the oriented edge x -> y, its attach point x and the
// super-tree's root as its new representative (each non-root piece is the
// child of exactly one edge: one write per piece; the super-root keeps its
// representative).
__device__ __forceinline__ void orient_one(const OrientArgs &a, long long i, bool down, unsigned ep) {
    const u64 k = a.er[i];
    const int x0 = (int)klo(k), x1 = (int)khi(k);
    const int p0 = LD(a.ep[2 * i]), p1 = LD(a.ep[2 * i + 1]);
    const int child = down ? p1 : p0;
    const int x = down ? x1 : x0, y = down ? x0 : x1;
    a.chx[i] = x;
    a.chy[i] = y;
    a.att_x[child] = x;
    a.att_ep[child] = ep;
    a.newrep[child] = LD(a.minp[LD(a.eroot[i])]);
    a.rep_ep[child] = ep;
}

// Wyllie list ranking of ncore list cells in shared memory by one block:
// val (svc) = cells from here to the end of the list, next pointers in snc
// (NIL at the end); svn / snn are the ping-pong buffers.  Returns the rounds
// taken (ERR_ROUNDS latched if the bound is hit) and leaves the ranks in
// *out (one of svc / svn).
__device__ int rank_block(Ctl *ctl, int *svc, int *svn, int *snc, int *snn, int ncore, int **out) {
    int r = 0;
    for (;; ++r) {
        int ch = 0;
        for (int i = threadIdx.x; i < ncore; i += blockDim.x) {
            const int sx = snc[i];
            if (sx != NIL) {
                svn[i] = svc[i] + svc[sx];
                snn[i] = snc[sx];
                ch = 1;
            } else {
                svn[i] = svc[i];
                snn[i] = NIL;
            }
        }
        const int any = __syncthreads_or(ch);
        int *t = svc; svc = svn; svn = t;
        t = snc; snc = snn; snn = t;
        if (!any) break;
        if (r >= MAX_ROUNDS) {
            if (threadIdx.x == 0) atomicOr(&ctl->err, ERR_ROUNDS);
            break;
        }
    }
    *out = svc;
    return r + 1;
}

// The core of the super-forest (the edges that are not leaf edges, listed
// in cel) oriented by one block: adjacency ranges claimed by the first arc
// of each core piece, arcs placed, Euler successors (as in the grid phases
// of k_orient) written straight into shared memory, ranked there, and each
// core edge oriented by its arc that comes first.  Block barriers only.
__device__ void orient_small_core(Ctl *ctl, const OrientArgs &a, const int *cel, long long nce, unsigned ep) {
    __shared__ int s_nc;
    if (threadIdx.x == 0) s_nc = 0;
    __syncthreads();
    for (long long t = threadIdx.x; t < 2 * nce; t += blockDim.x) {
        const long long j = 2 * (long long)LD(cel[t >> 1]) + (t & 1);
        const int id = LD(a.eid[j]);
        if (atomicCAS(&a.poff[id], -1, -2) == -1) a.poff[id] = atomicAdd(&s_nc, LD(a.cdeg[id]));
    }
    __syncthreads();
    const int ncore = s_nc;
    for (long long t = threadIdx.x; t < 2 * nce; t += blockDim.x) {
        const long long j = 2 * (long long)LD(cel[t >> 1]) + (t & 1);
        const int id = LD(a.eid[j]);
        const int slot = a.poff[id] + atomicAdd(&a.pcur[id], 1);
        a.adj[slot] = (int)j;
        a.apos[j] = slot;
    }
    __syncthreads();
    extern __shared__ int s_rank[];
    int *svc = s_rank, *svn = svc + ORIENT_SMEM_ARCS, *snc = svn + ORIENT_SMEM_ARCS, *snn = snc + ORIENT_SMEM_ARCS;
    for (long long t = threadIdx.x; t < 2 * nce; t += blockDim.x) {
        const long long j = 2 * (long long)LD(cel[t >> 1]) + (t & 1);
        const long long tw = j ^ 1;
        const int hid = LD(a.eid[tw]);   // the arc's head = the twin's source
        const int start = a.poff[hid], end = start + LD(a.cdeg[hid]);
        const int nx = a.apos[tw] + 1;
        int succ;
        if (nx == end) {
            const bool is_root = LD(a.minp[LD(a.eroot[j >> 1])]) == LD(a.ep[tw]);
            succ = is_root ? NIL : start;
        } else {
            succ = nx;
        }
        const int si = a.apos[j];
        snc[si] = succ;
        svc[si] = 1;
    }
    __syncthreads();
    int *rank = nullptr;
    const int rounds = rank_block(ctl, svc, svn, snc, snn, ncore, &rank);
    for (long long t = threadIdx.x; t < nce; t += blockDim.x) {
        const long long i = LD(cel[t]);
        orient_one(a, i, rank[a.apos[2 * i]] > rank[a.apos[2 * i + 1]], ep);
    }
    if (threadIdx.x == 0) {
        ctl->ncore = (u64)ncore;
        ctl->rank_rounds = rounds;
    }
}

// Orientation of E_r (Algorithm 2, phase 2).  The replacement edges form a
// forest over the pieces (the super-forest); each super-tree is rooted at
// its piece with the smallest root id.  A non-root piece with a single
// replacement edge is a leaf: its parent is its only neighbour, no tour
// needed.  The rest (the core, a tree per super-tree that still holds the
// root) is rooted by the Euler tour technique: circular adjacency lists give
// the successor of arc a->b as the arc after b->a in b's list; the circuit is
// opened at the root, the arcs are ranked by Wyllie's pointer jumping, and
// each edge is oriented by its arc that comes first.  The child piece P of
// edge {x, y} (x in P) gets the oriented replacement edge x -> y; every piece
// of the super-tree gets the root as its new representative.
__global__ void __launch_bounds__(ORIENT_THREADS) k_orient(Ctl *ctl, OrientArgs a) {
    if (*(volatile int *)&ctl->skip) return;
    const long long ner = (long long)ctl->ner;
    const unsigned ep = ctl->epoch;
    u64 *bar = &ctl->bar[2];
    // Arc j of edge j/2 runs from the piece of its (j odd ? larger : smaller)
    // endpoint to the other piece.  Phase 1 caches each arc's source piece
    // (ep), later phases its dense id (eid) and each edge's super-tree root
    // (eroot), so no phase re-walks rep / pidx / the hook forest.
    // phase 1: dense ids for the pieces touched by E_r
    if (gtid() == 0) ctl->ncore = ctl->cnt[0] = ctl->cnt[1] = 0;
    // the path walks after this kernel follow parent pointers one dependent
    // load at a time: pull the forest into L2 now, while the phases below
    // wait at their barriers (one 128-byte line per thread or so)
    if (ner > 0) l2_prefetch(a.parent, 4 * a.n, gtid(), gstride());
    // (block-uniform loop: the dense ids are reserved once per block)
    for (long long b0 = (long long)blockIdx.x * blockDim.x; b0 < 2 * ner; b0 += gstride()) {
        const long long j = b0 + threadIdx.x;
        bool first = false;
        int p = 0;
        if (j < 2 * ner) {
            u64 k = a.er[j >> 1];
            p = a.rep[(j & 1) ? khi(k) : klo(k)];
            a.ep[j] = p;
            // one lane per piece among the warp's lanes claims it (a piece
            // such as the giant one is an endpoint of most of the edges)
            unsigned grp = __match_any_sync(__activemask(), p);
            bool lead = (int)(threadIdx.x & 31) == __ffs(grp) - 1;
            first = lead && __ldcg(&a.pstamp[p]) != ep && atomicExch(&a.pstamp[p], ep) != ep;
        }
        long long id = block_append(&ctl->npc, first);
        if (first) {
            a.pidx[p] = (int)id;
            a.plist[id] = p;
            a.pdeg[id] = 0;
            a.cdeg[id] = 0;
            a.pcur[id] = 0;
            a.poff[id] = -1;   // (claimed by the core path for small cores)
            // the root piece of the hook forest holds its super-tree's slot
            if (find_root(a.comp, p, ctl) == p) a.minp[p] = INT_MAX;
        }
    }
    if (!grid_barrier(ctl, bar)) return;
    // phase 2: smallest piece id per super-tree, degrees (lanes with the
    // same target combine first: one super-tree or piece can collect most
    // of the batch's edges)
    for (long long j = gtid(); j < 2 * ner; j += gstride()) {
        int p = LD(a.ep[j]);
        int id = LD(a.pidx[p]);
        int root = find_root(a.comp, p, ctl);
        a.eid[j] = id;
        if (!(j & 1)) a.eroot[j >> 1] = root;
        unsigned act = __activemask();
        unsigned g1 = __match_any_sync(act, root);
        int pm = (int)__reduce_min_sync(g1, (unsigned)p);
        if ((int)(threadIdx.x & 31) == __ffs(g1) - 1) atomicMin(&a.minp[root], pm);
        unsigned g2 = __match_any_sync(act, id);
        if ((int)(threadIdx.x & 31) == __ffs(g2) - 1) atomicAdd(&a.pdeg[id], __popc(g2));
    }
    if (!grid_barrier(ctl, bar)) return;
    // phase 2b: leaf edges (a non-root piece with one edge); core degrees
    for (long long i = gtid(); i < ner; i += gstride()) {
        int p0 = LD(a.ep[2 * i]), p1 = LD(a.ep[2 * i + 1]);
        int id0 = LD(a.eid[2 * i]), id1 = LD(a.eid[2 * i + 1]);
        int sr = LD(a.minp[LD(a.eroot[i])]);
        bool leaf0 = LD(a.pdeg[id0]) == 1 && sr != p0;
        bool leaf1 = LD(a.pdeg[id1]) == 1 && sr != p1;
        unsigned char lf = leaf0 ? 1 : (leaf1 ? 2 : 0);
        a.lf[i] = lf;
        unsigned act = __activemask();
        unsigned core = __ballot_sync(act, !lf);
        if (!lf) {
            unsigned g0 = __match_any_sync(core, id0);
            if ((int)(threadIdx.x & 31) == __ffs(g0) - 1) atomicAdd(&a.cdeg[id0], __popc(g0));
            unsigned g1 = __match_any_sync(core, id1);
            if ((int)(threadIdx.x & 31) == __ffs(g1) - 1) atomicAdd(&a.cdeg[id1], __popc(g1));
        }
        // the core edges, listed for the one-block path of small cores
        if (!lf) {
            const int ld = __ffs(core) - 1;
            u64 b = 0;
            if ((int)(threadIdx.x & 31) == ld) b = atomicAdd(&ctl->cnt[0], (u64)__popc(core));
            b = __shfl_sync(core, b, ld);
            a.cel[b + __popc(core & ((1u << (threadIdx.x & 31)) - 1u))] = (int)i;
        }
    }
    if (!grid_barrier(ctl, bar)) return;
    {
        // A small core (small batches: tens of edges) is done by block 0
        // alone with block barriers (adjacency, Euler successors, ranking in
        // shared memory, orientation), while every block orients the leaf
        // edges.  A larger one first gets a second round of leaf raking
        // (phase 2c: on R-MAT it leaves about a tenth of the core), and
        // takes the grid phases below only if it is still large.
        long long nce = (long long)*(volatile u64 *)&ctl->cnt[0];
        const int *cel = a.cel;
        if (nce > ORIENT_SMALL_EDGES) {
            // phase 2c: a core piece with a single core edge that is not its
            // super-tree's root is a leaf of the remaining core; its edge is
            // oriented towards the other piece (lf) and both core degrees
            // drop.  Core degrees only fall, so a stale read can miss a leaf
            // but never make one up (the edge being looked at is still
            // alive, so a degree read as 1 is exactly 1), and both ends of
            // one edge cannot be such leaves (every core component holds its
            // root).  The edges left are listed again (second half of cel).
            int *cel2 = a.cel + ner;
            for (long long b0 = gtid() & ~31ll; b0 < nce; b0 += gstride()) {
                const long long t = b0 + (threadIdx.x & 31);
                bool keep = false;
                long long i = 0;
                if (t < nce) {
                    i = LD(a.cel[t]);
                    const int id0 = LD(a.eid[2 * i]), id1 = LD(a.eid[2 * i + 1]);
                    const int p0 = LD(a.ep[2 * i]), p1 = LD(a.ep[2 * i + 1]);
                    const int sr = LD(a.minp[LD(a.eroot[i])]);
                    const bool l0 = LD(a.cdeg[id0]) == 1 && p0 != sr;
                    const bool l1 = !l0 && LD(a.cdeg[id1]) == 1 && p1 != sr;
                    if (l0 || l1) {
                        a.lf[i] = l0 ? 1 : 2;
                        atomicSub(&a.cdeg[id0], 1);
                        atomicSub(&a.cdeg[id1], 1);
                    } else {
                        keep = true;
                    }
                }
                const unsigned km = __ballot_sync(0xffffffffu, keep);
                if (km) {
                    const int lane = threadIdx.x & 31, ld = __ffs(km) - 1;
                    u64 q0 = 0;
                    if (lane == ld) q0 = atomicAdd(&ctl->cnt[1], (u64)__popc(km));
                    q0 = __shfl_sync(0xffffffffu, q0, ld);
                    if (keep) cel2[q0 + __popc(km & ((1u << lane) - 1u))] = (int)i;
                }
            }
            if (!grid_barrier(ctl, bar)) return;
            nce = (long long)*(volatile u64 *)&ctl->cnt[1];
            cel = cel2;
        }
        if (nce <= ORIENT_SMALL_EDGES) {
            for (long long i = gtid(); i < ner; i += gstride()) {
                const unsigned char lf = LD(a.lf[i]);
                if (lf) orient_one(a, i, lf == 2, ep);
            }
            if (blockIdx.x == 0) orient_small_core(ctl, a, cel, nce, ep);
            return;
        }
    }
    // phase 3: adjacency ranges of the core pieces, reserved per block from
    // one cursor (ctl->ncore ends as the number of core arcs; the order of
    // the ranges is immaterial)
    const long long np = (long long)*(volatile u64 *)&ctl->npc;
    for (long long b0 = (long long)blockIdx.x * blockDim.x; b0 < np; b0 += gstride()) {
        const long long i = b0 + threadIdx.x;
        const long long d = i < np ? LD(a.cdeg[i]) : 0;
        const long long off = block_reserve(&ctl->ncore, d);
        if (i < np) a.poff[i] = (int)off;
    }
    if (!grid_barrier(ctl, bar)) return;
    // phase 4: place core arcs in their source piece's adjacency
    for (long long j = gtid(); j < 2 * ner; j += gstride()) {
        bool core = !LD(a.lf[j >> 1]);
        unsigned cm = __ballot_sync(__activemask(), core);
        if (!core) continue;
        int id = LD(a.eid[j]);
        unsigned grp = __match_any_sync(cm, id);
        int lane = threadIdx.x & 31, leader = __ffs(grp) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(&a.pcur[id], __popc(grp));
        base = __shfl_sync(grp, base, leader);
        int slot = LD(a.poff[id]) + base + __popc(grp & ((1u << lane) - 1u));
        a.adj[slot] = (int)j;
        a.apos[j] = slot;
    }
    if (!grid_barrier(ctl, bar)) return;
    // phase 5: Euler successors of core arcs, in slot space (the position of
    // an arc in the core adjacency array): the successor of arc a->b is the
    // slot after b->a's slot in b's list, wrapping to the list start; the
    // circuit is opened at each super-tree root
    for (long long j = gtid(); j < 2 * ner; j += gstride()) {
        if (LD(a.lf[j >> 1])) continue;
        long long tw = j ^ 1;
        int hid = LD(a.eid[tw]);                  // the arc's head = the twin's source
        int start = LD(a.poff[hid]), end = start + LD(a.cdeg[hid]);
        int nx = LD(a.apos[tw]) + 1;
        int succ;
        if (nx == end) {
            bool is_root = LD(a.minp[LD(a.eroot[j >> 1])]) == LD(a.ep[tw]);
            succ = is_root ? NIL : start;
        } else {
            succ = nx;
        }
        int si = LD(a.apos[j]);
        a.nx0[si] = succ;
        a.val0[si] = 1;
    }
    if (!grid_barrier(ctl, bar)) return;
    // phase 6: list ranking (Wyllie): val = arcs from here to the tour end.
    // A core of at most ORIENT_SMEM_ARCS arcs is ranked by block 0 alone in
    // shared memory (block barriers instead of grid barriers per round).
    const long long ncore = (long long)*(volatile u64 *)&ctl->ncore;
    int *vc = a.val0, *vn = a.val1, *nc = a.nx0, *nn = a.nx1;
    int r = 0;
    if (ncore <= ORIENT_SMEM_ARCS) {
        if (blockIdx.x == 0) {
            extern __shared__ int s_rank[];
            int *svc = s_rank, *svn = svc + ORIENT_SMEM_ARCS, *snc = svn + ORIENT_SMEM_ARCS,
                *snn = snc + ORIENT_SMEM_ARCS;
            for (long long i = threadIdx.x; i < ncore; i += blockDim.x) {
                svc[i] = LD(a.val0[i]);
                snc[i] = LD(a.nx0[i]);
            }
            __syncthreads();
            int *rank = nullptr;
            const int rounds = rank_block(ctl, svc, svn, snc, snn, (int)ncore, &rank);
            for (long long i = threadIdx.x; i < ncore; i += blockDim.x) a.val0[i] = rank[i];
            if (threadIdx.x == 0) ctl->rank_rounds = rounds;
        }
        if (!grid_barrier(ctl, bar)) return;
        vc = a.val0;
    } else {
        for (;; ++r) {
            if (r >= MAX_ROUNDS) {
                if (gtid() == 0) atomicOr(&ctl->err, ERR_ROUNDS);
                return;
            }
            if (gtid() == 0) ctl->flag[(r + 1) % 3] = 0;
            bool ch = false;
            for (long long i = gtid(); i < ncore; i += gstride()) {
                int sx = LD(nc[i]);
                if (sx != NIL) {
                    vn[i] = LD(vc[i]) + LD(vc[sx]);
                    nn[i] = LD(nc[sx]);
                    ch = true;
                } else {
                    vn[i] = LD(vc[i]);
                    nn[i] = NIL;
                }
            }
            if (__syncthreads_or(ch) && threadIdx.x == 0) atomicOr(&ctl->flag[r % 3], 1);
            if (!grid_barrier(ctl, bar)) return;
            int again = *(volatile int *)&ctl->flag[r % 3];
            int *t = vc; vc = vn; vn = t;
            t = nc; nc = nn; nn = t;
            if (!again) break;
        }
        if (gtid() == 0) ctl->rank_rounds = r + 1;
    }
    // phase 7: orient, attach points, new roots
    for (long long i = gtid(); i < ner; i += gstride()) {
        const unsigned char lf = LD(a.lf[i]);
        const bool down = lf ? lf == 2 : LD(vc[LD(a.apos[2 * i])]) > LD(vc[LD(a.apos[2 * i + 1])]);
        orient_one(a, i, down, ep);
    }
}

// Path reversal by walking (ReversePaths, Algorithm 1), one thread per
// oriented replacement edge x -> y: the path x = v0, v1 = parent[v0], ...,
// vL (the piece root) is reversed in place while it is walked (parent[v_j]
// <- v_{j-1}, parent[v0] <- y).  Each child piece has exactly one oriented
// edge and pieces are disjoint, so the walks never touch the same vertex.
// A walk that has not met its root after WALK_MAX steps restores the part
// it reversed and stamps its piece in long_ep: such pieces are reversed by
// the pointer-doubling marks instead.
__global__ void k_walk(Ctl *ctl, const int *chx, const int *chy, const int *rep, int *parent, unsigned *long_ep) {
    if (*(volatile int *)&ctl->skip) return;
    const unsigned ep = ctl->epoch;
    const long long ner = (long long)ctl->ner;
    long long rev = 0;
    GS_LOOP(i, ner) {
        const int x = chx[i];
        int prev = chy[i], cur = x, steps = 0;
        bool done = false;
        for (; steps < WALK_MAX; ++steps) {
            int nxt = parent[cur];
            parent[cur] = prev;
            if (nxt == cur) {
                done = true;
                break;
            }
            prev = cur;
            cur = nxt;
        }
        if (done) {
            rev += steps;   // the path's vertices below the root
        } else {
            // v0 .. v_{WALK_MAX-1} reversed, cur = v_WALK_MAX untouched
            int up = cur, v = prev;
            for (int t = 0; t < WALK_MAX; ++t) {
                int nv = parent[v];
                parent[v] = up;
                up = v;
                v = nv;
            }
            long_ep[rep[x]] = ep;
        }
    }
    if (rev) atomicAdd((u64 *)&ctl->reversed, (u64)rev);
}

// Path-reversal set-up fused with the representative refresh: a vertex of a
// piece that is re-rooted at an attach point x != its root is active (its
// old parent is saved, J0 seeded, x marked); every vertex of a merged piece
// takes the super-tree's root as its new rep.
// IP items per thread and iteration (IPT over a list, IPN over all
// vertices), k-major as in k_aff_collect, one slot reservation per block.
// Only the pieces stay in registers; the few items whose piece changed are
// handled from bit masks (the common item costs one stamp gather).
template <int IP>
__global__ void __launch_bounds__(BLK)
    k_active(const int *L, int use_list, long long cnt_static, Ctl *ctl, int *rep, const int *parent,
             const unsigned *sel_ep, const int *att_x, const unsigned *rep_ep, const int *newrep, int *act, int *pold,
             int *J0, unsigned char *mark, int *aidx, int *aroot) {
    static_assert(IP <= 32, "item masks are 32 bits");
    if (*(volatile int *)&ctl->skip) return;
    unsigned ep = ctl->epoch;
    long long cnt = use_list ? (long long)ctl->naff : cnt_static;
    const long long step = (long long)gridDim.x * blockDim.x * IP;
    for (long long b0 = (long long)blockIdx.x * blockDim.x * IP; b0 < cnt; b0 += step) {
        const long long i0 = b0 + threadIdx.x;
        int p[IP];
        if (use_list) {
#pragma unroll
            for (int k = 0; k < IP; ++k) {
                const long long i = i0 + (long long)k * blockDim.x;
                p[k] = i < cnt ? L[i] : 0;
            }
#pragma unroll
            for (int k = 0; k < IP; ++k) p[k] = i0 + (long long)k * blockDim.x < cnt ? rep[p[k]] : 0;
        } else {
#pragma unroll
            for (int k = 0; k < IP; ++k) {
                const long long i = i0 + (long long)k * blockDim.x;
                p[k] = i < cnt ? rep[i] : 0;
            }
        }
        // the pieces selected for the marks are re-rooted child pieces, all
        // of which get a new representative: one gather in the common case
        unsigned chg = 0;
#pragma unroll
        for (int k = 0; k < IP; ++k)
            if (i0 + (long long)k * blockDim.x < cnt && rep_ep[p[k]] == ep) chg |= 1u << k;
        unsigned on = 0;
        for (unsigned m = chg; m; m &= m - 1) {
            const int k = __ffs(m) - 1;
            const int pk = p[k];
            if (sel_ep[pk] == ep && att_x[pk] != pk) on |= 1u << k;
        }
        long long q = block_reserve(&ctl->nact, __popc(on));
        for (unsigned m = chg; m; m &= m - 1) {
            const int k = __ffs(m) - 1;
            const int pk = p[k];
            const long long i = i0 + (long long)k * blockDim.x;
            const int v = use_list ? L[i] : (int)i;
            if ((on >> k) & 1u) {
                const int pv = parent[v];
                act[q] = v;
                pold[q] = pv;
                J0[v] = pv;
                mark[v] = v == att_x[pk];
                aidx[v] = (int)q;   // dense index (Euler-tour marks)
                aroot[q] = pk;      // the piece root
                ++q;
            }
            rep[v] = newrep[pk];
        }
    }
}

// Mark every ancestor of each attach point x inside its piece by pointer
// doubling over the active vertices: round j, a marked v marks J_j[v] (its
// 2^j-th ancestor, clamped at the root) and J_{j+1} = J_j o J_j.  After
// round j the marks cover distances [0, 2^{j+1}); the loop stops once every
// J_{j+1} is a root, which bounds the path length.  Marks only ever land on
// ancestors of x, so reads racing with writes within a round are harmless.
__global__ void k_mark(Ctl *ctl, const int *act, int *J0, int *J1, unsigned char *mark, const int *parent) {
    if (*(volatile int *)&ctl->skip) return;
    long long na = (long long)ctl->nact;
    if (na == 0) {   // every path was walked (the same value in every block)
        if (gtid() == 0) ctl->mark_rounds = 0;
        return;
    }
    int *Jc = J0, *Jn = J1;
    int r = 0;
    for (;; ++r) {
        if (r >= MAX_ROUNDS) {
            if (gtid() == 0) atomicOr(&ctl->err, ERR_ROUNDS);
            return;
        }
        if (gtid() == 0) ctl->flag[(r + 1) % 3] = 0;
        bool more = false;
        const long long S = gstride();
        for (long long base = gtid(); base < na; base += S * JU) {
            int v[JU], w[JU], w2[JU];
            bool ok[JU];
            unsigned char mk[JU];
#pragma unroll
            for (int k = 0; k < JU; ++k) {
                long long i = base + k * S;
                ok[k] = i < na;
                v[k] = ok[k] ? act[i] : 0;
            }
#pragma unroll
            for (int k = 0; k < JU; ++k) {
                w[k] = ok[k] ? LD(Jc[v[k]]) : 0;
                mk[k] = ok[k] ? LD(mark[v[k]]) : 0;
            }
#pragma unroll
            for (int k = 0; k < JU; ++k) w2[k] = ok[k] ? LD(Jc[w[k]]) : 0;
#pragma unroll
            for (int k = 0; k < JU; ++k) {
                if (!ok[k]) continue;
                if (mk[k]) mark[w[k]] = 1;
                Jn[v[k]] = w2[k];
                more |= parent[w2[k]] != w2[k];
            }
        }
        if (__syncthreads_or(more) && threadIdx.x == 0) atomicOr(&ctl->flag[r % 3], 1);
        if (!grid_barrier(ctl, &ctl->bar[3])) return;
        int again = *(volatile int *)&ctl->flag[r % 3];
        int *t = Jc; Jc = Jn; Jn = t;
        if (!again) break;
    }
    if (gtid() == 0) ctl->mark_rounds = r + 1;
}

// ReversePaths + attach (Algorithm 1): for each marked non-root vertex u,
// parent'[old parent of u] = u (old parents come from the saved snapshot, so
// no thread reads a pointer another thread rewrites); then parent[x] = y for
// every oriented replacement edge x -> y.
__global__ void k_reverse(Ctl *ctl, const int *act, const int *pold, const unsigned char *mark, const int *chx,
                          const int *chy, int *parent, int walked) {
    if (*(volatile int *)&ctl->skip) return;
    long long na = (long long)ctl->nact, ner = (long long)ctl->ner;
    if (walked && na == 0) return;   // every piece was reversed and attached by its walk
    long long c = 0;
    GS_LOOP(i, na) {
        int v = act[i];
        int p = pold[i];
        if (mark[v] && p != v) {
            parent[p] = v;
            ++c;
        }
    }
    if (c) atomicAdd((u64 *)&ctl->reversed, (u64)c);
    GS_LOOP(i, ner) parent[chx[i]] = chy[i];
}

// Component labels: smallest vertex id per tree (drsf_labels).
__global__ void k_label_init(int n, int *tmp) {
    GS_LOOP(v, n) tmp[v] = INT_MAX;
}
__global__ void k_label_min(int n, const int *rep, int *tmp) {
    GS_LOOP(v, n) {
        int r = rep[v];
        unsigned same = __match_any_sync(__activemask(), r);
        // lanes hold increasing v: the lowest lane of each group has the minimum
        if ((threadIdx.x & 31) == __ffs(same) - 1) atomicMin(&tmp[r], (int)v);
    }
}
__global__ void k_label_out(int n, const int *rep, const int *tmp, int *out) {
    GS_LOOP(v, n) out[v] = tmp[rep[v]];
}

// Failure-detection self-test: block 1 never arrives at the barrier, so
// block 0's bounded wait runs out, latches ERR_TIMEOUT and returns.
__global__ void k_barrier_selftest(Ctl *ctl) {
    if (blockIdx.x != 0) return;
    grid_barrier(ctl, &ctl->bar[0]);
}

// ------------------------------------------------------------- wrappers

static unsigned gsz(long long n) { return grid_for(n, BLK, 152u * 16u); }

static unsigned coop_blocks(const void *fn, int nsm, int cap_per_sm) {
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, BLK, 0) != cudaSuccess || per < 1) per = 1;
    if (per > cap_per_sm) per = cap_per_sm;
    return (unsigned)(per * nsm);
}
// The vertex passes (k_aff_collect, k_active) loop over their range with
// the blocks that are resident at once: no partial last wave.
unsigned grid_vertex_pass(int nsm) {
    unsigned a = coop_blocks((const void *)k_aff_collect, nsm, 8), b = coop_blocks((const void *)k_active<IPN>, nsm, 8);
    return a < b ? a : b;
}
unsigned grid_list_pass(int nsm) { return coop_blocks((const void *)k_active<IPT>, nsm, 8); }
unsigned coop_blocks_jump(int nsm) {
    // the three root-search variants share one launch bound; take the least
    unsigned a = coop_blocks((const void *)k_jump<0>, nsm, 8), b = coop_blocks((const void *)k_jump<1>, nsm, 8),
             c = coop_blocks((const void *)k_jump<2>, nsm, 8);
    return a < b ? (a < c ? a : c) : (b < c ? b : c);
}
static unsigned coop_blocks_hook_t(const void *fn, int threads, int nsm) {
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, 0) != cudaSuccess || per < 1) per = 1;
    if (per > 1024 / threads) per = 1024 / threads;
    return (unsigned)(per * nsm);
}
unsigned coop_blocks_hook(int nsm) { return coop_blocks_hook_t((const void *)k_boruvka<1024>, 1024, nsm); }
unsigned coop_blocks_hook_small(int nsm) { return coop_blocks_hook_t((const void *)k_boruvka<256>, 256, nsm); }
unsigned coop_blocks_orient(int nsm) {
    cudaFuncSetAttribute((const void *)k_orient, cudaFuncAttributeMaxDynamicSharedMemorySize, ORIENT_SMEM_BYTES);
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void *)k_orient, ORIENT_THREADS,
                                                      ORIENT_SMEM_BYTES) != cudaSuccess ||
        per < 1)
        per = 1;
    if (per > 2) per = 2;
    return (unsigned)(per * nsm);
}
unsigned coop_blocks_mark(int nsm) { return coop_blocks((const void *)k_mark, nsm, 4); }

cudaError_t launch_begin(Ctl *ctl, int op, long long len, const int *batch, cudaStream_t s) {
    k_begin<<<1, 32, 0, s>>>(ctl, op, len, batch);
    return cudaGetLastError();
}
cudaError_t launch_aff_collect(const Dev &d, int n, const int *rep, const unsigned *aff_ep, int *A, int *rold,
                               unsigned *w, u64 *heavy, Ctl *ctl, const int *par, int *J, int roots_only,
                               cudaStream_t s) {
    k_aff_collect<<<d.grid_pass, BLK, 0, s>>>(n, rep, aff_ep, A, rold, w, heavy, ctl, par, J, roots_only);
    (void)d;
    return cudaGetLastError();
}
cudaError_t launch_detach(const Dev &d, Ctl *ctl, const int *cuts, const int *par, int *rep, Csr g, const u64 *ovf,
                          u64 ovf_cap, RowList rl, int *A, int *J1, unsigned *det_ep, unsigned *det_claim,
                          const int *rold, long long budget_v, long long budget_e, int max_levels, int *oc, int *op,
                          cudaStream_t s) {
    void *args[] = {(void *)&ctl,     (void *)&cuts,     (void *)&par,      (void *)&rep,        (void *)&g,
                    (void *)&ovf,     (void *)&ovf_cap,  (void *)&rl,       (void *)&A,          (void *)&J1,
                    (void *)&det_ep,  (void *)&det_claim, (void *)&rold,    (void *)&budget_v,   (void *)&budget_e,
                    (void *)&max_levels, (void *)&oc,    (void *)&op};
    return cudaLaunchCooperativeKernel((const void *)k_detach, d.coop_detach, BLK, args, 0, s);
}
cudaError_t launch_rootcheck(const Dev &d, Ctl *ctl, const int *cuts, const int *rold, const unsigned *rep_ep,
                             cudaStream_t s) {
    k_rootcheck<<<d.nsm, BLK, 0, s>>>(ctl, cuts, rold, rep_ep);
    return cudaGetLastError();
}
unsigned coop_blocks_detach(int nsm) { return coop_blocks((const void *)k_detach, nsm, 4); }
cudaError_t launch_jump_async(const Dev &d, const int *A, Ctl *ctl, int *J, int *X, int *Y, cudaStream_t s) {
    k_jump_async<<<d.coop_jump, BLK, 0, s>>>(A, ctl, J, X, Y);
    return cudaGetLastError();
}
cudaError_t launch_jump(const Dev &d, const int *A, int use_list, long long cnt_static, Ctl *ctl, const int *par,
                        int *J, int *J1, int *rep, RowList rl, int mode, const int *rold, unsigned *w, u64 *heavy,
                        Csr g, int sync_rounds, int *X, int *Y, const int *cuts, cudaStream_t s) {
    void *args[] = {(void *)&A,    (void *)&use_list, (void *)&cnt_static, (void *)&ctl, (void *)&par,
                    (void *)&J,    (void *)&J1,       (void *)&rep,        (void *)&rl,  (void *)&mode,
                    (void *)&rold, (void *)&w,        (void *)&heavy,      (void *)&g,   (void *)&X,
                    (void *)&Y,    (void *)&cuts};
    const void *fn = sync_rounds == 2 ? (const void *)k_jump<2>
                                      : (sync_rounds ? (const void *)k_jump<1> : (const void *)k_jump<0>);
    return cudaLaunchCooperativeKernel(fn, d.coop_jump, BLK, args, 0, s);
}
cudaError_t launch_boruvka(const Dev &d, Ctl *ctl, u64 *ck0, int *ca0, int *cb0, u64 *ck1, int *ca1, int *cb1,
                           HookSlots hs, u64 *er, long long er_cap, int init, bool large, cudaStream_t s) {
    void *args[] = {(void *)&ctl, (void *)&ck0, (void *)&ca0, (void *)&cb0, (void *)&ck1, (void *)&ca1,
                    (void *)&cb1, (void *)&hs, (void *)&er, (void *)&er_cap, (void *)&init};
    if (large)
        return cudaLaunchCooperativeKernel((const void *)k_boruvka<256>, d.coop_hook_small, 256, args, 0, s);
    return cudaLaunchCooperativeKernel((const void *)k_boruvka<1024>, d.coop_hook, 1024, args, 0, s);
}
cudaError_t launch_orient(const Dev &d, Ctl *ctl, OrientArgs a, cudaStream_t s) {
    void *args[] = {(void *)&ctl, (void *)&a};
    return cudaLaunchCooperativeKernel((const void *)k_orient, d.coop_orient, ORIENT_THREADS, args,
                                       ORIENT_SMEM_BYTES, s);
}
cudaError_t launch_walk(const Dev &d, Ctl *ctl, const int *chx, const int *chy, const int *rep, int *parent,
                        unsigned *long_ep, cudaStream_t s) {
    k_walk<<<d.grid, BLK, 0, s>>>(ctl, chx, chy, rep, parent, long_ep);
    return cudaGetLastError();
}
cudaError_t launch_active(const Dev &d, const int *L, int use_list, long long cnt_static, Ctl *ctl, int *rep,
                          const int *parent, const unsigned *sel_ep, const int *att_x, const unsigned *rep_ep,
                          const int *newrep, int *act, int *pold, int *J0, unsigned char *mark, int *aidx,
                          int *aroot, cudaStream_t s) {
    if (use_list)
        k_active<IPT><<<d.grid_list, BLK, 0, s>>>(L, use_list, cnt_static, ctl, rep, parent, sel_ep, att_x, rep_ep,
                                                  newrep, act, pold, J0, mark, aidx, aroot);
    else
        k_active<IPN><<<d.grid_pass, BLK, 0, s>>>(L, use_list, cnt_static, ctl, rep, parent, sel_ep, att_x, rep_ep,
                                                  newrep, act, pold, J0, mark, aidx, aroot);
    return cudaGetLastError();
}
cudaError_t launch_mark(const Dev &d, Ctl *ctl, const int *act, int *J0, int *J1, unsigned char *mark,
                        const int *parent, cudaStream_t s) {
    void *args[] = {(void *)&ctl, (void *)&act, (void *)&J0, (void *)&J1, (void *)&mark, (void *)&parent};
    return cudaLaunchCooperativeKernel((const void *)k_mark, d.coop_mark, BLK, args, 0, s);
}
cudaError_t launch_reverse(const Dev &d, Ctl *ctl, const int *act, const int *pold, const unsigned char *mark,
                           const int *chx, const int *chy, int *parent, int walked, cudaStream_t s) {
    k_reverse<<<d.grid, BLK, 0, s>>>(ctl, act, pold, mark, chx, chy, parent, walked);
    return cudaGetLastError();
}
cudaError_t launch_labels(int n, const int *rep, int *tmp, int *out, cudaStream_t s) {
    k_label_init<<<gsz(n), BLK, 0, s>>>(n, tmp);
    k_label_min<<<gsz(n), BLK, 0, s>>>(n, rep, tmp);
    k_label_out<<<gsz(n), BLK, 0, s>>>(n, rep, tmp, out);
    return cudaGetLastError();
}
cudaError_t launch_barrier_selftest(Ctl *ctl, cudaStream_t s) {
    void *args[] = {(void *)&ctl};
    return cudaLaunchCooperativeKernel((const void *)k_barrier_selftest, 2, 32, args, 0, s);
}
