// Graph storage kernels: slack CSR + edge index build, batch normalisation,
// insertion and deletion of the batch ("Insert/Delete B of edges to/from G",
// Algorithm 1), and the cross-edge scans that produce the candidate set
// (key edges with rep[u] != rep[v], Section II-A).
#include <climits>

#include "kernels.h"

#define GS_LOOP(i, n) \
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)(n); \
         i += (long long)gridDim.x * blockDim.x)

// Warp-aggregated counter increment.
__device__ __forceinline__ void agg_count(long long *ctr, bool pred, long long sign = 1) {
    unsigned m = __ballot_sync(__activemask(), pred);
    if (m && (threadIdx.x & 31) == __ffs(m) - 1 && pred)
        atomicAdd((u64 *)ctr, (u64)(sign * (long long)__popc(m)));
}

// ------------------------------------------------------------------ build

__global__ void k_check_range(const int *a, long long cnt, int n, int *bad) {
    GS_LOOP(i, cnt) {
        int x = a[i];
        if (x < 0 || x >= n) atomicOr(bad, 1);
    }
}

// Deduplicate the input edge list through the index; winners are appended.
__global__ void k_create_claim(const int *edges, long long m, Index ix, u64 *dkey, u64 *dslot, u64 *cnt,
                               long long *self_loops) {
    GS_LOOP(i, m) {
        int u = edges[2 * i], v = edges[2 * i + 1];
        bool keep = false;
        u64 key = 0;
        long long s = -1;
        if (u != v) {
            key = ekey((uint32_t)u, (uint32_t)v);
            s = index_claim(ix, key);
            keep = s >= 0;
        }
        agg_count(self_loops, u == v);
        long long p = agg_append(cnt, keep);
        if (keep) {
            dkey[p] = key;
            dslot[p] = (u64)s;
        }
    }
}

__global__ void k_degree(const u64 *dkey, long long m, int *deg) {
    GS_LOOP(i, m) {
        u64 k = dkey[i];
        atomicAdd(&deg[klo(k)], 1);
        atomicAdd(&deg[khi(k)], 1);
    }
}

// Row capacity: degree plus max(4, degree / 4) free slots.
__global__ void k_caps(const int *deg, int n, long long *cap) {
    GS_LOOP(u, n) {
        int d = deg[u];
        int slack = d / 4 > 4 ? d / 4 : 4;
        cap[u] = (long long)d + slack;
    }
}

// Exclusive scan of int64: tiles of SCAN_TILE elements.
#define SCAN_ITEMS 16
#define SCAN_TILE (BLK * SCAN_ITEMS)

__device__ long long block_excl_scan_i64(long long v, long long *total) {
    __shared__ long long ws[BLK / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        long long t = lane < BLK / 32 ? ws[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < BLK / 32) ws[lane] = t;
    }
    __syncthreads();
    long long pre = (w > 0 ? ws[w - 1] : 0) + x - v;
    *total = ws[BLK / 32 - 1];
    __syncthreads();
    return pre;
}

__global__ void k_scan_tiles(const long long *in, long long n, long long *bsum) {
    long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_ITEMS;
    long long s = 0;
    for (int j = 0; j < SCAN_ITEMS; ++j)
        if (base + j < n) s += in[base + j];
    long long tot;
    block_excl_scan_i64(s, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_sums(long long *bsum, long long nb) {
    // one block: exclusive scan of nb block sums in place
    long long per = (nb + BLK - 1) / BLK;
    long long lo = threadIdx.x * per, hi = lo + per < nb ? lo + per : nb;
    long long s = 0;
    for (long long i = lo; i < hi; ++i) s += bsum[i];
    long long tot;
    long long pre = block_excl_scan_i64(s, &tot);
    for (long long i = lo; i < hi; ++i) {
        long long t = bsum[i];
        bsum[i] = pre;
        pre += t;
    }
}

__global__ void k_scan_apply(const long long *in, long long *out, long long n, const long long *bsum) {
    long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_ITEMS;
    long long s = 0;
    for (int j = 0; j < SCAN_ITEMS; ++j)
        if (base + j < n) s += in[base + j];
    long long tot;
    long long pre = block_excl_scan_i64(s, &tot) + bsum[blockIdx.x];
    for (int j = 0; j < SCAN_ITEMS; ++j)
        if (base + j < n) {
            out[base + j] = pre;
            pre += in[base + j];
        }
    if (base <= n - 1 && base + SCAN_ITEMS > n - 1) out[n] = pre;   // total after the last element
}

// Place the deduplicated edges: append to both rows, record positions.
__global__ void k_fill(const u64 *dkey, const u64 *dslot, long long m, Csr g, Index ix) {
    GS_LOOP(i, m) {
        u64 k = dkey[i];
        uint32_t a = klo(k), b = khi(k);
        int pa = atomicAdd(&g.used[a], 1), pb = atomicAdd(&g.used[b], 1);
        long long qa = g.off[a] + pa, qb = g.off[b] + pb;
        g.col[qa] = (int)b;
        g.col[qb] = (int)a;
        ix.pu[dslot[i]] = (uint32_t)qa;
        ix.pv[dslot[i]] = (uint32_t)qb;
    }
}

// ------------------------------------------------------------ per batch

// Id validation of the batch: an out-of-range id skips the whole batch.
__global__ void k_validate_batch(int n, Ctl *ctl) {
    const int *batch = ctl->batch;
    const long long len = ctl->batch_len;
    GS_LOOP(i, 2 * len) {
        int x = batch[i];
        if (x < 0 || x >= n) {
            atomicOr(&ctl->err, ERR_BATCH_ID);
            ctl->skip = 1;
        }
    }
}

// Insert, step 1 (batch normalisation): drop self-loops, repeated pairs and
// edges already in G; claim an index slot for each new edge.
__global__ void k_ins_claim(Index ix, Ctl *ctl, u64 *nkey, u64 *nslot) {
    if (*(volatile int *)&ctl->skip) return;
    const int *batch = ctl->batch;
    const long long len = ctl->batch_len;
    // block-uniform loop: counters and the list append are aggregated per
    // block (one atomic per block instead of one per warp)
    long long loops = 0, drops = 0;
    for (long long b0 = (long long)blockIdx.x * blockDim.x; b0 < len; b0 += (long long)gridDim.x * blockDim.x) {
        const long long i = b0 + threadIdx.x;
        bool keep = false;
        u64 key = 0;
        long long s = -1;
        if (i < len) {
            int u = batch[2 * i], v = batch[2 * i + 1];
            if (u != v) {
                key = ekey((uint32_t)u, (uint32_t)v);
                s = index_claim(ix, key);
                if (s == LLONG_MIN) atomicOr(&ctl->err, ERR_CAPACITY);
                keep = s >= 0;
                drops += !keep;
            } else {
                ++loops;
            }
        }
        long long p = block_append(&ctl->nb, keep);
        if (keep) {
            nkey[p] = key;
            nslot[p] = (u64)s;
        }
    }
    block_add(&ctl->self_loops, loops);
    block_add(&ctl->dropped, drops);
}

// Insert, step 2: append each new edge to both CSR rows (warp-aggregated
// row cursors are per row, so plain atomics); an edge whose row is full goes
// whole to the overflow list.  The cross test of the insert case (M = B,
// Algorithm 1) is fused here: rep[u] != rep[v] makes a candidate.  With SG
// (the supergraph variant, Section III-A) a candidate goes into the pair
// table instead, which keeps the minimum key per pair of trees (one
// super-edge per pair; k_pairs_compact then lists them); without it (HS,
// Section III-B) every cross edge is a candidate of the hooking.
template <bool SG>
__global__ void k_ins_place(const u64 *nkey, const u64 *nslot, Ctl *ctl, Csr g, Index ix, u64 *ovf, u64 ovf_cap,
                            const int *rep, PairTable pt, u64 *ck, int *ca, int *cb, u64 cand_cap, HookSlots hs) {
    if (*(volatile int *)&ctl->skip) return;
    const unsigned ep = ctl->epoch;
    long long nb = (long long)ctl->nb;
    // block-uniform loop: the candidate append is aggregated per block
    for (long long b0 = (long long)blockIdx.x * blockDim.x; b0 < nb; b0 += (long long)gridDim.x * blockDim.x) {
        const long long i = b0 + threadIdx.x;
        bool cross = false;
        int ra = 0, rb = 0;
        u64 k = 0;
        if (i < nb) {
            k = nkey[i];
            u64 s = nslot[i];
            uint32_t a = klo(k), b = khi(k);
            long long oa = g.off[a], ob = g.off[b];
            long long capa = g.off[a + 1] - oa, capb = g.off[b + 1] - ob;
            // lanes appending to the same row take consecutive slots from one
            // atomic (a hub row receives many of a batch's edges)
            int pa = row_slot(g.used, (int)a), pb = row_slot(g.used, (int)b);
            bool fa = pa < capa, fb = pb < capb;
            if (fa && fb) {
                g.col[oa + pa] = (int)b;
                g.col[ob + pb] = (int)a;
                ix.pu[s] = (uint32_t)(oa + pa);
                ix.pv[s] = (uint32_t)(ob + pb);
            } else {
                // the consumed free slot (if any) stays -1
                u64 o = atomicAdd(&ctl->ovf_count, 1ull);
                if (o < ovf_cap) {
                    ovf[o] = k;
                    ix.pu[s] = POS_OVF;
                    ix.pv[s] = (uint32_t)o;
                } else {
                    atomicOr(&ctl->err, ERR_CAPACITY);
                }
                atomicAdd((u64 *)&ctl->overflow_total, 1ull);
                if (fa || fb) atomicAdd((u64 *)&ctl->ctomb, 1ull);
            }
            ra = rep[a];
            rb = rep[b];
            cross = ra != rb;
            if (SG && cross) cross = !pair_min(pt.pk, pt.mk, pt.mask, ra, rb, k);   // no slot: plain candidate
        }
        long long p = block_append(&ctl->ncand, cross);
        if (cross) {
            if ((u64)p < cand_cap) {
                ck[p] = k;
                ca[p] = ra;
                cb[p] = rb;
                // HS: these are all the candidates, so the hooking needs no
                // initialisation phase of its own (see HookSlots)
                if (!SG) {
                    hook_slot_init(hs, ra, ep);
                    hook_slot_init(hs, rb, ep);
                }
            } else {
                atomicOr(&ctl->err, ERR_CAPACITY);
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd((u64 *)&ctl->edges, (u64)nb);
}

// Delete, step 1: normalisation (absent edges and repeats dropped), removal
// from the index and the CSR, and the tree-edge cut of Algorithm 1: for a
// deleted edge {u, v} with parent[u] == v, parent[u] <- u (either
// orientation).  The old root of a cut tree is stamped "affected"; the cut
// vertex becomes a piece root and is stamped in cut_ep.
__global__ void k_del_claim(Index ix, Csr g, u64 *ovf, int *parent, const int *rep, Ctl *ctl, unsigned *aff_ep,
                            unsigned *cut_ep, int *cutlist, unsigned *w, int *rold) {
    if (*(volatile int *)&ctl->skip) return;
    const int *batch = ctl->batch;
    const long long len = ctl->batch_len;
    unsigned ep = ctl->epoch;
    // block-uniform loop: counters and the cut list append are aggregated
    // per block (one atomic per block instead of one per warp)
    long long loops = 0, drops = 0, wins = 0;
    for (long long b0 = (long long)blockIdx.x * blockDim.x; b0 < len; b0 += (long long)gridDim.x * blockDim.x) {
        const long long i = b0 + threadIdx.x;
        int c = -1, rc = -1;
        if (i < len) {
            int u = batch[2 * i], v = batch[2 * i + 1];
            bool won = false;
            if (u != v) {
                // loaded up front, beside the index probe: parent[u] changes in
                // this kernel only by the cut of the edge {u, parent[u]}, which
                // only the thread deleting that edge makes
                const int par_u = parent[u], par_v = parent[v], rep_u = rep[u], rep_v = rep[v];
                u64 key = ekey((uint32_t)u, (uint32_t)v);
                long long s = index_find(ix, key);
                if (s >= 0) won = atomicCAS(&ix.key[s], key, TOMB_KEY) == key;
                if (won) {
                    uint32_t pu = ix.pu[s], pv = ix.pv[s];
                    if (pu == POS_OVF) {
                        ovf[pv] = TOMB_KEY;
                    } else {
                        g.col[pu] = -1;
                        g.col[pv] = -1;
                    }
                    if (par_u == v) {
                        c = u;
                        rc = rep_u;
                    } else if (par_v == u) {
                        c = v;
                        rc = rep_v;
                    }
                    if (c >= 0) {
                        parent[c] = c;
                        cut_ep[c] = ep;
                        w[c] = 0;     // c roots a new piece: its weight slot
                        rold[c] = rc; // and the old root of its tree
                    }
                }
                wins += won;
                drops += !won;
            } else {
                ++loops;
            }
        }
        {
            // stamp the cut trees' old roots; lanes cutting the same tree
            // write once (most cuts can fall in one giant tree)
            int r = rc;
            unsigned m = __ballot_sync(0xffffffffu, c >= 0);
            if (c >= 0) {
                unsigned grp = __match_any_sync(m, r);
                if ((int)(threadIdx.x & 31) == __ffs(grp) - 1) aff_ep[r] = ep;
            }
        }
        long long p = block_append(&ctl->ncut, c >= 0);
        if (c >= 0) cutlist[p] = c;
    }
    block_add(&ctl->self_loops, loops);
    block_add(&ctl->dropped, drops);
    block_add(&ctl->htomb, wins);
    block_add(&ctl->edges, -wins);
    block_add((long long *)&ctl->nb, wins);
}

// Delete, cross-edge scan (key edges M = E(G) - E(F) - B, Algorithm 1,
// restricted).  The rows of the listed vertices (every vertex outside the
// piece left out of its cut tree) are flattened by the prefix sum roff and
// cut into tiles of 32 entries, whatever rows they fall in (load balanced:
// a hub row is spread over many warps, short rows share a tile); each warp
// takes a contiguous range of tiles.  For a tile the warp loads the list
// entries of the 32 rows starting at the tile's first row (one coalesced
// load per field) and lane e takes its row's fields from the lane that
// loaded them, so an entry costs one column load and one rep gather.  A
// live neighbour x of u in another piece gives the cross edge {u, x}; every
// cross edge has a listed endpoint and, when both are listed, the smaller
// id emits it.  Parallel edges between two pieces are reduced to the one
// with the minimum key, which is the only one that can be in the minimum
// spanning forest: lanes holding the same piece pair take the minimum
// first, then one lane updates the pair table.  A pair that finds no table
// slot is emitted as a plain candidate.  This reduction is the supergraph
// variant's super-edge dedupe (SG, Section III-A); with SG false (HS,
// Section III-B) every cross edge is emitted as a candidate of the hooking.
// Entry positions are below 2^32, so the tile arithmetic is 32-bit.
template <bool SG>
__global__ void k_scan_lb(RowList rl, Ctl *ctl, Csr g, const int *rep, PairTable pt, u64 *ck, int *ca, int *cb,
                          u64 cand_cap) {
    if (*(volatile int *)&ctl->skip) return;
    const unsigned nd = (unsigned)ctl->ndet;
    if (nd == 0) return;
    const unsigned E = rl.roff[nd];
    const unsigned NT = (E + 31) >> 5;
    const int lane = threadIdx.x & 31;
    const unsigned warp = (unsigned)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const unsigned nw = (unsigned)((gridDim.x * blockDim.x) >> 5);
    if (warp == 0 && lane == 0) atomicAdd((u64 *)&ctl->scanned, (u64)E);
    const unsigned per = (NT + nw - 1) / nw;
    const unsigned t_lo = warp * per, t_hi = t_lo + per < NT ? t_lo + per : NT;
    // the pair this lane updated last, its table slot and the minimum key
    // seen for it since: a hub row repeats one piece pair over many tiles,
    // so its minimum is kept in a register and written to the table once
    // when the pair changes (no probe, and no stream of atomics on one
    // slot from every tile of the row)
    u64 cpair = EMPTY_KEY, cslot = 0, cmin = EMPTY_KEY;
    for (unsigned T = t_lo; T < t_hi; ++T) {
        const unsigned t0 = T << 5;
        // window: rows r0 .. r0+31 from the tile's first row
        const unsigned wr = (unsigned)rl.tile[T] + lane;
        const bool wok = wr < nd;
        const unsigned wv = wok ? rl.roff[wr] : 0xFFFFFFFFu;
        const int wu = wok ? rl.D[wr] : 0;
        const unsigned wb = wok ? rl.base[wr] : 0;
        const int2 wm = wok ? rl.meta[wr] : make_int2(0, 0);
        // the rows after the first that start inside this tile set a bit at
        // their start position (a row that starts before the tile wraps to
        // a large offset); the row of position p is the first row plus the
        // number of such starts at positions <= p
        const unsigned pos = wv - t0;
        const unsigned bit = (lane > 0 && pos < 32) ? (1u << pos) : 0u;
        const unsigned starts = __reduce_or_sync(0xffffffffu, bit);
        const int c = __popc(starts & (lane == 31 ? 0xffffffffu : ((2u << lane) - 1u)));
        // all lanes take part in the shuffles
        const unsigned rstart = __shfl_sync(0xffffffffu, wv, c);
        const int u = __shfl_sync(0xffffffffu, wu, c);
        const unsigned rb = __shfl_sync(0xffffffffu, wb, c);
        const int ru = __shfl_sync(0xffffffffu, wm.x, c);
        const int hp = __shfl_sync(0xffffffffu, wm.y, c);
        const unsigned e = t0 + lane;
        const int x = e < E ? __ldcs(&g.col[(size_t)(rb + (e - rstart))]) : -1;
        const int rx = x >= 0 ? rep[x] : 0;
        const bool emit = x >= 0 && rx != ru && (rx == hp || u < x);
        const unsigned m = __ballot_sync(0xffffffffu, emit);
        if (!m) continue;
        bool raw = false;
        u64 key = 0;
        if (!SG) {
            raw = emit;
            key = ekey((uint32_t)u, (uint32_t)x);
        } else if (emit) {
            // one piece pair for the whole warp is the common case (a hub
            // row against one other piece): no match needed then
            const int ld = __ffs(m) - 1;
            const int lru = __shfl_sync(m, ru, ld), lrx = __shfl_sync(m, rx, ld);
            const unsigned grp = __all_sync(m, ru == lru && rx == lrx)
                                     ? m
                                     : __match_any_sync(m, ((u64)(unsigned)ru << 32) | (unsigned)rx);
            key = group_min_u64(grp, ekey((uint32_t)u, (uint32_t)x));
            if (lane == __ffs(grp) - 1) {
                const u64 pair = ru < rx ? ((u64)(unsigned)ru << 32) | (unsigned)rx
                                         : ((u64)(unsigned)rx << 32) | (unsigned)ru;
                if (pair == cpair) {
                    cmin = key < cmin ? key : cmin;
                } else {
                    const long long sl = pair_slot(pt.pk, pt.mask, pair);
                    if (sl >= 0) {
                        if (cpair != EMPTY_KEY) atomicMin(&pt.mk[cslot], cmin);
                        cpair = pair;
                        cslot = (u64)sl;
                        cmin = key;
                    } else {
                        raw = true;
                    }
                }
            }
        }
        const long long p = agg_append(&ctl->ncand, raw);
        if (raw) {
            if ((u64)p < cand_cap) {
                ck[p] = key;
                ca[p] = ru;
                cb[p] = rx;
            } else {
                atomicOr(&ctl->err, ERR_CAPACITY);
            }
        }
    }
    if (SG && cpair != EMPTY_KEY) atomicMin(&pt.mk[cslot], cmin);
}

// Delete, cross-edge scan of the overflow list (edges outside their rows),
// through the same pair table (SG) or straight to the candidates (HS).
template <bool SG>
__global__ void k_scan_ovf(const u64 *ovf, Ctl *ctl, const int *rep, PairTable pt, u64 *ck, int *ca, int *cb,
                           u64 cand_cap) {
    if (*(volatile int *)&ctl->skip) return;
    long long no = (long long)ctl->ovf_count;
    GS_LOOP(i, no) {
        u64 k = ovf[i];
        bool raw = false;
        int ra = -1, rb = -1;
        if (k != TOMB_KEY) {
            ra = rep[klo(k)];
            rb = rep[khi(k)];
            if (ra != rb) raw = !SG || !pair_min(pt.pk, pt.mk, pt.mask, ra, rb, k);
        }
        long long p = agg_append(&ctl->ncand, raw);
        if (raw) {
            if ((u64)p < cand_cap) {
                ck[p] = k;
                ca[p] = ra;
                cb[p] = rb;
            } else {
                atomicOr(&ctl->err, ERR_CAPACITY);
            }
        }
    }
}

// Move the pair table into the candidate list (one candidate per piece
// pair, its minimum key) and free the slots for the next batch.
__global__ void k_pairs_compact(Ctl *ctl, PairTable pt, u64 *ck, int *ca, int *cb, u64 cand_cap) {
    if (*(volatile int *)&ctl->skip) return;
    // four slots per thread and iteration, one counter reservation per
    // block (the table has far more slots than warps have lanes, and most
    // warps hold an occupied slot: a per-warp append would queue on the
    // counter)
    const long long T = (long long)pt.mask + 1;
    const long long S = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < T; base += 4 * S) {
        u64 pair[4], k[4];
        bool on[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            long long i = base + q * S + threadIdx.x;
            pair[q] = i < T ? pt.pk[i] : EMPTY_KEY;
            on[q] = pair[q] != EMPTY_KEY;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            k[q] = 0;
            if (on[q]) {
                long long i = base + q * S + threadIdx.x;
                k[q] = pt.mk[i];
                pt.pk[i] = EMPTY_KEY;
                pt.mk[i] = EMPTY_KEY;
            }
        }
        long long p[4];
        block_reserve4(&ctl->ncand, on, p);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (!on[q]) continue;
            if ((u64)p[q] < cand_cap) {
                ck[p[q]] = k[q];
                ca[p[q]] = (int)(pair[q] >> 32);
                cb[p[q]] = (int)(pair[q] & 0xFFFFFFFFu);
            } else {
                atomicOr(&ctl->err, ERR_CAPACITY);
            }
        }
    }
}

// Edge-list export (rebuild and drsf_export_edges): warp per row, pairs
// (u, x) with u < x, then the live overflow edges.
__global__ void k_extract(int n, Csr g, const u64 *ovf, const Ctl *ctl, int *out, long long cap, u64 *cnt,
                          int *bad) {
    int lane = threadIdx.x & 31;
    long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long u = warp; u < n; u += nw) {
        long long o = g.off[u];
        long long c = g.off[u + 1] - o;
        long long used = g.used[u];
        if (used > c) used = c;
        for (long long j0 = 0; j0 < used; j0 += 32) {
            long long j = j0 + lane;
            int x = j < used ? g.col[o + j] : -1;
            bool emit = x > (int)u;
            long long p = agg_append(cnt, emit);
            if (emit) {
                if (p < cap) {
                    out[2 * p] = (int)u;
                    out[2 * p + 1] = x;
                } else {
                    atomicOr(bad, 1);
                }
            }
        }
    }
    long long no = (long long)ctl->ovf_count;
    GS_LOOP(i, no) {
        u64 k = ovf[i];
        bool emit = k != TOMB_KEY;
        long long p = agg_append(cnt, emit);
        if (emit) {
            if (p < cap) {
                out[2 * p] = (int)klo(k);
                out[2 * p + 1] = (int)khi(k);
            } else {
                atomicOr(bad, 1);
            }
        }
    }
}

// DRSF_VALIDATE: every parent pointer must be an edge of G.
__global__ void k_check_tree_edges(int n, const int *parent, Index ix, int *bad) {
    GS_LOOP(v, n) {
        int p = parent[v];
        if (p != (int)v && index_find(ix, ekey((uint32_t)v, (uint32_t)p)) < 0) atomicOr(bad, 2);
    }
}

// DRSF_VALIDATE: no edge of G joins two different trees (one root per
// component, given acyclic pointers along edges of G).
__global__ void k_check_cross(const int *pairs, long long m, const int *rep, int *bad) {
    GS_LOOP(i, m) {
        if (rep[pairs[2 * i]] != rep[pairs[2 * i + 1]]) atomicOr(bad, 4);
    }
}

// ------------------------------------------------------------- wrappers

static unsigned gsz(long long n) { return grid_for(n, BLK, 152u * 16u); }

cudaError_t launch_check_range(const int *a, long long cnt, int n, int *bad, cudaStream_t s) {
    k_check_range<<<gsz(cnt), BLK, 0, s>>>(a, cnt, n, bad);
    return cudaGetLastError();
}
cudaError_t launch_create_claim(const int *edges, long long m, Index ix, u64 *dkey, u64 *dslot, u64 *cnt,
                                long long *self_loops, cudaStream_t s) {
    k_create_claim<<<gsz(m), BLK, 0, s>>>(edges, m, ix, dkey, dslot, cnt, self_loops);
    return cudaGetLastError();
}
cudaError_t launch_degree(const u64 *dkey, long long m, int *deg, cudaStream_t s) {
    k_degree<<<gsz(m), BLK, 0, s>>>(dkey, m, deg);
    return cudaGetLastError();
}
cudaError_t launch_caps(const int *deg, int n, long long *cap, cudaStream_t s) {
    k_caps<<<gsz(n), BLK, 0, s>>>(deg, n, cap);
    return cudaGetLastError();
}
cudaError_t launch_scan_i64(const long long *in, long long *out, long long n, long long *bsum, cudaStream_t s) {
    long long tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles < 1) tiles = 1;
    k_scan_tiles<<<(unsigned)tiles, BLK, 0, s>>>(in, n, bsum);
    k_scan_sums<<<1, BLK, 0, s>>>(bsum, tiles);
    k_scan_apply<<<(unsigned)tiles, BLK, 0, s>>>(in, out, n, bsum);
    return cudaGetLastError();
}
cudaError_t launch_fill(const u64 *dkey, const u64 *dslot, long long m, Csr g, Index ix, cudaStream_t s) {
    k_fill<<<gsz(m), BLK, 0, s>>>(dkey, dslot, m, g, ix);
    return cudaGetLastError();
}
// The batch kernels read the batch and its length from the control block;
// `len` only sizes their grid (a captured launch sequence is keyed by it).
cudaError_t launch_validate_batch(long long len, int n, Ctl *ctl, cudaStream_t s) {
    k_validate_batch<<<gsz(2 * len), BLK, 0, s>>>(n, ctl);
    return cudaGetLastError();
}
cudaError_t launch_ins_claim(long long len, Index ix, Ctl *ctl, u64 *nkey, u64 *nslot, cudaStream_t s) {
    k_ins_claim<<<gsz(len), BLK, 0, s>>>(ix, ctl, nkey, nslot);
    return cudaGetLastError();
}
cudaError_t launch_ins_place(const Dev &d, const u64 *nkey, const u64 *nslot, Ctl *ctl, Csr g, Index ix,
                             u64 *ovf, u64 ovf_cap, const int *rep, bool sg, PairTable pt, u64 *ck, int *ca, int *cb,
                             u64 cand_cap, HookSlots hs, cudaStream_t s) {
    if (sg)
        k_ins_place<true><<<d.grid, BLK, 0, s>>>(nkey, nslot, ctl, g, ix, ovf, ovf_cap, rep, pt, ck, ca, cb, cand_cap,
                                                 hs);
    else
        k_ins_place<false><<<d.grid, BLK, 0, s>>>(nkey, nslot, ctl, g, ix, ovf, ovf_cap, rep, pt, ck, ca, cb,
                                                  cand_cap, hs);
    return cudaGetLastError();
}
cudaError_t launch_del_claim(long long len, Index ix, Csr g, u64 *ovf, int *parent, const int *rep, Ctl *ctl,
                             unsigned *aff_ep, unsigned *cut_ep, int *cutlist, unsigned *w, int *rold,
                             cudaStream_t s) {
    k_del_claim<<<gsz(len), BLK, 0, s>>>(ix, g, ovf, parent, rep, ctl, aff_ep, cut_ep, cutlist, w, rold);
    return cudaGetLastError();
}
cudaError_t launch_scan_rows(const Dev &d, RowList rl, Ctl *ctl, Csr g, const int *rep, bool sg, PairTable pt,
                             u64 *ck, int *ca, int *cb, u64 cand_cap, cudaStream_t s) {
    if (sg)
        k_scan_lb<true><<<d.grid_scan, BLK, 0, s>>>(rl, ctl, g, rep, pt, ck, ca, cb, cand_cap);
    else
        k_scan_lb<false><<<d.grid_scan, BLK, 0, s>>>(rl, ctl, g, rep, pt, ck, ca, cb, cand_cap);
    return cudaGetLastError();
}
// Every warp of the row scan takes an equal share of the tiles, so the grid
// is exactly the blocks that are resident at once (no second wave).
unsigned scan_grid(int nsm) {
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void *)k_scan_lb<true>, BLK, 0) != cudaSuccess ||
        per < 1)
        per = 1;
    return (unsigned)(per * nsm);
}
cudaError_t launch_scan_ovf(const Dev &d, const u64 *ovf, Ctl *ctl, const int *rep, bool sg, PairTable pt, u64 *ck,
                            int *ca, int *cb, u64 cand_cap, cudaStream_t s) {
    if (sg)
        k_scan_ovf<true><<<d.nsm * 2, BLK, 0, s>>>(ovf, ctl, rep, pt, ck, ca, cb, cand_cap);
    else
        k_scan_ovf<false><<<d.nsm * 2, BLK, 0, s>>>(ovf, ctl, rep, pt, ck, ca, cb, cand_cap);
    return cudaGetLastError();
}
cudaError_t launch_pairs_compact(const Dev &d, Ctl *ctl, PairTable pt, u64 *ck, int *ca, int *cb, u64 cand_cap,
                                 cudaStream_t s) {
    k_pairs_compact<<<grid_for(((long long)pt.mask + 4) / 4, BLK, (unsigned)d.nsm * 8u), BLK, 0, s>>>(ctl, pt, ck, ca,
                                                                                                   cb, cand_cap);
    return cudaGetLastError();
}
cudaError_t launch_extract(const Dev &d, int n, Csr g, const u64 *ovf, u64 novf_max, Ctl *ctl, int *out,
                           long long cap, u64 *cnt, cudaStream_t s) {
    (void)novf_max;
    k_extract<<<d.grid, BLK, 0, s>>>(n, g, ovf, ctl, out, cap, cnt, (int *)(cnt + 1));
    return cudaGetLastError();
}
cudaError_t launch_check_tree_edges(int n, const int *parent, Index ix, int *bad, cudaStream_t s) {
    k_check_tree_edges<<<gsz(n), BLK, 0, s>>>(n, parent, ix, bad);
    return cudaGetLastError();
}
cudaError_t launch_check_cross(const int *pairs, long long m, const int *rep, int *bad, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    k_check_cross<<<gsz(m), BLK, 0, s>>>(pairs, m, rep, bad);
    return cudaGetLastError();
}
