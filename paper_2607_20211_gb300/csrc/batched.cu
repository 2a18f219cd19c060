// Batched form: many independent graphs updated by persistent kernels.
//
// The graphs live in one handle as their disjoint union: graph g owns the
// vertex range [voff[g], voff[g+1]) and the slice [boff[g], boff[g+1]) of the
// union batch.  Instead of running the grid-wide launch sequence once over
// the whole union, a persistent kernel keeps one group per graph: a group
// is a thread-block cluster (1 to 16 blocks on as many SMs, cluster
// barriers, the group's counters in the first block's shared memory reached
// through distributed shared memory).  Each group takes the next graph from
// a device-side queue and runs that graph's whole update (Algorithm 1) with
// group barriers only, then takes the next.  Graphs are put in size classes;
// each class has its own queue and its own kernel instance (block size,
// cluster size and blocks per SM tuned per class), and the classes run side
// by side on library streams.  The launch sequence of one call is captured
// once into a CUDA graph and replayed.
//
// The block-level steps follow the same readings as the grid path, so the
// result is the same forest bit for bit: minimum-key replacement edges
// (Boruvka on every cross edge), the super-tree rooted at its piece with the
// smallest root id (level-synchronous BFS over the replacement edges), paths
// reversed by one walking thread each, representatives refreshed.
#include <climits>
#include <cstring>
#include <vector>

#include <cooperative_groups.h>

#include "kernels.h"

#define BCH 2048         // candidate pool chunk (entries)
#define BMAXCH 4096      // chunks one block can hold for one graph (8M candidates)

namespace cg = cooperative_groups;

namespace {

#define BMAXCL 16        // largest cluster

// Loads of data that other blocks of the group may have written since the
// last group barrier go to L2 (each block runs on its own SM and L1).
#define GL(x) __ldcg(&(x))

// Per-group state for the graph in hand; the copy in the group's first
// block is the one in use.
struct BLocal {
    int chunk[BMAXCH];   // pool chunks holding this graph's candidates
    int nch;
    int nc;              // candidates
    int fail;
    int cnt[6];          // general per-step counters
    int ctot[BMAXCL];    // per-block totals of a group scan
    int g;
};

// The group: a cluster of `size` blocks; thread `tid` of `stride`.
struct Grp {
    BLocal *L;           // the first block's BLocal (distributed shared memory)
    BLocal *me;          // this block's own: its copy of the chunk table
    int rank, size, tid, stride;
};

__device__ __forceinline__ void gsync() { cg::this_cluster().sync(); }

__device__ __forceinline__ long long pool_at(const BLocal *L, long long i) {
    return (long long)L->chunk[i / BCH] * BCH + (i % BCH);
}

// Warp-aggregated increment of a group counter by the calling (active)
// lanes; returns this lane's slot.
__device__ __forceinline__ int gappend(int *ctr) {
    const unsigned m = __activemask();
    const int lane = threadIdx.x & 31, ld = __ffs(m) - 1;
    int base = 0;
    if (lane == ld) base = atomicAdd(ctr, __popc(m));
    base = __shfl_sync(m, base, ld);
    return base + __popc(m & ((1u << lane) - 1u));
}

// Exclusive scan of one int per thread over the block (every thread calls it).
template <int BT>
__device__ __forceinline__ int block_excl(int x, int *total) {
    __shared__ int s_w[BT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) s_w[w] = v;
    __syncthreads();
    if (w == 0) {
        int t = lane < BT / 32 ? s_w[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < BT / 32) s_w[lane] = t;
    }
    __syncthreads();
    const int before = w > 0 ? s_w[w - 1] : 0;
    *total = s_w[BT / 32 - 1];
    __syncthreads();
    return before + v - x;
}

// Exclusive scan over the group in (block rank, thread) order; every thread
// of the group calls it.
template <int BT>
__device__ __forceinline__ int grp_excl(const Grp &G, int x, int *total) {
    __shared__ int s_before, s_total;
    int btot = 0;
    const int local = block_excl<BT>(x, &btot);
    if (G.size == 1) {
        *total = btot;
        return local;
    }
    if (threadIdx.x == 0) G.L->ctot[G.rank] = btot;
    gsync();
    if (threadIdx.x == 0) {
        int before = 0, tot = 0;
        for (int r = 0; r < G.size; ++r) {
            const int t = G.L->ctot[r];
            before += r < G.rank ? t : 0;
            tot += t;
        }
        s_before = before;
        s_total = tot;
    }
    gsync();   // also keeps ctot from being overwritten by the next scan too early
    *total = s_total;
    return s_before + local;
}

// Root of x in the hook forest (path halving; no concurrent hooking).
__device__ __forceinline__ int bfind(int *comp, int x, int bound, Ctl *ctl) {
    for (int it = 0; it < bound; ++it) {
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

// Make room for `extra` more candidates (every thread of the group calls it).
// The first block hands out the chunks; every other block then copies the
// new chunk ids into its own table, so candidate addresses are looked up in
// local shared memory.
__device__ __forceinline__ bool pool_ensure(const Grp &G, const BState &S, long long extra) {
    gsync();
    if (G.tid == 0) {
        BLocal *L = G.L;
        const long long need = (long long)L->nc + extra;
        const u64 nchunks = S.pool_cap / BCH;
        while ((long long)L->nch * BCH < need && !L->fail) {
            u64 c = L->nch < BMAXCH ? atomicAdd(S.pool_ctr, 1ull) : nchunks;
            if (c >= nchunks) {
                L->fail = 1;
                atomicOr(&S.ctl->err, ERR_CAPACITY);
            } else {
                L->chunk[L->nch++] = (int)c;
            }
        }
    }
    gsync();
    if (G.rank != 0) {
        const int have = G.me->nch, now = G.L->nch;
        for (int j = have + (int)threadIdx.x; j < now; j += (int)blockDim.x) G.me->chunk[j] = G.L->chunk[j];
        __syncthreads();
        if (threadIdx.x == 0) G.me->nch = now;
        __syncthreads();
    }
    return !G.L->fail;
}

__device__ __forceinline__ void pool_put(const Grp &G, const BState &S, u64 k, int a, int b) {
    const long long p = pool_at(G.me, gappend(&G.L->nc));
    S.pk[p] = k;
    S.pa[p] = a;
    S.pb[p] = b;
}

// Slot of a piece pair in the pair table, claimed if absent (*fresh tells
// whether this call claimed it), or -1 when the probes found no slot.
__device__ __forceinline__ long long pair_claim(u64 *pk, u64 mask, u64 pair, bool *fresh) {
    u64 s = hslot(pair, mask);
    for (int p = 0; p < PAIR_PROBES; ++p) {
        const u64 cur = __ldcg(&pk[s]);
        if (cur == pair) {
            *fresh = false;
            return (long long)s;
        }
        if (cur == EMPTY_KEY) {
            const u64 old = atomicCAS(&pk[s], EMPTY_KEY, pair);
            if (old == EMPTY_KEY || old == pair) {
                *fresh = old == EMPTY_KEY;
                return (long long)s;
            }
        }
        s = (s + 1) & mask;
    }
    return -1;
}

// A cross edge of a delete batch through the pair table (the supergraph
// reduction, Section III-A): lanes of a warp with the same pair of pieces
// take their minimum key first; the pair's slot keeps the minimum, and the
// lane that claims a slot lists it as a candidate (key = slot, ends -1, to
// be replaced by the pair and its minimum key after the scan).  Called by
// the lanes that hold a cross edge.
__device__ __forceinline__ void cross_edge(const Grp &G, const BState &S, u64 key, int ra, int rb) {
    const u64 pair = ra < rb ? ((u64)(unsigned)ra << 32) | (unsigned)rb : ((u64)(unsigned)rb << 32) | (unsigned)ra;
    const unsigned grp = __match_any_sync(__activemask(), pair);
    const u64 kmin = group_min_u64(grp, key);
    if ((int)(threadIdx.x & 31) != __ffs(grp) - 1) return;
    bool fresh = false;
    const long long sl = pair_claim(S.pt_pk, S.pt_mask, pair, &fresh);
    if (sl < 0) {
        const long long p = pool_at(G.me, gappend(&G.L->nc));
        S.pk[p] = kmin;
        S.pa[p] = ra;
        S.pb[p] = rb;
        return;
    }
    atomicMin(&S.pt_mk[sl], kmin);
    if (fresh) {
        const long long p = pool_at(G.me, gappend(&G.L->nc));
        S.pk[p] = (u64)sl;
        S.pa[p] = -1;
        S.pb[p] = -1;
    }
}

// Group sum of per-thread counts into L->cnt[i] (callers reset it first).
__device__ __forceinline__ void gadd(const Grp &G, int i, int v) {
    v = __reduce_add_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&G.L->cnt[i], v);
}

// ------------------------------------------------------------ insert

template <int BT>
__device__ void b_insert(const Grp &G, const BState &S, const BDesc &d, long long b0, long long b1) {
    Ctl *ctl = S.ctl;
    BLocal *L = G.L;
    if (G.tid == 0) L->cnt[0] = L->cnt[1] = L->cnt[2] = 0;
    gsync();
    // normalisation and index claim: self-loops, repeats and existing edges
    // are dropped; kept keys go to the graph's slice of nkey / nslot
    int loops = 0, drops = 0;
    for (long long i = b0 + G.tid; i < b1; i += G.stride) {
        const int u = d.batch[2 * i], v = d.batch[2 * i + 1];
        if (u == v) {
            ++loops;
            continue;
        }
        const u64 key = ekey((uint32_t)u, (uint32_t)v);
        const long long s = index_claim(S.ix, key);
        if (s == LLONG_MIN) atomicOr(&ctl->err, ERR_CAPACITY);
        if (s >= 0) {
            const int p = gappend(&L->cnt[0]);
            S.nkey[b0 + p] = key;
            S.nslot[b0 + p] = (u64)s;
        } else {
            ++drops;
        }
    }
    gadd(G, 1, loops);
    gadd(G, 2, drops);
    gsync();
    const int nb = L->cnt[0];
    // CSR append (or overflow) and the cross test rep[u] != rep[v]
    for (int j0 = 0; j0 < nb; j0 += G.stride) {
        if (!pool_ensure(G, S, G.stride)) return;
        const int j = j0 + G.tid;
        if (j < nb) {
            const u64 k = GL(S.nkey[b0 + j]);
            const u64 s = GL(S.nslot[b0 + j]);
            const uint32_t a = klo(k), b = khi(k);
            const long long oa = S.g.off[a], ob = S.g.off[b];
            const long long capa = S.g.off[a + 1] - oa, capb = S.g.off[b + 1] - ob;
            const int pa = row_slot(S.g.used, (int)a), pb = row_slot(S.g.used, (int)b);
            const bool fa = pa < capa, fb = pb < capb;
            if (fa && fb) {
                S.g.col[oa + pa] = (int)b;
                S.g.col[ob + pb] = (int)a;
                S.ix.pu[s] = (uint32_t)(oa + pa);
                S.ix.pv[s] = (uint32_t)(ob + pb);
            } else {
                const u64 o = atomicAdd(&ctl->ovf_count, 1ull);
                if (o < S.ovf_cap) {
                    S.ovf[o] = k;
                    S.ix.pu[s] = POS_OVF;
                    S.ix.pv[s] = (uint32_t)o;
                } else {
                    atomicOr(&ctl->err, ERR_CAPACITY);
                }
                atomicAdd((u64 *)&ctl->overflow_total, 1ull);
                if (fa || fb) atomicAdd((u64 *)&ctl->ctomb, 1ull);
            }
            const int ra = GL(S.rep[a]), rb = GL(S.rep[b]);
            if (ra != rb) pool_put(G, S, k, ra, rb);
        }
    }
    gsync();
    if (G.tid == 0) {
        atomicAdd(&ctl->nb, (u64)nb);
        atomicAdd((u64 *)&ctl->edges, (u64)nb);
        atomicAdd((u64 *)&ctl->self_loops, (u64)L->cnt[1]);
        atomicAdd((u64 *)&ctl->dropped, (u64)L->cnt[2]);
    }
}

// ------------------------------------------------------------ delete

template <int BT>
__device__ void b_delete(const Grp &G, const BState &S, const BDesc &d, int v0, int v1, long long b0, long long b1,
                         unsigned ep, int g) {
    Ctl *ctl = S.ctl;
    BLocal *L = G.L;
    const int ng = v1 - v0;
    if (G.tid == 0) L->cnt[0] = L->cnt[1] = L->cnt[2] = L->cnt[3] = L->cnt[4] = L->cnt[5] = 0;
    gsync();
    // normalisation, removal and the cut of deleted tree edges
    int loops = 0, drops = 0, wins = 0, cuts = 0;
    for (long long i = b0 + G.tid; i < b1; i += G.stride) {
        const int u = d.batch[2 * i], v = d.batch[2 * i + 1];
        if (u == v) {
            ++loops;
            continue;
        }
        // parent[u] changes in this step only by the cut of {u, parent[u]},
        // which only the thread deleting that edge makes
        const int par_u = GL(S.parent[u]), par_v = GL(S.parent[v]), rep_u = GL(S.rep[u]), rep_v = GL(S.rep[v]);
        const u64 key = ekey((uint32_t)u, (uint32_t)v);
        const long long s = index_find(S.ix, key);
        const bool won = s >= 0 && atomicCAS(&S.ix.key[s], key, TOMB_KEY) == key;
        if (!won) {
            ++drops;
            continue;
        }
        ++wins;
        const uint32_t pu = S.ix.pu[s], pv = S.ix.pv[s];
        if (pu == POS_OVF) {
            S.ovf[pv] = TOMB_KEY;
        } else {
            S.g.col[pu] = -1;
            S.g.col[pv] = -1;
        }
        int c = -1, rc = -1;
        if (par_u == v) {
            c = u;
            rc = rep_u;
        } else if (par_v == u) {
            c = v;
            rc = rep_v;
        }
        if (c >= 0) {
            S.parent[c] = c;
            S.st_cut[c] = ep;
            S.st_aff[rc] = ep;
            ++cuts;
        }
    }
    gadd(G, 1, loops);
    gadd(G, 2, drops);
    gadd(G, 0, wins);
    gadd(G, 3, cuts);
    gsync();
    const int nwin = L->cnt[0], ncut = L->cnt[3];
    if (G.tid == 0) {
        atomicAdd(&ctl->nb, (u64)nwin);
        atomicAdd((u64 *)&ctl->edges, (u64)(-(long long)nwin));
        atomicAdd((u64 *)&ctl->htomb, (u64)nwin);
        atomicAdd(&ctl->ncut, (u64)ncut);
        atomicAdd((u64 *)&ctl->self_loops, (u64)L->cnt[1]);
        atomicAdd((u64 *)&ctl->dropped, (u64)L->cnt[2]);
    }
    gsync();
    if (ncut == 0) return;   // no tree changed: no candidates, nothing to re-root
    if (G.tid == 0) L->cnt[0] = L->cnt[4] = 0;
    gsync();
    // vertices of the cut trees, with the jump pointers seeded by the cut forest
    for (int v = v0 + G.tid; v < v1; v += G.stride) {
        if (GL(S.st_aff[GL(S.rep[v])]) == ep) {
            const int p = gappend(&L->cnt[0]);
            S.A[v0 + p] = v;
            S.J[v] = GL(S.parent[v]);
        }
    }
    gsync();
    const int na = L->cnt[0];
    // piece root of every listed vertex: pointer jumping with path halving
    // in place (each J[x] only moves to an ancestor, so concurrent walks
    // stay correct); the root goes to R[v]
    for (int k = G.tid; k < na; k += G.stride) {
        const int v = GL(S.A[v0 + k]);
        int x = v, root = -1;
        for (int it = 0; it <= ng + 1; ++it) {
            const int p = __ldcg(&S.J[x]);
            const int gp = __ldcg(&S.J[p]);
            if (p == gp) {
                root = p;
                break;
            }
            S.J[x] = gp;
            x = gp;
        }
        if (root < 0) {
            atomicOr(&ctl->err, ERR_ROUNDS);
            root = v;
        }
        S.R[v] = root;
    }
    gsync();
    // new representatives; vertices outside their tree's root piece (the
    // piece root is a cut vertex) are the detached ones whose rows are
    // scanned (every cross edge has an endpoint in a detached piece)
    for (int k = G.tid; k < na; k += G.stride) {
        const int v = GL(S.A[v0 + k]);
        const int rn = GL(S.R[v]);
        S.rep[v] = rn;
        // rows with no entries are left out of the row list
        if (GL(S.st_cut[rn]) == ep && GL(S.g.used[v]) > 0) S.Dv[v0 + gappend(&L->cnt[4])] = v;
    }
    gsync();
    const int nd = L->cnt[4];
    // row lengths -> entry offsets (group scan in chunks); a row's append
    // cursor passes its capacity when edges went to the overflow list.  The
    // flattened entries are cut into tiles of 32; each tile records the row
    // of its first entry (tiles of graph g start at off[v0] / 32 + g, so the
    // graphs' tile ranges do not overlap).
    const long long tb = (S.g.off[v0] >> 5) + g;
    int run = 0;
    for (int k0 = 0; k0 < nd; k0 += G.stride) {
        const int k = k0 + G.tid;
        int len = 0;
        if (k < nd) {
            const int v = GL(S.Dv[v0 + k]);
            len = min(GL(S.g.used[v]), (int)(S.g.off[v + 1] - S.g.off[v]));
        }
        int tot = 0;
        const int ex = grp_excl<BT>(G, len, &tot);
        if (k < nd) {
            const int o = run + ex;
            S.roff[v0 + k] = o;
            for (int T = (o + 31) >> 5; (T << 5) < o + len; ++T) S.tile[tb + T] = k;
        }
        run += tot;
    }
    const int E = run;
    gsync();
    // cross edges: every live entry {v, w} of a detached row with rep[w] !=
    // rep[v]; emitted from v when w lies in a root piece (its row is not
    // scanned) or v < w, so each cross edge once.  Each warp of the group
    // takes a contiguous range of tiles, so a lane's successive entries sit
    // in the same rows (a hub row spans many tiles): the lane keeps the pair
    // of pieces it updated last, its table slot and the running minimum in
    // registers and writes the minimum once when the pair changes.  Room in
    // the pool is made every four rounds (a lane lists at most one
    // candidate per round).
    {
        const int lane = (int)(threadIdx.x & 31);
        const int NT = (E + 31) >> 5;
        const int W = G.stride >> 5, wid = G.tid >> 5;
        const int per = (NT + W - 1) / W;
        const int t_lo = wid * per, t_hi = min(t_lo + per, NT);
        u64 cpair = EMPTY_KEY, cslot = 0, cmin = EMPTY_KEY;
        for (int it = 0; it < per; ++it) {
            if ((it & 3) == 0 && !pool_ensure(G, S, 4LL * G.stride)) return;
            const int T = t_lo + it;
            if (T >= t_hi) continue;   // warp-uniform
            // the rows of window r0 .. r0+31 (r0 = row of the tile's first
            // entry) hold every entry of the tile (no row is empty); lane j
            // loads row r0+j's start, vertex, CSR start and piece, and each
            // lane takes its row's fields from the lane that loaded them
            const int r0 = GL(S.tile[tb + T]);
            const int wr = r0 + lane;
            const bool wok = wr < nd;
            const int wo = wok ? GL(S.roff[v0 + wr]) : INT_MAX;
            const int wv = wok ? GL(S.Dv[v0 + wr]) : 0;
            const long long wb = wok ? S.g.off[wv] : 0;
            const int wp = wok ? GL(S.rep[wv]) : 0;
            const int t0 = T << 5;
            // rows after the first that start inside the tile mark their
            // start position; an entry's row is the first row plus the
            // number of marks at or before it
            const int pos = wo - t0;
            const unsigned bit = (lane > 0 && pos >= 0 && pos < 32) ? (1u << pos) : 0u;
            const unsigned starts = __reduce_or_sync(0xffffffffu, bit);
            const int c = __popc(starts & (lane == 31 ? 0xffffffffu : ((2u << lane) - 1u)));
            const int rstart = __shfl_sync(0xffffffffu, wo, c);
            const int v = __shfl_sync(0xffffffffu, wv, c);
            const long long rb = __shfl_sync(0xffffffffu, wb, c);
            const int rv = __shfl_sync(0xffffffffu, wp, c);
            const int e = t0 + lane;
            const int w = e < E ? GL(S.g.col[rb + (e - rstart)]) : -1;
            const int rw = w >= 0 ? GL(S.rep[w]) : rv;
            const bool emit = rw != rv && (GL(S.st_cut[rw]) != ep || v < w);
            const unsigned m = __ballot_sync(0xffffffffu, emit);
            if (!emit) continue;
            const u64 key = ekey((uint32_t)v, (uint32_t)w);
            const u64 pair = rv < rw ? ((u64)(unsigned)rv << 32) | (unsigned)rw : ((u64)(unsigned)rw << 32) | (unsigned)rv;
            // one pair for the whole warp is the common case (a hub row
            // against one other piece): no match needed then
            const int ld0 = __ffs(m) - 1;
            const u64 p0 = __shfl_sync(m, pair, ld0);
            const unsigned grp = __all_sync(m, pair == p0) ? m : __match_any_sync(m, pair);
            const u64 kmin = group_min_u64(grp, key);
            if (lane != __ffs(grp) - 1) continue;
            if (pair == cpair) {
                cmin = kmin < cmin ? kmin : cmin;
                continue;
            }
            bool fresh = false;
            const long long sl = pair_claim(S.pt_pk, S.pt_mask, pair, &fresh);
            if (sl < 0) {   // no slot: a plain candidate
                const long long p = pool_at(G.me, gappend(&G.L->nc));
                S.pk[p] = kmin;
                S.pa[p] = rv;
                S.pb[p] = rw;
                continue;
            }
            if (cpair != EMPTY_KEY) atomicMin(&S.pt_mk[cslot], cmin);
            cpair = pair;
            cslot = (u64)sl;
            cmin = kmin;
            if (fresh) {
                const long long p = pool_at(G.me, gappend(&G.L->nc));
                S.pk[p] = (u64)sl;
                S.pa[p] = -1;
                S.pb[p] = -1;
            }
        }
        if (cpair != EMPTY_KEY) atomicMin(&S.pt_mk[cslot], cmin);
    }
    // this graph's overflow edges (their positions were bucketed per graph
    // before the launch; an edge this batch deleted is a tombstone by now)
    const long long o0 = S.govf_start[g], o1 = S.govf_start[g + 1];
    for (long long q0 = o0; q0 < o1; q0 += G.stride) {
        if (!pool_ensure(G, S, G.stride)) return;
        const long long q = q0 + G.tid;
        if (q < o1) {
            const u64 k = GL(S.ovf[S.govf[q]]);
            if (k != TOMB_KEY) {
                const int ra = GL(S.rep[klo(k)]), rb = GL(S.rep[khi(k)]);
                if (ra != rb) cross_edge(G, S, k, ra, rb);
            }
        }
    }
    gsync();
    // the listed pair slots become candidates (pair, minimum key); each slot
    // is emptied for later calls, its key before its pair, so a slot that
    // another group claims next starts from an empty minimum
    const int nc = G.L->nc;
    for (int i = G.tid; i < nc; i += G.stride) {
        const long long p = pool_at(G.me, i);
        if (GL(S.pa[p]) != -1) continue;
        const u64 sl = GL(S.pk[p]);
        const u64 pair = GL(S.pt_pk[sl]);
        S.pk[p] = GL(S.pt_mk[sl]);
        S.pa[p] = (int)(pair >> 32);
        S.pb[p] = (int)(pair & 0xFFFFFFFFu);
        S.pt_mk[sl] = EMPTY_KEY;
        __threadfence();
        S.pt_pk[sl] = EMPTY_KEY;
    }
    gsync();
    if (G.tid == 0) {
        atomicAdd(&ctl->naff, (u64)na);
        atomicAdd(&ctl->ndet, (u64)nd);
        atomicAdd((u64 *)&ctl->scanned, (u64)E);
    }
}

// ------------------------------------------------------------ replacement, orientation, reversal

template <int BT>
__device__ void b_replace(const Grp &G, const BState &S, int v0, int v1, unsigned ep) {
    Ctl *ctl = S.ctl;
    BLocal *L = G.L;
    const int ng = v1 - v0;
    const int bound = ng + 2;
    gsync();
    const int nc = L->nc;
    gsync();
    if (G.tid == 0) {
        atomicAdd(&ctl->ncand, (u64)nc);
        L->cnt[0] = 0;   // replacement edges
    }
    // Boruvka with minimum-key hooking over the pieces.  A candidate whose
    // ends fall in one component, or that hooked, is marked dead (key
    // EMPTY_KEY) in place; the list is not compacted, so a round costs no
    // group scan, and dead entries cost one load per round.
    for (int i = G.tid; i < nc; i += G.stride) {
        const long long p = pool_at(G.me, i);
        const int a = GL(S.pa[p]), b = GL(S.pb[p]);
        S.comp[a] = a;
        S.comp[b] = b;
    }
    if (G.tid == 0) L->cnt[1] = L->cnt[5] = 0;   // alive counts of even / odd rounds
    gsync();
    int rounds = 0;
    for (;;) {
        if (rounds >= MAX_ROUNDS) {
            if (G.tid == 0) atomicOr(&ctl->err, ERR_ROUNDS);
            return;
        }
        int *alive_ctr = (rounds & 1) ? &L->cnt[5] : &L->cnt[1];
        int alive = 0;
        for (int i = G.tid; i < nc; i += G.stride) {
            const long long p = pool_at(G.me, i);
            if (GL(S.pk[p]) == EMPTY_KEY) continue;
            const int a = bfind(S.comp, GL(S.pa[p]), bound, ctl), b = bfind(S.comp, GL(S.pb[p]), bound, ctl);
            if (a == b) {
                S.pk[p] = EMPTY_KEY;
                continue;
            }
            S.pa[p] = a;
            S.pb[p] = b;
            S.best[a] = EMPTY_KEY;
            S.best[b] = EMPTY_KEY;
            ++alive;
        }
        alive = __reduce_add_sync(0xffffffffu, alive);
        if ((threadIdx.x & 31) == 0 && alive) atomicAdd(alive_ctr, alive);
        gsync();
        const int c = *alive_ctr;
        if (G.tid == 0) *((rounds & 1) ? &L->cnt[1] : &L->cnt[5]) = 0;   // next round's count
        if (c == 0) break;
        ++rounds;
        for (int i = G.tid; i < nc; i += G.stride) {
            const long long p = pool_at(G.me, i);
            const u64 k = GL(S.pk[p]);
            if (k == EMPTY_KEY) continue;
            atomicMin(&S.best[GL(S.pa[p])], k);
            atomicMin(&S.best[GL(S.pb[p])], k);
        }
        gsync();
        // hook along minimum edges (a mutual choice hooks the larger root
        // under the smaller); each hooking edge joins E_r
        for (int i = G.tid; i < nc; i += G.stride) {
            const long long p = pool_at(G.me, i);
            const u64 k = GL(S.pk[p]);
            if (k == EMPTY_KEY) continue;
            const int a = GL(S.pa[p]), b = GL(S.pb[p]);
            const bool ba = GL(S.best[a]) == k, bb = GL(S.best[b]) == k;
            if (!(ba || bb)) continue;
            if (ba && bb) S.comp[a > b ? a : b] = a > b ? b : a;
            else if (ba) S.comp[a] = b;
            else S.comp[b] = a;
            const int pe = gappend(&L->cnt[0]);
            if (pe < ng) S.er[v0 + pe] = k;
            else atomicOr(&ctl->err, ERR_CAPACITY);
            S.pk[p] = EMPTY_KEY;
        }
        gsync();
    }
    gsync();
    const int ner = min(L->cnt[0], ng);
    gsync();
    if (G.tid == 0) {
        atomicAdd(&ctl->ner, (u64)ner);
        atomicMax((unsigned long long *)&ctl->hook_rounds, (unsigned long long)rounds);
        L->cnt[2] = 0;   // dense pieces
        L->cnt[3] = 0;   // frontier list
        L->cnt[4] = 0;   // walks
    }
    gsync();
    if (ner == 0) return;
    // dense ids of the pieces touched by E_r
    for (int j = G.tid; j < ner; j += G.stride) {
        const u64 k = GL(S.er[v0 + j]);
        const int pc[2] = {GL(S.rep[klo(k)]), GL(S.rep[khi(k)])};
        for (int s = 0; s < 2; ++s) {
            const int p = pc[s];
            if (atomicExch(&S.st_piece[p], ep) != ep) {
                const int id = atomicAdd(&L->cnt[2], 1);
                S.pidx[p] = id;
                S.plist[v0 + id] = p;
                S.pdeg[v0 + id] = 0;
                S.pcur[v0 + id] = 0;
                S.minp[p] = INT_MAX;
            }
        }
    }
    gsync();
    const int np = L->cnt[2];
    // super-root of every super-tree: its piece with the smallest root id
    for (int i = G.tid; i < np; i += G.stride) {
        const int p = GL(S.plist[v0 + i]);
        atomicMin(&S.minp[bfind(S.comp, p, bound, ctl)], p);
    }
    for (int j = G.tid; j < ner; j += G.stride) {
        const u64 k = GL(S.er[v0 + j]);
        atomicAdd(&S.pdeg[v0 + GL(S.pidx[GL(S.rep[klo(k)])])], 1);
        atomicAdd(&S.pdeg[v0 + GL(S.pidx[GL(S.rep[khi(k)])])], 1);
    }
    gsync();
    // adjacency of the super-forest (arcs by source piece)
    int run = 0;
    for (int k0 = 0; k0 < np; k0 += G.stride) {
        const int k = k0 + G.tid;
        const int dg = k < np ? GL(S.pdeg[v0 + k]) : 0;
        int tot = 0;
        const int ex = grp_excl<BT>(G, dg, &tot);
        if (k < np) S.poff[v0 + k] = run + ex;
        run += tot;
    }
    gsync();
    for (int j = G.tid; j < ner; j += G.stride) {
        const u64 k = GL(S.er[v0 + j]);
        const int ia = GL(S.pidx[GL(S.rep[klo(k)])]), ib = GL(S.pidx[GL(S.rep[khi(k)])]);
        S.adj[2LL * v0 + GL(S.poff[v0 + ia]) + atomicAdd(&S.pcur[v0 + ia], 1)] = j;
        S.adj[2LL * v0 + GL(S.poff[v0 + ib]) + atomicAdd(&S.pcur[v0 + ib], 1)] = j;
    }
    for (int i = G.tid; i < np; i += G.stride) {
        const int p = GL(S.plist[v0 + i]);
        if (GL(S.minp[bfind(S.comp, p, bound, ctl)]) == p) {
            S.st_vis[p] = ep;
            S.newroot[p] = p;
            S.flist[v0 + atomicAdd(&L->cnt[3], 1)] = p;
        }
    }
    gsync();
    // level-synchronous BFS from the super-roots: the piece Q found through
    // replacement edge {x in Q, y in P} from frontier piece P gets the
    // oriented edge x -> y (its path x -> root(Q) is reversed below).  The
    // arcs of a level's frontier are flattened (prefix sum of the frontier
    // pieces' degrees) so a hub piece's arcs spread over the whole group.
    int lo = 0, hi = L->cnt[3];
    for (int lvl = 0; lo < hi; ++lvl) {
        if (lvl > np) {
            if (G.tid == 0) atomicOr(&ctl->err, ERR_ROUNDS);
            return;
        }
        int tarcs = 0;
        for (int f0 = lo; f0 < hi; f0 += G.stride) {
            const int f = f0 + G.tid;
            const int dg = f < hi ? GL(S.pdeg[v0 + GL(S.pidx[GL(S.flist[v0 + f])])]) : 0;
            int tot = 0;
            const int ex = grp_excl<BT>(G, dg, &tot);
            if (f < hi) S.roff[v0 + (f - lo)] = tarcs + ex;
            tarcs += tot;
        }
        gsync();
        const int nf = hi - lo;
        for (int t = G.tid; t < tarcs; t += G.stride) {
            int a_lo = 0, a_hi = nf - 1;   // last frontier entry whose arc offset is <= t
            while (a_lo < a_hi) {
                const int mid = (a_lo + a_hi + 1) >> 1;
                if (GL(S.roff[v0 + mid]) <= t) a_lo = mid;
                else a_hi = mid - 1;
            }
            const int P = GL(S.flist[v0 + lo + a_lo]);
            const int a = GL(S.poff[v0 + GL(S.pidx[P])]) + (t - GL(S.roff[v0 + a_lo]));
            const u64 k = GL(S.er[v0 + GL(S.adj[2LL * v0 + a])]);
            const int xl = (int)klo(k), xh = (int)khi(k);
            const int rl = GL(S.rep[xl]), rh = GL(S.rep[xh]);
            const int Q = rl == P ? rh : rl;
            // Q is P's parent piece (visited earlier) or its child, which no
            // other frontier piece touches
            if (GL(S.st_vis[Q]) == ep) continue;
            S.st_vis[Q] = ep;
            S.newroot[Q] = GL(S.newroot[P]);
            S.st_rr[Q] = ep;
            const int w = gappend(&L->cnt[4]);
            S.chx[v0 + w] = rl == Q ? xl : xh;
            S.chy[v0 + w] = rl == Q ? xh : xl;
            S.flist[v0 + gappend(&L->cnt[3])] = Q;
        }
        gsync();
        lo = hi;
        hi = L->cnt[3];
        gsync();
    }
    gsync();
    const int nw = L->cnt[4];
    // path reversal: the paths of different pieces are disjoint, so one
    // thread walks each and reverses it in place, then attaches x -> y
    int rev = 0;
    for (int w = G.tid; w < nw; w += G.stride) {
        int prev = GL(S.chy[v0 + w]), cur = GL(S.chx[v0 + w]);
        for (int it = 0; it <= ng; ++it) {
            const int nxt = GL(S.parent[cur]);
            S.parent[cur] = prev;
            if (nxt == cur) break;
            ++rev;
            prev = cur;
            cur = nxt;
        }
    }
    if (rev) atomicAdd((u64 *)&ctl->reversed, (u64)rev);
    gsync();
    // representatives of the re-rooted pieces: their super-tree's root
    for (int v = v0 + G.tid; v < v1; v += G.stride) {
        const int r = GL(S.rep[v]);
        if (GL(S.st_rr[r]) == ep) S.rep[v] = GL(S.newroot[r]);
    }
}

// The persistent kernel of one size class: groups (clusters) take graphs
// from the class's queue until it is empty.
template <int BT>
__global__ void __launch_bounds__(BT) k_bpersist(const BState *Sp, int cls, int q_lo, int q_hi) {
    __shared__ BLocal L_own;
    const BState &S = *Sp;
    cg::cluster_group cl = cg::this_cluster();
    Grp G;
    G.rank = (int)cl.block_rank();
    G.size = (int)cl.num_blocks();
    G.tid = G.rank * BT + (int)threadIdx.x;
    G.stride = G.size * BT;
    G.L = cl.map_shared_rank(&L_own, 0);
    G.me = &L_own;
    // every block of the group reads the same skip flag, so they all leave
    // together
    if (*(volatile int *)&S.ctl->skip) return;
    const BDesc d = *S.desc;
    const unsigned ep = S.ctl->epoch;
    for (;;) {
        gsync();
        if (G.tid == 0) {
            const unsigned u = atomicAdd(&S.qctr[cls], 1u);
            G.L->g = q_lo + (int)u < q_hi ? d.order[q_lo + u] : -1;
            G.L->nch = 0;
            G.L->nc = 0;
            G.L->fail = 0;
        }
        if (threadIdx.x == 0) L_own.nch = 0;   // this block's copy of the chunk table
        gsync();
        const int g = G.L->g;
        if (g < 0) break;
        const int v0 = (int)d.voff[g], v1 = (int)d.voff[g + 1];
        const long long b0 = d.boff[g], b1 = d.boff[g + 1];
        if (d.op == DRSF_INSERT) b_insert<BT>(G, S, d, b0, b1);
        else b_delete<BT>(G, S, d, v0, v1, b0, b1, ep, g);
        gsync();
        if (!G.L->fail) b_replace<BT>(G, S, v0, v1, ep);
    }
    // no block leaves while another may still read its shared memory
    gsync();
}

// Per-call reset (the epoch and counters of the control block, the queues,
// the pool, the overflow buckets).
__global__ void k_bbegin(const BState *Sp) {
    const BState &S = *Sp;
    const BDesc d = *S.desc;
    Ctl *ctl = S.ctl;
    if (threadIdx.x == 0) {
        ctl->epoch += 1;
        ctl->skip = 0;
        ctl->op = d.op;
        ctl->nb = ctl->ncut = ctl->naff = ctl->ndet = ctl->ncand = ctl->ner = ctl->npc = ctl->nact = 0;
        ctl->scanned = ctl->self_loops = ctl->dropped = ctl->tree_cut = 0;
        ctl->hook_rounds = ctl->rank_rounds = ctl->mark_rounds = ctl->jump_rounds = ctl->reversed = 0;
        ctl->jump_visits = 0;
        ctl->td = ctl->need_root = 0;
        ctl->det_levels = ctl->det_entries = 0;
        ctl->batch_len = d.len;
        for (int i = 0; i < 8; ++i) ctl->bar[i] = 0;
        *S.pool_ctr = 0;
    }
    if (threadIdx.x < BCLASSES) S.qctr[threadIdx.x] = 0;
    for (int i = threadIdx.x; i <= d.G; i += blockDim.x) {
        S.gcnt[i] = 0;
        S.gcur[i] = 0;
    }
}

__device__ __forceinline__ int graph_of(const long long *voff, int G, long long v) {
    int lo = 0, hi = G - 1;   // last graph whose start is <= v
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (voff[mid] <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Every batch edge must have both ends in its own graph's range (an edge
// between two graphs would merge them); else the call is skipped and
// DRSF_EINVAL latched.  One warp per graph.
__global__ void k_bvalidate(const BState *Sp) {
    const BState &S = *Sp;
    const BDesc d = *S.desc;
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long g = warp; g < d.G; g += nw) {
        const long long lo = d.voff[g], hi = d.voff[g + 1];
        bool bad = d.boff[g] > d.boff[g + 1] || lo > hi;
        for (long long i = d.boff[g] + lane; !bad && i < d.boff[g + 1]; i += 32) {
            const int u = d.batch[2 * i], v = d.batch[2 * i + 1];
            if (u < lo || u >= hi || v < lo || v >= hi) bad = true;
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) {
            atomicOr(&S.ctl->err, ERR_BATCH_ID);
            S.ctl->skip = 1;
        }
    }
}

// Overflow edges bucketed per graph (delete calls): count, offsets, fill.
__global__ void k_bovf_count(const BState *Sp) {
    const BState &S = *Sp;
    if (*(volatile int *)&S.ctl->skip) return;
    const BDesc d = *S.desc;
    if (d.op != DRSF_DELETE) return;
    const long long no = (long long)min(S.ctl->ovf_count, S.ovf_cap);
    const long long vlo = d.voff[0], vhi = d.voff[d.G];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < no; i += (long long)gridDim.x * blockDim.x) {
        const u64 k = S.ovf[i];
        if (k != TOMB_KEY && klo(k) >= vlo && klo(k) < vhi) atomicAdd(&S.gcnt[graph_of(d.voff, d.G, klo(k))], 1);
    }
}
__global__ void k_bovf_scan(const BState *Sp) {
    // one block: exclusive scan of the per-graph counts into govf_start
    const BState &S = *Sp;
    const BDesc d = *S.desc;
    __shared__ long long s_run;
    if (threadIdx.x == 0) s_run = 0;
    __syncthreads();
    for (int i0 = 0; i0 <= d.G; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        const int x = i < d.G ? S.gcnt[i] : 0;
        int tot = 0;
        const int ex = block_excl<256>(x, &tot);
        if (i <= d.G) S.govf_start[i] = s_run + ex;
        __syncthreads();
        if (threadIdx.x == 0) s_run += tot;
        __syncthreads();
    }
}
__global__ void k_bovf_fill(const BState *Sp) {
    const BState &S = *Sp;
    if (*(volatile int *)&S.ctl->skip) return;
    const BDesc d = *S.desc;
    if (d.op != DRSF_DELETE) return;
    const long long no = (long long)min(S.ctl->ovf_count, S.ovf_cap);
    const long long vlo = d.voff[0], vhi = d.voff[d.G];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < no; i += (long long)gridDim.x * blockDim.x) {
        const u64 k = S.ovf[i];
        if (k == TOMB_KEY || klo(k) < vlo || klo(k) >= vhi) continue;
        const int g = graph_of(d.voff, d.G, klo(k));
        S.govf[S.govf_start[g] + atomicAdd(&S.gcur[g], 1)] = (u64)i;   // position, read again after the claim
    }
}

// Per-call state and descriptor, written in stream order ahead of the
// captured launch sequence (which reads both from device memory, so one
// captured graph serves every call with the same launch shapes).
__global__ void k_bset(BState *dst_state, BState st, BDesc *dst_desc, BDesc d) {
    *dst_state = st;
    *dst_desc = d;
}

template <int BT>
cudaError_t bpersist_launch(const BState *S, int cls, int q_lo, int q_hi, unsigned grid, int cluster, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(BT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_bpersist<BT>, S, cls, q_lo, q_hi);
}

// Blocks of a persistent launch: every cluster that fits at once (capped at
// blocks_per_sm blocks per SM when given), a multiple of the cluster size.
template <int BT>
unsigned persist_blocks(int nsm, int per_sm, int cluster) {
    if (cluster > 8) cudaFuncSetAttribute(k_bpersist<BT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void *)k_bpersist<BT>, BT, 0) != cudaSuccess ||
        occ < 1)
        occ = 1;
    if (per_sm > 0 && per_sm < occ) occ = per_sm;
    unsigned want = (unsigned)(occ * nsm);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(want);
    cfg.blockDim = dim3(BT);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, k_bpersist<BT>, &cfg) == cudaSuccess && ncl > 0 &&
        (unsigned)(ncl * cluster) < want)
        want = (unsigned)(ncl * cluster);
    cudaGetLastError();
    want -= want % (unsigned)cluster;
    return want < (unsigned)cluster ? (unsigned)cluster : want;
}

}  // namespace

cudaError_t launch_bset(BState *dst_state, const BState &st, BDesc *dst_desc, const BDesc &d, cudaStream_t s) {
    k_bset<<<1, 1, 0, s>>>(dst_state, st, dst_desc, d);
    return cudaGetLastError();
}

cudaError_t launch_bprologue(const Dev &dv, const BState *S, cudaStream_t s) {
    k_bbegin<<<1, 256, 0, s>>>(S);
    k_bvalidate<<<dv.nsm * 4, 256, 0, s>>>(S);
    k_bovf_count<<<dv.nsm * 4, 256, 0, s>>>(S);
    k_bovf_scan<<<1, 256, 0, s>>>(S);
    k_bovf_fill<<<dv.nsm * 4, 256, 0, s>>>(S);
    return cudaGetLastError();
}

unsigned bpersist_grid(int nsm, int threads, int per_sm, int cluster) {
    switch (threads) {
    case 128: return persist_blocks<128>(nsm, per_sm, cluster);
    case 256: return persist_blocks<256>(nsm, per_sm, cluster);
    case 512: return persist_blocks<512>(nsm, per_sm, cluster);
    default: return persist_blocks<1024>(nsm, per_sm, cluster);
    }
}

cudaError_t launch_bpersist(const BState *S, int cls, int q_lo, int q_hi, int threads, unsigned grid, int cluster,
                            cudaStream_t s) {
    switch (threads) {
    case 128: return bpersist_launch<128>(S, cls, q_lo, q_hi, grid, cluster, s);
    case 256: return bpersist_launch<256>(S, cls, q_lo, q_hi, grid, cluster, s);
    case 512: return bpersist_launch<512>(S, cls, q_lo, q_hi, grid, cluster, s);
    default: return bpersist_launch<1024>(S, cls, q_lo, q_hi, grid, cluster, s);
    }
}
