// Host side of the D-RSF library: handle lifetime, graph storage build and
// rebuild, the per-batch launch sequence (Algorithm 1) and the C ABI of
// include/drsf.h.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "kernels.h"

namespace {

drsf_alloc_fn g_alloc = nullptr;
drsf_free_fn g_free = nullptr;
void *g_alloc_ctx = nullptr;

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct drsf_ctx {
    int n = 0;
    uint32_t flags = 0;
    int device = 0;
    Dev dev{};
    drsf_alloc_fn alloc = nullptr;
    drsf_free_fn dfree = nullptr;
    void *alloc_ctx = nullptr;
    std::vector<Buf> bufs;
    bool poisoned = false;
    int jump_sync = 2;   // root search: 2 asynchronous doubling, 1 synchronous rounds, 0 path halving
    int pending_einval = 0;
    int last_sg = 0;     // the last batch took the supergraph variant
    // captured per-batch launch sequences (CUDA graphs), valid for storage
    // generation u_gen; gen moves whenever a storage or batch buffer moves
    std::vector<std::pair<std::string, cudaGraphExec_t>> u_graphs;
    std::map<std::string, int> u_seen;   // uses of each shape (capture on the second)
    long long gen = 0, u_gen = 0;
    bool graphs_ok = true;
    cudaStream_t u_cap = nullptr;

    Ctl *ctl = nullptr;
    Ctl *ctl_host = nullptr;   // pinned

    // forest
    int *parent = nullptr, *rep = nullptr;
    // graph
    long long *off = nullptr;
    int *used = nullptr, *col = nullptr;
    long long col_cap = 0;
    Index ix{};
    u64 H = 0;
    u64 *ovf = nullptr;
    u64 ovf_cap = 0;
    // n-sized work arrays
    int *J0 = nullptr, *J1 = nullptr, *comp = nullptr, *minp = nullptr, *pidx = nullptr, *plist = nullptr;
    int *att_x = nullptr, *newrep = nullptr, *A = nullptr, *act = nullptr, *pold = nullptr, *D = nullptr;
    int *chx = nullptr, *chy = nullptr;
    unsigned *aff_ep = nullptr, *cut_ep = nullptr, *pstamp = nullptr, *att_ep = nullptr, *rep_ep = nullptr;
    unsigned *long_ep = nullptr, *hstamp = nullptr;
    unsigned *det_ep = nullptr, *det_claim = nullptr;   // top-down delete stamps
    bool detach = true;                                 // DRSF_DETACH=0 turns the top-down delete off
    long long detach_max = 1 << 15;                     // ... and it runs for batches up to this length
    bool detach_now = false;                            // this batch's choice
    u64 *best0 = nullptr, *best1 = nullptr, *er = nullptr, *heavy = nullptr;
    int *rold = nullptr, *cdeg = nullptr, *xlist = nullptr, *aidx = nullptr, *aroot = nullptr;
    int *oep = nullptr, *oeid = nullptr, *oeroot = nullptr;
    unsigned *roff = nullptr, *rbase = nullptr;
    int2 *rmeta = nullptr;
    int *tile = nullptr;          // row of each 32-entry tile of the scanned rows
    long long tile_cap = 0;
    unsigned char *lf = nullptr;
    unsigned *wgt = nullptr;
    PairTable pt{};
    unsigned char *mark = nullptr;
    int *pdeg = nullptr, *pcur = nullptr, *poff = nullptr, *adj = nullptr, *apos = nullptr;
    int *val0 = nullptr, *val1 = nullptr, *nx0 = nullptr, *nx1 = nullptr;
    long long *bsum = nullptr;
    // candidates
    u64 *ck[2] = {nullptr, nullptr};
    int *ca[2] = {nullptr, nullptr}, *cb[2] = {nullptr, nullptr};
    u64 cand_cap = 0;
    // batch work
    u64 *nkey = nullptr, *nslot = nullptr;
    int *cutlist = nullptr;
    long long batch_cap = 0;
    int *stage_dev = nullptr;
    int *stage_host = nullptr;   // pinned
    long long stage_cap = 0;
    cudaEvent_t stage_done = nullptr;
    bool stage_pending = false;
    // batched form (drsf_apply_batched): persistent per-graph kernels
    bool b_ready = false;
    BState *b_state = nullptr;    // device copies of the per-call state and descriptor
    BDesc *b_desc = nullptr;
    long long b_gcap = 0;         // graphs the per-graph arrays hold
    char *b_meta = nullptr;       // device: voff (G+1) | boff (G+1) | order (G)
    char *b_meta_host = nullptr;  // pinned staging of the same
    cudaEvent_t b_meta_done = nullptr;
    bool b_meta_pending = false;
    cudaStream_t b_cap = nullptr, b_cls[BCLASSES] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t b_fork = nullptr, b_join[BCLASSES] = {nullptr, nullptr, nullptr, nullptr};
    std::vector<std::pair<std::string, cudaGraphExec_t>> b_graphs;   // captured launch sequences
    BState b_st{};                // scratch pointers (pool, stamps, lists)
    u64 b_govf_cap = 0;
    long long b_tile_cap = 0;
    // host-side bounds that decide a storage rebuild without a device read
    long long occ_bound = 0;     // index slots in use (live + deleted)
    long long ovf_bound = 0;     // overflow entries
    long long ctomb_bound = 0;   // deleted CSR entries
    long long rebuilds = 0;
    // per-phase profiling
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev;      // pairs per (batch, phase)
    std::vector<int> prof_phase;           // op * DRSF_NUM_PHASES + phase of each pair
    int prof_op = 0;
    size_t prof_used = 0;                  // pairs used
    long long prof_batches = 0;
    long long prof_launch[2][DRSF_NUM_PHASES] = {{0}};
    long long prof_nb[2] = {0, 0};
};

// Phases of one batch, in launch order.
enum {
    PH_BEGIN = 0,     // k_begin + id validation
    PH_INS_CLAIM,     // insert: normalisation + index claim
    PH_INS_PLACE,     // insert: CSR append + cross test
    PH_DEL_CLAIM,     // delete: normalisation, removal, tree-edge cut
    PH_AFF,           // delete: affected-vertex list
    PH_JUMP,          // delete: pointer jumping (representatives)
    PH_SCAN,          // delete: cross-edge scan of detached rows + overflow
    PH_HOOK,          // hook-and-compress (replacement edges)
    PH_ORIENT,        // Euler-tour orientation
    PH_ACTIVE,        // path-reversal set-up + representative refresh
    PH_MARK,          // pointer-doubling marks
    PH_REVERSE        // path walks, reversal scatter + attach
};
static const char *kPhaseNames[DRSF_NUM_PHASES] = {
    "begin", "ins_claim", "ins_place", "del_claim", "affected", "jump", "scan", "hook", "orient", "active",
    "mark", "reverse"};

static RowList rows(drsf_ctx *h) { return RowList{h->D, h->roff, h->rbase, h->rmeta, h->tile}; }
static HookSlots hook_slots(drsf_ctx *h) { return HookSlots{h->hstamp, h->comp, h->best0, h->best1}; }

static void prof_begin(drsf_ctx *h, int phase, cudaStream_t s) {
    if (!h->prof_on || 2 * (h->prof_used + 1) > h->prof_ev.size()) return;
    cudaEventRecord(h->prof_ev[2 * h->prof_used], s);
    h->prof_phase[h->prof_used] = h->prof_op * DRSF_NUM_PHASES + phase;
}
static void prof_end(drsf_ctx *h, int phase, int launches, cudaStream_t s) {
    if (!h->prof_on || 2 * (h->prof_used + 1) > h->prof_ev.size()) return;
    cudaEventRecord(h->prof_ev[2 * h->prof_used + 1], s);
    h->prof_launch[h->prof_op][phase] += launches;
    h->prof_used++;
}

// ------------------------------------------------------------- memory

static void *raw_alloc(drsf_ctx *h, size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (h->alloc) {
        p = h->alloc(bytes, (drsf_stream)s, h->alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

static void raw_free(drsf_ctx *h, void *p, cudaStream_t s) {
    if (!p) return;
    if (h->dfree) h->dfree(p, (drsf_stream)s, h->alloc_ctx);
    else cudaFree(p);
}

template <class T>
static bool halloc(drsf_ctx *h, T **out, size_t count, cudaStream_t s) {
    void *p = raw_alloc(h, count * sizeof(T), s);
    if (!p) return false;
    h->bufs.push_back({p, count * sizeof(T)});
    *out = (T *)p;
    return true;
}

template <class T>
static void hfree(drsf_ctx *h, T **ptr, cudaStream_t s) {
    if (!*ptr) return;
    for (size_t i = 0; i < h->bufs.size(); ++i)
        if (h->bufs[i].p == (void *)*ptr) {
            h->bufs.erase(h->bufs.begin() + (long)i);
            break;
        }
    raw_free(h, (void *)*ptr, s);
    *ptr = nullptr;
}

#define CK(x)                                     \
    do {                                          \
        cudaError_t e_ = (x);                     \
        if (e_ != cudaSuccess) {                  \
            cudaGetLastError();                   \
            return DRSF_ECUDA;                    \
        }                                         \
    } while (0)
#define CKA(x)                                    \
    do {                                          \
        if (!(x)) return DRSF_ENOMEM;             \
    } while (0)

static u64 pow2_at_least(u64 x) {
    u64 p = 1024;
    while (p < x) p <<= 1;
    return p;
}

// ------------------------------------------------------------ storage

// Build the slack CSR, the edge index and the overflow list from an edge
// list on the device (create and rebuild).  Synchronises `s`.
static drsf_status build_graph(drsf_ctx *h, const int *edges, long long m, cudaStream_t s, long long *m_out,
                               long long *self_loops_out, long long extra) {
    const int n = h->n;
    // index sized for load <= 0.5 with headroom for insertions, at least
    // twice the batch that asked for the rebuild
    long long headroom = std::max<long long>(std::max<long long>(m / 2, 1 << 12), 2 * extra);
    u64 H = pow2_at_least((u64)(2 * (m + headroom)));
    Index ix{};
    CKA(halloc(h, &ix.key, H, s));
    CKA(halloc(h, &ix.pu, H, s));
    CKA(halloc(h, &ix.pv, H, s));
    ix.mask = H - 1;
    CK(cudaMemsetAsync(ix.key, 0xFF, H * sizeof(u64), s));

    u64 *dkey = nullptr, *dslot = nullptr, *cnt = nullptr;
    long long *tmp64 = nullptr, *bs = nullptr;
    int *deg = nullptr;
    CKA(halloc(h, &dkey, (size_t)std::max<long long>(m, 1), s));
    CKA(halloc(h, &dslot, (size_t)std::max<long long>(m, 1), s));
    CKA(halloc(h, &cnt, 4, s));
    CKA(halloc(h, &deg, (size_t)n, s));
    CKA(halloc(h, &tmp64, (size_t)n + 1, s));
    long long tiles = ((long long)n + 4095) / 4096 + 1;
    CKA(halloc(h, &bs, (size_t)tiles, s));
    CK(cudaMemsetAsync(cnt, 0, 4 * sizeof(u64), s));
    CK(cudaMemsetAsync(deg, 0, (size_t)n * sizeof(int), s));
    if (m > 0) CK(launch_create_claim(edges, m, ix, dkey, dslot, cnt, (long long *)(cnt + 1), s));
    u64 hc[2] = {0, 0};
    CK(cudaMemcpyAsync(hc, cnt, 2 * sizeof(u64), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    long long m2 = (long long)hc[0];
    CK(launch_degree(dkey, m2, deg, s));
    CK(launch_caps(deg, n, tmp64, s));
    long long *off = nullptr;
    CKA(halloc(h, &off, (size_t)n + 1, s));
    CK(launch_scan_i64(tmp64, off, n, bs, s));
    long long total = 0;
    CK(cudaMemcpyAsync(&total, off + n, sizeof(long long), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (total >= (long long)POS_OVF - 1) return DRSF_ENOMEM;   // positions are 32-bit
    int *col = nullptr, *used = nullptr;
    CKA(halloc(h, &col, (size_t)total, s));
    CKA(halloc(h, &used, (size_t)n, s));
    CK(cudaMemsetAsync(col, 0xFF, (size_t)total * sizeof(int), s));
    CK(cudaMemsetAsync(used, 0, (size_t)n * sizeof(int), s));
    Csr g{off, used, col};
    CK(launch_fill(dkey, dslot, m2, g, ix, s));
    u64 ovf_cap = std::max<u64>(std::max<u64>(1u << 16, (u64)m2 / 16), (u64)(2 * extra));
    u64 *ovf = nullptr;
    CKA(halloc(h, &ovf, ovf_cap, s));
    // candidate buffers: every live undirected edge at most once
    u64 need = (u64)total / 2 + ovf_cap + 1024;
    if (need > h->cand_cap) {
        for (int b = 0; b < 2; ++b) {
            hfree(h, &h->ck[b], s);
            hfree(h, &h->ca[b], s);
            hfree(h, &h->cb[b], s);
        }
        for (int b = 0; b < 2; ++b) {
            CKA(halloc(h, &h->ck[b], need, s));
            CKA(halloc(h, &h->ca[b], need, s));
            CKA(halloc(h, &h->cb[b], need, s));
        }
        h->cand_cap = need;
    }
    // tiles of the scanned rows: at most one per 32 CSR slots, plus one
    const long long ntile = total / 32 + 2;
    if (ntile > h->tile_cap) {
        hfree(h, &h->tile, s);
        CKA(halloc(h, &h->tile, (size_t)ntile, s));
        h->tile_cap = ntile;
    }
    CK(cudaStreamSynchronize(s));
    // swap in
    hfree(h, &h->ix.key, s);
    hfree(h, &h->ix.pu, s);
    hfree(h, &h->ix.pv, s);
    hfree(h, &h->off, s);
    hfree(h, &h->col, s);
    hfree(h, &h->used, s);
    hfree(h, &h->ovf, s);
    h->ix = ix;
    h->H = H;
    h->off = off;
    h->col = col;
    h->used = used;
    h->col_cap = total;
    h->ovf = ovf;
    h->ovf_cap = ovf_cap;
    hfree(h, &dkey, s);
    hfree(h, &dslot, s);
    hfree(h, &cnt, s);
    hfree(h, &deg, s);
    hfree(h, &tmp64, s);
    hfree(h, &bs, s);
    h->occ_bound = m2;
    h->ovf_bound = 0;
    h->ctomb_bound = 0;
    h->gen++;   // captured launch sequences point into the old storage
    *m_out = m2;
    if (self_loops_out) *self_loops_out = (long long)hc[1];
    return DRSF_OK;
}

static drsf_status ensure_batch(drsf_ctx *h, long long len, cudaStream_t s) {
    if (len <= h->batch_cap) return DRSF_OK;
    long long cap = std::max<long long>(len, 1 << 12);
    CK(cudaStreamSynchronize(s));
    hfree(h, &h->nkey, s);
    hfree(h, &h->nslot, s);
    hfree(h, &h->cutlist, s);
    hfree(h, &h->pt.pk, s);
    hfree(h, &h->pt.mk, s);
    CKA(halloc(h, &h->nkey, (size_t)cap, s));
    CKA(halloc(h, &h->nslot, (size_t)cap, s));
    CKA(halloc(h, &h->cutlist, (size_t)cap, s));
    // pair table: room for ~2 piece pairs per batch edge at load <= 1/2
    // (a pair that finds no slot falls back to a plain candidate)
    u64 T = pow2_at_least((u64)cap * 4);
    CKA(halloc(h, &h->pt.pk, T, s));
    CKA(halloc(h, &h->pt.mk, T, s));
    CK(cudaMemsetAsync(h->pt.pk, 0xFF, T * sizeof(u64), s));
    CK(cudaMemsetAsync(h->pt.mk, 0xFF, T * sizeof(u64), s));
    h->pt.mask = T - 1;
    h->batch_cap = cap;
    h->gen++;
    return DRSF_OK;
}

static drsf_status read_ctl(drsf_ctx *h, cudaStream_t s) {
    CK(cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return DRSF_OK;
}

// Extract the live edge list and rebuild CSR + index + overflow (compacts
// deleted entries, absorbs overflow edges, resizes the index).
static drsf_status rebuild(drsf_ctx *h, cudaStream_t s, long long extra) {
    drsf_status st = read_ctl(h, s);
    if (st) return st;
    long long live = h->ctl_host->edges;
    int *tmp = nullptr;
    u64 *cnt = nullptr;
    CKA(halloc(h, &tmp, (size_t)std::max<long long>(2 * live, 2), s));
    CKA(halloc(h, &cnt, 2, s));
    CK(cudaMemsetAsync(cnt, 0, 2 * sizeof(u64), s));
    Csr g{h->off, h->used, h->col};
    CK(launch_extract(h->dev, h->n, g, h->ovf, h->ovf_cap, h->ctl, tmp, live, cnt, s));
    u64 hc[2];
    CK(cudaMemcpyAsync(hc, cnt, sizeof hc, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if ((long long)hc[0] != live || ((int *)hc)[2] != 0) {
        h->poisoned = true;
        return DRSF_EPOISONED;
    }
    long long m2 = 0;
    st = build_graph(h, tmp, live, s, &m2, nullptr, extra);
    hfree(h, &tmp, s);
    hfree(h, &cnt, s);
    if (st) return st;
    // reset the storage counters of the control block
    Ctl c = *h->ctl_host;
    c.ovf_count = 0;
    c.edges = m2;
    c.htomb = 0;
    c.ctomb = 0;
    CK(cudaMemcpyAsync(h->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    h->rebuilds++;
    return DRSF_OK;
}

// Decide from host-side bounds whether the storage could run out during a
// batch of `len`; only then read the real counts (one synchronisation) and
// rebuild if needed.
static drsf_status storage_check(drsf_ctx *h, int op, long long len, cudaStream_t s) {
    if (op == DRSF_INSERT) {
        bool maybe = h->occ_bound + len > (long long)(0.7 * (double)h->H) ||
                     h->ovf_bound + len > (long long)h->ovf_cap;
        if (maybe) {
            drsf_status st = read_ctl(h, s);
            if (st) return st;
            long long occ = h->ctl_host->edges + h->ctl_host->htomb;
            long long ovfc = (long long)h->ctl_host->ovf_count;
            h->occ_bound = occ;
            h->ovf_bound = ovfc;
            if (occ + len > (long long)(0.7 * (double)h->H) || ovfc + len > (long long)h->ovf_cap) {
                st = rebuild(h, s, len);
                if (st) return st;
            }
        }
        h->occ_bound += len;
        h->ovf_bound += len;
    } else {
        h->ctomb_bound += 2 * len;
        if (h->ctomb_bound > h->col_cap / 4) {
            drsf_status st = read_ctl(h, s);
            if (st) return st;
            // deleted CSR entries = 2 * (deleted edges) - bounded by the
            // index tombstones (each deleted edge frees two CSR entries)
            long long ct = 2 * h->ctl_host->htomb + h->ctl_host->ctomb;
            h->ctomb_bound = ct;
            if (ct > h->col_cap / 4) {
                st = rebuild(h, s, len);
                if (st) return st;
            }
        }
    }
    return DRSF_OK;
}

static void set_dev(drsf_ctx *h) {
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != h->device) cudaSetDevice(h->device);
}

// -------------------------------------------------------------- create

static drsf_status alloc_work(drsf_ctx *h, cudaStream_t s) {
    size_t n = (size_t)h->n;
    CKA(halloc(h, &h->parent, n, s));
    CKA(halloc(h, &h->rep, n, s));
    CKA(halloc(h, &h->J0, n, s));
    CKA(halloc(h, &h->J1, n, s));
    CKA(halloc(h, &h->comp, n, s));
    CKA(halloc(h, &h->minp, n, s));
    CKA(halloc(h, &h->pidx, n, s));
    CKA(halloc(h, &h->plist, n + 1, s));
    CKA(halloc(h, &h->att_x, n, s));
    CKA(halloc(h, &h->newrep, n, s));
    CKA(halloc(h, &h->A, n, s));
    CKA(halloc(h, &h->act, n, s));
    CKA(halloc(h, &h->pold, n, s));
    CKA(halloc(h, &h->D, n, s));
    CKA(halloc(h, &h->chx, n, s));
    CKA(halloc(h, &h->chy, n, s));
    CKA(halloc(h, &h->aff_ep, n, s));
    CKA(halloc(h, &h->cut_ep, n, s));
    CKA(halloc(h, &h->pstamp, n, s));
    CKA(halloc(h, &h->att_ep, n, s));
    CKA(halloc(h, &h->long_ep, n, s));
    CKA(halloc(h, &h->hstamp, n, s));
    CKA(halloc(h, &h->rep_ep, n, s));
    CKA(halloc(h, &h->det_ep, n, s));
    CKA(halloc(h, &h->det_claim, n, s));
    CKA(halloc(h, &h->best0, n, s));
    CKA(halloc(h, &h->best1, n, s));
    CKA(halloc(h, &h->heavy, n, s));
    CKA(halloc(h, &h->rold, n, s));
    CKA(halloc(h, &h->roff, n + 1, s));
    CKA(halloc(h, &h->rbase, n, s));
    CKA(halloc(h, &h->rmeta, n, s));
    CKA(halloc(h, &h->xlist, n, s));
    CKA(halloc(h, &h->aidx, n, s));
    CKA(halloc(h, &h->aroot, n, s));
    CKA(halloc(h, &h->oep, 2 * n + 2, s));
    CKA(halloc(h, &h->oeid, 2 * n + 2, s));
    CKA(halloc(h, &h->oeroot, n + 1, s));
    CKA(halloc(h, &h->cdeg, n + 1, s));
    CKA(halloc(h, &h->lf, n + 1, s));
    CKA(halloc(h, &h->wgt, n, s));
    CKA(halloc(h, &h->er, n, s));
    CKA(halloc(h, &h->mark, n, s));
    CKA(halloc(h, &h->pdeg, n + 1, s));
    CKA(halloc(h, &h->pcur, n + 1, s));
    CKA(halloc(h, &h->poff, n + 1, s));
    CKA(halloc(h, &h->adj, 2 * n + 2, s));
    CKA(halloc(h, &h->apos, 2 * n + 2, s));
    CKA(halloc(h, &h->val0, 2 * n + 2, s));
    CKA(halloc(h, &h->val1, 2 * n + 2, s));
    CKA(halloc(h, &h->nx0, 2 * n + 2, s));
    CKA(halloc(h, &h->nx1, 2 * n + 2, s));
    CKA(halloc(h, &h->bsum, 8192, s));
    CKA(halloc(h, &h->ctl, 1, s));
    unsigned *eps[] = {h->aff_ep, h->cut_ep, h->pstamp, h->att_ep, h->rep_ep, h->long_ep, h->hstamp, h->det_ep,
                       h->det_claim};
    for (unsigned *e : eps) CK(cudaMemsetAsync(e, 0, n * sizeof(unsigned), s));
    CK(cudaMemsetAsync(h->ctl, 0, sizeof(Ctl), s));
    return DRSF_OK;
}

static void destroy_all(drsf_ctx *h) {
    if (!h) return;
    set_dev(h);
    cudaDeviceSynchronize();
    for (auto &b : h->bufs) raw_free(h, b.p, nullptr);
    h->bufs.clear();
    if (h->ctl_host) cudaFreeHost(h->ctl_host);
    if (h->stage_host) cudaFreeHost(h->stage_host);
    if (h->stage_done) cudaEventDestroy(h->stage_done);
    for (cudaEvent_t e : h->prof_ev) cudaEventDestroy(e);
    for (auto &ge : h->b_graphs) cudaGraphExecDestroy(ge.second);
    for (auto &ge : h->u_graphs) cudaGraphExecDestroy(ge.second);
    if (h->u_cap) cudaStreamDestroy(h->u_cap);
    if (h->b_meta_host) cudaFreeHost(h->b_meta_host);
    if (h->b_meta_done) cudaEventDestroy(h->b_meta_done);
    if (h->b_fork) cudaEventDestroy(h->b_fork);
    if (h->b_cap) cudaStreamDestroy(h->b_cap);
    for (int c = 0; c < BCLASSES; ++c) {
        if (h->b_join[c]) cudaEventDestroy(h->b_join[c]);
        if (h->b_cls[c]) cudaStreamDestroy(h->b_cls[c]);
    }
    delete h;
}

extern "C" {

drsf_status drsf_set_allocator(drsf_alloc_fn alloc, drsf_free_fn free_fn, void *ctx) {
    if ((alloc == nullptr) != (free_fn == nullptr)) return DRSF_EINVAL;
    g_alloc = alloc;
    g_free = free_fn;
    g_alloc_ctx = ctx;
    return DRSF_OK;
}

static drsf_status create_impl(drsf_ctx *h, const int32_t *edges, int64_t m, const int32_t *parent,
                               cudaStream_t s) {
    const int n = h->n;
    drsf_status st = alloc_work(h, s);
    if (st) return st;
    st = ensure_batch(h, 1, s);
    if (st) return st;
    CK(cudaMallocHost((void **)&h->ctl_host, sizeof(Ctl)));
    int *bad = nullptr;
    CKA(halloc(h, &bad, 4, s));
    CK(cudaMemsetAsync(bad, 0, 4 * sizeof(int), s));
    if (m > 0) CK(launch_check_range(edges, 2 * m, n, bad, s));
    CK(launch_check_range(parent, n, n, bad + 1, s));
    int hb[2] = {0, 0};
    CK(cudaMemcpyAsync(hb, bad, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hb[0] || hb[1]) return DRSF_EINVAL;
    long long m2 = 0, loops = 0;
    st = build_graph(h, edges, m, s, &m2, &loops, 0);
    if (st) return st;
    CK(cudaMemcpyAsync(h->parent, parent, (size_t)n * sizeof(int), cudaMemcpyDeviceToDevice, s));
    // representatives of F by pointer jumping over all vertices
    Csr g0{h->off, h->used, h->col};
    CK(launch_jump(h->dev, nullptr, 0, n, h->ctl, h->parent, h->J0, h->J1, h->rep, rows(h), 0, h->rold, h->wgt,
                   h->heavy, g0, h->jump_sync == 2 ? 1 : h->jump_sync, h->act, h->xlist, h->cutlist, s));
    Ctl c{};
    CK(cudaMemcpyAsync(&c, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (c.err & ERR_ROUNDS) return DRSF_ENOT_FOREST;   // pointers did not converge: a cycle
    if (c.err & ERR_TIMEOUT) return DRSF_ETIMEOUT;
    if (h->flags & DRSF_VALIDATE) {
        CK(cudaMemsetAsync(bad, 0, 4 * sizeof(int), s));
        CK(launch_check_tree_edges(n, h->parent, h->ix, bad, s));
        // every live edge must join two vertices of the same tree
        int *el = nullptr;
        u64 *cnt = nullptr;
        CKA(halloc(h, &el, (size_t)std::max<long long>(2 * m2, 2), s));
        CKA(halloc(h, &cnt, 2, s));
        CK(cudaMemsetAsync(cnt, 0, 2 * sizeof(u64), s));
        Csr g{h->off, h->used, h->col};
        CK(launch_extract(h->dev, n, g, h->ovf, h->ovf_cap, h->ctl, el, m2, cnt, s));
        CK(launch_check_cross(el, m2, h->rep, bad, s));
        CK(cudaMemcpyAsync(hb, bad, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        hfree(h, &el, s);
        hfree(h, &cnt, s);
        if (hb[0]) return DRSF_ENOT_FOREST;
    }
    hfree(h, &bad, s);
    c.edges = m2;
    c.self_loops = loops;
    CK(cudaMemcpyAsync(h->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    return DRSF_OK;
}

drsf_status drsf_create(int32_t n, const int32_t *edges, int64_t m, const int32_t *parent, uint32_t flags,
                        drsf_stream stream, drsf_handle *out) {
    if (!out) return DRSF_EINVAL;
    *out = nullptr;
    if (n < 1 || m < 0 || !parent || (m > 0 && !edges)) return DRSF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    drsf_ctx *h = new (std::nothrow) drsf_ctx();
    if (!h) return DRSF_ENOMEM;
    h->n = n;
    h->flags = flags;
    h->alloc = g_alloc;
    h->dfree = g_free;
    h->alloc_ctx = g_alloc_ctx;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        delete h;
        return DRSF_ECUDA;
    }
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device);
    if (nsm < 1 || !coop) {
        delete h;
        return DRSF_ECUDA;
    }
    h->dev.nsm = nsm;
    h->dev.grid = (unsigned)nsm * 8u;
    h->dev.coop_jump = coop_blocks_jump(nsm);
    h->dev.coop_hook = coop_blocks_hook(nsm);
    h->dev.coop_hook_small = coop_blocks_hook_small(nsm);
    h->dev.coop_orient = coop_blocks_orient(nsm);
    h->dev.coop_mark = coop_blocks_mark(nsm);
    h->dev.coop_bfs = coop_blocks_bfs(nsm);
    h->dev.grid_scan = scan_grid(nsm);
    h->dev.grid_pass = grid_vertex_pass(nsm);
    h->dev.grid_list = grid_list_pass(nsm);
    h->dev.coop_et = coop_blocks_et(nsm);
    h->dev.coop_detach = coop_blocks_detach(nsm);
    // root search of a delete batch: barrier-free doubling over per-warp
    // slices by default; DRSF_JUMP=sync selects synchronous doubling rounds,
    // DRSF_JUMP=halving the in-place path-halving walks
    const char *jm = getenv("DRSF_JUMP");
    h->jump_sync = jm && strcmp(jm, "halving") == 0 ? 0 : (jm && strcmp(jm, "sync") == 0 ? 1 : 2);
    // DRSF_GRAPHS=0: launch every batch's kernels one by one instead of
    // replaying a captured CUDA graph
    const char *gr = getenv("DRSF_GRAPHS");
    h->graphs_ok = !(gr && strcmp(gr, "0") == 0);
    // DRSF_DETACH=0: deletes find their detached vertices by pointer jumping
    // over the cut trees only (no top-down search first)
    const char *dt = getenv("DRSF_DETACH");
    h->detach = !(dt && strcmp(dt, "0") == 0);
    // DRSF_DETACH_MAX: the largest delete batch that tries it first
    const char *dm = getenv("DRSF_DETACH_MAX");
    if (dm) h->detach_max = atoll(dm);
    drsf_status st = create_impl(h, edges, m, parent, s);
    if (st != DRSF_OK) {
        destroy_all(h);
        return st;
    }
    *out = h;
    return DRSF_OK;
}

// Replacement-edge variant of a batch (Section III): the supergraph (SG)
// reduction of parallel cross edges, or hooking on every cross edge (HS).
// A flag forces one; otherwise the key-edge count |M| is compared with n
// (Section V: HS suits |M| >> n in the paper's implementations, SG the
// opposite; here the hooking's cost follows the candidate count, so the
// supergraph's reduction pays off when the key edges outnumber the
// vertices).  |M| is the batch for an insert and the non-tree edges of G
// for a delete, from the host-side bound on live edges (no device read).
static bool use_supergraph(const drsf_ctx *h, int op, long long len) {
    const bool sg = (h->flags & DRSF_REPL_SG) != 0, hs = (h->flags & DRSF_REPL_HS) != 0;
    if (sg != hs) return sg;
    long long keys = op == DRSF_INSERT ? len : std::max<long long>(0, h->occ_bound - (long long)h->n);
    return keys > (long long)h->n / 16;
}

// The launch sequence of one batch after k_begin (Algorithm 1).  Its
// launches depend on the handle's storage, the operation, the
// replacement-edge variant and, for the batch kernels' grids, `glen`; the
// batch itself is read from the control block, so one captured copy of the
// sequence serves every batch with the same key.
static drsf_status launch_rest(drsf_ctx *h, int op, bool sg, long long glen, cudaStream_t s) {
    Ctl *ctl = h->ctl;
    Csr g{h->off, h->used, h->col};
    CK(launch_validate_batch(glen, h->n, ctl, s));
    prof_end(h, PH_BEGIN, 2, s);
    if (op == DRSF_INSERT) {
        // Algorithm 1, insert: F^ = F, M = B; rep of the previous batch is current
        prof_begin(h, PH_INS_CLAIM, s);
        CK(launch_ins_claim(glen, h->ix, ctl, h->nkey, h->nslot, s));
        prof_end(h, PH_INS_CLAIM, 1, s);
        prof_begin(h, PH_INS_PLACE, s);
        CK(launch_ins_place(h->dev, h->nkey, h->nslot, ctl, g, h->ix, h->ovf, h->ovf_cap, h->rep, sg, h->pt,
                            h->ck[0], h->ca[0], h->cb[0], h->cand_cap, hook_slots(h), s));
        if (sg) CK(launch_pairs_compact(h->dev, ctl, h->pt, h->ck[0], h->ca[0], h->cb[0], h->cand_cap, s));
        prof_end(h, PH_INS_PLACE, sg ? 2 : 1, s);
    } else {
        // Algorithm 1, delete: remove B, cut tree edges, re-label the cut trees
        prof_begin(h, PH_DEL_CLAIM, s);
        CK(launch_del_claim(glen, h->ix, g, h->ovf, h->parent, h->rep, ctl, h->aff_ep, h->cut_ep, h->cutlist,
                            h->wgt, h->rold, s));
        prof_end(h, PH_DEL_CLAIM, 1, s);
        if (h->detach_now) {
            // the detached vertices top-down from the cut vertices; over its
            // budget it hands over to the pointer jumping below
            prof_begin(h, PH_JUMP, s);
            const long long n = h->n;
            CK(launch_detach(h->dev, ctl, h->cutlist, h->parent, h->rep, g, h->ovf, h->ovf_cap, rows(h), h->A, h->J1,
                             h->det_ep, h->det_claim, h->rold, std::max<long long>(1 << 16, n / 8),
                             std::max<long long>(1 << 20, 4 * n), DETACH_LEVELS, h->act, h->xlist, s));
            prof_end(h, PH_JUMP, 1, s);
        }
        prof_begin(h, PH_AFF, s);
        CK(launch_aff_collect(h->dev, h->n, h->rep, h->aff_ep, h->A, h->rold, h->wgt, h->heavy, ctl, h->parent,
                              h->jump_sync == 2 ? h->J0 : nullptr, 0, s));
        prof_end(h, PH_AFF, 1, s);
        prof_begin(h, PH_JUMP, s);
        if (h->jump_sync == 2) CK(launch_jump_async(h->dev, h->A, ctl, h->J0, h->act, h->xlist, s));
        CK(launch_jump(h->dev, h->A, 1, 0, ctl, h->parent, h->J0, h->J1, h->rep, rows(h), 1, h->rold, h->wgt,
                       h->heavy, g, h->jump_sync, h->act, h->xlist, h->cutlist, s));
        prof_end(h, PH_JUMP, h->jump_sync == 2 ? 2 : 1, s);   // the asynchronous doubling is a launch of its own
        prof_begin(h, PH_SCAN, s);
        CK(launch_scan_rows(h->dev, rows(h), ctl, g, h->rep, sg, h->pt, h->ck[0], h->ca[0], h->cb[0], h->cand_cap,
                            s));
        CK(launch_scan_ovf(h->dev, h->ovf, ctl, h->rep, sg, h->pt, h->ck[0], h->ca[0], h->cb[0], h->cand_cap, s));
        if (sg) CK(launch_pairs_compact(h->dev, ctl, h->pt, h->ck[0], h->ca[0], h->cb[0], h->cand_cap, s));
        prof_end(h, PH_SCAN, sg ? 3 : 2, s);
    }
    prof_begin(h, PH_HOOK, s);
    // an HS insert's candidates all come from k_ins_place, which set up
    // their hook-forest slots; otherwise the hooking sets them up itself
    // (inside the scan of a large delete that costs more than it saves)
    CK(launch_boruvka(h->dev, ctl, h->ck[0], h->ca[0], h->cb[0], h->ck[1], h->ca[1], h->cb[1], hook_slots(h), h->er,
                      h->n, (op == DRSF_INSERT && !sg) ? 0 : 1, glen > (1 << 18), s));
    prof_end(h, PH_HOOK, 1, s);
    OrientArgs oa{};
    oa.er = h->er;
    oa.rep = h->rep;
    oa.comp = h->comp;
    oa.minp = h->minp;
    oa.pidx = h->pidx;
    oa.plist = h->plist;
    oa.pstamp = h->pstamp;
    oa.pdeg = h->pdeg;
    oa.pcur = h->pcur;
    oa.poff = h->poff;
    oa.adj = h->adj;
    oa.apos = h->apos;
    oa.val0 = h->val0;
    oa.val1 = h->val1;
    oa.nx0 = h->nx0;
    oa.nx1 = h->nx1;
    oa.bsum = h->bsum;
    oa.chx = h->chx;
    oa.chy = h->chy;
    oa.att_ep = h->att_ep;
    oa.rep_ep = h->rep_ep;
    oa.att_x = h->att_x;
    oa.newrep = h->newrep;
    oa.lf = h->lf;
    oa.cdeg = h->cdeg;
    oa.ep = h->oep;
    oa.eid = h->oeid;
    oa.eroot = h->oeroot;
    oa.cel = h->nx1;   // (the grid ranking's second buffer: unused on the one-block path)
    oa.parent = h->parent;
    oa.n = h->n;
    prof_begin(h, PH_ORIENT, s);
    CK(launch_orient(h->dev, ctl, oa, s));
    prof_end(h, PH_ORIENT, 1, s);
    // Path reversal: by default short paths are reversed by walking and only
    // the pieces with long paths go through the marks; the Euler-tour
    // variant (Algorithm 3) takes every re-rooted piece.
    const bool euler = (h->flags & DRSF_EULER_REVERSAL) != 0;
    if (!euler) {
        prof_begin(h, PH_REVERSE, s);
        CK(launch_walk(h->dev, ctl, h->chx, h->chy, h->rep, h->parent, h->long_ep, s));
        prof_end(h, PH_REVERSE, 1, s);
    }
    const unsigned *sel = euler ? h->att_ep : h->long_ep;
    prof_begin(h, PH_ACTIVE, s);
    if (op == DRSF_DELETE && h->detach_now) {
        // after a top-down delete the affected list holds the detached
        // vertices only; a root piece that was re-rooted adds its vertices
        CK(launch_rootcheck(h->dev, ctl, h->cutlist, h->rold, h->rep_ep, s));
        CK(launch_aff_collect(h->dev, h->n, h->rep, h->aff_ep, h->A, h->rold, h->wgt, h->heavy, ctl, h->parent,
                              nullptr, 1, s));
    }
    if (op == DRSF_INSERT)
        CK(launch_active(h->dev, nullptr, 0, h->n, ctl, h->rep, h->parent, sel, h->att_x, h->rep_ep, h->newrep,
                         h->act, h->pold, h->J0, h->mark, h->aidx, h->aroot, s));
    else
        CK(launch_active(h->dev, h->A, 1, 0, ctl, h->rep, h->parent, sel, h->att_x, h->rep_ep, h->newrep, h->act,
                         h->pold, h->J0, h->mark, h->aidx, h->aroot, s));
    prof_end(h, PH_ACTIVE, 1, s);
    prof_begin(h, PH_MARK, s);
    if (euler) {
        // Algorithm 3: Euler-tour intervals of the re-rooted pieces
        EtArgs ea{};
        ea.act = h->act;
        ea.pold = h->pold;
        ea.aidx = h->aidx;
        ea.aroot = h->aroot;
        ea.att_x = h->att_x;
        ea.ccnt = h->pdeg;
        ea.ccur = h->pcur;
        ea.coff = h->poff;
        ea.kids = h->adj;
        ea.kpos = h->apos;
        ea.val0 = h->val0;
        ea.val1 = h->val1;
        ea.nx0 = h->nx0;
        ea.nx1 = h->nx1;
        ea.bsum = h->bsum;
        ea.mark = h->mark;
        CK(launch_et_marks(h->dev, ctl, ea, s));
    } else {
        CK(launch_mark(h->dev, ctl, h->act, h->J0, h->J1, h->mark, h->parent, s));
    }
    prof_end(h, PH_MARK, 1, s);
    prof_begin(h, PH_REVERSE, s);
    CK(launch_reverse(h->dev, ctl, h->act, h->pold, h->mark, h->chx, h->chy, h->parent, euler ? 0 : 1, s));
    prof_end(h, PH_REVERSE, 1, s);
    return DRSF_OK;
}

// Forget the captured launch sequences (the storage they point into moved).
static void drop_graphs(drsf_ctx *h) {
    for (auto &ge : h->u_graphs) cudaGraphExecDestroy(ge.second);
    h->u_graphs.clear();
}

static drsf_status apply_impl(drsf_ctx *h, int op, const int32_t *batch, int64_t len, cudaStream_t s) {
    drsf_status st = ensure_batch(h, len, s);
    if (st) return st;
    st = storage_check(h, op, len, s);
    if (st) return st;
    const bool sg = use_supergraph(h, op, len);
    h->last_sg = sg ? 1 : 0;
    // the top-down delete for small batches: its cost follows the detached
    // vertices' rows and its levels, the pointer jumping's the cut trees
    h->detach_now = op == DRSF_DELETE && h->detach && len <= h->detach_max;
    if (h->prof_on) {
        h->prof_batches++;
        h->prof_op = op;
        h->prof_nb[op]++;
    }
    prof_begin(h, PH_BEGIN, s);
    CK(launch_begin(h->ctl, op, len, batch, s));
    // per-phase profiling brackets the phases with events: launch directly
    if (h->prof_on || !h->graphs_ok) return launch_rest(h, op, sg, len, s);
    // otherwise replay the captured sequence for this (storage, op, variant,
    // grid size class of the batch kernels); capture it on first use
    long long glen = 4096;
    while (glen < len) glen <<= 2;
    if (h->u_gen != h->gen) {
        drop_graphs(h);
        h->u_seen.clear();
        h->u_gen = h->gen;
    }
    const std::string key = std::to_string(op) + ":" + std::to_string(sg ? 1 : 0) + ":" + std::to_string(glen) +
                            ":" + std::to_string(h->detach_now ? 1 : 0);
    cudaGraphExec_t exec = nullptr;
    for (auto &ge : h->u_graphs)
        if (ge.first == key) exec = ge.second;
    if (!exec) {
        // a shape is captured on its second use: recording and instantiating
        // costs more host time than one direct launch sequence, and a
        // handle that sees a shape once (a tenant with few batches) never
        // pays it
        int &seen = h->u_seen[key];
        if (++seen < 2) return launch_rest(h, op, sg, len, s);
        // recorded on a stream of the library's own (the caller's stream may
        // be the legacy default stream, which cannot be captured); nothing
        // runs while recording, the replay below is ordered on s
        if (!h->u_cap) CK(cudaStreamCreateWithFlags(&h->u_cap, cudaStreamNonBlocking));
        CK(cudaStreamBeginCapture(h->u_cap, cudaStreamCaptureModeThreadLocal));
        drsf_status rs = launch_rest(h, op, sg, glen, h->u_cap);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->u_cap, &graph);
        if (rs == DRSF_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (rs != DRSF_OK || e != cudaSuccess || !exec) {
            // capture not possible here: launch directly from now on
            cudaGetLastError();
            h->graphs_ok = false;
            return launch_rest(h, op, sg, len, s);
        }
        if (h->u_graphs.size() >= 16) {
            cudaGraphExecDestroy(h->u_graphs.front().second);
            h->u_graphs.erase(h->u_graphs.begin());
        }
        h->u_graphs.emplace_back(key, exec);
    }
    CK(cudaGraphLaunch(exec, s));
    return DRSF_OK;
}

// ------------------------------------------------------- batched form

// Scratch of the persistent per-graph kernels, allocated on first use.
static drsf_status batched_scratch(drsf_ctx *h, cudaStream_t s) {
    if (h->b_ready) return DRSF_OK;
    const size_t n = (size_t)h->n;
    BState &b = h->b_st;
    int **iv[] = {&b.J, &b.R, &b.A, &b.Dv, &b.roff, &b.comp, &b.minp, &b.pidx, &b.plist, &b.pdeg, &b.poff, &b.pcur,
                  &b.newroot, &b.flist, &b.chx, &b.chy};
    for (int **p : iv) CKA(halloc(h, p, n + 1, s));
    CKA(halloc(h, &b.adj, 2 * n + 2, s));
    unsigned **st[] = {&b.st_aff, &b.st_cut, &b.st_piece, &b.st_vis, &b.st_rr};
    for (unsigned **p : st) {
        CKA(halloc(h, p, n + 1, s));
        CK(cudaMemsetAsync(*p, 0, (n + 1) * sizeof(unsigned), s));
    }
    CKA(halloc(h, &b.best, n + 1, s));
    CKA(halloc(h, &b.er, n + 1, s));
    CKA(halloc(h, &b.pool_ctr, 1, s));
    CKA(halloc(h, &b.qctr, BCLASSES, s));
    CKA(halloc(h, &h->b_state, 1, s));
    CKA(halloc(h, &h->b_desc, 1, s));
    CK(cudaStreamCreateWithFlags(&h->b_cap, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->b_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->b_meta_done, cudaEventDisableTiming));
    for (int c = 0; c < BCLASSES; ++c) {
        CK(cudaStreamCreateWithFlags(&h->b_cls[c], cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&h->b_join[c], cudaEventDisableTiming));
    }
    h->b_ready = true;
    return DRSF_OK;
}

// Per-graph arrays for G graphs and the candidate pool for this call.
static drsf_status batched_capacity(drsf_ctx *h, long long G, long long len, cudaStream_t s) {
    BState &b = h->b_st;
    if (G > h->b_gcap) {
        CK(cudaStreamSynchronize(s));
        if (h->b_meta_host) cudaFreeHost(h->b_meta_host);
        h->b_meta_host = nullptr;
        hfree(h, &h->b_meta, s);
        hfree(h, &b.gcnt, s);
        hfree(h, &b.gcur, s);
        hfree(h, &b.govf_start, s);
        long long cap = std::max<long long>(G, 256);
        size_t bytes = (size_t)(2 * (cap + 1)) * sizeof(long long) + (size_t)cap * sizeof(int);
        CKA(halloc(h, &h->b_meta, bytes, s));
        CK(cudaMallocHost((void **)&h->b_meta_host, bytes));
        CKA(halloc(h, &b.gcnt, (size_t)cap + 1, s));
        CKA(halloc(h, &b.gcur, (size_t)cap + 1, s));
        CKA(halloc(h, &b.govf_start, (size_t)cap + 1, s));
        h->b_gcap = cap;
        h->b_meta_pending = false;
    }
    // candidates: at most the batch (insert) or every live edge (delete),
    // plus one partly used chunk per graph
    const u64 need = (u64)std::max<long long>(len, h->col_cap / 2 + (long long)h->ovf_cap) + (u64)(G + 1) * 2048u;
    if (need > b.pool_cap) {
        CK(cudaStreamSynchronize(s));
        hfree(h, &b.pk, s);
        hfree(h, &b.pa, s);
        hfree(h, &b.pb, s);
        CKA(halloc(h, &b.pk, need, s));
        CKA(halloc(h, &b.pa, need, s));
        CKA(halloc(h, &b.pb, need, s));
        b.pool_cap = need;
    }
    // tiles of the scanned rows: graph g's start at off[first vertex] / 32 + g
    const long long ntile = h->col_cap / 32 + G + 2;
    if (ntile > h->b_tile_cap) {
        CK(cudaStreamSynchronize(s));
        hfree(h, &b.tile, s);
        CKA(halloc(h, &b.tile, (size_t)ntile, s));
        h->b_tile_cap = ntile;
    }
    // overflow buckets: as large as the overflow list (which a rebuild resizes)
    if (!b.govf || h->b_govf_cap < h->ovf_cap) {
        CK(cudaStreamSynchronize(s));
        hfree(h, &b.govf, s);
        CKA(halloc(h, &b.govf, (size_t)h->ovf_cap, s));
        h->b_govf_cap = h->ovf_cap;
    }
    return DRSF_OK;
}

drsf_status drsf_apply_batched(drsf_handle h, drsf_op op, const int32_t *batch, int64_t len, int32_t num_graphs,
                               const int64_t *vertex_offsets, const int64_t *batch_offsets,
                               const drsf_batched_class *classes, int32_t num_classes, drsf_stream stream) {
    if (!h || (op != DRSF_INSERT && op != DRSF_DELETE) || len < 0 || (len > 0 && !batch) || num_graphs < 1 ||
        !vertex_offsets || !batch_offsets || !classes || num_classes < 1 || num_classes > BCLASSES)
        return DRSF_EINVAL;
    if (h->poisoned) return DRSF_EPOISONED;
    if (len > (int64_t)1 << 31) return DRSF_EINVAL;
    const long long G = num_graphs;
    if (vertex_offsets[0] < 0 || vertex_offsets[G] > h->n || batch_offsets[0] != 0 || batch_offsets[G] != len)
        return DRSF_EINVAL;
    for (long long g = 0; g < G; ++g)
        if (vertex_offsets[g + 1] < vertex_offsets[g] || batch_offsets[g + 1] < batch_offsets[g]) return DRSF_EINVAL;
    for (int c = 0; c < num_classes; ++c) {
        const int t = classes[c].block_threads, cb = classes[c].cluster_blocks;
        if ((t != 128 && t != 256 && t != 512 && t != 1024) || classes[c].blocks_per_sm < 0) return DRSF_EINVAL;
        if (cb != 1 && cb != 2 && cb != 4 && cb != 8 && cb != 16) return DRSF_EINVAL;
        if (c > 0 && classes[c].max_vertices <= classes[c - 1].max_vertices) return DRSF_EINVAL;
    }
    set_dev(h);
    cudaStream_t s = (cudaStream_t)stream;
    drsf_status st = ensure_batch(h, len, s);
    if (st) return st;
    st = storage_check(h, op, len, s);
    if (st) return st;
    st = batched_scratch(h, s);
    if (st) return st;
    st = batched_capacity(h, G, len, s);
    if (st) return st;
    BState &b = h->b_st;
    // queue order: size class by vertex count, then the largest work first
    // (batch edges + vertices) so the long graphs start early
    std::vector<std::vector<int>> per(num_classes);
    for (long long g = 0; g < G; ++g) {
        const long long nv = vertex_offsets[g + 1] - vertex_offsets[g];
        int c = 0;
        while (c < num_classes - 1 && nv > classes[c].max_vertices) ++c;
        per[c].push_back((int)g);
    }
    char *mh = h->b_meta_host;
    if (h->b_meta_pending) CK(cudaEventSynchronize(h->b_meta_done));
    long long *voff_h = (long long *)mh, *boff_h = voff_h + (G + 1);
    int *order_h = (int *)(boff_h + (G + 1));
    memcpy(voff_h, vertex_offsets, (size_t)(G + 1) * sizeof(long long));
    memcpy(boff_h, batch_offsets, (size_t)(G + 1) * sizeof(long long));
    int q[BCLASSES + 1] = {0};
    long long pos = 0;
    for (int c = 0; c < num_classes; ++c) {
        auto &v = per[c];
        std::stable_sort(v.begin(), v.end(), [&](int x, int y) {
            long long wx = (batch_offsets[x + 1] - batch_offsets[x]) + (vertex_offsets[x + 1] - vertex_offsets[x]);
            long long wy = (batch_offsets[y + 1] - batch_offsets[y]) + (vertex_offsets[y + 1] - vertex_offsets[y]);
            return wx > wy;
        });
        q[c] = (int)pos;
        for (int g : v) order_h[pos++] = g;
    }
    q[num_classes] = (int)pos;
    const size_t mbytes = (size_t)(2 * (G + 1)) * sizeof(long long) + (size_t)G * sizeof(int);
    long long *voff_d = (long long *)h->b_meta, *boff_d = voff_d + (G + 1);
    int *order_d = (int *)(boff_d + (G + 1));
    CK(cudaMemcpyAsync(h->b_meta, mh, mbytes, cudaMemcpyHostToDevice, s));
    CK(cudaEventRecord(h->b_meta_done, s));
    h->b_meta_pending = true;
    // the per-call state: current storage pointers + scratch
    b.ctl = h->ctl;
    b.parent = h->parent;
    b.rep = h->rep;
    b.g = Csr{h->off, h->used, h->col};
    b.ix = h->ix;
    b.ovf = h->ovf;
    b.ovf_cap = h->ovf_cap;
    b.nkey = h->nkey;
    b.nslot = h->nslot;
    b.pt_pk = h->pt.pk;
    b.pt_mk = h->pt.mk;
    b.pt_mask = h->pt.mask;
    b.desc = h->b_desc;
    BDesc d{};
    d.batch = batch;
    d.len = len;
    d.voff = voff_d;
    d.boff = boff_d;
    d.order = order_d;
    d.G = (int)G;
    d.op = (int)op;
    CK(launch_bset(h->b_state, b, h->b_desc, d, s));
    // one captured launch sequence per (op, class queues, launch shapes)
    std::string key = std::to_string((int)op);
    // the classes run side by side, each on a share of the GPU in
    // proportion to its vertices (a class's grid alone would fill the GPU
    // and the classes would then run one after another)
    double vsum[BCLASSES] = {0}, vtot = 0;
    for (int c = 0; c < num_classes; ++c) {
        for (int g : per[c]) vsum[c] += (double)(vertex_offsets[g + 1] - vertex_offsets[g]) + 1.0;
        vtot += vsum[c];
    }
    unsigned grid[BCLASSES] = {0};
    for (int c = 0; c < num_classes; ++c) {
        const unsigned cb = (unsigned)classes[c].cluster_blocks;
        grid[c] = bpersist_grid(h->dev.nsm, classes[c].block_threads, classes[c].blocks_per_sm,
                                classes[c].cluster_blocks);
        if (vtot > 0 && vsum[c] < vtot) {
            unsigned share = (unsigned)((double)(grid[c] / cb) * vsum[c] / vtot) * cb;
            grid[c] = share < cb ? cb : share;
        }
        key += "|" + std::to_string(q[c]) + ":" + std::to_string(q[c + 1]) + ":" +
               std::to_string(classes[c].block_threads) + ":" + std::to_string(grid[c]) + ":" +
               std::to_string(classes[c].cluster_blocks);
    }
    cudaGraphExec_t exec = nullptr;
    for (auto &ge : h->b_graphs)
        if (ge.first == key) exec = ge.second;
    if (!exec) {
        CK(cudaStreamBeginCapture(h->b_cap, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = launch_bprologue(h->dev, h->b_state, h->b_cap);
        if (e == cudaSuccess) e = cudaEventRecord(h->b_fork, h->b_cap);
        for (int c = 0; c < num_classes && e == cudaSuccess; ++c) {
            if (q[c + 1] == q[c]) continue;
            e = cudaStreamWaitEvent(h->b_cls[c], h->b_fork, 0);
            if (e == cudaSuccess)
                e = launch_bpersist(h->b_state, c, q[c], q[c + 1], classes[c].block_threads, grid[c],
                                    classes[c].cluster_blocks, h->b_cls[c]);
            if (e == cudaSuccess) e = cudaEventRecord(h->b_join[c], h->b_cls[c]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(h->b_cap, h->b_join[c], 0);
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(h->b_cap, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return DRSF_ECUDA;
        }
        if (h->b_graphs.size() >= 8) {
            cudaGraphExecDestroy(h->b_graphs.front().second);
            h->b_graphs.erase(h->b_graphs.begin());
        }
        h->b_graphs.emplace_back(key, exec);
    }
    CK(cudaGraphLaunch(exec, s));
    h->last_sg = 0;
    return DRSF_OK;
}

drsf_status drsf_apply(drsf_handle h, drsf_op op, const int32_t *batch, int64_t len, drsf_stream stream) {
    if (!h || (op != DRSF_INSERT && op != DRSF_DELETE) || len < 0 || (len > 0 && !batch)) return DRSF_EINVAL;
    if (h->poisoned) return DRSF_EPOISONED;
    if (len > (int64_t)1 << 31) return DRSF_EINVAL;
    set_dev(h);
    return apply_impl(h, (int)op, batch, len, (cudaStream_t)stream);
}

// Host staging of drsf_apply_host sized for `len` edges (grows only).
static drsf_status ensure_stage(drsf_ctx *h, long long len, cudaStream_t s) {
    if (len > h->stage_cap) {
        CK(cudaStreamSynchronize(s));
        if (h->stage_host) cudaFreeHost(h->stage_host);
        h->stage_host = nullptr;
        hfree(h, &h->stage_dev, s);
        long long cap = std::max<long long>(len, 1 << 16);
        CK(cudaMallocHost((void **)&h->stage_host, (size_t)cap * 2 * sizeof(int)));
        CKA(halloc(h, &h->stage_dev, (size_t)cap * 2, s));
        h->stage_cap = cap;
        if (!h->stage_done) CK(cudaEventCreateWithFlags(&h->stage_done, cudaEventDisableTiming));
        h->stage_pending = false;
    }
    return DRSF_OK;
}

drsf_status drsf_reserve(drsf_handle h, int64_t max_batch, drsf_stream stream) {
    if (!h || max_batch < 0 || max_batch > (int64_t)1 << 31) return DRSF_EINVAL;
    if (h->poisoned) return DRSF_EPOISONED;
    set_dev(h);
    cudaStream_t s = (cudaStream_t)stream;
    drsf_status st = ensure_batch(h, max_batch, s);
    if (st) return st;
    st = ensure_stage(h, max_batch, s);
    if (st) return st;
    CK(cudaStreamSynchronize(s));
    return DRSF_OK;
}

drsf_status drsf_apply_host(drsf_handle h, drsf_op op, const int32_t *batch, int64_t len, drsf_stream stream) {
    if (!h || (op != DRSF_INSERT && op != DRSF_DELETE) || len < 0 || (len > 0 && !batch)) return DRSF_EINVAL;
    if (h->poisoned) return DRSF_EPOISONED;
    if (len > (int64_t)1 << 31) return DRSF_EINVAL;
    set_dev(h);
    cudaStream_t s = (cudaStream_t)stream;
    drsf_status st = ensure_stage(h, len, s);
    if (st) return st;
    if (h->stage_pending) CK(cudaEventSynchronize(h->stage_done));   // previous copy out of the staging buffer
    if (len > 0) {
        memcpy(h->stage_host, batch, (size_t)len * 2 * sizeof(int));
        CK(cudaMemcpyAsync(h->stage_dev, h->stage_host, (size_t)len * 2 * sizeof(int), cudaMemcpyHostToDevice, s));
        CK(cudaEventRecord(h->stage_done, s));
        h->stage_pending = true;
    }
    return apply_impl(h, (int)op, h->stage_dev, len, s);
}

static drsf_status latched(drsf_ctx *h) {
    int e = h->ctl_host->err;
    if (e & (ERR_TIMEOUT | ERR_CAPACITY | ERR_ROUNDS)) {
        h->poisoned = true;
        return (e & ERR_TIMEOUT) ? DRSF_ETIMEOUT : DRSF_EPOISONED;
    }
    if (e & ERR_BATCH_ID) {
        // report once, then clear the bit
        int z = e & ~ERR_BATCH_ID;
        cudaMemcpy(&h->ctl->err, &z, sizeof(int), cudaMemcpyHostToDevice);
        return DRSF_EINVAL;
    }
    return DRSF_OK;
}

drsf_status drsf_sync(drsf_handle h, drsf_stream stream) {
    if (!h) return DRSF_EINVAL;
    if (h->poisoned) return DRSF_EPOISONED;
    set_dev(h);
    drsf_status st = read_ctl(h, (cudaStream_t)stream);
    if (st) return st;
    return latched(h);
}

drsf_status drsf_parent(drsf_handle h, int32_t *out, drsf_stream stream) {
    if (!h || !out) return DRSF_EINVAL;
    if (h->poisoned) return DRSF_EPOISONED;
    set_dev(h);
    CK(cudaMemcpyAsync(out, h->parent, (size_t)h->n * sizeof(int), cudaMemcpyDeviceToDevice,
                       (cudaStream_t)stream));
    return DRSF_OK;
}

drsf_status drsf_labels(drsf_handle h, int32_t *out, drsf_stream stream) {
    if (!h || !out) return DRSF_EINVAL;
    if (h->poisoned) return DRSF_EPOISONED;
    set_dev(h);
    CK(launch_labels(h->n, h->rep, h->J1, out, (cudaStream_t)stream));
    return DRSF_OK;
}

drsf_status drsf_stats(drsf_handle h, drsf_batch_stats *out, drsf_stream stream) {
    if (!h || !out) return DRSF_EINVAL;
    if (h->poisoned) return DRSF_EPOISONED;
    set_dev(h);
    drsf_status st = read_ctl(h, (cudaStream_t)stream);
    if (st) return st;
    const Ctl &c = *h->ctl_host;
    out->batch_len = c.batch_len;
    out->self_loops = c.self_loops;
    out->dropped = c.dropped;
    out->applied = (int64_t)c.nb;
    out->tree_cut = (int64_t)c.ncut;
    out->affected = (int64_t)c.naff;
    out->detached = (int64_t)c.ndet;
    out->scanned = c.scanned;
    out->candidates = (int64_t)c.ncand;
    out->hook_rounds = c.hook_rounds;
    out->replacement = (int64_t)c.ner;
    out->rank_rounds = c.rank_rounds;
    out->active = (int64_t)c.nact;
    out->reversed = c.reversed;
    out->mark_rounds = c.mark_rounds;
    out->jump_rounds = c.jump_rounds;
    out->edges = c.edges;
    out->overflow = (int64_t)c.ovf_count;
    out->rebuilds = h->rebuilds;
    out->jump_visits = c.jump_visits;
    out->supergraph = h->last_sg;
    out->detach_levels = c.det_levels;
    out->detach_entries = c.det_entries;
    out->core_arcs = (int64_t)c.ncore;
    return latched(h);
}

int32_t drsf_num_vertices(drsf_handle h) { return h ? h->n : 0; }

int64_t drsf_num_edges(drsf_handle h, drsf_stream stream) {
    drsf_batch_stats st;
    if (drsf_stats(h, &st, stream) != DRSF_OK) return -1;
    return st.edges;
}

drsf_status drsf_export_edges(drsf_handle h, int32_t *out, int64_t cap, int64_t *m_out, drsf_stream stream) {
    if (!h || !m_out || cap < 0 || (cap > 0 && !out)) return DRSF_EINVAL;
    if (h->poisoned) return DRSF_EPOISONED;
    set_dev(h);
    cudaStream_t s = (cudaStream_t)stream;
    u64 *cnt = nullptr;
    CKA(halloc(h, &cnt, 2, s));
    CK(cudaMemsetAsync(cnt, 0, 2 * sizeof(u64), s));
    Csr g{h->off, h->used, h->col};
    CK(launch_extract(h->dev, h->n, g, h->ovf, h->ovf_cap, h->ctl, out, cap, cnt, s));
    u64 hc[2];
    CK(cudaMemcpyAsync(hc, cnt, sizeof hc, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    hfree(h, &cnt, s);
    *m_out = (int64_t)hc[0];
    return ((int *)hc)[2] ? DRSF_EINVAL : DRSF_OK;
}

drsf_status drsf_profile_start(drsf_handle h, int64_t max_batches) {
    if (!h || max_batches < 1) return DRSF_EINVAL;
    set_dev(h);
    size_t pairs = (size_t)max_batches * DRSF_NUM_PHASES;
    while (h->prof_ev.size() < 2 * pairs) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        h->prof_ev.push_back(e);
    }
    h->prof_phase.assign(pairs, 0);
    h->prof_used = 0;
    h->prof_batches = 0;
    memset(h->prof_launch, 0, sizeof h->prof_launch);
    h->prof_nb[0] = h->prof_nb[1] = 0;
    h->prof_on = true;
    return DRSF_OK;
}

drsf_status drsf_profile_stop(drsf_handle h, drsf_profile_t *out, drsf_stream stream) {
    if (!h || !out) return DRSF_EINVAL;
    set_dev(h);
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    memset(out, 0, sizeof *out);
    for (size_t i = 0; i < h->prof_used; ++i) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, h->prof_ev[2 * i], h->prof_ev[2 * i + 1]));
        int k = h->prof_phase[i];
        out->ms[k / DRSF_NUM_PHASES][k % DRSF_NUM_PHASES] += ms;
    }
    for (int o = 0; o < 2; ++o) {
        for (int i = 0; i < DRSF_NUM_PHASES; ++i) out->launches[o][i] = h->prof_launch[o][i];
        out->batches[o] = h->prof_nb[o];
    }
    h->prof_on = false;
    return DRSF_OK;
}

const char *drsf_phase_name(int phase) {
    return phase >= 0 && phase < DRSF_NUM_PHASES ? kPhaseNames[phase] : "?";
}

drsf_status drsf_static_forest(drsf_handle h, int32_t *parent_out, int32_t *labels_out, int64_t *levels_out,
                               drsf_stream stream) {
    if (!h || !parent_out) return DRSF_EINVAL;
    if (h->poisoned) return DRSF_EPOISONED;
    set_dev(h);
    cudaStream_t s = (cudaStream_t)stream;
    int *comp = labels_out ? labels_out : h->pold;
    u64 *levels = (u64 *)h->bsum;   // scratch word
    Csr g{h->off, h->used, h->col};
    CK(launch_static_forest(h->dev, h->n, g, h->ovf, h->ctl, h->J1, comp, parent_out, h->act, h->xlist, levels,
                            s));
    if (levels_out) {
        long long lv = 0;
        CK(cudaMemcpyAsync(&lv, levels, sizeof lv, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        *levels_out = lv;
    }
    return DRSF_OK;
}

drsf_status drsf_stream_create(int priority, drsf_stream *out) {
    if (!out) return DRSF_EINVAL;
    *out = nullptr;
    int lo = 0, hi = 0;
    CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    // the runtime's range runs from lo (lowest) to hi (highest, numerically
    // smaller); clamp the request into it
    int p = priority < hi ? hi : (priority > lo ? lo : priority);
    cudaStream_t s = nullptr;
    CK(cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, p));
    *out = (drsf_stream)s;
    return DRSF_OK;
}

drsf_status drsf_stream_destroy(drsf_stream stream) {
    if (!stream) return DRSF_EINVAL;
    CK(cudaStreamDestroy((cudaStream_t)stream));
    return DRSF_OK;
}

drsf_status drsf_selftest_barrier_timeout(drsf_stream stream) {
    cudaStream_t s = (cudaStream_t)stream;
    Ctl *ctl = nullptr;
    CK(cudaMalloc(&ctl, sizeof(Ctl)));
    CK(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));
    cudaError_t e = launch_barrier_selftest(ctl, s);
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, &ctl->err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(ctl);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return DRSF_ECUDA;
    }
    return (err & ERR_TIMEOUT) ? DRSF_ETIMEOUT : DRSF_OK;
}

void drsf_destroy(drsf_handle h) { destroy_all(h); }

const char *drsf_error_string(drsf_status s) {
    switch (s) {
    case DRSF_OK: return "ok";
    case DRSF_EINVAL: return "invalid argument or vertex id out of range";
    case DRSF_ENOMEM: return "device memory allocation failed";
    case DRSF_ECUDA: return "CUDA runtime error";
    case DRSF_ENOT_FOREST: return "parent is not a rooted spanning forest of the graph";
    case DRSF_ETIMEOUT: return "a bounded device-side wait timed out";
    case DRSF_EPOISONED: return "handle unusable after an earlier device fault";
    }
    return "unknown status";
}

}  // extern "C"
