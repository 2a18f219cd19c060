// Launch wrappers of the D-RSF kernels (host side).  Each wrapper enqueues
// on `s` and returns the launch status.
#pragma once

#include "common.cuh"

// Fixed launch shapes.
#define BLK 256

struct Dev {
    int nsm;
    unsigned grid;        // grid-stride kernels: nsm * 8 blocks of BLK
    unsigned coop_jump;   // cooperative kernels: co-resident block counts
    unsigned coop_hook;        // (1024-thread blocks)
    unsigned coop_hook_small;  // (256-thread blocks, for large batches)
    unsigned coop_orient;
    unsigned coop_mark;
    unsigned coop_bfs;
    unsigned coop_et;
    unsigned coop_detach;
    unsigned grid_scan;   // row scan: the co-resident block count
    unsigned grid_pass;   // passes over all n vertices (affected list, insert refresh): co-resident blocks
    unsigned grid_list;   // passes over a vertex list (delete refresh): co-resident blocks
};

// graph.cu -------------------------------------------------------------
unsigned scan_grid(int nsm);
cudaError_t launch_check_range(const int *a, long long cnt, int n, int *bad, cudaStream_t s);
cudaError_t launch_create_claim(const int *edges, long long m, Index ix, u64 *dkey, u64 *dslot, u64 *cnt,
                                long long *self_loops, cudaStream_t s);
cudaError_t launch_degree(const u64 *dkey, long long m, int *deg, cudaStream_t s);
cudaError_t launch_caps(const int *deg, int n, long long *cap, cudaStream_t s);
cudaError_t launch_scan_i64(const long long *in, long long *out, long long n, long long *bsum, cudaStream_t s);
cudaError_t launch_fill(const u64 *dkey, const u64 *dslot, long long m, Csr g, Index ix, cudaStream_t s);
// (the batch kernels read the batch from the control block; len sizes the grid)
cudaError_t launch_validate_batch(long long len, int n, Ctl *ctl, cudaStream_t s);

cudaError_t launch_del_claim(long long len, Index ix, Csr g, u64 *ovf, int *parent, const int *rep, Ctl *ctl,
                             unsigned *aff_ep, unsigned *cut_ep, int *cutlist, unsigned *w, int *rold,
                             cudaStream_t s);
// The rows a delete batch scans for cross edges, one entry per listed
// vertex u: u itself, the exclusive prefix sum of the row lengths (roff[nd]
// = total), the row's start in the CSR, and (rep[u], piece left out of the
// scan in u's tree); and for each tile of 32 consecutive entries of the
// flattened rows, the row of its first entry.
struct RowList {
    int *D;
    unsigned *roff;   // entry counts and CSR positions are below 2^32
    unsigned *base;   // (checked at build)
    int2 *meta;
    int *tile;        // tile[T] = the row holding entry 32 T (tiles of 32 entries)
};
struct PairTable {
    u64 *pk;   // piece pair key, EMPTY_KEY when free
    u64 *mk;   // minimum edge key of the pair
    u64 mask;
};
// sg: supergraph variant (pair-table dedupe to one minimum-key edge per
// pair of trees), else every cross edge is a candidate (hooking variant)
cudaError_t launch_ins_claim(long long len, Index ix, Ctl *ctl, u64 *nkey, u64 *nslot, cudaStream_t s);
// (HS: the candidates' hook-forest slots are set up here, see HookSlots)
cudaError_t launch_ins_place(const Dev &d, const u64 *nkey, const u64 *nslot, Ctl *ctl, Csr g, Index ix,
                             u64 *ovf, u64 ovf_cap, const int *rep, bool sg, PairTable pt, u64 *ck, int *ca, int *cb,
                             u64 cand_cap, HookSlots hs, cudaStream_t s);
cudaError_t launch_scan_rows(const Dev &d, RowList rl, Ctl *ctl, Csr g, const int *rep, bool sg, PairTable pt,
                             u64 *ck, int *ca, int *cb, u64 cand_cap, cudaStream_t s);
cudaError_t launch_scan_ovf(const Dev &d, const u64 *ovf, Ctl *ctl, const int *rep, bool sg, PairTable pt, u64 *ck,
                            int *ca, int *cb, u64 cand_cap, cudaStream_t s);
cudaError_t launch_pairs_compact(const Dev &d, Ctl *ctl, PairTable pt, u64 *ck, int *ca, int *cb, u64 cand_cap,
                                 cudaStream_t s);
cudaError_t launch_extract(const Dev &d, int n, Csr g, const u64 *ovf, u64 novf_max, Ctl *ctl, int *out,
                           long long cap, u64 *cnt, cudaStream_t s);
cudaError_t launch_check_tree_edges(int n, const int *parent, Index ix, int *bad, cudaStream_t s);
cudaError_t launch_check_cross(const int *pairs, long long m, const int *rep, int *bad, cudaStream_t s);

// forest.cu ------------------------------------------------------------
cudaError_t launch_begin(Ctl *ctl, int op, long long len, const int *batch, cudaStream_t s);
cudaError_t launch_aff_collect(const Dev &d, int n, const int *rep, const unsigned *aff_ep, int *A, int *rold,
                               unsigned *w, u64 *heavy, Ctl *ctl, const int *par, int *J, int roots_only,
                               cudaStream_t s);
// delete: detached vertices top-down from the cut vertices (falls back to
// the pointer jumping above when over budget); root pieces to list after it.
// DETACH_LEVELS: its level limit (measured on R-MAT, where it pays, the
// search takes 2-7 levels; on deep trees each level costs about as much as
// a whole pointer-jumping round)
#define DETACH_LEVELS 16
cudaError_t launch_detach(const Dev &d, Ctl *ctl, const int *cuts, const int *par, int *rep, Csr g, const u64 *ovf,
                          u64 ovf_cap, RowList rl, int *A, int *J1, unsigned *det_ep, unsigned *det_claim,
                          const int *rold, long long budget_v, long long budget_e, int max_levels, int *oc, int *op,
                          cudaStream_t s);
cudaError_t launch_rootcheck(const Dev &d, Ctl *ctl, const int *cuts, const int *rold, const unsigned *rep_ep,
                             cudaStream_t s);
unsigned coop_blocks_detach(int nsm);
cudaError_t launch_jump_async(const Dev &d, const int *A, Ctl *ctl, int *J, int *X, int *Y, cudaStream_t s);
cudaError_t launch_jump(const Dev &d, const int *A, int use_list, long long cnt_static, Ctl *ctl, const int *par,
                        int *J, int *J1, int *rep, RowList rl, int mode, const int *rold, unsigned *w, u64 *heavy,
                        Csr g, int sync_rounds, int *X, int *Y, const int *cuts, cudaStream_t s);
// init: set up the candidates' endpoints first (0: their writer did, HookSlots);
// large: a batch whose candidates stay many past round 0 (smaller blocks)
cudaError_t launch_boruvka(const Dev &d, Ctl *ctl, u64 *ck0, int *ca0, int *cb0, u64 *ck1, int *ca1, int *cb1,
                           HookSlots hs, u64 *er, long long er_cap, int init, bool large, cudaStream_t s);
struct OrientArgs {
    const u64 *er;
    const int *rep;
    int *comp, *minp, *pidx, *plist;
    unsigned *pstamp;
    int *pdeg, *pcur, *poff, *adj, *apos;
    int *val0, *val1, *nx0, *nx1;
    long long *bsum;
    int *chx, *chy;
    unsigned *att_ep, *rep_ep;
    int *att_x, *newrep;
    unsigned char *lf;   // per replacement edge: 0 core, 1 lo-side piece is a leaf, 2 hi-side
    int *cdeg;           // core degree per dense piece
    int *ep, *eid;       // per arc: source piece, its dense id
    int *eroot;          // per edge: hook-forest root of its super-tree
    int *cel;            // core edges (for the one-block path of small cores)
    const int *parent;   // the forest: pulled into L2 for the walks that follow
    long long n;
};
cudaError_t launch_orient(const Dev &d, Ctl *ctl, OrientArgs a, cudaStream_t s);
cudaError_t launch_walk(const Dev &d, Ctl *ctl, const int *chx, const int *chy, const int *rep, int *parent,
                        unsigned *long_ep, cudaStream_t s);
cudaError_t launch_active(const Dev &d, const int *L, int use_list, long long cnt_static, Ctl *ctl, int *rep,
                          const int *parent, const unsigned *sel_ep, const int *att_x, const unsigned *rep_ep,
                          const int *newrep, int *act, int *pold, int *J0, unsigned char *mark, int *aidx,
                          int *aroot, cudaStream_t s);
cudaError_t launch_mark(const Dev &d, Ctl *ctl, const int *act, int *J0, int *J1, unsigned char *mark,
                        const int *parent, cudaStream_t s);
cudaError_t launch_reverse(const Dev &d, Ctl *ctl, const int *act, const int *pold, const unsigned char *mark,
                           const int *chx, const int *chy, int *parent, int walked, cudaStream_t s);
cudaError_t launch_labels(int n, const int *rep, int *tmp, int *out, cudaStream_t s);

unsigned coop_blocks_jump(int nsm);
unsigned grid_vertex_pass(int nsm);
unsigned grid_list_pass(int nsm);
unsigned coop_blocks_hook(int nsm);
unsigned coop_blocks_hook_small(int nsm);
unsigned coop_blocks_orient(int nsm);
unsigned coop_blocks_mark(int nsm);
cudaError_t launch_barrier_selftest(Ctl *ctl, cudaStream_t s);
// static.cu ------------------------------------------------------------
cudaError_t launch_static_forest(const Dev &d, int n, Csr g, const u64 *ovf, Ctl *ctl, int *lab, int *comp,
                                 int *parent, int *f0, int *f1, u64 *levels, cudaStream_t s);
unsigned coop_blocks_bfs(int nsm);
// euler.cu -------------------------------------------------------------
struct EtArgs {
    const int *act, *pold, *aidx, *aroot, *att_x;
    int *ccnt, *ccur, *coff, *kids, *kpos;
    int *val0, *val1, *nx0, *nx1;
    long long *bsum;
    unsigned char *mark;
};
cudaError_t launch_et_marks(const Dev &d, Ctl *ctl, EtArgs a, cudaStream_t s);
unsigned coop_blocks_et(int nsm);
// batched.cu -----------------------------------------------------------
// Persistent per-graph kernels over the disjoint union of many graphs.
#define BCLASSES 4
struct BDesc {               // per call
    const int *batch;        // union batch (ids offset per graph)
    long long len;
    const long long *voff;   // G + 1 vertex offsets
    const long long *boff;   // G + 1 batch offsets
    const int *order;        // graphs in queue order, class by class
    int G;
    int op;
};
struct BState {              // device pointers of one handle (per call)
    Ctl *ctl;
    int *parent, *rep;
    Csr g;
    Index ix;
    u64 *ovf;
    u64 ovf_cap;
    u64 *nkey, *nslot;       // batch-indexed
    // vertex-indexed scratch (graph g uses its own vertex range)
    int *J, *R, *A, *Dv, *roff, *comp, *minp, *pidx, *plist, *pdeg, *poff, *pcur, *newroot, *flist, *chx, *chy;
    int *adj;                // 2 per vertex
    int *tile;               // row of the first entry of each 32-entry tile of a graph's scanned rows
    unsigned *st_aff, *st_cut, *st_piece, *st_vis, *st_rr;   // epoch stamps
    u64 *best, *er;
    // candidate pool, handed out in chunks
    u64 *pk;
    int *pa, *pb;
    u64 pool_cap;
    u64 *pool_ctr;
    u64 *pt_pk, *pt_mk;      // pair table (shared with the grid path; empty between calls)
    u64 pt_mask;
    unsigned *qctr;          // queue counter per class
    int *gcnt, *gcur;        // overflow edges per graph
    long long *govf_start;
    u64 *govf;               // positions in ovf, grouped by graph
    BDesc *desc;
};
cudaError_t launch_bset(BState *dst_state, const BState &st, BDesc *dst_desc, const BDesc &d, cudaStream_t s);
cudaError_t launch_bprologue(const Dev &dv, const BState *S, cudaStream_t s);
unsigned bpersist_grid(int nsm, int threads, int per_sm, int cluster);
cudaError_t launch_bpersist(const BState *S, int cls, int q_lo, int q_hi, int threads, unsigned grid, int cluster,
                            cudaStream_t s);
