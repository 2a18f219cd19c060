// Path marking by the Euler tour (Algorithm 3, ReversePathsEulerTour), the
// alternative to pointer-doubling marks (selected with DRSF_EULER_REVERSAL).
//
// The re-rooted pieces (active vertices, listed densely by k_active) are
// toured: children lists from the old parent pointers, one down arc
// (parent -> v) and one up arc (v -> parent) per non-root vertex, successor
// of down(v) = down(first child of v) or up(v) for a leaf, successor of
// up(v) = down(next sibling of v) or up(parent of v), ending at the piece
// root.  Wyllie list ranking gives every arc its distance to the end of its
// piece's tour.  A vertex u is an ancestor-or-self of its piece's attach
// point x exactly when down(u) comes no later than down(x) and up(u) no
// earlier than up(x) (nested start/finish intervals); those vertices are
// marked, and k_reverse reverses their parent pointers as for the doubling
// marks.  The result is the same parent array.
#include <climits>

#include "kernels.h"

__device__ __forceinline__ long long etid() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long etstride() { return (long long)gridDim.x * blockDim.x; }

__global__ void k_et_marks(Ctl *ctl, EtArgs a) {
    if (*(volatile int *)&ctl->skip) return;
    u64 *bar = &ctl->bar[5];
    const long long na = (long long)ctl->nact;
    // phase 0: clear child counters
    for (long long q = etid(); q < na; q += etstride()) {
        a.ccnt[q] = 0;
        a.ccur[q] = 0;
    }
    if (!grid_barrier(ctl, bar)) return;
    // phase 1: children per active vertex (dense index of the old parent)
    for (long long q = etid(); q < na; q += etstride()) {
        int v = a.act[q], pv = a.pold[q];
        if (pv != v) atomicAdd(&a.ccnt[LD(a.aidx[pv])], 1);
    }
    if (!grid_barrier(ctl, bar)) return;
    // phase 2: exclusive scan of child counts (chunk sums, scan, rescans)
    const long long chunk = (na + gridDim.x - 1) / gridDim.x;
    const long long lo = (long long)blockIdx.x * chunk, hi = lo + chunk < na ? lo + chunk : na;
    {
        long long sacc = 0;
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) sacc += LD(a.ccnt[i]);
        long long tot;
        block_excl_scan_ll(sacc, &tot);
        if (threadIdx.x == 0) a.bsum[blockIdx.x] = tot;
    }
    if (!grid_barrier(ctl, bar)) return;
    if (blockIdx.x == 0) {
        long long nbk = gridDim.x;
        long long per = (nbk + blockDim.x - 1) / blockDim.x;
        long long l0 = threadIdx.x * per, l1 = l0 + per < nbk ? l0 + per : nbk;
        long long sacc = 0;
        for (long long i = l0; i < l1; ++i) sacc += LD(a.bsum[i]);
        long long tot;
        long long pre = block_excl_scan_ll(sacc, &tot);
        for (long long i = l0; i < l1; ++i) {
            long long t = LD(a.bsum[i]);
            a.bsum[i] = pre;
            pre += t;
        }
    }
    if (!grid_barrier(ctl, bar)) return;
    {
        long long carry = LD(a.bsum[blockIdx.x]);
        for (long long t0 = lo; t0 < hi; t0 += blockDim.x) {
            long long i = t0 + threadIdx.x;
            long long d = i < hi ? LD(a.ccnt[i]) : 0;
            long long tot;
            long long pre = block_excl_scan_ll(d, &tot);
            if (i < hi) a.coff[i] = (int)(carry + pre);
            carry += tot;
        }
    }
    if (!grid_barrier(ctl, bar)) return;
    // phase 3: children lists; kpos = slot of a vertex in its parent's list
    for (long long q = etid(); q < na; q += etstride()) {
        int v = a.act[q], pv = a.pold[q];
        if (pv == v) continue;
        int pq = LD(a.aidx[pv]);
        int slot = LD(a.coff[pq]) + atomicAdd(&a.ccur[pq], 1);
        a.kids[slot] = (int)q;
        a.kpos[q] = slot;
    }
    if (!grid_barrier(ctl, bar)) return;
    // phase 4: arc successors (down(q) = 2q, up(q) = 2q + 1)
    for (long long q = etid(); q < na; q += etstride()) {
        int v = a.act[q], pv = a.pold[q];
        if (pv == v) continue;   // the piece root has no arcs
        int c0 = LD(a.coff[q]), cn = LD(a.ccnt[q]);
        a.nx0[2 * q] = cn > 0 ? 2 * LD(a.kids[c0]) : (int)(2 * q + 1);
        int pq = LD(a.aidx[pv]);
        int nxt = LD(a.kpos[q]) + 1;
        int up;
        if (nxt < LD(a.coff[pq]) + LD(a.ccnt[pq])) up = 2 * LD(a.kids[nxt]);
        else up = a.pold[pq] == pv ? NIL : 2 * pq + 1;   // after the root's last child: end
        a.nx0[2 * q + 1] = up;
        a.val0[2 * q] = 1;
        a.val0[2 * q + 1] = 1;
    }
    if (!grid_barrier(ctl, bar)) return;
    // phase 5: Wyllie ranking: distance to the end of the piece's tour
    int *vc = a.val0, *vn = a.val1, *nc = a.nx0, *nn = a.nx1;
    int r = 0;
    for (;; ++r) {
        if (r >= MAX_ROUNDS) {
            if (etid() == 0) atomicOr(&ctl->err, ERR_ROUNDS);
            return;
        }
        if (etid() == 0) ctl->flag[(r + 1) % 3] = 0;
        bool ch = false;
        for (long long i = etid(); i < 2 * na; i += etstride()) {
            if (a.pold[i >> 1] == a.act[i >> 1]) continue;
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
    // phase 6: interval test against the piece's attach point
    for (long long q = etid(); q < na; q += etstride()) {
        int u = a.act[q];
        if (a.pold[q] == u) continue;   // the root needs no mark
        int x = a.att_x[a.aroot[q]];
        int qx = LD(a.aidx[x]);
        bool anc = qx == (int)q ||
                   (LD(vc[2 * q]) >= LD(vc[2 * qx]) && LD(vc[2 * qx + 1]) >= LD(vc[2 * q + 1]));
        a.mark[u] = anc ? 1 : 0;
    }
    if (etid() == 0) ctl->mark_rounds = r + 1;
}

cudaError_t launch_et_marks(const Dev &d, Ctl *ctl, EtArgs a, cudaStream_t s) {
    void *args[] = {(void *)&ctl, (void *)&a};
    return cudaLaunchCooperativeKernel((const void *)k_et_marks, d.coop_et, BLK, args, 0, s);
}

unsigned coop_blocks_et(int nsm) {
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void *)k_et_marks, BLK, 0) != cudaSuccess ||
        per < 1)
        per = 1;
    if (per > 4) per = 4;
    return (unsigned)(per * nsm);
}
