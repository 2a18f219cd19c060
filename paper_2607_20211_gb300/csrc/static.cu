// Static rooted spanning forest of the handle's current graph, from scratch
// (the plain alternative to the dynamic update that the paper compares
// against, Section V-B): connected components by hooking and compressing
// over every edge, then a multi-source BFS from each component's smallest
// vertex, parent = the vertex that first discovers a vertex.  The BFS parent
// of a vertex is whichever frontier vertex wins the claim, so the forest is
// a valid rooted spanning forest but not a fixed one; its roots and labels
// are fixed (the component minima).
#include <climits>

#include "kernels.h"

#define GS_LOOP(i, n) \
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)(n); \
         i += (long long)gridDim.x * blockDim.x)

__device__ __forceinline__ int cc_find(int *lab, int x) {
    for (int it = 0; it < (1 << 22); ++it) {
        int p = __ldcg(&lab[x]);
        if (p == x) return x;
        int gp = __ldcg(&lab[p]);
        if (gp != p) lab[x] = gp;   // halving: gp is still an ancestor
        x = gp;
    }
    return x;
}

__global__ void k_cc_init(int n, int *lab) {
    GS_LOOP(v, n) lab[v] = (int)v;
}

// Hook: for each edge, link the larger root under the smaller one
// (atomicCAS on the larger root, retried on contention).  Roots only ever
// point to smaller ids, so the forest stays acyclic and each component's
// final root is its smallest vertex.  A warp per CSR row (each edge taken
// from its smaller endpoint's row), then the overflow edges.
__device__ __forceinline__ void cc_union(int *lab, int a, int b) {
    for (int it = 0; it < (1 << 20); ++it) {
        int ra = cc_find(lab, a), rb = cc_find(lab, b);
        if (ra == rb) return;
        int hi = ra > rb ? ra : rb, lo = ra > rb ? rb : ra;
        if (atomicCAS(&lab[hi], hi, lo) == hi) return;
    }
}

__global__ void k_cc_hook(int n, Csr g, const u64 *ovf, const Ctl *ctl, int *lab) {
    int lane = threadIdx.x & 31;
    long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long u = warp; u < n; u += nw) {
        long long o = g.off[u];
        long long cap = g.off[u + 1] - o;
        long long used = g.used[u];
        if (used > cap) used = cap;
        for (long long j = lane; j < used; j += 32) {
            int x = g.col[o + j];
            if (x > (int)u) cc_union(lab, (int)u, x);
        }
    }
    const long long no = (long long)ctl->ovf_count;
    GS_LOOP(i, no) {
        u64 k = ovf[i];
        if (k != TOMB_KEY) cc_union(lab, (int)klo(k), (int)khi(k));
    }
}

// Component of every vertex by a read-only walk to its root, written to a
// separate array (a walk that rewrote the pointers it reads could race with
// another walk and leave a non-root behind); roots start the BFS
// (parent[r] = r), other vertices are unclaimed (-1).
__global__ void k_cc_roots(int n, const int *lab, int *comp, int *parent, int *frontier, u64 *fcount) {
    for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += (long long)gridDim.x * blockDim.x) {
        long long v = base + threadIdx.x;
        bool root = false;
        if (v < n) {
            int r = (int)v;
            for (int it = 0; it < (1 << 22); ++it) {
                int p = __ldcg(&lab[r]);
                if (p == r) break;
                r = p;
            }
            comp[v] = r;
            root = r == (int)v;
            parent[v] = root ? (int)v : -1;
        }
        long long p = block_append(fcount, root);
        if (root) frontier[p] = (int)v;
    }
}

// Level-synchronous multi-source BFS in one cooperative launch: a warp per
// frontier vertex streams its row; a neighbour claimed by atomicCAS on its
// parent joins the next frontier.  Frontiers alternate between two lists;
// counts live in ctl->cnt (3 slots, as in the other round loops).
__global__ void k_bfs(Ctl *ctl, Csr g, const u64 *ovf, int *parent, int *f0, int *f1, u64 *levels) {
    int lane = threadIdx.x & 31;
    long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    int r = 0;
    for (;; ++r) {
        const long long c = (long long)*(volatile u64 *)&ctl->cnt[r % 3];
        if (c == 0) break;
        if (r > (1 << 24)) {
            if (warp == 0 && lane == 0) atomicOr(&ctl->err, ERR_ROUNDS);
            return;
        }
        if (warp == 0 && lane == 0) ctl->cnt[(r + 2) % 3] = 0;
        const int *in = (r & 1) ? f1 : f0;
        int *out = (r & 1) ? f0 : f1;
        for (long long w = warp; w < c; w += nw) {
            int u = in[w];
            long long o = g.off[u];
            long long cap = g.off[u + 1] - o;
            long long used = g.used[u];
            if (used > cap) used = cap;
            for (long long j0 = 0; j0 < used; j0 += 32) {
                long long j = j0 + lane;
                int x = j < used ? g.col[o + j] : -1;
                bool claim = x >= 0 && __ldcg(&parent[x]) == -1 && atomicCAS(&parent[x], -1, u) == -1;
                long long p = agg_append(&ctl->cnt[(r + 1) % 3], claim);
                if (claim) out[p] = x;
            }
        }
        // overflow edges (outside their rows), both directions
        const long long no = (long long)ctl->ovf_count;
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < no;
             i += (long long)gridDim.x * blockDim.x) {
            u64 k = ovf[i];
            if (k == TOMB_KEY) continue;
            int a = (int)klo(k), b = (int)khi(k);
            int pa = __ldcg(&parent[a]), pb = __ldcg(&parent[b]);
            // an endpoint claimed in an earlier level discovers the other one
            if (pa != -1 && pb == -1 && atomicCAS(&parent[b], -1, a) == -1)
                out[atomicAdd(&ctl->cnt[(r + 1) % 3], 1ull)] = b;
            else if (pb != -1 && pa == -1 && atomicCAS(&parent[a], -1, b) == -1)
                out[atomicAdd(&ctl->cnt[(r + 1) % 3], 1ull)] = a;
        }
        if (!grid_barrier(ctl, &ctl->bar[4])) return;
    }
    if (warp == 0 && lane == 0) *levels = (u64)r;
}

unsigned coop_blocks_bfs(int nsm) {
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void *)k_bfs, BLK, 0) != cudaSuccess || per < 1)
        per = 1;
    if (per > 8) per = 8;
    return (unsigned)(per * nsm);
}

cudaError_t launch_static_forest(const Dev &d, int n, Csr g, const u64 *ovf, Ctl *ctl, int *lab, int *comp,
                                 int *parent, int *f0, int *f1, u64 *levels, cudaStream_t s) {
    unsigned gn = grid_for(n, BLK, 152u * 16u);
    cudaError_t e = cudaMemsetAsync(ctl->cnt, 0, sizeof(ctl->cnt), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(&ctl->bar[4], 0, sizeof(u64), s);   // BFS barrier counter
    if (e != cudaSuccess) return e;
    k_cc_init<<<gn, BLK, 0, s>>>(n, lab);
    k_cc_hook<<<d.grid, BLK, 0, s>>>(n, g, ovf, ctl, lab);
    k_cc_roots<<<gn, BLK, 0, s>>>(n, lab, comp, parent, f0, &ctl->cnt[0]);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&ctl, (void *)&g, (void *)&ovf, (void *)&parent, (void *)&f0, (void *)&f1,
                    (void *)&levels};
    return cudaLaunchCooperativeKernel((const void *)k_bfs, d.coop_bfs, BLK, args, 0, s);
}
