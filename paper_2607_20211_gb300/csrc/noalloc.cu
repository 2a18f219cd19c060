// Allocation-free forest labelling: drsf_forest_labels_noalloc.
//
// The same labels as drsf_labels (smallest vertex id of each tree), computed
// from a parent array the caller passes in, with all scratch memory in one
// fixed file-scope device array instead of memory obtained at run time.  It
// exists for callers that cannot allocate device memory when they need the
// answer: code that runs under a fixed device-memory budget reserved up
// front, code called from inside a device-memory allocator or its callbacks
// (where allocating again would re-enter the allocator), and latency-bound
// loops where cudaMalloc / cudaFree would synchronise the device.
//
// Limits and sharing:
//   - n <= DRSF_NOALLOC_MAX_N (2^20 vertices); larger n is rejected with
//     DRSF_EINVAL before any work is enqueued.
//   - The scratch array lives on every GPU that loads the library until the
//     process exits (12 MiB + a few bytes).  Every call on a device shares it
//     and it keeps the last call's contents; each call clears what must
//     start from a known value.  Calls that overlap on the GPU (different
//     streams, or threads) race on the array and give wrong results: order
//     them on one stream.
//   - The first call on a device looks up the device address of the array
//     (cudaGetSymbolAddress) with that device current and keeps it for the
//     life of the process; a cudaDeviceReset while the library is loaded is
//     not supported (the kept address would belong to the old context).
//   - Every call synchronises its stream and reads a status word back to
//     the host, so the call cannot be recorded into a CUDA graph.
#include <climits>
#include <mutex>

#include "kernels.h"

#define NOALLOC_MAX_N (1 << 20)

// [0, MAX): jump pointers J; [MAX, 2 MAX): root of each vertex R (written
// only by that vertex's thread); [2 MAX, 3 MAX): per-tree minimum; then a
// status word (bit 1: bad parent id, bit 2: walk bound exceeded, bit 4: a
// walk ended on a vertex that is not a root of the input, i.e. a cycle).
// The status word is cleared by a memset in stream order before the first
// kernel, never inside a multi-block launch that may also set it.
static __device__ __align__(256) int g_noalloc_scratch[3 * NOALLOC_MAX_N + 64];

namespace {
std::mutex g_na_mu;
int *g_na_ptr[256];   // device address of g_noalloc_scratch per device id
}

__global__ void k_na_init(const int *parent, int n, int *J, int *mn, int *status) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        int p = parent[v];
        if (p < 0 || p >= n) {
            atomicOr(status, 1);
            p = (int)v;
        }
        J[v] = p;
        mn[v] = INT_MAX;
    }
}

// Root of every vertex by in-place pointer jumping with path halving (every
// J[x] only moves to an ancestor of x, so concurrent walks stay correct).
// J[x] itself may be left pointing at a non-root ancestor by a late halving
// write of another walk, so the root goes to R[v], which only this thread
// writes.  On a cycle a halving step can make a cycle vertex point at
// itself (J[x] = x), which ends walks at a vertex whose input parent is not
// itself: that is checked against the input and reported as bit 4.
__global__ void k_na_roots(int n, const int *parent, int *J, int *R, int *status) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        int x = (int)v;
        int root = -1;
        // On a forest every step moves x at least two levels up (p is a
        // proper ancestor of x and gp one of p, whatever other walks wrote),
        // so a walk ends within depth / 2 + 1 <= n / 2 + 1 steps; a walk
        // that does not is on a cycle.
        const int bound = (n >> 1) + 2;
        for (int it = 0; it < bound; ++it) {
            int p = __ldcg(&J[x]);
            int gp = __ldcg(&J[p]);
            if (p == gp) {
                root = p;
                break;
            }
            J[x] = gp;
            x = gp;
        }
        if (root < 0) {
            atomicOr(status, 2);
            root = (int)v;
        } else {
            int pr = parent[root];   // a true root of the input points at itself
            if (pr != root && pr >= 0 && pr < n) atomicOr(status, 4);
        }
        R[v] = root;
    }
}

__global__ void k_na_min(int n, const int *R, int *mn) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        int r = __ldcg(&R[v]);
        unsigned same = __match_any_sync(__activemask(), r);
        if ((threadIdx.x & 31) == __ffs(same) - 1) atomicMin(&mn[r], (int)v);
    }
}

__global__ void k_na_out(int n, const int *R, const int *mn, int *out) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
        out[v] = __ldcg(&mn[__ldcg(&R[v])]);
}

extern "C" drsf_status drsf_forest_labels_noalloc(int32_t n, const int32_t *parent, int32_t *labels,
                                                  drsf_stream stream) {
    if (n < 1 || !parent || !labels) return DRSF_EINVAL;
    if (n > NOALLOC_MAX_N) return DRSF_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        cudaGetLastError();
        return DRSF_ECUDA;
    }
    int *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return DRSF_ECUDA;
            }
            g_na_ptr[dev] = (int *)p;
        }
        base = g_na_ptr[dev];
    }
    int *J = base, *R = base + NOALLOC_MAX_N, *mn = base + 2 * NOALLOC_MAX_N, *status = base + 3 * NOALLOC_MAX_N;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned g = grid_for(n, BLK, 152u * 16u);
    if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) {
        cudaGetLastError();
        return DRSF_ECUDA;
    }
    k_na_init<<<g, BLK, 0, s>>>(parent, n, J, mn, status);
    k_na_roots<<<g, BLK, 0, s>>>(n, parent, J, R, status);
    k_na_min<<<g, BLK, 0, s>>>(n, R, mn);
    k_na_out<<<g, BLK, 0, s>>>(n, R, mn, labels);
    int st = 0;
    if (cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return DRSF_ECUDA;
    }
    return st ? DRSF_EINVAL : DRSF_OK;
}
