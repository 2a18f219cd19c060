/*
 * drsf.h -- C ABI of the GB300 (sm_103a) dynamic rooted spanning forest
 * library.
 *
 * The library maintains a rooted spanning forest F of an undirected graph G
 * on one GPU under batches of edge insertions or deletions: the Dynamic
 * Rooted Spanning Forest (D-RSF) problem of Sahu, Singh, Nandy and
 * Ramakrishna, "Fully Dynamic Rooted Spanning Tree on GPU" (problem box,
 * Section I).  Input: G, a rooted spanning forest F of G, a batch B and an
 * operation op; output: a rooted spanning forest F' of G' = G + B (insert)
 * or G - B (delete).  The update follows Algorithm 1 (Section II): update
 * the graph, cut deleted tree edges, label every vertex with its tree root
 * by pointer jumping, find replacement edges among the cross edges by
 * hooking and compressing (Section III-B, Algorithm 2), orient them by an
 * Euler tour of the tree-of-trees (Section I preliminaries), then reverse
 * the affected root paths in parallel and attach (Algorithm 1, Section
 * III-C/D).
 *
 * Conventions
 *   - Vertex ids are int32 in [0, n); n <= 2^31 - 1.
 *   - Edges and batches are arrays of int32 pairs (u, v), row-major, i.e.
 *     element 2*i is u_i and 2*i+1 is v_i.  Edges are undirected.
 *   - parent[v] == v marks a root.
 *   - Pointers documented "device" must be CUDA device (or managed) memory
 *     readable by the stream's device; "host" pointers are ordinary or
 *     pinned host memory.
 *   - Every call is ordered on the given stream.  Calls on one handle must
 *     not overlap on different streams.
 *   - The caller owns all buffers it passes in; the library copies what it
 *     needs and never keeps caller pointers.  All library memory comes from
 *     the allocator registered with drsf_set_allocator (default cudaMalloc /
 *     cudaFree).
 *
 * Errors
 *   Every call returns a drsf_status.  drsf_apply checks its arguments on
 *   the host and returns without a host synchronisation; errors detected on
 *   the device (an out-of-range vertex id in a batch, a bounded wait that
 *   timed out) are latched in the handle and reported by the next
 *   drsf_stats / drsf_sync call (drsf_parent and drsf_labels only enqueue
 *   work and report a handle already known to be poisoned).  A batch with
 *   an out-of-range id is not applied at all (DRSF_EINVAL is reported once).
 *   A timeout or internal capacity fault poisons the handle
 *   (DRSF_EPOISONED from then on); destroy it.
 */
#ifndef DRSF_H
#define DRSF_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DRSF_API __attribute__((visibility("default")))
#else
#define DRSF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct drsf_ctx *drsf_handle;
/* A cudaStream_t, passed as an opaque pointer so that this header does not
 * need the CUDA headers.  NULL is the legacy default stream. */
typedef void *drsf_stream;

typedef enum {
    DRSF_OK = 0,
    DRSF_EINVAL = 1,      /* bad argument or out-of-range vertex id */
    DRSF_ENOMEM = 2,      /* allocation failed; the handle is unchanged */
    DRSF_ECUDA = 3,       /* a CUDA runtime call failed */
    DRSF_ENOT_FOREST = 4, /* DRSF_VALIDATE: parent is not a rooted spanning forest of G */
    DRSF_ETIMEOUT = 5,    /* a bounded device-side wait gave up */
    DRSF_EPOISONED = 6    /* an earlier device fault left the handle unusable */
} drsf_status;

typedef enum { DRSF_INSERT = 0, DRSF_DELETE = 1 } drsf_op;

enum {
    /* Minimum-key replacement edges and smallest-root-id super-roots: the
     * result is a function of the inputs alone (bit-identical parent arrays
     * run to run).  In the paper, which cross edge of a super-edge wins is
     * left to races between threads (Section III-A/B).  Here the
     * minimum-key rule is the only mode: it costs one 64-bit atomic minimum
     * per candidate, the same single atomic a first-winner hook would take,
     * so a non-deterministic mode would have nothing to gain and none is
     * built.  The flag is accepted and ignored. */
    DRSF_DETERMINISTIC = 1u,
    /* drsf_create checks on the device that parent is a rooted spanning
     * forest of G and fails with DRSF_ENOT_FOREST otherwise (synchronises). */
    DRSF_VALIDATE = 2u,
    /* Reverse every re-rooted tree's path through the Euler-tour intervals
     * of the re-rooted trees (Algorithm 3).  Default: paths of up to 64
     * edges are reversed by one walking thread each, longer ones through
     * pointer-doubling marks.  Same result. */
    DRSF_EULER_REVERSAL = 4u,
    /* Replacement-edge variant (Section III).  DRSF_REPL_SG, the supergraph
     * variant (Section III-A): the cross edges are reduced to one super-edge
     * per pair of trees (its minimum-key cross edge, through a hash table
     * keyed by the pair of roots), and the hooking then runs on the
     * supergraph.  DRSF_REPL_HS, hooking and shortcutting (Section III-B):
     * the hooking runs on every cross edge.  Neither flag (or both): chosen
     * per batch by comparing the number of key edges |M| with n, as the
     * paper's comparison of the two does (Section V, influencing factors):
     * SG when |M| > n / 16, where |M| is the batch length for an insert and
     * the non-tree edges of G (live edges - n) for a delete.  The result is
     * the same either way (the minimum-key forest does not depend on how
     * parallel super-edges are reduced). */
    DRSF_REPL_SG = 8u,
    DRSF_REPL_HS = 16u
};

/* Per-batch counters of the last applied batch (drsf_stats).  They count
 * the steps of Algorithm 1 (Section II-D) for one batch: the graph update
 * (applied, dropped), the cut of deleted tree edges and the pointer jumping
 * for representatives (tree_cut, affected, jump_rounds, jump_visits), the
 * cross-edge scan and hook-and-compress for replacement edges (Section II-A,
 * III-B: detached, scanned, candidates, hook_rounds, replacement), the
 * Euler-tour orientation (rank_rounds) and the path reversal (Section II-C,
 * III-C/D: active, reversed, mark_rounds). */
typedef struct {
    int64_t batch_len;     /* |B| as passed */
    int64_t self_loops;    /* dropped: u == v */
    int64_t dropped;       /* dropped: duplicate in B, or insert of an existing /
                              delete of an absent edge */
    int64_t applied;       /* edges actually inserted / deleted */
    int64_t tree_cut;      /* deleted edges that were tree edges (delete) */
    int64_t affected;      /* vertices of trees that lost an edge (delete) */
    int64_t detached;      /* rows scanned for cross edges: vertices of cut trees
                              outside the piece left out of the scan, the root
                              piece unless a detached piece has 4096 more
                              vertices, then the heaviest piece (delete) */
    int64_t scanned;       /* adjacency entries scanned for cross edges */
    int64_t candidates;    /* cross edges found */
    int64_t hook_rounds;   /* hook-and-compress rounds */
    int64_t replacement;   /* replacement edges |E_r| */
    int64_t rank_rounds;   /* list-ranking rounds of the Euler tour */
    int64_t active;        /* vertices of the re-rooted trees whose path goes
                              through the marks: trees whose path is longer
                              than 64 edges (all re-rooted trees with
                              DRSF_EULER_REVERSAL) */
    int64_t reversed;      /* vertices whose parent pointer was reversed */
    int64_t mark_rounds;   /* pointer-doubling rounds of the path reversal */
    int64_t jump_rounds;   /* pointer-jumping steps for representatives: the
                              most steps any warp took (asynchronous
                              doubling, the default), or the rounds of the
                              synchronous variant */
    int64_t edges;         /* |E(G')| after the batch */
    int64_t overflow;      /* edges held outside their CSR row (slack exhausted) */
    int64_t rebuilds;      /* CSR / index rebuilds so far */
    int64_t jump_visits;   /* vertex visits summed over the pointer-jumping steps */
    int64_t supergraph;    /* 1: the batch took the supergraph (SG) variant,
                              0: hooking on every cross edge (HS) */
    int64_t detach_levels; /* delete: levels of the top-down search for the
                              detached vertices (0: none, negative: it ran
                              over its budget and pointer jumping took over) */
    int64_t detach_entries;/* delete: adjacency entries that search read */
    int64_t core_arcs;     /* arcs of the super-forest core that the Euler
                              tour ranked (pieces with one replacement edge
                              are oriented without it) */
} drsf_batch_stats;

/* Allocator hooks.  alloc(bytes, stream, ctx) returns device memory or NULL;
 * free(ptr, stream, ctx) releases it.  Pass NULLs to restore cudaMalloc /
 * cudaFree.  Affects handles created afterwards.  Not thread-safe. */
typedef void *(*drsf_alloc_fn)(size_t bytes, drsf_stream stream, void *ctx);
typedef void (*drsf_free_fn)(void *ptr, drsf_stream stream, void *ctx);
DRSF_API drsf_status drsf_set_allocator(drsf_alloc_fn alloc, drsf_free_fn free_fn, void *ctx);

/*
 * drsf_create -- build the device state for the problem's inputs (problem
 * box, Section I): the undirected graph G and its rooted spanning forest F.
 *   n       number of vertices, 1 <= n <= 2^31 - 1
 *   edges   device, int32[2*m], the edge list of G; self-loops and repeated
 *           pairs are dropped; m may be 0 (edges may then be NULL)
 *   parent  device, int32[n], F as parent pointers (parent[r] == r at roots)
 *   flags   DRSF_DETERMINISTIC | DRSF_VALIDATE | DRSF_EULER_REVERSAL |
 *           DRSF_REPL_SG | DRSF_REPL_HS
 *   out     receives the handle (NULL on failure)
 * The graph is stored as a slack CSR (int64 row offsets, int32 columns) with
 * an open-addressing edge index for O(1) deletion.  Synchronises the stream
 * once (to size the CSR).  Without DRSF_VALIDATE, an F that is not a rooted
 * spanning forest of G gives undefined (but memory-safe) results.
 * The environment variable DRSF_JUMP, read here, selects the root search of
 * the handle's delete batches: unset, asynchronous pointer doubling (per-warp
 * slices stepping in place, no grid barrier between steps); "sync",
 * synchronous doubling rounds; "halving", path-halving walks.  All three give
 * the same representatives.  Before it, a delete batch first looks for its
 * detached vertices top-down from the cut vertices over tree children
 * (touching only the detached vertices' rows) and falls back to the root
 * search only when that search exceeds its budget; DRSF_DETACH=0 skips the
 * top-down search, DRSF_DETACH_MAX (default 32768) is the longest delete
 * batch that tries it.  DRSF_GRAPHS=0 launches every batch's kernels directly
 * instead of replaying a captured CUDA graph.
 * Errors: DRSF_EINVAL (n out of range, negative m, NULL pointers, an id out
 * of range), DRSF_ENOMEM, DRSF_ECUDA, DRSF_ENOT_FOREST.
 */
DRSF_API drsf_status drsf_create(int32_t n, const int32_t *edges, int64_t m, const int32_t *parent,
                        uint32_t flags, drsf_stream stream, drsf_handle *out);

/*
 * drsf_apply -- apply one batch (Algorithm 1, Section II-D).
 *   op     DRSF_INSERT (G' = G + B) or DRSF_DELETE (G' = G - B)
 *   batch  device, int32[2*len], the batch B as (u, v) pairs; len may be 0
 * Normalisation: self-loops, pairs repeated within B, insertion of an edge
 * already in G and deletion of an edge not in G are dropped and counted.
 * Asynchronous: returns once the work is enqueued on `stream`; no host
 * synchronisation unless the graph storage must grow (slack or index
 * exhausted), which the host detects from conservative bounds.
 * Errors (immediate): DRSF_EINVAL (bad op, negative len, NULL batch with
 * len > 0), DRSF_ENOMEM, DRSF_ECUDA, DRSF_EPOISONED.  An out-of-range id is
 * reported later as DRSF_EINVAL and the batch is skipped.
 */
DRSF_API drsf_status drsf_apply(drsf_handle h, drsf_op op, const int32_t *batch, int64_t len, drsf_stream stream);

/*
 * drsf_apply_host -- as drsf_apply, with `batch` in host memory (pinned for
 * a truly asynchronous copy).  The library stages it to the device on
 * `stream` before the update.  The host buffer may be reused once this call
 * returns (the library copies through its own pinned staging buffer).
 */
DRSF_API drsf_status drsf_apply_host(drsf_handle h, drsf_op op, const int32_t *batch, int64_t len,
                            drsf_stream stream);

/*
 * drsf_apply_batched -- the batched form: one update of many independent
 * graphs held by one handle as their disjoint union (not in the paper,
 * which updates one graph; each graph's update is Algorithm 1).  Graph g
 * owns vertices [vertex_offsets[g], vertex_offsets[g+1]) and the batch
 * slice [batch_offsets[g], batch_offsets[g+1]); no edge of G may join two
 * graphs, and every edge of a slice must have both ends in its graph's
 * range (else DRSF_EINVAL is latched and the call is skipped, as for an
 * out-of-range id).  Instead of the grid-wide launch sequence, persistent
 * kernels keep one group per graph, a thread-block cluster of
 * cluster_blocks blocks: each group takes the next graph from a
 * device-side queue (largest work first) and runs that graph's whole
 * update with cluster barriers only.  Graphs fall into size classes by
 * vertex count (class c takes graphs with more vertices than class c-1's
 * max_vertices and at most its own; the last class takes the rest); every
 * class has its own queue, block size, cluster size and blocks per SM, and
 * the classes run side by side.  The launch sequence is captured into a
 * CUDA graph on first use of a shape and replayed.  The result is the same
 * forest as drsf_apply with the same batch (minimum-key replacement edges,
 * smallest-root super-roots), and drsf_stats reports the union's counters.
 *   batch           device, int32[2*len] (ids of the union)
 *   vertex_offsets  host, int64[num_graphs + 1], non-decreasing, last <= n
 *   batch_offsets   host, int64[num_graphs + 1], first 0, last len
 *   classes         host, num_classes (1..4) entries, max_vertices increasing;
 *                   block_threads 128, 256, 512 or 1024; blocks_per_sm 0 =
 *                   as many as fit; cluster_blocks 1, 2, 4, 8 or 16
 * Asynchronous like drsf_apply (the host arrays are copied before return).
 * Errors: DRSF_EINVAL (arguments), DRSF_ENOMEM, DRSF_ECUDA, DRSF_EPOISONED.
 */
typedef struct {
    int32_t max_vertices;
    int32_t block_threads;
    int32_t blocks_per_sm;
    int32_t cluster_blocks;
} drsf_batched_class;
DRSF_API drsf_status drsf_apply_batched(drsf_handle h, drsf_op op, const int32_t *batch, int64_t len,
                                        int32_t num_graphs, const int64_t *vertex_offsets,
                                        const int64_t *batch_offsets, const drsf_batched_class *classes,
                                        int32_t num_classes, drsf_stream stream);

/*
 * drsf_reserve -- size the handle's per-batch buffers (device work lists,
 * pair table, the pinned host staging of drsf_apply_host) for batches of up
 * to max_batch edges now, so that later drsf_apply / drsf_apply_host calls
 * of at most that size neither allocate nor synchronise for them (storage
 * growth of the graph itself can still do so).  Not in the paper: for
 * serving loops, where an allocation or a synchronisation inside one
 * tenant's call stalls every other tenant's work.  Synchronises `stream`.
 * Errors: DRSF_EINVAL, DRSF_ENOMEM, DRSF_ECUDA, DRSF_EPOISONED.
 */
DRSF_API drsf_status drsf_reserve(drsf_handle h, int64_t max_batch, drsf_stream stream);

/*
 * drsf_stream_create / drsf_stream_destroy -- a CUDA stream of the caller's
 * own (non-blocking, priority clamped to the device's range; a smaller
 * number is a higher priority).  Not in the paper: a serving loop gives
 * every tenant its own streams, where a framework's stream pool would let
 * two tenants share one and queue behind each other.  The caller destroys
 * what it created.  Errors: DRSF_EINVAL, DRSF_ECUDA.
 */
DRSF_API drsf_status drsf_stream_create(int priority, drsf_stream *out);
DRSF_API drsf_status drsf_stream_destroy(drsf_stream stream);

/* drsf_parent -- the output of the D-RSF problem (problem box, Section I):
 * the rooted spanning forest F' of the updated graph G', as parent
 * pointers.  Copies
 * int32[n] (parent[r] == r at roots) to device buffer `out` on `stream`.
 * Does not synchronise.  Errors: DRSF_EINVAL (NULL handle or out),
 * DRSF_EPOISONED, DRSF_ECUDA. */
DRSF_API drsf_status drsf_parent(drsf_handle h, int32_t *out, drsf_stream stream);

/*
 * drsf_labels -- connected-component labels of G' (connectivity maintenance,
 * Section I contributions): out[v] = smallest vertex id of v's component,
 * written to device buffer int32[n] on `stream`.  Every tree of F' spans one
 * component, so the label is the minimum over v's tree.
 */
DRSF_API drsf_status drsf_labels(drsf_handle h, int32_t *out, drsf_stream stream);

/* drsf_stats -- the counters of the last batch's Algorithm 1 steps (see
 * drsf_batch_stats) into host struct `out`; synchronises `stream`; returns
 * any latched device error (DRSF_EINVAL once for a skipped batch with an
 * out-of-range id, DRSF_ETIMEOUT / DRSF_EPOISONED for a poisoned handle). */
DRSF_API drsf_status drsf_stats(drsf_handle h, drsf_batch_stats *out, drsf_stream stream);

/* drsf_sync -- synchronise `stream` and return any latched device error. */
DRSF_API drsf_status drsf_sync(drsf_handle h, drsf_stream stream);

/* drsf_num_vertices / drsf_num_edges -- sizes (num_edges synchronises). */
DRSF_API int32_t drsf_num_vertices(drsf_handle h);
DRSF_API int64_t drsf_num_edges(drsf_handle h, drsf_stream stream);

/* drsf_export_edges -- write the edge list of G' (int32[2*m], u < v per
 * pair, unspecified order) into device buffer `out` of capacity `cap` pairs;
 * *m_out receives the number of edges.  Synchronises. */
DRSF_API drsf_status drsf_export_edges(drsf_handle h, int32_t *out, int64_t cap, int64_t *m_out, drsf_stream stream);

/*
 * drsf_static_forest -- a rooted spanning forest of the handle's current
 * graph built from scratch, the static alternative the paper compares the
 * dynamic update with (Section V-B: connected components by hooking and
 * shortcutting, the component representatives, then parallel BFS from
 * them).  Components by hook-and-compress over every edge (larger root
 * under smaller, so each root is its component's smallest vertex), then a
 * level-synchronous multi-source BFS from those roots.
 *   parent_out  device int32[n]: a BFS forest (parent[r] == r at the
 *               component minima); which neighbour becomes a vertex's
 *               parent depends on thread timing, the roots do not
 *   labels_out  device int32[n] or NULL: smallest vertex id per component
 *   levels_out  host or NULL: BFS levels (synchronises when given)
 * Does not change the handle's forest.  Enqueued on `stream`.
 */
DRSF_API drsf_status drsf_static_forest(drsf_handle h, int32_t *parent_out, int32_t *labels_out,
                                        int64_t *levels_out, drsf_stream stream);

/*
 * Per-phase timing (instrumentation; not part of the paper).  Between
 * drsf_profile_start and drsf_profile_stop every drsf_apply brackets each
 * phase of the update with CUDA events on its stream; stop synchronises and
 * returns the summed device time and launch count of each phase over the
 * profiled batches.  max_batches bounds the event pool (batches beyond it
 * are not timed).  Phase names come from drsf_phase_name.
 */
#define DRSF_NUM_PHASES 12
typedef struct {
    double ms[2][DRSF_NUM_PHASES];        /* [op][phase] summed device time (ms) */
    int64_t launches[2][DRSF_NUM_PHASES]; /* [op][phase] kernel launches */
    int64_t batches[2];                   /* [op] batches timed */
} drsf_profile_t;
DRSF_API drsf_status drsf_profile_start(drsf_handle h, int64_t max_batches);
DRSF_API drsf_status drsf_profile_stop(drsf_handle h, drsf_profile_t *out, drsf_stream stream);
DRSF_API const char *drsf_phase_name(int phase);

/*
 * drsf_selftest_barrier_timeout -- failure-detection self-test (not part of
 * the paper).  Launches a two-block cooperative kernel in which one block
 * never reaches the grid barrier, so the other block's bounded wait (about
 * two seconds) runs out.  Returns DRSF_ETIMEOUT when the wait gave up and
 * reported it as designed, DRSF_OK if it did not time out, DRSF_ECUDA on a
 * launch failure.  Synchronises `stream`; the CUDA context stays usable.
 */
DRSF_API drsf_status drsf_selftest_barrier_timeout(drsf_stream stream);

/*
 * drsf_forest_labels_noalloc -- the labels of drsf_labels (smallest vertex
 * id of each tree) for a forest the caller passes as a parent array, with no
 * device memory allocated by the call: all scratch lives in one fixed
 * device array compiled into the library.  The paper has no counterpart; it
 * is for callers that cannot allocate when they need the answer (a device
 * memory budget reserved up front, code running inside an allocator or its
 * callbacks, latency-bound loops where cudaMalloc would synchronise).
 *   n       1 <= n <= DRSF_NOALLOC_MAX_N, else DRSF_EINVAL (nothing enqueued)
 *   parent  device, int32[n], parent[r] == r at roots
 *   labels  device, int32[n], output
 * Synchronises `stream` (it reads a status word back), so it cannot be
 * recorded into a CUDA graph; returns DRSF_EINVAL if parent has an id
 * outside [0, n) or a cycle.  Every call on a device shares the scratch
 * array (it keeps the last call's contents; each call re-initialises what
 * it reads, the status word by a memset in stream order): calls that
 * overlap on the GPU race, so order them on one stream.  The first call on
 * a device resolves the array's device address with that device current
 * and keeps it; a cudaDeviceReset while the library is loaded is not
 * supported.  The array (12 MiB) stays allocated on every GPU that loads
 * the library until exit.
 */
#define DRSF_NOALLOC_MAX_N (1 << 20)
DRSF_API drsf_status drsf_forest_labels_noalloc(int32_t n, const int32_t *parent, int32_t *labels,
                                               drsf_stream stream);

/* drsf_destroy -- release all device memory (synchronises the handle's last
 * stream).  NULL is a no-op. */
DRSF_API void drsf_destroy(drsf_handle h);

/* drsf_error_string -- static description of a status. */
DRSF_API const char *drsf_error_string(drsf_status s);

#ifdef __cplusplus
}
#endif
#endif /* DRSF_H */
