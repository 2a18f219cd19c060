/*
 * Seeded synthetic inputs for the dynamic rooted spanning forest batch update.
 *
 * This file generates graphs, initial forests and update batches.  It holds
 * none of the update method's arithmetic: it is shared, as input plumbing, by
 * the serial oracle tests and by the GPU library's tests and benchmark.
 *
 * Random numbers: SplitMix64 (G. L. Steele, D. Lea, C. H. Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014), written from its
 * published definition.  Every decision uses integer arithmetic only, so the
 * output is identical on x86_64 and aarch64.
 *
 * Graph families (stand-ins for the paper's datasets, Table III):
 *   - G(n, m) Erdos-Renyi: m distinct non-loop pairs, uniform.
 *   - R-MAT (Chakrabarti, Zhan, Faloutsos 2004) with the Graph500 initiator
 *     (0.57, 0.19, 0.19, 0.05): edge-factor * 2^scale sampled pairs by
 *     recursive quadrant choice, self-loops dropped, symmetrised,
 *     deduplicated, vertex ids permuted by Fisher-Yates.
 *   - W x H 4-neighbour grid, each edge kept with probability p, plus uniform
 *     long-range shortcuts (road-network stand-in).
 * Initial forest: FIFO BFS from the smallest vertex id of each component,
 * neighbours visited in increasing id, parent = first discoverer,
 * parent[root] = root.
 *
 * Edge keys are uint64 (min(u,v) << 32) | max(u,v).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s; } sm64;

static uint64_t sm64_next(sm64 *g) {
    uint64_t z = (g->s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* One independent stream per (seed, purpose). */
static sm64 sm64_stream(uint64_t seed, uint64_t purpose) {
    sm64 g;
    g.s = seed * 0xD1B54A32D192ED03ull ^ (purpose + 0x632BE59BD9B4E019ull);
    sm64_next(&g);
    sm64_next(&g);
    return g;
}

/* Uniform integer in [0, k) by the multiply-high method (k < 2^63). */
static uint64_t sm64_below(sm64 *g, uint64_t k) {
    return (uint64_t)(((unsigned __int128)sm64_next(g) * k) >> 64);
}

/* Bernoulli(num / 2^32). */
static int sm64_coin32(sm64 *g, uint32_t num) {
    return (uint32_t)(sm64_next(g) >> 32) < num;
}

static inline uint64_t ekey(uint32_t u, uint32_t v) {
    return u < v ? ((uint64_t)u << 32) | v : ((uint64_t)v << 32) | u;
}

/* ---------------------------------------------------------------- sorting */

/* LSD radix sort of uint64 keys, 16-bit digits; skips constant digits. */
static int radix_sort_u64(uint64_t *a, int64_t n) {
    if (n < 2) return 0;
    uint64_t *tmp = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    size_t *cnt = (size_t *)malloc(65536 * sizeof(size_t));
    if (!tmp || !cnt) { free(tmp); free(cnt); return -1; }
    uint64_t *src = a, *dst = tmp;
    for (int pass = 0; pass < 4; ++pass) {
        int sh = 16 * pass;
        memset(cnt, 0, 65536 * sizeof(size_t));
        for (int64_t i = 0; i < n; ++i) cnt[(src[i] >> sh) & 0xFFFF]++;
        int constant = 0;
        for (int d = 0; d < 65536; ++d) if (cnt[d] == (size_t)n) constant = 1;
        if (constant) continue;
        size_t acc = 0;
        for (int d = 0; d < 65536; ++d) { size_t c = cnt[d]; cnt[d] = acc; acc += c; }
        for (int64_t i = 0; i < n; ++i) dst[cnt[(src[i] >> sh) & 0xFFFF]++] = src[i];
        uint64_t *t = src; src = dst; dst = t;
    }
    if (src != a) memcpy(a, src, (size_t)n * sizeof(uint64_t));
    free(tmp);
    free(cnt);
    return 0;
}

static int64_t unique_sorted(uint64_t *a, int64_t n) {
    if (n == 0) return 0;
    int64_t w = 1;
    for (int64_t i = 1; i < n; ++i) if (a[i] != a[w - 1]) a[w++] = a[i];
    return w;
}

static int bsearch_u64(const uint64_t *a, int64_t n, uint64_t k) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (a[mid] < k) lo = mid + 1; else hi = mid;
    }
    return lo < n && a[lo] == k;
}

/* Small open-addressing set of uint64 keys (key 0 never stored: callers add 1). */
typedef struct { uint64_t *t; uint64_t mask; } kset;

static int kset_init(kset *s, int64_t want) {
    uint64_t cap = 16;
    while (cap < (uint64_t)want * 2 + 16) cap <<= 1;
    s->t = (uint64_t *)calloc(cap, sizeof(uint64_t));
    s->mask = cap - 1;
    return s->t ? 0 : -1;
}
static uint64_t kmix(uint64_t k) {
    k ^= k >> 33; k *= 0xff51afd7ed558ccdull; k ^= k >> 33; k *= 0xc4ceb9fe1a85ec53ull; k ^= k >> 33;
    return k;
}
/* returns 1 if inserted, 0 if present */
static int kset_add(kset *s, uint64_t key) {
    uint64_t k1 = key + 1;
    for (uint64_t i = kmix(k1) & s->mask;; i = (i + 1) & s->mask) {
        if (s->t[i] == k1) return 0;
        if (s->t[i] == 0) { s->t[i] = k1; return 1; }
    }
}
static int kset_has(const kset *s, uint64_t key) {
    uint64_t k1 = key + 1;
    for (uint64_t i = kmix(k1) & s->mask;; i = (i + 1) & s->mask) {
        if (s->t[i] == k1) return 1;
        if (s->t[i] == 0) return 0;
    }
}
static void kset_free(kset *s) { free(s->t); s->t = NULL; }

void gen_free(void *p) { free(p); }

/* ------------------------------------------------------------ generators */

/* G(n, m): m distinct non-loop pairs.  Returns sorted keys (malloc'd). */
int64_t gen_er(int32_t n, int64_t m, uint64_t seed, uint64_t **out) {
    *out = NULL;
    if (n < 2) return 0;
    uint64_t maxm = (uint64_t)n * (uint64_t)(n - 1) / 2;
    if ((uint64_t)m > maxm) m = (int64_t)maxm;
    sm64 g = sm64_stream(seed, 1);
    kset s;
    if (kset_init(&s, m)) return -1;
    uint64_t *k = (uint64_t *)malloc((size_t)(m ? m : 1) * sizeof(uint64_t));
    if (!k) { kset_free(&s); return -1; }
    int64_t c = 0;
    while (c < m) {
        uint32_t u = (uint32_t)sm64_below(&g, (uint64_t)n), v = (uint32_t)sm64_below(&g, (uint64_t)n);
        if (u == v) continue;
        uint64_t key = ekey(u, v);
        if (kset_add(&s, key)) k[c++] = key;
    }
    kset_free(&s);
    radix_sort_u64(k, c);
    *out = k;
    return c;
}

/* R-MAT.  Probabilities a, b, c are given as numerators over 2^32.
 * Samples ef * 2^scale pairs over [0, 2^scale), drops self-loops,
 * permutes ids over [0, 2^scale) by Fisher-Yates, keeps pairs with both
 * endpoints < n (n <= 2^scale), symmetrises and deduplicates. */
int64_t gen_rmat(int32_t scale, int32_t n, int64_t ef, uint32_t pa, uint32_t pb, uint32_t pc,
                 uint64_t seed, uint64_t **out) {
    *out = NULL;
    int64_t N = (int64_t)1 << scale;
    if (n <= 0 || n > N) n = (int32_t)N;
    int64_t ms = ef * N;
    uint64_t *k = (uint64_t *)malloc((size_t)(ms ? ms : 1) * sizeof(uint64_t));
    uint32_t *perm = (uint32_t *)malloc((size_t)N * sizeof(uint32_t));
    if (!k || !perm) { free(k); free(perm); return -1; }
    sm64 gp = sm64_stream(seed, 3);
    for (int64_t i = 0; i < N; ++i) perm[i] = (uint32_t)i;
    for (int64_t i = N - 1; i > 0; --i) {
        int64_t j = (int64_t)sm64_below(&gp, (uint64_t)(i + 1));
        uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    sm64 g = sm64_stream(seed, 2);
    uint64_t ta = pa, tb = (uint64_t)pa + pb, tc = (uint64_t)pa + pb + pc;
    int64_t c = 0;
    for (int64_t e = 0; e < ms; ++e) {
        uint32_t u = 0, v = 0;
        for (int l = 0; l < scale; ++l) {
            uint64_t r = sm64_next(&g) >> 32;
            uint32_t bu, bv;
            if (r < ta) { bu = 0; bv = 0; }
            else if (r < tb) { bu = 0; bv = 1; }
            else if (r < tc) { bu = 1; bv = 0; }
            else { bu = 1; bv = 1; }
            u = (u << 1) | bu;
            v = (v << 1) | bv;
        }
        if (u == v) continue;
        uint32_t pu = perm[u], pv = perm[v];
        if ((int64_t)pu >= n || (int64_t)pv >= n) continue;
        k[c++] = ekey(pu, pv);
    }
    free(perm);
    if (radix_sort_u64(k, c)) { free(k); return -1; }
    c = unique_sorted(k, c);
    *out = k;
    return c;
}

/* W x H grid, ids y*W + x; each right / down neighbour edge kept with
 * probability keep/2^32; plus `shortcuts` distinct uniform non-loop pairs
 * that are not grid edges already kept. */
int64_t gen_grid(int32_t W, int32_t H, uint32_t keep, int64_t shortcuts, uint64_t seed, uint64_t **out) {
    *out = NULL;
    int64_t n = (int64_t)W * H;
    int64_t cap = 2 * n + shortcuts + 1;
    uint64_t *k = (uint64_t *)malloc((size_t)cap * sizeof(uint64_t));
    if (!k) return -1;
    sm64 g = sm64_stream(seed, 4);
    int64_t c = 0;
    for (int32_t y = 0; y < H; ++y)
        for (int32_t x = 0; x < W; ++x) {
            uint32_t u = (uint32_t)((int64_t)y * W + x);
            if (x + 1 < W && sm64_coin32(&g, keep)) k[c++] = ekey(u, u + 1);
            if (y + 1 < H && sm64_coin32(&g, keep)) k[c++] = ekey(u, u + (uint32_t)W);
        }
    int64_t cg = c;
    if (radix_sort_u64(k, cg)) { free(k); return -1; }
    sm64 gs = sm64_stream(seed, 5);
    kset s;
    if (kset_init(&s, shortcuts)) { free(k); return -1; }
    int64_t added = 0;
    while (added < shortcuts && n > 1) {
        uint32_t u = (uint32_t)sm64_below(&gs, (uint64_t)n), v = (uint32_t)sm64_below(&gs, (uint64_t)n);
        if (u == v) continue;
        uint64_t key = ekey(u, v);
        if (bsearch_u64(k, cg, key)) continue;
        if (kset_add(&s, key)) { k[c++] = key; added++; }
    }
    kset_free(&s);
    radix_sort_u64(k, c);
    *out = k;
    return c;
}

/* FIFO BFS forest: roots are the smallest id of each component; neighbours
 * visited in increasing id; parent = first discoverer.  keys sorted. */
int gen_bfs_forest(int32_t n, const uint64_t *keys, int64_t m, int32_t *parent) {
    int64_t *off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *adj = (int32_t *)malloc((size_t)(2 * m + 1) * sizeof(int32_t));
    int32_t *q = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
    if (!off || !adj || !q) { free(off); free(adj); free(q); return -1; }
    for (int64_t i = 0; i < m; ++i) {
        off[(keys[i] >> 32) + 1]++;
        off[(keys[i] & 0xFFFFFFFFu) + 1]++;
    }
    for (int32_t v = 0; v < n; ++v) off[v + 1] += off[v];
    int64_t *cur = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    if (!cur) { free(off); free(adj); free(q); return -1; }
    memcpy(cur, off, (size_t)(n + 1) * sizeof(int64_t));
    /* keys sorted by (min, max): filling both sides in key order leaves every
     * adjacency row in increasing neighbour order. */
    for (int64_t i = 0; i < m; ++i) {
        uint32_t u = (uint32_t)(keys[i] >> 32), v = (uint32_t)(keys[i] & 0xFFFFFFFFu);
        adj[cur[u]++] = (int32_t)v;
    }
    for (int64_t i = 0; i < m; ++i) {
        uint32_t u = (uint32_t)(keys[i] >> 32), v = (uint32_t)(keys[i] & 0xFFFFFFFFu);
        adj[cur[v]++] = (int32_t)u;
    }
    /* rows now hold [larger neighbours ascending][smaller neighbours ascending];
     * merge into fully ascending order. */
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * 64);
    int64_t tcap = 64;
    for (int32_t v = 0; v < n; ++v) {
        int64_t a = off[v], b = off[v + 1], len = b - a;
        if (len < 2) continue;
        if (len > tcap) { free(tmp); tcap = len; tmp = (int32_t *)malloc((size_t)tcap * sizeof(int32_t)); }
        int64_t nl = 0;
        for (int64_t i = a; i < b; ++i) if (adj[i] > v) nl++;
        int64_t i = a, j = a + nl, o = 0;
        while (i < a + nl && j < b) tmp[o++] = adj[j] < adj[i] ? adj[j++] : adj[i++];
        while (i < a + nl) tmp[o++] = adj[i++];
        while (j < b) tmp[o++] = adj[j++];
        memcpy(adj + a, tmp, (size_t)len * sizeof(int32_t));
    }
    free(tmp);
    for (int32_t v = 0; v < n; ++v) parent[v] = -1;
    for (int32_t s = 0; s < n; ++s) {
        if (parent[s] != -1) continue;
        parent[s] = s;
        int64_t h = 0, t = 0;
        q[t++] = s;
        while (h < t) {
            int32_t u = q[h++];
            for (int64_t i = off[u]; i < off[u + 1]; ++i) {
                int32_t w = adj[i];
                if (parent[w] == -1) { parent[w] = u; q[t++] = w; }
            }
        }
    }
    free(cur); free(off); free(adj); free(q);
    return 0;
}

/* ----------------------------------------------------------------- batches */

/* b uniform new pairs (u != v, not in the sorted key set, distinct), written
 * as (u, v) in random orientation.  `local` > 0 restricts v to the
 * (2*local+1)^2 window around u on a W-wide grid (H = n / W). */
int gen_insert_batch(int32_t n, const uint64_t *keys, int64_t m, int64_t b, int32_t W, int32_t local,
                     uint64_t seed, int32_t *out) {
    sm64 g = sm64_stream(seed, 6);
    kset s;
    if (kset_init(&s, b)) return -1;
    int64_t c = 0, tries = 0;
    int32_t H = W > 0 ? n / W : 0;
    while (c < b) {
        if (++tries > 1000 * (b + 16)) { kset_free(&s); return -2; }
        uint32_t u = (uint32_t)sm64_below(&g, (uint64_t)n), v;
        if (local > 0) {
            int32_t ux = (int32_t)(u % (uint32_t)W), uy = (int32_t)(u / (uint32_t)W);
            int32_t dx = (int32_t)sm64_below(&g, (uint64_t)(2 * local + 1)) - local;
            int32_t dy = (int32_t)sm64_below(&g, (uint64_t)(2 * local + 1)) - local;
            int32_t vx = ux + dx, vy = uy + dy;
            if (vx < 0 || vx >= W || vy < 0 || vy >= H) continue;
            v = (uint32_t)vy * (uint32_t)W + (uint32_t)vx;
        } else {
            v = (uint32_t)sm64_below(&g, (uint64_t)n);
        }
        if (u == v) continue;
        uint64_t key = ekey(u, v);
        if (bsearch_u64(keys, m, key)) continue;
        if (!kset_add(&s, key)) continue;
        if (sm64_next(&g) & 1) { out[2 * c] = (int32_t)u; out[2 * c + 1] = (int32_t)v; }
        else { out[2 * c] = (int32_t)v; out[2 * c + 1] = (int32_t)u; }
        c++;
    }
    kset_free(&s);
    return 0;
}

/* b distinct existing edges: round(b * tree_num / 1000) uniform tree edges
 * {v, parent[v]} of the given forest, the rest uniform non-tree edges; if one
 * class runs short the other fills in.  Random orientation.  Returns the
 * number written (< b only if the graph has fewer than b edges). */
int64_t gen_delete_batch(int32_t n, const uint64_t *keys, int64_t m, const int32_t *parent, int64_t b,
                         int32_t tree_permille, uint64_t seed, int32_t *out) {
    sm64 g = sm64_stream(seed, 7);
    if (b > m) b = m;
    int64_t nt = 0;
    for (int32_t v = 0; v < n; ++v) if (parent[v] != v) nt++;
    int64_t nn = m - nt;
    int64_t want_t = (b * tree_permille + 500) / 1000;
    if (want_t > nt) want_t = nt;
    int64_t want_n = b - want_t;
    if (want_n > nn) { want_n = nn; want_t = b - want_n; }
    int32_t *tv = (int32_t *)malloc((size_t)(nt ? nt : 1) * sizeof(int32_t));
    if (!tv) return -1;
    int64_t c = 0;
    for (int32_t v = 0; v < n; ++v) if (parent[v] != v) tv[c++] = v;
    /* partial Fisher-Yates over tree children */
    int64_t o = 0;
    for (int64_t i = 0; i < want_t; ++i) {
        int64_t j = i + (int64_t)sm64_below(&g, (uint64_t)(nt - i));
        int32_t t = tv[i]; tv[i] = tv[j]; tv[j] = t;
        int32_t u = tv[i], v = parent[tv[i]];
        if (sm64_next(&g) & 1) { out[2 * o] = u; out[2 * o + 1] = v; }
        else { out[2 * o] = v; out[2 * o + 1] = u; }
        o++;
    }
    free(tv);
    kset s;
    if (kset_init(&s, want_n)) return -1;
    int64_t got = 0;
    while (got < want_n) {
        uint64_t key = keys[sm64_below(&g, (uint64_t)m)];
        uint32_t u = (uint32_t)(key >> 32), v = (uint32_t)(key & 0xFFFFFFFFu);
        if (parent[u] == (int32_t)v || parent[v] == (int32_t)u) continue;
        if (!kset_add(&s, key)) continue;
        if (sm64_next(&g) & 1) { out[2 * o] = (int32_t)u; out[2 * o + 1] = (int32_t)v; }
        else { out[2 * o] = (int32_t)v; out[2 * o + 1] = (int32_t)u; }
        o++;
        got++;
    }
    kset_free(&s);
    /* shuffle so tree and non-tree edges interleave */
    for (int64_t i = o - 1; i > 0; --i) {
        int64_t j = (int64_t)sm64_below(&g, (uint64_t)(i + 1));
        int32_t a0 = out[2 * i], a1 = out[2 * i + 1];
        out[2 * i] = out[2 * j]; out[2 * i + 1] = out[2 * j + 1];
        out[2 * j] = a0; out[2 * j + 1] = a1;
    }
    return o;
}

/* Sorted-key set update: G + B or G - B for a batch already known to be new
 * (insert) or present (delete), duplicates allowed.  Returns the new count;
 * *out is malloc'd. */
int64_t gen_apply_keys(const uint64_t *keys, int64_t m, const int32_t *batch, int64_t b, int32_t op,
                       uint64_t **out) {
    uint64_t *bk = (uint64_t *)malloc((size_t)(b ? b : 1) * sizeof(uint64_t));
    uint64_t *r = (uint64_t *)malloc((size_t)(m + b + 1) * sizeof(uint64_t));
    if (!bk || !r) { free(bk); free(r); return -1; }
    int64_t nb = 0;
    for (int64_t i = 0; i < b; ++i) {
        uint32_t u = (uint32_t)batch[2 * i], v = (uint32_t)batch[2 * i + 1];
        if (u != v) bk[nb++] = ekey(u, v);
    }
    radix_sort_u64(bk, nb);
    nb = unique_sorted(bk, nb);
    int64_t i = 0, j = 0, o = 0;
    if (op == 0) {
        while (i < m || j < nb) {
            if (j >= nb || (i < m && keys[i] < bk[j])) r[o++] = keys[i++];
            else if (i >= m || bk[j] < keys[i]) r[o++] = bk[j++];
            else { r[o++] = keys[i++]; j++; }
        }
    } else {
        while (i < m) {
            while (j < nb && bk[j] < keys[i]) j++;
            if (j < nb && bk[j] == keys[i]) { i++; continue; }
            r[o++] = keys[i++];
        }
    }
    free(bk);
    *out = r;
    return o;
}
