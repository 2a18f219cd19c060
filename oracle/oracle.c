/*
 * Serial CPU oracle for the Dynamic Rooted Spanning Forest (D-RSF) batch
 * update of Sahu, Singh, Nandy, Ramakrishna, "Fully Dynamic Rooted Spanning
 * Tree on GPU" (arXiv 2607.20211).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the GPU library is checked against.  Only the tests, the
 * smoke entry point and the benchmark's CPU-baseline leg may load it.  It
 * shares no code with the GPU path.
 *
 * Every step is serial and follows the paper's definitions:
 *   - problem statement (D-RSF box, Section I): G' = G + B or G - B, output a
 *     rooted spanning forest F' of G';
 *   - notation (Section II-A): F^ = F - B for delete, F^ = F for insert;
 *     rep[v] = root of v's tree in F^; cross edge: rep[u] != rep[v];
 *     replacement edges E_r: k - l cross edges, forming a spanning forest of
 *     the trees of F^ (k trees of F^, l components of G');
 *   - Algorithm 1: cut deleted tree edges (parent[u] <- u), representatives,
 *     oriented replacement edges, path reversal of (x, rep[x]) paths, then
 *     parent[x] <- y for each oriented replacement edge (x -> y);
 *   - Theorem 1 (Section II-D): each replacement edge removes one root.
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   - batch normalisation: self-loops dropped, duplicates within the batch
 *     dropped, inserting an existing edge or deleting an absent edge is a
 *     no-op (the paper's graphs are simple and undirected, Section V-A);
 *   - a deleted edge {a, b} is a tree edge iff parent[a] == b or
 *     parent[b] == a (Algorithm 1 comments assume the child is listed first);
 *   - E_r is the unique minimum spanning forest of the piece multigraph
 *     under edge key (min(u,v) << 32 | max(u,v)), taken by Kruskal; any
 *     forest meeting the Section II-A definition is valid, this one is the
 *     deterministic choice;
 *   - the root of each merged tree is the root of its piece with the
 *     smallest root id; the replacement edges are oriented away from it;
 *   - the "k - l" count and the root count are as in Theorem 1.
 *
 * Return codes: 0 ok, -1 invalid input (vertex id out of range),
 * -2 allocation failure.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- helpers */

static inline uint64_t okey(uint32_t u, uint32_t v) {
    return u < v ? ((uint64_t)u << 32) | v : ((uint64_t)v << 32) | u;
}
static inline uint32_t key_lo(uint64_t k) { return (uint32_t)(k >> 32); }
static inline uint32_t key_hi(uint64_t k) { return (uint32_t)(k & 0xFFFFFFFFu); }

/* Edge set: open addressing, linear probing, key+1 stored (0 = empty),
 * deleted entries marked with DEAD. */
#define DEAD 0xFFFFFFFFFFFFFFFFull
typedef struct { uint64_t *t; uint64_t mask; } eset;

static uint64_t ehash(uint64_t k) {
    k ^= k >> 31; k *= 0x7fb5d329728ea185ull; k ^= k >> 27; k *= 0x81dadef4bc2dd44dull; k ^= k >> 33;
    return k;
}
static int eset_init(eset *s, int64_t want) {
    uint64_t cap = 64;
    while (cap < (uint64_t)want * 2 + 64) cap <<= 1;
    s->t = (uint64_t *)calloc(cap, sizeof(uint64_t));
    s->mask = cap - 1;
    return s->t ? 0 : -2;
}
static int eset_has(const eset *s, uint64_t key) {
    uint64_t k1 = key + 1;
    for (uint64_t i = ehash(k1) & s->mask;; i = (i + 1) & s->mask) {
        if (s->t[i] == k1) return 1;
        if (s->t[i] == 0) return 0;
    }
}
static void eset_add(eset *s, uint64_t key) {
    uint64_t k1 = key + 1;
    for (uint64_t i = ehash(k1) & s->mask;; i = (i + 1) & s->mask) {
        if (s->t[i] == k1) return;
        if (s->t[i] == 0 || s->t[i] == DEAD) { s->t[i] = k1; return; }
    }
}
static void eset_del(eset *s, uint64_t key) {
    uint64_t k1 = key + 1;
    for (uint64_t i = ehash(k1) & s->mask;; i = (i + 1) & s->mask) {
        if (s->t[i] == k1) { s->t[i] = DEAD; return; }
        if (s->t[i] == 0) return;
    }
}

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : x > y;
}

/* Union-find over vertex ids: find with path halving, union links the
 * larger representative under the smaller one. */
static int32_t uf_find(int32_t *uf, int32_t x) {
    while (uf[x] != x) { uf[x] = uf[uf[x]]; x = uf[x]; }
    return x;
}
static int uf_union(int32_t *uf, int32_t a, int32_t b) {
    a = uf_find(uf, a); b = uf_find(uf, b);
    if (a == b) return 0;
    if (a < b) uf[b] = a; else uf[a] = b;
    return 1;
}

/* CSR adjacency of an edge-key list (used by BFS labelling). */
static int build_adj(int32_t n, const uint64_t *keys, int64_t m, int64_t **off_out, int32_t **adj_out) {
    int64_t *off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *adj = (int32_t *)malloc((size_t)(2 * m + 1) * sizeof(int32_t));
    int64_t *cur = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!off || !adj || !cur) { free(off); free(adj); free(cur); return -2; }
    for (int64_t i = 0; i < m; ++i) { off[key_lo(keys[i]) + 1]++; off[key_hi(keys[i]) + 1]++; }
    for (int32_t v = 0; v < n; ++v) off[v + 1] += off[v];
    memcpy(cur, off, ((size_t)n + 1) * sizeof(int64_t));
    for (int64_t i = 0; i < m; ++i) {
        uint32_t u = key_lo(keys[i]), v = key_hi(keys[i]);
        adj[cur[u]++] = (int32_t)v;
        adj[cur[v]++] = (int32_t)u;
    }
    free(cur);
    *off_out = off;
    *adj_out = adj;
    return 0;
}

/* ------------------------------------------------------------ labels (CC) */

/* Connected-component labels by BFS: label[v] = smallest vertex id of v's
 * component (connectivity maintenance, Section I contributions). */
int oracle_labels(int32_t n, const uint64_t *keys, int64_t m, int32_t *label) {
    for (int64_t i = 0; i < m; ++i)
        if (key_lo(keys[i]) >= (uint32_t)n || key_hi(keys[i]) >= (uint32_t)n) return -1;
    int64_t *off; int32_t *adj;
    if (build_adj(n, keys, m, &off, &adj)) return -2;
    int32_t *q = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    if (!q) { free(off); free(adj); return -2; }
    for (int32_t v = 0; v < n; ++v) label[v] = -1;
    for (int32_t s = 0; s < n; ++s) {       /* ascending: s is its component's minimum */
        if (label[s] != -1) continue;
        int64_t h = 0, t = 0;
        label[s] = s;
        q[t++] = s;
        while (h < t) {
            int32_t u = q[h++];
            for (int64_t i = off[u]; i < off[u + 1]; ++i)
                if (label[adj[i]] == -1) { label[adj[i]] = s; q[t++] = adj[i]; }
        }
    }
    free(q); free(off); free(adj);
    return 0;
}

/* ---------------------------------------------------------- exact checker */

/* Exact checker for "F is a rooted spanning forest of G" (D-RSF box,
 * Section I; rooted spanning forest definition, Section II-A):
 *   1  some parent[v] outside [0, n)
 *   2  some parent[v] != v with {v, parent[v]} not an edge of G
 *   3  the parent pointers contain a cycle
 *   4  some connected component of G has zero or several roots
 *   5  some vertex does not reach the root of its component
 * Returns 0 when all hold. */
int oracle_check_forest(int32_t n, const uint64_t *keys, int64_t m, const int32_t *parent) {
    int rc = 0;
    for (int32_t v = 0; v < n; ++v)
        if (parent[v] < 0 || parent[v] >= n) return 1;
    eset s;
    if (eset_init(&s, m)) return -2;
    for (int64_t i = 0; i < m; ++i) eset_add(&s, keys[i]);
    for (int32_t v = 0; v < n; ++v)
        if (parent[v] != v && !eset_has(&s, okey((uint32_t)v, (uint32_t)parent[v]))) { rc = 2; break; }
    free(s.t);
    if (rc) return rc;

    /* acyclicity: iterative three-colour walk (0 unseen, 1 on the current
     * walk, 2 known to end at a root) */
    uint8_t *col = (uint8_t *)calloc((size_t)n + 1, 1);
    int32_t *uf = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int32_t *root = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int32_t *cnt = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    if (!col || !uf || !root || !cnt) { free(col); free(uf); free(root); free(cnt); return -2; }
    for (int32_t v = 0; v < n && !rc; ++v) {
        int32_t x = v;
        while (col[x] == 0 && parent[x] != x) { col[x] = 1; x = parent[x]; }
        if (col[x] == 1) { rc = 3; break; }
        int32_t r = col[x] == 2 ? root[x] : x;   /* x is a root or already resolved */
        col[x] = 2; root[x] = r;
        for (int32_t y = v; col[y] == 1; y = parent[y]) { col[y] = 2; root[y] = r; }
    }
    if (!rc) {
        /* one root per connected component of G */
        for (int32_t v = 0; v < n; ++v) uf[v] = v;
        for (int64_t i = 0; i < m; ++i) uf_union(uf, (int32_t)key_lo(keys[i]), (int32_t)key_hi(keys[i]));
        for (int32_t v = 0; v < n; ++v) if (parent[v] == v) cnt[uf_find(uf, v)]++;
        for (int32_t v = 0; v < n && !rc; ++v) if (uf_find(uf, v) == v && cnt[v] != 1) rc = 4;
        /* every vertex reaches the root of its own component */
        for (int32_t v = 0; v < n && !rc; ++v)
            if (uf_find(uf, root[v]) != uf_find(uf, v) || parent[root[v]] != root[v]) rc = 5;
    }
    free(col); free(uf); free(root); free(cnt);
    return rc;
}

/* ------------------------------------------------------- the batch update */

typedef struct {
    int64_t batch_len;      /* |B| as given */
    int64_t self_loops;     /* dropped: u == v */
    int64_t duplicates;     /* dropped: repeated within the batch */
    int64_t ignored;        /* dropped: insert of an existing / delete of an absent edge */
    int64_t applied;        /* |B| after normalisation */
    int64_t tree_cut;       /* deleted edges that were tree edges of F */
    int64_t pieces;         /* k: trees of F^ */
    int64_t components;     /* l: components of G' */
    int64_t cross;          /* cross edges of G' w.r.t. F^ */
    int64_t replacement;    /* |E_r| */
    int64_t reversed;       /* vertices whose parent was reversed */
    int64_t m_out;          /* |E(G')| */
} oracle_stats;

/* 1 if the parent pointers are acyclic (every walk ends at a root). */
static int acyclic(int32_t n, const int32_t *par) {
    uint8_t *col = (uint8_t *)calloc((size_t)n + 1, 1);
    if (!col) return 0;
    int ok = 1;
    for (int32_t v = 0; v < n && ok; ++v) {
        int32_t x = v;
        while (col[x] == 0 && par[x] != x) { col[x] = 1; x = par[x]; }
        if (col[x] == 1) { ok = 0; break; }
        col[x] = 2;
        for (int32_t y = v; col[y] == 1; y = par[y]) col[y] = 2;
    }
    free(col);
    return ok;
}

/* rep[v]: root of v's tree in the forest par (serial walk, memoised). */
static void oracle_rep(int32_t n, const int32_t *par, int32_t *rep) {
    for (int32_t v = 0; v < n; ++v) rep[v] = -1;
    for (int32_t v = 0; v < n; ++v) {
        int32_t x = v;
        while (rep[x] == -1 && par[x] != x) x = par[x];
        int32_t r = rep[x] != -1 ? rep[x] : x;
        for (int32_t y = v; rep[y] == -1; y = par[y]) { rep[y] = r; if (par[y] == y) break; }
        rep[x] = r;
    }
}

/* Public: representatives of a forest (Algorithm 1, pointer-jumping line,
 * computed here by walking). */
int oracle_representatives(int32_t n, const int32_t *parent, int32_t *rep) {
    for (int32_t v = 0; v < n; ++v) if (parent[v] < 0 || parent[v] >= n) return -1;
    if (!acyclic(n, parent)) return -1;
    oracle_rep(n, parent, rep);
    return 0;
}

/*
 * One D-RSF batch update (Algorithm 1 with the readings above).
 *
 * In:  n; keys[m] the edge set of G (canonical keys, distinct); parent[n]
 *      a rooted spanning forest F of G; op 0 = insert, 1 = delete;
 *      batch[2*b] the batch B as (u, v) pairs.
 * Out: parent_out[n] = F'; repl_out (may be NULL, room for n keys) = E_r
 *      sorted by key, *nrepl_out its size; keys_out (may be NULL) receives a
 *      malloc'd, sorted copy of E(G') (free with oracle_free); stats (may be
 *      NULL).
 */
int oracle_apply(int32_t n, const uint64_t *keys, int64_t m, const int32_t *parent, int32_t op,
                 const int32_t *batch, int64_t b, int32_t *parent_out, uint64_t *repl_out,
                 int64_t *nrepl_out, uint64_t **keys_out, oracle_stats *stats) {
    oracle_stats st;
    memset(&st, 0, sizeof st);
    st.batch_len = b;
    if (keys_out) *keys_out = NULL;
    for (int64_t i = 0; i < 2 * b; ++i) if (batch[i] < 0 || batch[i] >= n) return -1;
    for (int32_t v = 0; v < n; ++v) if (parent[v] < 0 || parent[v] >= n) return -1;
    if (!acyclic(n, parent)) return -1;

    int rc = -2;
    eset g = {0}, seen = {0};
    uint64_t *bk = NULL, *cross = NULL, *er = NULL, *gk = NULL;
    int32_t *par = NULL, *rep = NULL, *uf = NULL, *sroot = NULL, *pdeg = NULL, *padj_e = NULL;
    int32_t *att_x = NULL, *att_y = NULL, *q = NULL, *vis = NULL, *lab = NULL;
    int64_t *poff = NULL;

    /* --- G' = G op B after normalisation (problem statement; graph update) */
    if (eset_init(&g, m + b) || eset_init(&seen, b)) goto out;
    for (int64_t i = 0; i < m; ++i) eset_add(&g, keys[i]);
    bk = (uint64_t *)malloc((size_t)(b + 1) * sizeof(uint64_t));
    if (!bk) goto out;
    int64_t nb = 0;
    for (int64_t i = 0; i < b; ++i) {
        uint32_t u = (uint32_t)batch[2 * i], v = (uint32_t)batch[2 * i + 1];
        if (u == v) { st.self_loops++; continue; }
        uint64_t k = okey(u, v);
        if (eset_has(&seen, k)) { st.duplicates++; continue; }
        eset_add(&seen, k);
        int present = eset_has(&g, k);
        if ((op == 0 && present) || (op != 0 && !present)) { st.ignored++; continue; }
        bk[nb++] = k;
    }
    st.applied = nb;
    for (int64_t i = 0; i < nb; ++i) { if (op == 0) eset_add(&g, bk[i]); else eset_del(&g, bk[i]); }
    int64_t m2 = op == 0 ? m + nb : m - nb;
    st.m_out = m2;
    gk = (uint64_t *)malloc((size_t)(m2 + 1) * sizeof(uint64_t));
    if (!gk) goto out;
    {
        int64_t c = 0;
        for (uint64_t i = 0; i <= g.mask; ++i)
            if (g.t[i] != 0 && g.t[i] != DEAD) gk[c++] = g.t[i] - 1;
    }

    /* --- F^: delete the tree edges of B (Algorithm 1, delete branch) */
    par = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    rep = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    uf = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    sroot = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    if (!par || !rep || !uf || !sroot) goto out;
    memcpy(par, parent, (size_t)n * sizeof(int32_t));
    if (op != 0)
        for (int64_t i = 0; i < nb; ++i) {
            int32_t a = (int32_t)key_lo(bk[i]), c = (int32_t)key_hi(bk[i]);
            if (par[a] == c) { par[a] = a; st.tree_cut++; }
            else if (par[c] == a) { par[c] = c; st.tree_cut++; }
        }

    /* --- rep[v] = root of v's tree in F^ (Algorithm 1, representatives) */
    oracle_rep(n, par, rep);
    for (int32_t v = 0; v < n; ++v) if (par[v] == v) st.pieces++;

    /* --- cross edges of G' w.r.t. F^ (Section II-A), all of them */
    int64_t nc = 0;
    cross = (uint64_t *)malloc((size_t)(m2 + 1) * sizeof(uint64_t));
    if (!cross) goto out;
    for (int64_t i = 0; i < m2; ++i)
        if (rep[key_lo(gk[i])] != rep[key_hi(gk[i])]) cross[nc++] = gk[i];
    st.cross = nc;

    /* --- E_r: Kruskal over pieces in increasing key order; the result is
     * the unique minimum spanning forest of the piece multigraph, so it has
     * k - l edges and at most one edge between any two pieces. */
    qsort(cross, (size_t)nc, sizeof(uint64_t), cmp_u64);
    for (int32_t v = 0; v < n; ++v) uf[v] = v;
    er = (uint64_t *)malloc((size_t)(n + 1) * sizeof(uint64_t));
    if (!er) goto out;
    int64_t ne = 0;
    for (int64_t i = 0; i < nc; ++i)
        if (uf_union(uf, rep[key_lo(cross[i])], rep[key_hi(cross[i])])) er[ne++] = cross[i];
    st.replacement = ne;

    /* --- super-root: per merged tree, the piece with the smallest root id */
    for (int32_t v = 0; v < n; ++v) sroot[v] = -1;
    for (int32_t p = 0; p < n; ++p)
        if (par[p] == p) {
            int32_t s = uf_find(uf, p);
            if (sroot[s] == -1 || p < sroot[s]) sroot[s] = p;
        }

    /* --- orient E_r: BFS over the super-forest (pieces joined by E_r) from
     * each super-root; the piece P first reached through edge {x, y} with
     * x in P gets the oriented replacement edge x -> y (Algorithm 2 output;
     * Algorithm 1 builds R from these). */
    pdeg = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    poff = (int64_t *)calloc((size_t)n + 2, sizeof(int64_t));
    padj_e = (int32_t *)malloc((size_t)(2 * ne + 1) * sizeof(int32_t));
    att_x = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    att_y = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    q = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    vis = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    if (!pdeg || !poff || !padj_e || !att_x || !att_y || !q || !vis) goto out;
    for (int64_t i = 0; i < ne; ++i) { pdeg[rep[key_lo(er[i])]]++; pdeg[rep[key_hi(er[i])]]++; }
    for (int32_t p = 0; p < n; ++p) poff[p + 1] = poff[p] + pdeg[p];
    for (int32_t p = 0; p < n; ++p) pdeg[p] = 0;
    for (int64_t i = 0; i < ne; ++i) {
        int32_t a = rep[key_lo(er[i])], c = rep[key_hi(er[i])];
        padj_e[poff[a] + pdeg[a]++] = (int32_t)i;
        padj_e[poff[c] + pdeg[c]++] = (int32_t)i;
    }
    for (int32_t p = 0; p < n; ++p) att_x[p] = -1;
    for (int32_t s = 0; s < n; ++s) {
        if (par[s] != s || sroot[uf_find(uf, s)] != s) continue;
        int64_t h = 0, t = 0;
        vis[s] = 1;
        q[t++] = s;
        while (h < t) {
            int32_t P = q[h++];
            for (int64_t j = poff[P]; j < poff[P + 1]; ++j) {
                uint64_t e = er[padj_e[j]];
                int32_t a = (int32_t)key_lo(e), c = (int32_t)key_hi(e);
                int32_t x = rep[a] == P ? c : a;     /* endpoint in the child piece */
                int32_t y = rep[a] == P ? a : c;     /* endpoint in P */
                int32_t Q = rep[x];
                if (vis[Q]) continue;
                vis[Q] = 1;
                att_x[Q] = x;
                att_y[Q] = y;
                q[t++] = Q;
            }
        }
    }

    /* --- ReversePaths for R = {(x, rep[x])}, then parent[x] <- y
     * (Algorithm 1).  Each path x -> ... -> root(P) lies inside its own piece,
     * so pieces are handled one after another: a linked-list reversal. */
    for (int32_t P = 0; P < n; ++P) {
        if (att_x[P] < 0) continue;
        int32_t prev = att_y[P], cur = att_x[P];
        for (;;) {
            int32_t nxt = par[cur];
            par[cur] = prev;
            if (cur != att_x[P]) st.reversed++;
            if (nxt == cur) break;          /* cur was the piece root */
            prev = cur;
            cur = nxt;
        }
    }
    {
        /* l: components of G' */
        lab = uf;
        for (int32_t v = 0; v < n; ++v) lab[v] = v;
        for (int64_t i = 0; i < m2; ++i) uf_union(lab, (int32_t)key_lo(gk[i]), (int32_t)key_hi(gk[i]));
        for (int32_t v = 0; v < n; ++v) if (uf_find(lab, v) == v) st.components++;
    }

    memcpy(parent_out, par, (size_t)n * sizeof(int32_t));
    if (repl_out) memcpy(repl_out, er, (size_t)ne * sizeof(uint64_t));
    if (nrepl_out) *nrepl_out = ne;
    if (keys_out) {
        qsort(gk, (size_t)m2, sizeof(uint64_t), cmp_u64);
        *keys_out = gk;
        gk = NULL;
    }
    rc = 0;
out:
    if (stats) *stats = st;
    free(g.t); free(seen.t); free(bk); free(cross); free(er); free(gk);
    free(par); free(rep); free(uf); free(sroot); free(pdeg); free(poff); free(padj_e);
    free(att_x); free(att_y); free(q); free(vis);
    return rc;
}

void oracle_free(void *p) { free(p); }
