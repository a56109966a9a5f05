/*
 * gc_oracle.c -- plain, slow, single-threaded CPU oracle for batch-dynamic
 * 4-node graphlet counting (FDGC / IGC).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header or table with the CUDA library, and the CUDA library never calls it.
 *
 * What it computes, and where each part comes from:
 *
 *  - The six connected induced 4-vertex graphlets, in the paper's order
 *    (Fig. 1): g1 3-path, g2 3-star, g3 4-cycle, g4 tailed triangle,
 *    g5 diamond, g6 4-clique.  Sec. 3 (Problem 1) defines the target as the
 *    frequency of connected induced size-4 graphlets.
 *
 *  - A static count in the style of PGD (Sec. 3, "PGD Algorithm"): iterate
 *    over edges, count per-edge triangles t_uv = |N(u) n N(v)| and degrees,
 *    count 4-cliques and 4-cycles by marking, and derive the remaining types
 *    by combinatorial identities.  The paper prints none of PGD's identities,
 *    so they are written out here from containment counts:
 *      P  = sum_{uv in E} (d_u-1)(d_v-1) - t_uv   non-induced 3-paths
 *      S  = sum_v C(d_v, 3)                       non-induced 3-stars
 *      TT = 1/2 sum_{uv in E} t_uv (d_u+d_v-4)    non-induced tailed triangles
 *      D  = sum_{uv in E} C(t_uv, 2)              non-induced diamonds
 *      K  = number of 4-cliques
 *      Q  = 1/2 sum_{u<w} C(|N(u) n N(w)|, 2)     non-induced 4-cycles
 *    and the induced counts follow by inverting the containment matrix
 *    (a 4-clique holds 6 diamonds, 3 four-cycles, 12 tailed triangles,
 *    4 stars, 12 three-paths; a diamond holds 1 four-cycle, 4 tailed
 *    triangles, 2 stars, 6 three-paths; a 4-cycle holds 4 three-paths; a
 *    tailed triangle holds 1 star and 2 three-paths).
 *    Two independent routes compute the sums: a literal one (per-edge
 *    merges, 4-cliques from the edges inside each edge's common
 *    neighbourhood, 4-cycles from common-neighbour counts of every vertex
 *    pair) and a degree-oriented one that is fast enough for large graphs.
 *
 *  - FDGC, Algorithm 2 (Sec. 4.3): H is the subgraph induced by the k-hop
 *    neighbourhood of the batch endpoints, G_a = (H \ D) u A,
 *    G_b = (H \ A) u D, C' = PGD(G_a) - PGD(G_b), F += C', then
 *    G <- G \ D u A.  IGC (Algorithm 1, Sec. 4.2) is the case D = {}.
 *    Batches are first normalised: pairs are unordered, repeats collapse,
 *    a pair both added and deleted is removed from both (Sec. 5, fully
 *    dynamic batches), inserting an existing edge or deleting a missing one
 *    is a no-op.  The k-hop neighbourhood is taken in G u A.
 *
 * Graphs are symmetric CSR arrays with int64 row offsets and int32 columns,
 * rows sorted ascending, no self-loops, no repeated entries.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)

typedef struct {
    int64_t n;
    const int64_t *rp;
    const int32_t *col;
} ograph;

static int64_t deg_of(const ograph *g, int64_t v) { return g->rp[v + 1] - g->rp[v]; }

/* position of v in the sorted row of u, or -1 */
static int64_t find_in_row(const ograph *g, int64_t u, int64_t v) {
    int64_t lo = g->rp[u], hi = g->rp[u + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (g->col[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    if (lo < g->rp[u + 1] && g->col[lo] == v) return lo;
    return -1;
}

static int has_edge(const ograph *g, int64_t u, int64_t v) { return find_in_row(g, u, v) >= 0; }

static int64_t choose2(int64_t x) { return x * (x - 1) / 2; }
static int64_t choose3(int64_t x) { return x * (x - 1) * (x - 2) / 6; }

/* ------------------------------------------------------------------------ */
/* Induced counts from the non-induced sums (containment inversion).        */
/* s = [P, S, TT, D, K, Q];  c = [g1 .. g6]                                  */
/* ------------------------------------------------------------------------ */
void or_counts_from_sums(const int64_t *s, int64_t *c) {
    int64_t P = s[0], S = s[1], TT = s[2], D = s[3], K = s[4], Q = s[5];
    int64_t g6 = K;
    int64_t g5 = D - 6 * K;
    int64_t g3 = Q - g5 - 3 * K;
    int64_t g4 = TT - 4 * g5 - 12 * K;
    int64_t g2 = S - g4 - 2 * g5 - 4 * K;
    int64_t g1 = P - 2 * g4 - 4 * g3 - 6 * g5 - 12 * K;
    c[0] = g1; c[1] = g2; c[2] = g3; c[3] = g4; c[4] = g5; c[5] = g6;
}

/* ------------------------------------------------------------------------ */
/* Literal sums.  out = [P, S, TT, D, K, Q, IC4]; IC4 is the induced 4-cycle */
/* count by PGD's per-edge rule (only when with_ic4 != 0, else -1):          */
/*   IC4 = 1/4 sum_{uv in E} #{(w,x): w in N(u)\N[v], x in N(v)\N[u], wx in E} */
/* ------------------------------------------------------------------------ */
/* 3-vertex graphlets (the by-product of PGD's per-edge triangle counts and
 * degrees, Sec. 3): out[0] induced 2-paths, out[1] triangles.
 * Triangles: every edge u < v adds |N(u) n N(v)| (a merge of the two sorted
 * rows); each triangle is seen from its three edges.  2-paths: every vertex
 * centres C(d, 2) pairs of its edges, of which the closed ones are the
 * triangle corners (three per triangle). */
int or_counts3(int64_t n, const int64_t *rp, const int32_t *col, int64_t *out) {
    ograph g = {n, rp, col};
    int64_t wedges = 0, tsum = 0;
    for (int64_t u = 0; u < n; u++) {
        wedges += choose2(deg_of(&g, u));
        for (int64_t i = g.rp[u]; i < g.rp[u + 1]; i++) {
            int64_t v = g.col[i];
            if (v <= u) continue;
            int64_t a = g.rp[u], b = g.rp[v];
            while (a < g.rp[u + 1] && b < g.rp[v + 1]) {
                if (g.col[a] < g.col[b]) a++;
                else if (g.col[a] > g.col[b]) b++;
                else { tsum++; a++; b++; }
            }
        }
    }
    out[0] = wedges - tsum;
    out[1] = tsum / 3;
    return 0;
}

int or_sums_literal(int64_t n, const int64_t *rp, const int32_t *col, int with_ic4, int64_t *out) {
    ograph g = {n, rp, col};
    int64_t P = 0, S = 0, TT2 = 0, D = 0, K6 = 0, Q2 = 0, IC4x4 = 0;
    int64_t maxd = 0;
    for (int64_t v = 0; v < n; v++) {
        int64_t d = deg_of(&g, v);
        if (d > maxd) maxd = d;
        S += choose3(d);
    }
    int32_t *common = (int32_t *)malloc(sizeof(int32_t) * (size_t)(maxd + 1));
    if (!common) return OR_ENOMEM;
    for (int64_t u = 0; u < n; u++) {
        int64_t du = deg_of(&g, u);
        for (int64_t p = rp[u]; p < rp[u + 1]; p++) {
            int64_t v = col[p];
            if (v <= u) continue;
            int64_t dv = deg_of(&g, v);
            /* common neighbours by merging the two sorted rows */
            int64_t t = 0, i = rp[u], j = rp[v];
            while (i < rp[u + 1] && j < rp[v + 1]) {
                if (col[i] < col[j]) i++;
                else if (col[i] > col[j]) j++;
                else { common[t++] = col[i]; i++; j++; }
            }
            P += (du - 1) * (dv - 1) - t;
            TT2 += t * (du + dv - 4);
            D += choose2(t);
            for (int64_t a = 0; a < t; a++)
                for (int64_t b = a + 1; b < t; b++)
                    if (has_edge(&g, common[a], common[b])) K6++;
            if (with_ic4) {
                for (int64_t a = rp[u]; a < rp[u + 1]; a++) {
                    int64_t w = col[a];
                    if (w == v || has_edge(&g, v, w)) continue;
                    for (int64_t b = rp[v]; b < rp[v + 1]; b++) {
                        int64_t x = col[b];
                        if (x == u || has_edge(&g, u, x)) continue;
                        if (has_edge(&g, w, x)) IC4x4++;
                    }
                }
            }
        }
    }
    free(common);
    /* Q: common-neighbour count c_uw of every pair u < w, by walking the
       wedges u - v - w; then sum C(c_uw, 2) */
    int64_t *cnt = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    int64_t *touched = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!cnt || !touched) { free(cnt); free(touched); return OR_ENOMEM; }
    for (int64_t u = 0; u < n; u++) {
        int64_t nt = 0;
        for (int64_t p = rp[u]; p < rp[u + 1]; p++) {
            int64_t v = col[p];
            for (int64_t q = rp[v]; q < rp[v + 1]; q++) {
                int64_t w = col[q];
                if (w <= u) continue;
                if (cnt[w]++ == 0) touched[nt++] = w;
            }
        }
        for (int64_t i = 0; i < nt; i++) {
            Q2 += choose2(cnt[touched[i]]);
            cnt[touched[i]] = 0;
        }
    }
    free(cnt);
    free(touched);
    out[0] = P;
    out[1] = S;
    out[2] = TT2 / 2;
    out[3] = D;
    out[4] = K6 / 6;
    out[5] = Q2 / 2;
    out[6] = with_ic4 ? IC4x4 / 4 : -1;
    /* the halvings above are exact: report if a sum was odd */
    if ((TT2 & 1) || (K6 % 6) || (Q2 & 1) || (with_ic4 && (IC4x4 & 3))) return OR_EINVAL;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Degree-oriented sums (fast enough for graphs with tens of millions of    */
/* edges).  Vertices are ranked by (degree, id); every edge points from the  */
/* lower to the higher rank.                                                 */
/*  - each triangle is listed once from its lowest vertex and credited to    */
/*    its three edges;                                                       */
/*  - each 4-clique is counted once from its lowest edge;                    */
/*  - each 4-cycle is counted once at its highest-ranked vertex u: for every */
/*    w of lower rank, c = #{v in N(u) n N(w): rank v < rank u}, add C(c,2). */
/* out = [P, S, TT, D, K, Q]                                                 */
/* ------------------------------------------------------------------------ */
static const int64_t *g_sort_deg;
static int cmp_rank(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    if (g_sort_deg[x] != g_sort_deg[y]) return g_sort_deg[x] < g_sort_deg[y] ? -1 : 1;
    return x < y ? -1 : (x > y);
}

int or_sums_oriented(int64_t n, const int64_t *rp, const int32_t *col, int64_t *out) {
    ograph g = {n, rp, col};
    int64_t nn = n > 0 ? n : 1;
    int64_t m2 = rp[n];
    int64_t *degv = (int64_t *)malloc(sizeof(int64_t) * (size_t)nn);
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)nn);
    int64_t *rank = (int64_t *)malloc(sizeof(int64_t) * (size_t)nn);
    int64_t *tslot = (int64_t *)calloc((size_t)(m2 > 0 ? m2 : 1), sizeof(int64_t));
    int64_t *orp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int32_t *ocol = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m2 / 2 + 1));
    int64_t *oslot = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m2 / 2 + 1));
    int64_t *cnt = (int64_t *)calloc((size_t)nn, sizeof(int64_t));
    int64_t *touched = (int64_t *)malloc(sizeof(int64_t) * (size_t)nn);
    int32_t *tbuf = NULL;
    int rc = OR_OK;
    if (!degv || !order || !rank || !tslot || !orp || !ocol || !oslot || !cnt || !touched) { rc = OR_ENOMEM; goto done; }
    for (int64_t v = 0; v < n; v++) { degv[v] = deg_of(&g, v); order[v] = v; }
    g_sort_deg = degv;
    qsort(order, (size_t)n, sizeof(int64_t), cmp_rank);
    for (int64_t i = 0; i < n; i++) rank[order[i]] = i;
    /* out-lists (higher-rank neighbours), kept in id order, with the slot of
       each entry in the full CSR */
    int64_t maxout = 0;
    orp[0] = 0;
    for (int64_t u = 0; u < n; u++) {
        int64_t c = orp[u];
        for (int64_t p = rp[u]; p < rp[u + 1]; p++)
            if (rank[col[p]] > rank[u]) { ocol[c] = col[p]; oslot[c] = p; c++; }
        orp[u + 1] = c;
        if (c - orp[u] > maxout) maxout = c - orp[u];
    }
    tbuf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(maxout + 1));
    if (!tbuf) { rc = OR_ENOMEM; goto done; }
    int64_t K = 0, Q2 = 0;
    for (int64_t u = 0; u < n; u++) {
        for (int64_t a = orp[u]; a < orp[u + 1]; a++) {
            int64_t v = ocol[a];
            /* T = N+(u) n N+(v) */
            int64_t t = 0, i = orp[u], j = orp[v];
            while (i < orp[u + 1] && j < orp[v + 1]) {
                if (ocol[i] < ocol[j]) i++;
                else if (ocol[i] > ocol[j]) j++;
                else {
                    int64_t w = ocol[i];
                    tbuf[t++] = (int32_t)w;
                    /* triangle {u, v, w}: credit its three edges, both directions */
                    int64_t s_uv = oslot[a], s_uw = oslot[i], s_vw = oslot[j];
                    int64_t r_vu = find_in_row(&g, v, u), r_wu = find_in_row(&g, w, u), r_wv = find_in_row(&g, w, v);
                    tslot[s_uv]++; tslot[s_uw]++; tslot[s_vw]++;
                    tslot[r_vu]++; tslot[r_wu]++; tslot[r_wv]++;
                    i++; j++;
                }
            }
            /* 4-cliques {u, v, x, y} with x -> y inside T */
            for (int64_t x = 0; x < t; x++) {
                int64_t xv = tbuf[x];
                int64_t p = orp[xv], q = 0;
                while (p < orp[xv + 1] && q < t) {
                    if (ocol[p] < tbuf[q]) p++;
                    else if (ocol[p] > tbuf[q]) q++;
                    else { K++; p++; q++; }
                }
            }
        }
    }
    /* 4-cycles by pivot */
    for (int64_t u = 0; u < n; u++) {
        int64_t nt = 0;
        for (int64_t p = rp[u]; p < rp[u + 1]; p++) {
            int64_t v = col[p];
            if (rank[v] >= rank[u]) continue;
            for (int64_t q = rp[v]; q < rp[v + 1]; q++) {
                int64_t w = col[q];
                if (rank[w] >= rank[u]) continue;
                if (cnt[w]++ == 0) touched[nt++] = w;
            }
        }
        for (int64_t i = 0; i < nt; i++) {
            Q2 += choose2(cnt[touched[i]]);
            cnt[touched[i]] = 0;
        }
    }
    int64_t P = 0, S = 0, TT2 = 0, D = 0;
    for (int64_t u = 0; u < n; u++) {
        int64_t du = degv[u];
        S += choose3(du);
        for (int64_t p = rp[u]; p < rp[u + 1]; p++) {
            int64_t v = col[p];
            if (v <= u) continue;
            int64_t dv = degv[v], t = tslot[p];
            P += (du - 1) * (dv - 1) - t;
            TT2 += t * (du + dv - 4);
            D += choose2(t);
        }
    }
    out[0] = P;
    out[1] = S;
    out[2] = TT2 / 2;
    out[3] = D;
    out[4] = K;
    out[5] = Q2;
    if (TT2 & 1) rc = OR_EINVAL;
done:
    free(degv); free(order); free(rank); free(tslot); free(orp); free(ocol); free(oslot);
    free(cnt); free(touched); free(tbuf);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Batch normalisation.                                                     */
/* ------------------------------------------------------------------------ */
static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y);
}

static int key_in(const uint64_t *arr, int64_t len, uint64_t key) {
    int64_t lo = 0, hi = len;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (arr[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo < len && arr[lo] == key;
}

static uint64_t canon_key(int64_t a, int64_t b) {
    return a < b ? ((uint64_t)a << 32) | (uint64_t)b : ((uint64_t)b << 32) | (uint64_t)a;
}

/* sort + collapse repeats in place; returns the new length */
static int64_t sort_unique(uint64_t *k, int64_t len) {
    if (len <= 0) return 0;
    qsort(k, (size_t)len, sizeof(uint64_t), cmp_u64);
    int64_t w = 1;
    for (int64_t i = 1; i < len; i++)
        if (k[i] != k[w - 1]) k[w++] = k[i];
    return w;
}

/*
 * stats[0..7] = raw inserts, raw deletes, repeated inserts, repeated deletes,
 *               pairs in both (cancelled), no-op inserts, no-op deletes, 0
 * A_out / D_out must hold n_ins / n_del keys.
 */
int or_normalize(int64_t n, const int64_t *rp, const int32_t *col,
                 const int32_t *ins, int64_t n_ins, const int32_t *del, int64_t n_del,
                 uint64_t *A_out, int64_t *nA, uint64_t *D_out, int64_t *nD, int64_t *stats) {
    ograph g = {n, rp, col};
    for (int64_t i = 0; i < n_ins; i++) {
        int64_t a = ins[2 * i], b = ins[2 * i + 1];
        if (a < 0 || b < 0 || a >= n || b >= n || a == b) return OR_EINVAL;
    }
    for (int64_t i = 0; i < n_del; i++) {
        int64_t a = del[2 * i], b = del[2 * i + 1];
        if (a < 0 || b < 0 || a >= n || b >= n || a == b) return OR_EINVAL;
    }
    uint64_t *ik = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n_ins + 1));
    uint64_t *dk = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n_del + 1));
    if (!ik || !dk) { free(ik); free(dk); return OR_ENOMEM; }
    for (int64_t i = 0; i < n_ins; i++) ik[i] = canon_key(ins[2 * i], ins[2 * i + 1]);
    for (int64_t i = 0; i < n_del; i++) dk[i] = canon_key(del[2 * i], del[2 * i + 1]);
    int64_t ui = sort_unique(ik, n_ins), ud = sort_unique(dk, n_del);
    int64_t cancelled = 0, noop_i = 0, noop_d = 0, a = 0, d = 0;
    for (int64_t i = 0; i < ui; i++) {
        if (key_in(dk, ud, ik[i])) { cancelled++; continue; }
        if (has_edge(&g, (int64_t)(ik[i] >> 32), (int64_t)(ik[i] & 0xFFFFFFFFu))) { noop_i++; continue; }
        A_out[a++] = ik[i];
    }
    for (int64_t i = 0; i < ud; i++) {
        if (key_in(ik, ui, dk[i])) continue;
        if (!has_edge(&g, (int64_t)(dk[i] >> 32), (int64_t)(dk[i] & 0xFFFFFFFFu))) { noop_d++; continue; }
        D_out[d++] = dk[i];
    }
    *nA = a;
    *nD = d;
    stats[0] = n_ins; stats[1] = n_del; stats[2] = n_ins - ui; stats[3] = n_del - ud;
    stats[4] = cancelled; stats[5] = noop_i; stats[6] = noop_d; stats[7] = 0;
    free(ik);
    free(dk);
    return OR_OK;
}

/* CSR on m canonical sorted unique keys over vertices 0..n-1.  Rows come out
   sorted because the keys are sorted. */
static int csr_from_sorted_keys(int64_t n, const uint64_t *keys, int64_t m, int64_t *rp, int32_t *col) {
    for (int64_t v = 0; v <= n; v++) rp[v] = 0;
    for (int64_t i = 0; i < m; i++) {
        rp[(keys[i] >> 32) + 1]++;
        rp[(keys[i] & 0xFFFFFFFFu) + 1]++;
    }
    for (int64_t v = 0; v < n; v++) rp[v + 1] += rp[v];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!fill) return OR_ENOMEM;
    for (int64_t v = 0; v < n; v++) fill[v] = rp[v];
    /* Row x holds the a of every key (a, x) -- all below x, met in
       increasing a -- followed by the b of every key (x, b) -- all above x,
       met in increasing b.  Two passes in key order therefore leave every
       row sorted. */
    for (int64_t i = 0; i < m; i++) {
        int64_t b = (int64_t)(keys[i] & 0xFFFFFFFFu);
        col[fill[b]++] = (int32_t)(keys[i] >> 32);
    }
    for (int64_t i = 0; i < m; i++) {
        int64_t a = (int64_t)(keys[i] >> 32);
        col[fill[a]++] = (int32_t)(keys[i] & 0xFFFFFFFFu);
    }
    free(fill);
    return OR_OK;
}

/* count edges of a CSR given as canonical keys into sums via a variant */
static int sums_of_keys(int64_t n, const uint64_t *keys, int64_t m, int variant, int64_t *sums) {
    int64_t *rp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int32_t *col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    if (!rp || !col) { free(rp); free(col); return OR_ENOMEM; }
    int rc = csr_from_sorted_keys(n, keys, m, rp, col);
    int64_t tmp[7];
    if (rc == OR_OK) {
        if (variant == 0) rc = or_sums_literal(n, rp, col, 0, tmp);
        else rc = or_sums_oriented(n, rp, col, tmp);
        for (int i = 0; i < 6; i++) sums[i] = tmp[i];
    }
    free(rp);
    free(col);
    return rc;
}

/*
 * One FDGC step (Algorithm 2).
 *   F        in/out: maintained counts (uint64, wraps mod 2^64)
 *   Ca, Cb   out:    induced counts of G_a and G_b
 *   sa, sb   out:    their sums [P, S, TT, D, K, Q]
 *   info     out:    [|A|, |D|, |W|, |E(G_a)|, |E(G_b)|, cancelled, no-ops, repeats]
 *   new_rp / new_col out: G \ D u A (new_col holds rp[n] + 2 n_ins entries)
 *   region   out (optional, may be NULL): the |W| vertices of the region, sorted
 *   variant  0 = literal sums, 1 = oriented sums
 */
int or_fdgc_step(int64_t n, const int64_t *rp, const int32_t *col,
                 const int32_t *ins, int64_t n_ins, const int32_t *del, int64_t n_del,
                 int hops, int variant, uint64_t *F, int64_t *Ca, int64_t *Cb,
                 int64_t *sa, int64_t *sb, int64_t *info,
                 int64_t *new_rp, int32_t *new_col, int32_t *region) {
    ograph g = {n, rp, col};
    int rc = OR_OK;
    uint64_t *A = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n_ins + 1));
    uint64_t *Dk = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n_del + 1));
    int64_t nA = 0, nD = 0, st[8];
    int64_t *dist = NULL, *queue = NULL, *widx = NULL, *arp = NULL;
    int32_t *acol = NULL;
    uint64_t *ka = NULL, *kb = NULL, *knew = NULL;
    if (!A || !Dk) { rc = OR_ENOMEM; goto out; }
    rc = or_normalize(n, rp, col, ins, n_ins, del, n_del, A, &nA, Dk, &nD, st);
    if (rc != OR_OK) goto out;

    /* adjacency of A, for the walk in G u A */
    arp = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
    acol = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * nA + 1));
    dist = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    widx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!arp || !acol || !dist || !queue || !widx) { rc = OR_ENOMEM; goto out; }
    for (int64_t i = 0; i < nA; i++) { arp[(A[i] >> 32) + 1]++; arp[(A[i] & 0xFFFFFFFFu) + 1]++; }
    for (int64_t v = 0; v < n; v++) arp[v + 1] += arp[v];
    {
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        if (!fill) { rc = OR_ENOMEM; goto out; }
        for (int64_t v = 0; v < n; v++) fill[v] = arp[v];
        for (int64_t i = 0; i < nA; i++) {
            int64_t a = (int64_t)(A[i] >> 32), b = (int64_t)(A[i] & 0xFFFFFFFFu);
            acol[fill[a]++] = (int32_t)b;
            acol[fill[b]++] = (int32_t)a;
        }
        free(fill);
    }

    /* breadth-first walk of depth `hops` from every endpoint, in G u A */
    for (int64_t v = 0; v < n; v++) dist[v] = -1;
    int64_t qh = 0, qt = 0;
    for (int64_t i = 0; i < nA; i++) {
        int64_t e[2] = {(int64_t)(A[i] >> 32), (int64_t)(A[i] & 0xFFFFFFFFu)};
        for (int s = 0; s < 2; s++) if (dist[e[s]] < 0) { dist[e[s]] = 0; queue[qt++] = e[s]; }
    }
    for (int64_t i = 0; i < nD; i++) {
        int64_t e[2] = {(int64_t)(Dk[i] >> 32), (int64_t)(Dk[i] & 0xFFFFFFFFu)};
        for (int s = 0; s < 2; s++) if (dist[e[s]] < 0) { dist[e[s]] = 0; queue[qt++] = e[s]; }
    }
    while (qh < qt) {
        int64_t x = queue[qh++];
        if (dist[x] >= hops) continue;
        for (int64_t p = rp[x]; p < rp[x + 1]; p++) {
            int64_t y = col[p];
            if (dist[y] < 0) { dist[y] = dist[x] + 1; queue[qt++] = y; }
        }
        for (int64_t p = arp[x]; p < arp[x + 1]; p++) {
            int64_t y = acol[p];
            if (dist[y] < 0) { dist[y] = dist[x] + 1; queue[qt++] = y; }
        }
    }
    int64_t nW = 0;
    for (int64_t v = 0; v < n; v++) {
        widx[v] = dist[v] >= 0 ? nW : -1;
        if (dist[v] >= 0) { if (region) region[nW] = (int32_t)v; nW++; }
    }

    /* H = G[W]; G_a = (H \ D) u A; G_b = (H \ A) u D, on region ids 0..|W|-1 */
    int64_t mH = 0;
    for (int64_t u = 0; u < n; u++) {
        if (widx[u] < 0) continue;
        for (int64_t p = rp[u]; p < rp[u + 1]; p++)
            if (col[p] > u && widx[col[p]] >= 0) mH++;
    }
    ka = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(mH + nA + 1));
    kb = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(mH + nD + 1));
    if (!ka || !kb) { rc = OR_ENOMEM; goto out; }
    int64_t ma = 0, mb = 0;
    for (int64_t u = 0; u < n; u++) {
        if (widx[u] < 0) continue;
        for (int64_t p = rp[u]; p < rp[u + 1]; p++) {
            int64_t v = col[p];
            if (v <= u || widx[v] < 0) continue;
            uint64_t gk = canon_key(u, v);
            uint64_t rk = canon_key(widx[u], widx[v]);
            if (!key_in(Dk, nD, gk)) ka[ma++] = rk;
            if (!key_in(A, nA, gk)) kb[mb++] = rk;
        }
    }
    for (int64_t i = 0; i < nA; i++)
        ka[ma++] = canon_key(widx[A[i] >> 32], widx[A[i] & 0xFFFFFFFFu]);
    for (int64_t i = 0; i < nD; i++)
        kb[mb++] = canon_key(widx[Dk[i] >> 32], widx[Dk[i] & 0xFFFFFFFFu]);
    ma = sort_unique(ka, ma);
    mb = sort_unique(kb, mb);
    rc = sums_of_keys(nW, ka, ma, variant, sa);
    if (rc != OR_OK) goto out;
    rc = sums_of_keys(nW, kb, mb, variant, sb);
    if (rc != OR_OK) goto out;
    or_counts_from_sums(sa, Ca);
    or_counts_from_sums(sb, Cb);
    for (int i = 0; i < 6; i++) F[i] = F[i] + (uint64_t)Ca[i] - (uint64_t)Cb[i];

    /* commit: G <- G \ D u A */
    {
        int64_t m0 = rp[n] / 2;
        knew = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m0 + nA + 1));
        if (!knew) { rc = OR_ENOMEM; goto out; }
        int64_t mn = 0;
        for (int64_t u = 0; u < n; u++)
            for (int64_t p = rp[u]; p < rp[u + 1]; p++) {
                int64_t v = col[p];
                if (v <= u) continue;
                uint64_t k = canon_key(u, v);
                if (!key_in(Dk, nD, k)) knew[mn++] = k;
            }
        for (int64_t i = 0; i < nA; i++) knew[mn++] = A[i];
        mn = sort_unique(knew, mn);
        rc = csr_from_sorted_keys(n, knew, mn, new_rp, new_col);
    }
    info[0] = nA; info[1] = nD; info[2] = nW; info[3] = ma; info[4] = mb;
    info[5] = st[4]; info[6] = st[5] + st[6]; info[7] = st[2] + st[3];
out:
    free(A); free(Dk); free(dist); free(queue); free(widx); free(arp); free(acol);
    free(ka); free(kb); free(knew);
    (void)g;
    return rc;
}
