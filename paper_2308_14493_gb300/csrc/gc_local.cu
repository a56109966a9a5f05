// gc_local.cu -- the edge-local delta: the change of the maintained counts
// from the terms a batch can change, without recounting a region.  An
// alternative to steps a1..a7 for small batches; the normalisation (a0) and
// the commit (a8) are shared with the region path.
//
// Why it is exact.  F(G_a) - F(G_b) is the image under the containment
// inversion (Sec. 3, PGD's closed forms) of the difference of the
// non-induced sums N = (P, S, TT, D, K, Q) of G_a and G_b (Lemma 2 takes the
// same difference over a region).  Let X be the changed pairs of the batch
// after normalisation and V_X their endpoints.
//  * S and sum C(d,2) add a function of each vertex degree: only vertices of
//    V_X change degree.
//  * P, TT, D and sum t add, per edge uw, a function of d_u, d_w and
//    t_uw = |N(u) n N(w)|.  A triangle uwz whose t changes holds a changed
//    pair, whose endpoints are two of u, w, z, so one of u, w is in V_X; so
//    every term that changes belongs to an edge with an endpoint in V_X.
//  * K and Q count subgraphs (4-cliques, 4-cycles): the copies that differ
//    between G_a and G_b are those holding a changed pair.  A copy in G_a
//    (G_b) is counted once, at the smallest inserted (deleted) pair it holds,
//    pairs ordered by the key (min id, max id).
// Everything else is equal in G_a and G_b and cancels.  So the path sums the
// a- and b-side terms of exactly those edges, vertices and subgraphs, and
// k_finalize_local turns their differences into the six induced deltas.
//
// Work is a list of probes: each intersection of two sorted rows iterates
// the shorter one and binary-searches the longer.  The probes of all rows
// are numbered through prefix sums (an exclusive scan of per-task counts)
// and dealt one per thread, so hub rows spread over the whole grid.
//
// Maintained triangle sums.  With T2[x] = sum of t_e over the edges e at x
// (twice the triangles at x) kept for the current graph, the per-edge t of
// the edges at V_X is not needed: TT = 1/2 sum_x T2(x) (d_x - 2) changes
// only at V_X and at the third vertices of triangles through changed pairs;
// P needs the degree products of the edges at V_X (a row scan) and the
// change of sum t; D = sum C(t_e, 2) changes only on edges whose t changes,
// and those are edges of triangles through changed pairs, found from the
// pairs' common-neighbour records (each such triangle taken once, at its
// smallest changed pair).  Only they need an intersection (for the old t).
// Without valid T2 (after a region batch) every edge at V_X is intersected.
//
// Rows.  A vertex of V_X reads its union row from U (N(u) u A_u, entries
// flagged FLAG_A / FLAG_B as in the region path, built over the full row).
// Any other vertex is untouched by the batch and reads its adjacency row
// directly (in both graphs: both flags implied).
#include "gc_internal.cuh"
#include "gc_kernels.cuh"

namespace gcx {

namespace {

constexpr uint32_t AB = FLAG_A | FLAG_B;

struct Row {
    const uint32_t* p;
    int len;
    uint32_t orf;  // flags implied for every entry (plain adjacency rows)
};

__device__ __forceinline__ bool in_x(const uint32_t* __restrict__ visited, uint32_t v) {
    return (visited[v >> 5] >> (v & 31)) & 1u;
}

struct LocalView {
    const uint32_t* visited;
    const long long* U_off;
    const uint32_t* U_col;
    const long long* row_start;
    const int32_t* deg;
    const int32_t* col;

    __device__ __forceinline__ Row row(uint32_t y) const {
        if (in_x(visited, y)) {
            const long long b = U_off[y];
            return Row{U_col + b, (int)(U_off[y + 1] - b), 0u};
        }
        return Row{(const uint32_t*)(col + row_start[y]), deg[y], AB};
    }
    __device__ __forceinline__ Row urow(uint32_t y) const {  // y in V_X
        const long long b = U_off[y];
        return Row{U_col + b, (int)(U_off[y + 1] - b), 0u};
    }
};

__device__ __forceinline__ uint32_t flags_at(const Row& r, int i) { return (r.p[i] | r.orf) & AB; }

// first position in r[lo, len) whose id is >= z
__device__ __forceinline__ int row_lower(const Row& r, int lo, uint32_t z) {
    int hi = r.len;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (vid(r.p[mid]) < z) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// position of id z in r[lo, len), or -1
__device__ __forceinline__ int row_find(const Row& r, int lo, uint32_t z) {
    const int p = row_lower(r, lo, z);
    return (p < r.len && vid(r.p[p]) == z) ? p : -1;
}

// last i in [lo, n) with pre[i] <= t (pre non-decreasing, pre[lo] <= t < pre[n])
__device__ __forceinline__ long long locate(const long long* __restrict__ pre, long long n, long long t,
                                            long long lo = 0) {
    long long hi = n;
    while (hi - lo > 1) {
        const long long mid = (lo + hi) >> 1;
        if (pre[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

// The same for the 32 consecutive t of a warp (t non-decreasing over the
// lanes; every lane calls it): one search for lane 0, then each lane steps
// forward over a few task boundaries, or searches the rest when there are
// more (runs of empty tasks).
__device__ __forceinline__ long long locate_warp(const long long* __restrict__ pre, long long n, long long t,
                                                 bool valid) {
    const long long t0 = __shfl_sync(FULL, t, 0);
    long long e = 0;
    if ((threadIdx.x & 31) == 0) e = locate(pre, n, t0);
    e = __shfl_sync(FULL, e, 0);
    if (valid) {
        for (int k = 0; e + 1 < n && pre[e + 1] <= t; k++) {
            if (k == 4) {
                e = locate(pre, n, t, e + 1);
                break;
            }
            e++;
        }
    }
    return e;
}

// The task that holds probe s, searched forward from task e (pre[e] <= s <
// pre[n]; every lane calls it with the same s and e): 32 task boundaries per
// coalesced load, so runs of empty tasks are crossed quickly; a binary search
// after four full windows.
__device__ __forceinline__ long long next_task(const long long* __restrict__ pre, long long n, long long s,
                                               long long e) {
    for (int it = 0; it < 4; it++) {
        const long long k = e + 1 + (threadIdx.x & 31);
        const unsigned m = __ballot_sync(FULL, k < n && pre[k] <= s);
        e += __popc(m);
        if (m != FULL) return e;
    }
    long long r = 0;
    if ((threadIdx.x & 31) == 0) r = locate(pre, n, s, e);
    return __shfl_sync(FULL, r, 0);
}

__device__ __forceinline__ unsigned long long pkey(uint32_t a, uint32_t b) {
    return a < b ? ((unsigned long long)a << 32) | b : ((unsigned long long)b << 32) | a;
}

// Changed pair slot i of the batch: kept insertion entries first, then kept
// deletions (both directions are listed; the slot with src < dst stands for
// the pair).  x = the graph the pair belongs to (FLAG_A inserted, FLAG_B
// deleted).
struct Pair {
    uint32_t a, b, x;
};
__device__ __forceinline__ Pair pair_at(const Ctl* c, const int32_t* __restrict__ srcA,
                                        const int32_t* __restrict__ dstA, const int32_t* __restrict__ srcD,
                                        const int32_t* __restrict__ dstD, long long i) {
    if (i < c->nA2) return Pair{(uint32_t)srcA[i], (uint32_t)dstA[i], FLAG_A};
    const long long j = i - c->nA2;
    return Pair{(uint32_t)srcD[j], (uint32_t)dstD[j], FLAG_B};
}

// For the 4-cycles through a pair, the neighbours w of one endpoint v are
// walked and each N(w) is intersected with the other endpoint's row; the
// endpoint with the cheaper walk was chosen by k_loc_pair_cost (walk[i] = 1:
// v = a).
__device__ __forceinline__ void c4_orient(const Pair& p, int walk_a, uint32_t* v, uint32_t* u) {
    *v = walk_a ? p.a : p.b;
    *u = walk_a ? p.b : p.a;
}

__device__ __forceinline__ void acc_warp(Ctl* c, int slot, unsigned long long x) {
    x = warp_sum_u64(x);
    if ((threadIdx.x & 31) == 0 && x) {
        const int stripe = (int)((blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) & (ACC_STRIPES - 1));
        atomicAdd(&c->accs[slot][stripe], x);
    }
}

// Position in U_col of the entry that stands for edge (x, y), x in V_X: the
// row of the lower endpoint when both are in V_X, else x's row (the entry
// the per-edge kernels take; the edge is in the union graph).
__device__ __forceinline__ long long canon_pos(const LocalView& V, uint32_t x, uint32_t y) {
    if (in_x(V.visited, y) && y < x) {
        const uint32_t t = x;
        x = y;
        y = t;
    }
    const Row r = V.urow(x);
    return V.U_off[x] + row_find(r, 0, y);
}

// packed common-neighbour record of a changed pair (u, v): id z, the flags of
// uz and vz (bit 0 FLAG_A, bit 1 FLAG_B), and whether z is in both rows
constexpr int T_FU = 32, T_FV = 34;
constexpr unsigned long long T_VALID = 1ull << 36;
__device__ __forceinline__ uint32_t t_flags(unsigned long long r, int at) {
    return (uint32_t)((r >> at) & 3ull) << 30;
}

}  // namespace

// ---- scratch bounds ---------------------------------------------------------

// After the union rows: the entry and pair-slot scans run only if their
// arrays fit.
__global__ void k_loc_check_rows(Ctl* c, long long cap) {
    pdl_enter();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const long long np = c->nA2 + c->nD2;
    c->l_np = np;
    bool ovf = c->nU > cap || np > cap;
    if (ovf) {
        c->lovf = 1;
        c->l_need = max(c->l_need, max(c->nU, np));
    }
    const bool run = !c->err && !c->lovf;
    c->l_len[0] = run ? c->nU : 0;
    c->l_len[1] = run ? np : 0;
}

// After the pair scans: common-neighbour records and 4-cycle tasks.
__global__ void k_loc_check_pairs(Ctl* c, long long cap) {
    pdl_enter();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const bool ovf = c->l_tot[1] > cap || c->l_tot[3] > cap;
    if (ovf) {
        c->lovf = 1;
        c->l_need = max(c->l_need, max(c->l_tot[1], c->l_tot[3]));
    }
    const bool run = !c->err && !c->lovf;
    c->l_len[2] = run ? c->l_tot[1] : 0;
    c->l_len[3] = run ? c->l_tot[3] : 0;
    if (!run) {
        c->l_len[0] = c->l_len[1] = 0;
        c->l_tot[0] = c->l_tot[2] = c->l_tot[4] = 0;
    }
}

// ---- triangles per edge with an endpoint in V_X -----------------------------

// Owner of every union-row entry: own[e] = u for the entries of u's row (a
// warp per vertex of V_X; a hub row is a long run of coalesced stores).
__global__ void k_loc_owner(const Ctl* c, const int32_t* __restrict__ wlist, LocalView V,
                            int32_t* __restrict__ own) {
    pdl_enter();
    const int nX = c->l_len[0] ? c->lvl[0] : 0;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < nX; i += nwarps) {
        const int32_t u = wlist[i];
        const long long b = V.U_off[u], e = V.U_off[u + 1];
        for (long long j = b + lane; j < e; j += 32) own[j] = u;
    }
}

// Probes of edge (u, w) for u in V_X: the shorter of the two rows.  An edge
// with both endpoints in V_X is taken from its lower endpoint only.
__global__ void k_loc_tri_cost(const Ctl* c, LocalView V, const int32_t* __restrict__ own,
                               int32_t* __restrict__ cost) {
    pdl_enter();
    const long long tot = c->l_len[0];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const uint32_t u = (uint32_t)own[e];
        const uint32_t w = vid(V.U_col[e]);
        int k = 0;
        if (!(in_x(V.visited, w) && w < u)) k = min((int)(V.U_off[u + 1] - V.U_off[u]), V.row(w).len);
        cost[e] = k;
    }
}

// ---- per-edge and per-vertex terms --------------------------------------------

// The a- and b-side terms of every edge with an endpoint in V_X (a thread
// per entry) and of every vertex of V_X, into the accumulator slots of the
// region path.
__global__ void k_loc_terms(Ctl* c, const int32_t* __restrict__ wlist, LocalView V,
                            const int32_t* __restrict__ own, const unsigned long long* __restrict__ tpack,
                            const int32_t* __restrict__ da, const int32_t* __restrict__ db) {
    pdl_enter();
    const long long tot = c->l_len[0];
    const int nX = tot ? c->lvl[0] : 0;
    const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    unsigned long long P[2] = {0, 0}, S[2] = {0, 0}, T[2] = {0, 0}, D[2] = {0, 0}, E[2] = {0, 0};
    unsigned long long T3[2] = {0, 0}, W2[2] = {0, 0};
    for (long long i = gid; i < nX; i += stride) {
        const uint32_t u = (uint32_t)wlist[i];
        S[0] += choose3((unsigned long long)da[u]);
        S[1] += choose3((unsigned long long)db[u]);
        W2[0] += choose2((unsigned long long)da[u]);
        W2[1] += choose2((unsigned long long)db[u]);
    }
    for (long long e = gid; e < tot; e += stride) {
        const uint32_t u = (uint32_t)own[e];
        const uint32_t fe = V.U_col[e];
        const uint32_t w = vid(fe);
        const bool wx = in_x(V.visited, w);
        if (wx && w < u) continue;
        const long long dau = da[u], dbu = db[u];
        const unsigned long long t = tpack[e];
        if (fe & FLAG_A) {
            const long long dw = wx ? da[w] : V.deg[w], tt = (long long)(t >> 32);
            P[0] += (unsigned long long)((dau - 1) * (dw - 1) - tt);
            T[0] += (unsigned long long)(tt * (dau + dw - 4));
            D[0] += choose2((unsigned long long)tt);
            T3[0] += (unsigned long long)tt;
            E[0] += 1;
        }
        if (fe & FLAG_B) {
            const long long dw = wx ? db[w] : V.deg[w], tt = (long long)(t & 0xFFFFFFFFull);
            P[1] += (unsigned long long)((dbu - 1) * (dw - 1) - tt);
            T[1] += (unsigned long long)(tt * (dbu + dw - 4));
            D[1] += choose2((unsigned long long)tt);
            T3[1] += (unsigned long long)tt;
            E[1] += 1;
        }
    }
    for (int g = 0; g < 2; g++) {
        const int o = 6 * g;
        acc_warp(c, o + 0, P[g]);
        acc_warp(c, o + 1, S[g]);
        acc_warp(c, o + 2, T[g]);
        acc_warp(c, o + 3, D[g]);
        acc_warp(c, 12 + g, E[g]);
        acc_warp(c, 16 + g, T3[g]);
        acc_warp(c, 18 + g, W2[g]);
    }
}

// ---- changed pairs: common neighbours and 4-cycle tasks -----------------------

// Per pair slot: probes of its common-neighbour list (shorter row) and the
// number of 4-cycle tasks (one per entry of the walked row).
__global__ void k_loc_pair_cost(const Ctl* c, LocalView V, const int32_t* __restrict__ srcA,
                                const int32_t* __restrict__ dstA, const int32_t* __restrict__ srcD,
                                const int32_t* __restrict__ dstD, int32_t* __restrict__ pcost,
                                int32_t* __restrict__ ccnt, int32_t* __restrict__ walk) {
    pdl_enter();
    // a warp per pair slot: the 4-cycle probes of walking either endpoint,
    // sum over its neighbours w of min(|N(w)|, |other row|)
    const long long np = c->l_len[1];
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = warp; i < np; i += nwarps) {
        const Pair p = pair_at(c, srcA, dstA, srcD, dstD, i);
        int k = 0, m = 0, wa = 0;
        if (p.a < p.b) {
            const Row ra = V.urow(p.a), rb = V.urow(p.b);
            unsigned long long ca = 0, cb = 0;
            for (int j = lane; j < ra.len; j += 32) ca += (unsigned long long)min(V.row(vid(ra.p[j])).len, rb.len);
            for (int j = lane; j < rb.len; j += 32) cb += (unsigned long long)min(V.row(vid(rb.p[j])).len, ra.len);
            ca = warp_sum_u64(ca);
            cb = warp_sum_u64(cb);
            wa = ca < cb || (ca == cb && ra.len >= rb.len);
            k = min(ra.len, rb.len);
            m = wa ? ra.len : rb.len;
        }
        if (lane == 0) {
            pcost[i] = k;
            ccnt[i] = m;
            walk[i] = wa;
        }
    }
}

// Common neighbours of each changed pair (u, v) = (a, b): one record per
// entry of the shorter row, in id order; valid when the id is in both rows.
__global__ void k_loc_common(const Ctl* c, LocalView V, const int32_t* __restrict__ srcA,
                             const int32_t* __restrict__ dstA, const int32_t* __restrict__ srcD,
                             const int32_t* __restrict__ dstD, const long long* __restrict__ ppre,
                             unsigned long long* __restrict__ rec) {
    pdl_enter();
    const long long np = c->l_len[1];
    const long long tot = c->l_len[2];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long tb = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); tb < tot; tb += stride) {
        const long long t = tb + (threadIdx.x & 31);
        const long long i = locate_warp(ppre, np, t, t < tot);
        if (t >= tot) continue;
        const int k = (int)(t - ppre[i]);
        const Pair p = pair_at(c, srcA, dstA, srcD, dstD, i);
        const Row ra = V.urow(p.a), rb = V.urow(p.b);
        uint32_t z, fa, fb;
        int q;
        if (ra.len <= rb.len) {
            z = vid(ra.p[k]);
            fa = flags_at(ra, k);
            q = row_find(rb, 0, z);
            fb = q < 0 ? 0u : flags_at(rb, q);
        } else {
            z = vid(rb.p[k]);
            fb = flags_at(rb, k);
            q = row_find(ra, 0, z);
            fa = q < 0 ? 0u : flags_at(ra, q);
        }
        unsigned long long r = z;
        if (q >= 0)
            r |= ((unsigned long long)(fa >> 30) << T_FU) | ((unsigned long long)(fb >> 30) << T_FV) | T_VALID;
        rec[t] = r;
    }
}

// ---- 4-cliques holding a changed pair -------------------------------------------

// For a common neighbour w of pair (u, v) in the pair's graph x, the
// 4-cliques {u, v, w, z} with z > w: probes of the shorter of the pair's
// remaining records and w's row beyond w.
__global__ void k_loc_k4_cost(const Ctl* c, LocalView V, const int32_t* __restrict__ srcA,
                              const int32_t* __restrict__ dstA, const int32_t* __restrict__ srcD,
                              const int32_t* __restrict__ dstD, const long long* __restrict__ ppre,
                              const unsigned long long* __restrict__ rec, int32_t* __restrict__ kcost) {
    pdl_enter();
    const long long np = c->l_len[1];
    const long long tot = c->l_len[2];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long tb = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); tb < tot; tb += stride) {
        const long long t = tb + (threadIdx.x & 31);
        const long long i = locate_warp(ppre, np, t, t < tot);
        if (t >= tot) continue;
        const unsigned long long r = rec[t];
        int k = 0;
        if (r & T_VALID) {
            const Pair p = pair_at(c, srcA, dstA, srcD, dstD, i);
            if (t_flags(r, T_FU) & t_flags(r, T_FV) & p.x) {
                const uint32_t w = (uint32_t)(r & 0xFFFFFFFFull);
                const Row rw = V.row(w);
                const int lr = rw.len - row_lower(rw, 0, w + 1);
                const long long lt = ppre[i + 1] - t - 1;
                k = (int)min((long long)lr, lt);
            }
        }
        kcost[t] = k;
    }
}

__global__ void k_loc_k4(Ctl* c, LocalView V, const int32_t* __restrict__ srcA, const int32_t* __restrict__ dstA,
                         const int32_t* __restrict__ srcD, const int32_t* __restrict__ dstD,
                         const long long* __restrict__ ppre, const unsigned long long* __restrict__ rec,
                         const long long* __restrict__ kpre) {
    pdl_enter();
    const long long np = c->l_len[1];
    const long long n = c->l_len[2];
    const long long tot = n ? kpre[n] : 0;
    unsigned long long ka = 0, kb = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long sb = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); sb < tot; sb += stride) {
        const long long s = sb + (threadIdx.x & 31);
        const long long t = locate_warp(kpre, n, s, s < tot);
        const long long i = locate_warp(ppre, np, t, s < tot);
        if (s >= tot) continue;
        const int k = (int)(s - kpre[t]);
        const Pair p = pair_at(c, srcA, dstA, srcD, dstD, i);
        const unsigned long long rw_rec = rec[t];
        const uint32_t w = (uint32_t)(rw_rec & 0xFFFFFFFFull);
        const Row rw = V.row(w);
        const int pos = row_lower(rw, 0, w + 1);
        const long long lt = ppre[i + 1] - t - 1;
        const int lr = rw.len - pos;
        uint32_t z, fuz = 0, fvz = 0, fwz = 0;
        bool ok = false;
        if (lt <= (long long)lr) {
            const unsigned long long rz = rec[t + 1 + k];
            z = (uint32_t)(rz & 0xFFFFFFFFull);
            if (rz & T_VALID) {
                const int q = row_find(rw, pos, z);
                if (q >= 0) {
                    ok = true;
                    fuz = t_flags(rz, T_FU);
                    fvz = t_flags(rz, T_FV);
                    fwz = flags_at(rw, q);
                }
            }
        } else {
            z = vid(rw.p[pos + k]);
            fwz = flags_at(rw, pos + k);
            // binary search of z among the pair's records after t (sorted by id)
            long long lo = t + 1, hi = ppre[i + 1];
            while (lo < hi) {
                const long long mid = (lo + hi) >> 1;
                if ((uint32_t)(rec[mid] & 0xFFFFFFFFull) < z) lo = mid + 1;
                else hi = mid;
            }
            if (lo < ppre[i + 1]) {
                const unsigned long long rz = rec[lo];
                if ((uint32_t)(rz & 0xFFFFFFFFull) == z && (rz & T_VALID)) {
                    ok = true;
                    fuz = t_flags(rz, T_FU);
                    fvz = t_flags(rz, T_FV);
                }
            }
        }
        if (!ok) continue;
        const uint32_t x = p.x;
        const uint32_t fuw = t_flags(rw_rec, T_FU), fvw = t_flags(rw_rec, T_FV);
        if (!(fuw & fvw & fuz & fvz & fwz & x)) continue;
        // counted at the smallest changed pair of graph x in the clique
        const unsigned long long kp = pkey(p.a, p.b);
        const uint32_t ids[5][2] = {{p.a, w}, {p.b, w}, {p.a, z}, {p.b, z}, {w, z}};
        const uint32_t fl[5] = {fuw, fvw, fuz, fvz, fwz};
        bool mine = true;
#pragma unroll
        for (int q = 0; q < 5; q++)
            if (fl[q] == x && pkey(ids[q][0], ids[q][1]) < kp) mine = false;
        if (!mine) continue;
        if (x == FLAG_A) ka++;
        else kb++;
    }
    acc_warp(c, 4, ka);
    acc_warp(c, 10, kb);
}

// ---- 4-cycles holding a changed pair ----------------------------------------------

// One task per entry w of the walked endpoint v's row; its probes: the
// shorter of w's row and the other endpoint u's row.
__global__ void k_loc_c4_tasks(const Ctl* c, LocalView V, const int32_t* __restrict__ srcA,
                               const int32_t* __restrict__ dstA, const int32_t* __restrict__ srcD,
                               const int32_t* __restrict__ dstD, const long long* __restrict__ cpre,
                               const int32_t* __restrict__ walk, int32_t* __restrict__ tpair,
                               int32_t* __restrict__ tent, int32_t* __restrict__ tcost) {
    pdl_enter();
    const long long np = c->l_len[1];
    const long long tot = c->l_len[3];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long tb = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); tb < tot; tb += stride) {
        const long long tau = tb + (threadIdx.x & 31);
        const long long i = locate_warp(cpre, np, tau, tau < tot);
        if (tau >= tot) continue;
        const int j = (int)(tau - cpre[i]);
        const Pair p = pair_at(c, srcA, dstA, srcD, dstD, i);
        uint32_t v, u;
        c4_orient(p, walk[i], &v, &u);
        const uint32_t e = V.urow(v).p[j];
        const uint32_t w = vid(e);
        int k = 0;
        if (w != u && (e & p.x)) k = min(V.row(w).len, (int)(V.U_off[u + 1] - V.U_off[u]));
        tpair[tau] = (int32_t)i;
        tent[tau] = j;
        tcost[tau] = k;
    }
}

// Each block takes one contiguous range of the probes (numbered pair by
// pair, then task by task).  Before walking it the block picks the pair with
// the most probes in the range and puts the other endpoint u's union row
// (entries with their flags) into a bucketed hash table in shared memory,
// when that row has between LC4_ROW_MIN and LC4_ROW_MAX entries and the
// range holds at least two probes of the pair per entry; the probes of that
// pair that walk N(w) then look z up there instead of binary-searching u's
// row in global memory.  Probes that walk u's row (N(w) the longer) search
// N(w) as before.  4 slots to a bucket, linear probing over buckets, at most
// 3/4 of the slots filled, so every lookup ends at an empty slot.
constexpr int LC4_BUCKETS = 4096;
constexpr int LC4_ROW_MAX = 3 * LC4_BUCKETS;
constexpr int LC4_ROW_MIN = 64;
constexpr uint32_t LC4_EMPTY = 0xFFFFFFFFu;  // ids stay below 2^30 - 1
constexpr size_t LC4_SMEM = (size_t)LC4_BUCKETS * sizeof(uint4);
constexpr int LC4_THREADS = 512;
// Probes a warp takes at a time from its block's range: about an eighth of
// a warp's share, a multiple of 32 between 128 and 2048.
constexpr int LC4_CHUNK = 2048;
__device__ __forceinline__ long long lc4_chunk(long long range) {
    const long long c = (range / (8 * (LC4_THREADS / 32)) + 31) & ~31ll;
    return c < 128 ? 128 : c > LC4_CHUNK ? LC4_CHUNK : c;
}
// Blocks that take part for tot probes: about one per LC4_BLOCK_PROBES, at
// least half and at most all of the launched grid (eight waves).  More and
// smaller ranges put more of the probes under a staged row, fewer and larger
// ones pay fewer table builds: 8 waves won at 10,000 updates on c3 (6.7
// against 7.2 ms), 4 at 1,000 (1.60 against 1.78 ms).
constexpr long long LC4_BLOCK_PROBES = 65536;
__device__ __forceinline__ long long lc4_blocks(long long tot) {
    const long long g = (long long)gridDim.x, want = tot / LC4_BLOCK_PROBES;
    return want < g / 2 ? g / 2 : want > g ? g : want;
}

__device__ __forceinline__ uint32_t lc4_bucket(uint32_t z, int lgb) { return (z * 0x9E3779B1u) >> (32 - lgb); }

__device__ __forceinline__ uint32_t lc4_find(const uint4* __restrict__ tab, int lgb, uint32_t z) {
    const uint32_t mask = (1u << lgb) - 1;
    uint32_t h = lc4_bucket(z, lgb);
    for (int it = 0; it <= (int)mask; it++) {
        const uint4 q = tab[h];
        if (vid(q.x) == z) return q.x;
        if (vid(q.y) == z) return q.y;
        if (vid(q.z) == z) return q.z;
        if (vid(q.w) == z) return q.w;
        if (q.w == LC4_EMPTY) break;  // slots fill in order within a bucket
        h = (h + 1) & mask;
    }
    return LC4_EMPTY;
}

// Fills the table with row r (the whole block calls it; LC4_ROW_MIN <=
// r.len <= LC4_ROW_MAX) and returns log2 of its bucket count.
__device__ __forceinline__ int lc4_stage(uint4* tab, const Row& r) {
    int lgb = 0;
    while ((2 << lgb) < r.len) lgb++;  // buckets >= len / 2
    lgb = min(lgb, 12);
    uint32_t* slot = reinterpret_cast<uint32_t*>(tab);
    for (int q = threadIdx.x; q < (4 << lgb); q += blockDim.x) slot[q] = LC4_EMPTY;
    __syncthreads();
    const uint32_t mask = (1u << lgb) - 1;
    for (int q = threadIdx.x; q < r.len; q += blockDim.x) {
        const uint32_t e = r.p[q] | r.orf;
        uint32_t h = lc4_bucket(vid(e), lgb);
        for (bool done = false; !done; h = (h + 1) & mask)
            for (int j = 0; j < 4 && !done; j++) done = atomicCAS(&slot[4 * h + j], LC4_EMPTY, e) == LC4_EMPTY;
    }
    __syncthreads();
    return lgb;
}

__global__ void __launch_bounds__(LC4_THREADS, 3) k_loc_c4(Ctl* c, LocalView V, const int32_t* __restrict__ srcA,
                                                const int32_t* __restrict__ dstA, const int32_t* __restrict__ srcD,
                                                const int32_t* __restrict__ dstD, const int32_t* __restrict__ walk,
                                                const int32_t* __restrict__ tpair, const int32_t* __restrict__ tent,
                                                const long long* __restrict__ tpre,
                                                const long long* __restrict__ cpre) {
    pdl_enter();
    extern __shared__ uint4 tab[];
    __shared__ unsigned long long s_best, s_chunk;
    __shared__ long long s_pair[2];
    const long long n = c->l_len[3];
    const long long tot = n ? tpre[n] : 0;
    const long long nb = lc4_blocks(tot);
    if (blockIdx.x >= nb) return;
    const long long lo = tot * blockIdx.x / nb, hi = tot * (blockIdx.x + 1) / nb;
    unsigned long long qa = 0, qb = 0;
    if (lo < hi) {
        // the pair with the most probes in [lo, hi) whose u row can be staged
        if (threadIdx.x == 0) {
            s_best = 0;
            s_chunk = (unsigned long long)lo;
            s_pair[0] = tpair[locate(tpre, n, lo)];
            s_pair[1] = tpair[locate(tpre, n, hi - 1)];
        }
        __syncthreads();
        for (long long i = s_pair[0] + threadIdx.x; i <= s_pair[1]; i += blockDim.x) {
            const long long ta = cpre[i], tb = cpre[i + 1];
            if (ta >= tb) continue;
            const long long cnt = min(hi, tpre[tb]) - max(lo, tpre[ta]);
            const Pair p = pair_at(c, srcA, dstA, srcD, dstD, i);
            const uint32_t u = walk[i] ? p.b : p.a;
            const long long len = V.U_off[u + 1] - V.U_off[u];
            if (len < LC4_ROW_MIN || len > LC4_ROW_MAX || cnt < 2 * len) continue;
            atomicMax(&s_best, ((unsigned long long)min(cnt, 0xFFFFFFFFll) << 32) | (unsigned long long)i);
        }
        __syncthreads();
        const unsigned long long best = s_best;
        const long long sp = best ? (long long)(uint32_t)best : -1;
        int lgb = 0;
        if (sp >= 0) {
            const Pair p = pair_at(c, srcA, dstA, srcD, dstD, sp);
            lgb = lc4_stage(tab, V.urow(walk[sp] ? p.b : p.a));
        }
        // the warps take chunks of the block's range in turn (probe costs
        // differ tenfold, so equal shares would leave warps idle) and walk
        // each chunk task by task: the task's pair, rows and walked entry
        // once, then its probes 32 at a time
        const int lane = threadIdx.x & 31;
        const long long chunk = lc4_chunk(hi - lo);
        long long tau = 0;
        if (lane == 0) tau = locate(tpre, n, lo);
        tau = __shfl_sync(FULL, tau, 0);
        for (long long s = 0, whi = 0;;) {
            if (s >= whi) {
                long long c0 = 0;
                if (lane == 0) c0 = (long long)atomicAdd(&s_chunk, (unsigned long long)chunk);
                c0 = __shfl_sync(FULL, c0, 0);
                if (c0 >= hi) break;
                s = c0;
                whi = min(hi, c0 + chunk);
            }
            tau = next_task(tpre, n, s, tau);
            const long long pe = tpre[tau + 1], pb = tpre[tau];
            const int k0 = (int)(s - pb), k1 = (int)(min(whi, pe) - pb);
            s = min(whi, pe);
            const int pi = tpair[tau];
            const Pair p = pair_at(c, srcA, dstA, srcD, dstD, pi);
            uint32_t v, u;
            c4_orient(p, walk[pi], &v, &u);
            const uint32_t ev = V.urow(v).p[tent[tau]];
            const uint32_t w = vid(ev), fvw = ev & AB, x = p.x;
            // the cycle u-v-w-z-u is counted at its smallest changed pair of graph x
            const unsigned long long kp = pkey(p.a, p.b);
            if (!(fvw & x) || (fvw == x && pkey(v, w) < kp)) continue;
            const Row ru = V.urow(u), rw = V.row(w);
            unsigned q4 = 0;
            const bool staged = pi == sp;
            // with u's row staged, a task whose N(w) is longer (at most four
            // times) still walks N(w) when the task lies wholly in this
            // block's range: its probe range [k0, k1) of u's row maps to the
            // proportional range of N(w), so the chunks that split the task
            // split N(w) exactly.  A task that a block boundary cuts keeps
            // walking u's row in both blocks, whichever pairs they stage.
            const bool walk_w =
                rw.len <= ru.len || (staged && pb >= lo && pe <= hi && rw.len <= 4 * ru.len);
            if (walk_w) {
                const int j0 = rw.len <= ru.len ? k0 : (int)((long long)k0 * rw.len / ru.len);
                const int j1 = rw.len <= ru.len ? k1 : (int)((long long)k1 * rw.len / ru.len);
                for (int k = j0 + lane; k < j1; k += 32) {
                    const uint32_t z = vid(rw.p[k]), fwz = flags_at(rw, k);
                    if (z == v || !(fwz & x)) continue;
                    uint32_t fuz;
                    if (staged) {
                        const uint32_t e = lc4_find(tab, lgb, z);
                        if (e == LC4_EMPTY) continue;
                        fuz = e & AB;
                    } else {
                        const int q = row_find(ru, 0, z);
                        if (q < 0) continue;
                        fuz = flags_at(ru, q);
                    }
                    if (!(fuz & x) || (fwz == x && pkey(w, z) < kp) || (fuz == x && pkey(u, z) < kp)) continue;
                    q4++;
                }
            } else {
                for (int k = k0 + lane; k < k1; k += 32) {
                    const uint32_t z = vid(ru.p[k]), fuz = flags_at(ru, k);
                    if (z == v || !(fuz & x)) continue;
                    const int q = row_find(rw, 0, z);
                    if (q < 0) continue;
                    const uint32_t fwz = flags_at(rw, q);
                    if (!(fwz & x) || (fwz == x && pkey(w, z) < kp) || (fuz == x && pkey(u, z) < kp)) continue;
                    q4++;
                }
            }
            if (x == FLAG_A) qa += q4;
            else qb += q4;
        }
    }
    acc_warp(c, 5, qa);
    acc_warp(c, 11, qb);
}

// t_e for G_a and G_b packed into tpack[e] (high 32 bits G_a, low 32 G_b).
// The probes are numbered edge by edge, and the edges of one owner u are
// consecutive.  Each block takes one contiguous range of the probes and
// stages the union row of the owner with the most probes in it (of the
// owners of its first, middle and last probe) in the shared-memory hash,
// under the same bounds as the 4-cycle kernel; that owner's edges whose probes
// walk N(w) look z up there.  The warps take chunks of the block's range in
// turn and walk each edge by edge: the edge's rows once, then its probes 32
// at a time, the hits summed over the warp before one atomic per edge and
// chunk.
__global__ void __launch_bounds__(LC4_THREADS, 3) k_loc_tri(const Ctl* c, LocalView V,
                                                            const long long* __restrict__ pre,
                                                            const int32_t* __restrict__ own,
                                                            unsigned long long* __restrict__ tpack) {
    pdl_enter();
    extern __shared__ uint4 tab[];
    __shared__ int32_t s_cand[3];
    __shared__ unsigned long long s_chunk;
    const long long n = c->l_len[0];
    if (n == 0) return;
    const long long tot = pre[n];
    const long long nb = lc4_blocks(tot);
    if (blockIdx.x >= nb) return;
    const long long lo = tot * blockIdx.x / nb, hi = tot * (blockIdx.x + 1) / nb;
    if (lo >= hi) return;
    if (threadIdx.x < 3) {
        const long long t = threadIdx.x == 0 ? lo : threadIdx.x == 1 ? lo + (hi - lo) / 2 : hi - 1;
        s_cand[threadIdx.x] = own[locate(pre, n, t)];
    }
    if (threadIdx.x == 0) s_chunk = (unsigned long long)lo;
    __syncthreads();
    long long su = -1, best = 0;
    for (int j = 0; j < 3; j++) {
        const uint32_t u = (uint32_t)s_cand[j];
        const long long b = V.U_off[u], e = V.U_off[u + 1];
        const long long cnt = min(hi, pre[e]) - max(lo, pre[b]);
        if (e - b < LC4_ROW_MIN || e - b > LC4_ROW_MAX || cnt < 2 * (e - b) || cnt <= best) continue;
        best = cnt;
        su = u;
    }
    int lgb = 0;
    if (su >= 0) lgb = lc4_stage(tab, V.urow((uint32_t)su));
    const int lane = threadIdx.x & 31;
    const long long chunk = lc4_chunk(hi - lo);
    long long e = 0;
    if (lane == 0) e = locate(pre, n, lo);
    e = __shfl_sync(FULL, e, 0);
    for (long long s = 0, whi = 0;;) {
        if (s >= whi) {
            long long c0 = 0;
            if (lane == 0) c0 = (long long)atomicAdd(&s_chunk, (unsigned long long)chunk);
            c0 = __shfl_sync(FULL, c0, 0);
            if (c0 >= hi) break;
            s = c0;
            whi = min(hi, c0 + chunk);
        }
        e = next_task(pre, n, s, e);
        const long long pe = pre[e + 1], pb = pre[e];
        const int k0 = (int)(s - pb), k1 = (int)(min(whi, pe) - pb);
        s = min(whi, pe);
        const uint32_t u = (uint32_t)own[e];
        const Row ru = V.urow(u);
        const Row rw = V.row(vid(V.U_col[e]));
        unsigned ca = 0, cb = 0;
        // with u's row staged, an edge whose N(w) is longer (at most four
        // times) and whose probes lie wholly in this block's range still walks
        // N(w), over the range proportional to its probe range of u's row (an
        // edge that a block boundary cuts walks the same row in both blocks)
        const bool staged = u == su;
        if (ru.len <= rw.len && !(staged && pb >= lo && pe <= hi && rw.len <= 4 * ru.len)) {
            for (int k = k0 + lane; k < k1; k += 32) {
                const uint32_t z = ru.p[k];
                const int q = row_find(rw, 0, vid(z));
                if (q < 0) continue;
                const uint32_t f = z & flags_at(rw, q);
                ca += (f & FLAG_A) != 0;
                cb += (f & FLAG_B) != 0;
            }
        } else if (staged) {
            const int j0 = rw.len < ru.len ? k0 : (int)((long long)k0 * rw.len / ru.len);
            const int j1 = rw.len < ru.len ? k1 : (int)((long long)k1 * rw.len / ru.len);
            for (int k = j0 + lane; k < j1; k += 32) {
                const uint32_t z = rw.p[k] | rw.orf;
                const uint32_t hit = lc4_find(tab, lgb, vid(z));
                if (hit == LC4_EMPTY) continue;
                const uint32_t f = z & hit;
                ca += (f & FLAG_A) != 0;
                cb += (f & FLAG_B) != 0;
            }
        } else {
            for (int k = k0 + lane; k < k1; k += 32) {
                const uint32_t z = rw.p[k] | rw.orf;
                const int q = row_find(ru, 0, vid(z));
                if (q < 0) continue;
                const uint32_t f = z & flags_at(ru, q);
                ca += (f & FLAG_A) != 0;
                cb += (f & FLAG_B) != 0;
            }
        }
        ca = __reduce_add_sync(FULL, ca);
        cb = __reduce_add_sync(FULL, cb);
        if (lane == 0 && (ca | cb)) atomicAdd(&tpack[e], ((unsigned long long)ca << 32) | cb);
    }
}

// ---- with maintained triangle sums ---------------------------------------------------

// T2 from a static count (U = G, both flags on every entry; tpack holds t of
// every out-entry).  T2 must be zero.
__global__ void k_t2_from_static(const Ctl* c, const int32_t* __restrict__ wlist, const long long* __restrict__ U_off,
                                 const uint32_t* __restrict__ U_col, const int32_t* __restrict__ U_split,
                                 const unsigned long long* __restrict__ tpack, unsigned long long* __restrict__ T2) {
    pdl_enter();
    const int nW = c->nW;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < nW; i += nwarps) {
        const int32_t u = wlist[i];
        const long long ob = U_off[u] + U_split[u], oe = U_off[u + 1];
        unsigned long long own = 0;
        for (long long e = ob + lane; e < oe; e += 32) {
            const unsigned long long t = tpack[e] >> 32;
            if (t) {
                own += t;
                atomicAdd(&T2[vid(U_col[e])], t);
            }
        }
        own = warp_sum_u64(own);
        if (lane == 0 && own) atomicAdd(&T2[u], own);
    }
}

// After a committed region batch: T2 of the vertices within one hop of the
// batch endpoints (the only vertices whose triangles can change), from the
// region pass's triangle counts in G_a.  Those counts are exact there: with
// k >= 2 hops, a vertex within one hop has its whole neighbourhood inside
// W.  First the one-hop vertices are marked and their T2 cleared ...
__global__ void k_t2_mark(const Ctl* c, const int32_t* __restrict__ wlist, uint32_t* __restrict__ mark,
                          unsigned long long* __restrict__ T2) {
    pdl_enter();
    if (c->err || !c->active) return;
    const int n1 = c->lvl[1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n1; i += gridDim.x * blockDim.x) {
        const uint32_t x = (uint32_t)wlist[i];
        atomicOr(&mark[x >> 5], 1u << (x & 31));
        T2[x] = 0;
    }
}

// ... then every out-entry u -> v of U adds its t to T2 of the marked ends
// (a warp per vertex of W: out-lists are short, hubs having the highest ids).
__global__ void k_t2_from_region(const Ctl* c, const int32_t* __restrict__ wlist, const long long* __restrict__ U_off,
                                 const uint32_t* __restrict__ U_col, const int32_t* __restrict__ U_split,
                                 const unsigned long long* __restrict__ tpack, const uint32_t* __restrict__ mark,
                                 unsigned long long* __restrict__ T2) {
    pdl_enter();
    if (c->err || !c->active) return;
    const int nW = c->nW;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < nW; i += nwarps) {
        const uint32_t u = (uint32_t)wlist[i];
        const bool mu = in_x(mark, u);
        unsigned long long own = 0;
        for (long long e = U_off[u] + U_split[u] + lane; e < U_off[u + 1]; e += 32) {
            const uint32_t f = U_col[e];
            if (!(f & FLAG_A)) continue;
            const unsigned long long t = tpack[e] >> 32;
            if (!t) continue;
            own += t;
            const uint32_t v = vid(f);
            if (in_x(mark, v)) atomicAdd(&T2[v], t);
        }
        own = warp_sum_u64(own);
        if (lane == 0 && mu && own) atomicAdd(&T2[u], own);
    }
}

// Triangles through changed pairs, each once at its smallest changed pair:
// delta = [in G_a] - [in G_b] goes to the change of t of its three edges
// (dcnt, at their entries), to twice the change of the triangles at its
// three vertices (dtri2), and to the change of sum t.  Third vertices
// outside V_X are listed after V_X in wlist.
__global__ void k_loc_tri_delta(Ctl* c, LocalView V, const int32_t* __restrict__ srcA,
                                const int32_t* __restrict__ dstA, const int32_t* __restrict__ srcD,
                                const int32_t* __restrict__ dstD, const long long* __restrict__ ppre,
                                const unsigned long long* __restrict__ rec, long long* __restrict__ dcnt,
                                long long* __restrict__ dtri2, uint32_t* __restrict__ visited2,
                                int32_t* __restrict__ wlist) {
    pdl_enter();
    const long long np = c->l_len[1];
    const long long tot = c->l_len[2];
    const int nX = c->lvl[0];
    long long s3 = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long tb = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); tb < tot; tb += stride) {
        const long long t = tb + (threadIdx.x & 31);
        const long long i = locate_warp(ppre, np, t, t < tot);
        if (t >= tot) continue;
        const unsigned long long r = rec[t];
        if (!(r & T_VALID)) continue;
        const Pair p = pair_at(c, srcA, dstA, srcD, dstD, i);
        const uint32_t w = (uint32_t)(r & 0xFFFFFFFFull);
        const uint32_t faw = t_flags(r, T_FU), fbw = t_flags(r, T_FV);
        const unsigned long long kp = pkey(p.a, p.b);
        if ((faw != AB && pkey(p.a, w) < kp) || (fbw != AB && pkey(p.b, w) < kp)) continue;
        const uint32_t f = p.x & faw & fbw;
        const long long d = ((f & FLAG_A) ? 1 : 0) - ((f & FLAG_B) ? 1 : 0);
        if (!d) continue;
        atomicAdd((unsigned long long*)&dcnt[canon_pos(V, p.a, p.b)], (unsigned long long)d);
        atomicAdd((unsigned long long*)&dcnt[canon_pos(V, p.a, w)], (unsigned long long)d);
        atomicAdd((unsigned long long*)&dcnt[canon_pos(V, p.b, w)], (unsigned long long)d);
        atomicAdd((unsigned long long*)&dtri2[p.a], (unsigned long long)(2 * d));
        atomicAdd((unsigned long long*)&dtri2[p.b], (unsigned long long)(2 * d));
        atomicAdd((unsigned long long*)&dtri2[w], (unsigned long long)(2 * d));
        if (!in_x(V.visited, w)) {
            const uint32_t bit = 1u << (w & 31);
            if (!(atomicOr(&visited2[w >> 5], bit) & bit)) wlist[nX + atomicAdd(&c->l_nw3, 1)] = (int32_t)w;
        }
        s3 += 3 * d;
    }
    acc_warp(c, 16, (unsigned long long)s3);   // change of sum t (G_a slot; the G_b slot stays 0)
    acc_warp(c, 0, (unsigned long long)(-s3)); // P = sum (d_u - 1)(d_w - 1) - sum t
}

// Intersections only for the common edges at V_X whose t changes (their old t).
__global__ void k_loc_dcost(const Ctl* c, LocalView V, const int32_t* __restrict__ own,
                            const long long* __restrict__ dcnt, int32_t* __restrict__ cost) {
    pdl_enter();
    const long long tot = c->l_len[0];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const uint32_t u = (uint32_t)own[e];
        const uint32_t fe = V.U_col[e];
        const uint32_t w = vid(fe);
        int k = 0;
        if ((fe & AB) == AB && dcnt[e] != 0 && !(in_x(V.visited, w) && w < u))
            k = min((int)(V.U_off[u + 1] - V.U_off[u]), V.row(w).len);
        cost[e] = k;
    }
}

// Per-edge terms at V_X (a thread per entry): degree products (P), edge
// counts, and C(t, 2) (D) of the edges whose t changes.
__global__ void k_loc_eterms(Ctl* c, LocalView V, const int32_t* __restrict__ own,
                             const unsigned long long* __restrict__ tpack, const long long* __restrict__ dcnt,
                             const int32_t* __restrict__ da, const int32_t* __restrict__ db) {
    pdl_enter();
    const long long tot = c->l_len[0];
    unsigned long long P[2] = {0, 0}, D[2] = {0, 0}, E[2] = {0, 0};
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const uint32_t u = (uint32_t)own[e];
        const uint32_t fe = V.U_col[e];
        const uint32_t w = vid(fe);
        const bool wx = in_x(V.visited, w);
        if (wx && w < u) continue;
        const uint32_t f = fe & AB;
        const long long dd = dcnt[e];
        if (f & FLAG_A) {
            const long long dw = wx ? da[w] : V.deg[w];
            P[0] += (unsigned long long)(((long long)da[u] - 1) * (dw - 1));
            E[0] += 1;
        }
        if (f & FLAG_B) {
            const long long dw = wx ? db[w] : V.deg[w];
            P[1] += (unsigned long long)(((long long)db[u] - 1) * (dw - 1));
            E[1] += 1;
        }
        if (f == AB) {
            if (dd) {
                const long long tb = (long long)(tpack[e] & 0xFFFFFFFFull);
                D[0] += choose2((unsigned long long)(tb + dd));
                D[1] += choose2((unsigned long long)tb);
            }
        } else if (f == FLAG_A) {
            D[0] += choose2((unsigned long long)dd);    // dd = triangles through the inserted edge
        } else {
            D[1] += choose2((unsigned long long)(-dd));  // -dd = triangles through the deleted edge
        }
    }
    for (int g = 0; g < 2; g++) {
        acc_warp(c, 6 * g + 0, P[g]);
        acc_warp(c, 6 * g + 3, D[g]);
        acc_warp(c, 12 + g, E[g]);
    }
}

// Per-vertex terms: S and sum C(d, 2) at V_X, 2 TT = sum T2(x) (d_x - 2) at
// V_X and at the third vertices; then T2 follows the batch (commit) and
// the changes are cleared.
__global__ void k_loc_vterms(Ctl* c, const int32_t* __restrict__ wlist, LocalView V,
                             unsigned long long* __restrict__ T2, long long* __restrict__ dtri2,
                             const int32_t* __restrict__ da, const int32_t* __restrict__ db, int commit) {
    pdl_enter();
    const int nX = c->l_len[0] ? c->lvl[0] : 0;
    const int nT = nX ? nX + c->l_nw3 : 0;
    const bool apply = commit && c->err == 0 && c->active && c->lovf == 0;
    unsigned long long S[2] = {0, 0}, W2[2] = {0, 0}, T[2] = {0, 0};
    const int nT_r = (nT + 31) & ~31;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nT_r; i += gridDim.x * blockDim.x) {
        if (i >= nT) continue;
        const uint32_t x = (uint32_t)wlist[i];
        const bool inX = i < nX;
        const long long dxa = inX ? da[x] : V.deg[x], dxb = inX ? db[x] : V.deg[x];
        const long long t2b = (long long)T2[x], dt = dtri2[x], t2a = t2b + dt;
        T[0] += (unsigned long long)(t2a * (dxa - 2));
        T[1] += (unsigned long long)(t2b * (dxb - 2));
        if (inX) {
            S[0] += choose3((unsigned long long)dxa);
            S[1] += choose3((unsigned long long)dxb);
            W2[0] += choose2((unsigned long long)dxa);
            W2[1] += choose2((unsigned long long)dxb);
        }
        if (apply) T2[x] = (unsigned long long)t2a;
        dtri2[x] = 0;
    }
    for (int g = 0; g < 2; g++) {
        acc_warp(c, 6 * g + 1, S[g]);
        acc_warp(c, 6 * g + 2, T[g]);
        acc_warp(c, 18 + g, W2[g]);
    }
}

// ---- closed forms on the differences -------------------------------------------------

// commit = 1: F += delta (the batch is applied); 0: the result is F + delta
// and F stays.  Nothing changes after a scratch overflow (the host re-runs
// the batch).  Ca holds the six induced deltas and sa the non-induced ones
// (Cb, sb zero).
__global__ void k_finalize_local(Ctl* c, int commit) {
    pdl_enter();
    if (blockIdx.x == 0 && threadIdx.x < NACC) {
        unsigned long long x = 0;
        for (int k = 0; k < ACC_STRIPES; k++) x += c->accs[threadIdx.x][k];
        c->acc[threadIdx.x] += x;
    }
    __syncwarp();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const unsigned long long* a = c->acc;
    const long long P = (long long)(a[0] - a[6]), S = (long long)(a[1] - a[7]);
    const long long TT = (long long)(a[2] - a[8]) / 2;  // both full sums are even
    const long long D = (long long)(a[3] - a[9]), K = (long long)(a[4] - a[10]), Q = (long long)(a[5] - a[11]);
    const long long g6 = K;
    const long long g5 = D - 6 * K;
    const long long g3 = Q - g5 - 3 * K;
    const long long g4 = TT - 4 * g5 - 12 * K;
    const long long g2 = S - g4 - 2 * g5 - 4 * K;
    const long long g1 = P - 2 * g4 - 4 * g3 - 6 * g5 - 12 * K;
    const long long d[6] = {g1, g2, g3, g4, g5, g6};
    const long long s[6] = {P, S, TT, D, K, Q};
    const long long t3 = (long long)(a[16] - a[17]);  // 3 x change of triangles
    const long long d3[2] = {(long long)(a[18] - a[19]) - t3, t3 / 3};
    const bool ok = c->err == 0 && c->active && c->lovf == 0;
    for (int i = 0; i < 6; i++) {
        c->Ca[i] = d[i];
        c->Cb[i] = 0;
        c->sa[i] = s[i];
        c->sb[i] = 0;
        if (commit && ok) c->F[i] += (unsigned long long)d[i];
        c->last_out[i] = commit ? c->F[i] : c->F[i] + (unsigned long long)d[i];
    }
    for (int i = 0; i < 2; i++) {
        c->C3a[i] = d3[i];
        c->C3b[i] = 0;
        if (commit && ok) c->F3[i] += (unsigned long long)d3[i];
        c->last_out3[i] = commit ? c->F3[i] : c->F3[i] + (unsigned long long)d3[i];
    }
    c->acc[14] = (unsigned long long)(c->l_tot[0] + c->l_tot[2] + c->l_tot[4]);  // probes
    c->acc[15] = 0;
}

// ---- launch sequence ---------------------------------------------------------------

// Blocks of the two kernels with a staged row: eight waves of the blocks
// that fit at once (the table takes 64 KB of shared memory; three 512-thread
// blocks share an SM), of which lc4_blocks takes part, so that ranges of
// unequal cost even out.
static int g_loc_per_sm[2] = {0, 0};

template <typename K>
static int staged_per_sm(K kernel) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LC4_SMEM);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, LC4_THREADS, LC4_SMEM) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 0;
    }
    return per_sm > 0 ? per_sm : 2;
}

void local_setup_attributes() {
    g_loc_per_sm[0] = staged_per_sm(k_loc_tri);
    g_loc_per_sm[1] = staged_per_sm(k_loc_c4);
}

// kind 0: the triangle kernel, 1: the 4-cycle kernel
static int staged_grid(int kind, int sms) { return 8 * sms * (g_loc_per_sm[kind] > 0 ? g_loc_per_sm[kind] : 2); }

int enqueue_local(const LocalArgs& a, cudaStream_t s, cudaEvent_t ev_tri, cudaEvent_t ev_sub, cudaEvent_t ev_fin,
                  int commit) {
    const int sms = a.sms;
    const int gw = 8 * sms, tpb = 256;
    const int sg = scan_grid(a.cap, sms);
    LocalView V{a.visited, a.U_off, a.U_col, a.row_start, a.deg, a.col};
    int nl = 0;
    pdl_launch(k_loc_check_rows, dim3(1), dim3(32), 0, s, a.ctl, a.cap);
    if (ev_tri) record_stage(ev_tri, s);
    pdl_launch(k_loc_owner, dim3(gw), dim3(tpb), 0, s, a.ctl, a.wlist, V, a.own);
    nl += 2;
    // changed pairs: common neighbours (4-cliques, triangles) and 4-cycle tasks
    pdl_launch(k_loc_pair_cost, dim3(gw), dim3(tpb), 0, s, a.ctl, V, a.srcA, a.dstA, a.srcD, a.dstD, a.pcost, a.ccnt,
               a.walk);
    nl++;
    nl += scan_i32_to_i64(a.pcost, a.ppre, &a.ctl->l_len[1], 0, a.bsum, sg, &a.ctl->l_tot[1], s);
    nl += scan_i32_to_i64(a.ccnt, a.cpre, &a.ctl->l_len[1], 0, a.bsum, sg, &a.ctl->l_tot[3], s);
    pdl_launch(k_loc_check_pairs, dim3(1), dim3(32), 0, s, a.ctl, a.cap);
    pdl_launch(k_loc_common, dim3(gw), dim3(tpb), 0, s, a.ctl, V, a.srcA, a.dstA, a.srcD, a.dstD, a.ppre, a.rec);
    nl += 2;
    if (a.T2) {
        // maintained triangle sums: intersect only the edges whose t changes
        pdl_launch(k_zero_u64, dim3(gw), dim3(tpb), 0, s, (unsigned long long*)a.dcnt, &a.ctl->l_len[0]);
        pdl_launch(k_loc_tri_delta, dim3(gw), dim3(tpb), 0, s, a.ctl, V, a.srcA, a.dstA, a.srcD, a.dstD, a.ppre, a.rec,
                   a.dcnt,
                                           a.dtri2, a.visited2, a.wlist_w);
        pdl_launch(k_loc_dcost, dim3(gw), dim3(tpb), 0, s, a.ctl, V, a.own, a.dcnt, a.cost);
        nl += 3;
        nl += scan_i32_to_i64(a.cost, a.pre, &a.ctl->l_len[0], 0, a.bsum, sg, &a.ctl->l_tot[0], s);
        pdl_launch(k_loc_tri, dim3(staged_grid(0, sms)), dim3(LC4_THREADS), LC4_SMEM, s, a.ctl, V, a.pre, a.own,
                   a.tpack);
        pdl_launch(k_loc_eterms, dim3(gw), dim3(tpb), 0, s, a.ctl, V, a.own, a.tpack, a.dcnt, a.da, a.db);
        pdl_launch(k_loc_vterms, dim3(gw), dim3(tpb), 0, s, a.ctl, a.wlist, V, a.T2, a.dtri2, a.da, a.db, commit);
        nl += 3;
    } else {
        // triangles of every edge at V_X, then their terms
        pdl_launch(k_loc_tri_cost, dim3(gw), dim3(tpb), 0, s, a.ctl, V, a.own, a.cost);
        nl++;
        nl += scan_i32_to_i64(a.cost, a.pre, &a.ctl->l_len[0], 0, a.bsum, sg, &a.ctl->l_tot[0], s);
        pdl_launch(k_loc_tri, dim3(staged_grid(0, sms)), dim3(LC4_THREADS), LC4_SMEM, s, a.ctl, V, a.pre, a.own,
                   a.tpack);
        pdl_launch(k_loc_terms, dim3(gw), dim3(tpb), 0, s, a.ctl, a.wlist, V, a.own, a.tpack, a.da, a.db);
        nl += 2;
    }
    if (ev_sub) record_stage(ev_sub, s);
    pdl_launch(k_loc_k4_cost, dim3(gw), dim3(tpb), 0, s, a.ctl, V, a.srcA, a.dstA, a.srcD, a.dstD, a.ppre, a.rec,
               a.kcost);
    nl++;
    nl += scan_i32_to_i64(a.kcost, a.kpre, &a.ctl->l_len[2], 0, a.bsum, sg, &a.ctl->l_tot[2], s);
    pdl_launch(k_loc_k4, dim3(gw), dim3(tpb), 0, s, a.ctl, V, a.srcA, a.dstA, a.srcD, a.dstD, a.ppre, a.rec, a.kpre);
    // the triangle probe offsets are free again: the 4-cycle tasks reuse them
    pdl_launch(k_loc_c4_tasks, dim3(gw), dim3(tpb), 0, s, a.ctl, V, a.srcA, a.dstA, a.srcD, a.dstD, a.cpre, a.walk,
               a.tpair, a.own,
                                      a.cost);
    nl += 2;
    nl += scan_i32_to_i64(a.cost, a.pre, &a.ctl->l_len[3], 0, a.bsum, sg, &a.ctl->l_tot[4], s);
    pdl_launch(k_loc_c4, dim3(staged_grid(1, sms)), dim3(LC4_THREADS), LC4_SMEM, s, a.ctl, V, a.srcA, a.dstA, a.srcD,
               a.dstD, a.walk, a.tpair, a.own, a.pre, a.cpre);
    nl++;
    if (ev_fin) record_stage(ev_fin, s);
    pdl_launch(k_finalize_local, dim3(1), dim3(32), 0, s, a.ctl, commit);
    nl++;
    return nl;
}

}  // namespace gcx
