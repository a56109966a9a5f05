// gc_batch.cu -- batch normalisation (step a0), the commit G <- G \ D u A
// (step a8, Algorithm 2), the slack-padded adjacency layout, and the
// device-side part of opening a graph.
//
// Batch keys.  Every pair (u, v) of a batch becomes two directed keys
//   (src << (S+1)) | (dst << 1) | op,  op = 0 insert, 1 delete,
// over internal ids, S = bits of n-1.  After sorting, the keys of one
// unordered pair sit together in both directions, so repeats, pairs present
// in both A and D (dropped from both, Sec. 5) and no-ops (insert of a present
// edge, delete of an absent one) are decided per run, identically for both
// directions.  The kept entries, still sorted, form per-vertex lists A_u and
// D_u, reached through segA / segD.
#include "gc_internal.cuh"
#include "gc_kernels.cuh"

namespace gcx {

__global__ void k_batch_keys(Ctl* c, const int32_t* __restrict__ perm, int n, int S, uint64_t* __restrict__ keys) {
    pdl_enter();
    long long ni = c->n_ins, nd = c->n_del, tot = ni + nd;
    const int32_t* ins = c->pairs_ins + 2 * c->ins_off;
    const int32_t* del = c->pairs_del + 2 * c->del_off;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        const int32_t* p = i < ni ? ins + 2 * i : del + 2 * (i - ni);
        uint64_t op = i < ni ? 0 : 1;
        int32_t x = p[0], y = p[1];
        if (x < 0 || y < 0 || x >= n || y >= n || x == y) {
            atomicExch(&c->err, -1);  // GC_EINVAL; the batch is then not applied
            keys[2 * i] = keys[2 * i + 1] = ~0ull;
            continue;
        }
        uint64_t a = (uint64_t)perm[x], b = (uint64_t)perm[y];
        keys[2 * i] = (a << (S + 1)) | (b << 1) | op;
        keys[2 * i + 1] = (b << (S + 1)) | (a << 1) | op;
    }
}

// ---- twin pass: two independent batches counted in one pass ---------------
// Both batches' pairs are keyed together, each key carrying its batch's tag:
// key = (a << (S + 2)) | (b << 2) | (tag << 1) | op.  Per vertex pair the
// group of keys decides, for each batch alone, what Algorithm 2's
// normalisation decides (repeats collapse, a pair in both A and D of one
// batch drops, no-ops drop); the kept entry of the pair carries the mask of
// the batches that insert (or delete) it, in its two low bits:
// dst = (b << 2) | mask.  A pair cannot be kept as an insertion by one batch
// and as a deletion by the other (one needs it absent, the other present).
__global__ void k_batch_keys_twin(Ctl* c, const int32_t* __restrict__ perm, int n, int S,
                                  uint64_t* __restrict__ keys) {
    pdl_enter();
    const long long n0 = c->tw_n[0], n1 = c->tw_n[1], n2 = c->tw_n[2], n3 = c->tw_n[3];
    const long long tot = n0 + n1 + n2 + n3;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        int seg = 0;
        long long j = i;
        if (j >= n0) { j -= n0; seg = 1;
            if (j >= n1) { j -= n1; seg = 2;
                if (j >= n2) { j -= n2; seg = 3; } } }
        const int32_t* base = (seg & 1) ? c->pairs_del : c->pairs_ins;
        const int32_t* p = base + 2 * (c->tw_off[seg] + j);
        const uint64_t op = seg & 1, tag = seg >> 1;
        const int32_t x = p[0], y = p[1];
        if (x < 0 || y < 0 || x >= n || y >= n || x == y) {
            atomicExch(&c->err, -1);  // checked on the host before a twin pass; never applied
            keys[2 * i] = keys[2 * i + 1] = ~0ull;
            continue;
        }
        const uint64_t a = (uint64_t)perm[x], b = (uint64_t)perm[y];
        keys[2 * i] = (a << (S + 2)) | (b << 2) | (tag << 1) | op;
        keys[2 * i + 1] = (b << (S + 2)) | (a << 2) | (tag << 1) | op;
    }
}

// what the group of keys of one vertex pair starting at i keeps, per batch:
// bit t of *ins / *del: batch t inserts / deletes it (before the existence
// test)
__device__ __forceinline__ void twin_group(const uint64_t* keys, long long i, long long nk, uint64_t pair, int* ins,
                                           int* del) {
    int hi[2] = {0, 0}, hd[2] = {0, 0};
    for (long long j = i; j < nk && (keys[j] >> 2) == pair; j++) {
        const int t = (int)((keys[j] >> 1) & 1);
        if (keys[j] & 1) hd[t] = 1;
        else hi[t] = 1;
    }
    *ins = (hi[0] && !hd[0] ? 1 : 0) | (hi[1] && !hd[1] ? 2 : 0);
    *del = (hd[0] && !hi[0] ? 1 : 0) | (hd[1] && !hi[1] ? 2 : 0);
}

__global__ void k_batch_decide_twin(const uint64_t* __restrict__ keys, Ctl* c, int S,
                                    const long long* __restrict__ row_start, const int32_t* __restrict__ deg,
                                    const int32_t* __restrict__ col, int32_t* __restrict__ keepA,
                                    int32_t* __restrict__ keepD) {
    pdl_enter();
    const long long nk = c->nkeys;
    const uint64_t idmask = (1ull << S) - 1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nk;
         i += (long long)gridDim.x * blockDim.x) {
        const uint64_t pair = keys[i] >> 2;
        int ka = 0, kd = 0;
        if (keys[i] != ~0ull && (i == 0 || (keys[i - 1] >> 2) != pair)) {
            int ins, del;
            twin_group(keys, i, nk, pair, &ins, &del);
            const int32_t src = (int32_t)(pair >> S), dst = (int32_t)(pair & idmask);
            const bool exists = sorted_contains(col + row_start[src], deg[src], dst);
            ka = (!exists && ins) ? 1 : 0;
            kd = (exists && del) ? 1 : 0;
        }
        keepA[i] = ka;
        keepD[i] = kd;
    }
}

__global__ void k_batch_compact_twin(const uint64_t* __restrict__ keys, const Ctl* c, int S,
                                     const int32_t* __restrict__ keepA, const int32_t* __restrict__ keepD,
                                     const long long* __restrict__ posA, const long long* __restrict__ posD,
                                     int32_t* __restrict__ srcA, int32_t* __restrict__ dstA,
                                     int32_t* __restrict__ srcD, int32_t* __restrict__ dstD) {
    pdl_enter();
    const long long nk = c->nkeys;
    const uint64_t idmask = (1ull << S) - 1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nk;
         i += (long long)gridDim.x * blockDim.x) {
        if (!keepA[i] && !keepD[i]) continue;
        const uint64_t pair = keys[i] >> 2;
        const int32_t src = (int32_t)(pair >> S), dst = (int32_t)(pair & idmask);
        int ins, del;
        twin_group(keys, i, nk, pair, &ins, &del);
        if (keepA[i]) {
            srcA[posA[i]] = src;
            dstA[posA[i]] = (dst << 2) | ins;
        }
        if (keepD[i]) {
            srcD[posD[i]] = src;
            dstD[posD[i]] = (dst << 2) | del;
        }
    }
}

// keep[i]: 1 = insert entry, 2 = delete entry, 0 = dropped / not a run head
__global__ void k_batch_decide(const uint64_t* __restrict__ keys, Ctl* c, int S,
                               const long long* __restrict__ row_start, const int32_t* __restrict__ deg,
                               const int32_t* __restrict__ col, int32_t* __restrict__ keepA,
                               int32_t* __restrict__ keepD) {
    pdl_enter();
    long long nk = c->nkeys;
    const uint64_t idmask = (1ull << S) - 1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nk;
         i += (long long)gridDim.x * blockDim.x) {
        uint64_t pair = keys[i] >> 1;
        int ka = 0, kd = 0;
        if (keys[i] != ~0ull && (i == 0 || (keys[i - 1] >> 1) != pair)) {
            bool has_ins = false, has_del = false;
            long long j = i;
            while (j < nk && (keys[j] >> 1) == pair) {
                if (keys[j] & 1) has_del = true;
                else has_ins = true;
                j++;
            }
            int32_t src = (int32_t)(pair >> S), dst = (int32_t)(pair & idmask);
            unsigned long long rep = (unsigned long long)(j - i) - (has_ins ? 1 : 0) - (has_del ? 1 : 0);
            if (rep) atomicAdd(&c->st[0], rep);
            if (has_ins && has_del) {
                atomicAdd(&c->st[1], 1ull);
            } else {
                bool exists = sorted_contains(col + row_start[src], deg[src], dst);
                if (has_ins) {
                    if (exists) atomicAdd(&c->st[2], 1ull);
                    else ka = 1;
                } else {
                    if (exists) kd = 1;
                    else atomicAdd(&c->st[3], 1ull);
                }
            }
        }
        keepA[i] = ka;
        keepD[i] = kd;
    }
}

__global__ void k_batch_compact(const uint64_t* __restrict__ keys, const Ctl* c, int S,
                                const int32_t* __restrict__ keepA, const int32_t* __restrict__ keepD,
                                const long long* __restrict__ posA, const long long* __restrict__ posD,
                                int32_t* __restrict__ srcA, int32_t* __restrict__ dstA,
                                int32_t* __restrict__ srcD, int32_t* __restrict__ dstD) {
    pdl_enter();
    long long nk = c->nkeys;
    const uint64_t idmask = (1ull << S) - 1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nk;
         i += (long long)gridDim.x * blockDim.x) {
        uint64_t pair = keys[i] >> 1;
        int32_t src = (int32_t)(pair >> S), dst = (int32_t)(pair & idmask);
        if (keepA[i]) {
            srcA[posA[i]] = src;
            dstA[posA[i]] = dst;
        }
        if (keepD[i]) {
            srcD[posD[i]] = src;
            dstD[posD[i]] = dst;
        }
    }
}

// seg[src] = [first, last+1) of src's run in the kept, sorted entry list
__global__ void k_batch_segments(const int32_t* __restrict__ src, const long long* d_len, int2* __restrict__ seg) {
    pdl_enter();
    long long n = *d_len;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x) {
        int32_t s = src[j];
        if (j == 0 || src[j - 1] != s) {
            long long e = j + 1;
            while (e < n && src[e] == s) e++;
            seg[s] = make_int2((int)j, (int)e);
        }
    }
}

__global__ void k_batch_clear_segments(const int32_t* __restrict__ src, const long long* d_len,
                                       int2* __restrict__ seg) {
    pdl_enter();
    long long n = *d_len;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x)
        seg[src[j]] = make_int2(0, 0);
}

// ---- commit ---------------------------------------------------------------
// The batch endpoints are exactly the level-0 entries of the region list.
__global__ void k_commit_plan(Ctl* c, const int32_t* __restrict__ wlist, const int2* __restrict__ segA,
                              const int2* __restrict__ segD, const int32_t* __restrict__ deg,
                              const int32_t* __restrict__ cap, const long long* __restrict__ row_start,
                              long long col_capacity, float slack, long long* __restrict__ plan_dst,
                              int32_t* __restrict__ plan_cap, int32_t* __restrict__ plan_deg,
                              long long* __restrict__ plan_scr) {
    pdl_enter();
    if (c->err || c->lovf) return;
    int ns = c->lvl[0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += gridDim.x * blockDim.x) {
        int32_t u = wlist[i];
        int2 a = segA[u], d = segD[u];
        int nd = deg[u] + (a.y - a.x) - (d.y - d.x);
        plan_deg[i] = nd;
        plan_scr[i] = (long long)atomicAdd(&c->scratch_tail, (unsigned long long)nd);
        if (nd > cap[u]) {
            int extra = (int)ceilf(slack * (float)nd);
            if (extra < 4) extra = 4;
            int ncap = nd + extra;
            unsigned long long at = atomicAdd(&c->pool_tail, (unsigned long long)ncap);
            if (at + (unsigned long long)ncap > (unsigned long long)col_capacity && atomicExch(&c->overflow, 1) == 0) {
                // no row is written; later batches of a run wait until the
                // host has grown the pool and finished this commit
                c->halt = 1;
                c->pend_ns = ns;
                c->pend_nA2 = c->nA2;
                c->pend_nD2 = c->nD2;
            }
            plan_dst[i] = (long long)at;
            plan_cap[i] = ncap;
        } else {
            plan_dst[i] = row_start[u];
            plan_cap[i] = cap[u];
        }
    }
}

// row \ D_u u A_u of every touched vertex into the scratch: a warp per
// short row, a block per long one (every entry placed by binary searches,
// so a hub row spreads over the block).
constexpr long long LONG_ROW = 4096;

__global__ void k_commit_merge(const Ctl* c, const int32_t* __restrict__ wlist, const int2* __restrict__ segA,
                               const int2* __restrict__ segD, const int32_t* __restrict__ dstA,
                               const int32_t* __restrict__ dstD, const int32_t* __restrict__ deg,
                               const long long* __restrict__ row_start, const int32_t* __restrict__ col,
                               const long long* __restrict__ plan_scr, uint32_t* __restrict__ scratch) {
    pdl_enter();
    if (c->err || c->overflow || c->lovf) return;
    const int ns = c->lvl[0];
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < ns; i += nwarps) {
        const int32_t u = wlist[i];
        const int2 a = segA[u], d = segD[u];
        if ((long long)deg[u] + (a.y - a.x) > LONG_ROW) continue;
        const int32_t* dl = dstD + d.x;
        const long long nd = d.y - d.x;
        warp_merge_row(col + row_start[u], deg[u], dstA + a.x, a.y - a.x, scratch + plan_scr[i], 0u,
                       [&](int32_t v) { return nd == 0 || !sorted_contains(dl, nd, v); },
                       [](int32_t) { return 0u; });
    }
    for (int i = blockIdx.x; i < ns; i += gridDim.x) {
        const int32_t u = wlist[i];
        const int2 a = segA[u], d = segD[u];
        if ((long long)deg[u] + (a.y - a.x) <= LONG_ROW) continue;
        block_merge_row(col + row_start[u], deg[u], dstA + a.x, a.y - a.x, dstD + d.x, d.y - d.x,
                        scratch + plan_scr[i], false, 0u, 0u, 0u);
    }
}

__global__ void k_commit_write(const Ctl* c, const int32_t* __restrict__ wlist, const long long* __restrict__ plan_dst,
                               const int32_t* __restrict__ plan_cap, const int32_t* __restrict__ plan_deg,
                               const long long* __restrict__ plan_scr, const uint32_t* __restrict__ scratch,
                               int32_t* __restrict__ deg, int32_t* __restrict__ cap,
                               long long* __restrict__ row_start, int32_t* __restrict__ col) {
    pdl_enter();
    if (c->err || c->overflow || c->lovf) return;
    const int ns = c->lvl[0];
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < ns; i += nwarps) {
        const int nd = plan_deg[i];
        if (nd > LONG_ROW) continue;
        const int32_t u = wlist[i];
        const long long dst = plan_dst[i], scr = plan_scr[i];
        for (int j = lane; j < nd; j += 32) col[dst + j] = (int32_t)scratch[scr + j];
        if (lane == 0) {
            deg[u] = nd;
            cap[u] = plan_cap[i];
            row_start[u] = dst;
        }
    }
    for (int i = blockIdx.x; i < ns; i += gridDim.x) {
        const int nd = plan_deg[i];
        if (nd <= LONG_ROW) continue;
        const int32_t u = wlist[i];
        const long long dst = plan_dst[i], scr = plan_scr[i];
        for (int j = threadIdx.x; j < nd; j += blockDim.x) col[dst + j] = (int32_t)scratch[scr + j];
        if (threadIdx.x == 0) {
            deg[u] = nd;
            cap[u] = plan_cap[i];
            row_start[u] = dst;
        }
    }
}

// ---- layout ---------------------------------------------------------------

__global__ void k_slack_caps(const int32_t* __restrict__ deg, int n, float slack, int32_t* __restrict__ cap) {
    pdl_enter();
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int d = deg[v];
        int extra = (int)ceilf(slack * (float)d);
        if (extra < 2) extra = 2;
        cap[v] = d + extra;
    }
}

__global__ void k_copy_rows(const int32_t* __restrict__ deg, int n, const long long* __restrict__ old_start,
                            const int32_t* __restrict__ old_col, const long long* __restrict__ new_start,
                            int32_t* __restrict__ new_col) {
    pdl_enter();
    int lane = threadIdx.x & 31;
    long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long v = warp; v < n; v += nwarps) {
        long long o = old_start[v], w = new_start[v];
        int d = deg[v];
        for (int j = lane; j < d; j += 32) new_col[w + j] = old_col[o + j];
    }
}

// ---- open -----------------------------------------------------------------

__global__ void k_degree_keys(const int32_t* __restrict__ rp, int n, int32_t* __restrict__ deg0,
                              uint64_t* __restrict__ keys) {
    pdl_enter();
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int d = rp[v + 1] - rp[v];
        deg0[v] = d;
        keys[v] = ((uint64_t)(uint32_t)d << 32) | (uint32_t)v;
    }
}

__global__ void k_perm_from_keys(const uint64_t* __restrict__ keys, int n, int32_t* __restrict__ perm,
                                 int32_t* __restrict__ iperm, const int32_t* __restrict__ deg0,
                                 int32_t* __restrict__ deg) {
    pdl_enter();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int32_t v = (int32_t)(keys[i] & 0xFFFFFFFFu);
        iperm[i] = v;
        perm[v] = i;
        deg[i] = deg0[v];
    }
}

__global__ void k_edge_keys(const int32_t* __restrict__ rp, const int32_t* __restrict__ col, int n,
                            const int32_t* __restrict__ perm, int S, uint64_t* __restrict__ keys,
                            int* __restrict__ bad) {
    pdl_enter();
    int lane = threadIdx.x & 31;
    long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long v = warp; v < n; v += nwarps) {
        uint64_t a = (uint64_t)perm[v];
        for (long long p = rp[v] + lane; p < rp[v + 1]; p += 32) {
            int32_t w = col[p];
            if (w < 0 || w >= n || w == v) {
                atomicExch(bad, 1);
                keys[p] = 0;
                continue;
            }
            keys[p] = (a << S) | (uint64_t)perm[w];
        }
    }
}

// After sorting: keys of row a are contiguous and sorted.  Rejects repeats
// and asymmetric entries; writes columns into the slack layout.
__global__ void k_fill_from_keys(const uint64_t* __restrict__ keys, long long m2, int n, int S,
                                 const long long* __restrict__ key_off, const long long* __restrict__ row_start,
                                 int32_t* __restrict__ col, int* __restrict__ bad) {
    pdl_enter();
    const uint64_t idmask = (1ull << S) - 1;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < m2;
         p += (long long)gridDim.x * blockDim.x) {
        uint64_t k = keys[p];
        long long a = (long long)(k >> S), b = (long long)(k & idmask);
        if (a >= n || b >= n) {
            atomicExch(bad, 1);
            continue;
        }
        long long j = p - key_off[a];
        if (j < 0 || j >= key_off[a + 1] - key_off[a]) {  // only after a rejected entry
            atomicExch(bad, 1);
            continue;
        }
        if (p > 0 && keys[p - 1] == k) atomicExch(bad, 2);
        // symmetric partner (b, a) must exist in row b
        long long lo = key_off[b], hi = key_off[b + 1];
        uint64_t want = ((uint64_t)b << S) | (uint64_t)a;
        while (lo < hi) {
            long long mid = (lo + hi) >> 1;
            if (keys[mid] < want) lo = mid + 1;
            else hi = mid;
        }
        if (lo >= key_off[b + 1] || keys[lo] != want) atomicExch(bad, 3);
        col[row_start[a] + j] = (int32_t)b;
    }
}

// ---- export ---------------------------------------------------------------

__global__ void k_export_rows(const int32_t* __restrict__ deg, int n, const long long* __restrict__ row_start,
                              const int32_t* __restrict__ col, const int32_t* __restrict__ perm,
                              const long long* __restrict__ out_off_ext, const int32_t* __restrict__ iperm,
                              int32_t* __restrict__ out_col) {
    pdl_enter();
    // warp per internal vertex i: external id x = iperm[i]; writes external
    // neighbour ids (unsorted; sorted on the host)
    int lane = threadIdx.x & 31;
    long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = warp; i < n; i += nwarps) {
        int32_t x = iperm[i];
        long long o = out_off_ext[x], s = row_start[i];
        int d = deg[i];
        for (int j = lane; j < d; j += 32) out_col[o + j] = iperm[col[s + j]];
    }
    (void)perm;
}

__global__ void k_ext_degrees(const int32_t* __restrict__ deg, const int32_t* __restrict__ iperm, int n,
                              int32_t* __restrict__ ext_deg) {
    pdl_enter();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) ext_deg[iperm[i]] = deg[i];
}

}  // namespace gcx
