// gc_region.cu -- the region of change (step a1) and the flagged region
// union graph (step a2).
//
// Region.  W is every vertex within k hops of a batch endpoint (Sec. 4.2:
// a 4-vertex graphlet has diameter at most 3; Algorithm 2 takes the k-hop
// neighbourhood of each changed pair).  The walk starts from all endpoints at
// once, level by level, over a vertex bitmap; each level appends the newly
// reached vertices to the region list, so level L occupies
// wlist[lvl[L-1] .. lvl[L]).  Every inserted or deleted pair joins two
// depth-0 vertices, so walking G alone reaches exactly what walking G u A does.
//
// Union graph.  Row u of U lists N(u) n W plus the insertions A_u, sorted by
// id, each entry tagged FLAG_A / FLAG_B (membership in G_a / G_b).  d_a(u)
// and d_b(u) are the degrees inside G_a and G_b (region-induced, as the
// counts of Algorithm 2 are taken in those graphs), and split(u) is the
// first position whose id exceeds u: the out-list N+(u).
#include "gc_internal.cuh"
#include "gc_kernels.cuh"

namespace gcx {

__device__ __forceinline__ bool in_region(const uint32_t* visited, int32_t v) {
    return (visited[v >> 5] >> (v & 31)) & 1u;
}

// mark v; if it was unmarked, append it to the region list (warp-aggregated)
__device__ __forceinline__ void visit_append(bool want, int32_t v, uint32_t* visited, int32_t* wlist, Ctl* c) {
    bool fresh = false;
    if (want) {
        uint32_t bit = 1u << (v & 31);
        if (!(visited[v >> 5] & bit)) fresh = !(atomicOr(&visited[v >> 5], bit) & bit);
    }
    unsigned m = __ballot_sync(FULL, fresh);
    if (m) {
        int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(&c->nW, __popc(m));
        base = __shfl_sync(FULL, base, leader);
        if (fresh) wlist[base + __popc(m & lanemask_lt())] = v;
    }
}

__global__ void k_bfs_sources(Ctl* c, const int32_t* __restrict__ srcA, const int32_t* __restrict__ srcD,
                              uint32_t* __restrict__ visited, int32_t* __restrict__ wlist) {
    pdl_enter();
    if (c->err) return;
    long long na = c->nA2, nd = c->nD2, tot = na + nd;
    long long stride = (long long)gridDim.x * blockDim.x;
    long long start = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    // the loop bound is warp-uniform so the ballot in visit_append is safe
    long long tot_r = (tot + 31) & ~31ll;
    for (long long i = start; i < tot_r; i += stride) {
        bool ok = i < tot;
        int32_t v = ok ? (i < na ? srcA[i] : srcD[i - na]) : 0;
        visit_append(ok, v, visited, wlist, c);
    }
}

__global__ void k_level_mark(Ctl* c, int L) { pdl_enter(); c->lvl[L] = c->nW; }

// The two-batch form's whole-graph pass: after the batch endpoints (level
// 0), every other vertex joins the region, so W = V and the counts of G_a and
// G_b are those of the whole graph after and before the batch.  An inactive
// batch (a halted run) keeps its empty region.
__global__ void k_region_rest(Ctl* c, int n, uint32_t* __restrict__ visited, int32_t* __restrict__ wlist) {
    pdl_enter();
    if (c->err || !c->active) return;
    const long long n_r = ((long long)n + 31) & ~31ll;  // warp-uniform bound for the ballot
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n_r;
         v += (long long)gridDim.x * blockDim.x)
        visit_append(v < n, (int32_t)(v < n ? v : 0), visited, wlist, c);
}

__global__ void k_bfs_expand(Ctl* c, int L, const long long* __restrict__ row_start, const int32_t* __restrict__ deg,
                             const int32_t* __restrict__ col, uint32_t* __restrict__ visited,
                             int32_t* __restrict__ wlist) {
    pdl_enter();
    if (c->err) return;
    int fb = L >= 2 ? c->lvl[L - 2] : 0;
    int fe = c->lvl[L - 1];
    int lane = threadIdx.x & 31;
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = fb + warp; i < fe; i += nwarps) {
        int32_t x = wlist[i];
        const int32_t* row = col + row_start[x];
        int d = deg[x];
        for (int b = 0; b < d; b += 32) {
            bool ok = b + lane < d;
            int32_t y = ok ? row[b + lane] : 0;
            visit_append(ok, y, visited, wlist, c);
        }
    }
}

// static count: W = V
__global__ void k_region_all(Ctl* c, int n, int32_t* __restrict__ wlist) {
    pdl_enter();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) wlist[i] = i;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->nW = n;
        for (int L = 0; L < MAX_HOPS + 2; L++) c->lvl[L] = n;
    }
}

__global__ void k_u_count(const Ctl* c, const int32_t* __restrict__ wlist, const uint32_t* __restrict__ visited,
                          const long long* __restrict__ row_start, const int32_t* __restrict__ deg,
                          const int32_t* __restrict__ col, const int2* __restrict__ segA,
                          int32_t* __restrict__ U_deg, int all) {
    pdl_enter();
    int nW = c->nW;
    int lane = threadIdx.x & 31;
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < nW; i += nwarps) {
        int32_t u = wlist[i];
        if (all) {  // the full row and the insertions
            if (lane == 0) U_deg[u] = deg[u] + (segA[u].y - segA[u].x);
            continue;
        }
        const int32_t* row = col + row_start[u];
        int d = deg[u], cnt = 0;
        for (int b = 0; b < d; b += 32) {
            bool ok = b + lane < d && (all || in_region(visited, row[b + lane]));
            cnt += __popc(__ballot_sync(FULL, ok));
        }
        if (lane == 0) {
            int2 a = segA[u];
            U_deg[u] = cnt + (a.y - a.x);
        }
    }
}

__global__ void k_u_fill(const Ctl* c, const int32_t* __restrict__ wlist, const uint32_t* __restrict__ visited,
                         const long long* __restrict__ row_start, const int32_t* __restrict__ deg,
                         const int32_t* __restrict__ col, const int2* __restrict__ segA,
                         const int2* __restrict__ segD, const int32_t* __restrict__ dstA,
                         const int32_t* __restrict__ dstD, const long long* __restrict__ U_off,
                         uint32_t* __restrict__ U_col, int32_t* __restrict__ U_split, int32_t* __restrict__ da,
                         int32_t* __restrict__ db, int all) {
    pdl_enter();
    int nW = c->nW;
    int lane = threadIdx.x & 31;
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < nW; i += nwarps) {
        int32_t u = wlist[i];
        int2 a = segA[u], d = segD[u];
        const int32_t* dl = dstD + d.x;
        long long nd = d.y - d.x, na = a.y - a.x;
        uint32_t* out = U_col + U_off[u];
        long long len = warp_merge_row(
            col + row_start[u], deg[u], dstA + a.x, na, out, FLAG_A,
            [&](int32_t v) { return all || in_region(visited, v); },
            [&](int32_t v) { return FLAG_B | ((nd == 0 || !sorted_contains(dl, nd, v)) ? FLAG_A : 0u); });
        __syncwarp();
        if (lane == 0) {
            U_split[u] = (int32_t)lower_bound_id(out, len, (uint32_t)u);
            da[u] = (int32_t)(len - nd);
            db[u] = (int32_t)(len - na);
        }
    }
}

// Twin pass (two independent batches, W = V): row u of U is N(u) plus the
// insertions of either batch; the kept entries carry the batches' mask in
// their two low bits (dst << 2 | mask, one entry per vertex pair, sorted).
// A G entry loses FLAG_A (FLAG_B) if the first (second) batch deletes it; an
// insertion has FLAG_A (FLAG_B) if the first (second) batch makes it.  Every
// entry is placed by binary searches: a row element after the insertions
// below it, an insertion after the row elements below it.
__global__ void k_u_count_twin(const Ctl* c, const int32_t* __restrict__ wlist, const int32_t* __restrict__ deg,
                               const int2* __restrict__ segA, int32_t* __restrict__ U_deg) {
    pdl_enter();
    const int nW = c->nW;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nW; i += gridDim.x * blockDim.x) {
        const int32_t u = wlist[i];
        U_deg[u] = deg[u] + (segA[u].y - segA[u].x);
    }
}

__global__ void k_u_fill_twin(const Ctl* c, const int32_t* __restrict__ wlist, const long long* __restrict__ row_start,
                              const int32_t* __restrict__ deg, const int32_t* __restrict__ col,
                              const int2* __restrict__ segA, const int2* __restrict__ segD,
                              const int32_t* __restrict__ dstA, const int32_t* __restrict__ dstD,
                              const long long* __restrict__ U_off, uint32_t* __restrict__ U_col,
                              int32_t* __restrict__ U_split, int32_t* __restrict__ da, int32_t* __restrict__ db) {
    pdl_enter();
    const int nW = c->nW;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < nW; i += nwarps) {
        const int32_t u = wlist[i];
        const int2 a = segA[u], d = segD[u];
        const int32_t* A = dstA + a.x;
        const int32_t* D = dstD + d.x;
        const long long na = a.y - a.x, nd = d.y - d.x;
        const int32_t* row = col + row_start[u];
        const int du = deg[u];
        uint32_t* out = U_col + U_off[u];
        for (int p = lane; p < du; p += 32) {
            const int32_t v = row[p];
            uint32_t fl = FLAG_A | FLAG_B;
            if (nd) {
                const long long q = lower_bound_i32(D, nd, v << 2);
                if (q < nd && (D[q] >> 2) == v) {
                    if (D[q] & 1) fl &= ~FLAG_A;
                    if (D[q] & 2) fl &= ~FLAG_B;
                }
            }
            out[p + (na ? lower_bound_i32(A, na, v << 2) : 0)] = (uint32_t)v | fl;
        }
        int cA = 0, cB = 0;  // insertions into G_a / G_b minus deletions from them
        for (long long q = lane; q < na; q += 32) {
            const int32_t x = A[q] >> 2, m = A[q] & 3;
            out[q + lower_bound_i32(row, du, x)] = (uint32_t)x | ((m & 1) ? FLAG_A : 0u) | ((m & 2) ? FLAG_B : 0u);
            cA += (m & 1) ? 1 : 0;
            cB += (m & 2) ? 1 : 0;
        }
        for (long long q = lane; q < nd; q += 32) {
            cA -= (D[q] & 1) ? 1 : 0;
            cB -= (D[q] & 2) ? 1 : 0;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cA += __shfl_xor_sync(FULL, cA, o);
            cB += __shfl_xor_sync(FULL, cB, o);
        }
        __syncwarp();
        if (lane == 0) {
            U_split[u] = (int32_t)(lower_bound_i32(row, du, u + 1) + (na ? lower_bound_i32(A, na, (u + 1) << 2) : 0));
            da[u] = du + cA;
            db[u] = du + cB;
        }
    }
}

// Union rows over the full adjacency (the edge-local path): a block per
// vertex, every entry placed by binary searches (hub rows spread over the
// block).  D entries stay with FLAG_B only, A entries get FLAG_A only.
__global__ void k_u_fill_all(const Ctl* c, const int32_t* __restrict__ wlist, const long long* __restrict__ row_start,
                             const int32_t* __restrict__ deg, const int32_t* __restrict__ col,
                             const int2* __restrict__ segA, const int2* __restrict__ segD,
                             const int32_t* __restrict__ dstA, const int32_t* __restrict__ dstD,
                             const long long* __restrict__ U_off, uint32_t* __restrict__ U_col,
                             int32_t* __restrict__ U_split, int32_t* __restrict__ da, int32_t* __restrict__ db) {
    pdl_enter();
    const int nW = c->nW;
    for (int i = blockIdx.x; i < nW; i += gridDim.x) {
        const int32_t u = wlist[i];
        const int2 a = segA[u], d = segD[u];
        const long long na = a.y - a.x, nd = d.y - d.x;
        const int32_t* row = col + row_start[u];
        const long long len = block_merge_row(row, deg[u], dstA + a.x, na, dstD + d.x, nd, U_col + U_off[u], true,
                                              FLAG_A | FLAG_B, FLAG_A, FLAG_B);
        if (threadIdx.x == 0) {
            U_split[u] = (int32_t)(lower_bound_i32(row, deg[u], u + 1) + lower_bound_i32(dstA + a.x, na, u + 1));
            da[u] = (int32_t)(len - nd);
            db[u] = (int32_t)(len - na);
        }
    }
}

}  // namespace gcx
