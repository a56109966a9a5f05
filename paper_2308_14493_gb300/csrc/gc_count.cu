// gc_count.cu -- PGD-style counting over the flagged region union graph
// (steps a3..a7): per-edge triangles, 4-cliques, 4-cycles, the per-edge and
// per-vertex terms, and the closed forms that turn them into the six induced
// graphlet counts of G_a and G_b (Sec. 3 "PGD Algorithm"; Algorithm 2).
//
// Non-induced sums per graph X (d = degree in X, t_uv = |N(u) n N(v)|):
//   P  = sum_{uv} (d_u-1)(d_v-1) - t_uv        3-paths
//   S  = sum_v C(d_v,3)                        3-stars
//   TT = 1/2 sum_{uv} t_uv (d_u+d_v-4)         tailed triangles
//   D  = sum_{uv} C(t_uv,2)                    diamonds
//   K  = #4-cliques,  Q = #4-cycles (not necessarily induced)
// Induced counts invert the containment of each graphlet in the larger ones:
//   g6 = K, g5 = D-6K, g3 = Q-g5-3K, g4 = TT-4g5-12K,
//   g2 = S-g4-2g5-4K, g1 = P-2g4-4g3-6g5-12K.
//
// Orientation: an edge points from its lower to its higher internal id.
//  * each triangle u<v<w is listed once, from edge u->v, as w in N+(u) n N+(v),
//    and credited to its three edges (one 64-bit atomic each: G_a count in the
//    high word, G_b count in the low word);
//  * each 4-clique u<v<w<x is counted once, from triangle (u,v,w), as
//    x in N+(u) n N+(v) n N+(w);
//  * each 4-cycle is counted once at its highest vertex u: for every w < u,
//    c_w = #{v in N(u) n N(w), v < u}, and the cycle count is sum_w C(c_w,2).
// An edge set counts for G_a (G_b) only if all its entries carry FLAG_A
// (FLAG_B), so one walk serves both graphs.
#include "gc_internal.cuh"
#include "gc_kernels.cuh"

namespace gcx {

__global__ void k_reset_count(Ctl* c) {
    int t = threadIdx.x;
    if (t < 16) c->acc[t] = 0;
    if (t < 8) c->work[t] = 0;
}

__global__ void k_zero_u64(unsigned long long* __restrict__ a, const long long* d_len) {
    long long n = *d_len;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] = 0;
}

__device__ __forceinline__ unsigned long long flag_inc(uint32_t f) {
    return ((f & FLAG_A) ? (1ull << 32) : 0ull) | ((f & FLAG_B) ? 1ull : 0ull);
}

// One warp per region vertex u; each lane takes one out-edge u->v and merges
// N+(u) (after v) with N+(v).
__global__ void k_tri_k4(Ctl* c, const int32_t* __restrict__ wlist, const long long* __restrict__ U_off,
                         const uint32_t* __restrict__ U_col, const int32_t* __restrict__ U_split,
                         unsigned long long* __restrict__ tpack) {
    int nW = c->nW;
    int lane = threadIdx.x & 31;
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int nwarps = (gridDim.x * blockDim.x) >> 5;
    unsigned long long ka = 0, kb = 0;
    for (int wi = warp; wi < nW; wi += nwarps) {
        int32_t u = wlist[wi];
        long long ob = U_off[u] + U_split[u], oe = U_off[u + 1];
        for (long long e = ob + lane; e < oe; e += 32) {
            uint32_t fe = U_col[e];
            uint32_t v = vid(fe);
            long long vb = U_off[v] + U_split[v], ve = U_off[v + 1];
            long long i = e + 1, j = vb;
            while (i < oe && j < ve) {
                uint32_t ei = U_col[i], ej = U_col[j];
                uint32_t x = vid(ei), y = vid(ej);
                if (x < y) {
                    i++;
                } else if (x > y) {
                    j++;
                } else {
                    uint32_t f = fe & ei & ej;
                    unsigned long long inc = flag_inc(f);
                    if (inc) {
                        atomicAdd(&tpack[e], inc);
                        atomicAdd(&tpack[i], inc);
                        atomicAdd(&tpack[j], inc);
                        // 4-cliques through triangle (u, v, x): z in N+(u) n N+(v) n N+(x)
                        long long wb = U_off[x] + U_split[x], we = U_off[x + 1];
                        long long p = i + 1, q = j + 1, r = wb;
                        while (p < oe && q < ve && r < we) {
                            uint32_t ep = U_col[p], eq = U_col[q], er = U_col[r];
                            uint32_t a = vid(ep), b = vid(eq), cc = vid(er);
                            uint32_t mx = max(a, max(b, cc));
                            if (a == mx && b == mx && cc == mx) {
                                uint32_t g = f & ep & eq & er;
                                ka += (g & FLAG_A) ? 1 : 0;
                                kb += (g & FLAG_B) ? 1 : 0;
                                p++;
                                q++;
                                r++;
                            } else {
                                if (a < mx) p++;
                                if (b < mx) q++;
                                if (cc < mx) r++;
                            }
                        }
                    }
                    i++;
                    j++;
                }
            }
        }
    }
    ka = warp_sum_u64(ka);
    kb = warp_sum_u64(kb);
    if (lane == 0 && (ka | kb)) {
        atomicAdd(&c->acc[4], ka);
        atomicAdd(&c->acc[10], kb);
    }
}

// One block per pivot u (dynamic queue).  Each block owns a dense counter
// array cnt[0..n) in global memory, zero between pivots: pass 1 adds the
// wedges u-v-w (v < u, w < u), pass 2 walks the same wedges and takes each
// counter with an exchange, so every w is summed once and left at zero.
__global__ void __launch_bounds__(256) k_c4(Ctl* c, const int32_t* __restrict__ wlist,
                                            const long long* __restrict__ U_off, const uint32_t* __restrict__ U_col,
                                            const int32_t* __restrict__ U_split,
                                            unsigned long long* __restrict__ cnt_all, int n) {
    __shared__ int s_idx;
    __shared__ unsigned long long s_q[2][8];
    unsigned long long* cnt = cnt_all + (size_t)blockIdx.x * n;
    int nW = c->nW;
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    unsigned long long qa = 0, qb = 0, wedges = 0;
    for (;;) {
        if (threadIdx.x == 0) s_idx = (int)atomicAdd(&c->work[0], 1u);
        __syncthreads();
        int idx = s_idx;
        __syncthreads();
        if (idx >= nW) break;
        int32_t u = wlist[idx];
        long long rb = U_off[u], nlow = U_split[u];
        for (int pass = 0; pass < 2; pass++) {
            for (long long k = warp; k < nlow; k += nwarps) {
                uint32_t fv = U_col[rb + k];
                uint32_t v = vid(fv);
                long long vb = U_off[v];
                long long lenv = lower_bound_id(U_col + vb, U_off[v + 1] - vb, (uint32_t)u);
                if (pass == 0 && lane == 0) wedges += (unsigned long long)lenv;
                for (long long q = lane; q < lenv; q += 32) {
                    uint32_t fw = U_col[vb + q];
                    uint32_t w = vid(fw);
                    if (pass == 0) {
                        unsigned long long inc = flag_inc(fv & fw);
                        if (inc) atomicAdd(&cnt[w], inc);
                    } else {
                        unsigned long long cw = atomicExch(&cnt[w], 0ull);
                        if (cw) {
                            qa += choose2(cw >> 32);
                            qb += choose2(cw & 0xFFFFFFFFull);
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
    qa = warp_sum_u64(qa);
    qb = warp_sum_u64(qb);
    if (lane == 0 && wedges) atomicAdd(&c->acc[15], wedges);
    if (lane == 0) {
        s_q[0][warp] = qa;
        s_q[1][warp] = qb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long ta = 0, tb = 0;
        for (int w = 0; w < nwarps; w++) {
            ta += s_q[0][w];
            tb += s_q[1][w];
        }
        if (ta | tb) {
            atomicAdd(&c->acc[5], ta);
            atomicAdd(&c->acc[11], tb);
        }
    }
}

__global__ void k_edge_terms(Ctl* c, const int32_t* __restrict__ wlist, const long long* __restrict__ U_off,
                             const uint32_t* __restrict__ U_col, const int32_t* __restrict__ U_split,
                             const unsigned long long* __restrict__ tpack, const int32_t* __restrict__ da,
                             const int32_t* __restrict__ db) {
    int nW = c->nW;
    int lane = threadIdx.x & 31;
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int nwarps = (gridDim.x * blockDim.x) >> 5;
    unsigned long long P[2] = {0, 0}, S[2] = {0, 0}, T[2] = {0, 0}, D[2] = {0, 0}, E[2] = {0, 0}, work = 0;
    for (int wi = warp; wi < nW; wi += nwarps) {
        int32_t u = wlist[wi];
        long long dau = da[u], dbu = db[u];
        if (lane == 0) {
            S[0] += choose3((unsigned long long)dau);
            S[1] += choose3((unsigned long long)dbu);
        }
        long long ob = U_off[u] + U_split[u], oe = U_off[u + 1];
        for (long long e = ob + lane; e < oe; e += 32) {
            uint32_t fe = U_col[e];
            uint32_t v = vid(fe);
            unsigned long long t = tpack[e];
            work += (unsigned long long)((oe - ob) + (U_off[v + 1] - U_off[v] - U_split[v]));
            if (fe & FLAG_A) {
                long long dv = da[v], tt = (long long)(t >> 32);
                P[0] += (unsigned long long)((dau - 1) * (dv - 1) - tt);
                T[0] += (unsigned long long)(tt * (dau + dv - 4));
                D[0] += choose2((unsigned long long)tt);
                E[0] += 1;
            }
            if (fe & FLAG_B) {
                long long dv = db[v], tt = (long long)(t & 0xFFFFFFFFull);
                P[1] += (unsigned long long)((dbu - 1) * (dv - 1) - tt);
                T[1] += (unsigned long long)(tt * (dbu + dv - 4));
                D[1] += choose2((unsigned long long)tt);
                E[1] += 1;
            }
        }
    }
#pragma unroll
    for (int g = 0; g < 2; g++) {
        P[g] = warp_sum_u64(P[g]);
        S[g] = warp_sum_u64(S[g]);
        T[g] = warp_sum_u64(T[g]);
        D[g] = warp_sum_u64(D[g]);
        E[g] = warp_sum_u64(E[g]);
    }
    if (lane == 0) {
        for (int g = 0; g < 2; g++) {
            int o = 6 * g;
            if (P[g]) atomicAdd(&c->acc[o + 0], P[g]);
            if (S[g]) atomicAdd(&c->acc[o + 1], S[g]);
            if (T[g]) atomicAdd(&c->acc[o + 2], T[g]);
            if (D[g]) atomicAdd(&c->acc[o + 3], D[g]);
            if (E[g]) atomicAdd(&c->acc[12 + g], E[g]);
        }
    }
    work = warp_sum_u64(work);
    if (lane == 0 && work) atomicAdd(&c->acc[14], work);
}

// mode 0: batch (F += C_a - C_b unless the batch was rejected); 1: static
__global__ void k_finalize(Ctl* c, int mode) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int g = 0; g < 2; g++) {
        const unsigned long long* s = c->acc + 6 * g;
        long long P = (long long)s[0], S = (long long)s[1], TT = (long long)(s[2] / 2), D = (long long)s[3],
                  K = (long long)s[4], Q = (long long)s[5];
        long long g6 = K;
        long long g5 = D - 6 * K;
        long long g3 = Q - g5 - 3 * K;
        long long g4 = TT - 4 * g5 - 12 * K;
        long long g2 = S - g4 - 2 * g5 - 4 * K;
        long long g1 = P - 2 * g4 - 4 * g3 - 6 * g5 - 12 * K;
        long long* C = g == 0 ? c->Ca : c->Cb;
        long long* sm = g == 0 ? c->sa : c->sb;
        C[0] = g1; C[1] = g2; C[2] = g3; C[3] = g4; C[4] = g5; C[5] = g6;
        sm[0] = P; sm[1] = S; sm[2] = TT; sm[3] = D; sm[4] = K; sm[5] = Q;
    }
    if (mode == 0 && c->err == 0)
        for (int i = 0; i < 6; i++) c->F[i] += (unsigned long long)(c->Ca[i] - c->Cb[i]);
}

}  // namespace gcx
