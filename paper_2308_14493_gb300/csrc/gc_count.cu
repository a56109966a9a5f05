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
//
// Triangles and 4-cliques, root-centred.  For a root u with out-list
// X = N+(u) (k entries), every v = X[q] is probed: each entry y of N+(v)
// that is also in X (binary search in shared memory) closes the triangle
// (u, v, y), listed exactly once (u < v < y).  It sets bit p = pos(y) of the
// local row q, and credits its three edges: (u,v) and (u,y) in a per-root
// shared-memory accumulator, (v,y) by one 64-bit atomic.  The rows are the
// adjacency of N+(u) as bitmasks, so the 4-cliques through u are
// sum over bits p of row q of popcount(row_q & row_p).  G_a and G_b get one
// row set each.  Roots are binned by k: a warp (k <= 32), a block
// (k <= TRI_KM), or per-edge merging (larger k).
//
// 4-cycles, pivot-centred.  Each 4-cycle is counted once at its highest
// vertex u: for every w < u, c_w = #{v in N(u) n N(w): v < u}, and the
// pivot contributes sum_w C(c_w, 2).  Counters are incremented one wedge
// u-v-w at a time and the increment returns the old value c, so the pivot's
// sum is accumulated on the fly as sum of old values (C(c+1,2) - C(c,2) = c);
// no reduction pass is needed.  Pivots are binned by the wedge bound
// w~ = sum of the degrees of the lower neighbours: registers (w~ <= 32, equal
// endpoints grouped by __match_any_sync), a per-warp or per-block hash table
// in shared memory, or, for the heavy pivots, a cluster of CTAs sharing one
// dense counter array in global memory.
//
// An edge set counts for G_a (G_b) only if all its entries carry FLAG_A
// (FLAG_B), so one walk serves both graphs.
#include <cooperative_groups.h>

#include <algorithm>

#include "gc_internal.cuh"
#include "gc_kernels.cuh"

namespace cg = cooperative_groups;

namespace gcx {

__global__ void k_reset_count(Ctl* c) {
    pdl_enter();
    int t = threadIdx.x;
    if (t < NACC) c->acc[t] = 0;
    for (int i = t; i < NACC * ACC_STRIPES; i += blockDim.x) (&c->accs[0][0])[i] = 0;
    if (t < NWORK) c->work[t] = 0;
    if (t < NBINS) c->nbin[t] = 0;
    if (t == 0) c->maxdeg = 0;
}

__global__ void k_zero_u64(unsigned long long* __restrict__ a, const long long* d_len) {
    pdl_enter();
    long long n = *d_len;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] = 0;
}

__device__ __forceinline__ unsigned long long flag_inc(uint32_t f) {
    return ((f & FLAG_A) ? (1ull << 32) : 0ull) | ((f & FLAG_B) ? 1ull : 0ull);
}

// Add a warp's sum to accumulator `slot`: one atomic per warp, on one of
// ACC_STRIPES copies chosen by the warp (thousands of warps adding to one
// address would queue at a single L2 slice); k_finalize sums the copies.
__device__ __forceinline__ void acc_add_warp(Ctl* c, int slot, unsigned long long x) {
    if ((threadIdx.x & 31) == 0 && x) {
        const int stripe = (int)((blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) & (ACC_STRIPES - 1));
        atomicAdd(&c->accs[slot][stripe], x);
    }
}
__device__ __forceinline__ void acc_add(Ctl* c, int slot, unsigned long long x) {
    acc_add_warp(c, slot, warp_sum_u64(x));
}

// index of id y in the sorted entries s[0..k), or -1 (the first probes of
// all lanes hit the same entries, which shared memory broadcasts)
__device__ __forceinline__ int find_pos(const uint32_t* s, int k, uint32_t y) {
    int lo = 0, hi = k;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (vid(s[mid]) < y) lo = mid + 1;
        else hi = mid;
    }
    return (lo < k && vid(s[lo]) == y) ? lo : -1;
}

// largest q in [0, k) with pre[q] <= t (pre[0] = 0 <= t < pre[k])
__device__ __forceinline__ int find_seg(const int* pre, int k, int t) {
    int lo = 0, hi = k;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (pre[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

// ---- binning ---------------------------------------------------------------

// Wedge bound of every 4-cycle pivot: w~(u) = sum of the union-graph degrees
// of its lower neighbours.  A warp per vertex (hubs with tens of thousands
// of lower neighbours spread over the grid like everyone else).
__global__ void k_wedge_bound(const Ctl* c, const int32_t* __restrict__ wlist, const long long* __restrict__ U_off,
                              const uint32_t* __restrict__ U_col, const int32_t* __restrict__ U_split,
                              long long* __restrict__ U_wt) {
    pdl_enter();
    const int nW = c->nW;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < nW; i += nwarps) {
        const int32_t u = wlist[i];
        const int sp = U_split[u];
        long long part = 0;
        if (sp >= 2) {
            const long long rb = U_off[u];
#pragma unroll 4
            for (int j = lane; j < sp; j += 32) {
                const uint32_t v = vid(U_col[rb + j]);
                part += U_off[v + 1] - U_off[v];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
        }
        if (lane == 0) U_wt[u] = part;
    }
}

// Work bins: triangle roots by out-degree, 4-cycle pivots by w~.
__global__ void k_bin(Ctl* c, const int32_t* __restrict__ wlist, const long long* __restrict__ U_off,
                      const int32_t* __restrict__ U_split, const long long* __restrict__ U_wt,
                      int32_t* __restrict__ bins, int n, Tuning t, long long chunk_cap) {
    pdl_enter();
    const int nW = c->nW;
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long nW_r = ((long long)nW + 31) & ~31ll;
    int dmax = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nW_r; i += stride) {
        const bool valid = i < nW;
        int tb = -1, cb = -1;
        const int32_t u = valid ? wlist[i] : 0;
        if (valid) {
            const long long rb = U_off[u], re = U_off[u + 1];
            const int split = U_split[u];
            const int k = (int)(re - rb) - split;
            dmax = max(dmax, (int)(re - rb));
            if (k >= 2)
                tb = k <= t.tri_warp_max    ? BIN_TRI_WARP
                     : k <= t.tri_small_max ? BIN_TRI_SMALL
                     : k <= t.tri_block_max ? BIN_TRI_BLOCK
                                            : BIN_TRI_MERGE;
            if (split >= 2) {
                const long long wt = U_wt[u];
                // the hash tier packs 16-bit counts: at most 2^16 - 1 lower neighbours
                cb = wt <= t.c4_reg_max                         ? BIN_C4_REG
                     : wt <= t.c4_warp_max                      ? BIN_C4_WARP
                     : wt <= min(t.c4_block_max, C4B_SMALL_MAX) ? BIN_C4_BSMALL
                     : wt <= t.c4_block_max                     ? BIN_C4_BLOCK
                     : (wt <= t.c4_cta_max && split < 65536)    ? BIN_C4_CTA
                     : (wt > t.c4_chunk_min && wt <= t.c4_chunk_max &&
                        (long long)split * (((long long)u + CH_R - 1) / CH_R + 1) <= chunk_cap) ? BIN_C4_CHUNK
                                                                                                 : BIN_C4_DENSE;
            }
        }
#pragma unroll 1
        for (int b = 0; b < NBINS; b++) {
            bool mine = valid && (tb == b || cb == b);
            unsigned m = __ballot_sync(FULL, mine);
            if (m) {
                int leader = __ffs(m) - 1, base = 0;
                if (lane == leader) base = atomicAdd(&c->nbin[b], __popc(m));
                base = __shfl_sync(FULL, base, leader);
                if (mine) bins[(size_t)b * n + base + __popc(m & lanemask_lt())] = u;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmax = max(dmax, __shfl_down_sync(FULL, dmax, o));
    if (lane == 0 && dmax) atomicMax(&c->maxdeg, dmax);
}

// ---- triangles and 4-cliques -------------------------------------------------

constexpr int TW = 8;  // warps per block of the warp-per-root kernel

__global__ void __launch_bounds__(TW * 32) k_tri_warp(Ctl* c, const int32_t* __restrict__ list,
                                                     const long long* __restrict__ U_off,
                                                     const uint32_t* __restrict__ U_col,
                                                     const int32_t* __restrict__ U_split,
                                                     unsigned long long* __restrict__ tpack) {
    pdl_enter();
    __shared__ uint32_t sX[TW][32];
    __shared__ long long sNb[TW][32];
    __shared__ int sPre[TW][33];
    __shared__ uint32_t sRA[TW][32], sRB[TW][32];
    __shared__ unsigned long long sTq[TW][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int cnt = c->nbin[BIN_TRI_WARP];
    unsigned long long ka = 0, kb = 0;
    for (int i = blockIdx.x * TW + w; i < cnt; i += gridDim.x * TW) {
        int32_t u = list[i];
        long long rb = U_off[u] + U_split[u];
        int k = (int)(U_off[u + 1] - rb);
        uint32_t x = lane < k ? U_col[rb + lane] : 0u;
        uint32_t xmax = vid(__shfl_sync(FULL, x, k - 1));
        int cq = 0;
        long long nb = 0;
        if (lane < k) {
            uint32_t v = vid(x);
            nb = U_off[v] + U_split[v];
            cq = (int)lower_bound_id(U_col + nb, U_off[v + 1] - nb, xmax + 1);
        }
        int inc = cq;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += y;
        }
        const int total = __shfl_sync(FULL, inc, 31);
        sX[w][lane] = x;
        sNb[w][lane] = nb;
        sPre[w][lane + 1] = inc;
        if (lane == 0) sPre[w][0] = 0;
        sRA[w][lane] = 0;
        sRB[w][lane] = 0;
        sTq[w][lane] = 0;
        __syncwarp();
        int q = 0;
        for (int t = lane; t < total; t += 32) {
            while (q + 1 < k && sPre[w][q + 1] <= t) q++;
            long long slot = sNb[w][q] + (t - sPre[w][q]);
            uint32_t e = U_col[slot];
            int p = find_pos(sX[w], k, vid(e));
            if (p < 0) continue;
            uint32_t f = sX[w][q] & sX[w][p] & e;
            unsigned long long iv = flag_inc(f);
            if (!iv) continue;
            if (f & FLAG_A) atomicOr(&sRA[w][q], 1u << p);
            if (f & FLAG_B) atomicOr(&sRB[w][q], 1u << p);
            atomicAdd(&sTq[w][q], iv);
            atomicAdd(&sTq[w][p], iv);
            atomicAdd(&tpack[slot], iv);
        }
        __syncwarp();
        if (lane < k) {
            uint32_t ra = sRA[w][lane], rbm = sRB[w][lane];
            for (uint32_t m = ra; m; m &= m - 1) ka += __popc(ra & sRA[w][__ffs(m) - 1]);
            for (uint32_t m = rbm; m; m &= m - 1) kb += __popc(rbm & sRB[w][__ffs(m) - 1]);
            unsigned long long tq = sTq[w][lane];
            if (tq) atomicAdd(&tpack[rb + lane], tq);
        }
        __syncwarp();
    }
    acc_add(c, 4, ka);
    acc_add(c, 10, kb);
}

// Shared memory of the block kernel for out-lists of up to KM entries.
template <int KM>
constexpr size_t tri_block_smem() {
    return (size_t)KM * 4 + (size_t)KM * 8 + (size_t)(KM + 8) * 4 + 2ull * KM * (KM / 32) * 4 + (size_t)KM * 8;
}
size_t tri_block_smem_bytes() { return tri_block_smem<TRI_KM>(); }

// Roots with 32 < k <= KM: one block per root.  The out-list X is held
// in shared memory; the candidates (every entry of N+(v) up to max X, for v
// in X) are dealt in warp-contiguous runs of 32, so a lane finds its row by
// stepping from the run's first row, and its position in X by binary search.
// Two instances: KM = TRI_KS for the many short lists (small shared
// footprint, many blocks per SM) and KM = TRI_KM for the long ones.
template <int KM, int BIN, int WORK>
__global__ void __launch_bounds__(256) k_tri_block(Ctl* c, const int32_t* __restrict__ list,
                                                  const long long* __restrict__ U_off,
                                                  const uint32_t* __restrict__ U_col,
                                                  const int32_t* __restrict__ U_split,
                                                  unsigned long long* __restrict__ tpack) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem[];
    long long* sNb = (long long*)smem;
    unsigned long long* sTq = (unsigned long long*)(smem + (size_t)KM * 8);
    uint32_t* sX = (uint32_t*)(smem + (size_t)KM * 16);
    int* sPre = (int*)(smem + (size_t)KM * 20);
    uint32_t* sRA = (uint32_t*)(smem + (size_t)KM * 24 + 32);
    uint32_t* sRB = sRA + KM * (KM / 32);
    __shared__ int s_idx;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NW = blockDim.x >> 5;
    const int cnt = c->nbin[BIN];
    unsigned long long ka = 0, kb = 0;
    for (;;) {
        if (tid == 0) s_idx = (int)atomicAdd(&c->work[WORK], 1u);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= cnt) break;
        int32_t u = list[idx];
        long long rb = U_off[u] + U_split[u];
        const int k = (int)(U_off[u + 1] - rb);
        const int W = (k + 31) >> 5;
        const uint32_t xmax = vid(U_col[rb + k - 1]);
        for (int t = tid; t < k; t += blockDim.x) {
            uint32_t x = U_col[rb + t];
            uint32_t v = vid(x);
            long long nb = U_off[v] + U_split[v];
            sX[t] = x;
            sNb[t] = nb;
            sPre[t + 1] = (int)lower_bound_id(U_col + nb, U_off[v + 1] - nb, xmax + 1);
            sTq[t] = 0;
        }
        for (int t = tid; t < k * W; t += blockDim.x) {
            sRA[t] = 0;
            sRB[t] = 0;
        }
        __syncthreads();
        if (warp == 0) {  // inclusive scan of sPre[1..k]
            int carry = 0;
            for (int b = 0; b < k; b += 32) {
                int x = b + lane < k ? sPre[b + lane + 1] : 0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    int y = __shfl_up_sync(FULL, x, o);
                    if (lane >= o) x += y;
                }
                if (b + lane < k) sPre[b + lane + 1] = x + carry;
                carry += __shfl_sync(FULL, x, 31);
            }
            if (lane == 0) sPre[0] = 0;
        }
        __syncthreads();
        const int total = sPre[k];
        for (int base = warp * 32; base < total; base += NW * 32) {
            const int t = base + lane;
            int q = find_seg(sPre, k, base);
            if (t < total) {
                while (q + 1 < k && sPre[q + 1] <= t) q++;
                const long long slot = sNb[q] + (t - sPre[q]);
                const uint32_t e = U_col[slot];
                const int p = find_pos(sX, k, vid(e));
                if (p >= 0) {
                    const uint32_t f = sX[q] & sX[p] & e;
                    const unsigned long long iv = flag_inc(f);
                    if (iv) {
                        if (f & FLAG_A) atomicOr(&sRA[q * W + (p >> 5)], 1u << (p & 31));
                        if (f & FLAG_B) atomicOr(&sRB[q * W + (p >> 5)], 1u << (p & 31));
                        atomicAdd(&sTq[q], iv);
                        atomicAdd(&sTq[p], iv);
                        atomicAdd(&tpack[slot], iv);
                    }
                }
            }
        }
        __syncthreads();
        for (int q = tid; q < k; q += blockDim.x) {
            const uint32_t* ra = sRA + q * W;
            const uint32_t* rbm = sRB + q * W;
            for (int i = 0; i < W; i++) {
                for (uint32_t m = ra[i]; m; m &= m - 1) {
                    int p = i * 32 + __ffs(m) - 1;
                    const uint32_t* rp = sRA + p * W;
                    for (int i2 = p >> 5; i2 < W; i2++) ka += __popc(ra[i2] & rp[i2]);
                }
                for (uint32_t m = rbm[i]; m; m &= m - 1) {
                    int p = i * 32 + __ffs(m) - 1;
                    const uint32_t* rp = sRB + p * W;
                    for (int i2 = p >> 5; i2 < W; i2++) kb += __popc(rbm[i2] & rp[i2]);
                }
            }
            unsigned long long tq = sTq[q];
            if (tq) atomicAdd(&tpack[rb + q], tq);
        }
        __syncthreads();
    }
    acc_add(c, 4, ka);
    acc_add(c, 10, kb);
}

// Roots with very long out-lists: one warp per root, one lane per out-edge
// u->v merging N+(u) (after v) with N+(v); 4-cliques by a three-way merge.
__global__ void k_tri_merge(Ctl* c, const int32_t* __restrict__ list, const long long* __restrict__ U_off,
                            const uint32_t* __restrict__ U_col, const int32_t* __restrict__ U_split,
                            unsigned long long* __restrict__ tpack) {
    pdl_enter();
    const int cnt = c->nbin[BIN_TRI_MERGE];
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    unsigned long long ka = 0, kb = 0;
    for (int wi = warp; wi < cnt; wi += nwarps) {
        int32_t u = list[wi];
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
    acc_add(c, 4, ka);
    acc_add(c, 10, kb);
}

// ---- 4-cycles ----------------------------------------------------------------

constexpr uint32_t EMPTY_KEY = 0xFFFFFFFFu;

// packed counter: G_a count in the high 16 bits, G_b count in the low 16
__device__ __forceinline__ uint32_t flag_inc16(uint32_t f) {
    return ((f & FLAG_A) ? 0x10000u : 0u) | ((f & FLAG_B) ? 1u : 0u);
}

// open-addressing insert; returns the counter's old value
__device__ __forceinline__ uint32_t hash_add(uint32_t* keys, uint32_t* cnts, int shift, uint32_t mask, uint32_t w,
                                             uint32_t inc) {
    uint32_t h = (w * 0x9E3779B1u) >> shift;
    for (;;) {
        uint32_t k = keys[h];
        if (k == w) return atomicAdd(&cnts[h], inc);
        if (k == EMPTY_KEY) {
            uint32_t prev = atomicCAS(&keys[h], EMPTY_KEY, w);
            if (prev == EMPTY_KEY || prev == w) return atomicAdd(&cnts[h], inc);
        }
        h = (h + 1) & mask;
    }
}

__device__ __forceinline__ int log2_table(long long wt, int lo_log, int hi_log) {
    int lg = lo_log;
    while (lg < hi_log && (1ll << lg) < 2 * wt) lg++;
    return lg;
}

// w~ <= 32: every wedge endpoint in one lane; equal endpoints are grouped
// with __match_any_sync and each group adds C(c, 2).
__global__ void __launch_bounds__(256) k_c4_reg(Ctl* c, const int32_t* __restrict__ list,
                                               const long long* __restrict__ U_off,
                                               const uint32_t* __restrict__ U_col,
                                               const int32_t* __restrict__ U_split) {
    pdl_enter();
    __shared__ long long sVb[8][32];
    __shared__ uint32_t sFv[8][32];
    __shared__ int sPre[8][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int cnt = c->nbin[BIN_C4_REG];
    unsigned long long qa = 0, qb = 0, wedges = 0;
    for (int i = blockIdx.x * 8 + w; i < cnt; i += gridDim.x * 8) {
        int32_t u = list[i];
        long long rb = U_off[u];
        int nlow = U_split[u];  // 2..32 here
        int dv = 0;
        if (lane < nlow) {
            uint32_t fv = U_col[rb + lane];
            uint32_t v = vid(fv);
            long long vb = U_off[v];
            dv = (int)(U_off[v + 1] - vb);
            sVb[w][lane] = vb;
            sFv[w][lane] = fv;
        }
        int inc = dv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += y;
        }
        const int total = __shfl_sync(FULL, inc, 31);  // <= 32
        sPre[w][lane + 1] = inc;
        if (lane == 0) sPre[w][0] = 0;
        __syncwarp();
        bool ok = false;
        uint32_t wv = 0, fl = 0;
        if (lane < total) {
            int j = find_seg(sPre[w], nlow, lane);
            uint32_t e = U_col[sVb[w][j] + (lane - sPre[w][j])];
            wv = vid(e);
            ok = wv < (uint32_t)u;
            fl = sFv[w][j] & e & (FLAG_A | FLAG_B);
        }
        unsigned okm = __ballot_sync(FULL, ok);
        if (lane == 0) wedges += __popc(okm);
        bool valid = ok && fl;
        unsigned peers = __match_any_sync(FULL, valid ? wv : (0x80000000u | (uint32_t)lane));
        unsigned ba = __ballot_sync(FULL, valid && (fl & FLAG_A));
        unsigned bb = __ballot_sync(FULL, valid && (fl & FLAG_B));
        if (valid && lane == __ffs(peers) - 1) {
            qa += choose2(__popc(peers & ba));
            qb += choose2(__popc(peers & bb));
        }
        __syncwarp();
    }
    acc_add(c, 5, qa);
    acc_add(c, 11, qb);
    acc_add(c, 15, wedges);
}

// Walk the wedges u-v-w of pivot u (w < u) for its lower neighbours
// v = N(u)[j], calling fn(w, flags) once per wedge.  The warp takes 32
// lower neighbours at a time and lays their rows end to end (a warp prefix
// sum over the nonempty rows); each lane then finds its row from a bitmask
// of row starts (one OR-reduction per 32 entries), so the loads of up to 128
// entries of many short rows are in flight together instead of one row after
// the other.  Entries at or above u are read and skipped.  Rows are taken in
// groups j0 = first, first + 32 * step, ...; scratch: 32 ints, 32 int64 and
// 32 uint32 of shared memory per warp.  Warp-uniform.
constexpr int WF_UNROLL = 4;
template <class Fn>
__device__ __forceinline__ void walk_flat(const long long* __restrict__ U_off, const uint32_t* __restrict__ U_col,
                                          uint32_t u, long long rb, int nlow, int first, int step, int* cpre,
                                          long long* cvb, uint32_t* cfv, Fn fn) {
    const int lane = threadIdx.x & 31;
    for (int j0 = first * 32; j0 < nlow; j0 += step * 32) {
        const int j = j0 + lane;
        int len = 0;
        long long vb = 0;
        uint32_t fv = 0;
        if (j < nlow) {
            fv = U_col[rb + j];
            const uint32_t v = vid(fv);
            vb = U_off[v];
            len = (int)(U_off[v + 1] - vb);
        }
        const unsigned ne = __ballot_sync(FULL, len > 0);
        if (!ne) continue;
        int inc = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += y;
        }
        const int total = __shfl_sync(FULL, inc, 31);
        const int k = __popc(ne);
        __syncwarp();
        if (len > 0) {
            const int slot = __popc(ne & lanemask_lt());
            cpre[slot] = inc - len;
            cvb[slot] = vb - (inc - len);
            cfv[slot] = fv;
        }
        __syncwarp();
        const int my_start = lane < k ? cpre[lane] : 0x7FFFFFFF;
        int R = 0;  // row holding position t0 (warp-uniform)
        for (int t0 = 0; t0 < total; t0 += 32 * WF_UNROLL) {
            uint32_t ev[WF_UNROLL], fr[WF_UNROLL];
#pragma unroll
            for (int q = 0; q < WF_UNROLL; q++) {
                const int tb = t0 + q * 32;
                ev[q] = 0xFFFFFFFFu;
                fr[q] = 0;
                if (tb < total) {
                    const unsigned bit = (my_start > tb && my_start < tb + 32) ? (1u << (my_start - tb)) : 0u;
                    const unsigned m = __reduce_or_sync(FULL, bit);
                    const int r = R + __popc(m & ((2u << lane) - 1u));
                    if (tb + lane < total) {
                        ev[q] = U_col[cvb[r] + tb + lane];
                        fr[q] = cfv[r];
                    }
                    int rn = R + __popc(m);
                    if (rn + 1 < k && cpre[rn + 1] == tb + 32) rn++;
                    R = rn;
                }
            }
#pragma unroll
            for (int q = 0; q < WF_UNROLL; q++) {
                const uint32_t w = vid(ev[q]);
                if (ev[q] != 0xFFFFFFFFu && w < u) fn(w, fr[q] & ev[q] & (FLAG_A | FLAG_B));
            }
        }
        __syncwarp();
    }
}

constexpr int C4W_WARPS = 4;
constexpr int C4W_SLOTS = 2 * C4_T1;

__global__ void __launch_bounds__(C4W_WARPS * 32) k_c4_warp(Ctl* c, const int32_t* __restrict__ list,
                                                          const long long* __restrict__ U_off,
                                                          const uint32_t* __restrict__ U_col,
                                                          const int32_t* __restrict__ U_split,
                                                          const long long* __restrict__ U_wt) {
    pdl_enter();
    __shared__ uint32_t sKey[C4W_WARPS][C4W_SLOTS];
    __shared__ uint32_t sCnt[C4W_WARPS][C4W_SLOTS];
    __shared__ int s_pre[C4W_WARPS][32];
    __shared__ long long s_vb[C4W_WARPS][32];
    __shared__ uint32_t s_fv[C4W_WARPS][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int cnt = c->nbin[BIN_C4_WARP];
    unsigned long long qa = 0, qb = 0, wedges = 0;
    uint32_t* keys = sKey[w];
    uint32_t* cnts = sCnt[w];
    for (int i = blockIdx.x * C4W_WARPS + w; i < cnt; i += gridDim.x * C4W_WARPS) {
        const uint32_t u = (uint32_t)list[i];
        const long long rb = U_off[u];
        const int nlow = U_split[u];
        const int lg = log2_table(U_wt[u], 5, 10);
        const uint32_t mask = (1u << lg) - 1;
        const int shift = 32 - lg;
        for (int s = lane; s <= (int)mask; s += 32) {
            keys[s] = EMPTY_KEY;
            cnts[s] = 0;
        }
        __syncwarp();
        walk_flat(U_off, U_col, u, rb, nlow, 0, 1, s_pre[w], s_vb[w], s_fv[w], [&](uint32_t wv, uint32_t fl) {
            wedges++;
            if (!fl) return;
            uint32_t old = hash_add(keys, cnts, shift, mask, wv, flag_inc16(fl));
            if (fl & FLAG_A) qa += old >> 16;
            if (fl & FLAG_B) qb += old & 0xFFFFu;
        });
        __syncwarp();
    }
    acc_add(c, 5, qa);
    acc_add(c, 11, qb);
    acc_add(c, 15, wedges);
}

// Prefix sums of the row lengths of lower neighbours rb[s0 .. s0+ns) of a
// pivot, so a pivot's wedges can be split evenly over many threads: wedge i
// of the segment lies in row j = find_seg(pre, ns, i), at U_col[vbs[j] + i]
// (vbs holds each row's start minus its prefix).
// Every thread of the block calls it; ends with __syncthreads().
__device__ __forceinline__ void wedge_segment_prefix(const long long* __restrict__ U_off,
                                                     const uint32_t* __restrict__ U_col, long long rb, int s0, int ns,
                                                     int* pre, long long* vbs, uint32_t* fvs, int* wtot) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    for (int j = tid; j < ns; j += blockDim.x) {
        uint32_t fv = U_col[rb + s0 + j];
        uint32_t v = vid(fv);
        long long vb = U_off[v];
        vbs[j] = vb;
        fvs[j] = fv;
        pre[j + 1] = (int)(U_off[v + 1] - vb);
    }
    __syncthreads();
    // two-level scan: each warp scans a contiguous slice, then the slice totals
    const int per = (ns + nwarps - 1) / nwarps;
    const int b0 = warp * per, b1 = min(ns, b0 + per);
    int carry = 0;
    for (int b = b0; b < b1; b += 32) {
        int x = b + lane < b1 ? pre[b + lane + 1] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        if (b + lane < b1) pre[b + lane + 1] = x + carry;
        carry += __shfl_sync(FULL, x, 31);
    }
    __shared__ int s_part[33];
    if (lane == 0) s_part[warp + 1] = carry;
    __syncthreads();
    if (tid == 0) {
        s_part[0] = 0;
        for (int w = 1; w <= nwarps; w++) s_part[w] += s_part[w - 1];
        pre[0] = 0;
        *wtot = s_part[nwarps];
    }
    __syncthreads();
    for (int j = b0 + lane; j < b1; j += 32) pre[j + 1] += s_part[warp];
    __syncthreads();
    // rebase: wedge i of row j is U_col[vbs[j] + i]
    for (int j = tid; j < ns; j += blockDim.x) vbs[j] -= pre[j];
    __syncthreads();
}

constexpr int C4D_SEG = 2048;  // lower neighbours per prefix segment
constexpr int C4D_UNROLL = 4;

// Block-wide walk over the elements of ns <= C4D_SEG rows laid end to end,
// so every warp of the block has work however the row lengths vary.  Row j
// has len_fn(j, &base, &flag) elements starting at U_col[base]; the prefix of
// the lengths goes to pre[0 .. ns] (block scan), each row's start minus its
// prefix to vbs[j] and its flag word to fvs[j].  Then each warp takes runs of
// 32 * C4D_UNROLL consecutive elements (binary search for the run's first
// row, then steps) and calls fn(j, p, e, f) for the element at position p of
// row j (e = its adjacency entry, f = the row's flag word), loads of a run in
// flight together.  Every thread of the block calls it; ends with
// __syncthreads().  Returns the number of elements.
template <class LenFn, class Fn>
__device__ __forceinline__ int block_walk_rows(const uint32_t* __restrict__ U_col, int ns, int* pre, long long* vbs,
                                               uint32_t* fvs, int* s_tot, LenFn len_fn, Fn fn) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    for (int j = tid; j < ns; j += blockDim.x) {
        long long b = 0;
        uint32_t f = 0;
        pre[j + 1] = len_fn(j, &b, &f);
        vbs[j] = b;
        fvs[j] = f;
    }
    __syncthreads();
    // two-level scan: each warp scans a contiguous slice, then the slice totals
    const int per = (ns + nwarps - 1) / nwarps;
    const int b0 = warp * per, b1 = min(ns, b0 + per);
    int carry = 0;
    for (int b = b0; b < b1; b += 32) {
        int x = b + lane < b1 ? pre[b + lane + 1] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        if (b + lane < b1) pre[b + lane + 1] = x + carry;
        carry += __shfl_sync(FULL, x, 31);
    }
    __shared__ int s_part[33];
    if (lane == 0) s_part[warp + 1] = carry;
    __syncthreads();
    if (tid == 0) {
        s_part[0] = 0;
        for (int w = 1; w <= nwarps; w++) s_part[w] += s_part[w - 1];
        pre[0] = 0;
        *s_tot = s_part[nwarps];
    }
    __syncthreads();
    for (int j = b0 + lane; j < b1; j += 32) pre[j + 1] += s_part[warp];
    __syncthreads();
    for (int j = tid; j < ns; j += blockDim.x) vbs[j] -= pre[j];
    __syncthreads();
    const int total = *s_tot;
    for (int base = warp * 32 * C4D_UNROLL; base < total; base += nwarps * 32 * C4D_UNROLL) {
        uint32_t e[C4D_UNROLL], f[C4D_UNROLL];
        int jr[C4D_UNROLL];
        int j = find_seg(pre, ns, base);
#pragma unroll
        for (int r = 0; r < C4D_UNROLL; r++) {
            const int i = base + r * 32 + lane;
            e[r] = 0xFFFFFFFFu;
            f[r] = 0;
            jr[r] = -1;
            if (i < total) {
                while (j + 1 < ns && pre[j + 1] <= i) j++;
                e[r] = U_col[vbs[j] + i];
                f[r] = fvs[j];
                jr[r] = j;
            }
        }
#pragma unroll
        for (int r = 0; r < C4D_UNROLL; r++)
            if (jr[r] >= 0) fn(jr[r], base + r * 32 + lane - pre[jr[r]], e[r], f[r]);
    }
    __syncthreads();
    return total;
}


// Medium pivots: one block per pivot, hash table of up to 2^LG slots in
// shared memory.  Two instances: 2^12 slots with 4 warps (several blocks per
// SM) for the smaller wedge bounds, each warp laying 32 rows end to end
// (walk_flat); 2^14 slots with 16 warps for the rest, the whole block laying
// all the pivot's rows end to end (block_walk_rows), so no warp waits idle at
// the block barrier while others walk long rows.
constexpr int C4B_SMALL_LG = 12, C4B_SMALL_THREADS = 128;
constexpr int C4B_BIG_LG = 14, C4B_BIG_THREADS = 512;
template <int LG, int THREADS>
constexpr size_t c4_block_smem() {
    return ((size_t)8 << LG) + (size_t)(THREADS / 32) * 32 * (4 + 8 + 4);
}

template <int LG, int THREADS, int BIN, int WORK, bool BLOCKWIDE>
__global__ void __launch_bounds__(THREADS) k_c4_block(Ctl* c, const int32_t* __restrict__ list,
                                                      const long long* __restrict__ U_off,
                                                      const uint32_t* __restrict__ U_col,
                                                      const int32_t* __restrict__ U_split,
                                                      const long long* __restrict__ U_wt) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* keys = (uint32_t*)smem;
    uint32_t* cnts = keys + (1 << LG);
    long long* w_vb = (long long*)(cnts + (1 << LG));
    int* w_pre = (int*)(w_vb + THREADS);
    uint32_t* w_fv = (uint32_t*)(w_pre + THREADS);
    __shared__ int s_idx;
    constexpr int SEG = BLOCKWIDE ? C4D_SEG : 1;
    __shared__ int s_pre[SEG + 1], s_tot;
    __shared__ long long s_vb[SEG];
    __shared__ uint32_t s_fv[SEG];
    const int tid = threadIdx.x, warp = tid >> 5, nwarps = THREADS >> 5;
    const int cnt = c->nbin[BIN];
    unsigned long long qa = 0, qb = 0, wedges = 0;
    for (;;) {
        if (tid == 0) s_idx = (int)atomicAdd(&c->work[WORK], 1u);
        __syncthreads();
        const int idx = s_idx;
        if (idx >= cnt) break;
        const uint32_t u = (uint32_t)list[idx];
        const long long rb = U_off[u];
        const int nlow = U_split[u];
        const int lg = log2_table(U_wt[u], 6, LG);
        const uint32_t mask = (1u << lg) - 1;
        const int shift = 32 - lg;
        for (int s = tid; s <= (int)mask; s += THREADS) {
            keys[s] = EMPTY_KEY;
            cnts[s] = 0;
        }
        __syncthreads();
        auto count = [&](uint32_t wv, uint32_t fl) {
            wedges++;
            if (!fl) return;
            uint32_t old = hash_add(keys, cnts, shift, mask, wv, flag_inc16(fl));
            if (fl & FLAG_A) qa += old >> 16;
            if (fl & FLAG_B) qb += old & 0xFFFFu;
        };
        if constexpr (BLOCKWIDE) {
            for (int s0 = 0; s0 < nlow; s0 += SEG) {
                const int ns = min(SEG, nlow - s0);
                block_walk_rows(
                    U_col, ns, s_pre, s_vb, s_fv, &s_tot,
                    [&](int j, long long* b, uint32_t* f) {
                        const uint32_t fv = U_col[rb + s0 + j];
                        const uint32_t v = vid(fv);
                        *b = U_off[v];
                        *f = fv;
                        return (int)(U_off[v + 1] - *b);
                    },
                    [&](int, int, uint32_t e, uint32_t f) {
                        const uint32_t wv = vid(e);
                        if (wv < u) count(wv, f & e & (FLAG_A | FLAG_B));
                    });
            }
        } else {
            walk_flat(U_off, U_col, u, rb, nlow, warp, nwarps, w_pre + warp * 32, w_vb + warp * 32,
                      w_fv + warp * 32, count);
            __syncthreads();
        }
    }
    acc_add(c, 5, qa);
    acc_add(c, 11, qb);
    acc_add(c, 15, wedges);
}

// Reductions in L2 that return nothing (the compiler may otherwise merge
// them with the returning atomics of the other path).
__device__ __forceinline__ void red_add_u32(uint32_t* p, uint32_t v) {
    asm volatile("red.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_add_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("red.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <bool CLUSTER>
__device__ __forceinline__ void group_sync() {
    if constexpr (CLUSTER) {
        __threadfence();
        cg::this_cluster().sync();
    } else {
        __syncthreads();
    }
}

// Heavy pivots, dense counter array in global memory (16/16-bit packed
// counts while every degree is below 2^16, else 32/32 in 64-bit words).
// CLUSTER = true: a cluster of CTAs takes one pivot at a time and shares one
// array (the instance launched); CLUSTER = false: one CTA per pivot with its
// own array.  The pivot's wedges are numbered through per-segment prefix
// sums and dealt in warp-contiguous chunks to every thread of the group
// (coalesced, balanced even when one lower neighbour has a very long row).
// Two ways through a pivot, each ending with group barriers:
//   w~ > u / 16 (many wedges for its id range): increments by L2 reductions,
//     then one coalesced sweep of the counters of [0, u) that adds C(c_w, 2)
//     and clears them;
//   otherwise: increments that return the old value (summed on the fly),
//     then the same wedges walked again to clear what they touched.
// While every degree is below 2^16 (narrow layout), a wedge in both graphs
// adds 1 to a 16-bit count of its endpoint, two endpoints to a 32-bit word,
// so the counters of a cluster take 2 bytes per id (half of a 16/16 pair
// per id): the L2 holds them and more of the adjacency, and random L2
// reductions run faster on the smaller footprint (130 against 100 G/s for
// 61 against 122 MB in all, by a probe on this GPU).  The few wedges in one
// graph only (through a changed pair) count in separate 16/16 counters and
// are listed; after the increments, each listed wedge adds the both-graph
// count of its endpoint (the cross term of C(c_ab + c_x, 2)) and clears
// its counter, before the sweep or the clearing walk.
template <bool CLUSTER>
__global__ void __launch_bounds__(C4_DENSE_THREADS, 1) k_c4_dense_t(Ctl* c, const int32_t* __restrict__ list,
                                                                const long long* __restrict__ U_off,
                                                                const uint32_t* __restrict__ U_col,
                                                                const int32_t* __restrict__ U_split,
                                                                const long long* __restrict__ U_wt,
                                                                unsigned long long* __restrict__ arrays, int n) {
    pdl_enter();
    int rank = 0, ncta = 1;
    if constexpr (CLUSTER) {
        cg::cluster_group cl = cg::this_cluster();
        rank = (int)cl.block_rank();
        ncta = (int)cl.num_blocks();
    }
    const int gid = blockIdx.x / ncta;
    // per-group regions start on 16-byte boundaries (vectorised sweeps)
    unsigned long long* a64 = arrays + (size_t)gid * (size_t)dense_stride(n);
    const bool wide = c->maxdeg >= 65536;
    // Narrow layout (every degree below 2^16), in 32-bit words of the region:
    //   cab  one 16-bit count per id of the wedges in both graphs, two ids
    //        to a word (id w in half w & 1), 16-byte aligned;
    //   cx   16/16 counts (G_a high, G_b low) of the wedges in one graph only;
    //   lcount, lst  the list of those wedges (id | bit 31 for G_b) of the
    //        pivot being counted, lcap entries (none when the region has no
    //        room, on tiny graphs).
    uint32_t* a32 = (uint32_t*)a64;
    const long long words = 2 * dense_stride(n);
    const long long off_ab = ((long long)n + 3) & ~3ll, len_ab = (((long long)n + 1) / 2 + 3) & ~3ll;
    uint32_t* cx = a32;
    uint32_t* cab = a32 + off_ab;
    uint32_t* lcount = a32 + off_ab + len_ab;
    uint32_t* lst = lcount + 4;
    const long long lcap = min(words - (off_ab + len_ab + 4), 0x7FFFFFFFll);
    __shared__ int s_tot;
    __shared__ int s_pre[C4D_SEG + 1];
    __shared__ long long s_vb[C4D_SEG];
    __shared__ uint32_t s_fv[C4D_SEG];
    const long long T = (long long)ncta * blockDim.x;
    const long long g = (long long)rank * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int gwarp = rank * (int)(blockDim.x >> 5) + (int)(threadIdx.x >> 5);
    const int NW = ncta * (int)(blockDim.x >> 5);
    const int bin = CLUSTER ? BIN_C4_DENSE : BIN_C4_CTA;
    const int cnt = c->nbin[bin];
    unsigned long long qa = 0, qb = 0, wedges = 0, nred = 0, natom = 0;
    // Pivot indices: the group's first thread takes the next pivot from the
    // work counter while the current one is processed, into one of two slots
    // (iteration t reads slot t & 1, fills slot (t + 1) & 1); the barrier at
    // the end of each pivot publishes it, so fetching costs no barrier of
    // its own.  A slot is refilled only after every CTA has passed the
    // barrier that follows its last read.
    __shared__ int s_next[2];
    const int work_slot = CLUSTER ? WORK_C4_DENSE : WORK_C4_CTA;
    if (rank == 0 && threadIdx.x == 0) s_next[0] = (int)atomicAdd(&c->work[work_slot], 1u);
    group_sync<CLUSTER>();
    for (int iter = 0;; iter++) {
        int idx;
        if constexpr (CLUSTER) idx = *cg::this_cluster().map_shared_rank(&s_next[iter & 1], 0);
        else idx = s_next[iter & 1];
        if (idx >= cnt) break;
        if (rank == 0 && threadIdx.x == 0) s_next[(iter + 1) & 1] = (int)atomicAdd(&c->work[work_slot], 1u);
        const int32_t u = list[idx];
        const long long rb = U_off[u];
        const int nlow = U_split[u];
        // A pivot with many wedges for its id range (w~ > u / 16) increments
        // without taking old values, then sweeps the counters of [0, u)
        // once, coalesced: each c_w gives C(c_w, 2) and is cleared.  Smaller
        // pivots take old values and clear by walking their wedges again.
        // (With 16-bit counts the sweep reads u / 2 bytes; u / 16 beat u / 8,
        // u / 4 and u / 32 on the 1.6M-vertex graph.)
        const bool sweep = U_wt[u] * 16 > (long long)u;
        // One walk over the pivot's wedges.  mode 0: increments; mode 1:
        // cross terms of the wedges of one graph only (narrow layout); mode
        // 2: clearing what mode 0 touched.
        auto walk = [&](int mode) {
            for (int s0 = 0; s0 < nlow; s0 += C4D_SEG) {
                const int ns = min(C4D_SEG, nlow - s0);
                // a single-segment pivot keeps its prefix for the later walks
                if (mode == 0 || nlow > C4D_SEG)
                    wedge_segment_prefix(U_off, U_col, rb, s0, ns, s_pre, s_vb, s_fv, &s_tot);
                const int total = s_tot;
                // each warp takes C4D_UNROLL consecutive chunks of 32 wedges;
                // a lane finds its row by stepping forward from the chunk's
                // first row (rows average tens of entries, so a step or two)
                const int wstep = NW * 32 * C4D_UNROLL;
                for (int base = gwarp * 32 * C4D_UNROLL; base < total; base += wstep) {
                    uint32_t e[C4D_UNROLL], f[C4D_UNROLL];
                    int j = find_seg(s_pre, ns, (int)base);
                    const int end = min(total, base + 32 * C4D_UNROLL);
                    if (j + 1 >= ns || s_pre[j + 1] >= end) {
                        // the whole chunk lies in one row: its base and flags are uniform
                        const long long vb = s_vb[j];
                        const uint32_t fv = s_fv[j];
#pragma unroll
                        for (int r = 0; r < C4D_UNROLL; r++) {
                            const int i = base + r * 32 + lane;
                            e[r] = i < total ? U_col[vb + i] : 0xFFFFFFFFu;
                            f[r] = fv;
                        }
                    } else {
#pragma unroll
                        for (int r = 0; r < C4D_UNROLL; r++) {
                            const int i = base + r * 32 + lane;
                            e[r] = 0xFFFFFFFFu;
                            f[r] = 0;
                            if (i < total) {
                                while (j + 1 < ns && s_pre[j + 1] <= i) j++;
                                e[r] = U_col[s_vb[j] + i];
                                f[r] = s_fv[j];
                            }
                        }
                    }
#pragma unroll
                    for (int r = 0; r < C4D_UNROLL; r++) {
                        const uint32_t wv = vid(e[r]);
                        if (wv >= (uint32_t)u) continue;
                        const uint32_t fl = f[r] & e[r] & (FLAG_A | FLAG_B);
                        if (mode == 0) wedges++;
                        if (!fl) continue;
                        if (wide) {
                            if (mode == 2) {
                                a64[wv] = 0ull;
                            } else if (sweep) {
                                nred++;
                                red_add_u64(&a64[wv], flag_inc(fl));
                            } else {
                                natom++;
                                const unsigned long long old = atomicAdd(&a64[wv], flag_inc(fl));
                                if (fl & FLAG_A) qa += old >> 32;
                                if (fl & FLAG_B) qb += old & 0xFFFFFFFFull;
                            }
                            continue;
                        }
                        const int sh = (int)(wv & 1u) * 16;
                        if (fl == (FLAG_A | FLAG_B)) {
                            if (mode == 2) {
                                cab[wv >> 1] = 0u;
                            } else if (mode == 0) {
                                if (sweep) {
                                    nred++;
                                    red_add_u32(&cab[wv >> 1], 1u << sh);
                                } else {
                                    natom++;
                                    const uint32_t c = (atomicAdd(&cab[wv >> 1], 1u << sh) >> sh) & 0xFFFFu;
                                    qa += c;
                                    qb += c;
                                }
                            }
                        } else if (mode == 0) {
                            // one graph only: its own count by a returning
                            // atomic, the wedge listed for the cross term
                            natom++;
                            const uint32_t old = atomicAdd(&cx[wv], flag_inc16(fl));
                            if (fl & FLAG_A) qa += old >> 16;
                            else qb += old & 0xFFFFu;
                            if (lcap > 0) {
                                const uint32_t at = atomicAdd(lcount, 1u);
                                if (at < (uint32_t)lcap) lst[at] = wv | (fl == FLAG_B ? 0x80000000u : 0u);
                            }
                        } else if (mode == 1) {
                            const uint64_t c = (__ldcg(&cab[wv >> 1]) >> sh) & 0xFFFFu;
                            if (fl & FLAG_A) qa += c;
                            else qb += c;
                            cx[wv] = 0u;
                        }
                    }
                }
                __syncthreads();  // the next segment reuses the shared arrays
            }
        };
        walk(0);
        group_sync<CLUSTER>();
        if (!wide) {
            // c_a(w) = c_ab(w) + c_a-only(w): C(c_a, 2) = C(c_ab, 2) +
            // C(c_a-only, 2) + c_ab(w) c_a-only(w).  The second term was summed
            // on arrival; the cross term adds c_ab(w) once per listed wedge
            // (the whole walk again if the list overflowed).  Without room for
            // a list (tiny graphs) the walk always runs.
            // The list's entries are zeroed as they are taken: the region is
            // read as 32/32 counters once some degree reaches 2^16.
            const uint32_t nl = lcap > 0 ? __ldcg(lcount) : 1u;
            if (nl) {
                if (nl <= (uint32_t)lcap) {
                    for (long long i = g; i < (long long)nl; i += T) {
                        const uint32_t x = __ldcg(&lst[i]);
                        lst[i] = 0u;
                        const uint32_t wv = x & 0x7FFFFFFFu;
                        const uint64_t c = (__ldcg(&cab[wv >> 1]) >> ((wv & 1u) * 16)) & 0xFFFFu;
                        if (x >> 31) qb += c;
                        else qa += c;
                        cx[wv] = 0u;
                    }
                } else {
                    walk(1);
                    for (long long i = g; i < lcap; i += T) lst[i] = 0u;
                }
                group_sync<CLUSTER>();  // every cross term read before the clearing
                if (lcap > 0 && rank == 0 && threadIdx.x == 0) *lcount = 0u;
            }
        }
        if (sweep) {
            if (wide) {
                for (long long w = g; w < u; w += T) {
                    const unsigned long long x = __ldcg(&a64[w]);
                    if (x) {
                        qa += choose2(x >> 32);
                        qb += choose2(x & 0xFFFFFFFFull);
                        a64[w] = 0ull;
                    }
                }
            } else {
                // eight 16-bit counts per 16-byte load (the counts of ids in
                // both graphs add to both sides)
                const long long q4 = ((long long)u + 7) / 8;
                uint4* a4 = (uint4*)cab;
                for (long long i = g; i < q4; i += T) {
                    const uint4 x = __ldcg(&a4[i]);
                    if (x.x | x.y | x.z | x.w) {
                        const uint32_t xs[4] = {x.x, x.y, x.z, x.w};
                        unsigned long long t = 0;
#pragma unroll
                        for (int k = 0; k < 4; k++) t += choose2(xs[k] >> 16) + choose2(xs[k] & 0xFFFFu);
                        qa += t;
                        qb += t;
                        a4[i] = make_uint4(0, 0, 0, 0);
                    }
                }
            }
        } else {
            walk(2);
        }
        group_sync<CLUSTER>();
    }
    // no CTA leaves while another may still read its shared memory
    group_sync<CLUSTER>();
    acc_add(c, 5, qa);
    acc_add(c, 11, qb);
    acc_add(c, 15, wedges);
    if (CLUSTER) {
        acc_add(c, 20, wedges);
        acc_add(c, 21, nred);
        acc_add(c, 22, natom);
    }
}

// Heavy pivots, counters in shared memory.  Shared-memory atomics are about
// twenty times faster than L2 atomics, but a pivot's endpoints w range over
// [0, u), far more ids than shared memory holds.  So the id range is cut
// into chunks of CH_R ids (one chunk of counters fills the shared array) and
// the pivot is counted chunk by chunk.  Every adjacency row is sorted, so the
// entries of a lower neighbour's row inside chunk b are one contiguous run.
// One CTA takes one pivot at a time:
//   phase 1  a warp per lower neighbour v = N(u)[j] reads its row once
//            (until the first id >= u) and writes where each chunk's run
//            starts: T[b][j] for b = 0 .. NCH (T[NCH][j] = end of the ids
//            below u).  T lies in the CTA's own scratch, chunk-major, so
//            phase 2 reads it coalesced.
//   phase 2  for every chunk b: each warp takes 32 lower neighbours, lays
//            their runs end to end (a warp prefix sum over the nonempty
//            runs), finds each lane's run from a bitmask of run starts
//            (one OR-reduction per 32 wedges) and increments the counter of
//            each endpoint by a shared-memory atomic that returns the old
//            value c (adding c accumulates sum C(c_w, 2) as in the other
//            4-cycle kernels); then the chunk's counters are cleared.
// Counters are packed 16/16 bits (G_a / G_b) while every degree is below
// 2^16; with larger degrees they are 32/32 bits in 64-bit words and each
// chunk is walked twice, one half of its ids at a time.  A pivot whose table
// (lower neighbours x (NCH + 1)) exceeds the CTA's scratch stays in the dense
// tier (k_bin checks it).
constexpr int CH_THREADS = 1024;

constexpr int CH_UNROLL = 4;
size_t c4_chunk_smem_bytes() { return (size_t)CH_BYTES + (CH_THREADS / 32) * 32 * (4 + 8 + 4); }
int c4_chunk_width(long long n) { return (int)((n + CH_R - 1) / CH_R) + 1; }
long long c4_chunk_cap(long long n) {
    // run-bound entries per CTA: room for lower neighbour counts up to 16,384
    // at this graph's chunk count, between 2^16 and 2^20 entries
    const long long e = (long long)c4_chunk_width(n) * 16384;
    return std::min<long long>(1ll << 20, std::max<long long>(1ll << 16, e));
}
// bytes of one CTA's scratch: T (int32[cap]), row starts (int64[cap / 2]),
// row flags (uint32[cap / 2])

template <bool WIDE>
__device__ __forceinline__ void chunk_walk(const uint32_t* __restrict__ U_col, const int32_t* __restrict__ T,
                                           const long long* __restrict__ rbase, const uint32_t* __restrict__ rflag,
                                           int nlow, int b, uint32_t u, uint32_t lo_id, uint32_t hi_id,
                                           unsigned char* smem, int* w_pre, long long* w_vb, uint32_t* w_fv,
                                           unsigned long long& qa, unsigned long long& qb,
                                           unsigned long long& wedges, bool count_wedges) {
    uint32_t* cnt32 = (uint32_t*)smem;
    unsigned long long* cnt64 = (unsigned long long*)smem;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
    int* cpre = w_pre + warp * 32;
    long long* cvb = w_vb + warp * 32;
    uint32_t* cfv = w_fv + warp * 32;
    const int32_t* Tb = T + (size_t)b * nlow;
    const int32_t* Tn = Tb + nlow;
    for (int j0 = warp * 32; j0 < nlow; j0 += NW * 32) {
        const int j = j0 + lane;
        int len = 0, s = 0;
        if (j < nlow) {
            s = Tb[j];
            len = Tn[j] - s;
        }
        const unsigned ne = __ballot_sync(FULL, len > 0);
        if (!ne) continue;
        int inc = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += y;
        }
        const int total = __shfl_sync(FULL, inc, 31);
        const int k = __popc(ne);
        __syncwarp();
        if (len > 0) {
            // nonempty runs, compacted: run r starts at cpre[r] of the laid-out
            // sequence; its wedge i is U_col[cvb[r] + i]
            const int slot = __popc(ne & lanemask_lt());
            cpre[slot] = inc - len;
            cvb[slot] = rbase[j] + s - (inc - len);
            cfv[slot] = rflag[j];
        }
        __syncwarp();
        const int my_start = lane < k ? cpre[lane] : 0x7FFFFFFF;
        int R = 0;  // run holding position t0 (warp-uniform)
        for (int t0 = 0; t0 < total; t0 += 32 * CH_UNROLL) {
            uint32_t ev[CH_UNROLL], fr[CH_UNROLL];
#pragma unroll
            for (int q = 0; q < CH_UNROLL; q++) {
                const int tb = t0 + q * 32;
                ev[q] = 0xFFFFFFFFu;
                fr[q] = 0;
                if (tb < total) {
                    // starts of runs inside (tb, tb + 32): bit (start - tb)
                    const unsigned bit =
                        (my_start > tb && my_start < tb + 32) ? (1u << (my_start - tb)) : 0u;
                    const unsigned m = __reduce_or_sync(FULL, bit);
                    const int r = R + __popc(m & ((2u << lane) - 1u));
                    const int t = tb + lane;
                    if (t < total) {
                        ev[q] = U_col[cvb[r] + t];
                        fr[q] = cfv[r];
                    }
                    // run holding tb + 32: the last lane's, or the next one if
                    // a run starts exactly there
                    int rn = R + __popc(m);
                    if (rn + 1 < k && cpre[rn + 1] == tb + 32) rn++;
                    R = rn;
                }
            }
#pragma unroll
            for (int q = 0; q < CH_UNROLL; q++) {
                const uint32_t e = ev[q];
                if (e == 0xFFFFFFFFu) continue;
                const uint32_t w = vid(e);
                if (count_wedges) wedges++;
                if (WIDE && (w < lo_id || w >= hi_id)) continue;
                const uint32_t fl = fr[q] & e & (FLAG_A | FLAG_B);
                if (!fl) continue;
                if (WIDE) {
                    const unsigned long long inc2 =
                        ((fl & FLAG_A) ? (1ull << 32) : 0ull) | ((fl & FLAG_B) ? 1ull : 0ull);
                    const unsigned long long old = atomicAdd(&cnt64[w - lo_id], inc2);
                    if (fl & FLAG_A) qa += old >> 32;
                    if (fl & FLAG_B) qb += old & 0xFFFFFFFFull;
                } else {
                    const uint32_t old = atomicAdd(&cnt32[w - lo_id], flag_inc16(fl));
                    if (fl & FLAG_A) qa += old >> 16;
                    if (fl & FLAG_B) qb += old & 0xFFFFu;
                }
            }
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(CH_THREADS, 1) k_c4_chunk(Ctl* c, const int32_t* __restrict__ list,
                                                        const long long* __restrict__ U_off,
                                                        const uint32_t* __restrict__ U_col,
                                                        const int32_t* __restrict__ U_split,
                                                        unsigned char* __restrict__ scratch, long long cap) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char ch_smem[];
    int* w_pre = (int*)(ch_smem + CH_BYTES);
    long long* w_vb = (long long*)(w_pre + CH_THREADS);
    uint32_t* w_fv = (uint32_t*)(w_vb + CH_THREADS);
    __shared__ int s_idx;
    unsigned char* mine = scratch + (size_t)blockIdx.x * c4_chunk_cta_bytes(cap);
    int32_t* T = (int32_t*)mine;
    long long* rbase = (long long*)(mine + (size_t)cap * 4);
    uint32_t* rflag = (uint32_t*)(mine + (size_t)cap * 4 + (size_t)(cap / 2) * 8);
    const bool wide = c->maxdeg >= 65536;
    const int cnt = c->nbin[BIN_C4_CHUNK];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
    unsigned long long qa = 0, qb = 0, wedges = 0;
    uint4* c4 = (uint4*)ch_smem;
    for (int i = threadIdx.x; i < CH_BYTES / 16; i += blockDim.x) c4[i] = make_uint4(0, 0, 0, 0);
    for (;;) {
        if (threadIdx.x == 0) s_idx = (int)atomicAdd(&c->work[WORK_C4_CHUNK], 1u);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= cnt) break;
        const uint32_t u = (uint32_t)list[idx];
        const long long rb = U_off[u];
        const int nlow = U_split[u];
        const int nch = (int)(((long long)u + CH_R - 1) / CH_R);
        // phase 1: run starts of every lower neighbour's row, per chunk
        for (int j = warp; j < nlow; j += NW) {
            const uint32_t fv = U_col[rb + j];
            const uint32_t v = vid(fv);
            const long long vb = U_off[v];
            const int d = (int)(U_off[v + 1] - vb);
            if (lane == 0) {
                rbase[j] = vb;
                rflag[j] = fv;
            }
            int prev = -1;  // chunk of the entry before this step's first
            for (int q0 = 0;; q0 += 32) {
                const int q = q0 + lane;
                int cb = nch;  // past the row, or an id >= u: the end of the runs
                if (q < d) {
                    const uint32_t w = vid(U_col[vb + q]);
                    if (w < u) cb = (int)(w / CH_R);
                }
                int ca = __shfl_up_sync(FULL, cb, 1);
                if (lane == 0) ca = prev;
                for (int bb = ca + 1; bb <= cb; bb++) T[(size_t)bb * nlow + j] = q;
                prev = __shfl_sync(FULL, cb, 31);
                if (prev == nch) break;  // every chunk bound is written
            }
        }
        __syncthreads();
        // phase 2: chunk by chunk
        for (int b = 0; b < nch; b++) {
            const int halves = wide ? 2 : 1;
            for (int h = 0; h < halves; h++) {
                const uint32_t span = wide ? CH_R / 2 : CH_R;
                const uint32_t lo_id = (uint32_t)b * CH_R + h * span;
                const uint32_t hi_id = min(lo_id + span, u);
                if (lo_id >= hi_id) continue;
                if (wide) chunk_walk<true>(U_col, T, rbase, rflag, nlow, b, u, lo_id, hi_id, ch_smem, w_pre, w_vb,
                                           w_fv, qa, qb, wedges, h == 0);
                else chunk_walk<false>(U_col, T, rbase, rflag, nlow, b, u, lo_id, hi_id, ch_smem, w_pre, w_vb,
                                       w_fv, qa, qb, wedges, true);
                __syncthreads();
                // clear the counters this chunk used (16-byte granules)
                const long long granules = ((long long)(hi_id - lo_id) * (wide ? 8 : 4) + 15) / 16;
                for (long long i = threadIdx.x; i < granules; i += blockDim.x) c4[i] = make_uint4(0, 0, 0, 0);
                __syncthreads();
            }
        }
    }
    acc_add(c, 5, qa);
    acc_add(c, 11, qb);
    acc_add(c, 15, wedges);
    acc_add(c, 20, wedges);
}

// Open-addressing insert into a table in global memory.  A slot holds
// (w + 1) << 32 | packed counts, 0 = empty; counts stay below 2^16 because a
// pivot of this tier has fewer than 2^16 lower neighbours.  Returns the
// packed counts before the increment.
// Slot = [epoch 2 | id + 1 30 | G_a count 16 | G_b count 16].  A slot whose
// epoch is not the current one (0: never used) is free: a pivot's keys only
// ever turn free slots into current ones, so linear probing still stops at
// the first free slot, and the entries of the previous pivots need no
// clearing until the epochs wrap.
__device__ __forceinline__ uint32_t ghash_add(unsigned long long* tab, int shift, uint32_t mask, uint32_t w,
                                              uint32_t inc, uint32_t epoch) {
    uint32_t h = (w * 0x9E3779B1u) >> shift;
    const unsigned long long key = (unsigned long long)((w + 1) | (epoch << 30)) << 32;
    for (;;) {
        unsigned long long cur = __ldcg(&tab[h]);  // from L2: slots change only by atomics
        if ((uint32_t)(cur >> 62) != epoch) {
            const unsigned long long got = atomicCAS(&tab[h], cur, key | inc);
            if (got == cur) return 0u;
            cur = got;  // taken meanwhile, by a key of this pivot
        }
        if ((cur & 0xFFFFFFFF00000000ull) == key) return (uint32_t)atomicAdd(&tab[h], (unsigned long long)inc);
        h = (h + 1) & mask;
    }
}

// Medium pivots (C4_T2 < w~ <= t3): one CTA per pivot with its own hash
// table in global memory, sized to the pivot (twice the next power of two of
// w~), so the tables of all CTAs stay small enough for L2.  The wedges are
// dealt in warp-contiguous chunks as in the dense kernel.  A CTA's pivots
// take epochs 1, 2, 3 in turn; the part of the table those three used is
// cleared by a vectorised fill after the third (and at the end), so the
// tables are zero between launches.
__global__ void __launch_bounds__(C4_DENSE_THREADS, 1) k_c4_hash(Ctl* c, const int32_t* __restrict__ list,
                                                             const long long* __restrict__ U_off,
                                                             const uint32_t* __restrict__ U_col,
                                                             const int32_t* __restrict__ U_split,
                                                             unsigned long long* __restrict__ tables,
                                                             long long table_words) {
    pdl_enter();
    unsigned long long* tab = tables + (size_t)blockIdx.x * (size_t)table_words;
    __shared__ int s_idx, s_tot;
    __shared__ unsigned long long s_wt;
    __shared__ int s_pre[C4D_SEG + 1];
    __shared__ long long s_vb[C4D_SEG];
    __shared__ uint32_t s_fv[C4D_SEG];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NW = blockDim.x >> 5;
    const int cnt = c->nbin[BIN_C4_CTA];
    unsigned long long qa = 0, qb = 0, wedges = 0;
    uint32_t epoch = 1;
    int lg_used = 0;  // largest table of the pivots since the last clearing
    uint4* t4 = (uint4*)tab;
    for (;;) {
        if (tid == 0) {
            s_idx = (int)atomicAdd(&c->work[WORK_C4_CTA], 1u);
            s_wt = 0;
        }
        __syncthreads();
        const int idx = s_idx;
        if (idx >= cnt) break;
        const int32_t u = list[idx];
        const long long rb = U_off[u];
        const int nlow = U_split[u];
        unsigned long long wt = 0;
        for (int j = tid; j < nlow; j += blockDim.x) {
            uint32_t v = vid(U_col[rb + j]);
            wt += (unsigned long long)(U_off[v + 1] - U_off[v]);
        }
        wt = warp_sum_u64(wt);
        if (lane == 0 && wt) atomicAdd(&s_wt, wt);
        __syncthreads();
        int lg = 6;
        while ((1ll << lg) < 2 * (long long)s_wt && (1ll << lg) < table_words) lg++;
        const uint32_t mask = (1u << lg) - 1;
        const int shift = 32 - lg;
        for (int s0 = 0; s0 < nlow; s0 += C4D_SEG) {
            const int ns = min(C4D_SEG, nlow - s0);
            wedge_segment_prefix(U_off, U_col, rb, s0, ns, s_pre, s_vb, s_fv, &s_tot);
            const int total = s_tot;
            const int wstep = NW * 32 * C4D_UNROLL;
            for (int base = warp * 32 * C4D_UNROLL; base < total; base += wstep) {
                uint32_t e[C4D_UNROLL], f[C4D_UNROLL];
                int j = find_seg(s_pre, ns, (int)base);
                const int end = min(total, base + 32 * C4D_UNROLL);
                if (j + 1 >= ns || s_pre[j + 1] >= end) {
                    const long long vb = s_vb[j];
                    const uint32_t fv = s_fv[j];
#pragma unroll
                    for (int r = 0; r < C4D_UNROLL; r++) {
                        const int i = base + r * 32 + lane;
                        e[r] = i < total ? U_col[vb + i] : 0xFFFFFFFFu;
                        f[r] = fv;
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < C4D_UNROLL; r++) {
                        const int i = base + r * 32 + lane;
                        e[r] = 0xFFFFFFFFu;
                        f[r] = 0;
                        if (i < total) {
                            while (j + 1 < ns && s_pre[j + 1] <= i) j++;
                            e[r] = U_col[s_vb[j] + i];
                            f[r] = s_fv[j];
                        }
                    }
                }
#pragma unroll
                for (int r = 0; r < C4D_UNROLL; r++) {
                    uint32_t wv = vid(e[r]);
                    if (wv >= (uint32_t)u) continue;
                    wedges++;
                    uint32_t fl = f[r] & e[r] & (FLAG_A | FLAG_B);
                    if (!fl) continue;
                    uint32_t old = ghash_add(tab, shift, mask, wv, flag_inc16(fl), epoch);
                    if (fl & FLAG_A) qa += old >> 16;
                    if (fl & FLAG_B) qb += old & 0xFFFFu;
                }
            }
            __syncthreads();
        }
        lg_used = max(lg_used, lg);
        if (epoch == 3) {
            for (long long i = tid; i < (1ll << lg_used) / 2; i += blockDim.x) t4[i] = make_uint4(0, 0, 0, 0);
            __syncthreads();
            epoch = 1;
            lg_used = 0;
        } else {
            epoch++;
        }
    }
    for (long long i = tid; i < (1ll << lg_used) / 2 && lg_used > 0; i += blockDim.x) t4[i] = make_uint4(0, 0, 0, 0);
    acc_add(c, 5, qa);
    acc_add(c, 11, qb);
    acc_add(c, 15, wedges);
}

// ---- per-edge terms and closed forms ----------------------------------------

__global__ void k_edge_terms(Ctl* c, const int32_t* __restrict__ wlist, const long long* __restrict__ U_off,
                             const uint32_t* __restrict__ U_col, const int32_t* __restrict__ U_split,
                             const unsigned long long* __restrict__ tpack, const int32_t* __restrict__ da,
                             const int32_t* __restrict__ db) {
    pdl_enter();
    int nW = c->nW;
    int lane = threadIdx.x & 31;
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int nwarps = (gridDim.x * blockDim.x) >> 5;
    unsigned long long P[2] = {0, 0}, S[2] = {0, 0}, T[2] = {0, 0}, D[2] = {0, 0}, E[2] = {0, 0}, work = 0;
    unsigned long long T3[2] = {0, 0}, W2[2] = {0, 0};  // sum of t_e; sum of C(d, 2)
    for (int wi = warp; wi < nW; wi += nwarps) {
        int32_t u = wlist[wi];
        long long dau = da[u], dbu = db[u];
        if (lane == 0) {
            S[0] += choose3((unsigned long long)dau);
            S[1] += choose3((unsigned long long)dbu);
            W2[0] += choose2((unsigned long long)dau);
            W2[1] += choose2((unsigned long long)dbu);
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
                T3[0] += (unsigned long long)tt;
                E[0] += 1;
            }
            if (fe & FLAG_B) {
                long long dv = db[v], tt = (long long)(t & 0xFFFFFFFFull);
                P[1] += (unsigned long long)((dbu - 1) * (dv - 1) - tt);
                T[1] += (unsigned long long)(tt * (dbu + dv - 4));
                D[1] += choose2((unsigned long long)tt);
                T3[1] += (unsigned long long)tt;
                E[1] += 1;
            }
        }
    }
#pragma unroll
    for (int g = 0; g < 2; g++) {
        P[g] = warp_sum_u64(P[g]);
        S[g] = warp_sum_u64(S[g]);
        T3[g] = warp_sum_u64(T3[g]);
        W2[g] = warp_sum_u64(W2[g]);
        T[g] = warp_sum_u64(T[g]);
        D[g] = warp_sum_u64(D[g]);
        E[g] = warp_sum_u64(E[g]);
    }
    for (int g = 0; g < 2; g++) {
        const int o = 6 * g;
        acc_add_warp(c, o + 0, P[g]);
        acc_add_warp(c, o + 1, S[g]);
        acc_add_warp(c, o + 2, T[g]);
        acc_add_warp(c, o + 3, D[g]);
        acc_add_warp(c, 12 + g, E[g]);
        acc_add_warp(c, 16 + g, T3[g]);
        acc_add_warp(c, 18 + g, W2[g]);
    }
    acc_add(c, 14, work);
}

// mode 0: batch (F += C_a - C_b unless the batch was rejected); 1: static
__global__ void k_finalize(Ctl* c, int mode) {
    pdl_enter();
    // fold the striped accumulators (one warp: lane i sums slot i's copies
    // and slot i + 16's if any)
    if (blockIdx.x == 0 && threadIdx.x < NACC) {
        unsigned long long x = 0;
        for (int k = 0; k < ACC_STRIPES; k++) x += c->accs[threadIdx.x][k];
        c->acc[threadIdx.x] += x;
    }
    __syncwarp();
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
    // mode 0: committed batch, F += C_a - C_b; mode 2: independent batch,
    // the result is F + C_a - C_b and F stays; mode 1: static count; mode 3:
    // a committed batch whose pass covered every vertex, so C_a and C_b are
    // the whole graph's counts after and before it: F = C_a, and C_b is the
    // result of the batch before it (committed without a count of its own);
    // mode 4: see below
    const bool ok = c->err == 0 && c->active;
    for (int i = 0; i < 6; i++) {
        unsigned long long d = (unsigned long long)(c->Ca[i] - c->Cb[i]);
        if (mode == 0 && ok) c->F[i] += d;
        if (mode == 3 && ok) {
            c->prev_out[i] = (unsigned long long)c->Cb[i];
            c->F[i] = (unsigned long long)c->Ca[i];
        }
        c->last_out[i] = mode == 2 ? c->F[i] + d : c->F[i];
        // mode 4: two independent batches counted over every vertex (the
        // twin pass): C_a and C_b are the whole graph's counts with the
        // first and with the second batch applied; F stays
        if (mode == 4) {
            c->last_out[i] = (unsigned long long)c->Ca[i];
            c->prev_out[i] = (unsigned long long)c->Cb[i];
        }
    }
    // 3-vertex graphlets from the same sums: triangles = (sum t_e) / 3,
    // induced 2-paths = sum C(d, 2) - 3 triangles
    for (int g = 0; g < 2; g++) {
        long long* C3 = g == 0 ? c->C3a : c->C3b;
        const unsigned long long t3 = c->acc[16 + g], w2 = c->acc[18 + g];
        C3[0] = (long long)(w2 - t3);
        C3[1] = (long long)(t3 / 3);
    }
    for (int i = 0; i < 2; i++) {
        unsigned long long d = (unsigned long long)(c->C3a[i] - c->C3b[i]);
        if (mode == 0 && ok) c->F3[i] += d;
        if (mode == 3 && ok) c->F3[i] = (unsigned long long)c->C3a[i];
        c->last_out3[i] = mode == 2 ? c->F3[i] + d : c->F3[i];
    }
}

}  // namespace gcx

// ---- launch sequence of one counting pass -------------------------------------

namespace gcx {

void count_setup_attributes() {
    cudaFuncSetAttribute(k_tri_block<TRI_KM, BIN_TRI_BLOCK, WORK_TRI_BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tri_block_smem<TRI_KM>());
    cudaFuncSetAttribute(k_tri_block<TRI_KS, BIN_TRI_SMALL, WORK_TRI_SMALL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tri_block_smem<TRI_KS>());
    cudaFuncSetAttribute(k_c4_block<C4B_SMALL_LG, C4B_SMALL_THREADS, BIN_C4_BSMALL, WORK_C4_BSMALL, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)c4_block_smem<C4B_SMALL_LG, C4B_SMALL_THREADS>());
    cudaFuncSetAttribute(k_c4_block<C4B_BIG_LG, C4B_BIG_THREADS, BIN_C4_BLOCK, WORK_C4_BLOCK, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)c4_block_smem<C4B_BIG_LG, C4B_BIG_THREADS>());
    cudaFuncSetAttribute(k_c4_dense_t<true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(k_c4_chunk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c4_chunk_smem_bytes());
}

// Cluster size of the heavy 4-cycle kernel: the one that keeps the most
// CTAs resident (8-CTA clusters fill all 152 SMs of a GB300, 16-CTA ones
// only 112), unless the caller asks for a size.
int dense_cluster_plan(int want, int sms, int* size_out) {
    int best_size = 8, best_active = 0;
    const int sizes[2] = {8, 16};
    for (int i = 0; i < 2; i++) {
        int cs = sizes[i];
        if (want && want != cs) continue;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cs * std::max(1, sms / cs));
        cfg.blockDim = dim3(C4_DENSE_THREADS);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int active = 0;
        if (cudaOccupancyMaxActiveClusters(&active, k_c4_dense_t<true>, &cfg) != cudaSuccess) {
            cudaGetLastError();
            active = 0;
        }
        active = std::min(active, std::max(1, sms / cs));
        if (active * cs > best_active * best_size) {
            best_size = cs;
            best_active = active;
        }
    }
    *size_out = best_size;
    return best_active > 0 ? best_active : std::max(1, sms / best_size);
}

// The caller's bin boundaries, clamped to what the kernels and the scratch
// of this pass can take.
Tuning effective_tuning(const CountArgs& a) {
    Tuning t = a.tune;
    t.tri_warp_max = std::max(1, std::min(t.tri_warp_max, 32));
    t.tri_small_max = std::max(t.tri_warp_max, std::min(t.tri_small_max, TRI_KS));
    t.tri_block_max = std::max(t.tri_small_max, std::min(t.tri_block_max, TRI_KM));
    t.c4_reg_max = std::max(1, std::min(t.c4_reg_max, 32));
    t.c4_warp_max = std::max(t.c4_reg_max, std::min(t.c4_warp_max, C4_T1));
    t.c4_block_max = std::max(t.c4_warp_max, std::min(t.c4_block_max, C4_T2));
    t.c4_cta_max = std::max<long long>(t.c4_block_max, std::min<long long>(t.c4_cta_max, a.cta_table_words / 2));
    if (!a.chunk_scratch || a.chunk_cap <= 0 || t.c4_chunk_min <= 0) t.c4_chunk_min = NEVER;
    t.c4_chunk_min = std::max<long long>(t.c4_chunk_min, t.c4_cta_max);
    if (t.c4_chunk_max <= 0) t.c4_chunk_max = NEVER;
    if (t.c4_chunk_max <= t.c4_chunk_min) t.c4_chunk_min = NEVER;  // empty chunked bin
    return t;
}

int enqueue_counting(const CountArgs& a, cudaStream_t s, cudaEvent_t ev_tri, cudaEvent_t ev_c4, cudaEvent_t ev_end,
                     int mode) {
    const int sms = a.sms;
    int nl = 0;
    auto lists = [&](int b) { return a.bins + (size_t)b * a.n_alloc; };
    long long nw = a.n_alloc > 0 ? a.n_alloc : 1;
    int gb = (int)std::min<long long>((nw + 255) / 256, 8LL * sms);
    const Tuning t = effective_tuning(a);
    pdl_launch(k_wedge_bound, dim3(8 * sms), dim3(256), 0, s, a.ctl, a.wlist, a.U_off, a.U_col, a.U_split, a.U_wt);
    pdl_launch(k_bin, dim3(gb), dim3(256), 0, s, a.ctl, a.wlist, a.U_off, a.U_split, a.U_wt, a.bins, a.n_alloc, t,
               t.c4_chunk_min < NEVER ? a.chunk_cap : 0ll);
    nl += 2;
    // The triangle kernels and the 4-cycle tiers are independent: with
    // auxiliary streams they run side by side (a fork after the binning, a
    // join before the edge terms), which fills the GPU when each tier alone
    // has little work.  ev_tri marks the fork, ev_c4 the end of the triangle
    // branch, ev_end the end of the 4-cycle branches.
    const bool par = a.aux[0] && a.aux[1] && a.aux[2];
    cudaStream_t sT = par ? a.aux[0] : s, sC1 = par ? a.aux[1] : s, sC2 = par ? a.aux[2] : s;
    if (ev_tri) record_stage(ev_tri, s);
    if (par) {
        cudaEventRecord(a.fork, s);
        for (int i = 0; i < 3; i++) cudaStreamWaitEvent(a.aux[i], a.fork, 0);
    }
    k_tri_warp<<<4 * sms, TW * 32, 0, sT>>>(a.ctl, lists(BIN_TRI_WARP), a.U_off, a.U_col, a.U_split, a.tpack);
    k_tri_block<TRI_KS, BIN_TRI_SMALL, WORK_TRI_SMALL><<<8 * sms, 256, tri_block_smem<TRI_KS>(), sT>>>(
        a.ctl, lists(BIN_TRI_SMALL), a.U_off, a.U_col, a.U_split, a.tpack);
    k_tri_block<TRI_KM, BIN_TRI_BLOCK, WORK_TRI_BLOCK><<<2 * sms, 256, tri_block_smem<TRI_KM>(), sT>>>(
        a.ctl, lists(BIN_TRI_BLOCK), a.U_off, a.U_col, a.U_split, a.tpack);
    k_tri_merge<<<sms, 256, 0, sT>>>(a.ctl, lists(BIN_TRI_MERGE), a.U_off, a.U_col, a.U_split, a.tpack);
    nl += 4;
    if (ev_c4) record_stage(ev_c4, sT);
    k_c4_reg<<<4 * sms, 256, 0, sC1>>>(a.ctl, lists(BIN_C4_REG), a.U_off, a.U_col, a.U_split);
    k_c4_warp<<<7 * sms, C4W_WARPS * 32, 0, sC1>>>(a.ctl, lists(BIN_C4_WARP), a.U_off, a.U_col, a.U_split,
                                                   a.U_wt);
    k_c4_block<C4B_SMALL_LG, C4B_SMALL_THREADS, BIN_C4_BSMALL, WORK_C4_BSMALL, false>
        <<<6 * sms, C4B_SMALL_THREADS, c4_block_smem<C4B_SMALL_LG, C4B_SMALL_THREADS>(), sC1>>>(
            a.ctl, lists(BIN_C4_BSMALL), a.U_off, a.U_col, a.U_split, a.U_wt);
    k_c4_block<C4B_BIG_LG, C4B_BIG_THREADS, BIN_C4_BLOCK, WORK_C4_BLOCK, true>
        <<<sms, C4B_BIG_THREADS, c4_block_smem<C4B_BIG_LG, C4B_BIG_THREADS>(), sC1>>>(
            a.ctl, lists(BIN_C4_BLOCK), a.U_off, a.U_col, a.U_split, a.U_wt);
    if (a.ev_heavy[0]) record_stage(a.ev_heavy[0], sC2);
    {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(a.dense_cluster_size * a.dense_clusters);
        cfg.blockDim = dim3(C4_DENSE_THREADS);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = sC2;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = a.dense_cluster_size;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaLaunchKernelEx(&cfg, k_c4_dense_t<true>, a.ctl, (const int32_t*)lists(BIN_C4_DENSE),
                           (const long long*)a.U_off, (const uint32_t*)a.U_col, (const int32_t*)a.U_split,
                           (const long long*)a.U_wt, a.dense, a.n_alloc);
    }
    if (t.c4_chunk_min < NEVER) {
        k_c4_chunk<<<sms, CH_THREADS, c4_chunk_smem_bytes(), sC2>>>(a.ctl, lists(BIN_C4_CHUNK), a.U_off, a.U_col,
                                                                    a.U_split, a.chunk_scratch, a.chunk_cap);
        nl += 1;
    }
    if (a.ev_heavy[1]) record_stage(a.ev_heavy[1], sC2);
    k_c4_hash<<<a.cta_groups, C4_DENSE_THREADS, 0, s>>>(a.ctl, lists(BIN_C4_CTA), a.U_off, a.U_col, a.U_split,
                                                        a.cta_tables, a.cta_table_words);
    nl += 5;
    if (par) {
        cudaEventRecord(a.join[1], sC1);
        cudaEventRecord(a.join[2], sC2);
        cudaStreamWaitEvent(s, a.join[1], 0);
        cudaStreamWaitEvent(s, a.join[2], 0);
    }
    if (ev_end) record_stage(ev_end, s);
    if (par) {
        cudaEventRecord(a.join[0], sT);
        cudaStreamWaitEvent(s, a.join[0], 0);
    }
    k_edge_terms<<<8 * sms, 256, 0, s>>>(a.ctl, a.wlist, a.U_off, a.U_col, a.U_split, a.tpack, a.da, a.db);
    pdl_launch(k_finalize, dim3(1), dim3(32), 0, s, a.ctl, mode);
    nl += 2;
    return nl;
}

}  // namespace gcx
