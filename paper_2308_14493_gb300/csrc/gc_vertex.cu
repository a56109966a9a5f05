// gc_vertex.cu -- per-vertex (local) graphlet counts of the current graph:
// for every vertex v, how many induced connected 4-vertex graphlets hold v
// in each orbit 4..14 (3-path end, middle; 3-star leaf, centre; 4-cycle;
// tailed triangle tail end, other corner, attachment; diamond degree-2,
// degree-3 corner; 4-clique), and their sums per graphlet [g1..g6].
//
// The containment identity behind the global counts (Sec. 3, PGD's closed
// forms) holds per vertex and role: a 4-set S of induced type g holding v
// in orbit o contains a fixed number of copies of each subgraph H with v
// in role r, so the non-induced role counts are N_r(v) = sum_o M[r][o]
// I_o(v), M triangular.  The role counts (d degrees, t_e triangles per
// edge, tri(v) = T2[v] / 2, s(u) = sum_{w in N(u)} (d_w - 1)):
//   3-path   end sum_{u in N(v)} (s(u) - (d_v - 1)) - 2 tri(v);
//            middle sum_{u in N(v)} ((d_v - 1)(d_u - 1) - t_vu)
//   3-star   leaf sum_{u in N(v)} C(d_u - 1, 2); centre C(d_v, 3)
//   4-cycle  counted once at its highest vertex u with opposite corner w:
//            c_w = common lower neighbours, C(c_w, 2) cycles credit u and
//            w, and each middle vertex a of a wedge u-a-w gets c_w - 1
//   tailed triangle  tail end sum_z (tri(z) - t_vz); other corner
//            sum_y t_vy (d_y - 2); attachment tri(v)(d_v - 2)
//   diamond  degree-2 corner: for each triangle {v, a, b}, t_ab - 1;
//            degree-3 corner sum_u C(t_vu, 2)
//   4-clique listed once (oriented), each of its four vertices credited
// NV[v] holds the eleven role counts in orbit order.  The input is the
// union graph U of a static count (both flags on every entry, t of each
// out-entry in tpack, T2 filled, w~ per pivot in U_wt).
//
// The second half of the file gives the same per edge (ten edge orbits,
// k_e_*), and the 4-cycle walk of the heavy pivots shared by both
// (k_c4_group: a few pivots at a time over the whole grid, their counters
// resident in L2).
#include "gc_internal.cuh"
#include "gc_kernels.cuh"

namespace gcx {

// role slots of NV, in orbit order 4..14
enum { R_PEND, R_PMID, R_SLEAF, R_SCTR, R_C4, R_TTAIL, R_TOTH, R_TATT, R_D2, R_D3, R_K4, NROLE };
// per-entry credit slots of the per-edge counts (the two entries of an edge are added at the end)
enum { E_OPP, E_OUTER, E_C4, E_K4, NEROLE };

// t of every entry (out-entries carry it; an in-entry reads its twin).
__global__ void k_v_tsym(const Ctl* c, const int32_t* __restrict__ wlist, const long long* __restrict__ U_off,
                         const uint32_t* __restrict__ U_col, const int32_t* __restrict__ U_split,
                         const unsigned long long* __restrict__ tpack, uint32_t* __restrict__ tall) {
    pdl_enter();
    const int nW = c->nW;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < nW; i += nwarps) {
        const uint32_t u = (uint32_t)wlist[i];
        for (long long e = U_off[u] + U_split[u] + lane; e < U_off[u + 1]; e += 32) {
            const uint32_t t = (uint32_t)(tpack[e] >> 32);
            const uint32_t v = vid(U_col[e]);
            tall[e] = t;
            const long long vb = U_off[v];
            tall[vb + lower_bound_id(U_col + vb, U_split[v], u)] = t;
        }
    }
}

// s(u) = sum over the neighbours w of (d_w - 1)
__global__ void k_v_s(const Ctl* c, const int32_t* __restrict__ wlist, const long long* __restrict__ U_off,
                      const uint32_t* __restrict__ U_col, long long* __restrict__ sdeg) {
    pdl_enter();
    const int nW = c->nW;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < nW; i += nwarps) {
        const uint32_t u = (uint32_t)wlist[i];
        long long sum = 0;
        for (long long e = U_off[u] + lane; e < U_off[u + 1]; e += 32) {
            const uint32_t w = vid(U_col[e]);
            sum += U_off[w + 1] - U_off[w] - 1;
        }
        sum = (long long)warp_sum_u64((unsigned long long)sum);
        if (lane == 0) sdeg[u] = sum;
    }
}

// The row terms of each vertex: 3-path end and middle, 3-star leaf and
// centre, tailed triangle tail end, other corner and attachment, diamond
// degree-3 corner.
__global__ void k_v_terms(const Ctl* c, const int32_t* __restrict__ wlist, const long long* __restrict__ U_off,
                          const uint32_t* __restrict__ U_col, const uint32_t* __restrict__ tall,
                          const long long* __restrict__ sdeg, const unsigned long long* __restrict__ T2,
                          long long* __restrict__ NV) {
    pdl_enter();
    const int nW = c->nW;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < nW; i += nwarps) {
        const uint32_t v = (uint32_t)wlist[i];
        const long long rb = U_off[v], re = U_off[v + 1];
        const long long d = re - rb, trv = (long long)(T2[v] / 2);
        long long pe = 0, pm = 0, sl = 0, tl = 0, to = 0, d3 = 0;
        for (long long e = rb + lane; e < re; e += 32) {
            const uint32_t u = vid(U_col[e]);
            const long long du = U_off[u + 1] - U_off[u], t = tall[e];
            pe += sdeg[u] - (d - 1);
            pm += (d - 1) * (du - 1) - t;
            sl += (du - 1) * (du - 2) / 2;
            tl += (long long)(T2[u] / 2) - t;
            to += t * (du - 2);
            d3 += t * (t - 1) / 2;
        }
        pe = (long long)warp_sum_u64((unsigned long long)pe);
        pm = (long long)warp_sum_u64((unsigned long long)pm);
        sl = (long long)warp_sum_u64((unsigned long long)sl);
        tl = (long long)warp_sum_u64((unsigned long long)tl);
        to = (long long)warp_sum_u64((unsigned long long)to);
        d3 = (long long)warp_sum_u64((unsigned long long)d3);
        if (lane == 0) {
            long long* o = NV + NROLE * (size_t)v;
            o[R_PEND] += pe - 2 * trv;
            o[R_PMID] += pm;
            o[R_SLEAF] += sl;
            o[R_SCTR] += d * (d - 1) * (d - 2) / 6;
            o[R_TTAIL] += tl;
            o[R_TOTH] += to;
            o[R_TATT] += trv * (d - 2);
            o[R_D3] += d3;
        }
    }
}

// Triangles u < v < y (each once): the degree-2 corner part of the
// diamonds (t of the opposite edge - 1 to each corner); 4-cliques
// u < v < y < z (each once) credited to their four vertices.  A warp per
// root u, a lane per out-edge (out-lists are short in the degree order).
__global__ void k_v_tri_k4(const Ctl* c, const int32_t* __restrict__ wlist, const long long* __restrict__ U_off,
                           const uint32_t* __restrict__ U_col, const int32_t* __restrict__ U_split,
                           const uint32_t* __restrict__ tall, long long* __restrict__ NV) {
    pdl_enter();
    const int nW = c->nW;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int wi = warp; wi < nW; wi += nwarps) {
        const uint32_t u = (uint32_t)wlist[wi];
        const long long ob = U_off[u] + U_split[u], oe = U_off[u + 1];
        for (long long e = ob + lane; e < oe; e += 32) {
            const uint32_t v = vid(U_col[e]);
            const long long vb = U_off[v] + U_split[v], ve = U_off[v + 1];
            long long i = e + 1, j = vb;
            long long k4u = 0;
            while (i < oe && j < ve) {
                const uint32_t x = vid(U_col[i]), y = vid(U_col[j]);
                if (x < y) {
                    i++;
                } else if (x > y) {
                    j++;
                } else {
                    // triangle (u, v, y): t of uv, uy, vy at e, i, j
                    atomicAdd((unsigned long long*)&NV[NROLE * (size_t)u + R_D2],
                              (unsigned long long)((long long)tall[j] - 1));
                    atomicAdd((unsigned long long*)&NV[NROLE * (size_t)v + R_D2],
                              (unsigned long long)((long long)tall[i] - 1));
                    atomicAdd((unsigned long long*)&NV[NROLE * (size_t)y + R_D2],
                              (unsigned long long)((long long)tall[e] - 1));
                    // 4-cliques (u, v, y, z), z > y in N+(u), N+(v), N+(y)
                    const long long yb = U_off[y] + U_split[y], ye = U_off[y + 1];
                    long long p = i + 1, q = j + 1, r = yb, kk = 0;
                    while (p < oe && q < ve && r < ye) {
                        const uint32_t a = vid(U_col[p]), b = vid(U_col[q]), cc = vid(U_col[r]);
                        const uint32_t mx = max(a, max(b, cc));
                        if (a == mx && b == mx && cc == mx) {
                            atomicAdd((unsigned long long*)&NV[NROLE * (size_t)a + R_K4], 1ull);
                            kk++;
                            p++;
                            q++;
                            r++;
                        } else {
                            if (a < mx) p++;
                            if (b < mx) q++;
                            if (cc < mx) r++;
                        }
                    }
                    if (kk) {
                        atomicAdd((unsigned long long*)&NV[NROLE * (size_t)v + R_K4], (unsigned long long)kk);
                        atomicAdd((unsigned long long*)&NV[NROLE * (size_t)y + R_K4], (unsigned long long)kk);
                        k4u += kk;
                    }
                    i++;
                    j++;
                }
            }
            if (k4u) atomicAdd((unsigned long long*)&NV[NROLE * (size_t)u + R_K4], (unsigned long long)k4u);
        }
    }
}

// 4-cycles, a block per pivot u (its highest vertex) with one dense counter
// array of n words per block: walk 1 counts c_w over the wedges u-a-w
// (a, w below u), walk 2 credits each middle a with c_w - 1, walk 3 takes
// and clears c_w, crediting w and u with C(c_w, 2).
__global__ void __launch_bounds__(1024) k_v_c4(const Ctl* c, const int32_t* __restrict__ wlist,
                                               const long long* __restrict__ U_off,
                                               const uint32_t* __restrict__ U_col,
                                               const int32_t* __restrict__ U_split, uint32_t* __restrict__ cnt_all,
                                               int n, const uint8_t* __restrict__ heavy,
                                               long long* __restrict__ NV) {
    pdl_enter();
    const int nW = c->nW;
    uint32_t* cnt = cnt_all + (size_t)blockIdx.x * (size_t)n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NWp = blockDim.x >> 5;
    __shared__ unsigned long long s_u[32];
    for (int pi = blockIdx.x; pi < nW; pi += gridDim.x) {
        const uint32_t u = (uint32_t)wlist[pi];
        if (heavy && heavy[u]) continue;  // taken by k_c4_group (same for the whole block)
        const long long rb = U_off[u];
        const int nlow = U_split[u];
        unsigned long long usum = 0;
        for (int pass = 0; pass < 3; pass++) {
            for (int j = warp; j < nlow; j += NWp) {
                const uint32_t a = vid(U_col[rb + j]);
                const long long ab = U_off[a], ae = U_off[a + 1];
                long long asum = 0;
                for (long long q = ab + lane; q < ae; q += 32) {
                    const uint32_t w = vid(U_col[q]);
                    if (w >= u) break;  // rows are sorted: the rest is above u
                    if (pass == 0) {
                        atomicAdd(&cnt[w], 1u);
                    } else if (pass == 1) {
                        asum += (long long)__ldcg(&cnt[w]) - 1;
                    } else {
                        const uint32_t old = atomicExch(&cnt[w], 0u);
                        if (old >= 2) {
                            const unsigned long long cy = (unsigned long long)old * (old - 1) / 2;
                            atomicAdd((unsigned long long*)&NV[NROLE * (size_t)w + R_C4], cy);
                            usum += cy;
                        }
                    }
                }
                if (pass == 1) {
                    asum = (long long)warp_sum_u64((unsigned long long)asum);
                    if (lane == 0 && asum) atomicAdd((unsigned long long*)&NV[NROLE * (size_t)a + R_C4],
                        (unsigned long long)asum);
                }
            }
            __threadfence();
            __syncthreads();
        }
        usum = warp_sum_u64(usum);
        if (lane == 0) s_u[warp] = usum;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long t = 0;
            for (int w = 0; w < NWp; w++) t += s_u[w];
            if (t) atomicAdd((unsigned long long*)&NV[NROLE * (size_t)u + R_C4], t);  // other blocks credit u too
        }
        __syncthreads();
    }
}

// Heavy 4-cycle pivots of the local counts: w~(u) (the sum of the degrees
// of u's lower neighbours, from the static pass) at least heavy_min.  They
// are listed for k_c4_group and flagged so that the per-block walk skips
// them.
__global__ void k_c4_heavy_mark(const Ctl* c, const int32_t* __restrict__ wlist, const long long* __restrict__ U_wt,
                                long long heavy_min, uint8_t* __restrict__ heavy, int32_t* __restrict__ hlist,
                                int* __restrict__ hcount) {
    pdl_enter();
    const int nW = c->nW;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nW; i += gridDim.x * blockDim.x) {
        const int32_t u = wlist[i];
        const bool h = U_wt[u] >= heavy_min;
        heavy[u] = h ? 1 : 0;
        if (h) hlist[atomicAdd(hcount, 1)] = u;
    }
}

// One walk of the 4-cycle counting for up to C4G heavy pivots at once
// (hlist[first .. first + count)), each with its own dense counter array of
// n words (C4G arrays of 4 n bytes stay resident in L2 on graphs of a few
// million vertices).  The whole grid shares the work: the (pivot, lower
// neighbour a) pairs of the group are numbered and dealt to warps, the
// lanes of a warp walk a's row below the pivot.  The three walks are three
// launches (pass 0 count c_w, 1 credit c_w - 1, 2 clear), so the kernel
// boundary is the only barrier between them.  EDGE: credits go to the two
// entries of each wedge (per-edge 4-cycle role), else to the middle vertex
// a in pass 1 and to the corners w and u with C(c_w, 2) in pass 2.
template <bool EDGE>
__global__ void k_c4_group(const int32_t* __restrict__ hlist, int first, int count,
                           const long long* __restrict__ U_off, const uint32_t* __restrict__ U_col,
                           const int32_t* __restrict__ U_split, uint32_t* __restrict__ cnt_g, int n, int pass,
                           long long* __restrict__ acc) {
    pdl_enter();
    const int lane = threadIdx.x & 31;
    const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    // lane p < count holds slot p: its pivot and the inclusive prefix of the
    // lower-neighbour counts
    uint32_t up = 0;
    long long nl = 0;
    if (lane < count) {
        up = (uint32_t)hlist[first + lane];
        nl = U_split[up];
    }
    long long incl = nl;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    const long long total = __shfl_sync(FULL, incl, 31);
    const long long excl = incl - nl;
    for (long long k = gwarp; k < total; k += nwarps) {
        const int p = __popc(__ballot_sync(FULL, incl <= k));  // the slot holding pair k
        const uint32_t u = __shfl_sync(FULL, up, p);
        const long long j = k - __shfl_sync(FULL, excl, p);
        uint32_t* cnt = cnt_g + (size_t)p * (size_t)n;
        const long long ea = U_off[u] + j;  // entry (u, a)
        const uint32_t a = vid(U_col[ea]);
        const long long ab = U_off[a], ae = U_off[a + 1];
        long long asum = 0;
        unsigned long long usum = 0;
        for (long long q = ab + lane; q < ae; q += 32) {
            const uint32_t w = vid(U_col[q]);
            if (w >= u) break;  // rows are sorted: the rest is above u
            if (pass == 0) {
                atomicAdd(&cnt[w], 1u);
            } else if (pass == 1) {
                const long long x = (long long)__ldcg(&cnt[w]) - 1;
                if (x > 0) {
                    if (EDGE) atomicAdd((unsigned long long*)&acc[NEROLE * (size_t)q + E_C4], (unsigned long long)x);
                    asum += x;
                }
            } else if (EDGE) {
                cnt[w] = 0u;
            } else {
                const uint32_t old = atomicExch(&cnt[w], 0u);
                if (old >= 2) {
                    const unsigned long long cy = (unsigned long long)old * (old - 1) / 2;
                    atomicAdd((unsigned long long*)&acc[NROLE * (size_t)w + R_C4], cy);
                    usum += cy;
                }
            }
        }
        if (pass == 1) {
            asum = (long long)warp_sum_u64((unsigned long long)asum);
            if (lane == 0 && asum) {
                if (EDGE) atomicAdd((unsigned long long*)&acc[NEROLE * (size_t)ea + E_C4], (unsigned long long)asum);
                else atomicAdd((unsigned long long*)&acc[NROLE * (size_t)a + R_C4], (unsigned long long)asum);
            }
        } else if (pass == 2 && !EDGE) {
            usum = warp_sum_u64(usum);
            if (lane == 0 && usum) atomicAdd((unsigned long long*)&acc[NROLE * (size_t)u + R_C4], usum);
        }
    }
}

// The heavy pivots: mark them, read their number back, then three launches
// per group of C4G.  Returns the launches made, or -1 on a CUDA error.
template <bool EDGE>
static int enqueue_heavy_c4(const HeavyC4& h, Ctl* ctl, const int32_t* wlist, const long long* U_off,
                            const uint32_t* U_col, const int32_t* U_split, int n, int sms, long long* acc,
                            cudaStream_t s) {
    if (h.heavy_min <= 0) return 0;
    int nl = 0;
    if (cudaMemsetAsync(h.hcount, 0, sizeof(int), s) != cudaSuccess) return -1;
    pdl_launch(k_c4_heavy_mark, dim3(std::max(1, std::min(8 * sms, (n + 255) / 256))), dim3(256), 0, s, ctl, wlist,
               h.U_wt, h.heavy_min, h.heavy, h.hlist, h.hcount);
    nl++;
    int H = 0;
    if (cudaMemcpyAsync(&H, h.hcount, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return -1;
    for (int first = 0; first < H; first += C4G) {
        const int cnt = std::min(C4G, H - first);
        for (int pass = 0; pass < 3; pass++) {
            pdl_launch(k_c4_group<EDGE>, dim3(8 * sms), dim3(256), 0, s, (const int32_t*)h.hlist, first, cnt, U_off,
                       U_col, U_split, h.cnt_g, n, pass, acc);
            nl++;
        }
    }
    return nl;
}

// Orbit counts per vertex by the triangular role containment; out[k v + j]
// by external id: the eleven orbits (k = 11) or their sums per graphlet
// (k = 6).
__global__ void k_v_finalize(const long long* __restrict__ NV, int n, const int32_t* __restrict__ iperm, int k,
                             unsigned long long* __restrict__ out) {
    pdl_enter();
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const long long* r = NV + NROLE * (size_t)v;
        const long long o14 = r[R_K4];
        const long long o13 = r[R_D3] - 3 * o14;
        const long long o12 = r[R_D2] - 3 * o14;
        const long long o11 = r[R_TATT] - 2 * o13 - 3 * o14;
        const long long o10 = r[R_TOTH] - 2 * o12 - 2 * o13 - 6 * o14;
        const long long o9 = r[R_TTAIL] - 2 * o12 - 3 * o14;
        const long long o8 = r[R_C4] - o12 - o13 - 3 * o14;
        const long long o7 = r[R_SCTR] - o11 - o13 - o14;
        const long long o6 = r[R_SLEAF] - o9 - o10 - 2 * o12 - o13 - 3 * o14;
        const long long o5 = r[R_PMID] - 2 * o8 - o10 - 2 * o11 - 2 * o12 - 4 * o13 - 6 * o14;
        const long long o4 = r[R_PEND] - 2 * o8 - 2 * o9 - o10 - 4 * o12 - 2 * o13 - 6 * o14;
        unsigned long long* o = out + (size_t)k * iperm[v];
        if (k == 11) {
            const long long orb[11] = {o4, o5, o6, o7, o8, o9, o10, o11, o12, o13, o14};
            for (int j = 0; j < 11; j++) o[j] = (unsigned long long)orb[j];
        } else {
            o[0] = (unsigned long long)(o4 + o5);
            o[1] = (unsigned long long)(o6 + o7);
            o[2] = (unsigned long long)o8;
            o[3] = (unsigned long long)(o9 + o10 + o11);
            o[4] = (unsigned long long)(o12 + o13);
            o[5] = (unsigned long long)o14;
        }
    }
}

// ---------------------------------------------------------------------
// Per-edge (local) counts.  The same containment identity holds per edge
// {u, v} and edge role, with the edge orbits 0..9 (3-path end, middle
// edge; 3-star edge; 4-cycle edge; tailed triangle tail, triangle edge
// opposite the attachment, triangle edge at the attachment; diamond outer
// edge, chord; 4-clique edge).  The non-induced role counts of the edge
// (tri(x) = T2[x] / 2, s(x) = sum_{w in N(x)} (d_w - 1)):
//   3-path end   (s(v) - (d_u - 1) - t) + (s(u) - (d_v - 1) - t)
//   3-path middle (d_u - 1)(d_v - 1) - t;  3-star C(d_u - 1, 2) + C(d_v - 1, 2)
//   4-cycle      credited by the pivot walk below
//   tail         (tri(u) - t) + (tri(v) - t);  attachment t (d_u + d_v - 4)
//   opposite     sum over triangles {u, v, w} of d_w - 2
//   diamond outer  sum over triangles {u, v, w} of t_uw + t_vw - 2
//   chord C(t, 2);  4-clique credited by the clique listing
// Credits land on either entry of the edge; the finalize adds both.

// One sort key per entry: the out-entry (x < y) of an edge gets its
// external pair (lo << nb) | hi, every in-entry the largest nb-bit pair,
// so after the sort the first m keys are the edges in external order.
__global__ void k_e_keys(const Ctl* c, const int32_t* __restrict__ wlist, const long long* __restrict__ U_off,
                         const uint32_t* __restrict__ U_col, const int32_t* __restrict__ U_split,
                         const int32_t* __restrict__ iperm, int nb, unsigned long long* __restrict__ keys) {
    pdl_enter();
    const int nW = c->nW;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const unsigned long long none = (1ull << (2 * nb)) - 1;
    for (int i = warp; i < nW; i += nwarps) {
        const uint32_t u = (uint32_t)wlist[i];
        const long long ob = U_off[u] + U_split[u];
        const unsigned long long a = (unsigned long long)iperm[u];
        for (long long e = U_off[u] + lane; e < U_off[u + 1]; e += 32) {
            if (e < ob) {
                keys[e] = none;
            } else {
                const unsigned long long b = (unsigned long long)iperm[vid(U_col[e])];
                keys[e] = a < b ? (a << nb) | b : (b << nb) | a;
            }
        }
    }
}

// Triangles u < v < y (each once) credit the opposite and diamond-outer
// terms of their three edges; 4-cliques u < v < y < z (each once) credit
// their six edges.  A warp per root u, a lane per out-edge e = (u, v).
__global__ void k_e_tri_k4(const Ctl* c, const int32_t* __restrict__ wlist, const long long* __restrict__ U_off,
                           const uint32_t* __restrict__ U_col, const int32_t* __restrict__ U_split,
                           const uint32_t* __restrict__ tall, long long* __restrict__ NE) {
    pdl_enter();
    const int nW = c->nW;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int wi = warp; wi < nW; wi += nwarps) {
        const uint32_t u = (uint32_t)wlist[wi];
        const long long ob = U_off[u] + U_split[u], oe = U_off[u + 1];
        const long long du = U_off[u + 1] - U_off[u];
        for (long long e = ob + lane; e < oe; e += 32) {
            const uint32_t v = vid(U_col[e]);
            const long long vb = U_off[v] + U_split[v], ve = U_off[v + 1];
            const long long dv = U_off[v + 1] - U_off[v], te = tall[e];
            long long i = e + 1, j = vb;
            long long opp = 0, outer = 0, k4 = 0;
            while (i < oe && j < ve) {
                const uint32_t x = vid(U_col[i]), y = vid(U_col[j]);
                if (x < y) {
                    i++;
                } else if (x > y) {
                    j++;
                } else {
                    // triangle (u, v, y): edges uv, uy, vy at e, i, j
                    const long long dy = U_off[y + 1] - U_off[y], ti = tall[i], tj = tall[j];
                    opp += dy - 2;
                    outer += ti + tj - 2;
                    atomicAdd((unsigned long long*)&NE[NEROLE * (size_t)i + E_OPP], (unsigned long long)(dv - 2));
                    atomicAdd((unsigned long long*)&NE[NEROLE * (size_t)i + E_OUTER],
                              (unsigned long long)(te + tj - 2));
                    atomicAdd((unsigned long long*)&NE[NEROLE * (size_t)j + E_OPP], (unsigned long long)(du - 2));
                    atomicAdd((unsigned long long*)&NE[NEROLE * (size_t)j + E_OUTER],
                              (unsigned long long)(te + ti - 2));
                    // 4-cliques (u, v, y, z), z > y: edges uz, vz, yz at p, q, r
                    const long long yb = U_off[y] + U_split[y], ye = U_off[y + 1];
                    long long p = i + 1, q = j + 1, r = yb, kk = 0;
                    while (p < oe && q < ve && r < ye) {
                        const uint32_t a = vid(U_col[p]), b = vid(U_col[q]), cc = vid(U_col[r]);
                        const uint32_t mx = max(a, max(b, cc));
                        if (a == mx && b == mx && cc == mx) {
                            atomicAdd((unsigned long long*)&NE[NEROLE * (size_t)p + E_K4], 1ull);
                            atomicAdd((unsigned long long*)&NE[NEROLE * (size_t)q + E_K4], 1ull);
                            atomicAdd((unsigned long long*)&NE[NEROLE * (size_t)r + E_K4], 1ull);
                            kk++;
                            p++;
                            q++;
                            r++;
                        } else {
                            if (a < mx) p++;
                            if (b < mx) q++;
                            if (cc < mx) r++;
                        }
                    }
                    if (kk) {
                        atomicAdd((unsigned long long*)&NE[NEROLE * (size_t)i + E_K4], (unsigned long long)kk);
                        atomicAdd((unsigned long long*)&NE[NEROLE * (size_t)j + E_K4], (unsigned long long)kk);
                        k4 += kk;
                    }
                    i++;
                    j++;
                }
            }
            if (opp) atomicAdd((unsigned long long*)&NE[NEROLE * (size_t)e + E_OPP], (unsigned long long)opp);
            if (outer) atomicAdd((unsigned long long*)&NE[NEROLE * (size_t)e + E_OUTER], (unsigned long long)outer);
            if (k4) atomicAdd((unsigned long long*)&NE[NEROLE * (size_t)e + E_K4], (unsigned long long)k4);
        }
    }
}

// 4-cycles per edge, a block per pivot u (the highest vertex of the cycle)
// with one dense counter array of n words per block: walk 1 counts c_w over
// the wedges u-a-w (a, w below u); walk 2 credits each wedge's two edges
// u-a and a-w with c_w - 1 (the cycles u-a-w-b, b another middle); walk 3
// clears the counters.
__global__ void __launch_bounds__(1024) k_e_c4(const Ctl* c, const int32_t* __restrict__ wlist,
                                               const long long* __restrict__ U_off,
                                               const uint32_t* __restrict__ U_col,
                                               const int32_t* __restrict__ U_split, uint32_t* __restrict__ cnt_all,
                                               int n, const uint8_t* __restrict__ heavy,
                                               long long* __restrict__ NE) {
    pdl_enter();
    const int nW = c->nW;
    uint32_t* cnt = cnt_all + (size_t)blockIdx.x * (size_t)n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NWp = blockDim.x >> 5;
    for (int pi = blockIdx.x; pi < nW; pi += gridDim.x) {
        const uint32_t u = (uint32_t)wlist[pi];
        if (heavy && heavy[u]) continue;  // taken by k_c4_group (same for the whole block)
        const long long rb = U_off[u];
        const int nlow = U_split[u];
        for (int pass = 0; pass < 3; pass++) {
            for (int j = warp; j < nlow; j += NWp) {
                const uint32_t a = vid(U_col[rb + j]);
                const long long ab = U_off[a], ae = U_off[a + 1];
                long long asum = 0;
                for (long long q = ab + lane; q < ae; q += 32) {
                    const uint32_t w = vid(U_col[q]);
                    if (w >= u) break;  // rows are sorted: the rest is above u
                    if (pass == 0) {
                        atomicAdd(&cnt[w], 1u);
                    } else if (pass == 1) {
                        const long long x = (long long)__ldcg(&cnt[w]) - 1;
                        if (x > 0) {
                            atomicAdd((unsigned long long*)&NE[NEROLE * (size_t)q + E_C4], (unsigned long long)x);
                            asum += x;
                        }
                    } else {
                        cnt[w] = 0u;
                    }
                }
                if (pass == 1) {
                    asum = (long long)warp_sum_u64((unsigned long long)asum);
                    if (lane == 0 && asum)
                        atomicAdd((unsigned long long*)&NE[NEROLE * (size_t)(rb + j) + E_C4], (unsigned long long)asum);
                }
            }
            __threadfence();
            __syncthreads();
        }
    }
}

// Orbit counts per edge by the triangular edge-role containment.  A warp
// per vertex x, a lane per out-entry e = (x, y); the credits of the twin
// entry (x in y's row) are added, the edge's row in the output is the rank
// of its key among the sorted keys.  out[k row + j]: the ten edge orbits
// (k = 10) or their sums per graphlet (k = 6); edges[2 row] = (lo, hi).
__global__ void k_e_finalize(const Ctl* c, const int32_t* __restrict__ wlist, const long long* __restrict__ U_off,
                             const uint32_t* __restrict__ U_col, const int32_t* __restrict__ U_split,
                             const uint32_t* __restrict__ tall, const long long* __restrict__ sdeg,
                             const unsigned long long* __restrict__ T2, const long long* __restrict__ NE,
                             const int32_t* __restrict__ iperm, const unsigned long long* __restrict__ skeys,
                             int nb, long long m, int k, unsigned long long* __restrict__ out,
                             int32_t* __restrict__ edges) {
    pdl_enter();
    const int nW = c->nW;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < nW; i += nwarps) {
        const uint32_t x = (uint32_t)wlist[i];
        const long long dx = U_off[x + 1] - U_off[x], trx = (long long)(T2[x] / 2), sx = sdeg[x];
        const unsigned long long ex = (unsigned long long)iperm[x];
        for (long long e = U_off[x] + U_split[x] + lane; e < U_off[x + 1]; e += 32) {
            const uint32_t y = vid(U_col[e]);
            const long long yb = U_off[y];
            const long long tw = yb + lower_bound_id(U_col + yb, U_split[y], x);
            const long long dy = U_off[y + 1] - yb, t = tall[e];
            const long long* ra = NE + NEROLE * (size_t)e;
            const long long* rt = NE + NEROLE * (size_t)tw;
            const long long n_opp = ra[E_OPP] + rt[E_OPP], n_outer = ra[E_OUTER] + rt[E_OUTER];
            const long long n_c4 = ra[E_C4] + rt[E_C4], n_k4 = ra[E_K4] + rt[E_K4];
            const long long n_pend = (sdeg[y] - (dx - 1) - t) + (sx - (dy - 1) - t);
            const long long n_pmid = (dx - 1) * (dy - 1) - t;
            const long long n_star = (dx - 1) * (dx - 2) / 2 + (dy - 1) * (dy - 2) / 2;
            const long long n_tail = (trx - t) + ((long long)(T2[y] / 2) - t);
            const long long n_att = t * (dx + dy - 4);
            const long long n_chord = t * (t - 1) / 2;
            const long long i9 = n_k4;
            const long long i8 = n_chord - i9;
            const long long i7 = n_outer - 4 * i9;
            const long long i6 = n_att - 4 * i8 - i7 - 4 * i9;
            const long long i5 = n_opp - i7 - 2 * i9;
            const long long i4 = n_tail - i7 - 2 * i9;
            const long long i3 = n_c4 - i7 - 2 * i9;
            const long long i2 = n_star - i6 - i4 - 2 * i8 - i7 - 2 * i9;
            const long long i1 = n_pmid - i3 - i6 - 2 * i8 - i7 - 2 * i9;
            const long long i0 = n_pend - 2 * i3 - 2 * i5 - 2 * i4 - 3 * i7 - 4 * i9;
            // rank of the key among the m sorted edge keys
            const unsigned long long ey = (unsigned long long)iperm[y];
            const unsigned long long lo = ex < ey ? ex : ey, hi = ex < ey ? ey : ex;
            const unsigned long long key = (lo << nb) | hi;
            long long a = 0, b = m;
            while (a < b) {
                const long long mid = (a + b) >> 1;
                if (skeys[mid] < key) a = mid + 1;
                else b = mid;
            }
            unsigned long long* o = out + (size_t)k * a;
            if (k == 10) {
                o[0] = (unsigned long long)i0; o[1] = (unsigned long long)i1; o[2] = (unsigned long long)i2;
                o[3] = (unsigned long long)i3; o[4] = (unsigned long long)i4; o[5] = (unsigned long long)i5;
                o[6] = (unsigned long long)i6; o[7] = (unsigned long long)i7; o[8] = (unsigned long long)i8;
                o[9] = (unsigned long long)i9;
            } else {
                o[0] = (unsigned long long)(i0 + i1);
                o[1] = (unsigned long long)i2;
                o[2] = (unsigned long long)i3;
                o[3] = (unsigned long long)(i4 + i5 + i6);
                o[4] = (unsigned long long)(i7 + i8);
                o[5] = (unsigned long long)i9;
            }
            if (edges) {
                edges[2 * a] = (int32_t)lo;
                edges[2 * a + 1] = (int32_t)hi;
            }
        }
    }
}

int enqueue_edge_counts(const EdgeArgs& a, cudaStream_t s) {
    const int gw = 8 * a.sms, tpb = 256;
    int nl = 0;
    pdl_launch(k_v_tsym, dim3(gw), dim3(tpb), 0, s, a.ctl, a.wlist, a.U_off, a.U_col, a.U_split, a.tpack, a.tall);
    pdl_launch(k_v_s, dim3(gw), dim3(tpb), 0, s, a.ctl, a.wlist, a.U_off, a.U_col, a.sdeg);
    pdl_launch(k_e_keys, dim3(gw), dim3(tpb), 0, s, a.ctl, a.wlist, a.U_off, a.U_col, a.U_split, a.iperm, a.nb,
               a.keys);
    nl += 3;
    nl += radix_sort_u64((uint64_t*)a.keys, (uint64_t*)a.keys_tmp, a.d_count, a.nU, 2 * a.nb, a.hist, a.sort_grid, s);
    pdl_launch(k_e_tri_k4, dim3(gw), dim3(tpb), 0, s, a.ctl, a.wlist, a.U_off, a.U_col, a.U_split, a.tall, a.NE);
    const int nh = enqueue_heavy_c4<true>(a.hv, a.ctl, a.wlist, a.U_off, a.U_col, a.U_split, a.n, a.sms, a.NE, s);
    if (nh < 0) return -1;
    nl += nh;
    pdl_launch(k_e_c4, dim3(a.c4_blocks), dim3(1024), 0, s, a.ctl, a.wlist, a.U_off, a.U_col, a.U_split, a.cnt, a.n,
               nh > 0 ? (const uint8_t*)a.hv.heavy : nullptr, a.NE);
    pdl_launch(k_e_finalize, dim3(gw), dim3(tpb), 0, s, a.ctl, a.wlist, a.U_off, a.U_col, a.U_split, a.tall, a.sdeg,
               a.T2, a.NE, a.iperm, a.keys, a.nb, a.m, a.orbits ? 10 : 6, a.out, a.edges);
    nl += 3;
    return nl;
}

int enqueue_vertex_counts(const VertexArgs& a, cudaStream_t s) {
    const int gw = 8 * a.sms, tpb = 256;
    int nl = 0;
    pdl_launch(k_v_tsym, dim3(gw), dim3(tpb), 0, s, a.ctl, a.wlist, a.U_off, a.U_col, a.U_split, a.tpack, a.tall);
    pdl_launch(k_v_s, dim3(gw), dim3(tpb), 0, s, a.ctl, a.wlist, a.U_off, a.U_col, a.sdeg);
    pdl_launch(k_v_terms, dim3(gw), dim3(tpb), 0, s, a.ctl, a.wlist, a.U_off, a.U_col, a.tall, a.sdeg, a.T2, a.NV);
    pdl_launch(k_v_tri_k4, dim3(gw), dim3(tpb), 0, s, a.ctl, a.wlist, a.U_off, a.U_col, a.U_split, a.tall, a.NV);
    const int nh = enqueue_heavy_c4<false>(a.hv, a.ctl, a.wlist, a.U_off, a.U_col, a.U_split, a.n, a.sms, a.NV, s);
    if (nh < 0) return -1;
    nl += nh;
    pdl_launch(k_v_c4, dim3(a.c4_blocks), dim3(1024), 0, s, a.ctl, a.wlist, a.U_off, a.U_col, a.U_split, a.cnt, a.n,
               nh > 0 ? (const uint8_t*)a.hv.heavy : nullptr, a.NV);
    pdl_launch(k_v_finalize, dim3((a.n + 255) / 256), dim3(256), 0, s, a.NV, a.n, a.iperm, a.orbits ? 11 : 6, a.out);
    nl += 6;
    return nl;
}

}  // namespace gcx
