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
// out-entry in tpack, T2 filled).
#include "gc_internal.cuh"
#include "gc_kernels.cuh"

namespace gcx {

// role slots of NV, in orbit order 4..14
enum { R_PEND, R_PMID, R_SLEAF, R_SCTR, R_C4, R_TTAIL, R_TOTH, R_TATT, R_D2, R_D3, R_K4, NROLE };

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
                                               int n, long long* __restrict__ NV) {
    pdl_enter();
    const int nW = c->nW;
    uint32_t* cnt = cnt_all + (size_t)blockIdx.x * (size_t)n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NWp = blockDim.x >> 5;
    __shared__ unsigned long long s_u[32];
    for (int pi = blockIdx.x; pi < nW; pi += gridDim.x) {
        const uint32_t u = (uint32_t)wlist[pi];
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

int enqueue_vertex_counts(const VertexArgs& a, cudaStream_t s) {
    const int gw = 8 * a.sms, tpb = 256;
    int nl = 0;
    pdl_launch(k_v_tsym, dim3(gw), dim3(tpb), 0, s, a.ctl, a.wlist, a.U_off, a.U_col, a.U_split, a.tpack, a.tall);
    pdl_launch(k_v_s, dim3(gw), dim3(tpb), 0, s, a.ctl, a.wlist, a.U_off, a.U_col, a.sdeg);
    pdl_launch(k_v_terms, dim3(gw), dim3(tpb), 0, s, a.ctl, a.wlist, a.U_off, a.U_col, a.tall, a.sdeg, a.T2, a.NV);
    pdl_launch(k_v_tri_k4, dim3(gw), dim3(tpb), 0, s, a.ctl, a.wlist, a.U_off, a.U_col, a.U_split, a.tall, a.NV);
    pdl_launch(k_v_c4, dim3(a.c4_blocks), dim3(1024), 0, s, a.ctl, a.wlist, a.U_off, a.U_col, a.U_split, a.cnt, a.n,
               a.NV);
    pdl_launch(k_v_finalize, dim3((a.n + 255) / 256), dim3(256), 0, s, a.NV, a.n, a.iperm, a.orbits ? 11 : 6, a.out);
    nl += 6;
    return nl;
}

}  // namespace gcx
