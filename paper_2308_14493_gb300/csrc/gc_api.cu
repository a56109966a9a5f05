// gc_api.cu -- the C ABI (include/gc.h): handle state, device buffers and the
// launch sequence of one batch of Algorithm 2 (FDGC, Sec. 4.3):
//
//   a0 normalise the batch (sort directed keys, drop repeats, pairs in both
//      lists, no-ops)                                    gc_batch.cu
//   a1 k-hop region W from every endpoint               gc_region.cu
//   a2 flagged union graph U = G[W] u A, degrees in G_a and G_b
//   a3 per-edge triangles of G_a and G_b                 gc_count.cu
//   a4 4-cliques, a5 4-cycles, a6 per-edge / per-vertex terms
//   a7 closed forms: C_a, C_b, F += C_a - C_b
//   a8 commit G <- G \ D u A into the slack-padded rows  gc_batch.cu
//
// Every stage reads its sizes from the device control block, so the host
// only enqueues work.  The plain form enqueues one batch and reads the
// control block back once.  The batched form captures the same sequence once
// in a CUDA graph that takes its batch from a device-side cursor, and replays
// it for every batch of a run without host round trips.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "gc.h"
#include "gc_internal.cuh"
#include "gc_kernels.cuh"

using namespace gcx;

namespace {

thread_local std::string t_open_error;

template <class T>
struct Buf {
    T* p = nullptr;
    size_t cap = 0;
};

constexpr int TPB = 256;

int bitlen(long long x) {
    int b = 0;
    while (x > 0) {
        b++;
        x >>= 1;
    }
    return b;
}

}  // namespace

struct gc_graph {
    int dev = 0, n = 0, S = 1, sms = 148, hops = 3;
    float slack = 0.25f;
    cudaStream_t s = nullptr;
    bool own_stream = false;
    gc_options opt{};
    // persistent state
    int32_t *perm = nullptr, *iperm = nullptr, *deg = nullptr, *cap = nullptr, *col = nullptr;
    long long* row_start = nullptr;
    long long col_capacity = 0;
    Ctl* ctl = nullptr;
    Ctl* h_ctl = nullptr;            // pinned mirror
    long long* desc = nullptr;       // device run descriptor: [pair bases, then 4 words per batch]
    long long* h_desc = nullptr;     // pinned staging of the descriptor
    long long desc_cap = 0;          // words of desc / h_desc
    int2 *segA = nullptr, *segD = nullptr;
    uint32_t* visited = nullptr;
    int32_t *wlist = nullptr, *U_deg = nullptr, *U_split = nullptr, *da = nullptr, *db = nullptr;
    long long* U_off = nullptr;
    long long* U_wt = nullptr;           // wedge bound per 4-cycle pivot
    // scratch that grows with the batch or the graph
    Buf<uint32_t> U_col;
    Buf<unsigned long long> tpack;
    Buf<uint64_t> keys, keys_tmp;
    Buf<int32_t> keepA, keepD, srcA, dstA, srcD, dstD, plan_cap, plan_deg, pairs;
    Buf<long long> posA, posD, plan_dst, plan_scr, bsum;
    Buf<uint32_t> hist;
    Buf<unsigned long long> out_dev;     // per-batch results of a batched run
    Buf<int32_t> vids, vdeg;             // vertex deletion: ids and their degrees
    Buf<long long> voff;                 // vertex deletion: pair offsets
    Buf<unsigned long long> dense;       // counter arrays of the heaviest 4-cycle pivots (per cluster)
    int dense_clusters = 0;
    int dense_cluster_size = 8;
    Buf<unsigned long long> cta_tables;  // hash tables of the medium 4-cycle pivots (per CTA)
    int cta_groups = 0;
    Buf<unsigned char> chunk_table;      // per-CTA run bounds of the chunked 4-cycle kernel
    long long chunk_cap = 0;             // run-bound entries per CTA in it
    Tuning tune = default_tuning();     // bin boundaries of the counting pass
    long long loc_heavy_min = 65536;   // w~ from which local-count 4-cycle pivots take k_c4_group (0 = never)
    int32_t* bins = nullptr;             // NBINS * n work lists of the counting pass
    // captured batch graph and the shape it was captured for
    cudaGraphExec_t gexec = nullptr;
    long long g_nk = -1;
    int g_commit = -1;
    unsigned long long g_gen = 0;
    int g_launches = 0;                  // kernels in one replay
    // the same for the plain form: one batch per call, stage events recorded
    cudaGraphExec_t pexec = nullptr;
    long long p_nk = -1;
    int p_commit = -1;
    unsigned long long p_gen = 0;
    int p_launches = 0;
    // the same for the edge-local form of the plain path
    cudaGraphExec_t lexec = nullptr;
    long long l_nk = -1;
    int l_commit = -1;
    unsigned long long l_gen = 0;
    int l_launches = 0;
    // scratch of the edge-local path (entries each; offsets one more)
    Buf<int32_t> l_cost, l_own, l_pcost, l_ccnt, l_kcost, l_tpair, l_walk;
    Buf<long long> l_pre, l_ppre, l_cpre, l_kpre;
    Buf<unsigned long long> l_rec;
    Buf<long long> l_dcnt;
    long long l_cap = 0;
    int l_t2 = -1;                       // captured with maintained triangle sums
    int p_t2 = -1;                       // the same for the plain region form
    int g_t2 = -1;                       // and for the batched region form
    // the two-batch form of sequential runs: [0] commits a batch without a
    // count, [1] counts the next one over every vertex (enqueue_batch roles)
    // and [2] the twin pass of independent runs
    cudaGraphExec_t qexec[3] = {nullptr, nullptr, nullptr};
    long long q_nk[3] = {-1, -1, -1};
    unsigned long long q_gen[3] = {0, 0, 0};
    int q_launches[3] = {0, 0, 0};
    long long pair_min_share = 700;      // per mille of 2m (gc_tuning.pair_min_share)
    long long pair_hint = 0;             // size of the smallest first batch of a run whose region met it (0: none)
    // maintained triangle sums of the edge-local path: T2[x] = sum of t_e
    // over the edges at x, valid after a static count and kept by local
    // batches (a region batch makes it stale)
    unsigned long long* T2 = nullptr;
    long long* dtri2 = nullptr;          // zero between batches
    uint32_t* visited2 = nullptr;
    bool t2_valid = false;
    unsigned long long buf_gen = 1;      // bumped whenever a buffer moves
    // host mirror
    uint64_t F[6] = {0, 0, 0, 0, 0, 0};
    uint64_t F3[2] = {0, 0};  // maintained 3-vertex counts: induced 2-paths, triangles
    long long m = 0;
    gc_stats st{};
    std::string err;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEvent_t ev[10] = {};  // stage boundaries, see gc_stats.ms_stage; [8], [9] around the
                              // heavy-pivot 4-cycle kernels (ms_stage[7])
    cudaStream_t aux[3] = {};   // side streams of the counting pass
    cudaEvent_t fork = nullptr, join[3] = {};
    int launches = 0;        // kernels launched by the current call
    // device bytes held, for admission control
    std::unordered_map<void*, size_t> held;
    long long bytes_held = 0;
};

// ---------------------------------------------------------------------------
// memory
// ---------------------------------------------------------------------------
static void* dalloc(gc_graph* g, size_t bytes) {
    if (bytes < 16) bytes = 16;
    void* p = nullptr;
    if (g->opt.alloc) {
        p = g->opt.alloc(bytes, (void*)g->s, g->opt.ctx);
    } else if (cudaMallocAsync(&p, bytes, g->s) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        g->held[p] = bytes;
        g->bytes_held += (long long)bytes;
    }
    return p;
}

static void dfree(gc_graph* g, void* p) {
    if (!p) return;
    auto it = g->held.find(p);
    if (it != g->held.end()) {
        g->bytes_held -= (long long)it->second;
        g->held.erase(it);
    }
    if (g->opt.free) g->opt.free(p, (void*)g->s, g->opt.ctx);
    else cudaFreeAsync(p, g->s);
}

template <class T>
static bool ensure(gc_graph* g, Buf<T>& b, size_t count) {
    if (b.p && b.cap >= count) return true;
    size_t nc = std::max<size_t>(count + count / 4, 64);
    dfree(g, b.p);
    b.p = (T*)dalloc(g, nc * sizeof(T));
    b.cap = b.p ? nc : 0;
    g->buf_gen++;
    return b.p != nullptr;
}

template <class T>
static void release(gc_graph* g, Buf<T>& b) {
    dfree(g, b.p);
    b.p = nullptr;
    b.cap = 0;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            g->err = std::string(#call) + ": " + cudaGetErrorString(e_);                  \
            return GC_ECUDA;                                                              \
        }                                                                                 \
    } while (0)

#define CKL()                                                                             \
    do {                                                                                  \
        cudaError_t e_ = cudaGetLastError();                                              \
        if (e_ != cudaSuccess) {                                                          \
            g->err = std::string("kernel launch: ") + cudaGetErrorString(e_);             \
            return GC_ECUDA;                                                              \
        }                                                                                 \
    } while (0)

static int nomem(gc_graph* g, const char* what) {
    g->err = std::string("device allocation failed: ") + what;
    return GC_ENOMEM;
}

static int grid_elems(gc_graph* g, long long n) {
    long long b = (n + TPB - 1) / TPB;
    if (b < 1) b = 1;
    if (b > 8LL * g->sms) b = 8LL * g->sms;
    return (int)b;
}
static int grid_warps(gc_graph* g) { return 8 * g->sms; }  // 8 warps per block

// ---------------------------------------------------------------------------
// small device helpers local to this file
// ---------------------------------------------------------------------------
namespace gcx {

// desc: [0] insertion pair base, [1] deletion pair base, then per batch
// [ins_off, n_ins, del_off, n_del]; the batch is the one at the run cursor.
// A halted run (a commit waiting for pool space) makes every later batch
// empty and inactive.
__global__ void k_begin_batch(Ctl* c, const long long* desc) {
    pdl_enter();
    if (threadIdx.x != 0) return;
    const bool run = c->halt == 0;
    c->active = run ? 1 : 0;
    // the descriptor is rewritten by host copies between calls: read it
    // from L2, never through the read-only cache path
    const long long* b = desc + 2 + 4 * (long long)c->cur;
    c->pairs_ins = (const int32_t*)__ldcg(desc);
    c->pairs_del = (const int32_t*)__ldcg(desc + 1);
    c->ins_off = run ? __ldcg(b) : 0;
    c->n_ins = run ? __ldcg(b + 1) : 0;
    c->del_off = run ? __ldcg(b + 2) : 0;
    c->n_del = run ? __ldcg(b + 3) : 0;
    c->nkeys = 2 * (c->n_ins + c->n_del);
    c->nA2 = c->nD2 = 0;
    for (int k = 0; k < 8; k++) c->st[k] = 0;
    c->nW = 0;
    for (int k = 0; k < MAX_HOPS + 2; k++) c->lvl[k] = 0;
    c->nU = 0;
    c->scratch_tail = 0;
    c->overflow = 0;
    c->err = 0;
    c->lovf = 0;
    c->l_np = 0;
    c->l_need = 0;
    c->l_nw3 = 0;
    for (int k = 0; k < 4; k++) c->l_len[k] = 0;
    for (int k = 0; k < 5; k++) c->l_tot[k] = 0;
}

// The twin pass's batches cur and cur + 1: both pair lists (the keys kernel
// reads four segments: insertions and deletions of each).
__global__ void k_begin_twin(Ctl* c, const long long* desc) {
    pdl_enter();
    if (threadIdx.x != 0) return;
    c->active = 1;
    c->pairs_ins = (const int32_t*)__ldcg(desc);
    c->pairs_del = (const int32_t*)__ldcg(desc + 1);
    long long tot = 0;
    for (int b = 0; b < 2; b++) {
        const long long* d = desc + 2 + 4 * (long long)(c->cur + b);
        c->tw_off[2 * b] = __ldcg(d);
        c->tw_n[2 * b] = __ldcg(d + 1);
        c->tw_off[2 * b + 1] = __ldcg(d + 2);
        c->tw_n[2 * b + 1] = __ldcg(d + 3);
        tot += c->tw_n[2 * b] + c->tw_n[2 * b + 1];
    }
    c->n_ins = c->tw_n[0] + c->tw_n[2];
    c->n_del = c->tw_n[1] + c->tw_n[3];
    c->ins_off = c->del_off = 0;
    c->nkeys = 2 * tot;
    c->nA2 = c->nD2 = 0;
    for (int k = 0; k < 8; k++) c->st[k] = 0;
    c->nW = 0;
    for (int k = 0; k < MAX_HOPS + 2; k++) c->lvl[k] = 0;
    c->nU = 0;
    c->scratch_tail = 0;
    c->overflow = 0;
    c->err = 0;
    c->lovf = 0;
}

// result of the current batch to out[cur], advance the cursor.  form 1:
// the second batch of a two-batch pass also writes the first one's result;
// form 2: a twin pass writes the results of batches cur and cur + 1
__global__ void k_end_batch(Ctl* c, unsigned long long* out, int commit, int form) {
    pdl_enter();
    if (threadIdx.x != 0 || !c->active) return;
    if (form == 1 && c->cur > 0 && !c->err)
        for (int k = 0; k < 6; k++) out[6 * (long long)(c->cur - 1) + k] = c->prev_out[k];
    if (form == 2) {
        for (int k = 0; k < 6; k++) {
            out[6 * (long long)c->cur + k] = c->last_out[k];
            out[6 * (long long)(c->cur + 1) + k] = c->prev_out[k];
        }
        c->cur += 2;
        return;
    }
    for (int k = 0; k < 6; k++) out[6 * (long long)c->cur + k] = c->last_out[k];
    if (commit && !c->err && !c->lovf) c->m_delta += c->nA2 / 2 - c->nD2 / 2;
    c->cur++;
}

// every pair of a run in range and not a self-loop (bad = 1 otherwise)
__global__ void k_run_pairs_check(const long long* desc, int k, int n, int* bad) {
    pdl_enter();
    const int32_t* ins = (const int32_t*)__ldcg(desc);
    const int32_t* del = (const int32_t*)__ldcg(desc + 1);
    for (int b = blockIdx.y; b < k; b += gridDim.y) {
        const long long* d = desc + 2 + 4 * (long long)b;
        const long long io = __ldcg(d), ni = __ldcg(d + 1), dof = __ldcg(d + 2), nd = __ldcg(d + 3);
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ni + nd;
             i += (long long)gridDim.x * blockDim.x) {
            const int32_t* p = i < ni ? ins + 2 * (io + i) : del + 2 * (dof + i - ni);
            const int32_t x = p[0], y = p[1];
            if (x < 0 || y < 0 || x >= n || y >= n || x == y) atomicExch(bad, 1);
        }
    }
}

__global__ void k_run_reset(Ctl* c) {
    pdl_enter();
    if (threadIdx.x != 0) return;
    c->cur = 0;
    c->halt = 0;
    c->m_delta = 0;
}

// restore the kept-entry counts of the batch whose commit is pending
__global__ void k_resume_pending(Ctl* c) {
    pdl_enter();
    if (threadIdx.x != 0) return;
    c->nA2 = c->pend_nA2;
    c->nD2 = c->pend_nD2;
    c->lvl[0] = c->pend_ns;
    c->active = 1;
    c->err = 0;
}

__global__ void k_halt_clear(Ctl* c) {
    pdl_enter();
    if (threadIdx.x == 0) c->halt = 0;
}

__global__ void k_commit_reset(Ctl* c, unsigned long long pool_tail, int set_pool) {
    pdl_enter();
    if (threadIdx.x != 0) return;
    c->scratch_tail = 0;
    c->overflow = 0;
    if (set_pool) c->pool_tail = pool_tail;
}

// Vertex deletion as an edge batch: the degrees of the listed vertices, then
// every incident edge as an (external id) pair.
__global__ void k_vertex_degrees(const int32_t* __restrict__ ids, long long k, const int32_t* __restrict__ perm,
                                 const int32_t* __restrict__ deg, int32_t* __restrict__ vdeg) {
    pdl_enter();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < k; i += (long long)gridDim.x * blockDim.x)
        vdeg[i] = deg[perm[ids[i]]];
}
__global__ void k_vertex_pairs(const int32_t* __restrict__ ids, long long k, const int32_t* __restrict__ perm,
                               const int32_t* __restrict__ iperm, const long long* __restrict__ row_start,
                               const int32_t* __restrict__ deg, const int32_t* __restrict__ col,
                               const long long* __restrict__ off, int32_t* __restrict__ pairs) {
    pdl_enter();
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = warp; i < k; i += nwarps) {
        const int32_t v = ids[i];
        const int32_t iv = perm[v];
        const long long rb = row_start[iv];
        const int d = deg[iv];
        int32_t* o = pairs + 2 * off[i];
        for (int j = lane; j < d; j += 32) {
            o[2 * j] = v;
            o[2 * j + 1] = iperm[col[rb + j]];
        }
    }
}

// New vertices ids [n0, n1): internal id = external id, no edges (a zero
// capacity row: the first insertion moves it to the pool).
__global__ void k_init_new_vertices(int32_t* perm, int32_t* iperm, int32_t* deg, int32_t* cap, long long* row_start,
                                    int n0, int n1) {
    pdl_enter();
    for (long long i = n0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n1;
         i += (long long)gridDim.x * blockDim.x) {
        perm[i] = (int32_t)i;
        iperm[i] = (int32_t)i;
        deg[i] = 0;
        cap[i] = 0;
        row_start[i] = 0;
    }
}

__global__ void k_set_F(Ctl* c) {
    pdl_enter();
    if (threadIdx.x < 6) c->F[threadIdx.x] = (unsigned long long)c->Ca[threadIdx.x];
    if (threadIdx.x < 2) c->F3[threadIdx.x] = (unsigned long long)c->C3a[threadIdx.x];
}

__global__ void k_mark_active(Ctl* c) {
    pdl_enter();
    if (threadIdx.x == 0) c->active = 1;
}

}  // namespace gcx

// ---------------------------------------------------------------------------
// pipeline pieces
// ---------------------------------------------------------------------------
static int plan_region_buffers(gc_graph* g, long long max_edges, long long n_ins) {
    size_t ucap = (size_t)(2 * max_edges + 2 * n_ins + 64);
    if (!ensure(g, g->U_col, ucap)) return nomem(g, "region adjacency");
    if (!ensure(g, g->tpack, ucap)) return nomem(g, "triangle counters");
    return GC_OK;
}

static int plan_batch_buffers(gc_graph* g, long long nk) {
    size_t nkb = (size_t)std::max<long long>(nk, 1);
    if (!ensure(g, g->keys, nkb) || !ensure(g, g->keys_tmp, nkb) || !ensure(g, g->keepA, nkb) ||
        !ensure(g, g->keepD, nkb) || !ensure(g, g->posA, nkb + 1) || !ensure(g, g->posD, nkb + 1) ||
        !ensure(g, g->srcA, nkb) || !ensure(g, g->dstA, nkb) || !ensure(g, g->srcD, nkb) ||
        !ensure(g, g->dstD, nkb) || !ensure(g, g->plan_dst, nkb) || !ensure(g, g->plan_scr, nkb) ||
        !ensure(g, g->plan_cap, nkb) || !ensure(g, g->plan_deg, nkb))
        return nomem(g, "batch scratch");
    if (!ensure(g, g->hist, (size_t)256 * radix_grid(nk, g->sms))) return nomem(g, "sort histogram");
    return GC_OK;
}

// Bytes that ensure(b, count) would add.
template <class T>
static long long grow_bytes(const Buf<T>& b, size_t count) {
    if (b.p && b.cap >= count) return 0;
    size_t nc = std::max<size_t>(count + count / 4, 64);
    return (long long)(nc * sizeof(T)) - (long long)(b.cap * sizeof(T));
}

// Device bytes a batch of n_ins + n_del pairs would add to what the handle
// holds: its scratch growth, plus a re-layout of the adjacency when the
// pool's free space at the end of the last batch may not take the insertions.
static long long predict_batch_bytes(const gc_graph* g, long long n_ins, long long n_del) {
    // batch scratch is sized for the captured shape: the next power of two of the keys
    size_t nk = 1;
    while (nk < (size_t)std::max<long long>(2 * (n_ins + n_del), 1)) nk <<= 1;
    long long b = grow_bytes(g->keys, nk) + grow_bytes(g->keys_tmp, nk) + grow_bytes(g->keepA, nk) +
                  grow_bytes(g->keepD, nk) + grow_bytes(g->posA, nk + 1) + grow_bytes(g->posD, nk + 1) +
                  grow_bytes(g->srcA, nk) + grow_bytes(g->dstA, nk) + grow_bytes(g->srcD, nk) +
                  grow_bytes(g->dstD, nk) + grow_bytes(g->plan_dst, nk) + grow_bytes(g->plan_scr, nk) +
                  grow_bytes(g->plan_cap, nk) + grow_bytes(g->plan_deg, nk) +
                  grow_bytes(g->hist, (size_t)256 * radix_grid((long long)nk, g->sms)) +
                  grow_bytes(g->pairs, nk) + grow_bytes(g->out_dev, 6);
    const size_t ucap = (size_t)(2 * g->m + 4 * n_ins + 64);
    b += grow_bytes(g->U_col, ucap) + grow_bytes(g->tpack, ucap);
    const long long pool_free = g->col_capacity - (long long)g->h_ctl->pool_tail;
    if (n_ins > 0 && pool_free < 8 * n_ins) {
        // new rows with fresh slack and a new pool, while the old ones live
        const double rows = (double)(2 * (g->m + n_ins)) * (1.0 + 2.0 * g->slack) + 8.0 * n_ins + 4096;
        b += (long long)(4.0 * rows) + 8LL * (g->n + 1);
    }
    return b;
}

static void release_local(gc_graph* g) {
    release(g, g->l_cost);
    release(g, g->l_own);
    release(g, g->l_pcost);
    release(g, g->l_ccnt);
    release(g, g->l_kcost);
    release(g, g->l_tpair);
    release(g, g->l_walk);
    release(g, g->l_pre);
    release(g, g->l_ppre);
    release(g, g->l_cpre);
    release(g, g->l_kpre);
    release(g, g->l_rec);
    release(g, g->l_dcnt);
    g->l_cap = 0;
}

// Scratch of the edge-local path for `cap` entries per array.
static int ensure_local(gc_graph* g, long long cap) {
    if (g->l_cap >= cap) return GC_OK;
    const size_t c = (size_t)cap;
    if (!ensure(g, g->l_cost, c) || !ensure(g, g->l_own, c) || !ensure(g, g->l_pcost, c) ||
        !ensure(g, g->l_ccnt, c) || !ensure(g, g->l_kcost, c) || !ensure(g, g->l_tpair, c) ||
        !ensure(g, g->l_walk, c) ||
        !ensure(g, g->l_pre, c + 1) || !ensure(g, g->l_ppre, c + 1) || !ensure(g, g->l_cpre, c + 1) ||
        !ensure(g, g->l_kpre, c + 1) || !ensure(g, g->l_rec, c) || !ensure(g, g->l_dcnt, c)) {
        release_local(g);  // no array is left half-grown (l_cap = 0)
        return nomem(g, "edge-local scratch");
    }
    // ensure() may round up; the usable capacity is the smallest array's
    size_t m = std::min({g->l_cost.cap, g->l_own.cap, g->l_pcost.cap, g->l_ccnt.cap, g->l_kcost.cap,
                         g->l_tpair.cap, g->l_walk.cap, g->l_rec.cap, g->l_dcnt.cap, g->l_pre.cap - 1, g->l_ppre.cap - 1, g->l_cpre.cap - 1,
                         g->l_kpre.cap - 1});
    g->l_cap = (long long)m;
    g->buf_gen++;  // captured graphs hold the old pointers
    return GC_OK;
}

// Free the scratch that the next batch re-creates on demand.
static void trim_scratch(gc_graph* g) {
    if (g->s) cudaStreamSynchronize(g->s);
    for (int i = 0; i < 3; i++)
        if (g->qexec[i]) {
            cudaGraphExecDestroy(g->qexec[i]);
            g->qexec[i] = nullptr;
        }
    if (g->gexec) {
        cudaGraphExecDestroy(g->gexec);
        g->gexec = nullptr;
    }
    if (g->pexec) {
        cudaGraphExecDestroy(g->pexec);
        g->pexec = nullptr;
    }
    if (g->lexec) {
        cudaGraphExecDestroy(g->lexec);
        g->lexec = nullptr;
    }
    release_local(g);
    release(g, g->U_col);
    release(g, g->tpack);
    release(g, g->keys);
    release(g, g->keys_tmp);
    release(g, g->keepA);
    release(g, g->keepD);
    release(g, g->srcA);
    release(g, g->dstA);
    release(g, g->srcD);
    release(g, g->dstD);
    release(g, g->plan_cap);
    release(g, g->plan_deg);
    release(g, g->pairs);
    release(g, g->posA);
    release(g, g->posD);
    release(g, g->plan_dst);
    release(g, g->plan_scr);
    release(g, g->out_dev);
    g->buf_gen++;
    if (g->s) cudaStreamSynchronize(g->s);
}

// Scratch of the chunked 4-cycle kernel: per CTA, the run bounds of one
// pivot's lower neighbours (c4_chunk_cap entries for this n), allocated when
// a tuning first enables that tier.
static bool ensure_chunk_table(gc_graph* g) {
    const long long cap = c4_chunk_cap(std::max(g->n, 1));
    if (!ensure(g, g->chunk_table, (size_t)g->sms * c4_chunk_cta_bytes(cap))) return false;
    g->chunk_cap = cap;
    return true;
}

static int ensure_desc(gc_graph* g, long long words) {
    if (g->desc && g->desc_cap >= words) return GC_OK;
    long long nc = std::max<long long>(words + words / 4, 64);
    if (g->h_desc) cudaFreeHost(g->h_desc);
    dfree(g, g->desc);
    g->h_desc = nullptr;
    g->desc = (long long*)dalloc(g, sizeof(long long) * (size_t)nc);
    g->buf_gen++;
    if (!g->desc || cudaMallocHost((void**)&g->h_desc, sizeof(long long) * (size_t)nc) != cudaSuccess) {
        g->desc_cap = 0;
        return nomem(g, "batch descriptor");
    }
    g->desc_cap = nc;
    return GC_OK;
}

// U build + counting + closed forms.
//   fin: k_finalize mode (0 committed batch, 1 static, 2 independent batch)
//   set_F: a static count that initialises F; timed: record stage events
// all: the region is every vertex (no per-entry region test in the union
// graph); twin: the twin pass's union graph of two batches
static int count_region(gc_graph* g, int fin, bool set_F, bool timed, bool twin = false, bool all = false) {
    cudaStream_t s = g->s;
    int gw = grid_warps(g);
    pdl_launch(k_reset_count, dim3(1), dim3(32), 0, s, g->ctl);
    CK(cudaMemsetAsync(g->U_deg, 0, sizeof(int32_t) * (size_t)std::max(g->n, 1), s));
    if (twin)
        pdl_launch(k_u_count_twin, dim3(grid_elems(g, g->n)), dim3(TPB), 0, s, g->ctl, g->wlist, g->deg, g->segA,
                   g->U_deg);
    else
        pdl_launch(k_u_count, dim3(gw), dim3(TPB), 0, s, g->ctl, g->wlist, g->visited, g->row_start, g->deg, g->col,
                   g->segA, g->U_deg, all ? 1 : 0);
    g->launches += 2;
    g->launches += scan_i32_to_i64(g->U_deg, g->U_off, nullptr, g->n, g->bsum.p, scan_grid(g->n, g->sms), &g->ctl->nU,
                                   s);
    if (twin)
        pdl_launch(k_u_fill_twin, dim3(gw), dim3(TPB), 0, s, g->ctl, g->wlist, g->row_start, g->deg, g->col, g->segA,
                   g->segD, g->dstA.p, g->dstD.p, g->U_off, g->U_col.p, g->U_split, g->da, g->db);
    else
        pdl_launch(k_u_fill, dim3(gw), dim3(TPB), 0, s, g->ctl, g->wlist, g->visited, g->row_start, g->deg, g->col,
                   g->segA, g->segD, g->dstA.p, g->dstD.p, g->U_off, g->U_col.p, g->U_split, g->da, g->db,
                   all ? 1 : 0);
    pdl_launch(k_zero_u64, dim3(grid_elems(g, (long long)g->U_col.cap)), dim3(TPB), 0, s, g->tpack.p, &g->ctl->nU);
    g->launches += 2;
    CountArgs ca;
    ca.ctl = g->ctl;
    ca.wlist = g->wlist;
    ca.U_off = g->U_off;
    ca.U_col = g->U_col.p;
    ca.U_split = g->U_split;
    ca.U_wt = g->U_wt;
    ca.da = g->da;
    ca.db = g->db;
    ca.tpack = g->tpack.p;
    ca.bins = g->bins;
    ca.dense = g->dense.p;
    ca.n_alloc = std::max(g->n, 1);
    ca.dense_clusters = g->dense_clusters;
    ca.dense_cluster_size = g->dense_cluster_size;
    ca.cta_tables = g->cta_tables.p;
    ca.cta_table_words = 2 * C4_T3;
    ca.cta_groups = g->cta_groups;
    ca.chunk_scratch = g->chunk_table.p;
    ca.chunk_cap = g->chunk_table.p ? g->chunk_cap : 0;
    ca.tune = g->tune;
    ca.sms = g->sms;
    for (int i = 0; i < 3; i++) {
        ca.aux[i] = g->opt.serial_count ? nullptr : g->aux[i];
        ca.join[i] = g->join[i];
    }
    ca.fork = g->fork;
    ca.ev_heavy[0] = timed ? g->ev[8] : nullptr;
    ca.ev_heavy[1] = timed ? g->ev[9] : nullptr;
    g->launches += enqueue_counting(ca, s, timed ? g->ev[3] : nullptr, timed ? g->ev[4] : nullptr,
                                    timed ? g->ev[5] : nullptr, fin);
    if (set_F) {
        pdl_launch(k_set_F, dim3(1), dim3(32), 0, s, g->ctl);
        g->launches++;
    }
    if (timed) CK(record_stage(g->ev[6], s));
    CKL();
    return GC_OK;
}

// Edge-local delta: union rows of the batch endpoints V_X (full rows), then
// the local terms, 4-cliques and 4-cycles and their closed forms.
static int count_local(gc_graph* g, int commit, bool timed, bool t2) {
    cudaStream_t s = g->s;
    int gw = grid_warps(g);
    pdl_launch(k_reset_count, dim3(1), dim3(32), 0, s, g->ctl);
    if (t2) CK(cudaMemsetAsync(g->visited2, 0, sizeof(uint32_t) * (size_t)((g->n + 31) / 32 + 1), s));
    CK(cudaMemsetAsync(g->U_deg, 0, sizeof(int32_t) * (size_t)std::max(g->n, 1), s));
    pdl_launch(k_u_count, dim3(gw), dim3(TPB), 0, s, g->ctl, g->wlist, g->visited, g->row_start, g->deg, g->col,
               g->segA, g->U_deg, 1);
    g->launches += 2;
    g->launches += scan_i32_to_i64(g->U_deg, g->U_off, nullptr, g->n, g->bsum.p, scan_grid(g->n, g->sms), &g->ctl->nU,
                                   s);
    pdl_launch(k_u_fill_all, dim3(gw), dim3(TPB), 0, s, g->ctl, g->wlist, g->row_start, g->deg, g->col, g->segA,
               g->segD, g->dstA.p,
                                    g->dstD.p, g->U_off, g->U_col.p, g->U_split, g->da, g->db);
    pdl_launch(k_zero_u64, dim3(grid_elems(g, (long long)g->U_col.cap)), dim3(TPB), 0, s, g->tpack.p, &g->ctl->nU);
    g->launches += 2;
    LocalArgs la;
    la.ctl = g->ctl;
    la.wlist = g->wlist;
    la.visited = g->visited;
    la.U_off = g->U_off;
    la.U_col = g->U_col.p;
    la.row_start = g->row_start;
    la.deg = g->deg;
    la.col = g->col;
    la.da = g->da;
    la.db = g->db;
    la.tpack = g->tpack.p;
    la.srcA = g->srcA.p;
    la.dstA = g->dstA.p;
    la.srcD = g->srcD.p;
    la.dstD = g->dstD.p;
    la.cost = g->l_cost.p;
    la.own = g->l_own.p;
    la.pcost = g->l_pcost.p;
    la.ccnt = g->l_ccnt.p;
    la.kcost = g->l_kcost.p;
    la.tpair = g->l_tpair.p;
    la.walk = g->l_walk.p;
    la.pre = g->l_pre.p;
    la.ppre = g->l_ppre.p;
    la.cpre = g->l_cpre.p;
    la.kpre = g->l_kpre.p;
    la.rec = g->l_rec.p;
    la.dcnt = g->l_dcnt.p;
    la.T2 = t2 ? g->T2 : nullptr;
    la.dtri2 = g->dtri2;
    la.visited2 = g->visited2;
    la.wlist_w = g->wlist;
    la.bsum = g->bsum.p;
    la.cap = g->l_cap;
    la.n = std::max(g->n, 1);
    la.sms = g->sms;
    g->launches += enqueue_local(la, s, timed ? g->ev[3] : nullptr, timed ? g->ev[4] : nullptr,
                                 timed ? g->ev[5] : nullptr, commit);
    if (timed) CK(record_stage(g->ev[6], s));
    CKL();
    return GC_OK;
}

static int enqueue_commit(gc_graph* g) {
    cudaStream_t s = g->s;
    int gw = grid_warps(g);
    pdl_launch(k_commit_plan, dim3(grid_elems(g, std::max<long long>(g->keys.cap, 1))), dim3(TPB), 0, s, g->ctl,
               g->wlist, g->segA, g->segD, g->deg, g->cap, g->row_start, g->col_capacity, g->slack,
        g->plan_dst.p, g->plan_cap.p, g->plan_deg.p, g->plan_scr.p);
    // the region adjacency buffer is free again and is large enough for every
    // rewritten row: use it as the merge scratch
    pdl_launch(k_commit_merge, dim3(gw), dim3(TPB), 0, s, g->ctl, g->wlist, g->segA, g->segD, g->dstA.p, g->dstD.p,
               g->deg, g->row_start,
                                      g->col, g->plan_scr.p, g->U_col.p);
    pdl_launch(k_commit_write, dim3(gw), dim3(TPB), 0, s, g->ctl, g->wlist, g->plan_dst.p, g->plan_cap.p, g->plan_deg.p,
                                      g->plan_scr.p, g->U_col.p, g->deg, g->cap, g->row_start, g->col);
    g->launches += 3;
    CKL();
    return GC_OK;
}

static int enqueue_segments(gc_graph* g, bool clear) {
    int ge = grid_elems(g, std::max<long long>(g->keys.cap, 1));
    if (clear) {
        pdl_launch(k_batch_clear_segments, dim3(ge), dim3(TPB), 0, g->s, g->srcA.p, &g->ctl->nA2, g->segA);
        pdl_launch(k_batch_clear_segments, dim3(ge), dim3(TPB), 0, g->s, g->srcD.p, &g->ctl->nD2, g->segD);
    } else {
        pdl_launch(k_batch_segments, dim3(ge), dim3(TPB), 0, g->s, g->srcA.p, &g->ctl->nA2, g->segA);
        pdl_launch(k_batch_segments, dim3(ge), dim3(TPB), 0, g->s, g->srcD.p, &g->ctl->nD2, g->segD);
    }
    g->launches += 2;
    CKL();
    return GC_OK;
}

// One batch of Algorithm 2, all stages, on g->s, taken from the run cursor
// of the device descriptor (captured once per batch shape, replayed per
// batch).  Grids are sized for batches of up to max_nk directed keys; the
// actual sizes are read on the device.
//   commit:     apply G <- G \ D u A (else an independent what-if batch)
//   timed:      record the stage events (event-record nodes in the graph)
//   local:      the edge-local delta instead of the region recount
// role 0: the batch as Algorithm 2 (region, recount of G_a and G_b, commit);
// the two-batch form (sequential runs whose regions cover the graph): role 1
// normalises and commits the first batch of a pair without counting, role 2
// counts the second over every vertex (C_b = the whole graph after the first
// batch, C_a = after the second) and commits it; role 3 (independent runs):
// the twin pass, batches cur and cur + 1 keyed together with a batch tag and
// counted over every vertex, G_a = G with the first, G_b = G with the second
// (no commit).
static int enqueue_batch(gc_graph* g, long long max_nk, bool commit, bool timed, bool local = false,
                         bool t2 = false, int role = 0) {
    cudaStream_t s = g->s;
    if (timed) CK(record_stage(g->ev[0], s));
    const bool twin = role == 3;
    if (twin) pdl_launch(k_begin_twin, dim3(1), dim3(32), 0, s, g->ctl, g->desc);
    else pdl_launch(k_begin_batch, dim3(1), dim3(32), 0, s, g->ctl, g->desc);
    g->launches++;
    const long long nkb = std::max<long long>(max_nk, 1);
    const int ge = grid_elems(g, nkb);
    if (max_nk > 0) {
        if (twin)
            pdl_launch(k_batch_keys_twin, dim3(grid_elems(g, nkb / 2)), dim3(TPB), 0, s, g->ctl, g->perm, g->n, g->S,
                       g->keys.p);
        else
            pdl_launch(k_batch_keys, dim3(grid_elems(g, nkb / 2)), dim3(TPB), 0, s, g->ctl, g->perm, g->n, g->S,
                       g->keys.p);
        g->launches++;
        g->launches += radix_sort_u64(g->keys.p, g->keys_tmp.p, &g->ctl->nkeys, nkb, 2 * g->S + (twin ? 2 : 1),
                                      g->hist.p, radix_grid(nkb, g->sms), s);
        if (twin)
            pdl_launch(k_batch_decide_twin, dim3(ge), dim3(TPB), 0, s, g->keys.p, g->ctl, g->S, g->row_start, g->deg,
                       g->col, g->keepA.p, g->keepD.p);
        else
            pdl_launch(k_batch_decide, dim3(ge), dim3(TPB), 0, s, g->keys.p, g->ctl, g->S, g->row_start, g->deg,
                       g->col, g->keepA.p, g->keepD.p);
        g->launches++;
        int sg = scan_grid(nkb, g->sms);
        g->launches += scan_i32_to_i64(g->keepA.p, g->posA.p, &g->ctl->nkeys, 0, g->bsum.p, sg, &g->ctl->nA2, s);
        g->launches += scan_i32_to_i64(g->keepD.p, g->posD.p, &g->ctl->nkeys, 0, g->bsum.p, sg, &g->ctl->nD2, s);
        if (twin)
            pdl_launch(k_batch_compact_twin, dim3(ge), dim3(TPB), 0, s, g->keys.p, g->ctl, g->S, g->keepA.p,
                       g->keepD.p, g->posA.p, g->posD.p, g->srcA.p, g->dstA.p, g->srcD.p, g->dstD.p);
        else
            pdl_launch(k_batch_compact, dim3(ge), dim3(TPB), 0, s, g->keys.p, g->ctl, g->S, g->keepA.p, g->keepD.p,
                       g->posA.p, g->posD.p, g->srcA.p, g->dstA.p, g->srcD.p, g->dstD.p);
        g->launches++;
        int rc = enqueue_segments(g, false);
        if (rc) return rc;
    }
    if (timed) CK(record_stage(g->ev[1], s));
    CK(cudaMemsetAsync(g->visited, 0, sizeof(uint32_t) * (size_t)((g->n + 31) / 32 + 1), s));
    pdl_launch(k_bfs_sources, dim3(ge), dim3(TPB), 0, s, g->ctl, g->srcA.p, g->srcD.p, g->visited, g->wlist);
    pdl_launch(k_level_mark, dim3(1), dim3(1), 0, s, g->ctl, 0);
    g->launches += 2;
    if (role == 2 || role == 3) {
        pdl_launch(k_region_rest, dim3(grid_elems(g, g->n)), dim3(TPB), 0, s, g->ctl, g->n, g->visited, g->wlist);
        g->launches++;
    }
    for (int L = 1; L <= (local || role == 1 ? 0 : g->hops); L++) {
        if (role == 0) {
            pdl_launch(k_bfs_expand, dim3(grid_warps(g)), dim3(TPB), 0, s, g->ctl, L, g->row_start, g->deg, g->col,
                       g->visited, g->wlist);
            g->launches++;
        }
        pdl_launch(k_level_mark, dim3(1), dim3(1), 0, s, g->ctl, L);
        g->launches++;
    }
    CKL();
    if (timed) CK(record_stage(g->ev[2], s));
    int rc = GC_OK;
    if (role != 1) {
        rc = local ? count_local(g, commit ? 1 : 0, timed, t2)
                   : count_region(g, role == 2 ? 3 : role == 3 ? 4 : (commit ? 0 : 2), false, timed, twin,
                                  role == 2);
        if (rc) return rc;
    }
    if (!local && commit && t2 && role == 0) {
        // keep the triangle sums of the edge-local path
        CK(cudaMemsetAsync(g->visited2, 0, sizeof(uint32_t) * (size_t)((g->n + 31) / 32 + 1), s));
        pdl_launch(k_t2_mark, dim3(grid_warps(g)), dim3(TPB), 0, s, g->ctl, g->wlist, g->visited2, g->T2);
        pdl_launch(k_t2_from_region, dim3(grid_warps(g)), dim3(TPB), 0, s, g->ctl, g->wlist, g->U_off, g->U_col.p,
                   g->U_split,
                                                       g->tpack.p, g->visited2, g->T2);
        g->launches += 2;
        CKL();
    }
    if (commit) {
        rc = enqueue_commit(g);
        if (rc) return rc;
    }
    if (timed) CK(record_stage(g->ev[7], s));
    if (max_nk > 0) {
        rc = enqueue_segments(g, true);
        if (rc) return rc;
    }
    pdl_launch(k_end_batch, dim3(1), dim3(32), 0, s, g->ctl, g->out_dev.p, commit ? 1 : 0,
               role == 2 ? 1 : role == 3 ? 2 : 0);
    g->launches++;
    CKL();
    return GC_OK;
}

// Re-lay every row with fresh slack; the pool beyond the rows gets
// pool_extra slots more than the usual slack share.
static int relayout(gc_graph* g, long long pool_extra) {
    cudaStream_t s = g->s;
    int n = g->n;
    long long* new_start = (long long*)dalloc(g, sizeof(long long) * (size_t)(n + 1));
    if (!new_start) return nomem(g, "row offsets");
    pdl_launch(k_slack_caps, dim3(grid_elems(g, n)), dim3(TPB), 0, s, g->deg, n, g->slack, g->cap);
    scan_i32_to_i64(g->cap, new_start, nullptr, n, g->bsum.p, scan_grid(n, g->sms), nullptr, s);
    long long total = 0;
    CK(cudaMemcpyAsync(&total, new_start + n, sizeof(long long), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    long long pool = std::max<long long>((long long)(total * g->slack), 4096) + pool_extra;
    long long ncap = total + pool;
    int32_t* ncol = (int32_t*)dalloc(g, sizeof(int32_t) * (size_t)ncap);
    if (!ncol) {
        dfree(g, new_start);
        return nomem(g, "adjacency pool");
    }
    pdl_launch(k_copy_rows, dim3(grid_warps(g)), dim3(TPB), 0, s, g->deg, n, g->row_start, g->col, new_start, ncol);
    pdl_launch(k_commit_reset, dim3(1), dim3(32), 0, s, g->ctl, (unsigned long long)total, 1);
    CKL();
    dfree(g, g->col);
    dfree(g, g->row_start);
    g->col = ncol;
    g->row_start = new_start;
    g->col_capacity = ncap;
    g->buf_gen++;  // captured graphs hold the old adjacency pointers
    return GC_OK;
}

static int read_ctl(gc_graph* g) {
    CK(cudaMemcpyAsync(g->h_ctl, g->ctl, offsetof(Ctl, accs), cudaMemcpyDeviceToHost, g->s));
    CK(cudaStreamSynchronize(g->s));
    return GC_OK;
}

// A commit ran out of pool space: the rows are untouched.  Grow the pool and
// commit the pending batch again (its kept entries are still in scratch).
static int finish_pending_commit(gc_graph* g, int* relayouts) {
    for (int tries = 0;; tries++) {
        const Ctl& c = *g->h_ctl;
        long long extra = 4 * (c.pend_nA2 + c.pend_nD2) + 1024;
        for (int i = 0; i < tries; i++) extra *= 2;
        int rc = relayout(g, extra);
        if (rc) return rc;
        (*relayouts)++;
        pdl_launch(k_resume_pending, dim3(1), dim3(32), 0, g->s, g->ctl);
        pdl_launch(k_halt_clear, dim3(1), dim3(32), 0, g->s, g->ctl);
        CKL();
        rc = enqueue_segments(g, false);
        if (rc) return rc;
        rc = enqueue_commit(g);
        if (rc) return rc;
        rc = read_ctl(g);
        if (rc) return rc;
        if (!g->h_ctl->overflow) break;
        if (tries >= 4) {
            g->err = "adjacency pool could not be grown enough";
            return GC_ENOMEM;
        }
    }
    int rc = enqueue_segments(g, true);
    if (rc) return rc;
    pdl_launch(k_halt_clear, dim3(1), dim3(32), 0, g->s, g->ctl);
    CKL();
    return read_ctl(g);
}

static float elapsed(cudaEvent_t a, cudaEvent_t b) {
    float x = 0.f;
    if (cudaEventElapsedTime(&x, a, b) != cudaSuccess) {
        cudaGetLastError();  // a stage the call did not run; not an error of the call
        x = 0.f;
    }
    return x;
}

// Stage times of gc_stats.ms_stage from the boundary events ev[lo .. hi].
// The triangle stage (ev3 -> ev4) and the 4-cycle stage (ev3 -> ev5) run
// side by side from the same fork; the edge terms start after both.
static void stage_times(gc_graph* g, int lo, int hi) {
    for (int i = 0; i < 8; i++) g->st.ms_stage[i] = 0.f;
    for (int i = lo; i < hi; i++) {
        if (i == 4) g->st.ms_stage[4] = elapsed(g->ev[3], g->ev[5]);
        else if (i == 5) g->st.ms_stage[5] = std::min(elapsed(g->ev[4], g->ev[6]), elapsed(g->ev[5], g->ev[6]));
        else g->st.ms_stage[i] = elapsed(g->ev[i], g->ev[i + 1]);
    }
    // the heavy-pivot 4-cycle kernels alone, on their own stream
    if (lo <= 4 && hi > 4) g->st.ms_stage[7] = elapsed(g->ev[8], g->ev[9]);
}

static void fill_stats(gc_graph* g, const Ctl& c) {
    gc_stats& t = g->st;
    t.n_ins = c.nA2 / 2;
    t.n_del = c.nD2 / 2;
    t.repeats = (long long)c.st[0] / 2;
    t.cancelled = (long long)c.st[1] / 2;
    t.noop_ins = (long long)c.st[2] / 2;
    t.noop_del = (long long)c.st[3] / 2;
    t.region_vertices = c.nW;
    t.region_entries = c.nU;
    t.edges_a = (long long)c.acc[12];
    t.edges_b = (long long)c.acc[13];
    t.work_triangles = (long long)c.acc[14];
    t.work_wedges = (long long)c.acc[15];
    t.work_wedges_heavy = (long long)c.acc[20];
    t.l2_red_heavy = (long long)c.acc[21];
    t.l2_atom_heavy = (long long)c.acc[22];
    for (int i = 0; i < 6; i++) {
        t.Ca[i] = c.Ca[i];
        t.Cb[i] = c.Cb[i];
        t.sums_a[i] = c.sa[i];
        t.sums_b[i] = c.sb[i];
    }
    for (int i = 0; i < 2; i++) {
        t.C3a[i] = c.C3a[i];
        t.C3b[i] = c.C3b[i];
    }
}

// Capture the per-batch launch sequence (batch from the run cursor) into
// *exec; timed: with the stage events as event-record nodes.
static int capture_batch(gc_graph* g, long long shape_nk, bool commit, bool timed, cudaGraphExec_t* exec,
                         int* launches, bool local = false, bool t2 = false, int role = 0) {
    cudaStream_t s = g->s;
    if (*exec) {
        cudaGraphExecDestroy(*exec);
        *exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const int lsave = g->launches;
    g->launches = 0;
    int rc = enqueue_batch(g, shape_nk, commit, timed, local, t2, role);
    cudaError_t ce = cudaStreamEndCapture(s, &graph);
    *launches = g->launches;
    g->launches = lsave;
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (ce != cudaSuccess) {
        g->err = std::string("graph capture: ") + cudaGetErrorString(ce);
        return GC_ECUDA;
    }
    ce = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
        *exec = nullptr;
        g->err = std::string("graph instantiate: ") + cudaGetErrorString(ce);
        return GC_ECUDA;
    }
    return GC_OK;
}

// One batch whose pairs are already in device memory (plain form): the
// batch's launch sequence is captured once per batch shape (grids sized for
// the next power of two of its keys) with its stage events, then replayed
// with the batch described on the device.
static int apply_device(gc_graph* g, const int32_t* d_ins, long long n_ins, const int32_t* d_del,
                        long long n_del, int commit, uint64_t out[6]) {
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = g->s;
    const long long nk = 2 * (n_ins + n_del);
    long long shape_nk = 1;
    while (shape_nk < nk) shape_nk <<= 1;
    int rc = plan_batch_buffers(g, shape_nk);
    if (rc) return rc;
    rc = plan_region_buffers(g, g->m, n_ins);
    if (rc) return rc;
    rc = ensure_desc(g, 6);
    if (rc) return rc;
    if (!ensure(g, g->out_dev, 6)) return nomem(g, "batch results");
    // small batches may take the edge-local delta (same counts, work
    // proportional to the rows the batch touches instead of a region)
    bool local = g->opt.local_max_pairs > 0 && n_ins + n_del <= (long long)g->opt.local_max_pairs;
    for (int attempt = 0;; attempt++) {
        if (local && ensure_local(g, std::max<long long>(g->l_cap, 1LL << 20)) != GC_OK) {
            g->err.clear();  // no room for the local scratch: the region form does the batch
            local = false;
        }
        cudaGraphExec_t* ex = local ? &g->lexec : &g->pexec;
        long long* ex_nk = local ? &g->l_nk : &g->p_nk;
        int* ex_commit = local ? &g->l_commit : &g->p_commit;
        unsigned long long* ex_gen = local ? &g->l_gen : &g->p_gen;
        int* ex_launches = local ? &g->l_launches : &g->p_launches;
        // maintained triangle sums: used by the local form, kept by the
        // region form while the local form is enabled
        const bool t2 = g->t2_valid && (local || g->opt.local_max_pairs > 0);
        int* ex_t2 = local ? &g->l_t2 : &g->p_t2;
        if (!*ex || *ex_nk != shape_nk || *ex_commit != commit || *ex_gen != g->buf_gen || *ex_t2 != (int)t2) {
            rc = capture_batch(g, shape_nk, commit != 0, true, ex, ex_launches, local, t2);
            if (rc) return rc;
            *ex_nk = shape_nk;
            *ex_commit = commit;
            *ex_gen = g->buf_gen;
            *ex_t2 = (int)t2;
        }
        g->h_desc[0] = (long long)d_ins;
        g->h_desc[1] = (long long)d_del;
        g->h_desc[2] = 0;
        g->h_desc[3] = n_ins;
        g->h_desc[4] = 0;
        g->h_desc[5] = n_del;
        CK(cudaMemcpyAsync(g->desc, g->h_desc, 6 * sizeof(long long), cudaMemcpyHostToDevice, s));
        pdl_launch(k_run_reset, dim3(1), dim3(32), 0, s, g->ctl);
        CKL();
        g->launches = *ex_launches + 1;
        CK(cudaEventRecord(g->e0, s));
        CK(cudaGraphLaunch(*ex, s));
        CK(cudaEventRecord(g->e1, s));
        rc = read_ctl(g);
        if (rc) return rc;
        if (g->h_ctl->err) {
            g->err = "batch rejected on the device: a pair is a self-loop or names a vertex outside [0, n)";
            return GC_EINVAL;
        }
        if (!(local && g->h_ctl->lovf)) break;
        // the local scratch was too small and nothing was applied: grow it
        // to what the batch needed (each of the two bound checks can report
        // its own need), else take the region path
        const long long need = g->h_ctl->l_need;
        if (attempt >= 2 || ensure_local(g, need + need / 4 + 1024) != GC_OK) {
            g->err.clear();
            local = false;
        }
    }
    int relayouts = 0;
    if (commit && g->h_ctl->overflow) {
        rc = finish_pending_commit(g, &relayouts);
        if (rc) return rc;
    }
    Ctl c = *g->h_ctl;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, g->e0, g->e1);
    fill_stats(g, c);
    g->st.n_ins_raw = n_ins;
    g->st.n_del_raw = n_del;
    g->st.ms_device = ms;
    g->st.relayouts = relayouts;
    g->st.launches = g->launches;
    // [0] normalise: ev0->ev1, [1] region: ev1->ev2, [2] union graph: ev2->ev3,
    // [3] triangles: ev3->ev4, [4] 4-cycles: ev4->ev5, [5] terms: ev5->ev6, [6] commit: ev6->ev7
    // (the edge-local path runs its stages one after the other)
    if (local) {
        for (int i = 0; i < 8; i++) g->st.ms_stage[i] = i < 7 ? elapsed(g->ev[i], g->ev[i + 1]) : 0.f;
    } else {
        stage_times(g, 0, 7);
    }
    g->st.path = local ? 1 : 0;
    if (commit && !local && g->opt.local_max_pairs <= 0) g->t2_valid = false;  // not kept without the local form
    if (commit) {
        for (int i = 0; i < 6; i++) g->F[i] = c.F[i];
        for (int i = 0; i < 2; i++) g->F3[i] = c.F3[i];
        g->m += c.nA2 / 2 - c.nD2 / 2;
    }
    g->st.num_edges = g->m;
    if (out)
        for (int i = 0; i < 6; i++) out[i] = c.last_out[i];
    g->st.ms_wall = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return GC_OK;
}

// Batched form: k batches whose pairs are in device memory, described by
// h_batches[k][4] = {ins_off, n_ins, del_off, n_del} (in pairs, relative to
// d_ins / d_del).  One captured graph per batch shape, replayed k times.
static int apply_batches_region(gc_graph* g, const int32_t* d_ins, const int32_t* d_del, const long long* h_batches,
                                int k, int independent, uint64_t* out) {
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = g->s;
    const bool commit = !independent;
    // the triangle sums of the edge-local form are kept while it is enabled
    const bool t2 = g->t2_valid && g->opt.local_max_pairs > 0;
    if (commit && !t2) g->t2_valid = false;
    long long max_nk = 0, max_ins = 0, sum_ins = 0, raw_ins = 0, raw_del = 0;
    for (int i = 0; i < k; i++) {
        long long ni = h_batches[4 * i + 1], nd = h_batches[4 * i + 3];
        max_nk = std::max(max_nk, 2 * (ni + nd));
        max_ins = std::max(max_ins, ni);
        sum_ins += ni;
        raw_ins = ni;
        raw_del = nd;
    }
    // grids are sized by powers of two of the largest batch, so runs of
    // similar shape share one captured graph
    long long shape_nk = 1;
    while (shape_nk < max_nk) shape_nk <<= 1;
    int rc = GC_OK;
    int relayouts = 0;
    if (commit && sum_ins > 0) {
        // room for the whole run's insertions and the rows they relocate, so
        // the replays are not halted by a full pool mid-run
        const long long need = 8 * sum_ins;
        const long long pool_free = g->col_capacity - (long long)g->h_ctl->pool_tail;
        if (pool_free < need) {
            rc = relayout(g, need);
            if (rc) return rc;
            relayouts++;
        }
    }
    // the twin pass of independent runs keys two batches at once
    const bool twin_ok = !commit && k >= 3 && g->pair_min_share > 0 && g->n < (1 << 29);
    long long twin_nk = 1;
    if (twin_ok)
        while (twin_nk < 2 * max_nk) twin_nk <<= 1;
    rc = plan_batch_buffers(g, twin_ok ? twin_nk : shape_nk);
    if (rc) return rc;
    rc = plan_region_buffers(g, g->m + (commit ? sum_ins : (twin_ok ? 2 : 1) * max_ins), (twin_ok ? 2 : 1) * max_ins);
    if (rc) return rc;
    rc = ensure_desc(g, 2 + 4LL * k);
    if (rc) return rc;
    if (!ensure(g, g->out_dev, (size_t)6 * std::max(k, 1))) return nomem(g, "batch results");
    g->h_desc[0] = (long long)d_ins;
    g->h_desc[1] = (long long)d_del;
    std::memcpy(g->h_desc + 2, h_batches, sizeof(long long) * 4 * (size_t)k);
    CK(cudaMemcpyAsync(g->desc, g->h_desc, sizeof(long long) * (2 + 4 * (size_t)k), cudaMemcpyHostToDevice, s));
    pdl_launch(k_run_reset, dim3(1), dim3(32), 0, s, g->ctl);
    CKL();
    // (re)capture the per-batch graph when its shape or any buffer changed
    if (!g->gexec || g->g_nk != shape_nk || g->g_commit != (int)commit || g->g_gen != g->buf_gen ||
        g->g_t2 != (int)t2) {
        rc = capture_batch(g, shape_nk, commit, false, &g->gexec, &g->g_launches, false, t2);
        if (rc) return rc;
        g->g_nk = shape_nk;
        g->g_commit = (int)commit;
        g->g_gen = g->buf_gen;
        g->g_t2 = (int)t2;
    }
    // the two-batch form: a sequential run of at least three batches whose
    // pairs pass the device check (a bad pair makes its batch a no-op, which
    // the pairing does not model).  Batch 0 runs as Algorithm 2 and its region
    // decides whether the rest go in pairs; a run whose batch 0 is at least as
    // large as the first batch of an earlier run that went in pairs starts
    // them at batch 0 (regions grow with their endpoints, and a pair is exact
    // whatever the region: the choice is one of speed only).
    bool pair_ok = (commit || twin_ok) && k >= 3 && g->pair_min_share > 0;
    const long long size0 = h_batches[1] + h_batches[3];
    if (pair_ok) {
        CK(cudaMemsetAsync(g->hist.p, 0, sizeof(int), s));
        k_run_pairs_check<<<dim3(64, (unsigned)std::min(k, 64)), TPB, 0, s>>>(g->desc, k, g->n, (int*)g->hist.p);
        CKL();
        int bad = 0;
        CK(cudaMemcpyAsync(&bad, g->hist.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        pair_ok = bad == 0;
    }
    bool pairs = false;  // batches base .. k-1 go in pairs
    int base = 1;
    if (pair_ok && g->pair_hint > 0 && size0 >= g->pair_hint) {
        pairs = true;
        base = 0;
        pair_ok = false;
    }
    int pairs_used = 0;
    auto role_of = [&](int i) {
        if (!pairs || i < base) return 0;
        if ((i - base) % 2 == 0) return i + 1 < k ? (commit ? 1 : 3) : 0;
        return 2;  // (independent runs never reach this: a twin pass takes two batches)
    };
    auto ensure_exec = [&](int role) -> int {
        if (role == 0) return GC_OK;
        const int q = role - 1;
        const long long nk = role == 3 ? twin_nk : shape_nk;
        if (!g->qexec[q] || g->q_nk[q] != nk || g->q_gen[q] != g->buf_gen) {
            int r = capture_batch(g, nk, role != 3, false, &g->qexec[q], &g->q_launches[q], false, false, role);
            if (r) return r;
            g->q_nk[q] = nk;
            g->q_gen[q] = g->buf_gen;
        }
        return GC_OK;
    };
    CK(cudaEventRecord(g->e0, s));
    int done = 0;
    long long launches = 0;
    while (done < k) {
        const int upto = (pair_ok && !pairs && done == 0) ? 1 : k;
        for (int i = done; i < upto;) {
            const int role = role_of(i);
            rc = ensure_exec(role);
            if (rc) return rc;
            CK(cudaGraphLaunch(role == 0 ? g->gexec : g->qexec[role - 1], s));
            launches += role == 0 ? g->g_launches : g->q_launches[role - 1];
            pairs_used += (role == 2 || role == 3) ? 1 : 0;
            i += role == 3 ? 2 : 1;
        }
        rc = read_ctl(g);
        if (rc) return rc;
        done = g->h_ctl->cur;
        if (pair_ok && !pairs && upto == 1 && done >= 1) {
            // batch 0's region against the graph's adjacency entries
            pairs = (double)g->h_ctl->nU * 1000.0 >= (double)g->pair_min_share * 2.0 * (double)g->m;
            pair_ok = false;
            if (pairs) g->pair_hint = g->pair_hint > 0 ? std::min(g->pair_hint, size0) : size0;
        }
        if (g->h_ctl->halt) {
            // batch done-1 is counted (or, first of a pair, only normalised)
            // but its commit waits for pool space
            rc = finish_pending_commit(g, &relayouts);
            if (rc) return rc;
            if (g->g_gen != g->buf_gen) {
                // the adjacency moved: capture again for the remaining batches
                rc = capture_batch(g, shape_nk, commit, false, &g->gexec, &g->g_launches, false, t2);
                if (rc) return rc;
                g->g_gen = g->buf_gen;
            }
        }
    }
    if (pairs_used && commit) g->t2_valid = false;  // first batches of pairs did not keep the triangle sums
    CK(cudaEventRecord(g->e1, s));
    std::vector<unsigned long long> res((size_t)6 * std::max(k, 1));
    CK(cudaMemcpyAsync(res.data(), g->out_dev.p, sizeof(unsigned long long) * 6 * (size_t)k, cudaMemcpyDeviceToHost,
                       s));
    rc = read_ctl(g);
    if (rc) return rc;
    const Ctl& c = *g->h_ctl;
    if (commit) {
        for (int i = 0; i < 6; i++) g->F[i] = c.F[i];
        for (int i = 0; i < 2; i++) g->F3[i] = c.F3[i];
        g->m += c.m_delta;
    }
    if (out)
        for (long long i = 0; i < 6LL * k; i++) out[i] = (uint64_t)res[(size_t)i];
    float ms = 0.f;
    cudaEventElapsedTime(&ms, g->e0, g->e1);
    fill_stats(g, c);
    g->st.n_ins_raw = raw_ins;
    g->st.n_del_raw = raw_del;
    g->st.ms_device = ms;
    g->st.relayouts = relayouts;
    g->st.launches = (int)launches;
    g->st.path = pairs_used ? 2 : 0;
    for (int i = 0; i < 8; i++) g->st.ms_stage[i] = 0.f;
    g->st.num_edges = g->m;
    g->st.ms_wall = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return GC_OK;
}

static int count_static(gc_graph* g, bool set_F, uint64_t out[6]) {
    cudaStream_t s = g->s;
    int rc = plan_region_buffers(g, g->m, 0);
    if (rc) return rc;
    g->launches = 0;
    CK(cudaMemsetAsync(g->visited, 0xFF, sizeof(uint32_t) * (size_t)((g->n + 31) / 32 + 1), s));
    pdl_launch(k_region_all, dim3(grid_elems(g, g->n)), dim3(TPB), 0, s, g->ctl, g->n, g->wlist);
    pdl_launch(k_mark_active, dim3(1), dim3(32), 0, s, g->ctl);
    g->launches += 2;
    CKL();
    CK(cudaEventRecord(g->ev[2], s));
    rc = count_region(g, 1, set_F, true, false, true);
    if (rc) return rc;
    // the static pass also gives the triangle sums of the edge-local path
    CK(cudaMemsetAsync(g->T2, 0, 8 * (size_t)std::max(g->n, 1), s));
    pdl_launch(k_t2_from_static, dim3(grid_warps(g)), dim3(TPB), 0, s, g->ctl, g->wlist, g->U_off, g->U_col.p,
               g->U_split, g->tpack.p,
                                                   g->T2);
    g->launches++;
    CKL();
    rc = read_ctl(g);
    if (rc) return rc;
    g->t2_valid = true;
    if (out)
        for (int i = 0; i < 6; i++) out[i] = (uint64_t)g->h_ctl->Ca[i];
    if (set_F) {
        for (int i = 0; i < 6; i++) g->F[i] = (uint64_t)g->h_ctl->Ca[i];
        for (int i = 0; i < 2; i++) g->F3[i] = (uint64_t)g->h_ctl->C3a[i];
    }
    // a static count leaves its stage times in the stats record
    stage_times(g, 2, 6);
    if (cudaEventElapsedTime(&g->st.ms_device, g->ev[2], g->ev[6]) != cudaSuccess) cudaGetLastError();
    fill_stats(g, *g->h_ctl);
    g->st.launches = g->launches;
    return GC_OK;
}

// ---------------------------------------------------------------------------
// open / close
// ---------------------------------------------------------------------------
static void destroy(gc_graph* g) {
    if (!g) return;
    if (g->s) cudaStreamSynchronize(g->s);
    if (g->gexec) cudaGraphExecDestroy(g->gexec);
    for (int i = 0; i < 3; i++)
        if (g->qexec[i]) cudaGraphExecDestroy(g->qexec[i]);
    if (g->pexec) cudaGraphExecDestroy(g->pexec);
    if (g->lexec) cudaGraphExecDestroy(g->lexec);
    release_local(g);
    int32_t* p32[] = {g->perm, g->iperm, g->deg, g->cap, g->col, g->wlist, g->U_deg, g->U_split, g->da, g->db};
    for (auto p : p32) dfree(g, p);
    dfree(g, g->row_start);
    dfree(g, g->U_off);
    dfree(g, g->U_wt);
    dfree(g, g->ctl);
    dfree(g, g->desc);
    dfree(g, g->segA);
    dfree(g, g->segD);
    dfree(g, g->visited);
    dfree(g, g->visited2);
    dfree(g, g->T2);
    dfree(g, g->dtri2);
    release(g, g->U_col);
    release(g, g->tpack);
    release(g, g->keys);
    release(g, g->keys_tmp);
    release(g, g->keepA);
    release(g, g->keepD);
    release(g, g->srcA);
    release(g, g->dstA);
    release(g, g->srcD);
    release(g, g->dstD);
    release(g, g->plan_cap);
    release(g, g->plan_deg);
    release(g, g->pairs);
    release(g, g->posA);
    release(g, g->posD);
    release(g, g->plan_dst);
    release(g, g->plan_scr);
    release(g, g->bsum);
    release(g, g->hist);
    release(g, g->out_dev);
    release(g, g->vids);
    release(g, g->vdeg);
    release(g, g->voff);
    release(g, g->dense);
    release(g, g->cta_tables);
    release(g, g->chunk_table);
    dfree(g, g->bins);
    if (g->s) cudaStreamSynchronize(g->s);
    if (g->h_ctl) cudaFreeHost(g->h_ctl);
    if (g->h_desc) cudaFreeHost(g->h_desc);
    if (g->e0) cudaEventDestroy(g->e0);
    for (auto e : g->ev)
        if (e) cudaEventDestroy(e);
    if (g->e1) cudaEventDestroy(g->e1);
    for (int i = 0; i < 3; i++) {
        if (g->aux[i]) cudaStreamDestroy(g->aux[i]);
        if (g->join[i]) cudaEventDestroy(g->join[i]);
    }
    if (g->fork) cudaEventDestroy(g->fork);
    if (g->own_stream && g->s) cudaStreamDestroy(g->s);
    delete g;
}

static int open_device(gc_graph* g, const int32_t* row_ptr, const int32_t* colh) {
    const int n = g->n;
    const long long m2 = n > 0 ? row_ptr[n] : 0;
    cudaStream_t s = g->s;
    size_t nn = (size_t)std::max(n, 1);
    g->perm = (int32_t*)dalloc(g, 4 * nn);
    g->iperm = (int32_t*)dalloc(g, 4 * nn);
    g->deg = (int32_t*)dalloc(g, 4 * nn);
    g->cap = (int32_t*)dalloc(g, 4 * nn);
    g->wlist = (int32_t*)dalloc(g, 4 * nn);
    g->U_deg = (int32_t*)dalloc(g, 4 * nn);
    g->U_split = (int32_t*)dalloc(g, 4 * nn);
    g->da = (int32_t*)dalloc(g, 4 * nn);
    g->db = (int32_t*)dalloc(g, 4 * nn);
    g->row_start = (long long*)dalloc(g, 8 * (nn + 1));
    g->U_off = (long long*)dalloc(g, 8 * (nn + 1));
    g->U_wt = (long long*)dalloc(g, 8 * nn);
    g->ctl = (Ctl*)dalloc(g, sizeof(Ctl));
    g->segA = (int2*)dalloc(g, sizeof(int2) * nn);
    g->segD = (int2*)dalloc(g, sizeof(int2) * nn);
    g->visited = (uint32_t*)dalloc(g, 4 * ((nn + 31) / 32 + 1));
    g->visited2 = (uint32_t*)dalloc(g, 4 * ((nn + 31) / 32 + 1));
    g->T2 = (unsigned long long*)dalloc(g, 8 * nn);
    g->dtri2 = (long long*)dalloc(g, 8 * nn);
    if (!g->visited2 || !g->T2 || !g->dtri2) return nomem(g, "triangle sums");
    CK(cudaMemsetAsync(g->dtri2, 0, 8 * nn, s));
    CK(cudaMemsetAsync(g->T2, 0, 8 * nn, s));
    if (!g->perm || !g->iperm || !g->deg || !g->cap || !g->wlist || !g->U_deg || !g->U_split || !g->da || !g->db ||
        !g->row_start || !g->U_off || !g->U_wt || !g->ctl || !g->segA || !g->segD || !g->visited)
        return nomem(g, "graph state");
    if (ensure_desc(g, 16)) return GC_ENOMEM;
    if (!ensure(g, g->bsum, 1024)) return nomem(g, "scan scratch");
    CK(cudaMemsetAsync(g->segA, 0, sizeof(int2) * nn, s));
    CK(cudaMemsetAsync(g->segD, 0, sizeof(int2) * nn, s));
    Ctl zero{};
    *g->h_ctl = zero;
    CK(cudaMemcpyAsync(g->ctl, g->h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, s));

    // temporaries of the open
    int32_t* d_rp = (int32_t*)dalloc(g, 4 * (nn + 1));
    int32_t* d_col = (int32_t*)dalloc(g, 4 * (size_t)std::max<long long>(m2, 1));
    int32_t* deg0 = (int32_t*)dalloc(g, 4 * nn);
    long long* key_off = (long long*)dalloc(g, 8 * (nn + 1));
    int* bad = (int*)dalloc(g, sizeof(int));
    size_t kcount = (size_t)std::max<long long>(std::max<long long>(m2, n), 1);
    uint64_t* k1 = (uint64_t*)dalloc(g, 8 * kcount);
    uint64_t* k2 = (uint64_t*)dalloc(g, 8 * kcount);
    int rg = radix_grid((long long)kcount, g->sms);
    if (!d_rp || !d_col || !deg0 || !key_off || !bad || !k1 || !k2 || !ensure(g, g->hist, (size_t)256 * rg)) {
        dfree(g, d_rp); dfree(g, d_col); dfree(g, deg0); dfree(g, key_off); dfree(g, bad); dfree(g, k1); dfree(g, k2);
        return nomem(g, "open scratch");
    }
    int rc = GC_OK;
    do {
        if (n > 0) {
            if (cudaMemcpyAsync(d_rp, row_ptr, 4 * (size_t)(n + 1), cudaMemcpyHostToDevice, s) != cudaSuccess ||
                (m2 > 0 && cudaMemcpyAsync(d_col, colh, 4 * (size_t)m2, cudaMemcpyHostToDevice, s) != cudaSuccess)) {
                g->err = "copying the CSR to the device failed";
                rc = GC_ECUDA;
                break;
            }
        }
        if (cudaMemsetAsync(bad, 0, sizeof(int), s) != cudaSuccess) { rc = GC_ECUDA; break; }
        // internal order: ascending initial degree, ties by id
        long long maxdeg = 0;
        for (int v = 0; v < n; v++) maxdeg = std::max<long long>(maxdeg, (long long)row_ptr[v + 1] - row_ptr[v]);
        g->h_desc[8] = n;
        g->h_desc[9] = m2;
        if (cudaMemcpyAsync(g->desc + 8, g->h_desc + 8, 2 * sizeof(long long), cudaMemcpyHostToDevice, s) !=
            cudaSuccess) { rc = GC_ECUDA; break; }
        if (n > 0) {
            pdl_launch(k_degree_keys, dim3(grid_elems(g, n)), dim3(TPB), 0, s, d_rp, n, deg0, k1);
            radix_sort_u64(k1, k2, g->desc + 8, n, 32 + bitlen(maxdeg), g->hist.p, radix_grid(n, g->sms), s);
            pdl_launch(k_perm_from_keys, dim3(grid_elems(g, n)), dim3(TPB), 0, s, k1, n, g->perm, g->iperm, deg0,
                       g->deg);
        }
        if (m2 > 0) {
            pdl_launch(k_edge_keys, dim3(grid_warps(g)), dim3(TPB), 0, s, d_rp, d_col, n, g->perm, g->S, k1, bad);
            radix_sort_u64(k1, k2, g->desc + 9, m2, 2 * g->S, g->hist.p, rg, s);
        }
        if (n > 0) {
            scan_i32_to_i64(g->deg, key_off, nullptr, n, g->bsum.p, scan_grid(n, g->sms), nullptr, s);
            pdl_launch(k_slack_caps, dim3(grid_elems(g, n)), dim3(TPB), 0, s, g->deg, n, g->slack, g->cap);
            scan_i32_to_i64(g->cap, g->row_start, nullptr, n, g->bsum.p, scan_grid(n, g->sms), nullptr, s);
        }
        long long total = 0;
        if (n > 0 &&
            cudaMemcpyAsync(&total, g->row_start + n, sizeof(long long), cudaMemcpyDeviceToHost, s) != cudaSuccess) {
            rc = GC_ECUDA;
            break;
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            g->err = std::string("open: ") + cudaGetErrorString(cudaGetLastError());
            rc = GC_ECUDA;
            break;
        }
        long long pool = std::max<long long>((long long)(total * g->slack), 4096);
        g->col_capacity = total + pool;
        g->col = (int32_t*)dalloc(g, 4 * (size_t)g->col_capacity);
        if (!g->col) {
            rc = nomem(g, "adjacency");
            break;
        }
        if (m2 > 0)
            pdl_launch(k_fill_from_keys, dim3(grid_elems(g, m2)), dim3(TPB), 0, s, k1, m2, n, g->S, key_off,
                       g->row_start, g->col, bad);
        pdl_launch(k_commit_reset, dim3(1), dim3(32), 0, s, g->ctl, (unsigned long long)total, 1);
        int hbad = 0;
        if (cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            g->err = std::string("open: ") + cudaGetErrorString(cudaGetLastError());
            rc = GC_ECUDA;
            break;
        }
        if (hbad) {
            g->err = hbad == 1 ? "CSR has a self-loop or a neighbour outside [0, n)"
                     : hbad == 2 ? "CSR has a repeated entry in a row"
                                 : "CSR is not symmetric";
            rc = GC_EINVAL;
            break;
        }
    } while (0);
    cudaStreamSynchronize(s);
    dfree(g, d_rp); dfree(g, d_col); dfree(g, deg0); dfree(g, key_off); dfree(g, bad); dfree(g, k1); dfree(g, k2);
    if (rc) return rc;
    g->m = m2 / 2;
    // counting pass: work lists, one dense counter array per cluster of the
    // heaviest 4-cycle pivots and one hash table per CTA of the medium ones
    // (all kept zero between pivots)
    count_setup_attributes();
    local_setup_attributes();
    g->bins = (int32_t*)dalloc(g, sizeof(int32_t) * (size_t)NBINS * nn);
    g->dense_clusters = dense_cluster_plan(g->opt.dense_cluster, g->sms, &g->dense_cluster_size);
    if (!g->bins || !ensure(g, g->dense, (size_t)g->dense_clusters * (size_t)dense_stride((long long)nn)))
        return nomem(g, "counting work lists");
    CK(cudaMemsetAsync(g->dense.p, 0, 8 * g->dense.cap, s));
    g->cta_groups = g->sms;
    if (!ensure(g, g->cta_tables, (size_t)g->cta_groups * 2 * C4_T3)) return nomem(g, "4-cycle hash tables");
    if (g->tune.c4_chunk_min < NEVER && !ensure_chunk_table(g)) return nomem(g, "4-cycle chunk table");
    CK(cudaMemsetAsync(g->cta_tables.p, 0, 8 * g->cta_tables.cap, s));
    return count_static(g, true, nullptr);
}

// host-side checks of a batch's pairs
static int check_pairs(gc_graph* g, const int32_t* p, int64_t k, const char* what) {
    for (int64_t i = 0; i < k; i++) {
        int32_t a = p[2 * i], b = p[2 * i + 1];
        if (a < 0 || b < 0 || a >= g->n || b >= g->n || a == b) {
            g->err = std::string(what) + " " + std::to_string(i) +
                     " is a self-loop or names a vertex outside [0, n)";
            return GC_EINVAL;
        }
    }
    return GC_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
// Make the handle's device current for the calling thread (a thread other
// than the one that opened the handle starts on device 0).
static bool on_device(gc_graph* g) {
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess) return false;
    return d == g->dev || cudaSetDevice(g->dev) == cudaSuccess;
}

extern "C" {

void gc_default_options(gc_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->region_hops = 3;
    opt->slack = 0.25f;
}

int gc_open(int32_t n, const int32_t* row_ptr, const int32_t* col, const gc_options* opt, gc_graph** out) {
    t_open_error.clear();
    if (!out) {
        t_open_error = "out is NULL";
        return GC_EINVAL;
    }
    *out = nullptr;
    if (n < 0 || n >= (1 << 30)) {
        t_open_error = "n must be in [0, 2^30)";
        return GC_EINVAL;
    }
    if (n > 0 && !row_ptr) {
        t_open_error = "row_ptr is NULL";
        return GC_EINVAL;
    }
    if (n > 0) {
        if (row_ptr[0] != 0) {
            t_open_error = "row_ptr[0] must be 0";
            return GC_EINVAL;
        }
        for (int v = 0; v < n; v++)
            if (row_ptr[v + 1] < row_ptr[v]) {
                t_open_error = "row_ptr must be non-decreasing";
                return GC_EINVAL;
            }
        if (row_ptr[n] > 0 && !col) {
            t_open_error = "col is NULL";
            return GC_EINVAL;
        }
        if (row_ptr[n] % 2) {
            t_open_error = "CSR of an undirected graph has an even number of entries";
            return GC_EINVAL;
        }
    }
    gc_options o;
    gc_default_options(&o);
    if (opt) {
        o = *opt;
        if (o.region_hops == 0) o.region_hops = 3;
        if (o.slack <= 0.f) o.slack = 0.25f;
    }
    if (o.region_hops < 2 || o.region_hops > MAX_HOPS) {
        t_open_error = "region_hops must be in [2, 8]";
        return GC_EINVAL;
    }
    if ((o.alloc == nullptr) != (o.free == nullptr)) {
        t_open_error = "alloc and free callbacks come together";
        return GC_EINVAL;
    }
    if (o.dense_cluster != 0 && o.dense_cluster != 8 && o.dense_cluster != 16) {
        t_open_error = "dense_cluster must be 0, 8 or 16";
        return GC_EINVAL;
    }
    gc_graph* g = new gc_graph();
    g->opt = o;
    g->n = n;
    g->S = std::max(1, bitlen(n > 0 ? n - 1 : 0));
    if (o.chunk_threshold > 0) g->tune.c4_chunk_min = o.chunk_threshold;
    g->hops = o.region_hops;
    g->slack = o.slack;
    int rc = GC_OK;
    do {
        if (o.device > 0 && cudaSetDevice(o.device) != cudaSuccess) {
            t_open_error = "cudaSetDevice failed";
            rc = GC_ECUDA;
            break;
        }
        if (cudaGetDevice(&g->dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->dev) != cudaSuccess) {
            t_open_error = std::string("no usable CUDA device: ") + cudaGetErrorString(cudaGetLastError());
            rc = GC_ECUDA;
            break;
        }
        if (o.stream) {
            g->s = (cudaStream_t)o.stream;
        } else {
            if (cudaStreamCreateWithFlags(&g->s, cudaStreamNonBlocking) != cudaSuccess) {
                t_open_error = "cudaStreamCreate failed";
                rc = GC_ECUDA;
                break;
            }
            g->own_stream = true;
        }
        if (cudaMallocHost((void**)&g->h_ctl, sizeof(Ctl)) != cudaSuccess ||
            cudaEventCreate(&g->e0) != cudaSuccess || cudaEventCreate(&g->e1) != cudaSuccess ||
            [&] {
                for (auto& e : g->ev)
                    if (cudaEventCreate(&e) != cudaSuccess) return true;
                return false;
            }()) {
            t_open_error = "host allocation failed";
            rc = GC_ENOMEM;
            break;
        }
        // side streams of the counting pass (they inherit nothing from the
        // caller's stream: every use is fenced by events on it)
        bool aux_ok = cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming) == cudaSuccess;
        for (int i = 0; i < 3 && aux_ok; i++)
            aux_ok = cudaStreamCreateWithFlags(&g->aux[i], cudaStreamNonBlocking) == cudaSuccess &&
                     cudaEventCreateWithFlags(&g->join[i], cudaEventDisableTiming) == cudaSuccess;
        if (!aux_ok) {
            t_open_error = "cudaStreamCreate failed";
            rc = GC_ECUDA;
            break;
        }
        rc = open_device(g, row_ptr, col);
        if (rc) t_open_error = g->err;
    } while (0);
    if (rc) {
        destroy(g);
        return rc;
    }
    *out = g;
    return GC_OK;
}

int gc_count_static(gc_graph* g, uint64_t out[6]) {
    if (!g || !out) return GC_EINVAL;
    if (!on_device(g)) {
        g->err = "cudaSetDevice failed";
        return GC_ECUDA;
    }
    g->err.clear();
    return count_static(g, false, out);
}

int gc_counts3(const gc_graph* g, uint64_t out[2]) {
    if (!g || !out) return GC_EINVAL;
    out[0] = g->F3[0];
    out[1] = g->F3[1];
    return GC_OK;
}

int gc_counts_all(const gc_graph* g, uint64_t out[22]) {
    if (!g || !out) return GC_EINVAL;
    typedef unsigned __int128 u128;
    const u128 n = (u128)(uint64_t)g->n, m = (u128)(uint64_t)g->m;
    const u128 g1 = g->F[0], g2 = g->F[1], g3 = g->F[2], g4 = g->F[3], g5 = g->F[4], g6 = g->F[5];
    const u128 tri = g->F3[1], wedges = (u128)g->F3[0] + 3 * (u128)g->F3[1];
    auto c2 = [](u128 x) -> u128 { return x < 2 ? 0 : x * (x - 1) / 2; };
    auto c4 = [](u128 x) -> u128 { return x < 4 ? 0 : x * (x - 1) / 2 * (x - 2) / 3 * (x - 3) / 4; };
    u128 c[11];
    c[0] = g1; c[1] = g2; c[2] = g3; c[3] = g4; c[4] = g5; c[5] = g6;
    if (g->n < 4) {
        for (int i = 6; i < 11; i++) c[i] = 0;
    } else {
        const u128 t_iso = tri * (n - 3) - g4 - 2 * g5 - 4 * g6;
        const u128 w_iso = wedges * (n - 3) - (2 * g1 + 3 * g2 + 4 * g3 + 5 * g4 + 8 * g5 + 12 * g6 + 3 * t_iso);
        const u128 two = (c2(m) - wedges) - (g1 + 2 * g3 + g4 + 2 * g5 + 3 * g6);
        const u128 one = m * c2(n - 2) -
                         (2 * (w_iso + two) + 3 * (t_iso + g1 + g2) + 4 * (g3 + g4) + 5 * g5 + 6 * g6);
        const u128 empty = c4(n) - (one + w_iso + two + t_iso + g1 + g2 + g3 + g4 + g5 + g6);
        c[6] = t_iso; c[7] = w_iso; c[8] = two; c[9] = one; c[10] = empty;
    }
    for (int i = 0; i < 11; i++) {
        out[2 * i] = (uint64_t)c[i];
        out[2 * i + 1] = (uint64_t)(c[i] >> 64);
    }
    return GC_OK;
}

// Scratch of the heavy 4-cycle pivots of the local counts (none when the
// grouped walk is off); returns false when an allocation failed.
static bool alloc_heavy(gc_graph* g, HeavyC4& h) {
    h.heavy_min = g->loc_heavy_min;
    h.U_wt = g->U_wt;
    h.heavy = nullptr;
    h.hlist = nullptr;
    h.hcount = nullptr;
    h.cnt_g = nullptr;
    if (h.heavy_min <= 0) return true;
    const size_t n = (size_t)std::max(g->n, 1);
    h.heavy = (uint8_t*)dalloc(g, n);
    h.hlist = (int32_t*)dalloc(g, 4 * n);
    h.hcount = (int*)dalloc(g, 16);
    h.cnt_g = (uint32_t*)dalloc(g, 4 * (size_t)C4G * n);
    return h.heavy && h.hlist && h.hcount && h.cnt_g &&
           cudaMemsetAsync(h.cnt_g, 0, 4 * (size_t)C4G * n, g->s) == cudaSuccess;
}

static void free_heavy(gc_graph* g, HeavyC4& h) {
    if (h.heavy) dfree(g, h.heavy);
    if (h.hlist) dfree(g, h.hlist);
    if (h.hcount) dfree(g, h.hcount);
    if (h.cnt_g) dfree(g, h.cnt_g);
}

static int vertex_counts(gc_graph* g, uint64_t* out, int orbits) {
    if (!g || (!out && g->n > 0)) return GC_EINVAL;
    if (!on_device(g)) {
        g->err = "cudaSetDevice failed";
        return GC_ECUDA;
    }
    g->err.clear();
    if (g->n == 0) return GC_OK;
    // the union graph, per-entry t and T2 of the current graph
    int rc = count_static(g, false, nullptr);
    if (rc) return rc;
    cudaStream_t s = g->s;
    const size_t n = (size_t)g->n;
    const long long nU = std::max<long long>(g->h_ctl->nU, 1);
    // one dense counter array per 4-cycle block, at most 2 GB in all
    const int blocks = (int)std::max<long long>(1, std::min<long long>(g->sms, (2LL << 30) / (4LL * (long long)n)));
    uint32_t* tall = (uint32_t*)dalloc(g, 4 * (size_t)nU);
    long long* sdeg = (long long*)dalloc(g, 8 * n);
    const int k = orbits ? 11 : 6;
    long long* NV = (long long*)dalloc(g, 88 * n);
    uint32_t* cnt = (uint32_t*)dalloc(g, 4 * n * (size_t)blocks);
    unsigned long long* dout = (unsigned long long*)dalloc(g, 8 * (size_t)k * n);
    HeavyC4 hv;
    const bool hv_ok = alloc_heavy(g, hv);
    auto cleanup = [&]() {
        dfree(g, tall);
        dfree(g, sdeg);
        dfree(g, NV);
        dfree(g, cnt);
        dfree(g, dout);
        free_heavy(g, hv);
    };
    if (!tall || !sdeg || !NV || !cnt || !dout || !hv_ok) {
        cleanup();
        return nomem(g, "per-vertex counts");
    }
    if (cudaMemsetAsync(NV, 0, 88 * n, s) != cudaSuccess || cudaMemsetAsync(cnt, 0, 4 * n * (size_t)blocks, s) != cudaSuccess) {
        cleanup();
        g->err = "cudaMemsetAsync failed";
        return GC_ECUDA;
    }
    VertexArgs va;
    va.ctl = g->ctl;
    va.wlist = g->wlist;
    va.U_off = g->U_off;
    va.U_col = g->U_col.p;
    va.U_split = g->U_split;
    va.tpack = g->tpack.p;
    va.T2 = g->T2;
    va.tall = tall;
    va.sdeg = sdeg;
    va.NV = NV;
    va.cnt = cnt;
    va.c4_blocks = blocks;
    va.n = (int)n;
    va.iperm = g->iperm;
    va.out = dout;
    va.orbits = orbits;
    va.sms = g->sms;
    va.hv = hv;
    cudaError_t ce = cudaEventRecord(g->e0, s);
    g->launches = enqueue_vertex_counts(va, s);
    if (g->launches < 0 && ce == cudaSuccess) ce = cudaErrorUnknown;
    if (ce == cudaSuccess) ce = cudaEventRecord(g->e1, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(out, dout, 8 * (size_t)k * n, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce == cudaSuccess) ce = cudaGetLastError();
    float ms = 0.f;
    if (ce == cudaSuccess && cudaEventElapsedTime(&ms, g->e0, g->e1) == cudaSuccess) g->st.ms_device = ms;
    cleanup();
    if (ce != cudaSuccess) {
        g->err = std::string("per-vertex counts: ") + cudaGetErrorString(ce);
        return GC_ECUDA;
    }
    g->st.launches = g->launches;
    return GC_OK;
}

int gc_vertex_counts(gc_graph* g, uint64_t* out) { return vertex_counts(g, out, 0); }

int gc_vertex_orbits(gc_graph* g, uint64_t* out) { return vertex_counts(g, out, 1); }

static int edge_counts(gc_graph* g, int32_t* edges, uint64_t* out, int orbits) {
    if (!g || (g->m > 0 && !out)) return GC_EINVAL;
    if (!on_device(g)) {
        g->err = "cudaSetDevice failed";
        return GC_ECUDA;
    }
    g->err.clear();
    if (g->m == 0) return GC_OK;
    // the union graph, per-entry t and T2 of the current graph
    int rc = count_static(g, false, nullptr);
    if (rc) return rc;
    cudaStream_t s = g->s;
    const size_t n = (size_t)g->n;
    const long long nU = g->h_ctl->nU, m = nU / 2;
    if (nU != 2 * g->m) {
        g->err = "per-edge counts: the union graph does not hold every edge twice";
        return GC_ECUDA;
    }
    const int blocks = (int)std::max<long long>(1, std::min<long long>(g->sms, (2LL << 30) / (4LL * (long long)n)));
    const int sg = radix_grid(nU, g->sms);
    const int k = orbits ? 10 : 6;
    uint32_t* tall = (uint32_t*)dalloc(g, 4 * (size_t)nU);
    long long* sdeg = (long long*)dalloc(g, 8 * n);
    long long* NE = (long long*)dalloc(g, 32 * (size_t)nU);
    unsigned long long* keys = (unsigned long long*)dalloc(g, 8 * (size_t)nU);
    unsigned long long* ktmp = (unsigned long long*)dalloc(g, 8 * (size_t)nU);
    uint32_t* hist = (uint32_t*)dalloc(g, 4 * 256 * (size_t)sg);
    uint32_t* cnt = (uint32_t*)dalloc(g, 4 * n * (size_t)blocks);
    unsigned long long* dout = (unsigned long long*)dalloc(g, 8 * (size_t)k * (size_t)m);
    int32_t* dedges = edges ? (int32_t*)dalloc(g, 8 * (size_t)m) : nullptr;
    HeavyC4 hv;
    const bool hv_ok = alloc_heavy(g, hv);
    auto cleanup = [&]() {
        free_heavy(g, hv);
        dfree(g, tall);
        dfree(g, sdeg);
        dfree(g, NE);
        dfree(g, keys);
        dfree(g, ktmp);
        dfree(g, hist);
        dfree(g, cnt);
        dfree(g, dout);
        if (dedges) dfree(g, dedges);
    };
    if (!tall || !sdeg || !NE || !keys || !ktmp || !hist || !cnt || !dout || (edges && !dedges) || !hv_ok) {
        cleanup();
        return nomem(g, "per-edge counts");
    }
    if (cudaMemsetAsync(NE, 0, 32 * (size_t)nU, s) != cudaSuccess ||
        cudaMemsetAsync(cnt, 0, 4 * n * (size_t)blocks, s) != cudaSuccess) {
        cleanup();
        g->err = "cudaMemsetAsync failed";
        return GC_ECUDA;
    }
    EdgeArgs ea;
    ea.ctl = g->ctl;
    ea.wlist = g->wlist;
    ea.U_off = g->U_off;
    ea.U_col = g->U_col.p;
    ea.U_split = g->U_split;
    ea.tpack = g->tpack.p;
    ea.T2 = g->T2;
    ea.tall = tall;
    ea.sdeg = sdeg;
    ea.NE = NE;
    ea.keys = keys;
    ea.keys_tmp = ktmp;
    ea.hist = hist;
    ea.sort_grid = sg;
    ea.d_count = &g->ctl->nU;
    ea.nU = nU;
    ea.m = m;
    ea.nb = g->S;
    ea.cnt = cnt;
    ea.c4_blocks = blocks;
    ea.n = (int)n;
    ea.iperm = g->iperm;
    ea.out = dout;
    ea.edges = dedges;
    ea.orbits = orbits;
    ea.sms = g->sms;
    ea.hv = hv;
    cudaError_t ce = cudaEventRecord(g->e0, s);
    g->launches = enqueue_edge_counts(ea, s);
    if (g->launches < 0 && ce == cudaSuccess) ce = cudaErrorUnknown;
    if (ce == cudaSuccess) ce = cudaEventRecord(g->e1, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(out, dout, 8 * (size_t)k * (size_t)m, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess && edges) ce = cudaMemcpyAsync(edges, dedges, 8 * (size_t)m, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce == cudaSuccess) ce = cudaGetLastError();
    float ms = 0.f;
    if (ce == cudaSuccess && cudaEventElapsedTime(&ms, g->e0, g->e1) == cudaSuccess) g->st.ms_device = ms;
    cleanup();
    if (ce != cudaSuccess) {
        g->err = std::string("per-edge counts: ") + cudaGetErrorString(ce);
        return GC_ECUDA;
    }
    g->st.launches = g->launches;
    return GC_OK;
}

int gc_edge_counts(gc_graph* g, int32_t* edges, uint64_t* out) { return edge_counts(g, edges, out, 0); }

int gc_edge_orbits(gc_graph* g, int32_t* edges, uint64_t* out) { return edge_counts(g, edges, out, 1); }

int gc_counts(const gc_graph* g, uint64_t out[6]) {
    if (!g || !out) return GC_EINVAL;
    for (int i = 0; i < 6; i++) out[i] = g->F[i];
    return GC_OK;
}

static int batch_host(gc_graph* g, const int32_t* ins, int64_t n_ins, const int32_t* del, int64_t n_del, int commit,
                      uint64_t out[6]) {
    if (!g) return GC_EINVAL;
    if (!on_device(g)) {
        g->err = "cudaSetDevice failed";
        return GC_ECUDA;
    }
    auto t0 = std::chrono::steady_clock::now();
    g->err.clear();
    if (n_ins < 0 || n_del < 0 || (n_ins > 0 && !ins) || (n_del > 0 && !del)) {
        g->err = "batch arrays: negative size or NULL pointer";
        return GC_EINVAL;
    }
    if (n_ins + n_del > (1LL << 29)) {
        g->err = "batch too large";
        return GC_EINVAL;
    }
    int rc = check_pairs(g, ins, n_ins, "insertion");
    if (rc) return rc;
    rc = check_pairs(g, del, n_del, "deletion");
    if (rc) return rc;
    size_t np = (size_t)(n_ins + n_del);
    if (!ensure(g, g->pairs, 2 * std::max<size_t>(np, 1))) return nomem(g, "batch staging");
    if (n_ins) CK(cudaMemcpyAsync(g->pairs.p, ins, 8 * (size_t)n_ins, cudaMemcpyHostToDevice, g->s));
    if (n_del) CK(cudaMemcpyAsync(g->pairs.p + 2 * n_ins, del, 8 * (size_t)n_del, cudaMemcpyHostToDevice, g->s));
    rc = apply_device(g, g->pairs.p, n_ins, g->pairs.p + 2 * n_ins, n_del, commit, out);
    g->st.ms_wall = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return rc;
}

int gc_apply_batch(gc_graph* g, const int32_t* ins, int64_t n_ins, const int32_t* del, int64_t n_del,
                   uint64_t out[6]) {
    return batch_host(g, ins, n_ins, del, n_del, 1, out);
}

int gc_count_batch(gc_graph* g, const int32_t* ins, int64_t n_ins, const int32_t* del, int64_t n_del,
                   uint64_t out[6]) {
    return batch_host(g, ins, n_ins, del, n_del, 0, out);
}

static int batch_device(gc_graph* g, const int32_t* d_ins, int64_t n_ins, const int32_t* d_del, int64_t n_del,
                        int commit, uint64_t out[6]) {
    if (!g) return GC_EINVAL;
    if (!on_device(g)) {
        g->err = "cudaSetDevice failed";
        return GC_ECUDA;
    }
    g->err.clear();
    if (n_ins < 0 || n_del < 0 || (n_ins > 0 && !d_ins) || (n_del > 0 && !d_del) || n_ins + n_del > (1LL << 29)) {
        g->err = "batch arrays: bad size or NULL pointer";
        return GC_EINVAL;
    }
    return apply_device(g, d_ins, n_ins, d_del, n_del, commit, out);
}

int gc_apply_batch_device(gc_graph* g, const int32_t* d_ins, int64_t n_ins, const int32_t* d_del, int64_t n_del,
                          uint64_t out[6]) {
    return batch_device(g, d_ins, n_ins, d_del, n_del, 1, out);
}

int gc_count_batch_device(gc_graph* g, const int32_t* d_ins, int64_t n_ins, const int32_t* d_del, int64_t n_del,
                          uint64_t out[6]) {
    return batch_device(g, d_ins, n_ins, d_del, n_del, 0, out);
}

// Append k isolated vertices: the per-vertex state is copied into arrays of
// the new size (scratch is re-made), the id width of the batch keys follows
// n, and every captured batch graph is dropped.
static int grow_vertices(gc_graph* g, long long k) {
    cudaStream_t s = g->s;
    const int n0 = g->n, n1 = (int)(n0 + k);
    const size_t nn = (size_t)std::max(n1, 1), old_nn = (size_t)std::max(n0, 1);
    auto grow = [&](void** p, size_t elem, size_t count_new, size_t count_old, bool keep) -> bool {
        void* q = dalloc(g, elem * count_new);
        if (!q) return false;
        if (keep && n0 > 0) {
            if (cudaMemcpyAsync(q, *p, elem * count_old, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return false;
        }
        dfree(g, *p);
        *p = q;
        return true;
    };
    bool ok = grow((void**)&g->perm, 4, nn, old_nn, true) && grow((void**)&g->iperm, 4, nn, old_nn, true) &&
              grow((void**)&g->deg, 4, nn, old_nn, true) && grow((void**)&g->cap, 4, nn, old_nn, true) &&
              grow((void**)&g->row_start, 8, nn + 1, old_nn, true) && grow((void**)&g->wlist, 4, nn, 0, false) &&
              grow((void**)&g->U_deg, 4, nn, 0, false) && grow((void**)&g->U_split, 4, nn, 0, false) &&
              grow((void**)&g->da, 4, nn, 0, false) && grow((void**)&g->db, 4, nn, 0, false) &&
              grow((void**)&g->U_off, 8, nn + 1, 0, false) && grow((void**)&g->U_wt, 8, nn, 0, false) &&
              grow((void**)&g->segA, sizeof(int2), nn, 0, false) && grow((void**)&g->segD, sizeof(int2), nn, 0,
                   false) &&
              grow((void**)&g->visited, 4, (nn + 31) / 32 + 1, 0, false) &&
              grow((void**)&g->visited2, 4, (nn + 31) / 32 + 1, 0, false) &&
              grow((void**)&g->T2, 8, nn, old_nn, true) && grow((void**)&g->dtri2, 8, nn, 0, false) &&
              grow((void**)&g->bins, 4, (size_t)NBINS * nn, 0, false);
    if (!ok) return nomem(g, "vertex arrays");
    CK(cudaMemsetAsync(g->segA, 0, sizeof(int2) * nn, s));
    CK(cudaMemsetAsync(g->segD, 0, sizeof(int2) * nn, s));
    // new vertices are isolated: no triangles
    CK(cudaMemsetAsync(g->dtri2, 0, 8 * nn, s));
    {
        const size_t kept = n0 > 0 ? (size_t)n0 : 0;
        CK(cudaMemsetAsync(g->T2 + kept, 0, 8 * (nn - kept), s));
    }
    pdl_launch(k_init_new_vertices, dim3(grid_elems(g, k)), dim3(TPB), 0, s, g->perm, g->iperm, g->deg, g->cap,
               g->row_start, n0, n1);
    CKL();
    release(g, g->dense);
    if (!ensure(g, g->dense, (size_t)g->dense_clusters * (size_t)dense_stride((long long)nn)))
        return nomem(g, "4-cycle counter arrays");
    CK(cudaMemsetAsync(g->dense.p, 0, 8 * g->dense.cap, s));
    g->n = n1;
    g->S = std::max(1, bitlen(n1 > 0 ? n1 - 1 : 0));
    if (g->chunk_table.p) {
        release(g, g->chunk_table);
        if (!ensure_chunk_table(g)) return nomem(g, "4-cycle chunk table");
    }
    for (int i = 0; i < 3; i++)
        if (g->qexec[i]) {
            cudaGraphExecDestroy(g->qexec[i]);
            g->qexec[i] = nullptr;
        }
    if (g->gexec) {
        cudaGraphExecDestroy(g->gexec);
        g->gexec = nullptr;
    }
    if (g->pexec) {
        cudaGraphExecDestroy(g->pexec);
        g->pexec = nullptr;
    }
    if (g->lexec) {
        cudaGraphExecDestroy(g->lexec);
        g->lexec = nullptr;
    }
    g->buf_gen++;
    CK(cudaStreamSynchronize(s));
    return GC_OK;
}

int gc_add_vertices(gc_graph* g, int64_t k, int32_t* first_id) {
    if (!g) return GC_EINVAL;
    if (!on_device(g)) {
        g->err = "cudaSetDevice failed";
        return GC_ECUDA;
    }
    g->err.clear();
    if (k < 0 || (long long)g->n + k >= (1ll << 30)) {
        g->err = "vertex count: negative, or n would reach 2^30";
        return GC_EINVAL;
    }
    if (first_id) *first_id = g->n;
    if (k == 0) return GC_OK;
    return grow_vertices(g, k);
}

int32_t gc_num_vertices(const gc_graph* g) { return g ? g->n : -1; }

int gc_delete_vertices(gc_graph* g, const int32_t* ids, int64_t k, uint64_t out[6]) {
    if (!g) return GC_EINVAL;
    if (!on_device(g)) {
        g->err = "cudaSetDevice failed";
        return GC_ECUDA;
    }
    g->err.clear();
    if (k < 0 || (k > 0 && !ids)) {
        g->err = "vertex list: negative size or NULL pointer";
        return GC_EINVAL;
    }
    for (int64_t i = 0; i < k; i++)
        if (ids[i] < 0 || ids[i] >= g->n) {
            g->err = "vertex id outside [0, n)";
            return GC_EINVAL;
        }
    cudaStream_t s = g->s;
    const size_t kk = (size_t)std::max<int64_t>(k, 1);
    if (!ensure(g, g->vids, kk) || !ensure(g, g->vdeg, kk) || !ensure(g, g->voff, kk + 1))
        return nomem(g, "vertex list");
    long long total = 0;
    if (k > 0) {
        CK(cudaMemcpyAsync(g->vids.p, ids, 4 * (size_t)k, cudaMemcpyHostToDevice, s));
        pdl_launch(k_vertex_degrees, dim3(grid_elems(g, k)), dim3(TPB), 0, s, g->vids.p, k, g->perm, g->deg, g->vdeg.p);
        CKL();
        scan_i32_to_i64(g->vdeg.p, g->voff.p, nullptr, k, g->bsum.p, scan_grid(k, g->sms), nullptr, s);
        CK(cudaMemcpyAsync(&total, g->voff.p + k, sizeof(long long), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    if (!ensure(g, g->pairs, 2 * (size_t)std::max<long long>(total, 1))) return nomem(g, "vertex edges");
    if (total > 0) {
        pdl_launch(k_vertex_pairs, dim3(grid_warps(g)), dim3(TPB), 0, s, g->vids.p, k, g->perm, g->iperm, g->row_start,
                   g->deg, g->col,
                                                     g->voff.p, g->pairs.p);
        CKL();
    }
    // an edge between two listed vertices appears twice; normalisation collapses it
    return apply_device(g, g->pairs.p, 0, g->pairs.p, total, 1, out);
}

// A run of batches: those of at most local_max_pairs pairs take the
// edge-local delta one at a time (in order, when the run commits), the
// others run as captured region runs.
static int apply_batches_device(gc_graph* g, const int32_t* d_ins, const int32_t* d_del, const long long* h_batches,
                                int k, int independent, uint64_t* out) {
    const long long L = g->opt.local_max_pairs;
    int nloc = 0;
    for (int i = 0; i < k; i++) nloc += (L > 0 && h_batches[4 * i + 1] + h_batches[4 * i + 3] <= L) ? 1 : 0;
    if (nloc == 0) return apply_batches_region(g, d_ins, d_del, h_batches, k, independent, out);
    auto t0 = std::chrono::steady_clock::now();
    const int commit = independent ? 0 : 1;
    float ms = 0.f;
    int launches = 0, relayouts = 0;
    std::vector<long long> sub;
    std::vector<int> idx;
    std::vector<uint64_t> tmp;
    auto run_region = [&]() -> int {
        if (idx.empty()) return GC_OK;
        tmp.assign(6 * idx.size(), 0);
        int rc = apply_batches_region(g, d_ins, d_del, sub.data(), (int)idx.size(), independent, tmp.data());
        if (rc) return rc;
        if (out)
            for (size_t j = 0; j < idx.size(); j++)
                for (int q = 0; q < 6; q++) out[6 * (size_t)idx[j] + q] = tmp[6 * j + q];
        ms += g->st.ms_device;
        launches += g->st.launches;
        relayouts += g->st.relayouts;
        sub.clear();
        idx.clear();
        return GC_OK;
    };
    for (int i = 0; i < k; i++) {
        const long long* b = h_batches + 4 * (size_t)i;
        if (!(L > 0 && b[1] + b[3] <= L)) {
            sub.insert(sub.end(), b, b + 4);
            idx.push_back(i);
            continue;
        }
        if (commit) {
            int rc = run_region();  // batches before this one first
            if (rc) return rc;
        }
        uint64_t o[6];
        int rc = apply_device(g, d_ins + 2 * b[0], b[1], d_del + 2 * b[2], b[3], commit, o);
        if (rc) return rc;
        if (out)
            for (int q = 0; q < 6; q++) out[6 * (size_t)i + q] = o[q];
        ms += g->st.ms_device;
        launches += g->st.launches;
        relayouts += g->st.relayouts;
    }
    int rc = run_region();
    if (rc) return rc;
    g->st.ms_device = ms;
    g->st.launches = launches;
    g->st.relayouts = relayouts;
    g->st.ms_wall = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return GC_OK;
}

int gc_apply_batches(gc_graph* g, const int32_t* const* ins, const int64_t* n_ins, const int32_t* const* del,
                     const int64_t* n_del, int32_t k, int32_t independent, uint64_t* out) {
    if (!g || k < 0 || (k > 0 && (!n_ins || !n_del || !ins || !del))) return GC_EINVAL;
    if (!on_device(g)) {
        g->err = "cudaSetDevice failed";
        return GC_ECUDA;
    }
    g->err.clear();
    if (k == 0) return GC_OK;
    long long tot = 0;
    for (int32_t i = 0; i < k; i++) {
        if (n_ins[i] < 0 || n_del[i] < 0 || (n_ins[i] > 0 && !ins[i]) || (n_del[i] > 0 && !del[i])) {
            g->err = "batch arrays: negative size or NULL pointer";
            return GC_EINVAL;
        }
        if (n_ins[i] + n_del[i] > (1LL << 29)) {
            g->err = "batch too large";
            return GC_EINVAL;
        }
        int rc = check_pairs(g, ins[i], n_ins[i], "insertion");
        if (rc) return rc;
        rc = check_pairs(g, del[i], n_del[i], "deletion");
        if (rc) return rc;
        tot += n_ins[i] + n_del[i];
    }
    // all batches in one upload: insertions then deletions of each batch
    if (!ensure(g, g->pairs, 2 * (size_t)std::max<long long>(tot, 1))) return nomem(g, "batch staging");
    std::vector<long long> d((size_t)4 * k);
    long long off = 0;
    for (int32_t i = 0; i < k; i++) {
        if (n_ins[i]) CK(cudaMemcpyAsync(g->pairs.p + 2 * off, ins[i], 8 * (size_t)n_ins[i], cudaMemcpyHostToDevice, g->s));
        d[4 * i] = off;
        d[4 * i + 1] = n_ins[i];
        off += n_ins[i];
        if (n_del[i]) CK(cudaMemcpyAsync(g->pairs.p + 2 * off, del[i], 8 * (size_t)n_del[i], cudaMemcpyHostToDevice, g->s));
        d[4 * i + 2] = off;
        d[4 * i + 3] = n_del[i];
        off += n_del[i];
    }
    return apply_batches_device(g, g->pairs.p, g->pairs.p, d.data(), k, independent, out);
}

int gc_apply_batches_device(gc_graph* g, const int32_t* d_pairs, const int64_t* batches, int32_t k,
                            int32_t independent, uint64_t* out) {
    if (!g || k < 0 || (k > 0 && (!d_pairs || !batches))) return GC_EINVAL;
    if (!on_device(g)) {
        g->err = "cudaSetDevice failed";
        return GC_ECUDA;
    }
    g->err.clear();
    if (k == 0) return GC_OK;
    for (int32_t i = 0; i < k; i++) {
        const int64_t* b = batches + 4 * (size_t)i;
        if (b[0] < 0 || b[1] < 0 || b[2] < 0 || b[3] < 0 || b[1] + b[3] > (1LL << 29)) {
            g->err = "batch descriptor: negative offset or size, or batch too large";
            return GC_EINVAL;
        }
    }
    return apply_batches_device(g, d_pairs, d_pairs, (const long long*)batches, k, independent, out);
}

int gc_batch_stats(const gc_graph* g, gc_stats* s) {
    if (!g || !s) return GC_EINVAL;
    *s = g->st;
    return GC_OK;
}

int64_t gc_num_edges(const gc_graph* g) { return g ? g->m : -1; }

int gc_export_csr(gc_graph* g, int32_t* row_ptr, int32_t* col) {
    if (!g || !row_ptr || (g->m > 0 && !col)) return GC_EINVAL;
    if (!on_device(g)) {
        g->err = "cudaSetDevice failed";
        return GC_ECUDA;
    }
    int n = g->n;
    std::vector<int32_t> deg(n), iperm(n);
    std::vector<long long> rs(n);
    std::vector<int32_t> hc((size_t)g->col_capacity);
    CK(cudaStreamSynchronize(g->s));
    if (n > 0) {
        CK(cudaMemcpy(deg.data(), g->deg, 4 * (size_t)n, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(iperm.data(), g->iperm, 4 * (size_t)n, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(rs.data(), g->row_start, 8 * (size_t)n, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(hc.data(), g->col, 4 * (size_t)g->col_capacity, cudaMemcpyDeviceToHost));
    }
    std::vector<int32_t> ext_deg(n);
    for (int i = 0; i < n; i++) ext_deg[iperm[i]] = deg[i];
    row_ptr[0] = 0;
    for (int x = 0; x < n; x++) row_ptr[x + 1] = row_ptr[x] + ext_deg[x];
    for (int i = 0; i < n; i++) {
        int32_t x = iperm[i];
        int32_t* o = col + row_ptr[x];
        for (int j = 0; j < deg[i]; j++) o[j] = iperm[hc[(size_t)rs[i] + j]];
        std::sort(o, o + deg[i]);
    }
    return GC_OK;
}

static void tuning_to_abi(const Tuning& t, long long local_max_pairs, long long heavy_min, gc_tuning* o) {
    std::memset(o, 0, sizeof(*o));
    o->tri_warp_max = t.tri_warp_max;
    o->tri_small_max = t.tri_small_max;
    o->tri_block_max = t.tri_block_max;
    o->c4_reg_max = t.c4_reg_max;
    o->c4_warp_max = t.c4_warp_max;
    o->c4_block_max = t.c4_block_max;
    o->c4_cta_max = t.c4_cta_max;
    o->c4_chunk_min = t.c4_chunk_min >= NEVER ? 0 : t.c4_chunk_min;
    o->c4_chunk_max = t.c4_chunk_max >= NEVER ? 0 : t.c4_chunk_max;
    o->local_max_pairs = local_max_pairs;
    o->local_c4_heavy_min = heavy_min;
}

int gc_get_tuning(const gc_graph* g, gc_tuning* t) {
    if (!g || !t) return GC_EINVAL;
    tuning_to_abi(g->tune, g->opt.local_max_pairs, g->loc_heavy_min, t);
    t->pair_min_share = g->pair_min_share;
    return GC_OK;
}

int gc_set_tuning(gc_graph* g, const gc_tuning* t) {
    if (!g || !t) return GC_EINVAL;
    if (t->tri_warp_max < 1 || t->tri_small_max < 1 || t->tri_block_max < 1 || t->c4_reg_max < 1 || t->c4_warp_max < 1 ||
        t->c4_block_max < 1 || t->c4_cta_max < 1 || t->c4_chunk_min < 0 || t->c4_chunk_max < 0 ||
        t->local_max_pairs < 0 || t->local_c4_heavy_min < 0 || t->pair_min_share < 0) {
        g->err = "tuning: every bound must be positive (c4_chunk_min, local_max_pairs, local_c4_heavy_min and "
                 "pair_min_share may be 0)";
        return GC_EINVAL;
    }
    Tuning n;
    n.tri_warp_max = t->tri_warp_max;
    n.tri_small_max = t->tri_small_max;
    n.tri_block_max = t->tri_block_max;
    n.c4_reg_max = t->c4_reg_max;
    n.c4_warp_max = t->c4_warp_max;
    n.c4_block_max = t->c4_block_max;
    n.c4_cta_max = t->c4_cta_max;
    n.c4_chunk_min = t->c4_chunk_min == 0 ? NEVER : t->c4_chunk_min;
    n.c4_chunk_max = t->c4_chunk_max == 0 ? NEVER : t->c4_chunk_max;
    if (n.c4_chunk_min < NEVER && !ensure_chunk_table(g)) return nomem(g, "4-cycle chunk table");
    g->tune = n;
    g->opt.local_max_pairs = (int32_t)std::min<int64_t>(t->local_max_pairs, INT32_MAX);
    g->loc_heavy_min = t->local_c4_heavy_min;
    g->pair_min_share = t->pair_min_share;
    g->pair_hint = 0;
    return GC_OK;
}

// Best of `reps` static counts under the current tuning.
static int time_static(gc_graph* g, int reps, float* ms, uint64_t out[6]) {
    float best = 1e30f;
    for (int r = 0; r < reps; r++) {
        int rc = count_static(g, false, out);
        if (rc) return rc;
        best = std::min(best, g->st.ms_device);
    }
    *ms = best;
    return GC_OK;
}

// splitmix64 of a draw index (Steele, Lea and Flood, OOPSLA 2014)
__device__ __forceinline__ unsigned long long mix64(unsigned long long seed, unsigned long long i) {
    unsigned long long z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// the vertex owning directed entry r of the degree prefix sums cum
__device__ __forceinline__ long long entry_owner(const long long* __restrict__ cum, int n, long long r) {
    long long lo = 0, hi = n;  // last u with cum[u] <= r
    while (hi - lo > 1) {
        const long long mid = (lo + hi) >> 1;
        if (cum[mid] <= r) lo = mid;
        else hi = mid;
    }
    return lo;
}

// A calibration batch as external-id pairs: k deletions of edges drawn
// uniformly (with repetition) from the current graph (draw i picks directed
// entry h(seed, i) mod 2m), then k insertions between two vertices drawn
// in proportion to degree (mostly non-edges, as the batch recipe's
// insertions; a present edge is a no-op).
__global__ void k_sample_edges(const long long* __restrict__ cum, int n, const long long* __restrict__ row_start,
                               const int32_t* __restrict__ col, const int32_t* __restrict__ iperm,
                               unsigned long long seed, int k, int32_t* __restrict__ pairs) {
    pdl_enter();
    const unsigned long long m2 = (unsigned long long)cum[n];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * k; i += gridDim.x * blockDim.x) {
        const long long r = (long long)(mix64(seed, (unsigned long long)i) % m2);
        const int32_t u = (int32_t)entry_owner(cum, n, r);
        int32_t v;
        if (i < k) {
            v = col[row_start[u] + (r - cum[u])];
        } else {
            const unsigned long long r2 = mix64(seed ^ 0x5851F42D4C957F2Dull, (unsigned long long)i) % m2;
            v = (int32_t)entry_owner(cum, n, (long long)r2);
            if (v == u) v = (u + 1) % n;
        }
        pairs[2 * i] = iperm[u];
        pairs[2 * i + 1] = iperm[v];
    }
}

// The edge-local threshold by measurement (see gc_autotune).
static int calibrate_local(gc_graph* g, int reps) {
    const int32_t saved = g->opt.local_max_pairs;
    if (g->m < 64 || g->n < 2) {
        g->opt.local_max_pairs = 0;
        return GC_OK;
    }
    cudaStream_t s = g->s;
    const long long kmax = std::min<long long>(g->m / 4, 1LL << 17);
    if (!ensure(g, g->pairs, 2 * (size_t)std::max<long long>(kmax, 8))) return nomem(g, "calibration pairs");
    // each calibration batch: k / 2 deletions, then k / 2 insertions
    // degree prefix sums (the union-graph offsets are free between batches)
    g->launches += scan_i32_to_i64(g->deg, g->U_off, nullptr, g->n, g->bsum.p, scan_grid(g->n, g->sms), nullptr, s);
    long long thr = 0;
    for (long long k = 8; k <= kmax; k *= 2) {
        const long long half = k / 2;
        k_sample_edges<<<grid_elems(g, k), TPB, 0, s>>>(g->U_off, g->n, g->row_start, g->col, g->iperm,
                                                        0x5DEECE66Dull + (unsigned long long)k, (int)half, g->pairs.p);
        CKL();
        float best[2] = {1e30f, 1e30f};
        uint64_t res[2][6];
        for (int form = 0; form < 2; form++) {
            g->opt.local_max_pairs = form == 0 ? (int32_t)k : 0;
            for (int r = 0; r < std::max(reps, 1) + 1; r++) {  // the first run captures
                // half deletions, half insertions (the second half of the pairs)
                int rc = apply_device(g, g->pairs.p + 2 * half, half, g->pairs.p, half, 0, res[form]);
                if (rc) {
                    g->opt.local_max_pairs = saved;
                    return rc;
                }
                if (r > 0) best[form] = std::min(best[form], g->st.ms_device);
            }
        }
        if (std::memcmp(res[0], res[1], sizeof(res[0])) != 0) {
            g->opt.local_max_pairs = saved;
            g->err = "autotune: the edge-local and region results differ";
            return GC_ECUDA;
        }
        if (best[0] < best[1]) thr = k;
        else break;
    }
    g->opt.local_max_pairs = (int32_t)thr;
    return GC_OK;
}

int gc_autotune(gc_graph* g, int32_t reps, gc_tuning* best, float* best_ms) {
    if (!g) return GC_EINVAL;
    if (!on_device(g)) {
        g->err = "cudaSetDevice failed";
        return GC_ECUDA;
    }
    g->err.clear();
    if (reps <= 0) reps = 2;
    Tuning cur = g->tune;
    uint64_t ref[6], got[6];
    float cur_ms = 0.f;
    int rc = time_static(g, reps, &cur_ms, ref);
    if (rc) return rc;
    // candidate values per boundary; coordinate descent, at most three sweeps
    // (a bound below the tier beneath it empties the tier; the chunked
    // kernel only takes pivots above c4_cta_max, so lowering that one after
    // c4_chunk_min opens the chunked tier to medium pivots)
    const long long cand[9][6] = {
        {16, 32, -1, -1, -1, -1},                          // tri_warp_max
        {64, 128, -1, -1, -1, -1},                         // tri_small_max
        {256, 512, -1, -1, -1, -1},                        // tri_block_max
        {16, 32, -1, -1, -1, -1},                          // c4_reg_max
        {128, 512, -1, -1, -1, -1},                        // c4_warp_max
        {512, 2048, 8192, -1, -1, -1},                     // c4_block_max
        {2048, 8192, 16384, 32768, -1, -1},                // c4_cta_max
        {NEVER, 2048, 8192, 32768, 262144, 1048576},       // c4_chunk_min
        {NEVER, 131072, 524288, 2097152, -1, -1}            // c4_chunk_max
    };
    auto field = [](Tuning& t, int i) -> long long {
        switch (i) {
            case 0: return t.tri_warp_max;
            case 1: return t.tri_small_max;
            case 2: return t.tri_block_max;
            case 3: return t.c4_reg_max;
            case 4: return t.c4_warp_max;
            case 5: return t.c4_block_max;
            case 6: return t.c4_cta_max;
            case 7: return t.c4_chunk_min;
            default: return t.c4_chunk_max;
        }
    };
    auto set = [](Tuning& t, int i, long long v) {
        switch (i) {
            case 0: t.tri_warp_max = (int)v; break;
            case 1: t.tri_small_max = (int)v; break;
            case 2: t.tri_block_max = (int)v; break;
            case 3: t.c4_reg_max = (int)v; break;
            case 4: t.c4_warp_max = (int)v; break;
            case 5: t.c4_block_max = (int)v; break;
            case 6: t.c4_cta_max = v; break;
            case 7: t.c4_chunk_min = v; break;
            default: t.c4_chunk_max = v; break;
        }
    };
    const bool chunk_ok = ensure_chunk_table(g);
    for (int sweep = 0; sweep < 3; sweep++) {
        bool moved = false;
        for (int i = 8; i >= 0; i--) {
            if (i >= 7 && !chunk_ok) continue;
            for (int k = 0; k < 6; k++) {
                const long long v = cand[i][k];
                if (v < 0 || v == field(cur, i)) continue;
                Tuning t = cur;
                set(t, i, v);
                g->tune = t;
                float ms = 0.f;
                rc = time_static(g, reps, &ms, got);
                if (rc) {
                    g->tune = cur;
                    return rc;
                }
                if (std::memcmp(got, ref, sizeof(ref)) != 0) {
                    g->tune = cur;
                    g->err = "autotune: counts differ between bin boundaries";
                    return GC_ECUDA;
                }
                if (ms < 0.97f * cur_ms) {
                    cur = t;
                    cur_ms = ms;
                    moved = true;
                }
            }
        }
        if (!moved) break;
    }
    g->tune = cur;
    rc = calibrate_local(g, reps);
    if (rc) return rc;
    if (best) {
        tuning_to_abi(cur, g->opt.local_max_pairs, g->loc_heavy_min, best);
        best->pair_min_share = g->pair_min_share;
    }
    if (best_ms) *best_ms = cur_ms;
    return GC_OK;
}

int64_t gc_device_bytes(const gc_graph* g) { return g ? g->bytes_held : -1; }

int64_t gc_batch_bytes(const gc_graph* g, int64_t n_ins, int64_t n_del) {
    if (!g || n_ins < 0 || n_del < 0) return -1;
    return predict_batch_bytes(g, n_ins, n_del);
}

int gc_trim(gc_graph* g) {
    if (!g) return GC_EINVAL;
    if (!on_device(g)) {
        g->err = "cudaSetDevice failed";
        return GC_ECUDA;
    }
    trim_scratch(g);
    return GC_OK;
}

const char* gc_last_error(const gc_graph* g) { return g ? g->err.c_str() : t_open_error.c_str(); }

void gc_close(gc_graph* g) {
    if (g) on_device(g);
    destroy(g);
}

}  // extern "C"
