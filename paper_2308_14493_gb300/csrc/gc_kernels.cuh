// gc_kernels.cuh -- declarations of the kernels, for the launchers in gc_api.cu.
#pragma once

#include "gc_internal.cuh"

namespace gcx {

// gc_batch.cu
__global__ void k_batch_keys(Ctl* c, const int32_t* perm, int n, int S, uint64_t* keys);
__global__ void k_batch_decide(const uint64_t* keys, Ctl* c, int S, const long long* row_start, const int32_t* deg,
                               const int32_t* col, int32_t* keepA, int32_t* keepD);
__global__ void k_batch_compact(const uint64_t* keys, const Ctl* c, int S, const int32_t* keepA,
                                const int32_t* keepD, const long long* posA, const long long* posD, int32_t* srcA,
                                int32_t* dstA, int32_t* srcD, int32_t* dstD);
__global__ void k_batch_segments(const int32_t* src, const long long* d_len, int2* seg);
__global__ void k_batch_clear_segments(const int32_t* src, const long long* d_len, int2* seg);
__global__ void k_commit_plan(Ctl* c, const int32_t* wlist, const int2* segA, const int2* segD, const int32_t* deg,
                              const int32_t* cap, const long long* row_start, long long col_capacity, float slack,
                              long long* plan_dst, int32_t* plan_cap, int32_t* plan_deg, long long* plan_scr);
__global__ void k_commit_merge(const Ctl* c, const int32_t* wlist, const int2* segA, const int2* segD,
                               const int32_t* dstA, const int32_t* dstD, const int32_t* deg,
                               const long long* row_start, const int32_t* col, const long long* plan_scr,
                               uint32_t* scratch);
__global__ void k_commit_write(const Ctl* c, const int32_t* wlist, const long long* plan_dst,
                               const int32_t* plan_cap, const int32_t* plan_deg, const long long* plan_scr,
                               const uint32_t* scratch, int32_t* deg, int32_t* cap, long long* row_start,
                               int32_t* col);
__global__ void k_slack_caps(const int32_t* deg, int n, float slack, int32_t* cap);
__global__ void k_copy_rows(const int32_t* deg, int n, const long long* old_start, const int32_t* old_col,
                            const long long* new_start, int32_t* new_col);
__global__ void k_degree_keys(const int32_t* rp, int n, int32_t* deg0, uint64_t* keys);
__global__ void k_perm_from_keys(const uint64_t* keys, int n, int32_t* perm, int32_t* iperm, const int32_t* deg0,
                                 int32_t* deg);
__global__ void k_edge_keys(const int32_t* rp, const int32_t* col, int n, const int32_t* perm, int S,
                            uint64_t* keys, int* bad);
__global__ void k_fill_from_keys(const uint64_t* keys, long long m2, int n, int S, const long long* key_off,
                                 const long long* row_start, int32_t* col, int* bad);
__global__ void k_export_rows(const int32_t* deg, int n, const long long* row_start, const int32_t* col,
                              const int32_t* perm, const long long* out_off_ext, const int32_t* iperm,
                              int32_t* out_col);
__global__ void k_ext_degrees(const int32_t* deg, const int32_t* iperm, int n, int32_t* ext_deg);

// gc_region.cu
__global__ void k_bfs_sources(Ctl* c, const int32_t* srcA, const int32_t* srcD, uint32_t* visited, int32_t* wlist);
__global__ void k_level_mark(Ctl* c, int L);
__global__ void k_region_rest(Ctl* c, int n, uint32_t* visited, int32_t* wlist);
__global__ void k_u_count_twin(const Ctl* c, const int32_t* wlist, const int32_t* deg, const int2* segA,
                               int32_t* U_deg);
__global__ void k_u_fill_twin(const Ctl* c, const int32_t* wlist, const long long* row_start, const int32_t* deg,
                              const int32_t* col, const int2* segA, const int2* segD, const int32_t* dstA,
                              const int32_t* dstD, const long long* U_off, uint32_t* U_col, int32_t* U_split,
                              int32_t* da, int32_t* db);
__global__ void k_batch_keys_twin(Ctl* c, const int32_t* perm, int n, int S, uint64_t* keys);
__global__ void k_batch_decide_twin(const uint64_t* keys, Ctl* c, int S, const long long* row_start,
                                    const int32_t* deg, const int32_t* col, int32_t* keepA, int32_t* keepD);
__global__ void k_batch_compact_twin(const uint64_t* keys, const Ctl* c, int S, const int32_t* keepA,
                                     const int32_t* keepD, const long long* posA, const long long* posD,
                                     int32_t* srcA, int32_t* dstA, int32_t* srcD, int32_t* dstD);
__global__ void k_bfs_expand(Ctl* c, int L, const long long* row_start, const int32_t* deg, const int32_t* col,
                             uint32_t* visited, int32_t* wlist);
__global__ void k_region_all(Ctl* c, int n, int32_t* wlist);
// all = 1: every entry of each row (the edge-local path), else N(u) n W
__global__ void k_u_count(const Ctl* c, const int32_t* wlist, const uint32_t* visited, const long long* row_start,
                          const int32_t* deg, const int32_t* col, const int2* segA, int32_t* U_deg, int all);
__global__ void k_u_fill(const Ctl* c, const int32_t* wlist, const uint32_t* visited, const long long* row_start,
                         const int32_t* deg, const int32_t* col, const int2* segA, const int2* segD,
                         const int32_t* dstA, const int32_t* dstD, const long long* U_off, uint32_t* U_col,
                         int32_t* U_split, int32_t* da, int32_t* db, int all);

__global__ void k_u_fill_all(const Ctl* c, const int32_t* wlist, const long long* row_start, const int32_t* deg,
                             const int32_t* col, const int2* segA, const int2* segD, const int32_t* dstA,
                             const int32_t* dstD, const long long* U_off, uint32_t* U_col, int32_t* U_split,
                             int32_t* da, int32_t* db);

// gc_count.cu
__global__ void k_reset_count(Ctl* c);
__global__ void k_zero_u64(unsigned long long* a, const long long* d_len);
__global__ void k_edge_terms(Ctl* c, const int32_t* wlist, const long long* U_off, const uint32_t* U_col,
                             const int32_t* U_split, const unsigned long long* tpack, const int32_t* da,
                             const int32_t* db);
__global__ void k_finalize(Ctl* c, int mode);

// Device buffers of one counting pass over a region union graph.
struct CountArgs {
    Ctl* ctl;
    const int32_t* wlist;          // region vertices (c->nW of them)
    const long long* U_off;        // n_alloc + 1
    const uint32_t* U_col;         // flagged entries
    const int32_t* U_split;        // start of the out-list per vertex
    long long* U_wt;               // n_alloc: wedge bound per pivot (written by the pass)
    const int32_t* da;             // degree in G_a
    const int32_t* db;             // degree in G_b
    unsigned long long* tpack;     // per-entry triangle counters, zeroed
    int32_t* bins;                 // NBINS * n_alloc
    unsigned long long* dense;     // dense_clusters * dense_stride(n_alloc) zeroed words
    int n_alloc;                   // vertex id bound
    int dense_clusters;            // clusters of the heavy 4-cycle kernel
    int dense_cluster_size;        // CTAs per such cluster (8 or 16)
    unsigned long long* cta_tables; // cta_groups * cta_table_words zeroed words
    long long cta_table_words;      // power of two; pivots up to half of it use the hash tier
    int cta_groups;                 // CTAs of the medium 4-cycle kernel (one table each)
    unsigned char* chunk_scratch;   // sms * c4_chunk_cta_bytes(chunk_cap): per-CTA run bounds of the chunked kernel
    long long chunk_cap;            // run-bound entries per CTA (0: the chunked tier is off)
    Tuning tune;                    // bin boundaries (clamped to the capacities)
    int sms;
    cudaStream_t aux[3] = {nullptr, nullptr, nullptr};  // side streams of the counting pass (or none)
    cudaEvent_t fork = nullptr;     // fork / join events for them (timing disabled)
    cudaEvent_t join[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t ev_heavy[2] = {nullptr, nullptr};  // around the heavy-pivot 4-cycle kernels, on their stream
};
Tuning effective_tuning(const CountArgs& a);
// Dynamic shared-memory limits of the counting kernels (once per device).
void count_setup_attributes();
void local_setup_attributes();
size_t c4_chunk_smem_bytes();
int c4_chunk_width(long long n);                 // id-range chunks + 1
long long c4_chunk_cap(long long n);             // run-bound entries per CTA for ids below n
// bytes of one CTA's scratch of the chunked kernel: run bounds int32[cap],
// row starts int64[cap / 2], row flags uint32[cap / 2]
__host__ __device__ inline size_t c4_chunk_cta_bytes(long long cap) {
    return (size_t)cap * 4 + (size_t)(cap / 2) * 12;
}
// Cluster shape of the heavy 4-cycle kernel: CTAs per cluster (want = 0:
// 16 if the device can co-schedule it, else 8) and the number of clusters.
int dense_cluster_plan(int want, int sms, int* size_out);

// 64-bit words of one cluster's counter region in the heavy 4-cycle kernel
// for n vertices: an even count (16-byte aligned regions) with room for the
// narrow layout's arrays, list counter and padding at every n.
__host__ __device__ constexpr long long dense_stride(long long n) { return ((n + 1) & ~1ll) + 8; }
// Device buffers of the edge-local path (gc_local.cu).  V_X = wlist[0 ..
// lvl[0]), marked in `visited`; its union rows in U_off / U_col, degrees in
// G_a / G_b in da / db.  The scratch arrays hold `cap` entries (the offset
// arrays cap + 1); a batch that needs more sets Ctl::lovf and l_need.
struct LocalArgs {
    Ctl* ctl;
    const int32_t* wlist;
    const uint32_t* visited;
    const long long* U_off;
    const uint32_t* U_col;
    const long long* row_start;
    const int32_t* deg;
    const int32_t* col;
    const int32_t* da;
    const int32_t* db;
    unsigned long long* tpack;     // per-entry triangle counters, zeroed
    const int32_t *srcA, *dstA, *srcD, *dstD;  // kept directed entries of the batch
    int32_t *cost, *own, *pcost, *ccnt, *kcost, *tpair, *walk;
    long long *pre, *ppre, *cpre, *kpre;
    unsigned long long* rec;
    long long* dcnt;               // per-entry change of t (cap entries)
    // maintained triangle sums (null: not valid, every edge at V_X is intersected)
    unsigned long long* T2;        // n: sum of t_e over the edges at each vertex
    long long* dtri2;              // n zeroed words: its change in the batch (cleared after)
    uint32_t* visited2;            // n bits, zeroed: third vertices already listed
    int32_t* wlist_w;              // = wlist (third vertices are appended after V_X)
    long long* bsum;               // 1024 words
    long long cap;
    int n;                         // vertex id bound (U_off has n + 1 entries)
    int sms;
};
// T2 (zeroed) from a static count: sum of t_e over the edges at each vertex.
__global__ void k_t2_from_static(const Ctl* c, const int32_t* wlist, const long long* U_off, const uint32_t* U_col,
                                 const int32_t* U_split, const unsigned long long* tpack, unsigned long long* T2);
// T2 of the vertices within one hop of a committed region batch (mark, then add).
__global__ void k_t2_mark(const Ctl* c, const int32_t* wlist, uint32_t* mark, unsigned long long* T2);
__global__ void k_t2_from_region(const Ctl* c, const int32_t* wlist, const long long* U_off, const uint32_t* U_col,
                                 const int32_t* U_split, const unsigned long long* tpack, const uint32_t* mark,
                                 unsigned long long* T2);
// Enqueue the edge-local delta (after the union rows of V_X); events mark
// the triangle stage, the 4-clique / 4-cycle stage and the closed forms.
int enqueue_local(const LocalArgs& a, cudaStream_t s, cudaEvent_t ev_tri, cudaEvent_t ev_sub, cudaEvent_t ev_fin,
                  int commit);

// Per-vertex graphlet counts of a static pass (gc_vertex.cu).
// Heavy 4-cycle pivots of the per-vertex and per-edge counts (gc_vertex.cu):
// pivots with w~ >= heavy_min are walked C4G at a time by the whole grid,
// each with its own counter array in cnt_g; heavy_min = 0 leaves every
// pivot to the per-block walk.
constexpr int C4G = 8;
struct HeavyC4 {
    long long heavy_min;
    const long long* U_wt;         // w~ per pivot (static pass)
    uint8_t* heavy;                // n flags
    int32_t* hlist;                // n
    int* hcount;                   // 1
    uint32_t* cnt_g;               // C4G * n, zeroed
};

struct VertexArgs {
    Ctl* ctl;
    const int32_t* wlist;          // all vertices (c->nW = n)
    const long long* U_off;
    const uint32_t* U_col;
    const int32_t* U_split;
    const unsigned long long* tpack;
    const unsigned long long* T2;
    uint32_t* tall;                // nU: t of every entry
    long long* sdeg;               // n
    long long* NV;                 // 11 n role counts, zeroed
    uint32_t* cnt;                 // c4_blocks * n, zeroed
    int c4_blocks;
    int n;
    const int32_t* iperm;
    unsigned long long* out;       // 6 n (graphlets) or 11 n (orbits), by external id
    int orbits;
    int sms;
    HeavyC4 hv;
};
// Returns the kernels launched, or -1 on a CUDA error.
int enqueue_vertex_counts(const VertexArgs& a, cudaStream_t s);

struct EdgeArgs {
    Ctl* ctl;
    const int32_t* wlist;          // all vertices (c->nW = n)
    const long long* U_off;
    const uint32_t* U_col;
    const int32_t* U_split;
    const unsigned long long* tpack;
    const unsigned long long* T2;
    uint32_t* tall;                // nU: t of every entry
    long long* sdeg;               // n
    long long* NE;                 // 4 nU per-entry credits, zeroed
    unsigned long long* keys;      // nU sort keys (the first m sorted are the edges)
    unsigned long long* keys_tmp;  // nU
    uint32_t* hist;                // 256 sort_grid
    int sort_grid;
    const long long* d_count;      // device copy of nU
    long long nU, m;
    int nb;                        // bits of an external id
    uint32_t* cnt;                 // c4_blocks * n, zeroed
    int c4_blocks;
    int n;
    const int32_t* iperm;
    unsigned long long* out;       // 10 m (edge orbits) or 6 m (graphlets), by external (lo, hi) order
    int32_t* edges;                // 2 m: (lo, hi) per output row
    int orbits;
    int sms;
    HeavyC4 hv;
};
// Returns the kernels launched, or -1 on a CUDA error.
int enqueue_edge_counts(const EdgeArgs& a, cudaStream_t s);

// Enqueue the counting kernels (binning, triangles / 4-cliques, 4-cycles,
// edge terms, closed forms with k_finalize(mode)); events, when given, are
// recorded before the triangle, 4-cycle and edge-term stages.  Returns the
// number of kernels launched.
int enqueue_counting(const CountArgs& a, cudaStream_t s, cudaEvent_t ev_tri, cudaEvent_t ev_c4, cudaEvent_t ev_end,
                     int mode);

}  // namespace gcx
