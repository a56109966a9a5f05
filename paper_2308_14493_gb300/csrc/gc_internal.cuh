// gc_internal.cuh -- shared definitions of the CUDA graphlet-counting library.
//
// Vertex numbering.  The library renumbers vertices once, at open, in
// ascending order of their initial degree (ties by id).  Every adjacency row
// is kept sorted by this internal id, and each edge is oriented from its
// lower to its higher internal id.  Any total order gives exact counts; the
// degree order keeps out-lists short (hubs point to few vertices).
//
// Region union graph U.  For a batch B = A u D (Algorithm 2, Sec. 4.3) the
// region is W, the k-hop neighbourhood of the batch endpoints.  G_a and G_b
// share every edge of G[W] except the batch pairs, so both are stored as one
// adjacency structure U = G[W] u A whose entries carry two membership bits:
//   FLAG_A  the edge is in G_a = (H \ D) u A  (every entry except D pairs)
//   FLAG_B  the edge is in G_b = (H \ A) u D  (every entry except A pairs)
// One pass over U then counts both graphs.  A full static count is the
// special case W = V, no batch, both bits on every entry.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gcx {

constexpr uint32_t ID_MASK = 0x3FFFFFFFu;  // vertex id (n < 2^30)
constexpr uint32_t FLAG_A = 0x40000000u;   // entry belongs to G_a
constexpr uint32_t FLAG_B = 0x80000000u;   // entry belongs to G_b
constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int MAX_HOPS = 8;

// Work bins of the counting pass: region bins[b * n ...] holds the vertices
// of bin b.  Triangle roots by out-degree k; 4-cycle pivots by the wedge
// bound w~ = sum of the degrees of the lower neighbours.
enum {
    // (default boundaries; the Tuning below moves them at run time)
    BIN_TRI_WARP = 0,   // 2 <= k <= 32                   warp per root
    BIN_TRI_BLOCK = 1,  // TRI_KS < k <= TRI_KM            block per root
    BIN_TRI_MERGE = 2,  // k > TRI_KM                      merge per out-edge
    BIN_C4_REG = 3,     // w~ <= 32                        registers (match)
    BIN_C4_WARP = 4,    // w~ <= C4_T1                     warp hash in shared memory
    BIN_C4_BLOCK = 5,   // C4B_SMALL_MAX < w~ <= C4_T2     block hash in shared memory
    BIN_C4_DENSE = 6,   // C4_T3 < w~ <= c4_chunk_min      cluster, shared dense counter array
    BIN_C4_CTA = 7,     // C4_T2 < w~ <= C4_T3             CTA, own hash table in global memory
    BIN_C4_CHUNK = 8,   // w~ > c4_chunk_min (off)         CTA, shared-memory counters over id-range chunks
    BIN_TRI_SMALL = 9,  // 32 < k <= TRI_KS                block per root, small shared footprint
    BIN_C4_BSMALL = 10, // w~ <= C4B_SMALL_MAX             block hash in shared memory, small table
    NBINS = 11
};

// Work counters (Ctl::work) of the kernels that take their roots or pivots
// one at a time; kernels that run side by side need different counters.
enum {
    WORK_TRI_BLOCK = 1,   // k_tri_block, long out-lists
    WORK_C4_BLOCK = 2,    // k_c4_block, large table
    WORK_C4_DENSE = 3,    // k_c4_dense_t, clusters
    WORK_C4_CTA = 4,      // k_c4_hash (and k_c4_dense_t without clusters)
    WORK_C4_CHUNK = 5,    // k_c4_chunk
    WORK_TRI_SMALL = 6,   // k_tri_block, short out-lists
    WORK_C4_BSMALL = 7,   // k_c4_block, small table
    NWORK = 8
};

constexpr int ACC_STRIPES = 32;  // copies of each accumulator (spreads the atomics of many warps)
constexpr int NACC = 23;         // accumulator slots (see Ctl::acc)

// Device control block: sizes produced and consumed on the device, so a
// batch's kernels never wait for the host between stages.
struct Ctl {
    long long n_ins, n_del;          // raw pairs of the batch
    long long nkeys;                 // directed batch keys = 2 (n_ins + n_del)
    long long nA2, nD2;              // kept directed insertion / deletion entries
    unsigned long long st[8];        // [0] repeats [1] cancelled [2] no-op ins [3] no-op del (directed)
    int nW;                          // region size
    int lvl[MAX_HOPS + 2];           // lvl[L]: end of BFS level L in the region list
    long long nU;                    // entries of the region union graph
    unsigned long long acc[NACC];    // [0..5] sums of G_a, [6..11] sums of G_b: P, S, 2TT, D, K, Q
                                     // [12] |E(G_a)|, [13] |E(G_b)|, [14] triangle work, [15] wedges
                                     // [16] sum of t_e in G_a (3 triangles), [17] in G_b,
                                     // [18] sum C(d,2) in G_a (2-paths), [19] in G_b
                                     // heavy-pivot 4-cycle tier: [20] wedges, [21] L2
                                     // reductions, [22] L2 atomics returning the old value
    unsigned long long F[6];         // maintained counts
    long long Ca[6], Cb[6];          // induced counts of G_a, G_b of the last pass
    long long sa[6], sb[6];          // their non-induced sums (TT halved)
    unsigned long long pool_tail;    // first free column slot of the adjacency pool
    unsigned long long scratch_tail; // bump pointer of the commit scratch
    int overflow;                    // commit needs a re-layout
    int err;                         // GC_E* code raised on the device
    unsigned work[NWORK];            // dynamic work counters (WORK_*)
    int nbin[NBINS];                 // sizes of the work bins (see gc_count.cu)
    int maxdeg;                      // largest union-graph degree in the region
    // batch source and sequencing (a captured batch graph reads these)
    const int32_t* pairs_ins;        // base of the insertion pairs
    const int32_t* pairs_del;        // base of the deletion pairs
    long long ins_off, del_off;      // offsets (in pairs) of the current batch
    long long tw_off[4], tw_n[4];    // a twin pass (two independent batches): ins / del of the
                                     // first, ins / del of the second, offsets and sizes
    int cur;                         // index of the current batch in a run
    int active;                      // the current batch runs (no commit is pending)
    int halt;                        // a commit ran out of pool space; later batches wait
    int pend_ns;                     // endpoints of the batch whose commit is pending
    long long pend_nA2, pend_nD2;    // its kept directed insertion / deletion entries
    long long m_delta;               // net edges committed during a run
    unsigned long long last_out[6];  // counts after the current batch
    unsigned long long prev_out[6];  // counts before it, when its pass counted both whole graphs
                                     // (the two-batch form: out of the batch before it)
    // 3-vertex graphlets, [0] induced 2-path (open wedge), [1] triangle
    unsigned long long F3[2];        // maintained
    long long C3a[2], C3b[2];        // of G_a, G_b of the last pass
    unsigned long long last_out3[2]; // after the current batch
    // edge-local path (gc_local.cu)
    int lovf;                        // a local scratch array was too small: nothing applied
    long long l_np;                  // changed-pair slots (kept directed entries)
    long long l_len[4];              // lengths of its scans: [0] union entries [1] pair slots
                                     // [2] common-neighbour records [3] 4-cycle tasks (0: skip)
    long long l_tot[5];              // totals: [0] triangle probes [1] records [2] 4-clique probes
                                     // [3] 4-cycle tasks [4] 4-cycle probes
    long long l_need;                // entries the largest local array needed
    int l_nw3;                       // third vertices listed after V_X (maintained triangle sums)
    // (device-only tail: the host mirror copies the block up to here)
    unsigned long long accs[NACC][ACC_STRIPES];  // acc, striped: kernels add here, k_finalize sums
};

constexpr int TRI_KM = 512;
constexpr int TRI_KS = 128;
constexpr int C4_T1 = 512;
constexpr int C4_T2 = 8192;
constexpr int C4B_SMALL_MAX = 2048;  // block-hash pivots up to this bound use the small table
constexpr long long C4_T3 = 32768;
constexpr int C4_CLUSTER = 8;       // CTAs per cluster of the dense 4-cycle kernel
constexpr int CH_BYTES = 196608;    // shared counter bytes of the chunked 4-cycle kernel
constexpr int CH_R = CH_BYTES / 4;  // ids per chunk (49,152)

// Bin boundaries of the counting pass (upper bounds of each tier; each at
// most the capacity its kernel was compiled for).  Chosen per graph by the
// autotuner or set by the caller.
struct Tuning {
    int tri_warp_max;        // out-degree k: warp kernel up to this (<= 32)
    int tri_small_max;       // small-footprint block kernel up to this (<= TRI_KS)
    int tri_block_max;       // block kernel up to this (<= TRI_KM), merge beyond
    int c4_reg_max;          // wedge bound w~: registers up to this (<= 32)
    int c4_warp_max;         // warp hash (<= C4_T1)
    int c4_block_max;        // block hash (<= C4_T2)
    long long c4_cta_max;    // global hash tables (<= half the table words)
    long long c4_chunk_min;  // chunked shared-memory kernel above this ...
    long long c4_chunk_max;  // ... and up to this (the cluster kernel takes the rest)
};
constexpr long long NEVER = 1ll << 62;
inline Tuning default_tuning() { return Tuning{32, TRI_KS, TRI_KM, 32, C4_T1, C4_T2, C4_T3, NEVER, NEVER}; }
constexpr int C4_DENSE_THREADS = 1024;

// Handle-independent launch geometry.
struct Dims {
    int sms;
};

// Stage-boundary event: inside a stream capture it becomes an event-record
// node that records at every replay (a plain record there would only order
// the capture); outside a capture an ordinary record.
inline cudaError_t record_stage(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaError_t r = cudaStreamIsCapturing(s, &st);
    if (r != cudaSuccess) return r;
    return st == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                                               : cudaEventRecord(e, s);
}

__device__ __forceinline__ uint32_t vid(uint32_t e) { return e & ID_MASK; }

// Programmatic dependent launch: a kernel launched by pdl_launch may be
// scheduled while the kernel before it in the stream is still running;
// it waits here (first statement) until that kernel has finished and its
// writes are visible, then lets the next kernel be scheduled in turn.  The
// launch latency of a chain of small kernels is hidden this way.  Without
// a programmatic dependency both instructions are no-ops.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" :::);
}

template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(FULL, x, o);
    return x;
}

// first index in sorted a[0..len) whose id is >= key
__device__ __forceinline__ long long lower_bound_id(const uint32_t* a, long long len, uint32_t key) {
    long long lo = 0, hi = len;
    while (lo < hi) {
        long long mid = (lo + hi) >> 1;
        if ((a[mid] & ID_MASK) < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ long long lower_bound_i32(const int32_t* a, long long len, int32_t key) {
    long long lo = 0, hi = len;
    while (lo < hi) {
        long long mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ unsigned long long choose2(unsigned long long x) { return x * (x - 1) / 2; }
__device__ __forceinline__ unsigned long long choose3(unsigned long long x) {
    return x < 3 ? 0ull : x * (x - 1) / 2 * (x - 2) / 3;
}

// Warp-cooperative merge of one sorted adjacency row with a sorted list of
// insertions (ids absent from the row).  Row entries failing keep(v) are
// dropped; kept ones are written as v | tag(v); insertions as a | ins_tag.
// The output is sorted by id.  All 32 lanes must call it together.
// Returns the number of entries written.
template <class KeepF, class TagF>
__device__ __forceinline__ long long warp_merge_row(const int32_t* __restrict__ row, long long d,
                                                    const int32_t* __restrict__ ins, long long na,
                                                    uint32_t* __restrict__ out, uint32_t ins_tag, KeepF keep,
                                                    TagF tag) {
    const int lane = threadIdx.x & 31;
    long long obase = 0, ia = 0;
    for (long long cb = 0; cb < d; cb += 32) {
        long long idx = cb + lane;
        bool valid = idx < d;
        int32_t v = valid ? row[idx] : 0x7fffffff;
        bool kp = valid && keep(v);
        unsigned km = __ballot_sync(FULL, kp);
        int32_t vlast = row[(cb + 31 < d - 1) ? cb + 31 : d - 1];
        long long ib = ia;
        for (;;) {  // insertions in [ia, na) below vlast form a prefix
            long long j = ib + lane;
            unsigned m = __ballot_sync(FULL, j < na && ins[j] < vlast);
            ib += __popc(m);
            if (m != FULL) break;
        }
        if (kp) {
            long long lb = lower_bound_i32(ins + ia, ib - ia, v);
            out[obase + __popc(km & lanemask_lt()) + lb] = (uint32_t)v | tag(v);
        }
        for (long long j = ia; j < ib; j++) {
            int32_t a = ins[j];
            unsigned below = __ballot_sync(FULL, kp && v < a);
            if (lane == 0) out[obase + (j - ia) + __popc(below)] = (uint32_t)a | ins_tag;
        }
        obase += __popc(km) + (ib - ia);
        ia = ib;
    }
    for (long long j = ia + lane; j < na; j += 32) out[obase + (j - ia)] = (uint32_t)ins[j] | ins_tag;
    return obase + (na - ia);
}

// Block-cooperative merge of one sorted row with sorted insertions `ins`
// (ids absent from the row) and sorted deletions `del` (ids present in it):
// every entry finds its output position by binary searches in the others,
// so a long row spreads over the block.  keep_del: deletions stay, tagged
// del_tag (else they are dropped); other row entries get row_tag,
// insertions ins_tag.  The output is sorted by id.  Every thread of the
// block calls it; returns the output length.
__device__ __forceinline__ long long block_merge_row(const int32_t* __restrict__ row, long long d,
                                                     const int32_t* __restrict__ ins, long long na,
                                                     const int32_t* __restrict__ del, long long nd,
                                                     uint32_t* __restrict__ out, bool keep_del, uint32_t row_tag,
                                                     uint32_t ins_tag, uint32_t del_tag) {
    for (long long j = threadIdx.x; j < d; j += blockDim.x) {
        const int32_t v = row[j];
        const long long db = lower_bound_i32(del, nd, v);
        const bool is_del = db < nd && del[db] == v;
        if (is_del && !keep_del) continue;
        out[j - (keep_del ? 0 : db) + lower_bound_i32(ins, na, v)] = (uint32_t)v | (is_del ? del_tag : row_tag);
    }
    for (long long i = threadIdx.x; i < na; i += blockDim.x) {
        const int32_t a = ins[i];
        const long long rb = lower_bound_i32(row, d, a);
        const long long db = keep_del ? 0 : lower_bound_i32(del, nd, a);
        out[i + rb - db] = (uint32_t)a | ins_tag;
    }
    return d + na - (keep_del ? 0 : nd);
}

__device__ __forceinline__ bool sorted_contains(const int32_t* a, long long len, int32_t key) {
    long long p = lower_bound_i32(a, len, key);
    return p < len && a[p] == key;
}

// ---- host-side launchers implemented in the .cu files -------------------

// gc_sort.cu
// Sort `keys` (uint64) of device-resident length *d_count (<= max_count) by
// their low `bits` bits.  `tmp` holds max_count keys; `hist` holds 256 * grid
// words.  The sorted keys end in `keys`.
// Returns the number of kernels launched.
int radix_sort_u64(uint64_t* keys, uint64_t* tmp, const long long* d_count, long long max_count, int bits,
                   uint32_t* hist, int grid, cudaStream_t s);
int radix_grid(long long max_count, int sms);
// Exclusive prefix sum of int32 in[0..len) into int64 out[0..len], out[len] = total.
// len = *d_len when d_len != null, else host_len.  `bsum` holds `grid` int64.
// If total_out != null the total is also stored there.
int scan_i32_to_i64(const int32_t* in, long long* out, const long long* d_len, long long host_len,
                    long long* bsum, int grid, long long* total_out, cudaStream_t s);
int scan_grid(long long max_len, int sms);

}  // namespace gcx
