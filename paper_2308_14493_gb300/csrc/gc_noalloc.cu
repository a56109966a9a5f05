// gc_noalloc.cu -- a static graphlet count that allocates no memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the
// moment they need a count: a service whose device memory is entirely
// reserved up front by another allocator, a real-time loop that cannot take
// the implicit device synchronisation and latency of a fresh allocation, or
// a plug-in running inside a host process that forbids new device
// allocations after start-up.  gc_count_static_noalloc serves them: it counts
// the six graphlets of a small graph that the caller already holds in device
// memory, using only the fixed scratch array below.
//
// The scratch is one file-scope __device__ array.  Every GPU that loads this
// library keeps it, zero-initialised, until the process exits.  Host code
// must not pass the array's name to a kernel (in host code it is only a
// host-side stand-in); the device address is fetched once per device with
// cudaGetSymbolAddress on the first call made with that device current.
// All calls share the array and it keeps the last call's contents, so each
// call clears what must start at zero, and calls that overlap on the GPU
// (different streams, or different host threads) race.
#include <algorithm>
#include <mutex>

#include "gc.h"
#include "gc_internal.cuh"
#include "gc_kernels.cuh"

using namespace gcx;

namespace {

constexpr int NA_MAX_N = GC_NOALLOC_MAX_VERTICES;      // vertices
constexpr long long NA_MAX_E = GC_NOALLOC_MAX_ENTRIES;  // directed adjacency entries (2m)
constexpr int NA_DENSE_CLUSTERS = 2;                   // clusters of the heaviest 4-cycle pivots
constexpr int NA_CTA_GROUPS = 4;                       // CTAs of the medium 4-cycle pivots
constexpr long long NA_TABLE_WORDS = 1 << 15;          // hash table words per such CTA
constexpr int NA_TPB = 256;

// byte offsets of the pieces inside the scratch array
constexpr size_t al(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t OFF_CTL = 0;
constexpr size_t OFF_UOFF = al(OFF_CTL + sizeof(Ctl));
constexpr size_t OFF_WT = al(OFF_UOFF + 8 * (size_t)(NA_MAX_N + 1));
constexpr size_t OFF_SPLIT = al(OFF_WT + 8 * (size_t)NA_MAX_N);
constexpr size_t OFF_DA = al(OFF_SPLIT + 4 * (size_t)NA_MAX_N);
constexpr size_t OFF_DB = al(OFF_DA + 4 * (size_t)NA_MAX_N);
constexpr size_t OFF_WL = al(OFF_DB + 4 * (size_t)NA_MAX_N);
constexpr size_t OFF_UCOL = al(OFF_WL + 4 * (size_t)NA_MAX_N);
constexpr size_t OFF_TPACK = al(OFF_UCOL + 4 * (size_t)NA_MAX_E);
constexpr size_t OFF_BINS = al(OFF_TPACK + 8 * (size_t)NA_MAX_E);
constexpr size_t OFF_DENSE = al(OFF_BINS + 4 * (size_t)NA_MAX_N * NBINS);
constexpr size_t OFF_CTA = al(OFF_DENSE + 8 * (size_t)dense_stride(NA_MAX_N) * NA_DENSE_CLUSTERS);
constexpr size_t OFF_ERR = al(OFF_CTA + 8 * (size_t)NA_TABLE_WORDS * NA_CTA_GROUPS);
constexpr size_t SCRATCH_BYTES = al(OFF_ERR + 16);

__device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

std::mutex g_mu;
void* g_base[128] = {};  // device address of the scratch array, per device ordinal
int g_sms[128] = {};     // multiprocessors per device

// Checks the caller's CSR (sorted rows, ids in range, no self-loops,
// symmetric) and builds the flagged union-graph view the counting kernels read:
// every entry belongs to both graphs, so both counts equal the static count.
// Edges are oriented by the caller's ids as they are (no degree renumbering,
// which would need scratch of its own): a 4-cycle pivot u walks every lower
// neighbour's row, so the wedge work is at most sum over edges of the lower
// endpoint's degree (m * d_max) rather than the degree-ordered bound that
// gc_count_static reaches after renumbering.  Any order gives exact counts;
// at the 16,384-vertex cap the worst case stays small.
__global__ void k_na_build(const int32_t* __restrict__ rp, const int32_t* __restrict__ col, int n, long long nnz,
                           Ctl* c, long long* __restrict__ U_off, uint32_t* __restrict__ U_col,
                           int32_t* __restrict__ U_split, int32_t* __restrict__ da, int32_t* __restrict__ db,
                           int32_t* __restrict__ wlist, int* __restrict__ bad) {
    long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    if (tid == 0) {
        if (rp[0] != 0 || rp[n] != nnz) atomicExch(bad, 1);
        c->nW = n;
        for (int i = 0; i < MAX_HOPS + 2; i++) c->lvl[i] = n;
    }
    for (long long v = tid; v < n; v += stride) {
        long long b = rp[v], e = rp[v + 1];
        if (b < 0 || e < b || e > nnz) {
            atomicExch(bad, 1);
            U_off[v] = 0;
            U_split[v] = 0;
            da[v] = db[v] = 0;
        } else {
            U_off[v] = b;
            da[v] = db[v] = (int32_t)(e - b);
            long long lo = b, hi = e;  // first entry above v
            while (lo < hi) {
                long long mid = (lo + hi) >> 1;
                if (col[mid] <= v) lo = mid + 1;
                else hi = mid;
            }
            U_split[v] = (int32_t)(lo - b);
        }
        wlist[v] = (int32_t)v;
    }
    if (tid == 0) U_off[n] = nnz;
}

__global__ void k_na_fill(const int32_t* __restrict__ rp, const int32_t* __restrict__ col, int n, long long nnz,
                          uint32_t* __restrict__ U_col, int* __restrict__ bad) {
    // warp per row
    int lane = threadIdx.x & 31;
    long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    if (*bad) return;
    for (long long v = warp; v < n; v += nwarps) {
        long long b = rp[v], e = rp[v + 1];
        for (long long p = b + lane; p < e; p += 32) {
            int32_t w = col[p];
            bool ok = w >= 0 && w < n && w != v && (p == b || col[p - 1] < w);
            if (ok) {  // symmetric partner (w, v)
                long long lo = rp[w], hi = rp[w + 1];
                while (lo < hi) {
                    long long mid = (lo + hi) >> 1;
                    if (col[mid] < v) lo = mid + 1;
                    else hi = mid;
                }
                ok = lo < rp[w + 1] && col[lo] == v;
            }
            if (!ok) {
                atomicExch(bad, 1);
                continue;
            }
            U_col[p] = (uint32_t)w | FLAG_A | FLAG_B;
        }
    }
}

__global__ void k_na_reset(Ctl* c, int* bad) {
    if (threadIdx.x == 0) {
        *bad = 0;
        c->err = 0;
        c->nU = 0;
    }
}

}  // namespace

extern "C" int gc_count_static_noalloc(int32_t n, const int32_t* d_row_ptr, const int32_t* d_col, int64_t nnz,
                                       void* stream, uint64_t out[6]) {
    if (!out || n < 0 || nnz < 0 || !d_row_ptr || (nnz > 0 && !d_col)) return GC_EINVAL;
    if (n > NA_MAX_N || nnz > NA_MAX_E) return GC_EINVAL;  // beyond the fixed scratch
    if (n == 0) {
        if (nnz != 0) return GC_EINVAL;
        for (int i = 0; i < 6; i++) out[i] = 0;
        return GC_OK;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return GC_ECUDA;
    void* base = nullptr;
    int sms = 0;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_base[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) return GC_ECUDA;
            if (cudaDeviceGetAttribute(&g_sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
                return GC_ECUDA;
            count_setup_attributes();
            g_base[dev] = p;
        }
        base = g_base[dev];
        sms = g_sms[dev];
    }
    unsigned char* b = (unsigned char*)base;
    Ctl* ctl = (Ctl*)(b + OFF_CTL);
    long long* U_off = (long long*)(b + OFF_UOFF);
    int32_t* U_split = (int32_t*)(b + OFF_SPLIT);
    long long* U_wt = (long long*)(b + OFF_WT);
    int32_t* da = (int32_t*)(b + OFF_DA);
    int32_t* db = (int32_t*)(b + OFF_DB);
    int32_t* wlist = (int32_t*)(b + OFF_WL);
    uint32_t* U_col = (uint32_t*)(b + OFF_UCOL);
    unsigned long long* tpack = (unsigned long long*)(b + OFF_TPACK);
    int32_t* bins = (int32_t*)(b + OFF_BINS);
    unsigned long long* dense = (unsigned long long*)(b + OFF_DENSE);
    unsigned long long* cta_tables = (unsigned long long*)(b + OFF_CTA);
    int* bad = (int*)(b + OFF_ERR);
    cudaStream_t s = (cudaStream_t)stream;
    int nn = n > 0 ? n : 1;
    int grid = (int)((std::max<long long>(n, nnz) + NA_TPB - 1) / NA_TPB);
    if (grid < 1) grid = 1;
    if (grid > 1024) grid = 1024;
    // what must start at zero: flags, accumulators, triangle counters and the
    // 4-cycle counters (an interrupted earlier call may have left them dirty)
    const bool stale = cudaPeekAtLastError() != cudaSuccess;
    k_na_reset<<<1, 32, 0, s>>>(ctl, bad);
    // per-cluster counter regions of dense_stride(n) words
    if (cudaMemsetAsync(tpack, 0, 8 * (size_t)std::max<long long>(nnz, 1), s) != cudaSuccess ||
        cudaMemsetAsync(dense, 0, 8 * (size_t)dense_stride(nn) * NA_DENSE_CLUSTERS, s) != cudaSuccess ||
        cudaMemsetAsync(cta_tables, 0, 8 * (size_t)NA_TABLE_WORDS * NA_CTA_GROUPS, s) != cudaSuccess)
        return GC_ECUDA;
    k_reset_count<<<1, 32, 0, s>>>(ctl);
    k_na_build<<<grid, NA_TPB, 0, s>>>(d_row_ptr, d_col, n, nnz, ctl, U_off, U_col, U_split, da, db, wlist, bad);
    k_na_fill<<<grid, NA_TPB, 0, s>>>(d_row_ptr, d_col, n, nnz, U_col, bad);
    // a launch that failed shows in the runtime's last error; a failure
    // while the kernels run shows in the synchronisation's own result.  An
    // error the caller's earlier work left pending is not read or cleared
    // (it stays with its owner), and then launch errors are not told apart.
    if (!stale && cudaGetLastError() != cudaSuccess) return GC_ECUDA;
    // the counting kernels index by the ids they read, so they run only on a
    // CSR that passed the checks
    int hbad = 0;
    if (cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return GC_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GC_ECUDA;
    if (hbad) return GC_EINVAL;
    CountArgs ca;
    ca.ctl = ctl;
    ca.wlist = wlist;
    ca.U_off = U_off;
    ca.U_col = U_col;
    ca.U_split = U_split;
    ca.U_wt = U_wt;
    ca.da = da;
    ca.db = db;
    ca.tpack = tpack;
    ca.bins = bins;
    ca.dense = dense;
    ca.n_alloc = nn;
    ca.dense_clusters = NA_DENSE_CLUSTERS;
    ca.dense_cluster_size = 8;
    ca.cta_tables = cta_tables;
    ca.cta_table_words = NA_TABLE_WORDS;
    ca.chunk_scratch = nullptr;  // no chunked 4-cycle tier in the fixed scratch
    ca.chunk_cap = 0;
    ca.tune = default_tuning();
    ca.cta_groups = NA_CTA_GROUPS;
    ca.sms = sms;
    enqueue_counting(ca, s, nullptr, nullptr, nullptr, 1);
    if (!stale && cudaGetLastError() != cudaSuccess) return GC_ECUDA;
    long long Ca[6];
    if (cudaMemcpyAsync(Ca, ctl->Ca, sizeof(Ca), cudaMemcpyDeviceToHost, s) != cudaSuccess) return GC_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GC_ECUDA;
    for (int i = 0; i < 6; i++) out[i] = (uint64_t)Ca[i];
    return GC_OK;
}
