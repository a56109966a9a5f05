// gc_sort.cu -- device-wide primitives with device-resident lengths:
// LSD radix sort of uint64 keys and exclusive prefix sums.
//
// Both use a fixed grid whose blocks each own one contiguous chunk of the
// input, so the chunk bounds depend only on the length read on the device.
// That keeps every launch shape independent of the data, which lets a whole
// batch pipeline be captured once in a CUDA graph and replayed for batches of
// any size up to the planned maximum.
#include "gc_internal.cuh"

namespace gcx {

namespace {

constexpr int RS_BLOCK = 256;  // threads per block = number of 8-bit digits
constexpr int RS_WARPS = RS_BLOCK / 32;

__device__ __forceinline__ void chunk_of(long long n, long long& beg, long long& end) {
    long long G = gridDim.x;
    long long chunk = (n + G - 1) / G;
    beg = (long long)blockIdx.x * chunk;
    end = beg + chunk < n ? beg + chunk : n;
    if (beg > n) beg = n;
}

__global__ void __launch_bounds__(RS_BLOCK) k_rs_hist(const uint64_t* __restrict__ keys, const long long* d_count,
                                                     int shift, uint32_t* __restrict__ hist) {
    pdl_enter();
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    long long beg, end;
    chunk_of(*d_count, beg, end);
    for (long long i = beg + threadIdx.x; i < end; i += RS_BLOCK) atomicAdd(&h[(keys[i] >> shift) & 255], 1u);
    __syncthreads();
    hist[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// In-place exclusive scan of a[0..len) by one block of 1024 threads: each
// thread sums a contiguous slice, the 1024 slice sums are scanned with warp
// shuffles (two levels), then each thread rewrites its slice.
__global__ void __launch_bounds__(1024) k_scan_u32_one_block(uint32_t* a, int len) {
    pdl_enter();
    __shared__ uint32_t wsum[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int per = (len + 1023) / 1024;
    const int beg = t * per, end = min(beg + per, len);
    uint32_t s = 0;
    for (int i = beg; i < end; i++) s += a[i];
    uint32_t x = s;  // inclusive scan within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    uint32_t run = x - s + (warp > 0 ? wsum[warp - 1] : 0u);
    for (int i = beg; i < end; i++) {
        const uint32_t v = a[i];
        a[i] = run;
        run += v;
    }
}

// Stable scatter: each tile of RS_BLOCK keys is ranked within warps with
// __match_any_sync, warp counts are scanned per digit, and a running
// per-digit base carries the order across tiles.
__global__ void __launch_bounds__(RS_BLOCK) k_rs_scatter(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                                                        const long long* d_count, int shift,
                                                        const uint32_t* __restrict__ offs) {
    pdl_enter();
    __shared__ uint32_t base[256];
    __shared__ uint32_t wcnt[RS_WARPS][256];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    base[t] = offs[(size_t)t * gridDim.x + blockIdx.x];
    long long beg, end;
    chunk_of(*d_count, beg, end);
    for (long long tile = beg; tile < end; tile += RS_BLOCK) {
#pragma unroll
        for (int w = 0; w < RS_WARPS; w++) wcnt[w][t] = 0;
        __syncthreads();
        long long i = tile + t;
        bool valid = i < end;
        uint64_t key = valid ? in[i] : 0;
        unsigned d = valid ? (unsigned)((key >> shift) & 255) : 256u + (unsigned)lane;
        unsigned peers = __match_any_sync(FULL, d);
        unsigned rank = __popc(peers & lanemask_lt());
        if (valid && lane == __ffs(peers) - 1) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; w++) {
            uint32_t c = wcnt[w][t];
            wcnt[w][t] = run;
            run += c;
        }
        __syncthreads();
        if (valid) out[base[d] + wcnt[warp][d] + rank] = key;
        __syncthreads();
        base[t] += run;
    }
}

__global__ void k_copy_u64(const uint64_t* __restrict__ in, uint64_t* __restrict__ out, const long long* d_count) {
    pdl_enter();
    long long n = *d_count;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = in[i];
}

// ---- scan -----------------------------------------------------------------

constexpr int SC_BLOCK = 512;

__device__ __forceinline__ long long block_incl_scan_i64(long long x, long long* sh) {
    // sh: at least 32 entries
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        sh[lane] = w;
    }
    __syncthreads();
    long long r = x + (warp > 0 ? sh[warp - 1] : 0);
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SC_BLOCK) k_scan_partials(const int32_t* __restrict__ in, const long long* d_len,
                                                           long long host_len, long long* __restrict__ bsum) {
    pdl_enter();
    __shared__ long long sh[32];
    long long n = d_len ? *d_len : host_len;
    long long beg, end;
    chunk_of(n, beg, end);
    long long s = 0;
    for (long long i = beg + threadIdx.x; i < end; i += SC_BLOCK) s += in[i];
    s = block_incl_scan_i64(s, sh);
    if (threadIdx.x == SC_BLOCK - 1) bsum[blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024) k_scan_top(long long* bsum, int G) {
    pdl_enter();
    __shared__ long long sh[32];
    // G <= 1024
    long long x = threadIdx.x < G ? bsum[threadIdx.x] : 0;
    long long inc = block_incl_scan_i64(x, sh);
    if (threadIdx.x < G) bsum[threadIdx.x] = inc - x;
}

__global__ void __launch_bounds__(SC_BLOCK) k_scan_apply(const int32_t* __restrict__ in, long long* __restrict__ out,
                                                        const long long* d_len, long long host_len,
                                                        const long long* __restrict__ bsum, long long* total_out) {
    pdl_enter();
    __shared__ long long sh[32];
    long long n = d_len ? *d_len : host_len;
    long long beg, end;
    chunk_of(n, beg, end);
    long long run = bsum[blockIdx.x];
    for (long long tile = beg; tile < end; tile += SC_BLOCK) {
        long long i = tile + threadIdx.x;
        long long x = i < end ? in[i] : 0;
        long long inc = block_incl_scan_i64(x, sh);
        if (i < end) out[i] = run + inc - x;
        // total of this tile = inclusive value of the last thread
        __shared__ long long tile_total;
        if (threadIdx.x == SC_BLOCK - 1) tile_total = inc;
        __syncthreads();
        run += tile_total;
        __syncthreads();
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        out[n] = run;
        if (total_out) *total_out = run;
    }
}

}  // namespace

// One block per 1024 keys (four tiles: short serial scatter loops for the
// small sorts of a batch), at most two per SM.
int radix_grid(long long max_count, int sms) {
    long long g = (max_count + 1023) / 1024;
    if (g < 1) g = 1;
    if (g > 2L * sms) g = 2L * sms;
    if (g > 1024) g = 1024;
    return (int)g;
}

int radix_sort_u64(uint64_t* keys, uint64_t* tmp, const long long* d_count, long long max_count, int bits,
                   uint32_t* hist, int grid, cudaStream_t s) {
    int passes = (bits + 7) / 8;
    int launches = 3 * passes;
    uint64_t* a = keys;
    uint64_t* b = tmp;
    for (int p = 0; p < passes; p++) {
        int shift = 8 * p;
        pdl_launch(k_rs_hist, dim3(grid), dim3(RS_BLOCK), 0, s, a, d_count, shift, hist);
        pdl_launch(k_scan_u32_one_block, dim3(1), dim3(1024), 0, s, hist, 256 * grid);
        pdl_launch(k_rs_scatter, dim3(grid), dim3(RS_BLOCK), 0, s, a, b, d_count, shift, hist);
        uint64_t* t = a;
        a = b;
        b = t;
    }
    if (a != keys) {
        int g = (int)((max_count + 255) / 256);
        if (g < 1) g = 1;
        if (g > 2048) g = 2048;
        pdl_launch(k_copy_u64, dim3(g), dim3(256), 0, s, a, keys, d_count);
        launches++;
    }
    return launches;
}

int scan_grid(long long max_len, int sms) {
    long long g = (max_len + 8191) / 8192;
    if (g < 1) g = 1;
    if (g > 4L * sms) g = 4L * sms;
    if (g > 1024) g = 1024;
    return (int)g;
}

int scan_i32_to_i64(const int32_t* in, long long* out, const long long* d_len, long long host_len, long long* bsum,
                    int grid, long long* total_out, cudaStream_t s) {
    pdl_launch(k_scan_partials, dim3(grid), dim3(SC_BLOCK), 0, s, in, d_len, host_len, bsum);
    pdl_launch(k_scan_top, dim3(1), dim3(1024), 0, s, bsum, grid);
    pdl_launch(k_scan_apply, dim3(grid), dim3(SC_BLOCK), 0, s, in, out, d_len, host_len, bsum, total_out);
    return 3;
}

}  // namespace gcx
