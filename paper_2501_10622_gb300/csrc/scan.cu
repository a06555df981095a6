// scan.cu -- exclusive prefix sum of uint32 arrays (reduce, scan block sums,
// scan + add).  Used for the deposit bins, the seed ranks and the compaction
// of kept halos.  No spin waits: three plain launches.
#include <algorithm>

#include "internal.cuh"

namespace cwthf {
namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanThreads * kScanItems;  // 4096 values per block

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread; *total gets the block sum.
// Every thread of the block must call it (it synchronises the block).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* total) {
    constexpr int kWarps = kScanThreads / 32;
    __shared__ uint32_t warp_off[kWarps + 1];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t inc = warp_incl_scan(v);
    if (lane == 31) warp_off[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = (lane < kWarps) ? warp_off[lane] : 0u;
        uint32_t si = warp_incl_scan(s);
        if (lane < kWarps) warp_off[lane] = si - s;
        if (lane == kWarps - 1) warp_off[kWarps] = si;
    }
    __syncthreads();
    uint32_t excl = inc - v + warp_off[wid];
    *total = warp_off[kWarps];
    __syncthreads();  // warp_off may be reused by the next call
    return excl;
}

// Length of the scan: n, or the device value *d_n clamped to the capacity n.
__device__ __forceinline__ int64_t scan_len(int64_t n, const uint32_t* d_n) {
    return d_n ? min(int64_t(*d_n), n) : n;
}

__global__ void __launch_bounds__(kScanThreads) k_block_sums(const uint32_t* __restrict__ in, int64_t n,
                                                             const uint32_t* d_n, uint32_t* __restrict__ sums) {
    int64_t len = scan_len(n, d_n);
    int64_t base = int64_t(blockIdx.x) * kScanChunk;
    if (base >= len) return;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t idx = base + int64_t(i) * kScanThreads + threadIdx.x;
        if (idx < len) s += in[idx];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ uint32_t ws[kScanThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kScanThreads / 32; w++) t += ws[w];
        sums[blockIdx.x] = t;
    }
}

// One block scans the (<= 32 * kScanThreads * ...) block sums in place, sequential chunks.
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(uint32_t* sums, int64_t nblocks_cap, int64_t n,
                                                            const uint32_t* d_n) {
    int64_t len = scan_len(n, d_n);
    int64_t nb = (len + kScanChunk - 1) / kScanChunk;
    if (nb > nblocks_cap) nb = nblocks_cap;
    uint32_t carry = 0;
    for (int64_t base = 0; base < nb; base += kScanThreads) {
        int64_t idx = base + threadIdx.x;
        uint32_t v = idx < nb ? sums[idx] : 0u;
        uint32_t tot;
        uint32_t ex = block_excl_scan(v, &tot);
        if (idx < nb) sums[idx] = ex + carry;
        carry += tot;
    }
    if (threadIdx.x == 0) sums[nblocks_cap] = carry;  // grand total
}

__global__ void __launch_bounds__(kScanThreads) k_scan_add(const uint32_t* in, int64_t n, const uint32_t* d_n,
                                                           const uint32_t* __restrict__ sums, int64_t nblocks_cap,
                                                           uint32_t* out) {
    int64_t len = scan_len(n, d_n);
    int64_t base = int64_t(blockIdx.x) * kScanChunk;
    if (blockIdx.x == 0 && threadIdx.x == 0) out[len] = sums[nblocks_cap];
    if (base >= len) return;
    // each thread owns kScanItems consecutive values
    uint32_t v[kScanItems];
    uint32_t local = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t idx = base + int64_t(threadIdx.x) * kScanItems + i;
        v[i] = idx < len ? in[idx] : 0u;
        local += v[i];
    }
    uint32_t tot;  // block_excl_scan synchronises: every value is read before any is written
    uint32_t ex = block_excl_scan(local, &tot) + sums[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t idx = base + int64_t(threadIdx.x) * kScanItems + i;
        if (idx < len) out[idx] = ex;
        ex += v[i];
    }
}

int scan_generic(cwthf_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n_cap, const uint32_t* d_n,
                 cudaStream_t s) {
    int64_t nb = (n_cap + kScanChunk - 1) / kScanChunk;
    if (nb < 1) nb = 1;
    if (size_t(nb) + 2 > ctx->scan_tmp_cap) return CWTHF_E_INVALID_ARG;
    uint32_t* sums = ctx->scan_tmp;
    CWTHF_LAUNCH(ctx, s, "k_block_sums", k_block_sums<<<unsigned(nb), kScanThreads, 0, s>>>(in, n_cap, d_n, sums));
    CWTHF_LAUNCH(ctx, s, "k_scan_sums", k_scan_sums<<<1, kScanThreads, 0, s>>>(sums, nb, n_cap, d_n));
    CWTHF_LAUNCH(ctx, s, "k_scan_add", k_scan_add<<<unsigned(nb), kScanThreads, 0, s>>>(in, n_cap, d_n, sums, nb, out));
    return cuda_status(cudaGetLastError());
}

}  // namespace

size_t scan_tmp_words(int64_t n_cap) { return size_t((n_cap + kScanChunk - 1) / kScanChunk) + 2; }

int scan_u32(cwthf_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s) {
    return scan_generic(ctx, in, out, n, nullptr, s);
}

int scan_u32_dev(cwthf_ctx* ctx, const uint32_t* in, uint32_t* out, const uint32_t* d_n, int64_t n_cap,
                 cudaStream_t s) {
    return scan_generic(ctx, in, out, n_cap, d_n, s);
}

// The same three launches on caller-provided block-sum storage (no context).
int scan_u32_scratch(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp, size_t tmp_cap, cudaStream_t s) {
    int64_t nb = std::max<int64_t>((n + kScanChunk - 1) / kScanChunk, 1);
    if (size_t(nb) + 2 > tmp_cap) return CWTHF_E_INVALID_ARG;
    k_block_sums<<<unsigned(nb), kScanThreads, 0, s>>>(in, n, nullptr, tmp);
    k_scan_sums<<<1, kScanThreads, 0, s>>>(tmp, nb, n, nullptr);
    k_scan_add<<<unsigned(nb), kScanThreads, 0, s>>>(in, n, nullptr, tmp, nb, out);
    return cuda_status(cudaGetLastError());
}

}  // namespace cwthf
