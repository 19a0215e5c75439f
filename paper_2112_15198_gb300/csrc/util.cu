// Device-wide exclusive scan and stable LSD radix sort used by the plan builder.
#include <cstdio>
#include <cstdlib>

#include "ifgf_internal.cuh"

namespace ifgf {

std::atomic<int64_t> g_launches{0};
std::atomic<int64_t> g_fail_alloc_in{0};

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t& total) {
    __shared__ int32_t warp_sums[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int32_t w = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;  // inclusive
    }
    __syncthreads();
    total = warp_sums[(blockDim.x >> 5) - 1];
    int32_t before = warp ? warp_sums[warp - 1] : 0;
    __syncthreads();
    return before + x - v;
}

__global__ void k_scan_reduce(const int32_t* __restrict__ in, int64_t n, int32_t* __restrict__ sums) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += in[base + i];
    int32_t tot;
    block_exclusive_scan(s, tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_down(const int32_t* in, int64_t n, const int32_t* __restrict__ offs, int32_t* out) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int32_t v[kScanItems];
    int32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0;
        s += v[i];
    }
    int32_t tot;
    int32_t pre = block_exclusive_scan(s, tot) + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = pre;
        pre += v[i];
    }
}

// ---- radix sort ----------------------------------------------------------------------
constexpr int kRsThreads = 256;
constexpr int kRsItems = 16;
constexpr int kRsTile = kRsThreads * kRsItems;
constexpr int kRsWarps = kRsThreads / 32;

__global__ void k_rs_hist(const uint64_t* __restrict__ keys, int64_t n, int shift, int32_t* __restrict__ hist,
                          int nblk) {
    __shared__ int32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
#pragma unroll 4
    for (int i = 0; i < kRsItems; ++i) {
        int64_t idx = base + (int64_t)i * kRsThreads + threadIdx.x;
        if (idx < n) atomicAdd(&cnt[(keys[idx] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: items are ranked chunk by chunk (256 consecutive items per chunk), inside a
// chunk by warp then lane, so equal digits keep their input order.
__global__ void k_rs_scatter(const uint64_t* __restrict__ kin, const int32_t* __restrict__ vin,
                             uint64_t* __restrict__ kout, int32_t* __restrict__ vout, int64_t n, int shift,
                             const int32_t* __restrict__ offs, int nblk) {
    __shared__ int32_t base[256];
    __shared__ int32_t wcnt[kRsWarps][256];
    __shared__ int32_t wpre[kRsWarps][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    base[threadIdx.x] = offs[(int64_t)threadIdx.x * nblk + blockIdx.x];
    for (int w = 0; w < kRsWarps; ++w) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t tile = (int64_t)blockIdx.x * kRsTile;
    const unsigned lt = (1u << lane) - 1u;
    for (int c = 0; c < kRsItems; ++c) {
        const int64_t idx = tile + (int64_t)c * kRsThreads + threadIdx.x;
        const bool valid = idx < n;
        uint64_t key = valid ? kin[idx] : 0;
        int32_t val = valid ? vin[idx] : 0;
        const int digit = valid ? (int)((key >> shift) & 255u) : 256;
        const unsigned peers = __match_any_sync(0xffffffffu, digit);
        const int rank = __popc(peers & lt);
        const int leader = __ffs(peers) - 1;
        if (valid && lane == leader) wcnt[warp][digit] = __popc(peers);
        __syncthreads();
        {
            int32_t s = 0;
            for (int w = 0; w < kRsWarps; ++w) {
                wpre[w][threadIdx.x] = s;
                s += wcnt[w][threadIdx.x];
            }
            wcnt[0][threadIdx.x] = s;  // chunk total of this digit (row 0 reused after reading)
        }
        __syncthreads();
        if (valid) {
            const int64_t pos = (int64_t)base[digit] + wpre[warp][digit] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        base[threadIdx.x] += wcnt[0][threadIdx.x];
        for (int w = 0; w < kRsWarps; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
    }
}

}  // namespace

void exclusive_scan_i32(Plan& p, const int32_t* in, int32_t* out, int64_t n) {
    if (n <= 0) return;
    const int64_t nblk = (n + kScanTile - 1) / kScanTile;
    if (nblk == 1) {
        IFGF_LAUNCH(k_scan_down, 1, kScanThreads, 0, p.stream, in, n, (const int32_t*)nullptr, out);
        return;
    }
    const size_t mark = p.allocs.size();
    int32_t* sums = dalloc<int32_t>(p, (size_t)nblk);
    IFGF_LAUNCH(k_scan_reduce, (unsigned)nblk, kScanThreads, 0, p.stream, in, n, sums);
    exclusive_scan_i32(p, sums, sums, nblk);
    IFGF_LAUNCH(k_scan_down, (unsigned)nblk, kScanThreads, 0, p.stream, in, n, (const int32_t*)sums, out);
    dfree_from(p, mark);
}

void radix_sort_pairs(Plan& p, uint64_t* keys, int32_t* vals, int64_t n, int end_bit) {
    if (n <= 1) return;
    const int nblk = (int)((n + kRsTile - 1) / kRsTile);
    const size_t mark = p.allocs.size();
    uint64_t* k2 = dalloc<uint64_t>(p, (size_t)n);
    int32_t* v2 = dalloc<int32_t>(p, (size_t)n);
    int32_t* hist = dalloc<int32_t>(p, (size_t)256 * nblk);
    uint64_t *ka = keys, *kb = k2;
    int32_t *va = vals, *vb = v2;
    int passes = 0;
    for (int shift = 0; shift < end_bit; shift += 8, ++passes) {
        IFGF_LAUNCH(k_rs_hist, nblk, kRsThreads, 0, p.stream, ka, n, shift, hist, nblk);
        exclusive_scan_i32(p, hist, hist, (int64_t)256 * nblk);
        IFGF_LAUNCH(k_rs_scatter, nblk, kRsThreads, 0, p.stream, ka, va, kb, vb, n, shift, hist, nblk);
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        IFGF_CUDA(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, p.stream));
        IFGF_CUDA(cudaMemcpyAsync(vals, va, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, p.stream));
    }
    dfree_from(p, mark);
}

}  // namespace ifgf
