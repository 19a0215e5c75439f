// Morton point order without device allocation.
//
// Some callers cannot allocate device memory at the moment they need the point order: their
// device memory is entirely owned by another allocator (a framework's caching pool or an arena
// reserved up front), or they run in loops where cudaMalloc/cudaFree are not acceptable because
// they can synchronise the device or fail under memory pressure.  This file gives them the
// root cube, the level-21 Morton keys and the stable key sort of the plan builder in a variant
// whose scratch is a fixed static device array instead of per-call allocations.  The caller
// passes the points and both outputs; the scratch holds the second half of the sort's
// ping-pong buffers, the per-tile digit histograms and the bounding-box partials.
#include <cmath>
#include <mutex>
#include <string>

#include "ifgf_internal.cuh"

namespace ifgf {
namespace {

constexpr int64_t kMaxPoints = IFGF_NOALLOC_MAX_POINTS;
constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;
constexpr int kMaxTiles = (int)(kMaxPoints / kTile);
constexpr int kBboxBlocks = 256;
constexpr int kScanThreads = 1024;

struct Scratch {
    double bbox[kBboxBlocks * 7];
    uint64_t keys[kMaxPoints];
    int32_t vals[kMaxPoints];
    int32_t hist[256 * kMaxTiles];
};

// The scratch: every device that loads the library holds it until the process exits.  Every
// call reuses it, so calls that overlap on the GPU (two streams, or two host threads) race.
static __device__ __align__(256) Scratch g_scratch;

std::mutex g_mu;
void* g_addr[128] = {nullptr};

__global__ void na_bbox(const double* __restrict__ X, int64_t N, Scratch* sc) {
    __shared__ double smin[3][kThreads], smax[3][kThreads];
    __shared__ int sbad[kThreads];
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        for (int c = 0; c < 3; ++c) {
            const double v = X[(int64_t)c * N + i];
            if (!isfinite(v)) bad = 1;
            mn[c] = fmin(mn[c], v);
            mx[c] = fmax(mx[c], v);
        }
    }
    for (int c = 0; c < 3; ++c) {
        smin[c][threadIdx.x] = mn[c];
        smax[c][threadIdx.x] = mx[c];
    }
    sbad[threadIdx.x] = bad;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            for (int c = 0; c < 3; ++c) {
                smin[c][threadIdx.x] = fmin(smin[c][threadIdx.x], smin[c][threadIdx.x + o]);
                smax[c][threadIdx.x] = fmax(smax[c][threadIdx.x], smax[c][threadIdx.x + o]);
            }
            sbad[threadIdx.x] |= sbad[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int c = 0; c < 3; ++c) {
            sc->bbox[blockIdx.x * 7 + c] = smin[c][0];
            sc->bbox[blockIdx.x * 7 + 3 + c] = smax[c][0];
        }
        sc->bbox[blockIdx.x * 7 + 6] = sbad[0];
    }
}

__global__ void na_keys(const double* __restrict__ X, int64_t N, double a0, double a1, double a2, double H1,
                        uint64_t* __restrict__ keys, int32_t* __restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double a[3] = {a0, a1, a2};
    uint32_t k[3];
    for (int c = 0; c < 3; ++c) {
        const double u = __ddiv_rn(__dsub_rn(X[(int64_t)c * N + i], a[c]), H1);
        double f = floor(__dmul_rn(u, 1048576.0));
        f = fmin(fmax(f, 0.0), 1048575.0);
        k[c] = (uint32_t)f;
    }
    keys[i] = morton3(k[0], k[1], k[2]);
    vals[i] = (int32_t)i;
}

__global__ void na_hist(const uint64_t* __restrict__ keys, int64_t n, int shift, int32_t* __restrict__ hist, int nblk) {
    __shared__ int32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int i = 0; i < kItems; ++i) {
        const int64_t idx = base + (int64_t)i * kThreads + threadIdx.x;
        if (idx < n) atomicAdd(&cnt[(keys[idx] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive scan of the (at most 65,536) histogram entries in one block.
__global__ void na_scan(int32_t* __restrict__ h, int n) {
    __shared__ int32_t warp_sums[32];
    const int per = (n + kScanThreads - 1) / kScanThreads;
    const int b = threadIdx.x * per;
    int32_t s = 0;
    for (int i = 0; i < per; ++i)
        if (b + i < n) s += h[b + i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t x = s;
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int32_t w = warp_sums[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;
    }
    __syncthreads();
    int32_t pre = (warp ? warp_sums[warp - 1] : 0) + x - s;
    for (int i = 0; i < per; ++i)
        if (b + i < n) {
            const int32_t v = h[b + i];
            h[b + i] = pre;
            pre += v;
        }
}

// Stable scatter: chunks of 256 consecutive items, ranked by warp then lane inside a chunk.
__global__ void na_scatter(const uint64_t* __restrict__ kin, const int32_t* __restrict__ vin,
                           uint64_t* __restrict__ kout, int32_t* __restrict__ vout, int64_t n, int shift,
                           const int32_t* __restrict__ offs, int nblk) {
    constexpr int W = kThreads / 32;
    __shared__ int32_t base[256];
    __shared__ int32_t wcnt[W][256];
    __shared__ int32_t wpre[W][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    base[threadIdx.x] = offs[(int64_t)threadIdx.x * nblk + blockIdx.x];
    for (int w = 0; w < W; ++w) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t tile = (int64_t)blockIdx.x * kTile;
    const unsigned lt = (1u << lane) - 1u;
    for (int c = 0; c < kItems; ++c) {
        const int64_t idx = tile + (int64_t)c * kThreads + threadIdx.x;
        const bool valid = idx < n;
        const uint64_t key = valid ? kin[idx] : 0;
        const int32_t val = valid ? vin[idx] : 0;
        const int digit = valid ? (int)((key >> shift) & 255u) : 256;
        const unsigned peers = __match_any_sync(0xffffffffu, digit);
        const int rank = __popc(peers & lt);
        if (valid && lane == __ffs(peers) - 1) wcnt[warp][digit] = __popc(peers);
        __syncthreads();
        int32_t s = 0;
        for (int w = 0; w < W; ++w) {
            wpre[w][threadIdx.x] = s;
            s += wcnt[w][threadIdx.x];
        }
        __syncthreads();
        if (valid) {
            const int64_t pos = (int64_t)base[digit] + wpre[warp][digit] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        base[threadIdx.x] += s;
        for (int w = 0; w < W; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
    }
}

}  // namespace
}  // namespace ifgf

using namespace ifgf;

extern "C" ifgf_status ifgf_morton_order_noalloc(const double* points, int64_t N, int32_t* perm, uint64_t* keys,
                                                 void* stream) {
    if (!points || !perm || !keys) {
        set_last_error("points, perm and keys must be device pointers");
        return IFGF_ERR_INVALID_ARG;
    }
    if (N < 2 || N > kMaxPoints) {
        set_last_error("N must be in [2, " + std::to_string(kMaxPoints) + "] for the allocation-free sort");
        return IFGF_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // Launch errors are read back through the runtime's last-error state at the end, so an error
    // left pending by the caller's earlier work is cleared here rather than reported as ours.
    cudaGetLastError();
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
        cudaGetLastError();
        set_last_error("cudaGetDevice failed");
        return IFGF_ERR_CUDA;
    }
    Scratch* sc = nullptr;
    {
        // One-time set-up per device, with that device current: the host-side name of the
        // scratch array is not its device address, so ask the runtime for it.
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void* ptr = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
            if (e != cudaSuccess || !ptr) {
                cudaGetLastError();
                set_last_error(std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
                return IFGF_ERR_CUDA;
            }
            g_addr[dev] = ptr;
        }
        sc = static_cast<Scratch*>(g_addr[dev]);
    }
    const int nb = (int)std::min<int64_t>(kBboxBlocks, (N + kThreads - 1) / kThreads);
    na_bbox<<<nb, kThreads, 0, s>>>(points, N, sc);
    g_launches.fetch_add(1);
    double part[kBboxBlocks * 7];
    cudaError_t e = cudaMemcpyAsync(part, sc->bbox, sizeof(double) * 7 * nb, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_last_error(std::string("bounding box: ") + cudaGetErrorString(e));
        return IFGF_ERR_CUDA;
    }
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = 0; b < nb; ++b) {
        if (part[b * 7 + 6] != 0.0) {
            set_last_error("non-finite coordinate");
            return IFGF_ERR_INVALID_ARG;
        }
        for (int c = 0; c < 3; ++c) {
            mn[c] = std::min(mn[c], part[b * 7 + c]);
            mx[c] = std::max(mx[c], part[b * 7 + 3 + c]);
        }
    }
    double ext = 0.0;
    for (int c = 0; c < 3; ++c) ext = std::max(ext, mx[c] - mn[c]);
    if (!(ext > 0.0)) {
        set_last_error("all points coincide");
        return IFGF_ERR_INVALID_ARG;
    }
    const double H1 = ext * (1.0 + std::ldexp(1.0, -20));
    double a[3];
    for (int c = 0; c < 3; ++c) a[c] = 0.5 * (mn[c] + mx[c]) - 0.5 * H1;
    na_keys<<<(unsigned)((N + kThreads - 1) / kThreads), kThreads, 0, s>>>(points, N, a[0], a[1], a[2], H1, keys, perm);
    const int nblk = (int)((N + kTile - 1) / kTile);
    uint64_t *ka = keys, *kb = sc->keys;
    int32_t *va = perm, *vb = sc->vals;
    for (int shift = 0; shift < 3 * (kKeyLevel - 1); shift += 8) {
        na_hist<<<nblk, kThreads, 0, s>>>(ka, N, shift, sc->hist, nblk);
        na_scan<<<1, kScanThreads, 0, s>>>(sc->hist, 256 * nblk);
        na_scatter<<<nblk, kThreads, 0, s>>>(ka, va, kb, vb, N, shift, sc->hist, nblk);
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    g_launches.fetch_add(1 + 3 * 8);
    // 8 passes: the sorted keys and permutation are back in the caller's buffers.
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(std::string("launch: ") + cudaGetErrorString(e));
        return IFGF_ERR_CUDA;
    }
    return IFGF_OK;
}
