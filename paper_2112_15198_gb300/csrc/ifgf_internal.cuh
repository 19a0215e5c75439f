// Internal data structures and device helpers of the GB300 IFGF library.
//
// Geometry conventions (shared by the plan builder and the apply kernels):
//  - Root cube B^1 (Sec. 2): a = centre(bbox) - H1/2, H1 = largest extent * (1 + 2^-20).
//  - Level-d boxes have side H_d = H1 / 2^(d-1); the grid unit is u = H_D / 2, so every box
//    centre lies at a + u * (odd integer vector) and offsets between centres are exact small
//    integers in grid units.
//  - Each sorted point keeps its FP32 offset from its leaf centre in grid units, so the
//    offset of a point from any box centre is (exact integer) + (FP32 leaf offset).
//  - Cone segments of level d: uniform grids over s = h_d / r in [0, eta], theta in [0, pi],
//    phi in [0, 2 pi), h_d = sqrt(3)/2 H_d, eta = sqrt(3)/3 (Sec. 2, box-centred cones).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "ifgf.h"

namespace ifgf {

constexpr int kKeyLevel = 21;  // finest level of the sort key: 20 bits per axis
constexpr int kMaxLevel = 21;
constexpr int kMaxNbr = 27;    // |N B| <= 27
constexpr int kMaxCous = 189;  // |M B| <= 189 (Sec. 3.3)
constexpr int kMaxOrder = 8;

extern std::atomic<int64_t> g_launches;
// Fault injection for tests (ifgf_debug_fail_allocation): when positive, the device allocation
// that brings it to zero fails as if the device were out of memory.
extern std::atomic<int64_t> g_fail_alloc_in;

// Per-level cone grid: counts, exact-classification tables and interpolation-node tables.
struct LevelGrid {
    int ns, nt, np, C;         // cone counts per direction, C = ns*nt*np
    float hg;                  // circumradius h_d in grid units
    float s_scale, t_scale, p_scale;  // ns/eta, nt/pi, np/(2 pi): candidate bins
    float s2w, t2w, p2w;       // 2/ds, 2/dt, 2/dp: local coordinate scales
    float ms, tA, tB, mp;      // edge margins of the classification's fast path (bin widths)
    double ds64, dt64, dp64;   // interval widths
    double h64;                // circumradius in physical units
    const float* R2;           // [ns]  (h/(i ds))^2, grid units
    const float* C2;           // [nt]  cos^2(i pi/nt)
    const int* cpos;           // [nt]  cos(i pi/nt) >= 0
    const float* cph;          // [np]  cos(2 pi j/np)
    const float* sph;          // [np]  sin(2 pi j/np)
    const float* rho;          // [ns*Ps] node radius h/s in grid units
    const float* ctn;          // [nt*Pt] cos of theta nodes
    const float* stn;          // [nt*Pt] sin of theta nodes
    const float* cpn;          // [np*Pp] cos of phi nodes
    const float* spn;          // [np*Pp] sin of phi nodes
    const float* snode;        // [ns*Ps] s of nodes (FP32)
    const double* snode64;     // [ns*Ps] s of nodes
    const double* tnode64;     // [nt*Pt] theta of nodes
    const double* pnode64;     // [np*Pp] phi of nodes
};

// ---- bounds checks (builds with -DIFGF_CHECKS) ------------------------------------------
// In a checked build the cone lookups test the box and the cone they return, the kernels test
// the list and table indices they derive before using them, and the plan's index lists are
// validated once they are built; a failed test records IFGF_ERR_INTERNAL in the plan's status
// word and the access is skipped.  Other builds compile the tests away.
#ifdef IFGF_CHECKS
constexpr bool kChecks = true;
#else
constexpr bool kChecks = false;
#endif
__device__ __forceinline__ bool in_bounds(int64_t i, int64_t n, int* st) {
    if (!kChecks || (i >= 0 && i < n)) return true;
    if (st) atomicCAS(st, 0, (int)IFGF_ERR_INTERNAL);
    return false;
}

// Cone lookup (box, gamma) -> index of the relevant cone, or -1. Dense levels keep the table
// slot[box * C + gamma] (one load); levels whose table would be too large keep only the
// cone list, sorted by (box, gamma), with the first cone of every box (binary search).
// Sparse levels may also keep rows[box * nrow + w] = the first cone of the box whose gamma is at
// least w * np (w = is * nt + it, one row per (s, theta) bin, the next box's first row closing
// the last), so that a search covers the few relevant cones of one phi-row instead of the box.
struct ConeMap {
    const int32_t* slot;  // dense table, or nullptr
    int32_t C;
    const int32_t* bcs;   // [n+1] first cone of every box (sparse levels)
    const int32_t* gam;   // [nc] cone index gamma of every cone (sparse levels)
    const int32_t* rows;  // [n * nrow + 1] row starts (sparse levels), or nullptr
    int32_t nrow, np;     // rows per box (ns * nt) and the phi count
    // A rank of a distributed apply holds some of the level's cones: g2l maps a cone's index in the
    // level's list to its block in the rank's buffer, -1 when the rank does not hold it.
    const int32_t* g2l = nullptr;
    int32_t nbox = 0;      // boxes of the level (checked builds)
    int64_t nc = 0;        // relevant cones of the level (checked builds)
    int* status = nullptr; // status word for failed checks
    __device__ __forceinline__ int find(int box, int gamma) const {
        const int s = find_global(box, gamma);
        return (g2l && s >= 0) ? __ldg(&g2l[s]) : s;
    }
    __device__ __forceinline__ int find_global(int box, int gamma) const {
        if (!in_bounds(box, nbox, status) || !in_bounds(gamma, C, status)) return -1;
        if constexpr (kChecks) {
            const int s = find_unchecked(box, gamma);
            return in_bounds(s + 1, nc + 1, status) ? s : -1;
        }
        return find_unchecked(box, gamma);
    }
    __device__ __forceinline__ int find_unchecked(int box, int gamma) const {
        if (slot) return __ldg(&slot[(int64_t)box * C + gamma]);
        int lo, end;
        if (rows) {
            const int64_t w = (int64_t)box * nrow + gamma / np;
            lo = __ldg(&rows[w]);
            end = __ldg(&rows[w + 1]);
        } else {
            lo = __ldg(&bcs[box]);
            end = __ldg(&bcs[box + 1]);
        }
        int hi = end;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(&gam[mid]) < gamma) lo = mid + 1;
            else hi = mid;
        }
        return (lo < end && __ldg(&gam[lo]) == gamma) ? lo : -1;
    }
};

struct Level {
    int32_t n = 0;                 // relevant boxes R_B^d
    uint64_t* key = nullptr;       // [n] Morton keys, ascending
    int32_t* start = nullptr;      // [n+1] sorted point ranges
    int32_t* parent = nullptr;     // [n] box index at level d-1
    int32_t* cstart = nullptr;     // [n+1] first child at level d+1
    int4* k = nullptr;             // [n] integer box coordinates
    int32_t* pbox = nullptr;       // [N] box of every sorted point
    int32_t* nnb = nullptr;        // [n]
    int32_t* nb = nullptr;         // [n*27] ascending
    int32_t* ncs = nullptr;        // [n]
    int32_t* cs = nullptr;         // [n*189] ascending
    LevelGrid g{};
    int64_t nc = 0;                // relevant cones R_C^d
    int32_t* slot = nullptr;       // [n*C] cone index or -1 (dense levels; nullptr when sparse)
    int32_t* bcs = nullptr;        // [n+1] first cone of every box (sparse levels)
    int32_t* rows = nullptr;       // [n * ns * nt + 1] row starts of the cone list (sparse levels)
    ConeMap cmap(int* st = nullptr) const {
        return ConeMap{slot, g.C, bcs, cone_gam, rows, g.ns * g.nt, g.np, nullptr, n, nc, st};
    }
    int32_t* cone_box = nullptr;   // [nc]
    int32_t* cone_gam = nullptr;   // [nc]
    float* phtab = nullptr;        // [28] (kappa H_d sqrt(m)) mod 2 pi, m = |k_A - k_B|^2
    std::vector<int32_t> host_grid;  // (ns, nt, np)
    // Node tables of this level's relevant cones seen from the child grid (level d+1): the
    // child cone, local coordinates and G ratio of node n of cone index gamma in the child at
    // octant o depend only on (gamma, o, n), not on the box, so they are computed once per
    // distinct gamma and shared by every box (row g = distinct gamma, entry (g*8 + o)*P + n).
    int32_t n_gam = 0;             // rows (0: no tables, the kernels compute the geometry)
    int32_t* gam_list = nullptr;   // [n_gam] gamma of each row
    int32_t* cone_gidx = nullptr;  // [nc] row of each relevant cone
    // Entries of a row are stored in the order of their child cone (stable in the node index).
    float4* tab_t = nullptr;       // (t_s, t_theta, t_phi, node index in the parent cone)
    float2* tab_r = nullptr;       // G(x, x_k) / G(x, x_j)
    int32_t* tab_k = nullptr;      // [n_gam*8] distinct child cones of the row (K <= kTabList)
    int32_t* tab_list = nullptr;   // [n_gam*8][kTabList] their child cone indices
    int16_t* tab_perm = nullptr;   // [n_gam*8*P] node index of each sorted entry
    // Segments: runs of <= kSegLen sorted entries with one child cone, packed as
    // first entry | length << 8 | list position << 16.
    int32_t* tab_nseg = nullptr;   // [n_gam*8]
    int32_t* tab_seg = nullptr;    // [n_gam*8*P]
    int32_t* tab_run = nullptr;    // [n_gam*8][kTabList+1] first segment of each child cone, then nseg
    // Levels without node tables (mixed precision, orders (3,5,5)): relevant cones grouped by
    // cone index. gorder lists them by (block of boxes, gamma, box); gchunk[c]..gchunk[c+1] is a
    // chunk of at most kChunkBoxes cones of one gamma, whose node classification seen from the
    // eight child octants is computed once for the whole chunk (activation of the next level).
    int64_t n_gchunk = 0;
    int32_t* gorder = nullptr;     // [nc]
    int32_t* gchunk = nullptr;     // [n_gchunk+1]
    // Propagation into this level (as the parent level): cone boundaries of its slices.
    std::vector<int64_t> pslice;
    // Kernel choices of the propagation from this level into level d-1 where level d-1 has node
    // tables (-1: the built-in choice), set by ifgf_plan_set_knob or the autotuner:
    //   knob_many (mixed, kMmaMinRhs densities or more): 0 mma.sync tiles, 1 tcgen05 + TMEM;
    //   knob_few (mixed, fewer densities): 0 the node-table warp kernel, 1 the per-cone kernel.
    int8_t knob_many = -1;
    int8_t knob_few = -1;
};
constexpr int kTabList = 80;   // distinct child cones a row may list: at most one per node (75)
constexpr int kSlotCache = 32; // child-cone slots a warp of the node-table propagation keeps in shared memory
constexpr int kSegLen = 8;  // nodes of one child cone evaluated by one thread
constexpr int kChunkBoxes = 8;  // cones (of one gamma, different boxes) per chunk

struct Plan {
    int64_t N = 0;
    int D = 0;
    double kappa = 0;
    int Ps = 3, Pt = 5, Pp = 5, P = 75;
    int cstride = 76;              // complex entries per cone and density vector
    int precision = IFGF_PREC_MIXED;
    int max_nrhs = 1;
    int rhs_block = 1;             // densities per level sweep (coefficient buffers hold this many)
    int knob_block = -1;           // densities per block of the many-density kernels (8, 16, 32; -1 by nrhs)
    double a[3] = {0, 0, 0};
    double H1 = 0, u = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    int32_t* perm = nullptr;       // [N] sorted -> caller index
    uint64_t* key = nullptr;       // [N] sorted keys
    double* Xs = nullptr;          // [3][N] sorted coordinates
    float4* off = nullptr;         // [N] leaf offsets (grid units), w unused
    Level L[kMaxLevel + 1];
    float* Wf = nullptr;           // analysis matrices Ws | Wt | Wp (FP32)
    double* Wd = nullptr;          // same in FP64
    void* a_s = nullptr;           // sorted densities [nrhs][N]
    void* I_s = nullptr;           // sorted output [nrhs][N]
    // Coefficient arena of arena_cones cone blocks (each rhs_block densities x cstride). Level d
    // lives at the start of the arena when D - d is even and at its end otherwise, so the
    // propagation into level d-1 writes at the other end while it reads level d; done in slices
    // of parent cones (Level::pslice), the reads still ahead never meet the writes, and the
    // arena needs about max_d n_c(d) (1 + 1/slices) cones instead of two full levels.
    char* arena = nullptr;
    int64_t arena_cones = 0;
    int* d_status = nullptr;       // sticky device status
    std::vector<void*> allocs;
};

// ---- errors -------------------------------------------------------------------------
struct Error {
    ifgf_status status;
    std::string what;
};
void set_last_error(const std::string& s);
[[noreturn]] void fail(ifgf_status s, const std::string& what);
void cuda_check(cudaError_t e, const char* what);
#define IFGF_CUDA(expr) ::ifgf::cuda_check((expr), #expr)

// The library's stream-ordered memory pool of a device (created on first use; freed memory
// stays cached up to a quarter of the device memory).
cudaMemPool_t device_pool(int device);
// Bytes the pool of a device holds but does not use (available to the next allocations).
size_t pool_cached_bytes(int device);

template <class T>
T* dalloc(Plan& p, size_t count) {
    void* ptr = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    if (g_fail_alloc_in.load(std::memory_order_relaxed) > 0 && g_fail_alloc_in.fetch_sub(1) == 1)
        fail(IFGF_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed (injected)");
    cudaMemPool_t pool = device_pool(p.device);
    cudaError_t e = cudaMallocFromPoolAsync(&ptr, bytes, pool, p.stream);
    if (e != cudaSuccess) {  // return the pool's cached memory to the device and try once more
        cudaGetLastError();
        cudaStreamSynchronize(p.stream);
        cudaMemPoolTrimTo(pool, 0);
        e = cudaMallocFromPoolAsync(&ptr, bytes, pool, p.stream);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(IFGF_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    p.allocs.push_back(ptr);
    return static_cast<T*>(ptr);
}

// Stream-ordered release of every allocation made after `mark` (temporaries of one stage).
inline void dfree_from(Plan& p, size_t mark) {
    while (p.allocs.size() > mark) {
        cudaFreeAsync(p.allocs.back(), p.stream);
        p.allocs.pop_back();
    }
}

// Stream-ordered release of one allocation.
inline void dfree_ptr(Plan& p, void* ptr) {
    for (size_t i = p.allocs.size(); i-- > 0;)
        if (p.allocs[i] == ptr) {
            cudaFreeAsync(ptr, p.stream);
            p.allocs.erase(p.allocs.begin() + (std::ptrdiff_t)i);
            return;
        }
}

inline unsigned grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    return (unsigned)b;
}

#define IFGF_LAUNCH(kernel, grid, block, smem, stream, ...)                     \
    do {                                                                       \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);            \
        ::ifgf::g_launches.fetch_add(1, std::memory_order_relaxed);            \
        ::ifgf::cuda_check(cudaGetLastError(), #kernel);                       \
    } while (0)

// ---- live kernel timing (opt-in; CUDA events around each hot kernel) -------------------
// TK_PROP: propagation from node tables; TK_PROP_GEN: propagation that computes the node geometry.
enum TimingKind {
    TK_PERM = 0, TK_NEAR = 1, TK_LEAF = 2, TK_PROP = 3, TK_INTERP = 4, TK_PLAN = 5, TK_PROP_GEN = 6, TK_COUNT = 7
};
static_assert(TK_COUNT == IFGF_TIMING_KINDS, "timing kinds of the header");
struct TimedScope {
    TimedScope(int kind, cudaStream_t s);
    ~TimedScope();
    int kind;
    int level = -1;
    cudaStream_t stream;
    cudaEvent_t start = nullptr;
};
// Tags the timed scopes of the calling thread with an octree level while it lives (the level
// sweeps set it, so that the autotuner can read kernel times per level).
struct TimingLevel {
    explicit TimingLevel(int d);
    ~TimingLevel();
    int prev;
};
// Kernel times collected since the last collection, in total per kind and per (kind, level);
// clears them (ifgf_timing_collect reports the totals).
void timing_collect_levels(double* ms, int64_t* launches, double (*by_level)[kMaxLevel + 1]);
// Switches the kernel timing on or off and returns the previous setting.
bool timing_switch(bool on);

// ---- autotuner cache (tune.cu) ---------------------------------------------------------
std::map<std::string, std::string> tune_cache_read(const std::string& path);
void tune_cache_write(const std::string& path, const std::map<std::string, std::string>& add);
std::string tune_gpu_key(int device);
std::string tune_rhs_bucket(int nrhs);
int tune_log2(int64_t n);

// ---- scan / sort utilities (util.cu) --------------------------------------------------
// Exclusive prefix sum of n int32 values into out (may alias in); returns nothing; the
// total is out[n-1] + in[n-1] (callers read it back when needed).
void exclusive_scan_i32(Plan& p, const int32_t* in, int32_t* out, int64_t n);
// Stable LSD radix sort of (key, val) pairs over key bits [0, end_bit); result in keys/vals.
void radix_sort_pairs(Plan& p, uint64_t* keys, int32_t* vals, int64_t n, int end_bit);

// ---- stages -----------------------------------------------------------------------------
void build_plan(Plan& p, const double* points, const ifgf_options& opt, int levels);
// Coefficient arena layout: slices per level and arena size for at most `budget` bytes per
// density (cone blocks of cstride complex values); returns the arena size in cones, 0 if the
// levels cannot be laid out in the budget. slices = 0: one slice if it fits, else 64.
int64_t layout_arena(Plan& p, size_t budget_per_rhs, int slices);
// Level d's first cone block in the arena for blocks of nb densities.
inline char* level_coef(const Plan& p, int d, int nb) {
    const size_t csz = p.precision == IFGF_PREC_MIXED ? 8 : 16;
    const size_t cone = (size_t)nb * p.cstride * csz;
    return ((p.D - d) % 2 == 0) ? p.arena : p.arena + (size_t)(p.arena_cones - p.L[d].nc) * cone;
}
void destroy_plan(Plan& p);
// Steps of one rank of a distributed apply (apply.cu; mixed precision, at most 3 value sets):
// near field of the leaf boxes [b0, b1) and LevelDEvaluations of the level-D cones [c_lo, c_hi)
// (whose boxes are [lb0, lb1)), written at coefD; Interpolation(d) of the targets [i0, i1); and
// Propagation(d) of the level-(d-1) cones [lo, hi), parent cone lo written at cp.  Sorted
// densities as and results Is are [nrhs][N]; cone lookups go through cm (with the rank's map).
void shard_near_leaf(Plan& p, const float2* as, int nrhs, float2* Is, int64_t b0, int64_t b1, int64_t lb0, int64_t lb1,
                     int64_t c_lo, int64_t c_hi, float2* coefD, cudaStream_t s);
void shard_interp(Plan& p, int d, int nrhs, float2* Is, const ConeMap& cm, const float2* coef, int64_t i0, int64_t i1,
                  cudaStream_t s);
void shard_prop(Plan& p, int d, int nrhs, int64_t lo, int64_t hi, const ConeMap& cm, const float2* cc, float2* cp,
                cudaStream_t s);
// Propagation of the parent cones [lo, lo + n) of level d-1 (node tables) for nrhs densities on
// the tcgen05 tensor cores (prop_tc.cu); child coefficients cc, parent cone lo written at cp.
void launch_prop_tc_tab(const Plan& p, int d, int nrhs, int64_t lo, int64_t n, const float2* cc, float2* cp,
                        cudaStream_t s);
// Caller order <-> sorted order of [nrhs][N] complex vectors of the plan's precision.
void permute_points(Plan& p, const void* in, int nrhs, void* out, bool to_sorted, cudaStream_t s);
void apply_plan(Plan& p, const void* dens, int nrhs, void* out, cudaStream_t s, bool near, int64_t mask);
// Green tensor c (alpha delta_ij / r + r_i r_j / r^3): the Stokeslet (c = 1/(8 pi mu), alpha = 1)
// or Kelvin's solution of linear elasticity (c = 1/(16 pi mu (1 - nu)), alpha = 3 - 4 nu).
struct TensorKernel {
    double c = 0.039788735772973836;  // 1/(8 pi)
    double alpha = 1.0;
};
// forces and vel: [nf][3][N] float (mixed plans) or double (FP64 plans).
void apply_plan_stokes(Plan& p, const void* forces, int nf, void* vel, const TensorKernel& tk, cudaStream_t s,
                       bool near, int64_t mask);

// =========================================================================================
// Device helpers
// =========================================================================================

// r^2 = (vx*vx + vy*vy) + vz*vz, each operation correctly rounded (no contraction).
__device__ __forceinline__ float rn_r2(float vx, float vy, float vz) {
    return __fadd_rn(__fadd_rn(__fmul_rn(vx, vx), __fmul_rn(vy, vy)), __fmul_rn(vz, vz));
}

// Exact cone classification of an FP32 grid-unit offset v (r2 = rn_r2(v)).  Each bin index
// is the number of edges the point lies on or beyond, decided by correctly rounded FP32
// products/sums and comparisons; (is, it, ip) enter as candidate bins from approximate
// spherical coordinates and leave as the exact counts, reached by stepping across edges (the
// edge predicates are monotone in the edge index).
//   s:     edge i (1 <= i < ns) passed iff r2 <= R2[i]                 (s >= i ds)
//   theta: edge i (1 <= i < nt) passed iff vz <= cos(theta_i) r, in squared form
//   phi:   edge j (1 <= j < np) passed iff phi >= phi_j, from the half plane left of edge j
//          and the lower half plane H; 0 on the z axis.
__device__ __forceinline__ void classify_exact(const LevelGrid& g, float vx, float vy, float vz, float r2, int& is,
                                               int& it, int& ip) {
    is = min(max(is, 0), g.ns - 1);
    while (is > 0 && !(r2 <= __ldg(&g.R2[is]))) --is;
    while (is + 1 < g.ns && (r2 <= __ldg(&g.R2[is + 1]))) ++is;

    const float z2 = __fmul_rn(vz, vz);
    const bool zneg = vz < 0.0f;
    it = min(max(it, 0), g.nt - 1);
    auto Q = [&](int i) -> bool {
        const float c2r = __fmul_rn(__ldg(&g.C2[i]), r2);
        return __ldg(&g.cpos[i]) ? (zneg || z2 <= c2r) : (zneg && z2 >= c2r);
    };
    while (it > 0 && !Q(it)) --it;
    while (it + 1 < g.nt && Q(it + 1)) ++it;

    if (vx == 0.0f && vy == 0.0f) {
        ip = 0;
        return;
    }
    const bool H = (vy < 0.0f) || (vy == 0.0f && vx < 0.0f);
    auto GE = [&](int j) -> bool {
        const bool Lj = __fsub_rn(__fmul_rn(__ldg(&g.cph[j]), vy), __fmul_rn(__ldg(&g.sph[j]), vx)) >= 0.0f;
        const int j2 = 2 * j;
        return j2 < g.np ? (Lj || H) : (j2 == g.np ? H : (Lj && H));
    };
    ip = min(max(ip, 0), g.np - 1);
    while (ip > 0 && !GE(ip)) --ip;
    while (ip + 1 < g.np && GE(ip + 1)) ++ip;
}

// Fast path of the exact classification.  (fs, ft, fp) are the approximate bin coordinates
// s ns/eta, theta nt/pi, phi np/(2 pi) of the offset v, (is, it, ip) their integer parts.  The
// approximate coordinates differ from the true ones by a few 1e-7 (relative for s, radians for the
// angles), and each exact edge test decides as the true geometry does unless the point lies within
// a few 1e-7 of the edge (for theta, within about 1.5e-7 / tan(theta_i) of edge i, which grows
// near the poles).  Where every coordinate lies inside its candidate bin by more than the level's
// margins (about eight times those bounds), the candidate bins are the exact ones; the polar theta
// bins, points on the axis and points beyond the grid take the exact tests.
__device__ __forceinline__ bool bins_certain(const LevelGrid& g, float vx, float vy, float fs, float ft, float fp,
                                             int is, int it, int ip) {
    if ((unsigned)is >= (unsigned)g.ns || (unsigned)ip >= (unsigned)g.np) return false;
    const int k = min(it, g.nt - 1 - it);  // bins between this one and the nearest polar bin
    if (k <= 0 || (vx == 0.0f && vy == 0.0f)) return false;
    const float es = fs - (float)is, et = ft - (float)it, ep = fp - (float)ip;
    const float ms = g.ms * (float)(is + 1);
    const float mt = g.tA + __fdividef(g.tB, (float)k);
    const bool s_ok = (is == 0 || es > ms) && (is == g.ns - 1 || es < 1.0f - ms);
    return s_ok && et > mt && et < 1.0f - mt && ep > g.mp && ep < 1.0f - g.mp;
}

// atan2 for evaluation coordinates: octant symmetry reduces the argument to t in [0, 1], where
// atan(t) = t P(t^2) with an odd polynomial of degree 15 fitted to atan by iteratively
// reweighted least squares on Chebyshev nodes (near-minimax); max error 1.4e-7 rad in FP32.
__device__ __forceinline__ float fast_atan2(float y, float x) {
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    const float t = mx > 0.0f ? __fdividef(mn, mx) : 0.0f;
    const float u = t * t;
    float p = -0.004054564982652664f;
    p = fmaf(p, u, 0.021862955763936043f);
    p = fmaf(p, u, -0.055912334471940994f);
    p = fmaf(p, u, 0.0964219868183136f);
    p = fmaf(p, u, -0.1390863060951233f);
    p = fmaf(p, u, 0.19946566224098206f);
    p = fmaf(p, u, -0.33329859375953674f);
    p = fmaf(p, u, 0.9999993443489075f);
    float r = p * t;
    if (ay > ax) r = 1.57079632679489662f - r;
    if (x < 0.0f) r = 3.14159265358979324f - r;
    return copysignf(r, y);
}

// Cone of a grid-unit offset v (exact bins) and its local coordinates (t_s, t_theta, t_phi)
// in [-1, 1] (slightly beyond near edges), from approximate spherical coordinates.
struct ConeLocal {
    int is, it, ip;
    float ts, tt, tp;
    float r;  // |v| (approximate)
    __device__ __forceinline__ int gamma(const LevelGrid& g) const { return (is * g.nt + it) * g.np + ip; }
};

__device__ __forceinline__ ConeLocal locate_f32(const LevelGrid& g, float vx, float vy, float vz) {
    const float r2 = rn_r2(vx, vy, vz);
    const float rinv = rsqrtf(r2);
    const float s = g.hg * rinv;
    const float rxy2 = fmaf(vx, vx, vy * vy);
    const float rxy = rxy2 > 0.0f ? rxy2 * rsqrtf(rxy2) : 0.0f;
    const float th = fast_atan2(rxy, vz);
    float ph = fast_atan2(vy, vx);
    if (ph < 0.0f) ph += 6.28318530717958647692f;
    ConeLocal o;
    const float fs = s * g.s_scale, ft = th * g.t_scale, fp = ph * g.p_scale;
    o.is = (int)fs;
    o.it = (int)ft;
    o.ip = (int)fp;
    if (!bins_certain(g, vx, vy, fs, ft, fp, o.is, o.it, o.ip)) classify_exact(g, vx, vy, vz, r2, o.is, o.it, o.ip);
    o.r = r2 * rinv;
    o.ts = fmaf(s, g.s2w, -(float)(2 * o.is + 1));
    o.tt = fmaf(th, g.t2w, -(float)(2 * o.it + 1));
    float tp = fmaf(ph, g.p2w, -(float)(2 * o.ip + 1));
    const float span = (float)(2 * g.np);  // 2 pi in local units
    if (tp > (float)g.np) tp -= span;
    if (tp < -(float)g.np) tp += span;
    o.tp = tp;
    return o;
}

// Classification only (plan-time activation and the FP64 path).
__device__ __forceinline__ int classify_f32(const LevelGrid& g, float vx, float vy, float vz) {
    const float r2 = rn_r2(vx, vy, vz);
    const float s = g.hg * rsqrtf(r2);
    const float rxy2 = fmaf(vx, vx, vy * vy);
    const float rxy = rxy2 > 0.0f ? rxy2 * rsqrtf(rxy2) : 0.0f;
    float ph = fast_atan2(vy, vx);
    if (ph < 0.0f) ph += 6.28318530717958647692f;
    const float fs = s * g.s_scale, ft = fast_atan2(rxy, vz) * g.t_scale, fp = ph * g.p_scale;
    int is = (int)fs, it = (int)ft, ip = (int)fp;
    if (!bins_certain(g, vx, vy, fs, ft, fp, is, it, ip)) classify_exact(g, vx, vy, vz, r2, is, it, ip);
    return (is * g.nt + it) * g.np + ip;
}

// FP64 local coordinates of a physical offset v inside cone gamma of a level grid.
__device__ __forceinline__ void local_f64(const LevelGrid& g, int gam, double vx, double vy, double vz, double& ts,
                                          double& tt, double& tp, double& r) {
    const int ip = gam % g.np;
    const int it = (gam / g.np) % g.nt;
    const int is = gam / (g.np * g.nt);
    const double rxy = sqrt(vx * vx + vy * vy);
    r = sqrt(vx * vx + vy * vy + vz * vz);
    const double s = g.h64 / r;
    const double th = atan2(rxy, vz);
    const double ph = atan2(vy, vx);
    ts = (s - g.ds64 * (is + 0.5)) / (0.5 * g.ds64);
    tt = (th - g.dt64 * (it + 0.5)) / (0.5 * g.dt64);
    double dph = ph - g.dp64 * (ip + 0.5);
    const double twopi = 6.283185307179586476925286766559;
    if (dph > 3.14159265358979323846) dph -= twopi;
    if (dph > 3.14159265358979323846) dph -= twopi;
    if (dph <= -3.14159265358979323846) dph += twopi;
    if (dph <= -3.14159265358979323846) dph += twopi;
    tp = dph / (0.5 * g.dp64);
}

// Chebyshev polynomials T_0..T_{P-1}(t) by the three-term recurrence.
template <int P, class T>
__device__ __forceinline__ void cheb_T(T t, T* v) {
    v[0] = T(1);
    if (P > 1) v[1] = t;
    const T t2 = t + t;
#pragma unroll
    for (int n = 2; n < P; ++n) v[n] = t2 * v[n - 1] - v[n - 2];
}

// One row (fixed a, b) of the phi contraction: bb = sum_q c_q T_q with packed FP32x2 FMAs.
__device__ __forceinline__ float2 row5(float2 c0, float2 c1, float2 c2, float2 c3, float2 c4, const float* Tp) {
    float2 bb = make_float2(c0.x, c0.y);  // T_0 = 1
    bb = __ffma2_rn(c1, make_float2(Tp[1], Tp[1]), bb);
    bb = __ffma2_rn(c2, make_float2(Tp[2], Tp[2]), bb);
    bb = __ffma2_rn(c3, make_float2(Tp[3], Tp[3]), bb);
    bb = __ffma2_rn(c4, make_float2(Tp[4], Tp[4]), bb);
    return bb;
}

// Loads of coefficients: through the non-coherent read-only path, or (kCoh) as ordinary cached
// loads, for data that other blocks of the same launch wrote before this block's acquire (the
// read-only path is reserved to data that no block writes during the launch).
template <bool kCoh, class T>
__device__ __forceinline__ T ld_ro(const T* p) {
    if constexpr (kCoh) return __ldca(p);
    else return __ldg(p);
}

// Interpolant sum_abc c_abc T_a(ts) T_b(tt) T_c(tp), contracted phi, then theta, then s, with
// packed FP32x2 FMAs (re and im share the real basis weight).  For P_phi = 5 two consecutive
// rows (10 complex = 80 bytes, 16-byte aligned for an even row) are read with five 128-bit
// loads; the coefficient block of a cone must be 16-byte aligned.
template <int PS, int PT, int PP, bool kCoh = false>
__device__ __forceinline__ float2 interp_f32(const float2* __restrict__ c, float ts, float tt, float tp) {
    float Ts[PS], Tt[PT], Tp[PP];
    cheb_T<PS>(ts, Ts);
    cheb_T<PT>(tt, Tt);
    cheb_T<PP>(tp, Tp);
    if constexpr (PP == 5) {
        constexpr int R = PS * PT;
        const float4* c4 = reinterpret_cast<const float4*>(c);
        float2 aa[PS];
#pragma unroll
        for (int a = 0; a < PS; ++a) aa[a] = make_float2(0.f, 0.f);
        // fold row r = a*PT + b into aa[a] with weight T_b(tt) as soon as it is formed
        auto fold = [&](int rr, float2 row) {
            const int a = rr / PT, b = rr - (rr / PT) * PT;
            aa[a] = __ffma2_rn(row, make_float2(Tt[b], Tt[b]), aa[a]);
        };
#pragma unroll
        for (int m = 0; m < R / 2; ++m) {
            const float4 v0 = ld_ro<kCoh>(c4 + 5 * m + 0), v1 = ld_ro<kCoh>(c4 + 5 * m + 1), v2 = ld_ro<kCoh>(c4 + 5 * m + 2);
            const float4 v3 = ld_ro<kCoh>(c4 + 5 * m + 3), v4 = ld_ro<kCoh>(c4 + 5 * m + 4);
            fold(2 * m, row5(make_float2(v0.x, v0.y), make_float2(v0.z, v0.w), make_float2(v1.x, v1.y),
                             make_float2(v1.z, v1.w), make_float2(v2.x, v2.y), Tp));
            fold(2 * m + 1, row5(make_float2(v2.z, v2.w), make_float2(v3.x, v3.y), make_float2(v3.z, v3.w),
                                 make_float2(v4.x, v4.y), make_float2(v4.z, v4.w), Tp));
        }
        if constexpr (R % 2 == 1) {
            const float4 v0 = ld_ro<kCoh>(c4 + 5 * (R / 2) + 0), v1 = ld_ro<kCoh>(c4 + 5 * (R / 2) + 1);
            const float2 v2 = ld_ro<kCoh>(c + 10 * (R / 2) + 4);
            fold(R - 1, row5(make_float2(v0.x, v0.y), make_float2(v0.z, v0.w), make_float2(v1.x, v1.y),
                             make_float2(v1.z, v1.w), v2, Tp));
        }
        float2 acc = aa[0];
#pragma unroll
        for (int a = 1; a < PS; ++a) acc = __ffma2_rn(aa[a], make_float2(Ts[a], Ts[a]), acc);
        return acc;
    } else {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int a = 0; a < PS; ++a) {
            float2 aa = make_float2(0.f, 0.f);
#pragma unroll
            for (int b = 0; b < PT; ++b) {
                float2 bb = make_float2(0.f, 0.f);
#pragma unroll
                for (int q = 0; q < PP; ++q) {
                    const float2 co = ld_ro<kCoh>(c + (a * PT + b) * PP + q);
                    bb = __ffma2_rn(co, make_float2(Tp[q], Tp[q]), bb);
                }
                aa = __ffma2_rn(bb, make_float2(Tt[b], Tt[b]), aa);
            }
            acc = __ffma2_rn(aa, make_float2(Ts[a], Ts[a]), acc);
        }
        return acc;
    }
}

// The contraction of interp_f32 for R points of one cone: every coefficient row is loaded
// once and applied to all R points, so the coefficient bytes moved into registers per point
// drop by R. Row (a, b) enters point q with weight T_a(ts_q) T_b(tt_q).
// kShared: the coefficient block was staged in shared memory (same layout) and is read with
// plain loads; otherwise it is read from global memory through the read-only path.
template <int PS, int PT, int PP, int R, bool kShared = false, bool kCoh = false>
__device__ __forceinline__ void interp_f32_seg(const float2* __restrict__ c, const float* ts, const float* tt,
                                               const float* tp, float2* out) {
    float Ts[R][PS], Tt[R][PT], Tp[R][PP];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        cheb_T<PS>(ts[q], Ts[q]);
        cheb_T<PT>(tt[q], Tt[q]);
        cheb_T<PP>(tp[q], Tp[q]);
        out[q] = make_float2(0.f, 0.f);
    }
    auto fold = [&](int rr, const float2* row) {
        const int a = rr / PT, b = rr - (rr / PT) * PT;
#pragma unroll
        for (int q = 0; q < R; ++q) {
            float2 bb = row[0];
#pragma unroll
            for (int k = 1; k < PP; ++k) bb = __ffma2_rn(row[k], make_float2(Tp[q][k], Tp[q][k]), bb);
            const float w = Ts[q][a] * Tt[q][b];
            out[q] = __ffma2_rn(bb, make_float2(w, w), out[q]);
        }
    };
    constexpr int NR = PS * PT;
    if constexpr (PP == 5) {
        const float4* c4 = reinterpret_cast<const float4*>(c);
        auto ld4 = [&](int i) -> float4 {
            if constexpr (kShared) return c4[i];
            else return ld_ro<kCoh>(c4 + i);
        };
#pragma unroll
        for (int m = 0; m < NR / 2; ++m) {
            const float4 v0 = ld4(5 * m + 0), v1 = ld4(5 * m + 1), v2 = ld4(5 * m + 2);
            const float4 v3 = ld4(5 * m + 3), v4 = ld4(5 * m + 4);
            const float2 r0[5] = {make_float2(v0.x, v0.y), make_float2(v0.z, v0.w), make_float2(v1.x, v1.y),
                                  make_float2(v1.z, v1.w), make_float2(v2.x, v2.y)};
            const float2 r1[5] = {make_float2(v2.z, v2.w), make_float2(v3.x, v3.y), make_float2(v3.z, v3.w),
                                  make_float2(v4.x, v4.y), make_float2(v4.z, v4.w)};
            fold(2 * m, r0);
            fold(2 * m + 1, r1);
        }
        if constexpr (NR % 2 == 1) {
            const float4 v0 = ld4(5 * (NR / 2) + 0), v1 = ld4(5 * (NR / 2) + 1);
            float2 v2;
            if constexpr (kShared) v2 = c[10 * (NR / 2) + 4];
            else v2 = ld_ro<kCoh>(c + 10 * (NR / 2) + 4);
            const float2 r0[5] = {make_float2(v0.x, v0.y), make_float2(v0.z, v0.w), make_float2(v1.x, v1.y),
                                  make_float2(v1.z, v1.w), v2};
            fold(NR - 1, r0);
        }
    } else {
#pragma unroll 1
        for (int rr = 0; rr < NR; ++rr) {
            float2 row[PP];
#pragma unroll
            for (int k = 0; k < PP; ++k) {
                if constexpr (kShared) row[k] = c[rr * PP + k];
                else row[k] = ld_ro<kCoh>(c + rr * PP + k);
            }
            // rr is not a compile-time constant here: weights by explicit selection
            const int a = rr / PT, b = rr - (rr / PT) * PT;
#pragma unroll
            for (int q = 0; q < R; ++q) {
                float2 bb = row[0];
#pragma unroll
                for (int k = 1; k < PP; ++k) bb = __ffma2_rn(row[k], make_float2(Tp[q][k], Tp[q][k]), bb);
                float wa = Ts[q][0], wb = Tt[q][0];
#pragma unroll
                for (int i = 1; i < PS; ++i) wa = a == i ? Ts[q][i] : wa;
#pragma unroll
                for (int i = 1; i < PT; ++i) wb = b == i ? Tt[q][i] : wb;
                const float w = wa * wb;
                out[q] = __ffma2_rn(bb, make_float2(w, w), out[q]);
            }
        }
    }
}

template <int PS, int PT, int PP>
__device__ __forceinline__ double2 interp_f64(const double2* __restrict__ c, double ts, double tt, double tp) {
    double Ts[PS], Tt[PT], Tp[PP];
    cheb_T<PS>(ts, Ts);
    cheb_T<PT>(tt, Tt);
    cheb_T<PP>(tp, Tp);
    double2 acc = make_double2(0., 0.);
#pragma unroll
    for (int a = 0; a < PS; ++a) {
        double2 aa = make_double2(0., 0.);
#pragma unroll
        for (int b = 0; b < PT; ++b) {
            double2 bb = make_double2(0., 0.);
#pragma unroll
            for (int q = 0; q < PP; ++q) {
                const double2 co = c[(a * PT + b) * PP + q];
                bb.x = fma(co.x, Tp[q], bb.x);
                bb.y = fma(co.y, Tp[q], bb.y);
            }
            aa.x = fma(bb.x, Tt[b], aa.x);
            aa.y = fma(bb.y, Tt[b], aa.y);
        }
        acc.x = fma(aa.x, Ts[a], acc.x);
        acc.y = fma(aa.y, Ts[a], acc.y);
    }
    return acc;
}

// Reduction of an angle to [-pi, pi] (Cody and Waite's method: 2 pi = c1 + c2 + c3 with c1
// short enough that k*c1 is exact; each step is one fused multiply-add).
__device__ __forceinline__ float reduce_2pi(float x) {
    const float k = rintf(x * 0.159154943091895335768883763f);
    float r = fmaf(-k, 6.28125f, x);
    r = fmaf(-k, 0.0019353071693331003f, r);
    r = fmaf(-k, 1.0253131677018246e-11f, r);
    return r;
}

// exp(i x) for an FP32 phase, after reduction.
__device__ __forceinline__ float2 cis_f32(float x) {
    float s, c;
    __sincosf(reduce_2pi(x), &s, &c);
    return make_float2(c, s);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ void set_status(int* st, int code) { atomicCAS(st, 0, code); }

// ---- tensor-core helpers (warp-level mma.sync, TF32, 3xTF32 split precision) ----------------
// Fragment layout of mma.m16n8k8 (row.col), g = lane / 4, t = lane % 4:
//   A (16x8):  a0 (g, t), a1 (g+8, t), a2 (g, t+4), a3 (g+8, t+4)
//   B (8x8):   b0 (t, g), b1 (t+4, g)
//   C (16x8):  c0 (g, 2t), c1 (g, 2t+1), c2 (g+8, 2t), c3 (g+8, 2t+1)
// x = hi + lo for 3xTF32 products: hi keeps the sign, exponent and 10 leading mantissa bits of
// x (the 13 low bits cleared), so |lo| < 2^-10 |x| and lo = x - hi is exact in FP32. The tensor
// core reads the 10 leading mantissa bits of lo, which leaves a relative error below 2^-20 |x|
// in hi + lo; with the dropped lo*lo term a product keeps about 19 bits.
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
    hi = __float_as_uint(x) & 0xffffe000u;
    lo = __float_as_uint(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// C += A B with A = ah + al, B = bh + bl to FP32 accuracy: al bh + ah bl + ah bh.
__device__ __forceinline__ void mma_3xtf32(float (&c)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                           const uint32_t (&bh)[2], const uint32_t (&bl)[2]) {
    mma_tf32(c, al, bh);
    mma_tf32(c, ah, bl);
    mma_tf32(c, ah, bh);
}

// Multi-density interpolant contraction for one warp: 16 points (rows r0 = g, r1 = g + 8,
// whose Chebyshev values this thread holds), the coefficient block of one cone for 4*NT
// densities starting at rhs0 (row p = coefficient index, columns (density, re/im)), rows whose
// mask bit is clear contribute zero.  c[j] receives the C fragment of n-tile j.
template <int N>
__device__ __forceinline__ float pick(const float (&v)[N], int i) {  // v[i] without local memory
    float r = v[0];
#pragma unroll
    for (int k = 1; k < N; ++k) r = (i == k) ? v[k] : r;
    return r;
}

template <int PS, int PT, int PP, int NT>
__device__ __forceinline__ void mma_interp_block(const float (&Ts0)[PS], const float (&Tt0)[PT],
                                                 const float (&Tp0)[PP], const float (&Ts1)[PS],
                                                 const float (&Tt1)[PT], const float (&Tp1)[PP], bool row0,
                                                 bool row1, const float2* __restrict__ coef, int64_t cone_base,
                                                 int nrhs, int rhs0, int cstride, float (&c)[NT][4]) {
    constexpr int P = PS * PT * PP;
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    // density columns of this thread in every n-tile: (rhs, re/im) = (rhs0 + (8j + g)/2, g & 1)
    const float* blk[NT];
    bool colok[NT];
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        const int rhs = rhs0 + ((j * 8 + g) >> 1);
        colok[j] = rhs < nrhs;
        blk[j] = reinterpret_cast<const float*>(coef + (cone_base * nrhs + (colok[j] ? rhs : 0)) * cstride) + (g & 1);
    }
#pragma unroll 1
    for (int kk = 0; kk < (P + 7) / 8; ++kk) {
        const int p0 = kk * 8 + t, p1 = p0 + 4;
        const int a0 = p0 / (PT * PP), b0 = (p0 / PP) % PT, q0 = p0 % PP;
        const int a1 = p1 / (PT * PP), b1 = (p1 / PP) % PT, q1 = p1 % PP;
        const bool ok0 = p0 < P, ok1 = p1 < P;
        const float A0 = (row0 && ok0) ? pick(Ts0, a0) * pick(Tt0, b0) * pick(Tp0, q0) : 0.f;
        const float A1 = (row1 && ok0) ? pick(Ts1, a0) * pick(Tt1, b0) * pick(Tp1, q0) : 0.f;
        const float A2 = (row0 && ok1) ? pick(Ts0, a1) * pick(Tt0, b1) * pick(Tp0, q1) : 0.f;
        const float A3 = (row1 && ok1) ? pick(Ts1, a1) * pick(Tt1, b1) * pick(Tp1, q1) : 0.f;
        uint32_t ah[4], al[4];
        tf32_split(A0, ah[0], al[0]);
        tf32_split(A1, ah[1], al[1]);
        tf32_split(A2, ah[2], al[2]);
        tf32_split(A3, ah[3], al[3]);
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            const float B0 = (colok[j] && ok0) ? __ldg(blk[j] + 2 * p0) : 0.f;
            const float B1 = (colok[j] && ok1) ? __ldg(blk[j] + 2 * p1) : 0.f;
            uint32_t bh[2], bl[2];
            tf32_split(B0, bh[0], bl[0]);
            tf32_split(B1, bh[1], bl[1]);
            mma_3xtf32(c[j], ah, al, bh, bl);
        }
    }
}

// Morton interleave of three 21-bit coordinates (bit 3b = x_b, 3b+1 = y_b, 3b+2 = z_b).
__host__ __device__ __forceinline__ uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}
__host__ __device__ __forceinline__ uint32_t compact3(uint64_t x) {
    x &= 0x1249249249249249ull;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
    x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
    x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
    x = (x ^ (x >> 32)) & 0x1fffffull;
    return (uint32_t)x;
}
__host__ __device__ __forceinline__ uint64_t morton3(uint32_t x, uint32_t y, uint32_t z) {
    return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

}  // namespace ifgf
