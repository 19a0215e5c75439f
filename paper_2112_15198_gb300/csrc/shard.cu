// Distribution of the method over several GPUs (Sec. 3.2).
//
// Decomposition (Sec. 3.2.1): the points in intervals of whole leaf boxes of the Morton order with
// nearly equal point counts, and every level's relevant cones in contiguous intervals of the cone
// order, which may split co-centred cones between ranks.  The two partition functions are plain
// host code; they depend only on the sorted box point ranges and the cone counts, which every rank
// derives identically from the same points.
//
// A shard is one rank's part of a plan.  Every rank builds the same plan (tree, lists and relevant
// cones are integers, a small fraction of the coefficient memory) and holds coefficients only for
// its own cones and for the cones of other ranks that its steps read: the cones its targets look
// up in Interpolation(d) and the child cones its parent cones look up in Propagation(d) (the data
// of the paper's two communication algorithms), found by marking kernels that repeat those
// lookups.  Per level the rank's coefficient buffer holds its own cones first, then the needed
// cones in ascending cone order; a map from the level's cone index to the block in that buffer
// (-1 where not held) is what the apply kernels' lookups go through.  The data movement between
// ranks is left to the caller (the Python binding uses torch.distributed): for level d it fills
// the needed part of the buffer from the owners' own parts (ifgf_shard_pack) before
// ifgf_shard_level(d) runs.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "ifgf_internal.cuh"

using namespace ifgf;

struct ifgf_shard_s {
    Plan* plan = nullptr;
    int nranks = 1, rank = 0, max_nrhs = 1;
    std::vector<int64_t> box_bounds, pt_bounds;  // [nranks + 1] leaf boxes, sorted points
    int64_t b0 = 0, b1 = 0, p0 = 0, p1 = 0;      // own leaf boxes and points
    int64_t lb0 = 0, lb1 = 0;                    // leaf boxes of the own level-D cones
    struct Lev {
        std::vector<int64_t> bounds;      // [nranks + 1] cone intervals
        int64_t c0 = 0, c1 = 0;           // own cones
        std::vector<uint8_t> looked;      // per cone: bit 0 Interpolation, bit 1 Propagation lookups
        std::vector<int64_t> need;        // cones of other ranks read, ascending
        int32_t* g2l = nullptr;           // [nc] block in coef, or -1
        float2* coef = nullptr;           // (own + needed) blocks of max_nrhs x cstride
    } L[kMaxLevel + 1];
    std::vector<int64_t> need_pts;        // points of other ranks read, ascending
    std::vector<void*> allocs;
};

namespace ifgf {
ifgf::Plan* plan_of(ifgf_plan p);  // api.cu
ifgf_status guard_call(const std::function<void()>& f);
}  // namespace ifgf

namespace {
constexpr int kT = 256;

template <class T>
T* shard_alloc(ifgf_shard_s& sh, size_t count) {
    void* ptr = nullptr;
    const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    if (cudaMallocFromPoolAsync(&ptr, bytes, device_pool(sh.plan->device), sh.plan->stream) != cudaSuccess) {
        cudaGetLastError();
        fail(IFGF_ERR_OOM, "shard allocation of " + std::to_string(bytes) + " bytes failed");
    }
    sh.allocs.push_back(ptr);
    return static_cast<T*>(ptr);
}

void shard_free(ifgf_shard_s& sh) {
    for (void* ptr : sh.allocs) cudaFreeAsync(ptr, sh.plan->stream);
    sh.allocs.clear();
    cudaStreamSynchronize(sh.plan->stream);
}

// Interpolation(d) lookups of the points [p0, p1): for every cousin box of a point's level-d box,
// the relevant cone that contains the point (as the interpolation kernels find it).
__global__ void k_look_interp(int64_t p0, int64_t p1, int D, int d, const int32_t* __restrict__ pbox_d,
                              const int32_t* __restrict__ pbox_D, const int4* __restrict__ kD,
                              const int4* __restrict__ kd, const int32_t* __restrict__ ncs,
                              const int32_t* __restrict__ cs, const float4* __restrict__ off, LevelGrid g, ConeMap cm,
                              uint8_t* __restrict__ flags, int* __restrict__ status) {
    const int64_t i = p0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p1) return;
    const int A = pbox_d[i];
    const int4 kl = kD[pbox_D[i]];
    const float4 o = off[i];
    const int sh = D - d;
    for (int t = 0; t < ncs[A]; ++t) {
        const int B = cs[(int64_t)A * kMaxCous + t];
        if (!in_bounds(B, cm.nbox, status)) continue;
        const int4 kb = kd[B];
        const float vx = __fadd_rn((float)((2 * kl.x + 1) - ((2 * kb.x + 1) << sh)), o.x);
        const float vy = __fadd_rn((float)((2 * kl.y + 1) - ((2 * kb.y + 1) << sh)), o.y);
        const float vz = __fadd_rn((float)((2 * kl.z + 1) - ((2 * kb.z + 1) << sh)), o.z);
        const int s = cm.find_global(B, classify_f32(g, vx, vy, vz));
        if (s < 0) set_status(status, IFGF_ERR_INTERNAL);
        else flags[s] = 1;
    }
}

// Propagation(d) lookups of the level-(d-1) cones [lo, hi): every node of each, in each child box,
// the relevant child cone that contains it.
__global__ void k_look_prop(int64_t lo, int64_t hi, int Ps, int Pt, int Pp, int D, int d,
                            const int32_t* __restrict__ pcone_box, const int32_t* __restrict__ pcone_gam,
                            const int4* __restrict__ kp, const int32_t* __restrict__ pcstart,
                            const int4* __restrict__ kd, LevelGrid gp, LevelGrid g, ConeMap cm,
                            uint8_t* __restrict__ flags, int* __restrict__ status) {
    const int P = Ps * Pt * Pp;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (hi - lo) * P) return;
    const int64_t pc = lo + t / P;
    const int n = (int)(t % P);
    const int jb = pcone_box[pc], gam = pcone_gam[pc];
    const int ip = gam % gp.np, it = (gam / gp.np) % gp.nt, is = gam / (gp.np * gp.nt);
    const int c = n % Pp, b = (n / Pp) % Pt, a = n / (Pp * Pt);
    const float rho = gp.rho[is * Ps + a];
    const float st = gp.stn[it * Pt + b], ct = gp.ctn[it * Pt + b];
    const float cp = gp.cpn[ip * Pp + c], sp = gp.spn[ip * Pp + c];
    const float qx = __fmul_rn(rho, __fmul_rn(st, cp)), qy = __fmul_rn(rho, __fmul_rn(st, sp));
    const float qz = __fmul_rn(rho, ct);
    const int4 kj = kp[jb];
    const int sh = D - d;
    for (int kb = pcstart[jb]; kb < pcstart[jb + 1]; ++kb) {
        const int4 kk = kd[kb];
        const float ox = (float)((2 * (kk.x - 2 * kj.x) - 1) << sh);
        const float oy = (float)((2 * (kk.y - 2 * kj.y) - 1) << sh);
        const float oz = (float)((2 * (kk.z - 2 * kj.z) - 1) << sh);
        const int s = cm.find_global(kb, classify_f32(g, __fsub_rn(qx, ox), __fsub_rn(qy, oy), __fsub_rn(qz, oz)));
        if (s < 0) set_status(status, IFGF_ERR_INTERNAL);
        else flags[s] = 1;
    }
}

// Points read by the near field of the leaf boxes [b0, b1) (their neighbour boxes' points) and by
// LevelDEvaluations of the cones of the leaf boxes [lb0, lb1); one block per box.
__global__ void k_look_points(int64_t b0, int64_t b1, int64_t lb0, int64_t lb1, const int32_t* __restrict__ startD,
                              const int32_t* __restrict__ nnb, const int32_t* __restrict__ nb,
                              uint8_t* __restrict__ flags) {
    const int64_t b = blockIdx.x;
    if (b >= b0 && b < b1)
        for (int t = 0; t < nnb[b]; ++t) {
            const int q = nb[b * kMaxNbr + t];
            for (int j = startD[q] + threadIdx.x; j < startD[q + 1]; j += blockDim.x) flags[j] = 1;
        }
    if (b >= lb0 && b < lb1)
        for (int j = startD[b] + threadIdx.x; j < startD[b + 1]; j += blockDim.x) flags[j] = 1;
}

// dst[j] = block ids[j] - c0 of src (blocks of `len` float4).
__global__ void k_pack(const int64_t* __restrict__ ids, int64_t n, int64_t c0, const float4* __restrict__ src,
                       int64_t len, float4* __restrict__ dst) {
    const int64_t j = blockIdx.x;
    if (j >= n) return;
    const float4* s = src + (ids[j] - c0) * len;
    for (int64_t k = threadIdx.x; k < len; k += blockDim.x) dst[j * len + k] = s[k];
}

template <class T>
std::vector<T> to_host(const T* d, int64_t n, cudaStream_t s) {
    std::vector<T> h((size_t)std::max<int64_t>(n, 0));
    if (n > 0) {
        IFGF_CUDA(cudaMemcpyAsync(h.data(), d, sizeof(T) * n, cudaMemcpyDeviceToHost, s));
        IFGF_CUDA(cudaStreamSynchronize(s));
    }
    return h;
}
}  // namespace

extern "C" {

ifgf_status ifgf_partition_boxes(const int64_t* box_start, int64_t nbox, int32_t nranks, int64_t* out_bounds) {
    if (!box_start || !out_bounds || nbox < 1 || nranks < 1) {
        set_last_error("partition of boxes: NULL array, no box or no rank");
        return IFGF_ERR_INVALID_ARG;
    }
    const int64_t N = box_start[nbox];
    if (box_start[0] != 0 || N < 1) {
        set_last_error("partition of boxes: point ranges must start at 0 and hold at least one point");
        return IFGF_ERR_INVALID_ARG;
    }
    for (int64_t b = 0; b < nbox; ++b)
        if (box_start[b + 1] < box_start[b]) {
            set_last_error("partition of boxes: point ranges must be non-decreasing");
            return IFGF_ERR_INVALID_ARG;
        }
    // Bound r is the box boundary whose point offset is nearest to r N / nranks (the lower one on a
    // tie), kept non-decreasing; rank r owns the boxes [bound r, bound r+1).
    out_bounds[0] = 0;
    out_bounds[nranks] = nbox;
    for (int32_t r = 1; r < nranks; ++r) {
        const double t = (double)N * r / nranks;
        const int64_t* hi = std::lower_bound(box_start, box_start + nbox + 1, (int64_t)std::ceil(t));
        int64_t b = hi - box_start;
        if (b > 0 && (t - (double)box_start[b - 1]) <= ((double)box_start[std::min(b, nbox)] - t)) --b;
        b = std::min(std::max(b, out_bounds[r - 1]), nbox);
        out_bounds[r] = b;
    }
    return IFGF_OK;
}

ifgf_status ifgf_partition_cones(int64_t nc, int32_t nranks, int64_t* out_bounds) {
    if (!out_bounds || nc < 0 || nranks < 1) {
        set_last_error("partition of cones: NULL array, negative count or no rank");
        return IFGF_ERR_INVALID_ARG;
    }
    // Rank r owns the cones [floor(r nc / nranks), floor((r + 1) nc / nranks)): interval sizes
    // differ by at most one.
    for (int32_t r = 0; r <= nranks; ++r) out_bounds[r] = (int64_t)((__int128)nc * r / nranks);
    return IFGF_OK;
}

}  // extern "C"

extern "C" {

ifgf_status ifgf_shard_create(ifgf_plan plan, int32_t nranks, int32_t rank, int32_t max_nrhs, ifgf_shard* out) {
    if (!plan || !out || nranks < 1 || rank < 0 || rank >= nranks || max_nrhs < 1 || max_nrhs > 3) {
        set_last_error("shard: NULL plan or handle, rank outside [0, nranks), or max_nrhs outside [1, 3]");
        return IFGF_ERR_INVALID_ARG;
    }
    Plan& p = *plan_of(plan);
    if (p.precision != IFGF_PREC_MIXED) {
        set_last_error("shards are built for mixed-precision plans");
        return IFGF_ERR_UNSUPPORTED;
    }
    ifgf_shard_s* sh = new ifgf_shard_s();
    sh->plan = &p;
    sh->nranks = nranks;
    sh->rank = rank;
    sh->max_nrhs = max_nrhs;
    ifgf_status st = guard_call([&] {
        IFGF_CUDA(cudaSetDevice(p.device));
        cudaStream_t s = p.stream;
        const int D = p.D;
        Level& LD = p.L[D];
        // points: intervals of whole leaf boxes
        auto st32 = to_host(LD.start, (int64_t)LD.n + 1, s);
        std::vector<int64_t> bst(st32.begin(), st32.end());
        sh->box_bounds.assign(nranks + 1, 0);
        if (ifgf_partition_boxes(bst.data(), LD.n, nranks, sh->box_bounds.data()) != IFGF_OK)
            fail(IFGF_ERR_INTERNAL, "partition of the leaf boxes failed");
        sh->pt_bounds.resize(nranks + 1);
        for (int r = 0; r <= nranks; ++r) sh->pt_bounds[r] = bst[sh->box_bounds[r]];
        sh->b0 = sh->box_bounds[rank];
        sh->b1 = sh->box_bounds[rank + 1];
        sh->p0 = sh->pt_bounds[rank];
        sh->p1 = sh->pt_bounds[rank + 1];
        // cones: contiguous intervals of each level's cone order
        for (int d = 3; d <= D; ++d) {
            auto& L = sh->L[d];
            L.bounds.assign(nranks + 1, 0);
            ifgf_partition_cones(p.L[d].nc, nranks, L.bounds.data());
            L.c0 = L.bounds[rank];
            L.c1 = L.bounds[rank + 1];
        }
        if (sh->L[D].c1 > sh->L[D].c0) {
            auto cb = to_host(LD.cone_box, LD.nc, s);
            sh->lb0 = cb[sh->L[D].c0];
            sh->lb1 = (int64_t)cb[sh->L[D].c1 - 1] + 1;
        }
        // what the rank's steps read: cones per level, points
        for (int d = 3; d <= D; ++d) {
            Level& Lv = p.L[d];
            auto& L = sh->L[d];
            const size_t nf = (size_t)std::max<int64_t>(Lv.nc, 1);
            uint8_t* fi = shard_alloc<uint8_t>(*sh, nf);  // looked up by Interpolation(d)
            uint8_t* fp = shard_alloc<uint8_t>(*sh, nf);  // looked up by Propagation(d)
            IFGF_CUDA(cudaMemsetAsync(fi, 0, nf, s));
            IFGF_CUDA(cudaMemsetAsync(fp, 0, nf, s));
            if (sh->p1 > sh->p0)
                IFGF_LAUNCH(k_look_interp, grid_for(sh->p1 - sh->p0, kT), kT, 0, s, sh->p0, sh->p1, D, d, Lv.pbox, LD.pbox,
                            LD.k, Lv.k, Lv.ncs, Lv.cs, p.off, Lv.g, Lv.cmap(p.d_status), fi, p.d_status);
            if (d > 3) {
                Level& Lp = p.L[d - 1];
                const int64_t lo = sh->L[d - 1].c0, hi = sh->L[d - 1].c1;
                if (hi > lo)
                    IFGF_LAUNCH(k_look_prop, grid_for((hi - lo) * p.P, kT), kT, 0, s, lo, hi, p.Ps, p.Pt, p.Pp, D, d,
                                Lp.cone_box, Lp.cone_gam, Lp.k, Lp.cstart, Lv.k, Lp.g, Lv.g, Lv.cmap(p.d_status), fp, p.d_status);
            }
            L.looked = to_host(fi, Lv.nc, s);
            const auto lp = to_host(fp, Lv.nc, s);
            for (int64_t c = 0; c < Lv.nc; ++c) L.looked[c] |= (uint8_t)(lp[c] << 1);
            std::vector<int32_t> g2l((size_t)std::max<int64_t>(Lv.nc, 1), -1);
            for (int64_t c = L.c0; c < L.c1; ++c) g2l[c] = (int32_t)(c - L.c0);
            for (int64_t c = 0; c < Lv.nc; ++c)
                if (L.looked[c] && (c < L.c0 || c >= L.c1)) {
                    g2l[c] = (int32_t)((L.c1 - L.c0) + (int64_t)L.need.size());
                    L.need.push_back(c);
                }
            L.g2l = shard_alloc<int32_t>(*sh, g2l.size());
            IFGF_CUDA(cudaMemcpyAsync(L.g2l, g2l.data(), sizeof(int32_t) * g2l.size(), cudaMemcpyHostToDevice, s));
            const int64_t held = (L.c1 - L.c0) + (int64_t)L.need.size();
            L.coef = shard_alloc<float2>(*sh, (size_t)std::max<int64_t>(held, 1) * max_nrhs * p.cstride);
            IFGF_CUDA(cudaStreamSynchronize(s));  // the host copy of g2l outlives no iteration
        }
        uint8_t* pflags = shard_alloc<uint8_t>(*sh, (size_t)p.N);
        IFGF_CUDA(cudaMemsetAsync(pflags, 0, (size_t)p.N, s));
        IFGF_LAUNCH(k_look_points, (unsigned)LD.n, 128, 0, s, sh->b0, sh->b1, sh->lb0, sh->lb1, LD.start, LD.nnb, LD.nb,
                    pflags);
        auto pf = to_host(pflags, p.N, s);
        for (int64_t i = 0; i < p.N; ++i)
            if (pf[i] && (i < sh->p0 || i >= sh->p1)) sh->need_pts.push_back(i);
        int dst = 0;
        IFGF_CUDA(cudaMemcpy(&dst, p.d_status, sizeof(int), cudaMemcpyDeviceToHost));
        if (dst != 0) fail((ifgf_status)dst, "a lookup of the shard's steps found no relevant cone");
    });
    if (st != IFGF_OK) {
        shard_free(*sh);
        delete sh;
        return st;
    }
    *out = sh;
    return IFGF_OK;
}

ifgf_status ifgf_shard_query(ifgf_shard sh, int32_t what, int32_t level, int64_t* host_buf, int64_t* inout_count) {
    if (!sh || !inout_count) {
        set_last_error("NULL shard or count");
        return IFGF_ERR_INVALID_ARG;
    }
    const bool lev_ok = level >= 3 && level <= sh->plan->D;
    std::vector<int64_t> res;
    switch (what) {
        case IFGF_SQ_POINTS: res = {sh->p0, sh->p1}; break;
        case IFGF_SQ_BOXES: res = {sh->b0, sh->b1}; break;
        case IFGF_SQ_POINT_BOUNDS: res = sh->pt_bounds; break;
        case IFGF_SQ_NEED_POINTS: res = sh->need_pts; break;
        case IFGF_SQ_CONES:
        case IFGF_SQ_CONE_BOUNDS:
        case IFGF_SQ_NEED_CONES:
        case IFGF_SQ_LOOKED_INTERP:
        case IFGF_SQ_LOOKED_PROP: {
            if (!lev_ok) {
                set_last_error("level outside [3, D]");
                return IFGF_ERR_INVALID_ARG;
            }
            const auto& L = sh->L[level];
            if (what == IFGF_SQ_CONES) res = {L.c0, L.c1};
            else if (what == IFGF_SQ_CONE_BOUNDS) res = L.bounds;
            else if (what == IFGF_SQ_NEED_CONES) res = L.need;
            else {
                const uint8_t bit = what == IFGF_SQ_LOOKED_INTERP ? 1 : 2;
                for (size_t c = 0; c < L.looked.size(); ++c)
                    if (L.looked[c] & bit) res.push_back((int64_t)c);
            }
            break;
        }
        default:
            set_last_error("unknown shard query");
            return IFGF_ERR_INVALID_ARG;
    }
    const int64_t cap = *inout_count;
    *inout_count = (int64_t)res.size();
    if (host_buf && cap >= (int64_t)res.size() && !res.empty())
        std::memcpy(host_buf, res.data(), sizeof(int64_t) * res.size());
    return IFGF_OK;
}

ifgf_status ifgf_shard_coefficients(ifgf_shard sh, int32_t level, int32_t nrhs, void** buf, int64_t* block_bytes) {
    if (!sh || !buf || !block_bytes || level < 3 || level > sh->plan->D || nrhs < 1 || nrhs > sh->max_nrhs) {
        set_last_error("shard coefficients: NULL argument, level outside [3, D] or nrhs outside [1, max_nrhs]");
        return IFGF_ERR_INVALID_ARG;
    }
    *buf = sh->L[level].coef;
    *block_bytes = (int64_t)nrhs * sh->plan->cstride * (int64_t)sizeof(float2);
    return IFGF_OK;
}

ifgf_status ifgf_shard_pack(ifgf_shard sh, int32_t level, int32_t nrhs, const int64_t* ids, int64_t n, void* dst,
                            void* stream) {
    if (!sh || level < 3 || level > sh->plan->D || nrhs < 1 || nrhs > sh->max_nrhs || n < 0 || (n > 0 && (!ids || !dst))) {
        set_last_error("shard pack: invalid argument");
        return IFGF_ERR_INVALID_ARG;
    }
    return guard_call([&] {
        IFGF_CUDA(cudaSetDevice(sh->plan->device));
        const auto& L = sh->L[level];
        const int64_t len = (int64_t)nrhs * sh->plan->cstride / 2;  // float4 per block (cstride is even)
        if (n > 0)
            IFGF_LAUNCH(k_pack, (unsigned)n, 128, 0, (cudaStream_t)stream, ids, n, L.c0, (const float4*)L.coef, len,
                        (float4*)dst);
    });
}

ifgf_status ifgf_shard_unpack(ifgf_shard sh, int32_t level, int32_t nrhs, const void* src, int64_t first, int64_t n,
                              void* stream) {
    if (!sh || level < 3 || level > sh->plan->D || nrhs < 1 || nrhs > sh->max_nrhs || first < 0 || n < 0 ||
        first + n > (int64_t)sh->L[level].need.size() || (n > 0 && !src)) {
        set_last_error("shard unpack: invalid argument or blocks beyond the needed cones");
        return IFGF_ERR_INVALID_ARG;
    }
    return guard_call([&] {
        IFGF_CUDA(cudaSetDevice(sh->plan->device));
        const auto& L = sh->L[level];
        const size_t block = (size_t)nrhs * sh->plan->cstride * sizeof(float2);
        if (n > 0)
            IFGF_CUDA(cudaMemcpyAsync(reinterpret_cast<char*>(L.coef) + (size_t)((L.c1 - L.c0) + first) * block, src,
                                      (size_t)n * block, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    });
}

ifgf_status ifgf_shard_near_leaf(ifgf_shard sh, const void* dens_sorted, int32_t nrhs, void* out_sorted, void* stream) {
    if (!sh || !dens_sorted || !out_sorted || nrhs < 1 || nrhs > sh->max_nrhs) {
        set_last_error("shard near/leaf: NULL buffer or nrhs outside [1, max_nrhs]");
        return IFGF_ERR_INVALID_ARG;
    }
    return guard_call([&] {
        Plan& p = *sh->plan;
        IFGF_CUDA(cudaSetDevice(p.device));
        const auto& L = sh->L[p.D];
        shard_near_leaf(p, (const float2*)dens_sorted, nrhs, (float2*)out_sorted, sh->b0, sh->b1, sh->lb0, sh->lb1, L.c0,
                        L.c1, L.coef, (cudaStream_t)stream);
    });
}

ifgf_status ifgf_shard_level(ifgf_shard sh, int32_t level, int32_t nrhs, void* out_sorted, void* stream) {
    if (!sh || !out_sorted || level < 3 || level > sh->plan->D || nrhs < 1 || nrhs > sh->max_nrhs) {
        set_last_error("shard level: NULL buffer, level outside [3, D] or nrhs outside [1, max_nrhs]");
        return IFGF_ERR_INVALID_ARG;
    }
    return guard_call([&] {
        Plan& p = *sh->plan;
        IFGF_CUDA(cudaSetDevice(p.device));
        cudaStream_t s = (cudaStream_t)stream;
        const auto& L = sh->L[level];
        ConeMap cm = p.L[level].cmap(p.d_status);
        cm.g2l = L.g2l;
        shard_interp(p, level, nrhs, (float2*)out_sorted, cm, L.coef, sh->p0, sh->p1, s);
        if (level > 3) {
            const auto& Lp = sh->L[level - 1];
            shard_prop(p, level, nrhs, Lp.c0, Lp.c1, cm, L.coef, Lp.coef, s);
        }
    });
}

ifgf_status ifgf_shard_destroy(ifgf_shard sh) {
    if (!sh) return IFGF_OK;
    cudaSetDevice(sh->plan->device);
    shard_free(*sh);
    delete sh;
    return IFGF_OK;
}

}  // extern "C"
