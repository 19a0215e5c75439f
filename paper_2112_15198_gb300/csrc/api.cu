// extern "C" boundary of the library: argument checks, plan lifetime, queries, errors.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <tuple>
#include <string>
#include <vector>

#include "ifgf_internal.cuh"

namespace ifgf {

namespace {
thread_local std::string t_last_error;
}

void set_last_error(const std::string& s) { t_last_error = s; }

void fail(ifgf_status s, const std::string& what) { throw Error{s, what}; }

void cuda_check(cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(IFGF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }
}

namespace {
struct TimingState {
    std::mutex mu;
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<std::tuple<int, int, cudaEvent_t, cudaEvent_t>> pending;  // kind, level, start, end
    double ms[TK_COUNT] = {0};
    int64_t launches[TK_COUNT] = {0};
    double by_level[TK_COUNT][kMaxLevel + 1] = {};
    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
};
TimingState& timing() {
    static TimingState t;
    return t;
}
thread_local int g_timing_level = -1;
}  // namespace

TimingLevel::TimingLevel(int d) : prev(g_timing_level) { g_timing_level = d; }
TimingLevel::~TimingLevel() { g_timing_level = prev; }

bool timing_switch(bool on) {
    TimingState& t = timing();
    std::lock_guard<std::mutex> lk(t.mu);
    const bool was = t.on;
    t.on = on;
    return was;
}

void timing_collect_levels(double* ms, int64_t* launches, double (*by_level)[kMaxLevel + 1]) {
    TimingState& t = timing();
    std::lock_guard<std::mutex> lk(t.mu);
    for (auto& [k, lev, a, b] : t.pending) {
        float el = 0.f;
        if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&el, a, b) != cudaSuccess)
            cuda_check(cudaGetLastError(), "kernel timing");
        t.ms[k] += el;
        t.launches[k] += 1;
        if (lev >= 0 && lev <= kMaxLevel) t.by_level[k][lev] += el;
        t.pool.push_back(a);
        t.pool.push_back(b);
    }
    t.pending.clear();
    for (int k = 0; k < TK_COUNT; ++k) {
        if (ms) ms[k] = t.ms[k];
        if (launches) launches[k] = t.launches[k];
        for (int d = 0; d <= kMaxLevel; ++d) {
            if (by_level) by_level[k][d] = t.by_level[k][d];
            t.by_level[k][d] = 0;
        }
        t.ms[k] = 0;
        t.launches[k] = 0;
    }
}

TimedScope::TimedScope(int k, cudaStream_t s) : kind(k), level(g_timing_level), stream(s) {
    TimingState& t = timing();
    std::lock_guard<std::mutex> lk(t.mu);
    if (!t.on) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return;  // no timing events inside a graph capture
    }
    start = t.get();
    cudaEventRecord(start, s);
}

TimedScope::~TimedScope() {
    if (!start) return;
    TimingState& t = timing();
    std::lock_guard<std::mutex> lk(t.mu);
    cudaEvent_t end = t.get();
    cudaEventRecord(end, stream);
    t.pending.emplace_back(kind, level, start, end);
}

namespace {
std::mutex g_pool_mutex;
std::vector<std::pair<int, cudaMemPool_t>> g_pools;
}  // namespace

cudaMemPool_t device_pool(int device) {
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    for (auto& e : g_pools)
        if (e.first == device) return e.second;
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool = nullptr;
    IFGF_CUDA(cudaMemPoolCreate(&pool, &props));
    size_t free_b = 0, total_b = 0;
    IFGF_CUDA(cudaMemGetInfo(&free_b, &total_b));
    uint64_t keep = total_b / 4;
    IFGF_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    g_pools.emplace_back(device, pool);
    return pool;
}

size_t pool_cached_bytes(int device) {
    cudaMemPool_t pool = device_pool(device);
    uint64_t reserved = 0, used = 0;
    cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved);
    cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used);
    return reserved > used ? (size_t)(reserved - used) : 0;
}

void destroy_plan(Plan& p) {
    for (size_t i = p.allocs.size(); i-- > 0;) cudaFreeAsync(p.allocs[i], p.stream);
    p.allocs.clear();
    cudaStreamSynchronize(p.stream);
}

namespace {

// Analysis matrix W[n][j] = (2 - delta_{n0})/P cos(n (2j+1) pi / (2P)) of the Chebyshev
// interpolant on first-kind nodes ("generate interpolant", Algorithm 1).
void analysis(int P, std::vector<double>& W) {
    for (int n = 0; n < P; ++n)
        for (int j = 0; j < P; ++j)
            W.push_back((n == 0 ? 1.0 : 2.0) / P * std::cos(M_PI * n * (2.0 * j + 1.0) / (2.0 * P)));
}

ifgf_status guard(const std::function<void()>& f) {
    try {
        f();
        return IFGF_OK;
    } catch (const Error& e) {
        set_last_error(e.what);
        return e.status;
    } catch (const std::bad_alloc&) {
        set_last_error("host allocation failed");
        return IFGF_ERR_OOM;
    } catch (...) {
        set_last_error("unexpected exception");
        return IFGF_ERR_INTERNAL;
    }
}
}  // namespace

ifgf_status guard_call(const std::function<void()>& f) { return guard(f); }

}  // namespace ifgf

// The opaque handle of the C ABI is the plan itself.
struct ifgf_plan_s : public ifgf::Plan {};

namespace ifgf {
Plan* plan_of(ifgf_plan p) { return p; }
}  // namespace ifgf

using namespace ifgf;

extern "C" {

void ifgf_options_default(ifgf_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->struct_size = (int32_t)sizeof(ifgf_options);
    opt->precision = IFGF_PREC_MIXED;
    opt->base_cones[0] = 2;
    opt->base_cones[1] = 4;
    opt->base_cones[2] = 8;
    opt->leaf_target = 64;
    opt->max_nrhs = 1;
    opt->tau = 0.5;
}

ifgf_status ifgf_plan_create(const double* points, int64_t N, double kappa, const int32_t* orders, int32_t levels,
                             const ifgf_options* opt_in, void* stream, ifgf_plan* out_plan) {
    if (!out_plan) {
        set_last_error("out_plan is NULL");
        return IFGF_ERR_INVALID_ARG;
    }
    ifgf_options opt;
    ifgf_options_default(&opt);
    if (opt_in) {
        if (opt_in->struct_size != (int32_t)sizeof(ifgf_options)) {
            set_last_error("ifgf_options.struct_size mismatch");
            return IFGF_ERR_INVALID_ARG;
        }
        opt = *opt_in;
    }
    const int Ps = orders ? orders[0] : 3, Pt = orders ? orders[1] : 5, Pp = orders ? orders[2] : 5;
    std::string why;
    if (!points) why = "points is NULL";
    else if (N < 2 || N >= ((int64_t)1 << 31) - 1) why = "N out of range [2, 2^31)";
    else if (!(kappa >= 0.0) || !std::isfinite(kappa)) why = "kappa must be finite and >= 0";
    else if (levels != 0 && (levels < 3 || levels > kMaxLevel)) why = "levels must be 0 or in [3, 21]";
    else if (opt.precision != IFGF_PREC_FP64 && opt.precision != IFGF_PREC_MIXED) why = "unknown precision";
    else if (opt.base_cones[0] < 1 || opt.base_cones[1] < 1 || opt.base_cones[2] < 4 || (opt.base_cones[2] & 1))
        why = "base_cones must be >= (1, 1, 4) with an even azimuthal count";
    else if (opt.leaf_target < 1) why = "leaf_target must be >= 1";
    else if (opt.max_nrhs < 1 || opt.max_nrhs > 65535) why = "max_nrhs out of range";
    else if (opt.rhs_block < 0) why = "rhs_block must be >= 0";
    else if (opt.cone_table < 0 || opt.cone_table > 2) why = "cone_table must be 0, 1 or 2";
    else if (opt.prop_slices < 0 || opt.prop_slices > 4096) why = "prop_slices must be in [0, 4096]";
    else if (!(opt.tau > 0.0) || !std::isfinite(opt.tau)) why = "tau must be finite and > 0";
    else if (Ps < 1 || Pt < 1 || Pp < 1) why = "orders must be >= 1";
    if (!why.empty()) {
        set_last_error(why);
        return IFGF_ERR_INVALID_ARG;
    }
    if (!((Ps == 3 && Pt == 5 && Pp == 5) || (Ps == 5 && Pt == 7 && Pp == 7))) {
        set_last_error("orders other than (3,5,5) and (5,7,7) are not built");
        return IFGF_ERR_UNSUPPORTED;
    }
    ifgf_plan_s* p = nullptr;
    ifgf_status st = guard([&] {
        p = new ifgf_plan_s();
        p->N = N;
        p->kappa = kappa;
        p->Ps = Ps;
        p->Pt = Pt;
        p->Pp = Pp;
        p->P = Ps * Pt * Pp;
        p->precision = opt.precision;
        p->max_nrhs = opt.max_nrhs;
        p->cstride = p->precision == IFGF_PREC_MIXED ? ((p->P + 1) & ~1) : p->P;
        p->stream = (cudaStream_t)stream;
        IFGF_CUDA(cudaGetDevice(&p->device));
        {
            cudaPointerAttributes attr;
            IFGF_CUDA(cudaPointerGetAttributes(&attr, points));
            if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
                fail(IFGF_ERR_INVALID_ARG, "points must be device memory");
        }
        p->d_status = dalloc<int>(*p, 1);
        IFGF_CUDA(cudaMemsetAsync(p->d_status, 0, sizeof(int), p->stream));
        {
            TimedScope ts_(TK_PLAN, p->stream);
            build_plan(*p, points, opt, levels);
        }
        std::vector<double> W;
        analysis(Ps, W);
        analysis(Pt, W);
        analysis(Pp, W);
        std::vector<float> Wf(W.begin(), W.end());
        p->Wd = dalloc<double>(*p, W.size());
        p->Wf = dalloc<float>(*p, Wf.size());
        IFGF_CUDA(cudaMemcpyAsync(p->Wd, W.data(), sizeof(double) * W.size(), cudaMemcpyHostToDevice, p->stream));
        IFGF_CUDA(cudaMemcpyAsync(p->Wf, Wf.data(), sizeof(float) * Wf.size(), cudaMemcpyHostToDevice, p->stream));
        const size_t csz = p->precision == IFGF_PREC_MIXED ? sizeof(float2) : sizeof(double2);
        // Coefficient arena for a block of densities: half of the free device memory when that
        // holds it, else up to 90% (minus the density and output buffers); ifgf_apply sweeps the
        // levels once per block (a multiple of 4 densities when blocked).
        {
            size_t free_b = 0, total_b = 0;
            IFGF_CUDA(cudaMemGetInfo(&free_b, &total_b));
            free_b += pool_cached_bytes(p->device);  // memory the pool holds for reuse
            const size_t io = 2 * (size_t)N * p->max_nrhs * csz + ((size_t)1 << 28);
            const size_t usable = free_b > io ? free_b - io : 0;
            int64_t M = layout_arena(*p, usable / 2, opt.prop_slices);
            size_t budget = usable / 2;
            if (M == 0) {
                budget = usable / 10 * 9;
                M = layout_arena(*p, budget, opt.prop_slices);
            }
            if (M == 0) fail(IFGF_ERR_OOM, "the coefficient arena of one density does not fit in device memory");
            p->arena_cones = M;
            const size_t per_rhs = (size_t)M * p->cstride * csz;
            const size_t fit = std::max<size_t>(1, budget / std::max<size_t>(per_rhs, 1));
            int blk = (int)std::min<size_t>((size_t)p->max_nrhs, fit);
            if (blk < p->max_nrhs && blk >= 8) blk &= ~3;
            if (opt.rhs_block > 0) blk = std::min(opt.rhs_block, p->max_nrhs);
            p->rhs_block = std::max(1, blk);
        }
        p->arena = dalloc<char>(*p, (size_t)p->arena_cones * p->rhs_block * p->cstride * csz);
        p->a_s = dalloc<char>(*p, (size_t)N * p->max_nrhs * csz);
        p->I_s = dalloc<char>(*p, (size_t)N * p->max_nrhs * csz);
        IFGF_CUDA(cudaStreamSynchronize(p->stream));
    });
    if (st != IFGF_OK) {
        if (p) {
            destroy_plan(*p);
            delete p;
        }
        return st;
    }
    *out_plan = p;
    return IFGF_OK;
}

ifgf_status ifgf_apply_ex(ifgf_plan plan, const void* densities, int32_t nrhs, void* out, void* stream,
                          int32_t near, int64_t level_mask) {
    if (!plan || !densities || !out) {
        set_last_error("NULL plan, densities or out");
        return IFGF_ERR_INVALID_ARG;
    }
    if (nrhs < 1 || nrhs > plan->max_nrhs) {
        set_last_error("nrhs must be in [1, max_nrhs]");
        return IFGF_ERR_INVALID_ARG;
    }
    if (densities == out) {
        set_last_error("out must not alias densities");
        return IFGF_ERR_INVALID_ARG;
    }
    return guard([&] {
        IFGF_CUDA(cudaSetDevice(plan->device));
        apply_plan(*plan, densities, nrhs, out, (cudaStream_t)stream, near != 0, level_mask);
    });
}

ifgf_status ifgf_apply(ifgf_plan plan, const void* densities, int32_t nrhs, void* out, void* stream) {
    return ifgf_apply_ex(plan, densities, nrhs, out, stream, 1, -1);
}

namespace {

// Shared checks and dispatch of the tensor-kernel applies (Stokeslet, Kelvin's solution).
ifgf_status apply_tensor(ifgf_plan plan, const void* forces, int32_t nfield, void* out, void* stream, int32_t near,
                         int64_t level_mask, const TensorKernel& tk, const char* name) {
    if (!plan || !forces || !out) {
        set_last_error("NULL plan, forces or output");
        return IFGF_ERR_INVALID_ARG;
    }
    if (forces == out) {
        set_last_error("the output must not alias the forces");
        return IFGF_ERR_INVALID_ARG;
    }
    if (plan->kappa != 0.0) {
        set_last_error(std::string("the ") + name + " kernel needs a plan created with kappa = 0");
        return IFGF_ERR_INVALID_ARG;
    }
    if (nfield < 1 || (3 * (int64_t)nfield + 1) / 2 > plan->max_nrhs) {
        set_last_error("nfield must be in [1, 2 max_nrhs / 3]");
        return IFGF_ERR_INVALID_ARG;
    }
    return guard([&] {
        IFGF_CUDA(cudaSetDevice(plan->device));
        apply_plan_stokes(*plan, forces, nfield, out, tk, (cudaStream_t)stream, near != 0, level_mask);
    });
}

}  // namespace

ifgf_status ifgf_apply_stokes_ex(ifgf_plan plan, const void* forces, int32_t nfield, void* velocity, void* stream,
                                 int32_t near, int64_t level_mask) {
    return apply_tensor(plan, forces, nfield, velocity, stream, near, level_mask, TensorKernel{}, "Stokes");
}

ifgf_status ifgf_apply_stokes(ifgf_plan plan, const void* forces, int32_t nfield, void* velocity, void* stream) {
    return ifgf_apply_stokes_ex(plan, forces, nfield, velocity, stream, 1, -1);
}

ifgf_status ifgf_apply_elastic_ex(ifgf_plan plan, const void* forces, int32_t nfield, void* displacement,
                                  double shear_modulus, double poisson_ratio, void* stream, int32_t near,
                                  int64_t level_mask) {
    if (!(shear_modulus > 0.0) || !std::isfinite(shear_modulus) || !(poisson_ratio > -1.0) ||
        !(poisson_ratio <= 0.5)) {
        set_last_error("shear_modulus must be finite and > 0, poisson_ratio in (-1, 0.5]");
        return IFGF_ERR_INVALID_ARG;
    }
    TensorKernel tk;
    tk.c = 1.0 / (16.0 * M_PI * shear_modulus * (1.0 - poisson_ratio));
    tk.alpha = 3.0 - 4.0 * poisson_ratio;
    return apply_tensor(plan, forces, nfield, displacement, stream, near, level_mask, tk, "elasticity");
}

ifgf_status ifgf_apply_elastic(ifgf_plan plan, const void* forces, int32_t nfield, void* displacement,
                               double shear_modulus, double poisson_ratio, void* stream) {
    return ifgf_apply_elastic_ex(plan, forces, nfield, displacement, shear_modulus, poisson_ratio, stream, 1, -1);
}

ifgf_status ifgf_plan_destroy(ifgf_plan plan) {
    if (!plan) return IFGF_OK;
    ifgf_status st = guard([&] {
        cudaSetDevice(plan->device);
        destroy_plan(*plan);
    });
    delete plan;
    return st;
}

ifgf_status ifgf_plan_query(ifgf_plan plan, int32_t what, int32_t level, int64_t* host_buf, int64_t* inout_count) {
    if (!plan || !inout_count) {
        set_last_error("NULL plan or count");
        return IFGF_ERR_INVALID_ARG;
    }
    Plan& p = *plan;
    if (level < 0 || level > kMaxLevel) {
        set_last_error("level out of range");
        return IFGF_ERR_INVALID_ARG;
    }
    std::vector<int64_t> res;
    ifgf_status st = guard([&] {
        IFGF_CUDA(cudaSetDevice(p.device));
        IFGF_CUDA(cudaDeviceSynchronize());
        auto get32 = [&](const int32_t* d, int64_t n) {
            std::vector<int32_t> h((size_t)std::max<int64_t>(n, 0));
            if (n > 0) IFGF_CUDA(cudaMemcpy(h.data(), d, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
            return h;
        };
        const bool lev_ok = level >= 1 && level <= p.D;
        const Level& L = p.L[lev_ok ? level : 1];
        auto need = [&](bool ok) {
            if (!ok) fail(IFGF_ERR_INVALID_ARG, "item unavailable at this level");
        };
        switch (what) {
            case IFGF_Q_PERM: {
                auto h = get32(p.perm, p.N);
                res.assign(h.begin(), h.end());
                break;
            }
            case IFGF_Q_KEYS: {
                std::vector<uint64_t> h((size_t)p.N);
                IFGF_CUDA(cudaMemcpy(h.data(), p.key, sizeof(uint64_t) * p.N, cudaMemcpyDeviceToHost));
                res.assign(h.begin(), h.end());
                break;
            }
            case IFGF_Q_BOX_KEYS: {
                need(lev_ok);
                std::vector<uint64_t> h((size_t)L.n);
                IFGF_CUDA(cudaMemcpy(h.data(), L.key, sizeof(uint64_t) * L.n, cudaMemcpyDeviceToHost));
                res.assign(h.begin(), h.end());
                break;
            }
            case IFGF_Q_BOX_START: {
                need(lev_ok);
                auto h = get32(L.start, (int64_t)L.n + 1);
                res.assign(h.begin(), h.end());
                break;
            }
            case IFGF_Q_BOX_PARENT: {
                need(lev_ok);
                auto h = get32(L.parent, L.n);
                res.assign(h.begin(), h.end());
                break;
            }
            case IFGF_Q_BOX_COORDS: {
                need(lev_ok);
                std::vector<int4> h((size_t)L.n);
                IFGF_CUDA(cudaMemcpy(h.data(), L.k, sizeof(int4) * L.n, cudaMemcpyDeviceToHost));
                for (const int4& v : h) res.insert(res.end(), {v.x, v.y, v.z});
                break;
            }
            case IFGF_Q_CHILD_START: {
                need(lev_ok);
                auto h = get32(L.cstart, (int64_t)L.n + 1);
                res.assign(h.begin(), h.end());
                break;
            }
            case IFGF_Q_NBR_COUNT:
            case IFGF_Q_NBR_LIST: {
                need(lev_ok && level >= 2);
                auto c = get32(L.nnb, L.n);
                if (what == IFGF_Q_NBR_COUNT) {
                    res.assign(c.begin(), c.end());
                } else {
                    auto l = get32(L.nb, (int64_t)L.n * kMaxNbr);
                    for (int64_t b = 0; b < L.n; ++b)
                        for (int t = 0; t < c[b]; ++t) res.push_back(l[b * kMaxNbr + t]);
                }
                break;
            }
            case IFGF_Q_COUS_COUNT:
            case IFGF_Q_COUS_LIST: {
                need(lev_ok && level >= 3);
                auto c = get32(L.ncs, L.n);
                if (what == IFGF_Q_COUS_COUNT) {
                    res.assign(c.begin(), c.end());
                } else {
                    auto l = get32(L.cs, (int64_t)L.n * kMaxCous);
                    for (int64_t b = 0; b < L.n; ++b)
                        for (int t = 0; t < c[b]; ++t) res.push_back(l[b * kMaxCous + t]);
                }
                break;
            }
            case IFGF_Q_CONE_BOX: {
                need(lev_ok && level >= 3);
                auto h = get32(L.cone_box, L.nc);
                res.assign(h.begin(), h.end());
                break;
            }
            case IFGF_Q_CONE_GAMMA: {
                need(lev_ok && level >= 3);
                auto h = get32(L.cone_gam, L.nc);
                res.assign(h.begin(), h.end());
                break;
            }
            case IFGF_Q_GRID: {
                need(lev_ok && level >= 3);
                res.assign(L.host_grid.begin(), L.host_grid.end());
                break;
            }
            case IFGF_Q_INFO: {
                res.assign(44, 0);
                res[0] = p.N;
                res[1] = p.D;
                for (int d = 1; d <= p.D; ++d) {
                    res[1 + d] = p.L[d].n;
                    if (d >= 3) res[22 + d] = p.L[d].nc;
                }
                break;
            }
            case IFGF_Q_WORK: {
                // Exact work of one apply: near pairs, leaf pairs (whole plan); interpolation and
                // propagation evaluations of the requested level.
                need(lev_ok && level >= 3);
                const Level& LD = p.L[p.D];
                auto sD = get32(LD.start, (int64_t)LD.n + 1);
                auto cD = get32(LD.nnb, LD.n);
                auto lD = get32(LD.nb, (int64_t)LD.n * kMaxNbr);
                int64_t near = 0;
                for (int64_t b = 0; b < LD.n; ++b) {
                    int64_t nbpts = 0;
                    for (int t = 0; t < cD[b]; ++t) {
                        const int q = lD[b * kMaxNbr + t];
                        nbpts += sD[q + 1] - sD[q];
                    }
                    near += (int64_t)(sD[b + 1] - sD[b]) * nbpts;
                }
                near -= p.N;
                auto cbD = get32(LD.cone_box, LD.nc);
                int64_t leaf = 0;
                for (int64_t c = 0; c < LD.nc; ++c) leaf += (int64_t)p.P * (sD[cbD[c] + 1] - sD[cbD[c]]);
                auto st_ = get32(L.start, (int64_t)L.n + 1);
                auto nc = get32(L.ncs, L.n);
                int64_t interp = 0;
                for (int64_t b = 0; b < L.n; ++b) interp += (int64_t)(st_[b + 1] - st_[b]) * nc[b];
                int64_t prop = 0;
                if (level > 3) {
                    const Level& Lp = p.L[level - 1];
                    auto cb = get32(Lp.cone_box, Lp.nc);
                    auto cst = get32(Lp.cstart, (int64_t)Lp.n + 1);
                    for (int64_t c = 0; c < Lp.nc; ++c) prop += (int64_t)p.P * (cst[cb[c] + 1] - cst[cb[c]]);
                }
                res = {near, leaf, interp, prop};
                break;
            }
            case IFGF_Q_TABLES: {
                need(lev_ok && level >= 3);
                res = {(int64_t)L.n_gam};
                break;
            }
            case IFGF_Q_STATUS: {
                int h = 0;
                IFGF_CUDA(cudaMemcpy(&h, p.d_status, sizeof(int), cudaMemcpyDeviceToHost));
                res = {h};
                break;
            }
            default:
                fail(IFGF_ERR_INVALID_ARG, "unknown query");
        }
    });
    if (st != IFGF_OK) return st;
    const int64_t cap = *inout_count;
    *inout_count = (int64_t)res.size();
    if (host_buf && cap >= (int64_t)res.size() && !res.empty())
        std::memcpy(host_buf, res.data(), sizeof(int64_t) * res.size());
    return IFGF_OK;
}

const char* ifgf_status_string(ifgf_status s) {
    switch (s) {
        case IFGF_OK: return "ok";
        case IFGF_ERR_INVALID_ARG: return "invalid argument";
        case IFGF_ERR_OOM: return "out of device memory";
        case IFGF_ERR_CUDA: return "CUDA error";
        case IFGF_ERR_TIMEOUT: return "device wait timed out";
        case IFGF_ERR_INTERNAL: return "internal consistency check failed";
        case IFGF_ERR_UNSUPPORTED: return "unsupported by this build";
    }
    return "unknown status";
}

const char* ifgf_last_error(void) { return t_last_error.c_str(); }

int64_t ifgf_launch_count(void) { return g_launches.load(); }

void ifgf_debug_fail_allocation(int64_t n) { g_fail_alloc_in.store(n > 0 ? n : 0); }

int32_t ifgf_checked_build(void) { return kChecks ? 1 : 0; }

ifgf_status ifgf_debug_corrupt_cousin(ifgf_plan plan, int32_t level) {
    if (!kChecks) {
        set_last_error("corrupting a list is allowed in checked builds only");
        return IFGF_ERR_UNSUPPORTED;
    }
    if (!plan || level < 3 || level > plan->D) {
        set_last_error("NULL plan or level outside [3, D]");
        return IFGF_ERR_INVALID_ARG;
    }
    Plan& p = *plan;
    return guard([&] {
        IFGF_CUDA(cudaSetDevice(p.device));
        IFGF_CUDA(cudaDeviceSynchronize());
        Level& L = p.L[level];
        std::vector<int32_t> cnt((size_t)L.n);
        IFGF_CUDA(cudaMemcpy(cnt.data(), L.ncs, sizeof(int32_t) * L.n, cudaMemcpyDeviceToHost));
        for (int32_t b = 0; b < L.n; ++b)
            if (cnt[b] > 0) {
                const int32_t bad = L.n + 7;  // a box index past the level's boxes
                IFGF_CUDA(cudaMemcpy(L.cs + (int64_t)b * kMaxCous, &bad, sizeof(int32_t), cudaMemcpyHostToDevice));
                return;
            }
        fail(IFGF_ERR_INVALID_ARG, "no box of the level has a cousin");
    });
}

ifgf_status ifgf_permute(ifgf_plan plan, const void* in, int32_t nrhs, void* out, int32_t to_sorted, void* stream) {
    if (!plan || !in || !out || in == out || nrhs < 1) {
        set_last_error("permute: NULL or aliased buffers, or nrhs < 1");
        return IFGF_ERR_INVALID_ARG;
    }
    return guard([&] {
        IFGF_CUDA(cudaSetDevice(plan->device));
        permute_points(*plan, in, nrhs, out, to_sorted != 0, (cudaStream_t)stream);
    });
}

ifgf_status ifgf_plan_set_knob(ifgf_plan plan, int32_t knob, int32_t level, int32_t value) {
    if (!plan) {
        set_last_error("NULL plan");
        return IFGF_ERR_INVALID_ARG;
    }
    Plan& p = *plan;
    if (knob == IFGF_KNOB_RHS_BLOCK) {
        if (value != -1 && value != 8 && value != 16 && value != 32) {
            set_last_error("densities per block must be 8, 16 or 32 (or -1)");
            return IFGF_ERR_INVALID_ARG;
        }
        p.knob_block = value;
        return IFGF_OK;
    }
    if (knob != IFGF_KNOB_PROP_MANY && knob != IFGF_KNOB_PROP_FEW) {
        set_last_error("unknown knob");
        return IFGF_ERR_INVALID_ARG;
    }
    if (level < 4 || level > p.D || value < -1 || value > 1) {
        set_last_error("knob level must be in [4, D] and its value in {-1, 0, 1}");
        return IFGF_ERR_INVALID_ARG;
    }
    (knob == IFGF_KNOB_PROP_MANY ? p.L[level].knob_many : p.L[level].knob_few) = (int8_t)value;
    return IFGF_OK;
}

ifgf_status ifgf_plan_get_knob(ifgf_plan plan, int32_t knob, int32_t level, int32_t* value) {
    if (!plan || !value) {
        set_last_error("NULL plan or value pointer");
        return IFGF_ERR_INVALID_ARG;
    }
    Plan& p = *plan;
    if (knob == IFGF_KNOB_RHS_BLOCK) {
        *value = p.knob_block;
        return IFGF_OK;
    }
    if ((knob != IFGF_KNOB_PROP_MANY && knob != IFGF_KNOB_PROP_FEW) || level < 4 || level > p.D) {
        set_last_error("unknown knob or level out of [4, D]");
        return IFGF_ERR_INVALID_ARG;
    }
    const Level& L = p.L[level];
    const int v = knob == IFGF_KNOB_PROP_MANY ? L.knob_many : L.knob_few;
    *value = p.L[level - 1].n_gam > 0 ? (v < 0 ? 0 : v) : -1;
    return IFGF_OK;
}

ifgf_status ifgf_debug_drop_cone(ifgf_plan plan, int32_t level, int64_t cone) {
    if (!plan) {
        set_last_error("NULL plan");
        return IFGF_ERR_INVALID_ARG;
    }
    Plan& p = *plan;
    if (level < 3 || level > p.D || cone < 0 || cone >= p.L[level].nc) {
        set_last_error("level or cone out of range");
        return IFGF_ERR_INVALID_ARG;
    }
    Level& L = p.L[level];
    if (!L.slot) {
        set_last_error("the level keeps sorted cone lists, not a dense table");
        return IFGF_ERR_UNSUPPORTED;
    }
    return guard([&] {
        IFGF_CUDA(cudaSetDevice(p.device));
        IFGF_CUDA(cudaDeviceSynchronize());
        int32_t box = 0, gam = 0;
        IFGF_CUDA(cudaMemcpy(&box, L.cone_box + cone, sizeof(int32_t), cudaMemcpyDeviceToHost));
        IFGF_CUDA(cudaMemcpy(&gam, L.cone_gam + cone, sizeof(int32_t), cudaMemcpyDeviceToHost));
        const int32_t none = -1;
        IFGF_CUDA(cudaMemcpy(L.slot + (int64_t)box * L.g.C + gam, &none, sizeof(int32_t), cudaMemcpyHostToDevice));
    });
}

void ifgf_timing_enable(int32_t on) {
    TimingState& t = timing();
    std::lock_guard<std::mutex> lk(t.mu);
    t.on = on != 0;
}

ifgf_status ifgf_release_cached_memory(void) {
    std::vector<std::pair<int, cudaMemPool_t>> pools;
    {
        std::lock_guard<std::mutex> lock(g_pool_mutex);
        pools = g_pools;
    }
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto& e : pools) {
        if (cudaSetDevice(e.first) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemPoolTrimTo(e.second, 0) != cudaSuccess) {
            set_last_error(std::string("releasing cached memory: ") + cudaGetErrorString(cudaGetLastError()));
            cudaSetDevice(cur);
            return IFGF_ERR_CUDA;
        }
    }
    cudaSetDevice(cur);
    return IFGF_OK;
}

ifgf_status ifgf_timing_collect(double* ms, int64_t* launches) {
    return guard([&] { timing_collect_levels(ms, launches, nullptr); });
}

}  // extern "C"
