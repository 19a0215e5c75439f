// Batched apply of many plans (mixed precision, orders (3,5,5), one density each) as one short
// launch sequence over work queues that span all problems of the batch:
//   permutation in | near field | LevelDEvaluations | propagation | interpolation | permutation out.
// Each launch takes its work units (leaf boxes, groups of parent cones, blocks of targets) from
// a list that mixes every problem, largest first, so small problems fill the GPU together
// instead of each running a sequence of nearly empty launches.
//
// The propagation is one persistent kernel for all levels of all problems: its blocks take
// items (a problem, a level d, a run of parent cones at level d-1) from a queue ordered by the
// distance of d from the problem's leaf level, and an item whose child level is not complete
// waits on the problem's per-level completion counter (Algorithm 7 reads every child cone).
// Items only wait on items earlier in the queue, which running blocks hold, so every wait ends;
// the waits are nonetheless bounded: after wait_limit polls a block records IFGF_ERR_TIMEOUT in
// the batch's status word and skips its item, and every later wait gives up at once.
//
// Every work unit runs the device bodies of the single-plan kernels (bodies_f32.cuh) on the
// same data, so each problem's result is bit-identical to its own ifgf_apply.  Coefficients of
// all levels are kept (the single-plan arena reuses its storage level by level, which a queue
// that runs levels of different problems side by side cannot), and the propagation reads child
// coefficients written during the same launch with ordinary loads after the acquire of its wait
// (never through the read-only path).
#include <algorithm>
#include <numeric>

#include "batch_queue.cuh"
#include "bodies_f32.cuh"

namespace ifgf {
namespace {

constexpr int kQP = 75;  // orders (3,5,5)
constexpr int kMaxPhases = 2 * kMaxLevel;  // propagation launches (runs of one kernel kind)

// Level d of problem p: its interpolation and its propagation into level d-1.
struct QLevel {
    // interpolation to the targets of level d
    const int32_t* pbox = nullptr;   // [N] box of every sorted point at level d
    const int4* k = nullptr;
    const int32_t* ncs = nullptr;
    const int32_t* cs = nullptr;
    ConeMap cm{};
    LevelGrid g{};
    const float* phtab = nullptr;
    const float2* coef = nullptr;    // coefficients of level d (batch storage)
    float2* iacc = nullptr;          // [N] the level-d interpolation sums of the targets
    int sh = 0;
    int problem = 0;
    float ku = 0;                    // kappa u of the problem
    // propagation into level d-1 (ncp = 0: none)
    int64_t ncp = 0;
    int tabled = 0;
    const int32_t* pcone_box = nullptr;
    const int32_t* pcone_gam = nullptr;
    const int32_t* cone_gidx = nullptr;
    const int4* kp = nullptr;
    const int32_t* pcstart = nullptr;
    LevelGrid gp{};
    const float4* tab_t = nullptr;
    const float2* tab_r = nullptr;
    const int32_t* tab_k = nullptr;
    const int32_t* tab_list = nullptr;
    const int16_t* tab_perm = nullptr;
    const int32_t* tab_nseg = nullptr;
    const int32_t* tab_seg = nullptr;
    float2* cparent = nullptr;
};

// Problem p: its leaf level, points and buffers.
struct QProblem {
    int64_t N = 0;
    int D = 0;
    int lv0 = 0;                     // QLevel index of level 3 (level d at lv0 + d - 3)
    float ku = 0, inv4piu = 0, kh = 0, hinv = 0;
    const int32_t* perm = nullptr;
    const float4* off = nullptr;
    float2* as = nullptr;
    float2* Is = nullptr;
    const int4* kD = nullptr;
    const int32_t* startD = nullptr;
    const int32_t* nnb = nullptr;
    const int32_t* nb = nullptr;
    const int32_t* bcs = nullptr;
    const int32_t* pboxD = nullptr;
    const int32_t* cone_gamD = nullptr;
    LevelGrid gD{};
    int ncD = 0;
    float2* coefD = nullptr;
    const float* W = nullptr;
    int cstride = 0;
    int* status = nullptr;
};

struct QItem {
    int32_t lv;   // QLevel of the propagation
    int32_t dep;  // counter that must reach need[dep] first (-1: none)
    int32_t c0, c1;  // parent cones [c0, c1) at level d-1
};

// ---- elementwise and one-block-per-unit launches --------------------------------------------
// Units are (problem, first index or box) pairs.
__global__ void __launch_bounds__(256) k_q_perm_in(const QProblem* __restrict__ pb, const int2* __restrict__ units,
                                                   const float2* const* __restrict__ dens) {
    const int2 u = units[blockIdx.x];
    const QProblem& P = pb[u.x];
    const int64_t i = (int64_t)u.y + threadIdx.x;
    if (i >= P.N) return;
    P.as[i] = dens[u.x][P.perm[i]];
}

// The near-field sum plus the level sums D, D-1, ..., 3, added in that order (the order in which
// the single-plan sweep adds them to its output, so that the sums round identically), written in
// the caller's point order.
__global__ void __launch_bounds__(256) k_q_perm_out(const QProblem* __restrict__ pb, const QLevel* __restrict__ lv,
                                                    const int2* __restrict__ units, float2* const* __restrict__ outs) {
    const int2 u = units[blockIdx.x];
    const QProblem& P = pb[u.x];
    const int64_t i = (int64_t)u.y + threadIdx.x;
    if (i >= P.N) return;
    float2 v = P.Is[i];
    for (int d = P.D; d >= 3; --d) {
        const float2 a = lv[P.lv0 + d - 3].iacc[i];
        v = make_float2(v.x + a.x, v.y + a.y);
    }
    outs[u.x][P.perm[i]] = v;
}

__global__ void __launch_bounds__(kNearThreads) k_q_near(const QProblem* __restrict__ pb, const int2* __restrict__ units) {
    const int2 u = units[blockIdx.x];
    const QProblem& P = pb[u.x];
    near_box_f32(P.kD, P.startD, P.nnb, P.nb, P.off, P.as, P.Is, P.N, P.ku, P.inv4piu, u.y, 0);
}

__global__ void __launch_bounds__(kLeafThreads) k_q_leaf(const QProblem* __restrict__ pb, const int2* __restrict__ units) {
    const int2 u = units[blockIdx.x];
    const QProblem& P = pb[u.x];
    leaf_box_f32<3, 5, 5>(P.bcs, P.cone_gamD, P.gD, P.startD, P.off, P.as, P.N, P.kh, P.hinv, P.W, P.coefD, P.cstride,
                          1, u.y, 0, 0, P.ncD);
}

// Interpolation (Algorithm 8) of 256 targets of one level of one problem (unit: QLevel, first
// target) into that level's sums.
__global__ void __launch_bounds__(256, 4) k_q_interp(const QProblem* __restrict__ pb, const QLevel* __restrict__ lv,
                                                     const int2* __restrict__ units) {
    const int2 u = units[blockIdx.x];
    const QLevel& L = lv[u.x];
    const QProblem& P = pb[L.problem];
    const int64_t i = (int64_t)u.y + threadIdx.x;
    if (i >= P.N) return;
    float2 acc[1];
    interp_target_f32<3, 5, 5, 1, false, const ConeMap&, const LevelGrid&>(i, 0, 1, L.sh, L.pbox, P.pboxD, P.kD, L.k, L.ncs, L.cs, P.off, L.cm, L.g,
                                         L.coef, L.phtab, P.ku, P.inv4piu, P.cstride, 1, P.status, acc);
    L.iacc[i] = acc[0];
}

// ---- the persistent propagation -------------------------------------------------------------
__device__ __forceinline__ int load_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0 waits until the counter reaches target: false after `limit` polls (recording
// IFGF_ERR_TIMEOUT) or as soon as another block has recorded a failure.
__device__ bool wait_counter(const int* counter, int target, int64_t limit, int* bstatus) {
    for (int64_t it = 0;; ++it) {
        if (load_acquire(counter) >= target) return true;
        if ((it & 63) == 63 && load_acquire(bstatus) != 0) return false;
        if (it >= limit) {
            atomicCAS(bstatus, 0, (int)IFGF_ERR_TIMEOUT);
            return false;
        }
        __nanosleep(256);
    }
}

// The persistent propagation over one run of levels of one kind: kTab, levels whose parent level
// has node tables, one warp per parent cone, kWarpCones warps per block (the standalone node-table
// kernel's shape); otherwise the per-cone kernel's block of kPropThreads threads and kPropCones
// cones per step.  ctr: the next item of this launch; done: completed items per QLevel; need:
// items per QLevel.
template <bool kTab>
__global__ void __launch_bounds__(kTab ? 32 * kWarpCones : kPropThreads, kTab ? 8 : 5)
k_q_prop(const QLevel* __restrict__ lv, const QItem* __restrict__ items, int nitems, const int* __restrict__ need,
         int* head, int* done, int* bstatus, const float* __restrict__ W, int cstride, int64_t limit, int withhold) {
    __shared__ int s_item, s_ok;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(head, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const QItem q = items[it];
        if (tid == 0) s_ok = q.dep < 0 || wait_counter(done + q.dep, need[q.dep], limit, bstatus);
        __syncthreads();  // with the acquire of thread 0: the child level is visible to the block
        if (s_ok) {
            const QLevel& L = lv[q.lv];
            if constexpr (kTab) {
                __shared__ WarpSmem<kQP> ws[kWarpCones];
                const int warp = tid >> 5;
                for (int64_t pc = q.c0 + warp; pc < q.c1; pc += kWarpCones)
                    prop_cone_warp_f32<3, 5, 5, 1, true, WarpSmem<kQP>>(
                        &ws[warp], q.c1, L.pcone_box, L.cone_gidx, L.kp, L.pcstart, L.k, L.cm, L.tab_t, L.tab_r,
                        L.tab_k, L.tab_list, L.tab_perm, L.tab_nseg, L.tab_seg, L.coef, L.cparent, W, cstride, 1,
                        L.cm.status, pc, tid & 31);
            } else {
                __shared__ PropSmem<kQP> gs;
                for (int64_t pc0 = q.c0; pc0 < q.c1; pc0 += kPropCones) {
                    prop_cones_f32<3, 5, 5, true>(gs, q.c1, L.pcone_box, L.pcone_gam, L.kp, L.pcstart, L.gp, L.k,
                                                  L.cm, L.g, L.coef, L.cparent, L.sh, L.ku, W, cstride, 1,
                                                  L.cm.status, pc0, 0);
                    __syncthreads();  // the next pair reuses the block's shared memory
                }
            }
            __threadfence();  // this thread's coefficients, device-wide, before the count
        }
        __syncthreads();
        if (tid == 0 && s_ok && it != withhold) atomicAdd(done + q.lv, 1);
    }
}

}  // namespace

struct BatchQueue {
    std::vector<Plan*> plans;
    int device = 0;
    int nsm = 0;
    std::vector<QProblem> hp;
    std::vector<QLevel> hl;
    std::vector<QItem> hitems;
    std::vector<int> hneed;
    std::vector<int64_t> first_item;      // [problem * (kMaxLevel + 1) + level]
    std::vector<int> phase_begin;         // first item of every launch, then the item count
    std::vector<int> phase_tab;           // 1: the launch runs node-table levels
    QProblem* dp = nullptr;
    QLevel* dl = nullptr;
    QItem* ditems = nullptr;
    int* dneed = nullptr;
    int* dctr = nullptr;                  // status, heads[kMaxPhases], done[nlv]
    int2* u_perm = nullptr;
    int2* u_interp = nullptr;
    int64_t n_interp = 0;
    int2* u_near = nullptr;
    int2* u_leaf = nullptr;
    int64_t n_perm = 0, n_near = 0, n_leaf = 0;
    void** dio = nullptr;                 // [2 n]: densities, then outputs
    std::vector<const void*> io_dens;
    std::vector<void*> io_outs;
    char* coef = nullptr;                 // coefficients of every level of every problem
    int cones_per_item = -1;              // split the items were built with
    std::vector<void*> owned;
};

namespace {

template <class T>
T* upload_vec(BatchQueue& q, const std::vector<T>& h) {
    void* p = nullptr;
    const size_t bytes = std::max<size_t>(16, h.size() * sizeof(T));
    IFGF_CUDA(cudaMalloc(&p, bytes));
    q.owned.push_back(p);
    if (!h.empty()) IFGF_CUDA(cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return (T*)p;
}

// Propagation items.  A problem's propagation levels D..4 fall into runs of one kind (from a
// level with node tables or not); runs go to alternating launches, node-table launches at even
// indices (phase), so that each launch runs one kernel shape.  Within a launch: stage
// s = D_p - d (the distance of the child level from the leaves) first, then problems with more
// cones at that stage first; within a level, runs of cpi parent cones in cone order (a multiple
// of the warps and cones per step of both kernels).  An item waits for the items of the problem's
// level d+1 when they are in the same launch (an earlier launch has finished before it starts).
void build_items(BatchQueue& q, int cpi) {
    q.hitems.clear();
    q.hneed.assign(q.hl.size(), 0);
    const size_t np = q.plans.size();
    q.first_item.assign(np * (kMaxLevel + 1), -1);
    struct Job {
        int phase, stage, p, d;
        int64_t ncp;
    };
    std::vector<Job> jobs;
    std::vector<int> phase_of(np * (kMaxLevel + 1), -1);
    for (size_t p = 0; p < np; ++p) {
        const QProblem& P = q.hp[p];
        int ph = -1, kind = -1;
        for (int d = P.D; d >= 4; --d) {
            const QLevel& L = q.hl[P.lv0 + d - 3];
            if (L.ncp == 0) continue;
            if (L.tabled != kind) {
                ph = ph < 0 ? (L.tabled ? 0 : 1) : ph + 1;
                kind = L.tabled;
            }
            phase_of[p * (kMaxLevel + 1) + d] = ph;
            jobs.push_back(Job{ph, P.D - d, (int)p, d, L.ncp});
        }
    }
    std::stable_sort(jobs.begin(), jobs.end(), [](const Job& a, const Job& b) {
        if (a.phase != b.phase) return a.phase < b.phase;
        if (a.stage != b.stage) return a.stage < b.stage;
        return a.ncp > b.ncp;
    });
    q.phase_begin.clear();
    q.phase_tab.clear();
    for (const Job& j : jobs) {
        while ((int)q.phase_begin.size() <= j.phase) {
            q.phase_begin.push_back((int)q.hitems.size());
            q.phase_tab.push_back(q.phase_begin.size() % 2 == 1 ? 1 : 0);
        }
        const QProblem& P = q.hp[j.p];
        const int lv = P.lv0 + j.d - 3;
        const bool same = j.d < P.D && phase_of[(size_t)j.p * (kMaxLevel + 1) + j.d + 1] == j.phase;
        q.first_item[(size_t)j.p * (kMaxLevel + 1) + j.d] = (int64_t)q.hitems.size();
        for (int64_t c = 0; c < j.ncp; c += cpi) {
            q.hitems.push_back(QItem{lv, same ? lv + 1 : -1, (int32_t)c, (int32_t)std::min<int64_t>(j.ncp, c + cpi)});
            ++q.hneed[lv];
        }
    }
    q.phase_begin.push_back((int)q.hitems.size());
}

}  // namespace

bool queue_eligible(const std::vector<Plan*>& plans, const int32_t* nrhs, std::string* why) {
    for (size_t i = 0; i < plans.size(); ++i) {
        const Plan& p = *plans[i];
        std::string w;
        if (p.precision != IFGF_PREC_MIXED) w = "not mixed precision";
        else if (p.Ps != 3 || p.Pt != 5 || p.Pp != 5) w = "orders other than (3,5,5)";
        else if (nrhs && nrhs[i] != 1) w = "more than one density";
        else if (p.device != plans[0]->device) w = "another device";
        if (!w.empty()) {
            if (why) *why = "batch entry " + std::to_string(i) + ": " + w;
            return false;
        }
    }
    return true;
}

BatchQueue* queue_create(const std::vector<Plan*>& plans) {
    BatchQueue* qp = new BatchQueue();
    BatchQueue& q = *qp;
    try {
        q.plans = plans;
        q.device = plans[0]->device;
        IFGF_CUDA(cudaSetDevice(q.device));
        IFGF_CUDA(cudaDeviceGetAttribute(&q.nsm, cudaDevAttrMultiProcessorCount, q.device));
        // coefficient storage: every level of every problem, 256-byte aligned blocks
        std::vector<int64_t> off;
        int64_t total = 0;
        for (Plan* pp : plans) {
            for (int d = 3; d <= pp->D; ++d) {
                off.push_back(total);
                total += (pp->L[d].nc * pp->cstride * (int64_t)sizeof(float2) + 255) / 256 * 256;
            }
        }
        IFGF_CUDA(cudaMalloc((void**)&q.coef, std::max<int64_t>(total, 256)));
        q.owned.push_back(q.coef);
        size_t k = 0;
        std::vector<int2> u_perm, u_near, u_leaf, u_interp;
        int64_t acc_total = 0;
        for (Plan* pp : plans) acc_total += pp->N * (int64_t)(pp->D - 2);
        float2* iacc = nullptr;
        IFGF_CUDA(cudaMalloc((void**)&iacc, std::max<int64_t>(acc_total, 1) * sizeof(float2)));
        q.owned.push_back(iacc);
        int64_t acc_at = 0;
        std::vector<int> by_size(plans.size());
        std::iota(by_size.begin(), by_size.end(), 0);
        std::stable_sort(by_size.begin(), by_size.end(), [&](int a, int b) { return plans[a]->N > plans[b]->N; });
        for (size_t i = 0; i < plans.size(); ++i) {
            Plan& p = *plans[i];
            Level& LD = p.L[p.D];
            QProblem P;
            P.N = p.N;
            P.D = p.D;
            P.lv0 = (int)q.hl.size();
            P.ku = (float)(p.kappa * p.u);
            P.inv4piu = (float)(1.0 / (4.0 * M_PI * p.u));
            P.kh = (float)(p.kappa * LD.g.h64);
            P.hinv = 1.0f / LD.g.hg;
            P.perm = p.perm;
            P.off = p.off;
            P.as = (float2*)p.a_s;
            P.Is = (float2*)p.I_s;
            P.kD = LD.k;
            P.startD = LD.start;
            P.nnb = LD.nnb;
            P.nb = LD.nb;
            P.bcs = LD.bcs;
            P.pboxD = LD.pbox;
            P.cone_gamD = LD.cone_gam;
            P.gD = LD.g;
            P.ncD = (int)LD.nc;
            P.W = p.Wf;
            P.cstride = p.cstride;
            P.status = p.d_status;
            for (int d = 3; d <= p.D; ++d) {
                Level& L = p.L[d];
                QLevel Q;
                Q.pbox = L.pbox;
                Q.k = L.k;
                Q.ncs = L.ncs;
                Q.cs = L.cs;
                Q.cm = L.cmap(p.d_status);
                Q.g = L.g;
                Q.phtab = L.phtab;
                Q.coef = (const float2*)(q.coef + off[k + d - 3]);
                Q.iacc = iacc + acc_at;
                acc_at += p.N;
                Q.sh = p.D - d;
                Q.problem = (int)i;
                Q.ku = P.ku;
                if (d >= 4 && p.L[d - 1].nc > 0) {
                    Level& Lp = p.L[d - 1];
                    Q.ncp = Lp.nc;
                    Q.tabled = Lp.n_gam > 0 && L.knob_few != 1;
                    Q.pcone_box = Lp.cone_box;
                    Q.pcone_gam = Lp.cone_gam;
                    Q.cone_gidx = Lp.cone_gidx;
                    Q.kp = Lp.k;
                    Q.pcstart = Lp.cstart;
                    Q.gp = Lp.g;
                    Q.tab_t = Lp.tab_t;
                    Q.tab_r = Lp.tab_r;
                    Q.tab_k = Lp.tab_k;
                    Q.tab_list = Lp.tab_list;
                    Q.tab_perm = Lp.tab_perm;
                    Q.tab_nseg = Lp.tab_nseg;
                    Q.tab_seg = Lp.tab_seg;
                    Q.cparent = (float2*)(q.coef + off[k + d - 4]);
                }
                q.hl.push_back(Q);
            }
            P.coefD = (float2*)(q.coef + off[k + p.D - 3]);
            k += p.D - 2;
            q.hp.push_back(P);
        }
        for (int i : by_size) {
            Plan& p = *plans[i];
            const Level& LD = p.L[p.D];
            for (int64_t t = 0; t < p.N; t += 256) u_perm.push_back(make_int2(i, (int)t));
            for (int d = p.D; d >= 3; --d)
                for (int64_t t = 0; t < p.N; t += 256) u_interp.push_back(make_int2(q.hp[i].lv0 + d - 3, (int)t));
            for (int b = 0; b < LD.n; ++b) u_near.push_back(make_int2(i, b));
            if (LD.nc > 0)
                for (int b = 0; b < LD.n; ++b) u_leaf.push_back(make_int2(i, b));
        }
        q.n_perm = (int64_t)u_perm.size();
        q.n_near = (int64_t)u_near.size();
        q.n_leaf = (int64_t)u_leaf.size();
        q.u_perm = upload_vec(q, u_perm);
        q.n_interp = (int64_t)u_interp.size();
        q.u_interp = upload_vec(q, u_interp);
        q.u_near = upload_vec(q, u_near);
        q.u_leaf = upload_vec(q, u_leaf);
        q.dp = upload_vec(q, q.hp);
        q.dl = upload_vec(q, q.hl);
        q.dctr = upload_vec(q, std::vector<int>(q.hl.size() + 1 + kMaxPhases, 0));
        q.dio = upload_vec(q, std::vector<void*>(2 * plans.size(), nullptr));
    } catch (...) {
        queue_destroy(qp);
        throw;
    }
    return qp;
}

void queue_destroy(BatchQueue* q) {
    if (!q) return;
    cudaSetDevice(q->device);
    for (void* p : q->owned) cudaFree(p);
    delete q;
}

void queue_set_io(BatchQueue* q, const void* const* dens, void* const* outs, cudaStream_t s) {
    const size_t n = q->plans.size();
    bool same = q->io_dens.size() == n;
    for (size_t i = 0; same && i < n; ++i) same = q->io_dens[i] == dens[i] && q->io_outs[i] == outs[i];
    if (same) return;
    q->io_dens.assign(dens, dens + n);
    q->io_outs.assign(outs, outs + n);
    std::vector<void*> h(2 * n);
    for (size_t i = 0; i < n; ++i) {
        h[i] = const_cast<void*>(dens[i]);
        h[n + i] = outs[i];
    }
    // pageable source: the copy is staged before this call returns, ordered on s
    IFGF_CUDA(cudaMemcpyAsync(q->dio, h.data(), h.size() * sizeof(void*), cudaMemcpyHostToDevice, s));
    IFGF_CUDA(cudaStreamSynchronize(s));
}

void queue_prepare(BatchQueue* q, const QueueConfig& c) {
    BatchQueue& Q = *q;
    const int cpi = std::max(4, c.cones_per_item / 4 * 4);
    if (cpi != Q.cones_per_item) {
        build_items(Q, cpi);
        for (void* p : {(void*)Q.ditems, (void*)Q.dneed}) {
            if (!p) continue;
            Q.owned.erase(std::find(Q.owned.begin(), Q.owned.end(), p));
            IFGF_CUDA(cudaFree(p));
        }
        Q.ditems = upload_vec(Q, Q.hitems);
        Q.dneed = upload_vec(Q, Q.hneed);
        Q.cones_per_item = cpi;
    }
}

void queue_record(BatchQueue* q, const QueueConfig& c, cudaStream_t s, const std::vector<cudaStream_t>* branches,
                  const std::vector<cudaEvent_t>* ev) {
    BatchQueue& Q = *q;
    if (Q.cones_per_item != std::max(4, c.cones_per_item / 4 * 4))
        fail(IFGF_ERR_INTERNAL, "queue recorded before its items were built");
    const size_t n = Q.plans.size();
    const float2* const* dens = (const float2* const*)Q.dio;
    float2* const* outs = (float2* const*)(Q.dio + n);
    IFGF_CUDA(cudaMemsetAsync(Q.dctr, 0, (Q.hl.size() + 1 + kMaxPhases) * sizeof(int), s));
    IFGF_LAUNCH(k_q_perm_in, (unsigned)Q.n_perm, 256, 0, s, Q.dp, Q.u_perm, dens);
    if (Q.n_near > 0) IFGF_LAUNCH(k_q_near, (unsigned)Q.n_near, kNearThreads, 0, s, Q.dp, Q.u_near);
    if (Q.n_leaf > 0) IFGF_LAUNCH(k_q_leaf, (unsigned)Q.n_leaf, kLeafThreads, 0, s, Q.dp, Q.u_leaf);
    const int wh = c.withhold >= 0 ? (int)queue_first_item(q, c.withhold / 64, c.withhold % 64) : -1;
    int* bstatus = Q.dctr;
    int* heads = Q.dctr + 1;
    int* done = Q.dctr + 1 + kMaxPhases;
    if (branches && !branches->empty()) {
        // each plan's own propagation kernels, problems spread over concurrent branches
        const size_t kb = branches->size();
        IFGF_CUDA(cudaEventRecord((*ev)[0], s));
        for (size_t j = 0; j < kb; ++j) IFGF_CUDA(cudaStreamWaitEvent((*branches)[j], (*ev)[0], 0));
        for (size_t i = 0; i < n; ++i) {
            Plan& p = *Q.plans[i];
            const QProblem& P = Q.hp[i];
            for (int d = p.D; d >= 4; --d) {
                const QLevel& L = Q.hl[P.lv0 + d - 3];
                if (L.ncp > 0) shard_prop(p, d, 1, 0, L.ncp, L.cm, L.coef, L.cparent, (*branches)[i % kb]);
            }
        }
        for (size_t j = 0; j < kb; ++j) {
            IFGF_CUDA(cudaEventRecord((*ev)[j + 1], (*branches)[j]));
            IFGF_CUDA(cudaStreamWaitEvent(s, (*ev)[j + 1], 0));
        }
    }
    for (size_t ph = 0; !(branches && !branches->empty()) && ph + 1 < Q.phase_begin.size(); ++ph) {
        const int i0 = Q.phase_begin[ph], n = Q.phase_begin[ph + 1] - i0;
        if (n <= 0) continue;
        const int w = wh >= i0 && wh < i0 + n ? wh - i0 : -1;
        const bool tab = Q.phase_tab[ph] != 0;
        int occ = 0;
        if (tab)
            IFGF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_q_prop<true>, 32 * kWarpCones, 0));
        else
            IFGF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_q_prop<false>, kPropThreads, 0));
        occ = std::max(occ, 1);
        const int per_sm = c.blocks_per_sm > 0 ? std::min(c.blocks_per_sm, occ) : occ;
        const unsigned blocks = (unsigned)std::min<int64_t>((int64_t)per_sm * Q.nsm, n);
        if (tab)
            IFGF_LAUNCH(k_q_prop<true>, blocks, 32 * kWarpCones, 0, s, Q.dl, Q.ditems + i0, n, Q.dneed, heads + ph,
                        done, bstatus, Q.plans[0]->Wf, Q.plans[0]->cstride, c.wait_limit, w);
        else
            IFGF_LAUNCH(k_q_prop<false>, blocks, kPropThreads, 0, s, Q.dl, Q.ditems + i0, n, Q.dneed, heads + ph,
                        done, bstatus, Q.plans[0]->Wf, Q.plans[0]->cstride, c.wait_limit, w);
    }
    IFGF_LAUNCH(k_q_interp, (unsigned)Q.n_interp, 256, 0, s, Q.dp, Q.dl, Q.u_interp);
    IFGF_LAUNCH(k_q_perm_out, (unsigned)Q.n_perm, 256, 0, s, Q.dp, Q.dl, Q.u_perm, outs);
}

int64_t queue_items(const BatchQueue* q) { return (int64_t)q->hitems.size(); }

int64_t queue_first_item(const BatchQueue* q, int problem, int level) {
    if (problem < 0 || (size_t)problem >= q->plans.size() || level < 0 || level > kMaxLevel) return -1;
    if (q->first_item.empty()) return -1;
    return q->first_item[(size_t)problem * (kMaxLevel + 1) + level];
}

int queue_status(BatchQueue* q) {
    IFGF_CUDA(cudaSetDevice(q->device));
    IFGF_CUDA(cudaDeviceSynchronize());
    int st = 0;
    IFGF_CUDA(cudaMemcpy(&st, q->dctr, sizeof(int), cudaMemcpyDeviceToHost));
    return st;
}

}  // namespace ifgf
