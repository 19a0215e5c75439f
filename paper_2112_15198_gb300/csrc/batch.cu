// Batched apply: many plans evaluated as one CUDA-graph launch sequence.
//
// The first ifgf_batch_apply with a given set of buffers captures the apply of every plan on
// private streams into a CUDA graph (problem i on branch i mod 8 of a fork/join, so independent
// problems run concurrently); later calls with the same buffers replay it with one
// cudaGraphLaunch on the caller's stream (different buffers trigger a new capture).
// The problems of the batch share the launch sequence, not their data: each plan keeps its
// own tree, cones and scratch.
#include <algorithm>
#include <cstdio>
#include <functional>
#include <string>
#include <vector>

#include "batch_queue.cuh"
#include "ifgf_internal.cuh"

struct ifgf_plan_s;  // opaque handle of api.cu (derives from ifgf::Plan)

struct ifgf_batch_s {
    std::vector<ifgf::Plan*> plans;
    int device = 0;
    cudaStream_t cap = nullptr;
    // independent problems run on kBranches concurrent branches of the graph (captured on
    // forked streams), so that small problems fill the GPU together
    std::vector<cudaStream_t> branch;
    std::vector<cudaEvent_t> ev;  // fork event, then one join event per branch
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> dens;
    std::vector<void*> outs;
    std::vector<int32_t> nrhs;
    int64_t launches_per_replay = 0;
    // queue mode (batch_queue.cu): -1 where eligible, 0 never, 1 always
    int mode = -1;                  // 2: queue sequence with each plan's propagation on branches
    int last_mode = -1;
    ifgf::QueueConfig qc;
    ifgf::BatchQueue* queue = nullptr;
    cudaGraph_t qgraph = nullptr;
    cudaGraphExec_t qexec = nullptr;
    int64_t q_launches = 0;
};

namespace ifgf {
ifgf::Plan* plan_of(ifgf_plan p);  // api.cu
ifgf_status guard_call(const std::function<void()>& f);
}  // namespace ifgf

using namespace ifgf;

namespace {
constexpr int kBranches = 8;
void drop_graph(ifgf_batch_s& b) {
    if (b.exec) cudaGraphExecDestroy(b.exec);
    if (b.graph) cudaGraphDestroy(b.graph);
    b.exec = nullptr;
    b.graph = nullptr;
}
void drop_qgraph(ifgf_batch_s& b) {
    if (b.qexec) cudaGraphExecDestroy(b.qexec);
    if (b.qgraph) cudaGraphDestroy(b.qgraph);
    b.qexec = nullptr;
    b.qgraph = nullptr;
}
}  // namespace

extern "C" {

ifgf_status ifgf_batch_create(const ifgf_plan* plans, int32_t n, ifgf_batch* out_batch) {
    if (!plans || n < 1 || !out_batch) {
        set_last_error("batch needs at least one plan and an output handle");
        return IFGF_ERR_INVALID_ARG;
    }
    for (int32_t i = 0; i < n; ++i) {
        if (!plans[i]) {
            set_last_error("NULL plan in batch");
            return IFGF_ERR_INVALID_ARG;
        }
        // a plan owns its scratch and coefficient buffers: two entries of one plan would run on
        // concurrent branches and overwrite each other's intermediate results
        for (int32_t j = 0; j < i; ++j)
            if (plans[j] == plans[i]) {
                set_last_error("plan " + std::to_string(i) + " repeats plan " + std::to_string(j) +
                               " of the batch");
                return IFGF_ERR_INVALID_ARG;
            }
    }
    ifgf_batch_s* b = new ifgf_batch_s();
    ifgf_status st = guard_call([&] {
        for (int32_t i = 0; i < n; ++i) b->plans.push_back(plan_of(plans[i]));
        b->device = b->plans[0]->device;
        for (Plan* p : b->plans)
            if (p->device != b->device) fail(IFGF_ERR_INVALID_ARG, "plans of a batch must share one device");
        IFGF_CUDA(cudaSetDevice(b->device));
        IFGF_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
        const int nb = (int)std::min<size_t>(kBranches, b->plans.size());
        for (int i = 0; i < nb; ++i) {
            cudaStream_t st2 = nullptr;
            IFGF_CUDA(cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking));
            b->branch.push_back(st2);
        }
        for (int i = 0; i <= nb; ++i) {
            cudaEvent_t e = nullptr;
            IFGF_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            b->ev.push_back(e);
        }
    });
    if (st != IFGF_OK) {
        for (cudaStream_t x : b->branch) cudaStreamDestroy(x);
        for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
        if (b->cap) cudaStreamDestroy(b->cap);
        delete b;
        return st;
    }
    *out_batch = b;
    return IFGF_OK;
}

ifgf_status ifgf_batch_apply(ifgf_batch b, const void* const* dens, const int32_t* nrhs, void* const* outs,
                             void* stream) {
    if (!b || !dens || !nrhs || !outs) {
        set_last_error("NULL batch or buffer arrays");
        return IFGF_ERR_INVALID_ARG;
    }
    const size_t n = b->plans.size();
    for (size_t i = 0; i < n; ++i) {
        if (!dens[i] || !outs[i] || dens[i] == outs[i]) {
            set_last_error("batch entry " + std::to_string(i) + ": NULL or aliased buffers");
            return IFGF_ERR_INVALID_ARG;
        }
        if (nrhs[i] < 1 || nrhs[i] > b->plans[i]->max_nrhs) {
            set_last_error("batch entry " + std::to_string(i) + ": nrhs out of range");
            return IFGF_ERR_INVALID_ARG;
        }
    }
    std::string why;
    const bool eligible = queue_eligible(b->plans, nrhs, &why);
    if ((b->mode == 1 || b->mode == 2) && !eligible) {
        set_last_error("queue mode: " + why);
        return IFGF_ERR_UNSUPPORTED;
    }
    // -1: the built-in choice, the graph sequence (fastest on the uneven 64-problem batch measured;
    // ifgf_batch_autotune chooses per batch)
    const int eff = b->mode == -1 ? 0 : b->mode;
    if (eff != 0) {
        return guard_call([&] {
            IFGF_CUDA(cudaSetDevice(b->device));
            if (!b->queue) b->queue = queue_create(b->plans);
            queue_set_io(b->queue, dens, outs, (cudaStream_t)stream);
            if (!b->qexec) {
                queue_prepare(b->queue, b->qc);
                const int64_t l0 = g_launches.load();
                IFGF_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
                try {
                    if (eff == 2)
                        queue_record(b->queue, b->qc, b->cap, &b->branch, &b->ev);
                    else
                        queue_record(b->queue, b->qc, b->cap);
                } catch (...) {
                    cudaGraph_t g = nullptr;
                    cudaStreamEndCapture(b->cap, &g);
                    if (g) cudaGraphDestroy(g);
                    cudaGetLastError();
                    throw;
                }
                IFGF_CUDA(cudaStreamEndCapture(b->cap, &b->qgraph));
                IFGF_CUDA(cudaGraphInstantiate(&b->qexec, b->qgraph, 0));
                b->q_launches = g_launches.load() - l0;
                g_launches.fetch_sub(b->q_launches);  // counted when replayed
            }
            IFGF_CUDA(cudaGraphLaunch(b->qexec, (cudaStream_t)stream));
            g_launches.fetch_add(b->q_launches);
            b->last_mode = eff;
        });
    }
    return guard_call([&] {
        IFGF_CUDA(cudaSetDevice(b->device));
        b->last_mode = 0;
        bool same = b->exec != nullptr && b->dens.size() == n;
        for (size_t i = 0; same && i < n; ++i)
            same = b->dens[i] == dens[i] && b->outs[i] == outs[i] && b->nrhs[i] == nrhs[i];
        if (!same) {
            drop_graph(*b);
            const int64_t l0 = g_launches.load();
            IFGF_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
            try {
                // fork: every branch waits for the capture stream, runs every kb-th problem in order,
                // and the capture stream joins all branches
                const size_t kb = b->branch.size();
                IFGF_CUDA(cudaEventRecord(b->ev[0], b->cap));
                for (size_t j = 0; j < kb; ++j) IFGF_CUDA(cudaStreamWaitEvent(b->branch[j], b->ev[0], 0));
                for (size_t i = 0; i < n; ++i)
                    apply_plan(*b->plans[i], dens[i], nrhs[i], outs[i], b->branch[i % kb], true, -1);
                for (size_t j = 0; j < kb; ++j) {
                    IFGF_CUDA(cudaEventRecord(b->ev[j + 1], b->branch[j]));
                    IFGF_CUDA(cudaStreamWaitEvent(b->cap, b->ev[j + 1], 0));
                }
            } catch (...) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(b->cap, &g);
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                throw;
            }
            IFGF_CUDA(cudaStreamEndCapture(b->cap, &b->graph));
            IFGF_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
            b->launches_per_replay = g_launches.load() - l0;
            g_launches.fetch_sub(b->launches_per_replay);  // counted when replayed, not when captured
            b->dens.assign(dens, dens + n);
            b->outs.assign(outs, outs + n);
            b->nrhs.assign(nrhs, nrhs + n);
        }
        IFGF_CUDA(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
        g_launches.fetch_add(b->launches_per_replay);
    });
}

ifgf_status ifgf_batch_set(ifgf_batch b, int32_t what, int64_t value) {
    if (!b) {
        set_last_error("NULL batch");
        return IFGF_ERR_INVALID_ARG;
    }
    bool ok = true;
    switch (what) {
        case IFGF_BATCH_MODE:
            ok = value >= -1 && value <= 2;
            if (ok) b->mode = (int)value;
            break;
        case IFGF_BATCH_CONES_PER_ITEM:
            ok = value >= 4 && value <= (1 << 20);
            if (ok) b->qc.cones_per_item = (int)value;
            break;
        case IFGF_BATCH_BLOCKS_PER_SM:
            ok = value >= 0 && value <= 64;
            if (ok) b->qc.blocks_per_sm = (int)value;
            break;
        case IFGF_BATCH_WAIT_LIMIT:
            ok = value >= 0;
            if (ok) b->qc.wait_limit = value;
            break;
        case IFGF_BATCH_WITHHOLD:
            if (value < 0) {
                b->qc.withhold = -1;
            } else {
                const int64_t prob = value / 64, lev = value % 64;
                ok = prob < (int64_t)b->plans.size() && lev >= 4 && lev <= b->plans[prob]->D;
                if (ok) b->qc.withhold = (int)value;
            }
            break;
        default:
            ok = false;
    }
    if (!ok) {
        set_last_error("unknown batch setting or value out of range");
        return IFGF_ERR_INVALID_ARG;
    }
    drop_qgraph(*b);  // the next queue apply records the sequence with the new settings
    return IFGF_OK;
}

ifgf_status ifgf_batch_get(ifgf_batch b, int32_t what, int64_t* value) {
    if (!b || !value) {
        set_last_error("NULL batch or value pointer");
        return IFGF_ERR_INVALID_ARG;
    }
    switch (what) {
        case IFGF_BATCH_MODE: *value = b->mode; return IFGF_OK;
        case IFGF_BATCH_CONES_PER_ITEM: *value = b->qc.cones_per_item; return IFGF_OK;
        case IFGF_BATCH_BLOCKS_PER_SM: *value = b->qc.blocks_per_sm; return IFGF_OK;
        case IFGF_BATCH_WAIT_LIMIT: *value = b->qc.wait_limit; return IFGF_OK;
        case IFGF_BATCH_LAST_MODE: *value = b->last_mode; return IFGF_OK;
        case IFGF_BATCH_ITEMS: *value = b->queue ? queue_items(b->queue) : 0; return IFGF_OK;
        case IFGF_BATCH_STATUS:
            if (!b->queue) {
                *value = IFGF_OK;
                return IFGF_OK;
            }
            return guard_call([&] { *value = queue_status(b->queue); });
        default:
            set_last_error("unknown batch query");
            return IFGF_ERR_INVALID_ARG;
    }
}

ifgf_status ifgf_batch_autotune(ifgf_batch b, const void* const* dens, const int32_t* nrhs, void* const* outs,
                                const char* cache_path, void* stream, int32_t* from_cache) {
    if (!b || !dens || !nrhs || !outs) {
        set_last_error("NULL batch or buffer arrays");
        return IFGF_ERR_INVALID_ARG;
    }
    if (from_cache) *from_cache = 1;
    const bool eligible = queue_eligible(b->plans, nrhs, nullptr);
    int64_t total = 0, largest = 0;
    int rmax = 1;
    for (size_t i = 0; i < b->plans.size(); ++i) {
        total += b->plans[i]->N;
        largest = std::max<int64_t>(largest, b->plans[i]->N);
        rmax = std::max<int>(rmax, nrhs[i]);
    }
    struct Cand {
        int mode, cpi, bps;
    };
    std::vector<Cand> cands{{0, 16, 0}};
    if (eligible) {
        cands.push_back({2, 16, 0});
        for (int cpi : {8, 16, 32, 64})
            for (int bps : {0, 2}) cands.push_back({1, cpi, bps});
    }
    Cand best = cands.back();
    ifgf_status st = guard_call([&] {
        IFGF_CUDA(cudaSetDevice(b->device));
        const std::string key = "batch|" + tune_gpu_key(b->device) + "|n=" + std::to_string(tune_log2((int64_t)b->plans.size())) +
                                "|N=" + std::to_string(tune_log2(total)) + "|M=" + std::to_string(tune_log2(largest)) +
                                "|r=" + tune_rhs_bucket(rmax) + "|q=" + (eligible ? "1" : "0");
        std::map<std::string, std::string> cache;
        if (cache_path) cache = tune_cache_read(cache_path);
        auto it = cache.find(key);
        if (it != cache.end() && std::sscanf(it->second.c_str(), "%d,%d,%d", &best.mode, &best.cpi, &best.bps) == 3 &&
            (best.mode == 0 || eligible))
            return;
        if (from_cache) *from_cache = 0;
        cudaStream_t s = (cudaStream_t)stream;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        IFGF_CUDA(cudaEventCreate(&e0));
        IFGF_CUDA(cudaEventCreate(&e1));
        double best_ms = 1e300;
        for (const Cand& c : cands) {
            b->mode = c.mode;
            b->qc.cones_per_item = c.cpi;
            b->qc.blocks_per_sm = c.bps;
            drop_qgraph(*b);
            ifgf_status r = ifgf_batch_apply(b, dens, nrhs, outs, stream);  // capture and warm-up
            if (r != IFGF_OK) fail(r, "batch apply while tuning");
            std::vector<double> ms;
            for (int k = 0; k < 3; ++k) {
                IFGF_CUDA(cudaEventRecord(e0, s));
                r = ifgf_batch_apply(b, dens, nrhs, outs, stream);
                if (r != IFGF_OK) fail(r, "batch apply while tuning");
                IFGF_CUDA(cudaEventRecord(e1, s));
                IFGF_CUDA(cudaEventSynchronize(e1));
                float t = 0.f;
                IFGF_CUDA(cudaEventElapsedTime(&t, e0, e1));
                ms.push_back(t);
            }
            std::sort(ms.begin(), ms.end());
            if (ms[1] < best_ms) {
                best_ms = ms[1];
                best = c;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (cache_path)
            tune_cache_write(cache_path, {{key, std::to_string(best.mode) + "," + std::to_string(best.cpi) + "," +
                                                    std::to_string(best.bps)}});
    });
    b->mode = best.mode;
    b->qc.cones_per_item = best.cpi;
    b->qc.blocks_per_sm = best.bps;
    drop_qgraph(*b);
    return st;
}

ifgf_status ifgf_batch_destroy(ifgf_batch b) {
    if (!b) return IFGF_OK;
    cudaSetDevice(b->device);
    drop_graph(*b);
    drop_qgraph(*b);
    ifgf::queue_destroy(b->queue);
    for (cudaStream_t x : b->branch) cudaStreamDestroy(x);
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return IFGF_OK;
}

}  // extern "C"
