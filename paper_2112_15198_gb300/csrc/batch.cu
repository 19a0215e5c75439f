// Batched apply: many plans evaluated as one CUDA-graph launch sequence.
//
// The first ifgf_batch_apply with a given set of buffers captures the apply of every plan on
// private streams into a CUDA graph (problem i on branch i mod 8 of a fork/join, so independent
// problems run concurrently); later calls with the same buffers replay it with one
// cudaGraphLaunch on the caller's stream (different buffers trigger a new capture).
// The problems of the batch share the launch sequence, not their data: each plan keeps its
// own tree, cones and scratch.
#include <algorithm>
#include <functional>
#include <string>
#include <vector>

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
    return guard_call([&] {
        IFGF_CUDA(cudaSetDevice(b->device));
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

ifgf_status ifgf_batch_destroy(ifgf_batch b) {
    if (!b) return IFGF_OK;
    cudaSetDevice(b->device);
    drop_graph(*b);
    for (cudaStream_t x : b->branch) cudaStreamDestroy(x);
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return IFGF_OK;
}

}  // extern "C"
