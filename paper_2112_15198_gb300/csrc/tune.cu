// Autotuner: chooses a plan's kernel knobs (and, in batch.cu, a batch's launch sequence) by
// timing the candidates on the plan's own data, and keeps the choices in an on-disk cache keyed
// by (GPU, SM count, orders, densities, size bucket), so that the next plan of the same shape
// on the same GPU takes them without measuring.
//
// Cache file: text, one entry per line, "<key> <value>"; later lines override earlier ones.
// Writes go to a temporary file that replaces the cache (rename), so that a reader never sees
// half a file.
#include <algorithm>
#include <cmath>
#include <functional>
#include <cstdio>
#include <fstream>
#include <map>
#include <sstream>

#include "ifgf_internal.cuh"

struct ifgf_plan_s;

namespace ifgf {

Plan* plan_of(ifgf_plan p);  // api.cu
ifgf_status guard_call(const std::function<void()>& f);

std::map<std::string, std::string> tune_cache_read(const std::string& path) {
    std::map<std::string, std::string> m;
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {
        const size_t sp = line.rfind(' ');
        if (sp == std::string::npos || sp == 0) continue;
        m[line.substr(0, sp)] = line.substr(sp + 1);
    }
    return m;
}

void tune_cache_write(const std::string& path, const std::map<std::string, std::string>& add) {
    std::map<std::string, std::string> m = tune_cache_read(path);
    for (auto& kv : add) m[kv.first] = kv.second;
    const std::string tmp = path + ".tmp" + std::to_string((long long)std::hash<std::string>{}(path) & 0xffff);
    {
        std::ofstream f(tmp, std::ios::trunc);
        if (!f) fail(IFGF_ERR_INVALID_ARG, "cannot write the tuning cache next to " + path);
        for (auto& kv : m) f << kv.first << ' ' << kv.second << '\n';
        if (!f) fail(IFGF_ERR_INVALID_ARG, "cannot write the tuning cache " + tmp);
    }
    if (std::rename(tmp.c_str(), path.c_str()) != 0) {
        std::remove(tmp.c_str());
        fail(IFGF_ERR_INVALID_ARG, "cannot replace the tuning cache " + path);
    }
}

// "<gpu name>/<SMs>" of a device, spaces replaced, for cache keys.
std::string tune_gpu_key(int device) {
    cudaDeviceProp prop;
    IFGF_CUDA(cudaGetDeviceProperties(&prop, device));
    std::string name = prop.name;
    for (char& c : name)
        if (c == ' ' || c == '|') c = '_';
    return name + "/" + std::to_string(prop.multiProcessorCount);
}

// Densities bucket of a cache key: 1, 2-3, 4-8, 9-16, 17-32, 33+.
std::string tune_rhs_bucket(int nrhs) {
    if (nrhs <= 1) return "1";
    if (nrhs <= 3) return "2-3";
    if (nrhs <= 8) return "4-8";
    if (nrhs <= 16) return "9-16";
    if (nrhs <= 32) return "17-32";
    return "33+";
}

int tune_log2(int64_t n) { return n <= 1 ? 0 : (int)std::floor(std::log2((double)n)); }

namespace {

__global__ void k_fill_density(float2* a, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // a bounded, non-constant pattern; the values do not change the kernels' work
    const float t = (float)(i % 9973) * 6.2831853f / 9973.f;
    a[i] = make_float2(__sinf(t), __cosf(2.f * t));
}

struct Timed {
    double total = 0;                     // ms of the whole apply
    double level[kMaxLevel + 1] = {};     // ms of the propagation from level d (both kinds)
};

Timed time_apply(Plan& p, const float2* dens, int nrhs, float2* out, cudaStream_t s, int reps) {
    apply_plan(p, dens, nrhs, out, s, true, -1);  // warm-up (and first-use setup)
    IFGF_CUDA(cudaStreamSynchronize(s));
    timing_collect_levels(nullptr, nullptr, nullptr);
    cudaEvent_t a = nullptr, b = nullptr;
    IFGF_CUDA(cudaEventCreate(&a));
    IFGF_CUDA(cudaEventCreate(&b));
    Timed t;
    std::vector<double> totals;
    for (int r = 0; r < reps; ++r) {
        IFGF_CUDA(cudaEventRecord(a, s));
        apply_plan(p, dens, nrhs, out, s, true, -1);
        IFGF_CUDA(cudaEventRecord(b, s));
        IFGF_CUDA(cudaEventSynchronize(b));
        float ms = 0.f;
        IFGF_CUDA(cudaEventElapsedTime(&ms, a, b));
        totals.push_back(ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    double by[TK_COUNT][kMaxLevel + 1];
    timing_collect_levels(nullptr, nullptr, by);
    std::sort(totals.begin(), totals.end());
    t.total = totals[totals.size() / 2];
    for (int d = 0; d <= kMaxLevel; ++d) t.level[d] = (by[TK_PROP][d] + by[TK_PROP_GEN][d]) / reps;
    return t;
}

}  // namespace
}  // namespace ifgf

using namespace ifgf;

extern "C" {

ifgf_status ifgf_plan_autotune(ifgf_plan plan, int32_t nrhs, const char* cache_path, void* stream,
                               int32_t* from_cache) {
    if (!plan || nrhs < 1) {
        set_last_error("NULL plan or nrhs < 1");
        return IFGF_ERR_INVALID_ARG;
    }
    Plan& p = *plan_of(plan);
    if (nrhs > p.max_nrhs) {
        set_last_error("nrhs above the plan's max_nrhs");
        return IFGF_ERR_INVALID_ARG;
    }
    if (from_cache) *from_cache = 1;
    const bool many = nrhs >= 4;
    const bool knobs = p.precision == IFGF_PREC_MIXED && p.Ps == 3 && p.Pt == 5 && p.Pp == 5;
    if (!knobs) return IFGF_OK;  // no kernel choices outside the mixed (3,5,5) path
    return guard_call([&] {
        IFGF_CUDA(cudaSetDevice(p.device));
        cudaStream_t s = (cudaStream_t)stream;
        const std::string pre = "plan|" + tune_gpu_key(p.device) + "|o=3.5.5|r=" + tune_rhs_bucket(nrhs);
        // the levels whose choice matters: propagation from d into a level with node tables
        std::vector<int> lv;
        std::vector<std::string> key(kMaxLevel + 1);
        for (int d = 4; d <= p.D; ++d)
            if (p.L[d - 1].nc > 0 && p.L[d - 1].n_gam > 0) {
                lv.push_back(d);
                key[d] = pre + (many ? "|many" : "|few") + "|c=" + std::to_string(tune_log2(p.L[d].nc)) + "|p=" +
                         std::to_string(tune_log2(p.L[d - 1].nc));
            }
        const std::string bkey = pre + "|block|n=" + std::to_string(tune_log2(p.N));
        std::map<std::string, std::string> cache;
        if (cache_path) cache = tune_cache_read(cache_path);
        bool hit = true;
        for (int d : lv) hit = hit && cache.count(key[d]);
        if (many) hit = hit && cache.count(bkey);
        auto set_level = [&](int d, int v) { (many ? p.L[d].knob_many : p.L[d].knob_few) = (int8_t)v; };
        if (hit) {
            for (int d : lv) set_level(d, std::stoi(cache[key[d]]));
            if (many) p.knob_block = std::stoi(cache[bkey]);
            return;
        }
        if (from_cache) *from_cache = 0;
        // measure: every candidate on every level at once, per-level propagation times
        const int64_t n = (int64_t)nrhs * p.N;
        float2* dens = nullptr;
        float2* out = nullptr;
        IFGF_CUDA(cudaMallocAsync((void**)&dens, n * sizeof(float2), device_pool(p.device), s));
        IFGF_CUDA(cudaMallocAsync((void**)&out, n * sizeof(float2), device_pool(p.device), s));
        const bool was_on = timing_switch(true);
        std::map<std::string, std::string> found;
        try {
            IFGF_LAUNCH(k_fill_density, (unsigned)((n + 255) / 256), 256, 0, s, dens, n);
            std::vector<int> blocks = many ? std::vector<int>{8, 16, 32} : std::vector<int>{-1};
            double best_total = 1e300;
            for (int blk : blocks) {
                p.knob_block = blk;
                Timed t[2];
                for (int v = 0; v < 2; ++v) {
                    for (int d : lv) set_level(d, v);
                    t[v] = time_apply(p, dens, nrhs, out, s, 2);
                }
                // the whole apply with the faster kernel on every level
                double total = t[0].total;
                std::vector<int> pick(kMaxLevel + 1, 0);
                for (int d : lv) {
                    pick[d] = t[1].level[d] < t[0].level[d] ? 1 : 0;
                    total -= t[0].level[d] - t[pick[d]].level[d];
                }
                if (total < best_total) {
                    best_total = total;
                    for (int d : lv) found[key[d]] = std::to_string(pick[d]);
                    if (many) found[bkey] = std::to_string(blk);
                }
            }
        } catch (...) {
            timing_switch(was_on);
            cudaFreeAsync(dens, s);
            cudaFreeAsync(out, s);
            throw;
        }
        timing_switch(was_on);
        IFGF_CUDA(cudaFreeAsync(dens, s));
        IFGF_CUDA(cudaFreeAsync(out, s));
        for (int d : lv) set_level(d, std::stoi(found[key[d]]));
        if (many) p.knob_block = std::stoi(found[bkey]);
        if (cache_path) tune_cache_write(cache_path, found);
    });
}

}  // extern "C"
