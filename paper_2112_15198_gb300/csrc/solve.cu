// Solver integration: restarted GMRES with the IFGF apply as its matrix-vector product, for
// second-kind systems (alpha I + beta A W) x = b, A the operator of Eq. (1) on the plan's points
// and W a diagonal of quadrature weights.  The paper evaluates A alone; inside an iterative
// solver for an integral equation is where such an apply is used.  The near field stays the
// naive point sum of Eq. (1): singular quadratures are not part of the paper.
//
// Krylov vectors live on the device in the plan's precision; inner products are accumulated in
// FP64 in a fixed order (per-block partial sums, then one block that adds them in block order),
// so a solve is reproducible.  The small Hessenberg least-squares problem runs on the host.
#include <algorithm>
#include <cmath>
#include <complex>
#include <functional>
#include <vector>

#include "ifgf_internal.cuh"

struct ifgf_plan_s;

namespace ifgf {

Plan* plan_of(ifgf_plan p);  // api.cu
ifgf_status guard_call(const std::function<void()>& f);

namespace {

using cd = std::complex<double>;
constexpr int kRed = 256;          // threads of the reduction blocks
constexpr int kRedBlocks = 296;    // blocks of the first reduction pass (two per SM)

template <class T>
struct Cx;
template <>
struct Cx<float2> {
    using R = float;
    __device__ static double2 ld(const float2& v) { return make_double2(v.x, v.y); }
    __device__ static float2 st(double re, double im) { return make_float2((float)re, (float)im); }
};
template <>
struct Cx<double2> {
    using R = double;
    __device__ static double2 ld(const double2& v) { return v; }
    __device__ static double2 st(double re, double im) { return make_double2(re, im); }
};

// u = w o x (weights real, NULL: u = x)
template <class T>
__global__ void k_weight(const T* __restrict__ x, const typename Cx<T>::R* __restrict__ w, T* __restrict__ u, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 v = Cx<T>::ld(x[i]);
    const double s = w ? (double)w[i] : 1.0;
    u[i] = Cx<T>::st(v.x * s, v.y * s);
}

// y = alpha x + beta a
template <class T>
__global__ void k_combine(const T* __restrict__ x, const T* __restrict__ a, double2 alpha, double2 beta, T* __restrict__ y,
                          int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 xv = Cx<T>::ld(x[i]), av = Cx<T>::ld(a[i]);
    const double re = alpha.x * xv.x - alpha.y * xv.y + beta.x * av.x - beta.y * av.y;
    const double im = alpha.x * xv.y + alpha.y * xv.x + beta.x * av.y + beta.y * av.x;
    y[i] = Cx<T>::st(re, im);
}

// partial[blockIdx.x][j] = sum over this block's elements of conj(V_j) w, j < k
template <class T>
__global__ void __launch_bounds__(kRed) k_dots(const T* __restrict__ V, int64_t n, int k, const T* __restrict__ w,
                                              double2* __restrict__ partial) {
    __shared__ double2 red[kRed];
    for (int j = 0; j < k; ++j) {
        double2 acc = make_double2(0.0, 0.0);
        const T* v = V + (int64_t)j * n;
        for (int64_t i = (int64_t)blockIdx.x * kRed + threadIdx.x; i < n; i += (int64_t)gridDim.x * kRed) {
            const double2 a = Cx<T>::ld(v[i]), b = Cx<T>::ld(w[i]);
            acc.x += a.x * b.x + a.y * b.y;
            acc.y += a.x * b.y - a.y * b.x;
        }
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int o = kRed / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) {
                red[threadIdx.x].x += red[threadIdx.x + o].x;
                red[threadIdx.x].y += red[threadIdx.x + o].y;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * k + j] = red[0];
        __syncthreads();
    }
}

// out[j] = sum over blocks of partial[b][j], in block order
__global__ void k_dots_sum(const double2* __restrict__ partial, int nb, int k, double2* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    double2 s = make_double2(0.0, 0.0);
    for (int b = 0; b < nb; ++b) {
        s.x += partial[(int64_t)b * k + j].x;
        s.y += partial[(int64_t)b * k + j].y;
    }
    out[j] = s;
}

// w -= sum_j h_j V_j  (sign = -1) or x += sum_j h_j V_j (sign = +1)
template <class T>
__global__ void k_update(const T* __restrict__ V, int64_t n, int k, const double2* __restrict__ h, double sign,
                         T* __restrict__ w) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 a = Cx<T>::ld(w[i]);
    for (int j = 0; j < k; ++j) {
        const double2 v = Cx<T>::ld(V[(int64_t)j * n + i]);
        const double2 c = h[j];
        a.x += sign * (c.x * v.x - c.y * v.y);
        a.y += sign * (c.x * v.y + c.y * v.x);
    }
    w[i] = Cx<T>::st(a.x, a.y);
}

template <class T>
__global__ void k_scale(T* __restrict__ v, int64_t n, double s) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 a = Cx<T>::ld(v[i]);
    v[i] = Cx<T>::st(a.x * s, a.y * s);
}

template <class T>
__global__ void k_copy(const T* __restrict__ a, T* __restrict__ b, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}

template <class T>
struct Gmres {
    Plan& p;
    cudaStream_t s;
    int64_t n;
    int m;
    const typename Cx<T>::R* wt;
    double2 alpha, beta;
    T* V = nullptr;  // m + 1 Krylov vectors of n
    T* u = nullptr;
    T* au = nullptr;
    T* w = nullptr;
    double2* partial = nullptr;
    double2* dots = nullptr;
    double2* hdev = nullptr;
    int64_t applies = 0;

    unsigned g(int64_t k) const { return (unsigned)((k + 255) / 256); }
    T* vec(int j) { return V + (int64_t)j * n; }

    // y = alpha x + beta A (W x)
    void op(const T* x, T* y) {
        IFGF_LAUNCH(k_weight<T>, g(n), 256, 0, s, x, wt, u, n);
        apply_plan(p, u, 1, au, s, true, -1);
        ++applies;
        IFGF_LAUNCH(k_combine<T>, g(n), 256, 0, s, x, au, alpha, beta, y, n);
    }
    // conj(rows[j]) . v for the k vectors starting at rows
    std::vector<cd> dot(const T* rows, int k, const T* v) {
        IFGF_LAUNCH(k_dots<T>, kRedBlocks, kRed, 0, s, rows, n, k, v, partial);
        IFGF_LAUNCH(k_dots_sum, (unsigned)((k + 63) / 64), 64, 0, s, partial, kRedBlocks, k, dots);
        std::vector<double2> h(k);
        IFGF_CUDA(cudaMemcpyAsync(h.data(), dots, k * sizeof(double2), cudaMemcpyDeviceToHost, s));
        IFGF_CUDA(cudaStreamSynchronize(s));
        std::vector<cd> out(k);
        for (int j = 0; j < k; ++j) out[j] = cd(h[j].x, h[j].y);
        return out;
    }
    double norm(const T* v) { return std::sqrt(std::max(0.0, dot(v, 1, v)[0].real())); }
    // target += sign * sum_j c_j V_j
    void update(int k, const std::vector<cd>& c, double sign, T* target) {
        std::vector<double2> h(k);
        for (int j = 0; j < k; ++j) h[j] = make_double2(c[j].real(), c[j].imag());
        IFGF_CUDA(cudaMemcpyAsync(hdev, h.data(), k * sizeof(double2), cudaMemcpyHostToDevice, s));
        IFGF_LAUNCH(k_update<T>, g(n), 256, 0, s, V, n, k, hdev, sign, target);
    }

    // Restarted GMRES(m) from the initial guess in x; returns the iterations and the residual
    // norm of the last step's estimate.
    int run(const T* b, T* x, int max_iters, double tol, double& est) {
        const double bn = norm(b);
        const double target = tol * (bn > 0 ? bn : 1.0);
        int it = 0;
        est = 0;
        std::vector<std::vector<cd>> H(m + 1, std::vector<cd>(m, cd(0)));
        std::vector<double> cs(m);
        std::vector<cd> sn(m), gv(m + 1);
        while (true) {
            op(x, w);  // r = b - op(x) into V_0
            IFGF_LAUNCH(k_combine<T>, g(n), 256, 0, s, b, w, make_double2(1, 0), make_double2(-1, 0), vec(0), n);
            const double r0 = norm(vec(0));
            est = r0;
            if (r0 <= target || it >= max_iters) return it;
            IFGF_LAUNCH(k_scale<T>, g(n), 256, 0, s, vec(0), n, 1.0 / r0);
            std::fill(gv.begin(), gv.end(), cd(0));
            gv[0] = r0;
            int k = 0;
            for (; k < m && it < max_iters; ++k) {
                op(vec(k), w);
                // classical Gram-Schmidt, twice
                std::vector<cd> h = dot(V, k + 1, w);
                update(k + 1, h, -1.0, w);
                std::vector<cd> h2 = dot(V, k + 1, w);
                update(k + 1, h2, -1.0, w);
                for (int i = 0; i <= k; ++i) H[i][k] = h[i] + h2[i];
                const double hn = norm(w);
                H[k + 1][k] = hn;
                if (hn > 0) {
                    IFGF_LAUNCH(k_copy<T>, g(n), 256, 0, s, w, vec(k + 1), n);
                    IFGF_LAUNCH(k_scale<T>, g(n), 256, 0, s, vec(k + 1), n, 1.0 / hn);
                }
                for (int i = 0; i < k; ++i) {  // earlier rotations
                    const cd a = H[i][k], c = H[i + 1][k];
                    H[i][k] = cs[i] * a + sn[i] * c;
                    H[i + 1][k] = -std::conj(sn[i]) * a + cs[i] * c;
                }
                const cd a = H[k][k], c = H[k + 1][k];
                const double na = std::abs(a), nr = std::sqrt(na * na + std::norm(c));
                if (nr == 0) {
                    cs[k] = 1;
                    sn[k] = 0;
                } else if (na == 0) {
                    cs[k] = 0;
                    sn[k] = std::conj(c) / nr;
                } else {
                    cs[k] = na / nr;
                    sn[k] = (a / na) * std::conj(c) / nr;
                }
                H[k][k] = cs[k] * a + sn[k] * c;
                H[k + 1][k] = 0;
                gv[k + 1] = -std::conj(sn[k]) * gv[k];
                gv[k] = cs[k] * gv[k];
                ++it;
                est = std::abs(gv[k + 1]);
                if (est <= target || hn == 0) {
                    ++k;
                    break;
                }
            }
            // x += V y, H y = g (upper triangular, k unknowns)
            std::vector<cd> y(k);
            for (int i = k - 1; i >= 0; --i) {
                cd t = gv[i];
                for (int j = i + 1; j < k; ++j) t -= H[i][j] * y[j];
                y[i] = H[i][i] != cd(0) ? t / H[i][i] : cd(0);
            }
            update(k, y, 1.0, x);
            if (est <= target || it >= max_iters) {
                // the true residual of the final iterate
                op(x, w);
                IFGF_LAUNCH(k_combine<T>, g(n), 256, 0, s, b, w, make_double2(1, 0), make_double2(-1, 0), vec(0), n);
                est = norm(vec(0));
                if (est <= target || it >= max_iters) return it;
            }
        }
    }
};

template <class T>
void solve(Plan& p, const void* b, void* x, double2 alpha, double2 beta, const void* weights, int m, int max_iters,
           double tol, cudaStream_t s, int32_t* iters, double* rel) {
    Gmres<T> G{p, s, p.N, m, (const typename Cx<T>::R*)weights, alpha, beta};
    const int64_t n = p.N;
    cudaMemPool_t pool = device_pool(p.device);
    std::vector<void*> mem;
    auto get = [&](size_t bytes) {
        void* q = nullptr;
        IFGF_CUDA(cudaMallocAsync(&q, std::max<size_t>(bytes, 16), pool, s));
        mem.push_back(q);
        return q;
    };
    try {
        G.V = (T*)get((size_t)(m + 1) * n * sizeof(T));
        G.u = (T*)get(n * sizeof(T));
        G.au = (T*)get(n * sizeof(T));
        G.w = (T*)get(n * sizeof(T));
        G.partial = (double2*)get((size_t)kRedBlocks * (m + 1) * sizeof(double2));
        G.dots = (double2*)get((size_t)(m + 1) * sizeof(double2));
        G.hdev = (double2*)get((size_t)(m + 1) * sizeof(double2));
        double est = 0;
        const int it = G.run((const T*)b, (T*)x, max_iters, tol, est);
        const double bn = G.norm((const T*)b);
        if (iters) *iters = it;
        if (rel) *rel = bn > 0 ? est / bn : est;
    } catch (...) {
        for (void* q : mem) cudaFreeAsync(q, s);
        throw;
    }
    for (void* q : mem) IFGF_CUDA(cudaFreeAsync(q, s));
    IFGF_CUDA(cudaStreamSynchronize(s));
}

}  // namespace
}  // namespace ifgf

using namespace ifgf;

extern "C" ifgf_status ifgf_gmres(ifgf_plan plan, const void* b, void* x, const double* alpha, const double* beta,
                                  const void* weights, int32_t restart, int32_t max_iters, double tol, void* stream,
                                  int32_t* iters, double* rel_residual) {
    if (!plan || !b || !x || !alpha || !beta) {
        set_last_error("NULL plan, right-hand side, solution or coefficient");
        return IFGF_ERR_INVALID_ARG;
    }
    if (b == x || weights == b || weights == x) {
        set_last_error("the right-hand side, the solution and the weights must not alias");
        return IFGF_ERR_INVALID_ARG;
    }
    if (restart < 1 || restart > 128 || max_iters < 1 || !(tol > 0) || !std::isfinite(tol)) {
        set_last_error("restart must be in [1, 128], max_iters >= 1 and tol > 0");
        return IFGF_ERR_INVALID_ARG;
    }
    Plan& p = *plan_of(plan);
    return guard_call([&] {
        IFGF_CUDA(cudaSetDevice(p.device));
        const double2 a = make_double2(alpha[0], alpha[1]), bt = make_double2(beta[0], beta[1]);
        if (p.precision == IFGF_PREC_MIXED)
            solve<float2>(p, b, x, a, bt, weights, restart, max_iters, tol, (cudaStream_t)stream, iters, rel_residual);
        else
            solve<double2>(p, b, x, a, bt, weights, restart, max_iters, tol, (cudaStream_t)stream, iters, rel_residual);
    });
}
