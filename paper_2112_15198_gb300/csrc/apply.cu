// Apply kernels of the IFGF operator (Algorithm 5 with the parallel loops of Algorithms 6-8)
// and the level-D neighbour sums ("LevelDSingularInteractions", Sec. 2).
//
// Two arithmetic variants share the plan and its exact FP32 cone classification:
//   mixed  FP32 arithmetic on grid-unit offsets (exact integer box-centre differences plus
//          FP32 leaf offsets); the large centred-factor phases kappa |x - x_B| are split into
//          a per-level FP64 table of (kappa |c_A - c_B|) mod 2 pi and a small FP32 correction;
//          the analytic factor and the propagation ratio are written in cancellation-free
//          forms whose phases stay below kappa h_d.
//   fp64   every value in FP64 on physical coordinates.
#include <algorithm>
#include <cmath>

#include "bodies_f32.cuh"
#include "ifgf_internal.cuh"

namespace ifgf {
namespace {

constexpr int kThreads = 256;

// ---- permutations -----------------------------------------------------------------------
template <class T>
__global__ void k_perm_in(const T* __restrict__ a, const int32_t* __restrict__ perm, int64_t N, T* __restrict__ as) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t r = blockIdx.y;
    as[r * N + i] = a[r * N + perm[i]];
}

template <class T>
__global__ void k_perm_out(const T* __restrict__ Is, const int32_t* __restrict__ perm, int64_t N, T* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t r = blockIdx.y;
    out[r * N + perm[i]] = Is[r * N + i];
}

// ---- near field --------------------------------------------------------------------------
// One block per leaf box (near_box_f32): leaf boxes [l0, l0 + gridDim.x), value set blockIdx.y.
__global__ void __launch_bounds__(kNearThreads)
k_near_tile_f32(const int4* __restrict__ kD, const int32_t* __restrict__ startD, const int32_t* __restrict__ nnb,
                const int32_t* __restrict__ nb, const float4* __restrict__ off, const float2* __restrict__ as,
                float2* __restrict__ Is, int64_t N, float ku, float inv4piu, int l0) {
    near_box_f32(kD, startD, nnb, nb, off, as, Is, N, ku, inv4piu, l0 + (int)blockIdx.x, (int64_t)blockIdx.y);
}

__global__ void k_near_f64(int64_t N, const int32_t* __restrict__ pboxD, const int32_t* __restrict__ startD,
                           const int32_t* __restrict__ nnb, const int32_t* __restrict__ nb,
                           const double* __restrict__ Xs, const double2* __restrict__ as, double2* __restrict__ Is,
                           double kappa) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t r = blockIdx.y;
    const int l = pboxD[i];
    const double xi = Xs[i], yi = Xs[N + i], zi = Xs[2 * N + i];
    const double2* ar = as + r * N;
    double2 acc = make_double2(0., 0.);
    const double inv4pi = 0.079577471545947667884441881686257181;
    for (int t = 0; t < nnb[l]; ++t) {
        const int q = nb[(int64_t)l * kMaxNbr + t];
        for (int j = startD[q]; j < startD[q + 1]; ++j) {
            if (j == i) continue;
            const double dx = xi - Xs[j], dy = yi - Xs[N + j], dz = zi - Xs[2 * N + j];
            const double rr = sqrt(dx * dx + dy * dy + dz * dz);
            double sn, cs;
            sincos(kappa * rr, &sn, &cs);
            const double w = inv4pi / rr;
            acc = make_double2(acc.x + (ar[j].x * cs - ar[j].y * sn) * w, acc.y + (ar[j].x * sn + ar[j].y * cs) * w);
        }
    }
    Is[r * N + i] = acc;
}

// ---- coefficient generation ("generate interpolant") -------------------------------------
// Chebyshev coefficients of the P node values held in smem f (index (i*PT + j)*PP + k), by the
// separable analysis matrices Ws | Wt | Wp; g is scratch of the same size.
template <int PS, int PT, int PP, class T2, class R>
__device__ __forceinline__ T2 cheb_coeffs_smem(T2* f, T2* g, const R* __restrict__ W, int n) {
    constexpr int P = PS * PT * PP;
    const R* Ws = W;
    const R* Wt = W + PS * PS;
    const R* Wp = Wt + PT * PT;
    const int c = n % PP, b = (n / PP) % PT, a = n / (PP * PT);
    if (n < P) {
        T2 acc{};
        const T2* row = f + (a * PT + b) * PP;
#pragma unroll
        for (int k = 0; k < PP; ++k) {
            const R w = Wp[c * PP + k];
            acc.x += w * row[k].x;
            acc.y += w * row[k].y;
        }
        g[n] = acc;
    }
    __syncthreads();
    if (n < P) {
        T2 acc{};
#pragma unroll
        for (int j = 0; j < PT; ++j) {
            const R w = Wt[b * PT + j];
            const T2 v = g[(a * PT + j) * PP + c];
            acc.x += w * v.x;
            acc.y += w * v.y;
        }
        f[n] = acc;
    }
    __syncthreads();
    T2 out{};
    if (n < P) {
#pragma unroll
        for (int i = 0; i < PS; ++i) {
            const R w = Ws[a * PS + i];
            const T2 v = f[(i * PT + b) * PP + c];
            out.x += w * v.x;
            out.y += w * v.y;
        }
    }
    return out;
}

// ---- LevelDEvaluations (Algorithm 6) ------------------------------------------------------
// One block per relevant leaf cone, one thread per interpolation node y:
//   F(y) = sum_{x' in B} a(x') g_k(y, x'),  g_k = G(y,x')/G(y,x_k)  (Eq. (3)),
// with y = x_k + (h/s) yhat and u = (x' - x_k)/h:
//   g_k = exp(i kappa h (s|u|^2 - 2 yhat.u) / (|yhat - s u| + 1)) / |yhat - s u|.

// LevelDEvaluations with one block per leaf box (leaf_box_f32): leaf boxes [b0, b0 + gridDim.x),
// value set blockIdx.y.
template <int PS, int PT, int PP>
__global__ void __launch_bounds__(kLeafThreads)
k_leaf_box_f32(const int32_t* __restrict__ bcs, const int32_t* __restrict__ cone_gam, LevelGrid g,
               const int32_t* __restrict__ startD, const float4* __restrict__ off, const float2* __restrict__ as,
               int64_t N, float kh, float hinv, const float* __restrict__ W, float2* __restrict__ coef, int cstride,
               int nrhs, int b0, int c_lo, int c_hi) {
    leaf_box_f32<PS, PT, PP>(bcs, cone_gam, g, startD, off, as, N, kh, hinv, W, coef, cstride, nrhs,
                             b0 + (int)blockIdx.x, (int)blockIdx.y, c_lo, c_hi);
}

template <int PS, int PT, int PP>
__global__ void k_leaf_f64(const int32_t* __restrict__ cone_box, const int32_t* __restrict__ cone_gam, LevelGrid g,
                           const int32_t* __restrict__ startD, const int4* __restrict__ kD,
                           const double* __restrict__ Xs, const double2* __restrict__ as, int64_t N, double kappa,
                           double a0, double a1, double a2, double HD, const double* __restrict__ W,
                           double2* __restrict__ coef, int cstride, int nrhs) {
    constexpr int P = PS * PT * PP;
    __shared__ double2 f[P], tmp[P];
    const int cone = blockIdx.x;
    const int r = blockIdx.y;
    const int n = threadIdx.x;
    const int b = cone_box[cone];
    if (n < P) {
        const int gam = cone_gam[cone];
        const int ip = gam % g.np, it = (gam / g.np) % g.nt, is = gam / (g.np * g.nt);
        const int ic = n % PP, ib = (n / PP) % PT, ia = n / (PP * PT);
        const int4 k = kD[b];
        const double xc = a0 + (k.x + 0.5) * HD, yc = a1 + (k.y + 0.5) * HD, zc = a2 + (k.z + 0.5) * HD;
        const double s = g.snode64[is * PS + ia], th = g.tnode64[it * PT + ib], ph = g.pnode64[ip * PP + ic];
        const double rr = g.h64 / s;
        const double yx = xc + rr * sin(th) * cos(ph), yy = yc + rr * sin(th) * sin(ph), yz = zc + rr * cos(th);
        const double rk = sqrt((yx - xc) * (yx - xc) + (yy - yc) * (yy - yc) + (yz - zc) * (yz - zc));
        const double2* ar = as + (int64_t)r * N;
        double2 acc = make_double2(0., 0.);
        for (int j = startD[b]; j < startD[b + 1]; ++j) {
            const double dx = yx - Xs[j], dy = yy - Xs[N + j], dz = yz - Xs[2 * N + j];
            const double dist = sqrt(dx * dx + dy * dy + dz * dz);
            double sn, cs;
            sincos(kappa * (dist - rk), &sn, &cs);
            const double w = rk / dist;
            acc = make_double2(acc.x + (ar[j].x * cs - ar[j].y * sn) * w, acc.y + (ar[j].x * sn + ar[j].y * cs) * w);
        }
        f[n] = acc;
    }
    __syncthreads();
    const double2 c = cheb_coeffs_smem<PS, PT, PP>(f, tmp, W, n);
    if (n < P) coef[((int64_t)cone * nrhs + r) * cstride + n] = c;
}

// Node offset (grid units, FP32) of node n of cone gamma from the centre of its box: the same
// correctly rounded products as the plan's activation, so the classification agrees with it.
__device__ __forceinline__ float3 node_grid(const LevelGrid& gp, int Ps, int Pt, int Pp, int gam, int n) {
    const int ip = gam % gp.np, it = (gam / gp.np) % gp.nt, is = gam / (gp.np * gp.nt);
    const int c = n % Pp, b = (n / Pp) % Pt, a = n / (Pp * Pt);
    const float rho = gp.rho[is * Ps + a];
    const float st = gp.stn[it * Pt + b], ct = gp.ctn[it * Pt + b];
    const float cp = gp.cpn[ip * Pp + c], sp = gp.spn[ip * Pp + c];
    return make_float3(__fmul_rn(rho, __fmul_rn(st, cp)), __fmul_rn(rho, __fmul_rn(st, sp)), __fmul_rn(rho, ct));
}

// ---- Propagation(d) (Algorithm 7) -----------------------------------------------------------
// Propagation, kPropCones parent cones per block (prop_cones_f32), value set blockIdx.y.
template <int PS, int PT, int PP>
__global__ void __launch_bounds__(kPropThreads, 8)
k_prop_f32(int64_t ncp, const int32_t* __restrict__ pcone_box, const int32_t* __restrict__ pcone_gam,
           const int4* __restrict__ kp, const int32_t* __restrict__ pcstart, LevelGrid gp,
           const int4* __restrict__ kd, ConeMap cm, LevelGrid g,
           const float2* __restrict__ cchild, float2* __restrict__ cparent, int sh, float ku,
           const float* __restrict__ W, int cstride, int nrhs, int* __restrict__ status) {
    __shared__ PropSmem<PS * PT * PP> sm;
    prop_cones_f32<PS, PT, PP, false>(sm, ncp, pcone_box, pcone_gam, kp, pcstart, gp, kd, cm, g, cchild, cparent, sh,
                                      ku, W, cstride, nrhs, status, (int64_t)blockIdx.x * kPropCones,
                                      (int)blockIdx.y);
}

// Propagation from the node tables, one warp per parent cone (prop_cone_warp_f32).
template <int PS, int PT, int PP, int NSETS>
__global__ void __launch_bounds__(32 * kWarpCones, 9)
k_prop_warp_f32(int64_t ncp, const int32_t* __restrict__ pcone_box, const int32_t* __restrict__ cone_gidx,
                const int4* __restrict__ kp, const int32_t* __restrict__ pcstart, const int4* __restrict__ kd,
                ConeMap cm, const float4* __restrict__ tab_t, const float2* __restrict__ tab_r,
                const int32_t* __restrict__ tab_k, const int32_t* __restrict__ tab_list,
                const int16_t* __restrict__ tab_perm, const int32_t* __restrict__ tab_nseg,
                const int32_t* __restrict__ tab_seg, const float2* __restrict__ cchild, float2* __restrict__ cparent,
                const float* __restrict__ W, int cstride, int nrhs, int* __restrict__ status) {
    const int64_t pc = (int64_t)blockIdx.x * kWarpCones + (threadIdx.x >> 5);
    prop_cone_warp_f32<PS, PT, PP, NSETS, false, void>(nullptr, ncp, pcone_box, cone_gidx, kp, pcstart, kd, cm, tab_t, tab_r,
                                                 tab_k, tab_list, tab_perm, tab_nseg, tab_seg, cchild, cparent, W,
                                                 cstride, nrhs, status, pc, threadIdx.x & 31);
}

template <int PS, int PT, int PP>
__global__ void k_prop_f64(const int32_t* __restrict__ pcone_box, const int32_t* __restrict__ pcone_gam,
                           const int4* __restrict__ kp, const int32_t* __restrict__ pcstart, LevelGrid gp,
                           const int4* __restrict__ kd, ConeMap cm, LevelGrid g,
                           const double2* __restrict__ cchild, double2* __restrict__ cparent, int sh, double kappa,
                           double a0, double a1, double a2, double Hd, const double* __restrict__ W, int cstride,
                           int nrhs, int* __restrict__ status) {
    constexpr int P = PS * PT * PP;
    __shared__ double2 f[P], tmp[P];
    const int pc = blockIdx.x;
    const int r = blockIdx.y;
    const int n = threadIdx.x;
    if (n < P) {
        const int jb = pcone_box[pc];
        const int gam = pcone_gam[pc];
        const float3 q = node_grid(gp, PS, PT, PP, gam, n);
        const int4 kj = kp[jb];
        const double Hp = 2.0 * Hd;
        const double xj = a0 + (kj.x + 0.5) * Hp, yj = a1 + (kj.y + 0.5) * Hp, zj = a2 + (kj.z + 0.5) * Hp;
        const int ip = gam % gp.np, it = (gam / gp.np) % gp.nt, is = gam / (gp.np * gp.nt);
        const int ic = n % PP, ib = (n / PP) % PT, ia = n / (PP * PT);
        const double s = gp.snode64[is * PS + ia], th = gp.tnode64[it * PT + ib], ph = gp.pnode64[ip * PP + ic];
        const double rr = gp.h64 / s;
        const double yx = xj + rr * sin(th) * cos(ph), yy = yj + rr * sin(th) * sin(ph), yz = zj + rr * cos(th);
        const double rj = sqrt((yx - xj) * (yx - xj) + (yy - yj) * (yy - yj) + (yz - zj) * (yz - zj));
        double2 acc = make_double2(0., 0.);
        for (int kb = pcstart[jb]; kb < pcstart[jb + 1]; ++kb) {
            const int4 kk = kd[kb];
            const float ox = (float)((2 * (kk.x - 2 * kj.x) - 1) << sh);
            const float oy = (float)((2 * (kk.y - 2 * kj.y) - 1) << sh);
            const float oz = (float)((2 * (kk.z - 2 * kj.z) - 1) << sh);
            const int gam = classify_f32(g, __fsub_rn(q.x, ox), __fsub_rn(q.y, oy), __fsub_rn(q.z, oz));
            const int sl = cm.find(kb, gam);
            if (sl < 0) {
                set_status(status, IFGF_ERR_INTERNAL);
                continue;
            }
            const double xk = a0 + (kk.x + 0.5) * Hd, yk = a1 + (kk.y + 0.5) * Hd, zk = a2 + (kk.z + 0.5) * Hd;
            double ts, tt, tp, rk;
            local_f64(g, gam, yx - xk, yy - yk, yz - zk, ts, tt, tp, rk);
            const double2 F = interp_f64<PS, PT, PP>(cchild + ((int64_t)sl * nrhs + r) * cstride, ts, tt, tp);
            double sn, cs;
            sincos(kappa * (rk - rj), &sn, &cs);
            const double w = rj / rk;
            const double2 t = cmul(F, make_double2(cs * w, sn * w));
            acc.x += t.x;
            acc.y += t.y;
        }
        f[n] = acc;
    }
    __syncthreads();
    const double2 c = cheb_coeffs_smem<PS, PT, PP>(f, tmp, W, n);
    if (n < P) cparent[((int64_t)pc * nrhs + r) * cstride + n] = c;
}

// ---- Interpolation(d) (Algorithm 8) -----------------------------------------------------------
// One thread per target (interp_target_f32), NR value sets per thread (grid row y covers sets
// [NR y, NR y + NR)), added to Is.
template <int PS, int PT, int PP, int NR>
__global__ void __launch_bounds__(kThreads, NR == 1 ? 5 : 4) k_interp_f32(int64_t N, int sh, const int32_t* __restrict__ pbox_d, const int32_t* __restrict__ pbox_D,
                             const int4* __restrict__ kD, const int4* __restrict__ kd, const int32_t* __restrict__ ncs,
                             const int32_t* __restrict__ cs, const float4* __restrict__ off,
                             ConeMap cm, LevelGrid g, const float2* __restrict__ coef,
                             const float* __restrict__ phtab, float ku, float inv4piu, float2* __restrict__ Is,
                             int cstride, int nrhs, int* __restrict__ status, int64_t i0, int64_t i1) {
    // targets [i0, i1) of the sorted points; Is is [nrhs][N]
    const int64_t i = i0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= i1) return;
    const int r0 = blockIdx.y * NR;
    const int nv = min(NR, nrhs - r0);
    float2 acc[NR];
    interp_target_f32<PS, PT, PP, NR, false>(i, r0, nv, sh, pbox_d, pbox_D, kD, kd, ncs, cs, off, cm, g, coef, phtab,
                                             ku, inv4piu, cstride, nrhs, status, acc);
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        if (r < nv) {
            float2* dst = Is + (int64_t)(r0 + r) * N + i;
            const float2 prev = *dst;
            *dst = make_float2(prev.x + acc[r].x, prev.y + acc[r].y);
        }
    }
}

template <int PS, int PT, int PP>
__global__ void k_interp_f64(int64_t N, int sh, const int32_t* __restrict__ pbox_d, const int32_t* __restrict__ pbox_D,
                             const int4* __restrict__ kD, const int4* __restrict__ kd, const int32_t* __restrict__ ncs,
                             const int32_t* __restrict__ cs, const float4* __restrict__ off,
                             const double* __restrict__ Xs, ConeMap cm, LevelGrid g,
                             const double2* __restrict__ coef, double kappa, double a0, double a1, double a2,
                             double Hd, double2* __restrict__ Is, int cstride, int nrhs, int* __restrict__ status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int r = blockIdx.y;
    const int A = pbox_d[i];
    const int4 kl = kD[pbox_D[i]];
    const float4 o = off[i];
    const double xi = Xs[i], yi = Xs[N + i], zi = Xs[2 * N + i];
    const double inv4pi = 0.079577471545947667884441881686257181;
    double2 acc = make_double2(0., 0.);
    for (int t = 0; t < ncs[A]; ++t) {
        const int B = cs[(int64_t)A * kMaxCous + t];
        if (!in_bounds(B, cm.nbox, status)) continue;
        const int4 kb = kd[B];
        const float vx = __fadd_rn((float)((2 * kl.x + 1) - ((2 * kb.x + 1) << sh)), o.x);
        const float vy = __fadd_rn((float)((2 * kl.y + 1) - ((2 * kb.y + 1) << sh)), o.y);
        const float vz = __fadd_rn((float)((2 * kl.z + 1) - ((2 * kb.z + 1) << sh)), o.z);
        const int gam = classify_f32(g, vx, vy, vz);
        const int s = cm.find(B, gam);
        if (s < 0) {
            set_status(status, IFGF_ERR_INTERNAL);
            continue;
        }
        const double xb = a0 + (kb.x + 0.5) * Hd, yb = a1 + (kb.y + 0.5) * Hd, zb = a2 + (kb.z + 0.5) * Hd;
        double ts, tt, tp, rr;
        local_f64(g, gam, xi - xb, yi - yb, zi - zb, ts, tt, tp, rr);
        const double2 F = interp_f64<PS, PT, PP>(coef + ((int64_t)s * nrhs + r) * cstride, ts, tt, tp);
        double sn, c;
        sincos(kappa * rr, &sn, &c);
        const double w = inv4pi / rr;
        const double2 tv = cmul(F, make_double2(c * w, sn * w));
        acc.x += tv.x;
        acc.y += tv.y;
    }
    double2* dst = Is + (int64_t)r * N + i;
    const double2 prev = *dst;
    *dst = make_double2(prev.x + acc.x, prev.y + acc.y);
}

// ---- many densities: tensor-core contractions (3xTF32) -----------------------------------------
// With nrhs densities the interpolant of a cone at a set of points is the dense product
// [points x P basis] * [P coefficients x (nrhs x re/im)]: one warp takes 16 points, and for each
// distinct cone among them an m16n8k8 TF32 MMA block (3xTF32 for FP32 accuracy) over 4*NT
// densities; the complex factor of each point is applied to its row in the epilogue.
constexpr int kMmaMinRhs = 4;    // densities from which the tensor-core kernels are used
constexpr int kChunk = 16;       // points per warp in the tensor-core kernels

// Distinct-cone loop of one warp: rows (r0, r1) of this thread carry cones a0, a1 (or are done);
// the warp visits each distinct cone once, calling body(alpha, mask0, mask1).
template <class Body>
__device__ __forceinline__ void for_each_cone(int a0, int a1, bool pend0, bool pend1, Body&& body) {
    for (int guard = 0; guard < 2 * kChunk; ++guard) {
        const unsigned pend = __ballot_sync(0xffffffffu, pend0 || pend1);
        if (!pend) break;
        const int src = __ffs(pend) - 1;
        const int alpha = __shfl_sync(0xffffffffu, pend0 ? a0 : a1, src);
        const bool m0 = pend0 && a0 == alpha, m1 = pend1 && a1 == alpha;
        body(alpha, m0, m1);
        pend0 = pend0 && !m0;
        pend1 = pend1 && !m1;
    }
}

template <int PS, int PT, int PP, int NT>
__global__ void __launch_bounds__(32 * ((PS * PT * PP + kChunk - 1) / kChunk))
k_prop_mma(int64_t ncp, const int32_t* __restrict__ pcone_box, const int32_t* __restrict__ pcone_gam,
           const int4* __restrict__ kp, const int32_t* __restrict__ pcstart, LevelGrid gp,
           const int4* __restrict__ kd, ConeMap cm, LevelGrid g,
           const float2* __restrict__ cchild, float2* __restrict__ cparent, int sh, float ku,
           const float* __restrict__ W, int cstride, int nrhs, int* __restrict__ status) {
    constexpr int P = PS * PT * PP;
    constexpr int NR = 4 * NT;
    constexpr int NTHR = 32 * ((P + kChunk - 1) / kChunk);
    __shared__ float2 f[NR][P], tmp[NR][P];
    const int64_t pc = blockIdx.x;
    const int rhs0 = blockIdx.y * NR;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gq = lane >> 2, tq = lane & 3;
    const int n0 = warp * kChunk + gq, n1 = n0 + 8;
    const bool v0 = n0 < P, v1 = n1 < P;
    const int jb = pcone_box[pc], gam = pcone_gam[pc];
    const int4 kj = kp[jb];
    auto node = [&](int n) -> float4 {
        const int ip = gam % gp.np, it = (gam / gp.np) % gp.nt, is = gam / (gp.np * gp.nt);
        const int qc = n % PP, qb = (n / PP) % PT, qa = n / (PP * PT);
        const float rho = gp.rho[is * PS + qa];
        const float st = gp.stn[it * PT + qb], ct = gp.ctn[it * PT + qb];
        const float cp = gp.cpn[ip * PP + qc], sp = gp.spn[ip * PP + qc];
        const float qx = __fmul_rn(rho, __fmul_rn(st, cp)), qy = __fmul_rn(rho, __fmul_rn(st, sp));
        const float qz = __fmul_rn(rho, ct);
        return make_float4(qx, qy, qz, sqrtf(fmaf(qx, qx, fmaf(qy, qy, qz * qz))));
    };
    const float4 q0 = v0 ? node(n0) : make_float4(0.f, 0.f, 1.f, 1.f);
    const float4 q1 = v1 ? node(n1) : make_float4(0.f, 0.f, 1.f, 1.f);
    const float oo = 3.0f * (float)(1 << sh) * (float)(1 << sh);
    float acc[NT][4];
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    for (int kb = pcstart[jb]; kb < pcstart[jb + 1]; ++kb) {
        const int4 kk = kd[kb];
        const float ox = (float)((2 * (kk.x - 2 * kj.x) - 1) << sh);
        const float oy = (float)((2 * (kk.y - 2 * kj.y) - 1) << sh);
        const float oz = (float)((2 * (kk.z - 2 * kj.z) - 1) << sh);
        const ConeLocal c0 = locate_f32(g, __fsub_rn(q0.x, ox), __fsub_rn(q0.y, oy), __fsub_rn(q0.z, oz));
        const ConeLocal c1 = locate_f32(g, __fsub_rn(q1.x, ox), __fsub_rn(q1.y, oy), __fsub_rn(q1.z, oz));
        auto ratio = [&](const float4& q, const ConeLocal& cl) -> float2 {
            const float qo = fmaf(q.x, ox, fmaf(q.y, oy, q.z * oz));
            const float dr = __fdividef(fmaf(-2.f, qo, oo), cl.r + q.w);
            const float2 e = cis_f32(ku * dr);
            const float w = __fdividef(q.w, cl.r);
            return make_float2(e.x * w, e.y * w);
        };
        const float2 rt0 = ratio(q0, c0), rt1 = ratio(q1, c1);
        float Ts0[PS], Tt0[PT], Tp0[PP], Ts1[PS], Tt1[PT], Tp1[PP];
        cheb_T<PS>(c0.ts, Ts0);
        cheb_T<PT>(c0.tt, Tt0);
        cheb_T<PP>(c0.tp, Tp0);
        cheb_T<PS>(c1.ts, Ts1);
        cheb_T<PT>(c1.tt, Tt1);
        cheb_T<PP>(c1.tp, Tp1);
        for_each_cone(c0.gamma(g), c1.gamma(g), v0, v1, [&](int alpha, bool m0, bool m1) {
            const int s = cm.find(kb, alpha);
            if (s < 0) {
                if (m0 || m1) set_status(status, IFGF_ERR_INTERNAL);
                return;
            }
            float c[NT][4];
#pragma unroll
            for (int j = 0; j < NT; ++j) c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.f;
            mma_interp_block<PS, PT, PP, NT>(Ts0, Tt0, Tp0, Ts1, Tt1, Tp1, m0, m1, cchild, s, nrhs, rhs0, cstride, c);
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                if (m0) {
                    acc[j][0] += rt0.x * c[j][0] - rt0.y * c[j][1];
                    acc[j][1] += rt0.x * c[j][1] + rt0.y * c[j][0];
                }
                if (m1) {
                    acc[j][2] += rt1.x * c[j][2] - rt1.y * c[j][3];
                    acc[j][3] += rt1.x * c[j][3] + rt1.y * c[j][2];
                }
            }
        });
    }
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        const int rl = j * 4 + tq;
        if (v0) f[rl][n0] = make_float2(acc[j][0], acc[j][1]);
        if (v1) f[rl][n1] = make_float2(acc[j][2], acc[j][3]);
    }
    __syncthreads();
    // Chebyshev coefficients of every density's node values (phi, theta, s passes)
    const float* Ws = W;
    const float* Wt = W + PS * PS;
    const float* Wp = Wt + PT * PT;
    for (int x = threadIdx.x; x < NR * P; x += NTHR) {
        const int rl = x / P, n = x - (x / P) * P;
        const int qc = n % PP, qb = (n / PP) % PT, qa = n / (PP * PT);
        float2 a = make_float2(0.f, 0.f);
        const float2* rw = &f[rl][(qa * PT + qb) * PP];
#pragma unroll
        for (int k = 0; k < PP; ++k) {
            const float w = Wp[qc * PP + k];
            a.x = fmaf(w, rw[k].x, a.x);
            a.y = fmaf(w, rw[k].y, a.y);
        }
        tmp[rl][n] = a;
    }
    __syncthreads();
    for (int x = threadIdx.x; x < NR * P; x += NTHR) {
        const int rl = x / P, n = x - (x / P) * P;
        const int qc = n % PP, qb = (n / PP) % PT, qa = n / (PP * PT);
        float2 a = make_float2(0.f, 0.f);
#pragma unroll
        for (int jj = 0; jj < PT; ++jj) {
            const float w = Wt[qb * PT + jj];
            const float2 v = tmp[rl][(qa * PT + jj) * PP + qc];
            a.x = fmaf(w, v.x, a.x);
            a.y = fmaf(w, v.y, a.y);
        }
        f[rl][n] = a;
    }
    __syncthreads();
    for (int x = threadIdx.x; x < NR * P; x += NTHR) {
        const int rl = x / P, n = x - (x / P) * P;
        if (rhs0 + rl >= nrhs) continue;
        const int qc = n % PP, qb = (n / PP) % PT, qa = n / (PP * PT);
        float2 a = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < PS; ++i) {
            const float w = Ws[qa * PS + i];
            const float2 v = f[rl][(i * PT + qb) * PP + qc];
            a.x = fmaf(w, v.x, a.x);
            a.y = fmaf(w, v.y, a.y);
        }
        cparent[(pc * nrhs + rhs0 + rl) * cstride + n] = a;
    }
}

// Propagation with many densities from the node tables (orders (3,5,5)). For a child cone
// alpha and a segment of <= 8 nodes of the parent cone that fall in it, the values of 8
// densities are the dense product
//     V[density][node] = sum_k C_alpha,density[k] W[k][node],  W[k][node] = T_a(t_s) T_b(t_theta) T_c(t_phi),
// one m16n8k8 tile per k-step in 3xTF32: A rows are re (row g) and im (row g + 8) of density g,
// K slot (k-step kk, column j) holds coefficient (r, c) with c = kk / 2, r = 8 (kk % 2) + j
// (r = 5a + b < 15; slot r = 15 is zero), and the 8 columns are the segment's nodes. Warp w
// owns densities 8w..8w+7 of the block for every node, so it accumulates the ratio-weighted
// products of all children into shared memory in a fixed order; its A fragments stay in
// registers for all segments of one child cone.
template <int NT>
__global__ void __launch_bounds__(16 * NT)
k_prop_mma_tab(int64_t ncp, const int32_t* __restrict__ pcone_box, const int32_t* __restrict__ cone_gidx,
               const int4* __restrict__ kp, const int32_t* __restrict__ pcstart, const int4* __restrict__ kd,
               ConeMap cm, const float4* __restrict__ tab_t,
               const float2* __restrict__ tab_r, const int32_t* __restrict__ tab_k,
               const int32_t* __restrict__ tab_list, const int16_t* __restrict__ tab_perm,
               const int32_t* __restrict__ tab_seg, const int32_t* __restrict__ tab_run,
               const float2* __restrict__ cchild, float2* __restrict__ cparent, const float* __restrict__ W,
               int cstride, int nrhs, int* __restrict__ status) {
    constexpr int PS = 3, PT = 5, PP = 5, P = 75;
    constexpr int NR = 4 * NT;         // densities of the block
    constexpr int NTHR = 16 * NT;      // NR / 8 warps
    static_assert(NR % 8 == 0, "a warp owns 8 densities");
    __shared__ float2 f[NR][P], tmp[NR][P];
    const int64_t pc = blockIdx.x;
    const int rhs0 = blockIdx.y * NR;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    for (int x = tid; x < NR * P; x += NTHR) f[x / P][x % P] = make_float2(0.f, 0.f);
    __syncthreads();
    const int jb = pcone_box[pc];
    const int g8 = cone_gidx[pc] * 8;
    const int4 kj = kp[jb];
    const int dens = rhs0 + 8 * warp + g;  // density of A rows g / g + 8
    const int dl = 8 * warp + g;           // its row in f
    const int kb0 = pcstart[jb], nch = pcstart[jb + 1] - kb0;
    // the children's rows, then the slots of their child cones (list positions below
    // kSlotCache), looked up by the whole block at once before the products
    __shared__ int s_row[8], s_K[8], s_sl[8][kSlotCache];
    if (tid < nch) {
        const int4 kk4 = kd[kb0 + tid];
        const int row = g8 + ((kk4.x - 2 * kj.x) | ((kk4.y - 2 * kj.y) << 1) | ((kk4.z - 2 * kj.z) << 2));
        s_row[tid] = row;
        s_K[tid] = __ldg(&tab_k[row]);
    }
    __syncthreads();
    for (int x = tid; x < nch * kSlotCache; x += NTHR) {
        const int ch = x / kSlotCache, kl = x - ch * kSlotCache;
        if (kl < s_K[ch]) s_sl[ch][kl] = cm.find(kb0 + ch, __ldg(&tab_list[(int64_t)s_row[ch] * kTabList + kl]));
    }
    __syncthreads();
    for (int ch = 0; ch < nch; ++ch) {
        const int kb = kb0 + ch;
        const int row = s_row[ch];
        const int64_t rowP = (int64_t)row * P;
        const int K = s_K[ch];
        for (int kl = 0; kl < K; ++kl) {
            const int sl = kl < kSlotCache ? s_sl[ch][kl] : cm.find(kb, __ldg(&tab_list[(int64_t)row * kTabList + kl]));
            if (sl < 0) set_status(status, IFGF_ERR_INTERNAL);
            const float2* blk = (sl >= 0 && dens < nrhs) ? cchild + ((int64_t)sl * nrhs + dens) * cstride : nullptr;
            uint32_t ah[10][4], al[10][4];
#pragma unroll
            for (int kk = 0; kk < 10; ++kk) {
                const int c = kk >> 1, r0 = 8 * (kk & 1) + t, r1 = r0 + 4;
                float2 v0 = make_float2(0.f, 0.f), v1 = make_float2(0.f, 0.f);
                if (blk) {
                    v0 = __ldg(blk + r0 * PP + c);
                    if (r1 < PS * PT) v1 = __ldg(blk + r1 * PP + c);
                }
                tf32_split(v0.x, ah[kk][0], al[kk][0]);
                tf32_split(v0.y, ah[kk][1], al[kk][1]);
                tf32_split(v1.x, ah[kk][2], al[kk][2]);
                tf32_split(v1.y, ah[kk][3], al[kk][3]);
            }
            const int sg0 = __ldg(&tab_run[(int64_t)row * (kTabList + 1) + kl]);
            const int sg1 = __ldg(&tab_run[(int64_t)row * (kTabList + 1) + kl + 1]);
            // segment descriptor and node coordinates one segment ahead of the contraction
            int pk = sg0 < sg1 ? __ldg(&tab_seg[rowP + sg0]) : 0;
            float4 t4 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (g < ((pk >> 8) & 0xff)) t4 = __ldg(&tab_t[rowP + (pk & 0xff) + g]);
            for (int sg = sg0; sg < sg1; ++sg) {
                const int pk_next = sg + 1 < sg1 ? __ldg(&tab_seg[rowP + sg + 1]) : 0;
                const int64_t e0 = rowP + (pk & 0xff);
                const int len = (pk >> 8) & 0xff;
                // weights of node g of the segment: U[q] = T_a(t_s) T_b(t_theta) for r = t + 4q
                float Uq[4] = {0.f, 0.f, 0.f, 0.f}, Tp[PP];
#pragma unroll
                for (int c = 0; c < PP; ++c) Tp[c] = 0.f;
                if (g < len) {
                    float Ts[PS], Tt[PT];
                    cheb_T<PS>(t4.x, Ts);
                    cheb_T<PT>(t4.y, Tt);
                    cheb_T<PP>(t4.z, Tp);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int rr = t + 4 * q, a = rr / PT;
                        Uq[q] = rr < PS * PT ? pick<PS>(Ts, a) * pick<PT>(Tt, rr - a * PT) : 0.f;
                    }
                }
                // two accumulator chains (even / odd k-steps) to overlap the MMA latency
                float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
                for (int kk = 0; kk < 10; ++kk) {
                    const int c = kk >> 1, h = kk & 1;
                    uint32_t bh[2], bl[2];
                    tf32_split(Uq[2 * h] * Tp[c], bh[0], bl[0]);
                    tf32_split(Uq[2 * h + 1] * Tp[c], bh[1], bl[1]);
                    mma_3xtf32(acc[h], ah[kk], al[kk], bh, bl);
                }
                t4 = make_float4(0.f, 0.f, 0.f, 0.f);
                if (g < ((pk_next >> 8) & 0xff)) t4 = __ldg(&tab_t[rowP + (pk_next & 0xff) + g]);
#pragma unroll
                for (int e = 0; e < 2; ++e) {  // (density g; nodes 2t, 2t+1 of the segment)
                    const int q = 2 * t + e;
                    if (q < len) {
                        const float2 v = cmul(make_float2(acc[0][e] + acc[1][e], acc[0][2 + e] + acc[1][2 + e]),
                                              __ldg(&tab_r[e0 + q]));
                        float2& dst = f[dl][__ldg(&tab_perm[e0 + q])];
                        dst.x += v.x;
                        dst.y += v.y;
                    }
                }
                pk = pk_next;
                __syncwarp();
            }
        }
    }
    __syncthreads();
    // Chebyshev coefficients of every density's node values (phi, theta, s passes)
    const float* Ws = W;
    const float* Wt = W + PS * PS;
    const float* Wp = Wt + PT * PT;
    for (int x = tid; x < NR * P; x += NTHR) {
        const int rl = x / P, n = x - (x / P) * P;
        const int qc = n % PP, qb = (n / PP) % PT, qa = n / (PP * PT);
        float2 a = make_float2(0.f, 0.f);
        const float2* rw = &f[rl][(qa * PT + qb) * PP];
#pragma unroll
        for (int k = 0; k < PP; ++k) {
            const float w = Wp[qc * PP + k];
            a.x = fmaf(w, rw[k].x, a.x);
            a.y = fmaf(w, rw[k].y, a.y);
        }
        tmp[rl][n] = a;
    }
    __syncthreads();
    for (int x = tid; x < NR * P; x += NTHR) {
        const int rl = x / P, n = x - (x / P) * P;
        const int qc = n % PP, qb = (n / PP) % PT, qa = n / (PP * PT);
        float2 a = make_float2(0.f, 0.f);
#pragma unroll
        for (int jj = 0; jj < PT; ++jj) {
            const float w = Wt[qb * PT + jj];
            const float2 v = tmp[rl][(qa * PT + jj) * PP + qc];
            a.x = fmaf(w, v.x, a.x);
            a.y = fmaf(w, v.y, a.y);
        }
        f[rl][n] = a;
    }
    __syncthreads();
    for (int x = tid; x < NR * P; x += NTHR) {
        const int rl = x / P, n = x - (x / P) * P;
        if (rhs0 + rl >= nrhs) continue;
        const int qc = n % PP, qb = (n / PP) % PT, qa = n / (PP * PT);
        float2 a = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < PS; ++i) {
            const float w = Ws[qa * PS + i];
            const float2 v = f[rl][(i * PT + qb) * PP + qc];
            a.x = fmaf(w, v.x, a.x);
            a.y = fmaf(w, v.y, a.y);
        }
        cparent[(pc * nrhs + rhs0 + rl) * cstride + n] = a;
    }
}

// Near field and leaf evaluation with a block of NR densities: the kernel value of each pair is
// computed once and applied to every density of the block.
template <int NR>
__global__ void k_near_f32_multi(int64_t N, const int32_t* __restrict__ pboxD, const int4* __restrict__ kD,
                                 const int32_t* __restrict__ startD, const int32_t* __restrict__ nnb,
                                 const int32_t* __restrict__ nb, const float4* __restrict__ off,
                                 const float2* __restrict__ as, float2* __restrict__ Is, float ku, float inv4piu,
                                 int nrhs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int rhs0 = blockIdx.y * NR;
    const int l = pboxD[i];
    const int4 kl = kD[l];
    const float4 oi = off[i];
    float2 acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = make_float2(0.f, 0.f);
    for (int t = 0; t < nnb[l]; ++t) {
        const int q = nb[(int64_t)l * kMaxNbr + t];
        const int4 kq = kD[q];
        const float bx = (float)(2 * (kl.x - kq.x)) + oi.x;
        const float by = (float)(2 * (kl.y - kq.y)) + oi.y;
        const float bz = (float)(2 * (kl.z - kq.z)) + oi.z;
        for (int j = startD[q]; j < startD[q + 1]; ++j) {
            if (j == i) continue;
            const float4 oj = __ldg(&off[j]);
            const float vx = bx - oj.x, vy = by - oj.y, vz = bz - oj.z;
            const float r2 = fmaf(vx, vx, fmaf(vy, vy, vz * vz));
            const float rinv = rsqrtf(r2);
            const float2 e = cis_f32(ku * (r2 * rinv));
            const float w = inv4piu * rinv;
            const float2 gk = make_float2(e.x * w, e.y * w);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                if (rhs0 + r >= nrhs) break;
                const float2 aj = __ldg(&as[(int64_t)(rhs0 + r) * N + j]);
                acc[r] = __ffma2_rn(make_float2(aj.x, aj.x), gk, acc[r]);
                acc[r] = __ffma2_rn(make_float2(-aj.y, aj.y), make_float2(gk.y, gk.x), acc[r]);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r)
        if (rhs0 + r < nrhs) Is[(int64_t)(rhs0 + r) * N + i] = acc[r];
}

// Chebyshev coefficients of NR value sets f[r][.] of one cone (separable analysis by the
// matrices Ws | Wt | Wp, last index first), stored to out[r * cstride + m] for r < nv; tmp is
// scratch of the same size. Every thread of the block calls it (it synchronises the block).
template <int PS, int PT, int PP, int NR>
__device__ __forceinline__ void cone_coeffs_block(float2 (*f)[PS * PT * PP], float2 (*tmp)[PS * PT * PP],
                                                  const float* __restrict__ W, float2* __restrict__ out, int cstride,
                                                  int nv) {
    constexpr int P = PS * PT * PP;
    constexpr int BT = ((P + 31) / 32) * 32;
    const float* Ws = W;
    const float* Wt = W + PS * PS;
    const float* Wp = Wt + PT * PT;
    for (int x = threadIdx.x; x < NR * P; x += BT) {
        const int rl = x / P, m = x - (x / P) * P;
        const int qc = m % PP, qb = (m / PP) % PT, qa = m / (PP * PT);
        float2 a = make_float2(0.f, 0.f);
        const float2* rw = &f[rl][(qa * PT + qb) * PP];
#pragma unroll
        for (int k = 0; k < PP; ++k) {
            const float w = Wp[qc * PP + k];
            a.x = fmaf(w, rw[k].x, a.x);
            a.y = fmaf(w, rw[k].y, a.y);
        }
        tmp[rl][m] = a;
    }
    __syncthreads();
    for (int x = threadIdx.x; x < NR * P; x += BT) {
        const int rl = x / P, m = x - (x / P) * P;
        const int qc = m % PP, qb = (m / PP) % PT, qa = m / (PP * PT);
        float2 a = make_float2(0.f, 0.f);
#pragma unroll
        for (int jj = 0; jj < PT; ++jj) {
            const float w = Wt[qb * PT + jj];
            const float2 v = tmp[rl][(qa * PT + jj) * PP + qc];
            a.x = fmaf(w, v.x, a.x);
            a.y = fmaf(w, v.y, a.y);
        }
        f[rl][m] = a;
    }
    __syncthreads();
    for (int x = threadIdx.x; x < NR * P; x += BT) {
        const int rl = x / P, m = x - (x / P) * P;
        if (rl >= nv) continue;
        const int qc = m % PP, qb = (m / PP) % PT, qa = m / (PP * PT);
        float2 a = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < PS; ++i) {
            const float w = Ws[qa * PS + i];
            const float2 v = f[rl][(i * PT + qb) * PP + qc];
            a.x = fmaf(w, v.x, a.x);
            a.y = fmaf(w, v.y, a.y);
        }
        out[(int64_t)rl * cstride + m] = a;
    }
}

template <int PS, int PT, int PP, int NR>
__global__ void k_leaf_f32_multi(const int32_t* __restrict__ cone_box, const int32_t* __restrict__ cone_gam,
                                 LevelGrid g, const int32_t* __restrict__ startD, const float4* __restrict__ off,
                                 const float2* __restrict__ as, int64_t N, float kh, float hinv,
                                 const float* __restrict__ W, float2* __restrict__ coef, int cstride, int nrhs) {
    constexpr int P = PS * PT * PP;
    __shared__ float2 f[NR][P], tmp[NR][P];
    const int cone = blockIdx.x;
    const int rhs0 = blockIdx.y * NR;
    const int n = threadIdx.x;
    const int b = cone_box[cone];
    if (n < P) {
        const int gam = cone_gam[cone];
        const int ip = gam % g.np, it = (gam / g.np) % g.nt, is = gam / (g.np * g.nt);
        const int ic = n % PP, ib = (n / PP) % PT, ia = n / (PP * PT);
        const float s = g.snode[is * PS + ia];
        const float st = g.stn[it * PT + ib], ct = g.ctn[it * PT + ib];
        const float yx = st * g.cpn[ip * PP + ic], yy = st * g.spn[ip * PP + ic], yz = ct;
        float2 acc[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[r] = make_float2(0.f, 0.f);
        for (int j = startD[b]; j < startD[b + 1]; ++j) {
            const float4 o = __ldg(&off[j]);
            const float ux = o.x * hinv, uy = o.y * hinv, uz = o.z * hinv;
            const float wx = fmaf(-s, ux, yx), wy = fmaf(-s, uy, yy), wz = fmaf(-s, uz, yz);
            const float q = fmaf(wx, wx, fmaf(wy, wy, wz * wz));
            const float rq = rsqrtf(q);
            const float uu = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
            const float yu = fmaf(yx, ux, fmaf(yy, uy, yz * uz));
            const float ph = kh * __fdividef(fmaf(s, uu, -2.f * yu), fmaf(q, rq, 1.f));
            const float2 e = cis_f32(ph);
            const float2 gk = make_float2(e.x * rq, e.y * rq);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                if (rhs0 + r >= nrhs) break;
                const float2 aj = __ldg(&as[(int64_t)(rhs0 + r) * N + j]);
                acc[r] = __ffma2_rn(make_float2(aj.x, aj.x), gk, acc[r]);
                acc[r] = __ffma2_rn(make_float2(-aj.y, aj.y), make_float2(gk.y, gk.x), acc[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) f[r][n] = acc[r];
    }
    __syncthreads();
    cone_coeffs_block<PS, PT, PP, NR>(f, tmp, W, coef + ((int64_t)cone * nrhs + rhs0) * cstride, cstride,
                                      nrhs - rhs0);
}

// ---- Stokes and elasticity kernels ----------------------------------------------------------
// Green tensors of the form S_ij(x,y) = c (alpha delta_ij/r + r_i r_j/r^3) with r = x - y, acting
// on real force vectors (the Stokes and elasticity equations are among the kernels Sec. 2 names
// for Eq. (1)): the Stokeslet (c = 1/(8 pi mu), alpha = 1) and Kelvin's solution of linear
// elasticity (c = 1/(16 pi mu (1 - nu)), alpha = 3 - 4 nu). Their centred factor is the Laplace
// one, G_0(x,x_k) = 1/(4 pi |x - x_k|), and their analytic factor S(x,x')/G_0(x,x_k) (Eq. (3))
// is smooth in the cone variables, so that each velocity (displacement) component is carried
// through propagation and interpolation as a kappa = 0 value set. The kernels stage alpha f and
// use beta = 1/alpha: S f = c (alpha f + r (r . alpha f) beta / r^2) / |r|.
// The three real components of force field f occupy reals q = 3f + c of the complex slots, slot
// q/2, real part for even q: ceil(3 nf / 2) complex sets. Forces in Morton order are SoA,
// fs[(3 f + c) N + j]; the kernels below take fields in pairs starting at an even field (three
// complete slots), or the last field of an odd count alone (two slots, the second's imaginary
// part zero).

// Near field: the tiling and the S-way split of a target's sources of k_near_tile_f32, with the
// NF force vectors of each staged source held in shared memory next to its position.
template <int NF>
__global__ void __launch_bounds__(kNearThreads)
k_near_stokes_f32(const int4* __restrict__ kD, const int32_t* __restrict__ startD, const int32_t* __restrict__ nnb,
                  const int32_t* __restrict__ nb, const float4* __restrict__ off, const float* __restrict__ fs,
                  float2* __restrict__ Is, int64_t N, float alpha, float beta, float cu, int f0) {
    __shared__ float4 s_p[kNearTile];  // source position in the target box's grid frame; w = source index
    __shared__ float4 s_f[NF][kNearTile];
    const int l = blockIdx.x;
    const int f = f0 + NF * blockIdx.y;
    const int tid = threadIdx.x;
    const int t0 = startD[l], m = startD[l + 1] - t0;
    const int4 kl = kD[l];
    int S = 1;
    while (S < 32 && 2 * S * m <= kNearThreads) S *= 2;
    const int per_pass = kNearThreads / S;
    const int cnt = nnb[l];
    for (int base = 0; base < m; base += per_pass) {
        const int tl = base + tid / S, part = tid % S;
        const bool active = tl < m;
        const int i = t0 + (active ? tl : 0);
        const float4 oi = off[i];
        float acc[NF][3];
#pragma unroll
        for (int r = 0; r < NF; ++r) acc[r][0] = acc[r][1] = acc[r][2] = 0.f;
        for (int nq = 0; nq < cnt; ++nq) {
            const int q = nb[(int64_t)l * kMaxNbr + nq];
            const int4 kq = kD[q];
            const float sx = (float)(2 * (kl.x - kq.x)), sy = (float)(2 * (kl.y - kq.y)),
                        sz = (float)(2 * (kl.z - kq.z));
            const int j0 = startD[q], j1 = startD[q + 1];
            for (int tb = j0; tb < j1; tb += kNearTile) {
                const int nt = min(kNearTile, j1 - tb);
                __syncthreads();
                if (tid < nt) {
                    const int j = tb + tid;
                    const float4 oj = __ldg(&off[j]);
                    s_p[tid] = make_float4(oj.x - sx, oj.y - sy, oj.z - sz, __int_as_float(j));
#pragma unroll
                    for (int r = 0; r < NF; ++r) {
                        const float* fr = fs + (int64_t)3 * (f + r) * N + j;
                        s_f[r][tid] = make_float4(alpha * __ldg(fr), alpha * __ldg(fr + N), alpha * __ldg(fr + 2 * N), 0.f);
                    }
                }
                __syncthreads();
                if (active) {
                    for (int k = part; k < nt; k += S) {
                        const float4 pj = s_p[k];
                        if (__float_as_int(pj.w) == i) continue;
                        const float vx = oi.x - pj.x, vy = oi.y - pj.y, vz = oi.z - pj.z;
                        const float r2 = fmaf(vx, vx, fmaf(vy, vy, vz * vz));
                        const float rinv = rsqrtf(r2);
                        const float rinv2 = rinv * rinv * beta;
#pragma unroll
                        for (int r = 0; r < NF; ++r) {
                            const float4 fj = s_f[r][k];  // alpha f
                            const float t = fmaf(vx, fj.x, fmaf(vy, fj.y, vz * fj.z)) * rinv2;
                            acc[r][0] = fmaf(rinv, fmaf(t, vx, fj.x), acc[r][0]);
                            acc[r][1] = fmaf(rinv, fmaf(t, vy, fj.y), acc[r][1]);
                            acc[r][2] = fmaf(rinv, fmaf(t, vz, fj.z), acc[r][2]);
                        }
                    }
                }
            }
        }
        for (int o = S / 2; o >= 1; o >>= 1) {  // the S partial sums of a target, fixed order
#pragma unroll
            for (int r = 0; r < NF; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) acc[r][c] += __shfl_xor_sync(0xffffffffu, acc[r][c], o);
        }
        if (active && part == 0) {
            float2* o = Is + (int64_t)(3 * f / 2) * N + i;
            o[0] = make_float2(acc[0][0] * cu, acc[0][1] * cu);
            if constexpr (NF == 2) {
                o[N] = make_float2(acc[0][2] * cu, acc[1][0] * cu);
                o[2 * N] = make_float2(acc[1][1] * cu, acc[1][2] * cu);
            } else {
                o[N] = make_float2(acc[0][2] * cu, 0.f);
            }
        }
    }
}

// Leaf level (Algorithm 6) for these kernels, one block per leaf box as in k_leaf_box_f32: the box's
// sources (u = (x' - x_k)/h and the NF force vectors) are staged in shared memory once per pass and
// swept by every (cone, node) of the box, NCP cones at a time. At node y = x_k + (h/s) yhat the
// analytic factor is S(y, x')/G_0(y, x_k) = 4 pi c rq (alpha I + w w^T rq^2) with w = yhat - s u
// and rq = 1/|w|; the factor 4 pi c (fscale) is applied to the coefficients. Then one warp per
// (cone, complex set) computes the coefficients.
template <int PS, int PT, int PP, int NF>
__global__ void __launch_bounds__(kLeafThreads)
k_leaf_stokes_f32(const int32_t* __restrict__ bcs, const int32_t* __restrict__ cone_gam, LevelGrid g,
                  const int32_t* __restrict__ startD, const float4* __restrict__ off, const float* __restrict__ fs,
                  int64_t N, float hinv, const float* __restrict__ W, float2* __restrict__ coef, int cstride,
                  int nrhs, float alpha, float beta, float fscale, int f0) {
    constexpr int P = PS * PT * PP;
    constexpr int NS = NF == 2 ? 3 : 2;  // complex sets of the block's fields
    constexpr int NW = kLeafThreads / 32;
    constexpr int NCP = P <= 75 ? 16 : 2;  // cones per pass (shared memory below 48 KB)
    __shared__ float4 s_u[kLeafSrc];
    __shared__ float4 s_f[NF][kLeafSrc];
    __shared__ float2 v[NCP][NS][P];
    __shared__ float2 tmp[NW][P];
    const int b = blockIdx.x;
    const int f = f0 + NF * blockIdx.y;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int c0 = bcs[b], c1 = bcs[b + 1];
    if (c0 == c1) return;
    const int j0 = startD[b], j1 = startD[b + 1];
    const float* Ws = W;
    const float* Wt = W + PS * PS;
    const float* Wp = Wt + PT * PT;
    for (int cc = c0; cc < c1; cc += NCP) {
        const int ncc = min(NCP, c1 - cc);
        const int items = ncc * P;
        for (int t0 = j0; t0 < j1; t0 += kLeafSrc) {
            const int nt = min(kLeafSrc, j1 - t0);
            __syncthreads();
            if (tid < nt) {
                const int j = t0 + tid;
                const float4 o = __ldg(&off[j]);
                s_u[tid] = make_float4(o.x * hinv, o.y * hinv, o.z * hinv, 0.f);
#pragma unroll
                for (int r = 0; r < NF; ++r) {
                    const float* fr = fs + (int64_t)3 * (f + r) * N + j;
                    s_f[r][tid] = make_float4(alpha * __ldg(fr), alpha * __ldg(fr + N), alpha * __ldg(fr + 2 * N), 0.f);
                }
            }
            __syncthreads();
            for (int item = tid; item < items; item += kLeafThreads) {
                const int cl = item / P, n = item - (item / P) * P;
                const int gam = __ldg(&cone_gam[cc + cl]);
                const int ip = gam % g.np, it = (gam / g.np) % g.nt, is = gam / (g.np * g.nt);
                const int ic = n % PP, ib = (n / PP) % PT, ia = n / (PP * PT);
                const float sn = __ldg(&g.snode[is * PS + ia]);
                const float st = __ldg(&g.stn[it * PT + ib]), ct = __ldg(&g.ctn[it * PT + ib]);
                const float yx = st * __ldg(&g.cpn[ip * PP + ic]), yy = st * __ldg(&g.spn[ip * PP + ic]), yz = ct;
                float acc[NF][3];
                if (t0 == j0) {
#pragma unroll
                    for (int r = 0; r < NF; ++r) acc[r][0] = acc[r][1] = acc[r][2] = 0.f;
                } else {
                    const float2 a0 = v[cl][0][n], a1 = v[cl][1][n];
                    acc[0][0] = a0.x;
                    acc[0][1] = a0.y;
                    acc[0][2] = a1.x;
                    if constexpr (NF == 2) {
                        const float2 a2 = v[cl][2][n];
                        acc[1][0] = a1.y;
                        acc[1][1] = a2.x;
                        acc[1][2] = a2.y;
                    }
                }
#pragma unroll 2
                for (int j = 0; j < nt; ++j) {
                    const float4 u = s_u[j];
                    const float wx = fmaf(-sn, u.x, yx), wy = fmaf(-sn, u.y, yy), wz = fmaf(-sn, u.z, yz);
                    const float q = fmaf(wx, wx, fmaf(wy, wy, wz * wz));
                    const float rq = rsqrtf(q);
                    const float rq2 = rq * rq * beta;
#pragma unroll
                    for (int r = 0; r < NF; ++r) {
                        const float4 fj = s_f[r][j];  // alpha f
                        const float t = fmaf(wx, fj.x, fmaf(wy, fj.y, wz * fj.z)) * rq2;
                        acc[r][0] = fmaf(rq, fmaf(t, wx, fj.x), acc[r][0]);
                        acc[r][1] = fmaf(rq, fmaf(t, wy, fj.y), acc[r][1]);
                        acc[r][2] = fmaf(rq, fmaf(t, wz, fj.z), acc[r][2]);
                    }
                }
                v[cl][0][n] = make_float2(acc[0][0], acc[0][1]);
                if constexpr (NF == 2) {
                    v[cl][1][n] = make_float2(acc[0][2], acc[1][0]);
                    v[cl][2][n] = make_float2(acc[1][1], acc[1][2]);
                } else {
                    v[cl][1][n] = make_float2(acc[0][2], 0.f);
                }
            }
        }
        __syncthreads();
        for (int x = warp; x < ncc * NS; x += NW) {  // coefficient transform, one warp per (cone, set)
            const int cl = x / NS, sl = x - (x / NS) * NS;
            float2* fv = v[cl][sl];
            float2* tv = tmp[warp];
            for (int n = lane; n < P; n += 32) {
                const int qc = n % PP, qb = (n / PP) % PT, qa = n / (PP * PT);
                float2 a = make_float2(0.f, 0.f);
#pragma unroll
                for (int k = 0; k < PP; ++k) {
                    const float w = Wp[qc * PP + k];
                    const float2 z = fv[(qa * PT + qb) * PP + k];
                    a.x = fmaf(w, z.x, a.x);
                    a.y = fmaf(w, z.y, a.y);
                }
                tv[n] = a;
            }
            __syncwarp();
            for (int n = lane; n < P; n += 32) {
                const int qc = n % PP, qb = (n / PP) % PT, qa = n / (PP * PT);
                float2 a = make_float2(0.f, 0.f);
#pragma unroll
                for (int k = 0; k < PT; ++k) {
                    const float w = Wt[qb * PT + k];
                    const float2 z = tv[(qa * PT + k) * PP + qc];
                    a.x = fmaf(w, z.x, a.x);
                    a.y = fmaf(w, z.y, a.y);
                }
                fv[n] = a;
            }
            __syncwarp();
            for (int n = lane; n < P; n += 32) {
                const int qc = n % PP, qb = (n / PP) % PT, qa = n / (PP * PT);
                float2 a = make_float2(0.f, 0.f);
#pragma unroll
                for (int k = 0; k < PS; ++k) {
                    const float w = Ws[qa * PS + k];
                    const float2 z = fv[(k * PT + qb) * PP + qc];
                    a.x = fmaf(w, z.x, a.x);
                    a.y = fmaf(w, z.y, a.y);
                }
                coef[((int64_t)(cc + cl) * nrhs + 3 * f / 2 + sl) * cstride + n] = make_float2(fscale * a.x, fscale * a.y);
            }
            __syncwarp();
        }
    }
}

// FP64 near field for these kernels (physical coordinates, one thread per target as k_near_f64):
// NF force fields starting at the even field f0 + NF blockIdx.y, written to their complex slots.
template <int NF>
__global__ void k_near_stokes_f64(int64_t N, const int32_t* __restrict__ pboxD, const int32_t* __restrict__ startD,
                                  const int32_t* __restrict__ nnb, const int32_t* __restrict__ nb,
                                  const double* __restrict__ Xs, const double* __restrict__ fs,
                                  double2* __restrict__ Is, double alpha, double c, int f0) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int f = f0 + NF * blockIdx.y;
    const int l = pboxD[i];
    const double xi = Xs[i], yi = Xs[N + i], zi = Xs[2 * N + i];
    double acc[NF][3];
#pragma unroll
    for (int r = 0; r < NF; ++r) acc[r][0] = acc[r][1] = acc[r][2] = 0.0;
    for (int t = 0; t < nnb[l]; ++t) {
        const int q = nb[(int64_t)l * kMaxNbr + t];
        for (int j = startD[q]; j < startD[q + 1]; ++j) {
            if (j == i) continue;
            const double vx = xi - Xs[j], vy = yi - Xs[N + j], vz = zi - Xs[2 * N + j];
            const double r2 = vx * vx + vy * vy + vz * vz;
            const double rr = sqrt(r2);
#pragma unroll
            for (int r = 0; r < NF; ++r) {
                const double* fr = fs + (int64_t)3 * (f + r) * N + j;
                const double fx = fr[0], fy = fr[N], fz = fr[2 * N];
                const double t3 = (vx * fx + vy * fy + vz * fz) / r2;
                acc[r][0] += (alpha * fx + t3 * vx) / rr;
                acc[r][1] += (alpha * fy + t3 * vy) / rr;
                acc[r][2] += (alpha * fz + t3 * vz) / rr;
            }
        }
    }
    double2* o = Is + (int64_t)(3 * f / 2) * N + i;
    o[0] = make_double2(c * acc[0][0], c * acc[0][1]);
    if constexpr (NF == 2) {
        o[N] = make_double2(c * acc[0][2], c * acc[1][0]);
        o[2 * N] = make_double2(c * acc[1][1], c * acc[1][2]);
    } else {
        o[N] = make_double2(c * acc[0][2], 0.0);
    }
}

// FP64 leaf level for these kernels (one block per leaf cone, one thread per node, as k_leaf_f64):
// the analytic factor S(y, x')/G_0(y, x_k) = 4 pi |y - x_k| S(y, x'), then the coefficients of
// each complex set of the block's fields.
template <int PS, int PT, int PP, int NF>
__global__ void k_leaf_stokes_f64(const int32_t* __restrict__ cone_box, const int32_t* __restrict__ cone_gam,
                                  LevelGrid g, const int32_t* __restrict__ startD, const int4* __restrict__ kD,
                                  const double* __restrict__ Xs, const double* __restrict__ fs, int64_t N, double a0,
                                  double a1, double a2, double HD, const double* __restrict__ W,
                                  double2* __restrict__ coef, int cstride, int nrhs, double alpha, double c, int f0) {
    constexpr int P = PS * PT * PP;
    constexpr int NS = NF == 2 ? 3 : 2;
    __shared__ double2 v[NS][P], tmp[P];
    const int cone = blockIdx.x;
    const int f = f0 + NF * blockIdx.y;
    const int n = threadIdx.x;
    const int b = cone_box[cone];
    if (n < P) {
        const int gam = cone_gam[cone];
        const int ip = gam % g.np, it = (gam / g.np) % g.nt, is = gam / (g.np * g.nt);
        const int ic = n % PP, ib = (n / PP) % PT, ia = n / (PP * PT);
        const int4 k = kD[b];
        const double xc = a0 + (k.x + 0.5) * HD, yc = a1 + (k.y + 0.5) * HD, zc = a2 + (k.z + 0.5) * HD;
        const double s = g.snode64[is * PS + ia], th = g.tnode64[it * PT + ib], ph = g.pnode64[ip * PP + ic];
        const double rr = g.h64 / s;
        const double yx = xc + rr * sin(th) * cos(ph), yy = yc + rr * sin(th) * sin(ph), yz = zc + rr * cos(th);
        const double rk = sqrt((yx - xc) * (yx - xc) + (yy - yc) * (yy - yc) + (yz - zc) * (yz - zc));
        double acc[NF][3];
#pragma unroll
        for (int r = 0; r < NF; ++r) acc[r][0] = acc[r][1] = acc[r][2] = 0.0;
        for (int j = startD[b]; j < startD[b + 1]; ++j) {
            const double vx = yx - Xs[j], vy = yy - Xs[N + j], vz = yz - Xs[2 * N + j];
            const double r2 = vx * vx + vy * vy + vz * vz;
            const double dist = sqrt(r2);
#pragma unroll
            for (int r = 0; r < NF; ++r) {
                const double* fr = fs + (int64_t)3 * (f + r) * N + j;
                const double fx = fr[0], fy = fr[N], fz = fr[2 * N];
                const double t3 = (vx * fx + vy * fy + vz * fz) / r2;
                acc[r][0] += (alpha * fx + t3 * vx) / dist;
                acc[r][1] += (alpha * fy + t3 * vy) / dist;
                acc[r][2] += (alpha * fz + t3 * vz) / dist;
            }
        }
        const double w = 4.0 * M_PI * rk * c;
        v[0][n] = make_double2(w * acc[0][0], w * acc[0][1]);
        if constexpr (NF == 2) {
            v[1][n] = make_double2(w * acc[0][2], w * acc[1][0]);
            v[2][n] = make_double2(w * acc[1][1], w * acc[1][2]);
        } else {
            v[1][n] = make_double2(w * acc[0][2], 0.0);
        }
    }
    __syncthreads();
#pragma unroll
    for (int sl = 0; sl < NS; ++sl) {
        const double2 cf = cheb_coeffs_smem<PS, PT, PP>(v[sl], tmp, W, n);
        if (n < P) coef[((int64_t)cone * nrhs + 3 * f / 2 + sl) * cstride + n] = cf;
    }
}

// FP64 velocities back to the caller's order.
__global__ void k_perm_out_stokes_f64(const double2* __restrict__ Is, const int32_t* __restrict__ perm, int64_t N,
                                      double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int q = blockIdx.y;
    const double2 v = Is[(int64_t)(q >> 1) * N + i];
    out[(int64_t)q * N + perm[i]] = (q & 1) ? v.y : v.x;
}

// Velocities back to the caller's order: real q of the slots -> out[q][perm[i]].
__global__ void k_perm_out_stokes(const float2* __restrict__ Is, const int32_t* __restrict__ perm, int64_t N,
                                  float* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int q = blockIdx.y;
    const float2 v = Is[(int64_t)(q >> 1) * N + i];
    out[(int64_t)q * N + perm[i]] = (q & 1) ? v.y : v.x;
}

// ---- driver -------------------------------------------------------------------------------
// Mixed precision with many densities: tensor-core propagation and interpolation, density-
// blocked near field and leaf evaluation.
// Propagation into level d-1, slice by slice in the order the coefficient arena requires (the
// parents are written at the other end of the arena from the children being read): launch(lo, n)
// runs the parent cones [lo, lo + n).
template <class F>
void for_each_slice(const Plan& p, int d, F&& launch) {
    const std::vector<int64_t>& b = p.L[d - 1].pslice;
    const int ks = (int)b.size() - 1;
    const bool child_at_start = (p.D - d) % 2 == 0;
    for (int j = 0; j < ks; ++j) {
        const int i = child_at_start ? ks - 1 - j : j;
        if (b[i + 1] > b[i]) launch(b[i], b[i + 1] - b[i]);
    }
}

// Interpolation to the targets [i0, i1) of level d for nrhs value sets, from the coefficients c
// found through cm: one set per thread for a single set, else two or four sets per thread sharing
// the geometry.
template <int PS, int PT, int PP>
void launch_interp_f32(Plan& p, int d, int nrhs, float2* Is, cudaStream_t s, ConeMap cm, const float2* c, int64_t i0,
                       int64_t i1) {
    const int64_t N = p.N;
    Level& L = p.L[d];
    Level& LD = p.L[p.D];
    const int sh = p.D - d;
    const float ku = (float)(p.kappa * p.u);
    const float inv4piu = (float)(1.0 / (4.0 * M_PI * p.u));
    const unsigned gx = grid_for(i1 - i0, kThreads);
    if (i1 <= i0) return;
    if (nrhs == 1)
        IFGF_LAUNCH((k_interp_f32<PS, PT, PP, 1>), dim3(gx, 1), kThreads, 0, s, N, sh, L.pbox, LD.pbox, LD.k, L.k,
                    L.ncs, L.cs, p.off, cm, L.g, c, L.phtab, ku, inv4piu, Is, p.cstride, nrhs, p.d_status, i0, i1);
    else if (nrhs <= 3)
        IFGF_LAUNCH((k_interp_f32<PS, PT, PP, 2>), dim3(gx, (nrhs + 1) / 2), kThreads, 0, s, N, sh, L.pbox, LD.pbox,
                    LD.k, L.k, L.ncs, L.cs, p.off, cm, L.g, c, L.phtab, ku, inv4piu, Is, p.cstride, nrhs, p.d_status, i0,
                    i1);
    else
        IFGF_LAUNCH((k_interp_f32<PS, PT, PP, 4>), dim3(gx, (nrhs + 3) / 4), kThreads, 0, s, N, sh, L.pbox, LD.pbox,
                    LD.k, L.k, L.ncs, L.cs, p.off, cm, L.g, c, L.phtab, ku, inv4piu, Is, p.cstride, nrhs, p.d_status, i0,
                    i1);
}

// Interpolation to every target of level d from the level's coefficients.
template <int PS, int PT, int PP>
void launch_interp_f32(Plan& p, int d, int nrhs, float2* Is, cudaStream_t s) {
    launch_interp_f32<PS, PT, PP>(p, d, nrhs, Is, s, p.L[d].cmap(p.d_status), (const float2*)level_coef(p, d, nrhs), 0, p.N);
}

// Levels D..3 of the many-density path: interpolation to the targets of level d (Algorithm 8),
// then propagation into level d-1 (Algorithm 7) on the tensor cores.
template <int NT, int PS, int PT, int PP>
void sweep_levels_mma(Plan& p, int nrhs, float2* Is, cudaStream_t s, int64_t mask) {
    constexpr int P = PS * PT * PP;
    constexpr int NR = 4 * NT;
    const int D = p.D;
    const float ku = (float)(p.kappa * p.u);
    const unsigned rb = (unsigned)((nrhs + NR - 1) / NR);
    for (int d = D; d >= 3; --d) {
        TimingLevel tl_(d);
        Level& L = p.L[d];
        const int sh = D - d;
        if ((mask >> d) & 1) {
            TimedScope ts_(TK_INTERP, s);
            launch_interp_f32<PS, PT, PP>(p, d, nrhs, Is, s);
        }
        if (d == 3) break;
        Level& Lp = p.L[d - 1];
        const float2* cc = (const float2*)level_coef(p, d, nrhs);
        float2* cp = (float2*)level_coef(p, d - 1, nrhs);
        const int64_t cone = (int64_t)nrhs * p.cstride;
        if (Lp.nc > 0 && Lp.n_gam > 0 && L.knob_many == 1) {
            // node-table levels on the fifth-generation tensor cores (tcgen05, TMEM accumulators)
            TimedScope ts_(TK_PROP, s);
            for_each_slice(p, d, [&](int64_t lo, int64_t n) { launch_prop_tc_tab(p, d, nrhs, lo, n, cc, cp + lo * cone, s); });
        } else if (Lp.nc > 0 && Lp.n_gam > 0) {
            TimedScope ts_(TK_PROP, s);
            for_each_slice(p, d, [&](int64_t lo, int64_t n) {
                IFGF_LAUNCH(k_prop_mma_tab<NT>, dim3((unsigned)n, rb), 16 * NT, 0, s, n, Lp.cone_box + lo,
                            Lp.cone_gidx + lo, Lp.k, Lp.cstart, L.k, L.cmap(p.d_status), Lp.tab_t, Lp.tab_r, Lp.tab_k, Lp.tab_list,
                            Lp.tab_perm, Lp.tab_seg, Lp.tab_run, cc, cp + lo * cone, p.Wf, p.cstride, nrhs, p.d_status);
            });
        } else if (Lp.nc > 0) {
            TimedScope ts_(TK_PROP_GEN, s);
            for_each_slice(p, d, [&](int64_t lo, int64_t n) {
                IFGF_LAUNCH((k_prop_mma<PS, PT, PP, NT>), dim3((unsigned)n, rb), 32 * ((P + kChunk - 1) / kChunk), 0, s,
                            n, Lp.cone_box + lo, Lp.cone_gam + lo, Lp.k, Lp.cstart, Lp.g, L.k, L.cmap(p.d_status), L.g, cc,
                            cp + lo * cone, sh, ku, p.Wf, p.cstride, nrhs, p.d_status);
            });
        }
    }
}

template <int NT, int PS, int PT, int PP>
void run_apply_multi_nt(Plan& p, const void* dens, int nrhs, void* out, cudaStream_t s, bool near, int64_t mask) {
    constexpr int P = PS * PT * PP;
    constexpr int BT = ((P + 31) / 32) * 32;
    constexpr int NRB = 8;  // densities per near-field / leaf block
    const int64_t N = p.N;
    const int D = p.D;
    const double u = p.u;
    Level& LD = p.L[D];
    const float ku = (float)(p.kappa * u);
    const float inv4piu = (float)(1.0 / (4.0 * M_PI * u));
    float2* as = (float2*)p.a_s;
    float2* Is = (float2*)p.I_s;
    const dim3 gN(grid_for(N, kThreads), nrhs);
    const unsigned rb8 = (unsigned)((nrhs + NRB - 1) / NRB);
    {
        TimedScope ts_(TK_PERM, s);
        IFGF_LAUNCH(k_perm_in<float2>, gN, kThreads, 0, s, (const float2*)dens, p.perm, N, as);
    }
    if (near) {
        TimedScope ts_(TK_NEAR, s);
        IFGF_LAUNCH(k_near_f32_multi<NRB>, dim3(grid_for(N, kThreads), rb8), kThreads, 0, s, N, LD.pbox, LD.k, LD.start,
                    LD.nnb, LD.nb, p.off, as, Is, ku, inv4piu, nrhs);
    } else {
        IFGF_CUDA(cudaMemsetAsync(Is, 0, sizeof(float2) * N * nrhs, s));
    }
    if (LD.nc > 0) {
        TimedScope ts_(TK_LEAF, s);
        IFGF_LAUNCH((k_leaf_f32_multi<PS, PT, PP, NRB>), dim3((unsigned)LD.nc, rb8), BT, 0, s, LD.cone_box,
                    LD.cone_gam, LD.g, LD.start, p.off, as, N, (float)(p.kappa * LD.g.h64), 1.0f / LD.g.hg, p.Wf,
                    (float2*)level_coef(p, D, nrhs), p.cstride, nrhs);
    }
    sweep_levels_mma<NT, PS, PT, PP>(p, nrhs, Is, s, mask);
    {
        TimedScope ts_(TK_PERM, s);
        IFGF_LAUNCH(k_perm_out<float2>, gN, kThreads, 0, s, Is, p.perm, N, (float2*)out);
    }
}

template <int PS, int PT, int PP>
void run_apply_multi(Plan& p, const void* dens, int nrhs, void* out, cudaStream_t s, bool near, int64_t mask) {
    if constexpr (PS == 3 && PT == 5 && PP == 5) {
        if (nrhs <= 8)
            run_apply_multi_nt<2, PS, PT, PP>(p, dens, nrhs, out, s, near, mask);
        else if (nrhs <= 16)
            run_apply_multi_nt<4, PS, PT, PP>(p, dens, nrhs, out, s, near, mask);
        else
            run_apply_multi_nt<8, PS, PT, PP>(p, dens, nrhs, out, s, near, mask);
    } else {
        fail(IFGF_ERR_UNSUPPORTED, "tensor-core path built for orders (3,5,5) only");
    }
}

// Propagation of the parent cones [lo, lo + n) of level d-1 (mixed precision, nrhs <= 3 value
// sets): child coefficients cc found through cm (level d), parent coefficients written from cp
// on (parent cone lo at cp); node tables where level d-1 has them.
template <int PS, int PT, int PP>
void launch_prop_f32(Plan& p, int d, int nrhs, int64_t lo, int64_t n, ConeMap cm, const float2* cc, float2* cp,
                     cudaStream_t s) {
    Level& L = p.L[d];
    Level& Lp = p.L[d - 1];
    const int sh = p.D - d;
    const float ku = (float)(p.kappa * p.u);
    if (n <= 0) return;
    if (Lp.n_gam > 0 && PS * PT * PP <= 75 && L.knob_few != 1) {  // tables are built for (3,5,5) only
        TimedScope ts_(TK_PROP, s);
        constexpr int TS = PS * PT * PP <= 75 ? PS : 3, TT = PS * PT * PP <= 75 ? PT : 5,
                      TP = PS * PT * PP <= 75 ? PP : 5;
        const dim3 grid((unsigned)((n + kWarpCones - 1) / kWarpCones), 1);
        if (nrhs == 1)
            IFGF_LAUNCH((k_prop_warp_f32<TS, TT, TP, 1>), grid, 32 * kWarpCones, 0, s, n, Lp.cone_box + lo,
                        Lp.cone_gidx + lo, Lp.k, Lp.cstart, L.k, cm, Lp.tab_t, Lp.tab_r, Lp.tab_k, Lp.tab_list,
                        Lp.tab_perm, Lp.tab_nseg, Lp.tab_seg, cc, cp, p.Wf, p.cstride, nrhs, p.d_status);
        else
            IFGF_LAUNCH((k_prop_warp_f32<TS, TT, TP, 0>), grid, 32 * kWarpCones, 0, s, n, Lp.cone_box + lo,
                        Lp.cone_gidx + lo, Lp.k, Lp.cstart, L.k, cm, Lp.tab_t, Lp.tab_r, Lp.tab_k, Lp.tab_list,
                        Lp.tab_perm, Lp.tab_nseg, Lp.tab_seg, cc, cp, p.Wf, p.cstride, nrhs, p.d_status);
    } else {
        TimedScope ts_(TK_PROP_GEN, s);
        IFGF_LAUNCH((k_prop_f32<PS, PT, PP>), dim3((unsigned)((n + kPropCones - 1) / kPropCones), nrhs), kPropThreads,
                    0, s, n, Lp.cone_box + lo, Lp.cone_gam + lo, Lp.k, Lp.cstart, Lp.g, L.k, cm, L.g, cc, cp, sh, ku,
                    p.Wf, p.cstride, nrhs, p.d_status);
    }
}

// Levels D..3 of the mixed path with few densities: interpolation to the targets of level d
// (Algorithm 8), then propagation into level d-1 (Algorithm 7), from node tables where the
// level has them.
template <int PS, int PT, int PP>
void sweep_levels_f32(Plan& p, int nrhs, float2* Is, cudaStream_t s, int64_t mask) {
    const int D = p.D;
    for (int d = D; d >= 3; --d) {
        TimingLevel tl_(d);
        Level& L = p.L[d];
        if ((mask >> d) & 1) {
            TimedScope ts_(TK_INTERP, s);
            launch_interp_f32<PS, PT, PP>(p, d, nrhs, Is, s);
        }
        if (d == 3) break;
        Level& Lp = p.L[d - 1];
        const float2* cc = (const float2*)level_coef(p, d, nrhs);
        float2* cp = (float2*)level_coef(p, d - 1, nrhs);
        const int64_t cone = (int64_t)nrhs * p.cstride;
        if (Lp.nc > 0)
            for_each_slice(p, d, [&](int64_t lo, int64_t n) {
                launch_prop_f32<PS, PT, PP>(p, d, nrhs, lo, n, L.cmap(p.d_status), cc, cp + lo * cone, s);
            });
    }
}

// The mixed-precision level sweep for nrhs value sets: tensor-core kernels from kMmaMinRhs sets on.
template <int PS, int PT, int PP>
void sweep_levels_mixed(Plan& p, int nrhs, float2* Is, cudaStream_t s, int64_t mask) {
    if constexpr (PS == 3 && PT == 5 && PP == 5) {
        if (nrhs >= kMmaMinRhs) {
            const int blk = p.knob_block > 0 ? p.knob_block : nrhs <= 8 ? 8 : nrhs <= 16 ? 16 : 32;
            if (blk == 8)
                sweep_levels_mma<2, PS, PT, PP>(p, nrhs, Is, s, mask);
            else if (blk == 16)
                sweep_levels_mma<4, PS, PT, PP>(p, nrhs, Is, s, mask);
            else
                sweep_levels_mma<8, PS, PT, PP>(p, nrhs, Is, s, mask);
            return;
        }
    }
    sweep_levels_f32<PS, PT, PP>(p, nrhs, Is, s, mask);
}

// Levels D..3 of the FP64 path: interpolation to the targets of level d (Algorithm 8), then
// propagation into level d-1 (Algorithm 7).
template <int PS, int PT, int PP>
void sweep_levels_f64(Plan& p, int nrhs, double2* Is, cudaStream_t s, int64_t mask) {
    constexpr int BT = ((PS * PT * PP + 31) / 32) * 32;
    const int64_t N = p.N;
    const int D = p.D;
    Level& LD = p.L[D];
    const dim3 gN(grid_for(N, kThreads), nrhs);
    for (int d = D; d >= 3; --d) {
        Level& L = p.L[d];
        const int sh = D - d;
        const double Hd = std::ldexp(p.H1, 1 - d);
        if ((mask >> d) & 1) {
            TimedScope ts_(TK_INTERP, s);
            IFGF_LAUNCH((k_interp_f64<PS, PT, PP>), gN, kThreads, 0, s, N, sh, L.pbox, LD.pbox, LD.k, L.k, L.ncs, L.cs,
                        p.off, p.Xs, L.cmap(p.d_status), L.g, (const double2*)level_coef(p, d, nrhs), p.kappa, p.a[0], p.a[1],
                        p.a[2], Hd, Is, p.cstride, nrhs, p.d_status);
        }
        if (d == 3) break;
        Level& Lp = p.L[d - 1];
        if (Lp.nc > 0) {
            TimedScope ts_(TK_PROP_GEN, s);
            const double2* cc = (const double2*)level_coef(p, d, nrhs);
            double2* cp = (double2*)level_coef(p, d - 1, nrhs);
            const int64_t cone = (int64_t)nrhs * p.cstride;
            for_each_slice(p, d, [&](int64_t lo, int64_t n) {
                IFGF_LAUNCH((k_prop_f64<PS, PT, PP>), dim3((unsigned)n, nrhs), BT, 0, s, Lp.cone_box + lo,
                            Lp.cone_gam + lo, Lp.k, Lp.cstart, Lp.g, L.k, L.cmap(p.d_status), L.g, cc, cp + lo * cone, sh,
                            p.kappa, p.a[0], p.a[1], p.a[2], Hd, p.Wd, p.cstride, nrhs, p.d_status);
            });
        }
    }
}

template <int PS, int PT, int PP>
void run_apply(Plan& p, const void* dens, int nrhs, void* out, cudaStream_t s, bool near, int64_t mask) {
    constexpr int P = PS * PT * PP;
    constexpr int BT = ((P + 31) / 32) * 32;
    const int64_t N = p.N;
    const int D = p.D;
    const dim3 gN(grid_for(N, kThreads), nrhs);
    const bool mixed = p.precision == IFGF_PREC_MIXED;
    const double u = p.u;
    const double HD = std::ldexp(p.H1, 1 - D);
    Level& LD = p.L[D];
    if (mixed && nrhs >= kMmaMinRhs && PS == 3 && PT == 5 && PP == 5) {
        run_apply_multi<PS, PT, PP>(p, dens, nrhs, out, s, near, mask);
    } else if (mixed) {
        const float ku = (float)(p.kappa * u);
        const float inv4piu = (float)(1.0 / (4.0 * M_PI * u));
        float2* as = (float2*)p.a_s;
        float2* Is = (float2*)p.I_s;
        {
            TimedScope ts_(TK_PERM, s);
            IFGF_LAUNCH(k_perm_in<float2>, gN, kThreads, 0, s, (const float2*)dens, p.perm, N, as);
        }
        if (near)
            {
                TimedScope ts_(TK_NEAR, s);
                IFGF_LAUNCH(k_near_tile_f32, dim3((unsigned)LD.n, nrhs), kNearThreads, 0, s, LD.k, LD.start, LD.nnb,
                            LD.nb, p.off, as, Is, N, ku, inv4piu, 0);
            }
        else
            IFGF_CUDA(cudaMemsetAsync(Is, 0, sizeof(float2) * N * nrhs, s));
        const float kh = (float)(p.kappa * LD.g.h64);
        if (LD.nc > 0)
            {
                TimedScope ts_(TK_LEAF, s);
                IFGF_LAUNCH((k_leaf_box_f32<PS, PT, PP>), dim3((unsigned)LD.n, nrhs), kLeafThreads, 0, s, LD.bcs,
                            LD.cone_gam, LD.g, LD.start, p.off, as, N, kh, 1.0f / LD.g.hg, p.Wf,
                            (float2*)level_coef(p, D, nrhs), p.cstride, nrhs, 0, 0, (int)LD.nc);
            }
        sweep_levels_f32<PS, PT, PP>(p, nrhs, Is, s, mask);
        {
            TimedScope ts_(TK_PERM, s);
            IFGF_LAUNCH(k_perm_out<float2>, gN, kThreads, 0, s, Is, p.perm, N, (float2*)out);
        }
    } else {
        double2* as = (double2*)p.a_s;
        double2* Is = (double2*)p.I_s;
        {
            TimedScope ts_(TK_PERM, s);
            IFGF_LAUNCH(k_perm_in<double2>, gN, kThreads, 0, s, (const double2*)dens, p.perm, N, as);
        }
        if (near)
            {
                TimedScope ts_(TK_NEAR, s);
                IFGF_LAUNCH(k_near_f64, gN, kThreads, 0, s, N, LD.pbox, LD.start, LD.nnb, LD.nb, p.Xs, as, Is, p.kappa);
            }
        else
            IFGF_CUDA(cudaMemsetAsync(Is, 0, sizeof(double2) * N * nrhs, s));
        if (LD.nc > 0)
            {
                TimedScope ts_(TK_LEAF, s);
                IFGF_LAUNCH((k_leaf_f64<PS, PT, PP>), dim3((unsigned)LD.nc, nrhs), BT, 0, s, LD.cone_box, LD.cone_gam,
                            LD.g, LD.start, LD.k, p.Xs, as, N, p.kappa, p.a[0], p.a[1], p.a[2], HD, p.Wd,
                            (double2*)level_coef(p, D, nrhs), p.cstride, nrhs);
            }
        sweep_levels_f64<PS, PT, PP>(p, nrhs, Is, s, mask);
        {
            TimedScope ts_(TK_PERM, s);
            IFGF_LAUNCH(k_perm_out<double2>, gN, kThreads, 0, s, Is, p.perm, N, (double2*)out);
        }
    }
}

// Apply of S = c (alpha I/r + r r^T/r^3) to nf force fields ([nf][3][N] float, caller's order)
// into velocities (displacements) of the same layout: near field and leaf level of this kernel,
// then the kappa = 0 level sweep on the ceil(3 nf / 2) complex slots.
template <int PS, int PT, int PP>
void run_apply_stokes_f64(Plan& p, const double* forces, int nf, double* vel, const TensorKernel& tk, cudaStream_t s,
                          bool near, int64_t mask) {
    constexpr int BT = ((PS * PT * PP + 31) / 32) * 32;
    const int64_t N = p.N;
    const int D = p.D;
    Level& LD = p.L[D];
    const int nreal = 3 * nf, slots = (nreal + 1) / 2, pairs = nf / 2;
    double* fs = (double*)p.a_s;
    double2* Is = (double2*)p.I_s;
    const double c = tk.c, alpha = tk.alpha;
    const dim3 gR(grid_for(N, kThreads), nreal);
    {
        TimedScope ts_(TK_PERM, s);
        IFGF_LAUNCH(k_perm_in<double>, gR, kThreads, 0, s, forces, p.perm, N, fs);
    }
    if (near) {
        TimedScope ts_(TK_NEAR, s);
        const unsigned gx = grid_for(N, kThreads);
        if (pairs > 0)
            IFGF_LAUNCH(k_near_stokes_f64<2>, dim3(gx, pairs), kThreads, 0, s, N, LD.pbox, LD.start, LD.nnb, LD.nb,
                        p.Xs, fs, Is, alpha, c, 0);
        if (nf & 1)
            IFGF_LAUNCH(k_near_stokes_f64<1>, dim3(gx, 1), kThreads, 0, s, N, LD.pbox, LD.start, LD.nnb, LD.nb, p.Xs,
                        fs, Is, alpha, c, nf - 1);
    } else {
        IFGF_CUDA(cudaMemsetAsync(Is, 0, sizeof(double2) * N * slots, s));
    }
    if (LD.nc > 0) {
        TimedScope ts_(TK_LEAF, s);
        double2* cD = (double2*)level_coef(p, D, slots);
        const double HD = std::ldexp(p.H1, 1 - D);
        if (pairs > 0)
            IFGF_LAUNCH((k_leaf_stokes_f64<PS, PT, PP, 2>), dim3((unsigned)LD.nc, pairs), BT, 0, s, LD.cone_box,
                        LD.cone_gam, LD.g, LD.start, LD.k, p.Xs, fs, N, p.a[0], p.a[1], p.a[2], HD, p.Wd, cD,
                        p.cstride, slots, alpha, c, 0);
        if (nf & 1)
            IFGF_LAUNCH((k_leaf_stokes_f64<PS, PT, PP, 1>), dim3((unsigned)LD.nc, 1), BT, 0, s, LD.cone_box,
                        LD.cone_gam, LD.g, LD.start, LD.k, p.Xs, fs, N, p.a[0], p.a[1], p.a[2], HD, p.Wd, cD,
                        p.cstride, slots, alpha, c, nf - 1);
    }
    sweep_levels_f64<PS, PT, PP>(p, slots, Is, s, mask);
    {
        TimedScope ts_(TK_PERM, s);
        IFGF_LAUNCH(k_perm_out_stokes_f64, gR, kThreads, 0, s, Is, p.perm, N, vel);
    }
}

template <int PS, int PT, int PP>
void run_apply_stokes(Plan& p, const float* forces, int nf, float* vel, const TensorKernel& tk, cudaStream_t s,
                      bool near, int64_t mask) {
    const int64_t N = p.N;
    const int D = p.D;
    Level& LD = p.L[D];
    const int nreal = 3 * nf, slots = (nreal + 1) / 2, pairs = nf / 2;
    float* fs = (float*)p.a_s;
    float2* Is = (float2*)p.I_s;
    const float alpha = (float)tk.alpha, beta = (float)(1.0 / tk.alpha);
    const float cu = (float)(tk.c / p.u), fscale = (float)(4.0 * M_PI * tk.c);
    const dim3 gR(grid_for(N, kThreads), nreal);
    {
        TimedScope ts_(TK_PERM, s);
        IFGF_LAUNCH(k_perm_in<float>, gR, kThreads, 0, s, forces, p.perm, N, fs);
    }
    if (near) {
        TimedScope ts_(TK_NEAR, s);
        if (pairs > 0)
            IFGF_LAUNCH(k_near_stokes_f32<2>, dim3((unsigned)LD.n, pairs), kNearThreads, 0, s, LD.k, LD.start, LD.nnb,
                        LD.nb, p.off, fs, Is, N, alpha, beta, cu, 0);
        if (nf & 1)
            IFGF_LAUNCH(k_near_stokes_f32<1>, dim3((unsigned)LD.n, 1), kNearThreads, 0, s, LD.k, LD.start, LD.nnb,
                        LD.nb, p.off, fs, Is, N, alpha, beta, cu, nf - 1);
    } else {
        IFGF_CUDA(cudaMemsetAsync(Is, 0, sizeof(float2) * N * slots, s));
    }
    if (LD.nc > 0) {
        TimedScope ts_(TK_LEAF, s);
        float2* cD = (float2*)level_coef(p, D, slots);
        const float hinv = 1.0f / LD.g.hg;
        if (pairs > 0)
            IFGF_LAUNCH((k_leaf_stokes_f32<PS, PT, PP, 2>), dim3((unsigned)LD.n, pairs), kLeafThreads, 0, s, LD.bcs,
                        LD.cone_gam, LD.g, LD.start, p.off, fs, N, hinv, p.Wf, cD, p.cstride, slots, alpha, beta,
                        fscale, 0);
        if (nf & 1)
            IFGF_LAUNCH((k_leaf_stokes_f32<PS, PT, PP, 1>), dim3((unsigned)LD.n, 1), kLeafThreads, 0, s, LD.bcs,
                        LD.cone_gam, LD.g, LD.start, p.off, fs, N, hinv, p.Wf, cD, p.cstride, slots, alpha, beta,
                        fscale, nf - 1);
    }
    sweep_levels_mixed<PS, PT, PP>(p, slots, Is, s, mask);
    {
        TimedScope ts_(TK_PERM, s);
        IFGF_LAUNCH(k_perm_out_stokes, gR, kThreads, 0, s, Is, p.perm, N, vel);
    }
}

}  // namespace

// ---- steps of one rank of a distributed apply (Sec. 3.2), mixed precision, nrhs <= 3 ------------
namespace {
template <int PS, int PT, int PP>
void shard_near_leaf_t(Plan& p, const float2* as, int nrhs, float2* Is, int64_t b0, int64_t b1, int64_t lb0,
                       int64_t lb1, int64_t c_lo, int64_t c_hi, float2* coefD, cudaStream_t s) {
    const int64_t N = p.N;
    Level& LD = p.L[p.D];
    const float ku = (float)(p.kappa * p.u);
    const float inv4piu = (float)(1.0 / (4.0 * M_PI * p.u));
    if (b1 > b0) {
        TimedScope ts_(TK_NEAR, s);
        IFGF_LAUNCH(k_near_tile_f32, dim3((unsigned)(b1 - b0), nrhs), kNearThreads, 0, s, LD.k, LD.start, LD.nnb, LD.nb,
                    p.off, as, Is, N, ku, inv4piu, (int)b0);
    }
    if (c_hi > c_lo) {
        TimedScope ts_(TK_LEAF, s);
        IFGF_LAUNCH((k_leaf_box_f32<PS, PT, PP>), dim3((unsigned)(lb1 - lb0), nrhs), kLeafThreads, 0, s, LD.bcs,
                    LD.cone_gam, LD.g, LD.start, p.off, as, N, (float)(p.kappa * LD.g.h64), 1.0f / LD.g.hg, p.Wf, coefD,
                    p.cstride, nrhs, (int)lb0, (int)c_lo, (int)c_hi);
    }
}
}  // namespace

void shard_near_leaf(Plan& p, const float2* as, int nrhs, float2* Is, int64_t b0, int64_t b1, int64_t lb0, int64_t lb1,
                     int64_t c_lo, int64_t c_hi, float2* coefD, cudaStream_t s) {
    if (p.Ps == 3 && p.Pt == 5 && p.Pp == 5)
        shard_near_leaf_t<3, 5, 5>(p, as, nrhs, Is, b0, b1, lb0, lb1, c_lo, c_hi, coefD, s);
    else
        shard_near_leaf_t<5, 7, 7>(p, as, nrhs, Is, b0, b1, lb0, lb1, c_lo, c_hi, coefD, s);
}

void shard_interp(Plan& p, int d, int nrhs, float2* Is, const ConeMap& cm, const float2* coef, int64_t i0, int64_t i1,
                  cudaStream_t s) {
    TimedScope ts_(TK_INTERP, s);
    if (p.Ps == 3 && p.Pt == 5 && p.Pp == 5)
        launch_interp_f32<3, 5, 5>(p, d, nrhs, Is, s, cm, coef, i0, i1);
    else
        launch_interp_f32<5, 7, 7>(p, d, nrhs, Is, s, cm, coef, i0, i1);
}

void shard_prop(Plan& p, int d, int nrhs, int64_t lo, int64_t hi, const ConeMap& cm, const float2* cc, float2* cp,
                cudaStream_t s) {
    if (p.Ps == 3 && p.Pt == 5 && p.Pp == 5)
        launch_prop_f32<3, 5, 5>(p, d, nrhs, lo, hi - lo, cm, cc, cp, s);
    else
        launch_prop_f32<5, 7, 7>(p, d, nrhs, lo, hi - lo, cm, cc, cp, s);
}

void permute_points(Plan& p, const void* in, int nrhs, void* out, bool to_sorted, cudaStream_t s) {
    const dim3 gN(grid_for(p.N, kThreads), nrhs);
    TimedScope ts_(TK_PERM, s);
    if (p.precision == IFGF_PREC_MIXED) {
        if (to_sorted)
            IFGF_LAUNCH(k_perm_in<float2>, gN, kThreads, 0, s, (const float2*)in, p.perm, p.N, (float2*)out);
        else
            IFGF_LAUNCH(k_perm_out<float2>, gN, kThreads, 0, s, (const float2*)in, p.perm, p.N, (float2*)out);
    } else {
        if (to_sorted)
            IFGF_LAUNCH(k_perm_in<double2>, gN, kThreads, 0, s, (const double2*)in, p.perm, p.N, (double2*)out);
        else
            IFGF_LAUNCH(k_perm_out<double2>, gN, kThreads, 0, s, (const double2*)in, p.perm, p.N, (double2*)out);
    }
}

void apply_plan(Plan& p, const void* dens, int nrhs, void* out, cudaStream_t s, bool near, int64_t mask) {
    // densities in blocks of at most rhs_block, one level sweep per block
    const size_t csz = p.precision == IFGF_PREC_MIXED ? sizeof(float2) : sizeof(double2);
    for (int r0 = 0; r0 < nrhs; r0 += p.rhs_block) {
        const int nb = std::min(p.rhs_block, nrhs - r0);
        const void* d = static_cast<const char*>(dens) + (size_t)r0 * p.N * csz;
        void* o = static_cast<char*>(out) + (size_t)r0 * p.N * csz;
        if (p.Ps == 3 && p.Pt == 5 && p.Pp == 5)
            run_apply<3, 5, 5>(p, d, nb, o, s, near, mask);
        else if (p.Ps == 5 && p.Pt == 7 && p.Pp == 7)
            run_apply<5, 7, 7>(p, d, nb, o, s, near, mask);
        else
            fail(IFGF_ERR_UNSUPPORTED, "interpolation orders not built");
    }
}

void apply_plan_stokes(Plan& p, const void* forces, int nf, void* vel, const TensorKernel& tk, cudaStream_t s,
                       bool near, int64_t mask) {
    // force fields in blocks whose ceil(3 nfb / 2) slots fit the arena's rhs_block value sets;
    // an even block size keeps every block but the last free of a half-empty slot
    int nfb = std::min(2 * p.rhs_block / 3, 21844);  // 3 nfb real sets fit a grid's y extent
    if (nfb >= 2) nfb &= ~1;
    if (nfb < 1) fail(IFGF_ERR_UNSUPPORTED, "the coefficient arena holds fewer than two value sets");
    const bool mixed = p.precision == IFGF_PREC_MIXED;
    const size_t rsz = mixed ? sizeof(float) : sizeof(double);
    for (int f0 = 0; f0 < nf; f0 += nfb) {
        const int nb = std::min(nfb, nf - f0);
        const void* f = static_cast<const char*>(forces) + (size_t)3 * f0 * p.N * rsz;
        void* u = static_cast<char*>(vel) + (size_t)3 * f0 * p.N * rsz;
        const bool o355 = p.Ps == 3 && p.Pt == 5 && p.Pp == 5, o577 = p.Ps == 5 && p.Pt == 7 && p.Pp == 7;
        if (!o355 && !o577) fail(IFGF_ERR_UNSUPPORTED, "interpolation orders not built");
        if (mixed && o355)
            run_apply_stokes<3, 5, 5>(p, (const float*)f, nb, (float*)u, tk, s, near, mask);
        else if (mixed)
            run_apply_stokes<5, 7, 7>(p, (const float*)f, nb, (float*)u, tk, s, near, mask);
        else if (o355)
            run_apply_stokes_f64<3, 5, 5>(p, (const double*)f, nb, (double*)u, tk, s, near, mask);
        else
            run_apply_stokes_f64<5, 7, 7>(p, (const double*)f, nb, (double*)u, tk, s, near, mask);
    }
}

}  // namespace ifgf
