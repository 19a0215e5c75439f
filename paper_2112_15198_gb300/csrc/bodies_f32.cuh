// Device bodies of the mixed-precision apply kernels for one density set (or a few): the level-D
// neighbour sums, LevelDEvaluations, both propagation kernels and the interpolation to a target.
// The kernels of apply.cu launch them one work unit per block (or warp, or thread); the batched
// apply runs the same bodies over work queues of many plans, so both compute identical values.
#pragma once
#include <type_traits>

#include "ifgf_internal.cuh"

namespace ifgf {

// ---- near field --------------------------------------------------------------------------
// I(x_l) = sum over the points x_m of the 27 neighbour leaves of leaf(x_l), m != l, of a_m G.

// Near field with one block per leaf box (the paper's LevelDSingularInteractions): the sources of
// the box's neighbourhood are staged in shared memory in tiles of kNearTile (coalesced 128-bit
// offset and 64-bit density loads), each shifted once to the target box's frame. With m targets
// in the box, S = 2^k <= min(32, kNearThreads / m) threads share a target and take every S-th
// source of a tile; their partial sums are combined by warp shuffles in a fixed order.
constexpr int kNearThreads = 128;
constexpr int kNearTile = 128;
__device__ __forceinline__ void near_box_f32(const int4* __restrict__ kD, const int32_t* __restrict__ startD, const int32_t* __restrict__ nnb,
                const int32_t* __restrict__ nb, const float4* __restrict__ off, const float2* __restrict__ as,
                float2* __restrict__ Is, int64_t N, float ku, float inv4piu, int l, int64_t r) {
    __shared__ float4 s_p[kNearTile];  // source position in the target box's grid frame; w = source index
    __shared__ float2 s_a[kNearTile];
    const int tid = threadIdx.x;
    const int t0 = startD[l], m = startD[l + 1] - t0;
    const int4 kl = kD[l];
    const float2* ar = as + r * N;
    int S = 1;
    while (S < 32 && 2 * S * m <= kNearThreads) S *= 2;
    const int per_pass = kNearThreads / S;  // targets per pass
    const int cnt = nnb[l];
    for (int base = 0; base < m; base += per_pass) {
        const int tl = base + tid / S, part = tid % S;
        const bool active = tl < m;
        const int i = t0 + (active ? tl : 0);
        const float4 oi = off[i];
        float2 acc = make_float2(0.f, 0.f);
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
                    const float4 oj = __ldg(&off[tb + tid]);
                    s_p[tid] = make_float4(oj.x - sx, oj.y - sy, oj.z - sz, __int_as_float(tb + tid));
                    s_a[tid] = __ldg(&ar[tb + tid]);
                }
                __syncthreads();
                if (active) {
                    for (int k = part; k < nt; k += S) {
                        const float4 pj = s_p[k];
                        if (__float_as_int(pj.w) == i) continue;
                        const float vx = oi.x - pj.x, vy = oi.y - pj.y, vz = oi.z - pj.z;
                        const float r2 = fmaf(vx, vx, fmaf(vy, vy, vz * vz));
                        const float rinv = rsqrtf(r2);
                        const float2 e = cis_f32(ku * (r2 * rinv));
                        const float w = inv4piu * rinv;
                        const float2 aj = s_a[k];
                        const float2 g = make_float2(e.x * w, e.y * w);
                        acc = __ffma2_rn(make_float2(aj.x, aj.x), g, acc);
                        acc = __ffma2_rn(make_float2(-aj.y, aj.y), make_float2(g.y, g.x), acc);
                    }
                }
            }
        }
        for (int o = S / 2; o >= 1; o >>= 1) {  // the S partial sums of a target, fixed order
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        if (active && part == 0) Is[r * N + i] = acc;
    }
}

// LevelDEvaluations with one block per leaf box: the box's sources (offset from the centre in
// units of h, |u|^2 and the density) are staged in shared memory once and swept by every
// (cone, node) of the box, up to 32 cones at a time (8 for larger orders). For the node x = x_k + (h/s) y (|y| = 1)
// and the source x' = x_k + h u, |x - x'|^2 / r^2 = q = 1 + s (s |u|^2 - 2 y.u), so
//     g_k(x, x') = q^(-1/2) exp(i kappa h (s |u|^2 - 2 y.u) / (1 + q^(1/2))),
// free of cancellation; then the coefficient transform of each cone by one warp.
constexpr int kLeafThreads = 256;
constexpr int kLeafSrc = 256;    // sources staged per pass
constexpr int kLeafCones = 32;   // cones of the box per pass
template <int PS, int PT, int PP>
__device__ __forceinline__ void leaf_box_f32(const int32_t* __restrict__ bcs, const int32_t* __restrict__ cone_gam, LevelGrid g,
               const int32_t* __restrict__ startD, const float4* __restrict__ off, const float2* __restrict__ as,
               int64_t N, float kh, float hinv, const float* __restrict__ W, float2* __restrict__ coef, int cstride,
               int nrhs, int b, int r, int c_lo, int c_hi) {
    constexpr int P = PS * PT * PP;
    constexpr int NW = kLeafThreads / 32;
    constexpr int NCP = P <= 75 ? kLeafCones : 8;  // cones per pass (shared memory below 48 KB)
    __shared__ float4 s_u[kLeafSrc];   // (u, |u|^2)
    __shared__ float2 s_a[kLeafSrc];
    __shared__ float2 f[NCP][P];
    __shared__ float2 tmp[NW][P];
    // leaf box b, value set r; only the cones [c_lo, c_hi) are evaluated, cone c is written at
    // block c - c_lo of coef
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int c0 = max(bcs[b], c_lo), c1 = min(bcs[b + 1], c_hi);
    if (c0 == c1) return;
    const int j0 = startD[b], j1 = startD[b + 1];
    const float2* ar = as + (int64_t)r * N;
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
                const float4 o = __ldg(&off[t0 + tid]);
                const float ux = o.x * hinv, uy = o.y * hinv, uz = o.z * hinv;
                s_u[tid] = make_float4(ux, uy, uz, fmaf(ux, ux, fmaf(uy, uy, uz * uz)));
                s_a[tid] = __ldg(&ar[t0 + tid]);
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
                float2 acc = t0 == j0 ? make_float2(0.f, 0.f) : f[cl][n];
#pragma unroll 4
                for (int j = 0; j < nt; ++j) {
                    const float4 u = s_u[j];
                    const float yu = fmaf(yx, u.x, fmaf(yy, u.y, yz * u.z));
                    const float num = fmaf(sn, u.w, -2.f * yu);
                    const float q = fmaf(sn, num, 1.f);
                    const float rq = rsqrtf(q);
                    const float2 e = cis_f32(kh * __fdividef(num, fmaf(q, rq, 1.f)));
                    const float2 gk = make_float2(e.x * rq, e.y * rq);
                    const float2 aj = s_a[j];
                    acc = __ffma2_rn(make_float2(aj.x, aj.x), gk, acc);
                    acc = __ffma2_rn(make_float2(-aj.y, aj.y), make_float2(gk.y, gk.x), acc);
                }
                f[cl][n] = acc;
            }
        }
        __syncthreads();
        for (int cl = warp; cl < ncc; cl += NW) {  // coefficient transform, one warp per cone
            float2* fv = f[cl];
            float2* tv = tmp[warp];
            for (int n = lane; n < P; n += 32) {
                const int qc = n % PP, qb = (n / PP) % PT, qa = n / (PP * PT);
                float2 a = make_float2(0.f, 0.f);
#pragma unroll
                for (int k = 0; k < PP; ++k) {
                    const float w = Wp[qc * PP + k];
                    const float2 v = fv[(qa * PT + qb) * PP + k];
                    a.x = fmaf(w, v.x, a.x);
                    a.y = fmaf(w, v.y, a.y);
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
                    const float2 v = tv[(qa * PT + k) * PP + qc];
                    a.x = fmaf(w, v.x, a.x);
                    a.y = fmaf(w, v.y, a.y);
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
                    const float2 v = fv[(k * PT + qb) * PP + qc];
                    a.x = fmaf(w, v.x, a.x);
                    a.y = fmaf(w, v.y, a.y);
                }
                coef[((int64_t)(cc + cl - c_lo) * nrhs + r) * cstride + n] = a;
            }
            __syncwarp();
        }
    }
}

// One block per relevant parent cone (j, gamma) at level d-1, one thread per node x:
//   F_j(x) = sum over relevant children B_k of B_j of I_P C_{k;alpha}(x) G(x,x_k)/G(x,x_j),
//   G(x,x_k)/G(x,x_j) = (r_j/r_k) exp(i kappa (r_k - r_j)),  r_k - r_j = (|o|^2 - 2 q.o)/(r_k + r_j),
// q the node offset from x_j and o the child-centre offset; then the parent interpolant.
// Block work layout: kPropCones consecutive parent cones; the (cone, child, node) evaluations
// of the block are flattened over its threads (no idle lanes beyond the last round); node
// offsets are staged in shared memory; values are summed over children in child order, then
// the parent interpolants are generated.
constexpr int kPropCones = 2;
constexpr int kPropThreads = 128;

template <int P>
struct PropSmem {
    float2 vals[kPropCones][8][P];
    float4 qn[kPropCones][P];
    float2 f[kPropCones][P], tmp[kPropCones][P];
    int off[kPropCones + 1], kb0[kPropCones], jb[kPropCones];
};

// Parent cones [pc0, pc0 + kPropCones) of value set r, kPropThreads threads.  kCoh: the child
// coefficients were written by other blocks of the same launch (no read-only-path loads).
template <int PS, int PT, int PP, bool kCoh>
__device__ __forceinline__ void prop_cones_f32(PropSmem<PS * PT * PP>& sm, int64_t ncp, const int32_t* __restrict__ pcone_box, const int32_t* __restrict__ pcone_gam,
           const int4* __restrict__ kp, const int32_t* __restrict__ pcstart, LevelGrid gp,
           const int4* __restrict__ kd, ConeMap cm, LevelGrid g,
           const float2* __restrict__ cchild, float2* __restrict__ cparent, int sh, float ku,
           const float* __restrict__ W, int cstride, int nrhs, int* __restrict__ status, int64_t pc0, int r) {
    constexpr int P = PS * PT * PP;
    constexpr int NC = kPropCones;
    const int tid = threadIdx.x;
    if (tid == 0) {
        int acc = 0;
        for (int c = 0; c < NC; ++c) {
            sm.off[c] = acc;
            const int64_t pc = pc0 + c;
            if (pc < ncp) {
                const int jb = pcone_box[pc];
                sm.jb[c] = jb;
                sm.kb0[c] = pcstart[jb];
                acc += (pcstart[jb + 1] - pcstart[jb]) * P;
            } else {
                sm.jb[c] = -1;
                sm.kb0[c] = 0;
            }
        }
        sm.off[NC] = acc;
    }
    // node offsets from the parent centre (grid units, the plan's exact products) and |q|
    for (int x = tid; x < NC * P; x += kPropThreads) {
        const int c = x / P, n = x - (x / P) * P;
        const int64_t pc = pc0 + c;
        if (pc < ncp) {
            const int gam = pcone_gam[pc];
            const int ip = gam % gp.np, it = (gam / gp.np) % gp.nt, is = gam / (gp.np * gp.nt);
            const int qc = n % PP, qb = (n / PP) % PT, qa = n / (PP * PT);
            const float rho = gp.rho[is * PS + qa];
            const float st = gp.stn[it * PT + qb], ct = gp.ctn[it * PT + qb];
            const float cp = gp.cpn[ip * PP + qc], sp = gp.spn[ip * PP + qc];
            const float qx = __fmul_rn(rho, __fmul_rn(st, cp)), qy = __fmul_rn(rho, __fmul_rn(st, sp));
            const float qz = __fmul_rn(rho, ct);
            sm.qn[c][n] = make_float4(qx, qy, qz, sqrtf(fmaf(qx, qx, fmaf(qy, qy, qz * qz))));
        }
    }
    __syncthreads();
    const float oo = 3.0f * (float)(1 << sh) * (float)(1 << sh);
    const int total = sm.off[NC];
    for (int item = tid; item < total; item += kPropThreads) {
        int c = 0;
#pragma unroll
        for (int k = 1; k < NC; ++k) c += item >= sm.off[k];
        const int rem = item - sm.off[c];
        const int ch = rem / P, n = rem - ch * P;
        const int kb = sm.kb0[c] + ch;
        const int4 kj = kp[sm.jb[c]];
        const int4 kk = kd[kb];
        const float4 q = sm.qn[c][n];
        const float ox = (float)((2 * (kk.x - 2 * kj.x) - 1) << sh);
        const float oy = (float)((2 * (kk.y - 2 * kj.y) - 1) << sh);
        const float oz = (float)((2 * (kk.z - 2 * kj.z) - 1) << sh);
        const ConeLocal cl = locate_f32(g, __fsub_rn(q.x, ox), __fsub_rn(q.y, oy), __fsub_rn(q.z, oz));
        const int s = cm.find(kb, cl.gamma(g));
        float2 t = make_float2(0.f, 0.f);
        if (s < 0) {
            set_status(status, IFGF_ERR_INTERNAL);
        } else {
            const float2 F = interp_f32<PS, PT, PP, kCoh>(cchild + ((int64_t)s * nrhs + r) * cstride, cl.ts, cl.tt, cl.tp);
            // G(x,x_k)/G(x,x_j) = (r_j/r_k) exp(i kappa (r_k - r_j)), r_k - r_j = (|o|^2 - 2 q.o)/(r_k + r_j)
            const float qo = fmaf(q.x, ox, fmaf(q.y, oy, q.z * oz));
            const float dr = __fdividef(fmaf(-2.f, qo, oo), cl.r + q.w);
            const float2 e = cis_f32(ku * dr);
            const float w = __fdividef(q.w, cl.r);
            t = cmul(F, make_float2(e.x * w, e.y * w));
        }
        sm.vals[c][ch][n] = t;
    }
    __syncthreads();
    // sum over children in child order, then the Chebyshev coefficients (phi, theta, s passes)
    const float* Ws = W;
    const float* Wt = W + PS * PS;
    const float* Wp = Wt + PT * PT;
    for (int x = tid; x < NC * P; x += kPropThreads) {
        const int c = x / P, n = x - (x / P) * P;
        const int nch = (sm.off[c + 1] - sm.off[c]) / P;
        float2 a = make_float2(0.f, 0.f);
        for (int ch = 0; ch < nch; ++ch) {
            a.x += sm.vals[c][ch][n].x;
            a.y += sm.vals[c][ch][n].y;
        }
        sm.f[c][n] = a;
    }
    __syncthreads();
    for (int x = tid; x < NC * P; x += kPropThreads) {
        const int c = x / P, n = x - (x / P) * P;
        const int qc = n % PP, qb = (n / PP) % PT, qa = n / (PP * PT);
        float2 acc = make_float2(0.f, 0.f);
        const float2* row = &sm.f[c][(qa * PT + qb) * PP];
#pragma unroll
        for (int k = 0; k < PP; ++k) {
            const float w = Wp[qc * PP + k];
            acc.x = fmaf(w, row[k].x, acc.x);
            acc.y = fmaf(w, row[k].y, acc.y);
        }
        sm.tmp[c][n] = acc;
    }
    __syncthreads();
    for (int x = tid; x < NC * P; x += kPropThreads) {
        const int c = x / P, n = x - (x / P) * P;
        const int qc = n % PP, qb = (n / PP) % PT, qa = n / (PP * PT);
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < PT; ++j) {
            const float w = Wt[qb * PT + j];
            const float2 v = sm.tmp[c][(qa * PT + j) * PP + qc];
            acc.x = fmaf(w, v.x, acc.x);
            acc.y = fmaf(w, v.y, acc.y);
        }
        sm.f[c][n] = acc;
    }
    __syncthreads();
    for (int x = tid; x < NC * P; x += kPropThreads) {
        const int c = x / P, n = x - (x / P) * P;
        const int64_t pc = pc0 + c;
        if (pc >= ncp) continue;
        const int qc = n % PP, qb = (n / PP) % PT, qa = n / (PP * PT);
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < PS; ++i) {
            const float w = Ws[qa * PS + i];
            const float2 v = sm.f[c][(i * PT + qb) * PP + qc];
            acc.x = fmaf(w, v.x, acc.x);
            acc.y = fmaf(w, v.y, acc.y);
        }
        cparent[(pc * nrhs + r) * cstride + n] = acc;
    }
}

// Propagation from the node tables of the parent level (orders (3,5,5), mixed precision): the
// geometry of every (cone index, child octant, node) was computed once at plan time, so an
// evaluation is a table read, the child cone's slot, the interpolant contraction and the complex
// ratio. One warp per parent cone, no block-wide barrier: the warp resolves its children's rows
// and child-cone slots, stages the child cones' coefficient blocks in shared memory with
// coalesced asynchronous copies, evaluates half-segments (up to 4 nodes of one child cone per
// lane, sharing each coefficient row), sums the children in order and forms the coefficients,
// synchronising only itself.
constexpr int kWarpCones = 2;  // warps (parent cones) per block
constexpr int kWarpStage = 8; // child-cone coefficient blocks staged in shared memory per warp
constexpr int kStage4 = 39;    // float4 per staged block (38 used at P = 75; odd, so lanes reading different
                               // blocks at one offset hit different banks)
// NSETS = 1: one value set (grid row y = 0); NSETS = 0: all nrhs sets in turn, sharing the rows,
// list entries and child-cone slots resolved once per warp.
template <int P>
struct WarpSmem {
    float2 vals[8][P];
    float4 cbuf[kWarpStage * kStage4];
    int slot[8][kSlotCache];  // global slot, -1 missing, -2 - j staged as block j
    int row[8], goff[9], koff[9];
    int dsl[kWarpStage];      // global slot of every staged block
};

// Parent cone pc, one warp (lane = lane index).  The warp's shared memory is wp (a WarpSmem of a
// persistent kernel), or, with WS = void, per-warp arrays of the block declared here for blocks of
// kWarpCones warps (the form whose register allocation the standalone kernel keeps).  kCoh: the
// child coefficients were written by other blocks of the same launch (no read-only-path loads).
template <int PS, int PT, int PP, int NSETS, bool kCoh, class WS>
__device__ __forceinline__ void prop_cone_warp_f32(WS* wp, int64_t ncp, const int32_t* __restrict__ pcone_box, const int32_t* __restrict__ cone_gidx,
                const int4* __restrict__ kp, const int32_t* __restrict__ pcstart, const int4* __restrict__ kd,
                ConeMap cm, const float4* __restrict__ tab_t, const float2* __restrict__ tab_r,
                const int32_t* __restrict__ tab_k, const int32_t* __restrict__ tab_list,
                const int16_t* __restrict__ tab_perm, const int32_t* __restrict__ tab_nseg,
                const int32_t* __restrict__ tab_seg, const float2* __restrict__ cchild, float2* __restrict__ cparent,
                const float* __restrict__ W, int cstride, int nrhs, int* __restrict__ status, int64_t pc, int lane) {
    constexpr int P = PS * PT * PP;
    constexpr int R = kSegLen / 2;  // a thread evaluates half a segment
    if (pc >= ncp) return;  // the whole warp leaves; nothing below synchronises the block
    float2 (*vals)[P];
    int (*s_slot)[kSlotCache];
    int *s_row, *s_goff, *s_koff, *s_dsl;
    float4* cbuf;
    if constexpr (std::is_same<WS, void>::value) {
        __shared__ float2 s_vals_w[kWarpCones][8][P];
        __shared__ float4 s_cbuf_w[kWarpCones][kWarpStage * kStage4];
        __shared__ int s_slot_w[kWarpCones][8][kSlotCache];  // global slot, -1 missing, -2 - j staged as block j
        __shared__ int s_row_w[kWarpCones][8], s_goff_w[kWarpCones][9], s_koff_w[kWarpCones][9];
        __shared__ int s_dsl_w[kWarpCones][kWarpStage];  // global slot of every staged block
        const int warp = threadIdx.x >> 5;
        vals = s_vals_w[warp];
        s_slot = s_slot_w[warp];
        s_row = s_row_w[warp];
        s_goff = s_goff_w[warp];
        s_koff = s_koff_w[warp];
        s_dsl = s_dsl_w[warp];
        cbuf = s_cbuf_w[warp];
    } else {
        vals = wp->vals;
        s_slot = wp->slot;
        s_row = wp->row;
        s_goff = wp->goff;
        s_koff = wp->koff;
        s_dsl = wp->dsl;
        cbuf = wp->cbuf;
    }
    const int jb = pcone_box[pc];
    const int k0 = pcstart[jb], nch = pcstart[jb + 1] - k0;
    const int g8 = cone_gidx[pc] * 8;
    int nseg = 0, K = 0;
    if (lane < nch) {
        const int4 kj = kp[jb];
        const int4 kk = kd[k0 + lane];
        const int row = g8 + ((kk.x - 2 * kj.x) | ((kk.y - 2 * kj.y) << 1) | ((kk.z - 2 * kj.z) << 2));
        s_row[lane] = row;
        nseg = __ldg(&tab_nseg[row]);
        K = __ldg(&tab_k[row]);
    }
    int incl = nseg, kincl = K;  // inclusive prefixes over the children (lanes 0..7)
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o), w = __shfl_up_sync(0xffffffffu, kincl, o);
        if (lane >= o) {
            incl += v;
            kincl += w;
        }
    }
    if (lane < 8) {
        s_goff[lane + 1] = incl;
        s_koff[lane + 1] = kincl;
    }
    if (lane == 0) s_goff[0] = s_koff[0] = 0;
    __syncwarp();
    // child-cone slots: distinct block j = koff[ch] + kl (list entry kl of child ch; the
    // children's lists are disjoint), one block per lane over all children at once; the first
    // kWarpStage blocks are copied to shared memory with coalesced asynchronous copies, the rest
    // are read from global memory
    for (int j = lane; j < s_koff[nch]; j += 32) {
        int ch = 0;
        while (ch + 1 < nch && s_koff[ch + 1] <= j) ++ch;
        const int kl = j - s_koff[ch];
        if (kl < kSlotCache) {
            const int sl = cm.find(k0 + ch, __ldg(&tab_list[(int64_t)s_row[ch] * kTabList + kl]));
            const bool staged = sl >= 0 && j < kWarpStage;
            s_slot[ch][kl] = staged ? -2 - j : sl;
            if (j < kWarpStage) s_dsl[j] = sl;
        }
    }
    __syncwarp();
    const int nst = min(s_koff[nch], kWarpStage);
    const float* Ws = W;
    const float* Wt = W + PS * PS;
    const float* Wp = Wt + PT * PT;
    const int nsets = NSETS ? NSETS : nrhs;
    for (int r = 0; r < nsets; ++r) {
    constexpr int Q4 = (P + 1) / 2;  // float4 of a coefficient block (P complex values, cstride even)
    static_assert(Q4 <= kStage4, "a staged coefficient block must fit its shared-memory slot");
    for (int x = lane; x < nst * Q4; x += 32) {
        const int j = x / Q4, q = x - (x / Q4) * Q4;
        const int sl = s_dsl[j];
        if (sl < 0) continue;  // missing cone: reported where it is used
        const float4* src = reinterpret_cast<const float4*>(cchild + ((int64_t)sl * nrhs + r) * cstride) + q;
        const unsigned dst = (unsigned)__cvta_generic_to_shared(cbuf + j * kStage4 + q);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_all;" ::: "memory");
    __syncwarp();
    const int total = 2 * s_goff[nch];
    int ch = 0;  // a lane's items only move forward over the children
    for (int item = lane; item < total; item += 32) {
        const int seg = item >> 1, half = item & 1;
        while (ch + 1 < nch && s_goff[ch + 1] <= seg) ++ch;
        const int64_t rowP = (int64_t)s_row[ch] * P;
        const int sg = __ldg(&tab_seg[rowP + (seg - s_goff[ch])]);
        const int j0 = (sg & 0xff) + R * half, len = min(R, ((sg >> 8) & 0xff) - R * half), kl = sg >> 16;
        if (len <= 0) continue;
        // the rare list positions past the cache (rows whose nodes spread over many child cones)
        const int sv = kl < kSlotCache ? s_slot[ch][kl]
                                       : cm.find(k0 + ch, __ldg(&tab_list[(int64_t)s_row[ch] * kTabList + kl]));
        float ts[R], tt[R], tp[R];
        float2 ratio[R], F[R];
        int node[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int64_t e = rowP + j0 + min(q, len - 1);  // short segments repeat their last node
            const float4 t4 = __ldg(&tab_t[e]);
            ts[q] = t4.x;
            tt[q] = t4.y;
            tp[q] = t4.z;
            node[q] = __float_as_int(t4.w);
            ratio[q] = __ldg(&tab_r[e]);
        }
        if (sv <= -2) {
            interp_f32_seg<PS, PT, PP, R, true>(reinterpret_cast<const float2*>(cbuf + (-2 - sv) * kStage4), ts, tt,
                                                tp, F);
        } else if (sv >= 0) {
            interp_f32_seg<PS, PT, PP, R, false, kCoh>(cchild + ((int64_t)sv * nrhs + r) * cstride, ts, tt, tp, F);
        } else {
            set_status(status, IFGF_ERR_INTERNAL);
#pragma unroll
            for (int q = 0; q < R; ++q) F[q] = make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < R; ++q)
            if (q < len && in_bounds(node[q], P, status)) vals[ch][node[q]] = cmul(F[q], ratio[q]);
    }
    __syncwarp();
    for (int n = lane; n < P; n += 32) {  // sum over children, in child order
        float2 a = vals[0][n];
        for (int ch = 1; ch < nch; ++ch) {
            a.x += vals[ch][n].x;
            a.y += vals[ch][n].y;
        }
        vals[0][n] = a;
    }
    __syncwarp();
    for (int n = lane; n < P; n += 32) {
        const int qc = n % PP, qb = (n / PP) % PT, qa = n / (PP * PT);
        float2 acc = make_float2(0.f, 0.f);
        const float2* rw = &vals[0][(qa * PT + qb) * PP];
#pragma unroll
        for (int k = 0; k < PP; ++k) {
            const float w = Wp[qc * PP + k];
            acc.x = fmaf(w, rw[k].x, acc.x);
            acc.y = fmaf(w, rw[k].y, acc.y);
        }
        vals[1][n] = acc;
    }
    __syncwarp();
    for (int n = lane; n < P; n += 32) {
        const int qc = n % PP, qb = (n / PP) % PT, qa = n / (PP * PT);
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < PT; ++j) {
            const float w = Wt[qb * PT + j];
            const float2 v = vals[1][(qa * PT + j) * PP + qc];
            acc.x = fmaf(w, v.x, acc.x);
            acc.y = fmaf(w, v.y, acc.y);
        }
        vals[2][n] = acc;
    }
    __syncwarp();
    for (int n = lane; n < P; n += 32) {
        const int qc = n % PP, qb = (n / PP) % PT, qa = n / (PP * PT);
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < PS; ++i) {
            const float w = Ws[qa * PS + i];
            const float2 v = vals[2][(i * PT + qb) * PP + qc];
            acc.x = fmaf(w, v.x, acc.x);
            acc.y = fmaf(w, v.y, acc.y);
        }
        cparent[(pc * nrhs + r) * cstride + n] = acc;
    }
    __syncwarp();  // the next set reuses the staged blocks and the value rows
    }
}

// ---- Interpolation(d) (Algorithm 8) -----------------------------------------------------------
// One thread per target x: for every B_k in M^d(x) (the cousins of x's level-d box, Eq. (8)),
// add I_P C_{k;gamma}(x) G(x, x_k).  Mixed variant: |x - x_k| = |c_A - c_k + d_A| with the
// integer centre offset c_A - c_k = 2^(D-d+1) n, so
//   kappa |x - x_k| = (kappa H_d sqrt(|n|^2) mod 2 pi) + kappa u (2 c.d_A + |d_A|^2)/(|x - x_k| + |c|).
// interp_target_f32: the level-d sum of target i (CM, LG: the cone map and the grid by value, or
// by const reference where they sit in global memory), for the value sets [r0, r0 + nv), nv <= NR, into
// acc; the target's geometry, the cone lookup and the centred factor are computed once for all
// of them.
template <int PS, int PT, int PP, int NR, bool kCoh, class CM = ConeMap, class LG = LevelGrid>
__device__ __forceinline__ void interp_target_f32(int64_t i, int r0, int nv, int sh, const int32_t* __restrict__ pbox_d,
                                                  const int32_t* __restrict__ pbox_D, const int4* __restrict__ kD,
                                                  const int4* __restrict__ kd, const int32_t* __restrict__ ncs,
                                                  const int32_t* __restrict__ cs, const float4* __restrict__ off,
                                                  CM cm, LG g, const float2* __restrict__ coef,
                                                  const float* __restrict__ phtab, float ku, float inv4piu, int cstride,
                                                  int nrhs, int* __restrict__ status, float2 (&acc)[NR]) {
    const int A = pbox_d[i];
    const int4 kl = kD[pbox_D[i]];
    const int4 kA = kd[A];
    const float4 o = off[i];
    const float dax = (float)((2 * kl.x + 1) - ((2 * kA.x + 1) << sh)) + o.x;
    const float day = (float)((2 * kl.y + 1) - ((2 * kA.y + 1) << sh)) + o.y;
    const float daz = (float)((2 * kl.z + 1) - ((2 * kA.z + 1) << sh)) + o.z;
    const float dd = fmaf(dax, dax, fmaf(day, day, daz * daz));
    const float cscale = (float)(2 << sh);
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = make_float2(0.f, 0.f);
    const int nc = ncs[A];
    for (int t = 0; t < nc; ++t) {
        const int B = cs[(int64_t)A * kMaxCous + t];
        if (!in_bounds(B, cm.nbox, status)) continue;
        const int4 kb = kd[B];
        const float vx = __fadd_rn((float)((2 * kl.x + 1) - ((2 * kb.x + 1) << sh)), o.x);
        const float vy = __fadd_rn((float)((2 * kl.y + 1) - ((2 * kb.y + 1) << sh)), o.y);
        const float vz = __fadd_rn((float)((2 * kl.z + 1) - ((2 * kb.z + 1) << sh)), o.z);
        const ConeLocal cl = locate_f32(g, vx, vy, vz);
        const int s = cm.find(B, cl.gamma(g));
        if (s < 0) {
            set_status(status, IFGF_ERR_INTERNAL);
            continue;
        }
        const int nx = kA.x - kb.x, ny = kA.y - kb.y, nz = kA.z - kb.z;
        const int nn = nx * nx + ny * ny + nz * nz;
        const float cx = cscale * nx, cy = cscale * ny, cz = cscale * nz;
        const float cn = cscale * sqrtf((float)nn);
        const float num = fmaf(2.f, fmaf(cx, dax, fmaf(cy, day, cz * daz)), dd);
        const float corr = __fdividef(num, cl.r + cn);
        const float2 e = cis_f32(fmaf(ku, corr, __ldg(&phtab[nn])));
        const float w = __fdividef(inv4piu, cl.r);
        const float2 ew = make_float2(e.x * w, e.y * w);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            if (r < nv) {
                const float2 F =
                    interp_f32<PS, PT, PP, kCoh>(coef + ((int64_t)s * nrhs + r0 + r) * cstride, cl.ts, cl.tt, cl.tp);
                const float2 tv = cmul(F, ew);
                acc[r].x += tv.x;
                acc[r].y += tv.y;
            }
        }
    }
}

}  // namespace ifgf
