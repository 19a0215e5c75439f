// Plan construction on the GPU: the octree of Sec. 2 with the Morton order of Sec. 3.2.1,
// neighbour and cousin sets of Eq. (2), and the relevant cone segments of Eq. (4).
//
// All heavy steps run as device kernels; the host only reads back sizes (bounding box,
// boxes per level, cones per level) to size the next allocations.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ifgf_internal.cuh"

namespace ifgf {
namespace {

constexpr int kThreads = 256;

// ---- bounding box -----------------------------------------------------------------------
__global__ void k_bbox_partial(const double* __restrict__ X, int64_t N, double* __restrict__ part) {
    __shared__ double smin[3][kThreads], smax[3][kThreads];
    __shared__ int sbad[kThreads];
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double v = X[(int64_t)c * N + i];
            if (!isfinite(v)) bad = 1;
            mn[c] = fmin(mn[c], v);
            mx[c] = fmax(mx[c], v);
        }
    }
    for (int c = 0; c < 3; ++c) {
        smin[c][threadIdx.x] = mn[c];
        smax[c][threadIdx.x] = mx[c];
    }
    sbad[threadIdx.x] = bad;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            for (int c = 0; c < 3; ++c) {
                smin[c][threadIdx.x] = fmin(smin[c][threadIdx.x], smin[c][threadIdx.x + o]);
                smax[c][threadIdx.x] = fmax(smax[c][threadIdx.x], smax[c][threadIdx.x + o]);
            }
            sbad[threadIdx.x] |= sbad[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int c = 0; c < 3; ++c) {
            part[blockIdx.x * 7 + c] = smin[c][0];
            part[blockIdx.x * 7 + 3 + c] = smax[c][0];
        }
        part[blockIdx.x * 7 + 6] = sbad[0];
    }
}

// ---- keys -------------------------------------------------------------------------------
// Level-21 box index k = floor(u 2^20) (clamped), u = (x - a)/H1, then the Morton key.
__global__ void k_keys(const double* __restrict__ X, int64_t N, double a0, double a1, double a2, double H1,
                       uint64_t* __restrict__ keys, int32_t* __restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double a[3] = {a0, a1, a2};
    uint32_t k[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double u = __ddiv_rn(__dsub_rn(X[(int64_t)c * N + i], a[c]), H1);
        double f = floor(__dmul_rn(u, 1048576.0));
        f = fmin(fmax(f, 0.0), 1048575.0);
        k[c] = (uint32_t)f;
    }
    keys[i] = morton3(k[0], k[1], k[2]);
    vals[i] = (int32_t)i;
}

__global__ void k_gather_points(const double* __restrict__ X, int64_t N, const int32_t* __restrict__ perm,
                                double* __restrict__ Xs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t o = perm[i];
#pragma unroll
    for (int c = 0; c < 3; ++c) Xs[(int64_t)c * N + i] = X[(int64_t)c * N + o];
}

// Coarsest level at which the keys of points i-1 and i differ: boxes split there and below.
__global__ void k_level_split(const uint64_t* __restrict__ keys, int64_t N, uint8_t* __restrict__ d0,
                              unsigned long long* __restrict__ hist) {
    __shared__ unsigned int h[24];
    if (threadIdx.x < 24) h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        int lev = 0;
        if (i > 0) {
            const uint64_t x = keys[i] ^ keys[i - 1];
            if (x == 0)
                lev = 22;
            else
                lev = kKeyLevel - (63 - __clzll((long long)x)) / 3;
            atomicAdd(&h[lev], 1u);
        }
        d0[i] = (uint8_t)lev;
    }
    __syncthreads();
    if (threadIdx.x < 24 && h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], (unsigned long long)h[threadIdx.x]);
}

__global__ void k_level_flags(const uint8_t* __restrict__ d0, int64_t N, int d, int32_t* __restrict__ flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    flag[i] = (i == 0 || (int)d0[i] <= d) ? 1 : 0;
}

__global__ void k_level_boxes(const int32_t* __restrict__ flag, const int32_t* __restrict__ pos,
                              const uint64_t* __restrict__ keys, int64_t N, int d, int32_t nbox,
                              int32_t* __restrict__ start, uint64_t* __restrict__ bkey, int4* __restrict__ bk,
                              int32_t* __restrict__ pbox) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) start[nbox] = (int32_t)N;
    if (i >= N) return;
    const int32_t f = flag[i], b = pos[i] + f - 1;
    pbox[i] = b;
    if (f) {
        const uint64_t key = keys[i] >> (3 * (kKeyLevel - d));
        start[b] = (int32_t)i;
        bkey[b] = key;
        bk[b] = make_int4((int)compact3(key), (int)compact3(key >> 1), (int)compact3(key >> 2), 0);
    }
}

__global__ void k_parents(const int32_t* __restrict__ start, int32_t n, const int32_t* __restrict__ pbox_up,
                          int32_t* __restrict__ parent) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    parent[b] = pbox_up ? pbox_up[start[b]] : -1;
}

__global__ void k_child_start(const int32_t* __restrict__ parent_child, int32_t nchild, int32_t nparent,
                              int32_t* __restrict__ cstart) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c == 0) cstart[nparent] = nchild;
    if (c >= nchild) return;
    const int p = parent_child[c];
    if (c == 0 || parent_child[c - 1] != p) cstart[p] = c;
}

// Offset of every sorted point from its leaf centre in grid units u = H_D/2, rounded to FP32.
__global__ void k_offsets(const double* __restrict__ Xs, int64_t N, double a0, double a1, double a2, double H1,
                          double scale, const int32_t* __restrict__ pboxD, const int4* __restrict__ kD,
                          float4* __restrict__ off) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int4 k = kD[pboxD[i]];
    const double a[3] = {a0, a1, a2};
    const int kk[3] = {k.x, k.y, k.z};
    float o[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double u = __ddiv_rn(__dsub_rn(Xs[(int64_t)c * N + i], a[c]), H1);
        const double t = __dmul_rn(u, scale);
        o[c] = __double2float_rn(__dsub_rn(t, (double)(2 * (int64_t)kk[c] + 1)));
    }
    off[i] = make_float4(o[0], o[1], o[2], 0.f);
}

__device__ __forceinline__ int find_box(const uint64_t* __restrict__ keys, int n, uint64_t key) {
    int lo = 0, hi = n - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const uint64_t k = keys[mid];
        if (k == key) return mid;
        if (k < key)
            lo = mid + 1;
        else
            hi = mid - 1;
    }
    return -1;
}

// Neighbours N B (Eq. (2)): relevant boxes with ||j - k||_inf <= 1, ascending.  The 27
// candidate lookups fill a register array (fully unrolled), then an ascending selection pass
// writes the list.
__global__ void k_neighbours(const uint64_t* __restrict__ keys, const int4* __restrict__ bk, int n, int d,
                             int32_t* __restrict__ nnb, int32_t* __restrict__ nb) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const int4 k = bk[b];
    const int side = 1 << (d - 1);
    int found[kMaxNbr];
#pragma unroll
    for (int c = 0; c < kMaxNbr; ++c) {
        const int x = k.x + (c % 3) - 1, y = k.y + ((c / 3) % 3) - 1, z = k.z + (c / 9) - 1;
        const bool in = x >= 0 && y >= 0 && z >= 0 && x < side && y < side && z < side;
        found[c] = in ? find_box(keys, n, morton3((uint32_t)x, (uint32_t)y, (uint32_t)z)) : -1;
    }
    int cnt = 0, last = -1;
    for (int t = 0; t < kMaxNbr; ++t) {
        int best = 0x7fffffff;
#pragma unroll
        for (int c = 0; c < kMaxNbr; ++c)
            if (found[c] > last && found[c] < best) best = found[c];
        if (best == 0x7fffffff) break;
        nb[(int64_t)b * kMaxNbr + cnt++] = best;
        last = best;
    }
    nnb[b] = cnt;
}

// Cousins M B (Eq. (2)): children of the parent's neighbours that are not neighbours.  The
// parent's neighbours are ascending and children are contiguous, so the list is ascending.
__global__ void k_cousins(const int4* __restrict__ bk, const int32_t* __restrict__ parent, int n,
                          const int32_t* __restrict__ pnnb, const int32_t* __restrict__ pnb,
                          const int32_t* __restrict__ pcstart, int32_t* __restrict__ ncs, int32_t* __restrict__ cs) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const int4 k = bk[b];
    const int pb = parent[b];
    int cnt = 0;
    for (int t = 0; t < pnnb[pb]; ++t) {
        const int q = pnb[(int64_t)pb * kMaxNbr + t];
        for (int c = pcstart[q]; c < pcstart[q + 1]; ++c) {
            const int4 kc = bk[c];
            const int m = max(abs(kc.x - k.x), max(abs(kc.y - k.y), abs(kc.z - k.z)));
            if (m > 1 && cnt < kMaxCous) cs[(int64_t)b * kMaxCous + cnt++] = c;
        }
    }
    ncs[b] = cnt;
}

// ---- cone activation (Eq. (4), discrete form) -------------------------------------------
// A relevant (box, gamma) is recorded either as a flag of the dense n_d x C_d table or as the
// key box * C + gamma in an open-addressing hash set (sparse levels). In the hash set the lanes
// of a warp that hold the same key insert it once.
constexpr unsigned long long kEmptyKey = ~0ull;
constexpr int kMaxProbe = 128;
struct ConeMark {
    int32_t* dense;             // [n*C] flags, or nullptr
    unsigned long long* hkeys;  // [hmask + 1] keys or kEmptyKey
    unsigned long long hmask;
    int64_t C;
    int* overflow;
    __device__ __forceinline__ void mark(int box, int gamma) const {
        const unsigned long long key = (unsigned long long)box * (unsigned long long)C + (unsigned long long)gamma;
        if (dense) {
            dense[key] = 1;
            return;
        }
        const unsigned same = __match_any_sync(__activemask(), key);
        if ((int)(threadIdx.x & 31) != __ffs(same) - 1) return;  // one lane per distinct key
        unsigned long long h = (key * 0x9E3779B97F4A7C15ull) >> 17;
        for (int probe = 0; probe < kMaxProbe; ++probe, ++h) {
            h &= hmask;
            const unsigned long long cur = __ldcg(&hkeys[h]);
            if (cur == key) return;
            if (cur == kEmptyKey) {
                const unsigned long long prev = atomicCAS(&hkeys[h], kEmptyKey, key);
                if (prev == kEmptyKey || prev == key) return;
            }
        }
        atomicExch(overflow, 1);  // table too full: the level is redone with a larger one
    }
};

// Cousin points x in V B: every point marks, in each cousin box of its level-d box, the cone
// that contains it.
__global__ void k_mark_cousin_points(int64_t N, int D, int d, const int32_t* __restrict__ pbox_d,
                                     const int32_t* __restrict__ pbox_D, const int4* __restrict__ kD,
                                     const int4* __restrict__ kd, const int32_t* __restrict__ ncs,
                                     const int32_t* __restrict__ cs, const float4* __restrict__ off, LevelGrid g,
                                     ConeMark mark) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int A = pbox_d[i];
    const int4 kl = kD[pbox_D[i]];
    const float4 o = off[i];
    const int sh = D - d;
    const int nc = ncs[A];
    for (int t = 0; t < nc; ++t) {
        const int B = cs[(int64_t)A * kMaxCous + t];
        const int4 kb = kd[B];
        const float vx = __fadd_rn((float)((2 * kl.x + 1) - ((2 * kb.x + 1) << sh)), o.x);
        const float vy = __fadd_rn((float)((2 * kl.y + 1) - ((2 * kb.y + 1) << sh)), o.y);
        const float vz = __fadd_rn((float)((2 * kl.z + 1) - ((2 * kb.z + 1) << sh)), o.z);
        mark.mark(B, classify_f32(g, vx, vy, vz));
    }
}

// Node offset (grid units) of node n of cone gamma, from the parent's node tables.
__device__ __forceinline__ float3 node_grid(const LevelGrid& gp, int Ps, int Pt, int Pp, int gam, int n) {
    const int ip = gam % gp.np, it = (gam / gp.np) % gp.nt, is = gam / (gp.np * gp.nt);
    const int c = n % Pp, b = (n / Pp) % Pt, a = n / (Pp * Pt);
    const float rho = gp.rho[is * Ps + a];
    const float st = gp.stn[it * Pt + b], ct = gp.ctn[it * Pt + b];
    const float cp = gp.cpn[ip * Pp + c], sp = gp.spn[ip * Pp + c];
    return make_float3(__fmul_rn(rho, __fmul_rn(st, cp)), __fmul_rn(rho, __fmul_rn(st, sp)), __fmul_rn(rho, ct));
}

// Nodes of the relevant parent cones: every node of every relevant level-(d-1) cone marks,
// in each child box of the cone's box, the cone that contains it.
__global__ void k_mark_parent_nodes(int64_t ncp, int P, int Ps, int Pt, int Pp, int D, int d,
                                    const int32_t* __restrict__ pcone_box, const int32_t* __restrict__ pcone_gam,
                                    const int4* __restrict__ kp, const int32_t* __restrict__ pcstart,
                                    const int4* __restrict__ kd, LevelGrid gp, LevelGrid g, ConeMark mark) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncp * P) return;
    const int64_t pc = t / P;
    const int n = (int)(t - pc * P);
    const int jb = pcone_box[pc];
    const float3 q = node_grid(gp, Ps, Pt, Pp, pcone_gam[pc], n);
    const int4 kj = kp[jb];
    const int sh = D - d;
    for (int kb = pcstart[jb]; kb < pcstart[jb + 1]; ++kb) {
        const int4 kk = kd[kb];
        const float ox = (float)((2 * (kk.x - 2 * kj.x) - 1) << sh);
        const float oy = (float)((2 * (kk.y - 2 * kj.y) - 1) << sh);
        const float oz = (float)((2 * (kk.z - 2 * kj.z) - 1) << sh);
        mark.mark(kb, classify_f32(g, __fsub_rn(q.x, ox), __fsub_rn(q.y, oy), __fsub_rn(q.z, oz)));
    }
}

// ---- node tables (translation invariance of the propagation geometry) ------------------
__global__ void k_flag_gamma(const int32_t* __restrict__ cone_gam, int64_t nc, int32_t* __restrict__ flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nc) flags[cone_gam[i]] = 1;
}

__global__ void k_gamma_rows(const int32_t* __restrict__ flags, const int32_t* __restrict__ pos, int C,
                             int32_t* __restrict__ gam_list) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < C && flags[i]) gam_list[pos[i]] = i;
}

__global__ void k_cone_rows(const int32_t* __restrict__ cone_gam, int64_t nc, const int32_t* __restrict__ pos,
                            int32_t* __restrict__ cone_gidx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nc) cone_gidx[i] = pos[cone_gam[i]];
}

// Entry (g*8 + o)*P + n: node n of cone index gam_list[g] of the parent grid, seen from the
// child centre at octant o (bit 0: +x half, bit 1: +y, bit 2: +z); offsets in child grid units.
__global__ void k_node_tables(int64_t total, const int32_t* __restrict__ gam_list, int Ps, int Pt, int Pp, int sh,
                              LevelGrid gp, LevelGrid g, float ku, float4* __restrict__ tab_t,
                              float2* __restrict__ tab_r) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int P = Ps * Pt * Pp;
    const int n = (int)(e % P);
    const int o = (int)((e / P) % 8);
    const int gam = gam_list[e / (8 * (int64_t)P)];
    const int ip = gam % gp.np, it = (gam / gp.np) % gp.nt, is = gam / (gp.np * gp.nt);
    const int qc = n % Pp, qb = (n / Pp) % Pt, qa = n / (Pp * Pt);
    const float rho = gp.rho[is * Ps + qa];
    const float st = gp.stn[it * Pt + qb], ct = gp.ctn[it * Pt + qb];
    const float cp = gp.cpn[ip * Pp + qc], sp = gp.spn[ip * Pp + qc];
    const float qx = __fmul_rn(rho, __fmul_rn(st, cp)), qy = __fmul_rn(rho, __fmul_rn(st, sp));
    const float qz = __fmul_rn(rho, ct);
    const float ox = (float)((2 * (o & 1) - 1) << sh);
    const float oy = (float)((2 * ((o >> 1) & 1) - 1) << sh);
    const float oz = (float)((2 * ((o >> 2) & 1) - 1) << sh);
    const ConeLocal cl = locate_f32(g, __fsub_rn(qx, ox), __fsub_rn(qy, oy), __fsub_rn(qz, oz));
    const float rj = sqrtf(fmaf(qx, qx, fmaf(qy, qy, qz * qz)));
    const float oo = 3.0f * (float)(1 << sh) * (float)(1 << sh);
    const float qo = fmaf(qx, ox, fmaf(qy, oy, qz * oz));
    // G(x,x_k)/G(x,x_j) = (r_j/r_k) exp(i kappa (r_k - r_j)), r_k - r_j = (|o|^2 - 2 q.o)/(r_k + r_j)
    const float dr = fmaf(-2.f, qo, oo) / (cl.r + rj);
    const float2 ex = cis_f32(ku * dr);
    const float w = rj / cl.r;
    tab_t[e] = make_float4(cl.ts, cl.tt, cl.tp, __int_as_float(cl.gamma(g)));
    tab_r[e] = make_float2(ex.x * w, ex.y * w);
}

// Distinct child cones of each table row (gamma, octant): the list, and the row's entries sorted
// by their position in it, with the node index in tab_t.w (replacing the cone index).  Rows are built from the 75-node classification, so
// K <= 75 <= kTabList; a row past kTabList would make the build drop the level's tables.
__global__ void k_node_lists(int P, float4* __restrict__ tab_t, float2* __restrict__ tab_r,
                             int32_t* __restrict__ tab_k, int32_t* __restrict__ tab_list,
                             int16_t* __restrict__ tab_perm, int32_t* __restrict__ tab_nseg,
                             int32_t* __restrict__ tab_seg, int32_t* __restrict__ tab_run,
                             int* __restrict__ overflow) {
    __shared__ int alpha[128];  // child cone of each node
    __shared__ int first[128];  // 1 if the node is the first with its child cone
    __shared__ int idx[128];    // list position, defined where first[] is set
    __shared__ int kpos[128];   // list position of every node
    __shared__ int segst[128];  // 1 if the sorted entry starts a segment
    const int64_t row = blockIdx.x;
    const int n = threadIdx.x;
    if (n < P) alpha[n] = __float_as_int(tab_t[row * P + n].w);
    segst[n] = 0;
    __syncthreads();
    if (n < P) {
        int f = 1;
        for (int m = 0; m < n; ++m)
            if (alpha[m] == alpha[n]) f = 0;
        first[n] = f;
    }
    __syncthreads();
    if (n == 0) {
        int K = 0;
        for (int m = 0; m < P; ++m) {
            if (first[m]) {
                if (K < kTabList) tab_list[row * kTabList + K] = alpha[m];
                idx[m] = K++;
            }
        }
        tab_k[row] = K;
        if (K > kTabList) atomicExch(overflow, 1);
    }
    __syncthreads();
    if (n < P) {
        int k = 0;
        for (int m = 0; m <= n; ++m)
            if (first[m] && alpha[m] == alpha[n]) k = idx[m];
        kpos[n] = k;
    }
    __syncthreads();
    // stable position of node n among the row's nodes ordered by child cone; the run of its
    // child cone starts at `before` and holds `cnt` entries
    int k = 0, pos = 0, before = 0, cnt = 0;
    float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 rr = make_float2(0.f, 0.f);
    if (n < P) {
        k = kpos[n];
        for (int m = 0; m < P; ++m) {
            pos += (kpos[m] < k) || (kpos[m] == k && m < n);
            before += kpos[m] < k;
            cnt += kpos[m] == k;
        }
        t = tab_t[row * P + n];
        t.w = __int_as_float(n);  // node index in the parent cone (as tab_perm)
        rr = tab_r[row * P + n];
        segst[pos] = (pos - before) % kSegLen == 0;
    }
    __syncthreads();  // every entry is read before any is moved
    if (n < P) {
        tab_t[row * P + pos] = t;
        tab_r[row * P + pos] = rr;
        tab_perm[row * P + pos] = (int16_t)n;
        if (segst[pos]) {
            int sidx = 0;
            for (int j = 0; j < pos; ++j) sidx += segst[j];
            const int len = min(kSegLen, before + cnt - pos);
            tab_seg[row * P + sidx] = pos | (len << 8) | (k << 16);
        }
        if (first[n] && k < kTabList) {  // first segment of this child cone's run
            int rs = 0;
            for (int j = 0; j < before; ++j) rs += segst[j];
            tab_run[row * (kTabList + 1) + k] = rs;
        }
        if (n == 0) {
            int ns = 0;
            for (int j = 0; j < P; ++j) ns += segst[j];
            tab_nseg[row] = ns;
            int K = 0;
            for (int m = 0; m < P; ++m) K += first[m];
            tab_run[row * (kTabList + 1) + min(K, kTabList)] = ns;
        }
    }
}

// Cones grouped by cone index: key = (box >> bb_shift, gamma), stably sorted (the cone list is
// already in box order), then cut into chunks of at most kChunkBoxes cones of one key.
__global__ void k_gamma_keys(int64_t nc, const int32_t* __restrict__ cone_box, const int32_t* __restrict__ cone_gam,
                             int bb_shift, int C, uint64_t* __restrict__ keys, int32_t* __restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    keys[i] = (uint64_t)(cone_box[i] >> bb_shift) * (uint64_t)C + (uint64_t)cone_gam[i];
    vals[i] = (int32_t)i;
}
__global__ void k_gamma_chunk_flags(int64_t n, const uint64_t* __restrict__ keys, int32_t* __restrict__ flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int f = 1;
    if (i > 0 && keys[i] == keys[i - 1]) {
        int64_t lo = 0, hi = i;  // first index with this key
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (keys[mid] < keys[i]) lo = mid + 1;
            else hi = mid;
        }
        f = (i - lo) % kChunkBoxes == 0;
    }
    flags[i] = f;
}
__global__ void k_gamma_chunk_fill(int64_t n, const int32_t* __restrict__ flags, const int32_t* __restrict__ pos,
                                   int32_t* __restrict__ gchunk) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (flags[i]) gchunk[pos[i]] = (int32_t)i;
    if (i == n - 1) gchunk[pos[i] + flags[i]] = (int32_t)n;  // end of the last chunk
}

// Activation from the nodes of the relevant parent cones, one warp per chunk (kMarkWarps chunks
// per block, no block-wide barrier): the child cone of node n seen from child octant o is
// classified once for the chunk (it depends on (gamma, o, n) only), for the octants that some box
// of the chunk has a child at, and marked in every child at octant o of the chunk's boxes.
constexpr int kMarkWarps = 8;
__global__ void __launch_bounds__(32 * kMarkWarps, 6)
k_mark_parent_nodes_chunk(const int32_t* __restrict__ gchunk, int64_t nchunk, const int32_t* __restrict__ gorder,
                          const int32_t* __restrict__ pcone_box, const int32_t* __restrict__ pcone_gam,
                          const int4* __restrict__ kp, const int32_t* __restrict__ pcstart,
                          const int4* __restrict__ kd, int D, int d, LevelGrid gp, LevelGrid g, ConeMark mark) {
    constexpr int Ps = 3, Pt = 5, Pp = 5, P = 75;
    __shared__ int s_alpha_w[kMarkWarps][8][P];
    __shared__ float4 s_q_w[kMarkWarps][P];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * kMarkWarps + warp;
    if (c >= nchunk) return;  // the whole warp leaves; nothing below synchronises the block
    int(*s_alpha)[P] = s_alpha_w[warp];
    float4* s_q = s_q_w[warp];
    const int c0 = gchunk[c], nb = gchunk[c + 1] - c0;  // nb <= kChunkBoxes
    const int gam = pcone_gam[gorder[c0]];
    // the cone's node offsets from the box centre (grid units), once for all octants
    for (int n = lane; n < P; n += 32) {
        const float3 q = node_grid(gp, Ps, Pt, Pp, gam, n);
        s_q[n] = make_float4(q.x, q.y, q.z, 0.f);
    }
    // octants with a child in some box of the chunk: lane x takes child x & 7 of box x >> 3
    int om = 0;
    for (int x = lane; x < 8 * nb; x += 32) {
        const int jb = pcone_box[gorder[c0 + (x >> 3)]];
        const int kb = pcstart[jb] + (x & 7);
        if (kb < pcstart[jb + 1]) {
            const int4 kj = kp[jb], kk = kd[kb];
            om |= 1 << ((kk.x - 2 * kj.x) | ((kk.y - 2 * kj.y) << 1) | ((kk.z - 2 * kj.z) << 2));
        }
    }
    om = __reduce_or_sync(0xffffffffu, om);
    __syncwarp();  // the node offsets are visible to the whole warp
    const int sh = D - d;
    for (int x = lane; x < __popc(om) * P; x += 32) {
        const int oi = x / P, n = x - oi * P;
        unsigned m = (unsigned)om;  // the oi-th octant present (oi < popc(om), so m stays nonzero)
        for (int i = 0; i < oi; ++i) m &= m - 1;
        const int o = __ffs(m) - 1;
        const float4 q = s_q[n];
        const float ox = (float)((2 * (o & 1) - 1) << sh);
        const float oy = (float)((2 * ((o >> 1) & 1) - 1) << sh);
        const float oz = (float)((2 * ((o >> 2) & 1) - 1) << sh);
        s_alpha[o][n] = classify_f32(g, __fsub_rn(q.x, ox), __fsub_rn(q.y, oy), __fsub_rn(q.z, oz));
    }
    __syncwarp();
    for (int b = 0; b < nb; ++b) {
        const int jb = pcone_box[gorder[c0 + b]];
        const int k0 = pcstart[jb], nch = pcstart[jb + 1] - k0;
        const int4 kj = kp[jb];
        for (int ch = 0; ch < nch; ++ch) {
            const int4 kk = kd[k0 + ch];
            const int o = (kk.x - 2 * kj.x) | ((kk.y - 2 * kj.y) << 1) | ((kk.z - 2 * kj.z) << 2);
            // the 75 nodes fall in a few child cones: collect the distinct ones over all nodes (lane
            // g keeps the g-th), then mark each once
            int a[3];
            bool pend[3];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const int n = lane + 32 * j;
                pend[j] = n < P;
                a[j] = pend[j] ? s_alpha[o][n] : -1;
            }
            int mine = -1, G = 0;
            for (int guard = 0; guard < P; ++guard) {
                const unsigned b0 = __ballot_sync(0xffffffffu, pend[0]), b1 = __ballot_sync(0xffffffffu, pend[1]),
                               b2 = __ballot_sync(0xffffffffu, pend[2]);
                if (!(b0 | b1 | b2)) break;
                const int sj = b0 ? 0 : (b1 ? 1 : 2);
                const int src = __ffs(b0 ? b0 : (b1 ? b1 : b2)) - 1;
                const int v = __shfl_sync(0xffffffffu, sj == 0 ? a[0] : (sj == 1 ? a[1] : a[2]), src);
                if (lane == (G & 31)) mine = v;
                if ((G & 31) == 31) {  // 32 distinct cones collected: mark them before collecting more
                    mark.mark(k0 + ch, mine);
                    mine = -1;
                }
                ++G;
#pragma unroll
                for (int j = 0; j < 3; ++j) pend[j] = pend[j] && a[j] != v;
            }
            if (mine >= 0) mark.mark(k0 + ch, mine);
        }
    }
}

// Activation from the node tables: every node of every relevant parent cone marks the child
// cone its table entry names (the same exact classification, computed once per gamma).
__global__ void k_mark_parent_nodes_tab(int64_t ncp, const int32_t* __restrict__ pcone_box,
                                        const int32_t* __restrict__ cone_gidx, const int4* __restrict__ kp,
                                        const int32_t* __restrict__ pcstart, const int4* __restrict__ kd,
                                        const int32_t* __restrict__ tab_k, const int32_t* __restrict__ tab_list,
                                        ConeMark mark) {
    // one thread per (parent cone, child slot): the row's distinct child cones are marked in the child
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncp * 8) return;
    const int64_t pc = t >> 3;
    const int ch = (int)(t & 7);
    const int jb = pcone_box[pc];
    const int kb = pcstart[jb] + ch;
    if (kb >= pcstart[jb + 1]) return;
    const int4 kj = kp[jb];
    const int4 kk = kd[kb];
    const int o = (kk.x - 2 * kj.x) | ((kk.y - 2 * kj.y) << 1) | ((kk.z - 2 * kj.z) << 2);
    const int64_t row = (int64_t)cone_gidx[pc] * 8 + o;
    const int K = tab_k[row];
    for (int k = 0; k < K; ++k) mark.mark(kb, tab_list[row * kTabList + k]);
}


// Sparse levels: the hash set's keys become the cone list sorted by (box, gamma).
__global__ void k_hash_flags(int64_t H, const unsigned long long* __restrict__ hkeys, int32_t* __restrict__ flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < H) flags[i] = hkeys[i] != kEmptyKey;
}
__global__ void k_hash_gather(int64_t H, const unsigned long long* __restrict__ hkeys,
                              const int32_t* __restrict__ flags, const int32_t* __restrict__ pos,
                              uint64_t* __restrict__ keys, int32_t* __restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= H || !flags[i]) return;
    keys[pos[i]] = hkeys[i];
    vals[pos[i]] = pos[i];
}
__global__ void k_split_keys(int64_t nc, const uint64_t* __restrict__ keys, int64_t C, int32_t* __restrict__ cone_box,
                             int32_t* __restrict__ cone_gam) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    cone_box[i] = (int32_t)(keys[i] / (uint64_t)C);
    cone_gam[i] = (int32_t)(keys[i] % (uint64_t)C);
}
__global__ void k_box_cone_starts(int n, int64_t nc, const int32_t* __restrict__ cone_box, int32_t* __restrict__ bcs) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > n) return;
    int64_t lo = 0, hi = nc;  // first cone of a box >= b
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (cone_box[mid] < b) lo = mid + 1;
        else hi = mid;
    }
    bcs[b] = (int32_t)lo;
}

// Row starts of a sparse level's cone list: entry b * nrow + w is the first cone of box b with
// gamma >= w * np; entry n * nrow closes the last row.
__global__ void k_row_starts(int64_t total, int nrow, int np, const int32_t* __restrict__ bcs,
                             const int32_t* __restrict__ cone_gam, int32_t* __restrict__ rows) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e > total) return;
    const int64_t b = e / nrow;
    const int w = (int)(e - b * nrow);
    if (e == total) {
        rows[e] = bcs[b];  // b == n: one past the last cone
        return;
    }
    int lo = bcs[b], hi = bcs[b + 1];
    const int key = w * np;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cone_gam[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    rows[e] = lo;
}

__global__ void k_finalize_cones(int32_t* __restrict__ slot, const int32_t* __restrict__ pos, int64_t total, int C,
                                 int32_t* __restrict__ cone_box, int32_t* __restrict__ cone_gam) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    if (slot[e]) {
        const int32_t s = pos[e];
        slot[e] = s;
        cone_box[s] = (int32_t)(e / C);
        cone_gam[s] = (int32_t)(e % C);
    } else {
        slot[e] = -1;
    }
}

// ---- host-side tables (the same formulas as the method's statement; see readings) --------
double cheb_node(int j, int P) { return std::cos(M_PI * (2.0 * j + 1.0) / (2.0 * P)); }
double node_in(int idx, double w, double t) { return w * ((double)idx + 0.5 * (1.0 + t)); }

template <class T>
T* upload(Plan& p, const std::vector<T>& h) {
    T* d = dalloc<T>(p, h.size());
    if (!h.empty()) IFGF_CUDA(cudaMemcpyAsync(d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, p.stream));
    return d;
}

void build_grid(Plan& p, int d, const ifgf_options& opt, std::vector<std::vector<char>>& keep) {
    const double eta = std::sqrt(3.0) / 3.0;
    const double Hd = std::ldexp(p.H1, 1 - d);
    int e = 0;
    while (p.kappa > 0.0 && e < 24 && p.kappa * Hd > 2.0 * M_PI * opt.tau * std::ldexp(1.0, e) * (1.0 + std::ldexp(1.0, -10))) ++e;
    const int ns = opt.base_cones[0] << e, nt = opt.base_cones[1] << e, np = opt.base_cones[2] << e;
    LevelGrid& g = p.L[d].g;
    g.ns = ns;
    g.nt = nt;
    g.np = np;
    const int64_t C = (int64_t)ns * nt * np;
    if (C > (int64_t)1 << 30) fail(IFGF_ERR_UNSUPPORTED, "cone grid too fine for the dense cone table");
    g.C = (int)C;
    g.ds64 = eta / ns;
    g.dt64 = M_PI / nt;
    g.dp64 = 2.0 * M_PI / np;
    g.h64 = 0.5 * std::sqrt(3.0) * Hd;
    const double hgd = std::sqrt(3.0) * std::ldexp(1.0, p.D - d);
    g.hg = (float)hgd;
    g.s_scale = (float)(ns / eta);
    g.t_scale = (float)(nt / M_PI);
    g.p_scale = (float)(np / (2.0 * M_PI));
    // Margins (in bin widths) of the classification's fast path: farther from every edge of its
    // candidate bin than these, a point provably has the bins that the exact edge tests give
    // (bounds of the approximate coordinates and of the tests' rounding, times about eight).
    g.ms = 4e-6f;                                        // s: relative, times (bin + 1)
    g.tA = (float)(4e-6 * nt / M_PI);                    // theta: approximation error
    g.tB = (float)(1.2e-6 * (double)nt * nt / (2.0 * M_PI));  // theta: edge test near the poles
    g.mp = (float)(8e-6 * np / (2.0 * M_PI));            // phi
    g.s2w = (float)(2.0 / g.ds64);
    g.t2w = (float)(2.0 / g.dt64);
    g.p2w = (float)(2.0 / g.dp64);
    std::vector<float> R2(ns, INFINITY), C2(nt), cph(np), sph(np);
    std::vector<int> cpos(nt);
    for (int i = 1; i < ns; ++i) {
        const double R = hgd / ((double)i * g.ds64);
        R2[i] = (float)(R * R);
    }
    for (int i = 0; i < nt; ++i) {
        const double c = std::cos(M_PI * (double)i / (double)nt);
        C2[i] = (float)(c * c);
        cpos[i] = c >= 0.0;
    }
    for (int j = 0; j < np; ++j) {
        cph[j] = (float)std::cos(2.0 * M_PI * (double)j / (double)np);
        sph[j] = (float)std::sin(2.0 * M_PI * (double)j / (double)np);
    }
    std::vector<float> rho(ns * p.Ps), sn(ns * p.Ps), ctn(nt * p.Pt), stn(nt * p.Pt), cpn(np * p.Pp), spn(np * p.Pp);
    std::vector<double> sn64(ns * p.Ps), tn64(nt * p.Pt), pn64(np * p.Pp);
    for (int is = 0; is < ns; ++is)
        for (int a = 0; a < p.Ps; ++a) {
            const double s = node_in(is, g.ds64, cheb_node(a, p.Ps));
            rho[is * p.Ps + a] = (float)(hgd / s);
            sn[is * p.Ps + a] = (float)s;
            sn64[is * p.Ps + a] = s;
        }
    for (int it = 0; it < nt; ++it)
        for (int b = 0; b < p.Pt; ++b) {
            const double th = node_in(it, g.dt64, cheb_node(b, p.Pt));
            ctn[it * p.Pt + b] = (float)std::cos(th);
            stn[it * p.Pt + b] = (float)std::sin(th);
            tn64[it * p.Pt + b] = th;
        }
    for (int ip = 0; ip < np; ++ip)
        for (int c = 0; c < p.Pp; ++c) {
            const double ph = node_in(ip, g.dp64, cheb_node(c, p.Pp));
            cpn[ip * p.Pp + c] = (float)std::cos(ph);
            spn[ip * p.Pp + c] = (float)std::sin(ph);
            pn64[ip * p.Pp + c] = ph;
        }
    g.R2 = upload(p, R2);
    g.C2 = upload(p, C2);
    g.cpos = upload(p, cpos);
    g.cph = upload(p, cph);
    g.sph = upload(p, sph);
    g.rho = upload(p, rho);
    g.snode = upload(p, sn);
    g.ctn = upload(p, ctn);
    g.stn = upload(p, stn);
    g.cpn = upload(p, cpn);
    g.spn = upload(p, spn);
    g.snode64 = upload(p, sn64);
    g.tnode64 = upload(p, tn64);
    g.pnode64 = upload(p, pn64);
    // Centred-factor phase of the box-centre offset (kappa H_d sqrt(m)) mod 2 pi, m = |k_A - k_B|^2.
    std::vector<float> ph(28);
    for (int m = 0; m < 28; ++m) ph[m] = (float)std::fmod(p.kappa * Hd * std::sqrt((double)m), 2.0 * M_PI);
    p.L[d].phtab = upload(p, ph);
    p.L[d].host_grid = {ns, nt, np};
    (void)keep;
}

template <class T>
T read_one(Plan& p, const T* d) {
    T h;
    IFGF_CUDA(cudaMemcpyAsync(&h, d, sizeof(T), cudaMemcpyDeviceToHost, p.stream));
    IFGF_CUDA(cudaStreamSynchronize(p.stream));
    return h;
}

__global__ void k_dup_check(const double* __restrict__ Xs, int64_t N, const uint64_t* __restrict__ keys,
                            int* __restrict__ flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    // Coincident points share their level-21 key, and equal keys are contiguous.
    for (int64_t j = i + 1; j < N && keys[j] == keys[i]; ++j)
        if (Xs[i] == Xs[j] && Xs[N + i] == Xs[N + j] && Xs[2 * N + i] == Xs[2 * N + j]) atomicExch(flag, 1);
}

}  // namespace

// Chunks of cones of one gamma (see k_gamma_keys) for a level without node tables. Boxes are
// blocked so that a block of boxes holds about kChunkBoxes cones of each cone index, which
// keeps the chunks full and the child cones of consecutive chunks close together. Chunks that
// would hold fewer than two cones on average are not kept.
void build_gamma_chunks(Plan& p, int dp) {
    Level& Lp = p.L[dp];
    Lp.n_gchunk = 0;
    const int64_t nc = Lp.nc;
    if (nc == 0) return;
    const int C = Lp.g.C;
    const double occ = (double)nc / ((double)Lp.n * (double)C);
    int bb_shift = 4;
    while (bb_shift < 30 && (double)((int64_t)1 << bb_shift) * occ < (double)kChunkBoxes) ++bb_shift;
    const uint64_t maxkey = (uint64_t)(Lp.n >> bb_shift) * (uint64_t)C + (uint64_t)C;
    int end_bit = 1;
    while (end_bit < 64 && (maxkey >> end_bit) != 0) ++end_bit;
    uint64_t* keys = dalloc<uint64_t>(p, (size_t)nc);
    int32_t* order = dalloc<int32_t>(p, (size_t)nc);
    IFGF_LAUNCH(k_gamma_keys, grid_for(nc, kThreads), kThreads, 0, p.stream, nc, Lp.cone_box, Lp.cone_gam, bb_shift,
                C, keys, order);
    radix_sort_pairs(p, keys, order, nc, end_bit);
    int32_t* flags = dalloc<int32_t>(p, (size_t)nc);
    int32_t* pos = dalloc<int32_t>(p, (size_t)nc);
    IFGF_LAUNCH(k_gamma_chunk_flags, grid_for(nc, kThreads), kThreads, 0, p.stream, nc, keys, flags);
    exclusive_scan_i32(p, flags, pos, nc);
    const int64_t nchunk = (int64_t)read_one(p, pos + (nc - 1)) + read_one(p, flags + (nc - 1));
    dfree_ptr(p, keys);
    if ((double)nc < 2.0 * (double)nchunk) {
        dfree_ptr(p, flags);
        dfree_ptr(p, pos);
        dfree_ptr(p, order);
        return;
    }
    int32_t* gchunk = dalloc<int32_t>(p, (size_t)nchunk + 1);
    IFGF_LAUNCH(k_gamma_chunk_fill, grid_for(nc, kThreads), kThreads, 0, p.stream, nc, flags, pos, gchunk);
    dfree_ptr(p, flags);
    dfree_ptr(p, pos);
    Lp.gorder = order;
    Lp.gchunk = gchunk;
    Lp.n_gchunk = nchunk;
}

// Node tables of level dp (for its children at dp+1), when the cone indices are shared by
// enough boxes and the tables stay small; otherwise the kernels compute the geometry.
void build_node_tables(Plan& p, int dp) {
    Level& Lp = p.L[dp];
    Level& L = p.L[dp + 1];
    Lp.n_gam = 0;
    if (Lp.nc == 0 || Lp.g.C > (1 << 27)) return;  // tables pay off only for few distinct gamma
    const int C = Lp.g.C;
    int32_t* flags = dalloc<int32_t>(p, C);
    int32_t* pos = dalloc<int32_t>(p, C);
    IFGF_CUDA(cudaMemsetAsync(flags, 0, sizeof(int32_t) * C, p.stream));
    IFGF_LAUNCH(k_flag_gamma, grid_for(Lp.nc, kThreads), kThreads, 0, p.stream, Lp.cone_gam, Lp.nc, flags);
    exclusive_scan_i32(p, flags, pos, C);
    const int32_t n_gam = read_one(p, pos + (C - 1)) + read_one(p, flags + (C - 1));
    const int64_t entries = (int64_t)n_gam * 8 * p.P;
    const double sharing = (double)Lp.nc / std::max(1, n_gam);
    // bytes: 30 per entry (coordinates, ratio, node, segment), lists and runs per row
    const int64_t bytes = entries * 30 + (int64_t)n_gam * 8 * (2 * kTabList + 3) * 4;
    // Tables of up to 1 GiB pay off from a sharing of 4; a level whose cone indices are each shared
    // by 16 cones or more may take up to 48 GiB (and at most a quarter of the free device memory):
    // on the 512-wavelength sphere the 38 GB tables of level 6 (sharing 128), on the 128-wavelength
    // oblate spheroid the 3.5 GB tables of level 5 (sharing 30), save more time in the propagation
    // and in the marking of relevant cones than they take to build.
    int64_t cap = (int64_t)1 << 30;
    if (sharing >= 16.0) {
        size_t free_b = 0, total_b = 0;
        IFGF_CUDA(cudaMemGetInfo(&free_b, &total_b));
        cap = std::max(cap, std::min((int64_t)48 << 30, (int64_t)((free_b + pool_cached_bytes(p.device)) / 4)));
    }
    if (sharing >= 4.0 && bytes <= cap) {
        Lp.n_gam = n_gam;
        Lp.gam_list = dalloc<int32_t>(p, n_gam);
        Lp.cone_gidx = dalloc<int32_t>(p, Lp.nc);
        Lp.tab_t = dalloc<float4>(p, entries);
        Lp.tab_r = dalloc<float2>(p, entries);
        IFGF_LAUNCH(k_gamma_rows, grid_for(C, kThreads), kThreads, 0, p.stream, flags, pos, C, Lp.gam_list);
        IFGF_LAUNCH(k_cone_rows, grid_for(Lp.nc, kThreads), kThreads, 0, p.stream, Lp.cone_gam, Lp.nc, pos,
                    Lp.cone_gidx);
        IFGF_LAUNCH(k_node_tables, grid_for(entries, kThreads), kThreads, 0, p.stream, entries, Lp.gam_list, p.Ps, p.Pt,
                    p.Pp, p.D - (dp + 1), Lp.g, L.g, (float)(p.kappa * p.u), Lp.tab_t, Lp.tab_r);
        Lp.tab_k = dalloc<int32_t>(p, (size_t)n_gam * 8);
        Lp.tab_list = dalloc<int32_t>(p, (size_t)n_gam * 8 * kTabList);
        Lp.tab_perm = dalloc<int16_t>(p, (size_t)entries);
        Lp.tab_nseg = dalloc<int32_t>(p, (size_t)n_gam * 8);
        Lp.tab_seg = dalloc<int32_t>(p, (size_t)entries);
        Lp.tab_run = dalloc<int32_t>(p, (size_t)n_gam * 8 * (kTabList + 1));
        int* ovf = dalloc<int>(p, 1);
        IFGF_CUDA(cudaMemsetAsync(ovf, 0, sizeof(int), p.stream));
        IFGF_LAUNCH(k_node_lists, (unsigned)(n_gam * 8), 128, 0, p.stream, p.P, Lp.tab_t, Lp.tab_r, Lp.tab_k,
                    Lp.tab_list, Lp.tab_perm, Lp.tab_nseg, Lp.tab_seg, Lp.tab_run, ovf);
        const int overflow = read_one(p, ovf);
        dfree_ptr(p, ovf);
        if (overflow) {  // some row has more distinct child cones than a list holds: no tables
            dfree_ptr(p, Lp.gam_list);
            dfree_ptr(p, Lp.cone_gidx);
            dfree_ptr(p, Lp.tab_t);
            dfree_ptr(p, Lp.tab_r);
            dfree_ptr(p, Lp.tab_k);
            dfree_ptr(p, Lp.tab_list);
            dfree_ptr(p, Lp.tab_perm);
            dfree_ptr(p, Lp.tab_nseg);
            dfree_ptr(p, Lp.tab_seg);
            dfree_ptr(p, Lp.tab_run);
            Lp.n_gam = 0;
        }
    }
    dfree_ptr(p, flags);
    dfree_ptr(p, pos);
}

// ---- validation of the plan's index lists (checked builds) -----------------------------
// Every index array must address its target array: values in [lo, hi), non-decreasing where they
// are offsets, and count-aware for the padded neighbour, cousin and table lists.
__global__ void k_chk_range(const int32_t* __restrict__ a, int64_t n, int64_t lo, int64_t hi, int monotone,
                            int* __restrict__ st) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    in_bounds((int64_t)a[i] - lo, hi - lo, st);
    if (monotone && i > 0 && a[i] < a[i - 1]) atomicCAS(st, 0, (int)IFGF_ERR_INTERNAL);
}
__global__ void k_chk_range16(const int16_t* __restrict__ a, int64_t n, int hi, int* __restrict__ st) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) in_bounds(a[i], hi, st);
}
__global__ void k_chk_lists(const int32_t* __restrict__ cnt, const int32_t* __restrict__ list, int64_t n, int stride,
                            int maxcnt, int64_t hi, int* __restrict__ st) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const int c = cnt[b];
    if (!in_bounds(c, maxcnt + 1, st)) return;
    for (int t = 0; t < c; ++t) in_bounds(list[b * stride + t], hi, st);
}
// child box k of parent j: k_child - 2 k_parent in {0, 1}^3 (the octant used by the node tables)
__global__ void k_chk_octants(const int4* __restrict__ kd, const int32_t* __restrict__ parent, int n,
                              const int4* __restrict__ kp, int np, int* __restrict__ st) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const int j = parent[b];
    if (!in_bounds(j, np, st)) return;
    const int ox = kd[b].x - 2 * kp[j].x, oy = kd[b].y - 2 * kp[j].y, oz = kd[b].z - 2 * kp[j].z;
    in_bounds(ox | oy | oz, 2, st);
}
// segments of the node tables: first entry + length within the row, list position within its list
__global__ void k_chk_segments(const int32_t* __restrict__ nseg, const int32_t* __restrict__ seg,
                               const int32_t* __restrict__ tab_k, int64_t rows, int P, int* __restrict__ st) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const int ns = nseg[r];
    if (!in_bounds(ns, P + 1, st)) return;
    for (int t = 0; t < ns; ++t) {
        const int sg = seg[r * P + t];
        const int j0 = sg & 0xff, len = (sg >> 8) & 0xff, kl = sg >> 16;
        in_bounds(j0 + len - 1, P, st);
        in_bounds(kl, min(tab_k[r], kTabList), st);
    }
}

void validate_plan(Plan& p) {
    cudaStream_t s = p.stream;
    int* st = p.d_status;
    const int64_t N = p.N;
    auto range = [&](const int32_t* a, int64_t n, int64_t lo, int64_t hi, bool mono) {
        if (a && n > 0) IFGF_LAUNCH(k_chk_range, grid_for(n, kThreads), kThreads, 0, s, a, n, lo, hi, mono ? 1 : 0, st);
    };
    range(p.perm, N, 0, N, false);
    for (int d = 1; d <= p.D; ++d) {
        Level& L = p.L[d];
        range(L.start, (int64_t)L.n + 1, 0, N + 1, true);
        range(L.pbox, N, 0, L.n, true);
        if (d > 1) {
            range(L.parent, L.n, 0, p.L[d - 1].n, true);
            IFGF_LAUNCH(k_chk_octants, grid_for(L.n, kThreads), kThreads, 0, s, L.k, L.parent, L.n, p.L[d - 1].k,
                        p.L[d - 1].n, st);
        }
        if (d < p.D) range(L.cstart, (int64_t)L.n + 1, 0, (int64_t)p.L[d + 1].n + 1, true);
        if (L.nnb) IFGF_LAUNCH(k_chk_lists, grid_for(L.n, kThreads), kThreads, 0, s, L.nnb, L.nb, L.n, kMaxNbr, kMaxNbr, L.n, st);
        if (L.ncs) IFGF_LAUNCH(k_chk_lists, grid_for(L.n, kThreads), kThreads, 0, s, L.ncs, L.cs, L.n, kMaxCous, kMaxCous, L.n, st);
        if (d < 3) continue;
        range(L.cone_box, L.nc, 0, L.n, true);
        range(L.cone_gam, L.nc, 0, L.g.C, false);
        range(L.slot, L.slot ? (int64_t)L.n * L.g.C : 0, -1, L.nc, false);
        range(L.bcs, L.bcs ? (int64_t)L.n + 1 : 0, 0, L.nc + 1, true);
        range(L.rows, L.rows ? (int64_t)L.n * L.g.ns * L.g.nt + 1 : 0, 0, L.nc + 1, true);
        range(L.gorder, L.gorder ? L.nc : 0, 0, L.nc, false);
        range(L.gchunk, L.gchunk ? L.n_gchunk + 1 : 0, 0, L.nc + 1, true);
        if (L.n_gam > 0 && d < p.D) {
            const int64_t rows = (int64_t)L.n_gam * 8;
            range(L.cone_gidx, L.nc, 0, L.n_gam, false);
            range(L.gam_list, L.n_gam, 0, L.g.C, true);
            range(L.tab_k, rows, 0, kTabList + 1, false);
            range(L.tab_nseg, rows, 0, p.P + 1, false);
            IFGF_LAUNCH(k_chk_lists, grid_for(rows, kThreads), kThreads, 0, s, L.tab_k, L.tab_list, rows, kTabList,
                        kTabList, p.L[d + 1].g.C, st);
            IFGF_LAUNCH(k_chk_segments, grid_for(rows, kThreads), kThreads, 0, s, L.tab_nseg, L.tab_seg, L.tab_k, rows,
                        p.P, st);
            IFGF_LAUNCH(k_chk_range16, grid_for(rows * p.P, kThreads), kThreads, 0, s, L.tab_perm, rows * p.P, p.P, st);
        }
    }
    int h = 0;
    IFGF_CUDA(cudaMemcpyAsync(&h, st, sizeof(int), cudaMemcpyDeviceToHost, s));
    IFGF_CUDA(cudaStreamSynchronize(s));
    if (h != 0) fail(IFGF_ERR_INTERNAL, "plan validation found an index outside its array");
}

void build_plan(Plan& p, const double* X, const ifgf_options& opt, int levels) {
    const int64_t N = p.N;
    cudaStream_t s = p.stream;

    // Root cube.
    const int nb = (int)std::min<int64_t>(1024, (N + kThreads - 1) / kThreads);
    double* part = dalloc<double>(p, (size_t)nb * 7);
    IFGF_LAUNCH(k_bbox_partial, nb, kThreads, 0, s, X, N, part);
    std::vector<double> hp((size_t)nb * 7);
    IFGF_CUDA(cudaMemcpyAsync(hp.data(), part, sizeof(double) * nb * 7, cudaMemcpyDeviceToHost, s));
    IFGF_CUDA(cudaStreamSynchronize(s));
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = 0; b < nb; ++b) {
        if (hp[b * 7 + 6] != 0.0) fail(IFGF_ERR_INVALID_ARG, "non-finite coordinate");
        for (int c = 0; c < 3; ++c) {
            mn[c] = std::min(mn[c], hp[b * 7 + c]);
            mx[c] = std::max(mx[c], hp[b * 7 + 3 + c]);
        }
    }
    double ext = 0.0;
    for (int c = 0; c < 3; ++c) ext = std::max(ext, mx[c] - mn[c]);
    if (!(ext > 0.0)) fail(IFGF_ERR_INVALID_ARG, "all points coincide");
    p.H1 = ext * (1.0 + std::ldexp(1.0, -20));
    for (int c = 0; c < 3; ++c) p.a[c] = 0.5 * (mn[c] + mx[c]) - 0.5 * p.H1;

    // Morton keys and the sorted order (ties by the caller's index: the sort is stable).
    p.key = dalloc<uint64_t>(p, N);
    p.perm = dalloc<int32_t>(p, N);
    IFGF_LAUNCH(k_keys, grid_for(N, kThreads), kThreads, 0, s, X, N, p.a[0], p.a[1], p.a[2], p.H1, p.key, p.perm);
    radix_sort_pairs(p, p.key, p.perm, N, 3 * (kKeyLevel - 1));
    p.Xs = dalloc<double>(p, 3 * (size_t)N);
    IFGF_LAUNCH(k_gather_points, grid_for(N, kThreads), kThreads, 0, s, X, N, p.perm, p.Xs);

    // Boxes per level.
    uint8_t* d0 = dalloc<uint8_t>(p, N);
    unsigned long long* hist = dalloc<unsigned long long>(p, 24);
    IFGF_CUDA(cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * 24, s));
    IFGF_LAUNCH(k_level_split, grid_for(N, kThreads), kThreads, 0, s, p.key, N, d0, hist);
    unsigned long long hh[24];
    IFGF_CUDA(cudaMemcpyAsync(hh, hist, sizeof(hh), cudaMemcpyDeviceToHost, s));
    int* dflag = dalloc<int>(p, 1);
    IFGF_CUDA(cudaMemsetAsync(dflag, 0, sizeof(int), s));
    IFGF_LAUNCH(k_dup_check, grid_for(N, kThreads), kThreads, 0, s, p.Xs, N, p.key, dflag);
    int dup = 0;
    IFGF_CUDA(cudaMemcpyAsync(&dup, dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    IFGF_CUDA(cudaStreamSynchronize(s));
    if (dup) fail(IFGF_ERR_INVALID_ARG, "two points share all three coordinates");
    int64_t nd[kMaxLevel + 2];
    {
        int64_t acc = 1;
        for (int d = 1; d <= kMaxLevel; ++d) {
            acc += (int64_t)hh[d];
            nd[d] = acc;
        }
    }
    int D = levels;
    if (D == 0) {
        D = kMaxLevel;
        for (int d = 3; d <= kMaxLevel; ++d)
            if (N <= (int64_t)opt.leaf_target * nd[d]) {
                D = d;
                break;
            }
    }
    p.D = D;
    p.u = std::ldexp(p.H1, -D);

    int32_t* flag = dalloc<int32_t>(p, N);
    int32_t* pos = dalloc<int32_t>(p, N);
    for (int d = 1; d <= D; ++d) p.L[d].n = (int32_t)nd[d];
    for (int d = 1; d <= D; ++d) {
        Level& L = p.L[d];
        L.start = dalloc<int32_t>(p, (size_t)L.n + 1);
        L.key = dalloc<uint64_t>(p, L.n);
        L.k = dalloc<int4>(p, L.n);
        L.pbox = dalloc<int32_t>(p, N);
        IFGF_LAUNCH(k_level_flags, grid_for(N, kThreads), kThreads, 0, s, d0, N, d, flag);
        exclusive_scan_i32(p, flag, pos, N);
        IFGF_LAUNCH(k_level_boxes, grid_for(N, kThreads), kThreads, 0, s, flag, pos, p.key, N, d, L.n, L.start, L.key,
                    L.k, L.pbox);
    }
    dfree_ptr(p, flag);
    dfree_ptr(p, pos);
    dfree_ptr(p, d0);
    dfree_ptr(p, hist);
    dfree_ptr(p, dflag);
    dfree_ptr(p, part);
    for (int d = 1; d <= D; ++d) {
        Level& L = p.L[d];
        L.parent = dalloc<int32_t>(p, L.n);
        IFGF_LAUNCH(k_parents, grid_for(L.n, kThreads), kThreads, 0, s, L.start, L.n, d > 1 ? p.L[d - 1].pbox : nullptr,
                    L.parent);
    }
    for (int d = 1; d <= D; ++d) {
        Level& L = p.L[d];
        L.cstart = dalloc<int32_t>(p, (size_t)L.n + 1);
        if (d < D)
            IFGF_LAUNCH(k_child_start, grid_for(p.L[d + 1].n, kThreads), kThreads, 0, s, p.L[d + 1].parent,
                        p.L[d + 1].n, L.n, L.cstart);
        else
            IFGF_CUDA(cudaMemsetAsync(L.cstart, 0, sizeof(int32_t) * ((size_t)L.n + 1), s));
    }
    p.off = dalloc<float4>(p, N);
    IFGF_LAUNCH(k_offsets, grid_for(N, kThreads), kThreads, 0, s, p.Xs, N, p.a[0], p.a[1], p.a[2], p.H1,
                std::ldexp(1.0, D), p.L[D].pbox, p.L[D].k, p.off);

    // Neighbours (levels 2..D) and cousins (levels 3..D).
    for (int d = 2; d <= D; ++d) {
        Level& L = p.L[d];
        L.nnb = dalloc<int32_t>(p, L.n);
        L.nb = dalloc<int32_t>(p, (size_t)L.n * kMaxNbr);
        IFGF_LAUNCH(k_neighbours, grid_for(L.n, kThreads), kThreads, 0, s, L.key, L.k, L.n, d, L.nnb, L.nb);
    }
    for (int d = 3; d <= D; ++d) {
        Level& L = p.L[d];
        Level& Lp = p.L[d - 1];
        L.ncs = dalloc<int32_t>(p, L.n);
        L.cs = dalloc<int32_t>(p, (size_t)L.n * kMaxCous);
        IFGF_LAUNCH(k_cousins, grid_for(L.n, kThreads), kThreads, 0, s, L.k, L.parent, L.n, Lp.nnb, Lp.nb, Lp.cstart,
                    L.ncs, L.cs);
    }

    // Cone grids and the relevant cones, top-down d = 3..D (level d needs level d-1).
    std::vector<std::vector<char>> keep;
    for (int d = 3; d <= D; ++d) build_grid(p, d, opt, keep);
    for (int d = 3; d <= D; ++d) {
        Level& L = p.L[d];
        const int64_t total = (int64_t)L.n * L.g.C;
        const bool dense = opt.cone_table == 1 || (opt.cone_table == 0 && total < ((int64_t)1 << 31));
        if (dense && total >= ((int64_t)1 << 31)) fail(IFGF_ERR_UNSUPPORTED, "dense cone table exceeds 2^31 entries");
        // one activation pass (both sources of Eq. (4)) into the given recorder
        auto activate = [&](const ConeMark& cm) {
            IFGF_LAUNCH(k_mark_cousin_points, grid_for(N, kThreads), kThreads, 0, s, N, D, d, L.pbox, p.L[D].pbox,
                        p.L[D].k, L.k, L.ncs, L.cs, p.off, L.g, cm);
            if (d > 3) {
                Level& Lp = p.L[d - 1];
                if (Lp.nc > 0 && Lp.n_gam > 0)
                    IFGF_LAUNCH(k_mark_parent_nodes_tab, grid_for(Lp.nc * 8, kThreads), kThreads, 0, s, Lp.nc,
                                Lp.cone_box, Lp.cone_gidx, Lp.k, Lp.cstart, L.k, Lp.tab_k, Lp.tab_list, cm);
                else if (Lp.nc > 0 && Lp.n_gchunk > 0)
                    IFGF_LAUNCH(k_mark_parent_nodes_chunk, (unsigned)((Lp.n_gchunk + kMarkWarps - 1) / kMarkWarps),
                                32 * kMarkWarps, 0, s, Lp.gchunk, (int64_t)Lp.n_gchunk, Lp.gorder, Lp.cone_box, Lp.cone_gam, Lp.k, Lp.cstart, L.k, D, d, Lp.g, L.g, cm);
                else if (Lp.nc > 0)
                    IFGF_LAUNCH(k_mark_parent_nodes, grid_for(Lp.nc * p.P, kThreads), kThreads, 0, s, Lp.nc, p.P, p.Ps,
                                p.Pt, p.Pp, D, d, Lp.cone_box, Lp.cone_gam, Lp.k, Lp.cstart, L.k, Lp.g, L.g, cm);
            }
        };
        if (dense) {
            L.slot = dalloc<int32_t>(p, total);
            IFGF_CUDA(cudaMemsetAsync(L.slot, 0, sizeof(int32_t) * total, s));
            activate(ConeMark{L.slot, nullptr, 0, L.g.C, nullptr});
            int32_t* cpos = dalloc<int32_t>(p, total);
            exclusive_scan_i32(p, L.slot, cpos, total);
            const int32_t last_pos = read_one(p, cpos + (total - 1));
            const int32_t last_flag = read_one(p, L.slot + (total - 1));
            L.nc = (int64_t)last_pos + last_flag;
            L.cone_box = dalloc<int32_t>(p, L.nc);
            L.cone_gam = dalloc<int32_t>(p, L.nc);
            IFGF_LAUNCH(k_finalize_cones, grid_for(total, kThreads), kThreads, 0, s, L.slot, cpos, total, L.g.C,
                        L.cone_box, L.cone_gam);
            dfree_ptr(p, cpos);
            L.bcs = dalloc<int32_t>(p, (size_t)L.n + 1);
            IFGF_LAUNCH(k_box_cone_starts, grid_for((int64_t)L.n + 1, kThreads), kThreads, 0, s, L.n, L.nc, L.cone_box,
                        L.bcs);
        } else {
            // hash set of (box, gamma) keys, grown until every insertion finds room
            const int64_t guess = std::max<int64_t>({(int64_t)1 << 20, N / 2, d > 3 ? p.L[d - 1].nc : 0});
            int64_t H = (int64_t)1 << 20;
            while (H < 4 * guess && H < ((int64_t)1 << 31)) H <<= 1;
            unsigned long long* hk = nullptr;
            int* ovf = dalloc<int>(p, 1);
            for (;;) {
                hk = dalloc<unsigned long long>(p, (size_t)H);
                IFGF_CUDA(cudaMemsetAsync(hk, 0xff, sizeof(unsigned long long) * H, s));
                IFGF_CUDA(cudaMemsetAsync(ovf, 0, sizeof(int), s));
                activate(ConeMark{nullptr, hk, (unsigned long long)(H - 1), L.g.C, ovf});
                if (!read_one(p, ovf)) break;
                dfree_ptr(p, hk);
                if (H >= ((int64_t)1 << 31)) fail(IFGF_ERR_OOM, "cone hash set cannot grow further");
                H <<= 1;
            }
            dfree_ptr(p, ovf);
            int32_t* flags = dalloc<int32_t>(p, (size_t)H);
            int32_t* pos = dalloc<int32_t>(p, (size_t)H);
            IFGF_LAUNCH(k_hash_flags, grid_for(H, kThreads), kThreads, 0, s, H, hk, flags);
            exclusive_scan_i32(p, flags, pos, H);
            L.nc = (int64_t)read_one(p, pos + (H - 1)) + read_one(p, flags + (H - 1));
            uint64_t* keys = dalloc<uint64_t>(p, (size_t)std::max<int64_t>(L.nc, 1));
            int32_t* vals = dalloc<int32_t>(p, (size_t)std::max<int64_t>(L.nc, 1));
            IFGF_LAUNCH(k_hash_gather, grid_for(H, kThreads), kThreads, 0, s, H, hk, flags, pos, keys, vals);
            dfree_ptr(p, hk);
            dfree_ptr(p, flags);
            dfree_ptr(p, pos);
            const uint64_t maxkey = (uint64_t)L.n * (uint64_t)L.g.C;
            int end_bit = 1;
            while (end_bit < 64 && (maxkey >> end_bit) != 0) ++end_bit;
            radix_sort_pairs(p, keys, vals, L.nc, end_bit);
            L.cone_box = dalloc<int32_t>(p, std::max<int64_t>(L.nc, 1));
            L.cone_gam = dalloc<int32_t>(p, std::max<int64_t>(L.nc, 1));
            IFGF_LAUNCH(k_split_keys, grid_for(L.nc, kThreads), kThreads, 0, s, L.nc, keys, (int64_t)L.g.C, L.cone_box,
                        L.cone_gam);
            dfree_ptr(p, keys);
            dfree_ptr(p, vals);
            L.bcs = dalloc<int32_t>(p, (size_t)L.n + 1);
            IFGF_LAUNCH(k_box_cone_starts, grid_for((int64_t)L.n + 1, kThreads), kThreads, 0, s, L.n, L.nc, L.cone_box,
                        L.bcs);
            // row index of the sorted list while it stays within a memory budget (4 bytes per row)
            const int64_t nrow = (int64_t)L.g.ns * L.g.nt;
            const int64_t rtotal = (int64_t)L.n * nrow;
            if (rtotal < ((int64_t)1 << 31) && rtotal * 4 <= ((int64_t)1 << 30)) {
                L.rows = dalloc<int32_t>(p, (size_t)rtotal + 1);
                IFGF_LAUNCH(k_row_starts, grid_for(rtotal + 1, kThreads), kThreads, 0, s, rtotal, (int)nrow, L.g.np,
                            L.bcs, L.cone_gam, L.rows);
            }
        }
        if (d < D && p.precision == IFGF_PREC_MIXED && p.Ps == 3 && p.Pt == 5 && p.Pp == 5) {
            build_node_tables(p, d);
            if (L.n_gam == 0) build_gamma_chunks(p, d);
        }
    }
    if constexpr (kChecks) validate_plan(p);
}

namespace {
// Child cones read by the parent-cone slice [lo, hi): [c_lo, c_hi).
__global__ void k_slice_children(int ns, const int64_t* __restrict__ b, const int32_t* __restrict__ pcone_box,
                                 const int32_t* __restrict__ pcstart, const int32_t* __restrict__ bcs,
                                 int64_t* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    const int64_t lo = b[i], hi = b[i + 1];
    out[2 * i] = bcs[pcstart[pcone_box[lo]]];
    out[2 * i + 1] = bcs[pcstart[pcone_box[hi - 1] + 1]];
}
}  // namespace

// Arena cones needed when every propagation runs in k slices of equal parent-cone counts (the
// slice boundaries are stored in the parent levels). With the child level at the start of the
// arena, the parents go to its end, slices in descending order: slice [lo, hi) writes from
// M - n_p + lo on while the children it and the later slices read lie below c_hi, so
// M >= n_p - lo + c_hi. With the children at the end, ascending slices: M >= n_c + hi - c_lo.
static int64_t arena_for_slices(Plan& p, int k) {
    int64_t M = 0;
    for (int d = 3; d <= p.D; ++d) M = std::max<int64_t>(M, p.L[d].nc);
    for (int d = p.D; d >= 4; --d) {
        Level& Lc = p.L[d];
        Level& Lp = p.L[d - 1];
        std::vector<int64_t> b;
        const int ks = (int)std::max<int64_t>(1, std::min<int64_t>(k, Lp.nc));
        for (int i = 0; i <= ks; ++i) b.push_back(Lp.nc * i / ks);
        Lp.pslice = b;
        if (Lp.nc == 0) continue;
        int64_t* db = dalloc<int64_t>(p, b.size());
        int64_t* dout = dalloc<int64_t>(p, 2 * (size_t)ks);
        IFGF_CUDA(cudaMemcpyAsync(db, b.data(), sizeof(int64_t) * b.size(), cudaMemcpyHostToDevice, p.stream));
        IFGF_LAUNCH(k_slice_children, grid_for(ks, 128), 128, 0, p.stream, ks, db, Lp.cone_box, Lp.cstart, Lc.bcs,
                    dout);
        std::vector<int64_t> c(2 * (size_t)ks);
        IFGF_CUDA(cudaMemcpyAsync(c.data(), dout, sizeof(int64_t) * c.size(), cudaMemcpyDeviceToHost, p.stream));
        IFGF_CUDA(cudaStreamSynchronize(p.stream));
        dfree_ptr(p, db);
        dfree_ptr(p, dout);
        const bool child_at_start = (p.D - d) % 2 == 0;
        for (int i = 0; i < ks; ++i) {
            const int64_t need = child_at_start ? Lp.nc - b[i] + c[2 * i + 1] : Lc.nc + b[i + 1] - c[2 * i];
            M = std::max(M, need);
        }
    }
    return std::max<int64_t>(M, 1);
}

int64_t layout_arena(Plan& p, size_t budget_per_rhs, int slices) {
    const size_t cone = (size_t)p.cstride * (p.precision == IFGF_PREC_MIXED ? 8 : 16);
    if (slices > 0) {
        const int64_t Mk = arena_for_slices(p, slices);
        return (size_t)Mk * cone <= budget_per_rhs ? Mk : 0;
    }
    int64_t M = arena_for_slices(p, 1);  // one launch per level: two full levels
    if ((size_t)M * cone <= budget_per_rhs) return M;
    M = arena_for_slices(p, 64);
    return (size_t)M * cone <= budget_per_rhs ? M : 0;
}

}  // namespace ifgf
