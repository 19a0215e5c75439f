// Propagation with many densities on the fifth-generation tensor cores (tcgen05, TMEM
// accumulators), levels with node tables, orders (3,5,5), mixed precision.
//
// For a parent cone (j, gamma) and a child box B_k, the nodes of the parent cone that fall in one
// child cone alpha form one contiguous run of the node-table row (gamma, octant of B_k).  For the
// NR densities r of a block, the values of Algorithm 7 at those nodes are the product
//     V[node][r] = sum_k W[node][k] C_alpha,r[k],   W[node][k] = T_a(t_s) T_b(t_theta) T_c(t_phi),
// with k = (a, b, c) the coefficient index (75, padded to K = 80).  One block takes one parent
// cone: for every (child, alpha) group it writes W (the group's nodes as rows, M = 128) and the
// coefficients of alpha (one row per density and real/imaginary part, N = 2 NR) to shared memory,
// one thread issues the products as tcgen05.mma kind::tf32 into a TMEM accumulator, in 3xTF32
// (x = hi + lo, products hi hi + hi lo + lo hi, FP32 accumulation), and every thread then reads its
// node's row of the accumulator, multiplies by the node's propagation ratio and adds it to the node
// values.  The groups of all children are added in a fixed order (no float atomics), and the
// parent interpolants are generated as in the other propagation kernels.
//
// Shared-memory operands use the canonical layout without swizzling: 8-row x 16-byte core
// matrices, core (row block, k block) at byte ((row / 8) * 20 + k / 4) * 128; the descriptors give
// the byte distance between core matrices along K (128) and between 8-row blocks (2560).  A group
// has at most 75 nodes, so the weight tiles hold 80 rows; the products read 128, and rows 80..127
// of a tile fall on the next buffer of the same shared-memory block (their accumulator rows are
// never read).
#include <cstdint>

#include "ifgf_internal.cuh"

namespace ifgf {
namespace {

constexpr int kTcThreads = 128;  // four warps: the 128 TMEM lanes of the accumulator
constexpr int kTcK = 80;         // 75 coefficients padded to a multiple of 8
constexpr int kTcKB = kTcK / 4;  // 16-byte k blocks per row
constexpr int kTcARows = 80;              // weight rows stored per tile (a group has <= 75 nodes)
constexpr int kTcATile = kTcARows * kTcK * 4;  // bytes of one weight tile
constexpr int kTcWaitLimit = 1 << 24;     // polls of an mbarrier before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row, k) in a K-major operand tile
__device__ __forceinline__ int tile_off(int row, int k) {
    return ((row >> 3) * kTcKB + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

// Shared-memory matrix descriptor: start address, byte distance between core matrices along K
// (leading) and between 8-row blocks (stride), descriptor version 1, no swizzling.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lead, uint32_t stride) {
    return (uint64_t)((addr >> 4) & 0x3fff) | ((uint64_t)((lead >> 4) & 0x3fff) << 16) |
           ((uint64_t)((stride >> 4) & 0x3fff) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major, N, M = 128.
__host__ __device__ constexpr uint32_t tf32_idesc(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Wait for phase `parity` of an mbarrier, at most kTcWaitLimit polls; false if it never completed.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (int it = 0; it < kTcWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 32 consecutive accumulator columns of this warp's 32 TMEM lanes (lane = row of the thread).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// x = hi + lo for 3xTF32: hi keeps the 10 leading mantissa bits (exactly representable in TF32)
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
    hi = __uint_as_float(__float_as_uint(x) & 0xffffe000u);
    lo = x - hi;
}

template <int NR>
__global__ void __launch_bounds__(kTcThreads)
k_prop_tc_tab(int64_t ncp, const int32_t* __restrict__ pcone_box, const int32_t* __restrict__ cone_gidx,
              const int4* __restrict__ kp, const int32_t* __restrict__ pcstart, const int4* __restrict__ kd, ConeMap cm,
              const float4* __restrict__ tab_t, const float2* __restrict__ tab_r, const int32_t* __restrict__ tab_k,
              const int32_t* __restrict__ tab_list, const int16_t* __restrict__ tab_perm,
              const int32_t* __restrict__ tab_seg, const int32_t* __restrict__ tab_run,
              const float2* __restrict__ cchild, float2* __restrict__ cparent, const float* __restrict__ W, int cstride,
              int nrhs, int* __restrict__ status) {
    constexpr int PS = 3, PT = 5, PP = 5, P = 75, N = 2 * NR;
    constexpr int kBTile = N * kTcK * 4;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* a_hi = smem;
    unsigned char* a_lo = a_hi + kTcATile;
    unsigned char* b_hi = a_lo + kTcATile;
    unsigned char* b_lo = b_hi + kBTile;
    float2* f = reinterpret_cast<float2*>(b_lo + kBTile);  // [NR][P] node values
    float* wst = reinterpret_cast<float*>(f + NR * P);     // [P][20]: T_a T_b (15) and T_c (5) of a node
    uint64_t* bar = reinterpret_cast<uint64_t*>(wst + P * 20);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t pc = blockIdx.x;
    const int rhs0 = blockIdx.y * NR;

    // zero the padded coefficients k = 75..79 of every operand row (never written afterwards)
    for (int x = tid; x < kTcARows * 5; x += kTcThreads) {
        const int row = x / 5, k = P + x % 5;
        *reinterpret_cast<float*>(a_hi + tile_off(row, k)) = 0.f;
        *reinterpret_cast<float*>(a_lo + tile_off(row, k)) = 0.f;
        if (row < N) {
            *reinterpret_cast<float*>(b_hi + tile_off(row, k)) = 0.f;
            *reinterpret_cast<float*>(b_lo + tile_off(row, k)) = 0.f;
        }
    }
    for (int x = tid; x < NR * P; x += kTcThreads) f[x] = make_float2(0.f, 0.f);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"((uint32_t)(N < 32 ? 32 : N))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t ubar = smem_u32(bar);
    uint32_t parity = 0;
    bool ok = true;

    const int jb = pcone_box[pc];
    const int g8 = cone_gidx[pc] * 8;
    const int4 kj = kp[jb];
    for (int kb = pcstart[jb]; kb < pcstart[jb + 1] && ok; ++kb) {
        const int4 kk = kd[kb];
        const int row = g8 + ((kk.x - 2 * kj.x) | ((kk.y - 2 * kj.y) << 1) | ((kk.z - 2 * kj.z) << 2));
        const int64_t rowP = (int64_t)row * P;
        const int K = min(__ldg(&tab_k[row]), kTabList);
        for (int kl = 0; kl < K && ok; ++kl) {
            // the group: entries [e0, e1) of the row (nodes of child cone kl)
            const int sg0 = __ldg(&tab_run[(int64_t)row * (kTabList + 1) + kl]);
            const int sg1 = __ldg(&tab_run[(int64_t)row * (kTabList + 1) + kl + 1]);
            if (sg1 <= sg0) continue;
            const int s0 = __ldg(&tab_seg[rowP + sg0]), s1 = __ldg(&tab_seg[rowP + sg1 - 1]);
            const int e0 = s0 & 0xff, e1 = (s1 & 0xff) + ((s1 >> 8) & 0xff), ns = e1 - e0;
            const int sl = cm.find(kb, __ldg(&tab_list[(int64_t)row * kTabList + kl]));
            if (sl < 0) {
                if (tid == 0) set_status(status, IFGF_ERR_INTERNAL);
                continue;
            }
            // basis values of the group's nodes
            if (tid < ns) {
                const float4 t4 = __ldg(&tab_t[rowP + e0 + tid]);
                float Ts[PS], Tt[PT], Tp[PP];
                cheb_T<PS>(t4.x, Ts);
                cheb_T<PT>(t4.y, Tt);
                cheb_T<PP>(t4.z, Tp);
                float* w = wst + tid * 20;
#pragma unroll
                for (int a = 0; a < PS; ++a)
#pragma unroll
                    for (int b = 0; b < PT; ++b) w[a * PT + b] = Ts[a] * Tt[b];
#pragma unroll
                for (int c = 0; c < PP; ++c) w[15 + c] = Tp[c];
            }
            __syncthreads();
            // A: W[node][k] for the group's nodes, four k per item (k < 75)
            for (int x = tid; x < ns * 19; x += kTcThreads) {
                const int r = x / 19, kq = x - r * 19;
                const float* w = wst + r * 20;
                float hi[4], lo[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int k = 4 * kq + i;
                    const float v = k < P ? w[k / 5] * w[15 + k % 5] : 0.f;
                    split_tf32(v, hi[i], lo[i]);
                }
                *reinterpret_cast<float4*>(a_hi + tile_off(r, 4 * kq)) = make_float4(hi[0], hi[1], hi[2], hi[3]);
                *reinterpret_cast<float4*>(a_lo + tile_off(r, 4 * kq)) = make_float4(lo[0], lo[1], lo[2], lo[3]);
            }
            // B: the coefficients of alpha, row 2 d + part = part of density rhs0 + d (zero past nrhs)
            for (int x = tid; x < N * 19; x += kTcThreads) {
                const int j = x / 19, kq = x - j * 19;
                const int d = rhs0 + (j >> 1);
                float hi[4], lo[4];
                const float2* c = cchild + ((int64_t)sl * nrhs + (d < nrhs ? d : 0)) * cstride;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int k = 4 * kq + i;
                    float v = 0.f;
                    if (k < P && d < nrhs) {
                        const float2 cv = __ldg(c + k);
                        v = (j & 1) ? cv.y : cv.x;
                    }
                    split_tf32(v, hi[i], lo[i]);
                }
                *reinterpret_cast<float4*>(b_hi + tile_off(j, 4 * kq)) = make_float4(hi[0], hi[1], hi[2], hi[3]);
                *reinterpret_cast<float4*>(b_lo + tile_off(j, 4 * kq)) = make_float4(lo[0], lo[1], lo[2], lo[3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // operands visible to the tensor core
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                constexpr uint32_t idesc = tf32_idesc(N);
                constexpr uint32_t lead = 128, stride = kTcKB * 128;
                const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo), bh = smem_u32(b_hi), bl = smem_u32(b_lo);
#pragma unroll 1
                for (int ks = 0; ks < kTcK / 8; ++ks) {  // 8 tf32 = two k blocks per instruction
                    const uint32_t o = ks * 256;
                    tc_mma(tmem, smem_desc(ah + o, lead, stride), smem_desc(bh + o, lead, stride), idesc, ks > 0);
                    tc_mma(tmem, smem_desc(ah + o, lead, stride), smem_desc(bl + o, lead, stride), idesc, 1);
                    tc_mma(tmem, smem_desc(al + o, lead, stride), smem_desc(bh + o, lead, stride), idesc, 1);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(ubar)
                             : "memory");
            }
            ok = __syncthreads_and(mbar_wait(ubar, parity)) != 0;  // one decision for the whole block
            if (!ok && tid == 0) set_status(status, IFGF_ERR_TIMEOUT);
            parity ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (ok) {
                // epilogue: row r of the accumulator is node r of the group
                const int r = warp * 32 + lane;
#pragma unroll
                for (int c0 = 0; c0 < N; c0 += 32) {
                    float v[32];
                    tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
                    if (r < ns) {
                        const int n = __ldg(&tab_perm[rowP + e0 + r]);
                        const float2 ratio = __ldg(&tab_r[rowP + e0 + r]);
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const int d = c0 / 2 + q;
                            if (d < NR) {
                                const float2 t = cmul(make_float2(v[2 * q], v[2 * q + 1]), ratio);
                                float2& acc = f[d * P + n];
                                acc = make_float2(acc.x + t.x, acc.y + t.y);
                            }
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();  // the next group overwrites the operands and the accumulator
        }
    }
    // Chebyshev coefficients of every density's node values (phi, theta, s passes; A tile as scratch)
    const float* Ws = W;
    const float* Wt = W + PS * PS;
    const float* Wp = Wt + PT * PT;
    float2* tmp = reinterpret_cast<float2*>(a_hi);
    for (int x = tid; x < NR * P; x += kTcThreads) {
        const int rl = x / P, n = x - (x / P) * P;
        const int qc = n % PP, qb = (n / PP) % PT, qa = n / (PP * PT);
        float2 a = make_float2(0.f, 0.f);
        const float2* rw = &f[rl * P + (qa * PT + qb) * PP];
#pragma unroll
        for (int k = 0; k < PP; ++k) {
            const float w = Wp[qc * PP + k];
            a.x = fmaf(w, rw[k].x, a.x);
            a.y = fmaf(w, rw[k].y, a.y);
        }
        tmp[x] = a;
    }
    __syncthreads();
    for (int x = tid; x < NR * P; x += kTcThreads) {
        const int rl = x / P, n = x - (x / P) * P;
        const int qc = n % PP, qb = (n / PP) % PT, qa = n / (PP * PT);
        float2 a = make_float2(0.f, 0.f);
#pragma unroll
        for (int jj = 0; jj < PT; ++jj) {
            const float w = Wt[qb * PT + jj];
            const float2 v = tmp[rl * P + (qa * PT + jj) * PP + qc];
            a.x = fmaf(w, v.x, a.x);
            a.y = fmaf(w, v.y, a.y);
        }
        f[x] = a;
    }
    __syncthreads();
    for (int x = tid; x < NR * P; x += kTcThreads) {
        const int rl = x / P, n = x - (x / P) * P;
        if (rhs0 + rl >= nrhs) continue;
        const int qc = n % PP, qb = (n / PP) % PT, qa = n / (PP * PT);
        float2 a = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < PS; ++i) {
            const float w = Ws[qa * PS + i];
            const float2 v = f[rl * P + (i * PT + qb) * PP + qc];
            a.x = fmaf(w, v.x, a.x);
            a.y = fmaf(w, v.y, a.y);
        }
        cparent[(pc * nrhs + rhs0 + rl) * cstride + n] = a;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((uint32_t)(N < 32 ? 32 : N))
                     : "memory");
}

template <int NR>
size_t tc_smem_bytes() {
    const size_t bytes = (size_t)2 * kTcATile + (size_t)2 * (2 * NR) * kTcK * 4 + (size_t)NR * 75 * sizeof(float2) +
                         (size_t)75 * 20 * sizeof(float) + 16;
    // the products read 128 rows of the second weight tile: they must lie inside the block
    return bytes > (size_t)kTcATile + 128 * kTcK * 4 ? bytes : (size_t)kTcATile + 128 * kTcK * 4;
}

template <int NR>
void launch_tc(const Plan& p, int d, int nrhs, int64_t lo, int64_t n, const float2* cc, float2* cp, cudaStream_t s) {
    const Level& L = p.L[d];
    const Level& Lp = p.L[d - 1];
    const size_t smem = tc_smem_bytes<NR>();
    static bool attr_set = false;  // per process: the kernel's shared-memory limit
    if (!attr_set) {
        IFGF_CUDA(cudaFuncSetAttribute(k_prop_tc_tab<NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_set = true;
    }
    const unsigned rb = (unsigned)((nrhs + NR - 1) / NR);
    IFGF_LAUNCH(k_prop_tc_tab<NR>, dim3((unsigned)n, rb), kTcThreads, smem, s, n, Lp.cone_box + lo, Lp.cone_gidx + lo,
                Lp.k, Lp.cstart, L.k, L.cmap(p.d_status), Lp.tab_t, Lp.tab_r, Lp.tab_k, Lp.tab_list, Lp.tab_perm,
                Lp.tab_seg, Lp.tab_run, cc, cp, p.Wf, p.cstride, nrhs, p.d_status);
}

}  // namespace

void launch_prop_tc_tab(const Plan& p, int d, int nrhs, int64_t lo, int64_t n, const float2* cc, float2* cp,
                        cudaStream_t s) {
    if (n > 0) launch_tc<16>(p, d, nrhs, lo, n, cc, cp, s);  // blocks of 16 densities
}

}  // namespace ifgf
