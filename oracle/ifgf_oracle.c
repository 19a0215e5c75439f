/*
 * IFGF oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously structured CPU statement of what the GPU path
 * computes.  Only the tests, __graft_entry__.smoke() and the bench's CPU
 * baseline / reference legs load this file; the product library never does,
 * and this file shares no code, header or table generator with it.
 *
 * Contents
 *   O1  orc_direct_sum      the discrete operator of Eq. (1), FP64, compensated sums.
 *   O2  orc_plan_create     octree, neighbour/cousin sets (Sec. 2, Eq. (2)), Morton
 *                           order (Sec. 3.2.1), cone segments and the relevant-cone
 *                           recursion of Eq. (4), cone order (Sec. 3.2.1).
 *       orc_apply           near field ("LevelDSingularInteractions", Sec. 2),
 *                           LevelDEvaluations (Algorithm 6), then for d = D..3
 *                           Interpolation(d) (Algorithm 8) and Propagation(d)
 *                           (Algorithm 7), as ordered by Algorithm 5.
 *   S1  orc_stokes_direct_sum   Eq. (1) with the Stokes Green tensor (the Stokeslet),
 *                           one of the kernels Sec. 2 names, FP64, compensated sums.
 *   S2  orc_apply_stokes    the same IFGF steps for the Stokeslet on a kappa = 0 plan.
 *   E1  orc_elastic_direct_sum  Eq. (1) with Kelvin's solution of linear elasticity.
 *   E2  orc_apply_elastic   the IFGF steps for Kelvin's solution on a kappa = 0 plan.
 *   M1  orc_shard_cones, orc_shard_points   the data one rank of a distributed run reads
 *                           (Sec. 3.2): the cones its Interpolation and Propagation look up and
 *                           the points its near field and LevelDEvaluations read.
 *
 * The paper defers the numerical details of IFGF (analytic factor, the
 * singularity-resolving radial variable, interpolation nodes, cone counts) to
 * its companion paper.  This file fixes them by the following readings, each
 * written out where it is used:
 *   - analytic factor g_k(x,x') = G(x,x')/G(x,x_k), so that Eq. (3) holds exactly;
 *   - box-centred spherical coordinates (s, theta, phi) with s = h_d / |x - x_k|,
 *     h_d = sqrt(3)/2 H_d (box circumradius), s in [0, eta], eta = sqrt(3)/3;
 *   - uniform cone grids (n_s, n_theta, n_phi) per level: a base grid, doubled in
 *     all three directions e_d times, e_d the smallest e >= 0 with
 *     kappa*H_d <= 2*pi*tau*2^e*(1 + 2^-10) (boxes of at most tau*2^e wavelengths, with a
 *     margin for the 2^-20 enlargement of the root cube);
 *   - tensor-product Chebyshev interpolation on first-kind nodes of orders
 *     (P_s, P_theta, P_phi); "generate interpolant" = Chebyshev coefficients by
 *     discrete cosine orthogonality;
 *   - the cone that contains a point is decided by a fixed sequence of correctly
 *     rounded FP32 operations on the point's offset from the box centre in grid
 *     units (see classify()), so that any implementation that performs the same
 *     IEEE operations reproduces the relevant-cone lists bit for bit;
 *   - the relevant-cone test of Eq. (4) is taken in its discrete form: a cone is
 *     relevant iff a cousin point or a node of a relevant parent cone lies in it;
 *   - the point order is the sort by the 60-bit level-21 Morton key, ties broken
 *     by the original index (the paper leaves the order inside a box arbitrary);
 *   - Stokes kernel: the Stokeslet at unit viscosity,
 *     S_ij(x,y) = (delta_ij/r + (x_i-y_i)(x_j-y_j)/r^3)/(8 pi), acting on real force
 *     vectors f_m; its centred factor is the Laplace one, G_0(x,x_k) = 1/(4 pi |x-x_k|),
 *     and its analytic factor S_ij(x,x')/G_0(x,x_k) (Eq. (3) with a matrix-valued G),
 *     so that propagation and interpolation are those of the kappa = 0 kernel applied
 *     to each of the three velocity components;
 *   - elasticity kernel: Kelvin's solution for a point force in an infinite isotropic solid
 *     with shear modulus mu and Poisson ratio nu,
 *     K_ij(x,y) = ((3-4nu) delta_ij/r + (x_i-y_i)(x_j-y_j)/r^3)/(16 pi mu (1-nu)),
 *     factored like the Stokeslet.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared  (no -ffast-math:
 * classification relies on IEEE single precision without contraction).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define KEY_LEVEL 21 /* finest level used for sorting: 20 bits per axis, 60-bit keys */
#define MAX_LEVEL 21
#define MAX_NBR 27
#define MAX_COUS 189

typedef double complex cplx;

/* ------------------------------------------------------------------------- */
/* O1: direct evaluation of Eq. (1)                                           */
/* ------------------------------------------------------------------------- */

/* Helmholtz Green function of Eq. (1): G(x,y) = exp(i kappa r) / (4 pi r), r = |x - y|. */
static cplx green(double kappa, double r) {
    return cexp(I * kappa * r) / (4.0 * M_PI * r);
}

/* Neumaier compensated accumulation of one real sum. */
typedef struct {
    double s, c;
} ksum;
static inline void ksum_add(ksum* k, double v) {
    double t = k->s + v;
    if (fabs(k->s) >= fabs(v))
        k->c += (k->s - t) + v;
    else
        k->c += (v - t) + k->s;
    k->s = t;
}

/*
 * I(x_l) = sum_{m != l} a_m G(x_l, x_m)   (Eq. (1)), for the M target indices tgt[],
 * every density vector r < nrhs.  a is [nrhs][N] complex128, out is [nrhs][M].
 * The kernel value of a pair is computed once and applied to every density.
 */
void orc_direct_sum(int64_t N, const double* x, const double* y, const double* z, double kappa,
                    int nrhs, const cplx* a, int64_t M, const int64_t* tgt, cplx* out) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < M; ++t) {
        const int64_t l = tgt[t];
        ksum* acc = (ksum*)calloc((size_t)2 * nrhs, sizeof(ksum));
        for (int64_t m = 0; m < N; ++m) {
            if (m == l) continue;
            double dx = x[l] - x[m], dy = y[l] - y[m], dz = z[l] - z[m];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            cplx g = green(kappa, r);
            for (int q = 0; q < nrhs; ++q) {
                cplx v = a[(int64_t)q * N + m] * g;
                ksum_add(&acc[2 * q], creal(v));
                ksum_add(&acc[2 * q + 1], cimag(v));
            }
        }
        for (int q = 0; q < nrhs; ++q)
            out[(int64_t)q * M + t] = (acc[2 * q].s + acc[2 * q].c) + I * (acc[2 * q + 1].s + acc[2 * q + 1].c);
        free(acc);
    }
}

/* Stokeslet at unit viscosity for the separation v = x - y (a reading; Sec. 2 names the
 * Stokes equations among the kernels of Eq. (1)):
 * S_ij = (delta_ij / r + v_i v_j / r^3) / (8 pi). */
static void stokeslet(const double* v, double S[3][3]) {
    const double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            S[i][j] = ((i == j ? 1.0 / r : 0.0) + v[i] * v[j] / (r * r * r)) / (8.0 * M_PI);
}

/* Kelvin's solution of the Navier equations of linear elasticity for the separation v = x - y
 * (displacement at x due to a unit point force at y; shear modulus mu, Poisson ratio nu):
 * K_ij = ((3 - 4 nu) delta_ij / r + v_i v_j / r^3) / (16 pi mu (1 - nu)). */
static void kelvinlet(const double* v, double mu, double nu, double S[3][3]) {
    const double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            S[i][j] = ((i == j ? (3.0 - 4.0 * nu) / r : 0.0) + v[i] * v[j] / (r * r * r)) /
                      (16.0 * M_PI * mu * (1.0 - nu));
}

/* Green tensor of kind 1 (Stokeslet) or 2 (Kelvin's solution with mu, nu). */
static void green_tensor(int kind, double mu, double nu, const double* v, double S[3][3]) {
    if (kind == 1)
        stokeslet(v, S);
    else
        kelvinlet(v, mu, nu, S);
}

/* u_i(x_l) = sum_{m != l} sum_j T_ij(x_l, x_m) f_j(x_m) for the Green tensor T of `kind`. */
static void tensor_direct_sum(int kind, double mu, double nu, int64_t N, const double* x, const double* y,
                              const double* z, int nf, const double* f, int64_t M, const int64_t* tgt,
                              double* out) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < M; ++t) {
        const int64_t l = tgt[t];
        ksum* acc = (ksum*)calloc((size_t)3 * nf, sizeof(ksum));
        for (int64_t m = 0; m < N; ++m) {
            if (m == l) continue;
            const double v[3] = {x[l] - x[m], y[l] - y[m], z[l] - z[m]};
            double S[3][3];
            green_tensor(kind, mu, nu, v, S);
            for (int q = 0; q < nf; ++q)
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
                        ksum_add(&acc[3 * q + i], S[i][j] * f[((int64_t)3 * q + j) * N + m]);
        }
        for (int c = 0; c < 3 * nf; ++c) out[(int64_t)c * M + t] = acc[c].s + acc[c].c;
        free(acc);
    }
}

/*
 * S1: u_i(x_l) = sum_{m != l} sum_j S_ij(x_l, x_m) f_j(x_m)  (Eq. (1) with the Stokeslet),
 * at the M target indices tgt[], for every force field s < nf.  f is [nf][3][N] real,
 * out is [nf][3][M].
 */
void orc_stokes_direct_sum(int64_t N, const double* x, const double* y, const double* z, int nf,
                           const double* f, int64_t M, const int64_t* tgt, double* out) {
    tensor_direct_sum(1, 1.0, 0.5, N, x, y, z, nf, f, M, tgt, out);
}

/* E1: the same with Kelvin's solution (shear modulus mu, Poisson ratio nu). */
void orc_elastic_direct_sum(int64_t N, const double* x, const double* y, const double* z, double mu, double nu,
                            int nf, const double* f, int64_t M, const int64_t* tgt, double* out) {
    tensor_direct_sum(2, mu, nu, N, x, y, z, nf, f, M, tgt, out);
}

/* ------------------------------------------------------------------------- */
/* O2: plain CPU IFGF                                                          */
/* ------------------------------------------------------------------------- */

typedef struct {
    /* cone grid of one level and its classification / node tables */
    int ns, nt, np;
    int64_t C;            /* ns*nt*np */
    double ds, dt, dp;    /* interval widths in s, theta, phi */
    double h;             /* circumradius h_d = sqrt(3)/2 H_d (physical units) */
    float hg;             /* circumradius in grid units */
    float* R2;            /* [ns]  (hg / (i ds))^2 in grid units, i >= 1 */
    float* C2;            /* [nt]  cos(i pi / nt)^2 */
    unsigned char* cpos;  /* [nt]  cos(i pi / nt) >= 0 */
    float* cph;           /* cos(2 pi j / np) */
    float* sph;           /* sin(2 pi j / np) */
    /* node tables for the points of this level's cones, as classified from a child */
    float* rho;           /* [ns*Ps]  hg / s_node (grid units) */
    float *ctn, *stn;     /* [nt*Pt]  cos/sin of theta nodes */
    float *cpn, *spn;     /* [np*Pp]  cos/sin of phi nodes */
} orc_grid;

typedef struct {
    int64_t n;         /* relevant boxes at this level */
    uint64_t* key;     /* Morton key of each box (ascending) */
    int64_t* start;    /* [n+1] first sorted point of each box */
    int64_t* parent;   /* index in level d-1 */
    int64_t* cstart;   /* [n+1] first child in level d+1 (children are contiguous) */
    int32_t* k;        /* [n][3] integer box coordinates */
    int32_t* nnb;      /* neighbour count (Eq. (2), N B) */
    int64_t* nb;       /* [n][27] neighbour boxes, ascending */
    int32_t* ncs;      /* cousin count (Eq. (2), M B) */
    int64_t* cs;       /* [n][189] cousin boxes, ascending */
    int64_t* pbox;     /* [N] box of each sorted point at this level */
    /* cones (levels 3..D) */
    orc_grid g;
    int64_t nc;        /* relevant cones R_C^d (Eq. (5)) */
    int64_t* cone_box; /* [nc] co-centred box */
    int32_t* cone_gam; /* [nc] linear cone index gamma */
    int64_t* slot;     /* [n*C] index into the cone list, or -1 if not relevant */
    int64_t work_int;  /* interpolation evaluations at this level */
    int64_t work_prop; /* propagation evaluations from this level into d-1 */
} orc_level;

typedef struct {
    int64_t N;
    int D;
    double kappa;
    int Ps, Pt, Pp, P;
    double a[3], H1;
    int64_t* perm;     /* sorted position -> original index */
    uint64_t* key;     /* sorted level-21 keys */
    double* X[3];      /* sorted coordinates */
    float* off;        /* [N][3] offset from the leaf centre in grid units (H_D/2) */
    orc_level L[MAX_LEVEL + 1];
    double *Ws, *Wt, *Wp; /* 1-D Chebyshev analysis matrices [P][P] */
    double *ts, *tt, *tp; /* Chebyshev nodes of the first kind */
    int64_t work_near, work_leaf;
    int status;
} orc_plan;

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_OOM = 2, ORC_ERR_INTERNAL = 5 };

static void* xcalloc(size_t n, size_t s) {
    void* p = calloc(n ? n : 1, s);
    return p;
}

/* Morton bit interleave: bit 3b <- kx bit b, 3b+1 <- ky bit b, 3b+2 <- kz bit b (Sec. 3.2.1). */
static uint64_t morton(uint32_t kx, uint32_t ky, uint32_t kz) {
    uint64_t key = 0;
    for (int b = 0; b < 21; ++b) {
        key |= (uint64_t)((kx >> b) & 1u) << (3 * b);
        key |= (uint64_t)((ky >> b) & 1u) << (3 * b + 1);
        key |= (uint64_t)((kz >> b) & 1u) << (3 * b + 2);
    }
    return key;
}
static void demorton(uint64_t key, int32_t* k) {
    k[0] = k[1] = k[2] = 0;
    for (int b = 0; b < 21; ++b) {
        k[0] |= (int32_t)((key >> (3 * b)) & 1u) << b;
        k[1] |= (int32_t)((key >> (3 * b + 1)) & 1u) << b;
        k[2] |= (int32_t)((key >> (3 * b + 2)) & 1u) << b;
    }
}

typedef struct {
    uint64_t key;
    int64_t idx;
} keyidx;
static int cmp_keyidx(const void* A, const void* B) {
    const keyidx* a = (const keyidx*)A;
    const keyidx* b = (const keyidx*)B;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx);
}
static int cmp_i64(const void* A, const void* B) {
    int64_t a = *(const int64_t*)A, b = *(const int64_t*)B;
    return a < b ? -1 : (a > b);
}

/* Binary search of a box key among the ascending keys of one level; -1 if the box is not relevant. */
static int64_t find_box(const orc_level* L, uint64_t key) {
    int64_t lo = 0, hi = L->n - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (L->key[mid] == key) return mid;
        if (L->key[mid] < key)
            lo = mid + 1;
        else
            hi = mid - 1;
    }
    return -1;
}

/* Chebyshev node of the first kind t_j = cos((2j+1) pi / (2P)). */
static double cheb_node(int j, int P) { return cos(M_PI * (2.0 * j + 1.0) / (2.0 * P)); }

/* Position of node t in interval idx of width w: w*(idx + (1+t)/2). */
static double node_in(int idx, double w, double t) { return w * ((double)idx + 0.5 * (1.0 + t)); }

/* Analysis matrix W[n][j] = (2 - delta_{n0})/P cos(n (2j+1) pi / (2P)). */
static double* cheb_analysis(int P) {
    double* W = (double*)xcalloc((size_t)P * P, sizeof(double));
    for (int n = 0; n < P; ++n)
        for (int j = 0; j < P; ++j)
            W[n * P + j] = (n == 0 ? 1.0 : 2.0) / P * cos(M_PI * n * (2.0 * j + 1.0) / (2.0 * P));
    return W;
}

/* Chebyshev polynomials T_0..T_{P-1} at t by the three-term recurrence (valid also for |t| > 1). */
static void cheb_T(double t, int P, double* T) {
    T[0] = 1.0;
    if (P > 1) T[1] = t;
    for (int n = 2; n < P; ++n) T[n] = 2.0 * t * T[n - 1] - T[n - 2];
}

/*
 * "Generate interpolant" (Algorithm 1): Chebyshev coefficients of the values f at the
 * tensor-product nodes, c_abc = sum_ijk Ws[a][i] Wt[b][j] Wp[c][k] f_ijk, index (i*Pt + j)*Pp + k.
 */
static void cheb3_coeffs(const orc_plan* p, const cplx* f, cplx* c) {
    for (int a = 0; a < p->Ps; ++a)
        for (int b = 0; b < p->Pt; ++b)
            for (int cc = 0; cc < p->Pp; ++cc) {
                cplx acc = 0;
                for (int i = 0; i < p->Ps; ++i)
                    for (int j = 0; j < p->Pt; ++j)
                        for (int k = 0; k < p->Pp; ++k)
                            acc += p->Ws[a * p->Ps + i] * p->Wt[b * p->Pt + j] * p->Wp[cc * p->Pp + k] *
                                   f[(i * p->Pt + j) * p->Pp + k];
                c[(a * p->Pt + b) * p->Pp + cc] = acc;
            }
}

/* Evaluate the interpolant sum_abc c_abc T_a(ts) T_b(tt) T_c(tp). */
static cplx cheb3_eval(const orc_plan* p, const cplx* c, double ts, double tt, double tp) {
    double Ts[32], Tt[32], Tp[32];
    cheb_T(ts, p->Ps, Ts);
    cheb_T(tt, p->Pt, Tt);
    cheb_T(tp, p->Pp, Tp);
    cplx acc = 0;
    for (int a = 0; a < p->Ps; ++a)
        for (int b = 0; b < p->Pt; ++b)
            for (int cc = 0; cc < p->Pp; ++cc) acc += c[(a * p->Pt + b) * p->Pp + cc] * (Ts[a] * Tt[b] * Tp[cc]);
    return acc;
}

/*
 * Cone containing a point (Sec. 3.2.2: spherical coordinates about the box centre, then the
 * segment index).  Input: the point's offset v from the box centre in grid units, as FP32.
 * Only correctly rounded FP32 products/sums and comparisons are used, in a fixed order, and
 * each bin index is a COUNT of edges that the point lies on or beyond, so every correct
 * implementation of the same IEEE operations reproduces it bit for bit:
 *   r2 = (vx*vx + vy*vy) + vz*vz;
 *   is = #{ i in [1, ns-1] : r2 <= R2[i] }          R2[i] = (h/(i ds))^2, i.e. s >= i ds;
 *   it = #{ i in [1, nt-1] : vz <= cos(theta_i) r } theta_i = i pi/nt, taken in squared form:
 *          cos >= 0:  vz < 0  or  vz*vz <= C2[i]*r2;   cos < 0:  vz < 0  and  vz*vz >= C2[i]*r2;
 *   ip = #{ j in [1, np-1] : phi >= phi_j }          phi_j = 2 pi j/np, with the lower half plane
 *          H = (vy < 0 or (vy == 0 and vx < 0)) and L_j = (cos(phi_j) vy - sin(phi_j) vx >= 0):
 *          2j < np: L_j or H;   2j == np: H;   2j > np: L_j and H;   ip = 0 on the z axis.
 * Bins are half-open [edge_i, edge_{i+1}); the top edges (s = eta, theta = pi) join the last bin
 * and phi wraps.  Linear index gamma = (is*nt + it)*np + ip: radial first, then elevation, then
 * azimuth (the order of co-centred cones, Sec. 3.2.1).
 */
static int64_t classify(const orc_grid* g, float vx, float vy, float vz) {
    float r2 = (vx * vx + vy * vy) + vz * vz;
    int is = 0;
    for (int i = 1; i < g->ns; ++i)
        if (r2 <= g->R2[i]) ++is;
    float z2 = vz * vz;
    int it = 0;
    for (int i = 1; i < g->nt; ++i) {
        float c2r = g->C2[i] * r2;
        int q = g->cpos[i] ? (vz < 0.0f || z2 <= c2r) : (vz < 0.0f && z2 >= c2r);
        if (q) ++it;
    }
    int ip = 0;
    if (!(vx == 0.0f && vy == 0.0f)) {
        int H = (vy < 0.0f) || (vy == 0.0f && vx < 0.0f);
        for (int j = 1; j < g->np; ++j) {
            int Lj = (g->cph[j] * vy - g->sph[j] * vx) >= 0.0f;
            int ge = (2 * j < g->np) ? (Lj || H) : (2 * j == g->np) ? H : (Lj && H);
            if (ge) ++ip;
        }
    }
    return ((int64_t)is * g->nt + it) * g->np + ip;
}

/* Local coordinates t in [-1,1] (slightly beyond near cone edges) of a point v relative to the
 * centre of a level's box, inside cone gamma; v is in physical units. */
static void local_coords(const orc_grid* g, int64_t gamma, const double* v, double* ts, double* tt,
                         double* tp) {
    int ip = (int)(gamma % g->np);
    int it = (int)((gamma / g->np) % g->nt);
    int is = (int)(gamma / ((int64_t)g->np * g->nt));
    double rxy = sqrt(v[0] * v[0] + v[1] * v[1]);
    double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double s = g->h / r;
    double th = atan2(rxy, v[2]);
    double ph = atan2(v[1], v[0]);
    *ts = (s - g->ds * (is + 0.5)) / (0.5 * g->ds);
    *tt = (th - g->dt * (it + 0.5)) / (0.5 * g->dt);
    double dphi = ph - g->dp * (ip + 0.5);
    while (dphi > M_PI) dphi -= 2.0 * M_PI;
    while (dphi <= -M_PI) dphi += 2.0 * M_PI;
    *tp = dphi / (0.5 * g->dp);
}

static void box_centre(const orc_plan* p, int d, const int32_t* k, double* c) {
    double Hd = ldexp(p->H1, 1 - d);
    for (int i = 0; i < 3; ++i) c[i] = p->a[i] + ((double)k[i] + 0.5) * Hd;
}

/* Physical position of node (a,b,c) of cone gamma of a level-d box with centre xc. */
static void node_pos(const orc_plan* p, const orc_grid* g, int64_t gamma, int a, int b, int c,
                     const double* xc, double* y) {
    int ip = (int)(gamma % g->np);
    int it = (int)((gamma / g->np) % g->nt);
    int is = (int)(gamma / ((int64_t)g->np * g->nt));
    double s = node_in(is, g->ds, p->ts[a]);
    double th = node_in(it, g->dt, p->tt[b]);
    double ph = node_in(ip, g->dp, p->tp[c]);
    double r = g->h / s;
    y[0] = xc[0] + r * sin(th) * cos(ph);
    y[1] = xc[1] + r * sin(th) * sin(ph);
    y[2] = xc[2] + r * cos(th);
}

/* FP32 node offset (grid units) from the centre of its own box, from the node tables. */
static void node_grid(const orc_plan* p, const orc_grid* g, int64_t gamma, int a, int b, int c, float* q) {
    int ip = (int)(gamma % g->np);
    int it = (int)((gamma / g->np) % g->nt);
    int is = (int)(gamma / ((int64_t)g->np * g->nt));
    float rho = g->rho[is * p->Ps + a];
    float st = g->stn[it * p->Pt + b], ctt = g->ctn[it * p->Pt + b];
    float cp = g->cpn[ip * p->Pp + c], sp = g->spn[ip * p->Pp + c];
    q[0] = rho * (st * cp);
    q[1] = rho * (st * sp);
    q[2] = rho * ctt;
}

static void free_level(orc_level* L) {
    free(L->key); free(L->start); free(L->parent); free(L->cstart); free(L->k);
    free(L->nnb); free(L->nb); free(L->ncs); free(L->cs); free(L->pbox);
    free(L->g.R2); free(L->g.C2); free(L->g.cpos); free(L->g.cph); free(L->g.sph); free(L->g.rho);
    free(L->g.ctn); free(L->g.stn); free(L->g.cpn); free(L->g.spn);
    free(L->cone_box); free(L->cone_gam); free(L->slot);
    memset(L, 0, sizeof(*L));
}

void orc_plan_destroy(orc_plan* p) {
    if (!p) return;
    free(p->perm); free(p->key);
    for (int i = 0; i < 3; ++i) free(p->X[i]);
    free(p->off);
    for (int d = 0; d <= MAX_LEVEL; ++d) free_level(&p->L[d]);
    free(p->Ws); free(p->Wt); free(p->Wp); free(p->ts); free(p->tt); free(p->tp);
    free(p);
}

/* Offset (grid units, FP32) of sorted point i from the centre of level-d box b, for
 * classification: integer centre difference plus the point's leaf offset. */
static void point_grid_offset(const orc_plan* p, int d, int64_t i, int64_t b, float* v) {
    const orc_level* LD = &p->L[p->D];
    const orc_level* Ld = &p->L[d];
    const int32_t* kl = &LD->k[3 * LD->pbox[i]];
    const int32_t* kb = &Ld->k[3 * b];
    int sh = p->D - d;
    for (int c = 0; c < 3; ++c) {
        int64_t m = (2 * (int64_t)kl[c] + 1) - ((2 * (int64_t)kb[c] + 1) << sh);
        v[c] = (float)m + p->off[3 * i + c];
    }
}

/*
 * Build the plan: tree (Sec. 2, Sec. 3.2.1-3.2.2), neighbour and cousin sets (Eq. (2)),
 * cone grids and the relevant cones of Eq. (4), top-down d = 3..D.
 * x,y,z: N points in the caller's order.  levels = 0 picks the smallest D >= 3 whose mean
 * relevant-leaf occupancy N/n_D is at most leaf_target.
 */
orc_plan* orc_plan_create(int64_t N, const double* x, const double* y, const double* z, double kappa,
                          int Ps, int Pt, int Pp, int levels, int leaf_target, int bns, int bnt, int bnp,
                          double tau, int* status) {
    *status = ORC_ERR_ARG;
    if (N < 2 || !(kappa >= 0.0) || !isfinite(kappa) || Ps < 1 || Pt < 1 || Pp < 1 || Ps > 32 ||
        Pt > 32 || Pp > 32 || (levels != 0 && (levels < 3 || levels > MAX_LEVEL)) || bns < 1 ||
        bnt < 1 || bnp < 4 || leaf_target < 1)
        return NULL;
    orc_plan* p = (orc_plan*)xcalloc(1, sizeof(orc_plan));
    p->N = N;
    p->kappa = kappa;
    p->Ps = Ps; p->Pt = Pt; p->Pp = Pp; p->P = Ps * Pt * Pp;

    /* Root cube B^1 (Sec. 2): centre of the bounding box, side = largest extent (1 + 2^-20). */
    const double* X0[3] = {x, y, z};
    double mn[3], mx[3];
    for (int c = 0; c < 3; ++c) {
        mn[c] = X0[c][0];
        mx[c] = X0[c][0];
        for (int64_t i = 0; i < N; ++i) {
            double v = X0[c][i];
            if (!isfinite(v)) { orc_plan_destroy(p); return NULL; }
            if (v < mn[c]) mn[c] = v;
            if (v > mx[c]) mx[c] = v;
        }
    }
    double ext = 0.0;
    for (int c = 0; c < 3; ++c) if (mx[c] - mn[c] > ext) ext = mx[c] - mn[c];
    if (!(ext > 0.0)) { orc_plan_destroy(p); return NULL; }
    p->H1 = ext * (1.0 + ldexp(1.0, -20));
    for (int c = 0; c < 3; ++c) p->a[c] = 0.5 * (mn[c] + mx[c]) - 0.5 * p->H1;

    /* Level-21 box index of every point: k = floor(u * 2^20), u = (x - a) / H1. */
    keyidx* ki = (keyidx*)xcalloc((size_t)N, sizeof(keyidx));
    double* U = (double*)xcalloc((size_t)N * 3, sizeof(double));
    for (int64_t i = 0; i < N; ++i) {
        uint32_t k[3];
        for (int c = 0; c < 3; ++c) {
            double u = (X0[c][i] - p->a[c]) / p->H1;
            U[3 * i + c] = u;
            double f = floor(u * 1048576.0);
            if (f < 0.0) f = 0.0;
            if (f > 1048575.0) f = 1048575.0;
            k[c] = (uint32_t)f;
        }
        ki[i].key = morton(k[0], k[1], k[2]);
        ki[i].idx = i;
    }
    /* Morton order of the points, ties by original index (Sec. 3.2.1). */
    qsort(ki, (size_t)N, sizeof(keyidx), cmp_keyidx);
    p->perm = (int64_t*)xcalloc((size_t)N, sizeof(int64_t));
    p->key = (uint64_t*)xcalloc((size_t)N, sizeof(uint64_t));
    for (int c = 0; c < 3; ++c) p->X[c] = (double*)xcalloc((size_t)N, sizeof(double));
    for (int64_t i = 0; i < N; ++i) {
        p->perm[i] = ki[i].idx;
        p->key[i] = ki[i].key;
        for (int c = 0; c < 3; ++c) p->X[c][i] = X0[c][ki[i].idx];
    }
    free(ki);

    /* Number of levels. */
    int D = levels;
    if (D == 0) {
        D = MAX_LEVEL;
        for (int d = 3; d <= MAX_LEVEL; ++d) {
            int sh = 3 * (KEY_LEVEL - d);
            int64_t nd = 1;
            for (int64_t i = 1; i < N; ++i)
                if ((p->key[i] >> sh) != (p->key[i - 1] >> sh)) ++nd;
            if (N <= (int64_t)leaf_target * nd) { D = d; break; }
        }
    }
    p->D = D;

    /* Relevant boxes of every level (Sec. 2, R_B^d) with their point ranges. */
    for (int d = 1; d <= D; ++d) {
        orc_level* L = &p->L[d];
        int sh = 3 * (KEY_LEVEL - d);
        int64_t nd = 1;
        for (int64_t i = 1; i < N; ++i)
            if ((p->key[i] >> sh) != (p->key[i - 1] >> sh)) ++nd;
        L->n = nd;
        L->key = (uint64_t*)xcalloc((size_t)nd, sizeof(uint64_t));
        L->start = (int64_t*)xcalloc((size_t)nd + 1, sizeof(int64_t));
        L->k = (int32_t*)xcalloc((size_t)nd * 3, sizeof(int32_t));
        L->pbox = (int64_t*)xcalloc((size_t)N, sizeof(int64_t));
        int64_t b = -1;
        for (int64_t i = 0; i < N; ++i) {
            if (i == 0 || (p->key[i] >> sh) != (p->key[i - 1] >> sh)) {
                ++b;
                L->key[b] = p->key[i] >> sh;
                L->start[b] = i;
                demorton(L->key[b], &L->k[3 * b]);
            }
            L->pbox[i] = b;
        }
        L->start[nd] = N;
    }
    /* Parent and child links. */
    for (int d = 1; d <= D; ++d) {
        orc_level* L = &p->L[d];
        L->parent = (int64_t*)xcalloc((size_t)L->n, sizeof(int64_t));
        for (int64_t b = 0; b < L->n; ++b) L->parent[b] = d > 1 ? p->L[d - 1].pbox[L->start[b]] : -1;
    }
    for (int d = 1; d <= D; ++d) {
        orc_level* L = &p->L[d];
        L->cstart = (int64_t*)xcalloc((size_t)L->n + 1, sizeof(int64_t));
        if (d < D) {
            orc_level* Lc = &p->L[d + 1];
            int64_t c = 0;
            for (int64_t b = 0; b < L->n; ++b) {
                while (c < Lc->n && Lc->parent[c] < b) ++c;
                L->cstart[b] = c;
            }
            L->cstart[L->n] = Lc->n;
        }
    }
    /* Leaf offsets in grid units u = H_D / 2: (x - a)/u - (2 k_D + 1), rounded to FP32. */
    p->off = (float*)xcalloc((size_t)N * 3, sizeof(float));
    for (int64_t i = 0; i < N; ++i) {
        const int32_t* kl = &p->L[D].k[3 * p->L[D].pbox[i]];
        int64_t o = p->perm[i];
        for (int c = 0; c < 3; ++c) {
            double t = U[3 * o + c] * ldexp(1.0, D);
            p->off[3 * i + c] = (float)(t - (double)(2 * (int64_t)kl[c] + 1));
        }
    }
    free(U);

    /* Neighbours N B (Eq. (2)): relevant boxes with ||j - k||_inf <= 1, the box itself included. */
    for (int d = 2; d <= D; ++d) {
        orc_level* L = &p->L[d];
        int64_t side = (int64_t)1 << (d - 1);
        L->nnb = (int32_t*)xcalloc((size_t)L->n, sizeof(int32_t));
        L->nb = (int64_t*)xcalloc((size_t)L->n * MAX_NBR, sizeof(int64_t));
        for (int64_t b = 0; b < L->n; ++b) {
            const int32_t* k = &L->k[3 * b];
            int cnt = 0;
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int64_t j0 = k[0] + dx, j1 = k[1] + dy, j2 = k[2] + dz;
                        if (j0 < 0 || j1 < 0 || j2 < 0 || j0 >= side || j1 >= side || j2 >= side) continue;
                        int64_t q = find_box(L, morton((uint32_t)j0, (uint32_t)j1, (uint32_t)j2));
                        if (q >= 0) L->nb[b * MAX_NBR + cnt++] = q;
                    }
            qsort(&L->nb[b * MAX_NBR], (size_t)cnt, sizeof(int64_t), cmp_i64);
            L->nnb[b] = cnt;
        }
    }
    /* Cousins M B (Eq. (2)): children of the parent's neighbours that are not neighbours. */
    for (int d = 3; d <= D; ++d) {
        orc_level* L = &p->L[d];
        orc_level* Lp = &p->L[d - 1];
        L->ncs = (int32_t*)xcalloc((size_t)L->n, sizeof(int32_t));
        L->cs = (int64_t*)xcalloc((size_t)L->n * MAX_COUS, sizeof(int64_t));
        for (int64_t b = 0; b < L->n; ++b) {
            const int32_t* k = &L->k[3 * b];
            int64_t pb = L->parent[b];
            int cnt = 0;
            for (int t = 0; t < Lp->nnb[pb]; ++t) {
                int64_t q = Lp->nb[pb * MAX_NBR + t];
                for (int64_t c = Lp->cstart[q]; c < Lp->cstart[q + 1]; ++c) {
                    const int32_t* kc = &L->k[3 * c];
                    int64_t m = 0;
                    for (int i = 0; i < 3; ++i) {
                        int64_t e = kc[i] - k[i];
                        if (e < 0) e = -e;
                        if (e > m) m = e;
                    }
                    if (m > 1) L->cs[b * MAX_COUS + cnt++] = c;
                }
            }
            qsort(&L->cs[b * MAX_COUS], (size_t)cnt, sizeof(int64_t), cmp_i64);
            L->ncs[b] = cnt;
        }
    }

    /* Chebyshev nodes and analysis matrices. */
    p->ts = (double*)xcalloc(Ps, sizeof(double));
    p->tt = (double*)xcalloc(Pt, sizeof(double));
    p->tp = (double*)xcalloc(Pp, sizeof(double));
    for (int j = 0; j < Ps; ++j) p->ts[j] = cheb_node(j, Ps);
    for (int j = 0; j < Pt; ++j) p->tt[j] = cheb_node(j, Pt);
    for (int j = 0; j < Pp; ++j) p->tp[j] = cheb_node(j, Pp);
    p->Ws = cheb_analysis(Ps);
    p->Wt = cheb_analysis(Pt);
    p->Wp = cheb_analysis(Pp);

    /* Cone grids: the base grid, doubled in all three directions e_d times, where e_d is the
     * smallest e >= 0 with kappa*H_d <= 2 pi tau 2^e (1 + 2^-10) (boxes of at most tau*2^e
     * wavelengths; the margin keeps the 2^-20 enlargement of the root cube from tipping a box
     * whose side is tau*2^e wavelengths into the next grid).
     * Above tau wavelengths each level up thus splits every cone into eight (Sec. 3.3). */
    const double eta = sqrt(3.0) / 3.0;
    for (int d = D; d >= 3; --d) {
        double Hd = ldexp(p->H1, 1 - d);
        int e = 0;
        while (kappa > 0.0 && e < 24 && kappa * Hd > 2.0 * M_PI * tau * ldexp(1.0, e) * (1.0 + ldexp(1.0, -10))) ++e;
        int gns = bns << e, gnt = bnt << e, gnp = bnp << e;
        orc_grid* g = &p->L[d].g;
        g->ns = gns; g->nt = gnt; g->np = gnp;
        g->C = (int64_t)gns * gnt * gnp;
        g->ds = eta / gns;
        g->dt = M_PI / gnt;
        g->dp = 2.0 * M_PI / gnp;
        g->h = 0.5 * sqrt(3.0) * Hd;
        double hgd = sqrt(3.0) * ldexp(1.0, D - d);
        g->hg = (float)hgd;
        g->R2 = (float*)xcalloc((size_t)gns, sizeof(float));
        for (int i = 1; i < gns; ++i) {
            double R = hgd / ((double)i * g->ds);
            g->R2[i] = (float)(R * R);
        }
        g->C2 = (float*)xcalloc((size_t)gnt, sizeof(float));
        g->cpos = (unsigned char*)xcalloc((size_t)gnt, 1);
        for (int i = 0; i < gnt; ++i) {
            double c = cos(M_PI * (double)i / (double)gnt);
            g->C2[i] = (float)(c * c);
            g->cpos[i] = c >= 0.0;
        }
        g->cph = (float*)xcalloc((size_t)gnp, sizeof(float));
        g->sph = (float*)xcalloc((size_t)gnp, sizeof(float));
        for (int j = 0; j < gnp; ++j) {
            g->cph[j] = (float)cos(2.0 * M_PI * (double)j / (double)gnp);
            g->sph[j] = (float)sin(2.0 * M_PI * (double)j / (double)gnp);
        }
        g->rho = (float*)xcalloc((size_t)gns * Ps, sizeof(float));
        for (int is = 0; is < gns; ++is)
            for (int a = 0; a < Ps; ++a) g->rho[is * Ps + a] = (float)(hgd / node_in(is, g->ds, p->ts[a]));
        g->ctn = (float*)xcalloc((size_t)gnt * Pt, sizeof(float));
        g->stn = (float*)xcalloc((size_t)gnt * Pt, sizeof(float));
        for (int it = 0; it < gnt; ++it)
            for (int b = 0; b < Pt; ++b) {
                double th = node_in(it, g->dt, p->tt[b]);
                g->ctn[it * Pt + b] = (float)cos(th);
                g->stn[it * Pt + b] = (float)sin(th);
            }
        g->cpn = (float*)xcalloc((size_t)gnp * Pp, sizeof(float));
        g->spn = (float*)xcalloc((size_t)gnp * Pp, sizeof(float));
        for (int ip = 0; ip < gnp; ++ip)
            for (int c = 0; c < Pp; ++c) {
                double ph = node_in(ip, g->dp, p->tp[c]);
                g->cpn[ip * Pp + c] = (float)cos(ph);
                g->spn[ip * Pp + c] = (float)sin(ph);
            }
    }

    /* Relevant cones, Eq. (4) in its discrete form, top-down d = 3..D. */
    int bad = 0;
    for (int d = 3; d <= D; ++d) {
        orc_level* L = &p->L[d];
        orc_grid* g = &L->g;
        unsigned char* mark = (unsigned char*)xcalloc((size_t)(L->n * g->C), 1);
        if (!mark) { orc_plan_destroy(p); *status = ORC_ERR_OOM; return NULL; }
#pragma omp parallel for schedule(dynamic, 8) reduction(| : bad)
        for (int64_t b = 0; b < L->n; ++b) {
            unsigned char* mb = mark + b * g->C;
            /* cousin points x in V B (Eq. (2)) */
            for (int t = 0; t < L->ncs[b]; ++t) {
                int64_t q = L->cs[b * MAX_COUS + t];
                for (int64_t i = L->start[q]; i < L->start[q + 1]; ++i) {
                    float v[3];
                    point_grid_offset(p, d, i, b, v);
                    if (v[0] == 0.0f && v[1] == 0.0f && v[2] == 0.0f) bad = 1;
                    mb[classify(g, v[0], v[1], v[2])] = 1;
                }
            }
            /* nodes of the relevant cones of the parent box */
            if (d > 3) {
                orc_level* Lp = &p->L[d - 1];
                int64_t pb = L->parent[b];
                const int32_t* kb = &L->k[3 * b];
                const int32_t* kp = &Lp->k[3 * pb];
                float o[3];
                for (int c = 0; c < 3; ++c)
                    o[c] = (float)(((int64_t)2 * (kb[c] - 2 * kp[c]) - 1) * ((int64_t)1 << (D - d)));
                for (int64_t sl = 0; sl < Lp->g.C; ++sl) {
                    int64_t cone = Lp->slot[pb * Lp->g.C + sl];
                    if (cone < 0) continue;
                    for (int a = 0; a < Ps; ++a)
                        for (int bb = 0; bb < Pt; ++bb)
                            for (int c = 0; c < Pp; ++c) {
                                float q[3];
                                node_grid(p, &Lp->g, sl, a, bb, c, q);
                                float v0 = q[0] - o[0], v1 = q[1] - o[1], v2 = q[2] - o[2];
                                mb[classify(g, v0, v1, v2)] = 1;
                            }
                }
            }
        }
        /* Cone list in the order of Sec. 3.2.1: box Morton order, then gamma. */
        int64_t nc = 0;
        L->slot = (int64_t*)xcalloc((size_t)(L->n * g->C), sizeof(int64_t));
        for (int64_t e = 0; e < L->n * g->C; ++e) {
            if (mark[e])
                L->slot[e] = nc++;
            else
                L->slot[e] = -1;
        }
        L->nc = nc;
        L->cone_box = (int64_t*)xcalloc((size_t)nc, sizeof(int64_t));
        L->cone_gam = (int32_t*)xcalloc((size_t)nc, sizeof(int32_t));
        for (int64_t e = 0; e < L->n * g->C; ++e)
            if (mark[e]) {
                L->cone_box[L->slot[e]] = e / g->C;
                L->cone_gam[L->slot[e]] = (int32_t)(e % g->C);
            }
        free(mark);
    }
    p->status = bad ? ORC_ERR_INTERNAL : ORC_OK;
    *status = p->status;
    return p;
}

/* Coincident-point check: 1 if two points share all three coordinates. */
int orc_has_duplicates(const orc_plan* p) {
    for (int64_t b = 0; b < p->L[p->D].n; ++b)
        for (int64_t i = p->L[p->D].start[b]; i < p->L[p->D].start[b + 1]; ++i)
            for (int64_t j = i + 1; j < p->L[p->D].start[b + 1]; ++j)
                if (p->X[0][i] == p->X[0][j] && p->X[1][i] == p->X[1][j] && p->X[2][i] == p->X[2][j])
                    return 1;
    return 0;
}

/*
 * Apply the operator (Algorithm 5 with the parallel loops of Algorithms 6-8).
 * a: [nrhs][N] complex128 in the caller's point order; out: same layout, overwritten.
 * near != 0 adds the level-D neighbour interactions; bit d of level_mask adds the
 * level-d cousin interpolations (all levels: ~0).
 */
/*
 * The IFGF apply on nrhs channels.  Helmholtz (kind = 0): channel q is density vector q.
 * Green tensors (kind 1 Stokeslet, kind 2 Kelvin's solution with mu, nu; kappa = 0): channel
 * 3s+j holds component j of force field s (real values in complex storage); the near field and
 * the leaf evaluation contract the tensor with the force vector, everything after the leaf
 * level acts on each channel alone, as it does for the kappa = 0 kernel.
 */
static int apply_impl(orc_plan* p, int kind, double mu, double nu, int nrhs, const cplx* a, cplx* out, int near,
                      int64_t level_mask) {
    const int stokes = kind != 0;
    const int64_t N = p->N;
    const int D = p->D, P = p->P, Ps = p->Ps, Pt = p->Pt, Pp = p->Pp;
    const double kappa = p->kappa;
    cplx* as = (cplx*)xcalloc((size_t)N * nrhs, sizeof(cplx));
    cplx* I_ = (cplx*)xcalloc((size_t)N * nrhs, sizeof(cplx));
    for (int q = 0; q < nrhs; ++q)
        for (int64_t i = 0; i < N; ++i) as[(int64_t)q * N + i] = a[(int64_t)q * N + p->perm[i]];
    int bad = 0;
    orc_level* LD = &p->L[D];

    /* LevelDSingularInteractions: sum over U B (neighbour-box points), m != l. */
    int64_t wnear = 0;
    if (near) {
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : wnear)
        for (int64_t b = 0; b < LD->n; ++b)
            for (int64_t i = LD->start[b]; i < LD->start[b + 1]; ++i)
                for (int t = 0; t < LD->nnb[b]; ++t) {
                    int64_t q = LD->nb[b * MAX_NBR + t];
                    for (int64_t j = LD->start[q]; j < LD->start[q + 1]; ++j) {
                        if (j == i) continue;
                        double dx = p->X[0][i] - p->X[0][j], dy = p->X[1][i] - p->X[1][j],
                               dz = p->X[2][i] - p->X[2][j];
                        ++wnear;
                        if (stokes) {
                            const double v[3] = {dx, dy, dz};
                            double S[3][3];
                            green_tensor(kind, mu, nu, v, S);
                            for (int q = 0; q < nrhs / 3; ++q)
                                for (int c = 0; c < 3; ++c)
                                    for (int e = 0; e < 3; ++e)
                                        I_[(int64_t)(3 * q + c) * N + i] += S[c][e] * as[(int64_t)(3 * q + e) * N + j];
                            continue;
                        }
                        cplx g = green(kappa, sqrt(dx * dx + dy * dy + dz * dz));
                        for (int r = 0; r < nrhs; ++r) I_[(int64_t)r * N + i] += as[(int64_t)r * N + j] * g;
                    }
                }
    }
    p->work_near = wnear;

    /* LevelDEvaluations (Algorithm 6): F_k^D at the nodes of every relevant leaf cone
     * (Eq. (3): F = sum a(x') g_k(x,x'), g_k = G(x,x')/G(x,x_k)), then its interpolant. */
    cplx* coef = (cplx*)xcalloc((size_t)LD->nc * P * nrhs, sizeof(cplx));
    int64_t wleaf = 0;
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : wleaf)
    for (int64_t cone = 0; cone < LD->nc; ++cone) {
        int64_t b = LD->cone_box[cone];
        int64_t gam = LD->cone_gam[cone];
        double xc[3];
        box_centre(p, D, &LD->k[3 * b], xc);
        cplx* f = (cplx*)xcalloc((size_t)P * nrhs, sizeof(cplx));
        for (int aa = 0; aa < Ps; ++aa)
            for (int bb = 0; bb < Pt; ++bb)
                for (int cc = 0; cc < Pp; ++cc) {
                    double yv[3];
                    node_pos(p, &LD->g, gam, aa, bb, cc, xc, yv);
                    int n = (aa * Pt + bb) * Pp + cc;
                    double r = sqrt((yv[0] - xc[0]) * (yv[0] - xc[0]) + (yv[1] - xc[1]) * (yv[1] - xc[1]) +
                                    (yv[2] - xc[2]) * (yv[2] - xc[2]));
                    for (int64_t j = LD->start[b]; j < LD->start[b + 1]; ++j) {
                        double dx = yv[0] - p->X[0][j], dy = yv[1] - p->X[1][j], dz = yv[2] - p->X[2][j];
                        ++wleaf;
                        if (stokes) {
                            /* analytic factor S_ij(y, x') / G_0(y, x_k), G_0(y, x_k) = 1/(4 pi r) */
                            const double v[3] = {dx, dy, dz};
                            double S[3][3];
                            green_tensor(kind, mu, nu, v, S);
                            for (int q = 0; q < nrhs / 3; ++q)
                                for (int c = 0; c < 3; ++c)
                                    for (int e = 0; e < 3; ++e)
                                        f[(int64_t)(3 * q + c) * P + n] +=
                                            (4.0 * M_PI * r) * S[c][e] * as[(int64_t)(3 * q + e) * N + j];
                            continue;
                        }
                        double dist = sqrt(dx * dx + dy * dy + dz * dz);
                        cplx g = (r / dist) * cexp(I * kappa * (dist - r));
                        for (int q = 0; q < nrhs; ++q) f[(int64_t)q * P + n] += as[(int64_t)q * N + j] * g;
                    }
                }
        for (int q = 0; q < nrhs; ++q) cheb3_coeffs(p, f + (int64_t)q * P, coef + (cone * nrhs + q) * P);
        free(f);
    }
    p->work_leaf = wleaf;

    for (int d = D; d >= 3; --d) {
        orc_level* L = &p->L[d];
        orc_grid* g = &L->g;
        /* Interpolation(d) (Algorithm 8): for every point x and every box B in M^d(x) (Eq. (8)),
         * add I_P C_{k;gamma}(x) G(x, x_k).  The cousin relation is symmetric, so M^d(x) is the
         * cousin set of the level-d box that contains x. */
        int64_t wint = 0;
        if ((level_mask >> d) & 1) {
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : wint) reduction(| : bad)
            for (int64_t i = 0; i < N; ++i) {
                int64_t bx = L->pbox[i];
                for (int t = 0; t < L->ncs[bx]; ++t) {
                    int64_t B = L->cs[bx * MAX_COUS + t];
                    float v[3];
                    point_grid_offset(p, d, i, B, v);
                    int64_t gam = classify(g, v[0], v[1], v[2]);
                    int64_t cone = L->slot[B * g->C + gam];
                    if (cone < 0) { bad = 1; continue; }
                    double xc[3], vv[3];
                    box_centre(p, d, &L->k[3 * B], xc);
                    for (int c = 0; c < 3; ++c) vv[c] = p->X[c][i] - xc[c];
                    double ts, tt, tp;
                    local_coords(g, gam, vv, &ts, &tt, &tp);
                    cplx G = green(kappa, sqrt(vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2]));
                    ++wint;
                    for (int q = 0; q < nrhs; ++q)
                        I_[(int64_t)q * N + i] += cheb3_eval(p, coef + (cone * nrhs + q) * P, ts, tt, tp) * G;
                }
            }
        }
        L->work_int = wint;
        if (d == 3) break;
        /* Propagation(d) (Algorithm 7): for every relevant parent cone (j, gamma) at level d-1,
         * every relevant child B_k of B_j and every node x of the cone, add
         * I_P C_{k;alpha}(x) G(x, x_k) / G(x, x_j); then generate the parent interpolants. */
        orc_level* Lp = &p->L[d - 1];
        cplx* pcoef = (cplx*)xcalloc((size_t)Lp->nc * P * nrhs, sizeof(cplx));
        int64_t wprop = 0;
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : wprop) reduction(| : bad)
        for (int64_t pc = 0; pc < Lp->nc; ++pc) {
            int64_t jb = Lp->cone_box[pc];
            int64_t pg = Lp->cone_gam[pc];
            double xj[3];
            box_centre(p, d - 1, &Lp->k[3 * jb], xj);
            cplx* f = (cplx*)xcalloc((size_t)P * nrhs, sizeof(cplx));
            for (int64_t kb = Lp->cstart[jb]; kb < Lp->cstart[jb + 1]; ++kb) {
                double xk[3];
                box_centre(p, d, &L->k[3 * kb], xk);
                const int32_t* kk = &L->k[3 * kb];
                const int32_t* kj = &Lp->k[3 * jb];
                float o[3];
                for (int c = 0; c < 3; ++c)
                    o[c] = (float)(((int64_t)2 * (kk[c] - 2 * kj[c]) - 1) * ((int64_t)1 << (D - d)));
                for (int aa = 0; aa < Ps; ++aa)
                    for (int bb = 0; bb < Pt; ++bb)
                        for (int cc = 0; cc < Pp; ++cc) {
                            int n = (aa * Pt + bb) * Pp + cc;
                            float q[3];
                            node_grid(p, &Lp->g, pg, aa, bb, cc, q);
                            int64_t gam = classify(g, q[0] - o[0], q[1] - o[1], q[2] - o[2]);
                            int64_t cone = L->slot[kb * g->C + gam];
                            if (cone < 0) { bad = 1; continue; }
                            double yv[3], vv[3];
                            node_pos(p, &Lp->g, pg, aa, bb, cc, xj, yv);
                            for (int c = 0; c < 3; ++c) vv[c] = yv[c] - xk[c];
                            double ts, tt, tp;
                            local_coords(g, gam, vv, &ts, &tt, &tp);
                            double rk = sqrt(vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2]);
                            double rj = sqrt((yv[0] - xj[0]) * (yv[0] - xj[0]) + (yv[1] - xj[1]) * (yv[1] - xj[1]) +
                                             (yv[2] - xj[2]) * (yv[2] - xj[2]));
                            cplx ratio = green(kappa, rk) / green(kappa, rj);
                            ++wprop;
                            for (int r = 0; r < nrhs; ++r)
                                f[(int64_t)r * P + n] += cheb3_eval(p, coef + (cone * nrhs + r) * P, ts, tt, tp) * ratio;
                        }
            }
            for (int r = 0; r < nrhs; ++r) cheb3_coeffs(p, f + (int64_t)r * P, pcoef + (pc * nrhs + r) * P);
            free(f);
        }
        L->work_prop = wprop;
        free(coef);
        coef = pcoef;
    }
    free(coef);
    for (int q = 0; q < nrhs; ++q)
        for (int64_t i = 0; i < N; ++i) out[(int64_t)q * N + p->perm[i]] = I_[(int64_t)q * N + i];
    free(as);
    free(I_);
    return bad ? ORC_ERR_INTERNAL : ORC_OK;
}

int orc_apply(orc_plan* p, int nrhs, const cplx* a, cplx* out, int near, int64_t level_mask) {
    return apply_impl(p, 0, 0.0, 0.0, nrhs, a, out, near, level_mask);
}

static int apply_tensor(orc_plan* p, int kind, double mu, double nu, int nf, const double* f, double* u, int near,
                        int64_t level_mask) {
    if (p->kappa != 0.0 || nf < 1) return ORC_ERR_ARG;
    const int64_t n = (int64_t)3 * nf * p->N;
    cplx* a = (cplx*)xcalloc((size_t)n, sizeof(cplx));
    cplx* o = (cplx*)xcalloc((size_t)n, sizeof(cplx));
    for (int64_t i = 0; i < n; ++i) a[i] = f[i];
    int st = apply_impl(p, kind, mu, nu, 3 * nf, a, o, near, level_mask);
    for (int64_t i = 0; i < n; ++i) u[i] = creal(o[i]);
    free(a);
    free(o);
    return st;
}

/* S2: u = IFGF approximation of S1 at every point; f and u are [nf][3][N] real in the
 * caller's point order.  The plan must have kappa = 0. */
int orc_apply_stokes(orc_plan* p, int nf, const double* f, double* u, int near, int64_t level_mask) {
    return apply_tensor(p, 1, 1.0, 0.5, nf, f, u, near, level_mask);
}

/* E2: the IFGF approximation of E1, as orc_apply_stokes. */
int orc_apply_elastic(orc_plan* p, double mu, double nu, int nf, const double* f, double* u, int near,
                      int64_t level_mask) {
    if (!(mu > 0.0) || !(nu > -1.0) || !(nu <= 0.5)) return ORC_ERR_ARG;
    return apply_tensor(p, 2, mu, nu, nf, f, u, near, level_mask);
}

/* ------------------------------------------------------------------------- */
/* Introspection for tests                                                     */
/* ------------------------------------------------------------------------- */

enum {
    ORC_Q_PERM = 0,
    ORC_Q_KEYS = 1,
    ORC_Q_BOX_KEYS = 2,
    ORC_Q_BOX_START = 3,
    ORC_Q_BOX_PARENT = 4,
    ORC_Q_NBR_COUNT = 5,
    ORC_Q_NBR_LIST = 6,
    ORC_Q_COUS_COUNT = 7,
    ORC_Q_COUS_LIST = 8,
    ORC_Q_CONE_BOX = 9,
    ORC_Q_CONE_GAMMA = 10,
    ORC_Q_GRID = 11,
    ORC_Q_WORK = 12,
    ORC_Q_CHILD_START = 13,
};

/* ------------------------------------------------------------------------- */
/* Distribution over ranks (Sec. 3.2): what one rank reads                     */
/* ------------------------------------------------------------------------- */

/*
 * The level-d cones a rank reads, for the rank that owns the sorted points [pt_lo, pt_hi) and the
 * level-(d-1) relevant cones [pc_lo, pc_hi).  need[c] (c a level-d cone index) receives
 *   bit 0  when Interpolation(d) of one of the rank's points looks the cone up: for each point x
 *          and each box B in M^d(x) (the cousins of x's level-d box), the cone of B containing x
 *          (the lookups of Algorithm 8 whose data CommunicateInterpolationData gathers);
 *   bit 1  when Propagation(d) of one of the rank's parent cones looks it up: for each parent cone,
 *          each relevant child box of its box and each interpolation node, the child cone
 *          containing the node (the lookups of Algorithm 7 gathered by CommunicatePropagationData).
 * need is cleared first.  Returns 0, or ORC_ERR_INTERNAL when a lookup finds no relevant cone.
 */
int orc_shard_cones(const orc_plan* p, int d, int64_t pt_lo, int64_t pt_hi, int64_t pc_lo, int64_t pc_hi,
                    unsigned char* need) {
    if (d < 3 || d > p->D) return ORC_ERR_ARG;
    const orc_level* L = &p->L[d];
    const orc_grid* g = &L->g;
    memset(need, 0, (size_t)L->nc);
    int bad = 0;
    for (int64_t i = pt_lo; i < pt_hi; ++i) {
        const int64_t A = L->pbox[i];
        for (int t = 0; t < L->ncs[A]; ++t) {
            const int64_t B = L->cs[A * MAX_COUS + t];
            float v[3];
            point_grid_offset(p, d, i, B, v);
            const int64_t cone = L->slot[B * g->C + classify(g, v[0], v[1], v[2])];
            if (cone < 0) bad = 1;
            else need[cone] |= 1;
        }
    }
    if (d > 3) {
        const orc_level* Lp = &p->L[d - 1];
        for (int64_t pc = pc_lo; pc < pc_hi; ++pc) {
            const int64_t jb = Lp->cone_box[pc];
            const int32_t* kp = &Lp->k[3 * jb];
            for (int64_t kb = Lp->cstart[jb]; kb < Lp->cstart[jb + 1]; ++kb) {
                const int32_t* kk = &L->k[3 * kb];
                float o[3];
                for (int c = 0; c < 3; ++c)
                    o[c] = (float)(((int64_t)2 * (kk[c] - 2 * kp[c]) - 1) * ((int64_t)1 << (p->D - d)));
                for (int a = 0; a < p->Ps; ++a)
                    for (int b = 0; b < p->Pt; ++b)
                        for (int c = 0; c < p->Pp; ++c) {
                            float q[3];
                            node_grid(p, &Lp->g, Lp->cone_gam[pc], a, b, c, q);
                            const int64_t cone = L->slot[kb * g->C + classify(g, q[0] - o[0], q[1] - o[1], q[2] - o[2])];
                            if (cone < 0) bad = 1;
                            else need[cone] |= 2;
                        }
            }
        }
    }
    return bad ? ORC_ERR_INTERNAL : ORC_OK;
}

/*
 * The sorted points a rank reads besides its own, for the rank that owns the sorted points
 * [pt_lo, pt_hi) and the level-D relevant cones [c_lo, c_hi): need[i] receives bit 0 for the
 * points of the level-D neighbours of its points' boxes (the near field, Sec. 2) and bit 1 for the
 * points of the boxes of its level-D cones (LevelDEvaluations, Algorithm 6); need is cleared first.
 */
void orc_shard_points(const orc_plan* p, int64_t pt_lo, int64_t pt_hi, int64_t c_lo, int64_t c_hi,
                      unsigned char* need) {
    const orc_level* LD = &p->L[p->D];
    memset(need, 0, (size_t)p->N);
    for (int64_t i = pt_lo; i < pt_hi; ++i) {
        const int64_t b = LD->pbox[i];
        for (int t = 0; t < LD->nnb[b]; ++t) {
            const int64_t q = LD->nb[b * MAX_NBR + t];
            for (int64_t j = LD->start[q]; j < LD->start[q + 1]; ++j) need[j] |= 1;
        }
    }
    for (int64_t c = c_lo; c < c_hi; ++c) {
        const int64_t b = LD->cone_box[c];
        for (int64_t j = LD->start[b]; j < LD->start[b + 1]; ++j) need[j] |= 2;
    }
}

/* Copies an integer array of the plan into buf (int64) when buf != NULL; returns its length. */
int64_t orc_get(const orc_plan* p, int what, int d, int64_t* buf) {
    if (d < 0 || d > MAX_LEVEL) return -1;
    const orc_level* L = &p->L[d];
    int64_t n = 0;
    switch (what) {
        case ORC_Q_PERM:
            n = p->N;
            if (buf) for (int64_t i = 0; i < n; ++i) buf[i] = p->perm[i];
            return n;
        case ORC_Q_KEYS:
            n = p->N;
            if (buf) for (int64_t i = 0; i < n; ++i) buf[i] = (int64_t)p->key[i];
            return n;
        case ORC_Q_BOX_KEYS:
            if (buf) for (int64_t i = 0; i < L->n; ++i) buf[i] = (int64_t)L->key[i];
            return L->n;
        case ORC_Q_BOX_START:
            if (buf) for (int64_t i = 0; i <= L->n; ++i) buf[i] = L->start[i];
            return L->n + 1;
        case ORC_Q_BOX_PARENT:
            if (buf) for (int64_t i = 0; i < L->n; ++i) buf[i] = L->parent[i];
            return L->n;
        case ORC_Q_CHILD_START:
            if (buf) for (int64_t i = 0; i <= L->n; ++i) buf[i] = L->cstart[i];
            return L->n + 1;
        case ORC_Q_NBR_COUNT:
            if (!L->nnb) return -1;
            if (buf) for (int64_t i = 0; i < L->n; ++i) buf[i] = L->nnb[i];
            return L->n;
        case ORC_Q_NBR_LIST:
            if (!L->nnb) return -1;
            for (int64_t i = 0; i < L->n; ++i)
                for (int t = 0; t < L->nnb[i]; ++t) {
                    if (buf) buf[n] = L->nb[i * MAX_NBR + t];
                    ++n;
                }
            return n;
        case ORC_Q_COUS_COUNT:
            if (!L->ncs) return -1;
            if (buf) for (int64_t i = 0; i < L->n; ++i) buf[i] = L->ncs[i];
            return L->n;
        case ORC_Q_COUS_LIST:
            if (!L->ncs) return -1;
            for (int64_t i = 0; i < L->n; ++i)
                for (int t = 0; t < L->ncs[i]; ++t) {
                    if (buf) buf[n] = L->cs[i * MAX_COUS + t];
                    ++n;
                }
            return n;
        case ORC_Q_CONE_BOX:
            if (buf) for (int64_t i = 0; i < L->nc; ++i) buf[i] = L->cone_box[i];
            return L->nc;
        case ORC_Q_CONE_GAMMA:
            if (buf) for (int64_t i = 0; i < L->nc; ++i) buf[i] = L->cone_gam[i];
            return L->nc;
        case ORC_Q_GRID:
            if (buf) { buf[0] = L->g.ns; buf[1] = L->g.nt; buf[2] = L->g.np; }
            return 3;
        case ORC_Q_WORK:
            if (buf) { buf[0] = p->work_near; buf[1] = p->work_leaf; buf[2] = L->work_int; buf[3] = L->work_prop; }
            return 4;
        default:
            return -1;
    }
}

/* info: [N, D, n_1..n_21 (boxes), nc_1..nc_21 (cones)] = 44 entries; geom: [a0,a1,a2,H1]. */
void orc_info(const orc_plan* p, int64_t* info, double* geom) {
    info[0] = p->N;
    info[1] = p->D;
    for (int d = 1; d <= MAX_LEVEL; ++d) {
        info[1 + d] = p->L[d].n;
        info[22 + d] = p->L[d].nc;
    }
    if (geom) {
        geom[0] = p->a[0]; geom[1] = p->a[1]; geom[2] = p->a[2]; geom[3] = p->H1;
    }
}

/* FP32 leaf offsets [N][3] (grid units). */
void orc_offsets(const orc_plan* p, float* buf) { memcpy(buf, p->off, sizeof(float) * 3 * p->N); }

/* Classification of FP32 grid-unit offsets v[n][3] in the cone grid of level d. */
void orc_classify(const orc_plan* p, int d, int64_t n, const float* v, int64_t* out) {
    for (int64_t i = 0; i < n; ++i) out[i] = classify(&p->L[d].g, v[3 * i], v[3 * i + 1], v[3 * i + 2]);
}

/* One cone's interpolant: coefficients from node values, and evaluation at local
 * coordinates t[n][3] -- exposed so that tests can check polynomial reproduction. */
void orc_cheb3(const orc_plan* p, const cplx* f, cplx* c) { cheb3_coeffs(p, f, c); }
void orc_cheb3_eval(const orc_plan* p, const cplx* c, int64_t n, const double* t, cplx* out) {
    for (int64_t i = 0; i < n; ++i) out[i] = cheb3_eval(p, c, t[3 * i], t[3 * i + 1], t[3 * i + 2]);
}
void orc_cheb_nodes(const orc_plan* p, double* ts, double* tt, double* tp) {
    memcpy(ts, p->ts, sizeof(double) * p->Ps);
    memcpy(tt, p->tt, sizeof(double) * p->Pt);
    memcpy(tp, p->tp, sizeof(double) * p->Pp);
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
