/*
 * ifgf.h -- C ABI of the GB300 IFGF operator-apply library.
 *
 * The library evaluates the discrete operator of Eq. (1) of "Massively Parallelized
 * Interpolated Factored Green Function Method" (Bauinger & Bruno):
 *
 *     I(x_l) = sum_{m != l} a_m G(x_l, x_m),   G(x,y) = exp(i kappa |x-y|) / (4 pi |x-y|),
 *
 * over N surface points x_1..x_N (kappa = 0 gives the Laplace kernel 1/(4 pi r)), with the
 * IFGF method of Sec. 2 of that paper: an octree of N-point boxes, box-centred cone
 * segments, the factorisation G(x,x') = G(x,x_k) g_k(x,x') of Eq. (3), and the three
 * functions LevelDEvaluations, Propagation and Interpolation (Algorithms 1-8), plus the
 * level-D neighbour interactions ("LevelDSingularInteractions", Sec. 2).
 *
 * Conventions
 *   - Every pointer named "device" must be CUDA device memory of the current device.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *   - Functions return an ifgf_status and never abort or throw; ifgf_last_error() gives a
 *     thread-local text for the last failure of the calling thread.
 *   - Complex numbers are interleaved (re, im) pairs: complex128 = 2 x double,
 *     complex64 = 2 x float.
 */
#ifndef IFGF_H
#define IFGF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ifgf_plan_s* ifgf_plan;
typedef struct ifgf_batch_s* ifgf_batch;

typedef enum {
    IFGF_OK = 0,
    IFGF_ERR_INVALID_ARG = 1, /* bad argument: see ifgf_plan_create / ifgf_apply */
    IFGF_ERR_OOM = 2,         /* device allocation failed; nothing leaked */
    IFGF_ERR_CUDA = 3,        /* a CUDA call failed; the text names it */
    IFGF_ERR_TIMEOUT = 4,     /* a bounded device wait expired */
    IFGF_ERR_INTERNAL = 5,    /* a device-side consistency check failed (e.g. cone lookup miss) */
    IFGF_ERR_UNSUPPORTED = 6  /* valid request outside what this build supports */
} ifgf_status;

typedef enum {
    IFGF_PREC_FP64 = 0,  /* every floating-point step in FP64 (complex128 in/out) */
    IFGF_PREC_MIXED = 1  /* FP32 arithmetic; grid-relative coordinates and large phases
                            kept exact or reduced in extended precision (complex64 in/out) */
} ifgf_precision;

/*
 * Method parameters.  Defaults (ifgf_options_default): MIXED, base cone grid (2, 4, 8),
 * tau = 0.5, leaf_target = 64, max_nrhs = 1.
 *   base_cones  (n_s, n_theta, n_phi) of the cone grid of boxes of at most tau wavelengths;
 *               level d uses the base grid doubled e times in all three directions, e the
 *               smallest integer with kappa H_d <= 2 pi tau 2^e (1 + 2^-10) (n_phi >= 4, even).
 *   leaf_target when levels == 0, D is the smallest level >= 3 whose mean relevant-leaf
 *               occupancy N / n_D is at most leaf_target.
 *   max_nrhs    largest nrhs that ifgf_apply will accept (buffers are sized for it).
 *   rhs_block   the coefficient buffer holds this many densities; ifgf_apply sweeps the levels
 *               once per block of densities (0: the largest block, up to max_nrhs, whose
 *               coefficients fit in half the free device memory at plan time, or in 90% of it
 *               when not even one density fits in half).
 *   cone_table  how a level finds the relevant cone of (box, cone index): 0 automatic (a dense
 *               n_d x C_d table while it has fewer than 2^31 entries, else the sorted cone list
 *               searched per box), 1 always dense (IFGF_ERR_UNSUPPORTED beyond 2^31 entries),
 *               2 always the sorted list.  Results do not depend on the choice.
 *   prop_slices the coefficients of consecutive levels share one buffer; propagation writes the
 *               parent level in this many slices so that it never overwrites child coefficients
 *               still to be read (0: one slice when two full levels fit the memory budget, else
 *               64).  More slices need less memory and more launches; results do not change.
 */
typedef struct {
    int32_t struct_size;   /* sizeof(ifgf_options) */
    int32_t precision;     /* ifgf_precision */
    int32_t base_cones[3];
    int32_t leaf_target;
    int32_t max_nrhs;
    int32_t rhs_block;     /* densities per level sweep; 0 = as many as fit half the free memory */
    double tau;
    int32_t cone_table;    /* 0 automatic, 1 dense, 2 sorted list */
    int32_t prop_slices;   /* 0 automatic, else propagation in this many slices (>= 1) */
} ifgf_options;

/* Fill *opt with the defaults listed above, struct_size included (host only; no device call). */
void ifgf_options_default(ifgf_options* opt);

/*
 * Build a plan: the Morton octree of the points and its relevant boxes (Sec. 2; Morton
 * order of Sec. 3.2.1), neighbour and cousin sets (Eq. (2)), the cone grids and the
 * relevant cone segments of Eq. (4) for levels 3..D in the order of Sec. 3.2.1, and the
 * apply buffers.  Runs on `stream` and returns after it has completed.
 *
 *   points   device, 3*N doubles, structure of arrays: x[0..N), y[0..N), z[0..N), in the
 *            caller's order.  Read only; the plan keeps its own sorted copy.
 *   N        number of points, 2 <= N < 2^31.
 *   kappa    wavenumber, finite and >= 0.
 *   orders   (P_s, P_theta, P_phi) interpolation orders (each >= 1), or NULL for (3, 5, 5).
 *            This build has kernels for (3,5,5) and (5,7,7); other valid orders return
 *            IFGF_ERR_UNSUPPORTED.
 *   levels   number of octree levels D in [3, 21], or 0 to choose it from leaf_target.
 *   opt      NULL for the defaults.
 *   out_plan receives the plan; unchanged on failure.
 *
 * Errors: IFGF_ERR_INVALID_ARG for N out of range, a non-finite coordinate, kappa < 0 or
 * non-finite, an order below 1, levels outside {0} U [3, 21], all points coincident, or
 * two points sharing all three coordinates (G is singular there); IFGF_ERR_UNSUPPORTED for
 * orders without kernels in this build, and when cone_table = 1 and a level's dense cone
 * table would exceed 2^31 entries; IFGF_ERR_OOM
 * (including a coefficient buffer of one density that does not fit), IFGF_ERR_CUDA.
 */
ifgf_status ifgf_plan_create(const double* points, int64_t N, double kappa, const int32_t* orders,
                             int32_t levels, const ifgf_options* opt, void* stream, ifgf_plan* out_plan);

/*
 * Apply the operator: out = I(a) (Algorithm 5 with the target- and cone-parallel loops of
 * Algorithms 6-8, plus the level-D neighbour sums).  Asynchronous on `stream`; the plan
 * owns its scratch, so one plan must not be applied concurrently on two streams.
 *
 *   densities device, [nrhs][N] complex128 (FP64 plan) or complex64 (MIXED plan), the
 *             caller's point order.  Read only.
 *   nrhs      1 <= nrhs <= opt.max_nrhs.
 *   out       device, same layout and type as densities; overwritten.  Must not alias it.
 *
 * Device-side consistency failures (a cone lookup that misses) are recorded in the plan
 * and returned by the next ifgf_plan_query(IFGF_Q_STATUS).
 */
ifgf_status ifgf_apply(ifgf_plan plan, const void* densities, int32_t nrhs, void* out, void* stream);

/*
 * Same as ifgf_apply, restricted to some contributions (for staged checks):
 *   near        nonzero adds the level-D neighbour interactions;
 *   level_mask  bit d adds the level-d cousin interpolations (all: -1).
 */
ifgf_status ifgf_apply_ex(ifgf_plan plan, const void* densities, int32_t nrhs, void* out, void* stream,
                          int32_t near, int64_t level_mask);

/*
 * Stokes kernel: velocities of point forces in Stokes flow at unit viscosity,
 *     u_i(x_l) = sum_{m != l} sum_j S_ij(x_l, x_m) f_j(x_m),
 *     S_ij(x, y) = (delta_ij / r + (x_i - y_i)(x_j - y_j) / r^3) / (8 pi),  r = |x - y|,
 * i.e. Eq. (1) with the Green tensor of the Stokes equations (one of the kernels Sec. 2 names),
 * evaluated by the same IFGF steps: the centred factor is the Laplace one, 1/(4 pi |x - x_k|),
 * and the analytic factor of Eq. (3) is S(x, x') divided by it.  Asynchronous on `stream`, like
 * ifgf_apply.
 *
 *   plan      created with kappa = 0 and opt.max_nrhs >= ceil(3 nfield / 2) (the three velocity
 *             components of a field are carried as real and imaginary parts of complex value
 *             sets, two per set).
 *   forces    device, [nfield][3][N] float32 (MIXED plan) or float64 (FP64 plan), component-major
 *             per field, the caller's point order.  Read only.
 *   nfield    number of force fields, >= 1.
 *   velocity  device, same layout and type as forces; overwritten.  Must not alias it.
 *
 * Errors: IFGF_ERR_INVALID_ARG for NULL pointers, aliasing, kappa != 0 or nfield out of range.
 */
ifgf_status ifgf_apply_stokes(ifgf_plan plan, const void* forces, int32_t nfield, void* velocity, void* stream);

/* ifgf_apply_stokes restricted to some contributions, as ifgf_apply_ex. */
ifgf_status ifgf_apply_stokes_ex(ifgf_plan plan, const void* forces, int32_t nfield, void* velocity, void* stream,
                                 int32_t near, int64_t level_mask);

/*
 * Elasticity kernel: displacements of point forces in an infinite homogeneous isotropic elastic
 * solid (Kelvin's solution of the Navier equations, one of the kernels Sec. 2 names),
 *     u_i(x_l) = sum_{m != l} sum_j K_ij(x_l, x_m) f_j(x_m),
 *     K_ij(x, y) = ((3 - 4 nu) delta_ij / r + (x_i - y_i)(x_j - y_j) / r^3) / (16 pi mu (1 - nu)),
 * evaluated as ifgf_apply_stokes does (same centred factor, plan requirements, layouts,
 * asynchrony and errors); at nu = 1/2 it is the Stokeslet divided by mu.
 *
 *   shear_modulus  mu, finite and > 0.
 *   poisson_ratio  nu, in (-1, 1/2].
 *
 * Errors: as ifgf_apply_stokes, plus IFGF_ERR_INVALID_ARG for mu or nu out of range.
 */
ifgf_status ifgf_apply_elastic(ifgf_plan plan, const void* forces, int32_t nfield, void* displacement,
                               double shear_modulus, double poisson_ratio, void* stream);

/* ifgf_apply_elastic restricted to some contributions, as ifgf_apply_ex. */
ifgf_status ifgf_apply_elastic_ex(ifgf_plan plan, const void* forces, int32_t nfield, void* displacement,
                                  double shear_modulus, double poisson_ratio, void* stream, int32_t near,
                                  int64_t level_mask);

/* Release the plan and all its device memory to the library's pool (synchronous; see
 * ifgf_release_cached_memory).  NULL is accepted. */
ifgf_status ifgf_plan_destroy(ifgf_plan plan);

/* Settings of ifgf_batch_set / ifgf_batch_get (described below). */
typedef enum {
    IFGF_BATCH_MODE = 0,
    IFGF_BATCH_CONES_PER_ITEM = 1,
    IFGF_BATCH_BLOCKS_PER_SM = 2,
    IFGF_BATCH_WAIT_LIMIT = 3,
    IFGF_BATCH_WITHHOLD = 4,
    IFGF_BATCH_STATUS = 5,
    IFGF_BATCH_LAST_MODE = 6,
    IFGF_BATCH_ITEMS = 7
} ifgf_batch_setting;
/*
 * Batched evaluation of many independent problems (each its own plan, e.g. bodies of different
 * sizes): the operator of Eq. (1) is applied to every plan, and each result is bit-identical to
 * the plan's own ifgf_apply.  Two launch sequences are built:
 *   queue  (plans of mixed precision with orders (3,5,5), one density each) one short sequence
 *          over work lists that mix all problems, largest first: permutation in, near field,
 *          LevelDEvaluations (Algorithm 6), the propagation (Algorithm 7), interpolation
 *          (Algorithm 8, one level per work unit) and permutation out with the level sums added
 *          in the single-plan order.  The propagation is either a persistent kernel per run of
 *          levels of one kind, whose blocks take runs of parent cones from a queue ordered by the
 *          distance of the child level from the problem's leaves (a run whose child level is not
 *          complete waits on the problem's per-level counter; waits bounded by
 *          IFGF_BATCH_WAIT_LIMIT polls, see ifgf_batch_set), or each plan's own per-level kernels
 *          on concurrent branches.  It keeps the coefficients and interpolation sums of every
 *          level of every problem (device memory owned by the batch, allocated at the first
 *          queue apply).
 *   graph  (any plans) each plan's own apply captured on branch i mod 8 of a fork/join, so that
 *          independent problems run concurrently.
 * Either sequence is captured into a CUDA graph by the first ifgf_batch_apply and replayed with
 * one graph launch on `stream` by later calls (the graph sequence is captured again when the
 * buffers change; the queue sequence reads the buffer pointers from a table that the call
 * updates, synchronising `stream` when they changed).  Plans must live on one device, must
 * outlive the batch, and must not be applied elsewhere while the batch runs (they own their
 * scratch).  Kernel knobs of the plans are read when the queue is built.
 *
 *   plans  n distinct plan handles (not owned); a handle that appears twice returns
 *          IFGF_ERR_INVALID_ARG, since each plan's buffers can serve one problem at a time.
 *   dens   n device pointers, plan i's densities as in ifgf_apply.
 *   nrhs   n counts, 1 <= nrhs[i] <= that plan's max_nrhs.
 *   outs   n device pointers, plan i's outputs.
 *
 * ifgf_batch_set / ifgf_batch_get (host; a change takes effect at the next apply):
 *   IFGF_BATCH_MODE            -1 (default) the built-in choice, the graph sequence; 0 graph;
 *                              1 queue with the persistent propagation; 2 queue with each plan's
 *                              propagation on branches (1 and 2: ifgf_batch_apply returns
 *                              IFGF_ERR_UNSUPPORTED when the plans do not allow them).
 *   IFGF_BATCH_CONES_PER_ITEM  parent cones per propagation queue item, >= 4 (rounded down to a
 *                              multiple of 4; default 16).
 *   IFGF_BATCH_BLOCKS_PER_SM   resident blocks per SM of the persistent propagation (0: as many
 *                              as fit, the default).
 *   IFGF_BATCH_WAIT_LIMIT      polls of a dependency counter (about 0.3 us each) before the
 *                              waiting block records IFGF_ERR_TIMEOUT in the batch's status word
 *                              and skips its item; later waits then give up at once (default 2^24).
 *   IFGF_BATCH_WITHHOLD        test only: problem * 64 + level d (4 <= d <= D of that problem):
 *                              the first queue item of the propagation from level d is never
 *                              counted as complete, so the items of level d-1 wait until their
 *                              limit; -1 turns it off.
 *   get only: IFGF_BATCH_STATUS (synchronises the device; the status word of the last queue
 *   sequence, IFGF_OK or IFGF_ERR_TIMEOUT, reset by every queue apply), IFGF_BATCH_LAST_MODE (the
 *   sequence the last apply ran: 0, 1 or 2 as IFGF_BATCH_MODE, -1 none), IFGF_BATCH_ITEMS
 *   (propagation queue items of the last queue sequence).
 * Errors: IFGF_ERR_INVALID_ARG for a NULL handle or pointer, an unknown code or a value out of
 * range.
 */
ifgf_status ifgf_batch_create(const ifgf_plan* plans, int32_t n, ifgf_batch* out_batch);
ifgf_status ifgf_batch_apply(ifgf_batch batch, const void* const* dens, const int32_t* nrhs, void* const* outs,
                             void* stream);
ifgf_status ifgf_batch_destroy(ifgf_batch batch);
ifgf_status ifgf_batch_set(ifgf_batch batch, int32_t what, int64_t value);
ifgf_status ifgf_batch_get(ifgf_batch batch, int32_t what, int64_t* value);

/*
 * Autotuner of a batch: times ifgf_batch_apply with the given buffers (three replays after a
 * warm-up) for the graph sequence and, where the plans allow it, the queue sequence with branch
 * propagation and with the persistent propagation at 8, 16, 32 and 64 parent cones per item and
 * 0 or 2 blocks per SM; sets the fastest (IFGF_BATCH_MODE,
 * IFGF_BATCH_CONES_PER_ITEM, IFGF_BATCH_BLOCKS_PER_SM).  Choices are cached in cache_path (NULL:
 * no cache) under a key of the GPU, the number of problems, their total and largest N (floor
 * log2 each), the densities bucket and whether the queue applies; with a cache hit nothing is
 * measured.  The outputs hold a valid result of the batch afterwards.  Arguments as
 * ifgf_batch_apply; from_cache: optional output, 1 if nothing was measured.
 * Errors: those of ifgf_batch_apply, IFGF_ERR_INVALID_ARG for an unwritable cache.
 */
ifgf_status ifgf_batch_autotune(ifgf_batch batch, const void* const* dens, const int32_t* nrhs, void* const* outs,
                                const char* cache_path, void* stream, int32_t* from_cache);

/*
 * Introspection (synchronous).  Copies the requested array into host_buf as int64 values
 * when host_buf != NULL and *inout_count is large enough; always stores the element count
 * in *inout_count.  `level` selects the octree level where the item is per level.
 */
enum {
    IFGF_Q_PERM = 0,        /* [N] sorted position -> caller index */
    IFGF_Q_KEYS = 1,        /* [N] sorted 60-bit level-21 Morton keys */
    IFGF_Q_BOX_KEYS = 2,    /* [n_d] Morton keys of the relevant boxes */
    IFGF_Q_BOX_START = 3,   /* [n_d + 1] first sorted point of each box */
    IFGF_Q_BOX_PARENT = 4,  /* [n_d] parent box (level d-1), -1 at level 1 */
    IFGF_Q_NBR_COUNT = 5,   /* [n_d] neighbour counts (levels >= 2) */
    IFGF_Q_NBR_LIST = 6,    /* concatenated ascending neighbour lists */
    IFGF_Q_COUS_COUNT = 7,  /* [n_d] cousin counts (levels >= 3) */
    IFGF_Q_COUS_LIST = 8,   /* concatenated ascending cousin lists */
    IFGF_Q_CONE_BOX = 9,    /* [c_d] box of each relevant cone, in cone order */
    IFGF_Q_CONE_GAMMA = 10, /* [c_d] linear cone index (is*nt + it)*np + ip */
    IFGF_Q_GRID = 11,       /* [3] (n_s, n_theta, n_phi) of level d */
    IFGF_Q_INFO = 12,       /* [44] N, D, n_1..n_21, c_1..c_21 */
    IFGF_Q_WORK = 13,       /* [4] near pairs, leaf pairs, level-d interpolations, level-d propagations */
    IFGF_Q_STATUS = 14,     /* [1] sticky device status (ifgf_status) */
    IFGF_Q_CHILD_START = 15, /* [n_d + 1] first child box in level d+1 */
    IFGF_Q_BOX_COORDS = 16,  /* [n_d * 3] integer box coordinates (k_x, k_y, k_z) */
    IFGF_Q_TABLES = 17       /* [1] node-table rows of level d (distinct cone indices whose node
                                geometry seen from the children is tabled); 0 when propagation into
                                level d computes the geometry per node */
};
ifgf_status ifgf_plan_query(ifgf_plan plan, int32_t what, int32_t level, int64_t* host_buf, int64_t* inout_count);

typedef enum { IFGF_KNOB_PROP_MANY = 0, IFGF_KNOB_PROP_FEW = 1, IFGF_KNOB_RHS_BLOCK = 2 } ifgf_knob;
/*
 * Kernel choices ("knobs") of a plan's mixed-precision apply.  Every choice computes the same
 * values of Algorithm 7; they differ in speed and in the rounding order of the FP32 sums.  A
 * value of -1 restores the built-in choice.
 *   IFGF_KNOB_PROP_MANY, per level d (the propagation from level d into level d-1, 4 <= d <= D),
 *     in effect where level d-1 has node tables and nrhs >= 4: 0 warp-level mma.sync tiles
 *     (built-in), 1 tcgen05 products with TMEM accumulators; both 3xTF32.
 *   IFGF_KNOB_PROP_FEW, per level d, in effect where level d-1 has node tables and nrhs < 4:
 *     0 the node-table warp kernel (built-in), 1 the per-cone kernel that computes the geometry.
 *   IFGF_KNOB_RHS_BLOCK, plan-wide (level ignored), nrhs >= 4: densities per block of the
 *     many-density kernels, 8, 16 or 32 (built-in, -1: the smallest of them >= nrhs, else 32).
 * ifgf_plan_get_knob returns the choice in effect for a level knob (-1 where level d-1 has no
 * node tables, so that the knob has no effect) and the value set for IFGF_KNOB_RHS_BLOCK.
 * Host only, no synchronisation; the next apply uses the new choice.
 * Errors: IFGF_ERR_INVALID_ARG (NULL plan or value pointer, unknown knob, level or value out of
 * range).
 */
ifgf_status ifgf_plan_set_knob(ifgf_plan plan, int32_t knob, int32_t level, int32_t value);
ifgf_status ifgf_plan_get_knob(ifgf_plan plan, int32_t knob, int32_t level, int32_t* value);

/*
 * Autotuner of the knobs above: for an apply with nrhs densities it times, on the plan's own
 * tree and cones with synthetic densities, each candidate kernel of every level whose parent
 * level has node tables (per-level propagation times from CUDA events around the launches) and,
 * from 4 densities on, each density block (8, 16, 32, by the time of the whole apply with the
 * faster kernel on every level), and sets the fastest.  The choices are stored in the text file
 * cache_path (created or rewritten whole; NULL: no cache) under keys made of the GPU's name and
 * SM count, the orders, the densities bucket (1, 2-3, 4-8, 9-16, 17-32, 33+) and the size
 * bucket (floor log2 of the level's cone counts, of N for the block); when every key is already
 * there the choices are taken from the file without measuring.  Plans other than mixed
 * precision with orders (3,5,5) have no choices: the call returns IFGF_OK and changes nothing.
 *
 *   nrhs        1 <= nrhs <= the plan's max_nrhs.
 *   stream      cudaStream_t as void*; the measurement runs on it (about six applies for
 *               1-3 densities, fourteen from 4 on) and the call returns after it.
 *   from_cache  optional output: 1 if nothing was measured.
 * The library's kernel timing (ifgf_timing_enable) is used and its collected totals are
 * discarded.  Errors: IFGF_ERR_INVALID_ARG (NULL plan, nrhs out of range, unwritable cache),
 * IFGF_ERR_OOM, IFGF_ERR_CUDA.
 */
ifgf_status ifgf_plan_autotune(ifgf_plan plan, int32_t nrhs, const char* cache_path, void* stream,
                               int32_t* from_cache);

/*
 * Solver integration: restarted GMRES(restart) for the second-kind system
 *     (alpha I + beta A W) x = b,
 * A the plan's operator of Eq. (1) (one ifgf_apply per iteration, the plan's precision) and W the
 * diagonal of the quadrature weights.  This is the use of the apply that the paper's Sec. 1-2
 * describe (the matrix-vector product of an iterative solver for a boundary integral equation);
 * the near field stays the point sum of Eq. (1): singular quadratures are not part of the paper.
 * Arnoldi with classical Gram-Schmidt applied twice; inner products accumulated in FP64 in a
 * fixed order (a solve is reproducible); Givens least squares on the host.
 *
 *   b, x         device, N complex values in the caller's point order (complex64 on a mixed plan,
 *                complex128 on an FP64 plan); x holds the initial guess and receives the solution.
 *   alpha, beta  host, 2 doubles each (real, imaginary part).
 *   weights      device, N reals (float32 mixed / float64 FP64) or NULL (all ones).
 *   restart      Krylov dimension per cycle, 1..128;  max_iters >= 1 (applies of A, not counting
 *                one per restart for the residual);  tol > 0: stop when |b - (alpha + beta A W) x|
 *                <= tol |b| (GMRES's estimate; the final residual is recomputed).
 *   iters, rel_residual  optional host outputs: iterations done, final relative residual.
 * Synchronous on `stream` (the host reads inner products every iteration).  Scratch: restart + 4
 * vectors of N from the library's pool.  Errors: IFGF_ERR_INVALID_ARG (NULL or aliased
 * pointers, parameters out of range), IFGF_ERR_OOM, IFGF_ERR_CUDA.
 */
ifgf_status ifgf_gmres(ifgf_plan plan, const void* b, void* x, const double* alpha, const double* beta,
                       const void* weights, int32_t restart, int32_t max_iters, double tol, void* stream,
                       int32_t* iters, double* rel_residual);

/*
 * Distribution over several GPUs (Sec. 3.2), one rank per GPU.
 *
 * ifgf_partition_boxes: the Morton-ordered leaf boxes in nranks intervals with point counts as
 *   close as possible to N / nranks (Sec. 3.2.1): bound r is the box boundary whose point offset
 *   box_start[b] is nearest to r N / nranks (the lower one on a tie), non-decreasing; rank r owns
 *   boxes [out_bounds[r], out_bounds[r+1]).  box_start: host, [nbox + 1] sorted point offsets
 *   (box_start[0] = 0, non-decreasing); out_bounds: host, [nranks + 1].  Host only.
 * ifgf_partition_cones: a level's nc relevant cones, in the cone order of Sec. 3.2.1, in nranks
 *   contiguous intervals of nearly equal size (co-centred cones may fall to different ranks):
 *   out_bounds[r] = floor(r nc / nranks).  Host only.
 * Errors: IFGF_ERR_INVALID_ARG for NULL arrays, nranks < 1, nbox < 1 or nc < 0, or ranges that do
 * not start at 0 or decrease.
 */
ifgf_status ifgf_partition_boxes(const int64_t* box_start, int64_t nbox, int32_t nranks, int64_t* out_bounds);
ifgf_status ifgf_partition_cones(int64_t nc, int32_t nranks, int64_t* out_bounds);

typedef struct ifgf_shard_s* ifgf_shard;
/*
 * One rank's part of a plan (Sec. 3.2): it owns the points of an interval of leaf boxes and, at
 * every level, an interval of the relevant cones (the partitions above), and it holds
 * coefficients only for its own cones and for the cones of other ranks its steps read.  Those are
 * the cones its points look up in Interpolation(d) and the child cones its parent cones look up in
 * Propagation(d) (Algorithms 7 and 8 restricted to the rank; the data of the paper's two
 * communication algorithms).  Every rank builds the same plan from the same points; the shard
 * borrows it (the plan must outlive the shard and must not be applied while shard steps run).
 * Mixed-precision plans, up to max_nrhs <= 3 value sets per step.  Synchronous.
 *
 * An apply on a rank runs, on `stream`:
 *   ifgf_shard_near_leaf   the near field of its points and LevelDEvaluations of its level-D cones;
 *   for d = D .. 3:
 *     (the caller fills the level-d blocks of the cones in IFGF_SQ_NEED_CONES, in that order,
 *      after the rank's own blocks in ifgf_shard_coefficients' buffer, from their owners'
 *      buffers: ifgf_shard_pack on the owner, then any transport)
 *     ifgf_shard_level(d)  Interpolation(d) of its points, then (d > 3) Propagation(d) of its
 *                          level-(d-1) cones into its own level-(d-1) blocks.
 * Densities and results are [nrhs][N] complex64 vectors in the sorted point order (ifgf_permute
 * converts); a rank reads the densities of its points and of IFGF_SQ_NEED_POINTS, and writes the
 * results of its own points only (the near field sets them, the levels add to them).  A rank's
 * results are bit-identical to those of ifgf_apply on the same points.
 *
 *   ifgf_shard_create       plan, nranks >= 1, 0 <= rank < nranks, 1 <= max_nrhs <= 3.
 *   ifgf_shard_query        as ifgf_plan_query, with the IFGF_SQ_* items below.
 *   ifgf_shard_coefficients device pointer of the level's buffer (own blocks, then the needed
 *                           ones) and the bytes of one cone block at nrhs value sets.
 *   ifgf_shard_pack         dst (device) <- the rank's own level blocks of the n cones ids
 *                           (device, int64, each within the rank's own interval), in that order.
 *   ifgf_shard_unpack       the n blocks at src (device) become needed cones first .. first + n - 1
 *                           (positions in IFGF_SQ_NEED_CONES) of the level's buffer.
 * Errors: IFGF_ERR_INVALID_ARG (NULL handle or buffer, rank, level or nrhs out of range),
 * IFGF_ERR_UNSUPPORTED (an FP64 plan), IFGF_ERR_OOM, IFGF_ERR_CUDA, and IFGF_ERR_INTERNAL from
 * ifgf_shard_create when a lookup finds no relevant cone.
 */
enum {
    IFGF_SQ_POINTS = 0,         /* [2] first and end sorted point of the rank */
    IFGF_SQ_BOXES = 1,          /* [2] first and end leaf box of the rank */
    IFGF_SQ_CONES = 2,          /* [2] first and end relevant cone of the rank at `level` */
    IFGF_SQ_NEED_CONES = 3,     /* [m] cones of other ranks read at `level`, ascending */
    IFGF_SQ_NEED_POINTS = 4,    /* [m] sorted points of other ranks read, ascending */
    IFGF_SQ_POINT_BOUNDS = 5,   /* [nranks + 1] sorted point intervals of all ranks */
    IFGF_SQ_CONE_BOUNDS = 6,    /* [nranks + 1] cone intervals of all ranks at `level` */
    IFGF_SQ_LOOKED_INTERP = 7,  /* [m] cones the rank's Interpolation(level) looks up (own ones too) */
    IFGF_SQ_LOOKED_PROP = 8     /* [m] cones the rank's Propagation(level) looks up (own ones too) */
};
ifgf_status ifgf_shard_create(ifgf_plan plan, int32_t nranks, int32_t rank, int32_t max_nrhs, ifgf_shard* out);
ifgf_status ifgf_shard_query(ifgf_shard shard, int32_t what, int32_t level, int64_t* host_buf, int64_t* inout_count);
ifgf_status ifgf_shard_coefficients(ifgf_shard shard, int32_t level, int32_t nrhs, void** buf, int64_t* block_bytes);
ifgf_status ifgf_shard_pack(ifgf_shard shard, int32_t level, int32_t nrhs, const int64_t* ids, int64_t n, void* dst,
                            void* stream);
ifgf_status ifgf_shard_unpack(ifgf_shard shard, int32_t level, int32_t nrhs, const void* src, int64_t first, int64_t n,
                              void* stream);
ifgf_status ifgf_shard_near_leaf(ifgf_shard shard, const void* dens_sorted, int32_t nrhs, void* out_sorted,
                                 void* stream);
ifgf_status ifgf_shard_level(ifgf_shard shard, int32_t level, int32_t nrhs, void* out_sorted, void* stream);
ifgf_status ifgf_shard_destroy(ifgf_shard shard);

/*
 * Reorder [nrhs][N] complex vectors of the plan's precision (complex64 MIXED, complex128 FP64)
 * between the caller's point order and the plan's sorted order (Sec. 3.2.1): to_sorted != 0 gives
 * out[r][i] = in[r][perm[i]], else out[r][perm[i]] = in[r][i].  Device buffers, asynchronous on
 * `stream`; out must not alias in.  Errors: IFGF_ERR_INVALID_ARG.
 */
ifgf_status ifgf_permute(ifgf_plan plan, const void* in, int32_t nrhs, void* out, int32_t to_sorted, void* stream);

/* Text of a status code, and the calling thread's last error detail. */
const char* ifgf_status_string(ifgf_status s);
const char* ifgf_last_error(void);

/* Number of kernels this library has launched in this process (all plans). */
int64_t ifgf_launch_count(void);

/*
 * Device memory of plans comes from one stream-ordered memory pool per device owned by this
 * library; memory freed by ifgf_plan_destroy stays cached in the pool (up to a quarter of the
 * device's memory) for the next plan.  This call returns every cached, unused byte of the pools
 * to the device.  It synchronises each device that has a pool; plans remain valid.
 */
ifgf_status ifgf_release_cached_memory(void);

/*
 * Opt-in live timing of the hot kernels: while enabled, every launch of a timed kernel is
 * bracketed by CUDA events on its own stream.  ifgf_timing_collect waits for the recorded
 * events, writes per-kind totals (milliseconds, launch counts) into ms[IFGF_TIMING_KINDS] /
 * launches[IFGF_TIMING_KINDS] (either may be NULL) and resets them.  Kinds: 0 permutations,
 * 1 near field, 2 leaf evaluation, 3 propagation into levels with node tables, 4 interpolation,
 * 5 whole plan construction, 6 propagation into levels without node tables (the kernels compute
 * each node's geometry; every FP64 propagation).
 */
#define IFGF_TIMING_KINDS 7
void ifgf_timing_enable(int32_t on);
ifgf_status ifgf_timing_collect(double* ms, int64_t* launches);

/*
 * Fault injection for tests.  Neither call is needed in normal use.
 *
 * ifgf_debug_fail_allocation(n): for n >= 1, the n-th device allocation the library makes from
 * now on (in any plan) fails as if the device were out of memory, once; n = 0 turns the hook
 * off.  The failing call returns IFGF_ERR_OOM after releasing everything it had allocated.
 *
 * ifgf_debug_drop_cone(plan, level, cone): removes relevant cone `cone` (an index of
 * IFGF_Q_CONE_BOX at `level`) from the level's dense cone table, so that every lookup of it by
 * the apply misses.  The kernels then treat its coefficients as zero and record
 * IFGF_ERR_INTERNAL in the plan's status (ifgf_plan_query(IFGF_Q_STATUS)); no memory outside
 * the plan's buffers is touched.  The plan stays usable but its results are no longer those of
 * the method.  Synchronous.  Errors: IFGF_ERR_INVALID_ARG (NULL plan, level or cone out of
 * range), IFGF_ERR_UNSUPPORTED (the level keeps sorted cone lists instead of a dense table).
 */
void ifgf_debug_fail_allocation(int64_t n);
ifgf_status ifgf_debug_drop_cone(ifgf_plan plan, int32_t level, int64_t cone);

/*
 * Checked builds (compiled with -DIFGF_CHECKS; the Python binding loads one when IFGF_CHECKS=1):
 * every cone lookup tests its box and the cone it returns, the interpolation tests every cousin
 * box it reads, and ifgf_plan_create validates every index list of the plan (ranges, offsets,
 * table segments) before returning; a failed test records IFGF_ERR_INTERNAL in the plan's status
 * word (ifgf_plan_create returns it) and the access is skipped, so the device never traps.
 * ifgf_checked_build returns 1 in such a build, 0 otherwise.
 * ifgf_debug_corrupt_cousin(plan, level), in checked builds only, replaces the first cousin of the
 * level's first box that has one by a box index past the level's boxes, so that the next apply's
 * checks report it (IFGF_ERR_UNSUPPORTED in other builds, where it would be read out of bounds).
 */
int32_t ifgf_checked_build(void);
ifgf_status ifgf_debug_corrupt_cousin(ifgf_plan plan, int32_t level);

/*
 * Allocation-free Morton order of N points.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory when they need the order, because
 * their device memory is wholly owned by another allocator (a framework's caching pool or an
 * arena reserved up front) or because cudaMalloc/cudaFree, which can synchronise the device
 * and fail under memory pressure, are not acceptable in their loop.
 *
 * It computes what ifgf_plan_create computes first: the root cube, the level-21 Morton keys
 * and the stable key sort (ties by the caller's index), so perm and keys equal
 * IFGF_Q_PERM / IFGF_Q_KEYS of a plan built from the same points.
 *
 *   points  device, 3*N doubles, x[0..N), y[0..N), z[0..N).  Read only.
 *   N       2 <= N <= IFGF_NOALLOC_MAX_POINTS; larger N returns IFGF_ERR_INVALID_ARG.
 *   perm    device, int32[N], output: sorted position -> caller index.
 *   keys    device, uint64[N], output: sorted keys.
 *   stream  cudaStream_t as void*.
 *
 * Memory: it calls no allocation routine.  Its scratch is one static device array of
 * about 12.6 MB (second sort buffers for 2^20 points, digit histograms, bounding-box partials)
 * that every device which loads this library holds until the process exits.  The first call
 * on a device looks up that array's device address (cudaGetSymbolAddress, with the device
 * current); make that first call before any stream capture.  All calls share the array and
 * each call overwrites what it reads, so calls that overlap on the GPU (two streams, or two
 * host threads) race and must be serialised by the caller.  Every call synchronises `stream`:
 * it returns after the bounding box has been read back to the host, with the keys and the
 * sort queued on `stream` behind it.  The device address found by the first call is kept for
 * the life of the process; after a cudaDeviceReset it is stale, so this entry point must not
 * be used on a device that has been reset.  A CUDA error left pending by the caller's earlier
 * work (cudaGetLastError) is cleared on entry.
 * Errors: IFGF_ERR_INVALID_ARG (NULL pointer, N out of range, non-finite coordinate, all
 * points coincident), IFGF_ERR_CUDA.
 */
#define IFGF_NOALLOC_MAX_POINTS (1 << 20)
ifgf_status ifgf_morton_order_noalloc(const double* points, int64_t N, int32_t* perm, uint64_t* keys, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* IFGF_H */
