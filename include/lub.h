/*
 * liblub -- lubrication corrections for near-contact spheroids, spheres and
 * plane walls, after Janoschek, Harting & Toschi, "Accurate lubrication
 * corrections for spherical and non-spherical particles in discretized fluid
 * simulations" (arXiv:1308.6482), on one NVIDIA GB300 GPU (sm_103a).
 *
 * The correction of one step is four calls, enqueued in order on one CUDA
 * stream:
 *
 *   lub_pairs_build     candidate pairs (Sec. III A pre-filters)
 *   lub_closest_points  closest points, normal and signed gap (Sec. III A)
 *   lub_resistance      curvatures, K~ and the pair force/torque
 *                       (Sec. III B, Eqs. lub:resistance-correction,
 *                       lub:model and the Appendix)
 *   lub_apply           per-particle force and torque (Sec. III B)
 *
 * Conventions shared by every call
 *   - Every array argument is DEVICE memory owned by the caller, unless the
 *     argument's comment says "host".  The library never frees, resizes or
 *     keeps caller memory beyond the call.
 *   - Calls only enqueue work on `stream` (a cudaStream_t passed as void*;
 *     NULL = the legacy default stream) and return without synchronising,
 *     except where a host-side output is requested (stated per call).
 *   - Particle arrays are structure-of-arrays with n entries each.  The
 *     quaternion is scalar-first; the particle's body z axis is its axis of
 *     rotational symmetry (semi-axis r_par); body x and y carry r_perp
 *     (Eq. lub:spheroid).  The rotation used is that of q/|q|.
 *   - Per-pair arrays are structure-of-arrays with `capacity` entries per
 *     component: component c of pair k is at [c * capacity + k].
 *   - Pair k processes pair_i[k] and pair_j[k]; pair_j[k] = -1 - w denotes
 *     plane wall w.  Calls that take d_count process min(*d_count, capacity)
 *     pairs, reading *d_count on the device (no host round trip).
 *   - Return value: LUB_OK (0) or a negative LUB_ERR_* code; lub_last_error()
 *     returns a message for the context's last failure.  No call aborts,
 *     exits or traps the GPU.  Problems of one pair (overlap, no convergence,
 *     bad index or shape) go to that pair's status byte, not the return code.
 *   - Units are lattice units; mu = rho nu (1/6 at tau = 1, Sec. II).
 *   - Thread safety: one context per host thread, or external locking.
 */
#ifndef LUB_H
#define LUB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define LUB_OK            0
#define LUB_ERR_ARG      (-1) /* invalid argument (null pointer, size, domain) */
#define LUB_ERR_CAPACITY (-2) /* more candidate pairs than capacity */
#define LUB_ERR_CUDA     (-3) /* a CUDA runtime call failed */
#define LUB_ERR_TIMEOUT  (-4) /* a bounded device wait ran out */
#define LUB_ERR_NOMEM    (-5) /* the context could not allocate its scratch */
#define LUB_ERR_LIMIT    (-6) /* input larger than a fixed limit of lub_pairs_build_static */
#define LUB_ERR_INTERNAL (-7) /* a kernel's own range check failed: a defect of the library; the
                                 call's outputs are invalid (reported by lub_pairs_build) */

/* lub_params.precision */
#define LUB_FP64  0 /* every step in double precision */
#define LUB_MIXED 1 /* FP32 Newton, curvature, K~ and sums; for every pair
                       the gap and one float-float Newton step of the normal
                       (~48 bits, on the FP32 pipe) and the normal relative
                       surface velocity in float-float; a pair whose FP32
                       Newton did not converge is solved again in FP64 */

/* lub_params.warm_start */
#define LUB_WARM_NONE     0 /* Newton starts from the line of centres (Sec. III A) */
#define LUB_MODEL_FULL 0
#define LUB_MODEL_NORMAL 1
#define LUB_WARM_PREVIOUS 1 /* Newton starts from the normal passed in n (in/out) */
#define LUB_WARM_MLP      2 /* every FP64 Newton solve starts from the learned
                               network's prediction (lub_mlp_set must have
                               installed a network): in LUB_FP64 every pair's;
                               in LUB_MIXED the FP32 stage starts from the line
                               of centres and only the pairs it fails (solved
                               again in FP64) start from the network, since an
                               FP32 iteration costs less than the network */
#define LUB_WARM_MLP_ALL  3 /* every Newton solve starts from the network's
                               prediction, the FP32 stage of LUB_MIXED too (the
                               same as LUB_WARM_MLP in LUB_FP64) */

/* per-pair status bits */
#define LUB_ST_OVERLAP    1  /* h <= 0 */
#define LUB_ST_NOCONV     2  /* Newton did not converge within max_newton */
#define LUB_ST_DEGENERATE 4  /* bad index, non-positive or non-finite shape, coincident centres */
#define LUB_ST_FP64       8  /* mixed mode: the FP32 Newton did not converge and
                                 the pair was solved again in FP64 */

typedef struct lub_ctx lub_ctx;

typedef struct {
    const double *x, *y, *z;          /* centre r_i                        [n] */
    const float *qw, *qx, *qy, *qz;   /* orientation quaternion            [n] */
    const float *r_par, *r_perp;      /* semi-axes R_par, R_perp (> 0)     [n] */
    const float *vx, *vy, *vz;        /* translational velocity v_i        [n] */
    const float *wx, *wy, *wz;        /* angular velocity omega_i          [n] */
    int32_t n;                        /* number of particles (>= 0)            */
    float max_semi_axis;              /* upper bound of max(r_par, r_perp) over
                                         all particles; used by lub_pairs_build
                                         to size its cell grid.  0 = the call
                                         computes it (one stream synchronise) */
    const int32_t *batch_offsets;     /* ensemble mode (no counterpart in the
                                         paper, which treats one suspension):
                                         HOST array [n_batches + 1]; suspension b
                                         owns particles [batch_offsets[b],
                                         batch_offsets[b + 1]), offsets
                                         non-decreasing from 0 to n.  NULL: one
                                         suspension (n_batches ignored)          */
    int32_t n_batches;                /* number of suspensions (>= 1) when
                                         batch_offsets is set                    */
} lub_particles;

typedef struct {
    double L[3];          /* box edge lengths; positions need not be wrapped     */
    int32_t periodic[3];  /* 1 = periodic along that axis (minimum image)        */
    int32_t n_walls;      /* 0, 1 or 2 plane walls normal to z                    */
    double wall_z[2];     /* wall w is the plane z = wall_z[w]                    */
    int32_t wall_dir[2];  /* +1: fluid on the z > wall_z side, -1: z < wall_z     */
} lub_domain;

typedef struct {
    double mu;            /* dynamic viscosity (1/6 at tau = 1)                      */
    double delta_n;       /* cut-off of K33 (Eq. results:cutoffs: 2/3)                */
    double delta_t;       /* cut-off of the other translational elements (1/2)       */
    double delta_r;       /* cut-off of K44, K45, K54, K55 (1/4)                      */
    double h_c;           /* contact cut-off of Eq. lub:model (0 = none: h <= 0 pairs
                             contribute nothing and are flagged OVERLAP)               */
    double eps_c;         /* stiffness of the Hookean repulsion, Eq. lub:frep         */
    double list_cutoff;   /* Delta_L: pairs with a possible gap below this are listed */
    int32_t precision;    /* LUB_FP64 or LUB_MIXED                                     */
    double fp64_switch;   /* reserved (kept for the layout): mixed mode refines
                             every pair's normal beyond FP32, since the force
                             bound needs it at every gap                          */
    int32_t max_newton;   /* Newton iteration cap per precision stage (1..64)          */
    double newton_tol;    /* step-size tolerance (radians) of the FP32 stage: Newton
                             stops after a step shorter than this (quadratic
                             convergence leaves an error of order tol^2); an FP64
                             solve stops after a step below 1e-7 rad              */
    int32_t warm_start;   /* LUB_WARM_NONE, LUB_WARM_PREVIOUS or LUB_WARM_MLP          */
    int32_t model;        /* LUB_MODEL_FULL: all 16 elements of K~; LUB_MODEL_NORMAL:
                             the normal element K~33 alone ("normal only" of Sec.
                             IV C; for two spheres Ladd's Eq. methods:llub)        */
} lub_params;

/* Ensemble mode.  With particles.batch_offsets set, the particle arrays hold
 * n_batches independent suspensions back to back and every call taking a
 * lub_domain reads dom[0 .. n_batches-1] (host memory), the box and walls of
 * each suspension.  Pairs never cross suspensions; pair lists carry global
 * particle indices, and a wall pair (i, -1 - w) names wall w of i's
 * suspension.  Each stage runs as one launch over all suspensions, so an
 * ensemble step costs the same number of launches as one suspension.  The
 * library keeps device copies of the per-suspension tables in the context and
 * uploads them (one stream synchronise) only when they change; a call whose
 * tables differ from the previous call's fails with LUB_ERR_ARG while the
 * stream is being captured into a CUDA graph.  A captured graph replays with
 * the context's current tables and scratch: make one eager call of the
 * largest ensemble before capturing. */

/* Fill *p with the paper's values: mu = 1/6, Delta_n = 2/3, Delta_t = 1/2,
 * Delta_r = 1/4 (Eq. results:cutoffs), h_c = eps_c = 0, list_cutoff = 1,
 * LUB_MIXED, fp64_switch = 1e-3, max_newton = 32, newton_tol = 1e-4,
 * LUB_WARM_NONE, LUB_MODEL_FULL. */
void lub_default_params(lub_params *p);

/* Waits for the stream, then reports whether a bounded device wait of any
 * call on this context timed out since the previous lub_sync_status (the
 * look-back of a scan in lub_pairs_build or deterministic lub_apply, an
 * mbarrier wait of the tcgen05 network), and clears that record.  A wait
 * that runs out sets a bit in the context's device status word and returns
 * instead of spinning on; the results of that call are then unreliable.
 * No counterpart in the paper.  Errors: LUB_ERR_TIMEOUT, LUB_ERR_CUDA,
 * LUB_ERR_ARG. */
int lub_sync_status(lub_ctx *ctx, void *stream);

/* Create a context (library-owned scratch, grown on demand by the calls that
 * need it: lub_pairs_build and deterministic lub_apply).  *ctx receives the
 * handle.  Errors: LUB_ERR_ARG (ctx NULL), LUB_ERR_NOMEM. */
int lub_ctx_create(lub_ctx **ctx);

/* Free the context and its device scratch (synchronises the device first). */
int lub_ctx_destroy(lub_ctx *ctx);

/* Message for the context's last error ("" if none); valid until the next
 * call on the same context.  ctx may be NULL (returns a generic message). */
const char *lub_last_error(const lub_ctx *ctx);

/*
 * Candidate pairs (Sec. III A).  A pair (i, j), i < j, is listed unless
 *   r_ij > Rmax_i + Rmax_j + Delta_L, or
 *   r_ij - sigma_i(r^_ij) > Rmax_j + Delta_L, or r_ij - sigma_j(r^_ij) > Rmax_i + Delta_L,
 * where r_ij is the minimum-image centre distance, Rmax = max(r_par, r_perp)
 * and sigma_k(e) the half-width of particle k along e (the plane test of
 * Sec. III A, with R_c = Rmax + Delta_L for particles of different size).
 * Particle w-wall pair (i, -1-w) is listed when the exact gap
 * wall_dir (z_i - wall_z) - sigma_i(e_z) < Delta_L.  The decisions are those
 * of double precision arithmetic: FP32 tests with a margin of 1e-5 (2 Rmax +
 * Delta_L + 1); every candidate inside that margin is tested again in
 * float-float (margin 1e-10 of the reach plus 3e-14 of the coordinates'
 * magnitude), and inside that margin in FP64.
 *
 * Order: particle pairs by (i, j) ascending, then wall pairs by (i, w).
 * Writes pair_i[k], pair_j[k] for k < min(count, capacity) and *d_count =
 * count (device int32).  The arrays also serve as the overflow store of the
 * build (pairs beyond 16 per particle, and, for inputs with more candidates
 * on the filters' edges than particles, the excess of those waiting for their
 * FP64 test; kept at their tail while it runs), so the call needs capacity
 * >= count + overflow entries, which is count for any ordinary suspension;
 * when that does not hold, *d_count receives the
 * sum (> capacity), the listed content is unspecified and the call returns
 * LUB_ERR_CAPACITY when h_count_or_null is given (host int32, receives that
 * required capacity; the call then synchronises `stream`).  A bounded wait
 * inside the build that times out gives LUB_ERR_TIMEOUT on that path.
 * Without h_count_or_null the call does not synchronise (unless
 * max_semi_axis is 0) and overflow is visible only through *d_count.
 * Periodic axes need L >= 2 (2 Rmax + Delta_L), and n <= 429,496,524 (five
 * sweep items per particle, indexed in int32) (else LUB_ERR_ARG).
 * Uses context scratch (cell grid, counts), grown with cudaMalloc as needed.
 */
int lub_pairs_build(lub_ctx *ctx, const lub_particles *p, const lub_domain *dom,
                    const lub_params *prm, int32_t *pair_i, int32_t *pair_j, int32_t capacity,
                    int32_t *d_count, int32_t *h_count_or_null, void *stream);

/*
 * Closest points and signed gap (Sec. III A, with the overlap extension).
 * For each pair, n* maximises g(n) = n.d - sigma_i(n) - sigma_j(n) over unit
 * n (d = minimum-image r_j - r_i), solved by Newton iteration on the sphere
 * from n = d/|d| (the paper's line-of-centres start), with
 * LUB_WARM_PREVIOUS from the n passed in, or with LUB_WARM_MLP from the
 * installed network's prediction (lub_mlp_set).  Outputs:
 *   n     [3][capacity] double: unit outward normal of i at y*_i (points i -> j)
 *   gap   [capacity] double: h = g(n*) (< 0 for overlap); y*_j - y*_i = h n
 *   status[capacity] uint8: LUB_ST_* bits
 *   iters [capacity] uint8: Newton iterations taken (the FP32 stage; the FP64 solve for a LUB_ST_FP64 pair), or NULL
 * Walls and two spheres use their closed forms (0 iterations).
 * y*_i = r_i + M_i n / sigma_i(n), y*_j = r_j - M_j n / sigma_j(n), with
 * M = Q diag(r_perp^2, r_perp^2, r_par^2) Q^T.
 */
int lub_closest_points(lub_ctx *ctx, const lub_particles *p, const lub_domain *dom,
                       const lub_params *prm, const int32_t *pair_i, const int32_t *pair_j,
                       const int32_t *d_count, int32_t capacity, double *n, double *gap,
                       uint8_t *status, uint8_t *iters, void *stream);

/*
 * Pair force and torque (Sec. III B, Eqs. lub:resistance,
 * lub:resistance-correction, lub:frep, lub:model; Appendix).  From n and gap
 * of lub_closest_points: principal directions and radii of curvature and the
 * cubic coefficients at y*_i and y*_j, the combined-gap eigenproblem, the 16
 * elements of K, K~ with the three cut-offs, the clipped gap and Hookean
 * repulsion, the surface velocities V = v + omega x (y* - r), and
 * (F_i, T_i) = mu K~ (V_j - V_i, Omega_j - Omega_i) turned into the lab frame.
 * Outputs (type float for LUB_MIXED, double for LUB_FP64):
 *   FT    [6][capacity]: F_i (lab) and T_i (lab, about y*_i)
 *   lever [6][capacity]: y*_i - r_i and y*_j - r_j (zero for a wall)
 * Pairs whose status has NOCONV or DEGENERATE, and pairs with h <= 0 when
 * h_c = 0 (OVERLAP is then set in status), get zeros.  status is read and
 * updated in place.
 */
int lub_resistance(lub_ctx *ctx, const lub_particles *p, const lub_domain *dom,
                   const lub_params *prm, const int32_t *pair_i, const int32_t *pair_j,
                   const int32_t *d_count, int32_t capacity, const double *n, const double *gap,
                   uint8_t *status, void *FT, void *lever, void *stream);

/*
 * Per-particle force and torque (Sec. III B):
 *   f_i += F_i,  t_i += T_i + (y*_i - r_i) x F_i,
 *   f_j -= F_i,  t_j += -T_i + (y*_j - r_j) x (-F_i)   (Eq. lub:resistance),
 * wall sides dropped.  force, torque: [3][n] of the precision's type
 * (float for LUB_MIXED, double for LUB_FP64).  accumulate = 0 zeroes them
 * first.  deterministic = 1 sums each particle's contributions in a fixed
 * order (pair index, then side), giving bitwise-reproducible results, using
 * context scratch; deterministic = 0 uses atomic adds.
 */
int lub_apply(lub_ctx *ctx, const int32_t *pair_i, const int32_t *pair_j, const int32_t *d_count,
              int32_t capacity, const void *FT, const void *lever, int32_t n, void *force,
              void *torque, int32_t precision, int32_t accumulate, int32_t deterministic,
              void *stream);

/*
 * Learned warm start of lub_closest_points (no counterpart in the paper: the
 * paper warm-starts from the previous time step, Sec. III A).  A network
 * 12 -> 128 -> 128 -> 4 with GELU activations maps a pair's relative pose to
 * the surface parameters (p_i, q_i, p_j, q_j) of Eq. lub:spheroid at its
 * closest points, as corrections to the parameters of the line-of-centres
 * start; the outward normals at the predicted points give Newton's start.
 *
 * Features (12 per pair): d = r_j - r_i (minimum image) in i's body frame over
 * R_perp,i (3); the relative rotation q_i^-1 q_j of the normalised
 * quaternions with w >= 0 (4); ln R_par,i, ln R_perp,i, ln R_par,j,
 * ln R_perp,j (4); asinh(g/a) with g = |d| - sigma_i(d^) - sigma_j(d^) and a
 * the smallest semi-axis (1); standardised as (f - mean) * istd.
 * Parameters: LUB_MLP_PARAMS floats [W1 | b1 | W2 | b2 | W3 | b3], W row-major
 * [out][in] (W1 128x12, W2 128x128, W3 4x128).
 */
#define LUB_MLP_PARAMS 18692
#define LUB_MLP_WORK_PER_SAMPLE 776

/* Install a network in the context (BF16 copy of params for the tensor
 * cores; mean, istd: device [12]).  params, mean, istd: device float.  The
 * first call allocates the context's copy. */
int lub_mlp_set(lub_ctx *ctx, const float *params, const float *mean, const float *istd, void *stream);

/* Tensor-core path of the network (no counterpart in the paper):
 * LUB_MLP_MMA_SYNC (default) runs it with warp-level mma.sync, one warp per
 * 32 pairs, activations in registers; LUB_MLP_TCGEN05 with tcgen05.mma, 128
 * pairs per CTA, accumulators in tensor memory, operands staged in shared
 * memory (weights by one bulk copy per CTA).  Same results up to the order
 * of the FP32 accumulation.  With LUB_MLP_MMA_SYNC, lub_closest runs the
 * network inside its own kernel (each warp infers the start normals of its
 * 32 pairs and solves them in the same launch); with LUB_MLP_TCGEN05 the
 * network is a launch of its own before the solve.  A bounded wait of the tcgen05 path that times
 * out sets bit 3 (value 8) of the context's flags and ends the kernel. */
#define LUB_MLP_MMA_SYNC 0
#define LUB_MLP_TCGEN05 1
int lub_mlp_engine(lub_ctx *ctx, int32_t engine);

/* The network's outputs for every pair on the tensor cores (BF16 weights and
 * activations, FP32 accumulate): pq [4][capacity] float, the predicted
 * corrections to (p_i, q_i, p_j, q_j) of the line-of-centres start;
 * pairs with a wall, bad indices or non-finite features get zeros. */
int lub_mlp_predict(lub_ctx *ctx, const lub_particles *p, const lub_domain *dom, const int32_t *pair_i,
                    const int32_t *pair_j, const int32_t *d_count, int32_t capacity, float *pq, void *stream);

/* Features of n pairs into feat [n][12] (device float); mean and istd (device
 * [12]) standardise them, or both NULL for the raw features. */
int lub_mlp_features(lub_ctx *ctx, const lub_particles *p, const lub_domain *dom, const int32_t *pair_i,
                     const int32_t *pair_j, int32_t n, const float *mean, const float *istd, float *feat,
                     void *stream);

/* Training step, forward and backward in FP32 on a batch of nb samples:
 * x [nb][12] standardised features, target [nb][4]: the corrections to the
 * surface parameters of the line-of-centres start, (p_i - p0_i,
 * wrap(q_i - q0_i), p_j - p0_j, wrap(q_j - q0_j)) with (p0, q0) those of the
 * support points of i along d^ and of j along -d^ (a zero output gives Newton
 * the line-of-centres start); weight [nb][4] or NULL (all 1).
 * loss = mean over the batch of 1/2 sum_o weight_o r_o^2, the azimuth errors
 * r_1, r_3 wrapped to (-pi, pi].  Writes grads [LUB_MLP_PARAMS] (d loss /
 * d params) and loss_rows [nb] (each sample's loss); work: nb *
 * LUB_MLP_WORK_PER_SAMPLE floats of scratch.  All device memory. */
int lub_mlp_forward_backward(lub_ctx *ctx, const float *params, const float *x, const float *target,
                             const float *weight, int32_t nb, float *grads, float *work, float *loss_rows,
                             void *stream);

/* Adam update of n parameters (step t >= 1) with moments m, v (device). */
int lub_mlp_adam(lub_ctx *ctx, float *params, const float *grads, float *m, float *v, int32_t n, int32_t t, float lr,
                 float beta1, float beta2, float eps, void *stream);

/*
 * The pair build of lub_pairs_build, for callers that cannot allocate device
 * memory.  The paper has no counterpart: this is an interface for host codes
 * that own a fixed device-memory budget and forbid allocation after
 * start-up, for instance because cudaMalloc synchronises the whole device
 * (stalling the other streams of a running simulation) and can fail in the
 * middle of a run.  Such callers cannot create a lub_ctx, so this call
 * takes none.
 *
 * It computes exactly what lub_pairs_build computes (same arguments, same
 * output order and *d_count), on a scratch array of LUB_STATIC_SCRATCH_BYTES
 * bytes that is a static device array of the library: every GPU that loads
 * the library holds it until the process exits.  It calls no cudaMalloc,
 * cudaFree or other allocating routine.  The caller still provides pair_i,
 * pair_j and d_count.
 *   - Limits: p->n <= LUB_STATIC_MAX_PARTICLES (else LUB_ERR_LIMIT, nothing
 *     enqueued); the cell grid is coarsened to at most LUB_STATIC_MAX_CELLS
 *     cells; p->max_semi_axis must be given (> 0, else LUB_ERR_ARG).
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current) and caches it; make
 *     that first call before any stream capture.
 *   - All calls share the array, which keeps the last call's contents (the
 *     call clears what must start at zero).  Calls whose work overlaps on the
 *     GPU, e.g. on two streams at once, race on it: serialise them.
 *   - Errors are return codes only (no context, no message).  Overflow of
 *     capacity is visible through *d_count only.
 */
#define LUB_STATIC_MAX_PARTICLES 65536
#define LUB_STATIC_MAX_CELLS     262144
#define LUB_STATIC_SCRATCH_BYTES 9437184
int lub_pairs_build_static(const lub_particles *p, const lub_domain *dom, const lub_params *prm,
                           int32_t *pair_i, int32_t *pair_j, int32_t capacity, int32_t *d_count,
                           void *stream);

/*
 * lub_resistance and lub_apply (atomic form) in one pass over the pairs: the
 * pair force is scattered to the particles straight from registers (the
 * fast path "write straight to force/torque").  Same arguments as
 * lub_resistance plus force and torque [3][n] (zeroed first unless
 * accumulate is set); FT and lever are written where given and skipped where
 * NULL.  Results as lub_resistance + lub_apply up to the order of the atomic
 * additions.
 */
int lub_resistance_apply(lub_ctx *ctx, const lub_particles *p, const lub_domain *dom, const lub_params *prm,
                         const int32_t *pair_i, const int32_t *pair_j, const int32_t *d_count, int32_t capacity,
                         const double *n, const double *gap, uint8_t *status, void *FT, void *lever, void *force,
                         void *torque, int32_t accumulate, void *stream);

/*
 * One call for the per-pair work of a step: lub_closest_points, lub_resistance
 * and lub_apply (atomic form) on the same arguments (Sec. III A, III B, Eq.
 * lub:resistance).
 *   - LUB_FP64: one pass over the pairs, each pair's closest points, gap and
 *     resistance staying in registers; the results are those of the three
 *     calls up to rounding (the same arithmetic, which the compiler may
 *     contract into multiply-adds differently inside the one kernel; the
 *     particle sums also add in another order).
 *   - LUB_MIXED: the kernels of lub_closest_points followed by those of
 *     lub_resistance_apply, on one set of per-call particle records (built
 *     once instead of once per call); the results are those of the two calls,
 *     the particle sums up to the order of the atomic additions.
 * n [3][cap] is required: it holds the start normals of a warm start
 * (LUB_WARM_PREVIOUS, LUB_WARM_MLP_ALL, LUB_WARM_MLP) and receives the
 * normals.  gap, status, iters, FT and lever are written where given and
 * skipped where NULL (in LUB_MIXED the context scratch holds gap and status
 * between the kernels when they are NULL).  force and torque [3][n] (float in
 * LUB_MIXED, double in LUB_FP64) are zeroed first unless accumulate is set.
 * Ensemble mode as for the separate calls.
 */
int lub_correct(lub_ctx *ctx, const lub_particles *p, const lub_domain *dom, const lub_params *prm,
                const int32_t *pair_i, const int32_t *pair_j, const int32_t *d_count, int32_t capacity, double *n,
                double *gap, uint8_t *status, uint8_t *iters, void *FT, void *lever, void *force, void *torque,
                int32_t accumulate, void *stream);

/*
 * Temporal warm start (Sec. III A: the paper starts each time step's
 * closest-point search from the previous step's solution).  For every pair
 * of the current list, copies into n [3][capacity] the normal that the
 * previous list (prev_i, prev_j, prev_n [3][prev_capacity], *prev_count
 * pairs, device) holds for the same pair (i, j) or wall pair (i, w), and
 * zero where the pair is new; lub_closest_points with warm_start =
 * LUB_WARM_PREVIOUS then starts Newton there (a zero or far-side start falls
 * back to the line of centres).  Both lists must be in the canonical order of
 * lub_pairs_build and index particles below n_particles; the current list
 * must not alias the previous one.  Works unchanged on ensemble lists (global
 * indices).  Asynchronous; context scratch of 8 bytes per particle (the
 * range of each particle's pairs in the previous list).
 */
int lub_carry_normals(lub_ctx *ctx, int32_t n_particles, const int32_t *prev_i, const int32_t *prev_j,
                      const double *prev_n, const int32_t *prev_count, int32_t prev_capacity, const int32_t *pair_i,
                      const int32_t *pair_j, const int32_t *d_count, int32_t capacity, double *n, void *stream);

/*
 * Link-based lubrication of Ding and Aidun (Sec. II, Eq. methods:dlub), the
 * correction the paper compares against, on a synthetic lattice: lattice
 * sites are the integer points of the box coordinates (spacing 1) and a site
 * belongs to a particle when it lies in or on its spheroid.  For every pair
 * (i, j) of the list and every D3Q19 link c_r (the 18 nonzero lattice
 * vectors, c_r = 1 or sqrt 2) that ends on a site of i and stems from a site
 * of j (not also in i), or from a fluid site (in neither particle) midway
 * along 2 c_r from a site of j, the partial force
 *   df = -3 q_bar mu / (2 c_r^2 lambda*) c^ (c^.(v_bi - v_bj)) (1/h*^2 - 1/c_r^2)
 * acts on i where 0 < h* < c_r, and -df on j.  h*: the distance along the
 * link(s) from where it leaves j's surface to where it enters i's; v_b: the
 * rigid-body velocities there; lambda*: the mean of the two surfaces' mean
 * curvatures there; j is taken at its minimum image from i.  Outputs, per
 * pair k (device arrays the caller owns):
 *   force   [3][capacity] double: the sum of df on i
 *   torque  [6][capacity] double: torque on i, then on j, about the centres
 *   n_links [capacity] int32 (may be NULL): the links that contributed
 * Wall pairs (j < 0) and invalid pairs give zeros.  mu is prm->mu; q_bar the
 * empirical weight (0.6 in the paper); the particles need v and w.  One warp
 * per pair; site membership in FP32 with an FP64 re-test near the surface,
 * the qualifying links in FP64.  Asynchronous on `stream`.
 */
int lub_links(lub_ctx *ctx, const lub_particles *p, const lub_domain *dom, const lub_params *prm,
              const int32_t *pair_i, const int32_t *pair_j, const int32_t *d_count, int32_t capacity,
              double q_bar, double *force, double *torque, int32_t *n_links, void *stream);

/*
 * Particle sub-step (Sec. II: the particle update is decoupled from the
 * lattice-Boltzmann step and runs at a fraction of it, typically 1/10, so the
 * strongly varying lubrication forces are followed while the forces from the
 * fluid stay constant over the LB step).  One explicit sub-step of length dt
 * for every particle, in double precision (semi-implicit Euler):
 *   v += dt (F_ext + f) / m;  r += dt v;
 *   L = I_lab w + dt (T_ext + t);  q <- exp(dt w_mid / 2) q with
 *   w_mid = I_lab(q)^-1 L;  w = I_lab(q_new)^-1 L,
 * m = density * 4/3 pi R_par R_perp^2, body inertia I_par = 2/5 m R_perp^2
 * about the symmetry axis and I_perp = 1/5 m (R_par^2 + R_perp^2).
 * force, torque: the lubrication force and torque [3][n] about the centres
 * (lub_apply / lub_resistance_apply output; float for LUB_MIXED, double for
 * LUB_FP64); f_ext, t_ext: [3][n] float or NULL (e.g. the fluid's, constant
 * over the LB step).  Writes x, y, z, the quaternion and the velocities of p
 * in place (they must be writable device memory).  Torque-free motion keeps
 * the angular momentum exactly.
 */
int lub_rigid_step(lub_ctx *ctx, const lub_particles *p, const void *force, const void *torque, int32_t precision,
                   const float *f_ext, const float *t_ext, double density, double dt, void *stream);

/*
 * Seeded random rigid motions (no counterpart in the paper: the input
 * preparation of time-stepped workloads, on the device so that a loop of
 * motions and correction steps can be captured into one CUDA graph).  Every
 * particle k is moved by a displacement with N(0, sigma_r^2) components and
 * rotated by exp(theta / 2) q, theta with N(0, sigma_t^2) components
 * (lattice units, radians).  The six normal draws come from Philox4x32-10
 * (Salmon et al., SC 2011) with counter (k, s, draw) and key seed, by the
 * Box-Muller transform, s = step + *step_dev (step_dev: NULL or a device
 * int64): the same (seed, s) gives the same motion on every call.  next_dev
 * (NULL or a device int64 other than step_dev) receives s + 1, so a graph
 * that captures several calls alternating two counters (step_dev, next_dev
 * = c0, c1, then c1, c0, ...) replays a fresh sequence of motions each time.
 * Writes x, y, z and the quaternion of p in place (writable device memory);
 * asynchronous on stream.  Errors: LUB_ERR_ARG.
 */
int lub_random_motion(lub_ctx *ctx, const lub_particles *p, uint64_t seed, int64_t step, const int64_t *step_dev,
                      int64_t *next_dev, double sigma_r, double sigma_t, void *stream);

/* ---------------------------------------------------------------------------
 * Launch-shape autotuner (no counterpart in the paper).  The tunable kernels
 * are persistent grid-stride loops; their shape is (threads per block, blocks
 * per SM), the grid being min(work / block, blocks_per_sm x SMs).
 * ------------------------------------------------------------------------- */
#define LUB_TUNE_CLOSEST_MIXED 0   /* lub_closest_points, LUB_MIXED, FP32 stage */
#define LUB_TUNE_CLOSEST_REFINE 1  /* lub_closest_points, LUB_MIXED, work list of FP64 solves */
#define LUB_TUNE_CLOSEST_FP64 2    /* lub_closest_points, LUB_FP64 */
#define LUB_TUNE_RESISTANCE 3      /* lub_resistance, lub_resistance_apply (and so
                                      lub_correct in LUB_MIXED) */
#define LUB_TUNE_APPLY 4           /* lub_apply, atomic form */
#define LUB_TUNE_SWEEP 5           /* lub_pairs_build, the cell sweep (one thread per
                                      particle slot: only the block counts, the grid
                                      follows) */
#define LUB_TUNE_COUNT 6

/* Time every candidate shape of the kernels a step with these arguments runs
 * (the four calls, in prm's precision, atomic lub_apply) and keep the fastest
 * in the context; later calls launch with them.  Runs the calls `reps` times
 * per candidate (>= 1), synchronises the stream, and overwrites the pair and
 * output arrays like a step does.  Not capturable: tune before capturing a
 * graph.  The shapes change no result except the order of atomic additions. */
int lub_autotune(lub_ctx *ctx, const lub_particles *p, const lub_domain *dom, const lub_params *prm,
                 int32_t *pair_i, int32_t *pair_j, int32_t capacity, int32_t *d_count, double *n, double *gap,
                 uint8_t *status, uint8_t *iters, void *FT, void *lever, void *force, void *torque, int32_t reps,
                 void *stream);

/* The shape kernel `kernel` (LUB_TUNE_*) launches with; 0 = the built-in
 * default.  lub_set_launch_shape with block = blocks_per_sm = 0 restores it;
 * otherwise block must be one of the kernel's candidates (a multiple of 32 up
 * to its limit: 128 for the closest-point and resistance kernels, 32 for the
 * work-list refinement, 256 for lub_apply and the sweep) and 1 <= blocks_per_sm <= 256. */
int lub_get_launch_shape(const lub_ctx *ctx, int32_t kernel, int32_t *block, int32_t *blocks_per_sm);
int lub_set_launch_shape(lub_ctx *ctx, int32_t kernel, int32_t block, int32_t blocks_per_sm);

/* ---------------------------------------------------------------------------
 * Kernel trace and pipe probes (no counterpart in the paper): measurement
 * support for per-kernel rooflines.
 * ------------------------------------------------------------------------- */
#define LUB_TRACE_SWEEP      0  /* lub_pairs_build: the cell sweep (k_pairs_sweep) */
#define LUB_TRACE_CLOSEST    1  /* lub_closest_points: the solve (FP32 stage, FP64 or learned kernel) */
#define LUB_TRACE_RESISTANCE 2  /* lub_resistance / lub_resistance_apply: the pair-force kernel */
#define LUB_TRACE_APPLY      3  /* lub_apply: the scatter kernel */
#define LUB_TRACE_COUNT      4

/* on != 0: from now on every eager call records a CUDA event on its stream
 * right before and right after each traced kernel (LUB_TRACE_*); nothing is
 * recorded while the stream is being captured into a graph.  The events
 * break the programmatic dependent-launch overlap around the traced kernels,
 * so traced calls are a little slower; the intervals are the kernels' own.
 * on = 0: stop and release the events.  Errors: LUB_ERR_ARG. */
int lub_trace_enable(lub_ctx *ctx, int32_t on);

/* Waits for the events of traced kernel `kernel` recorded since the last
 * read, then returns in *ms_total the sum of their intervals (milliseconds)
 * and in *launches their number, and forgets them.  Blocks the host.
 * Errors: LUB_ERR_ARG, LUB_ERR_CUDA. */
int lub_trace_read(lub_ctx *ctx, int32_t kernel, double *ms_total, int64_t *launches);

#define LUB_PROBE_FP32 0
#define LUB_PROBE_FP64 1
/* Sustained fused-multiply-add throughput of one pipe (LUB_PROBE_FP32 or
 * LUB_PROBE_FP64) at the current clocks, in TFLOP/s (2 FLOP per FMA): eight
 * independent FMA chains per thread, eight blocks of 256 threads per SM,
 * best of three timed launches after one warm-up (about 20 ms each).
 * Synchronises the stream.  Errors: LUB_ERR_ARG, LUB_ERR_CUDA. */
int lub_probe_peak(lub_ctx *ctx, int32_t pipe, double *tflops, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LUB_H */
