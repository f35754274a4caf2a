/*
 * rsot.h -- C ABI of librsot, a GB300 (sm_103a) implementation of the
 * entropy-regularised semi-discrete optimal transport (RSOT) dual evaluation
 * and its solver.
 *
 * Notation (Sec. 2-3 of the paper): quadrature points x_q in R^d with masses
 * m_q = rho_h(x_q) w_q (Remark 3.1), targets y_j with weights nu_j, dual
 * potentials psi in R^N, regularisation eps > 0, cost c(x,y) = |x - y|^2 / 2.
 *
 *   J(psi)        = sum_q m_q eps ln sum_j nu_j exp((psi_j - c(x_q,y_j))/eps)
 *                   - sum_j psi_j nu_j                       (Eq. discretized_functional)
 *   dJ/dpsi_k     = sum_q m_q p_k(x_q|psi) - nu_k            (Eq. discretized_gradient)
 *   p_k(x|psi)    = nu_k e^{(psi_k - c(x,y_k))/eps} / sum_j nu_j e^{(psi_j - c(x,y_j))/eps}
 *                                                            (Eq. final_plan_density)
 *
 * Truncation (Sec. 4.1, Algorithm 2) keeps, for each point, only the targets
 * with c(x_q, y_j) < C, i.e. |x_q - y_j| < radius with radius = sqrt(2 C).
 *
 * Conventions for every entry point
 *   - Array arguments are plain pointers.  Unless a comment says otherwise a
 *     pointer may address host memory or device memory of the current CUDA
 *     device (the library copies with cudaMemcpyDefault); row-major layout;
 *     the caller owns every buffer it passes and keeps ownership.
 *   - Outputs are written only when the call returns RSOT_OK.
 *   - Calls are synchronous with respect to their host-visible outputs and
 *     run on the stream set by rsot_set_stream (default: the legacy stream).
 *   - No call throws; errors are status codes.  A handle is not thread-safe.
 */
#ifndef RSOT_H
#define RSOT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rsot_problem rsot_problem;   /* opaque; owns its device memory */

typedef enum {
    RSOT_OK = 0,
    RSOT_ERR_ARG = 1,                 /* invalid argument (sizes, eps <= 0, null) */
    RSOT_ERR_CUDA = 2,                /* a CUDA runtime call failed              */
    RSOT_ERR_NONFINITE = 3,           /* psi, J or the gradient is not finite     */
    RSOT_ERR_EMPTY_NEIGHBORHOOD = 4,  /* a point had no target within the radius */
    RSOT_ERR_NOT_CONVERGED = 5,       /* the solver hit its iteration cap        */
    RSOT_ERR_LINESEARCH = 6,          /* the line search found no Wolfe step     */
    RSOT_ERR_TIMEOUT = 7,             /* a bounded device-side wait gave up      */
    RSOT_ERR_NOMEM = 8                /* device allocation failed                */
} rsot_status;

typedef enum {
    RSOT_FP64 = 0,        /* every operation in FP64                            */
    RSOT_MIXED = 1,       /* FP32 pair arithmetic (ex2.approx), FP64 reductions  */
    RSOT_COMPENSATED = 2  /* pair exponents as double-float FP32 pairs, ex2.approx,
                             compensated sums: ||g - grad J||_1 <= 6.5e-7 sum m_q
                             (RSOT_COMPENSATED_GRAD_REL), at FP32 throughput     */
} rsot_precision;

/* Bound of ||g - grad J||_1 / sum_q m_q for a gradient g computed with
 * RSOT_COMPENSATED, for any sizes, eps and potentials (the per-term error
 * budget of ex2.approx and of the compensated sums). */
#define RSOT_COMPENSATED_GRAD_REL 6.5e-7

/* Human-readable name of a status code (static string). */
const char *rsot_status_string(rsot_status s);

/* Version string of the library build (static string). */
const char *rsot_version(void);

/*
 * Create a problem: the discrete source measure sum_q m_q delta_{x_q}
 * (Remark 3.1) and the target measure sum_j nu_j delta_{y_j} (Sec. 2).
 *   d      : dimension, 2 or 3
 *   nq     : number of quadrature points, >= 1
 *   x      : nq*d doubles (row-major), mass: nq doubles, m_q >= 0
 *   n      : number of targets, >= 1
 *   y      : n*d doubles (row-major), nu: n doubles, nu_j > 0
 *   device_ptrs : 0 -- the inputs (host or device memory) are copied into
 *               device memory owned by the handle; the caller's buffers may
 *               be freed after the call.
 *               1 -- borrow: x, mass, y, nu must be device memory of the
 *               current device (else RSOT_ERR_ARG).  The handle reads mass
 *               and nu in place at every evaluation instead of copying them,
 *               so they must stay allocated and unchanged until
 *               rsot_destroy; x and y are read once, into the handle's own
 *               translated layouts (the cost is computed in coordinates
 *               centred on the data's bounding box).
 * Sum m_q and sum nu_j are used as given (the paper's normalisation sum = 1
 * is the caller's choice).
 * Errors: RSOT_ERR_ARG, RSOT_ERR_NOMEM, RSOT_ERR_CUDA.
 */
rsot_status rsot_create(int d, int64_t nq, const double *x, const double *mass,
                        int64_t n, const double *y, const double *nu, int device_ptrs,
                        rsot_problem **out);

/* Free every resource of the handle (NULL is accepted). */
void rsot_destroy(rsot_problem *p);

/* Use `stream` (a cudaStream_t; NULL = legacy default stream) for all work. */
rsot_status rsot_set_stream(rsot_problem *p, void *stream);

/*
 * Instruction form of the pair arithmetic of the mixed passes (Algorithm 2's
 * exponent (psi_j - c(x_q, y_j))/eps + ln nu_j).
 *   RSOT_PAIRS_FP32   : FP32 fused multiply-adds for every pair.
 *   RSOT_PAIRS_TENSOR : the exponent as a 16-term inner product on the tensor
 *     cores (mma.sync, f16 head/tail operand pairs, f32 accumulation; its
 *     error is within about twice the FP32 chain's, see below), falling back
 *     to the FP32 kernels by itself, per evaluation, when an operand leaves
 *     the f16 range.  Both passes form bitwise the same exponents.
 *   RSOT_PAIRS_AUTO (the default): every evaluation returned to the caller
 *     (rsot_eval_dual_grad, _tail, the maps) uses the FP32 form; inside
 *     rsot_solve and the batched and multilevel solvers, whose stop is
 *     certified on compensated or FP64 reference evaluations, the mixed
 *     iterations take the tensor-core form while the gradient is far above
 *     its rounding noise.
 * Neither form has a per-entry worst-case bound of 1e-6 at large eps-scaled
 * magnitudes (the FP32 rounding of the per-point shift and of the stage sums,
 * common to both, allows more for a target that collects a few percent of the
 * mass); the mixed tolerances are measured against the FP64 oracle.
 * Not a paper concept: a choice of kernel.
 * Errors: RSOT_ERR_ARG (NULL handle or unknown kind).
 */
typedef enum { RSOT_PAIRS_FP32 = 0, RSOT_PAIRS_TENSOR = 1, RSOT_PAIRS_AUTO = 2 } rsot_pair_kernel;
rsot_status rsot_set_pair_kernel(rsot_problem *p, rsot_pair_kernel kind);

/*
 * One evaluation of J(psi) and grad J(psi) -- Algorithm 2.
 *   psi       : n doubles (host or device)
 *   eps       : regularisation, > 0
 *   radius    : <= 0 or +inf -> dense evaluation over all pairs (Eq.
 *               discretized_functional / discretized_gradient);
 *               > 0 -> truncated: only pairs with |x_q - y_j| < radius
 *               (c < C with C = radius^2/2, Sec. 4.1)
 *   prec      : RSOT_FP64, RSOT_MIXED or RSOT_COMPENSATED (the truncated
 *               form decides membership c < C exactly as the FP64 path)
 *   J_out     : host pointer, 1 double
 *   grad_out  : n doubles (host or device)
 *   pairs_out : host pointer or NULL; receives sum_q |I_q|, the pairs whose
 *               terms entered the sums (nq*n when dense)
 * Errors: RSOT_ERR_ARG, RSOT_ERR_NONFINITE (psi not finite or J/grad not
 * finite), RSOT_ERR_EMPTY_NEIGHBORHOOD (truncated and some point kept no
 * target: Algorithm 2 skips such points; the outputs are not written, and
 * rsot_last_eval returns the evaluation with those points skipped),
 * RSOT_ERR_TIMEOUT, RSOT_ERR_CUDA.  On any error J_out, grad_out and
 * pairs_out are left untouched.
 */
rsot_status rsot_eval_dual_grad(rsot_problem *p, const double *psi, double eps,
                                double radius, rsot_precision prec,
                                double *J_out, double *grad_out, int64_t *pairs_out);

/*
 * Results of the last evaluation on this handle whose passes completed: the
 * last one that returned RSOT_OK, or one that returned
 * RSOT_ERR_EMPTY_NEIGHBORHOOD, whose points without a target Algorithm 2
 * skipped (their terms are absent from J and the gradient).
 *   J_out, pairs_out, empty_out : host pointers or NULL; empty_out receives
 *               the number of skipped points (0 when dense)
 *   grad_out  : n doubles (host or device) or NULL
 * Errors: RSOT_ERR_ARG when no evaluation has completed on this handle (or
 * another call, such as rsot_softmax_refine, has replaced its buffers),
 * RSOT_ERR_CUDA.
 */
rsot_status rsot_last_eval(rsot_problem *p, double *J_out, double *grad_out, int64_t *pairs_out,
                           int64_t *empty_out);

/*
 * One evaluation truncated by psi-aware cutoffs per pair (Sec. 4.1, App. B):
 *   I_q = { j : c(x_q, y_j) < alpha_q + beta_j },
 *   alpha_q = c(x_q, y_n) - psi_n - eps ln nu_n  (n = the nearest target of x_q,
 *             the lowest index among equal costs, found once per problem),
 *   beta_j  = psi_j + eps ln(1/tail).
 * The nearest target is always kept and each point's excluded terms sum to at
 * most tail * sum_j nu_j times its kept ones, so |J - J~| <= eps tail sum(nu)
 * sum(m) and |dJ/dpsi_j - dJ~/dpsi_j| <= tail (sum(nu) (dJ~/dpsi_j + nu_j) +
 * nu_j sum(m)) -- the guarantees of the radius of rsot_radius_for_tail, whose
 * cutoff bounds alpha_q + beta_j from above, with fewer pairs.
 *   tail : in (0, 1)
 * Other arguments, outputs and errors as rsot_eval_dual_grad (never
 * RSOT_ERR_EMPTY_NEIGHBORHOOD: every point keeps its nearest target).
 */
rsot_status rsot_eval_dual_grad_tail(rsot_problem *p, const double *psi, double eps,
                                     double tail, rsot_precision prec,
                                     double *J_out, double *grad_out, int64_t *pairs_out);

/*
 * Per-point log partition of the last successful rsot_eval_dual_grad call:
 *   L_q = ln sum_{j in I_q} nu_j exp((psi_j - c(x_q, y_j))/eps)
 * (the integrand of Eq. discretized_functional divided by eps; I_q all
 * targets when the evaluation was dense), in the precision of that call.
 *   L_out : nq doubles (host or device), in the caller's point order.
 * Errors: RSOT_ERR_ARG when no evaluation has succeeded on this handle.
 */
rsot_status rsot_point_log_partition(rsot_problem *p, double *L_out);

/*
 * ln D of the last successful evaluation, D = sum_q m_q / S_trunc(x_q) with
 * S_trunc(x_q) = exp(L_q) its (dense or truncated) per-point sum: the integrated
 * quantity of the integral cutoff (Sec. 4.1, Eq. truncation_cutoff_int)
 *   C_int = max_j psi_j + eps ln(eps D / (tau |J|)),
 * which keeps |J - J_trunc| <= tau |J| when D is taken at that cutoff (App. B).
 * +inf when a point with m_q > 0 had no target within the cutoff.
 * Errors: RSOT_ERR_ARG when no evaluation has succeeded on this handle.
 */
rsot_status rsot_log_integrated_D(rsot_problem *p, double *lnD_out);

/*
 * Covering cost C_0 = max_q min_j c(x_q, y_j) over the quadrature points
 * (App. B).  Depends on geometry only; computed once and cached.
 */
rsot_status rsot_covering_cost(rsot_problem *p, double *C0_out);

/*
 * Truncation radius for a tail tolerance (Sec. 4.1 and App. B, applied per
 * point): C = C_0 + Gamma + eps ln(1 / (nu_min tail)), Gamma = max psi -
 * min psi, radius = sqrt(2 C).  With this radius no point loses all its
 * targets, the excluded mass at every point is at most tail times the kept
 * mass, |J - J_trunc| <= eps tail sum_q m_q, and per target
 * |dJ/dpsi_j - dJ_trunc/dpsi_j| <= tail (sum_q m_q p~_qj + nu_j).
 *   psi : n doubles (host or device); tail in (0, 1).
 */
rsot_status rsot_radius_for_tail(rsot_problem *p, const double *psi, double eps,
                                 double tail, double *radius_out);

/*
 * The cost cutoffs of the truncated evaluation (Sec. 4.1, App. B), for a
 * potential psi (n doubles, host or device) at eps; M = max psi, m = min psi,
 * Gamma = M - m, C_0 = the covering cost (rsot_covering_cost):
 *   RSOT_CUTOFF_POINTWISE : C_pw = M + eps ln(max nu / param)      (Eq. cost_cutoff_delta;
 *                           param = delta_thr)
 *   RSOT_CUTOFF_INTEGRAL  : C_int = M + eps (ln eps + lnD - ln param - ln |J|)
 *                           (Eq. truncation_cutoff_int; param = tau, lnD = ln D as
 *                           returned by rsot_log_integrated_D, J the functional)
 *   RSOT_CUTOFF_GEOMETRIC : C_geom = max(C_0, C_0 + Gamma + eps ln(eps / (min nu param |J|)))
 *                           (Eq. truncation_cutoff_geom, App. B; param = tau)
 *   RSOT_CUTOFF_TAIL      : C = C_0 + Gamma + eps ln(1 / (min nu param))  (param = tail;
 *                           the cutoff of rsot_radius_for_tail)
 * The truncated evaluation keeps c(x_q, y_j) < C, i.e. radius sqrt(2 C).
 * J and lnD are read only by the kinds that use them.
 * Errors: RSOT_ERR_ARG (unknown kind, param <= 0, eps <= 0, J = 0 where used),
 * RSOT_ERR_NONFINITE (psi not finite), RSOT_ERR_CUDA.
 */
typedef enum {
    RSOT_CUTOFF_POINTWISE = 0,
    RSOT_CUTOFF_INTEGRAL = 1,
    RSOT_CUTOFF_GEOMETRIC = 2,
    RSOT_CUTOFF_TAIL = 3
} rsot_cutoff_kind;
rsot_status rsot_truncation_cutoff(rsot_problem *p, const double *psi, double eps, int kind,
                                   double param, double J, double lnD, double *C_out);

/*
 * Kernel tracing (no counterpart in the paper: a runtime facility).  While
 * enabled, every kernel the library launches is bracketed by CUDA events on
 * the handle's stream and its device time is accumulated per kernel name.
 * rsot_kernel_times copies up to `max` entries (static name strings, total
 * milliseconds, launch counts) and returns how many kernels have entries;
 * rsot_kernel_timing(p, 1) also clears the totals.
 */
rsot_status rsot_kernel_timing(rsot_problem *p, int enable);
int rsot_kernel_times(rsot_problem *p, const char **names, double *total_ms,
                      int64_t *launches, int max);

/*
 * Throughput probe of the special-function unit (no counterpart in the
 * paper): times `iters` rounds of independent ex2.approx.ftz.f32 on the
 * current device and returns the measured ex2 results per second.  Used as
 * the measured ceiling of the exponential-bound kernels.
 */
rsot_status rsot_probe_ex2_rate(int iters, double *ex2_per_s);

/*
 * Throughput probe of the FP64 pipe (no counterpart in the paper): times
 * `iters` rounds of independent FP64 fused multiply-adds on the current device
 * and returns the measured DFMA per second, the ceiling of the FP64 path
 * (whose exponential is the library's own, so its FP64 operations per pair
 * are known).
 */
rsot_status rsot_probe_dfma_rate(int iters, double *dfma_per_s);

/*
 * The FP64 path's exponential on the GPU, y_i = e^{x_i} (Tang's table-driven
 * method: 64 table values of 2^(j/64), Taylor polynomial of degree 6 on
 * |r| <= ln(2)/128; about 1 ulp; 0 below -745.2, +inf above 709.8, NaN kept),
 * exposed so that its accuracy can be tested.
 *   x, y : n doubles (host or device)
 */
rsot_status rsot_exp64(int64_t n, const double *x, double *y);

/*
 * Self-test of the bounded device-side waits (no counterpart in the paper:
 * failure detection).  Every wait of the library's kernels on a pipeline
 * stage (an mbarrier filled by a bulk copy) polls a bounded number of rounds
 * and, when they run out, records an error bit, lets the kernel's own copies
 * in flight land and returns, so the host reports RSOT_ERR_TIMEOUT and the
 * CUDA context stays usable.  This call runs that path on purpose: one CTA
 * waits `limit` rounds (1 <= limit <= 2^24) on a stage that no copy fills,
 * drains the one copy it did issue, and returns.
 * Returns RSOT_ERR_TIMEOUT when the wait ran out (the expected result),
 * RSOT_OK if it did not; RSOT_ERR_ARG, RSOT_ERR_NOMEM, RSOT_ERR_CUDA.
 */
rsot_status rsot_selftest_wait_timeout(long long limit, void *stream);

/*
 * Allocation-free dense evaluation (no counterpart in the paper: an interface
 * for callers that cannot allocate device memory themselves -- code whose
 * device memory belongs to another component, such as a framework's caching
 * allocator, or that runs under a fixed memory budget set at start-up).
 *
 * One dense mixed-precision evaluation of J and its gradient without a problem
 * handle and without calling cudaMalloc, cudaFree or any allocating library
 * routine.  It runs the FP32 pair kernels of RSOT_MIXED (RSOT_PAIRS_FP32), so
 * it agrees with rsot_eval_dual_grad(radius 0, RSOT_MIXED) within the mixed
 * path's tolerances (1e-5 relative on J, 1e-6 absolute per gradient entry),
 * not bit for bit.  Its scratch is one static device array of
 * RSOT_NOALLOC_SCRATCH_BYTES (57.6 MiB) inside librsot, which every GPU
 * that loads the library holds until the process exits.
 *   d, nq, n     : as rsot_create; nq <= RSOT_NOALLOC_MAX_NQ, n <= RSOT_NOALLOC_MAX_N
 *                  (larger sizes return RSOT_ERR_ARG without touching the GPU)
 *   x, mass, y, nu, psi : DEVICE pointers of the current device (row-major, as
 *                  rsot_create / eval); host pointers and other devices'
 *                  memory are rejected with RSOT_ERR_ARG
 *   eps          : > 0
 *   stream       : cudaStream_t for all work (NULL = legacy default stream)
 *   J_out        : HOST pointer, 1 double
 *   grad_out     : DEVICE pointer of the current device, n doubles
 * The call synchronises the stream before it returns (J_out is a host value),
 * so it cannot be captured in a CUDA graph.  The first call in a CUDA context
 * looks up the address of the static scratch in that context (with its device
 * current); later calls in the same context reuse it.  Every call shares the
 * one scratch array and leaves its contents behind: calls that overlap on the
 * GPU (other streams, other host threads) race and must be serialised by the
 * caller.  On an error J_out and grad_out are left untouched.
 * Errors: RSOT_ERR_ARG, RSOT_ERR_NONFINITE, RSOT_ERR_TIMEOUT, RSOT_ERR_CUDA.
 */
#define RSOT_NOALLOC_MAX_NQ 524288
#define RSOT_NOALLOC_MAX_N 65536
#define RSOT_NOALLOC_SCRATCH_BYTES 60393984
rsot_status rsot_eval_dense_noalloc(int d, int64_t nq, const double *x, const double *mass,
                                    int64_t n, const double *y, const double *nu,
                                    const double *psi, double eps, void *stream,
                                    double *J_out, double *grad_out);

/* Solver options (Algorithm 1 with the eps-schedule of Sec. 4.2). */
typedef struct {
    double eps;          /* final regularisation, > 0                              */
    double eps_start;    /* first stage of the eps-schedule; <= eps: no schedule   */
    double eps_factor;   /* stage ratio in (0,1), e.g. 0.5; the last stage is eps  */
    double tail;         /* > 0: truncate the mixed (and FP64 / compensated stage)
                            evaluations with the psi-aware cutoffs of this tail
                            (rsot_eval_dual_grad_tail).  The refinement's
                            compensated reference evaluations are truncated too
                            when tail <= 1e-8 (else dense, as are FP64 ones), and
                            the truncation bound tail sum(nu) (2 sum(m) + sum(nu))
                            on ||grad J~ - grad J||_1 is subtracted from tol_l1
                            with the compensated one, so a refined stop holds for
                            the untruncated J.  An eps-stage (or refinement
                            phase) whose first truncated evaluation keeps more
                            than 35 % of all pairs evaluates dense from that
                            point on (within tail of the truncated functional,
                            and cheaper there).  0: dense                      */
    double tol_l1;       /* stop when ||grad J||_1 <= tol_l1 (Remark 3.3)           */
    double stage_tol_l1; /* tolerance of the intermediate stages (<=0: 100 tol_l1:
                            they only warm-start the next stage)                 */
    int precision;       /* rsot_precision of the evaluations                       */
    int refine_fp64;     /* MIXED only: finish the last stage with the refinement on
                            reference evaluations (refine_precision; rsot_solve) */
    int lbfgs_m;         /* L-BFGS memory (<= 0: 10)                                */
    int max_iter;        /* iteration cap per stage (<= 0: 10000)                   */
    int verbose;         /* print one line per run to stderr                        */
    double mixed_tol_l1; /* MIXED + refine_fp64: the mixed phase of the last stage
                            stops here, the refinement takes over (<= 0: 1e-5)   */
    int refine_precision;/* reference evaluations of the refinement (and of the last
                            stage when precision is RSOT_COMPENSATED):
                            RSOT_COMPENSATED (default) stops at ||g||_1 <= tol_l1 -
                            RSOT_COMPENSATED_GRAD_REL sum m_q, which certifies
                            ||grad J||_1 <= tol_l1; it is used while that bound is
                            at most 0.8 tol_l1, else FP64.  Compensated references
                            of an untruncated solve of at least 2e10 pairs are
                            truncated at the psi-aware cutoffs of tail 1e-12, whose
                            bound joins the certified one (dense where they would
                            keep most pairs).
                            RSOT_FP64: always FP64, dense                        */
    double tau_int;      /* > 0 (with tail = 0): truncate each evaluation at the
                            integral cutoff C_int of this relative J tolerance,
                            D and J from the previous evaluation of the stage
                            (Sec. 4.1); the first evaluation of a stage is dense */
    double delta_pw;     /* > 0: truncate each evaluation at the pointwise cutoff
                            C_pw = max psi + eps ln(max nu / delta_pw) of the
                            current potential (Sec. 4.1, Eq. cost_cutoff_delta);
                            points left without a target are skipped, as
                            Algorithm 2 skips them                             */
    double tau_geom;     /* > 0: truncate each evaluation at the geometric cutoff
                            C_geom of this relative J tolerance (Sec. 4.1, Eq.
                            truncation_cutoff_geom, App. B), J from the previous
                            evaluation of the stage; the first one is dense.
                            At most one of tail, tau_int, delta_pw, tau_geom is
                            > 0; the refinement's references stay dense        */
} rsot_options;

/* Fill *o with the defaults (eps 1e-2, no schedule, dense, tol 1e-6, MIXED with
 * refinement against compensated evaluations, m = 10, 10000 iterations). */
void rsot_default_options(rsot_options *o);

/* Per-solve statistics. */
typedef struct {
    double J;            /* J at the returned psi (last stage's precision)       */
    double grad_l1;      /* ||grad J||_1 at the returned psi                      */
    int iters;           /* L-BFGS iterations over all stages                     */
    int evals;           /* dual evaluations over all stages                      */
    int stages;          /* eps stages run                                        */
    int64_t pairs;       /* pairs evaluated over all evaluations                  */
    double seconds;      /* wall time of the call                                 */
    int evals_prec[3];   /* evaluations by rsot_precision (index RSOT_FP64,
                            RSOT_MIXED, RSOT_COMPENSATED)                          */
    int64_t pairs_prec[3];  /* pairs evaluated by rsot_precision                   */
} rsot_solve_stats;

/*
 * Minimise J with FP64 L-BFGS on the host (two-loop recursion, strong-Wolfe
 * line search, curvature pairs in FP64), each evaluation on the GPU
 * (Algorithm 1), with eps-scheduling and warm start (Sec. 4.2).
 *   psi_inout : n doubles, HOST memory: the warm start on entry, the
 *               minimiser on return (also on NOT_CONVERGED / LINESEARCH,
 *               where it is the last accepted iterate).
 * precision RSOT_COMPENSATED runs every stage with compensated evaluations
 * (the last one to the certified tolerance, see refine_precision).
 * stats->grad_l1 is the L1 norm of the last gradient in the precision that
 * decided the stop.
 * Errors: RSOT_ERR_ARG, RSOT_ERR_NOT_CONVERGED, RSOT_ERR_LINESEARCH, and any
 * error of rsot_eval_dual_grad.
 */
rsot_status rsot_solve(rsot_problem *p, double *psi_inout, const rsot_options *opt,
                       rsot_solve_stats *stats);

/* ---------------------------------------------------------------------------
 * Batched problems: many RSOT problems of uneven size evaluated together.
 * One evaluation round is one CUDA graph: copy the potentials in, one
 * persistent launch per pass over a work queue of (problem, tile, chunk)
 * items, copy the gradients and J out.  The batched solver runs one L-BFGS
 * (Algorithm 1) per problem on the host, in lockstep: every round evaluates
 * the pending trial point of every unfinished problem.
 * ------------------------------------------------------------------------- */
typedef struct rsot_batch rsot_batch;   /* opaque; owns its device memory */

typedef struct {
    int d;                 /* 2 or 3                                              */
    int64_t nq;            /* quadrature points                                   */
    const double *x;       /* nq*d (host or device)                               */
    const double *mass;    /* nq                                                  */
    int64_t n;             /* targets                                             */
    const double *y;       /* n*d                                                 */
    const double *nu;      /* n                                                   */
} rsot_problem_desc;

/* Create a batch of `count` problems (inputs copied; buffers may be freed after). */
rsot_status rsot_batch_create(int count, const rsot_problem_desc *probs, rsot_batch **out);
void rsot_batch_destroy(rsot_batch *b);
rsot_status rsot_batch_set_stream(rsot_batch *b, void *stream);

/* Pair kernel of the batched mixed passes (see rsot_set_pair_kernel):
 * rsot_batch_eval uses the FP32 form unless RSOT_PAIRS_TENSOR; the batched
 * solver's rounds (and rsot_batch_tune, which times them) take the tensor-core
 * form under RSOT_PAIRS_AUTO when every problem is within its range, until a
 * problem's gradient approaches its noise.  Errors: RSOT_ERR_ARG, RSOT_ERR_CUDA. */
rsot_status rsot_batch_set_pair_kernel(rsot_batch *b, rsot_pair_kernel kind);

/* Total number of targets (length of the concatenated psi / gradient vectors). */
int64_t rsot_batch_total_targets(const rsot_batch *b);

/*
 * Autotuner (no counterpart in the paper): times one batched evaluation per
 * candidate work-item size at the given eps (count doubles, host) and psi
 * (concatenated, host), keeps the fastest, and rebuilds the CUDA graph.
 * *choice_out (nullable) receives the chosen pairs-per-item exponent.
 */
rsot_status rsot_batch_tune(rsot_batch *b, const double *psi_all, const double *eps,
                            int *choice_out);

/*
 * One batched dense mixed-precision evaluation (Eq. discretized_functional /
 * discretized_gradient for every problem).  All arrays are HOST memory:
 *   psi_all : concatenated potentials (problem order), total_targets doubles
 *   eps     : count doubles;  active: count bytes (NULL = all), 0 = skip problem
 *   J_out   : count doubles;  grad_all: total_targets doubles
 * Skipped problems' outputs are left untouched.
 */
rsot_status rsot_batch_eval(rsot_batch *b, const double *psi_all, const double *eps,
                            const unsigned char *active, double *J_out, double *grad_all);

/* Per-batch solve statistics. */
typedef struct {
    double seconds;            /* wall time of the call                               */
    double seconds_mixed;      /* batched mixed-precision rounds                      */
    double seconds_refine;     /* FP64 refinement                                     */
    int rounds;                /* batched evaluation rounds                           */
    int converged;             /* problems that reached tol_l1                        */
    double max_grad_l1;        /* largest final ||grad J||_1                          */
    int64_t evals;             /* evaluations summed over problems                    */
    int64_t evals_prec[3];     /* evaluations by rsot_precision (batched rounds are
                                  RSOT_MIXED; refinements add their own)             */
    int64_t pairs_prec[3];     /* pairs evaluated by rsot_precision                   */
} rsot_batch_stats;

/*
 * Solve every problem: per-problem final eps (count doubles, host), the
 * eps-schedule of `opt` (eps_start/eps_factor; a problem whose final eps is
 * above eps_start runs only its final stage), tol_l1, lbfgs_m, max_iter.
 * opt->precision = RSOT_MIXED runs the batched mixed rounds and then, with
 * refine_fp64, finishes each problem with the refinement of rsot_solve
 * (reference evaluations of opt->refine_precision) through its own problem
 * handle, problems spread over host threads with a stream each; RSOT_FP64
 * solves each problem in turn with FP64 evaluations (no batching).  psi_all: host, concatenated warm start in / solution out.
 * status_out (nullable): count ints; grad_l1_out (nullable): count doubles.
 */
rsot_status rsot_batch_solve(rsot_batch *b, double *psi_all, const double *eps,
                             const rsot_options *opt, int *status_out, double *grad_l1_out,
                             rsot_batch_stats *stats);

/* ---------------------------------------------------------------------------
 * Multilevel acceleration (Sec. 5).
 * ------------------------------------------------------------------------- */

/*
 * Weighted k-means of n points (Sec. 5.2: coarse targets are cluster
 * centroids, coarse weights the summed weights of the cluster).  Seeded
 * initial centres (a random subset of the points), `iters` Lloyd iterations:
 * assignment on the GPU (nearest centre in FP32, lowest index on ties),
 * update on the host in FP64 (deterministic); a cluster left empty restarts at
 * the point farthest from its centre.  The returned centres are the weighted
 * centroids of the final assignment (a cluster still empty after the last
 * iteration returns weight 0 and its last centre).
 *   y: n*d, w: n (host or device); centers_out: k*d, weights_out: k (host);
 *   assign_out: n (host, nullable).
 */
rsot_status rsot_kmeans(int d, int64_t n, const double *y, const double *w, int64_t k, int iters,
                        uint64_t seed, double *centers_out, double *weights_out,
                        int64_t *assign_out);

/*
 * Softmax refinement (Eq. softmax_refinement_formula): from the potential
 * psi_coarse on the targets of problem p (the coarse level, on p's source
 * points), the initial potential of the n_fine targets y_fine:
 *   psi_k = -eps ln sum_q m_q exp(-c(x_q, y_k)/eps) / S_c(x_q),
 *   S_c(x) = sum_j nu_j exp((psi_j - c(x, y_j))/eps).
 * Mixed precision (pass 1 of the coarse problem, a pass 2 over the fine
 * targets, FP64 sums).  psi_coarse, y_fine, psi_fine_out: host or device.
 */
rsot_status rsot_softmax_refine(rsot_problem *p, const double *psi_coarse, double eps,
                                int64_t n_fine, const double *y_fine, double *psi_fine_out);

#define RSOT_MAX_LEVELS 16

typedef struct {
    int d;
    int64_t nq;
    const double *x;      /* nq*d */
    const double *mass;   /* nq   */
} rsot_source_level;

typedef struct {
    int64_t n;
    const double *y;      /* n*d  */
    const double *nu;     /* n    */
} rsot_target_level;

typedef struct {
    int levels;                          /* L_max + 1                               */
    int src_level[RSOT_MAX_LEVELS];      /* i_s(l)                                  */
    int tgt_level[RSOT_MAX_LEVELS];      /* i_t(l)                                  */
    int transfer[RSOT_MAX_LEVELS];       /* 0 start, 1 injection, 2 softmax refine  */
    int iters[RSOT_MAX_LEVELS];
    int evals[RSOT_MAX_LEVELS];
    double seconds[RSOT_MAX_LEVELS];
    double grad_l1;                      /* final ||grad J||_1                      */
    double total_seconds;
} rsot_multilevel_stats;

/*
 * Combined multilevel solve (Sec. 5.3): source levels 0..L_mu (coarse to fine)
 * and target levels 0..L_nu (coarse to fine); at step l = 0..L_max the
 * problem (T_{i_s(l)}, nu^{i_t(l)}) with i_s = max(0, l - (L_max - L_mu)),
 * i_t = max(0, l - (L_max - L_nu)) is solved at eps_levels[l] (L_max + 1
 * values) by rsot_solve with `opt` (its eps-schedule applies to step 0 only;
 * steps before the last only warm-start the next one and stop at
 * max(tol_l1, mixed_tol_l1) without FP64 refinement); the potential moves to
 * the next step by softmax refinement when i_t increases and by injection
 * otherwise.  psi_out: host, n of the finest target level.
 */
rsot_status rsot_multilevel_solve(int n_src, const rsot_source_level *src, int n_tgt,
                                  const rsot_target_level *tgt, const double *eps_levels,
                                  const rsot_options *opt, double *psi_out,
                                  rsot_multilevel_stats *stats);

/* ---------------------------------------------------------------------------
 * Transport maps, centroids and barycenters (Sec. 6.2-6.3).  Each runs one
 * dense mixed evaluation at (psi, eps) and then one sum over its plan
 * p_qj (Eq. final_plan_density), FP32 pair arithmetic, FP64 across tiles.
 * ------------------------------------------------------------------------- */

/*
 * Transport maps of a plan (Sec. 6.3):
 *   T_out[q*d + k] = T_bary(x_q)_k = sum_j p_qj y_jk   (Eq. barycentric_map_registration)
 *   jstar_out[q]   = argmax_j p_qj                    (Eq. modal_map_registration;
 *                    the modal map is y_{jstar}; ties in FP32 go to the lowest j)
 * Either output may be NULL (not both); host or device memory.
 * Errors: RSOT_ERR_ARG, those of rsot_eval_dual_grad, RSOT_ERR_CUDA.
 */
rsot_status rsot_transport_maps(rsot_problem *p, const double *psi, double eps, double *T_out,
                                int64_t *jstar_out);

/*
 * Conditional centroids of a plan (Eq. barycenter_fixed_point):
 *   T_out[j*d + k] = (1/nu_j) sum_q m_q p_qj x_qk,  mass_out[j] = sum_q m_q p_qj
 * (mass_out may be NULL).  Host or device memory.
 * Errors: RSOT_ERR_ARG, those of rsot_eval_dual_grad, RSOT_ERR_CUDA.
 */
rsot_status rsot_centroids(rsot_problem *p, const double *psi, double eps, double *T_out,
                           double *mass_out);

typedef struct {
    int iterations;            /* Lloyd updates made                                */
    int converged;             /* 1 when the last RMS displacement <= tol_rms       */
    double rms_last;           /* RMS displacement of the last update               */
    int solve_iters, solve_evals;   /* summed over all RSOT solves                  */
    double seconds_solve, seconds_centroids, seconds_total;
} rsot_barycenter_stats;

/*
 * Barycenter with fixed weights nu by the damped Lloyd iteration of Sec. 6.2
 * (Eq. damped_lloyd): y <- (1 - theta) y + theta sum_i lambda_i T_i, T_i the
 * centroids of the optimal plan between source i (src[i], K sources of one
 * dimension d) and (y, nu), solved by rsot_solve with `opt` (its eps-schedule
 * on the first iteration only; later solves start from the previous
 * potential).  Stops when the RMS displacement sqrt(sum_j |dy_j|^2 / n) <=
 * tol_rms or after max_iter updates.  y_inout: host, n*d; nu, lambda: host.
 * Errors: RSOT_ERR_ARG, those of rsot_create / rsot_solve / rsot_centroids.
 */
rsot_status rsot_barycenter(int K, const rsot_source_level *src, const double *lambda,
                            int64_t n, double *y_inout, const double *nu,
                            const rsot_options *opt, double theta, int max_iter, double tol_rms,
                            rsot_barycenter_stats *stats);

/* ---------------------------------------------------------------------------
 * Learned warm start (no counterpart in the paper): an MLP psi_j ~ f(theta,
 * y_j) of width W with three SiLU hidden layers and a linear head, BF16
 * weights/activations in its GEMMs, FP32 accumulation, FP32 master weights,
 * Adam.  All arrays are FP32, host or device; inputs are rows of in_dim
 * values.
 * ------------------------------------------------------------------------- */
typedef struct rsot_mlp rsot_mlp;

rsot_status rsot_mlp_create(int in_dim, int width, uint64_t seed, rsot_mlp **out);
void rsot_mlp_destroy(rsot_mlp *m);
rsot_status rsot_mlp_set_stream(rsot_mlp *m, void *stream);
/* GEMM kernel of the network's layers (forward, back-propagation, weight
 * gradients): RSOT_MLP_GEMM_TCGEN05 (default: tcgen05.mma issued by one thread,
 * FP32 accumulators in tensor memory, operands by TMA tensor copies; where the
 * output width is at most 256 and a multiple of 32, a persistent kernel with
 * one CTA per SM, a copy warp, an MMA warp and 16 epilogue warps over two
 * accumulators, its outputs stored by TMA; otherwise 128 x 128 tiles),
 * RSOT_MLP_GEMM_TCGEN05_CPASYNC (the 128 x 128 tcgen05 kernel with cp.async
 * copies only) or RSOT_MLP_GEMM_MMA_SYNC (warp-level mma.sync m16n8k16).  Same
 * operands, K slices and epilogues; the sums differ only in the order of FP32
 * accumulation (the two tcgen05 forms give equal results).
 * Errors: RSOT_ERR_ARG (NULL handle or unknown kind).  Calls that run the
 * tcgen05 kernel return RSOT_ERR_TIMEOUT when one of its bounded waits gave up. */
enum { RSOT_MLP_GEMM_TCGEN05 = 0, RSOT_MLP_GEMM_MMA_SYNC = 1, RSOT_MLP_GEMM_TCGEN05_CPASYNC = 2 };
rsot_status rsot_mlp_set_gemm_kernel(rsot_mlp *m, int kind);
/* parameter block: W1 [W][in_pad], b1 [W], W2 [W][W], b2, W3 [W][W], b3, w4 [W], b4 [1];
 * in_pad = in_dim rounded up to 32 (padded columns are zero) */
int64_t rsot_mlp_num_params(const rsot_mlp *m);
rsot_status rsot_mlp_get_params(rsot_mlp *m, float *out);
rsot_status rsot_mlp_set_params(rsot_mlp *m, const float *in);
/* y_out[r] = f(x[r]) for r < rows */
rsot_status rsot_mlp_forward(rsot_mlp *m, int64_t rows, const float *x, float *y_out);
/* loss = mean_r (f(x_r) - y_r)^2 / 2 and its gradient (grad_out nullable, num_params floats) */
rsot_status rsot_mlp_gradients(rsot_mlp *m, int64_t rows, const float *x, const float *y,
                               float *loss_out, float *grad_out);
/* one Adam step (beta 0.9 / 0.999) on the loss of (x, y) with learning rate lr */
rsot_status rsot_mlp_train_step(rsot_mlp *m, int64_t rows, const float *x, const float *y,
                                float lr, float *loss_out);

#ifdef __cplusplus
}
#endif
#endif /* RSOT_H */
