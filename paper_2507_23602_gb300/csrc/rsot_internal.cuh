// Internal declarations shared by the librsot translation units.
//
// Layout in HBM (all device buffers owned by rsot_problem):
//   points  : FP32 translated coordinates, SoA xs[k * nq_pad + q] (k < d),
//             zero-padded to nq_pad (a multiple of the pass-1 point tile);
//             FP64 translated coordinates x64[q * d + k]; masses m_q (FP64)
//             and log2 m_q (FP64).
//   targets : FP64 translated coordinates y64[j * d + k], nu_j, ln nu_j.
//   per evaluation (mixed precision, log2 domain, see rsot_dense.cu):
//             target "dup" records  TRecDup[j]  = (w0,w0,w1,w1,w2,w2,c,c)
//             target "pair" records TRecPair[g] = (w0a,w0b,w1a,w1b,w2a,w2b,ca,cb)
//             pass-1 partials (M, S) per point and target chunk
//             point "dup" records   (x0,x0,x1,x1,x2,x2,u,u) for pass 2
//             pass-2 FP64 partial sums per point chunk and target
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rsot.h"

namespace rsot {

constexpr double kLog2e = 1.4426950408889634074;
constexpr double kLn2 = 0.69314718055994530942;
constexpr float kPadC = -1.0e30f;            // exponent of a padding target: ex2 -> 0

// Error bits written by kernels into ProblemDev::flags.
enum : int {
    kErrTimeout = 1,        // an mbarrier wait exceeded its iteration limit
    kErrNonfinitePsi = 2,   // psi had a NaN / Inf entry
    kErrBadCell = 4,        // a cell index fell outside the grid (truncated path)
};

struct __align__(16) Rec8 {   // 32-byte record: two float4
    float4 a;
    float4 b;
};

// Result block copied back to the host after each evaluation.
struct EvalResult {
    double J;
    double psic;        // psi_0 of the evaluation (the potential centre)
    long long pairs;
    long long empty;
    int flags;
    int gate;           // bit 0: an f16 operand is out of range (both passes take the FP32 kernels)
};

struct Grid;  // truncated-path cell grid (rsot_trunc.cu)
struct Rec16; // tensor-core operand record (rsot_tc.cuh)

}  // namespace rsot

struct rsot_problem {
    int d = 0;
    int dev = 0;
    int64_t nq = 0, n = 0;
    int64_t nq_pad = 0, n_pad = 0;
    cudaStream_t stream = nullptr;
    double origin[3] = {0, 0, 0};
    double msum = 0.0;          // sum_q m_q
    double hx = 0.0;            // sum_q m_q |x'_q|^2 / 2 (translated coordinates)
    double nu_min = 0.0, nu_max = 0.0;
    double diam2 = 0.0;         // squared diameter of the bounding box of points and targets
    int num_sms = 0;

    // static device data
    float *xs = nullptr;        // [d][nq_pad]
    double *x64 = nullptr;      // [nq][d]
    double *mass = nullptr;     // [nq]
    double *lmass2 = nullptr;   // [nq] log2 m_q (-inf if m_q == 0)
    double *y64 = nullptr;      // [n][d]
    double *nu = nullptr;       // [n]
    double *lnu = nullptr;      // [n] ln nu_j

    // per-evaluation scratch (mixed)
    rsot::Rec8 *tdup = nullptr;     // [n_pad]
    rsot::Rec8 *tpair = nullptr;    // [n_pad / 2]
    float2 *part1 = nullptr;        // [k1][nq_pad]
    rsot::Rec8 *pdup = nullptr;     // [nq_pad]
    double *part2 = nullptr;        // [s2][n_pad]
    double *blockJ = nullptr;       // [nblk_j]
    double *psinu = nullptr;        // [nblk_psi]
    int k1 = 0, chunk1 = 0;         // pass-1 target chunks
    int s2 = 0;                     // pass-2 point splits
    int64_t chunk2 = 0;
    int nblk_comb = 0, nblk_prep = 0;
    // tensor-core form of the pair arithmetic (rsot_tc.cuh)
    rsot::Rec16 *trec = nullptr;    // [n_pad] target operand records
    rsot::Rec16 *prec16 = nullptr;  // [nq_pad] point operand records (static)
    float *pu = nullptr;            // [nq_pad] pass-2 shifts u_q = log2 m_q - R_q
    float tc_P = 1.0f;              // point coordinate scale (power of two)
    int pair_kernel = 2;            // 0: FP32 passes, 1: tensor-core passes (FP32 fallback by
                                    // gate), 2: tensor-core passes when m_max nu_max <= kTcAuto
    double m_max = 0.0;             // max_q m_q
    // estimated L1 norm of the tensor-core rounding noise of a gradient,
    // 1.4e-5 sqrt(m_max) sum_j sqrt(nu_j) (see kTcAuto); solvers take the FP32
    // kernels once the gradient is within kTcNoiseFactor of it
    double tc_noise_l1 = 0.0;
    int pair_fp32_now = 0;          // set by a solver: this evaluation takes the FP32 kernels
    int in_solve = 0;               // set while rsot_solve runs on this handle
    int k1_tc = 0, chunk1_tc = 0;   // pass-1 target chunks of the tensor-core launch
    int s2_tc = 0;                  // pass-2 point splits of the tensor-core launch
    int64_t chunk2_tc = 0;
    // FP64 path scratch
    double *a64 = nullptr;          // [n_pad]   psi_j/eps + ln nu_j
    double *prec64 = nullptr;       // [nq_pad][4] (x0,x1,x2,u)
    int s2_64 = 0;
    int64_t chunk2_64 = 0;
    double *part2_64 = nullptr;     // [s2_64][n_pad]
    // compensated path scratch (rsot_df.cu), allocated on first use
    void *df_prec = nullptr;        // [nq_pad] point head/tail records (64 B)
    void *df_trec = nullptr;        // [n_pad] target head/tail records (64 B)
    double *df_part2 = nullptr;     // [df_s2][n_pad] pass-2 partials
    int df_s2 = 0;
    // truncated compensated passes: targets in the Morton order of the cell list,
    // blocks classified by balls (rsot_df.cu)
    double *df_beta_s = nullptr;    // [n_pad] beta in sorted order (per evaluation)
    float *df_beta_sf = nullptr;    // [n_pad] nb_j = b_j - 2k beta_j in FP32, sorted (per evaluation)
    float *df_alpha_f = nullptr;    // [nq_pad] A_q = k|x'_q|^2 - 2k alpha_q in FP32 (per evaluation)
    float4 *df_pb64 = nullptr;      // [nq_pad / 64] balls of 64 caller-order points (once)
    float4 *df_pb8 = nullptr;       // [nq_pad / 8] balls of 8 caller-order points (once)
    float2 *df_pa64 = nullptr, *df_pa8 = nullptr;    // alpha ranges of those point blocks
    float2 *df_tbe64 = nullptr, *df_tbe8 = nullptr;  // beta ranges of 64 / 8 sorted targets

    // truncation cutoffs per pair, c(x_q, y_j) < alpha_q + beta_j (rsot_cutoff.cu)
    int *nn = nullptr;              // [nq] nearest target of each point (once per problem)
    double *nn_c = nullptr;         // [nq] its cost
    double *alpha = nullptr;        // [nq_pad] per evaluation (-inf for padding)
    double *beta = nullptr;         // [n_pad]  per evaluation (-inf for padding)
    int cut_anchored = 0;           // alpha is anchored at the nearest targets (psi-aware)

    // staging for host psi / grad
    double *psi_dev = nullptr;      // [n]
    bool borrowed = false;          // mass and nu are the caller's device arrays (not freed)
    double *grad_dev = nullptr;     // [n] gradient of the last evaluation
    double *grad_host = nullptr;    // [n] pinned staging of host gradient outputs
    rsot::EvalResult *res_dev = nullptr;
    rsot::EvalResult *res_host = nullptr;   // pinned
    int *flags = nullptr;           // device error bits (inside res_dev)

    // per-point log partition of the last evaluation (see rsot_point_log_partition)
    double *lse_buf = nullptr;      // [nq_pad]: R_q (mixed, log2) or L'_q (FP64, natural)
    bool last_dense = true;         // the last evaluation's J, pair and empty-point counts
    double last_J = 0.0;            // (rsot_last_eval; its gradient stays in grad_dev)
    int64_t last_pairs = 0, last_empty = 0;
    int last_kind = -1;             // -1 none, 0 FP64 dense, 1 mixed dense, 2/3 truncated (FP64 /
                                    // mixed cell list), 4/5 compensated
                                    // FP64/mixed, 4/5 compensated dense/truncated
    double last_eps = 0.0;

    // covering cost cache
    double C0 = -1.0;

    // truncated path
    rsot::Grid *grid = nullptr;

    // kernel tracing (rsot_kernel_timing)
    int timing = 0;
    std::vector<cudaEvent_t> tr_events;                 // pool, reused
    std::vector<std::pair<const char *, int>> tr_open;  // (name, first event index)
    int tr_used = 0;
    std::vector<const char *> tr_names;
    std::vector<double> tr_total_ms;
    std::vector<int64_t> tr_count;
};

namespace rsot {

// Choice of the pair kernel of the mixed passes.  Every evaluation whose
// result goes back to the caller takes the FP32 pair arithmetic unless the
// caller asked for the tensor-core form (RSOT_PAIRS_TENSOR).  Inside the
// library's solvers (in_solve), whose stop is certified by compensated or
// FP64 reference evaluations, RSOT_PAIRS_AUTO lets the mixed L-BFGS iterations
// take the tensor-core form while its rounding noise is far below the
// gradient: the exponent's error is within about twice the FP32 chain's
// (measured maxima 5.7 and 2.7 units of 2^-24 times the sum of the magnitudes
// of its terms), random in sign, and a gradient entry sum_q m_q p_qj then
// scatters by ~1.4e-5 sqrt(m_max nu_max); where that scatter is no longer
// small (m_max nu_max > kTcAuto) or the gradient approaches it (pair_fp32_now,
// kTcNoiseFactor) the solver keeps the FP32 kernels, which converge further.
constexpr double kTcAuto = 2e-6;
constexpr double kTcNoiseFactor = 30.0;
inline bool use_tensor_pairs(const rsot_problem *p) {
    if (p->pair_kernel == 1) return true;
    return p->pair_kernel == 2 && p->in_solve && !p->pair_fp32_now && p->m_max * p->nu_max <= kTcAuto;
}

// ---- kernel tracing (rsot_api.cu) -------------------------------------------
// trace_begin/trace_end bracket one launch with events on p->stream when
// tracing is on; trace_collect (after a stream sync) accumulates durations.
void trace_begin(rsot_problem *p, const char *name);
void trace_end(rsot_problem *p);
void trace_collect(rsot_problem *p);

// ---- launch helpers implemented in rsot_dense.cu --------------------------
cudaError_t dense_alloc(rsot_problem *p);
void dense_free(rsot_problem *p);
cudaError_t launch_dense_mixed(rsot_problem *p, const double *psi_dev, double eps,
                               double *grad_dev);
cudaError_t launch_dense_fp64(rsot_problem *p, const double *psi_dev, double eps,
                              double *grad_dev);
cudaError_t launch_trunc_fp64(rsot_problem *p, const double *psi_dev, double eps, double *grad_dev);
cudaError_t launch_covering_cost(rsot_problem *p, double *C0_dev);
cudaError_t launch_psi_stats(rsot_problem *p, const double *psi_dev, double *out3_dev);
cudaError_t launch_point_L(rsot_problem *p, double *L_dev);
// Copy an evaluation's gradient src -> dst only when the result block reports
// success (no error bit, finite J, and with require_nonempty no empty point).
cudaError_t launch_commit_grad(const double *src, double *dst, int64_t n,
                               const EvalResult *res, int require_nonempty, cudaStream_t st);
cudaError_t launch_softmax_refine(rsot_problem *p, const double *psi_dev, double eps, int64_t nf,
                                  const double *yf_dev, double *out_dev);

// ---- truncation cutoffs (rsot_cutoff.cu): fill p->alpha / p->beta
cudaError_t cutoffs_uniform(rsot_problem *p, double C);
cudaError_t cutoffs_separable(rsot_problem *p, const double *psi_dev, double eps, double tail);
void cutoff_free(rsot_problem *p);
// ln sum_q m_q exp(-L_q) from natural per-point log partitions on the device
cudaError_t launch_log_D(rsot_problem *p, const double *L_dev, double *lnD);

// ---- compensated path (rsot_df.cu): dense, or truncated by p->alpha / p->beta
cudaError_t launch_compensated(rsot_problem *p, const double *psi_dev, double eps, bool trunc,
                               double *grad_dev);
void compensated_free(rsot_problem *p);
// Bound of ||g - grad J||_1 / sum_q m_q for a compensated gradient g (rsot_df.cu)
constexpr double kCompGradRel = 6.5e-7;

// ---- transport maps and centroids (rsot_maps.cu), after a dense mixed evaluation
cudaError_t launch_maps(rsot_problem *p, double eps, double *T_dev, int64_t *j_dev,
                        const double *origin_dev);
cudaError_t launch_centroids(rsot_problem *p, double *T_dev, double *mass_dev,
                             const double *origin_dev);

// ---- truncated path (rsot_trunc.cu) ----------------------------------------
// truncated by the cutoffs in p->alpha / p->beta
cudaError_t trunc_eval(rsot_problem *p, const double *psi_dev, double eps, int mixed,
                       double *grad_dev);
void trunc_free(rsot_problem *p);
cudaError_t trunc_point_L(rsot_problem *p, double *L_dev);
// the cell list's target order for the compensated passes (grid built on first
// use): perm (sorted -> caller index, -1 for padding), sorted FP64 coordinates
// [n_pad][d], balls of 8 and of 64 sorted targets [n_pad / 8], [n_pad / 64]
struct SortedTargets {
    const int *perm = nullptr;
    const double *y64 = nullptr;
    const float4 *ball8 = nullptr, *ball64 = nullptr;
};
cudaError_t trunc_sorted_targets(rsot_problem *p, SortedTargets *out);
// block data of the truncated block-skip passes from p->alpha / p->beta
// (rsot_df.cu): df_beta_s, df_alpha_f (A_q), balls and ranges of point and
// target blocks; T receives the sorted-target view
cudaError_t trunc_block_setup(rsot_problem *p, double eps, SortedTargets *T);

// ---- device helpers ----------------------------------------------------------
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float max3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// 2^k for an integer-valued float k <= 0 (exact; 0 below the normal range).
__device__ __forceinline__ float pow2_int_f(float k) {
    return k < -126.0f ? 0.0f : __int_as_float(((int)k + 127) << 23);
}
__device__ __forceinline__ double pow2_int_d(float k) {
    return k < -1022.0f ? 0.0 : __longlong_as_double((long long)((int)k + 1023) << 52);
}

// ---- mbarrier + bulk-copy (TMA) wrappers ------------------------------------
constexpr long long kWaitLimit = 1ll << 24;   // bounded spin: ~seconds at most

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *smem, const void *gmem, unsigned bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(smem)),
        "l"(gmem), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned phase) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Bounded wait; false when the limit is reached (the caller records an error).
__device__ __forceinline__ bool mbar_wait_n(uint64_t *bar, unsigned phase, long long limit) {
    for (long long i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned phase) {
    return mbar_wait_n(bar, phase, kWaitLimit);
}

// Classification of a block pair for the truncated passes: balls a, b (centre,
// radius; radius < 0: no member) of the two blocks and the (min, max) of their
// members' cutoff terms ra, rb (alpha of points, beta of targets; the pair is
// kept when |x - y|^2 / 2 < alpha_q + beta_j).  0: every pair outside, 1: every
// pair inside, 2: boundary (each pair tested).  The radii are widened /
// narrowed by 1e-4 relative, far more than the rounding of the pairwise tests.
// square root on the SFU (sqrt.approx, relative error about 2^-23): far inside
// the classification margins of 1e-4 relative
__device__ __forceinline__ float sqrt_sfu(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ int tp_class(float4 a, float4 b, float2 ra, float2 rb) {
    if (a.w < 0.f || b.w < 0.f) return 0;
    const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
    const float dist = sqrt_sfu(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    const float Rout = sqrt_sfu(fmaxf(0.f, 2.f * (ra.y + rb.y))) * (1.0f + 1e-4f) + 1e-6f;
    if (dist - a.w - b.w >= Rout) return 0;
    const float Rin = sqrt_sfu(fmaxf(0.f, 2.f * (ra.x + rb.x))) * (1.0f - 1e-4f) - 1e-6f;
    if (dist + a.w + b.w < Rin) return 1;
    return 2;
}

// Block-wide FP64 sum (blockDim.x a multiple of 32, <= 1024); result in thread 0.
__device__ __forceinline__ double block_sum_d(double v, double *sh /* >= 32 */) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;
}

}  // namespace rsot
