// Batched RSOT problems: one persistent launch per pass over a work queue of
// (problem, tile, chunk) items, one CUDA graph per evaluation round, and a
// lockstep host L-BFGS per problem (Algorithm 1) with per-problem
// eps-schedules (Sec. 4.2).
//
// Every problem keeps the single-problem layout of rsot_dense.cu (log2-domain
// target records, translated FP32 points), concatenated:
//   points  : problem p owns [pt_base, pt_base + nq_pad) (nq_pad a multiple of 1024)
//   targets : problem p owns [t_base, t_base + n_alloc)  (n_alloc a multiple of 1024)
//   psi     : problem p owns [psi_off, psi_off + n) of the caller's vector
// Pass 1 items: (p, point tile of 1024, target chunk); pass 2 items: (p, block
// of 1024 targets, point chunk).  Items of a problem are numbered
// tile-major / block-major from item*_base[p], so each point (target) finds
// the partials of its tile (block) without a table, and the merges run in a
// fixed order: the result does not depend on which CTA took which item.
// The work-item size (pairs per item, a power of two) is picked by an
// autotuner that times one round per candidate.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <thread>
#include <cmath>
#include <chrono>
#include <vector>

#include "rsot_inner.cuh"
#include "rsot_internal.cuh"
#include "rsot_tc.cuh"
#include "rsot_lbfgs.h"

namespace rsot {

struct BProb {
    int64_t nq, nq_pad, n, n_alloc, n_p1;
    int64_t pt_base, t_base, psi_off;
    int64_t item1_base, item2_base;
    int64_t chunk2;
    int d, nck1, chunk1, nsp2;
    int pblk_base, tblk_base;   // 256-blocks of points / targets
    double msum, hx;
    float tcP;                  // tensor-core point coordinate scale (rsot_tc.cuh)
};

}  // namespace rsot

struct rsot_batch {
    int count = 0, dev = 0, num_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<rsot_problem *> handles;
    std::vector<rsot::BProb> hp;
    std::vector<double> hnu;          // concatenated nu (caller order), for D in the solver
    rsot::BProb *dp = nullptr;
    int64_t tot_pts = 0, tot_t = 0, tot_n = 0;
    int64_t items1 = 0, items2 = 0, items1_cap = 0, items2_cap = 0;
    int nblk_p = 0, nblk_t = 0;
    int slots1 = 0, slots2 = 0;
    int *blk2prob_p = nullptr, *blk2prob_t = nullptr;
    int64_t *item1_base = nullptr, *item2_base = nullptr;   // count + 1
    float *xs = nullptr;
    double *mass = nullptr, *lm2 = nullptr, *y = nullptr, *nu = nullptr, *lnu = nullptr;
    rsot::Rec8 *tdup = nullptr, *tpair = nullptr, *pdup = nullptr;
    float2 *part1 = nullptr;
    double *part2 = nullptr, *blockJ = nullptr, *psinu = nullptr;
    double *psi_d = nullptr, *grad_d = nullptr, *eps_d = nullptr, *J_d = nullptr;
    unsigned char *active_d = nullptr;
    int *counters = nullptr;   // [0], [1]: work counters, [2]: error flags, [3]: f16 range gate
    rsot::Rec16 *prec16 = nullptr, *trec = nullptr;   // tensor-core operand records
    float *pu = nullptr;                              // pass-2 shifts u_q
    int pair_kernel = 2;       // as rsot_problem::pair_kernel
    bool tc_ok = false;        // every problem meets the automatic choice's bound
    int slots1_tc = 0, slots2_tc = 0;
    double *psi_h = nullptr, *grad_h = nullptr, *eps_h = nullptr, *J_h = nullptr;
    unsigned char *active_h = nullptr;
    int *flags_h = nullptr;
    cudaGraph_t graph = nullptr, graph32 = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphExec_t exec32 = nullptr;   // the same round on the FP32 pair kernels
    std::vector<double> tc_noise;       // per problem, as rsot_problem::tc_noise_l1
    int item_exp = 22;
};

namespace rsot {
namespace {

constexpr int B_T = 256;   // threads of the per-target / per-point kernels
constexpr int kRefineThreads = 8;   // host threads of the per-problem refinement

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

__device__ __forceinline__ int find_prob(const int64_t *__restrict__ base, int count, int64_t item) {
    int lo = 0, hi = count;   // base[lo] <= item < base[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (base[mid] <= item) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void k_bprep(const BProb *__restrict__ probs, const int *__restrict__ blk2prob,
                        const double *__restrict__ psi, const double *__restrict__ eps_v,
                        const unsigned char *__restrict__ active, const double *__restrict__ y,
                        const double *__restrict__ lnu, const double *__restrict__ nu,
                        Rec8 *__restrict__ tdup, Rec8 *__restrict__ tpair,
                        double *__restrict__ psinu, int *__restrict__ flags,
                        Rec16 *__restrict__ trec, int *__restrict__ gate) {
    __shared__ double sh[32];
    const int b = blockIdx.x;
    const int p = blk2prob[b];
    if (!active[p]) return;
    const BProb P = probs[p];
    const int64_t jl = (int64_t)(b - P.tblk_base) * B_T + threadIdx.x;
    const int64_t g = P.t_base + jl;
    const double eps = eps_v[p];
    const double psic = psi[P.psi_off];
    const double k = kLog2e / (2.0 * eps);
    double contrib = 0.0;
    float w[3] = {0.f, 0.f, 0.f};
    float c = kPadC;
    if (jl < P.n) {
        const double ps = psi[P.psi_off + jl];
        if (!isfinite(ps)) atomicOr(flags, kErrNonfinitePsi);
        const double bb = ((ps - psic) / eps + lnu[g]) * kLog2e;
        double yy = 0.0;
        for (int t = 0; t < 3; ++t) {
            const double yt = y[g * 3 + t];
            w[t] = (float)(2.0 * k * yt);
            yy += yt * yt;
        }
        c = (float)(bb - k * yy);
        contrib = ps * nu[g];
    }
    if (trec) {   // tensor-core operands: w / P and c (padding: c at the clamp)
        float W[3];
        bool ok = true;
        for (int t = 0; t < 3; ++t) {
            W[t] = (float)((double)w[t] / (double)P.tcP);
            ok = ok && fabsf(W[t]) < TC_RANGE;
        }
        const float C = fmaxf(c, -256.0f * TC_RANGE);
        ok = ok && C < 256.0f * TC_RANGE;
        if (!ok) atomicOr(gate, 1);
        trec[g] = make_target_rec(W, C);
    }
    Rec8 r;
    r.a = make_float4(w[0], w[0], w[1], w[1]);
    r.b = make_float4(w[2], w[2], c, c);
    tdup[g] = r;
    float *pr = reinterpret_cast<float *>(tpair + (g >> 1));
    const int l = (int)(g & 1);
    pr[0 + l] = w[0];
    pr[2 + l] = w[1];
    pr[4 + l] = w[2];
    pr[6 + l] = c;
    const double s = block_sum_d(contrib, sh);
    if (threadIdx.x == 0) psinu[b] = s;
}

// pass 1 over all problems (3-D arithmetic; 2-D problems carry x2 = y2 = 0)
__global__ void __launch_bounds__(P1_THREADS, 4)
    k_blse(const BProb *__restrict__ probs, int count, const int64_t *__restrict__ item1_base,
           const unsigned char *__restrict__ active, const float *__restrict__ xs,
           const Rec8 *__restrict__ tdup, float2 *__restrict__ part1, int *__restrict__ counter,
           int *__restrict__ flags, const int *__restrict__ gate = nullptr) {
    // as the fallback of the tensor-core pass, run only when the gate asks for it
    if (gate && !(*gate & 1)) return;
    __shared__ __align__(128) Rec8 sm[P1_STAGES][P1_TS];
    __shared__ __align__(8) uint64_t full[P1_STAGES];
    __shared__ int s_abort[2];
    __shared__ long long s_item;
    __shared__ int s_p;
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_abort[0] = s_abort[1] = 0;
        for (int s = 0; s < P1_STAGES; ++s) mbar_init(&full[s], 1);
        fence_barrier_init();
    }
    __syncthreads();
    const int64_t total = item1_base[count];
    unsigned git = 0;
    bool aborted = false;
    for (;;) {
        if (tid == 0) {
            const long long it = atomicAdd(counter, 1);
            s_item = it;
            if (it < total) s_p = find_prob(item1_base, count, it);
        }
        __syncthreads();
        const int64_t item = s_item;
        if (item >= total) break;
        const int p = s_p;
        if (active[p]) {
            const BProb P = probs[p];
            const int64_t local = item - P.item1_base;
            const int64_t tile = local / P.nck1;
            const int c = (int)(local % P.nck1);
            const int64_t t_begin = P.t_base + (int64_t)c * P.chunk1;
            const int ntile = (int)(min((int64_t)P.chunk1, P.n_p1 - (int64_t)c * P.chunk1) / P1_TS);
            if (tid == 0)
                for (int s = 0; s < 2 && s < ntile; ++s) {
                    const unsigned slot = (git + s) & 1u;
                    mbar_expect_tx(&full[slot], P1_TS * sizeof(Rec8));
                    bulk_g2s(sm[slot], tdup + t_begin + (int64_t)s * P1_TS, P1_TS * sizeof(Rec8),
                             &full[slot]);
                }
            const float *xb = xs + 3 * P.pt_base;
            float2 X[P1_PP][3];
#pragma unroll
            for (int pp = 0; pp < P1_PP; ++pp) {
                const int64_t q = tile * P1_TILE + 2 * (pp * P1_THREADS + tid);
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    X[pp][k] = *reinterpret_cast<const float2 *>(xb + k * P.nq_pad + q);
            }
            float2 M[P1_PP], Sf[P1_PP];
            double2 Sd[P1_PP];
#pragma unroll
            for (int pp = 0; pp < P1_PP; ++pp) {
                M[pp] = make_float2(kPadC, kPadC);
                Sf[pp] = make_float2(0.f, 0.f);
                Sd[pp] = make_double2(0.0, 0.0);
            }
            for (int it = 0; it < ntile; ++it) {
                const unsigned gs = git + it, slot = gs & 1u, ph = (gs >> 1) & 1u;
                if (!mbar_wait(&full[slot], ph)) {
                    s_abort[it & 1] = 1;
                    atomicOr(flags, kErrTimeout);
                } else {
                    lse_stage<3, P1_PP>(sm[slot], X, M, Sf, Sd);
                }
                __syncthreads();
                aborted = s_abort[it & 1] != 0;
                if (aborted) break;
                if (tid == 0 && it + 2 < ntile) {
                    mbar_expect_tx(&full[slot], P1_TS * sizeof(Rec8));
                    bulk_g2s(sm[slot], tdup + t_begin + (int64_t)(it + 2) * P1_TS,
                             P1_TS * sizeof(Rec8), &full[slot]);
                }
#pragma unroll
                for (int pp = 0; pp < P1_PP; ++pp) {
                    Sd[pp].x += (double)Sf[pp].x;
                    Sd[pp].y += (double)Sf[pp].y;
                    Sf[pp] = make_float2(0.f, 0.f);
                }
            }
            if (aborted) break;
            git += ntile;
#pragma unroll
            for (int pp = 0; pp < P1_PP; ++pp) {
                const int l = 2 * (pp * P1_THREADS + tid);
                *reinterpret_cast<float4 *>(part1 + item * P1_TILE + l) =
                    make_float4(M[pp].x, (float)Sd[pp].x, M[pp].y, (float)Sd[pp].y);
            }
        }
        __syncthreads();
    }
    if (aborted && tid == 0)
        for (int s = 0; s < 2; ++s) (void)mbar_wait(&full[s], 0u), (void)mbar_wait(&full[s], 1u);
}

__global__ void k_bcombine(const BProb *__restrict__ probs, const int *__restrict__ blk2prob,
                           const unsigned char *__restrict__ active,
                           const float2 *__restrict__ part1, const float *__restrict__ xs,
                           const double *__restrict__ mass, const double *__restrict__ lm2,
                           Rec8 *__restrict__ pdup, double *__restrict__ blockJ,
                           float *__restrict__ pu) {
    __shared__ double sh[32];
    const int b = blockIdx.x;
    const int p = blk2prob[b];
    if (!active[p]) return;
    const BProb P = probs[p];
    const int64_t ql = (int64_t)(b - P.pblk_base) * B_T + threadIdx.x;
    const int64_t g = P.pt_base + ql;
    double contrib = 0.0;
    float x[3];
    for (int t = 0; t < 3; ++t) x[t] = xs[3 * P.pt_base + t * P.nq_pad + ql];
    float u = kPadC;
    if (ql < P.nq) {
        const int64_t tile = ql / P1_TILE;
        const int l = (int)(ql % P1_TILE);
        const int64_t it0 = P.item1_base + tile * P.nck1;
        float mx = kPadC;
        for (int c = 0; c < P.nck1; ++c) mx = fmaxf(mx, part1[(it0 + c) * P1_TILE + l].x);
        double tot = 0.0;
        for (int c = 0; c < P.nck1; ++c) {
            const float2 v = part1[(it0 + c) * P1_TILE + l];
            tot += (double)v.y * pow2_int_d(v.x - mx);
        }
        const double R = (double)mx + log2(tot);
        if (mass[g] > 0.0) {
            contrib = mass[g] * R;
            u = (float)fmax(lm2[g] - R, -1.0e30);
        }
    }
    Rec8 r;
    r.a = make_float4(x[0], x[0], x[1], x[1]);
    r.b = make_float4(x[2], x[2], u, u);
    pdup[g] = r;
    if (pu) pu[g] = u;
    const double s = block_sum_d(contrib, sh);
    if (threadIdx.x == 0) blockJ[b] = s;
}

// ---- tensor-core passes over the batch (rsot_tc.cuh; stage bodies shared with
// the single-problem kernels): CTAs of 16 warps x 4 m-blocks = 1,024 points
// (pass 1) or targets (pass 2), 256-record stages released per warp.
constexpr int BT_THREADS = 512;
constexpr int BT_TS = 256;
static_assert(BT_THREADS / 32 * TC_MB * 16 == P1_TILE, "a pass-1 CTA covers a point tile");

// static point operand records (X = P x')
__global__ void k_bpoint_recs(const BProb *__restrict__ probs, const int *__restrict__ blk2prob,
                              const float *__restrict__ xs, Rec16 *__restrict__ prec) {
    const int b = blockIdx.x;
    const BProb P = probs[blk2prob[b]];
    const int64_t ql = (int64_t)(b - P.pblk_base) * B_T + threadIdx.x;
    float X[3];
    for (int k = 0; k < 3; ++k) X[k] = xs[3 * P.pt_base + k * P.nq_pad + ql] * P.tcP;
    prec[P.pt_base + ql] = make_point_rec(X, 0.0f);
}

__global__ void __launch_bounds__(BT_THREADS, 1)
    k_blse_tc(const BProb *__restrict__ probs, int count, const int64_t *__restrict__ item1_base,
              const unsigned char *__restrict__ active, const Rec16 *__restrict__ prec,
              const Rec16 *__restrict__ trec, float2 *__restrict__ part1,
              int *__restrict__ counter, int *__restrict__ flags, const int *__restrict__ gate) {
    if (*gate & 1) return;   // operands out of f16 range: the FP32 kernel runs
    __shared__ __align__(128) Rec16 sm[2][BT_TS];
    __shared__ __align__(8) uint64_t full[2], empty[2];
    __shared__ long long s_item;
    __shared__ int s_p, s_abort;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = lane >> 2, t = lane & 3;
    if (tid == 0) {
        for (int st = 0; st < 2; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], BT_THREADS / 32);
        }
        fence_barrier_init();
        s_abort = 0;
    }
    __syncthreads();
    const int64_t total = item1_base[count];
    const uint2 *pr = reinterpret_cast<const uint2 *>(prec);
    unsigned git = 0;
    bool aborted = false;
    for (;;) {
        if (tid == 0) {
            const long long it = atomicAdd(counter, 1);
            s_item = it;
            if (it < total) s_p = find_prob(item1_base, count, it);
        }
        __syncthreads();
        const int64_t item = s_item;
        if (item >= total) break;
        const int p = s_p;
        if (active[p]) {
            const BProb P = probs[p];
            const int64_t local = item - P.item1_base;
            const int64_t tile = local / P.nck1;
            const int c = (int)(local % P.nck1);
            const int64_t t_begin = P.t_base + (int64_t)c * P.chunk1;
            const int ntile = (int)(min((int64_t)P.chunk1, P.n_p1 - (int64_t)c * P.chunk1) / BT_TS);
            if (tid == 0)
                for (int st = 0; st < 2 && st < ntile; ++st) {
                    const unsigned slot = (git + st) & 1u;
                    mbar_expect_tx(&full[slot], BT_TS * sizeof(Rec16));
                    bulk_g2s(sm[slot], trec + t_begin + (int64_t)st * BT_TS, BT_TS * sizeof(Rec16),
                             &full[slot]);
                }
            const int64_t q0 = P.pt_base + tile * P1_TILE + warp * (TC_MB * 16);
            unsigned A[TC_MB][4];
            float2 M[TC_MB], Sf[TC_MB];
            double2 Sd[TC_MB];
#pragma unroll
            for (int m = 0; m < TC_MB; ++m) {
                tc_load_a(A[m], pr + (q0 + m * 16) * 4, g, t);
                M[m] = make_float2(-INFINITY, -INFINITY);
                Sf[m] = make_float2(0.f, 0.f);
                Sd[m] = make_double2(0.0, 0.0);
            }
            bool wabort = false;
            for (int it = 0; it < ntile; ++it) {
                const unsigned gs = git + it, slot = gs & 1u, ph = (gs >> 1) & 1u;
                if (!__all_sync(0xffffffffu, mbar_wait(&full[slot], ph))) {
                    s_abort = 1;
                    atomicOr(flags, kErrTimeout);
                    wabort = true;
                    break;
                }
                tc_lse_stage<BT_TS / 8>(reinterpret_cast<const uint2 *>(&sm[slot][0]) + lane, A, M, Sf, Sd);
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[slot]);
                if (warp == 0 && it + 2 < ntile) {
                    bool ok = true;
                    if (tid == 0) {
                        ok = mbar_wait(&empty[slot], ph);
                        if (ok) {
                            mbar_expect_tx(&full[slot], BT_TS * sizeof(Rec16));
                            bulk_g2s(sm[slot], trec + t_begin + (int64_t)(it + 2) * BT_TS,
                                     BT_TS * sizeof(Rec16), &full[slot]);
                        }
                    }
                    if (!__shfl_sync(0xffffffffu, ok, 0)) {
                        s_abort = 1;
                        atomicOr(flags, kErrTimeout);
                        wabort = true;
                        break;
                    }
                }
#pragma unroll
                for (int m = 0; m < TC_MB; ++m) {
                    Sd[m].x += (double)Sf[m].x;
                    Sd[m].y += (double)Sf[m].y;
                    Sf[m] = make_float2(0.f, 0.f);
                }
            }
            git += ntile;
            if (!wabort) {
#pragma unroll
                for (int m = 0; m < TC_MB; ++m) {
                    float mx = M[m].x, my = M[m].y;
                    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
                    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
                    my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, 1));
                    my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, 2));
                    double sx = M[m].x == -INFINITY ? 0.0 : Sd[m].x * pow2_int_d(M[m].x - mx);
                    double sy = M[m].y == -INFINITY ? 0.0 : Sd[m].y * pow2_int_d(M[m].y - my);
                    sx += __shfl_xor_sync(0xffffffffu, sx, 1);
                    sx += __shfl_xor_sync(0xffffffffu, sx, 2);
                    sy += __shfl_xor_sync(0xffffffffu, sy, 1);
                    sy += __shfl_xor_sync(0xffffffffu, sy, 2);
                    if (m == t) {
                        float2 *o = part1 + item * P1_TILE + warp * (TC_MB * 16) + m * 16 + g;
                        o[0] = mx == -INFINITY ? make_float2(kPadC, 0.f) : make_float2(mx, (float)sx);
                        o[8] = my == -INFINITY ? make_float2(kPadC, 0.f) : make_float2(my, (float)sy);
                    }
                }
            }
        }
        __syncthreads();   // end of the item: every warp is past its stages
        if (s_abort) {
            aborted = true;
            break;
        }
    }
    if (aborted && tid == 0)
        for (int st = 0; st < 2; ++st) (void)mbar_wait(&full[st], 0u), (void)mbar_wait(&full[st], 1u);
}

__global__ void __launch_bounds__(BT_THREADS, 1)
    k_bgrad_tc(const BProb *__restrict__ probs, int count, const int64_t *__restrict__ item2_base,
               const unsigned char *__restrict__ active, const Rec16 *__restrict__ trec,
               const Rec16 *__restrict__ prec, const float *__restrict__ pu,
               double *__restrict__ part2, int *__restrict__ counter, int *__restrict__ flags,
               const int *__restrict__ gate) {
    if (*gate & 1) return;   // operands out of f16 range: the FP32 kernel runs
    __shared__ __align__(128) Rec16 sm[2][BT_TS];
    __shared__ __align__(16) float su[2][BT_TS];
    __shared__ __align__(8) uint64_t full[2], empty[2];
    __shared__ long long s_item;
    __shared__ int s_p, s_abort;
    constexpr unsigned kStage = BT_TS * (sizeof(Rec16) + sizeof(float));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = lane >> 2, t = lane & 3;
    if (tid == 0) {
        for (int st = 0; st < 2; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], BT_THREADS / 32);
        }
        fence_barrier_init();
        s_abort = 0;
    }
    __syncthreads();
    const int64_t total = item2_base[count];
    const uint2 *tr = reinterpret_cast<const uint2 *>(trec);
    unsigned git = 0;
    bool aborted = false;
    for (;;) {
        if (tid == 0) {
            const long long it = atomicAdd(counter, 1);
            s_item = it;
            if (it < total) s_p = find_prob(item2_base, count, it);
        }
        __syncthreads();
        const int64_t item = s_item;
        if (item >= total) break;
        const int p = s_p;
        if (active[p]) {
            const BProb P = probs[p];
            const int64_t local = item - P.item2_base;
            const int64_t blk = local / P.nsp2;
            const int sp = (int)(local % P.nsp2);
            const int64_t p_begin = P.pt_base + (int64_t)sp * P.chunk2;
            const int ntile = (int)(min(P.chunk2, P.nq_pad - (int64_t)sp * P.chunk2) / BT_TS);
            if (tid == 0)
                for (int st = 0; st < 2 && st < ntile; ++st) {
                    const unsigned slot = (git + st) & 1u;
                    mbar_expect_tx(&full[slot], kStage);
                    bulk_g2s(sm[slot], prec + p_begin + (int64_t)st * BT_TS, BT_TS * sizeof(Rec16),
                             &full[slot]);
                    bulk_g2s(su[slot], pu + p_begin + (int64_t)st * BT_TS, BT_TS * sizeof(float),
                             &full[slot]);
                }
            const int64_t j0 = P.t_base + blk * 1024 + warp * (TC_MB * 16);
            unsigned A[TC_MB][4];
            double2 acc64[TC_MB];
#pragma unroll
            for (int m = 0; m < TC_MB; ++m) {
                tc_load_a(A[m], tr + (j0 + m * 16) * 4, g, t);
                acc64[m] = make_double2(0.0, 0.0);
            }
            bool wabort = false;
            for (int it = 0; it < ntile; ++it) {
                const unsigned gs = git + it, slot = gs & 1u, ph = (gs >> 1) & 1u;
                if (!__all_sync(0xffffffffu, mbar_wait(&full[slot], ph))) {
                    s_abort = 1;
                    atomicOr(flags, kErrTimeout);
                    wabort = true;
                    break;
                }
                tc_grad_stage<BT_TS / 8>(reinterpret_cast<const uint2 *>(&sm[slot][0]) + lane,
                                         reinterpret_cast<const float2 *>(&su[slot][0]) + t, A, acc64);
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[slot]);
                if (warp == 0 && it + 2 < ntile) {
                    bool ok = true;
                    if (tid == 0) {
                        ok = mbar_wait(&empty[slot], ph);
                        if (ok) {
                            mbar_expect_tx(&full[slot], kStage);
                            bulk_g2s(sm[slot], prec + p_begin + (int64_t)(it + 2) * BT_TS,
                                     BT_TS * sizeof(Rec16), &full[slot]);
                            bulk_g2s(su[slot], pu + p_begin + (int64_t)(it + 2) * BT_TS,
                                     BT_TS * sizeof(float), &full[slot]);
                        }
                    }
                    if (!__shfl_sync(0xffffffffu, ok, 0)) {
                        s_abort = 1;
                        atomicOr(flags, kErrTimeout);
                        wabort = true;
                        break;
                    }
                }
            }
            git += ntile;
            if (!wabort) {
#pragma unroll
                for (int m = 0; m < TC_MB; ++m) {
                    double x = acc64[m].x, y = acc64[m].y;
                    x += __shfl_xor_sync(0xffffffffu, x, 1);
                    x += __shfl_xor_sync(0xffffffffu, x, 2);
                    y += __shfl_xor_sync(0xffffffffu, y, 1);
                    y += __shfl_xor_sync(0xffffffffu, y, 2);
                    if (m == t) {
                        double *o = part2 + item * 1024 + warp * (TC_MB * 16) + m * 16 + g;
                        o[0] = x;
                        o[8] = y;
                    }
                }
            }
        }
        __syncthreads();
        if (s_abort) {
            aborted = true;
            break;
        }
    }
    if (aborted && tid == 0)
        for (int st = 0; st < 2; ++st) (void)mbar_wait(&full[st], 0u), (void)mbar_wait(&full[st], 1u);
}

constexpr int B_TPP = 4;   // pass 2: 1024 targets per block

__global__ void __launch_bounds__(P2_THREADS)
    k_bgrad(const BProb *__restrict__ probs, int count, const int64_t *__restrict__ item2_base,
            const unsigned char *__restrict__ active, const Rec8 *__restrict__ tpair,
            const Rec8 *__restrict__ pdup, double *__restrict__ part2, int *__restrict__ counter,
            int *__restrict__ flags, const int *__restrict__ gate = nullptr) {
    if (gate && !(*gate & 1)) return;
    __shared__ __align__(128) Rec8 sm[P2_STAGES][P2_TS];
    __shared__ __align__(8) uint64_t full[P2_STAGES];
    __shared__ int s_abort[2];
    __shared__ long long s_item;
    __shared__ int s_p;
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_abort[0] = s_abort[1] = 0;
        for (int s = 0; s < P2_STAGES; ++s) mbar_init(&full[s], 1);
        fence_barrier_init();
    }
    __syncthreads();
    const int64_t total = item2_base[count];
    unsigned git = 0;
    bool aborted = false;
    for (;;) {
        if (tid == 0) {
            const long long it = atomicAdd(counter, 1);
            s_item = it;
            if (it < total) s_p = find_prob(item2_base, count, it);
        }
        __syncthreads();
        const int64_t item = s_item;
        if (item >= total) break;
        const int p = s_p;
        if (active[p]) {
            const BProb P = probs[p];
            const int64_t local = item - P.item2_base;
            const int64_t blk = local / P.nsp2;
            const int s = (int)(local % P.nsp2);
            const int64_t p_begin = P.pt_base + (int64_t)s * P.chunk2;
            const int ntile = (int)(min(P.chunk2, P.nq_pad - (int64_t)s * P.chunk2) / P2_TS);
            if (tid == 0)
                for (int st = 0; st < 2 && st < ntile; ++st) {
                    const unsigned slot = (git + st) & 1u;
                    mbar_expect_tx(&full[slot], P2_TS * sizeof(Rec8));
                    bulk_g2s(sm[slot], pdup + p_begin + (int64_t)st * P2_TS, P2_TS * sizeof(Rec8),
                             &full[slot]);
                }
            const int64_t g0 = P.t_base / 2 + blk * (P2_THREADS * B_TPP);
            float2 W0[B_TPP], W1[B_TPP], W2[B_TPP], C[B_TPP];
            double2 acc64[B_TPP];
#pragma unroll
            for (int tp = 0; tp < B_TPP; ++tp) {
                const Rec8 r = tpair[g0 + tp * P2_THREADS + tid];
                W0[tp] = make_float2(r.a.x, r.a.y);
                W1[tp] = make_float2(r.a.z, r.a.w);
                W2[tp] = make_float2(r.b.x, r.b.y);
                C[tp] = make_float2(r.b.z, r.b.w);
                acc64[tp] = make_double2(0.0, 0.0);
            }
            for (int it = 0; it < ntile; ++it) {
                const unsigned gs = git + it, slot = gs & 1u, ph = (gs >> 1) & 1u;
                if (!mbar_wait(&full[slot], ph)) {
                    s_abort[it & 1] = 1;
                    atomicOr(flags, kErrTimeout);
                } else {
                    grad_stage<3, B_TPP>(sm[slot], W0, W1, W2, C, acc64);
                }
                __syncthreads();
                aborted = s_abort[it & 1] != 0;
                if (aborted) break;
                if (tid == 0 && it + 2 < ntile) {
                    mbar_expect_tx(&full[slot], P2_TS * sizeof(Rec8));
                    bulk_g2s(sm[slot], pdup + p_begin + (int64_t)(it + 2) * P2_TS,
                             P2_TS * sizeof(Rec8), &full[slot]);
                }
            }
            if (aborted) break;
            git += ntile;
#pragma unroll
            for (int tp = 0; tp < B_TPP; ++tp) {
                const int64_t j = 2 * (tp * P2_THREADS + tid);
                *reinterpret_cast<double2 *>(part2 + item * (2 * P2_THREADS * B_TPP) + j) = acc64[tp];
            }
        }
        __syncthreads();
    }
    if (aborted && tid == 0)
        for (int s = 0; s < 2; ++s) (void)mbar_wait(&full[s], 0u), (void)mbar_wait(&full[s], 1u);
}

__global__ void k_bfinal_grad(const BProb *__restrict__ probs, const int *__restrict__ blk2prob,
                              const unsigned char *__restrict__ active,
                              const double *__restrict__ part2, const double *__restrict__ nu,
                              double *__restrict__ grad) {
    const int b = blockIdx.x;
    const int p = blk2prob[b];
    if (!active[p]) return;
    const BProb P = probs[p];
    const int64_t jl = (int64_t)(b - P.tblk_base) * B_T + threadIdx.x;
    if (jl >= P.n) return;
    const int64_t blk = jl / (2 * P2_THREADS * B_TPP);
    const int l = (int)(jl % (2 * P2_THREADS * B_TPP));
    const int64_t it0 = P.item2_base + blk * P.nsp2;
    double g = 0.0;
    for (int s = 0; s < P.nsp2; ++s) g += part2[(it0 + s) * (2 * P2_THREADS * B_TPP) + l];
    grad[P.psi_off + jl] = g - nu[P.t_base + jl];
}

__global__ void k_bfinal_J(const BProb *__restrict__ probs, const unsigned char *__restrict__ active,
                           const double *__restrict__ blockJ, const double *__restrict__ psinu,
                           const double *__restrict__ psi, const double *__restrict__ eps_v,
                           double *__restrict__ J) {
    __shared__ double sh[32];
    const int p = blockIdx.x;
    if (!active[p]) return;
    const BProb P = probs[p];
    double a = 0.0, b = 0.0;
    const int nbp = (int)(P.nq_pad / B_T), nbt = (int)(P.n_alloc / B_T);
    for (int i = threadIdx.x; i < nbp; i += blockDim.x) a += blockJ[P.pblk_base + i];
    for (int i = threadIdx.x; i < nbt; i += blockDim.x) b += psinu[P.tblk_base + i];
    const double sa = block_sum_d(a, sh), sb = block_sum_d(b, sh);
    if (threadIdx.x == 0)
        J[p] = psi[P.psi_off] * P.msum - P.hx + eps_v[p] * kLn2 * sa - sb;
}

int occ(const void *fn, int threads) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, 0) != cudaSuccess || nb < 1)
        nb = 1;
    return nb;
}

rsot_status to_status(cudaError_t e) {
    if (e == cudaSuccess) return RSOT_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? RSOT_ERR_NOMEM : RSOT_ERR_CUDA;
}

// Item numbering for work items of about 2^e pairs.
void plan_items(rsot_batch *b, int e) {
    const int64_t pairs = (int64_t)1 << e;
    int64_t i1 = 0, i2 = 0;
    for (auto &P : b->hp) {
        const int64_t want1 = std::max<int64_t>(P1_TS, round_up(pairs / P1_TILE, P1_TS));
        int64_t ch1 = std::min(want1, P.n_p1);
        P.nck1 = (int)((P.n_p1 + ch1 - 1) / ch1);
        P.chunk1 = (int)round_up((P.n_p1 + P.nck1 - 1) / P.nck1, P1_TS);
        P.nck1 = (int)((P.n_p1 + P.chunk1 - 1) / P.chunk1);
        const int64_t want2 = std::max<int64_t>(P2_TS, round_up(pairs / 1024, P2_TS));
        int64_t ch2 = std::min(want2, P.nq_pad);
        P.nsp2 = (int)((P.nq_pad + ch2 - 1) / ch2);
        P.chunk2 = round_up((P.nq_pad + P.nsp2 - 1) / P.nsp2, P2_TS);
        P.nsp2 = (int)((P.nq_pad + P.chunk2 - 1) / P.chunk2);
        P.item1_base = i1;
        P.item2_base = i2;
        i1 += (P.nq_pad / P1_TILE) * P.nck1;
        i2 += (P.n_alloc / 1024) * P.nsp2;
    }
    b->items1 = i1;
    b->items2 = i2;
}

cudaError_t upload_plan(rsot_batch *b) {
    cudaError_t e;
    if (b->items1 > b->items1_cap) {
        cudaFree(b->part1);
        if ((e = cudaMalloc(&b->part1, (size_t)b->items1 * P1_TILE * sizeof(float2)))) return e;
        b->items1_cap = b->items1;
    }
    if (b->items2 > b->items2_cap) {
        cudaFree(b->part2);
        if ((e = cudaMalloc(&b->part2, (size_t)b->items2 * 1024 * sizeof(double)))) return e;
        b->items2_cap = b->items2;
    }
    std::vector<int64_t> i1(b->count + 1), i2(b->count + 1);
    for (int p = 0; p < b->count; ++p) {
        i1[p] = b->hp[p].item1_base;
        i2[p] = b->hp[p].item2_base;
    }
    i1[b->count] = b->items1;
    i2[b->count] = b->items2;
    if ((e = cudaMemcpy(b->dp, b->hp.data(), b->hp.size() * sizeof(BProb), cudaMemcpyHostToDevice)))
        return e;
    if ((e = cudaMemcpy(b->item1_base, i1.data(), i1.size() * 8, cudaMemcpyHostToDevice))) return e;
    return cudaMemcpy(b->item2_base, i2.data(), i2.size() * 8, cudaMemcpyHostToDevice);
}

// Record one evaluation round on b->stream (graph capture or direct launch).
cudaError_t enqueue_round(rsot_batch *b, bool force_fp32 = false) {
    cudaStream_t st = b->stream;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(b->psi_d, b->psi_h, b->tot_n * 8, cudaMemcpyHostToDevice, st))) return e;
    if ((e = cudaMemcpyAsync(b->eps_d, b->eps_h, b->count * 8, cudaMemcpyHostToDevice, st))) return e;
    if ((e = cudaMemcpyAsync(b->active_d, b->active_h, b->count, cudaMemcpyHostToDevice, st))) return e;
    if ((e = cudaMemsetAsync(b->counters, 0, 4 * sizeof(int), st))) return e;
    // tensor-core passes (automatic choice), FP32 passes as their fallback when an
    // operand leaves the f16 range (gate)
    const bool tc = !force_fp32 && (b->pair_kernel == 1 || (b->pair_kernel == 2 && b->tc_ok));
    int *gate = tc ? b->counters + 3 : nullptr;
    k_bprep<<<b->nblk_t, B_T, 0, st>>>(b->dp, b->blk2prob_t, b->psi_d, b->eps_d, b->active_d, b->y,
                                      b->lnu, b->nu, b->tdup, b->tpair, b->psinu, b->counters + 2,
                                      tc ? b->trec : nullptr, gate);
    if (tc)
        k_blse_tc<<<b->slots1_tc, BT_THREADS, 0, st>>>(b->dp, b->count, b->item1_base, b->active_d,
                                                       b->prec16, b->trec, b->part1, b->counters,
                                                       b->counters + 2, gate);
    k_blse<<<b->slots1, P1_THREADS, 0, st>>>(b->dp, b->count, b->item1_base, b->active_d, b->xs,
                                             b->tdup, b->part1, b->counters, b->counters + 2, gate);
    k_bcombine<<<b->nblk_p, B_T, 0, st>>>(b->dp, b->blk2prob_p, b->active_d, b->part1, b->xs,
                                         b->mass, b->lm2, b->pdup, b->blockJ,
                                         tc ? b->pu : nullptr);
    if (tc)
        k_bgrad_tc<<<b->slots2_tc, BT_THREADS, 0, st>>>(b->dp, b->count, b->item2_base, b->active_d,
                                                        b->trec, b->prec16, b->pu, b->part2,
                                                        b->counters + 1, b->counters + 2, gate);
    k_bgrad<<<b->slots2, P2_THREADS, 0, st>>>(b->dp, b->count, b->item2_base, b->active_d,
                                              b->tpair, b->pdup, b->part2, b->counters + 1,
                                              b->counters + 2, gate);
    k_bfinal_grad<<<b->nblk_t, B_T, 0, st>>>(b->dp, b->blk2prob_t, b->active_d, b->part2, b->nu,
                                            b->grad_d);
    k_bfinal_J<<<b->count, B_T, 0, st>>>(b->dp, b->active_d, b->blockJ, b->psinu, b->psi_d,
                                        b->eps_d, b->J_d);
    if ((e = cudaGetLastError())) return e;
    if ((e = cudaMemcpyAsync(b->grad_h, b->grad_d, b->tot_n * 8, cudaMemcpyDeviceToHost, st))) return e;
    if ((e = cudaMemcpyAsync(b->J_h, b->J_d, b->count * 8, cudaMemcpyDeviceToHost, st))) return e;
    return cudaMemcpyAsync(b->flags_h, b->counters + 2, sizeof(int), cudaMemcpyDeviceToHost, st);
}

cudaError_t capture(rsot_batch *b, bool force_fp32, cudaGraph_t *g, cudaGraphExec_t *x) {
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e) return e;
    cudaError_t e2 = enqueue_round(b, force_fp32);
    e = cudaStreamEndCapture(b->stream, g);
    if (e2) return e2;
    if (e) return e;
    return cudaGraphInstantiate(x, *g, 0);
}

cudaError_t build_graph(rsot_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->exec32) cudaGraphExecDestroy(b->exec32);
    if (b->graph32) cudaGraphDestroy(b->graph32);
    b->exec = b->exec32 = nullptr;
    b->graph = b->graph32 = nullptr;
    cudaError_t e = capture(b, false, &b->graph, &b->exec);
    if (!e) e = capture(b, true, &b->graph32, &b->exec32);
    return e;
}

// One round with the current host staging buffers (psi_h, eps_h, active_h);
// fp32: on the FP32 pair kernels whatever the automatic choice.
rsot_status run_round(rsot_batch *b, bool fp32 = false) {
    cudaGraphExec_t x = fp32 ? b->exec32 : b->exec;
    cudaError_t e = x ? cudaGraphLaunch(x, b->stream) : enqueue_round(b, fp32);
    if (!e) e = cudaStreamSynchronize(b->stream);
    if (e) return to_status(e);
    if (*b->flags_h & kErrTimeout) return RSOT_ERR_TIMEOUT;
    if (*b->flags_h & kErrNonfinitePsi) return RSOT_ERR_NONFINITE;
    return RSOT_OK;
}

}  // namespace
}  // namespace rsot

using namespace rsot;

extern "C" {

void rsot_batch_destroy(rsot_batch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->exec32) cudaGraphExecDestroy(b->exec32);
    if (b->graph32) cudaGraphDestroy(b->graph32);
    for (rsot_problem *h : b->handles) rsot_destroy(h);
    void *dev[] = {b->dp, b->blk2prob_p, b->blk2prob_t, b->item1_base, b->item2_base, b->xs,
                   b->mass, b->lm2, b->y, b->nu, b->lnu, b->tdup, b->tpair, b->pdup, b->part1,
                   b->part2, b->blockJ, b->psinu, b->psi_d, b->grad_d, b->eps_d, b->J_d,
                   b->active_d, b->counters, b->prec16, b->trec, b->pu};
    for (void *q : dev) cudaFree(q);
    void *host[] = {b->psi_h, b->grad_h, b->eps_h, b->J_h, b->active_h, b->flags_h};
    for (void *q : host)
        if (q) cudaFreeHost(q);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

int64_t rsot_batch_total_targets(const rsot_batch *b) { return b ? b->tot_n : 0; }

rsot_status rsot_batch_create(int count, const rsot_problem_desc *probs, rsot_batch **out) {
    if (!out || count < 1 || !probs) return RSOT_ERR_ARG;
    *out = nullptr;
    rsot_batch *b = new rsot_batch();
    b->count = count;
    cudaGetDevice(&b->dev);
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->dev);
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)) {
        delete b;
        return RSOT_ERR_CUDA;
    }
    b->own_stream = true;
    // host-side layouts
    std::vector<float> hxs;
    std::vector<double> hmass, hlm2, hy, hnu, hlnu;
    std::vector<int> bp, bt;
    bool tc_all = true;
    b->hp.resize(count);
    for (int p = 0; p < count; ++p) {
        const rsot_problem_desc &D = probs[p];
        if ((D.d != 2 && D.d != 3) || D.nq < 1 || D.n < 1 || !D.x || !D.mass || !D.y || !D.nu) {
            rsot_batch_destroy(b);
            return RSOT_ERR_ARG;
        }
        rsot_problem *h = nullptr;
        rsot_status s = rsot_create(D.d, D.nq, D.x, D.mass, D.n, D.y, D.nu, 0, &h);
        if (s) {
            rsot_batch_destroy(b);
            return s;
        }
        b->handles.push_back(h);
        std::vector<double> x((size_t)D.nq * D.d), m(D.nq), y((size_t)D.n * D.d), nu(D.n);
        cudaMemcpy(x.data(), D.x, x.size() * 8, cudaMemcpyDefault);
        cudaMemcpy(m.data(), D.mass, m.size() * 8, cudaMemcpyDefault);
        cudaMemcpy(y.data(), D.y, y.size() * 8, cudaMemcpyDefault);
        cudaMemcpy(nu.data(), D.nu, nu.size() * 8, cudaMemcpyDefault);
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (size_t i = 0; i < x.size(); ++i) {
            lo[i % D.d] = std::min(lo[i % D.d], x[i]);
            hi[i % D.d] = std::max(hi[i % D.d], x[i]);
        }
        for (size_t i = 0; i < y.size(); ++i) {
            lo[i % D.d] = std::min(lo[i % D.d], y[i]);
            hi[i % D.d] = std::max(hi[i % D.d], y[i]);
        }
        double o[3] = {0, 0, 0};
        for (int k = 0; k < D.d; ++k) o[k] = 0.5 * (lo[k] + hi[k]);
        BProb &P = b->hp[p];
        P.d = D.d;
        P.nq = D.nq;
        P.nq_pad = round_up(D.nq, P1_TILE);
        P.n = D.n;
        P.n_alloc = round_up(D.n, 1024);
        P.n_p1 = round_up(D.n, P1_TS);
        P.pt_base = b->tot_pts;
        P.t_base = b->tot_t;
        P.psi_off = b->tot_n;
        P.pblk_base = (int)(b->tot_pts / B_T);
        P.tblk_base = (int)(b->tot_t / B_T);
        const size_t xs0 = hxs.size();
        hxs.resize(xs0 + 3 * P.nq_pad, 0.0f);
        hmass.resize(b->tot_pts + P.nq_pad, 0.0);
        hlm2.resize(b->tot_pts + P.nq_pad, -INFINITY);
        double msum = 0.0, hxv = 0.0;
        for (int64_t q = 0; q < D.nq; ++q) {
            double r2 = 0.0;
            for (int k = 0; k < D.d; ++k) {
                const double v = x[q * D.d + k] - o[k];
                hxs[xs0 + k * P.nq_pad + q] = (float)v;
                r2 += v * v;
            }
            hmass[P.pt_base + q] = m[q];
            hlm2[P.pt_base + q] = m[q] > 0.0 ? log2(m[q]) : -INFINITY;
            msum += m[q];
            hxv += m[q] * 0.5 * r2;
        }
        P.msum = msum;
        P.hx = hxv;
        {   // tensor-core scale: P x' within [-32, 32] (a power of two)
            float xmax = 0.0f;
            for (int k = 0; k < 3; ++k)
                for (int64_t q = 0; q < D.nq; ++q) xmax = std::max(xmax, std::fabs(hxs[xs0 + k * P.nq_pad + q]));
            int ex = 0;
            if (xmax > 0.0f) std::frexp(xmax, &ex);
            P.tcP = std::ldexp(1.0f, 5 - ex);
            double mmax = 0.0, numax = 0.0;
            for (int64_t q = 0; q < D.nq; ++q) mmax = std::max(mmax, m[q]);
            double sq = 0.0;
            for (int64_t j = 0; j < D.n; ++j) {
                numax = std::max(numax, nu[j]);
                sq += std::sqrt(nu[j]);
            }
            tc_all = tc_all && mmax * numax <= kTcAuto;
            b->tc_noise.push_back(1.4e-5 * std::sqrt(mmax) * sq);
        }
        hy.resize(3 * (b->tot_t + P.n_alloc), 0.0);
        hnu.resize(b->tot_t + P.n_alloc, 0.0);
        hlnu.resize(b->tot_t + P.n_alloc, 0.0);
        for (int64_t j = 0; j < D.n; ++j) {
            for (int k = 0; k < D.d; ++k) hy[3 * (P.t_base + j) + k] = y[j * D.d + k] - o[k];
            hnu[P.t_base + j] = nu[j];
            hlnu[P.t_base + j] = log(nu[j]);
            b->hnu.push_back(nu[j]);
        }
        for (int64_t i = 0; i < P.nq_pad / B_T; ++i) bp.push_back(p);
        for (int64_t i = 0; i < P.n_alloc / B_T; ++i) bt.push_back(p);
        b->tot_pts += P.nq_pad;
        b->tot_t += P.n_alloc;
        b->tot_n += D.n;
    }
    b->nblk_p = (int)bp.size();
    b->nblk_t = (int)bt.size();
    cudaError_t e = cudaSuccess;
#define BALLOC(ptr, cnt) \
    if (!e) e = cudaMalloc(&(ptr), (size_t)(cnt) * sizeof(*(ptr)))
    BALLOC(b->dp, count);
    BALLOC(b->blk2prob_p, b->nblk_p);
    BALLOC(b->blk2prob_t, b->nblk_t);
    BALLOC(b->item1_base, count + 1);
    BALLOC(b->item2_base, count + 1);
    BALLOC(b->xs, hxs.size());
    BALLOC(b->mass, b->tot_pts);
    BALLOC(b->lm2, b->tot_pts);
    BALLOC(b->y, 3 * b->tot_t);
    BALLOC(b->nu, b->tot_t);
    BALLOC(b->lnu, b->tot_t);
    BALLOC(b->tdup, b->tot_t);
    BALLOC(b->tpair, b->tot_t / 2);
    BALLOC(b->pdup, b->tot_pts);
    BALLOC(b->blockJ, b->nblk_p);
    BALLOC(b->psinu, b->nblk_t);
    BALLOC(b->psi_d, b->tot_n);
    BALLOC(b->grad_d, b->tot_n);
    BALLOC(b->eps_d, count);
    BALLOC(b->J_d, count);
    BALLOC(b->active_d, count);
    BALLOC(b->counters, 4);
    BALLOC(b->prec16, b->tot_pts);
    BALLOC(b->trec, b->tot_t);
    BALLOC(b->pu, b->tot_pts);
#undef BALLOC
    if (!e) e = cudaMallocHost(&b->psi_h, b->tot_n * 8);
    if (!e) e = cudaMallocHost(&b->grad_h, b->tot_n * 8);
    if (!e) e = cudaMallocHost(&b->eps_h, count * 8);
    if (!e) e = cudaMallocHost(&b->J_h, count * 8);
    if (!e) e = cudaMallocHost(&b->active_h, count);
    if (!e) e = cudaMallocHost(&b->flags_h, sizeof(int));
    if (!e) e = cudaMemcpy(b->blk2prob_p, bp.data(), bp.size() * 4, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(b->blk2prob_t, bt.data(), bt.size() * 4, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(b->xs, hxs.data(), hxs.size() * 4, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(b->mass, hmass.data(), hmass.size() * 8, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(b->lm2, hlm2.data(), hlm2.size() * 8, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(b->y, hy.data(), hy.size() * 8, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(b->nu, hnu.data(), hnu.size() * 8, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(b->lnu, hlnu.data(), hlnu.size() * 8, cudaMemcpyHostToDevice);
    if (e) {
        cudaGetLastError();
        rsot_batch_destroy(b);
        return to_status(e);
    }
    b->tc_ok = tc_all;
    if (!e) e = cudaMemcpy(b->dp, b->hp.data(), b->hp.size() * sizeof(BProb), cudaMemcpyHostToDevice);
    if (!e) {
        k_bpoint_recs<<<b->nblk_p, B_T>>>(b->dp, b->blk2prob_p, b->xs, b->prec16);
        e = cudaDeviceSynchronize();
    }
    if (e) {
        cudaGetLastError();
        rsot_batch_destroy(b);
        return to_status(e);
    }
    b->slots1 = b->num_sms * occ((const void *)k_blse, P1_THREADS);
    b->slots2 = b->num_sms * occ((const void *)k_bgrad, P2_THREADS);
    b->slots1_tc = b->num_sms * occ((const void *)k_blse_tc, BT_THREADS);
    b->slots2_tc = b->num_sms * occ((const void *)k_bgrad_tc, BT_THREADS);
    plan_items(b, b->item_exp);
    e = upload_plan(b);
    if (!e) e = build_graph(b);
    if (e) {
        cudaGetLastError();
        rsot_batch_destroy(b);
        return to_status(e);
    }
    *out = b;
    return RSOT_OK;
}

rsot_status rsot_batch_set_pair_kernel(rsot_batch *b, rsot_pair_kernel kind) {
    if (!b || (kind != RSOT_PAIRS_FP32 && kind != RSOT_PAIRS_TENSOR && kind != RSOT_PAIRS_AUTO))
        return RSOT_ERR_ARG;
    b->pair_kernel = (int)kind;
    return to_status(build_graph(b));
}

rsot_status rsot_batch_set_stream(rsot_batch *b, void *stream) {
    if (!b || !stream) return RSOT_ERR_ARG;   // graph capture needs a non-default stream
    if (b->own_stream) cudaStreamDestroy(b->stream);
    b->own_stream = false;
    b->stream = (cudaStream_t)stream;
    return to_status(build_graph(b));
}

// One batched evaluation; solver_round: a round of the batched solver (the
// tensor-core form under RSOT_PAIRS_AUTO), else an evaluation returned to the
// caller (FP32 pair arithmetic unless RSOT_PAIRS_TENSOR)
static rsot_status batch_eval_impl(rsot_batch *b, const double *psi_all, const double *eps,
                                   const unsigned char *active, double *J_out, double *grad_all,
                                   bool solver_round) {
    if (!b || !psi_all || !eps || !J_out || !grad_all) return RSOT_ERR_ARG;
    for (int p = 0; p < b->count; ++p)
        if (!(eps[p] > 0.0) || !isfinite(eps[p])) return RSOT_ERR_ARG;
    memcpy(b->psi_h, psi_all, b->tot_n * 8);
    memcpy(b->eps_h, eps, b->count * 8);
    for (int p = 0; p < b->count; ++p) b->active_h[p] = active ? (active[p] ? 1 : 0) : 1;
    rsot_status s = run_round(b, !(b->pair_kernel == 1 || (b->pair_kernel == 2 && solver_round)));
    if (s) return s;
    for (int p = 0; p < b->count; ++p) {
        if (!b->active_h[p]) continue;
        J_out[p] = b->J_h[p];
        const BProb &P = b->hp[p];
        memcpy(grad_all + P.psi_off, b->grad_h + P.psi_off, P.n * 8);
    }
    return RSOT_OK;
}

rsot_status rsot_batch_eval(rsot_batch *b, const double *psi_all, const double *eps,
                            const unsigned char *active, double *J_out, double *grad_all) {
    return batch_eval_impl(b, psi_all, eps, active, J_out, grad_all, false);
}

rsot_status rsot_batch_tune(rsot_batch *b, const double *psi_all, const double *eps, int *choice_out) {
    if (!b || !psi_all || !eps) return RSOT_ERR_ARG;
    std::vector<double> J(b->count), g(b->tot_n);
    double best_t = INFINITY;
    int best = b->item_exp;
    for (int e = 21; e <= 24; ++e) {
        plan_items(b, e);
        cudaError_t ce = upload_plan(b);
        if (!ce) ce = build_graph(b);
        if (ce) return to_status(ce);
        // the solver's rounds are what the item size is tuned for
        rsot_status s = batch_eval_impl(b, psi_all, eps, nullptr, J.data(), g.data(), true);   // warm
        if (s) return s;
        const auto t0 = std::chrono::steady_clock::now();
        s = batch_eval_impl(b, psi_all, eps, nullptr, J.data(), g.data(), true);
        if (s) return s;
        const double t = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (t < best_t) {
            best_t = t;
            best = e;
        }
    }
    b->item_exp = best;
    plan_items(b, best);
    cudaError_t ce = upload_plan(b);
    if (!ce) ce = build_graph(b);
    if (choice_out) *choice_out = best;
    return to_status(ce);
}

rsot_status rsot_batch_solve(rsot_batch *b, double *psi_all, const double *eps,
                             const rsot_options *opt, int *status_out, double *grad_l1_out,
                             rsot_batch_stats *stats) {
    if (!b || !psi_all || !eps || !opt || !(opt->tol_l1 > 0.0)) return RSOT_ERR_ARG;
    const auto t0 = std::chrono::steady_clock::now();
    const int P = b->count;
    const int m = opt->lbfgs_m > 0 ? opt->lbfgs_m : 10;
    const int max_iter = opt->max_iter > 0 ? opt->max_iter : 10000;
    // intermediate eps stages only warm-start the next one: 100 tol_l1 unless given
    const double stage_tol = opt->stage_tol_l1 > 0.0 ? opt->stage_tol_l1 : rsot::kStageTolFactor * opt->tol_l1;
    // with FP64 refinement the batched mixed phase stops above the FP32 floor
    const double final_tol = (opt->precision == RSOT_MIXED && opt->refine_fp64)
                                 ? std::max(opt->tol_l1, opt->mixed_tol_l1 > 0.0 ? opt->mixed_tol_l1 : 1e-5)
                                 : opt->tol_l1;
    std::vector<int> st(P, RSOT_OK);
    std::vector<double> gl1(P, 0.0);
    int rounds = 0;
    int64_t evals = 0;
    int64_t evals_prec[3] = {0, 0, 0}, pairs_prec[3] = {0, 0, 0};
    double t_mixed = 0.0, t_ref = 0.0;
    // per-problem eps stages
    std::vector<std::vector<double>> stages(P);
    for (int p = 0; p < P; ++p) {
        if (opt->eps_start > eps[p] && opt->eps_factor > 0.0 && opt->eps_factor < 1.0)
            for (double e = opt->eps_start; e > eps[p] * (1.0 + 1e-12); e *= opt->eps_factor)
                stages[p].push_back(e);
        stages[p].push_back(eps[p]);
    }
    auto Dvec = [&](int p, double e) {
        const BProb &Q = b->hp[p];
        std::vector<double> D(Q.n);
        for (int64_t j = 0; j < Q.n; ++j) D[j] = e / b->hnu[Q.psi_off + j];
        return D;
    };
    auto xvec = [&](int p) {
        const BProb &Q = b->hp[p];
        return std::vector<double>(psi_all + Q.psi_off, psi_all + Q.psi_off + Q.n);
    };
    if (opt->precision == RSOT_MIXED) {
        std::vector<LbfgsMachine> mc(P);
        std::vector<int> si(P, 0);
        // latest gradient norm per problem: a round takes the tensor-core pair
        // kernels only while every active problem is far above their noise
        std::vector<double> last_l1(P, INFINITY);
        for (int p = 0; p < P; ++p) {
            const double e = stages[p][0];
            mc[p].start(xvec(p), stages[p].size() == 1 ? final_tol : stage_tol, m, max_iter,
                        Dvec(p, e), 1e-6);
            mc[p].set_stall_window(kMixedStallWindow);
            b->eps_h[p] = e;
        }
        for (;;) {
            bool any = false;
            for (int p = 0; p < P; ++p) {
                b->active_h[p] = mc[p].wants_eval() ? 1 : 0;
                if (b->active_h[p]) {
                    any = true;
                    const BProb &Q = b->hp[p];
                    memcpy(b->psi_h + Q.psi_off, mc[p].trial().data(), Q.n * 8);
                    b->eps_h[p] = stages[p][si[p]];
                }
            }
            if (!any) break;
            bool fp32 = false;
            for (int p = 0; p < P; ++p)
                if (b->active_h[p] && last_l1[p] < kTcNoiseFactor * b->tc_noise[p]) fp32 = true;
            rsot_status s = run_round(b, fp32);
            if (s) return s;
            ++rounds;
            for (int p = 0; p < P; ++p) {
                if (!b->active_h[p]) continue;
                const BProb &Q = b->hp[p];
                std::vector<double> g(b->grad_h + Q.psi_off, b->grad_h + Q.psi_off + Q.n);
                mc[p].feed(b->J_h[p], g);
                last_l1[p] = mc[p].grad_l1();
                ++evals;
                ++evals_prec[RSOT_MIXED];
                pairs_prec[RSOT_MIXED] += Q.nq * Q.n;
                if (mc[p].done()) {
                    const bool last = si[p] + 1 == (int)stages[p].size();
                    if (!last && (mc[p].status() == RSOT_OK || mc[p].status() == RSOT_ERR_LINESEARCH)) {
                        ++si[p];
                        const double e = stages[p][si[p]];
                        const bool fin = si[p] + 1 == (int)stages[p].size();
                        mc[p].start(mc[p].x(), fin ? final_tol : stage_tol, m, max_iter,
                                    Dvec(p, e), 1e-6);
                        mc[p].set_stall_window(kMixedStallWindow);
                    } else {
                        st[p] = mc[p].status();
                        gl1[p] = mc[p].grad_l1();
                        std::copy(mc[p].x().begin(), mc[p].x().end(), psi_all + Q.psi_off);
                    }
                }
            }
        }
        t_mixed = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (opt->refine_fp64) {
            // refinement (rsot_solve) of each problem through its own handle, from the
            // mixed solution: host threads take the problems largest first, each on
            // its own stream, so that the GPU runs several small problems at once
            std::vector<int> order;
            for (int p = 0; p < P; ++p)
                if (st[p] == RSOT_OK || st[p] == RSOT_ERR_LINESEARCH || st[p] == RSOT_ERR_NOT_CONVERGED)
                    order.push_back(p);
            std::sort(order.begin(), order.end(), [&](int a, int c) {
                return b->hp[a].nq * b->hp[a].n > b->hp[c].nq * b->hp[c].n;
            });
            const int nw = std::max(1, std::min<int>(kRefineThreads, (int)order.size()));
            std::vector<cudaStream_t> streams(nw, nullptr);
            for (int w = 0; w < nw; ++w)
                if (cudaStreamCreateWithFlags(&streams[w], cudaStreamNonBlocking) != cudaSuccess)
                    streams[w] = nullptr;
            std::atomic<int> next{0};
            std::vector<int64_t> wevals(nw, 0), wprec((size_t)nw * 6, 0);
            auto worker = [&](int w) {
                for (int i = next++; i < (int)order.size(); i = next++) {
                    const int p = order[i];
                    rsot_set_stream(b->handles[p], streams[w]);
                    rsot_options o = *opt;
                    o.eps = eps[p];
                    o.eps_start = 0.0;   // refinement of the batched result at the final eps
                    rsot_solve_stats ss;
                    const BProb &Q = b->hp[p];
                    st[p] = rsot_solve(b->handles[p], psi_all + Q.psi_off, &o, &ss);
                    gl1[p] = ss.grad_l1;
                    wevals[w] += ss.evals;
                    for (int k = 0; k < 3; ++k) {
                        wprec[(size_t)w * 6 + k] += ss.evals_prec[k];
                        wprec[(size_t)w * 6 + 3 + k] += ss.pairs_prec[k];
                    }
                    rsot_set_stream(b->handles[p], nullptr);
                }
            };
            std::vector<std::thread> pool;
            for (int w = 1; w < nw; ++w) pool.emplace_back(worker, w);
            worker(0);
            for (auto &th : pool) th.join();
            for (int w = 0; w < nw; ++w) {
                evals += wevals[w];
                for (int k = 0; k < 3; ++k) {
                    evals_prec[k] += wprec[(size_t)w * 6 + k];
                    pairs_prec[k] += wprec[(size_t)w * 6 + 3 + k];
                }
                if (streams[w]) cudaStreamDestroy(streams[w]);
            }
            t_ref = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() - t_mixed;
        }
    } else {
        // plain FP64: each problem in turn, no batching
        for (int p = 0; p < P; ++p) {
            rsot_options o = *opt;
            o.eps = eps[p];
            o.precision = RSOT_FP64;
            rsot_solve_stats ss;
            const BProb &Q = b->hp[p];
            st[p] = rsot_solve(b->handles[p], psi_all + Q.psi_off, &o, &ss);
            gl1[p] = ss.grad_l1;
            evals += ss.evals;
            for (int k = 0; k < 3; ++k) {
                evals_prec[k] += ss.evals_prec[k];
                pairs_prec[k] += ss.pairs_prec[k];
            }
        }
    }
    int conv = 0;
    double mx = 0.0;
    rsot_status worst = RSOT_OK;
    for (int p = 0; p < P; ++p) {
        if (status_out) status_out[p] = st[p];
        if (grad_l1_out) grad_l1_out[p] = gl1[p];
        if (st[p] == RSOT_OK) ++conv;
        else if (worst == RSOT_OK) worst = (rsot_status)st[p];
        mx = std::max(mx, gl1[p]);
    }
    if (stats) {
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        stats->seconds_mixed = t_mixed;
        stats->seconds_refine = t_ref;
        stats->rounds = rounds;
        stats->converged = conv;
        stats->max_grad_l1 = mx;
        stats->evals = evals;
        for (int k = 0; k < 3; ++k) {
            stats->evals_prec[k] = evals_prec[k];
            stats->pairs_prec[k] = pairs_prec[k];
        }
    }
    return worst;
}

}  // extern "C"
