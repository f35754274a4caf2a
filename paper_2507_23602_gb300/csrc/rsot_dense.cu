// Dense dual + gradient evaluation (Algorithm 2 with I_q = all targets).
//
// Mixed precision (FP32 pair arithmetic, FP64 reductions), log2 domain.
// With translated coordinates x' = x - o, y' = y - o, a centre psi_c = psi_0,
// k = log2(e) / (2 eps):
//     b_j = ((psi_j - psi_c)/eps + ln nu_j) log2 e
//     w_j = 2 k y'_j,  c_j = b_j - k |y'_j|^2           (per target, FP32)
//     r_qj = c_j + x'_q . w_j                           (d FFMA per pair)
//     log2( nu_j e^{(psi_j - c(x_q,y_j))/eps} ) = log2e psi_c/eps + r_qj - k |x'_q|^2
// so with R_q = log2 sum_j 2^{r_qj} (pass 1):
//     eps L_q = psi_c + eps ln2 R_q - |x'_q|^2 / 2
//     J = psi_c sum m - sum_q m_q |x'_q|^2/2 + eps ln2 sum_q m_q R_q - sum_j psi_j nu_j
//     m_q p_qj = 2^{ r_qj + log2 m_q - R_q }            (pass 2)
// which are Eq. discretized_functional and Eq. discretized_gradient.
//
// Pass 1 (K-LSE) is point-parallel: each thread holds 8 points as 4 float2
// pairs, target tiles are staged into shared memory by bulk async copies
// (cp.async.bulk + mbarrier, double buffered), and the running max / sum is
// kept per point with an integral shift M (lazy rescale when a sub-tile's
// max exceeds M + 32), ex2.approx.ftz per pair, FP64 flush per stage.
// Pass 2 (K-GRAD) is target-parallel: each thread holds 2*TPP targets as
// float2 pairs in registers, point records are staged into shared memory the
// same way, and each target accumulates sum_q m_q p_qj with no shuffles and
// no atomics; split partials over point chunks are summed in FP64 by a
// final kernel in a fixed order (deterministic).
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

#include <cuda.h>

#include "rsot_internal.cuh"
#include "rsot_inner.cuh"
#include "rsot_tc.cuh"
#include "rsot_exp64.cuh"

namespace rsot {
namespace {

constexpr int CB_THREADS = 256;                        // combine / prep kernels

constexpr int F_THREADS = 128;                         // FP64 kernels
constexpr int F_TS = 128;

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// ----------------------------------------------------------------------------
// Per-target records (step a1): dup records for pass 1, pair records for
// pass 2, and the block partials of sum_j psi_j nu_j.
// ----------------------------------------------------------------------------
__global__ void k_prep_mixed(const double *__restrict__ psi, const double *__restrict__ y64,
                             const double *__restrict__ lnu, const double *__restrict__ nu,
                             int64_t n, int64_t n_alloc, int d, double eps,
                             Rec8 *__restrict__ tdup, Rec8 *__restrict__ tpair,
                             double *__restrict__ psinu_part, int *__restrict__ flags,
                             Rec16 *__restrict__ trec, double inv_P, int *__restrict__ gate) {
    __shared__ double sh[32];
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double psic = psi[0];
    const double k = kLog2e / (2.0 * eps);
    double contrib = 0.0;
    if (j < n_alloc) {
        float w[3] = {0.f, 0.f, 0.f};
        float c = kPadC;
        float W[3] = {0.f, 0.f, 0.f};   // tensor-core operands: w / P and c
        float C = -256.0f * TC_RANGE;
        if (j < n) {
            const double ps = psi[j];
            if (!isfinite(ps)) atomicOr(flags, kErrNonfinitePsi);
            const double b = ((ps - psic) / eps + lnu[j]) * kLog2e;
            double yy = 0.0;
            bool ok = true;
            for (int t = 0; t < d; ++t) {
                const double yt = y64[j * d + t];
                w[t] = (float)(2.0 * k * yt);
                W[t] = (float)(2.0 * k * yt * inv_P);
                ok = ok && fabsf(W[t]) < TC_RANGE;
                yy += yt * yt;
            }
            const double cc = b - k * yy;
            c = (float)cc;
            // c below -256 TC_RANGE only makes the exponent more negative than
            // -1.5e7 + |X||W| < -1.3e7: clamping it leaves ex2 = 0 unchanged
            C = (float)fmax(cc, -256.0 * TC_RANGE);
            ok = ok && C < 256.0f * TC_RANGE;
            if (!ok && gate) atomicOr(gate, 1);
            contrib = ps * nu[j];
        }
        if (trec) trec[j] = make_target_rec(W, C);
        Rec8 r;
        r.a = make_float4(w[0], w[0], w[1], w[1]);
        r.b = make_float4(w[2], w[2], c, c);
        tdup[j] = r;
        float *pr = reinterpret_cast<float *>(tpair + (j >> 1));
        const int l = (int)(j & 1);
        pr[0 + l] = w[0];
        pr[2 + l] = w[1];
        pr[4 + l] = w[2];
        pr[6 + l] = c;
    }
    const double s = block_sum_d(contrib, sh);
    if (threadIdx.x == 0) psinu_part[blockIdx.x] = s;
}

// ----------------------------------------------------------------------------
// Pass 1: per-point log-sum-exp over one target chunk (step a2).
// ----------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(P1_THREADS, P1_MINB)
    k_lse_mixed(const float *__restrict__ xs, int64_t nq_pad, const Rec8 *__restrict__ tdup,
                int n_p1, int chunk, float2 *__restrict__ part, int *__restrict__ flags,
                const int *__restrict__ gate = nullptr, int need = 0) {
    // as the fallback of the tensor-core pass, run only when the gate asks for it
    if (gate && !(*gate & need)) return;
    __shared__ __align__(128) Rec8 sm[P1_STAGES][P1_TS];
    __shared__ __align__(8) uint64_t full[P1_STAGES];
    __shared__ int s_abort[2];   // indexed by iteration parity

    const int tid = threadIdx.x;
    const int64_t q0 = (int64_t)blockIdx.x * P1_TILE;
    const int kc = blockIdx.y;
    const int t_begin = kc * chunk;
    const int t_count = min(chunk, n_p1 - t_begin);
    const int ntile = t_count / P1_TS;

    float2 X[P1_PP][3];
#pragma unroll
    for (int pp = 0; pp < P1_PP; ++pp) {
        const int64_t q = q0 + 2 * (pp * P1_THREADS + tid);
#pragma unroll
        for (int k = 0; k < 3; ++k)
            X[pp][k] = (k < D) ? *reinterpret_cast<const float2 *>(xs + k * nq_pad + q)
                               : make_float2(0.f, 0.f);
    }
    float2 M[P1_PP], Sf[P1_PP];
    double2 Sd[P1_PP];
#pragma unroll
    for (int pp = 0; pp < P1_PP; ++pp) {
        M[pp] = make_float2(kPadC, kPadC);
        Sf[pp] = make_float2(0.f, 0.f);
        Sd[pp] = make_double2(0.0, 0.0);
    }

    if (tid == 0) {
        s_abort[0] = s_abort[1] = 0;
        for (int s = 0; s < P1_STAGES; ++s) mbar_init(&full[s], 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int s = 0; s < P1_STAGES && s < ntile; ++s) {
            mbar_expect_tx(&full[s], P1_TS * sizeof(Rec8));
            bulk_g2s(sm[s], tdup + t_begin + s * P1_TS, P1_TS * sizeof(Rec8), &full[s]);
        }
    }

    int issued = min(P1_STAGES, ntile);
    bool aborted = false;
    for (int it = 0; it < ntile; ++it) {
        const int s = it % P1_STAGES;
        const unsigned ph = (unsigned)(it / P1_STAGES) & 1u;
        const bool ok = mbar_wait(&full[s], ph);
        if (!ok) {
            s_abort[it & 1] = 1;
            atomicOr(flags, kErrTimeout);
        } else {
            lse_stage<D, P1_PP>(sm[s], X, M, Sf, Sd);
        }
        __syncthreads();
        aborted = s_abort[it & 1] != 0;
        if (aborted) break;
        if (tid == 0 && it + P1_STAGES < ntile) {
            mbar_expect_tx(&full[s], P1_TS * sizeof(Rec8));
            bulk_g2s(sm[s], tdup + t_begin + (it + P1_STAGES) * P1_TS, P1_TS * sizeof(Rec8),
                     &full[s]);
            ++issued;
        }
#pragma unroll
        for (int pp = 0; pp < P1_PP; ++pp) {
            Sd[pp].x += (double)Sf[pp].x;
            Sd[pp].y += (double)Sf[pp].y;
            Sf[pp] = make_float2(0.f, 0.f);
        }
    }
    if (aborted) {
        // drain copies still in flight (bounded) before the CTA exits
        if (tid == 0) {
            for (int it = 0; it < issued; ++it) {
                const int s = it % P1_STAGES;
                (void)mbar_wait(&full[s], (unsigned)(it / P1_STAGES) & 1u);
            }
        }
        return;
    }
#pragma unroll
    for (int pp = 0; pp < P1_PP; ++pp) {
        const int64_t q = q0 + 2 * (pp * P1_THREADS + tid);
        *reinterpret_cast<float4 *>(part + (int64_t)kc * nq_pad + q) =
            make_float4(M[pp].x, (float)Sd[pp].x, M[pp].y, (float)Sd[pp].y);
    }
}

// ----------------------------------------------------------------------------
// Merge the pass-1 chunk partials into R_q, write the pass-2 point records
// (x', u_q = log2 m_q - R_q) and the block partials of sum_q m_q R_q.
// ----------------------------------------------------------------------------
__global__ void k_combine(const float2 *__restrict__ part, int k1, int64_t nq_pad, int64_t nq,
                          const float *__restrict__ xs, int d, const double *__restrict__ lmass2,
                          const double *__restrict__ mass, Rec8 *__restrict__ pdup,
                          double *__restrict__ blockJ, double *__restrict__ lse_buf,
                          float *__restrict__ pu = nullptr) {
    __shared__ double sh[32];
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double contrib = 0.0;
    if (q < nq_pad) {
        float x[3] = {0.f, 0.f, 0.f};
        float u = kPadC;
        if (q < nq) {
            float mx = kPadC;
            for (int k = 0; k < k1; ++k) mx = fmaxf(mx, part[(int64_t)k * nq_pad + q].x);
            double tot = 0.0;
            for (int k = 0; k < k1; ++k) {
                const float2 v = part[(int64_t)k * nq_pad + q];
                tot += (double)v.y * pow2_int_d(v.x - mx);
            }
            const double R = (double)mx + log2(tot);
            lse_buf[q] = R;
            const double lm = lmass2[q];
            if (mass[q] > 0.0) {
                contrib = mass[q] * R;
                u = (float)fmax(lm - R, -1.0e30);
            }
            for (int t = 0; t < d; ++t) x[t] = xs[t * nq_pad + q];
        }
        Rec8 r;
        r.a = make_float4(x[0], x[0], x[1], x[1]);
        r.b = make_float4(x[2], x[2], u, u);
        pdup[q] = r;
        if (pu) pu[q] = u;   // pass-2 shift of the tensor-core kernel
    }
    const double s = block_sum_d(contrib, sh);
    if (threadIdx.x == 0) blockJ[blockIdx.x] = s;
}

// ----------------------------------------------------------------------------
// Pass 2: per-target sum over one point chunk of m_q p_qj (step a3).
// ----------------------------------------------------------------------------
template <int D, int TPP>
__global__ void __launch_bounds__(P2_THREADS, P2_MINB)
    k_grad_mixed(const Rec8 *__restrict__ tpair, const Rec8 *__restrict__ pdup, int64_t nq_pad,
                 int64_t chunk, double *__restrict__ part2, int64_t stride,
                 int *__restrict__ flags, const int *__restrict__ gate = nullptr, int need = 0) {
    if (gate && !(*gate & need)) return;
    __shared__ __align__(128) Rec8 sm[P2_STAGES][P2_TS];
    __shared__ __align__(8) uint64_t full[P2_STAGES];
    __shared__ int s_abort[2];   // indexed by iteration parity

    const int tid = threadIdx.x;
    const int64_t g0 = (int64_t)blockIdx.x * P2_THREADS * TPP;
    float2 W0[TPP], W1[TPP], W2[TPP], C[TPP];
#pragma unroll
    for (int tp = 0; tp < TPP; ++tp) {
        const Rec8 r = tpair[g0 + tp * P2_THREADS + tid];
        W0[tp] = make_float2(r.a.x, r.a.y);
        W1[tp] = make_float2(r.a.z, r.a.w);
        W2[tp] = make_float2(r.b.x, r.b.y);
        C[tp] = make_float2(r.b.z, r.b.w);
    }
    const int64_t p_begin = (int64_t)blockIdx.y * chunk;
    const int64_t p_count = min(chunk, nq_pad - p_begin);
    const int ntile = (int)(p_count / P2_TS);

    double2 acc64[TPP];
#pragma unroll
    for (int tp = 0; tp < TPP; ++tp) acc64[tp] = make_double2(0.0, 0.0);

    if (tid == 0) {
        s_abort[0] = s_abort[1] = 0;
        for (int s = 0; s < P2_STAGES; ++s) mbar_init(&full[s], 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int s = 0; s < P2_STAGES && s < ntile; ++s) {
            mbar_expect_tx(&full[s], P2_TS * sizeof(Rec8));
            bulk_g2s(sm[s], pdup + p_begin + (int64_t)s * P2_TS, P2_TS * sizeof(Rec8), &full[s]);
        }
    }
    int issued = min(P2_STAGES, ntile);
    bool aborted = false;
    for (int it = 0; it < ntile; ++it) {
        const int s = it % P2_STAGES;
        const unsigned ph = (unsigned)(it / P2_STAGES) & 1u;
        const bool ok = mbar_wait(&full[s], ph);
        if (!ok) {
            s_abort[it & 1] = 1;
            atomicOr(flags, kErrTimeout);
        } else {
            grad_stage<D, TPP>(sm[s], W0, W1, W2, C, acc64);
        }
        __syncthreads();
        aborted = s_abort[it & 1] != 0;
        if (aborted) break;
        if (tid == 0 && it + P2_STAGES < ntile) {
            mbar_expect_tx(&full[s], P2_TS * sizeof(Rec8));
            bulk_g2s(sm[s], pdup + p_begin + (int64_t)(it + P2_STAGES) * P2_TS,
                     P2_TS * sizeof(Rec8), &full[s]);
            ++issued;
        }
    }
    if (aborted) {
        if (tid == 0) {
            for (int it = 0; it < issued; ++it)
                (void)mbar_wait(&full[it % P2_STAGES], (unsigned)(it / P2_STAGES) & 1u);
        }
        return;
    }
#pragma unroll
    for (int tp = 0; tp < TPP; ++tp) {
        const int64_t j = 2 * (g0 + tp * P2_THREADS + tid);
        *reinterpret_cast<double2 *>(part2 + (int64_t)blockIdx.y * stride + j) = acc64[tp];
    }
}


// ----------------------------------------------------------------------------
// Tensor-core passes (rsot_tc.cuh).  Both passes form D = P_q . T_j, the
// exponent r_qj of every pair, with one mma.sync m16n8k16 per 16 points x 8
// targets: rows = points (A fragments of the point records), columns =
// targets (B fragments of the target records), f32 accumulation from zero.
// The two passes issue the same instruction on the same operands, so pass 2
// sees bitwise the exponents of pass 1 and the plan rows it forms sum to 1 as
// in the FP32 kernels; the per-point shift (-M_q in pass 1, u_q in pass 2) is
// one packed FP32 add per two pairs, ex2 reads the result, one packed add
// per two pairs accumulates.
//
// Pass 1 holds 4 m-blocks of 16 points per warp in registers and streams the
// target records (8 per n-block) through shared memory.  Lane (g, t) sums
// rows g and g + 8 over its columns 2t, 2t + 1 with its own integral shifts
// M; groups of 8 n-blocks are summed optimistically and redone exactly
// (maximum over the group, M raised to its ceiling, sums rescaled by a power
// of two) when a lane's group sum exceeds 2^60 or is not finite, or a shift
// is not yet set.  The 4 lanes of a row are merged at the end.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(TC_THREADS, TC_MINB)
    k_lse_tc(const Rec16 *__restrict__ prec, int64_t nq_pad, const Rec16 *__restrict__ trec,
             int n_p1, int chunk, float2 *__restrict__ part, int *__restrict__ flags,
             const int *__restrict__ gate) {
    if (gate && (*gate & 1)) return;   // operands out of f16 range: the FP32 kernel runs
    extern __shared__ __align__(128) unsigned char tc_smem[];
    Rec16 (*sm)[TC_TS] = reinterpret_cast<Rec16 (*)[TC_TS]>(tc_smem);   // [TC_STAGES][TC_TS]
    // full[s]: the stage's bytes landed; empty[s]: every warp is done with it
    __shared__ __align__(8) uint64_t full[TC_STAGES], empty[TC_STAGES];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = lane >> 2, t = lane & 3;
    const int64_t q0 = (int64_t)blockIdx.x * TC_ROWS + warp * (TC_MB * 16);
    const int kc = blockIdx.y;
    const int t_begin = kc * chunk;
    const int t_count = min(chunk, n_p1 - t_begin);
    const int ntile = t_count / TC_TS;

    unsigned A[TC_MB][4];
    float2 M[TC_MB], Sf[TC_MB];
    double2 Sd[TC_MB];
    const uint2 *pr = reinterpret_cast<const uint2 *>(prec);
#pragma unroll
    for (int m = 0; m < TC_MB; ++m) {
        tc_load_a(A[m], pr + (q0 + m * 16) * 4, g, t);
        M[m] = make_float2(-INFINITY, -INFINITY);
        Sf[m] = make_float2(0.f, 0.f);
        Sd[m] = make_double2(0.0, 0.0);
    }

    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], TC_WARPS);
        }
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int s = 0; s < TC_STAGES && s < ntile; ++s) {
            mbar_expect_tx(&full[s], TC_TS * sizeof(Rec16));
            bulk_g2s(sm[s], trec + t_begin + s * TC_TS, TC_TS * sizeof(Rec16), &full[s]);
        }
    }
    int issued = min(TC_STAGES, ntile);
    bool aborted = false;
    constexpr int NGRP = TC_NBS / TC_GROUP;
    // no block barrier in the loop: each warp waits for the data of a stage and
    // releases it; thread 0 refills a stage once all warps have released it
    for (int it = 0; it < ntile; ++it) {
        const int s = it % TC_STAGES;
        const unsigned ph = (unsigned)(it / TC_STAGES) & 1u;
        // warp-uniform decisions: the mma below needs every lane
        if (!__all_sync(0xffffffffu, mbar_wait(&full[s], ph))) {
            atomicOr(flags, kErrTimeout);
            aborted = true;
            break;
        }
        tc_lse_stage<TC_NBS>(reinterpret_cast<const uint2 *>(&sm[s][0]) + lane, A, M, Sf, Sd);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (warp == 0 && it + TC_STAGES < ntile) {
            bool ok = true;
            if (tid == 0) {
                ok = mbar_wait(&empty[s], ph);
                if (ok) {
                    mbar_expect_tx(&full[s], TC_TS * sizeof(Rec16));
                    bulk_g2s(sm[s], trec + t_begin + (it + TC_STAGES) * TC_TS,
                             TC_TS * sizeof(Rec16), &full[s]);
                    ++issued;
                }
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) {
                atomicOr(flags, kErrTimeout);
                aborted = true;
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
    // a warp whose wait expired leaves without writing (the error flag is set);
    // thread 0 drains its copies still in flight (bounded) before the CTA ends
    if (aborted) {
        if (tid == 0)
            for (int it = 0; it < issued; ++it)
                (void)mbar_wait(&full[it % TC_STAGES], (unsigned)(it / TC_STAGES) & 1u);
        return;
    }
    // merge the 4 lanes of each row: common shift = their maximum
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
        M[m] = make_float2(mx, my);
        Sd[m] = make_double2(sx, sy);
    }
#pragma unroll
    for (int m = 0; m < TC_MB; ++m) {
        if (m != t) continue;   // lane t writes m-block t
        const int64_t qa = q0 + m * 16 + g;
        float2 *o = part + (int64_t)kc * nq_pad;
        o[qa] = M[m].x == -INFINITY ? make_float2(kPadC, 0.f) : make_float2(M[m].x, (float)Sd[m].x);
        o[qa + 8] = M[m].y == -INFINITY ? make_float2(kPadC, 0.f) : make_float2(M[m].y, (float)Sd[m].y);
    }
}

// Pass 2: rows = targets (A fragments of the target records, 4 m-blocks of 16
// targets per warp, in registers), columns = points (records and shifts u_q
// streamed through shared memory, 8 per n-block).  The mma is symmetric in
// its operands bit for bit (checked on GB300: swapping the roles of the
// operands changed none of 2^21 results), so D here is bitwise the D of
// pass 1.  Lane (g, t) sums rows g and g + 8 over its columns 2t, 2t + 1,
// FP32 within a stage and FP64 across stages; the 4 lanes of a row are
// added at the end.
__global__ void __launch_bounds__(TC_THREADS, TC_MINB)
    k_grad_tc(const Rec16 *__restrict__ trec, const Rec16 *__restrict__ prec,
              const float *__restrict__ pu, int64_t nq_pad, int64_t chunk,
              double *__restrict__ part2, int64_t stride, int *__restrict__ flags,
              const int *__restrict__ gate) {
    if (gate && (*gate & 1)) return;   // out of f16 range: the FP32 kernel runs
    extern __shared__ __align__(128) unsigned char tc_smem[];
    Rec16 (*sm)[TC_TS] = reinterpret_cast<Rec16 (*)[TC_TS]>(tc_smem);   // [TC_STAGES][TC_TS]
    float (*su)[TC_TS] = reinterpret_cast<float (*)[TC_TS]>(tc_smem + TC_SMEM1);
    __shared__ __align__(8) uint64_t full[TC_STAGES], empty[TC_STAGES];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = lane >> 2, t = lane & 3;
    const int64_t j0 = (int64_t)blockIdx.x * TC_ROWS + warp * (TC_MB * 16);
    const uint2 *tr = reinterpret_cast<const uint2 *>(trec);
    unsigned A[TC_MB][4];
    double2 acc64[TC_MB];
#pragma unroll
    for (int m = 0; m < TC_MB; ++m) {
        tc_load_a(A[m], tr + (j0 + m * 16) * 4, g, t);
        acc64[m] = make_double2(0.0, 0.0);
    }
    const int64_t p_begin = (int64_t)blockIdx.y * chunk;
    const int64_t p_count = min(chunk, nq_pad - p_begin);
    const int ntile = (int)(p_count / TC_TS);
    constexpr unsigned kStageBytes = TC_TS * sizeof(Rec16) + TC_TS * sizeof(float);

    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], TC_WARPS);
        }
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int s = 0; s < TC_STAGES && s < ntile; ++s) {
            mbar_expect_tx(&full[s], kStageBytes);
            bulk_g2s(sm[s], prec + p_begin + (int64_t)s * TC_TS, TC_TS * sizeof(Rec16), &full[s]);
            bulk_g2s(su[s], pu + p_begin + (int64_t)s * TC_TS, TC_TS * sizeof(float), &full[s]);
        }
    }
    int issued = min(TC_STAGES, ntile);
    bool aborted = false;
    for (int it = 0; it < ntile; ++it) {
        const int s = it % TC_STAGES;
        const unsigned ph = (unsigned)(it / TC_STAGES) & 1u;
        if (!__all_sync(0xffffffffu, mbar_wait(&full[s], ph))) {
            atomicOr(flags, kErrTimeout);
            aborted = true;
            break;
        }
        tc_grad_stage<TC_NBS>(reinterpret_cast<const uint2 *>(&sm[s][0]) + lane,
                              reinterpret_cast<const float2 *>(&su[s][0]) + t, A, acc64);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (warp == 0 && it + TC_STAGES < ntile) {
            bool ok = true;
            if (tid == 0) {
                ok = mbar_wait(&empty[s], ph);
                if (ok) {
                    mbar_expect_tx(&full[s], kStageBytes);
                    bulk_g2s(sm[s], prec + p_begin + (int64_t)(it + TC_STAGES) * TC_TS,
                             TC_TS * sizeof(Rec16), &full[s]);
                    bulk_g2s(su[s], pu + p_begin + (int64_t)(it + TC_STAGES) * TC_TS,
                             TC_TS * sizeof(float), &full[s]);
                    ++issued;
                }
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) {
                atomicOr(flags, kErrTimeout);
                aborted = true;
                break;
            }
        }
    }
    if (aborted) {
        if (tid == 0)
            for (int it = 0; it < issued; ++it)
                (void)mbar_wait(&full[it % TC_STAGES], (unsigned)(it / TC_STAGES) & 1u);
        return;
    }
#pragma unroll
    for (int m = 0; m < TC_MB; ++m) {
        acc64[m].x += __shfl_xor_sync(0xffffffffu, acc64[m].x, 1);
        acc64[m].x += __shfl_xor_sync(0xffffffffu, acc64[m].x, 2);
        acc64[m].y += __shfl_xor_sync(0xffffffffu, acc64[m].y, 1);
        acc64[m].y += __shfl_xor_sync(0xffffffffu, acc64[m].y, 2);
    }
#pragma unroll
    for (int m = 0; m < TC_MB; ++m) {
        if (m != t) continue;   // lane t writes m-block t
        double *o = part2 + (int64_t)blockIdx.y * stride + j0 + m * 16 + g;
        o[0] = acc64[m].x;
        o[8] = acc64[m].y;
    }
}

// Point operand records (X = P x', no shift slots), once per problem.
__global__ void k_point_recs(const float *__restrict__ xs, int64_t nq_pad, int d, float P,
                             Rec16 *__restrict__ prec) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq_pad) return;
    float X[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) X[k] = k < d ? xs[k * nq_pad + q] * P : 0.0f;
    prec[q] = make_point_rec(X, 0.0f);
}

// grad_j = sum_s part2[s][j] - nu_j  (fixed order: deterministic)
__global__ void k_finalize_grad(const double *__restrict__ part2, int s2, int64_t stride,
                                const double *__restrict__ nu, int64_t n,
                                double *__restrict__ grad) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double g = 0.0;
    for (int s = 0; s < s2; ++s) g += part2[(int64_t)s * stride + j];
    grad[j] = g - nu[j];
}

// J from the block partials (one block).
__global__ void k_finalize_J(const double *__restrict__ blockJ, int nbj,
                             const double *__restrict__ psinu, int npn,
                             const double *__restrict__ psi, double eps, double msum, double hx,
                             int mixed, EvalResult *__restrict__ res) {
    __shared__ double sh[32];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nbj; i += blockDim.x) a += blockJ[i];
    for (int i = threadIdx.x; i < npn; i += blockDim.x) b += psinu[i];
    const double sa = block_sum_d(a, sh);
    const double sb = block_sum_d(b, sh);
    if (threadIdx.x == 0) {
        const double psic = psi[0];
        res->psic = psic;
        // mixed: sa = sum_q m_q R_q (log2, translated frame); FP64: sa = sum_q m_q eps L_q
        res->J = mixed ? (psic * msum - hx + eps * kLn2 * sa - sb) : (sa - sb);
    }
}

// ----------------------------------------------------------------------------
// FP64 path: same passes with FP64 arithmetic and CUDA's exp/log.
// ----------------------------------------------------------------------------
__global__ void k_prep_fp64(const double *__restrict__ psi, const double *__restrict__ lnu,
                            const double *__restrict__ nu, int64_t n, int64_t n_alloc, double eps,
                            double *__restrict__ a64, double *__restrict__ psinu_part,
                            int *__restrict__ flags) {
    __shared__ double sh[32];
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double contrib = 0.0;
    if (j < n_alloc) {
        double a = -INFINITY;
        if (j < n) {
            const double ps = psi[j];
            if (!isfinite(ps)) atomicOr(flags, kErrNonfinitePsi);
            a = (ps - psi[0]) / eps + lnu[j];
            contrib = ps * nu[j];
        }
        a64[j] = a;
    }
    const double s = block_sum_d(contrib, sh);
    if (threadIdx.x == 0) psinu_part[blockIdx.x] = s;
}

// TRUNC = false: dense; true: only pairs with c(x_q, y_j) < alpha_q + beta_j
// enter (Algorithm 2 with a cutoff per pair, rsot_cutoff.cu), and the number
// of such pairs and of empty points is counted.  The squared distance d2 =
// |x - y|^2 = 2 c enters as s = a_j - d2 / (2 eps); the cutoff test compares
// d2 < 2 alpha_q + 2 beta_j (the same decision as c < alpha_q + beta_j:
// doubling is exact).
template <int D, bool TRUNC>
__global__ void __launch_bounds__(F_THREADS)
    k_lse_fp64(const double *__restrict__ x64, int64_t nq, int64_t nq_pad,
               const double *__restrict__ y64, const double *__restrict__ a64, int64_t n,
               double half_inv_eps, const double *__restrict__ alpha, const double *__restrict__ beta,
               const double *__restrict__ psi, double eps,
               const double *__restrict__ mass, double *__restrict__ prec64,
               double *__restrict__ blockJ, double *__restrict__ lse_buf,
               EvalResult *__restrict__ res) {
    __shared__ double sy[F_TS][5];
    __shared__ double sh[32];
    __shared__ double2 s_tab[64];
    __shared__ unsigned long long s_cnt, s_empty;
    if (threadIdx.x == 0) s_cnt = s_empty = 0;
    load_exp2_tab(s_tab);
    const int64_t q = (int64_t)blockIdx.x * F_THREADS + threadIdx.x;
    double x[3] = {0.0, 0.0, 0.0};
    if (q < nq)
        for (int t = 0; t < D; ++t) x[t] = x64[q * D + t];
    const double aq2 = TRUNC && q < nq ? 2.0 * alpha[q] : INFINITY;
    double M = -INFINITY, S = 0.0;
    unsigned long long npair = 0;
    __syncthreads();
    for (int64_t t0 = 0; t0 < n; t0 += F_TS) {
        for (int i = threadIdx.x; i < F_TS; i += F_THREADS) {
            const int64_t j = t0 + i;
            if (j < n) {
                for (int t = 0; t < D; ++t) sy[i][t] = y64[j * D + t];
                sy[i][3] = a64[j];
                sy[i][4] = TRUNC ? 2.0 * beta[j] : 0.0;
            } else {
                sy[i][3] = -INFINITY;
                sy[i][4] = 0.0;
            }
        }
        __syncthreads();
        const int cnt = (int)min((int64_t)F_TS, n - t0);
        for (int i = 0; i < cnt; ++i) {
            double d2 = 0.0;
#pragma unroll
            for (int t = 0; t < D; ++t) {
                const double dd = x[t] - sy[i][t];
                d2 = fma(dd, dd, d2);
            }
            if (TRUNC) {
                if (!(d2 < aq2 + sy[i][4])) continue;
                ++npair;
            }
            const double s = fma(-d2, half_inv_eps, sy[i][3]);
            const double dlt = s - M;
            const double e = exp_tab(-fabs(dlt), s_tab);
            if (dlt > 0.0) {
                S = fma(S, e, 1.0);
                M = s;
            } else {
                S += e;
            }
        }
        __syncthreads();
    }
    double contrib = 0.0;
    if (q < nq_pad) {
        double u = -INFINITY;
        if (q < nq) {
            if (S > 0.0) {
                const double L = M + log(S);
                lse_buf[q] = L;
                if (mass[q] > 0.0) {
                    contrib = mass[q] * (psi[0] + eps * L);   // m_q eps L_q
                    u = log(mass[q]) - L;
                }
            } else {   // empty I_q: skipped by Algorithm 2
                lse_buf[q] = -INFINITY;
                atomicAdd(&s_empty, 1ull);
            }
            if (TRUNC) atomicAdd(&s_cnt, npair);
        }
        double *r = prec64 + q * 4;
        r[0] = x[0];
        r[1] = x[1];
        r[2] = x[2];
        r[3] = u;
    }
    const double s = block_sum_d(contrib, sh);
    if (threadIdx.x == 0) {
        blockJ[blockIdx.x] = s;
        if (s_cnt) atomicAdd(reinterpret_cast<unsigned long long *>(&res->pairs), s_cnt);
        if (s_empty) atomicAdd(reinterpret_cast<unsigned long long *>(&res->empty), s_empty);
    }
}

template <int D, bool TRUNC>
__global__ void __launch_bounds__(F_THREADS)
    k_grad_fp64(const double *__restrict__ y64, const double *__restrict__ a64, int64_t n,
                const double *__restrict__ prec64, int64_t nq_pad, int64_t chunk,
                double half_inv_eps, const double *__restrict__ alpha,
                const double *__restrict__ beta, double *__restrict__ part2, int64_t stride) {
    __shared__ double sp[F_TS][4];
    __shared__ double sa[F_TS];
    __shared__ double2 s_tab[64];
    load_exp2_tab(s_tab);
    const int64_t j = (int64_t)blockIdx.x * F_THREADS + threadIdx.x;
    double y[3] = {0.0, 0.0, 0.0};
    double a = -INFINITY, bj2 = 0.0;
    if (j < n) {
        for (int t = 0; t < D; ++t) y[t] = y64[j * D + t];
        a = a64[j];
        if (TRUNC) bj2 = 2.0 * beta[j];
    }
    const int64_t p_begin = (int64_t)blockIdx.y * chunk;
    const int64_t p_end = min(nq_pad, p_begin + chunk);
    double acc = 0.0;
    for (int64_t p0 = p_begin; p0 < p_end; p0 += F_TS) {
        for (int i = threadIdx.x; i < F_TS * 4; i += F_THREADS) {
            const int64_t idx = p0 * 4 + i;
            (&sp[0][0])[i] = (idx < p_end * 4) ? prec64[idx] : (((i & 3) == 3) ? -INFINITY : 0.0);
        }
        if (TRUNC)
            for (int i = threadIdx.x; i < F_TS; i += F_THREADS)
                sa[i] = p0 + i < p_end ? 2.0 * alpha[p0 + i] : -INFINITY;
        __syncthreads();
        const int cnt = (int)min((int64_t)F_TS, p_end - p0);
        for (int i = 0; i < cnt; ++i) {
            double d2 = 0.0;
#pragma unroll
            for (int t = 0; t < D; ++t) {
                const double dd = sp[i][t] - y[t];   // x - y, as in pass 1
                d2 = fma(dd, dd, d2);
            }
            if (TRUNC && !(d2 < sa[i] + bj2)) continue;
            acc += exp_tab(fma(-d2, half_inv_eps, a) + sp[i][3], s_tab);
        }
        __syncthreads();
    }
    if (j < stride) part2[(int64_t)blockIdx.y * stride + j] = acc;
}

// ----------------------------------------------------------------------------
// Covering cost: max_q min_j |x_q - y_j|^2 / 2 (FP32 distances, brute force).
// ----------------------------------------------------------------------------
__global__ void k_cover(const float *__restrict__ xs, int64_t nq, int64_t nq_pad,
                        const double *__restrict__ y64, int64_t n, int d,
                        float *__restrict__ block_max) {
    __shared__ float sy[256][3];
    __shared__ float smax[32];
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float x[3] = {0.f, 0.f, 0.f};
    if (q < nq)
        for (int t = 0; t < d; ++t) x[t] = xs[t * nq_pad + q];
    float best = INFINITY;
    for (int64_t t0 = 0; t0 < n; t0 += 256) {
        const int64_t j = t0 + threadIdx.x;
        for (int t = 0; t < 3; ++t) sy[threadIdx.x][t] = (j < n && t < d) ? (float)y64[j * d + t] : 0.f;
        __syncthreads();
        const int cnt = (int)min((int64_t)256, n - t0);
        for (int i = 0; i < cnt; ++i) {
            const float a = x[0] - sy[i][0], b = x[1] - sy[i][1], c = x[2] - sy[i][2];
            best = fminf(best, fmaf(a, a, fmaf(b, b, c * c)));
        }
        __syncthreads();
    }
    float v = (q < nq) ? best : 0.f;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, smax[w]);
        block_max[blockIdx.x] = m;
    }
}

__global__ void k_max_f(const float *__restrict__ v, int nb, double *__restrict__ out) {
    __shared__ float s[256];
    float m = 0.f;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) m = fmaxf(m, v[i]);
    s[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s[threadIdx.x] = fmaxf(s[threadIdx.x], s[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = 0.5 * (double)s[0];
}

// L_q from the stored per-point quantity of the last dense evaluation.
//   mixed : L_q = psi_c/eps + ln2 R_q - |x'_q|^2 / (2 eps)
//   FP64  : L_q = psi_c/eps + L'_q
__global__ void k_point_L(const double *__restrict__ lse_buf, const double *__restrict__ x64,
                          int64_t nq, int d, int kind, double eps,
                          const EvalResult *__restrict__ res, double *__restrict__ out) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const double base = res->psic / eps;
    if (kind == 1 || kind >= 4) {   // log2-domain R_q (mixed and compensated)
        double r2 = 0.0;
        for (int t = 0; t < d; ++t) r2 += x64[q * d + t] * x64[q * d + t];
        out[q] = base + kLn2 * lse_buf[q] - 0.5 * r2 / eps;
    } else {
        out[q] = base + lse_buf[q];
    }
}

// max psi, min psi (one block)
__global__ void k_psi_stats(const double *__restrict__ psi, int64_t n, double *__restrict__ out) {
    __shared__ double smx[256], smn[256];
    double mx = -INFINITY, mn = INFINITY;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        mx = fmax(mx, psi[i]);
        mn = fmin(mn, psi[i]);
    }
    smx[threadIdx.x] = mx;
    smn[threadIdx.x] = mn;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            smx[threadIdx.x] = fmax(smx[threadIdx.x], smx[threadIdx.x + o]);
            smn[threadIdx.x] = fmin(smn[threadIdx.x], smn[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = smx[0];
        out[1] = smn[0];
    }
}

// Split count s in [1, max_split] such that units * s work items fill the
// resident slots evenly (<= 5% idle in the last wave), smallest such s.
int pick_split(int64_t units, int64_t max_split, int64_t slots) {
    if (max_split < 1) max_split = 1;
    int best = 1;
    double best_eff = 0.0;
    for (int64_t s = 1; s <= max_split && s <= 256; ++s) {
        const int64_t items = units * s;
        const int64_t waves = (items + slots - 1) / slots;
        const double eff = (double)items / (double)(waves * slots);
        if (eff > best_eff + 0.01) {
            best_eff = eff;
            best = (int)s;
        }
        if (items >= slots && eff >= 0.95) return (int)s;
    }
    return best;
}

int occupancy(const void *fn, int threads, size_t dyn_smem) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, dyn_smem) != cudaSuccess ||
        nb < 1)
        nb = 1;
    return nb;
}

int pick_tpp(int64_t n) {
    // targets per pass-2 CTA = 128 * 2 * TPP; pick the largest TPP that wastes
    // at most 1/8 of the lanes on padding
    for (int tpp : {P2_TPP_MAX, 2}) {
        const int64_t blk = (int64_t)P2_THREADS * 2 * tpp;
        if (round_up(n, blk) - n <= n / 8) return tpp;
    }
    return 1;
}

}  // namespace

// ----------------------------------------------------------------------------
// allocation of the dense scratch
// ----------------------------------------------------------------------------
cudaError_t dense_alloc(rsot_problem *p) {
    cudaError_t e;
    const int64_t n_alloc = round_up(p->n, 1024);
    p->n_pad = n_alloc;
    const int64_t n_p1 = round_up(p->n, P1_TS);
    // pass-1 split over target chunks
    const int64_t tiles1 = p->nq_pad / P1_TILE;
    const void *f1 = (p->d == 3) ? (const void *)k_lse_mixed<3> : (const void *)k_lse_mixed<2>;
    const int64_t slots1 = (int64_t)p->num_sms * occupancy(f1, P1_THREADS, 0);
    p->k1 = pick_split(tiles1, n_p1 / P1_TS, slots1);
    p->chunk1 = (int)round_up((n_p1 + p->k1 - 1) / p->k1, P1_TS);
    p->k1 = (int)((n_p1 + p->chunk1 - 1) / p->chunk1);
    // pass-2 split over point chunks
    const int tpp = pick_tpp(p->n);
    const int64_t blk2 = (int64_t)P2_THREADS * 2 * tpp;
    const int64_t units2 = (p->n + blk2 - 1) / blk2;
    const void *f2 = (p->d == 3) ? (const void *)k_grad_mixed<3, 4> : (const void *)k_grad_mixed<2, 4>;
    const int64_t slots2 = (int64_t)p->num_sms * occupancy(f2, P2_THREADS, 0);
    p->s2 = pick_split(units2, p->nq_pad / P2_TS, slots2);
    p->chunk2 = round_up((p->nq_pad + p->s2 - 1) / p->s2, P2_TS);
    p->s2 = (int)((p->nq_pad + p->chunk2 - 1) / p->chunk2);
    // the same splits for the tensor-core passes (TC_ROWS points / targets per CTA);
    // their FP32 fallback (by the gate) runs with these chunks too
    const int64_t n_tc = round_up(p->n, TC_TS);
    if ((e = cudaFuncSetAttribute((const void *)k_lse_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)TC_SMEM1)))
        return e;
    if ((e = cudaFuncSetAttribute((const void *)k_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)TC_SMEM2)))
        return e;
    const int64_t slots_tc1 = (int64_t)p->num_sms * occupancy((const void *)k_lse_tc, TC_THREADS, TC_SMEM1);
    p->k1_tc = pick_split(p->nq_pad / TC_ROWS, n_tc / TC_TS, slots_tc1);
    p->chunk1_tc = (int)round_up((n_tc + p->k1_tc - 1) / p->k1_tc, TC_TS);
    p->k1_tc = (int)((n_tc + p->chunk1_tc - 1) / p->chunk1_tc);
    const int64_t slots_tc2 = (int64_t)p->num_sms * occupancy((const void *)k_grad_tc, TC_THREADS, TC_SMEM2);
    p->s2_tc = pick_split(n_alloc / TC_ROWS, p->nq_pad / TC_TS, slots_tc2);
    p->chunk2_tc = round_up((p->nq_pad + p->s2_tc - 1) / p->s2_tc, TC_TS);
    p->s2_tc = (int)((p->nq_pad + p->chunk2_tc - 1) / p->chunk2_tc);
    // FP64 split
    const int64_t units64 = (p->n + F_THREADS - 1) / F_THREADS;
    p->s2_64 = pick_split(units64, p->nq_pad / F_TS, (int64_t)p->num_sms * 8);
    p->chunk2_64 = round_up((p->nq_pad + p->s2_64 - 1) / p->s2_64, F_TS);
    p->s2_64 = (int)((p->nq_pad + p->chunk2_64 - 1) / p->chunk2_64);

    p->nblk_comb = (int)((p->nq_pad + CB_THREADS - 1) / CB_THREADS);
    p->nblk_prep = (int)((n_alloc + CB_THREADS - 1) / CB_THREADS);
    const int nbj = std::max<int64_t>(p->nblk_comb, (p->nq_pad + F_THREADS - 1) / F_THREADS);

    if ((e = cudaMalloc(&p->tdup, n_alloc * sizeof(Rec8)))) return e;
    if ((e = cudaMalloc(&p->tpair, (n_alloc / 2) * sizeof(Rec8)))) return e;
    const int k1max = std::max(p->k1, p->k1_tc), s2max = std::max(p->s2, p->s2_tc);
    if ((e = cudaMalloc(&p->part1, (size_t)k1max * p->nq_pad * sizeof(float2)))) return e;
    if ((e = cudaMalloc(&p->pdup, p->nq_pad * sizeof(Rec8)))) return e;
    if ((e = cudaMalloc(&p->part2, (size_t)s2max * n_alloc * sizeof(double)))) return e;
    if ((e = cudaMalloc(&p->trec, n_alloc * sizeof(Rec16)))) return e;
    if ((e = cudaMalloc(&p->prec16, p->nq_pad * sizeof(Rec16)))) return e;
    if ((e = cudaMalloc(&p->pu, p->nq_pad * sizeof(float)))) return e;
    k_point_recs<<<(unsigned)((p->nq_pad + 255) / 256), 256>>>(p->xs, p->nq_pad, p->d, p->tc_P,
                                                              p->prec16);
    if ((e = cudaStreamSynchronize(0))) return e;
    if ((e = cudaMalloc(&p->part2_64, (size_t)p->s2_64 * n_alloc * sizeof(double)))) return e;
    if ((e = cudaMalloc(&p->blockJ, (size_t)nbj * sizeof(double)))) return e;
    if ((e = cudaMalloc(&p->psinu, (size_t)p->nblk_prep * sizeof(double)))) return e;
    if ((e = cudaMalloc(&p->a64, n_alloc * sizeof(double)))) return e;
    if ((e = cudaMalloc(&p->prec64, (size_t)p->nq_pad * 4 * sizeof(double)))) return e;
    if ((e = cudaMalloc(&p->lse_buf, (size_t)p->nq_pad * sizeof(double)))) return e;
    return cudaSuccess;
}

void dense_free(rsot_problem *p) {
    cudaFree(p->trec);
    cudaFree(p->prec16);
    cudaFree(p->pu);
    cudaFree(p->tdup);
    cudaFree(p->tpair);
    cudaFree(p->part1);
    cudaFree(p->pdup);
    cudaFree(p->part2);
    cudaFree(p->part2_64);
    cudaFree(p->blockJ);
    cudaFree(p->psinu);
    cudaFree(p->a64);
    cudaFree(p->prec64);
    cudaFree(p->lse_buf);
}

template <int D>
static cudaError_t launch_mixed_d(rsot_problem *p, const double *psi, double eps, double *grad) {
    cudaStream_t st = p->stream;
    const int64_t n_p1 = round_up(p->n, P1_TS);
    // tensor-core passes by default; their FP32 kernels run as the fallback when
    // the prep or combine kernel finds an operand outside the f16 range (gate)
    const bool tc = use_tensor_pairs(p);
    int *gate = tc ? &p->res_dev->gate : nullptr;
    const int k1 = tc ? p->k1_tc : p->k1, chunk1 = tc ? p->chunk1_tc : p->chunk1;
    const int s2 = tc ? p->s2_tc : p->s2;
    const int64_t chunk2 = tc ? p->chunk2_tc : p->chunk2;
    trace_begin(p, "prep_targets_mixed");
    k_prep_mixed<<<p->nblk_prep, CB_THREADS, 0, st>>>(psi, p->y64, p->lnu, p->nu, p->n, p->n_pad,
                                                      p->d, eps, p->tdup, p->tpair, p->psinu,
                                                      p->flags, tc ? p->trec : nullptr,
                                                      1.0 / (double)p->tc_P, gate);
    trace_end(p);
    if (tc) {
        dim3 gt((unsigned)(p->nq_pad / TC_ROWS), (unsigned)k1);
        trace_begin(p, "lse_tc");
        k_lse_tc<<<gt, TC_THREADS, TC_SMEM1, st>>>(p->prec16, p->nq_pad, p->trec,
                                            (int)round_up(p->n, TC_TS), chunk1, p->part1,
                                            p->flags, gate);
        trace_end(p);
    }
    dim3 g1((unsigned)(p->nq_pad / P1_TILE), (unsigned)k1);
    trace_begin(p, "lse_mixed");
    k_lse_mixed<D><<<g1, P1_THREADS, 0, st>>>(p->xs, p->nq_pad, p->tdup, (int)n_p1, chunk1,
                                              p->part1, p->flags, gate, 1);
    trace_end(p);
    trace_begin(p, "combine_mixed");
    k_combine<<<p->nblk_comb, CB_THREADS, 0, st>>>(p->part1, k1, p->nq_pad, p->nq, p->xs, p->d,
                                                   p->lmass2, p->mass, p->pdup, p->blockJ,
                                                   p->lse_buf, tc ? p->pu : nullptr);
    trace_end(p);
    if (tc) {
        dim3 gt((unsigned)(p->n_pad / TC_ROWS), (unsigned)s2);
        trace_begin(p, "grad_tc");
        k_grad_tc<<<gt, TC_THREADS, TC_SMEM2, st>>>(p->trec, p->prec16, p->pu, p->nq_pad, chunk2,
                                             p->part2, p->n_pad, p->flags, gate);
        trace_end(p);
    }
    const int tpp = pick_tpp(p->n);
    const int64_t blk2 = (int64_t)P2_THREADS * 2 * tpp;
    dim3 g2((unsigned)((p->n + blk2 - 1) / blk2), (unsigned)s2);
    trace_begin(p, "grad_mixed");
    if (tpp == 4)
        k_grad_mixed<D, 4><<<g2, P2_THREADS, 0, st>>>(p->tpair, p->pdup, p->nq_pad, chunk2,
                                                      p->part2, p->n_pad, p->flags, gate, 1);
    else if (tpp == 2)
        k_grad_mixed<D, 2><<<g2, P2_THREADS, 0, st>>>(p->tpair, p->pdup, p->nq_pad, chunk2,
                                                      p->part2, p->n_pad, p->flags, gate, 1);
    else
        k_grad_mixed<D, 1><<<g2, P2_THREADS, 0, st>>>(p->tpair, p->pdup, p->nq_pad, chunk2,
                                                      p->part2, p->n_pad, p->flags, gate, 1);
    trace_end(p);
    trace_begin(p, "finalize_grad");
    k_finalize_grad<<<(unsigned)((p->n + 255) / 256), 256, 0, st>>>(p->part2, s2, p->n_pad,
                                                                    p->nu, p->n, grad);
    trace_end(p);
    trace_begin(p, "finalize_J");
    k_finalize_J<<<1, 256, 0, st>>>(p->blockJ, p->nblk_comb, p->psinu, p->nblk_prep, psi, eps,
                                    p->msum, p->hx, 1, p->res_dev);
    trace_end(p);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Softmax refinement (Eq. softmax_refinement_formula): with the coarse
// problem's pass 1 at psi (R_q, u_q = log2 m_q - R_q), the fine potential is
//   psi_k = -eps ln sum_q m_q exp(-c(x_q, y_k)/eps) / S_c(x_q)
//         = psi_c - eps ln sum_q 2^( -k|y'_k|^2 + x'_q.(2k y'_k) + u_q )
// i.e. a pass 2 over the fine targets with target records of b_k = 0.
// ----------------------------------------------------------------------------
__global__ void k_prep_fine(const double *__restrict__ yf, int64_t nf, int64_t nf_alloc, int d,
                            const double *__restrict__ origin3, double eps, Rec8 *__restrict__ tpair) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nf_alloc) return;
    const double k = kLog2e / (2.0 * eps);
    float w[3] = {0.f, 0.f, 0.f};
    float c = kPadC;
    if (j < nf) {
        double yy = 0.0;
        for (int t = 0; t < d; ++t) {
            const double yt = yf[j * d + t] - origin3[t];
            w[t] = (float)(2.0 * k * yt);
            yy += yt * yt;
        }
        c = (float)(-k * yy);
    }
    float *pr = reinterpret_cast<float *>(tpair + (j >> 1));
    const int l = (int)(j & 1);
    pr[0 + l] = w[0];
    pr[2 + l] = w[1];
    pr[4 + l] = w[2];
    pr[6 + l] = c;
}

__global__ void k_refine_final(const double *__restrict__ part2, int s2, int64_t stride, int64_t nf,
                               const double *__restrict__ psi_coarse, double eps,
                               double *__restrict__ out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nf) return;
    double s = 0.0;
    for (int i = 0; i < s2; ++i) s += part2[(int64_t)i * stride + j];
    out[j] = psi_coarse[0] - eps * log(s);
}

template <int D>
static cudaError_t softmax_refine_d(rsot_problem *p, const double *psi, double eps, int64_t nf,
                                    const double *yf, double *out) {
    cudaStream_t st = p->stream;
    cudaError_t e;
    const int64_t n_p1 = round_up(p->n, P1_TS);
    k_prep_mixed<<<p->nblk_prep, CB_THREADS, 0, st>>>(psi, p->y64, p->lnu, p->nu, p->n, p->n_pad,
                                                      p->d, eps, p->tdup, p->tpair, p->psinu,
                                                      p->flags, nullptr, 1.0, nullptr);
    dim3 g1((unsigned)(p->nq_pad / P1_TILE), (unsigned)p->k1);
    k_lse_mixed<D><<<g1, P1_THREADS, 0, st>>>(p->xs, p->nq_pad, p->tdup, (int)n_p1, p->chunk1,
                                              p->part1, p->flags);
    k_combine<<<p->nblk_comb, CB_THREADS, 0, st>>>(p->part1, p->k1, p->nq_pad, p->nq, p->xs, p->d,
                                                   p->lmass2, p->mass, p->pdup, p->blockJ,
                                                   p->lse_buf);
    const int64_t nf_alloc = round_up(nf, 1024);
    const int64_t blocks = nf_alloc / 1024;
    const void *f2 = (const void *)k_grad_mixed<D, 4>;
    int s2 = pick_split(blocks, p->nq_pad / P2_TS, (int64_t)p->num_sms * occupancy(f2, P2_THREADS, 0));
    const int64_t chunk2 = round_up((p->nq_pad + s2 - 1) / s2, P2_TS);
    s2 = (int)((p->nq_pad + chunk2 - 1) / chunk2);
    Rec8 *tpf = nullptr;
    double *part = nullptr, *org = nullptr;
    if ((e = cudaMallocAsync(&tpf, (nf_alloc / 2) * sizeof(Rec8), st))) return e;
    if ((e = cudaMallocAsync(&part, (size_t)s2 * nf_alloc * sizeof(double), st))) return e;
    if ((e = cudaMallocAsync(&org, 3 * sizeof(double), st))) return e;
    if ((e = cudaMemcpyAsync(org, p->origin, 3 * sizeof(double), cudaMemcpyHostToDevice, st))) return e;
    k_prep_fine<<<(unsigned)((nf_alloc + 255) / 256), 256, 0, st>>>(yf, nf, nf_alloc, p->d, org, eps, tpf);
    dim3 g2((unsigned)blocks, (unsigned)s2);
    k_grad_mixed<D, 4><<<g2, P2_THREADS, 0, st>>>(tpf, p->pdup, p->nq_pad, chunk2, part, nf_alloc,
                                                  p->flags);
    k_refine_final<<<(unsigned)((nf + 255) / 256), 256, 0, st>>>(part, s2, nf_alloc, nf, psi, eps, out);
    e = cudaGetLastError();
    cudaFreeAsync(tpf, st);
    cudaFreeAsync(part, st);
    cudaFreeAsync(org, st);
    return e;
}

cudaError_t launch_softmax_refine(rsot_problem *p, const double *psi_dev, double eps, int64_t nf,
                                  const double *yf_dev, double *out_dev) {
    return p->d == 3 ? softmax_refine_d<3>(p, psi_dev, eps, nf, yf_dev, out_dev)
                     : softmax_refine_d<2>(p, psi_dev, eps, nf, yf_dev, out_dev);
}

// gradient and log2-domain J from pass-2 partials [s2][n_pad] and nbj pass-1
// block partials of sum_q m_q R_q (the compensated path's finalisation)
cudaError_t launch_finalize_log2(rsot_problem *p, const double *psi, double eps,
                                 const double *part2, int s2, int nbj, double *grad) {
    cudaStream_t st = p->stream;
    trace_begin(p, "finalize_grad");
    k_finalize_grad<<<(unsigned)((p->n + 255) / 256), 256, 0, st>>>(part2, s2, p->n_pad, p->nu,
                                                                    p->n, grad);
    trace_end(p);
    trace_begin(p, "finalize_J");
    k_finalize_J<<<1, 256, 0, st>>>(p->blockJ, nbj, p->psinu, p->nblk_prep, psi, eps, p->msum,
                                    p->hx, 1, p->res_dev);
    trace_end(p);
    return cudaGetLastError();
}

cudaError_t launch_dense_mixed(rsot_problem *p, const double *psi, double eps, double *grad) {
    return p->d == 3 ? launch_mixed_d<3>(p, psi, eps, grad) : launch_mixed_d<2>(p, psi, eps, grad);
}

template <int D>
static cudaError_t launch_fp64_d(rsot_problem *p, const double *psi, double eps, double *grad,
                                 const double *alpha, const double *beta) {
    cudaStream_t st = p->stream;
    trace_begin(p, "prep_targets_fp64");
    k_prep_fp64<<<p->nblk_prep, CB_THREADS, 0, st>>>(psi, p->lnu, p->nu, p->n, p->n_pad, eps,
                                                     p->a64, p->psinu, p->flags);
    trace_end(p);
    const unsigned nb1 = (unsigned)((p->nq_pad + F_THREADS - 1) / F_THREADS);
    const double hinv = 0.5 * (1.0 / eps);   // exact halving of 1/eps
    trace_begin(p, "lse_fp64");
    if (alpha)
        k_lse_fp64<D, true><<<nb1, F_THREADS, 0, st>>>(p->x64, p->nq, p->nq_pad, p->y64, p->a64,
                                                       p->n, hinv, alpha, beta, psi, eps, p->mass,
                                                       p->prec64, p->blockJ, p->lse_buf, p->res_dev);
    else
        k_lse_fp64<D, false><<<nb1, F_THREADS, 0, st>>>(p->x64, p->nq, p->nq_pad, p->y64, p->a64,
                                                        p->n, hinv, alpha, beta, psi, eps, p->mass,
                                                        p->prec64, p->blockJ, p->lse_buf, p->res_dev);
    trace_end(p);
    dim3 g2((unsigned)((p->n + F_THREADS - 1) / F_THREADS), (unsigned)p->s2_64);
    trace_begin(p, "grad_fp64");
    if (alpha)
        k_grad_fp64<D, true><<<g2, F_THREADS, 0, st>>>(p->y64, p->a64, p->n, p->prec64, p->nq_pad,
                                                       p->chunk2_64, hinv, alpha, beta, p->part2_64,
                                                       p->n_pad);
    else
        k_grad_fp64<D, false><<<g2, F_THREADS, 0, st>>>(p->y64, p->a64, p->n, p->prec64, p->nq_pad,
                                                        p->chunk2_64, hinv, alpha, beta,
                                                        p->part2_64, p->n_pad);
    trace_end(p);
    trace_begin(p, "finalize_grad");
    k_finalize_grad<<<(unsigned)((p->n + 255) / 256), 256, 0, st>>>(p->part2_64, p->s2_64,
                                                                    p->n_pad, p->nu, p->n, grad);
    trace_end(p);
    trace_begin(p, "finalize_J");
    k_finalize_J<<<1, 256, 0, st>>>(p->blockJ, (int)nb1, p->psinu, p->nblk_prep, psi, eps, p->msum,
                                    0.0, 0, p->res_dev);
    trace_end(p);
    return cudaGetLastError();
}

cudaError_t launch_dense_fp64(rsot_problem *p, const double *psi, double eps, double *grad) {
    return p->d == 3 ? launch_fp64_d<3>(p, psi, eps, grad, nullptr, nullptr)
                     : launch_fp64_d<2>(p, psi, eps, grad, nullptr, nullptr);
}

// the cutoffs alpha_q + beta_j prepared in p->alpha / p->beta (rsot_cutoff.cu)
cudaError_t launch_trunc_fp64(rsot_problem *p, const double *psi, double eps, double *grad) {
    return p->d == 3 ? launch_fp64_d<3>(p, psi, eps, grad, p->alpha, p->beta)
                     : launch_fp64_d<2>(p, psi, eps, grad, p->alpha, p->beta);
}

cudaError_t launch_covering_cost(rsot_problem *p, double *C0_dev) {
    const int nb = (int)((p->nq + 255) / 256);
    float *bm = nullptr;
    cudaError_t e = cudaMallocAsync(&bm, (size_t)nb * sizeof(float), p->stream);
    if (e) return e;
    k_cover<<<nb, 256, 0, p->stream>>>(p->xs, p->nq, p->nq_pad, p->y64, p->n, p->d, bm);
    k_max_f<<<1, 256, 0, p->stream>>>(bm, nb, C0_dev);
    e = cudaGetLastError();
    cudaFreeAsync(bm, p->stream);
    return e;
}

cudaError_t launch_point_L(rsot_problem *p, double *L_dev) {
    k_point_L<<<(unsigned)((p->nq + 255) / 256), 256, 0, p->stream>>>(
        p->lse_buf, p->x64, p->nq, p->d, p->last_kind, p->last_eps, p->res_dev, L_dev);
    return cudaGetLastError();
}

// Outputs are written only on success: the evaluation's gradient reaches the
// caller's device buffer through this copy, which reads the result block on
// the device (after every pass on the stream) and copies nothing on an error.
__global__ void k_commit_grad(const double *__restrict__ src, double *__restrict__ dst, int64_t n,
                              const EvalResult *__restrict__ res, int require_nonempty) {
    const bool ok = res->flags == 0 && isfinite(res->J) && !(require_nonempty && res->empty > 0);
    if (!ok) return;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x)
        dst[j] = src[j];
}

cudaError_t launch_commit_grad(const double *src, double *dst, int64_t n, const EvalResult *res,
                               int require_nonempty, cudaStream_t st) {
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    k_commit_grad<<<(unsigned)blocks, 256, 0, st>>>(src, dst, n, res, require_nonempty);
    return cudaGetLastError();
}

cudaError_t launch_psi_stats(rsot_problem *p, const double *psi, double *out2) {
    k_psi_stats<<<1, 256, 0, p->stream>>>(psi, p->n, out2);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Allocation-free dense evaluation (rsot_eval_dense_noalloc).  The scratch of
// the mixed-precision dense passes lives in one file-scope device array of a
// fixed size instead of memory from cudaMalloc, for callers that must not
// allocate device memory themselves.  Host code reaches the array only
// through the address cudaGetSymbolAddress returns for the current device.
// ----------------------------------------------------------------------------
namespace {

constexpr int64_t NA_MAX_NQ = RSOT_NOALLOC_MAX_NQ;   // multiple of 1024
constexpr int64_t NA_MAX_N = RSOT_NOALLOC_MAX_N;     // multiple of 1024
constexpr int NA_MAX_S2 = 16;                        // pass-2 point splits
constexpr int NA_PTS_BLOCKS = (int)(NA_MAX_NQ / CB_THREADS);
// pass-1 partials: k1 target chunks x nq_pad points, k1 * nq_pad <= NA_K1_ROWS
// (small point sets take more chunks, so that the grid still fills the GPU)
constexpr int64_t NA_K1_ROWS = 4 * NA_MAX_NQ;
constexpr int NA_BBOX_BLOCKS = 1024;   // partial bounding boxes (6 doubles each)

constexpr size_t na_align(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t NA_OFF_RES = 0;
constexpr size_t NA_OFF_ORIGIN = na_align(NA_OFF_RES + sizeof(EvalResult));
constexpr size_t NA_OFF_BBOX = na_align(NA_OFF_ORIGIN + 4 * sizeof(double));
constexpr size_t NA_OFF_XS = na_align(NA_OFF_BBOX + 6 * NA_BBOX_BLOCKS * sizeof(double));
constexpr size_t NA_OFF_LM2 = na_align(NA_OFF_XS + 3 * NA_MAX_NQ * sizeof(float));
constexpr size_t NA_OFF_LSE = na_align(NA_OFF_LM2 + NA_MAX_NQ * sizeof(double));
constexpr size_t NA_OFF_PDUP = na_align(NA_OFF_LSE + NA_MAX_NQ * sizeof(double));
constexpr size_t NA_OFF_PART1 = na_align(NA_OFF_PDUP + NA_MAX_NQ * sizeof(Rec8));
constexpr size_t NA_OFF_TDUP = na_align(NA_OFF_PART1 + NA_K1_ROWS * sizeof(float2));
constexpr size_t NA_OFF_TPAIR = na_align(NA_OFF_TDUP + NA_MAX_N * sizeof(Rec8));
constexpr size_t NA_OFF_PART2 = na_align(NA_OFF_TPAIR + (NA_MAX_N / 2) * sizeof(Rec8));
constexpr size_t NA_OFF_BLOCKJ = na_align(NA_OFF_PART2 + (size_t)NA_MAX_S2 * NA_MAX_N * sizeof(double));
constexpr size_t NA_OFF_PSINU = na_align(NA_OFF_BLOCKJ + (NA_MAX_NQ / CB_THREADS) * sizeof(double));
constexpr size_t NA_OFF_PTS = na_align(NA_OFF_PSINU + (NA_MAX_N / CB_THREADS) * sizeof(double));
constexpr size_t NA_OFF_GRAD = na_align(NA_OFF_PTS + 2 * NA_PTS_BLOCKS * sizeof(double));
constexpr size_t NA_BYTES = na_align(NA_OFF_GRAD + NA_MAX_N * sizeof(double));
static_assert(NA_BYTES == RSOT_NOALLOC_SCRATCH_BYTES, "scratch size stated in rsot.h");

// Shared by every call on a device; holds the last call's contents.
static __device__ __align__(256) unsigned char g_na_scratch[NA_BYTES];

// Partial bounding boxes of points and targets: block b covers a grid-stride
// share of both sets and writes (lo[3], hi[3]) to part[6 b ..].
__global__ void k_na_bbox(const double *__restrict__ x, int64_t nq, const double *__restrict__ y,
                          int64_t n, int d, double *__restrict__ part) {
    __shared__ double slo[3][256], shi[3][256];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq + n; i += stride) {
        const double *v = i < nq ? x + i * d : y + (i - nq) * d;
        for (int k = 0; k < d; ++k) {
            lo[k] = fmin(lo[k], v[k]);
            hi[k] = fmax(hi[k], v[k]);
        }
    }
    for (int k = 0; k < 3; ++k) {
        slo[k][threadIdx.x] = lo[k];
        shi[k][threadIdx.x] = hi[k];
    }
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int k = 0; k < 3; ++k) {
                slo[k][threadIdx.x] = fmin(slo[k][threadIdx.x], slo[k][threadIdx.x + o]);
                shi[k][threadIdx.x] = fmax(shi[k][threadIdx.x], shi[k][threadIdx.x + o]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 3) {
        part[6 * blockIdx.x + threadIdx.x] = slo[threadIdx.x][0];
        part[6 * blockIdx.x + 3 + threadIdx.x] = shi[threadIdx.x][0];
    }
}

// bounding-box centre from the partial boxes (one block)
__global__ void k_na_origin(const double *__restrict__ part, int nparts, int d,
                            double *__restrict__ origin) {
    __shared__ double slo[3][256], shi[3][256];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = threadIdx.x; b < nparts; b += blockDim.x)
        for (int k = 0; k < 3; ++k) {
            lo[k] = fmin(lo[k], part[6 * b + k]);
            hi[k] = fmax(hi[k], part[6 * b + 3 + k]);
        }
    for (int k = 0; k < 3; ++k) {
        slo[k][threadIdx.x] = lo[k];
        shi[k][threadIdx.x] = hi[k];
    }
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int k = 0; k < 3; ++k) {
                slo[k][threadIdx.x] = fmin(slo[k][threadIdx.x], slo[k][threadIdx.x + o]);
                shi[k][threadIdx.x] = fmax(shi[k][threadIdx.x], shi[k][threadIdx.x + o]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) origin[k] = k < d ? 0.5 * (slo[k][0] + shi[k][0]) : 0.0;
}

// translated FP32 point coordinates (SoA, zero padded), log2 m_q, and block
// partials of sum m_q and sum m_q |x'_q|^2 / 2
__global__ void k_na_points(const double *__restrict__ x, const double *__restrict__ mass,
                            int64_t nq, int64_t nq_pad, int d, const double *__restrict__ origin,
                            float *__restrict__ xs, double *__restrict__ lm2,
                            double *__restrict__ pts_part) {
    __shared__ double sh[32];
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double m = 0.0, h = 0.0;
    if (q < nq_pad) {
        double r2 = 0.0;
        for (int k = 0; k < d; ++k) {
            const double v = q < nq ? x[q * d + k] - origin[k] : 0.0;
            xs[k * nq_pad + q] = (float)v;
            r2 += v * v;
        }
        if (q < nq) {
            m = mass[q];
            h = m * 0.5 * r2;
            lm2[q] = m > 0.0 ? log2(m) : -INFINITY;
        }
    }
    const double sm = block_sum_d(m, sh);
    const double shh = block_sum_d(h, sh);
    if (threadIdx.x == 0) {
        pts_part[2 * blockIdx.x] = sm;
        pts_part[2 * blockIdx.x + 1] = shh;
    }
}

// target records from the caller's raw targets (translated on the fly)
__global__ void k_na_targets(const double *__restrict__ psi, const double *__restrict__ y,
                             const double *__restrict__ nu, int64_t n, int64_t n_alloc, int d,
                             double eps, const double *__restrict__ origin, Rec8 *__restrict__ tdup,
                             Rec8 *__restrict__ tpair, double *__restrict__ psinu_part,
                             int *__restrict__ flags) {
    __shared__ double sh[32];
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double psic = psi[0];
    const double k = kLog2e / (2.0 * eps);
    double contrib = 0.0;
    if (j < n_alloc) {
        float w[3] = {0.f, 0.f, 0.f};
        float c = kPadC;
        if (j < n) {
            const double ps = psi[j];
            if (!isfinite(ps)) atomicOr(flags, kErrNonfinitePsi);
            const double b = ((ps - psic) / eps + log(nu[j])) * kLog2e;
            double yy = 0.0;
            for (int t = 0; t < d; ++t) {
                const double yt = y[j * d + t] - origin[t];
                w[t] = (float)(2.0 * k * yt);
                yy += yt * yt;
            }
            c = (float)(b - k * yy);
            contrib = ps * nu[j];
        }
        Rec8 r;
        r.a = make_float4(w[0], w[0], w[1], w[1]);
        r.b = make_float4(w[2], w[2], c, c);
        tdup[j] = r;
        float *pr = reinterpret_cast<float *>(tpair + (j >> 1));
        const int l = (int)(j & 1);
        pr[0 + l] = w[0];
        pr[2 + l] = w[1];
        pr[4 + l] = w[2];
        pr[6 + l] = c;
    }
    const double s = block_sum_d(contrib, sh);
    if (threadIdx.x == 0) psinu_part[blockIdx.x] = s;
}

// J = psi_c sum m - sum m |x'|^2/2 + eps ln2 sum_q m_q R_q - sum psi nu, to a host-visible result
__global__ void k_na_finalize_J(const double *__restrict__ blockJ, int nbj,
                                const double *__restrict__ psinu, int npn,
                                const double *__restrict__ pts_part, int npts,
                                const double *__restrict__ psi, double eps,
                                EvalResult *__restrict__ res) {
    __shared__ double sh[32];
    double a = 0.0, b = 0.0, m = 0.0, h = 0.0;
    for (int i = threadIdx.x; i < nbj; i += blockDim.x) a += blockJ[i];
    for (int i = threadIdx.x; i < npn; i += blockDim.x) b += psinu[i];
    for (int i = threadIdx.x; i < npts; i += blockDim.x) {
        m += pts_part[2 * i];
        h += pts_part[2 * i + 1];
    }
    const double sa = block_sum_d(a, sh), sb = block_sum_d(b, sh);
    const double smm = block_sum_d(m, sh), shh = block_sum_d(h, sh);
    if (threadIdx.x == 0) {
        res->psic = psi[0];
        res->J = psi[0] * smm - shh + eps * kLn2 * sa - sb;
    }
}

template <int D>
cudaError_t na_launch(unsigned char *base, int64_t nq, const double *x, const double *mass,
                      int64_t n, const double *y, const double *nu, const double *psi, double eps,
                      double *grad, cudaStream_t st, int num_sms) {
    EvalResult *res = reinterpret_cast<EvalResult *>(base + NA_OFF_RES);
    double *origin = reinterpret_cast<double *>(base + NA_OFF_ORIGIN);
    float *xs = reinterpret_cast<float *>(base + NA_OFF_XS);
    double *lm2 = reinterpret_cast<double *>(base + NA_OFF_LM2);
    double *lse = reinterpret_cast<double *>(base + NA_OFF_LSE);
    Rec8 *pdup = reinterpret_cast<Rec8 *>(base + NA_OFF_PDUP);
    float2 *part1 = reinterpret_cast<float2 *>(base + NA_OFF_PART1);
    Rec8 *tdup = reinterpret_cast<Rec8 *>(base + NA_OFF_TDUP);
    Rec8 *tpair = reinterpret_cast<Rec8 *>(base + NA_OFF_TPAIR);
    double *part2 = reinterpret_cast<double *>(base + NA_OFF_PART2);
    double *blockJ = reinterpret_cast<double *>(base + NA_OFF_BLOCKJ);
    double *psinu = reinterpret_cast<double *>(base + NA_OFF_PSINU);
    double *pts = reinterpret_cast<double *>(base + NA_OFF_PTS);
    double *bbox = reinterpret_cast<double *>(base + NA_OFF_BBOX);
    double *gscr = reinterpret_cast<double *>(base + NA_OFF_GRAD);

    const int64_t nq_pad = round_up(nq, P1_TILE);
    const int64_t n_alloc = round_up(n, 1024);
    const int64_t n_p1 = round_up(n, P1_TS);
    const int nb_pts = (int)(nq_pad / CB_THREADS);
    const int nb_prep = (int)(n_alloc / CB_THREADS);
    cudaError_t e = cudaMemsetAsync(res, 0, sizeof(EvalResult), st);
    if (e) return e;
    const int nbb = (int)std::min<int64_t>({(int64_t)NA_BBOX_BLOCKS, (int64_t)num_sms * 4,
                                            (nq + n + 255) / 256});
    k_na_bbox<<<nbb, 256, 0, st>>>(x, nq, y, n, D, bbox);
    k_na_origin<<<1, 256, 0, st>>>(bbox, nbb, D, origin);
    k_na_points<<<nb_pts, CB_THREADS, 0, st>>>(x, mass, nq, nq_pad, D, origin, xs, lm2, pts);
    k_na_targets<<<nb_prep, CB_THREADS, 0, st>>>(psi, y, nu, n, n_alloc, D, eps, origin, tdup,
                                                 tpair, psinu, &res->flags);
    // pass 1 split over target chunks as the handle path splits it, within the
    // partials' capacity
    const int64_t tiles1 = nq_pad / P1_TILE;
    const int64_t slots1 = (int64_t)num_sms * occupancy((const void *)k_lse_mixed<D>, P1_THREADS, 0);
    int k1 = pick_split(tiles1, std::min<int64_t>(n_p1 / P1_TS, NA_K1_ROWS / nq_pad), slots1);
    const int chunk1 = (int)round_up((n_p1 + k1 - 1) / k1, P1_TS);
    k1 = (int)((n_p1 + chunk1 - 1) / chunk1);
    dim3 g1((unsigned)tiles1, (unsigned)k1);
    k_lse_mixed<D><<<g1, P1_THREADS, 0, st>>>(xs, nq_pad, tdup, (int)n_p1, chunk1, part1,
                                              &res->flags);
    k_combine<<<nb_pts, CB_THREADS, 0, st>>>(part1, k1, nq_pad, nq, xs, D, lm2, mass, pdup, blockJ,
                                             lse);
    const int tpp = pick_tpp(n);
    const int64_t blk2 = (int64_t)P2_THREADS * 2 * tpp;
    const int64_t units2 = (n + blk2 - 1) / blk2;
    const void *f2 = (const void *)k_grad_mixed<D, 4>;
    int s2 = pick_split(units2, std::min<int64_t>(NA_MAX_S2, nq_pad / P2_TS),
                        (int64_t)num_sms * occupancy(f2, P2_THREADS, 0));
    const int64_t chunk2 = round_up((nq_pad + s2 - 1) / s2, P2_TS);
    s2 = (int)((nq_pad + chunk2 - 1) / chunk2);
    dim3 g2((unsigned)units2, (unsigned)s2);
    if (tpp == 4)
        k_grad_mixed<D, 4><<<g2, P2_THREADS, 0, st>>>(tpair, pdup, nq_pad, chunk2, part2, n_alloc,
                                                      &res->flags);
    else if (tpp == 2)
        k_grad_mixed<D, 2><<<g2, P2_THREADS, 0, st>>>(tpair, pdup, nq_pad, chunk2, part2, n_alloc,
                                                      &res->flags);
    else
        k_grad_mixed<D, 1><<<g2, P2_THREADS, 0, st>>>(tpair, pdup, nq_pad, chunk2, part2, n_alloc,
                                                      &res->flags);
    // the gradient goes to the scratch first; the caller's buffer receives it
    // only when the evaluation succeeded
    k_finalize_grad<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part2, s2, n_alloc, nu, n, gscr);
    k_na_finalize_J<<<1, 256, 0, st>>>(blockJ, nb_pts, psinu, nb_prep, pts, nb_pts, psi, eps, res);
    if ((e = cudaGetLastError())) return e;
    return launch_commit_grad(gscr, grad, n, res, 0, st);
}

// Unique id of the current CUDA context (cuCtxGetId through the runtime's
// driver entry point); 0 when there is none yet or the driver lacks the call.
unsigned long long current_context_id() {
    using CtxCur = CUresult (*)(CUcontext *);
    using CtxId = CUresult (*)(CUcontext, unsigned long long *);
    static const std::pair<CtxCur, CtxId> fns = [] {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) !=
                cudaSuccess || qa != cudaDriverEntryPointSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) !=
                cudaSuccess || qb != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return std::pair<CtxCur, CtxId>(nullptr, nullptr);
        }
        return std::pair<CtxCur, CtxId>(reinterpret_cast<CtxCur>(a), reinterpret_cast<CtxId>(b));
    }();
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!fns.first || !fns.second || fns.first(&c) != CUDA_SUCCESS || !c ||
        fns.second(c, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

}  // namespace

// Address of g_na_scratch in the current CUDA context.  The address belongs to
// the context (a device's primary context, re-created after cudaDeviceReset,
// or a context the caller created with the driver API), so it is looked up
// with cudaGetSymbolAddress once per context -- the first call in a context,
// with that context's device current -- and cached under the context's
// unique id.
static unsigned char *na_scratch_address() {
    static std::mutex mu;
    static std::vector<std::pair<unsigned long long, unsigned char *>> cache;
    std::lock_guard<std::mutex> lock(mu);
    unsigned long long id = current_context_id();
    if (id)
        for (const auto &c : cache)
            if (c.first == id) return c.second;
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_na_scratch) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (!id) id = current_context_id();   // the lookup made the context current
    if (id) {
        if (cache.size() >= 64) cache.erase(cache.begin());
        cache.emplace_back(id, static_cast<unsigned char *>(ptr));
    }
    return static_cast<unsigned char *>(ptr);
}

// device memory of the current device, or managed memory: the kernels here
// read it without peer access
static bool na_is_device(const void *p) {
    cudaPointerAttributes a;
    int dev = -1;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == dev);
}

rsot_status eval_dense_noalloc(int d, int64_t nq, const double *x, const double *mass, int64_t n,
                               const double *y, const double *nu, const double *psi, double eps,
                               void *stream, double *J_out, double *grad) {
    if ((d != 2 && d != 3) || nq < 1 || n < 1 || !(eps > 0.0) || !isfinite(eps) || !J_out)
        return RSOT_ERR_ARG;
    if (nq > NA_MAX_NQ || n > NA_MAX_N) return RSOT_ERR_ARG;   // beyond the static scratch
    if (!na_is_device(x) || !na_is_device(mass) || !na_is_device(y) || !na_is_device(nu) ||
        !na_is_device(psi) || !na_is_device(grad))
        return RSOT_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return RSOT_ERR_CUDA;
    }
    unsigned char *base = na_scratch_address();
    if (!base) return RSOT_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = d == 3 ? na_launch<3>(base, nq, x, mass, n, y, nu, psi, eps, grad, st, sms)
                           : na_launch<2>(base, nq, x, mass, n, y, nu, psi, eps, grad, st, sms);
    EvalResult r;
    if (!e) e = cudaMemcpyAsync(&r, base + NA_OFF_RES, sizeof(r), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e) {
        cudaGetLastError();
        return RSOT_ERR_CUDA;
    }
    if (r.flags & kErrTimeout) return RSOT_ERR_TIMEOUT;
    if ((r.flags & kErrNonfinitePsi) || !isfinite(r.J)) return RSOT_ERR_NONFINITE;
    *J_out = r.J;
    return RSOT_OK;
}

}  // namespace rsot

extern "C" rsot_status rsot_eval_dense_noalloc(int d, int64_t nq, const double *x,
                                               const double *mass, int64_t n, const double *y,
                                               const double *nu, const double *psi, double eps,
                                               void *stream, double *J_out, double *grad_out) {
    return rsot::eval_dense_noalloc(d, nq, x, mass, n, y, nu, psi, eps, stream, J_out, grad_out);
}

namespace {
// Self-test of the bounded waits.  One CTA issues a bulk copy into stage 0 and
// arms stage 1 for 16 bytes that no copy ever delivers; every thread waits on
// stage 1 with `limit` polling rounds, which runs out, and thread 0 records the
// timeout.  Before returning, the CTA waits (normal limit) for its own copy in
// stage 0 to land, so that nothing writes its shared memory after it exits.
__global__ void k_wait_selftest(const float4 *__restrict__ src, long long limit,
                                int *__restrict__ flags) {
    __shared__ __align__(128) float4 buf[64];
    __shared__ __align__(8) uint64_t bar[2];
    if (threadIdx.x == 0) {
        rsot::mbar_init(&bar[0], 1);
        rsot::mbar_init(&bar[1], 1);
        rsot::fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        rsot::mbar_expect_tx(&bar[0], (unsigned)sizeof(buf));
        rsot::bulk_g2s(buf, src, (unsigned)sizeof(buf), &bar[0]);
        rsot::mbar_expect_tx(&bar[1], 16u);    // never filled
    }
    __syncthreads();
    const bool got = rsot::mbar_wait_n(&bar[1], 0, limit);
    if (!got && threadIdx.x == 0) atomicOr(flags, rsot::kErrTimeout);
    if (!rsot::mbar_wait(&bar[0], 0) && threadIdx.x == 0) atomicOr(flags, rsot::kErrTimeout);
}

// 8 independent chains a <- a b + c per thread (b = 1 - 2^-20, c = 2^-21: a
// stays near its fixed point 1/2), one FP64 fused multiply-add each.
__global__ void k_probe_dfma(double *out, int iters) {
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = 0.5 + 0.01 * k + 1e-9 * threadIdx.x;
    const double b = 1.0 - 9.5367431640625e-07, c = 4.76837158203125e-07;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == 123.456) out[threadIdx.x] = s;   // keeps the chains alive
}

__global__ void k_exp64(const double *__restrict__ x, double *__restrict__ y, int64_t n) {
    __shared__ double2 s_tab[64];
    rsot::load_exp2_tab(s_tab);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = rsot::exp_tab(x[i], s_tab);
}

// 8 independent chains x <- ex2(x) / 2 per thread keep x in [1/2, 1].
__global__ void k_probe_ex2(float *out, int iters) {
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = 0.5f + 0.05f * k + 1e-6f * threadIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = rsot::ex2_approx(a[k]) * 0.5f;
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == 123.456f) out[threadIdx.x] = s;   // keeps the chains alive
}
}  // namespace

extern "C" rsot_status rsot_probe_ex2_rate(int iters, double *ex2_per_s) {
    if (iters < 1 || !ex2_per_s) return RSOT_ERR_ARG;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    float *out = nullptr;
    cudaEvent_t a, b;
    if (cudaMalloc(&out, 1024 * sizeof(float))) return RSOT_ERR_NOMEM;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int blocks = sms * 8, threads = 256;
    k_probe_ex2<<<blocks, threads>>>(out, iters);   // warm-up
    cudaEventRecord(a);
    k_probe_ex2<<<blocks, threads>>>(out, iters);
    cudaEventRecord(b);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (!e) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    if (e || ms <= 0.f) {
        cudaGetLastError();
        return RSOT_ERR_CUDA;
    }
    *ex2_per_s = (double)blocks * threads * 8.0 * iters / (ms * 1e-3);
    return RSOT_OK;
}

extern "C" rsot_status rsot_selftest_wait_timeout(long long limit, void *stream) {
    if (limit < 1 || limit > rsot::kWaitLimit) return RSOT_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    float4 *src = nullptr;
    int *flags = nullptr;
    int h = 0;
    cudaError_t e = cudaMalloc(&src, 64 * sizeof(float4));
    if (!e) e = cudaMalloc(&flags, sizeof(int));
    if (!e) e = cudaMemsetAsync(src, 0, 64 * sizeof(float4), st);
    if (!e) e = cudaMemsetAsync(flags, 0, sizeof(int), st);
    if (!e) {
        k_wait_selftest<<<1, 128, 0, st>>>(src, limit, flags);
        e = cudaGetLastError();
    }
    if (!e) e = cudaMemcpyAsync(&h, flags, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    cudaFree(src);
    cudaFree(flags);
    if (e) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? RSOT_ERR_NOMEM : RSOT_ERR_CUDA;
    }
    return (h & rsot::kErrTimeout) ? RSOT_ERR_TIMEOUT : RSOT_OK;
}

extern "C" rsot_status rsot_probe_dfma_rate(int iters, double *dfma_per_s) {
    if (iters < 1 || !dfma_per_s) return RSOT_ERR_ARG;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double *out = nullptr;
    cudaEvent_t a, b;
    if (cudaMalloc(&out, 1024 * sizeof(double))) return RSOT_ERR_NOMEM;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int blocks = sms * 8, threads = 256;
    k_probe_dfma<<<blocks, threads>>>(out, iters);   // warm-up
    cudaEventRecord(a);
    k_probe_dfma<<<blocks, threads>>>(out, iters);
    cudaEventRecord(b);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (!e) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    if (e || ms <= 0.f) {
        cudaGetLastError();
        return RSOT_ERR_CUDA;
    }
    *dfma_per_s = (double)blocks * threads * 8.0 * iters / (ms * 1e-3);
    return RSOT_OK;
}

extern "C" rsot_status rsot_exp64(int64_t n, const double *x, double *y) {
    if (n < 1 || !x || !y) return RSOT_ERR_ARG;
    double *dx = nullptr, *dy = nullptr;
    cudaError_t e = cudaMalloc(&dx, (size_t)n * 8);
    if (!e) e = cudaMalloc(&dy, (size_t)n * 8);
    if (!e) e = cudaMemcpy(dx, x, (size_t)n * 8, cudaMemcpyDefault);
    if (!e) {
        k_exp64<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256>>>(dx, dy, n);
        e = cudaGetLastError();
    }
    if (!e) e = cudaMemcpy(y, dy, (size_t)n * 8, cudaMemcpyDefault);
    cudaFree(dx);
    cudaFree(dy);
    if (e) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? RSOT_ERR_NOMEM : RSOT_ERR_CUDA;
    }
    return RSOT_OK;
}
