// Inner loops of the mixed-precision passes, shared by the single-problem,
// allocation-free and batched kernels.  Log2 domain: for a point x' and a
// target record (w_j, c_j), r_qj = c_j + x'.w_j (see rsot_dense.cu).
#pragma once

#include "rsot_internal.cuh"

namespace rsot {

// Tile shapes; the build may override them (-DRSOT_P1_PP=..., etc.) to tune.
#ifndef RSOT_P1_PP
#define RSOT_P1_PP 4
#endif
#ifndef RSOT_P1_MINB
#define RSOT_P1_MINB 4
#endif
#ifndef RSOT_P1_SUB
#define RSOT_P1_SUB 16
#endif
#ifndef RSOT_P2_MINB
#define RSOT_P2_MINB 1
#endif
#ifndef RSOT_P2_TPP
#define RSOT_P2_TPP 4
#endif
// Issue form of the per-pair additions (shift and accumulation):
//   0: packed FADD2 for both, 1: scalar FADD for both, 2: packed shift,
//   scalar accumulation.  The dot products always use packed FFMA2.
#ifndef RSOT_ADD_MODE
#define RSOT_ADD_MODE 0
#endif
inline constexpr int P1_THREADS = 128;
inline constexpr int P1_PP = RSOT_P1_PP;                      // point pairs per thread (<= 4)
inline constexpr int P1_TILE = P1_THREADS * 2 * P1_PP;        // points per CTA (divides 1024)
inline constexpr int P1_MINB = RSOT_P1_MINB;                  // resident CTAs per SM asked of ptxas
#ifndef RSOT_P1_TS
#define RSOT_P1_TS 512
#endif
#ifndef RSOT_P2_TS
#define RSOT_P2_TS 512
#endif
inline constexpr int P1_TS = RSOT_P1_TS;                      // targets per stage (divides 1024)
inline constexpr int P1_STAGES = 2;
inline constexpr int P1_SUB = RSOT_P1_SUB;                    // targets per optimistic sub-tile
inline constexpr int P2_MINB = RSOT_P2_MINB;
inline constexpr int P2_TPP_MAX = RSOT_P2_TPP;                // target pairs per thread (pass 2)
inline constexpr float P1_BIG = 1.152921504606846976e18f;     // 2^60: a sub-tile sum above it is redone

inline constexpr int P2_THREADS = 128;
inline constexpr int P2_TS = RSOT_P2_TS;                      // points per stage (divides 1024)
static_assert(1024 % P1_TS == 0 && 1024 % P2_TS == 0 && P1_TS % P1_SUB == 0, "stage shapes");
inline constexpr int P2_STAGES = 2;


__device__ __forceinline__ float2 add_shift(float2 a, float2 b) {
#if RSOT_ADD_MODE == 1
    return make_float2(a.x + b.x, a.y + b.y);
#else
    return __fadd2_rn(a, b);
#endif
}
__device__ __forceinline__ float2 add_acc(float2 a, float2 b) {
#if RSOT_ADD_MODE == 0
    return __fadd2_rn(a, b);
#else
    return make_float2(a.x + b.x, a.y + b.y);
#endif
}

// Exact sub-tile for one point pair: maximum of r over the sub-tile, shift M
// raised to ceil(max) when the maximum exceeds it (rescaling the running sums
// by an exact power of two), then the sum of 2^(r - M).
template <int D>
__device__ __forceinline__ float2 lse_exact_subtile(const Rec8 *T, const float2 (&X)[3], float2 &M,
                                                    float2 &Sf, double2 &Sd) {
    float mx = -INFINITY, my = -INFINITY;
#pragma unroll 4
    for (int t = 0; t < P1_SUB; ++t) {
        const float4 a = T[t].a, b = T[t].b;
        float2 r = make_float2(b.z, b.w);
        if (D == 3) r = __ffma2_rn(X[2], make_float2(b.x, b.y), r);
        r = __ffma2_rn(X[1], make_float2(a.z, a.w), r);
        r = __ffma2_rn(X[0], make_float2(a.x, a.y), r);
        mx = fmaxf(mx, r.x);
        my = fmaxf(my, r.y);
    }
    if (mx > M.x) {
        const float mn = ceilf(mx), dl = M.x - mn;
        Sf.x *= pow2_int_f(dl);
        Sd.x *= pow2_int_d(dl);
        M.x = mn;
    }
    if (my > M.y) {
        const float mn = ceilf(my), dl = M.y - mn;
        Sf.y *= pow2_int_f(dl);
        Sd.y *= pow2_int_d(dl);
        M.y = mn;
    }
    const float2 nm = make_float2(-M.x, -M.y);
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int t = 0; t < P1_SUB; ++t) {
        const float4 a = T[t].a, b = T[t].b;
        float2 r = make_float2(b.z, b.w);
        if (D == 3) r = __ffma2_rn(X[2], make_float2(b.x, b.y), r);
        r = __ffma2_rn(X[1], make_float2(a.z, a.w), r);
        r = __ffma2_rn(X[0], make_float2(a.x, a.y), r);
        const float2 e = __fadd2_rn(r, nm);
        acc = __fadd2_rn(acc, make_float2(ex2_approx(e.x), ex2_approx(e.y)));
    }
    return acc;
}

// One staged tile of P1_TS targets for PP point pairs: optimistic sub-tiles
// of P1_SUB targets with the running integral shift M, an exact sub-tile
// (raising M) when a sub-tile sum exceeds 2^60 or overflows.
template <int D, int PP>
__device__ __forceinline__ void lse_stage(const Rec8 *__restrict__ T, const float2 (&X)[PP][3],
                                          float2 (&M)[PP], float2 (&Sf)[PP], double2 (&Sd)[PP]) {
#pragma unroll 1
    for (int t0 = 0; t0 < P1_TS; t0 += P1_SUB) {
        float2 acc0[PP], acc1[PP], nm[PP];
#pragma unroll
        for (int pp = 0; pp < PP; ++pp) {
            acc0[pp] = make_float2(0.f, 0.f);
            acc1[pp] = make_float2(0.f, 0.f);
            nm[pp] = make_float2(-M[pp].x, -M[pp].y);
        }
#pragma unroll
        for (int t = 0; t < P1_SUB; ++t) {
            const float4 a = T[t0 + t].a;
            const float4 b = T[t0 + t].b;
            const float2 w0 = make_float2(a.x, a.y), w1 = make_float2(a.z, a.w);
            const float2 w2 = make_float2(b.x, b.y), c = make_float2(b.z, b.w);
#pragma unroll
            for (int pp = 0; pp < PP; ++pp) {
                float2 r = c;
                if (D == 3) r = __ffma2_rn(X[pp][2], w2, r);
                r = __ffma2_rn(X[pp][1], w1, r);
                r = __ffma2_rn(X[pp][0], w0, r);
                const float2 e = add_shift(r, nm[pp]);
                const float2 v = make_float2(ex2_approx(e.x), ex2_approx(e.y));
                if (t & 1) acc1[pp] = add_acc(acc1[pp], v);
                else acc0[pp] = add_acc(acc0[pp], v);
            }
        }
#pragma unroll
        for (int pp = 0; pp < PP; ++pp) {
            float2 sub = __fadd2_rn(acc0[pp], acc1[pp]);
            if (!(fmaxf(sub.x, sub.y) <= P1_BIG))
                sub = lse_exact_subtile<D>(T + t0, X[pp], M[pp], Sf[pp], Sd[pp]);
            Sf[pp] = __fadd2_rn(Sf[pp], sub);
        }
    }
}

// One staged tile of P2_TS point records (x0,x0,x1,x1,x2,x2,u,u) for TPP
// target pairs held in registers: acc64 += sum over the tile of
// 2^(c_j + x'.w_j + u_q) = sum_q m_q p_qj, FP32 within the tile, FP64 across.
template <int D, int TPP>
__device__ __forceinline__ void grad_stage(const Rec8 *__restrict__ T, const float2 (&W0)[TPP],
                                           const float2 (&W1)[TPP], const float2 (&W2)[TPP],
                                           const float2 (&C)[TPP], double2 (&acc64)[TPP]) {
    float2 acc[TPP];
#pragma unroll
    for (int tp = 0; tp < TPP; ++tp) acc[tp] = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int i = 0; i < P2_TS; ++i) {
        const float4 a = T[i].a;
        const float4 b = T[i].b;
        const float2 x0 = make_float2(a.x, a.y), x1 = make_float2(a.z, a.w);
        const float2 x2 = make_float2(b.x, b.y), u = make_float2(b.z, b.w);
#pragma unroll
        for (int tp = 0; tp < TPP; ++tp) {
            float2 t = C[tp];
            if (D == 3) t = __ffma2_rn(x2, W2[tp], t);
            t = __ffma2_rn(x1, W1[tp], t);
            t = __ffma2_rn(x0, W0[tp], t);
            t = add_shift(t, u);
            acc[tp] = add_acc(acc[tp], make_float2(ex2_approx(t.x), ex2_approx(t.y)));
        }
    }
#pragma unroll
    for (int tp = 0; tp < TPP; ++tp) {
        acc64[tp].x += (double)acc[tp].x;
        acc64[tp].y += (double)acc[tp].y;
    }
}

}  // namespace rsot
