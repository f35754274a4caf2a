// Tensor-core form of the pair arithmetic of both mixed passes.
//
// The exponent of every pair, r_qj = c_j + x'_q . w_j, is the inner product
// of a 16-slot point vector and a 16-slot target vector (f16 operands, f32
// accumulation in mma.sync m16n8k16):
//
//   point  [X0h X0l X0h  X1h X1l X1h  X2h X2l X2h  256 1/16  Sh Sl  0 0 0]
//   target [W0h W0h W0l  W1h W1h W1l  W2h W2h W2l  Ch  Cl    256 256 0 0 0]
//
// with X = P x' (P a power of two per problem, |X| <= 32), W = w / P, "h"/"l"
// the f16 head and tail of each value (v = h + l to ~2^-22 relative), and
// c split as Ch = f16(c / 256), Cl = f16(16 (c - 256 Ch)) so that the tail
// stays a normal f16 number for |c| from ~1e-2 to 1.5e7.  The three products per coordinate (Xh Wh + Xl Wh +
// Xh Wl) give the FP32 product to the same order; the dropped Xl Wl term is
// ~2^-24 relative.  The slots S (a shift folded into the product) are kept
// zero by the passes, which add their per-point shifts in FP32 so that both
// passes see bitwise the same r_qj.  Per pair the FP32 pipe is left with the
// shift and the accumulation (packed, one instruction per two pairs each)
// instead of three multiply-adds and two adds.
//
// Records are 32 bytes in the lane order of the mma fragments: segment t
// (8 bytes) holds slots (2t, 2t+1 | 2t+8, 2t+9), which is both the B fragment
// of lane (g, t) for column g and the A fragment half of lane (g, t) for a
// row.  Lane (g, t) of a warp reads record 8 nb + g, segment t, i.e. uint2
// index 32 nb + lane of a staged tile: one conflict-free 256-byte read per
// n-block.
#pragma once

#include <cuda_fp16.h>

#include "rsot_internal.cuh"

namespace rsot {

struct __align__(32) Rec16 {
    uint2 s[4];
};

// Shapes; the build may override them (-DRSOT_TC_TS=..., etc.) to tune.
#ifndef RSOT_TC_TS
#define RSOT_TC_TS 1024
#endif
#ifndef RSOT_TC_STAGES
#define RSOT_TC_STAGES 2
#endif
#ifndef RSOT_TC_MINB
#define RSOT_TC_MINB 2
#endif
inline constexpr int TC_THREADS = 256;               // 8 warps
inline constexpr int TC_WARPS = TC_THREADS / 32;
inline constexpr int TC_MB = 4;                       // 16-row m-blocks per warp
inline constexpr int TC_ROWS = TC_WARPS * TC_MB * 16; // points (pass 1) / targets (pass 2) per CTA
inline constexpr int TC_TS = RSOT_TC_TS;              // records per stage (multiple of 256)
inline constexpr int TC_STAGES = RSOT_TC_STAGES;
inline constexpr int TC_MINB = RSOT_TC_MINB;          // resident CTAs per SM asked of ptxas
inline constexpr int TC_NBS = TC_TS / 8;              // n-blocks per stage
inline constexpr int TC_GROUP = 8;                    // n-blocks per optimistic group
static_assert(TC_TS % 256 == 0 && 1024 % TC_TS == 0, "stages tile the 1024-padded arrays");
// dynamic shared memory: pass 1 stages target records; pass 2 point records and shifts
inline constexpr size_t TC_SMEM1 = (size_t)TC_STAGES * TC_TS * 32;
inline constexpr size_t TC_SMEM2 = TC_SMEM1 + (size_t)TC_STAGES * TC_TS * sizeof(float);
inline constexpr float TC_RANGE = 60000.0f;           // |f16 operand| bound (f16 max 65504)
inline constexpr float TC_BIG = 1.152921504606846976e18f;  // 2^60

__device__ __forceinline__ unsigned pack_h2(__half lo, __half hi) {
    return (unsigned)__half_as_ushort(lo) | ((unsigned)__half_as_ushort(hi) << 16);
}

// v ~ h + l with h = f16(v), l = f16(v - h)
__device__ __forceinline__ void split_h(float v, __half &h, __half &l) {
    h = __float2half_rn(v);
    l = __float2half_rn(v - __half2float(h));
}

// point vector: X = P x' (3 values, zero beyond d), S = s / 256
__device__ __forceinline__ Rec16 make_point_rec(const float (&X)[3], float S) {
    __half h0, l0, h1, l1, h2, l2, sh, sl;
    split_h(X[0], h0, l0);
    split_h(X[1], h1, l1);
    split_h(X[2], h2, l2);
    split_h(S, sh, sl);
    const __half c256 = __float2half_rn(256.0f), c16 = __float2half_rn(0.0625f);
    const __half z = __float2half_rn(0.0f);
    Rec16 r;
    r.s[0] = make_uint2(pack_h2(h0, l0), pack_h2(h2, c256));   // k0 k1 | k8 k9
    r.s[1] = make_uint2(pack_h2(h0, h1), pack_h2(c16, sh));    // k2 k3 | k10 k11
    r.s[2] = make_uint2(pack_h2(l1, h1), pack_h2(sl, z));      // k4 k5 | k12 k13
    r.s[3] = make_uint2(pack_h2(h2, l2), pack_h2(z, z));       // k6 k7 | k14 k15
    return r;
}

// target vector: W = w / P (3 values, zero beyond d) and c (|c| < 256 TC_RANGE)
__device__ __forceinline__ Rec16 make_target_rec(const float (&W)[3], float c) {
    __half h0, l0, h1, l1, h2, l2;
    split_h(W[0], h0, l0);
    split_h(W[1], h1, l1);
    split_h(W[2], h2, l2);
    const __half ch = __float2half_rn(c * (1.0f / 256.0f));
    const __half cl = __float2half_rn((c - 256.0f * __half2float(ch)) * 16.0f);
    const __half c256 = __float2half_rn(256.0f), z = __float2half_rn(0.0f);
    Rec16 r;
    r.s[0] = make_uint2(pack_h2(h0, h0), pack_h2(l2, ch));     // k0 k1 | k8 k9
    r.s[1] = make_uint2(pack_h2(l0, h1), pack_h2(cl, c256));   // k2 k3 | k10 k11
    r.s[2] = make_uint2(pack_h2(h1, l1), pack_h2(c256, z));    // k4 k5 | k12 k13
    r.s[3] = make_uint2(pack_h2(h2, h2), pack_h2(z, z));       // k6 k7 | k14 k15
    return r;
}

// D = A B (f16 x f16 -> f32, zero accumulator input)
__device__ __forceinline__ void mma_tc(float (&d)[4], const unsigned (&a)[4], uint2 b) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%10,%10,%10,%10};"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y), "f"(0.0f));
}

// A fragment of one m-block from the records of its rows g and g + 8
// (segment t of each): a0 = row g lo, a1 = row g+8 lo, a2 = row g hi, a3 = row g+8 hi.
__device__ __forceinline__ void load_a(unsigned (&a)[4], uint2 rg, uint2 rg8) {
    a[0] = rg.x;
    a[1] = rg8.x;
    a[2] = rg.y;
    a[3] = rg8.y;
}

// ---- stage bodies of the tensor-core passes (dense and batched kernels) ----
__device__ __forceinline__ void tc_raise(float &M, float mx, float &sf, double &sd) {
    const float mn = ceilf(mx);
    if (mn > M) {
        if (M != -INFINITY) {
            const float dl = M - mn;
            sf *= pow2_int_f(dl);
            sd *= pow2_int_d(dl);
        }
        M = mn;
    }
}

// exact redo of one group of TC_GROUP n-blocks (warp-uniform)
__device__ __forceinline__ void tc_exact_group(const uint2 *__restrict__ gb,
                                               const unsigned (&A)[TC_MB][4], float2 (&M)[TC_MB],
                                               float2 (&Sf)[TC_MB], double2 (&Sd)[TC_MB],
                                               float2 (&acc)[TC_MB]) {
#pragma unroll
    for (int m = 0; m < TC_MB; ++m) {
        float mg = -INFINITY, mg8 = -INFINITY;
#pragma unroll 2
        for (int i = 0; i < TC_GROUP; ++i) {
            float dd[4];
            mma_tc(dd, A[m], gb[32 * i]);
            mg = max3f(mg, dd[0], dd[1]);
            mg8 = max3f(mg8, dd[2], dd[3]);
        }
        tc_raise(M[m].x, mg, Sf[m].x, Sd[m].x);
        tc_raise(M[m].y, mg8, Sf[m].y, Sd[m].y);
        const float2 ng = make_float2(-M[m].x, -M[m].x), ng8 = make_float2(-M[m].y, -M[m].y);
        float2 a = make_float2(0.f, 0.f);
#pragma unroll 2
        for (int i = 0; i < TC_GROUP; ++i) {
            float dd[4];
            mma_tc(dd, A[m], gb[32 * i]);
            const float2 e01 = __fadd2_rn(make_float2(dd[0], dd[1]), ng);
            const float2 e23 = __fadd2_rn(make_float2(dd[2], dd[3]), ng8);
            a = __fadd2_rn(a, make_float2(ex2_approx(e01.x), ex2_approx(e23.x)));
            a = __fadd2_rn(a, make_float2(ex2_approx(e01.y), ex2_approx(e23.y)));
        }
        acc[m] = a;
    }
}

// A fragment of rows (g, g + 8) of a 16-point m-block whose records start at
// rec (uint2 view): segment t of row g and of row g + 8.
__device__ __forceinline__ void tc_load_a(unsigned (&a)[4], const uint2 *rec, int g, int t) {
    load_a(a, rec[g * 4 + t], rec[(g + 8) * 4 + t]);
}


// One stage of pass 1: NBS n-blocks of target records (uint2 view of the
// staged records, already offset by the lane), optimistic groups of
// TC_GROUP n-blocks with the exact redo; sums go to Sf (FP32, this stage).
template <int NBS>
__device__ __forceinline__ void tc_lse_stage(const uint2 *__restrict__ base,
                                             const unsigned (&A)[TC_MB][4], float2 (&M)[TC_MB],
                                             float2 (&Sf)[TC_MB], double2 (&Sd)[TC_MB]) {
    constexpr int NGRP_ = NBS / TC_GROUP;
    static_assert(NBS % TC_GROUP == 0, "whole groups per stage");

            float dc[TC_MB][4];
            {
                const uint2 b = base[0];
#pragma unroll
                for (int m = 0; m < TC_MB; ++m) mma_tc(dc[m], A[m], b);
            }
#pragma unroll 1
            for (int grp = 0; grp < NGRP_; ++grp) {
                float2 acc[TC_MB], ng[TC_MB], ng8[TC_MB];
#pragma unroll
                for (int m = 0; m < TC_MB; ++m) {
                    acc[m] = make_float2(0.f, 0.f);
                    ng[m] = make_float2(-M[m].x, -M[m].x);
                    ng8[m] = make_float2(-M[m].y, -M[m].y);
                }
#pragma unroll
                for (int i = 0; i < TC_GROUP; ++i) {
                    const int nb = grp * TC_GROUP + i;
                    const bool more = (i + 1 < TC_GROUP) || (grp + 1 < NGRP_);
                    float dn[TC_MB][4];
                    if (more) {
                        const uint2 b = base[32 * (nb + 1)];
#pragma unroll
                        for (int m = 0; m < TC_MB; ++m) mma_tc(dn[m], A[m], b);
                    }
#pragma unroll
                    for (int m = 0; m < TC_MB; ++m) {
                        const float2 e01 = __fadd2_rn(make_float2(dc[m][0], dc[m][1]), ng[m]);
                        const float2 e23 = __fadd2_rn(make_float2(dc[m][2], dc[m][3]), ng8[m]);
                        acc[m] = __fadd2_rn(acc[m], make_float2(ex2_approx(e01.x), ex2_approx(e23.x)));
                        acc[m] = __fadd2_rn(acc[m], make_float2(ex2_approx(e01.y), ex2_approx(e23.y)));
                    }
                    if (more) {
#pragma unroll
                        for (int m = 0; m < TC_MB; ++m)
#pragma unroll
                            for (int r = 0; r < 4; ++r) dc[m][r] = dn[m][r];
                    }
                }
                bool bad = false;
#pragma unroll
                for (int m = 0; m < TC_MB; ++m)
                    bad = bad || !(fmaxf(acc[m].x, acc[m].y) <= TC_BIG) || M[m].x == -INFINITY ||
                          M[m].y == -INFINITY;
                if (__any_sync(0xffffffffu, bad))
                    tc_exact_group(base + 32 * grp * TC_GROUP, A, M, Sf, Sd, acc);
#pragma unroll
                for (int m = 0; m < TC_MB; ++m) Sf[m] = __fadd2_rn(Sf[m], acc[m]);
            }
        }

// One stage of pass 2: NBS n-blocks of point records (uint2 view, offset by
// the lane) with their shifts (ub: float2 view of u offset by t, so that
// ub[4 nb] = (u_2t, u_2t+1) of n-block nb); FP32 within the stage, FP64 in acc64.
template <int NBS>
__device__ __forceinline__ void tc_grad_stage(const uint2 *__restrict__ base,
                                              const float2 *__restrict__ ub,
                                              const unsigned (&A)[TC_MB][4],
                                              double2 (&acc64)[TC_MB]) {

            float2 acc[TC_MB];
            float dc[TC_MB][4];
#pragma unroll
            for (int m = 0; m < TC_MB; ++m) acc[m] = make_float2(0.f, 0.f);
            float2 uc = ub[0];
            {
                const uint2 b = base[0];
#pragma unroll
                for (int m = 0; m < TC_MB; ++m) mma_tc(dc[m], A[m], b);
            }
#pragma unroll 4
            for (int nb = 0; nb < NBS; ++nb) {
                float dn[TC_MB][4];
                float2 un = uc;
                const bool more = nb + 1 < NBS;
                if (more) {
                    const uint2 b = base[32 * (nb + 1)];
                    un = ub[4 * (nb + 1)];
#pragma unroll
                    for (int m = 0; m < TC_MB; ++m) mma_tc(dn[m], A[m], b);
                }
#pragma unroll
                for (int m = 0; m < TC_MB; ++m) {
                    const float2 e01 = __fadd2_rn(make_float2(dc[m][0], dc[m][1]), uc);
                    const float2 e23 = __fadd2_rn(make_float2(dc[m][2], dc[m][3]), uc);
                    acc[m] = __fadd2_rn(acc[m], make_float2(ex2_approx(e01.x), ex2_approx(e23.x)));
                    acc[m] = __fadd2_rn(acc[m], make_float2(ex2_approx(e01.y), ex2_approx(e23.y)));
                }
                if (more) {
#pragma unroll
                    for (int m = 0; m < TC_MB; ++m)
#pragma unroll
                        for (int r = 0; r < 4; ++r) dc[m][r] = dn[m][r];
                    uc = un;
                }
            }
#pragma unroll
            for (int m = 0; m < TC_MB; ++m) {
                acc64[m].x += (double)acc[m].x;
                acc64[m].y += (double)acc[m].y;
            }
        }

}  // namespace rsot
