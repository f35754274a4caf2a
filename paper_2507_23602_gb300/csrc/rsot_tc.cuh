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

}  // namespace rsot
