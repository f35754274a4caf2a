// Compensated evaluation of Algorithm 2: the passes of the mixed path with the
// exponent of every pair carried as a double-float (an unevaluated sum of two
// FP32 numbers, ~44 significant bits) instead of one FP32 number.
//
// Log2 domain and translated coordinates as the mixed passes (rsot_dense.cu):
// r_qj = c_j + x'_q.w_j with w_j = 2k y'_j, c_j = b_j - k|y'_j|^2, k =
// log2(e)/(2 eps), every operand rounded from its FP64 value to head + tail.
// Each product x.w is formed exactly as ph + pe (pe = fma(x_h, w_h, -ph)) plus
// the cross terms x_h w_t + x_t w_h; the heads are summed with TwoSum, so r
// comes with an absolute error of a few 2^-44 |c| instead of 2^-24 |c|.  The
// shift by the running maximum (pass 1) or by u_q = log2 m_q - R_q (pass 2) is
// also a TwoSum, so 2^(r - M) = ex2.approx(a_h) (1 + a_t ln2 + O(a_t^2)), the
// tail a_t folded in as a separately accumulated first-order correction.  Sums
// are Kahan-compensated in FP32 within a tile and FP64 across tiles.
//
// Every step is an explicitly rounded add / mul / fma (no contraction), and
// each thread carries two pairs in the two lanes of the packed FP32x2
// instructions (add/sub/mul/fma .f32x2): two points per thread in pass 1, two
// targets in pass 2; the shared-memory records of the other side hold each
// value twice so that one 16-byte load gives both lanes' operand.
//
// Error budget, relative to each term (ex2.approx: measured <= 2^-22.71 over
// 3 x 2^30 arguments; the budget takes 2^-22.5):
//   one exponential            <= 2^-22.5 + 2^-26           ~ 1.8e-7
//   pass-1 normaliser S_q      <= 1.8e-7 + Kahan 2^-23      ~ 3.0e-7
//   pass-2 term m_q p_qj       <= 1.8e-7 + 3.0e-7 (via u_q) ~ 4.8e-7
//   pass-2 sum over q          <= 4.8e-7 + Kahan 2^-23      ~ 6.0e-7
// hence |g_j - dJ/dpsi_j| <= 6.0e-7 sum_q m_q p_qj and ||g - grad J||_1 <=
// 6.5e-7 sum_q m_q with a margin, whatever the sizes, eps or potentials: the
// solver certifies ||grad J||_1 <= tol from this evaluation (rsot_solve.cpp).
// J errs by <= eps 3e-7 sum_q m_q.
//
// Truncated form (Algorithm 2 with I_q = {j : c(x_q, y_j) < alpha_q + beta_j},
// rsot_cutoff.cu): membership is decided in FP32 where |c_32 - C_qj| exceeds a
// margin that bounds the FP32 distance and cutoff errors, else by the FP64 test
// of the FP64 path (same expression, same translated coordinates), so both
// paths keep the same pairs.
#include <math.h>

#include <algorithm>

#include "rsot_internal.cuh"

namespace rsot {

cudaError_t launch_finalize_log2(rsot_problem *p, const double *psi, double eps,
                                 const double *part2, int s2, int nbj, double *grad);

namespace {

constexpr int D_THREADS = 128;            // threads per block
constexpr int D_ROWS = 2 * D_THREADS;     // points (pass 1) / targets (pass 2) per block
constexpr int D_TS = 128;                 // records per shared-memory tile
constexpr int D_SUB = 8;                  // targets per max sub-tile (pass 1)
constexpr float kExcl = -1.0e30f;

// 64-byte record, every value twice: (v0h, v0h, v0t, v0t), (v1h, ...), (v2h, ...),
// (sh, sh, st, st) -- v = w (targets) or x' (points), s = c (targets) or u (points)
struct __align__(16) DRec {
    float4 a, b, c, d;
};


typedef float2 f2;
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
// a - b rounded once: the product b * -1 is exact
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ f2 lo2(float4 v) { return make_float2(v.x, v.y); }   // heads
__device__ __forceinline__ f2 hi2(float4 v) { return make_float2(v.z, v.w); }   // tails

// s + e = a + b exactly in each lane (Knuth's TwoSum)
__device__ __forceinline__ void two_sum2(f2 a, f2 b, f2 &s, f2 &e) {
    s = add2(a, b);
    const f2 bb = sub2(s, a);
    e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}
// s + e = a - b exactly in each lane (TwoSum of a and -b)
__device__ __forceinline__ void two_diff2(f2 a, f2 b, f2 &s, f2 &e) {
    s = sub2(a, b);
    const f2 bb = sub2(s, a);
    e = sub2(sub2(a, sub2(s, bb)), add2(b, bb));
}
__device__ __forceinline__ void kahan2(f2 &sum, f2 &comp, f2 v) {
    const f2 y = sub2(v, comp);
    const f2 t = add2(sum, y);
    comp = sub2(sub2(t, sum), y);
    sum = t;
}

// Operand held by the thread for its two lanes: head, tail, negated head.
struct Op2 {
    f2 h, t, nh;
};

// One coordinate: (s, lo) += R B with R the thread's operand and (Bh, Bt) the
// shared one: ph = R_h B_h exactly as -nph, pe = R_h B_h - ph, cross terms.
__device__ __forceinline__ void df_term2(const Op2 &R, f2 Bh, f2 Bt, f2 &s, f2 &lo) {
    const f2 nph = mul2(R.nh, Bh);
    const f2 pe = fma2(R.h, Bh, nph);
    lo = fma2(R.h, Bt, lo);
    lo = fma2(R.t, Bh, lo);
    lo = add2(lo, pe);
    f2 e;
    two_diff2(s, nph, s, e);
    lo = add2(lo, e);
}

template <int D>
__device__ __forceinline__ void df_exponent2(const Op2 *R, const DRec &B, f2 sh, f2 st, f2 &rh,
                                             f2 &rt) {
    f2 s = sh, lo = st;
    df_term2(R[0], lo2(B.a), hi2(B.a), s, lo);
    df_term2(R[1], lo2(B.b), hi2(B.b), s, lo);
    if (D == 3) df_term2(R[2], lo2(B.c), hi2(B.c), s, lo);
    rh = add2(s, lo);                // |lo| << |s|: Fast2Sum renormalisation
    rt = sub2(lo, sub2(rh, s));
}

__device__ __forceinline__ void split_f(double v, float &h, float &t) {
    h = (float)v;
    t = (float)(v - (double)h);
}

__device__ __forceinline__ DRec make_drec(const float *v /* 8: h,t pairs */) {
    DRec r;
    r.a = make_float4(v[0], v[0], v[1], v[1]);
    r.b = make_float4(v[2], v[2], v[3], v[3]);
    r.c = make_float4(v[4], v[4], v[5], v[5]);
    r.d = make_float4(v[6], v[6], v[7], v[7]);
    return r;
}

// the two lanes' operands from two records (lane 0 from r0, lane 1 from r1)
__device__ __forceinline__ void load_ops(const DRec &r0, const DRec &r1, Op2 *R, f2 &sh, f2 &st) {
    const float4 *a0 = &r0.a, *a1 = &r1.a;
    for (int t = 0; t < 3; ++t) {
        R[t].h = make_float2(a0[t].x, a1[t].x);
        R[t].t = make_float2(a0[t].z, a1[t].z);
        R[t].nh = make_float2(-a0[t].x, -a1[t].x);
    }
    sh = make_float2(r0.d.x, r1.d.x);
    st = make_float2(r0.d.z, r1.d.z);
}

// FP32 test c(x, y) < alpha + beta outside a margin that bounds the FP32
// errors (|c_32 - c| <= 2^-19 |coords|^2 + 2^-23 c from the rounded translated
// coordinates, their differences and squares; 2^-23 (|alpha| + |beta|) from the
// rounded cutoff; taken 4x); the FP64 test of the FP64 path decides inside it
// per-target records (rounded from FP64) and the block partials of sum psi nu
// (perm non-null: record j is target perm[j], the cell list's order)
// (nb non-null: nb[j] = b_j - 2k beta_j in FP32, the target's term of the
// truncation test on the exponent; +inf for padding)
__global__ void k_prep_df(const double *__restrict__ psi, const double *__restrict__ y64,
                          const double *__restrict__ lnu, const double *__restrict__ nu, int64_t n,
                          int64_t n_alloc, int d, double eps, const int *__restrict__ perm,
                          DRec *__restrict__ trec, double *__restrict__ psinu_part,
                          int *__restrict__ flags, const double *__restrict__ beta,
                          float *__restrict__ nb) {
    __shared__ double sh[32];
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double k = kLog2e / (2.0 * eps);
    double contrib = 0.0;
    if (j < n_alloc) {
        float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, kExcl, 0.f};
        if (j < n) {
            const int64_t o = perm ? (int64_t)perm[j] : j;
            const double ps = psi[o];
            if (!isfinite(ps)) atomicOr(flags, kErrNonfinitePsi);
            const double b = ((ps - psi[0]) / eps + lnu[o]) * kLog2e;
            double yy = 0.0;
            for (int t = 0; t < d; ++t) {
                const double yt = y64[o * d + t];
                split_f(2.0 * k * yt, v[2 * t], v[2 * t + 1]);
                yy += yt * yt;
            }
            split_f(fmax(b - k * yy, -1.0e29), v[6], v[7]);
            contrib = ps * nu[o];
            if (nb) nb[j] = (float)(b - 2.0 * k * beta[o]);
        } else if (nb) {
            nb[j] = INFINITY;
        }
        trec[j] = make_drec(v);
    }
    const double s = block_sum_d(contrib, sh);
    if (threadIdx.x == 0) psinu_part[blockIdx.x] = s;
}

// ---- block data of the truncated passes (targets in the cell list's order)
// ball (centre of the bounding box, radius to its corner, rounded up) of each
// block of B consecutive rows of c64 [cnt][d]; radius -1: no member
__global__ void k_df_balls(const double *__restrict__ c64, int64_t cnt, int d, int B, int64_t nblocks,
                           float4 *__restrict__ ball) {
    const int64_t bi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (bi >= nblocks) return;
    const int64_t a = bi * B, e = min((bi + 1) * B, cnt);
    if (a >= e) {
        ball[bi] = make_float4(0.f, 0.f, 0.f, -1.f);
        return;
    }
    double lo[3] = {0.0, 0.0, 0.0}, hi[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < d; ++k) lo[k] = hi[k] = c64[a * d + k];
    for (int64_t q = a + 1; q < e; ++q)
        for (int k = 0; k < d; ++k) {
            lo[k] = fmin(lo[k], c64[q * d + k]);
            hi[k] = fmax(hi[k], c64[q * d + k]);
        }
    double c[3] = {0.0, 0.0, 0.0}, r2 = 0.0;
    for (int k = 0; k < d; ++k) {
        c[k] = 0.5 * (lo[k] + hi[k]);
        r2 += 0.25 * (hi[k] - lo[k]) * (hi[k] - lo[k]);
    }
    ball[bi] = make_float4((float)c[0], (float)c[1], (float)c[2], (float)(sqrt(r2) * (1.0 + 1e-6) + 1e-9));
}

// (min, max) of v over blocks of B consecutive entries (v[perm[s]] when perm is
// given), rounded outwards to FP32; no member: (+inf, -inf)
__global__ void k_df_ranges(const double *__restrict__ v, const int *__restrict__ perm, int64_t cnt, int B,
                            int64_t nblocks, float2 *__restrict__ out) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblocks) return;
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t s = b * B; s < min((b + 1) * B, cnt); ++s) {
        const double a = v[perm ? (int64_t)perm[s] : s];
        lo = fmin(lo, a);
        hi = fmax(hi, a);
    }
    float flo = (float)lo, fhi = (float)hi;
    if ((double)flo > lo) flo = nextafterf(flo, -INFINITY);
    if ((double)fhi < hi) fhi = nextafterf(fhi, INFINITY);
    out[b] = make_float2(flo, fhi);
}

// out[s] = v[perm[s]] (v[s] without perm) for s < n, +inf beyond, in FP64
// (out, nullable) and rounded to FP32 (outf, nullable: the value the FP32
// pair tests use)
__global__ void k_df_gather(const double *__restrict__ v, const int *__restrict__ perm, int64_t n,
                            int64_t n_alloc, double *__restrict__ out, float *__restrict__ outf) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_alloc) return;
    const double x = s < n ? v[perm ? (int64_t)perm[s] : s] : INFINITY;
    if (out) out[s] = x;
    if (outf) outf[s] = (float)x;
}

// A[q] = k |x'_q|^2 - 2k alpha_q in FP32, the point's term of the truncation
// test on the exponent (+inf for padding)
__global__ void k_df_A(const double *__restrict__ x64, const double *__restrict__ alpha, int64_t nq,
                       int64_t nq_pad, int d, double k, float *__restrict__ A) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq_pad) return;
    if (q >= nq) {
        A[q] = INFINITY;
        return;
    }
    double r2 = 0.0;
    for (int t = 0; t < d; ++t) r2 += x64[q * d + t] * x64[q * d + t];
    A[q] = (float)(k * r2 - 2.0 * k * alpha[q]);
}

// The truncation test of a pair from its exponent: the pair is kept when
// c(x_q, y_j) < alpha_q + beta_j, i.e. r_qj > nb_j + A_q (r_qj = b_j - 2k c_qj
// + k |x'_q|^2 in the log2 domain).  With the double-float head rh of r_qj and
// nb_j, A_q rounded to FP32, the sign of rh - nb_j - A_q decides wherever it
// exceeds 2^-20 of the magnitudes (the FP32 and double-float errors are below
// 2^-22 of them); inside that band the FP64 cost decides (keep_fp64, the FP64
// path's own expression), so the kept pairs are exactly the FP64 path's.
// 1: kept, 0: excluded, -1: the FP64 test decides.
__device__ __forceinline__ int exp_test(float rh, float nb, float A) {
    const float v = (rh - nb) - A;
    const float mg = 0x1p-20f * (fabsf(rh) + fabsf(nb) + fabsf(A)) + 0x1p-100f;
    return v > mg ? 1 : (v < -mg ? 0 : -1);
}
template <int D>
__device__ __forceinline__ bool keep_fp64(const double *x64, const double *y64, double a64, double b64) {
    // the FP64 passes' test, written the same way: d2 = |x - y|^2 < 2 a + 2 b
    double d2 = 0.0;
#pragma unroll
    for (int t = 0; t < D; ++t) {
        const double dd = x64[t] - y64[t];
        d2 = fma(dd, dd, d2);
    }
    return d2 < 2.0 * a64 + 2.0 * b64;
}

// static point records (x' head/tail; the shift is written by pass 1)
__global__ void k_static_df(const double *__restrict__ x64, int64_t nq, int64_t nq_pad, int d,
                            DRec *__restrict__ prec) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nq_pad) {
        float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, kExcl, 0.f};
        if (i < nq)
            for (int t = 0; t < d; ++t) split_f(x64[i * d + t], v[2 * t], v[2 * t + 1]);
        prec[i] = make_drec(v);
    }
}

// Pass 1: R_q = log2 sum_{j in I_q} 2^{r_qj} with an integral running shift M,
// u_q = log2 m_q - R_q into the point record, sum_q m_q R_q by block.  Lane l
// of a thread is point blockIdx.x * D_ROWS + l * D_THREADS + threadIdx.x.
template <int D, bool TRUNC>
// (truncated: at most 96 registers, five blocks per SM, measured faster than four)
__global__ void __launch_bounds__(D_THREADS, TRUNC ? 5 : 1)
    k_lse_df(DRec *__restrict__ prec, const double *__restrict__ x64, int64_t nq, int64_t nq_pad,
             const DRec *__restrict__ trec, const double *__restrict__ y64, int64_t n,
             const double *__restrict__ alpha, const double *__restrict__ beta,
             const double *__restrict__ lmass2, const double *__restrict__ mass,
             const double *__restrict__ psi, double eps, double *__restrict__ blockJ,
             double *__restrict__ lse_buf, EvalResult *__restrict__ res,
             const float4 *__restrict__ pball64, const float2 *__restrict__ pal64,
             const float4 *__restrict__ tball8, const float2 *__restrict__ tbe8,
             const float *__restrict__ nbs, const float *__restrict__ Aq) {
    __shared__ DRec sm[D_TS];   // the block's target tile
    __shared__ float snb[D_TS];   // truncated: the tile's nb_j (exp_test)
    __shared__ unsigned s_live[D_THREADS / 32];   // truncated: live sub-tiles of each warp
    __shared__ double sh[32];
    __shared__ unsigned long long s_cnt, s_empty;
    if (threadIdx.x == 0) s_cnt = s_empty = 0;
    // truncated: a thread takes two consecutive points, a warp 64 (one ball)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t q[2];
    q[0] = (int64_t)blockIdx.x * D_ROWS + (TRUNC ? 2 * threadIdx.x : threadIdx.x);   // < nq_pad
    q[1] = q[0] + (TRUNC ? 1 : D_THREADS);
    const DRec p0 = prec[q[0]], p1 = prec[q[1]];
    Op2 X[3];
    f2 unused_h, unused_t;
    load_ops(p0, p1, X, unused_h, unused_t);
    float Ap[2] = {0.f, 0.f};   // truncated: A_q of the two points (exp_test)
    double a64[2] = {0.0, 0.0};
    if (TRUNC)
        for (int l = 0; l < 2; ++l) {
            Ap[l] = Aq[q[l]];
            a64[l] = alpha[q[l]];
        }
    const int64_t n_rec = (n + D_TS - 1) / D_TS * D_TS;
    float M[2] = {-INFINITY, -INFINITY};
    double S[2] = {0.0, 0.0};
    unsigned long long npair = 0;
    // truncated: the warp's 64 points against each sub-tile of 8 targets (ball
    // classes, bit maps lv / bd): outside sub-tiles are skipped, inside ones
    // need no pair test; a tile no warp needs is not loaded
    const int64_t wblk = (int64_t)blockIdx.x * (D_ROWS / 64) + warp;
    const float4 wb = TRUNC ? pball64[wblk] : make_float4(0.f, 0.f, 0.f, -1.f);
    const float2 wa = TRUNC ? pal64[wblk] : make_float2(0.f, 0.f);
    if constexpr (!TRUNC) {
        for (int64_t t0 = 0; t0 < n_rec; t0 += D_TS) {
            __syncthreads();
            for (int i = threadIdx.x; i < D_TS; i += D_THREADS) sm[i] = trec[t0 + i];
            __syncthreads();
            f2 s = make_float2(0.f, 0.f), comp = s, cs = s;
            for (int u0 = 0; u0 < D_TS; u0 += D_SUB) {
                f2 rh[D_SUB], rt[D_SUB];
                float mx0 = -INFINITY, mx1 = -INFINITY;
    #pragma unroll
                for (int i = 0; i < D_SUB; ++i) {
                    const DRec &B = sm[u0 + i];
                    df_exponent2<D>(X, B, lo2(B.d), hi2(B.d), rh[i], rt[i]);
                    mx0 = fmaxf(mx0, rh[i].x);
                    mx1 = fmaxf(mx1, rh[i].y);
                }
                if (mx0 > M[0] || mx1 > M[1]) {   // raise a shift to ceil(max): exact rescaling
                    float f[2] = {1.f, 1.f};
                    const float mx[2] = {mx0, mx1};
                    for (int l = 0; l < 2; ++l) {
                        if (mx[l] > M[l] && mx[l] > -1.0e29f) {
                            const float mn = ceilf(mx[l]);
                            if (M[l] != -INFINITY) {
                                f[l] = pow2_int_f(M[l] - mn);
                                S[l] *= pow2_int_d(M[l] - mn);
                            }
                            M[l] = mn;
                        }
                    }
                    const f2 ff = make_float2(f[0], f[1]);
                    s = mul2(s, ff);
                    comp = mul2(comp, ff);
                    cs = mul2(cs, ff);
                }
                // a lane with no kept pair yet subtracts a huge shift: its terms are 0
                const f2 Me = make_float2(M[0] == -INFINITY ? 1.0e30f : M[0],
                                          M[1] == -INFINITY ? 1.0e30f : M[1]);
    #pragma unroll
                for (int i = 0; i < D_SUB; ++i) {
                    f2 ah, ae;
                    two_diff2(rh[i], Me, ah, ae);
                    const f2 e = make_float2(ex2_approx(ah.x), ex2_approx(ah.y));
                    kahan2(s, comp, e);
                    cs = fma2(e, add2(ae, rt[i]), cs);
                }
            }
            S[0] += ((double)s.x - (double)comp.x) + kLn2 * (double)cs.x;
            S[1] += ((double)s.y - (double)comp.y) + kLn2 * (double)cs.y;
        }
    } else {
        // the warp's 64 points against every sub-tile of 8 targets of each tile
        // (ball classes, bit maps lv / bd): outside sub-tiles are skipped, inside
        // ones need no pair test; a tile that no warp of the block needs is not
        // loaded
        for (int64_t t0 = 0; t0 < n_rec; t0 += D_TS) {
            int c = 0;
            if (lane < D_TS / D_SUB) {
                const int64_t sb = t0 / D_SUB + lane;
                c = tp_class(wb, tball8[sb], wa, tbe8[sb]);
            }
            const unsigned lv = __ballot_sync(0xffffffffu, c != 0);
            const unsigned bd = __ballot_sync(0xffffffffu, c == 2);
            __syncthreads();   // the previous tile's readers are done
            if (lane == 0) s_live[warp] = lv;
            __syncthreads();
            unsigned any = 0;
            for (int w = 0; w < D_THREADS / 32; ++w) any |= s_live[w];
            if (!any) continue;   // block-uniform
            for (int i = threadIdx.x; i < D_TS; i += D_THREADS) {
                sm[i] = trec[t0 + i];
                snb[i] = nbs[t0 + i];
            }
            __syncthreads();
            if (!lv) continue;   // warp-uniform: the next tile's first barrier waits for the others
            f2 s = make_float2(0.f, 0.f), comp = s, cs = s;
            for (unsigned mm = lv; mm; mm &= mm - 1) {
                const int sub = __ffs(mm) - 1;
                const bool test = (bd >> sub) & 1u;
                const int u0 = sub * D_SUB;
                f2 rh[D_SUB], rt[D_SUB];
                float mx0 = -INFINITY, mx1 = -INFINITY;
#pragma unroll
                for (int i = 0; i < D_SUB; ++i) {
                    const int64_t j = t0 + u0 + i;
                    const DRec &B = sm[u0 + i];
                    df_exponent2<D>(X, B, lo2(B.d), hi2(B.d), rh[i], rt[i]);
                    for (int l = 0; l < 2; ++l) {
                        bool k = j < n && q[l] < nq;
                        if (k && test) {
                            const int e = exp_test(l ? rh[i].y : rh[i].x, snb[u0 + i], Ap[l]);
                            k = e > 0 || (e < 0 && keep_fp64<D>(x64 + q[l] * D, y64 + j * D, a64[l], beta[j]));
                        }
                        if (k) {
                            ++npair;
                        } else if (l == 0) {
                            rh[i].x = kExcl;
                            rt[i].x = 0.f;
                        } else {
                            rh[i].y = kExcl;
                            rt[i].y = 0.f;
                        }
                    }
                    mx0 = fmaxf(mx0, rh[i].x);
                    mx1 = fmaxf(mx1, rh[i].y);
                }
                if (mx0 > M[0] || mx1 > M[1]) {   // raise a shift to ceil(max): exact rescaling
                    float f[2] = {1.f, 1.f};
                    const float mx[2] = {mx0, mx1};
                    for (int l = 0; l < 2; ++l) {
                        if (mx[l] > M[l] && mx[l] > -1.0e29f) {
                            const float mn = ceilf(mx[l]);
                            if (M[l] != -INFINITY) {
                                f[l] = pow2_int_f(M[l] - mn);
                                S[l] *= pow2_int_d(M[l] - mn);
                            }
                            M[l] = mn;
                        }
                    }
                    const f2 ff = make_float2(f[0], f[1]);
                    s = mul2(s, ff);
                    comp = mul2(comp, ff);
                    cs = mul2(cs, ff);
                }
                const f2 Me = make_float2(M[0] == -INFINITY ? 1.0e30f : M[0],
                                          M[1] == -INFINITY ? 1.0e30f : M[1]);
#pragma unroll
                for (int i = 0; i < D_SUB; ++i) {
                    f2 ah, ae;
                    two_diff2(rh[i], Me, ah, ae);
                    const f2 e = make_float2(ex2_approx(ah.x), ex2_approx(ah.y));
                    kahan2(s, comp, e);
                    cs = fma2(e, add2(ae, rt[i]), cs);
                }
            }
            S[0] += ((double)s.x - (double)comp.x) + kLn2 * (double)cs.x;
            S[1] += ((double)s.y - (double)comp.y) + kLn2 * (double)cs.y;
        }
    }
    double contrib = 0.0;
    int empties = 0;
    for (int l = 0; l < 2; ++l) {
        const int64_t qq = q[l];
        float uh = kExcl, ut = 0.f;
        if (qq < nq) {
            if (S[l] > 0.0) {
                const double R = (double)M[l] + log2(S[l]);
                lse_buf[qq] = R;
                if (mass[qq] > 0.0) {
                    contrib += mass[qq] * R;
                    split_f(lmass2[qq] - R, uh, ut);
                }
            } else {   // empty I_q: skipped by Algorithm 2
                lse_buf[qq] = -INFINITY;
                ++empties;
                // the finalisation adds psi_c m_q - m_q |x'_q|^2 / 2 for every point
                // (sum m_q, hx): cancel this point's share in the log2 sum it scales
                if (mass[qq] > 0.0) {
                    double r2 = 0.0;
                    for (int t = 0; t < D; ++t) r2 += x64[qq * D + t] * x64[qq * D + t];
                    contrib -= mass[qq] * (psi[0] - 0.5 * r2) / (eps * kLn2);
                }
            }
        }
        prec[qq].d = make_float4(uh, uh, ut, ut);
    }
    if (TRUNC && npair) atomicAdd(&s_cnt, npair);
    if (empties) atomicAdd(&s_empty, (unsigned long long)empties);
    const double sum = block_sum_d(contrib, sh);
    if (threadIdx.x == 0) {
        blockJ[blockIdx.x] = sum;
        if (s_cnt) atomicAdd(reinterpret_cast<unsigned long long *>(&res->pairs), s_cnt);
        if (s_empty) atomicAdd(reinterpret_cast<unsigned long long *>(&res->empty), s_empty);
    }
}

// Pass 2: per target, sum over one point chunk of 2^{r_qj + u_q} = m_q p_qj.
// Lane l of a thread is target blockIdx.x * D_ROWS + l * D_THREADS + threadIdx.x.
template <int D, bool TRUNC>
__global__ void __launch_bounds__(D_THREADS)
    k_grad_df(const DRec *__restrict__ trec, const double *__restrict__ y64, int64_t n,
              int64_t n_alloc, const DRec *__restrict__ prec, const double *__restrict__ x64,
              int64_t nq, int64_t nq_pad, int64_t chunk, const double *__restrict__ alpha,
              const double *__restrict__ beta, double *__restrict__ part2, const int *__restrict__ perm,
              const float4 *__restrict__ tball64, const float2 *__restrict__ tbe64,
              const float4 *__restrict__ pball8, const float2 *__restrict__ pal8,
              const float *__restrict__ Aq, const float *__restrict__ nbs) {
    __shared__ DRec sm[D_TS];   // the block's point tile
    __shared__ float sA[D_TS];   // truncated: the tile's A_q (exp_test)
    __shared__ unsigned s_live[D_THREADS / 32];   // truncated: live sub-tiles of each warp
    // truncated: a thread takes two consecutive (sorted) targets, a warp 64 (one ball)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t j[2];
    j[0] = (int64_t)blockIdx.x * D_ROWS + (TRUNC ? 2 * threadIdx.x : threadIdx.x);   // < n_alloc
    j[1] = j[0] + (TRUNC ? 1 : D_THREADS);
    Op2 W[3];
    f2 Ch, Ct;
    load_ops(trec[j[0]], trec[j[1]], W, Ch, Ct);
    float nbl[2] = {0.f, 0.f};   // truncated: nb_j of the two targets (exp_test)
    if (TRUNC)
        for (int l = 0; l < 2; ++l) nbl[l] = nbs[j[l]];
    const int64_t p_begin = (int64_t)blockIdx.y * chunk;
    const int64_t p_end = min(nq_pad, p_begin + chunk);
    double acc0 = 0.0, acc1 = 0.0;
    // truncated: the warp's 64 targets against each sub-tile of 8 points (ball
    // classes, bit maps lv / bd): outside sub-tiles are skipped, inside ones need
    // no pair test; a tile no warp needs is not loaded
    const int64_t wblk = (int64_t)blockIdx.x * (D_ROWS / 64) + warp;
    const float4 wb = TRUNC ? tball64[wblk] : make_float4(0.f, 0.f, 0.f, -1.f);
    const float2 wr = TRUNC ? tbe64[wblk] : make_float2(0.f, 0.f);
    if constexpr (!TRUNC) {
        for (int64_t p0 = p_begin; p0 < p_end; p0 += D_TS) {
            __syncthreads();
            for (int i = threadIdx.x; i < D_TS; i += D_THREADS) sm[i] = prec[p0 + i];
            __syncthreads();
            f2 s = make_float2(0.f, 0.f), comp = s, cs = s;
    #pragma unroll 2
            for (int i = 0; i < D_TS; ++i) {
                const DRec &B = sm[i];
                f2 rh, rt;
                df_exponent2<D>(W, B, Ch, Ct, rh, rt);
                f2 th, te;
                two_sum2(rh, lo2(B.d), th, te);
                const f2 e = make_float2(ex2_approx(th.x), ex2_approx(th.y));
                kahan2(s, comp, e);
                cs = fma2(e, add2(add2(te, rt), hi2(B.d)), cs);
            }
            acc0 += ((double)s.x - (double)comp.x) + kLn2 * (double)cs.x;
            acc1 += ((double)s.y - (double)comp.y) + kLn2 * (double)cs.y;
        }
    } else {
        // the warp's 64 targets against every sub-tile of 8 points of each tile of
        // the chunk (ball classes, bit maps lv / bd): outside sub-tiles are
        // skipped, inside ones need no pair test; a tile that no warp of the
        // block needs is not loaded
        for (int64_t p0 = p_begin; p0 < p_end; p0 += D_TS) {
            int c = 0;
            if (lane < D_TS / D_SUB) {
                const int64_t sb = p0 / D_SUB + lane;
                c = tp_class(wb, pball8[sb], wr, pal8[sb]);
            }
            const unsigned lv = __ballot_sync(0xffffffffu, c != 0);
            const unsigned bd = __ballot_sync(0xffffffffu, c == 2);
            __syncthreads();   // the previous tile's readers are done
            if (lane == 0) s_live[warp] = lv;
            __syncthreads();
            unsigned any = 0;
            for (int w = 0; w < D_THREADS / 32; ++w) any |= s_live[w];
            if (!any) continue;   // block-uniform
            for (int i = threadIdx.x; i < D_TS; i += D_THREADS) {
                sm[i] = prec[p0 + i];
                sA[i] = Aq[p0 + i];
            }
            __syncthreads();
            if (!lv) continue;   // warp-uniform: the next tile's first barrier waits for the others
            f2 s = make_float2(0.f, 0.f), comp = s, cs = s;
            for (unsigned mm = lv; mm; mm &= mm - 1) {
                const int sub = __ffs(mm) - 1;
                const bool test = (bd >> sub) & 1u;
                const int u0 = sub * D_SUB;
#pragma unroll 2
                for (int i = u0; i < u0 + D_SUB; ++i) {
                    const int64_t qq = p0 + i;
                    const DRec &B = sm[i];
                    f2 rh, rt;
                    df_exponent2<D>(W, B, Ch, Ct, rh, rt);
                    f2 th, te;
                    two_sum2(rh, lo2(B.d), th, te);
                    f2 e = make_float2(ex2_approx(th.x), ex2_approx(th.y));
                    if (test) {
                        const float Ai = sA[i];
                        for (int l = 0; l < 2; ++l) {
                            bool k = qq < nq && j[l] < n;
                            if (k) {
                                const int c2 = exp_test(l ? rh.y : rh.x, nbl[l], Ai);
                                k = c2 > 0 ||
                                    (c2 < 0 && keep_fp64<D>(x64 + qq * D, y64 + j[l] * D, alpha[qq], beta[j[l]]));
                            }
                            if (!k) {
                                if (l) e.y = 0.f;
                                else e.x = 0.f;
                            }
                        }
                    }
                    kahan2(s, comp, e);
                    cs = fma2(e, add2(add2(te, rt), hi2(B.d)), cs);
                }
            }
            acc0 += ((double)s.x - (double)comp.x) + kLn2 * (double)cs.x;
            acc1 += ((double)s.y - (double)comp.y) + kLn2 * (double)cs.y;
        }
    }
    // truncated: j is a sorted index, the partial goes to the caller's target
    const int64_t o0 = (TRUNC && j[0] < n) ? (int64_t)perm[j[0]] : j[0];
    const int64_t o1 = (TRUNC && j[1] < n) ? (int64_t)perm[j[1]] : j[1];
    part2[(int64_t)blockIdx.y * n_alloc + o0] = acc0;
    part2[(int64_t)blockIdx.y * n_alloc + o1] = acc1;
}

int occupancy_df(const void *f) {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, D_THREADS, 0);
    return std::max(b, 1);
}

template <int D>
cudaError_t compensated_d(rsot_problem *p, const double *psi, double eps, bool trunc,
                          double *grad) {
    cudaStream_t st = p->stream;
    cudaError_t e;
    // point chunks of whole tiles for pass 2: enough blocks for four waves
    const int64_t tblocks = p->n_pad / D_ROWS, tiles = p->nq_pad / D_TS;
    const void *f2p = trunc ? (const void *)k_grad_df<D, true> : (const void *)k_grad_df<D, false>;
    const int64_t want = 4LL * p->num_sms * occupancy_df(f2p);
    int64_t s2 = std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(tiles, 64),
                                                        (want + tblocks - 1) / tblocks));
    const int64_t chunk = (tiles + s2 - 1) / s2 * D_TS;
    s2 = (p->nq_pad + chunk - 1) / chunk;
    if (!p->df_prec) {
        if ((e = cudaMalloc(&p->df_prec, (size_t)p->nq_pad * sizeof(DRec)))) return e;
        if ((e = cudaMalloc(&p->df_trec, (size_t)p->n_pad * sizeof(DRec)))) return e;
        const int64_t m = std::max(p->nq_pad, p->n_pad);
        k_static_df<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(p->x64, p->nq, p->nq_pad, p->d,
                                                                reinterpret_cast<DRec *>(p->df_prec));
        if ((e = cudaGetLastError())) return e;
    }
    if (p->df_s2 < s2) {
        cudaFree(p->df_part2);
        p->df_part2 = nullptr;
        p->df_s2 = 0;
        if ((e = cudaMalloc(&p->df_part2, (size_t)s2 * p->n_pad * sizeof(double)))) return e;
        p->df_s2 = (int)s2;
    }
    DRec *prec = reinterpret_cast<DRec *>(p->df_prec);
    DRec *trec = reinterpret_cast<DRec *>(p->df_trec);
    const double *alpha = trunc ? p->alpha : nullptr, *beta = trunc ? p->beta : nullptr;
    // truncated: targets in the cell list's order, blocks classified by balls
    SortedTargets T;
    const double *y64 = p->y64;
    if (trunc) {
        if ((e = trunc_block_setup(p, eps, &T))) return e;
        y64 = T.y64;
        beta = p->df_beta_s;
    }
    trace_begin(p, "prep_df");
    k_prep_df<<<p->nblk_prep, 256, 0, st>>>(psi, p->y64, p->lnu, p->nu, p->n, p->n_pad, p->d, eps,
                                           trunc ? T.perm : nullptr, trec, p->psinu, p->flags,
                                           p->beta, trunc ? p->df_beta_sf : nullptr);
    trace_end(p);
    const unsigned nb1 = (unsigned)(p->nq_pad / D_ROWS);
    trace_begin(p, "lse_df");
    if (trunc)
        k_lse_df<D, true><<<nb1, D_THREADS, 0, st>>>(prec, p->x64, p->nq, p->nq_pad, trec, y64, p->n, alpha,
                                                     beta, p->lmass2, p->mass, psi, eps, p->blockJ,
                                                     p->lse_buf, p->res_dev, p->df_pb64, p->df_pa64, T.ball8,
                                                     p->df_tbe8, p->df_beta_sf, p->df_alpha_f);
    else
        k_lse_df<D, false><<<nb1, D_THREADS, 0, st>>>(prec, p->x64, p->nq, p->nq_pad, trec, y64, p->n,
                                                      alpha, beta, p->lmass2, p->mass, psi, eps,
                                                      p->blockJ, p->lse_buf, p->res_dev, nullptr, nullptr,
                                                      nullptr, nullptr, nullptr, nullptr);
    trace_end(p);
    dim3 g2((unsigned)tblocks, (unsigned)s2);
    trace_begin(p, "grad_df");
    if (trunc)
        k_grad_df<D, true><<<g2, D_THREADS, 0, st>>>(trec, y64, p->n, p->n_pad, prec, p->x64, p->nq,
                                                     p->nq_pad, chunk, alpha, beta, p->df_part2, T.perm,
                                                     T.ball64, p->df_tbe64, p->df_pb8, p->df_pa8,
                                                     p->df_alpha_f, p->df_beta_sf);
    else
        k_grad_df<D, false><<<g2, D_THREADS, 0, st>>>(trec, y64, p->n, p->n_pad, prec, p->x64, p->nq,
                                                      p->nq_pad, chunk, alpha, beta, p->df_part2, nullptr,
                                                      nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    trace_end(p);
    if ((e = cudaGetLastError())) return e;
    return launch_finalize_log2(p, psi, eps, p->df_part2, (int)s2, (int)nb1, grad);
}

}  // namespace

// Block data of the truncated block-skip passes (compensated and FP32): the
// cell list's target order, balls of 64 / 8 caller-order points (once), beta in
// sorted order, A_q, and the alpha / beta ranges of the blocks (per evaluation,
// from p->alpha / p->beta).
cudaError_t trunc_block_setup(rsot_problem *p, double eps, SortedTargets *T) {
    cudaError_t e;
    cudaStream_t st = p->stream;
    if ((e = trunc_sorted_targets(p, T))) return e;
    const int d = p->d;
    auto nb = [](int64_t m) { return (unsigned)((m + 255) / 256); };
    if (!p->df_beta_s) {
        if ((e = cudaMalloc(&p->df_beta_s, (size_t)p->n_pad * sizeof(double)))) return e;
        if ((e = cudaMalloc(&p->df_beta_sf, (size_t)p->n_pad * sizeof(float)))) return e;   // nb_j
        if ((e = cudaMalloc(&p->df_alpha_f, (size_t)p->nq_pad * sizeof(float)))) return e;  // A_q
        if ((e = cudaMalloc(&p->df_pb64, (size_t)(p->nq_pad / 64) * sizeof(float4)))) return e;
        if ((e = cudaMalloc(&p->df_pb8, (size_t)(p->nq_pad / 8) * sizeof(float4)))) return e;
        if ((e = cudaMalloc(&p->df_pa64, (size_t)(p->nq_pad / 64) * sizeof(float2)))) return e;
        if ((e = cudaMalloc(&p->df_pa8, (size_t)(p->nq_pad / 8) * sizeof(float2)))) return e;
        if ((e = cudaMalloc(&p->df_tbe64, (size_t)(p->n_pad / 64) * sizeof(float2)))) return e;
        if ((e = cudaMalloc(&p->df_tbe8, (size_t)(p->n_pad / 8) * sizeof(float2)))) return e;
        k_df_balls<<<nb(p->nq_pad / 64), 256, 0, st>>>(p->x64, p->nq, d, 64, p->nq_pad / 64, p->df_pb64);
        k_df_balls<<<nb(p->nq_pad / 8), 256, 0, st>>>(p->x64, p->nq, d, 8, p->nq_pad / 8, p->df_pb8);
    }
    k_df_gather<<<nb(p->n_pad), 256, 0, st>>>(p->beta, T->perm, p->n, p->n_pad, p->df_beta_s, nullptr);
    k_df_A<<<nb(p->nq_pad), 256, 0, st>>>(p->x64, p->alpha, p->nq, p->nq_pad, d, kLog2e / (2.0 * eps),
                                          p->df_alpha_f);
    k_df_ranges<<<nb(p->nq_pad / 64), 256, 0, st>>>(p->alpha, nullptr, p->nq, 64, p->nq_pad / 64, p->df_pa64);
    k_df_ranges<<<nb(p->nq_pad / 8), 256, 0, st>>>(p->alpha, nullptr, p->nq, 8, p->nq_pad / 8, p->df_pa8);
    k_df_ranges<<<nb(p->n_pad / 64), 256, 0, st>>>(p->beta, T->perm, p->n, 64, p->n_pad / 64, p->df_tbe64);
    k_df_ranges<<<nb(p->n_pad / 8), 256, 0, st>>>(p->beta, T->perm, p->n, 8, p->n_pad / 8, p->df_tbe8);
    return cudaGetLastError();
}

// dense (Eq. discretized_functional / discretized_gradient), or the truncated
// sums over c(x_q, y_j) < alpha_q + beta_j (p->alpha, p->beta)
cudaError_t launch_compensated(rsot_problem *p, const double *psi, double eps, bool trunc,
                               double *grad) {
    return p->d == 3 ? compensated_d<3>(p, psi, eps, trunc, grad)
                     : compensated_d<2>(p, psi, eps, trunc, grad);
}

void compensated_free(rsot_problem *p) {
    cudaFree(p->df_prec);
    cudaFree(p->df_trec);
    cudaFree(p->df_part2);
    p->df_prec = p->df_trec = nullptr;
    p->df_part2 = nullptr;
    p->df_s2 = 0;
    void *blk[] = {p->df_beta_s, p->df_pb64, p->df_pb8, p->df_pa64, p->df_pa8,
                   p->df_tbe64, p->df_tbe8, p->df_beta_sf, p->df_alpha_f};
    for (void *q : blk) cudaFree(q);
    p->df_beta_s = nullptr;
    p->df_beta_sf = p->df_alpha_f = nullptr;
    p->df_pb64 = p->df_pb8 = nullptr;
    p->df_pa64 = p->df_pa8 = p->df_tbe64 = p->df_tbe8 = nullptr;
}

}  // namespace rsot
