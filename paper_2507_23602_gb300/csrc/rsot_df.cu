// Compensated evaluation of Algorithm 2: the passes of the mixed path with the
// exponent of every pair carried as a double-float (an unevaluated sum of two
// FP32 numbers, ~44 significant bits) instead of one FP32 number.
//
// Log2 domain and translated coordinates as the mixed passes (rsot_dense.cu):
// r_qj = c_j + x'_q.w_j with w_j = 2k y'_j, c_j = b_j - k|y'_j|^2, k =
// log2(e)/(2 eps), every operand rounded from its FP64 value to head + tail.
// Each product x.w is formed exactly as ph + pe (pe = fma(x, w, -ph)) plus the
// cross terms x_h w_t + x_t w_h; the heads are summed with TwoSum, so r comes
// with an absolute error of a few 2^-44 |c| instead of 2^-24 |c|.  The shift by
// the running maximum (pass 1) or by u_q = log2 m_q - R_q (pass 2) is also a
// TwoSum, so 2^(r - M) = ex2.approx(a_h) (1 + a_t ln2 + O(a_t^2)) with the tail
// a_t folded in as a separately accumulated first-order correction.  Sums are
// Kahan-compensated in FP32 within a tile and FP64 across tiles.
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
// Truncated form (Algorithm 2 with I_q = {j : c(x_q, y_j) < C}): membership is
// decided in FP32 where |c_32 - C| exceeds a margin that bounds the FP32
// distance error, else by the FP64 test of the FP64 path (same expression,
// same translated coordinates), so both paths keep the same pairs.
#include <math.h>

#include <algorithm>

#include "rsot_internal.cuh"

namespace rsot {

cudaError_t launch_finalize_log2(rsot_problem *p, const double *psi, double eps,
                                 const double *part2, int s2, int nbj, double *grad);

namespace {

constexpr int D_THREADS = 128;   // one point (pass 1) / one target (pass 2) per thread
constexpr int D_TS = 256;        // records per shared-memory tile (divides n_pad and nq_pad)
constexpr int D_SUB = 16;        // targets per max sub-tile (pass 1)
constexpr float kExcl = -1.0e30f;

struct __align__(16) DRec {      // head/tail pairs (v0h, v0t, v1h, v1t), (v2h, v2t, sh, st)
    float4 a, b;
};

// s + e = a + b exactly (Knuth's TwoSum; no ordering requirement)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void split_f(double v, float &h, float &t) {
    h = (float)v;
    t = (float)(v - (double)h);
}

// one coordinate's contribution x w = ph + (pe + x_h w_t + x_t w_h)
__device__ __forceinline__ void df_term(float xh, float xt, float wh, float wt, float &s,
                                        float &lo) {
    const float ph = xh * wh;
    const float pe = fmaf(xh, wh, -ph);
    lo += fmaf(xh, wt, fmaf(xt, wh, pe));
    float sn, se;
    two_sum(s, ph, sn, se);
    s = sn;
    lo += se;
}

// r = c + sum_t x_t w_t as (rh, rt); x from a point record, (w, c) from a
// target record
template <int D>
__device__ __forceinline__ void df_exponent(const DRec &x, const DRec &t, float &rh, float &rt) {
    float s = t.b.z, lo = t.b.w;
    df_term(x.a.x, x.a.y, t.a.x, t.a.y, s, lo);
    df_term(x.a.z, x.a.w, t.a.z, t.a.w, s, lo);
    if (D == 3) df_term(x.b.x, x.b.y, t.b.x, t.b.y, s, lo);
    rh = s + lo;                 // |lo| << |s|: Fast2Sum renormalisation
    rt = lo - (rh - s);
}

__device__ __forceinline__ void kahan(float &sum, float &comp, float v) {
    const float y = v - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

// FP32 distance test c(x, y) < C with the margin; the FP64 test of the FP64
// path decides pairs inside the margin
template <int D>
__device__ __forceinline__ bool keep_pair(const float *xf, const float *yf, float C, float margin,
                                          const double *x64, const double *y64, double C64) {
    float c2 = 0.f;
#pragma unroll
    for (int t = 0; t < D; ++t) {
        const float dd = xf[t] - yf[t];
        c2 = fmaf(dd, dd, c2);
    }
    const float c32 = 0.5f * c2;
    if (fabsf(c32 - C) > margin) return c32 < C;
    double c = 0.0;
#pragma unroll
    for (int t = 0; t < D; ++t) {
        const double dd = x64[t] - y64[t];
        c += dd * dd;
    }
    c *= 0.5;
    return c < C64;
}

// per-target records (rounded from FP64) and the block partials of sum psi nu
__global__ void k_prep_df(const double *__restrict__ psi, const double *__restrict__ y64,
                          const double *__restrict__ lnu, const double *__restrict__ nu, int64_t n,
                          int64_t n_alloc, int d, double eps, DRec *__restrict__ trec,
                          double *__restrict__ psinu_part, int *__restrict__ flags) {
    __shared__ double sh[32];
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double k = kLog2e / (2.0 * eps);
    double contrib = 0.0;
    if (j < n_alloc) {
        float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, kExcl, 0.f};
        if (j < n) {
            const double ps = psi[j];
            if (!isfinite(ps)) atomicOr(flags, kErrNonfinitePsi);
            const double b = ((ps - psi[0]) / eps + lnu[j]) * kLog2e;
            double yy = 0.0;
            for (int t = 0; t < d; ++t) {
                const double yt = y64[j * d + t];
                split_f(2.0 * k * yt, v[2 * t], v[2 * t + 1]);
                yy += yt * yt;
            }
            split_f(fmax(b - k * yy, -1.0e29), v[6], v[7]);
            contrib = ps * nu[j];
        }
        DRec r;
        r.a = make_float4(v[0], v[1], v[2], v[3]);
        r.b = make_float4(v[4], v[5], v[6], v[7]);
        trec[j] = r;
    }
    const double s = block_sum_d(contrib, sh);
    if (threadIdx.x == 0) psinu_part[blockIdx.x] = s;
}

// static point records (x' head/tail; the shift is written by pass 1) and
// FP32 target coordinates [3][n_alloc] for the truncation test
__global__ void k_static_df(const double *__restrict__ x64, int64_t nq, int64_t nq_pad,
                            const double *__restrict__ y64, int64_t n, int64_t n_alloc, int d,
                            DRec *__restrict__ prec, float *__restrict__ ys) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nq_pad) {
        float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (i < nq)
            for (int t = 0; t < d; ++t) split_f(x64[i * d + t], v[2 * t], v[2 * t + 1]);
        DRec r;
        r.a = make_float4(v[0], v[1], v[2], v[3]);
        r.b = make_float4(v[4], v[5], kExcl, 0.f);
        prec[i] = r;
    }
    if (i < n_alloc)
        for (int t = 0; t < 3; ++t)
            ys[t * n_alloc + i] = (i < n && t < d) ? (float)y64[i * d + t] : 1.0e30f;
}

// Pass 1: R_q = log2 sum_{j in I_q} 2^{r_qj} with an integral running shift M,
// u_q = log2 m_q - R_q into the point record, sum_q m_q R_q by block.
template <int D, bool TRUNC>
__global__ void __launch_bounds__(D_THREADS)
    k_lse_df(DRec *__restrict__ prec, const float *__restrict__ xs, const double *__restrict__ x64,
             int64_t nq, int64_t nq_pad, const DRec *__restrict__ trec,
             const float *__restrict__ ys, const double *__restrict__ y64, int64_t n,
             int64_t n_alloc, float C, float margin, double C64,
             const double *__restrict__ lmass2, const double *__restrict__ mass,
             const double *__restrict__ psi, double eps, double *__restrict__ blockJ,
             double *__restrict__ lse_buf, EvalResult *__restrict__ res) {
    __shared__ DRec sm[D_TS];
    __shared__ float sy[TRUNC ? 3 : 1][D_TS];
    __shared__ double sh[32];
    __shared__ unsigned long long s_cnt, s_empty;
    if (threadIdx.x == 0) s_cnt = s_empty = 0;
    const int64_t q = (int64_t)blockIdx.x * D_THREADS + threadIdx.x;   // < nq_pad
    const DRec pr = prec[q];
    float xf[3] = {0.f, 0.f, 0.f};
    if (TRUNC)
        for (int t = 0; t < D; ++t) xf[t] = xs[t * nq_pad + q];
    const int64_t qx = q < nq ? q : 0;   // FP64 coordinates for the rare exact test
    const int64_t n_rec = (n + D_TS - 1) / D_TS * D_TS;
    float M = -INFINITY;
    double S = 0.0;
    unsigned long long npair = 0;
    for (int64_t t0 = 0; t0 < n_rec; t0 += D_TS) {
        __syncthreads();
        for (int i = threadIdx.x; i < D_TS; i += D_THREADS) {
            sm[i] = trec[t0 + i];
            if (TRUNC)
                for (int t = 0; t < 3; ++t) sy[t][i] = ys[t * n_alloc + t0 + i];
        }
        __syncthreads();
        float s = 0.f, comp = 0.f, cs = 0.f;
        for (int u0 = 0; u0 < D_TS; u0 += D_SUB) {
            float rh[D_SUB], rt[D_SUB];
            float mx = -INFINITY;
#pragma unroll
            for (int i = 0; i < D_SUB; ++i) {
                df_exponent<D>(pr, sm[u0 + i], rh[i], rt[i]);
                if (TRUNC) {
                    const float yf[3] = {sy[0][u0 + i], sy[1][u0 + i], sy[2][u0 + i]};
                    const int64_t j = t0 + u0 + i;
                    const bool k = j < n && q < nq &&
                                   keep_pair<D>(xf, yf, C, margin, x64 + qx * D, y64 + j * D, C64);
                    if (k) {
                        ++npair;
                    } else {
                        rh[i] = kExcl;
                        rt[i] = 0.f;
                    }
                }
                mx = fmaxf(mx, rh[i]);
            }
            if (mx > M && mx > -1.0e29f) {   // raise the shift to ceil(max): exact rescaling
                const float mn = ceilf(mx);
                if (M != -INFINITY) {
                    const float f = pow2_int_f(M - mn);
                    s *= f;
                    comp *= f;
                    cs *= f;
                    S *= pow2_int_d(M - mn);
                }
                M = mn;
            }
            if (M == -INFINITY) continue;    // no pair kept so far
#pragma unroll
            for (int i = 0; i < D_SUB; ++i) {
                float ah, ae;
                two_sum(rh[i], -M, ah, ae);
                const float e = ex2_approx(ah);
                kahan(s, comp, e);
                cs = fmaf(e, ae + rt[i], cs);
            }
        }
        S += ((double)s - (double)comp) + kLn2 * (double)cs;
    }
    double contrib = 0.0;
    float uh = kExcl, ut = 0.f;
    if (q < nq) {
        if (S > 0.0) {
            const double R = (double)M + log2(S);
            lse_buf[q] = R;
            if (mass[q] > 0.0) {
                contrib = mass[q] * R;
                split_f(lmass2[q] - R, uh, ut);
            }
        } else {   // empty I_q: skipped by Algorithm 2
            lse_buf[q] = -INFINITY;
            atomicAdd(&s_empty, 1ull);
            // the finalisation adds psi_c m_q - m_q |x'_q|^2 / 2 for every point
            // (sum m_q, hx): cancel this point's share in the log2 sum it scales
            if (mass[q] > 0.0) {
                double r2 = 0.0;
                for (int t = 0; t < D; ++t) r2 += x64[q * D + t] * x64[q * D + t];
                contrib = -mass[q] * (psi[0] - 0.5 * r2) / (eps * kLn2);
            }
        }
        if (TRUNC) atomicAdd(&s_cnt, npair);
    }
    prec[q].b = make_float4(pr.b.x, pr.b.y, uh, ut);
    const double sum = block_sum_d(contrib, sh);
    if (threadIdx.x == 0) {
        blockJ[blockIdx.x] = sum;
        if (s_cnt) atomicAdd(reinterpret_cast<unsigned long long *>(&res->pairs), s_cnt);
        if (s_empty) atomicAdd(reinterpret_cast<unsigned long long *>(&res->empty), s_empty);
    }
}

// Pass 2: per target, sum over one point chunk of 2^{r_qj + u_q} = m_q p_qj.
template <int D, bool TRUNC>
__global__ void __launch_bounds__(D_THREADS)
    k_grad_df(const DRec *__restrict__ trec, const float *__restrict__ ys,
              const double *__restrict__ y64, int64_t n, int64_t n_alloc,
              const DRec *__restrict__ prec, const float *__restrict__ xs,
              const double *__restrict__ x64, int64_t nq, int64_t nq_pad, int64_t chunk, float C,
              float margin, double C64, double *__restrict__ part2) {
    __shared__ DRec sm[D_TS];
    __shared__ float sx[TRUNC ? 3 : 1][D_TS];
    const int64_t j = (int64_t)blockIdx.x * D_THREADS + threadIdx.x;   // < n_alloc
    const DRec tr = trec[j];
    float yf[3] = {0.f, 0.f, 0.f};
    if (TRUNC)
        for (int t = 0; t < D; ++t) yf[t] = ys[t * n_alloc + j];
    const int64_t jy = j < n ? j : 0;
    const int64_t p_begin = (int64_t)blockIdx.y * chunk;
    const int64_t p_end = min(nq_pad, p_begin + chunk);
    double acc = 0.0;
    for (int64_t p0 = p_begin; p0 < p_end; p0 += D_TS) {
        __syncthreads();
        for (int i = threadIdx.x; i < D_TS; i += D_THREADS) {
            sm[i] = prec[p0 + i];
            if (TRUNC)
                for (int t = 0; t < 3; ++t) sx[t][i] = t < D ? xs[t * nq_pad + p0 + i] : 0.f;
        }
        __syncthreads();
        float s = 0.f, comp = 0.f, cs = 0.f;
#pragma unroll 4
        for (int i = 0; i < D_TS; ++i) {
            float rh, rt;
            df_exponent<D>(sm[i], tr, rh, rt);
            float th, te;
            two_sum(rh, sm[i].b.z, th, te);
            float e = ex2_approx(th);
            if (TRUNC) {
                const float xf[3] = {sx[0][i], sx[1][i], sx[2][i]};
                const int64_t qq = p0 + i;
                const bool k = qq < nq && j < n &&
                               keep_pair<D>(xf, yf, C, margin, x64 + qq * D, y64 + jy * D, C64);
                if (!k) e = 0.f;
            }
            kahan(s, comp, e);
            cs = fmaf(e, te + rt + sm[i].b.w, cs);
        }
        acc += ((double)s - (double)comp) + kLn2 * (double)cs;
    }
    part2[(int64_t)blockIdx.y * n_alloc + j] = acc;
}

template <int D>
cudaError_t compensated_d(rsot_problem *p, const double *psi, double eps, double cutoff,
                          double *grad) {
    cudaStream_t st = p->stream;
    cudaError_t e;
    if (!p->df_prec) {
        if ((e = cudaMalloc(&p->df_prec, (size_t)p->nq_pad * sizeof(DRec)))) return e;
        if ((e = cudaMalloc(&p->df_trec, (size_t)p->n_pad * sizeof(DRec)))) return e;
        if ((e = cudaMalloc(&p->df_ys, (size_t)3 * p->n_pad * sizeof(float)))) return e;
        const int64_t m = std::max(p->nq_pad, p->n_pad);
        k_static_df<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(
            p->x64, p->nq, p->nq_pad, p->y64, p->n, p->n_pad, p->d,
            reinterpret_cast<DRec *>(p->df_prec), p->df_ys);
        if ((e = cudaGetLastError())) return e;
    }
    DRec *prec = reinterpret_cast<DRec *>(p->df_prec);
    DRec *trec = reinterpret_cast<DRec *>(p->df_trec);
    const bool trunc = cutoff < INFINITY;
    // |c_32 - c| <= 2^-19 max|coord|^2 + 2^-23 c (FP32 rounding of the translated
    // coordinates, their differences and squares); the margin is 4x that
    const float C = trunc ? (float)cutoff : 0.f;
    const float margin = trunc ? (float)std::ldexp(p->diam2 + cutoff, -17) : 0.f;
    trace_begin(p, "prep_df");
    k_prep_df<<<p->nblk_prep, 256, 0, st>>>(psi, p->y64, p->lnu, p->nu, p->n, p->n_pad, p->d, eps,
                                           trec, p->psinu, p->flags);
    trace_end(p);
    const unsigned nb1 = (unsigned)(p->nq_pad / D_THREADS);
    trace_begin(p, "lse_df");
    if (trunc)
        k_lse_df<D, true><<<nb1, D_THREADS, 0, st>>>(prec, p->xs, p->x64, p->nq, p->nq_pad, trec,
                                                     p->df_ys, p->y64, p->n, p->n_pad, C, margin,
                                                     cutoff, p->lmass2, p->mass, psi, eps,
                                                     p->blockJ, p->lse_buf, p->res_dev);
    else
        k_lse_df<D, false><<<nb1, D_THREADS, 0, st>>>(prec, p->xs, p->x64, p->nq, p->nq_pad, trec,
                                                      p->df_ys, p->y64, p->n, p->n_pad, C, margin,
                                                      cutoff, p->lmass2, p->mass, psi, eps,
                                                      p->blockJ, p->lse_buf, p->res_dev);
    trace_end(p);
    // point chunks of whole tiles, at most s2_64 of them (the FP64 partials buffer)
    const int64_t tiles = p->nq_pad / D_TS;
    const int64_t chunk = (tiles + p->s2_64 - 1) / p->s2_64 * D_TS;
    const int s2 = (int)((p->nq_pad + chunk - 1) / chunk);
    dim3 g2((unsigned)(p->n_pad / D_THREADS), (unsigned)s2);
    trace_begin(p, "grad_df");
    if (trunc)
        k_grad_df<D, true><<<g2, D_THREADS, 0, st>>>(trec, p->df_ys, p->y64, p->n, p->n_pad, prec,
                                                     p->xs, p->x64, p->nq, p->nq_pad, chunk, C,
                                                     margin, cutoff, p->part2_64);
    else
        k_grad_df<D, false><<<g2, D_THREADS, 0, st>>>(trec, p->df_ys, p->y64, p->n, p->n_pad, prec,
                                                      p->xs, p->x64, p->nq, p->nq_pad, chunk, C,
                                                      margin, cutoff, p->part2_64);
    trace_end(p);
    if ((e = cudaGetLastError())) return e;
    return launch_finalize_log2(p, psi, eps, p->part2_64, s2, (int)nb1, grad);
}

}  // namespace

// cutoff = +inf: dense (Eq. discretized_functional / discretized_gradient);
// else the truncated sums over c(x_q, y_j) < cutoff.
cudaError_t launch_compensated(rsot_problem *p, const double *psi, double eps, double cutoff,
                               double *grad) {
    return p->d == 3 ? compensated_d<3>(p, psi, eps, cutoff, grad)
                     : compensated_d<2>(p, psi, eps, cutoff, grad);
}

void compensated_free(rsot_problem *p) {
    cudaFree(p->df_prec);
    cudaFree(p->df_trec);
    cudaFree(p->df_ys);
    p->df_prec = p->df_trec = nullptr;
    p->df_ys = nullptr;
}

}  // namespace rsot
