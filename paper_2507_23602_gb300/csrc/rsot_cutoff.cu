// Truncation cutoffs per pair: I_q = { j : c(x_q, y_j) < alpha_q + beta_j }.
//
// Two forms share every truncated kernel (FP64, compensated and the cell-list
// mixed passes):
//   * uniform (a radius R, Algorithm 2 with C = R^2/2): alpha_q = C, beta_j = 0;
//   * separable, psi-aware (Sec. 4.1 / App. B's geometric argument anchored at
//     each point's own nearest target n(q) instead of the worst-covered point):
//       alpha_q = c(x_q, y_n) - psi_n - eps ln nu_n,  beta_j = psi_j + eps ln(1/tail).
//     The anchor's term s_qn = (psi_n - c_qn)/eps + ln nu_n is always kept
//     (alpha_q + beta_n - c_qn = eps ln(1/(nu_n tail)) > 0) and every excluded
//     term has exp(s_qj) <= tail nu_j exp(s_qn), so the excluded mass of every
//     point is at most tail sum_j nu_j times its truncated sum: |J - J~| <= eps
//     tail sum(nu) sum(m), as for the global tail radius, whose cutoff
//     C_0 + Gamma + eps ln(1/(nu_min tail)) bounds alpha_q + beta_j from above.
//
// n(q) is the nearest target in FP64 (translated coordinates), the lowest
// index among equal costs: an FP32 scan finds the smallest FP32 distance, a
// second scan evaluates in FP64 every target whose FP32 distance lies within
// the FP32 rounding bound of it.  Computed once per problem.
#include <math.h>

#include <algorithm>
#include <vector>

#include "rsot_internal.cuh"

namespace rsot {
namespace {

constexpr int NN_THREADS = 128;
constexpr int NN_TS = 512;   // targets per shared-memory tile

// FP32 translated target coordinates [3][n_alloc] (padding far away)
__global__ void k_targets_f32(const double *__restrict__ y64, int64_t n, int64_t n_alloc, int d,
                              float *__restrict__ ys) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_alloc) return;
    for (int t = 0; t < 3; ++t) ys[t * n_alloc + j] = (j < n && t < d) ? (float)y64[j * d + t] : 1.0e30f;
}

template <int D>
__global__ void __launch_bounds__(NN_THREADS)
    k_nearest(const float *__restrict__ xs, const double *__restrict__ x64, int64_t nq,
              int64_t nq_pad, const float *__restrict__ ys, const double *__restrict__ y64,
              int64_t n, int64_t n_alloc, float span2, int *__restrict__ nn,
              double *__restrict__ nn_c) {
    __shared__ float sy[3][NN_TS];
    const int64_t q = (int64_t)blockIdx.x * NN_THREADS + threadIdx.x;
    const int64_t qq = q < nq ? q : 0;
    float x[3] = {0.f, 0.f, 0.f};
    for (int t = 0; t < D; ++t) x[t] = xs[t * nq_pad + qq];
    double xd[3] = {0.0, 0.0, 0.0};
    for (int t = 0; t < D; ++t) xd[t] = x64[qq * D + t];
    const int64_t n_rec = (n + NN_TS - 1) / NN_TS * NN_TS;   // <= n_alloc
    float best = INFINITY;
    for (int pass = 0; pass < 2; ++pass) {
        // pass 1: smallest FP32 squared distance; pass 2: FP64 over the candidates
        // within its rounding bound (2^-18 |coords|^2 + 2^-22 d, doubled)
        const float thr = best + (span2 * 0x1p-16f + best * 0x1p-20f);
        double bc = INFINITY;
        int bj = 0;
        for (int64_t t0 = 0; t0 < n_rec; t0 += NN_TS) {
            __syncthreads();
            for (int i = threadIdx.x; i < NN_TS; i += NN_THREADS)
                for (int t = 0; t < 3; ++t) sy[t][i] = ys[t * n_alloc + t0 + i];
            __syncthreads();
            for (int i = 0; i < NN_TS; ++i) {
                float d2 = 0.f;
#pragma unroll
                for (int t = 0; t < D; ++t) {
                    const float dd = x[t] - sy[t][i];
                    d2 = fmaf(dd, dd, d2);
                }
                if (pass == 0) {
                    best = fminf(best, d2);
                } else if (d2 <= thr) {
                    const int64_t j = t0 + i;   // < n: padding is 1e30 away
                    double c = 0.0;
#pragma unroll
                    for (int t = 0; t < D; ++t) {
                        const double dd = xd[t] - y64[j * D + t];
                        c += dd * dd;
                    }
                    c *= 0.5;
                    if (c < bc) {   // ascending j: the lowest index wins ties
                        bc = c;
                        bj = (int)j;
                    }
                }
            }
        }
        if (pass == 1 && q < nq) {
            nn[q] = bj;
            nn_c[q] = bc;
        }
    }
}

// alpha_q = c(x_q, y_n) - psi_n - eps ln nu_n (points), beta_j = psi_j + eps ln(1/tail)
__global__ void k_separable(const int *__restrict__ nn, const double *__restrict__ nn_c,
                            const double *__restrict__ psi, const double *__restrict__ lnu,
                            int64_t nq, int64_t nq_pad, int64_t n, int64_t n_alloc, double eps,
                            double eps_ln_inv_tail, double *__restrict__ alpha,
                            double *__restrict__ beta) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nq_pad) {
        double a = -INFINITY;
        if (i < nq) {
            const int j = nn[i];
            a = nn_c[i] - psi[j] - eps * lnu[j];
        }
        alpha[i] = a;
    }
    if (i < n_alloc) beta[i] = i < n ? psi[i] + eps_ln_inv_tail : -INFINITY;
}

__global__ void k_uniform(int64_t nq, int64_t nq_pad, int64_t n, int64_t n_alloc, double C,
                          double *__restrict__ alpha, double *__restrict__ beta) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nq_pad) alpha[i] = i < nq ? C : -INFINITY;
    if (i < n_alloc) beta[i] = i < n ? 0.0 : -INFINITY;
}

cudaError_t cutoff_alloc(rsot_problem *p) {
    cudaError_t e;
    if (!p->alpha && (e = cudaMalloc(&p->alpha, (size_t)p->nq_pad * sizeof(double)))) return e;
    if (!p->beta && (e = cudaMalloc(&p->beta, (size_t)p->n_pad * sizeof(double)))) return e;
    return cudaSuccess;
}

}  // namespace

cudaError_t cutoffs_uniform(rsot_problem *p, double C) {
    cudaError_t e = cutoff_alloc(p);
    if (e) return e;
    const int64_t m = std::max(p->nq_pad, p->n_pad);
    k_uniform<<<(unsigned)((m + 255) / 256), 256, 0, p->stream>>>(p->nq, p->nq_pad, p->n, p->n_pad, C,
                                                                 p->alpha, p->beta);
    p->cut_anchored = 0;
    return cudaGetLastError();
}

cudaError_t cutoffs_separable(rsot_problem *p, const double *psi, double eps, double tail) {
    cudaError_t e = cutoff_alloc(p);
    if (e) return e;
    cudaStream_t st = p->stream;
    if (!p->nn) {
        if ((e = cudaMalloc(&p->nn, (size_t)p->nq * sizeof(int)))) return e;
        if ((e = cudaMalloc(&p->nn_c, (size_t)p->nq * sizeof(double)))) return e;
        float *ys = nullptr;
        if ((e = cudaMallocAsync(&ys, (size_t)3 * p->n_pad * sizeof(float), st))) return e;
        k_targets_f32<<<(unsigned)((p->n_pad + 255) / 256), 256, 0, st>>>(p->y64, p->n, p->n_pad, p->d, ys);
        // squared extent of the translated coordinates bounds their FP32 rounding
        const float span2 = (float)p->diam2;
        trace_begin(p, "nearest_targets");
        const unsigned nb = (unsigned)((p->nq + NN_THREADS - 1) / NN_THREADS);
        if (p->d == 3)
            k_nearest<3><<<nb, NN_THREADS, 0, st>>>(p->xs, p->x64, p->nq, p->nq_pad, ys, p->y64, p->n,
                                                    p->n_pad, span2, p->nn, p->nn_c);
        else
            k_nearest<2><<<nb, NN_THREADS, 0, st>>>(p->xs, p->x64, p->nq, p->nq_pad, ys, p->y64, p->n,
                                                    p->n_pad, span2, p->nn, p->nn_c);
        trace_end(p);
        cudaFreeAsync(ys, st);
        if ((e = cudaGetLastError())) return e;
    }
    const int64_t m = std::max(p->nq_pad, p->n_pad);
    k_separable<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(p->nn, p->nn_c, psi, p->lnu, p->nq,
                                                            p->nq_pad, p->n, p->n_pad, eps,
                                                            eps * log(1.0 / tail), p->alpha, p->beta);
    p->cut_anchored = 1;
    return cudaGetLastError();
}

// ln D with D = sum_q m_q exp(-L_q) (Sec. 4.1, Eq. truncation_cutoff_int):
// per-block (max, scaled sum) of v_q = ln m_q - L_q over points with m_q > 0;
// an empty point (L_q = -inf) with mass gives +inf
__global__ void k_log_D(const double *__restrict__ L, const double *__restrict__ mass, int64_t nq,
                        double2 *__restrict__ part) {
    __shared__ double smax[256], ssum[256];
    double mx = -INFINITY, sm = 0.0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq;
         q += (int64_t)gridDim.x * blockDim.x) {
        if (!(mass[q] > 0.0)) continue;
        const double v = log(mass[q]) - L[q];
        if (v > mx) {
            sm = (mx == -INFINITY ? 0.0 : sm * exp(mx - v)) + 1.0;
            mx = v;
        } else {
            sm += exp(v - mx);
        }
    }
    smax[threadIdx.x] = mx;
    ssum[threadIdx.x] = sm;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const double a = smax[threadIdx.x], b = smax[threadIdx.x + o];
            const double m2 = fmax(a, b);
            double s2 = 0.0;
            if (a != -INFINITY) s2 += ssum[threadIdx.x] * (a == INFINITY ? 1.0 : exp(a - m2));
            if (b != -INFINITY) s2 += ssum[threadIdx.x + o] * (b == INFINITY ? 1.0 : exp(b - m2));
            smax[threadIdx.x] = m2;
            ssum[threadIdx.x] = s2;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = make_double2(smax[0], ssum[0]);
}

cudaError_t launch_log_D(rsot_problem *p, const double *L_dev, double *lnD) {
    constexpr int NB = 120;
    double2 *part = nullptr;
    cudaError_t e = cudaMallocAsync(&part, NB * sizeof(double2), p->stream);
    if (e) return e;
    k_log_D<<<NB, 256, 0, p->stream>>>(L_dev, p->mass, p->nq, part);
    double2 h[NB];
    e = cudaMemcpyAsync(h, part, sizeof(h), cudaMemcpyDeviceToHost, p->stream);
    cudaFreeAsync(part, p->stream);
    if (!e) e = cudaStreamSynchronize(p->stream);
    if (e) return e;
    double mx = -INFINITY;
    for (int i = 0; i < NB; ++i) mx = fmax(mx, h[i].x);
    if (!isfinite(mx)) {
        *lnD = mx;
        return cudaSuccess;
    }
    double s = 0.0;
    for (int i = 0; i < NB; ++i)
        if (h[i].x != -INFINITY) s += h[i].y * exp(h[i].x - mx);
    *lnD = mx + log(s);
    return cudaSuccess;
}

void cutoff_free(rsot_problem *p) {
    cudaFree(p->nn);
    cudaFree(p->nn_c);
    cudaFree(p->alpha);
    cudaFree(p->beta);
    p->nn = nullptr;
    p->nn_c = nullptr;
    p->alpha = p->beta = nullptr;
}

}  // namespace rsot
