// Transport maps (Sec. 6.3), conditional centroids (Eq. barycenter_fixed_point)
// and the damped Lloyd iteration for barycenters (Eq. damped_lloyd, Sec. 6.2).
//
// Both maps and centroids are sums over the plan p_qj of Eq. final_plan_density,
// evaluated like the mixed dense passes (rsot_dense.cu: log2 domain, translated
// coordinates, r_qj = c_j + x'_q.w_j with w_j = 2k y'_j, FP32 pair arithmetic,
// FP64 across tiles):
//   T_bary(x_q) - o = sum_j 2^(r_qj - M) w_j / (2k sum_j 2^(r_qj - M))   (per point,
//                     an online max shift M as in pass 1)
//   j*(q)           = argmax_j r_qj  (the first maximum in index order)
//   a_j             = sum_q m_q p_qj = sum_q 2^(r_qj + u_q),  u_q = log2 m_q - R_q
//   T_j             = (sum_q m_q p_qj x'_q + o a_j) / nu_j               (per target,
//                     after a dense evaluation provides u_q)
// These are post-processing sums of one pass each; they run on the CUDA cores
// with plain cooperative staging (no tensor cores, no bulk copies).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "rsot_internal.cuh"

namespace rsot {
namespace {

constexpr int MP_THREADS = 128;   // maps: one point per thread
constexpr int MP_TS = 256;        // target records per shared-memory tile
constexpr int MP_SUB = 16;        // targets per max sub-tile
constexpr int CT_THREADS = 128;   // centroids: two targets per thread
constexpr int CT_TS = 256;        // point records per shared-memory tile

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// T_bary and j* per point over all target records (dup layout of the dense
// pass 1: (w0,w0,w1,w1), (w2,w2,c,c)); n_rec is a multiple of MP_TS.
__global__ void __launch_bounds__(MP_THREADS)
    k_maps(const float *__restrict__ xs, int64_t nq_pad, int64_t nq, int d,
           const Rec8 *__restrict__ tdup, int64_t n_rec, int64_t n, double inv2k,
           const double *__restrict__ origin, double *__restrict__ Tout,
           int64_t *__restrict__ jout) {
    __shared__ __align__(16) Rec8 sm[MP_TS];
    const int64_t q = (int64_t)blockIdx.x * MP_THREADS + threadIdx.x;
    const bool live = q < nq;
    float x[3] = {0.f, 0.f, 0.f};
    if (q < nq_pad)
        for (int k = 0; k < d; ++k) x[k] = xs[k * nq_pad + q];
    float M = -INFINITY, best = -INFINITY;
    int64_t bj = 0;
    double S = 0.0, A0 = 0.0, A1 = 0.0, A2 = 0.0;
    for (int64_t t0 = 0; t0 < n_rec; t0 += MP_TS) {
        __syncthreads();
        for (int i = threadIdx.x; i < MP_TS; i += MP_THREADS) sm[i] = tdup[t0 + i];
        __syncthreads();
        float s = 0.f, a0 = 0.f, a1 = 0.f, a2 = 0.f;
        for (int u0 = 0; u0 < MP_TS; u0 += MP_SUB) {
            float r[MP_SUB];
            float mx = -INFINITY;
#pragma unroll
            for (int i = 0; i < MP_SUB; ++i) {
                const float4 a = sm[u0 + i].a, b = sm[u0 + i].b;
                r[i] = fmaf(x[0], a.x, fmaf(x[1], a.z, fmaf(x[2], b.x, b.z)));
                mx = fmaxf(mx, r[i]);
                if (r[i] > best) {   // strict: the first maximum in index order
                    best = r[i];
                    bj = t0 + u0 + i;
                }
            }
            if (mx > M) {   // raise the shift to ceil(max), rescale by a power of two
                const float mn = ceilf(mx);
                if (M != -INFINITY) {
                    const float dl = M - mn;
                    s *= pow2_int_f(dl), a0 *= pow2_int_f(dl), a1 *= pow2_int_f(dl), a2 *= pow2_int_f(dl);
                    const double dd = pow2_int_d(dl);
                    S *= dd, A0 *= dd, A1 *= dd, A2 *= dd;
                }
                M = mn;
            }
#pragma unroll
            for (int i = 0; i < MP_SUB; ++i) {
                const float4 a = sm[u0 + i].a, b = sm[u0 + i].b;
                const float e = ex2_approx(r[i] - M);
                s += e;
                a0 = fmaf(e, a.x, a0);
                a1 = fmaf(e, a.z, a1);
                a2 = fmaf(e, b.x, a2);
            }
        }
        S += s, A0 += a0, A1 += a1, A2 += a2;
    }
    if (!live) return;
    if (jout) jout[q] = bj < n ? bj : n - 1;
    if (Tout) {
        const double A[3] = {A0, A1, A2};
        for (int k = 0; k < d; ++k) Tout[q * d + k] = origin[k] + A[k] / S * inv2k;
    }
}

// Per target pair: a_j = sum_q 2^(c_j + x'.w_j + u_q) and the x'-weighted sums,
// over one chunk of point records (dup layout of pass 2: (x0,x0,x1,x1),
// (x2,x2,u,u)); partials [split][n_alloc][4] in FP64.
__global__ void __launch_bounds__(CT_THREADS)
    k_centroid_part(const Rec8 *__restrict__ tpair, const Rec8 *__restrict__ pdup, int64_t nq_pad,
                    int64_t chunk, int64_t n_alloc, double *__restrict__ part) {
    __shared__ __align__(16) Rec8 sm[CT_TS];
    const int64_t jp = (int64_t)blockIdx.x * CT_THREADS + threadIdx.x;   // target pair
    const Rec8 tr = tpair[jp];
    const float2 W0 = make_float2(tr.a.x, tr.a.y), W1 = make_float2(tr.a.z, tr.a.w);
    const float2 W2 = make_float2(tr.b.x, tr.b.y), C = make_float2(tr.b.z, tr.b.w);
    const int64_t p0 = (int64_t)blockIdx.y * chunk, p1 = min(p0 + chunk, nq_pad);
    double a[4][2] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
    for (int64_t t0 = p0; t0 < p1; t0 += CT_TS) {
        __syncthreads();
        for (int i = threadIdx.x; i < CT_TS; i += CT_THREADS) sm[i] = pdup[t0 + i];
        __syncthreads();
        float2 s = make_float2(0.f, 0.f), s0 = s, s1 = s, s2 = s;
#pragma unroll 4
        for (int i = 0; i < CT_TS; ++i) {
            const float4 pa = sm[i].a, pb = sm[i].b;
            const float2 x0 = make_float2(pa.x, pa.y), x1 = make_float2(pa.z, pa.w);
            const float2 x2 = make_float2(pb.x, pb.y), u = make_float2(pb.z, pb.w);
            float2 r = __ffma2_rn(x2, W2, C);
            r = __ffma2_rn(x1, W1, r);
            r = __ffma2_rn(x0, W0, r);
            r = __fadd2_rn(r, u);
            const float2 e = make_float2(ex2_approx(r.x), ex2_approx(r.y));
            s = __fadd2_rn(s, e);
            s0 = __ffma2_rn(e, x0, s0);
            s1 = __ffma2_rn(e, x1, s1);
            s2 = __ffma2_rn(e, x2, s2);
        }
        a[3][0] += s.x, a[3][1] += s.y;
        a[0][0] += s0.x, a[0][1] += s0.y;
        a[1][0] += s1.x, a[1][1] += s1.y;
        a[2][0] += s2.x, a[2][1] += s2.y;
    }
    double *o = part + ((int64_t)blockIdx.y * n_alloc + 2 * jp) * 4;
    for (int h = 0; h < 2; ++h)
        for (int k = 0; k < 4; ++k) o[h * 4 + k] = a[k][h];
}

// fixed-order sum over the splits: T_j = (sum m p x' + o a_j) / nu_j, a_j
__global__ void k_centroid_final(const double *__restrict__ part, int splits, int64_t n_alloc,
                                 int64_t n, int d, const double *__restrict__ nu,
                                 const double *__restrict__ origin, double *__restrict__ T,
                                 double *__restrict__ mass) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = 0; i < splits; ++i)
        for (int k = 0; k < 4; ++k) s[k] += part[((int64_t)i * n_alloc + j) * 4 + k];
    for (int k = 0; k < d; ++k) T[j * d + k] = (s[k] + origin[k] * s[3]) / nu[j];
    if (mass) mass[j] = s[3];
}

}  // namespace

// T_bary / j* over the dense target records of the last mixed evaluation
cudaError_t launch_maps(rsot_problem *p, double eps, double *T_dev, int64_t *j_dev,
                        const double *origin_dev) {
    const int64_t n_rec = round_up(p->n, MP_TS);
    const double inv2k = 1.0 / (2.0 * kLog2e / (2.0 * eps));
    k_maps<<<(unsigned)((p->nq + MP_THREADS - 1) / MP_THREADS), MP_THREADS, 0, p->stream>>>(
        p->xs, p->nq_pad, p->nq, p->d, p->tdup, n_rec, p->n, inv2k, origin_dev, T_dev, j_dev);
    return cudaGetLastError();
}

// centroids over the pass-2 point records of the last mixed evaluation
cudaError_t launch_centroids(rsot_problem *p, double *T_dev, double *mass_dev,
                             const double *origin_dev) {
    cudaStream_t st = p->stream;
    const int64_t pairs_blocks = p->n_pad / 2 / CT_THREADS;   // n_pad is a multiple of 1024
    int splits = (int)std::max<int64_t>(1, std::min<int64_t>(64, (4 * p->num_sms + pairs_blocks - 1) / pairs_blocks));
    const int64_t chunk = round_up((p->nq_pad + splits - 1) / splits, CT_TS);
    splits = (int)((p->nq_pad + chunk - 1) / chunk);
    double *part = nullptr;
    cudaError_t e = cudaMallocAsync(&part, (size_t)splits * p->n_pad * 4 * sizeof(double), st);
    if (e) return e;
    dim3 grid((unsigned)pairs_blocks, (unsigned)splits);
    k_centroid_part<<<grid, CT_THREADS, 0, st>>>(p->tpair, p->pdup, p->nq_pad, chunk, p->n_pad, part);
    k_centroid_final<<<(unsigned)((p->n + 255) / 256), 256, 0, st>>>(part, splits, p->n_pad, p->n, p->d,
                                                                     p->nu, origin_dev, T_dev, mass_dev);
    e = cudaGetLastError();
    cudaFreeAsync(part, st);
    return e;
}

}  // namespace rsot
