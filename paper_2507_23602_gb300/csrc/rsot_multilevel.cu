// Multilevel acceleration (Sec. 5): target hierarchy by k-means (Sec. 5.2),
// softmax refinement of the potential between target levels (Eq.
// softmax_refinement_formula), injection between source levels, and the
// combined schedule of Sec. 5.3 with eps synchronised to the levels.
//
// k-means: the assignment step (nearest centre of every point) runs on the
// GPU -- FP32 expanded-form distances |c|^2 - 2 x.c in shared-memory tiles of
// centres, lowest index on ties -- and the update step (weighted centroids,
// cluster weights summed in FP64 in point order) on the host, so that the
// result is deterministic.  The initial centres are a seeded random subset of
// the points (splitmix64 on the seed).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <numeric>
#include <vector>

#include "rsot_internal.cuh"

namespace rsot {
namespace {

constexpr int KM_THREADS = 256;
constexpr int KM_TILE = 1024;   // centres per shared-memory tile

// centres as (-2c0, -2c1, -2c2, |c|^2) FP32; argmin_j |c_j|^2 - 2 x.c_j
__global__ void k_kmeans_assign(const float *__restrict__ x, int64_t n, const float4 *__restrict__ c4,
                                int64_t k, int *__restrict__ assign) {
    __shared__ float4 sc[KM_TILE];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float x0 = 0.f, x1 = 0.f, x2 = 0.f;
    if (i < n) {
        x0 = x[i * 3 + 0];
        x1 = x[i * 3 + 1];
        x2 = x[i * 3 + 2];
    }
    float best = INFINITY;
    int arg = 0;
    for (int64_t t0 = 0; t0 < k; t0 += KM_TILE) {
        for (int j = threadIdx.x; j < KM_TILE; j += blockDim.x)
            sc[j] = (t0 + j < k) ? c4[t0 + j] : make_float4(0.f, 0.f, 0.f, INFINITY);
        __syncthreads();
        const int cnt = (int)min((int64_t)KM_TILE, k - t0);
        for (int j = 0; j < cnt; ++j) {
            const float4 c = sc[j];
            const float v = fmaf(x0, c.x, fmaf(x1, c.y, fmaf(x2, c.z, c.w)));
            if (v < best) {
                best = v;
                arg = (int)(t0 + j);
            }
        }
        __syncthreads();
    }
    if (i < n) assign[i] = arg;
}

uint64_t splitmix64(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace
}  // namespace rsot

using namespace rsot;

extern "C" {

rsot_status rsot_kmeans(int d, int64_t n, const double *y, const double *w, int64_t k, int iters,
                        uint64_t seed, double *centers_out, double *weights_out,
                        int64_t *assign_out) {
    if ((d != 2 && d != 3) || n < 1 || k < 1 || k > n || iters < 0 || !y || !w || !centers_out ||
        !weights_out)
        return RSOT_ERR_ARG;
    std::vector<double> hy((size_t)n * d), hw(n);
    if (cudaMemcpy(hy.data(), y, hy.size() * 8, cudaMemcpyDefault) ||
        cudaMemcpy(hw.data(), w, hw.size() * 8, cudaMemcpyDefault)) {
        cudaGetLastError();
        return RSOT_ERR_CUDA;
    }
    // centre of the data (FP32 distances are taken in translated coordinates)
    double o[3] = {0, 0, 0};
    for (int t = 0; t < d; ++t) {
        double lo = INFINITY, hi = -INFINITY;
        for (int64_t i = 0; i < n; ++i) {
            lo = std::min(lo, hy[i * d + t]);
            hi = std::max(hi, hy[i * d + t]);
        }
        o[t] = 0.5 * (lo + hi);
    }
    std::vector<float> hx((size_t)n * 3, 0.f);
    for (int64_t i = 0; i < n; ++i)
        for (int t = 0; t < d; ++t) hx[i * 3 + t] = (float)(hy[i * d + t] - o[t]);
    // seeded initial centres: a partial Fisher-Yates shuffle of the indices
    std::vector<int64_t> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    uint64_t s = seed;
    for (int64_t i = 0; i < k; ++i) {
        const int64_t j = i + (int64_t)(splitmix64(s) % (uint64_t)(n - i));
        std::swap(idx[i], idx[j]);
    }
    std::vector<double> C((size_t)k * 3, 0.0);
    for (int64_t c = 0; c < k; ++c)
        for (int t = 0; t < d; ++t) C[c * 3 + t] = hy[idx[c] * d + t] - o[t];
    float *dx = nullptr;
    float4 *dc = nullptr;
    int *da = nullptr;
    cudaError_t e = cudaMalloc(&dx, hx.size() * 4);
    if (!e) e = cudaMalloc(&dc, k * sizeof(float4));
    if (!e) e = cudaMalloc(&da, n * sizeof(int));
    if (!e) e = cudaMemcpy(dx, hx.data(), hx.size() * 4, cudaMemcpyHostToDevice);
    std::vector<int> a(n, 0);
    std::vector<float4> c4(k);
    std::vector<double> W(k);
    for (int it = 0; !e && it <= iters; ++it) {
        for (int64_t c = 0; c < k; ++c) {
            const double cx = C[c * 3], cy = C[c * 3 + 1], cz = C[c * 3 + 2];
            c4[c] = make_float4((float)(-2.0 * cx), (float)(-2.0 * cy), (float)(-2.0 * cz),
                                (float)(cx * cx + cy * cy + cz * cz));
        }
        e = cudaMemcpy(dc, c4.data(), k * sizeof(float4), cudaMemcpyHostToDevice);
        if (e) break;
        k_kmeans_assign<<<(unsigned)((n + KM_THREADS - 1) / KM_THREADS), KM_THREADS>>>(dx, n, dc, k, da);
        e = cudaMemcpy(a.data(), da, n * sizeof(int), cudaMemcpyDeviceToHost);
        if (e) break;
        // update: weighted centroids in point order (FP64); empty clusters keep their centre
        std::vector<double> S((size_t)k * 3, 0.0);
        std::fill(W.begin(), W.end(), 0.0);
        for (int64_t i = 0; i < n; ++i) {
            const int c = a[i];
            W[c] += hw[i];
            for (int t = 0; t < d; ++t) S[(size_t)c * 3 + t] += hw[i] * (hy[i * d + t] - o[t]);
        }
        if (it == iters) break;   // the last assignment defines the clusters
        for (int64_t c = 0; c < k; ++c)
            if (W[c] > 0.0)
                for (int t = 0; t < d; ++t) C[c * 3 + t] = S[c * 3 + t] / W[c];
        // empty clusters restart at the points farthest from their centres
        // (largest distance first, lowest index on ties; each point used once)
        std::vector<int64_t> empty;
        for (int64_t c = 0; c < k; ++c)
            if (!(W[c] > 0.0)) empty.push_back(c);
        if (!empty.empty()) {
            std::vector<std::pair<double, int64_t>> far(n);
            for (int64_t i = 0; i < n; ++i) {
                double r = 0.0;
                for (int t = 0; t < d; ++t) {
                    const double v = hy[i * d + t] - o[t] - C[(size_t)a[i] * 3 + t];
                    r += v * v;
                }
                far[i] = {-r, i};
            }
            const size_t take = std::min(empty.size(), (size_t)n);
            std::partial_sort(far.begin(), far.begin() + take, far.end());
            for (size_t e2 = 0; e2 < take; ++e2)
                for (int t = 0; t < d; ++t)
                    C[empty[e2] * 3 + t] = hy[far[e2].second * d + t] - o[t];
        }
    }
    cudaFree(dx);
    cudaFree(dc);
    cudaFree(da);
    if (e) {
        cudaGetLastError();
        return RSOT_ERR_CUDA;
    }
    // final centres: centroids of the final clusters (cluster mass = summed weights)
    std::vector<double> S((size_t)k * 3, 0.0);
    for (int64_t i = 0; i < n; ++i)
        for (int t = 0; t < d; ++t) S[(size_t)a[i] * 3 + t] += hw[i] * (hy[i * d + t] - o[t]);
    for (int64_t c = 0; c < k; ++c) {
        for (int t = 0; t < d; ++t)
            centers_out[c * d + t] = (W[c] > 0.0 ? S[c * 3 + t] / W[c] : C[c * 3 + t]) + o[t];
        weights_out[c] = W[c];
    }
    if (assign_out)
        for (int64_t i = 0; i < n; ++i) assign_out[i] = a[i];
    return RSOT_OK;
}

rsot_status rsot_softmax_refine(rsot_problem *p, const double *psi_coarse, double eps, int64_t n_fine,
                                const double *y_fine, double *psi_fine_out) {
    if (!p || !psi_coarse || !y_fine || !psi_fine_out || n_fine < 1 || !(eps > 0.0)) return RSOT_ERR_ARG;
    cudaStream_t st = p->stream;
    const int d = p->d;
    p->last_kind = -1;   // its pass 1 replaces the per-point sums of the last evaluation
    double *dpsi = nullptr, *dyf = nullptr, *dout = nullptr;
    cudaError_t e = cudaMallocAsync(&dpsi, (size_t)p->n * 8, st);
    if (!e) e = cudaMallocAsync(&dyf, (size_t)n_fine * d * 8, st);
    if (!e) e = cudaMallocAsync(&dout, (size_t)n_fine * 8, st);
    if (!e) e = cudaMemcpyAsync(dpsi, psi_coarse, (size_t)p->n * 8, cudaMemcpyDefault, st);
    if (!e) e = cudaMemcpyAsync(dyf, y_fine, (size_t)n_fine * d * 8, cudaMemcpyDefault, st);
    if (!e) e = cudaMemsetAsync(p->res_dev, 0, sizeof(EvalResult), st);
    if (!e) e = launch_softmax_refine(p, dpsi, eps, n_fine, dyf, dout);
    if (!e) e = cudaMemcpyAsync(p->res_host, p->res_dev, sizeof(EvalResult), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    // the output is written only when the passes succeeded
    rsot_status s = RSOT_OK;
    if (!e) {
        if (p->res_host->flags & kErrTimeout) s = RSOT_ERR_TIMEOUT;
        else if (p->res_host->flags & kErrNonfinitePsi) s = RSOT_ERR_NONFINITE;
        else e = cudaMemcpyAsync(psi_fine_out, dout, (size_t)n_fine * 8, cudaMemcpyDefault, st);
    }
    cudaFreeAsync(dpsi, st);
    cudaFreeAsync(dyf, st);
    cudaFreeAsync(dout, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e) {
        cudaGetLastError();
        return RSOT_ERR_CUDA;
    }
    return s;
}

rsot_status rsot_multilevel_solve(int n_src, const rsot_source_level *src, int n_tgt,
                                  const rsot_target_level *tgt, const double *eps_levels,
                                  const rsot_options *opt, double *psi_out,
                                  rsot_multilevel_stats *stats) {
    if (n_src < 1 || n_tgt < 1 || !src || !tgt || !eps_levels || !opt || !psi_out) return RSOT_ERR_ARG;
    if (n_src > RSOT_MAX_LEVELS || n_tgt > RSOT_MAX_LEVELS) return RSOT_ERR_ARG;
    const auto t_all = std::chrono::steady_clock::now();
    const int Lmu = n_src - 1, Lnu = n_tgt - 1, Lmax = std::max(Lmu, Lnu);
    std::vector<double> psi;        // potential on the current target level
    int it_prev = -1;
    double eps_prev = eps_levels[0];
    rsot_status status = RSOT_OK;
    if (stats) memset(stats, 0, sizeof(*stats));
    for (int l = 0; l <= Lmax; ++l) {
        const int is = std::max(0, l - (Lmax - Lmu));
        const int itg = std::max(0, l - (Lmax - Lnu));
        const rsot_source_level &S = src[is];
        const rsot_target_level &T = tgt[itg];
        const double eps = eps_levels[l];
        const auto t0 = std::chrono::steady_clock::now();
        rsot_problem *p = nullptr;
        rsot_status s = rsot_create(S.d, S.nq, S.x, S.mass, T.n, T.y, T.nu, 0, &p);
        if (s) return s;
        int transfer = 0;   // 0 none (first level), 1 injection, 2 softmax refinement
        if (l == 0) {
            psi.assign(T.n, 0.0);
        } else if (itg == it_prev) {
            transfer = 1;   // same target level: the potential is used as it is
        } else {
            // the coarse target level on the current source level refines psi
            transfer = 2;
            const rsot_target_level &Tc = tgt[it_prev];
            rsot_problem *pc = nullptr;
            s = rsot_create(S.d, S.nq, S.x, S.mass, Tc.n, Tc.y, Tc.nu, 0, &pc);
            if (!s) {
                std::vector<double> fine(T.n);
                // the coarse pair (phi, psi) is optimal at the previous level's eps
                s = rsot_softmax_refine(pc, psi.data(), eps_prev, T.n, T.y, fine.data());
                psi.swap(fine);
            }
            rsot_destroy(pc);
            if (s) {
                rsot_destroy(p);
                return s;
            }
        }
        rsot_options o = *opt;
        o.eps = eps;
        if (l > 0) o.eps_start = 0.0;   // later levels start warm at their own eps
        if (l < Lmax) {
            // coarser levels only provide the warm start of the next one: mixed
            // evaluations, stopped at the mixed tolerance (no FP64 refinement)
            o.refine_fp64 = 0;
            o.tol_l1 = std::max(opt->tol_l1, opt->mixed_tol_l1 > 0.0 ? opt->mixed_tol_l1 : 1e-5);
        }
        rsot_solve_stats ss;
        s = rsot_solve(p, psi.data(), &o, &ss);
        rsot_destroy(p);
        if (stats) {
            stats->levels = l + 1;
            stats->src_level[l] = is;
            stats->tgt_level[l] = itg;
            stats->transfer[l] = transfer;
            stats->iters[l] = ss.iters;
            stats->evals[l] = ss.evals;
            stats->seconds[l] =
                std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            stats->grad_l1 = ss.grad_l1;
        }
        if (s && s != RSOT_ERR_NOT_CONVERGED && s != RSOT_ERR_LINESEARCH) return s;
        status = s;
        it_prev = itg;
        eps_prev = eps;
    }
    std::copy(psi.begin(), psi.end(), psi_out);
    if (stats)
        stats->total_seconds =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t_all).count();
    return status;
}

}  // extern "C"
