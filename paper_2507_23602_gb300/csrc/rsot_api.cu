// C ABI of librsot: problem setup, one dual evaluation, covering cost and
// truncation radius.  The solver lives in rsot_solve.cpp.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "rsot_internal.cuh"

using namespace rsot;

namespace {

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

bool is_device_ptr(const void *ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// 0: host memory, 1: device memory of the current device (or managed),
// -1: device memory of another device (rejected: kernels here would need
// peer access to read it)
int where_ptr(const void *ptr) {
    cudaPointerAttributes a;
    int dev = -1;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (a.type == cudaMemoryTypeManaged) return 1;
    if (a.type == cudaMemoryTypeDevice) return a.device == dev ? 1 : -1;
    return 0;
}

// device memory of the current device (or managed memory): what a kernel of
// this library may read without peer access
bool is_current_device_ptr(const void *ptr) {
    cudaPointerAttributes a;
    int dev = -1;
    if (!ptr || cudaPointerGetAttributes(&a, ptr) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == dev);
}

rsot_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return RSOT_OK;
    if (e == cudaErrorMemoryAllocation) return RSOT_ERR_NOMEM;
    return RSOT_ERR_CUDA;
}

template <class T>
cudaError_t upload(T **dst, const T *src, size_t count) {
    cudaError_t e = cudaMalloc(dst, count * sizeof(T));
    if (e) return e;
    return cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice);
}

struct NSum {   // Neumaier-compensated host sum
    double s = 0.0, c = 0.0;
    void add(double v) {
        const double t = s + v;
        c += (fabs(s) >= fabs(v)) ? (s - t) + v : (v - t) + s;
        s = t;
    }
    double val() const { return s + c; }
};

}  // namespace

namespace rsot {

void trace_begin(rsot_problem *p, const char *name) {
    if (!p->timing) return;
    if ((int)p->tr_events.size() < p->tr_used + 2) {
        for (int i = 0; i < 2; ++i) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            p->tr_events.push_back(e);
        }
    }
    p->tr_open.emplace_back(name, p->tr_used);
    cudaEventRecord(p->tr_events[p->tr_used], p->stream);
    p->tr_used += 2;
}

void trace_end(rsot_problem *p) {
    if (!p->timing || p->tr_open.empty()) return;
    cudaEventRecord(p->tr_events[p->tr_open.back().second + 1], p->stream);
}

void trace_collect(rsot_problem *p) {
    for (auto &o : p->tr_open) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p->tr_events[o.second], p->tr_events[o.second + 1]) !=
            cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        size_t k = 0;
        while (k < p->tr_names.size() && std::string(p->tr_names[k]) != o.first) ++k;
        if (k == p->tr_names.size()) {
            p->tr_names.push_back(o.first);
            p->tr_total_ms.push_back(0.0);
            p->tr_count.push_back(0);
        }
        p->tr_total_ms[k] += ms;
        p->tr_count[k] += 1;
    }
    p->tr_open.clear();
    p->tr_used = 0;
}

int64_t num_targets(const rsot_problem *p) { return p->n; }
int64_t num_points(const rsot_problem *p) { return p->nq; }
double mass_sum(const rsot_problem *p) { return p->msum; }
void copy_nu(const rsot_problem *p, double *out) {
    cudaMemcpy(out, p->nu, (size_t)p->n * sizeof(double), cudaMemcpyDeviceToHost);
}
int pair_kernel_of(const rsot_problem *p) { return p->pair_kernel; }
void set_in_solve(rsot_problem *p, int on) { p->in_solve = on; }
// A solver near convergence: the next mixed evaluations take the FP32 kernels
// when the gradient's L1 norm is within kTcNoiseFactor of the tensor-core noise.
void pair_kernel_for_gradient(rsot_problem *p, double grad_l1) {
    p->pair_fp32_now = grad_l1 < kTcNoiseFactor * p->tc_noise_l1 ? 1 : 0;
}
double tc_noise_l1_of(const rsot_problem *p) { return p->tc_noise_l1; }

}  // namespace rsot

extern "C" {

const char *rsot_status_string(rsot_status s) {
    switch (s) {
        case RSOT_OK: return "ok";
        case RSOT_ERR_ARG: return "invalid argument";
        case RSOT_ERR_CUDA: return "CUDA error";
        case RSOT_ERR_NONFINITE: return "non-finite value";
        case RSOT_ERR_EMPTY_NEIGHBORHOOD: return "a point has no target within the radius";
        case RSOT_ERR_NOT_CONVERGED: return "iteration limit reached";
        case RSOT_ERR_LINESEARCH: return "line search failed";
        case RSOT_ERR_TIMEOUT: return "device wait timed out";
        case RSOT_ERR_NOMEM: return "out of device memory";
    }
    return "unknown status";
}

const char *rsot_version(void) { return "rsot-gb300 0.1 (sm_103a)"; }

void rsot_destroy(rsot_problem *p) {
    if (!p) return;
    trunc_free(p);
    compensated_free(p);
    cutoff_free(p);
    dense_free(p);
    cudaFree(p->xs);
    cudaFree(p->x64);
    if (!p->borrowed) cudaFree(p->mass);
    cudaFree(p->lmass2);
    cudaFree(p->y64);
    if (!p->borrowed) cudaFree(p->nu);
    cudaFree(p->lnu);
    cudaFree(p->psi_dev);
    cudaFree(p->grad_dev);
    cudaFree(p->res_dev);
    if (p->res_host) cudaFreeHost(p->res_host);
    if (p->grad_host) cudaFreeHost(p->grad_host);
    for (cudaEvent_t e : p->tr_events) cudaEventDestroy(e);
    delete p;
}

rsot_status rsot_create(int d, int64_t nq, const double *x, const double *mass, int64_t n,
                        const double *y, const double *nu, int device_ptrs, rsot_problem **out) {
    if (!out) return RSOT_ERR_ARG;
    *out = nullptr;
    if ((d != 2 && d != 3) || nq < 1 || n < 1 || !x || !mass || !y || !nu) return RSOT_ERR_ARG;
    if (nq > (int64_t)1 << 31 || n > (int64_t)1 << 30) return RSOT_ERR_ARG;
    if (device_ptrs != 0 && device_ptrs != 1) return RSOT_ERR_ARG;
    if (device_ptrs && (!is_current_device_ptr(x) || !is_current_device_ptr(mass) ||
                        !is_current_device_ptr(y) || !is_current_device_ptr(nu)))
        return RSOT_ERR_ARG;

    std::vector<double> hx((size_t)nq * d), hm((size_t)nq), hy((size_t)n * d), hnu((size_t)n);
    if (cudaMemcpy(hx.data(), x, hx.size() * 8, cudaMemcpyDefault) ||
        cudaMemcpy(hm.data(), mass, hm.size() * 8, cudaMemcpyDefault) ||
        cudaMemcpy(hy.data(), y, hy.size() * 8, cudaMemcpyDefault) ||
        cudaMemcpy(hnu.data(), nu, hnu.size() * 8, cudaMemcpyDefault)) {
        cudaGetLastError();
        return RSOT_ERR_CUDA;
    }
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < nq; ++i) {
        if (!(hm[i] >= 0.0) || !isfinite(hm[i])) return RSOT_ERR_ARG;
        for (int k = 0; k < d; ++k) {
            const double v = hx[i * d + k];
            if (!isfinite(v)) return RSOT_ERR_ARG;
            lo[k] = std::min(lo[k], v);
            hi[k] = std::max(hi[k], v);
        }
    }
    for (int64_t j = 0; j < n; ++j) {
        if (!(hnu[j] > 0.0) || !isfinite(hnu[j])) return RSOT_ERR_ARG;
        for (int k = 0; k < d; ++k) {
            const double v = hy[j * d + k];
            if (!isfinite(v)) return RSOT_ERR_ARG;
            lo[k] = std::min(lo[k], v);
            hi[k] = std::max(hi[k], v);
        }
    }

    rsot_problem *p = new rsot_problem();
    p->d = d;
    p->nq = nq;
    p->n = n;
    cudaGetDevice(&p->dev);
    cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->dev);
    for (int k = 0; k < d; ++k) p->origin[k] = 0.5 * (lo[k] + hi[k]);
    p->diam2 = 0.0;
    for (int k = 0; k < d; ++k) p->diam2 += (hi[k] - lo[k]) * (hi[k] - lo[k]);
    p->nq_pad = round_up(nq, 1024);

    // translated coordinates (cost is translation invariant)
    std::vector<float> xs((size_t)d * p->nq_pad, 0.0f);
    std::vector<double> lm2((size_t)nq);
    NSum ms, hh;
    for (int64_t i = 0; i < nq; ++i) {
        double r2 = 0.0;
        for (int k = 0; k < d; ++k) {
            const double v = hx[i * d + k] - p->origin[k];
            hx[i * d + k] = v;
            xs[(size_t)k * p->nq_pad + i] = (float)v;
            r2 += v * v;
        }
        ms.add(hm[i]);
        hh.add(hm[i] * 0.5 * r2);
        p->m_max = std::max(p->m_max, hm[i]);
        lm2[i] = hm[i] > 0.0 ? log2(hm[i]) : -INFINITY;
    }
    p->msum = ms.val();
    p->hx = hh.val();
    // tensor-core operand scale: P x' within [-32, 32] (a power of two, exact)
    {
        float xmax = 0.0f;
        for (size_t i = 0; i < xs.size(); ++i) xmax = std::max(xmax, std::fabs(xs[i]));
        int ex = 0;
        if (xmax > 0.0f) std::frexp(xmax, &ex);
        p->tc_P = std::ldexp(1.0f, 5 - ex);
    }
    std::vector<double> lnu((size_t)n);
    p->nu_min = INFINITY;
    p->nu_max = 0.0;
    {
        double sq = 0.0;
        for (int64_t j = 0; j < n; ++j) sq += sqrt(hnu[j]);
        p->tc_noise_l1 = 1.4e-5 * sqrt(p->m_max) * sq;
    }
    for (int64_t j = 0; j < n; ++j) {
        for (int k = 0; k < d; ++k) hy[j * d + k] -= p->origin[k];
        lnu[j] = log(hnu[j]);
        p->nu_min = std::min(p->nu_min, hnu[j]);
        p->nu_max = std::max(p->nu_max, hnu[j]);
    }

    cudaError_t e = cudaSuccess;
    if (!e) e = upload(&p->xs, xs.data(), xs.size());
    if (!e) e = upload(&p->x64, hx.data(), hx.size());
    p->borrowed = device_ptrs == 1;
    if (p->borrowed) {
        p->mass = const_cast<double *>(mass);
        p->nu = const_cast<double *>(nu);
    }
    if (!e && !p->borrowed) e = upload(&p->mass, hm.data(), hm.size());
    if (!e) e = upload(&p->lmass2, lm2.data(), lm2.size());
    if (!e) e = upload(&p->y64, hy.data(), hy.size());
    if (!e && !p->borrowed) e = upload(&p->nu, hnu.data(), hnu.size());
    if (!e) e = upload(&p->lnu, lnu.data(), lnu.size());
    if (!e) e = dense_alloc(p);
    if (!e) e = cudaMalloc(&p->psi_dev, (size_t)n * 8);
    if (!e) e = cudaMalloc(&p->grad_dev, (size_t)n * 8);
    if (!e) e = cudaMalloc(&p->res_dev, sizeof(EvalResult) + 8 * sizeof(double));
    if (!e) e = cudaMallocHost(&p->res_host, sizeof(EvalResult) + 8 * sizeof(double));
    if (!e) e = cudaMallocHost(&p->grad_host, (size_t)n * 8);
    if (e) {
        cudaGetLastError();
        rsot_destroy(p);
        return from_cuda(e);
    }
    p->flags = &p->res_dev->flags;
    *out = p;
    return RSOT_OK;
}

rsot_status rsot_set_stream(rsot_problem *p, void *stream) {
    if (!p) return RSOT_ERR_ARG;
    p->stream = (cudaStream_t)stream;
    return RSOT_OK;
}

rsot_status rsot_set_pair_kernel(rsot_problem *p, rsot_pair_kernel kind) {
    if (!p || (kind != RSOT_PAIRS_FP32 && kind != RSOT_PAIRS_TENSOR && kind != RSOT_PAIRS_AUTO))
        return RSOT_ERR_ARG;
    p->pair_kernel = (int)kind;
    return RSOT_OK;
}

// One evaluation: dense (mode 0), truncated by a radius (mode 1, cutoff C =
// arg^2 / 2 for every pair) or by the separable psi-aware cutoffs (mode 2,
// tail = arg, rsot_cutoff.cu).
static rsot_status eval_impl(rsot_problem *p, const double *psi, double eps, int mode, double arg,
                             rsot_precision prec, double *J_out, double *grad_out,
                             int64_t *pairs_out) {
    if (!p || !psi || !J_out || !grad_out) return RSOT_ERR_ARG;
    if (!(eps > 0.0) || !isfinite(eps) || isnan(arg)) return RSOT_ERR_ARG;
    if (prec != RSOT_FP64 && prec != RSOT_MIXED && prec != RSOT_COMPENSATED) return RSOT_ERR_ARG;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        return RSOT_ERR_CUDA;
    }
    if (cur != p->dev) return RSOT_ERR_ARG;   // the handle's device must be current
    const int wpsi = where_ptr(psi), wgrad = where_ptr(grad_out);
    if (wpsi < 0 || wgrad < 0) return RSOT_ERR_ARG;
    cudaStream_t st = p->stream;
    const size_t nb = (size_t)p->n * sizeof(double);
    const double *psid = psi;
    cudaError_t e = cudaSuccess;
    if (wpsi == 0) {
        e = cudaMemcpyAsync(p->psi_dev, psi, nb, cudaMemcpyHostToDevice, st);
        psid = p->psi_dev;
    }
    // the passes write the handle's gradient; the caller's buffer receives it
    // only when the evaluation succeeds (a device-side conditional copy, or a
    // pinned staging copy for host memory)
    const bool gdev = wgrad == 1;
    double *gd = p->grad_dev;
    if (!e) e = cudaMemsetAsync(p->res_dev, 0, sizeof(EvalResult), st);
    // a radius beyond the diameter of the data keeps every pair: dense
    const bool dense = mode == 0 || (mode == 1 && (!(arg > 0.0) || isinf(arg) ||
                                                    arg * arg > p->diam2 * (1.0 + 1e-12)));
    if (!e && !dense) e = mode == 1 ? cutoffs_uniform(p, 0.5 * arg * arg) : cutoffs_separable(p, psid, eps, arg);
    if (!e) {
        if (prec == RSOT_COMPENSATED)
            e = launch_compensated(p, psid, eps, !dense, gd);
        else if (dense)
            e = (prec == RSOT_MIXED) ? launch_dense_mixed(p, psid, eps, gd)
                                     : launch_dense_fp64(p, psid, eps, gd);
        else
            e = trunc_eval(p, psid, eps, prec == RSOT_MIXED, gd);
    }
    if (!e && gdev && grad_out != gd)
        e = launch_commit_grad(gd, grad_out, p->n, p->res_dev, dense ? 0 : 1, st);
    if (!e && !gdev) e = cudaMemcpyAsync(p->grad_host, gd, nb, cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaMemcpyAsync(p->res_host, p->res_dev, sizeof(EvalResult), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e) {
        cudaGetLastError();
        p->tr_open.clear();
        p->tr_used = 0;
        return from_cuda(e);
    }
    trace_collect(p);
    const EvalResult r = *p->res_host;
    p->last_kind = -1;
    if (r.flags & kErrTimeout) return RSOT_ERR_TIMEOUT;
    if (r.flags & kErrBadCell) return RSOT_ERR_CUDA;
    if (r.flags & kErrNonfinitePsi) return RSOT_ERR_NONFINITE;
    if (r.flags) return RSOT_ERR_CUDA;   // an error bit this code does not know
    if (!isfinite(r.J)) return RSOT_ERR_NONFINITE;
    p->last_kind = prec == RSOT_COMPENSATED ? (dense ? 4 : 5)
                                            : dense ? (prec == RSOT_MIXED ? 1 : 0)
                                                    : (prec == RSOT_MIXED ? 3 : 2);
    p->last_eps = eps;
    p->last_dense = dense;
    p->last_J = r.J;
    p->last_pairs = dense ? p->nq * p->n : (int64_t)r.pairs;
    p->last_empty = dense ? 0 : (int64_t)r.empty;
    if (p->last_empty > 0) return RSOT_ERR_EMPTY_NEIGHBORHOOD;   // outputs untouched
    *J_out = r.J;
    if (pairs_out) *pairs_out = p->last_pairs;
    if (!gdev) memcpy(grad_out, p->grad_host, nb);
    return RSOT_OK;
}

rsot_status rsot_eval_dual_grad(rsot_problem *p, const double *psi, double eps, double radius,
                                rsot_precision prec, double *J_out, double *grad_out,
                                int64_t *pairs_out) {
    return eval_impl(p, psi, eps, 1, radius, prec, J_out, grad_out, pairs_out);
}

rsot_status rsot_eval_dual_grad_tail(rsot_problem *p, const double *psi, double eps, double tail,
                                     rsot_precision prec, double *J_out, double *grad_out,
                                     int64_t *pairs_out) {
    if (!(tail > 0.0) || !(tail < 1.0)) return RSOT_ERR_ARG;
    return eval_impl(p, psi, eps, 2, tail, prec, J_out, grad_out, pairs_out);
}

rsot_status rsot_last_eval(rsot_problem *p, double *J_out, double *grad_out, int64_t *pairs_out,
                           int64_t *empty_out) {
    if (!p || p->last_kind < 0) return RSOT_ERR_ARG;
    if (grad_out) {
        cudaError_t e = cudaMemcpyAsync(grad_out, p->grad_dev, (size_t)p->n * sizeof(double),
                                        cudaMemcpyDefault, p->stream);
        if (!e) e = cudaStreamSynchronize(p->stream);
        if (e) {
            cudaGetLastError();
            return from_cuda(e);
        }
    }
    if (J_out) *J_out = p->last_J;
    if (pairs_out) *pairs_out = p->last_pairs;
    if (empty_out) *empty_out = p->last_empty;
    return RSOT_OK;
}

rsot_status rsot_log_integrated_D(rsot_problem *p, double *lnD_out) {
    if (!p || !lnD_out || p->last_kind < 0) return RSOT_ERR_ARG;
    double *L = nullptr;
    cudaError_t e = cudaMallocAsync(&L, (size_t)p->nq * sizeof(double), p->stream);
    if (!e) e = (p->last_kind == 3) ? trunc_point_L(p, L) : launch_point_L(p, L);
    if (!e) e = launch_log_D(p, L, lnD_out);
    if (L) cudaFreeAsync(L, p->stream);
    if (!e) e = cudaStreamSynchronize(p->stream);
    if (e) {
        cudaGetLastError();
        return from_cuda(e);
    }
    return RSOT_OK;
}

rsot_status rsot_kernel_timing(rsot_problem *p, int enable) {
    if (!p) return RSOT_ERR_ARG;
    p->timing = enable ? 1 : 0;
    if (enable) {
        p->tr_names.clear();
        p->tr_total_ms.clear();
        p->tr_count.clear();
    }
    return RSOT_OK;
}

int rsot_kernel_times(rsot_problem *p, const char **names, double *total_ms, int64_t *launches,
                      int max) {
    if (!p) return 0;
    const int k = (int)p->tr_names.size();
    for (int i = 0; i < k && i < max; ++i) {
        if (names) names[i] = p->tr_names[i];
        if (total_ms) total_ms[i] = p->tr_total_ms[i];
        if (launches) launches[i] = p->tr_count[i];
    }
    return k;
}

rsot_status rsot_point_log_partition(rsot_problem *p, double *L_out) {
    if (!p || !L_out || p->last_kind < 0) return RSOT_ERR_ARG;
    const bool ddev = is_device_ptr(L_out);
    double *tgt = ddev ? L_out : nullptr;
    cudaError_t e = cudaSuccess;
    if (!ddev) e = cudaMallocAsync(&tgt, (size_t)p->nq * 8, p->stream);
    // the mixed truncated path keeps R_q in its sorted grid order; every other
    // path in lse_buf
    if (!e) e = (p->last_kind == 3) ? trunc_point_L(p, tgt) : launch_point_L(p, tgt);
    if (!e && !ddev)
        e = cudaMemcpyAsync(L_out, tgt, (size_t)p->nq * 8, cudaMemcpyDeviceToHost, p->stream);
    if (!ddev && tgt) cudaFreeAsync(tgt, p->stream);
    if (!e) e = cudaStreamSynchronize(p->stream);
    if (e) {
        cudaGetLastError();
        return from_cuda(e);
    }
    return RSOT_OK;
}

// Runs a dense mixed evaluation at (psi, eps) -- its records feed the maps and
// centroid kernels -- then `what` (0: maps, 1: centroids) into device or host
// outputs.
static rsot_status plan_sums(rsot_problem *p, const double *psi, double eps, int what, double *T_out,
                             int64_t *j_out, double *mass_out) {
    double J = 0.0;
    rsot_status s = rsot_eval_dual_grad(p, psi, eps, 0.0, RSOT_MIXED, &J, p->grad_dev, nullptr);
    if (s) return s;
    cudaStream_t st = p->stream;
    const int64_t rows = what == 0 ? p->nq : p->n;
    const size_t tb = (size_t)rows * p->d * sizeof(double);
    const bool tdev = !T_out || is_device_ptr(T_out);
    const bool jdev = !j_out || is_device_ptr(j_out);
    const bool mdev = !mass_out || is_device_ptr(mass_out);
    double *Td = tdev ? T_out : nullptr, *md = mdev ? mass_out : nullptr, *org = nullptr;
    int64_t *jd = jdev ? j_out : nullptr;
    cudaError_t e = cudaMallocAsync(&org, 3 * sizeof(double), st);
    if (!e) e = cudaMemcpyAsync(org, p->origin, 3 * sizeof(double), cudaMemcpyHostToDevice, st);
    if (!e && !tdev) e = cudaMallocAsync(&Td, tb, st);
    if (!e && !jdev) e = cudaMallocAsync(&jd, (size_t)rows * sizeof(int64_t), st);
    if (!e && !mdev) e = cudaMallocAsync(&md, (size_t)rows * sizeof(double), st);
    if (!e) {
        trace_begin(p, what == 0 ? "maps" : "centroids");
        e = what == 0 ? launch_maps(p, eps, Td, jd, org) : launch_centroids(p, Td, md, org);
        trace_end(p);
    }
    if (!e && !tdev) e = cudaMemcpyAsync(T_out, Td, tb, cudaMemcpyDeviceToHost, st);
    if (!e && !jdev) e = cudaMemcpyAsync(j_out, jd, (size_t)rows * sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (!e && !mdev) e = cudaMemcpyAsync(mass_out, md, (size_t)rows * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (org) cudaFreeAsync(org, st);
    if (!tdev && Td) cudaFreeAsync(Td, st);
    if (!jdev && jd) cudaFreeAsync(jd, st);
    if (!mdev && md) cudaFreeAsync(md, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e) {
        cudaGetLastError();
        p->tr_open.clear();
        p->tr_used = 0;
        return from_cuda(e);
    }
    trace_collect(p);
    return RSOT_OK;
}

rsot_status rsot_transport_maps(rsot_problem *p, const double *psi, double eps, double *T_out,
                                int64_t *jstar_out) {
    if (!p || !psi || (!T_out && !jstar_out) || !(eps > 0.0) || !isfinite(eps)) return RSOT_ERR_ARG;
    return plan_sums(p, psi, eps, 0, T_out, jstar_out, nullptr);
}

rsot_status rsot_centroids(rsot_problem *p, const double *psi, double eps, double *T_out,
                           double *mass_out) {
    if (!p || !psi || !T_out || !(eps > 0.0) || !isfinite(eps)) return RSOT_ERR_ARG;
    return plan_sums(p, psi, eps, 1, T_out, nullptr, mass_out);
}

rsot_status rsot_covering_cost(rsot_problem *p, double *C0_out) {
    if (!p || !C0_out) return RSOT_ERR_ARG;
    if (p->C0 < 0.0) {
        double *aux = reinterpret_cast<double *>(p->res_dev + 1);
        cudaError_t e = launch_covering_cost(p, aux);
        double v = 0.0;
        if (!e) e = cudaMemcpyAsync(&v, aux, 8, cudaMemcpyDeviceToHost, p->stream);
        if (!e) e = cudaStreamSynchronize(p->stream);
        if (e) {
            cudaGetLastError();
            return from_cuda(e);
        }
        p->C0 = v;
    }
    *C0_out = p->C0;
    return RSOT_OK;
}

// max and min of a potential (host or device memory)
static rsot_status psi_range(rsot_problem *p, const double *psi, double *mx_out, double *mn_out) {
    double mx = -INFINITY, mn = INFINITY;
    const int w = where_ptr(psi);
    if (w < 0) return RSOT_ERR_ARG;
    if (w == 1) {
        double *aux = reinterpret_cast<double *>(p->res_dev + 1) + 2;
        double h[2];
        cudaError_t e = launch_psi_stats(p, psi, aux);
        if (!e) e = cudaMemcpyAsync(h, aux, 16, cudaMemcpyDeviceToHost, p->stream);
        if (!e) e = cudaStreamSynchronize(p->stream);
        if (e) {
            cudaGetLastError();
            return from_cuda(e);
        }
        mx = h[0];
        mn = h[1];
    } else {
        for (int64_t j = 0; j < p->n; ++j) {
            if (!isfinite(psi[j])) return RSOT_ERR_NONFINITE;
            mx = std::max(mx, psi[j]);
            mn = std::min(mn, psi[j]);
        }
    }
    if (!isfinite(mx) || !isfinite(mn)) return RSOT_ERR_NONFINITE;
    *mx_out = mx;
    *mn_out = mn;
    return RSOT_OK;
}

rsot_status rsot_truncation_cutoff(rsot_problem *p, const double *psi, double eps, int kind,
                                   double param, double J, double lnD, double *C_out) {
    if (!p || !psi || !C_out || !(eps > 0.0) || !isfinite(eps) || !(param > 0.0)) return RSOT_ERR_ARG;
    if (kind < RSOT_CUTOFF_POINTWISE || kind > RSOT_CUTOFF_TAIL) return RSOT_ERR_ARG;
    if ((kind == RSOT_CUTOFF_INTEGRAL || kind == RSOT_CUTOFF_GEOMETRIC) && !(fabs(J) > 0.0))
        return RSOT_ERR_ARG;
    if (kind == RSOT_CUTOFF_TAIL && !(param < 1.0)) return RSOT_ERR_ARG;
    double mx = 0.0, mn = 0.0, C0 = 0.0;
    rsot_status s = psi_range(p, psi, &mx, &mn);
    if (s) return s;
    if (kind == RSOT_CUTOFF_GEOMETRIC || kind == RSOT_CUTOFF_TAIL)
        if ((s = rsot_covering_cost(p, &C0))) return s;
    double C = 0.0;
    switch (kind) {
        case RSOT_CUTOFF_POINTWISE:   // Eq. cost_cutoff_delta
            C = mx + eps * log(p->nu_max / param);
            break;
        case RSOT_CUTOFF_INTEGRAL:    // Eq. truncation_cutoff_int
            C = mx + eps * (log(eps) + lnD - log(param) - log(fabs(J)));
            break;
        case RSOT_CUTOFF_GEOMETRIC:   // Eq. truncation_cutoff_geom
            C = std::max(C0, C0 + (mx - mn) + eps * log(eps / (p->nu_min * param * fabs(J))));
            break;
        default:                      // the pointwise reading of App. B (tail)
            C = C0 + (mx - mn) + eps * log(1.0 / (p->nu_min * param));
    }
    if (isnan(C)) return RSOT_ERR_NONFINITE;
    *C_out = C;
    return RSOT_OK;
}

rsot_status rsot_radius_for_tail(rsot_problem *p, const double *psi, double eps, double tail,
                                 double *radius_out) {
    if (!p || !psi || !radius_out || !(eps > 0.0) || !(tail > 0.0) || !(tail < 1.0))
        return RSOT_ERR_ARG;
    double C = 0.0;
    rsot_status s = rsot_truncation_cutoff(p, psi, eps, RSOT_CUTOFF_TAIL, tail, 0.0, 0.0, &C);
    if (s) return s;
    *radius_out = sqrt(2.0 * C);
    return RSOT_OK;
}

}  // extern "C"
