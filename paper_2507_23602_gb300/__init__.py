"""Python binding of librsot (GB300 / sm_103a) -- argument marshalling only.

Every step of the dual evaluation and of the solver runs in librsot.so (CUDA
kernels plus the host L-BFGS driver in C++).  This module only converts
arrays to pointers and status codes to exceptions.  It never computes the
method on the CPU: when the library is missing, ``load()`` raises.

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA);
CUDA tensors are passed as device pointers, so device-resident inputs and
outputs stay on the GPU.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Optional

import numpy as np

__all__ = ["load", "lib_path", "RsotError", "Problem", "Batch", "MLP", "SolveOptions", "SolveStats",
           "FP64", "MIXED", "COMPENSATED", "COMPENSATED_GRAD_REL", "PAIRS_FP32", "PAIRS_TENSOR", "PAIRS_AUTO", "STATUS", "probe_ex2_rate", "probe_dfma_rate",
           "GEMM_TCGEN05", "GEMM_MMA_SYNC"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "librsot.so")
_lib = None

FP64, MIXED, COMPENSATED = 0, 1, 2
# ||g - grad J||_1 <= COMPENSATED_GRAD_REL * sum_q m_q for a COMPENSATED gradient
COMPENSATED_GRAD_REL = 6.5e-7
PAIRS_FP32, PAIRS_TENSOR, PAIRS_AUTO = 0, 1, 2
# cost cutoffs of Sec. 4.1 (rsot_truncation_cutoff)
CUTOFF_POINTWISE, CUTOFF_INTEGRAL, CUTOFF_GEOMETRIC, CUTOFF_TAIL = 0, 1, 2, 3
# GEMM kernels of the warm-start network (rsot_mlp_set_gemm_kernel)
GEMM_TCGEN05, GEMM_MMA_SYNC, GEMM_TCGEN05_CPASYNC = 0, 1, 2
STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "non-finite value",
          4: "empty neighbourhood", 5: "not converged", 6: "line search failed",
          7: "device wait timed out", 8: "out of device memory"}
RSOT_ERR_EMPTY_NEIGHBORHOOD = 4
# limits of the allocation-free entry point rsot_eval_dense_noalloc
NOALLOC_MAX_NQ, NOALLOC_MAX_N, NOALLOC_SCRATCH_BYTES = 524288, 65536, 60393984


class RsotError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = int(status)
        super().__init__(f"librsot: {what}: {STATUS.get(self.status, self.status)} ({self.status})")


class _Options(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("eps_start", ctypes.c_double),
                ("eps_factor", ctypes.c_double), ("tail", ctypes.c_double),
                ("tol_l1", ctypes.c_double), ("stage_tol_l1", ctypes.c_double),
                ("precision", ctypes.c_int), ("refine_fp64", ctypes.c_int),
                ("lbfgs_m", ctypes.c_int), ("max_iter", ctypes.c_int), ("verbose", ctypes.c_int),
                ("mixed_tol_l1", ctypes.c_double), ("refine_precision", ctypes.c_int),
                ("tau_int", ctypes.c_double), ("delta_pw", ctypes.c_double),
                ("tau_geom", ctypes.c_double)]


class _Desc(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("nq", ctypes.c_int64), ("x", ctypes.c_void_p),
                ("mass", ctypes.c_void_p), ("n", ctypes.c_int64), ("y", ctypes.c_void_p),
                ("nu", ctypes.c_void_p)]


class _BStats(ctypes.Structure):
    _fields_ = [("seconds", ctypes.c_double), ("seconds_mixed", ctypes.c_double),
                ("seconds_refine", ctypes.c_double), ("rounds", ctypes.c_int),
                ("converged", ctypes.c_int), ("max_grad_l1", ctypes.c_double),
                ("evals", ctypes.c_int64), ("evals_prec", ctypes.c_int64 * 3),
                ("pairs_prec", ctypes.c_int64 * 3)]


class _SrcLevel(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("nq", ctypes.c_int64), ("x", ctypes.c_void_p),
                ("mass", ctypes.c_void_p)]


class _TgtLevel(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("y", ctypes.c_void_p), ("nu", ctypes.c_void_p)]


MAX_LEVELS = 16


class _MLStats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("src_level", ctypes.c_int * MAX_LEVELS),
                ("tgt_level", ctypes.c_int * MAX_LEVELS), ("transfer", ctypes.c_int * MAX_LEVELS),
                ("iters", ctypes.c_int * MAX_LEVELS), ("evals", ctypes.c_int * MAX_LEVELS),
                ("seconds", ctypes.c_double * MAX_LEVELS), ("grad_l1", ctypes.c_double),
                ("total_seconds", ctypes.c_double)]


class _BaryStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("rms_last", ctypes.c_double),
                ("solve_iters", ctypes.c_int), ("solve_evals", ctypes.c_int),
                ("seconds_solve", ctypes.c_double), ("seconds_centroids", ctypes.c_double),
                ("seconds_total", ctypes.c_double)]


class _Stats(ctypes.Structure):
    _fields_ = [("J", ctypes.c_double), ("grad_l1", ctypes.c_double), ("iters", ctypes.c_int),
                ("evals", ctypes.c_int), ("stages", ctypes.c_int), ("pairs", ctypes.c_int64),
                ("seconds", ctypes.c_double), ("evals_prec", ctypes.c_int * 3),
                ("pairs_prec", ctypes.c_int64 * 3)]


@dataclasses.dataclass
class SolveOptions:
    eps: float = 1e-2
    eps_start: float = 0.0
    eps_factor: float = 0.5
    tail: float = 0.0
    tol_l1: float = 1e-6
    stage_tol_l1: float = 0.0
    precision: int = MIXED
    refine_fp64: bool = True
    lbfgs_m: int = 10
    max_iter: int = 10000
    verbose: bool = False
    mixed_tol_l1: float = 1e-5
    refine_precision: int = COMPENSATED
    tau_int: float = 0.0
    delta_pw: float = 0.0
    tau_geom: float = 0.0

    def _c(self):
        return _Options(self.eps, self.eps_start, self.eps_factor, self.tail, self.tol_l1,
                        self.stage_tol_l1, int(self.precision), int(bool(self.refine_fp64)),
                        int(self.lbfgs_m), int(self.max_iter), int(bool(self.verbose)),
                        float(self.mixed_tol_l1), int(self.refine_precision), float(self.tau_int),
                        float(self.delta_pw), float(self.tau_geom))


@dataclasses.dataclass
class SolveStats:
    status: int
    J: float
    grad_l1: float
    iters: int
    evals: int
    stages: int
    pairs: int
    seconds: float
    evals_prec: tuple = (0, 0, 0)   # by precision: FP64, MIXED, COMPENSATED
    pairs_prec: tuple = (0, 0, 0)


def lib_path() -> str:
    return _LIB_PATH


def load():
    """Load librsot.so (built in-tree by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"librsot.so is not built ({_LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(_LIB_PATH)
    vp, dp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)
    lib.rsot_status_string.restype = ctypes.c_char_p
    lib.rsot_status_string.argtypes = [ctypes.c_int]
    lib.rsot_version.restype = ctypes.c_char_p
    lib.rsot_create.argtypes = [ctypes.c_int, ctypes.c_int64, vp, vp, ctypes.c_int64, vp, vp,
                                ctypes.c_int, ctypes.POINTER(vp)]
    lib.rsot_destroy.argtypes = [vp]
    lib.rsot_destroy.restype = None
    lib.rsot_set_stream.argtypes = [vp, vp]
    lib.rsot_set_pair_kernel.argtypes = [vp, ctypes.c_int]
    lib.rsot_eval_dual_grad.argtypes = [vp, vp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                        dp, vp, i64p]
    lib.rsot_eval_dual_grad_tail.argtypes = [vp, vp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                        dp, vp, i64p]
    lib.rsot_log_integrated_D.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    lib.rsot_last_eval.argtypes = [vp, dp, vp, i64p, i64p]
    lib.rsot_covering_cost.argtypes = [vp, dp]
    lib.rsot_point_log_partition.argtypes = [vp, vp]
    lib.rsot_radius_for_tail.argtypes = [vp, vp, ctypes.c_double, ctypes.c_double, dp]
    lib.rsot_truncation_cutoff.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, dp]
    lib.rsot_default_options.argtypes = [ctypes.POINTER(_Options)]
    lib.rsot_default_options.restype = None
    lib.rsot_solve.argtypes = [vp, dp, ctypes.POINTER(_Options), ctypes.POINTER(_Stats)]
    lib.rsot_kernel_timing.argtypes = [vp, ctypes.c_int]
    lib.rsot_kernel_times.argtypes = [vp, ctypes.POINTER(ctypes.c_char_p), dp, i64p, ctypes.c_int]
    lib.rsot_kernel_times.restype = ctypes.c_int
    lib.rsot_probe_ex2_rate.argtypes = [ctypes.c_int, dp]
    lib.rsot_probe_dfma_rate.argtypes = [ctypes.c_int, dp]
    lib.rsot_exp64.argtypes = [ctypes.c_int64, vp, vp]
    lib.rsot_selftest_wait_timeout.argtypes = [ctypes.c_longlong, vp]
    lib.rsot_kmeans.argtypes = [ctypes.c_int, ctypes.c_int64, vp, vp, ctypes.c_int64, ctypes.c_int,
                                ctypes.c_uint64, dp, dp, i64p]
    lib.rsot_softmax_refine.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int64, vp, vp]
    lib.rsot_multilevel_solve.argtypes = [ctypes.c_int, ctypes.POINTER(_SrcLevel), ctypes.c_int,
                                          ctypes.POINTER(_TgtLevel), dp, ctypes.POINTER(_Options),
                                          dp, ctypes.POINTER(_MLStats)]
    lib.rsot_transport_maps.argtypes = [vp, vp, ctypes.c_double, vp, vp]
    lib.rsot_centroids.argtypes = [vp, vp, ctypes.c_double, vp, vp]
    lib.rsot_barycenter.argtypes = [ctypes.c_int, ctypes.POINTER(_SrcLevel), dp, ctypes.c_int64, dp,
                                    dp, ctypes.POINTER(_Options), ctypes.c_double, ctypes.c_int,
                                    ctypes.c_double, ctypes.POINTER(_BaryStats)]
    fp = ctypes.POINTER(ctypes.c_float)
    lib.rsot_mlp_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(vp)]
    lib.rsot_mlp_destroy.argtypes = [vp]
    lib.rsot_mlp_destroy.restype = None
    lib.rsot_mlp_set_stream.argtypes = [vp, vp]
    lib.rsot_mlp_set_gemm_kernel.argtypes = [vp, ctypes.c_int]
    lib.rsot_mlp_num_params.argtypes = [vp]
    lib.rsot_mlp_num_params.restype = ctypes.c_int64
    lib.rsot_mlp_get_params.argtypes = [vp, vp]
    lib.rsot_mlp_set_params.argtypes = [vp, vp]
    lib.rsot_mlp_forward.argtypes = [vp, ctypes.c_int64, vp, vp]
    lib.rsot_mlp_gradients.argtypes = [vp, ctypes.c_int64, vp, vp, fp, vp]
    lib.rsot_mlp_train_step.argtypes = [vp, ctypes.c_int64, vp, vp, ctypes.c_float, fp]
    lib.rsot_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(_Desc), ctypes.POINTER(vp)]
    lib.rsot_batch_destroy.argtypes = [vp]
    lib.rsot_batch_destroy.restype = None
    lib.rsot_batch_total_targets.argtypes = [vp]
    lib.rsot_batch_total_targets.restype = ctypes.c_int64
    lib.rsot_batch_eval.argtypes = [vp, dp, dp, ctypes.c_char_p, dp, dp]
    lib.rsot_batch_tune.argtypes = [vp, dp, dp, ctypes.POINTER(ctypes.c_int)]
    lib.rsot_batch_set_pair_kernel.argtypes = [vp, ctypes.c_int]
    lib.rsot_batch_solve.argtypes = [vp, dp, dp, ctypes.POINTER(_Options),
                                     ctypes.POINTER(ctypes.c_int), dp, ctypes.POINTER(_BStats)]
    _lib = lib
    return lib


def probe_ex2_rate(iters: int = 20000) -> float:
    """Measured ex2.approx results per second of the current device."""
    v = ctypes.c_double()
    _check(load().rsot_probe_ex2_rate(int(iters), ctypes.byref(v)), "probe_ex2_rate")
    return v.value


def probe_dfma_rate(iters: int = 4000) -> float:
    """Measured FP64 fused multiply-adds per second of the current device."""
    v = ctypes.c_double()
    _check(load().rsot_probe_dfma_rate(int(iters), ctypes.byref(v)), "probe_dfma_rate")
    return v.value


def _ptr(a):
    """(pointer, keep-alive object) for a numpy array or a torch tensor (float64)."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float64:
                a = a.to(torch.float64)
            a = a.contiguous()
            return ctypes.c_void_p(a.data_ptr()), a
    except ImportError:
        pass
    a = np.ascontiguousarray(a, dtype=np.float64)
    return ctypes.c_void_p(a.ctypes.data), a


def _is_cuda(a):
    try:
        import torch
        return isinstance(a, torch.Tensor) and a.is_cuda
    except ImportError:
        return False


def _check(st, what):
    if st != 0:
        raise RsotError(st, what)


class Problem:
    """An RSOT problem held on the GPU: quadrature points x (nq, d), masses
    (nq,), targets y (n, d), weights nu (n,).  With borrow=True the four
    arrays must be CUDA float64 tensors of the current device: the handle
    reads mass and nu in place (this object keeps them alive) instead of
    copying them."""

    def __init__(self, x, mass, y, nu, stream=None, borrow=False):
        lib = load()
        d = int(x.shape[1])
        self.d, self.nq, self.n = d, int(x.shape[0]), int(y.shape[0])
        px, kx = _ptr(x)
        pm, km = _ptr(mass)
        py, ky = _ptr(y)
        pn, kn = _ptr(nu)
        h = ctypes.c_void_p()
        _check(lib.rsot_create(d, self.nq, px, pm, self.n, py, pn, int(bool(borrow)),
                               ctypes.byref(h)), "create")
        self._borrowed = (km, kn) if borrow else None
        self._h = h
        self._lib = lib
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            except ImportError:
                stream = None
        self.set_stream(stream)

    def set_stream(self, stream):
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        _check(self._lib.rsot_set_stream(self._h, ctypes.c_void_p(s or 0)), "set_stream")

    def set_pair_kernel(self, kind):
        """PAIRS_AUTO (default), PAIRS_TENSOR or PAIRS_FP32 for the mixed dense passes."""
        _check(self._lib.rsot_set_pair_kernel(self._h, int(kind)), "set_pair_kernel")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.rsot_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def eval(self, psi, eps, radius=0.0, precision=MIXED, grad_out=None, allow_empty=False):
        """(J, grad, pairs): Eq. discretized_functional / discretized_gradient,
        dense when radius <= 0, else truncated at |x - y| < radius."""
        pp, kp = _ptr(psi)
        if grad_out is None:
            if _is_cuda(psi):
                import torch
                grad_out = torch.empty(self.n, dtype=torch.float64, device=psi.device)
            else:
                grad_out = np.empty(self.n)
        pg, kg = _ptr(grad_out)
        J = ctypes.c_double()
        pairs = ctypes.c_int64()
        st = self._lib.rsot_eval_dual_grad(self._h, pp, float(eps), float(radius), int(precision),
                                           ctypes.byref(J), pg, ctypes.byref(pairs))
        if allow_empty and st == RSOT_ERR_EMPTY_NEIGHBORHOOD:
            # the outputs are untouched on that status: the evaluation with the
            # empty points skipped comes from rsot_last_eval
            _check(self._lib.rsot_last_eval(self._h, ctypes.byref(J), pg, ctypes.byref(pairs), None),
                   "last_eval")
            st = 0
        if st != 0:
            raise RsotError(st, "eval_dual_grad")
        return J.value, grad_out, pairs.value

    def last_eval(self, grad_out=None):
        """(J, grad, pairs, empty) of the last evaluation whose passes completed,
        including one that skipped points without a target (Algorithm 2)."""
        if grad_out is None:
            grad_out = np.empty(self.n)
        pg, kg = _ptr(grad_out)
        J = ctypes.c_double()
        pairs = ctypes.c_int64()
        empty = ctypes.c_int64()
        _check(self._lib.rsot_last_eval(self._h, ctypes.byref(J), pg, ctypes.byref(pairs),
                                        ctypes.byref(empty)), "last_eval")
        return J.value, grad_out, pairs.value, empty.value

    def eval_tail(self, psi, eps, tail, precision=MIXED, grad_out=None):
        """(J, grad, pairs): Algorithm 2 truncated by the psi-aware cutoffs
        c(x_q, y_j) < alpha_q + beta_j of the given tail tolerance."""
        pp, kp = _ptr(psi)
        if grad_out is None:
            if _is_cuda(psi):
                import torch
                grad_out = torch.empty(self.n, dtype=torch.float64, device=psi.device)
            else:
                grad_out = np.empty(self.n)
        pg, kg = _ptr(grad_out)
        J = ctypes.c_double()
        pairs = ctypes.c_int64()
        st = self._lib.rsot_eval_dual_grad_tail(self._h, pp, float(eps), float(tail), int(precision),
                                                ctypes.byref(J), pg, ctypes.byref(pairs))
        if st != 0:
            raise RsotError(st, "eval_dual_grad_tail")
        return J.value, grad_out, pairs.value

    def log_integrated_D(self):
        """ln D = ln sum_q m_q / S_trunc(x_q) of the last evaluation (Sec. 4.1)."""
        v = ctypes.c_double()
        _check(self._lib.rsot_log_integrated_D(self._h, ctypes.byref(v)), "log_integrated_D")
        return v.value

    def point_log_partition(self, out=None):
        """L_q of the last evaluation (numpy unless `out` is given)."""
        if out is None:
            out = np.empty(self.nq)
        po, ko = _ptr(out)
        _check(self._lib.rsot_point_log_partition(self._h, po), "point_log_partition")
        return out

    def transport_maps(self, psi, eps, bary=True, modal=True):
        """Sec. 6.3: (T_bary [nq, d] or None, j* [nq] int64 or None); the modal
        map is y[j*]."""
        pp, kp = _ptr(psi)
        T = np.empty((self.nq, self.d)) if bary else None
        js = np.empty(self.nq, dtype=np.int64) if modal else None
        _check(self._lib.rsot_transport_maps(self._h, pp, float(eps),
                                             ctypes.c_void_p(T.ctypes.data) if bary else None,
                                             ctypes.c_void_p(js.ctypes.data) if modal else None),
               "transport_maps")
        return T, js

    def centroids(self, psi, eps):
        """Eq. barycenter_fixed_point: (T [n, d], transported mass a [n])."""
        pp, kp = _ptr(psi)
        T = np.empty((self.n, self.d))
        a = np.empty(self.n)
        _check(self._lib.rsot_centroids(self._h, pp, float(eps), ctypes.c_void_p(T.ctypes.data),
                                        ctypes.c_void_p(a.ctypes.data)), "centroids")
        return T, a

    def softmax_refine(self, psi_coarse, eps, y_fine):
        """Initial potential on the targets y_fine from psi_coarse on this
        problem's targets (Eq. softmax_refinement_formula)."""
        pc, kc = _ptr(psi_coarse)
        yf = np.ascontiguousarray(y_fine, dtype=np.float64)
        out = np.empty(yf.shape[0])
        _check(self._lib.rsot_softmax_refine(self._h, pc, float(eps), yf.shape[0],
                                             ctypes.c_void_p(yf.ctypes.data),
                                             ctypes.c_void_p(out.ctypes.data)), "softmax_refine")
        return out

    def kernel_timing(self, enable=True):
        """Bracket every library kernel with CUDA events (clears the totals)."""
        _check(self._lib.rsot_kernel_timing(self._h, int(bool(enable))), "kernel_timing")

    def kernel_times(self):
        """{kernel name: (total ms, launches)} accumulated while timing was on."""
        k = self._lib.rsot_kernel_times(self._h, None, None, None, 0)
        names = (ctypes.c_char_p * max(k, 1))()
        tot = (ctypes.c_double * max(k, 1))()
        cnt = (ctypes.c_int64 * max(k, 1))()
        self._lib.rsot_kernel_times(self._h, names, tot, cnt, k)
        return {names[i].decode(): (tot[i], cnt[i]) for i in range(k)}

    def covering_cost(self):
        v = ctypes.c_double()
        _check(self._lib.rsot_covering_cost(self._h, ctypes.byref(v)), "covering_cost")
        return v.value

    def truncation_cutoff(self, psi, eps, kind, param, J=0.0, lnD=0.0):
        """Cost cutoff C of Sec. 4.1 (kind: CUTOFF_POINTWISE, CUTOFF_INTEGRAL,
        CUTOFF_GEOMETRIC, CUTOFF_TAIL); the truncated evaluation keeps
        c(x, y) < C, i.e. radius sqrt(2 C)."""
        pp, kp = _ptr(psi)
        v = ctypes.c_double()
        _check(self._lib.rsot_truncation_cutoff(self._h, pp, float(eps), int(kind), float(param),
                                                float(J), float(lnD), ctypes.byref(v)),
               "truncation_cutoff")
        return v.value

    def radius_for_tail(self, psi, eps, tail):
        pp, kp = _ptr(psi)
        v = ctypes.c_double()
        _check(self._lib.rsot_radius_for_tail(self._h, pp, float(eps), float(tail), ctypes.byref(v)),
               "radius_for_tail")
        return v.value

    def solve(self, psi0=None, options: Optional[SolveOptions] = None, raise_on_error=True, **kw):
        """FP64 L-BFGS (host) over GPU evaluations; returns (psi, SolveStats)."""
        opts = options or SolveOptions(**kw)
        psi = np.zeros(self.n) if psi0 is None else np.array(psi0, dtype=np.float64, copy=True)
        o = opts._c()
        s = _Stats()
        st = self._lib.rsot_solve(self._h, psi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  ctypes.byref(o), ctypes.byref(s))
        stats = SolveStats(st, s.J, s.grad_l1, s.iters, s.evals, s.stages, s.pairs, s.seconds,
                           tuple(s.evals_prec), tuple(s.pairs_prec))
        if raise_on_error and st != 0:
            raise RsotError(st, "solve")
        return psi, stats


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Batch:
    """Many RSOT problems evaluated and solved together.  `problems` is a list of
    (x, mass, y, nu) tuples (numpy, host).  Potentials and gradients are the
    concatenation of the problems' vectors in list order."""

    def __init__(self, problems):
        lib = load()
        self._lib = lib
        self._keep = []
        descs = (_Desc * len(problems))()
        self.sizes = []
        for i, (x, m, y, nu) in enumerate(problems):
            arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, m, y, nu)]
            self._keep.append(arrs)
            x, m, y, nu = arrs
            descs[i] = _Desc(x.shape[1], x.shape[0], x.ctypes.data, m.ctypes.data, y.shape[0],
                             y.ctypes.data, nu.ctypes.data)
            self.sizes.append(y.shape[0])
        h = ctypes.c_void_p()
        _check(lib.rsot_batch_create(len(problems), descs, ctypes.byref(h)), "batch_create")
        self._keep = None
        self._h = h
        self.count = len(problems)
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        self.total = int(lib.rsot_batch_total_targets(h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.rsot_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def split(self, v):
        return [v[self.offsets[i]:self.offsets[i + 1]] for i in range(self.count)]

    def set_pair_kernel(self, kind):
        """PAIRS_AUTO (default), PAIRS_TENSOR or PAIRS_FP32 for the batched passes."""
        _check(self._lib.rsot_batch_set_pair_kernel(self._h, int(kind)), "batch_set_pair_kernel")

    def eval(self, psi_all, eps, active=None):
        psi_all = np.ascontiguousarray(psi_all, dtype=np.float64)
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        J = np.full(self.count, np.nan)
        g = np.full(self.total, np.nan)
        act = None if active is None else bytes(np.asarray(active, dtype=np.uint8))
        _check(self._lib.rsot_batch_eval(self._h, _dp(psi_all), _dp(eps), act, _dp(J), _dp(g)),
               "batch_eval")
        return J, g

    def tune(self, psi_all, eps):
        psi_all = np.ascontiguousarray(psi_all, dtype=np.float64)
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        c = ctypes.c_int()
        _check(self._lib.rsot_batch_tune(self._h, _dp(psi_all), _dp(eps), ctypes.byref(c)),
               "batch_tune")
        return c.value

    def solve(self, eps, psi0=None, options: Optional[SolveOptions] = None, raise_on_error=True,
              **kw):
        opts = options or SolveOptions(**kw)
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        psi = np.zeros(self.total) if psi0 is None else np.array(psi0, dtype=np.float64)
        st = (ctypes.c_int * self.count)()
        gl1 = np.zeros(self.count)
        s = _BStats()
        o = opts._c()
        rc = self._lib.rsot_batch_solve(self._h, _dp(psi), _dp(eps), ctypes.byref(o), st,
                                        _dp(gl1), ctypes.byref(s))
        if raise_on_error and rc != 0:
            raise RsotError(rc, "batch_solve")
        stats = {"status": rc, "statuses": list(st), "grad_l1": gl1, "seconds": s.seconds,
                 "seconds_mixed": s.seconds_mixed, "seconds_refine": s.seconds_refine,
                 "rounds": s.rounds, "converged": s.converged, "max_grad_l1": s.max_grad_l1,
                 "evals": s.evals, "evals_prec": list(s.evals_prec),
                 "pairs_prec": list(s.pairs_prec)}
        return psi, stats


def kmeans(y, w, k, iters=20, seed=6):
    """(centres, weights, assignment) of a weighted k-means (GPU assignment)."""
    lib = load()
    y = np.ascontiguousarray(y, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    d = y.shape[1]
    C = np.empty((k, d))
    W = np.empty(k)
    a = np.empty(y.shape[0], dtype=np.int64)
    _check(lib.rsot_kmeans(d, y.shape[0], ctypes.c_void_p(y.ctypes.data), ctypes.c_void_p(w.ctypes.data),
                           int(k), int(iters), int(seed), _dp(C), _dp(W),
                           a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))), "kmeans")
    return C, W, a


def multilevel_solve(sources, targets, eps_levels, options: Optional[SolveOptions] = None,
                     raise_on_error=True, **kw):
    """Combined multilevel solve (Sec. 5.3).  sources: list of (x, mass) coarse
    to fine; targets: list of (y, nu) coarse to fine; eps_levels: L_max + 1."""
    lib = load()
    keep = []
    S = (_SrcLevel * len(sources))()
    for i, (x, m) in enumerate(sources):
        x = np.ascontiguousarray(x, dtype=np.float64)
        m = np.ascontiguousarray(m, dtype=np.float64)
        keep += [x, m]
        S[i] = _SrcLevel(x.shape[1], x.shape[0], x.ctypes.data, m.ctypes.data)
    T = (_TgtLevel * len(targets))()
    for i, (y, nu) in enumerate(targets):
        y = np.ascontiguousarray(y, dtype=np.float64)
        nu = np.ascontiguousarray(nu, dtype=np.float64)
        keep += [y, nu]
        T[i] = _TgtLevel(y.shape[0], y.ctypes.data, nu.ctypes.data)
    eps = np.ascontiguousarray(eps_levels, dtype=np.float64)
    opts = options or SolveOptions(**kw)
    o = opts._c()
    psi = np.zeros(T[len(targets) - 1].n)
    st = _MLStats()
    rc = lib.rsot_multilevel_solve(len(sources), S, len(targets), T, _dp(eps), ctypes.byref(o),
                                   _dp(psi), ctypes.byref(st))
    if raise_on_error and rc != 0:
        raise RsotError(rc, "multilevel_solve")
    L = st.levels
    stats = {"status": rc, "levels": L, "src_level": list(st.src_level[:L]),
             "tgt_level": list(st.tgt_level[:L]), "transfer": list(st.transfer[:L]),
             "iters": list(st.iters[:L]), "evals": list(st.evals[:L]),
             "seconds": list(st.seconds[:L]), "grad_l1": st.grad_l1,
             "total_seconds": st.total_seconds}
    return psi, stats


def _fptr(a):
    """(pointer, keep) of a float32 numpy array or torch tensor (host or CUDA)."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            a = a.to(torch.float32).contiguous()
            return ctypes.c_void_p(a.data_ptr()), a
    except ImportError:
        pass
    a = np.ascontiguousarray(a, dtype=np.float32)
    return ctypes.c_void_p(a.ctypes.data), a


class MLP:
    """The warm-start network: in_dim -> width (SiLU) x3 -> 1."""

    def __init__(self, in_dim=18, width=256, seed=0, stream=None):
        lib = load()
        self._lib = lib
        h = ctypes.c_void_p()
        _check(lib.rsot_mlp_create(int(in_dim), int(width), int(seed), ctypes.byref(h)), "mlp_create")
        self._h = h
        self.in_dim, self.width = in_dim, width
        self.n_params = int(lib.rsot_mlp_num_params(h))
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            except ImportError:
                stream = None
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        _check(lib.rsot_mlp_set_stream(h, ctypes.c_void_p(s or 0)), "mlp_set_stream")

    def set_gemm_kernel(self, kind):
        """GEMM_TCGEN05 (default: TMA operand copies), GEMM_TCGEN05_CPASYNC or
        GEMM_MMA_SYNC for the layers' GEMMs."""
        _check(self._lib.rsot_mlp_set_gemm_kernel(self._h, int(kind)), "mlp_set_gemm_kernel")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.rsot_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        out = np.empty(self.n_params, dtype=np.float32)
        _check(self._lib.rsot_mlp_get_params(self._h, ctypes.c_void_p(out.ctypes.data)), "mlp_get")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(self._lib.rsot_mlp_set_params(self._h, ctypes.c_void_p(p.ctypes.data)), "mlp_set")

    def forward(self, x, out=None):
        px, kx = _fptr(x)
        rows = int(x.shape[0])
        if out is None:
            out = np.empty(rows, dtype=np.float32)
        po, ko = _fptr(out)
        _check(self._lib.rsot_mlp_forward(self._h, rows, px, po), "mlp_forward")
        return out

    def gradients(self, x, y):
        px, kx = _fptr(x)
        py, ky = _fptr(y)
        g = np.empty(self.n_params, dtype=np.float32)
        loss = ctypes.c_float()
        _check(self._lib.rsot_mlp_gradients(self._h, int(x.shape[0]), px, py, ctypes.byref(loss),
                                            ctypes.c_void_p(g.ctypes.data)), "mlp_gradients")
        return loss.value, g

    def train_step(self, x, y, lr):
        px, kx = _fptr(x)
        py, ky = _fptr(y)
        loss = ctypes.c_float()
        _check(self._lib.rsot_mlp_train_step(self._h, int(x.shape[0]), px, py, float(lr),
                                             ctypes.byref(loss)), "mlp_train_step")
        return loss.value


def barycenter(sources, weights, y0, nu, theta=0.5, max_iter=50, tol_rms=1e-6,
               options: Optional[SolveOptions] = None, raise_on_error=True, **kw):
    """Damped Lloyd barycenter (Sec. 6.2, Eq. damped_lloyd): sources = list of
    (x, mass) of one dimension, weights = lambda_i, y0 (n, d) the initial
    support with fixed weights nu.  Returns (y, stats)."""
    lib = load()
    keep = []
    S = (_SrcLevel * len(sources))()
    for i, (x, m) in enumerate(sources):
        x = np.ascontiguousarray(x, dtype=np.float64)
        m = np.ascontiguousarray(m, dtype=np.float64)
        keep += [x, m]
        S[i] = _SrcLevel(x.shape[1], x.shape[0], x.ctypes.data, m.ctypes.data)
    lam = np.ascontiguousarray(weights, dtype=np.float64)
    y = np.array(y0, dtype=np.float64, order="C", copy=True)
    nu = np.ascontiguousarray(nu, dtype=np.float64)
    opts = options or SolveOptions(**kw)
    o = opts._c()
    st = _BaryStats()
    rc = lib.rsot_barycenter(len(sources), S, _dp(lam), y.shape[0], _dp(y), _dp(nu), ctypes.byref(o),
                             float(theta), int(max_iter), float(tol_rms), ctypes.byref(st))
    if raise_on_error and rc != 0:
        raise RsotError(rc, "barycenter")
    stats = {f: getattr(st, f) for f, _ in _BaryStats._fields_}
    stats["status"] = rc
    return y, stats
