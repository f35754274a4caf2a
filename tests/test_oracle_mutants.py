"""Planted mistakes in the oracle must be caught by its pins.

Each case copies the oracle's C source, plants one plausible mistake (a
dropped term, a wrong sign, a swapped index, a wrong normaliser), builds the
mutant on the CPU and runs the pin checks of ``test_oracle_pins`` against it
through a stand-in module.  A mutant that every pin accepts fails this test.
"""
import ctypes
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from oracle import build as obuild

MUTANTS = {
    "drop_ln_nu": ("s[j] = (psi[j] - c) / eps + log(nu[j]);", "s[j] = (psi[j] - c) / eps;"),
    "sign_of_cost": ("s[j] = (psi[j] - c) / eps + log(nu[j]);", "s[j] = (psi[j] + c) / eps + log(nu[j]);"),
    "drop_psi_nu": ("nadd(&J, -psi[j] * nu[j]);", "(void)0;"),
    "drop_minus_nu": ("nadd(&a, -nu[j]);", "(void)0;"),
    "unnormalised_plan": ("nadd(&g[j], mass[q] * exp(s[j] - lnS));", "nadd(&g[j], mass[q] * exp(s[j] - smax));"),
    "no_eps_in_J": ("nadd(&jpart[t], mass[q] * eps * lnS);", "nadd(&jpart[t], mass[q] * lnS);"),
    "swapped_cost_index": ("double c = cost(d, xq, y + j * d);", "double c = cost(d, xq, y + (n - 1 - j) * d);"),
    "non_strict_cutoff": (": c < cutoff);", ": c <= cutoff + 1e-3);"),
    "mass_not_applied": ("nadd(&g[j], mass[q] * exp(s[j] - lnS));", "nadd(&g[j], exp(s[j] - lnS) / (double)nq);"),
}


def _build_mutant(name):
    src = open(obuild.SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) >= 1, name
    src = src.replace(old, new)
    tmpd = tempfile.mkdtemp(prefix="oracle_mut_")
    cpath = os.path.join(tmpd, "m.c")
    lpath = os.path.join(tmpd, "libm.so")
    open(cpath, "w").write(src)
    subprocess.run(["gcc", "-std=c99", "-O1", "-fPIC", "-shared", cpath, "-o", lpath, "-lm"], check=True)
    return lpath


def _mutant_dual_grad(lpath):
    lib = ctypes.CDLL(lpath)
    dp = ctypes.POINTER(ctypes.c_double)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.oracle_dual_grad.argtypes = [ctypes.c_int, ctypes.c_int64, dp, dp, ctypes.c_int64,
                                     dp, dp, dp, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, dp, dp, i64p, i64p]

    def dual_grad(x, mass, y, nu, psi, eps, cutoff=math.inf, threads=1):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, mass, y, nu, psi)]
        x, mass, y, nu, psi = arrs
        P = lambda a: a.ctypes.data_as(dp)
        g = np.empty(y.shape[0])
        J = ctypes.c_double()
        pr = ctypes.c_int64()
        em = ctypes.c_int64()
        rc = lib.oracle_dual_grad(x.shape[1], x.shape[0], P(x), P(mass), y.shape[0], P(y), P(nu),
                                  P(psi), eps, cutoff, 1, ctypes.byref(J), P(g),
                                  ctypes.byref(pr), ctypes.byref(em))
        assert rc == 0
        return J.value, g, pr.value, em.value
    return dual_grad


def _pins_pass(dual_grad):
    """A compact run of the independent pins; False as soon as one fails."""
    import test_oracle_pins as T
    orig = oracle.dual_grad
    oracle.dual_grad = dual_grad
    try:
        checks = [
            T.test_single_target_closed_form,
            lambda: T.test_gradient_mass_balance(5, 2),
            lambda: T.test_shift_invariance(0.5),
            lambda: T.test_gradient_central_differences(9, 2, 0.05),
            T.test_lse_sandwich,
            T.test_laguerre_limit_small_eps,
            T.test_two_target_1d_closed_form_and_convergence_order,
            T.test_truncation_pairs_match_brute_force_count,
            T.test_cutoff_infinite_is_dense_and_zero_is_empty,
        ]
        for c in checks:
            try:
                c()
            except AssertionError:
                return False
        return True
    finally:
        oracle.dual_grad = orig


def test_unmutated_oracle_passes_compact_pins():
    assert _pins_pass(oracle.dual_grad)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    lpath = _build_mutant(name)
    assert not _pins_pass(_mutant_dual_grad(lpath)), f"mutant {name} passed every pin"


# ---- transport maps and centroids (Sec. 6.2-6.3) ---------------------------
MUTANTS_MAPS = {
    "maps_drop_ln_nu": ("            double s = (psi[j] - cost(d, x + q * d, y + j * d)) / eps + log(nu[j]);\n            if (s > smax) {",
                        "            double s = (psi[j] - cost(d, x + q * d, y + j * d)) / eps;\n            if (s > smax) {"),
    "maps_wrong_coordinate": ("nadd(&W[k], e * y[j * d + k]);", "nadd(&W[k], e * y[j * d]);"),
    "maps_last_maximum_on_ties": ("            if (s > smax) {\n                smax = s;\n                arg = j;",
                                  "            if (s >= smax) {\n                smax = s;\n                arg = j;"),
    "centroids_normalised_by_mass": ("Tc[j * d + k] = nval(&A[j * 4 + k]) / nu[j];",
                                     "Tc[j * d + k] = nval(&A[j * 4 + k]) / nval(&A[j * 4 + 3]);"),
    "centroids_mass_not_applied": ("const double w = mass[q] * exp(row[j] - lnS);",
                                   "const double w = exp(row[j] - lnS) / (double)nq;"),
    "centroids_target_coordinates": ("nadd(&A[j * 4 + k], w * x[q * d + k]);",
                                     "nadd(&A[j * 4 + k], w * y[j * d + k]);"),
}


def _build_mutant_maps(name):
    src = open(obuild.SRC).read()
    old, new = MUTANTS_MAPS[name]
    assert src.count(old) >= 1, name
    src = src.replace(old, new, 1)
    tmpd = tempfile.mkdtemp(prefix="oracle_mut_")
    cpath = os.path.join(tmpd, "m.c")
    lpath = os.path.join(tmpd, "libm.so")
    open(cpath, "w").write(src)
    subprocess.run(["gcc", "-std=c99", "-O1", "-fPIC", "-shared", cpath, "-o", lpath, "-lm"], check=True)
    return lpath


def _mutant_maps(lpath):
    lib = ctypes.CDLL(lpath)
    dp = ctypes.POINTER(ctypes.c_double)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.oracle_transport_maps.argtypes = [ctypes.c_int, ctypes.c_int64, dp, ctypes.c_int64, dp, dp,
                                          dp, ctypes.c_double, ctypes.c_int, dp, i64p]
    lib.oracle_centroids.argtypes = [ctypes.c_int, ctypes.c_int64, dp, dp, ctypes.c_int64, dp, dp,
                                     dp, ctypes.c_double, dp, dp]
    F = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    P = lambda a: a.ctypes.data_as(dp)

    def transport_maps(x, y, nu, psi, eps, threads=1):
        x, y, nu, psi = F(x), F(y), F(nu), F(psi)
        T = np.zeros(x.shape)
        js = np.zeros(x.shape[0], dtype=np.int64)
        assert lib.oracle_transport_maps(x.shape[1], x.shape[0], P(x), y.shape[0], P(y), P(nu), P(psi),
                                         eps, 1, P(T), js.ctypes.data_as(i64p)) == 0
        return T, js

    def centroids(x, mass, y, nu, psi, eps):
        x, mass, y, nu, psi = F(x), F(mass), F(y), F(nu), F(psi)
        T = np.zeros(y.shape)
        a = np.zeros(y.shape[0])
        assert lib.oracle_centroids(x.shape[1], x.shape[0], P(x), P(mass), y.shape[0], P(y), P(nu),
                                    P(psi), eps, P(T), P(a)) == 0
        return T, a
    return transport_maps, centroids


def _map_pins_pass(transport_maps, centroids):
    import test_oracle_maps as T
    orig = (oracle.transport_maps, oracle.centroids)
    oracle.transport_maps, oracle.centroids = transport_maps, centroids
    try:
        checks = [T.test_single_target_maps_everything_to_it, T.test_two_targets_closed_form,
                  T.test_coincident_targets, T.test_modal_map_is_nearest_target_for_zero_potential,
                  T.test_maps_and_centroids_are_dual, T.test_centroids_of_a_point_mass]
        for c in checks:
            try:
                c()
            except AssertionError:
                return False
        return True
    finally:
        oracle.transport_maps, oracle.centroids = orig


def test_unmutated_maps_pass_compact_pins():
    assert _map_pins_pass(oracle.transport_maps, oracle.centroids)


@pytest.mark.parametrize("name", sorted(MUTANTS_MAPS))
def test_map_mutant_is_caught(name):
    lpath = _build_mutant_maps(name)
    assert not _map_pins_pass(*_mutant_maps(lpath)), f"mutant {name} passed every pin"


# ---- separable (psi-aware) truncation ----------------------------------------
MUTANTS_SEP = {
    "sep_minus_beta": ("alpha ? c < alpha[q] + beta[j]", "alpha ? c < alpha[q] - beta[j]"),
    "sep_point_index_for_target": ("alpha ? c < alpha[q] + beta[j]", "alpha ? c < alpha[q] + beta[q % n]"),
    "nearest_last_on_ties": ("            if (c < best) {\n                best = c;\n                bj = j;",
                             "            if (c <= best) {\n                best = c;\n                bj = j;"),
}


def _mutant_sep(lpath):
    lib = ctypes.CDLL(lpath)
    dp = ctypes.POINTER(ctypes.c_double)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.oracle_dual_grad_sep.argtypes = [ctypes.c_int, ctypes.c_int64, dp, dp, ctypes.c_int64, dp, dp,
                                         dp, ctypes.c_double, dp, dp, ctypes.c_int, dp, dp, i64p, i64p]
    lib.oracle_nearest.argtypes = [ctypes.c_int, ctypes.c_int64, dp, ctypes.c_int64, dp, ctypes.c_int,
                                   i64p, dp]
    F = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    P = lambda a: a.ctypes.data_as(dp)

    def dual_grad_sep(x, mass, y, nu, psi, eps, alpha, beta, threads=1):
        x, mass, y, nu, psi, alpha, beta = (F(a) for a in (x, mass, y, nu, psi, alpha, beta))
        g = np.empty(y.shape[0])
        J = ctypes.c_double()
        pr = ctypes.c_int64()
        em = ctypes.c_int64()
        assert lib.oracle_dual_grad_sep(x.shape[1], x.shape[0], P(x), P(mass), y.shape[0], P(y), P(nu),
                                        P(psi), eps, P(alpha), P(beta), 1, ctypes.byref(J), P(g),
                                        ctypes.byref(pr), ctypes.byref(em)) == 0
        return J.value, g, pr.value, em.value

    def nearest(x, y, threads=1):
        x, y = F(x), F(y)
        js = np.zeros(x.shape[0], dtype=np.int64)
        cs = np.zeros(x.shape[0])
        assert lib.oracle_nearest(x.shape[1], x.shape[0], P(x), y.shape[0], P(y), 1,
                                  js.ctypes.data_as(i64p), P(cs)) == 0
        return js, cs
    return dual_grad_sep, nearest


def _sep_pins_pass(dual_grad_sep, nearest):
    import test_oracle_separable as T
    orig = (oracle.dual_grad_sep, oracle.nearest)
    oracle.dual_grad_sep, oracle.nearest = dual_grad_sep, nearest
    try:
        checks = [lambda: T.test_nearest_matches_kdtree(2), T.test_nearest_takes_the_lowest_index_on_ties,
                  lambda: T.test_separable_matches_the_definition(2, 1e-3),
                  T.test_uniform_separable_cutoff_is_the_scalar_cutoff,
                  lambda: T.test_tail_guarantee_against_dense(1, 2, 0.01, 0.03, 1e-2, 0.5)]
        for c in checks:
            try:
                c()
            except AssertionError:
                return False
        return True
    finally:
        oracle.dual_grad_sep, oracle.nearest = orig


def test_unmutated_separable_passes_compact_pins():
    assert _sep_pins_pass(oracle.dual_grad_sep, oracle.nearest)


@pytest.mark.parametrize("name", sorted(MUTANTS_SEP))
def test_separable_mutant_is_caught(name):
    src = open(obuild.SRC).read()
    old, new = MUTANTS_SEP[name]
    assert src.count(old) >= 1, name
    tmpd = tempfile.mkdtemp(prefix="oracle_mut_")
    cpath = os.path.join(tmpd, "m.c")
    lpath = os.path.join(tmpd, "libm.so")
    open(cpath, "w").write(src.replace(old, new, 1))
    subprocess.run(["gcc", "-std=c99", "-O1", "-fPIC", "-shared", cpath, "-o", lpath, "-lm"], check=True)
    assert not _sep_pins_pass(*_mutant_sep(lpath)), f"mutant {name} passed every pin"


@pytest.mark.parametrize("wrong", ["drop_ln_nu_n", "global_min_psi"])
def test_wrong_separable_cutoffs_break_the_tail_guarantee(wrong, monkeypatch):
    """Plausible mistakes in the alpha/beta formula (Python side) are caught."""
    import test_oracle_separable as T

    def bad(x, y, nu, psi, eps, tail):
        jn, cn = oracle.nearest(x, y)
        if wrong == "drop_ln_nu_n":
            alpha = cn - psi[jn]
        else:
            alpha = cn - np.max(psi) - eps * np.log(nu[jn]) - 0.05
        return alpha, psi + eps * math.log(1.0 / tail)
    monkeypatch.setattr(T.truncation, "separable_cutoffs", bad)
    caught = False
    for args in [(1, 2, 0.01, 0.03, 1e-2, 0.5), (2, 3, 0.005, 0.01, 1e-4, 0.9), (3, 2, 0.002, 0.05, 1e-6, 0.9)]:
        try:
            T.test_tail_guarantee_against_dense(*args)
        except AssertionError:
            caught = True
    assert caught


# ---- integrated cutoff (Sec. 4.1, Eq. truncation_cutoff_int) ---------------------
@pytest.mark.parametrize("wrong", ["mass_not_applied", "log_partition_not_negated", "cutoff_ignored"])
def test_wrong_integrated_D_is_caught(wrong, monkeypatch):
    import test_oracle_integral as T
    good = oracle.integrated_D

    def bad(x, mass, y, nu, psi, eps, cutoff=math.inf, threads=0):
        if wrong == "cutoff_ignored":
            return good(x, mass, y, nu, psi, eps)
        lnD = good(x, mass, y, nu, psi, eps, cutoff)
        if wrong == "mass_not_applied":
            return lnD + math.log(len(mass)) + 0.0 * lnD
        m = np.asarray(mass)
        return -lnD + 2.0 * math.log(float(m.sum()))
    monkeypatch.setattr(oracle, "integrated_D", bad)
    caught = False
    for c in (T.test_single_target_closed_form, T.test_definition_by_brute_force,
              T.test_D_decreases_with_the_cutoff):
        try:
            c()
        except AssertionError:
            caught = True
    assert caught
