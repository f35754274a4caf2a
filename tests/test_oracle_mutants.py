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
    "non_strict_cutoff": ("in[j] = (unsigned char)(c < cutoff);", "in[j] = (unsigned char)(c <= cutoff + 1e-3);"),
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
