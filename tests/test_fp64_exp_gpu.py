"""The FP64 path's own exponential (Tang's table-driven method: 2^(j/64) from
a 64-entry table of head/tail pairs, a degree-6 Taylor polynomial on
|r| <= ln(2)/128) against the host's libm exp, and the probes of the pipes that
bound the evaluations.  Bound: 2 units in the last place for normal results
(the polynomial's remainder is below 3e-20 relative, the table pairs carry
2^(j/64) to about 2^-106, and the reduction, polynomial and final add round
about once each); subnormal results to within 2 units of 2^-1074; the special
values."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def exp64(x):
    import paper_2507_23602_gb300 as rs
    lib = rs.load()
    lib.rsot_exp64.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    assert lib.rsot_exp64(x.size, x.ctypes.data, y.ctypes.data) == 0
    return y


def test_exp64_within_two_ulp_of_libm():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-745.0, 709.0, 1_000_000), rng.uniform(-60.0, 0.0, 1_000_000),
                        rng.uniform(-1e-3, 1e-3, 100_000), np.arange(-1075, 1024) * np.log(2.0),
                        [0.0, -0.0, 1e-300, -1e-300]])
    y = exp64(x)
    ref = np.exp(x)
    normal = ref >= np.finfo(np.float64).tiny
    ulps = np.abs(y[normal] - ref[normal]) / np.spacing(ref[normal])
    assert np.max(ulps) <= 2.0, np.max(ulps)
    sub = ~normal & (x > -745.2)
    assert np.all(np.abs(y[sub] - ref[sub]) <= 2 * 2.0 ** -1074)


def test_exp64_special_values():
    x = np.array([-np.inf, np.inf, np.nan, -746.0, -745.1, 709.7, 709.9, 1e308, -1e308])
    y = exp64(x)
    assert y[0] == 0.0 and y[1] == np.inf and np.isnan(y[2]) and y[3] == 0.0
    assert 0.0 < y[4] < 1e-323
    assert np.isfinite(y[5]) and abs(y[5] - np.exp(709.7)) <= 2 * np.spacing(np.exp(709.7))
    assert y[6] == np.inf and y[7] == np.inf and y[8] == 0.0


def test_pipe_probes_report_rates():
    import paper_2507_23602_gb300 as rs
    lib = rs.load()
    v = ctypes.c_double()
    assert lib.rsot_probe_dfma_rate(2000, ctypes.byref(v)) == 0
    assert 1e11 < v.value < 1e15
    assert rs.probe_ex2_rate() > 1e12
