"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/*.h declares (no compute call: this runs without a GPU)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(rsot_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2507_23602_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path), path


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("rsot_create", "rsot_eval_dual_grad", "rsot_solve", "rsot_radius_for_tail",
              "rsot_destroy", "rsot_status_string", "rsot_covering_cost"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    so, path = lib
    for name in sorted(declared_functions()):
        assert hasattr(so, name), f"{name} declared in include/ but not exported by {path}"


def test_exports_are_unmangled_c_symbols(lib):
    _, path = lib
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    for name in declared_functions():
        assert name in exported


def test_status_strings_without_gpu(lib):
    so, _ = lib
    so.rsot_status_string.restype = ctypes.c_char_p
    so.rsot_version.restype = ctypes.c_char_p
    assert so.rsot_status_string(0) == b"ok"
    assert b"line search" in so.rsot_status_string(6)
    assert b"sm_103a" in so.rsot_version()


def test_argument_errors_need_no_gpu(lib):
    so, _ = lib
    h = ctypes.c_void_p()
    # d = 4 is rejected before any CUDA call
    assert so.rsot_create(4, 10, None, None, 5, None, None, 0, ctypes.byref(h)) == 1
    assert so.rsot_create(2, 0, None, None, 5, None, None, 0, ctypes.byref(h)) == 1
    assert so.rsot_eval_dual_grad(None, None, ctypes.c_double(0.1), ctypes.c_double(0.0), 1,
                                  None, None, None) == 1


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_2507_23602_gb300 as rs
    monkeypatch.setattr(rs, "_LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(rs, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        rs.load()


def test_binding_constants_match_the_header(lib):
    """Every enum value and numeric limit the binding restates equals the
    header's (a GEMM kind or status added to one side only fails here)."""
    import paper_2507_23602_gb300 as rs
    src = open(os.path.join(ROOT, "include", "rsot.h")).read()
    vals = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(RSOT_[A-Z0-9_]+)\s*=\s*(\d+)", src)}
    defs = {m.group(1): float(m.group(2))
            for m in re.finditer(r"#define\s+(RSOT_[A-Z0-9_]+)\s+([0-9.eE+-]+)\s*$", src, re.M)}
    prefixes = {"RSOT_MLP_GEMM_": "GEMM_", "RSOT_PAIRS_": "PAIRS_"}
    checked = 0
    for name, v in vals.items():
        if name.startswith("RSOT_ERR_") or name == "RSOT_OK":
            assert v in rs.STATUS, name
            checked += 1
            continue
        py = next((p2 + name[len(p1):] for p1, p2 in prefixes.items() if name.startswith(p1)),
                  name[len("RSOT_"):])
        assert getattr(rs, py) == v, (name, py)
        checked += 1
    assert set(rs.STATUS) == {v for n, v in vals.items() if n.startswith("RSOT_ERR_") or n == "RSOT_OK"}
    assert rs.COMPENSATED_GRAD_REL == defs["RSOT_COMPENSATED_GRAD_REL"]
    assert rs.MAX_LEVELS == defs["RSOT_MAX_LEVELS"]
    for name in ("NOALLOC_MAX_NQ", "NOALLOC_MAX_N", "NOALLOC_SCRATCH_BYTES"):
        assert getattr(rs, name) == defs["RSOT_" + name], name
    assert checked >= 18


def test_exp2_table_of_the_fp64_exponential():
    """The FP64 path's table: hi = 2^(j/64) rounded to FP64 and lo = the FP64
    value nearest 2^(j/64) - hi, checked in 200-bit arithmetic."""
    mpmath = pytest.importorskip("mpmath")
    src = open(os.path.join(ROOT, "paper_2507_23602_gb300", "csrc", "rsot_exp64.cuh")).read()
    body = src[src.index("kExp2Tab[64] = {"):]
    body = body[:body.index("};")]
    pairs = re.findall(r"\{([-0-9.e+]+),\s*([-0-9.e+]+)\}", body)
    assert len(pairs) == 64
    mpmath.mp.prec = 200
    for j, (hi, lo) in enumerate(pairs):
        t = mpmath.power(2, mpmath.mpf(j) / 64)
        assert float(hi) == float(t)
        assert float(lo) == float(t - mpmath.mpf(float(hi)))
