"""Host-side checks of the C ABI that need no GPU: the library loads, exports every symbol the
header declares, and rejects bad arguments before touching the device."""
import ctypes
import os
import re

import pytest

from paper_2105_08806_gb300 import _lib
from paper_2105_08806_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build()
    return _lib.lib()


def header_functions():
    text = open(os.path.join(ROOT, "include", "pg_boltz.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pg_boltz_\w+)\s*\(", text)))


def test_header_declares_binding_exports():
    assert header_functions() == sorted(_lib.EXPORTS)


def test_library_exports_every_declared_symbol(L):
    for name in header_functions():
        assert hasattr(L, name), name


def test_only_abi_symbols_are_exported(L):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    ours = {s for s in syms if s.startswith("pg_boltz")}
    assert ours == set(header_functions())


@pytest.mark.parametrize("args,needle", [
    ((4, 8, 8, 2.0, 0.0, 1e-6), "d must be"),
    ((2, 1, 8, 2.0, 0.0, 1e-6), "N out of range"),
    ((2, 8, 7, 2.0, 0.0, 1e-6), "M must be even"),
    ((2, 8, 8, -1.0, 0.0, 1e-6), "S must be positive"),
    ((2, 8, 8, 2.0, 1.5, 1e-6), "kernel_gamma"),
    ((2, 8, 8, 2.0, 0.0, 1e-20), "tol must be"),
])
def test_bad_arguments_rejected(L, args, needle):
    h = L.pg_boltz_plan(*args)
    assert not h
    assert needle in _lib.last_error()


def test_null_handles(L):
    assert L.pg_boltz_collide(None, None, None) == _lib.PG_ERR_ARG
    assert L.pg_boltz_moments(None, None) == _lib.PG_ERR_ARG
    assert L.pg_boltz_info(None, None) == _lib.PG_ERR_ARG
    assert L.pg_boltz_set_stream(None, None) == _lib.PG_ERR_ARG
    assert L.pg_boltz_evaluate(None, None, 1, None, None) == _lib.PG_ERR_ARG
    assert L.pg_boltz_batched_autotune(None, None, None, 2, None, None, None) == _lib.PG_ERR_ARG
    L.pg_boltz_destroy(None)  # NULL-safe


def test_extended_option_validation(L):
    o = _lib.Opts(d=2, N=8, M=8, S=2.0, kernel_gamma=0.0, tol=1e-6, upsampfac=9.0)
    assert not L.pg_boltz_plan_ex(ctypes.byref(o))
    assert "upsampfac" in _lib.last_error()
    o = _lib.Opts(d=2, N=8, M=8, S=2.0, kernel_gamma=0.0, tol=1e-6, map_log=3)
    assert not L.pg_boltz_plan_ex(ctypes.byref(o))
    assert "map_log" in _lib.last_error()
    o = _lib.Opts(d=2, N=8, M=8, S=2.0, kernel_gamma=0.0, tol=1e-6, angular_terms=9)
    assert not L.pg_boltz_plan_ex(ctypes.byref(o))
    assert "angular_terms" in _lib.last_error()
    o = _lib.Opts(d=2, N=8, M=8, S=2.0, kernel_gamma=0.0, tol=1e-6, angular_terms=2)  # NULL coefficients
    assert not L.pg_boltz_plan_ex(ctypes.byref(o))
    assert "angular_coef" in _lib.last_error()
    bad = (ctypes.c_double * 2)(1.0, float("nan"))
    o = _lib.Opts(d=2, N=8, M=8, S=2.0, kernel_gamma=0.0, tol=1e-6, angular_terms=2,
                  angular_coef=ctypes.cast(bad, ctypes.POINTER(ctypes.c_double)))
    assert not L.pg_boltz_plan_ex(ctypes.byref(o))
    assert "not finite" in _lib.last_error()
    n, m, sv, gv = (ctypes.c_int * 1)(8), (ctypes.c_int * 1)(8), (ctypes.c_double * 1)(2.0), (ctypes.c_double * 1)(0.0)
    o = _lib.Opts(d=2, tol=1e-6, angular_terms=1, angular_coef=ctypes.cast(sv, ctypes.POINTER(ctypes.c_double)))
    assert not L.pg_boltz_plan_batched_ex(ctypes.byref(o), 1, n, m, sv, gv)
    assert "VHS" in _lib.last_error()


@pytest.mark.parametrize("r", [0, 1])
@pytest.mark.parametrize("N,Lt", [(2, 5.0), (8, 8.83), (32, 14.35), (64, 13.24)])
def test_adaptive_scale_maps_first_interior_node_to_minus_L(L, r, N, Lt):
    """Section 5: S is chosen so that xi_2 and xi_{N+1} of the M_v = N + 2 CGL nodes map to -L and
    L; checked with the oracle's own map (an independent implementation of Eq. 1D_mapping)."""
    from oracle import oracle as O
    S = _lib.adaptive_scale(N, Lt, map_log=(r == 0))
    xi = O.cgl(N + 2)[0]
    v = O.v_of_xi(xi[1:-1], S, r)
    assert abs(v[0] + Lt) <= 1e-12 * Lt and abs(v[-1] - Lt) <= 1e-12 * Lt


def test_adaptive_scale_rejects_bad_arguments(L):
    out = ctypes.c_double(0.0)
    assert L.pg_boltz_adaptive_scale(1, 5.0, 0, ctypes.byref(out)) == _lib.PG_ERR_ARG
    assert L.pg_boltz_adaptive_scale(8, 0.0, 0, ctypes.byref(out)) == _lib.PG_ERR_ARG
    assert L.pg_boltz_adaptive_scale(8, float("inf"), 1, ctypes.byref(out)) == _lib.PG_ERR_ARG
    assert L.pg_boltz_adaptive_scale(8, 5.0, 0, None) == _lib.PG_ERR_ARG
