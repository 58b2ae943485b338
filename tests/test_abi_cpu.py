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
    assert L.pg_boltz_batched_autotune(None, None, None, 2, None, None, None, None) == _lib.PG_ERR_ARG
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


def _psi(t, beta):
    """Exponential-of-semicircle kernel psi(t) = exp(beta (sqrt(1 - t^2) - 1)), |t| < 1, else 0,
    in long double (in double the rounding of beta (sqrt - 1) alone is a few 1e-15)."""
    import numpy as np
    t = np.asarray(t, dtype=np.longdouble)
    om = 1 - t * t
    return np.where(om > 0, np.exp(np.longdouble(beta) * (np.sqrt(np.maximum(om, 0)) - 1)), 0)


def _poly_taps(w, P, c, y):
    """All w taps from the even/odd coefficient blocks (the FP64 spreading kernels' evaluation),
    summed in long double so that the comparison sees the fit, not this sum's rounding."""
    import numpy as np
    NE, NO = (P + 1) // 2, P // 2
    y = np.asarray(y, dtype=np.longdouble)
    c = [np.longdouble(v) for v in c]
    u = y * y
    taps = np.zeros((w, y.size), dtype=np.longdouble)
    for a in range((w + 1) // 2):
        blk = c[a * P:(a + 1) * P]
        e = np.zeros_like(y)
        for k in reversed(blk[:NE]):
            e = e * u + k
        o = np.zeros_like(y)
        for k in reversed(blk[NE:NE + NO]):
            o = o * u + k
        taps[a] = e + y * o if 2 * a + 1 != w else e
        taps[w - 1 - a] = e - y * o if 2 * a + 1 != w else e
    return taps


@pytest.mark.parametrize("sigma", [1.5, 2.0, 4.0])
@pytest.mark.parametrize("w", range(2, 17))
def test_kernel_poly_matches_kernel_definition(L, w, sigma):
    """Every tap of the polynomial form against psi at the tap's own t = (s + a - x) 2/w for
    points spread over a cell: within the kernel's own size at its support edge, exp(-beta)."""
    import numpy as np
    beta, P, c = _lib.kernel_poly(w, sigma)
    assert beta == pytest.approx(0.97 * np.pi * (1 - 0.5 / sigma) * w, rel=1e-15)
    assert P == (w + 3 if w < 12 else w + 1) and len(c) == (w + 1) // 2 * P
    x = 40.0 + np.linspace(0.0, 1.0, 1001, endpoint=False) + 0.5e-3
    s = np.floor(x - 0.5 * w) + 1
    y = 2.0 * (s - x) + (w - 1)  # exact: s - x and the sums are representable
    assert y.min() > -1 and y.max() <= 1
    taps = _poly_taps(w, P, c, y)
    exact = np.stack([_psi((s + a - x) * 2.0 / w, beta) for a in range(w)])
    err = float(np.abs(taps - exact).max())
    bound = (0.6 if (sigma == 2.0 and w >= 6) else 4.0) * np.exp(-beta) + 3e-16
    assert err <= bound, (w, sigma, err, np.exp(-beta))


def test_kernel_poly_rejects_bad_arguments(L):
    buf = (ctypes.c_double * 136)()
    P, beta = ctypes.c_int(0), ctypes.c_double(0.0)
    args = lambda w, sig, cap: (w, sig, buf, cap, ctypes.byref(P), ctypes.byref(beta))
    assert L.pg_boltz_kernel_poly(*args(1, 2.0, 136)) == _lib.PG_ERR_ARG
    assert L.pg_boltz_kernel_poly(*args(17, 2.0, 136)) == _lib.PG_ERR_ARG
    assert L.pg_boltz_kernel_poly(*args(8, 1.2, 136)) == _lib.PG_ERR_ARG
    assert L.pg_boltz_kernel_poly(*args(16, 2.0, 135)) == _lib.PG_ERR_ARG
    assert L.pg_boltz_kernel_poly(16, 2.0, None, 136, ctypes.byref(P), ctypes.byref(beta)) == _lib.PG_ERR_ARG
    assert L.pg_boltz_kernel_poly(*args(16, 0.0, 136)) == _lib.PG_OK and P.value == 17
