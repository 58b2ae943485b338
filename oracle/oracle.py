"""FP64 CPU oracle for Q_k = (Q(f_N, f_N), That_k) of arXiv 2105.08806.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  It shares no code with the CUDA library (``paper_2105_08806_gb300``);
neither side imports the other.

This module is the plain, slow definition of the discrete operator:

* Chebyshev polynomials by the three-term recurrence (Section 2.1).
* The maps v(xi), xi(v) and mu(xi) for r = 0 (logarithmic) and r = 1
  (algebraic), Section 2.1 Eq. 1D_mapping / 1D_mu_function and Remark.
* Chebyshev-Gauss-Lobatto nodes and weights for the weight
  (1 - xi^2)^(-1/2) (Section 4.1; the paper names the rule without writing it
  out, so the textbook rule is used: xi_i = -cos(pi (i-1)/(M_v-1)), weight
  pi/(M_v-1), halved at the two ends).
* Reconstruction of f_N at the nodes from its coefficients (Eq. fN_Expansion,
  Section 4.2 with M_v = N + 2).  The two end nodes map to v = -inf, +inf where
  f_N = 0, so they carry no weight and are dropped; the N interior nodes
  remain, each with weight pi/(N+1).
* The direct triple sum over (i, j, sigma_m) of the weak form
  (Eq. Qk_component) in ``pgb_oracle.c``.
* The projection f -> f~_k = (f, That_k) (Eq. MultiD_spectral_coef) used to
  prepare inputs, by Chebyshev-Gauss quadrature (the paper leaves this rule open).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from functools import lru_cache

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libpgb_oracle.so")


# ---------------------------------------------------------------- build / load
def build(force: bool = False) -> str:
    """Compile pgb_oracle.c with gcc into oracle/libpgb_oracle.so (plain C, -O2, pthreads)."""
    src = os.path.join(_HERE, "pgb_oracle.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu99", "-fPIC", "-shared", "-o", tmp, src,
                               "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


@lru_cache(maxsize=1)
def _lib():
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    common = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_int, dp, dp,
              ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, dp]
    lib.pgb_oracle_collide.argtypes = common + [ctypes.c_int, ip, ctypes.c_long, ctypes.c_long, dp, dp,
                                                ctypes.c_int]
    lib.pgb_oracle_collide.restype = ctypes.c_int
    lib.pgb_oracle_weak.argtypes = common + [ctypes.c_int, ip, dp, ctypes.c_int]
    lib.pgb_oracle_weak.restype = ctypes.c_int
    return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


# ------------------------------------------------------------ 1D numerics, §2.1
def c_k(k):
    """c_0 = pi, c_k = pi/2 for k >= 1 (Section 2.1, orthogonality of T_k)."""
    k = np.asarray(k)
    return np.where(k == 0, math.pi, math.pi / 2)


def cheb_T(kmax: int, x):
    """T_0..T_kmax at x by T_{k+1} = 2 x T_k - T_{k-1}; shape (kmax+1,) + x.shape."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty((kmax + 1,) + x.shape)
    out[0] = 1.0
    if kmax >= 1:
        out[1] = x
    for k in range(1, kmax):
        out[k + 1] = 2.0 * x * out[k] - out[k - 1]
    return out


def v_of_xi(xi, S, r):
    """v(xi): r=0 logarithmic v = (S/2) ln((1+xi)/(1-xi)); r=1 algebraic v = S xi/sqrt(1-xi^2)."""
    xi = np.asarray(xi, dtype=np.float64)
    if r == 0:
        return 0.5 * S * np.log((1 + xi) / (1 - xi))
    return S * xi / np.sqrt((1 - xi) * (1 + xi))


def xi_of_v(v, S, r):
    """xi(v): r=0 tanh(v/S); r=1 v/sqrt(S^2+v^2)."""
    v = np.asarray(v, dtype=np.float64)
    if r == 0:
        return np.tanh(v / S)
    return v / np.sqrt(S * S + v * v)


def mu_of_xi(xi, S, r):
    """mu(xi) = (1-xi^2)^((1+r)/4) / sqrt(S)   (Eq. 1D_mu_function)."""
    xi = np.asarray(xi, dtype=np.float64)
    return ((1 - xi) * (1 + xi)) ** ((1 + r) / 4.0) / math.sqrt(S)


def T_tilde(k, v, S, r):
    """Trial function T~_k(v) = mu^4 T_k(xi(v)) / sqrt(c_k)   (Eq. 1DCheby)."""
    xi = xi_of_v(v, S, r)
    return mu_of_xi(xi, S, r) ** 4 * cheb_T(k, xi)[k] / math.sqrt(c_k(k))


def T_hat(k, v, S, r):
    """Test function That_k(v) = mu^-2 T_k(xi(v)) / sqrt(c_k)   (Eq. 1DCheby)."""
    xi = xi_of_v(v, S, r)
    return mu_of_xi(xi, S, r) ** -2 * cheb_T(k, xi)[k] / math.sqrt(c_k(k))


def cgl(Mv: int):
    """All M_v Chebyshev-Gauss-Lobatto nodes/weights for the weight (1-xi^2)^(-1/2)."""
    i = np.arange(Mv)
    xi = -np.cos(math.pi * i / (Mv - 1))
    w = np.full(Mv, math.pi / (Mv - 1))
    w[0] *= 0.5
    w[-1] *= 0.5
    return xi, w


def interior_nodes(N: int, S: float, r: int):
    """Interior CGL nodes of M_v = N + 2 (Section 4.2): xi, v(xi), weight, mu(xi)^2."""
    xi, w = cgl(N + 2)
    xi, w = xi[1:-1], w[1:-1]
    return xi, v_of_xi(xi, S, r), w, mu_of_xi(xi, S, r) ** 2


# ------------------------------------------------------------------ sphere sets
def sphere_set(d: int, M: int, kind: str = "auto"):
    """Quadrature on S^{d-1}: points (M, d) and weights (M,).

    d = 2: M uniform polar angles 2 pi m / M, weight 2 pi / M (Section 4.1).
    d = 3: the paper's Lebedev rules are not available here, so an antipodal
    Fibonacci set is used: M/2 golden-angle points with heights
    1 - (2m+1)/(M/2) and azimuth m pi (3 - sqrt 5), plus their negatives,
    each of weight 4 pi / M.  kind="fibonacci" gives the plain (non-antipodal)
    M-point golden-angle set.
    """
    if d == 2:
        th = 2 * math.pi * np.arange(M) / M
        return np.stack([np.cos(th), np.sin(th)], axis=1), np.full(M, 2 * math.pi / M)
    if d != 3:
        raise ValueError("d must be 2 or 3")
    golden = math.pi * (3 - math.sqrt(5))
    if kind in ("auto", "antipodal"):
        if M % 2:
            raise ValueError("antipodal sphere set needs even M")
        h = M // 2
        m = np.arange(h)
        z = 1 - (2 * m + 1) / h
        rho = np.sqrt(1 - z * z)
        half = np.stack([rho * np.cos(m * golden), rho * np.sin(m * golden), z], axis=1)
        pts = np.concatenate([half, -half], axis=0)
    elif kind == "fibonacci":
        m = np.arange(M)
        z = 1 - (2 * m + 1) / M
        rho = np.sqrt(1 - z * z)
        pts = np.stack([rho * np.cos(m * golden), rho * np.sin(m * golden), z], axis=1)
    else:
        raise ValueError(kind)
    return pts, np.full(M, 4 * math.pi / M)


def sphere_area(d: int) -> float:
    return 2 * math.pi if d == 2 else 4 * math.pi


# ------------------------------------------------------------- reconstruction
def _apply_axis(mat, arr, axis):
    """Contract mat (out, in) with arr along `axis`."""
    return np.moveaxis(np.tensordot(mat, arr, axes=([1], [axis])), 0, axis)


def reconstruct(ftilde, d: int, N: int, S: float, r: int):
    """f_N at the interior nodes divided by mu^2:  g_i = mu(xi_i)^2 sum_k f~_k T_k(xi_i)/sqrt(c_k).

    f_N(v) = mu(xi)^4 sum_k f~_k T_k(xi)/sqrt(c_k)  (Eq. fN_Expansion with the
    tensor form of Eq. MultiD_spectral_coef), so g = f_N / mu^2 = mu^2 P.
    """
    ft = np.asarray(ftilde, dtype=np.float64).reshape((N + 1,) * d)
    xi, v, w, mu2 = interior_nodes(N, S, r)
    k = np.arange(N + 1)
    A = cheb_T(N, xi).T / np.sqrt(c_k(k))[None, :]  # (N interior, N+1)
    P = ft
    for ax in range(d):
        P = _apply_axis(A, P, ax)
    mu2_nd = mu2
    for _ in range(d - 1):
        mu2_nd = np.multiply.outer(mu2_nd, mu2)
    return mu2_nd * P


def fN_values(ftilde, d, N, S, r, pts):
    """f_N(v) at arbitrary points pts (P, d), straight from Eq. fN_Expansion."""
    ft = np.asarray(ftilde, dtype=np.float64).reshape((N + 1,) * d)
    pts = np.asarray(pts, dtype=np.float64)
    k = np.arange(N + 1)
    val = ft
    out = None
    tabs = []
    for l in range(d):
        xi = xi_of_v(pts[:, l], S, r)
        tabs.append(mu_of_xi(xi, S, r) ** 4 * cheb_T(N, xi) / np.sqrt(c_k(k))[:, None])  # (N+1, P)
    if d == 2:
        out = np.einsum("ab,ap,bp->p", val, tabs[0], tabs[1])
    else:
        out = np.einsum("abc,ap,bp,cp->p", val, tabs[0], tabs[1], tabs[2])
    return out


# ----------------------------------------------------------------- projection
def projection_nodes(Mp: int, S: float, r: int):
    """Mp Chebyshev-Gauss nodes xi_p = -cos((2p-1) pi / (2 Mp)), weight pi/Mp, and v(xi_p).

    The projection integral has the weight (1-xi^2)^(-1/2); the Gauss rule is exact for
    polynomial integrands of degree <= 2 Mp - 1 and, unlike the Lobatto rule, never needs
    the integrand at xi = +-1 (v = +-inf).
    """
    p = np.arange(1, Mp + 1)
    xi = -np.cos((2 * p - 1) * math.pi / (2 * Mp))
    return xi, v_of_xi(xi, S, r), np.full(Mp, math.pi / Mp)


def project(fun, d: int, N: int, S: float, r: int, Mp: int | None = None):
    """f~_k = (1/sqrt(c_k)) (mu^-4 f(v(xi)), T_k)_omega  (Eq. MultiD_spectral_coef), CGL quadrature.

    `fun` maps an (P, d) array of velocities to f values; Mp Chebyshev-Gauss nodes per axis
    (default 4 (N + 1)).
    """
    Mp = Mp or 4 * (N + 1)
    xi, v, w = projection_nodes(Mp, S, r)
    grids = np.meshgrid(*([v] * d), indexing="ij")
    pts = np.stack([gg.ravel() for gg in grids], axis=1)
    fv = np.asarray(fun(pts), dtype=np.float64).reshape((Mp,) * d)
    mu = mu_of_xi(xi, S, r)
    scale = w * mu ** -4
    val = fv
    k = np.arange(N + 1)
    A = (cheb_T(N, xi) / np.sqrt(c_k(k))[:, None]) * scale[None, :]  # (N+1, Mp)
    for ax in range(d):
        val = _apply_axis(A, val, ax)
    return val


# --------------------------------------------------------------- the operator
def all_modes(d: int, N: int):
    g = np.meshgrid(*([np.arange(N + 1)] * d), indexing="ij")
    return np.stack([x.ravel() for x in g], axis=1).astype(np.int32)


class Problem:
    """Quadrature data of one discrete operator: nodes, weights, g_i, sphere set, kernel."""

    def __init__(self, ftilde, d, N, M, S, gamma, r=1, sphere="auto", angular=None):
        self.d, self.N, self.M, self.S, self.gamma, self.r = d, N, M, float(S), float(gamma), int(r)
        xi, v, w, mu2 = interior_nodes(N, S, r)
        self.v1d = np.ascontiguousarray(v)
        self.Wnode = float(w[0] ** d)  # every interior weight is pi/(N+1)
        self.g = np.ascontiguousarray(reconstruct(ftilde, d, N, S, r).ravel())
        sig, wsig = sphere_set(d, M, sphere)
        self.sig = np.ascontiguousarray(sig.ravel())
        self.wsig = np.ascontiguousarray(wsig)
        # B = |v - v_*|^gamma / |S^{d-1}|  (VHS kernel, Section 3.1; constant 1/|S^{d-1}| as in Section 5 BKW tests)
        self.Bconst = 1.0 / sphere_area(d)
        # angular factor b(cos theta) = sum_p angular[p] cos^p theta of B(|g|, cos theta)
        # (Eq. collision_form); None: b = 1
        self.bcoef = np.ascontiguousarray(np.asarray(angular if angular is not None else [], dtype=np.float64))

    def _common(self):
        return (self.d, self.N, _dp(self.v1d), _dp(self.g), self.Wnode, self.M, _dp(self.sig),
                _dp(self.wsig), self.S, self.r, self.gamma, self.Bconst, int(self.bcoef.size),
                _dp(self.bcoef) if self.bcoef.size else None)


def collide_parts(ftilde, d, N, M, S, gamma, r=1, sphere="auto", modes=None, nthreads=None,
                  outer=None, angular=None):
    """(gain, loss) for the requested modes (default: all (N+1)^d, C-order).

    `outer` = (i_lo, i_hi) restricts the outer node sum to i_lo <= i < i_hi (C-order node
    index); the default is every node.
    """
    pb = Problem(ftilde, d, N, M, S, gamma, r, sphere, angular)
    modes = all_modes(d, N) if modes is None else np.ascontiguousarray(np.asarray(modes, dtype=np.int32))
    nm = modes.shape[0]
    gain = np.zeros(nm)
    loss = np.zeros(nm)
    i_lo, i_hi = outer if outer is not None else (0, N ** d)
    rc = _lib().pgb_oracle_collide(*pb._common(), nm, _ip(modes), int(i_lo), int(i_hi), _dp(gain), _dp(loss),
                                   int(nthreads or default_threads()))
    if rc != 0:
        raise RuntimeError(f"pgb_oracle_collide failed: {rc}")
    return gain, loss


def collide(ftilde, d, N, M, S, gamma, r=1, sphere="auto", modes=None, nthreads=None, angular=None):
    """Q_k = gain - loss (Section 4.2, Q = Q+ - Q-)."""
    gain, loss = collide_parts(ftilde, d, N, M, S, gamma, r, sphere, modes, nthreads, angular=angular)
    return gain - loss


PHI_ONE, PHI_V, PHI_V2, PHI_VV, PHI_VV2, PHI_V2V2, PHI_V4 = 0, 1, 2, 3, 4, 5, 6


def weak(ftilde, d, N, M, S, gamma, phis, r=1, sphere="auto", nthreads=None, angular=None):
    """sum qbar [phi(v') - phi(v_i)] and its scale for each (kind, a, b) in phis (Eq. weak)."""
    pb = Problem(ftilde, d, N, M, S, gamma, r, sphere, angular)
    ph = np.ascontiguousarray(np.asarray(phis, dtype=np.int32).reshape(-1, 3))
    out = np.zeros(2 * ph.shape[0])
    rc = _lib().pgb_oracle_weak(*pb._common(), ph.shape[0], _ip(ph), _dp(out),
                                int(nthreads or default_threads()))
    if rc != 0:
        raise RuntimeError(f"pgb_oracle_weak failed: {rc}")
    return out[0::2], out[1::2]


def mass_energy_coeffs(d: int, N: int, S: float):
    """Coefficients a_k with 1 = sum a_k That_k and |v|^2 = sum b_k That_k (r = 1, N >= 2).

    From the identities in the proof of the mass/energy theorem (Section 3.3):
    1   = sqrt(c0)/(2S) That_0 - sqrt(c2)/(2S) That_2,
    v^2 = sqrt(c0) S/2 That_0 + sqrt(c2) S/2 That_2.
    Returns two (N+1)^d arrays (C-order).
    """
    one = np.zeros(N + 1)
    one[0] = math.sqrt(math.pi) / (2 * S)
    one[2] = -math.sqrt(math.pi / 2) / (2 * S)
    sq = np.zeros(N + 1)
    sq[0] = math.sqrt(math.pi) * S / 2
    sq[2] = math.sqrt(math.pi / 2) * S / 2

    def outer(vs):
        out = vs[0]
        for x in vs[1:]:
            out = np.multiply.outer(out, x)
        return out

    mass = outer([one] * d)
    energy = np.zeros((N + 1,) * d)
    for l in range(d):
        energy = energy + outer([sq if m == l else one for m in range(d)])
    return mass.ravel(), energy.ravel()
