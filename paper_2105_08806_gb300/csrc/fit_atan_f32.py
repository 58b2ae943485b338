"""Fit the FP32 arctangent correction used by the spreading kernels (spread_impl.cuh).

For |u| <= 1 the kernels form atan(u) as the two terms u + u^3 R(u^2): the leading term u is
exact, and the correction u^3 R(u^2) (at most 0.215 in magnitude) is evaluated in FP32, so its
rounding is a few 1e-9 instead of the 6e-8 of an FP32 atan value.  R is a polynomial of degree
DEG in s = u^2, fitted to (atan(u) - u)/u^3 by iteratively reweighted least squares towards the
minimax error of atan(u) itself (weights u^3, then reweighted by the current error envelope)
on Chebyshev points of s in [0, 1].  Run it to print the coefficients (highest power first, as
the kernel's Horner loop takes them) and the fit's maximum error in FP64 and in FP32 arithmetic.

    python paper_2105_08806_gb300/csrc/fit_atan_f32.py
"""
import numpy as np

DEG = 9


def fit(deg=DEG, npts=4000, iters=60):
    k = np.arange(npts)
    s = 0.5 * (1 - np.cos(np.pi * (k + 0.5) / npts))  # Chebyshev points of s in [0, 1]
    u = np.sqrt(s)
    target = np.where(s > 1e-12, (np.arctan(u) - u) / np.maximum(u, 1e-300) ** 3, -1.0 / 3.0)
    V = np.vander(s, deg + 1, increasing=True)
    wgt = u ** 3 + 1e-30
    env = np.ones(npts)
    for _ in range(iters):
        sw = wgt * env
        c, *_ = np.linalg.lstsq(V * sw[:, None], target * sw, rcond=None)
        err = np.abs(wgt * (V @ c - target))
        # reweight towards equal error: raise weights where the local error envelope is large
        envl = np.maximum.accumulate(err[::-1])[::-1] * 0 + err
        env *= (envl / envl.max() + 1e-3) ** 0.5
        env /= env.max()
    return c


def atan_f32(u, c):
    """The kernel's evaluation in FP32: u + u^3 R(u^2) with R by Horner."""
    u = np.asarray(u, dtype=np.float32)
    s = u * u
    r = np.float32(c[-1])
    for cc in c[-2::-1]:
        r = np.float32(r * s + np.float32(cc))
    return u.astype(np.float64) + (u * s * r).astype(np.float64)


if __name__ == "__main__":
    c = fit()
    u = np.linspace(0, 1, 200001)
    ref = np.arctan(u)
    s = u * u
    r = np.polynomial.polynomial.polyval(s, c)
    print("max |error| (FP64 evaluation): %.3e" % np.max(np.abs(u + u ** 3 * r - ref)))
    uf = u.astype(np.float32).astype(np.float64)
    print("max |error| (FP32 evaluation, exact input): %.3e" % np.max(np.abs(atan_f32(uf, c) - np.arctan(uf))))
    print("coefficients of R, highest power first:")
    for cc in c[::-1]:
        print("    %.17gf," % cc)
