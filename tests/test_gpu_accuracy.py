"""Inverse evaluation on the GPU (pg_boltz_evaluate) against the oracle, and the accuracy study of
the 2D BKW test (Section 5.1.1, Test 01) run entirely through the library: projection of f_BKW,
the fast FP64 operator with NUFFT precision 1e-14, M_v = N + 2, M_sigma = N, and Q_N on the
paper's 200 x 200 grid over [-6.3, 6.3]^2 at t = 2.  For each N the best L2 error over a scan of S
is compared with the paper's table (Chebyshev-0: logarithmic map, Chebyshev-1: algebraic map)
within a factor 4 (the paper's S scan and norm are not restated)."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2105_08806_gb300 import PG_PREC_FP64
from paper_2105_08806_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2105_08806_gb300.build import build
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build()


@pytest.mark.parametrize("d,N,S,r", [(2, 12, 2.0, 1), (2, 40, 3.5, 0), (3, 9, 2.5, 1), (3, 7, 2.0, 0)])
@pytest.mark.parametrize("npts", [0, 1, 1000, 70001])
def test_evaluate_matches_oracle(d, N, S, r, npts):
    """u_N(v) from the nested-Clenshaw kernel against the oracle's direct sum (Eq. fN_Expansion)
    at random velocities, including far-field points where mu^4 underflows."""
    import torch
    from paper_2105_08806_gb300 import Plan
    rng = np.random.default_rng(100 * d + N + npts)
    coef = rng.standard_normal((N + 1) ** d) / (1 + np.arange((N + 1) ** d)) ** 0.5
    pts = rng.standard_normal((npts, d)) * 3.0
    if npts > 10:
        pts[:5] = [[1e3] * d, [-1e3] * d, [0.0] * d, [1e-300] * d, [-40.0] * d]
    out = torch.full((max(npts, 1),), float("nan"), dtype=torch.float64, device="cuda")
    with Plan(d, N, 4, S, 0.0, 1e-6, map_log=(r == 0)) as plan:
        plan.evaluate(torch.as_tensor(coef, device="cuda"), torch.as_tensor(pts.ravel(), device="cuda"), out)
        torch.cuda.synchronize()
    got = out.cpu().numpy()
    if npts == 0:
        assert math.isnan(got[0])  # nothing written
        return
    ref = O.fN_values(coef, d, N, S, r, pts)
    scale = np.abs(ref).max()
    assert np.abs(got[:npts] - ref).max() <= 1e-12 * scale


def _qbkw2(p, t):
    """Exact 2D BKW collision operator (Eq. 2d_bkw_rhs), B = 1/(2 pi)."""
    K = 1 - math.exp(-t / 8) / 2
    Kp = math.exp(-t / 8) / 16
    v2 = np.sum(p * p, axis=1)
    f = W.bkw_2d(p, t=t)
    return ((-2 / K + v2 / (2 * K * K)) * f
            + 1 / (2 * math.pi * K * K) * np.exp(-v2 / (2 * K)) * (2 - v2 / (2 * K * K))) * Kp


def _table(r):
    name = "bkw2d_chebyshev0_l2.txt" if r == 0 else "bkw2d_chebyshev1_l2.txt"
    rows = [l.split() for l in open(os.path.join(GOLDEN, name)) if l[0] != "#"]
    return {int(a): float(b) for a, b in rows}


def bkw2d_error(N, S, r, t=2.0):
    """L2 error of Q_N against Q_BKW on the 200^2 grid, every step on the GPU through the ABI."""
    import torch
    from paper_2105_08806_gb300 import Plan
    x = np.linspace(-6.3, 6.3, 200)
    X, Y = np.meshgrid(x, x, indexing="ij")
    grid = np.stack([X.ravel(), Y.ravel()], 1)
    h = x[1] - x[0]
    with Plan(2, N, N, S, 0.0, 1e-14, precision=PG_PREC_FP64, map_log=(r == 0)) as plan:
        v = np.array(plan.project_nodes())
        V = np.meshgrid(v, v, indexing="ij")
        fv = torch.as_tensor(W.bkw_2d(np.stack([a.ravel() for a in V], 1), t=t), device="cuda")
        f = torch.empty((N + 1) ** 2, dtype=torch.float64, device="cuda")
        plan.project(fv, f)
        Q = torch.empty_like(f)
        plan.collide(f, Q)
        QN = torch.empty(grid.shape[0], dtype=torch.float64, device="cuda")
        plan.evaluate(Q, torch.as_tensor(grid.ravel(), device="cuda"), QN)
        torch.cuda.synchronize()
    return math.sqrt(np.sum((QN.cpu().numpy() - _qbkw2(grid, t)) ** 2) * h * h)


# S windows (step 0.125) around each N's best S
SCANS = {
    (0, 8): (1.75, 2.75), (0, 16): (2.0, 3.25), (0, 24): (2.75, 4.0), (0, 32): (3.0, 4.5), (0, 40): (3.5, 5.0),
    (0, 48): (3.75, 4.75), (0, 56): (4.25, 5.25),
    (1, 8): (1.75, 2.75), (1, 16): (2.25, 3.5), (1, 24): (2.75, 4.25), (1, 32): (3.0, 5.0), (1, 40): (3.5, 5.5),
    (1, 48): (4.0, 6.0), (1, 56): (5.0, 6.5),
}


@pytest.mark.parametrize("r,N", sorted(SCANS))
def test_bkw2d_best_error_matches_paper(r, N):
    """Within a factor 4 of the paper's entry; below 1e-12 (the paper's entries there sit at its
    NUFFT's rounding floor) only the upper side is asserted."""
    lo, hi = SCANS[(r, N)]
    errs = {S: bkw2d_error(N, S, r) for S in np.arange(lo, hi + 1e-9, 0.125)}
    S_best = min(errs, key=errs.get)
    best = errs[S_best]
    paper = _table(r)[N]
    print(f"BKW2D r={r} N={N}: best L2 {best:.4e} at S={S_best:.3f} (paper {paper:.4e})")
    assert best < paper * 4, (r, N, S_best, best, paper)
    if paper > 1e-12:
        assert best > paper / 4, (r, N, S_best, best, paper)
