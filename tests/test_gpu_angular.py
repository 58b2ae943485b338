"""Collision kernels with an angular factor, B(|g|, cos theta) = |g|^gamma b(cos theta) / |S^{d-1}|
(Eq. collision_form, b a polynomial in cos theta), on the GPU against the FP64 oracle.

The spreading kernels add each unordered node pair once with b(c) + b(-c) (the two orders have
opposite cos theta at the same post-collision point); the loss sums b over the sphere set per pair.
Bars as in test_gpu_parity: 1e-10 relative L2 (FP64 path), 1e-5 of the gain norm (FP32 path).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2105_08806_gb300 import PG_PREC_FP32, PG_PREC_FP64, PG_SPHERE_FIBONACCI
from paper_2105_08806_gb300 import workloads as W

from _helpers import flat_index, gpu_collide, rel_l2, sample_modes

pytestmark = pytest.mark.gpu

ANG = [1.0, 0.5, 0.3, -0.2]  # b(c) = 1 + c/2 + 0.3 c^2 - 0.2 c^3 > 0 on [-1, 1]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2105_08806_gb300.build import build
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build()
    O.build()


def _maxwell3(d, seed=0):
    rng = np.random.default_rng(seed)
    comps = [(1 / 3, rng.uniform(-1, 1, d), rng.uniform(0.6, 1.4)) for _ in range(3)]
    return lambda p: sum(W.maxwellian(p, r, c, t) for r, c, t in comps)


CASES = [
    # d, N, M, S, gamma, map_log, sphere, angular coefficients
    (2, 10, 8, 2.0, 0.5, False, 0, ANG),
    (2, 9, 6, 1.5, 1.0, True, 0, [0.7, 0.0, 0.6]),
    (3, 5, 8, 2.0, 0.0, False, 0, ANG),
    # plain Fibonacci set: the odd part of b no longer drops out of the loss; all 8 terms
    (3, 4, 8, 2.0, 1.0, False, PG_SPHERE_FIBONACCI, ANG + [0.05, 0.0, 0.01, 0.02]),
]


@pytest.mark.parametrize("prec", [PG_PREC_FP64, PG_PREC_FP32])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"d{c[0]}N{c[1]}M{c[2]}g{c[4]}s{c[6]}b{len(c[7])}")
def test_angular_kernel_all_modes_match_oracle(case, prec):
    d, N, M, S, gamma, map_log, sphere, ang = case
    r = 0 if map_log else 1
    ft = O.project(_maxwell3(d, seed=N), d, N, S, r).ravel()
    gain, loss = O.collide_parts(ft, d, N, M, S, gamma, r=r, angular=ang,
                                 sphere="fibonacci" if sphere == PG_SPHERE_FIBONACCI else "auto")
    tol = 1e-13 if prec == PG_PREC_FP64 else 1e-7
    Q, info, mom = gpu_collide(ft, d, N, M, S, gamma, tol, map_log=map_log, precision=prec, sphere=sphere,
                               angular=ang)
    if prec == PG_PREC_FP64:
        assert rel_l2(Q, gain - loss) < 1e-10
    else:
        assert np.linalg.norm(Q - (gain - loss)) / np.linalg.norm(gain) < 1e-5
    assert abs(mom["norm_gain"] - np.linalg.norm(gain)) <= (1e-10 if prec == PG_PREC_FP64 else 1e-5) * np.linalg.norm(gain)


def test_odd_angular_kernel_gives_zero_operator():
    """b(cos theta) = cos theta with the uniform circle: the gain cancels between the orders of each
    pair and the loss's sphere sum vanishes, so Q = 0 (a zero-strength grid end to end) up to the
    rounding of the loss's sphere sums (FP32 pair terms in the FP32 path)."""
    d, N, M, S = 2, 12, 8, 2.0
    ft = O.project(_maxwell3(d, 3), d, N, S, 1).ravel()
    Qv, _, _ = gpu_collide(ft, d, N, M, S, 1.0, 1e-13, precision=PG_PREC_FP64)
    for prec, tol, bar in ((PG_PREC_FP64, 1e-13, 1e-12), (PG_PREC_FP32, 1e-6, 1e-7)):
        Q, _, _ = gpu_collide(ft, d, N, M, S, 1.0, tol, precision=prec, angular=[0.0, 1.0])
        assert np.abs(Q).max() <= bar * np.abs(Qv).max(), prec


def test_full_size_2d_hard_spheres_angular_fp32_sampled_modes():
    """The 2D hard-sphere workload at full size (N = 64, M = 32) with an angular factor, FP32
    spreading (tol 1e-6), on a seeded mode subset the oracle computes one by one."""
    w = W.c2_2d_vhs()
    d, N, M, S, gamma = w.d, w.N, w.M, w.S, w.gamma
    ft = O.project(w, d, N, S, 1).ravel()
    modes = sample_modes(d, N, 24, seed=13)
    gain, loss = O.collide_parts(ft, d, N, M, S, gamma, r=1, modes=modes, angular=ANG)
    Q, _, _ = gpu_collide(ft, d, N, M, S, gamma, 1e-6, precision=PG_PREC_FP32, angular=ANG)
    assert rel_l2(Q[flat_index(modes, N)], gain - loss) < 1e-5


@pytest.mark.parametrize("sphere", [0, PG_SPHERE_FIBONACCI])
def test_angular_weak_form_on_gpu(sphere):
    """Weak-form functionals (Eq. weak) with an angular kernel: conserved to 1e-12 of their scales
    with the antipodal set; equal to the oracle's with the plain Fibonacci set."""
    import torch
    from paper_2105_08806_gb300 import Plan
    d, N, M, S, gamma = 3, 5, 8, 2.0, 0.5
    ft = O.project(_maxwell3(d, 4), d, N, S, 1).ravel()
    f = torch.as_tensor(ft, device="cuda")
    with Plan(d, N, M, S, gamma, 1e-6, sphere=sphere, angular=ANG) as plan:
        res = plan.conservation(f)
    if sphere == 0:
        for val, scale in res:
            assert abs(val) <= 1e-12 * scale, res
    else:
        phis = [(0, 0, 0)] + [(1, l, 0) for l in range(d)] + [(2, 0, 0)]
        oval, _ = O.weak(ft, d, N, M, S, gamma, phis, r=1, sphere="fibonacci", angular=ANG)
        gval = np.array([v for v, _ in res])
        assert np.allclose(gval[1:], oval[1:], rtol=1e-10, atol=1e-14)
