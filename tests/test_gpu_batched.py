"""Batched plans: every cell of one pg_boltz_collide_batched call against the single-plan path
(same arithmetic, different launch structure) and, on small cells, against the FP64 oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2105_08806_gb300 import PG_PREC_FP32, PG_PREC_FP64
from paper_2105_08806_gb300 import workloads as W

from _helpers import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2105_08806_gb300.build import build
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build()


def _cells(d, n, seed):
    rng = np.random.default_rng(seed)
    Ns = rng.choice([4, 6, 8] if d == 2 else [4, 5], size=n)
    Ms = rng.choice([4, 8, 12] if d == 2 else [8, 16], size=n)
    Ss = rng.uniform(1.5, 3.0, size=n)
    gs = rng.choice([0.0, 0.5, 1.0], size=n)
    funs = []
    for c in range(n):
        comps = [(0.5, rng.uniform(-1, 1, d), rng.uniform(0.7, 1.3)) for _ in range(2)]
        funs.append(lambda p, comps=comps: sum(W.maxwellian(p, r, cc, t) for r, cc, t in comps))
    return Ns, Ms, Ss, gs, funs


def _run_batched(d, Ns, Ms, Ss, gs, fts, tol, prec, graph=True, calls=1):
    import torch
    from paper_2105_08806_gb300 import BatchedPlan
    with BatchedPlan(d, Ns, Ms, Ss, gs, tol, precision=prec) as bp:
        bp.use_graph(graph)
        f = torch.as_tensor(np.concatenate([np.ravel(x) for x in fts]), device="cuda")
        assert f.numel() == bp.n_modes
        Q = torch.empty_like(f)
        for _ in range(calls):
            bp.collide(f, Q)
        torch.cuda.synchronize()
        off = bp.offsets
        out = Q.cpu().numpy()
    return [out[off[c]:off[c + 1]] for c in range(len(Ns))]


def _plain(d, N, M, S, g, ft, tol, prec):
    from _helpers import gpu_collide
    Q, _, _ = gpu_collide(ft, d, N, M, S, g, tol, precision=prec)
    return Q


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("prec,tol,bar", [(PG_PREC_FP64, 1e-13, 1e-11), (PG_PREC_FP32, 1e-6, 2e-6)])
def test_batched_matches_single_plans(d, prec, tol, bar):
    Ns, Ms, Ss, gs, funs = _cells(d, 10, seed=3 + d)
    fts = [O.project(funs[c], d, int(Ns[c]), float(Ss[c]), 1).ravel() for c in range(len(Ns))]
    Qb = _run_batched(d, Ns, Ms, Ss, gs, fts, tol, prec)
    for c in range(len(Ns)):
        Qp = _plain(d, int(Ns[c]), int(Ms[c]), float(Ss[c]), float(gs[c]), fts[c], tol, prec)
        assert rel_l2(Qb[c], Qp) < bar, (c, rel_l2(Qb[c], Qp))


def test_batched_matches_oracle_on_small_cells():
    d = 2
    Ns, Ms, Ss, gs, funs = _cells(d, 6, seed=11)
    fts = [O.project(funs[c], d, int(Ns[c]), float(Ss[c]), 1).ravel() for c in range(len(Ns))]
    Qb = _run_batched(d, Ns, Ms, Ss, gs, fts, 1e-13, PG_PREC_FP64)
    for c in range(len(Ns)):
        ref = O.collide(fts[c], d, int(Ns[c]), int(Ms[c]), float(Ss[c]), float(gs[c]))
        assert rel_l2(Qb[c], ref) < 1e-10, c


def test_graph_replay_and_direct_launches_agree():
    d = 2
    Ns, Ms, Ss, gs, funs = _cells(d, 8, seed=21)
    fts = [O.project(funs[c], d, int(Ns[c]), float(Ss[c]), 1).ravel() for c in range(len(Ns))]
    a = _run_batched(d, Ns, Ms, Ss, gs, fts, 1e-6, PG_PREC_FP32, graph=True, calls=3)
    b = _run_batched(d, Ns, Ms, Ss, gs, fts, 1e-6, PG_PREC_FP32, graph=False, calls=1)
    for c in range(len(Ns)):
        assert np.array_equal(a[c], b[c])  # fixed-point sums: bitwise reproducible


def test_full_batched_workload_sampled_cells():
    """The 4096-cell batched 2D workload (N in {16,24,32}, M in {8,16,32}, gamma in {0,1}, S=3) in
    the FP32 path; a seeded sample of cells against single plans."""
    import torch
    from paper_2105_08806_gb300 import BatchedPlan, Plan
    cells = W.c5_batched_2d()
    d = 2
    Ns = [w.N for w in cells]
    Ms = [w.M for w in cells]
    Ss = [w.S for w in cells]
    gs = [w.gamma for w in cells]
    # inputs: each cell's density projected with a plan of its N (projection does not depend on M, gamma)
    fts = []
    plans = {}
    for w in cells:
        if w.N not in plans:
            plans[w.N] = Plan(d, w.N, 8, w.S, 0.0, 1e-6)
        pl = plans[w.N]
        v = np.array(pl.project_nodes())
        G = np.meshgrid(v, v, indexing="ij")
        fv = torch.as_tensor(w(np.stack([x.ravel() for x in G], 1)), device="cuda")
        out = torch.empty((w.N + 1) ** d, dtype=torch.float64, device="cuda")
        pl.project(fv, out)
        fts.append(out)
    torch.cuda.synchronize()
    for pl in plans.values():
        pl.close()
    f = torch.cat(fts)
    with BatchedPlan(d, Ns, Ms, Ss, gs, 1e-6, precision=PG_PREC_FP32) as bp:
        Q = torch.empty_like(f)
        bp.collide(f, Q)
        torch.cuda.synchronize()
        off = bp.offsets
        Qh = Q.cpu().numpy()
    # the batched and the single-plan kernels evaluate the same terms, but their FP32 point
    # arithmetic is compiled separately and may round differently; FP32 rounding scales with the
    # gain sum, and some cells are near equilibrium (|Q| << |Q+|), so the bar is 2e-6 of |Q+|
    from _helpers import gpu_collide
    rng = np.random.default_rng(5)
    for c in rng.choice(len(cells), size=12, replace=False):
        Qp, _, mom = gpu_collide(fts[c].cpu().numpy(), d, Ns[c], Ms[c], Ss[c], gs[c], 1e-6, precision=PG_PREC_FP32)
        assert np.linalg.norm(Qh[off[c]:off[c + 1]] - Qp) < 2e-6 * mom["norm_gain"], c


def test_batched_screened_matches_oracle():
    import torch
    from paper_2105_08806_gb300 import BatchedPlan
    d = 2
    Ns, Ms, Ss, gs, funs = _cells(d, 6, seed=31)
    fts = [O.project(funs[c], d, int(Ns[c]), float(Ss[c]), 1).ravel() for c in range(len(Ns))]
    with BatchedPlan(d, Ns, Ms, Ss, gs, 1e-13, precision=PG_PREC_FP64, screen=True) as bp:
        f = torch.as_tensor(np.concatenate(fts), device="cuda")
        Q = torch.empty_like(f)
        bp.collide(f, Q)
        torch.cuda.synchronize()
        off = bp.offsets
        Qh = Q.cpu().numpy()
    for c in range(len(Ns)):
        ref = O.collide(fts[c], d, int(Ns[c]), int(Ms[c]), float(Ss[c]), float(gs[c]))
        assert rel_l2(Qh[off[c]:off[c + 1]], ref) < 1e-10, c


def test_autotune_keeps_results_bitwise():
    """pg_boltz_batched_autotune times the persistent kernel's launch shapes and work-item sizes on
    the caller's data and keeps the fastest; the fixed-point sums depend on neither, so the results
    before and after tuning are identical, and the graph captured afterwards uses the new shape."""
    import torch
    from paper_2105_08806_gb300 import BatchedPlan
    d = 2
    Ns, Ms, Ss, gs, funs = _cells(d, 12, seed=41)
    fts = [O.project(funs[c], d, int(Ns[c]), float(Ss[c]), 1).ravel() for c in range(len(Ns))]
    with BatchedPlan(d, Ns, Ms, Ss, gs, 1e-6, precision=PG_PREC_FP32) as bp:
        f = torch.as_tensor(np.concatenate(fts), device="cuda")
        Q1 = torch.empty_like(f)
        bp.collide(f, Q1)
        Q2 = torch.empty_like(f)
        thr, blocks, items, ms = bp.autotune(f, Q2, trials=1)
        Q3 = torch.empty_like(f)
        bp.collide(f, Q3)
        torch.cuda.synchronize()
        info = bp.info()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert thr in (128, 256, 512, 1024) and blocks % sms == 0 and ms > 0
    assert items in (2 ** 15, 2 ** 16, 2 ** 17, 2 ** 18, 2 ** 19)
    assert (info["spread_threads"], info["spread_blocks"]) == (thr, blocks)
    assert torch.equal(Q1, Q2) and torch.equal(Q1, Q3)


def test_batched_alloc_failure_injection_leaves_no_plan():
    """An allocation failing at any of several points of batched plan creation raises and frees
    what was allocated; the next plan builds normally."""
    from paper_2105_08806_gb300 import BatchedPlan, PGBoltzError, lib
    try:
        for k in (1, 2, 8, 15):
            lib().pg_boltz_debug_fail_alloc(k)
            with pytest.raises(PGBoltzError) as ei:
                BatchedPlan(2, [8, 10], [8, 8], [2.0, 2.0], [0.0, 1.0], 1e-6, precision=PG_PREC_FP32)
            assert "injected" in str(ei.value)
    finally:
        lib().pg_boltz_debug_fail_alloc(0)
    with BatchedPlan(2, [8, 10], [8, 8], [2.0, 2.0], [0.0, 1.0], 1e-6, precision=PG_PREC_FP32):
        pass
