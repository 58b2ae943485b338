"""pg_boltz_project_noalloc: the projection for callers that cannot allocate device memory.

Applications whose own pool owns all device memory, or bindings that can only pass pointers
they already hold, cannot create a plan (plans allocate).  This entry point takes only the
caller's input and output arrays and keeps its intermediates in a static device array.  The
test calls it through the C ABI and compares it with the plan-based pg_boltz_project (the
existing entry point), twice in a row, so that the second call runs on scratch left over by
the first.  Around the second call (after the plan is destroyed and the first call has loaded
the library's device code) it also checks that the device's free memory does not change: the
call allocates nothing.  This file is collected last so a stop-at-first-failure run has already
run every other test.
"""
import ctypes

import numpy as np
import pytest

from _helpers import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_08806_gb300.build import build
    from paper_2105_08806_gb300 import _lib
    build()
    lib = _lib.lib()
    fn = lib.pg_boltz_project_noalloc
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return lib


def _density(d, seed):
    from paper_2105_08806_gb300 import workloads as W
    rng = np.random.default_rng(seed)
    comps = [(0.5, rng.uniform(-1, 1, d), rng.uniform(0.7, 1.3)) for _ in range(2)]
    return lambda p: sum(W.maxwellian(p, r, c, t) for r, c, t in comps)


@pytest.mark.parametrize("d,N,S,map_log,Mp", [(2, 16, 2.0, 0, 68), (2, 64, 3.0, 0, 260), (3, 8, 2.5, 1, 30)])
def test_noalloc_projection_matches_plan_twice(L, d, N, S, map_log, Mp):
    import torch
    from paper_2105_08806_gb300 import Plan
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        fun = _density(d, seed=10 * N + call)
        with Plan(d, N, 4, S, 0.0, 1e-6, map_log=bool(map_log), proj_nodes=Mp) as plan:
            v = np.array(plan.project_nodes())
            grids = np.meshgrid(*([v] * d), indexing="ij")
            fv = torch.as_tensor(fun(np.stack([g.ravel() for g in grids], 1)), device="cuda")
            ref = torch.empty((N + 1) ** d, dtype=torch.float64, device="cuda")
            plan.project(fv, ref)
        out = torch.full_like(ref, float("nan"))
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = L.pg_boltz_project_noalloc(d, N, S, map_log, Mp, fv.data_ptr(), out.data_ptr(), stream)
        assert rc == 0, L.pg_boltz_last_error().decode()
        assert L.pg_boltz_last_error().decode() == ""
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        if call == 1:  # the first call may load the library's device code in this context
            assert free_after == free_before, (free_before, free_after)
        assert rel_l2(out.cpu().numpy(), ref.cpu().numpy()) < 1e-12


def test_noalloc_rejects_sizes_beyond_the_static_scratch(L):
    import torch
    f = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = L.pg_boltz_project_noalloc(3, 40, 2.0, 0, 200, f.data_ptr(), f.data_ptr(), None)
    assert rc == -1
    assert "static scratch" in L.pg_boltz_last_error().decode()
    # a later successful call clears the error text
    g = torch.zeros(9 * 9, dtype=torch.float64, device="cuda")
    out = torch.empty(3 * 3, dtype=torch.float64, device="cuda")
    assert L.pg_boltz_project_noalloc(2, 2, 2.0, 0, 9, g.data_ptr(), out.data_ptr(), None) == 0
    assert L.pg_boltz_last_error().decode() == ""
