"""Shared test helpers: run the CUDA path through the C ABI and compare with the oracle."""
import numpy as np

from oracle import oracle as O


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu_collide(ft, d, N, M, S, gamma, tol, stream=None, **kw):
    """Q from libpgboltz.so for coefficients ft (numpy), plus the plan info and moments."""
    import torch

    from paper_2105_08806_gb300 import Plan

    f = torch.as_tensor(np.ascontiguousarray(np.asarray(ft, dtype=np.float64).ravel()), device="cuda")
    Q = torch.empty_like(f)
    with Plan(d, N, M, S, gamma, tol, **kw) as plan:
        if stream is not None:
            plan.set_stream(stream)
        plan.collide(f, Q)
        mom = plan.moments()
        info = plan.info()
    torch.cuda.synchronize()
    return Q.cpu().numpy(), info, mom


def sample_modes(d, N, count, seed):
    """Seeded mode subset that always holds 0, the {0,2}^d corners, (N,..,N) and the axes."""
    rng = np.random.default_rng(seed)
    fixed = [np.zeros(d, int), np.full(d, N)]
    for c in range(1 << d):
        fixed.append(np.array([2 * ((c >> (d - 1 - l)) & 1) for l in range(d)]))
    for l in range(d):
        e = np.zeros(d, int)
        e[l] = N
        fixed.append(e)
    rand = rng.integers(0, N + 1, size=(count, d))
    modes = np.unique(np.concatenate([np.array(fixed), rand]), axis=0)
    return modes.astype(np.int32)


def flat_index(modes, N):
    d = modes.shape[1]
    idx = np.zeros(modes.shape[0], dtype=np.int64)
    for l in range(d):
        idx = idx * (N + 1) + modes[:, l]
    return idx


def oracle_inputs(fun, d, N, S, r):
    return O.project(fun, d, N, S, r).ravel()
