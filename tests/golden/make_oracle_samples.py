"""Write the oracle's values of Q_k on a seeded mode subset of each single-plan workload.

The files oracle_<workload>.txt hold, for the seeded synthetic density of that workload
(paper_2105_08806_gb300/workloads.py, projected by the oracle's own Chebyshev-Gauss rule with
4 (N + 1) nodes per axis, Eq. MultiD_spectral_coef), the gain and loss parts of Q_k
(Eq. Qk_component, the discrete weak form summed directly by oracle/) for 64 seeded modes
plus the fixed ones (0, the {0,2}^d corners, (N,...,N) and the axis ends).  bench.py reads
them to state each workload's error against the oracle without running the oracle for
minutes; only this script, which calls nothing but oracle/ and the input generators,
writes them.

    python tests/golden/make_oracle_samples.py [workload ...]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2105_08806_gb300 import workloads as W  # noqa: E402

WORKLOADS = {"2d-maxwell": W.c1_2d_maxwell, "2d-hard-spheres": W.c2_2d_vhs, "3d-bkw": W.c3_3d_bkw,
             "3d-bimaxwell": W.c4_3d_bimaxwell}
COUNT, SEED = 64, 17


def mode_subset(d, N, count, seed):
    """Seeded modes plus 0, the {0,2}^d corners, (N,...,N) and the axis ends, sorted, unique."""
    rng = np.random.default_rng(seed)
    fixed = [np.zeros(d, int), np.full(d, N)]
    for c in range(1 << d):
        fixed.append(np.array([2 * ((c >> (d - 1 - l)) & 1) for l in range(d)]))
    for l in range(d):
        e = np.zeros(d, int)
        e[l] = N
        fixed.append(e)
    rand = rng.integers(0, N + 1, size=(count, d))
    return np.unique(np.concatenate([np.array(fixed), rand]), axis=0).astype(np.int32)


def path(name):
    return os.path.join(HERE, f"oracle_{name}.txt")


def load(name):
    """(modes (K, d) int, gain (K,), loss (K,)) from a written file."""
    a = np.loadtxt(path(name), comments="#", ndmin=2)
    d = a.shape[1] - 2
    return a[:, :d].astype(np.int64), a[:, d], a[:, d + 1]


def write(name):
    w = WORKLOADS[name]()
    d, N, M, S, g = w.d, w.N, w.M, w.S, w.gamma
    ft = O.project(w, d, N, S, 1).ravel()
    modes = mode_subset(d, N, COUNT, SEED)
    t0 = time.perf_counter()
    gain, loss = O.collide_parts(ft, d, N, M, S, g, r=1, modes=modes)
    dt = time.perf_counter() - t0
    with open(path(name), "w") as fh:
        fh.write(f"# oracle/ values of Q_k = gain - loss (Eq. Qk_component, discrete weak form, direct sum)\n")
        fh.write(f"# workload {name}: d={d} N={N} M={M} S={S} gamma={g} r=1; density workloads.{WORKLOADS[name].__name__}"
                 f", projected with {4 * (N + 1)} Chebyshev-Gauss nodes per axis\n")
        fh.write(f"# {len(modes)} modes (seed {SEED}); written by tests/golden/make_oracle_samples.py in {dt:.0f} s\n")
        fh.write("# " + " ".join(f"k{l + 1}" for l in range(d)) + " gain loss\n")
        for k, gn, ls in zip(modes, gain, loss):
            fh.write(" ".join(str(int(x)) for x in k) + f" {gn:.17e} {ls:.17e}\n")
    print(f"{name}: {len(modes)} modes in {dt:.1f} s", flush=True)


if __name__ == "__main__":
    for name in (sys.argv[1:] or list(WORKLOADS)):
        write(name)
