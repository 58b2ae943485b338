"""Host checks of the integer arithmetic the spreading kernels use in place of divisions
(spread_impl.cuh: node_axes, pair_cursor / pair_advance).  Both are exact by construction; these
tests check the construction itself for every node count a plan allows."""
import random

import numpy as np

K = 1597  # the row shear of the pair numbering (kPairShear)


def test_float_quotient_is_exact_for_every_plan_node_count():
    """q = trunc(fl32(fl32(k + 1/2) * fl32(1/N))) equals k // N for 0 <= k < N^d, for every N a plan
    takes (2D: N <= 512, 3D: N <= 128), as the kernels decode node indices."""
    for d, nmax in ((2, 512), (3, 128)):
        for N in range(2, nmax + 1):
            k = np.arange(N ** d, dtype=np.int64)
            inv = np.float32(1.0) / np.float32(N)
            q = np.trunc((k.astype(np.float32) + np.float32(0.5)) * inv).astype(np.int64)
            assert np.array_equal(q, k // N), (d, N)


def _direct(pr, nn):
    t, u = divmod(pr, nn)
    return t, u, (u if 2 * t == nn else (u + t * K) % nn)


def test_pair_cursor_matches_the_numbering():
    """Advancing (pr, t, u, i) by a stride with adds and conditional subtractions gives the same
    row, column and sheared node as decoding pr directly, across node counts and strides."""
    rng = random.Random(7)
    for _ in range(2000):
        nn = rng.choice([4, 9, 16, 27, 64, 256, 4096, 13824, 14400, 262144, 2097152, rng.randint(2, 5000)])
        npairs = nn * (nn + 1) // 2
        stride = rng.choice([1, 128, 1024, 152 * 1024, rng.randint(1, 10 ** 6)])
        pr = rng.randint(0, min(npairs - 1, 10 ** 7))
        t, u = divmod(pr, nn)
        i = (u + t * K) % nn
        dt, du = divmod(stride, nn)
        di, dk = (du + dt * K) % nn, K % nn
        for _ in range(40):
            if pr >= npairs:
                break
            assert (t, u, u if 2 * t == nn else i) == _direct(pr, nn), (nn, stride, pr)
            pr, t, u, i = pr + stride, t + dt, u + du, i + di
            if i >= nn:
                i -= nn
            if u >= nn:
                u, t, i = u - nn, t + 1, i + dk
                if i >= nn:
                    i -= nn
