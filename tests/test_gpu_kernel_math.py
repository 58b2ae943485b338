"""The FP32 spreading kernels' own arithmetic against FP64 references, through the C ABI.

* Grid coordinates (pg_boltz_grid_coords_f32): x = n z/(2 pi) with z = arccos(xi(v)) for the
  algebraic (r = 1) and logarithmic (r = 0) maps of Section 2.1, formed in FP32 as an exact cell
  plus a fraction in [0, 1) from the two-term arctangent u + u^3 R(u^2).  Bound: 1e-7 rad in z
  (r = 1) and 2e-7 rad (r = 0, where exp(-|v|/S) is an FP32 exponential), with no common offset
  (mean below 1e-8 rad); mu^-2 to 1e-6 relative (r = 1) and 1e-5 (r = 0, the same exponential).
* Measured peaks (pg_boltz_probe_pipes): positive, and FP32 FMA faster than FP64 FMA.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_08806_gb300.build import build
    build()
    return torch


def _velocities(S):
    rng = np.random.default_rng(3)
    v = np.concatenate([
        np.linspace(-4 * S, 4 * S, 20001),             # both branches |v/S| <= 1 and > 1
        S * np.tan(rng.uniform(-1.55, 1.55, 20000)),   # spread over the angles
        rng.uniform(-1e-3, 1e-3, 2000),                # around v = 0
        np.array([0.0, S, -S, 1e4, -1e4, 3e5, -3e5]),  # branch points and the far field
    ])
    return v.astype(np.float32)


@pytest.mark.parametrize("map_log,S,n", [(0, 3.0, 258), (0, 2.0, 72), (0, 2.5, 98), (1, 3.0, 258), (1, 2.0, 72)])
def test_fp32_grid_coordinates_against_fp64(torch_cuda, map_log, S, n):
    torch = torch_cuda
    from paper_2105_08806_gb300._lib import grid_coords_f32
    v = _velocities(S)
    vd = torch.as_tensor(v, device="cuda")
    cell = torch.empty(v.size, dtype=torch.float64, device="cuda")
    frac = torch.empty_like(cell)
    m2 = torch.empty_like(cell)
    grid_coords_f32(vd, S, bool(map_log), n, cell, frac, m2)
    torch.cuda.synchronize()
    cell, frac = cell.cpu().numpy(), frac.cpu().numpy()
    assert np.all(cell == np.floor(cell)) and np.all((frac >= 0) & (frac < 1))
    v64 = v.astype(np.float64)
    if map_log:
        xi = np.tanh(v64 / S)
        m2_ref = S * np.cosh(np.minimum(np.abs(v64 / S), 80.0))
    else:
        xi = v64 / np.sqrt(S * S + v64 * v64)
        m2_ref = (S * S + v64 * v64) / S
    z_ref = np.arccos(xi)
    z = (cell + frac) * 2 * math.pi / n
    err = z - z_ref
    bound = 2e-7 if map_log else 1e-7
    print(f"map_log={map_log} S={S} n={n}: max |z error| {np.abs(err).max():.2e} rad, mean {err.mean():.1e}")
    assert np.abs(err).max() < bound
    assert abs(err.mean()) < 1e-8
    ok = np.abs(v64 / S) < 60  # cosh overflows FP32 beyond
    rel = np.abs(m2.cpu().numpy()[ok] / m2_ref[ok] - 1)
    assert rel.max() < (1e-5 if map_log else 1e-6)


def test_probe_pipes(torch_cuda):
    from paper_2105_08806_gb300._lib import probe_pipes
    f32, f64, atom = probe_pipes()
    print(f"FP32 FMA {f32:.3e}/s, FP64 FMA {f64:.3e}/s, conflict-free shared atomics {atom:.3e}/s")
    assert f32 > 0 and f64 > 0 and atom > 0
    assert f32 > f64
