"""ctypes binding of libpgboltz.so (the C ABI in include/pg_boltz.h).

Argument marshalling only: every step of the collision operator runs in the
library's CUDA kernels.  Device arrays are passed as raw pointers; callers may
hand in torch CUDA tensors (float64, contiguous), whose data_ptr() is used.
There is no CPU fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
from functools import lru_cache

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libpgboltz.so")

PG_OK, PG_ERR_ARG, PG_ERR_NOMEM, PG_ERR_CUDA, PG_ERR_TIMEOUT, PG_ERR_STATE = 0, -1, -2, -3, -4, -5
PG_PREC_AUTO, PG_PREC_FP64, PG_PREC_FP32 = 0, 1, 2
PG_SPHERE_AUTO, PG_SPHERE_ANTIPODAL, PG_SPHERE_FIBONACCI = 0, 1, 2

# Every symbol the header declares (checked by the ABI test).
EXPORTS = (
    "pg_boltz_plan", "pg_boltz_plan_ex", "pg_boltz_set_stream", "pg_boltz_collide",
    "pg_boltz_moments", "pg_boltz_project_nodes", "pg_boltz_project", "pg_boltz_info",
    "pg_boltz_destroy", "pg_boltz_last_error", "pg_boltz_debug_fail_alloc", "pg_boltz_set_timing",
    "pg_boltz_stage_times", "pg_boltz_project_noalloc", "pg_boltz_probe_shared_atomics",
    "pg_boltz_plan_batched", "pg_boltz_plan_batched_ex", "pg_boltz_collide_batched", "pg_boltz_batched_offsets",
    "pg_boltz_batched_use_graph", "pg_boltz_rk4", "pg_boltz_conservation", "pg_boltz_evaluate",
    "pg_boltz_adaptive_scale", "pg_boltz_batched_autotune", "pg_boltz_kernel_poly", "pg_boltz_probe_pipes",
    "pg_boltz_grid_coords_f32",
)


class Opts(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int), ("N", ctypes.c_int), ("M", ctypes.c_int),
        ("S", ctypes.c_double), ("kernel_gamma", ctypes.c_double), ("tol", ctypes.c_double),
        ("map_log", ctypes.c_int), ("precision", ctypes.c_int), ("sphere", ctypes.c_int),
        ("upsampfac", ctypes.c_double), ("proj_nodes", ctypes.c_int),
        ("spread_threads", ctypes.c_int), ("spread_blocks_per_sm", ctypes.c_int), ("screen", ctypes.c_int),
        ("angular_terms", ctypes.c_int), ("angular_coef", ctypes.POINTER(ctypes.c_double)),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int), ("N", ctypes.c_int), ("M", ctypes.c_int), ("r", ctypes.c_int),
        ("precision", ctypes.c_int), ("sphere", ctypes.c_int),
        ("S", ctypes.c_double), ("kernel_gamma", ctypes.c_double), ("tol", ctypes.c_double),
        ("upsampfac", ctypes.c_double),
        ("n_grid", ctypes.c_int), ("n_fold", ctypes.c_int), ("kernel_width", ctypes.c_int),
        ("kernel_beta", ctypes.c_double), ("slabs", ctypes.c_int),
        ("spread_blocks", ctypes.c_int), ("spread_threads", ctypes.c_int),
        ("spread_smem_bytes", ctypes.c_size_t),
        ("points", ctypes.c_longlong), ("pairs", ctypes.c_longlong),
        ("proj_nodes", ctypes.c_int), ("launches_per_collide", ctypes.c_int),
        ("device_bytes", ctypes.c_size_t), ("kernels_per_collide", ctypes.c_int),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class PGBoltzError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


@lru_cache(maxsize=1)
def lib():
    """Load libpgboltz.so; raises if it has not been built (no fallback exists)."""
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2105_08806_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    L.pg_boltz_plan.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double]
    L.pg_boltz_plan.restype = vp
    L.pg_boltz_plan_ex.argtypes = [ctypes.POINTER(Opts)]
    L.pg_boltz_plan_ex.restype = vp
    L.pg_boltz_set_stream.argtypes = [vp, vp]
    L.pg_boltz_collide.argtypes = [vp, vp, vp]
    L.pg_boltz_moments.argtypes = [vp, dp]
    L.pg_boltz_project_nodes.argtypes = [vp, dp, ip]
    L.pg_boltz_project.argtypes = [vp, vp, vp]
    L.pg_boltz_evaluate.argtypes = [vp, vp, ctypes.c_longlong, vp, vp]
    L.pg_boltz_adaptive_scale.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, dp]
    L.pg_boltz_kernel_poly.argtypes = [ctypes.c_int, ctypes.c_double, dp, ctypes.c_int, ip, dp]
    L.pg_boltz_info.argtypes = [vp, ctypes.POINTER(Info)]
    L.pg_boltz_destroy.argtypes = [vp]
    L.pg_boltz_destroy.restype = None
    L.pg_boltz_last_error.restype = ctypes.c_char_p
    L.pg_boltz_debug_fail_alloc.argtypes = [ctypes.c_int]
    L.pg_boltz_debug_fail_alloc.restype = None
    ip_ = ctypes.POINTER(ctypes.c_int)
    L.pg_boltz_plan_batched.argtypes = [ctypes.c_int, ctypes.c_int, ip_, ip_, dp, dp, ctypes.c_double]
    L.pg_boltz_plan_batched.restype = vp
    L.pg_boltz_plan_batched_ex.argtypes = [ctypes.POINTER(Opts), ctypes.c_int, ip_, ip_, dp, dp]
    L.pg_boltz_plan_batched_ex.restype = vp
    L.pg_boltz_collide_batched.argtypes = [vp, vp, vp]
    L.pg_boltz_collide_batched.restype = ctypes.c_int
    L.pg_boltz_batched_offsets.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    L.pg_boltz_batched_offsets.restype = ctypes.c_int
    L.pg_boltz_batched_use_graph.argtypes = [vp, ctypes.c_int]
    L.pg_boltz_batched_autotune.argtypes = [vp, vp, vp, ctypes.c_int, ip, ip, ctypes.POINTER(ctypes.c_longlong), dp]
    L.pg_boltz_batched_use_graph.restype = ctypes.c_int
    L.pg_boltz_conservation.argtypes = [vp, vp, dp]
    L.pg_boltz_conservation.restype = ctypes.c_int
    L.pg_boltz_rk4.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int]
    L.pg_boltz_rk4.restype = ctypes.c_int
    L.pg_boltz_probe_shared_atomics.argtypes = [vp, dp]
    L.pg_boltz_probe_shared_atomics.restype = ctypes.c_int
    L.pg_boltz_probe_pipes.argtypes = [vp, dp]
    L.pg_boltz_probe_pipes.restype = ctypes.c_int
    L.pg_boltz_grid_coords_f32.argtypes = [vp, ctypes.c_longlong, ctypes.c_double, ctypes.c_int, ctypes.c_int, vp, vp,
                                           vp, vp]
    L.pg_boltz_grid_coords_f32.restype = ctypes.c_int
    L.pg_boltz_set_timing.argtypes = [vp, ctypes.c_int]
    L.pg_boltz_stage_times.argtypes = [vp, dp]
    for name in ("pg_boltz_set_timing", "pg_boltz_stage_times", "pg_boltz_set_stream", "pg_boltz_collide", "pg_boltz_moments", "pg_boltz_project_nodes",
                 "pg_boltz_project", "pg_boltz_info"):
        getattr(L, name).restype = ctypes.c_int
    return L


def last_error() -> str:
    return lib().pg_boltz_last_error().decode()


def _check(code):
    if code != PG_OK:
        raise PGBoltzError(code, last_error())


def _ptr(x):
    """Raw device pointer of a torch tensor (float64, contiguous, CUDA) or an int."""
    if isinstance(x, int):
        return x
    if not x.is_cuda or not x.is_contiguous() or str(x.dtype) != "torch.float64":
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return x.data_ptr()


def probe_shared_atomics(stream=None) -> float:
    """Measured int32 shared-memory atomic adds per second of the current GPU."""
    out = ctypes.c_double(0.0)
    raw = 0 if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _check(lib().pg_boltz_probe_shared_atomics(ctypes.c_void_p(raw), ctypes.byref(out)))
    return out.value


def probe_pipes(stream=None):
    """Measured (FP32 FMA/s, FP64 FMA/s, conflict-free int32 shared atomics/s) of the current GPU."""
    out = (ctypes.c_double * 3)()
    raw = 0 if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _check(lib().pg_boltz_probe_pipes(ctypes.c_void_p(raw), out))
    return tuple(out)


def grid_coords_f32(v, S: float, map_log: bool, n_grid: int, cell_out, frac_out, m2_out, stream=None):
    """FP32 spreading grid coordinates (cell, fraction in [0, 1)) and mu^-2 of float32 CUDA tensor v."""
    if str(v.dtype) != "torch.float32" or not v.is_cuda or not v.is_contiguous():
        raise ValueError("v must be a contiguous float32 CUDA tensor")
    raw = 0 if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _check(lib().pg_boltz_grid_coords_f32(ctypes.c_void_p(v.data_ptr()), v.numel(), float(S), int(bool(map_log)),
                                          int(n_grid), ctypes.c_void_p(_ptr(cell_out)), ctypes.c_void_p(_ptr(frac_out)),
                                          ctypes.c_void_p(_ptr(m2_out)), ctypes.c_void_p(raw)))


def adaptive_scale(N: int, L: float, map_log: bool = False) -> float:
    """S with v(xi_2) = -L for the M_v = N + 2 node grid (host-only, pg_boltz_adaptive_scale)."""
    out = ctypes.c_double(0.0)
    _check(lib().pg_boltz_adaptive_scale(int(N), float(L), int(bool(map_log)), ctypes.byref(out)))
    return out.value


def kernel_poly(w: int, upsampfac: float = 2.0):
    """(beta, P, coefficients) of the FP64 spreading kernels' polynomial form of the
    exponential-of-semicircle kernel (host-only, pg_boltz_kernel_poly): ceil(w/2) blocks of P."""
    cap = 8 * 17
    buf = (ctypes.c_double * cap)()
    terms = ctypes.c_int(0)
    beta = ctypes.c_double(0.0)
    _check(lib().pg_boltz_kernel_poly(int(w), float(upsampfac), buf, cap, ctypes.byref(terms), ctypes.byref(beta)))
    n = (int(w) + 1) // 2 * terms.value
    return beta.value, terms.value, list(buf[:n])


class Plan:
    """One collision-operator plan (pg_boltz_plan_ex).  Use as a context manager or call close()."""

    def __init__(self, d, N, M, S, kernel_gamma, tol, *, map_log=False, precision=PG_PREC_AUTO,
                 sphere=PG_SPHERE_AUTO, upsampfac=0.0, proj_nodes=0, spread_threads=0,
                 spread_blocks_per_sm=0, screen=False, angular=None):
        """angular: coefficients of b(cos theta) = sum_p angular[p] cos^p theta (at most 8), None: VHS."""
        ang = list(angular) if angular is not None else []
        coef = (ctypes.c_double * max(1, len(ang)))(*ang)
        o = Opts(d=d, N=N, M=M, S=S, kernel_gamma=kernel_gamma, tol=tol, map_log=int(map_log),
                 precision=precision, sphere=sphere, upsampfac=upsampfac, proj_nodes=proj_nodes,
                 spread_threads=spread_threads, spread_blocks_per_sm=spread_blocks_per_sm,
                 screen=int(screen), angular_terms=len(ang),
                 angular_coef=ctypes.cast(coef, ctypes.POINTER(ctypes.c_double)))
        h = lib().pg_boltz_plan_ex(ctypes.byref(o))
        if not h:
            raise PGBoltzError(PG_ERR_ARG, last_error())
        self._h = ctypes.c_void_p(h)
        self.d, self.N, self.M = d, N, M
        self.n_modes = (N + 1) ** d

    @property
    def handle(self):
        return self._h

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None for the default stream."""
        raw = 0 if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
        _check(lib().pg_boltz_set_stream(self._h, ctypes.c_void_p(raw)))

    def collide(self, f, Q):
        _check(lib().pg_boltz_collide(self._h, ctypes.c_void_p(_ptr(f)), ctypes.c_void_p(_ptr(Q))))

    def conservation(self, f):
        """Weak-form (value, scale) pairs for phi = 1, v_1..v_d, |v|^2 of the coefficients f."""
        n = 2 * (self.d + 2)
        out = (ctypes.c_double * n)()
        _check(lib().pg_boltz_conservation(self._h, ctypes.c_void_p(_ptr(f)), out))
        vals = list(out)
        return [(vals[2 * t], vals[2 * t + 1]) for t in range(self.d + 2)]

    def rk4(self, f, dt, nsteps):
        """nsteps classical RK4 steps of df/dt = Q(f) applied to f (device, in place)."""
        _check(lib().pg_boltz_rk4(self._h, ctypes.c_void_p(_ptr(f)), float(dt), int(nsteps)))

    def moments(self):
        out = (ctypes.c_double * 6)()
        _check(lib().pg_boltz_moments(self._h, out))
        keys = ("mass", "energy", "mass_gain", "energy_gain", "norm_Q", "norm_gain")
        return dict(zip(keys, list(out)))

    def set_timing(self, enable: bool):
        _check(lib().pg_boltz_set_timing(self._h, int(bool(enable))))

    def stage_times(self):
        """(reconstruct, loss, spread, transform) milliseconds of the last timed collide."""
        out = (ctypes.c_double * 4)()
        _check(lib().pg_boltz_stage_times(self._h, out))
        return list(out)

    def project_nodes(self):
        cnt = ctypes.c_int(0)
        _check(lib().pg_boltz_project_nodes(self._h, None, ctypes.byref(cnt)))
        buf = (ctypes.c_double * cnt.value)()
        _check(lib().pg_boltz_project_nodes(self._h, buf, ctypes.byref(cnt)))
        return list(buf)

    def project(self, fvals, ftilde):
        _check(lib().pg_boltz_project(self._h, ctypes.c_void_p(_ptr(fvals)), ctypes.c_void_p(_ptr(ftilde))))

    def evaluate(self, coef, pts, out):
        """u_N at the npts rows of pts (npts x d float64 CUDA tensor) into out (npts float64)."""
        npts = pts.numel() // self.d
        if pts.numel() != npts * self.d or out.numel() < npts or coef.numel() < (self.N + 1) ** self.d:
            raise ValueError("pts must hold npts x d values, out npts, coef (N+1)^d")
        _check(lib().pg_boltz_evaluate(self._h, ctypes.c_void_p(_ptr(coef)), npts,
                                       ctypes.c_void_p(_ptr(pts)), ctypes.c_void_p(_ptr(out))))

    def info(self) -> dict:
        inf = Info()
        _check(lib().pg_boltz_info(self._h, ctypes.byref(inf)))
        return inf.as_dict()

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().pg_boltz_destroy(self._h)
        self._h = ctypes.c_void_p(0)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchedPlan(Plan):
    """Many independent operators (pg_boltz_plan_batched_ex) evaluated by one call."""

    def __init__(self, d, N, M, S, kernel_gamma, tol, *, map_log=False, precision=PG_PREC_AUTO,
                 sphere=PG_SPHERE_AUTO, upsampfac=0.0, spread_threads=0, spread_blocks_per_sm=0,
                 screen=False):
        n = len(N)
        arr_i = ctypes.c_int * n
        arr_d = ctypes.c_double * n
        o = Opts(d=d, N=0, M=0, S=0.0, kernel_gamma=0.0, tol=tol, map_log=int(map_log), precision=precision,
                 sphere=sphere, upsampfac=upsampfac, proj_nodes=0, spread_threads=spread_threads,
                 spread_blocks_per_sm=spread_blocks_per_sm, screen=int(screen))
        h = lib().pg_boltz_plan_batched_ex(ctypes.byref(o), n, arr_i(*[int(x) for x in N]),
                                           arr_i(*[int(x) for x in M]), arr_d(*[float(x) for x in S]),
                                           arr_d(*[float(x) for x in kernel_gamma]))
        if not h:
            raise PGBoltzError(PG_ERR_ARG, last_error())
        self._h = ctypes.c_void_p(h)
        self.d, self.ncell = d, n
        off = (ctypes.c_longlong * (n + 1))()
        _check(lib().pg_boltz_batched_offsets(self._h, off))
        self.offsets = list(off)
        self.n_modes = self.offsets[-1]

    def collide(self, f, Q):
        _check(lib().pg_boltz_collide_batched(self._h, ctypes.c_void_p(_ptr(f)), ctypes.c_void_p(_ptr(Q))))

    def autotune(self, f, Q, trials=2):
        """Time the spreading launch shapes, then the work-item sizes, on (f, Q) and keep the fastest;
        returns (threads, blocks, item_points, ms)."""
        thr, blk, items, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_longlong(0), ctypes.c_double(0.0)
        _check(lib().pg_boltz_batched_autotune(self._h, ctypes.c_void_p(_ptr(f)), ctypes.c_void_p(_ptr(Q)), int(trials),
                                               ctypes.byref(thr), ctypes.byref(blk), ctypes.byref(items),
                                               ctypes.byref(ms)))
        return thr.value, blk.value, items.value, ms.value

    def use_graph(self, enable: bool):
        _check(lib().pg_boltz_batched_use_graph(self._h, int(bool(enable))))
