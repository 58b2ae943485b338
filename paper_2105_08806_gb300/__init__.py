"""GB300 (sm_103a) evaluation of the Petrov-Galerkin mapped-Chebyshev Boltzmann collision
operator Q(f, f) of arXiv 2105.08806 with the fast non-uniform-FFT algorithm (Section 4.2).

The compute path is the C ABI library libpgboltz.so (include/pg_boltz.h); this package is
its ctypes binding (``Plan``), its nvcc build script and the seeded input distributions.
"""
from ._lib import (BatchedPlan, Plan, PGBoltzError, adaptive_scale, kernel_poly, lib, last_error,  # noqa: F401
                   probe_shared_atomics)
from ._lib import PG_PREC_AUTO, PG_PREC_FP32, PG_PREC_FP64  # noqa: F401
from ._lib import PG_SPHERE_ANTIPODAL, PG_SPHERE_AUTO, PG_SPHERE_FIBONACCI  # noqa: F401
