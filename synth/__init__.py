"""Seeded synthetic inputs for FEWHA workloads.

This package is shared by the tests, the FP64 oracle's checks and the benchmark.
It holds workload descriptions (telescope, guide stars, layers, mirrors,
parameters), seeded von Karman phase screens with frozen flow, and a synthetic
Shack-Hartmann measurement simulation of the *true* atmosphere.  It holds none
of the reconstructor's arithmetic: no wavelet transform, no layer projection
operator, no slope operator of the reconstruction model, no prior, no solver.

Seeds (NumPy PCG64): truth screen k -> 1000 + k, noise of frame t -> 2000 + t,
wind -> 3000, batched instance i -> 4000 + i.
"""

from .configs import (  # noqa: F401
    tiny_scao, tiny_mcao, maory, realtime_loop, batched_instances, differentiable,
    workload_by_name, arcsec, with_elongation, paper_mcao, tiny_mcao_elongated,
)
from .atmosphere import TruthAtmosphere  # noqa: F401
from .sensor import simulate_slopes, slope_counts, slope_sequence, true_phase_at  # noqa: F401
