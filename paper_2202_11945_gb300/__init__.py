"""GB300-native FEWHA: the per-frame hot path of the Finite Element Wavelet Hybrid
Algorithm for MCAO tomography as sm_103a CUDA kernels behind a C ABI
(include/fewha.h), with a thin Python binding."""

from .fewha import (  # noqa: F401
    AUG_MAX_ITERS, FLAG_AUGMENTED, FLAG_CLOSED_LOOP, FLAG_GRAPH, FLAG_WARM_RESIDUAL, Batch, FewhaError, Reconstructor, lib, reconstruct_batched,
    structs_from_workload,
)
