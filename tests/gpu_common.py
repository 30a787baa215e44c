"""Shared helpers of the GPU parity tests (CUDA path through the C ABI vs the oracle)."""
import numpy as np
import torch

import oracle as O
import synth

# Tolerances, derived from the arithmetic:
#  FP64 operators: a handful of roundings per output, no cancellation amplification -> 1e-12
#  FP32 operators: up to ~100 roundings of 6e-8 per output (7 wavelet levels x 12 terms,
#                  9 layers x 4-point stencils) -> 1e-5 of the largest reference entry
#  frames: DM commands after the same PCG iterations; FP32 1e-4 relative L2 (the stated
#          target); FP64 1e-8 relative L2 (the oracle's own rounding in a layer's piston
#          coefficient is amplified by 1/(alpha D_LL) ~ 1e5)
TOL_OP = {64: 1e-12, 32: 1e-5}
TOL_FRAME = {64: 1e-8, 32: 1e-4}

_cache = {}


def recon(name, precision, graph=True, warm_residual=False):
    from paper_2202_11945_gb300 import Reconstructor
    return Reconstructor(synth.workload_by_name(name), precision=precision, graph=graph,
                         warm_residual=warm_residual)


def geometry(name):
    if name not in _cache:
        g = O.Geometry(synth.workload_by_name(name))
        _cache[name] = (g, O.prior_diag(g))
    return _cache[name]


def to_dev(x, precision):
    dt = torch.float32 if precision == 32 else torch.float64
    return torch.as_tensor(np.asarray(x), dtype=dt).cuda().contiguous()


def to_np(t):
    torch.cuda.synchronize()
    return t.detach().double().cpu().numpy()


def assert_close(gpu, ref, tol, what=""):
    gpu = np.asarray(gpu, float)
    ref = np.asarray(ref, float)
    assert gpu.shape == ref.shape, (what, gpu.shape, ref.shape)
    scale = max(np.abs(ref).max(), 1e-300)
    err = np.abs(gpu - ref).max() / scale
    assert err <= tol, "%s: max |gpu - oracle| / max |oracle| = %.3e > %.1e" % (what, err, tol)
    return err


def rel_l2(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
