"""fewha_apply_M_noalloc: the M-apply whose scratch is the library's static device block.

It exists for callers that may not allocate device memory when they need the operator
(for example a monitoring thread of a real-time loop that allocates everything at
start-up and forbids cudaMalloc afterwards).  Its result must equal the ordinary
fewha_apply_M on the same handle, call after call, although the static block keeps
whatever the previous call left in it.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
from tests.gpu_common import TOL_OP, assert_close, recon, to_dev, to_np

pytestmark = pytest.mark.gpu


def _noalloc(R, c, q):
    rc = R.L.fewha_apply_M_noalloc(R.h, ctypes.c_void_p(c.data_ptr()), ctypes.c_void_p(q.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc


# the elongated geometries exercise the LGS spot-elongation weighting (Eq. 3) of the
# single-CTA sensor kernel this entry point runs, against the cluster kernels of apply_M
@pytest.mark.parametrize("name,prec", [("tiny_mcao", 64), ("tiny_mcao", 32), ("maory", 32),
                                       ("maory", 64), ("tiny_mcao_elongated", 64),
                                       ("tiny_mcao_elongated", 32), ("paper_mcao", 32),
                                       ("paper_mcao", 64)])
def test_matches_apply_M_on_consecutive_calls(name, prec):
    R = recon(name, prec)
    rng = np.random.default_rng(77)
    for call in range(2):
        c = to_dev(rng.standard_normal(R.n_coeffs), prec)
        q_ref = to_np(R.apply_M(c))
        q = torch.full((R.n_coeffs,), float("nan"), dtype=R.dtype, device="cuda")
        assert _noalloc(R, c, q) == 0, R.L.fewha_last_error(R.h)
        assert_close(to_np(q), q_ref, TOL_OP[prec], "%s fp%d call %d" % (name, prec, call))
    R.close()


def test_rejects_an_instance_larger_than_the_block():
    wl = synth.maory()
    d = wl["layers"][0]["delta"]
    hs = np.linspace(0.0, 4500.0, 16)
    wl["layers"] = [dict(h=float(h), w=1.0 / 16, delta=d, n=128, levels=7) for h in hs]
    R = recon_from(wl, 64)
    c = torch.zeros(R.n_coeffs, dtype=torch.float64, device="cuda")
    q = torch.full((R.n_coeffs,), 7.0, dtype=torch.float64, device="cuda")
    assert _noalloc(R, c, q) == -6
    assert b"static block" in R.L.fewha_last_error(R.h)
    assert bool(torch.all(q == 7.0))          # nothing was launched
    R.close()


def recon_from(wl, prec):
    from paper_2202_11945_gb300 import Reconstructor
    return Reconstructor(wl, precision=prec)
