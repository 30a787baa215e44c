"""Reverse mode through the fixed-iteration frame on the CUDA path (fewha_frame_vjp)
against the FP64 oracle's reverse pass, through torch.autograd, and with the handle's
warm state left untouched."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from oracle import fewha_grad as G
from tests.gpu_common import TOL_FRAME, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

# The reverse pass keeps the forward vectors in the operator precision and forms its
# scalars in double on the host: FP64 follows the oracle to rounding.  The adjoint
# vectors carry a large piston component (J^-1 of a full-depth layer's piston coefficient
# is ~1 / (alpha D_LL) ~ 1e5), which the data path of every M apply and the final slope
# map leave out (Gamma annihilates constants), so float rounding of it cannot leak into
# the other components: the FP32 gradient then follows the oracle to ~1e-6 (CPU
# emulation with float rounding at every operator stage), checked at 1e-4.
TOL_GRAD = {64: 1e-8, 32: 1e-4}


def case(name):
    wl = synth.workload_by_name(name)
    ref = O.Reconstructor(wl)
    atm = synth.TruthAtmosphere(wl["truth"])
    ref.frame(synth.simulate_slopes(wl, 0, atm=atm))
    c0 = ref.c.copy()
    s = synth.simulate_slopes(wl, 1, atm=atm)
    g_a = np.random.default_rng(21).standard_normal(ref.geo.n_a)
    a, _, tape = G.unrolled_frame(ref.geo, s, c0, wl["params"]["iters"], ref.D)
    gs = G.unrolled_frame_vjp(ref.geo, tape, g_a)
    return wl, s, c0, g_a, a, gs


@pytest.mark.parametrize("name,prec", [("tiny_scao", 64), ("tiny_scao", 32), ("tiny_mcao", 64),
                                       ("tiny_mcao", 32), ("maory", 32), ("maory", 64)], ids=str)
def test_frame_vjp_matches_oracle(name, prec):
    from paper_2202_11945_gb300 import Reconstructor
    wl, s, c0, g_a, a_ref, gs_ref = case(name)
    R = Reconstructor(wl, precision=prec, graph=False)
    a, gs = R.frame_vjp(to_dev(s, prec), to_dev(c0, prec), to_dev(g_a, prec))
    assert rel_l2(to_np(a), a_ref) <= TOL_FRAME[prec], rel_l2(to_np(a), a_ref)
    g = to_np(gs)
    assert rel_l2(g, gs_ref) <= TOL_GRAD[prec], rel_l2(g, gs_ref)
    a2, none = R.frame_vjp(to_dev(s, prec), to_dev(c0, prec))        # forward only
    assert none is None and np.array_equal(to_np(a2), to_np(a))
    R.close()


def test_autograd_frame_and_untouched_warm_state():
    from paper_2202_11945_gb300 import Reconstructor
    from paper_2202_11945_gb300 import autograd as AG
    wl, s, c0, g_a, a_ref, gs_ref = case("tiny_mcao")
    A = Reconstructor(wl, precision=64, graph=True)
    B = Reconstructor(wl, precision=64, graph=True)
    s0 = to_dev(synth.simulate_slopes(wl, 0), 64)
    A.reconstruct(s0)
    B.reconstruct(s0)
    sl = to_dev(s, 64).requires_grad_(True)
    a = AG.frame(A, sl, to_dev(c0, 64))
    (a * to_dev(g_a, 64)).sum().backward()
    assert rel_l2(to_np(sl.grad), gs_ref) <= TOL_GRAD[64]
    # the vjp left A's frame state alone: its next frames equal B's bit for bit
    for t in (2, 3):
        st = to_dev(synth.simulate_slopes(wl, t), 64)
        assert np.array_equal(to_np(A.reconstruct(st)), to_np(B.reconstruct(st))), t
    A.close()
    B.close()
