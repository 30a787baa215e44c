"""Augmented PCG (Sec. 3.4, the augPCG step of Algorithm 1) on the CUDA path against the
FP64 oracle: frame sequences (explicit and warm initial residual), the graph and stream
forms, the directions dropped by a parameter update, and the argument limits."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from tests.gpu_common import TOL_FRAME, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

_atm = {}


def slopes(name, t):
    wl = synth.workload_by_name(name)
    if name not in _atm:
        _atm[name] = synth.TruthAtmosphere(wl["truth"])
    return synth.simulate_slopes(wl, t, atm=_atm[name])


def recon(name, prec, **kw):
    from paper_2202_11945_gb300 import Reconstructor
    return Reconstructor(synth.workload_by_name(name), precision=prec, augmented=True, **kw)


SEQ = [("tiny_scao", 64, 8, False), ("tiny_scao", 32, 8, False), ("tiny_mcao", 64, 8, True),
       ("tiny_mcao", 32, 8, False), ("tiny_mcao", 32, 8, True), ("maory", 32, 4, False),
       ("maory", 64, 3, True)]


@pytest.mark.parametrize("name,prec,frames,warm", SEQ, ids=lambda x: str(x))
def test_augmented_sequence_matches_oracle(name, prec, frames, warm):
    """Frame 0 unaugmented, then frames augmented by the previous frame's directions."""
    ref = O.Reconstructor(synth.workload_by_name(name))
    R = recon(name, prec, warm_residual=warm)
    for t in range(frames):
        s = slopes(name, t)
        a_ref = ref.frame(s, warm_residual=warm, augmented=True)
        a = to_np(R.reconstruct(to_dev(s, prec)))
        assert rel_l2(a, a_ref) <= TOL_FRAME[prec], (t, rel_l2(a, a_ref))
    R.close()


def test_residual_matches_oracle():
    """The recurrence residual and right-hand side of the last frame (FP64)."""
    ref = O.Reconstructor(synth.workload_by_name("tiny_mcao"))
    R = recon("tiny_mcao", 64)
    for t in range(3):
        s = slopes("tiny_mcao", t)
        ref.frame(s, augmented=True)
        R.reconstruct(to_dev(s, 64))
    r, _ = R.residual(with_b=False)       # the explicit frame forms r0 without b
    b = R.rhs(to_dev(slopes("tiny_mcao", 2), 64))
    b_ref = O.rhs(ref.geo, slopes("tiny_mcao", 2))
    r_ref = b_ref - O.apply_M(ref.geo, ref.c, ref.D)
    assert rel_l2(to_np(b), b_ref) <= 1e-12
    assert rel_l2(to_np(r), r_ref) <= 1e-6          # recurrence vs true residual of the oracle
    R.close()


def test_graph_and_stream_forms_are_bitwise_identical():
    A = recon("tiny_mcao", 32, graph=True)
    B = recon("tiny_mcao", 32, graph=False)
    for t in range(5):                                # both direction sets, each twice
        s = to_dev(slopes("tiny_mcao", t), 32)
        assert np.array_equal(to_np(A.reconstruct(s)), to_np(B.reconstruct(s))), t
    A.close()
    B.close()


def test_parameter_update_drops_the_directions():
    """After update_params the next frame runs unaugmented, from the carried c, with an
    explicit initial residual; later frames augment again."""
    name, alpha2 = "tiny_mcao", 2.0
    ref = O.Reconstructor(synth.workload_by_name(name))
    R = recon(name, 64, warm_residual=True)
    for t in range(3):
        s = slopes(name, t)
        ref.frame(s, warm_residual=True, augmented=True)
        R.reconstruct(to_dev(s, 64))
    R.update_params(alpha=alpha2)
    ref.geo.alpha = alpha2
    ref.J = O.precond_diag(ref.geo, ref.D)
    ref.Jinv = 1.0 / ref.J
    ref.dirs = None
    ref.b_prev = ref.r_prev = None
    for t in range(3, 6):
        s = slopes(name, t)
        a_ref = ref.frame(s, warm_residual=True, augmented=True)
        a = to_np(R.reconstruct(to_dev(s, 64)))
        assert rel_l2(a, a_ref) <= TOL_FRAME[64], (t, rel_l2(a, a_ref))
    R.close()


def test_augmentation_can_be_switched_on_and_off():
    """Turning it off gives plain frames; on again, the first frame is unaugmented (each
    switch is a parameter update, which also drops the directions)."""
    name = "tiny_scao"
    R = recon(name, 64)
    ref = O.Reconstructor(synth.workload_by_name(name))
    modes = [True, True, False, False, True, True]
    for t, aug in enumerate(modes):
        if t > 0 and aug != modes[t - 1]:
            R.update_params(augmented=aug)
            ref.dirs = None
        s = slopes(name, t)
        a_ref = ref.frame(s, augmented=aug)
        a = to_np(R.reconstruct(to_dev(s, 64)))
        assert rel_l2(a, a_ref) <= TOL_FRAME[64], (t, aug)
    R.close()


def test_limits_and_batches():
    from paper_2202_11945_gb300 import AUG_MAX_ITERS, Batch, FewhaError
    R = recon("tiny_scao", 32)
    with pytest.raises(FewhaError):
        R.update_params(iters=AUG_MAX_ITERS + 1)
    R.update_params(iters=AUG_MAX_ITERS)
    a = to_np(R.reconstruct(to_dev(slopes("tiny_scao", 0), 32)))
    assert np.all(np.isfinite(a))
    R.close()
    A, B = recon("tiny_scao", 32), recon("tiny_mcao", 32)
    bt = Batch([A, B])
    with pytest.raises(FewhaError):
        bt.reconstruct([to_dev(slopes("tiny_scao", 0), 32), to_dev(slopes("tiny_mcao", 0), 32)])
    bt.close()
    A.close()
    B.close()
