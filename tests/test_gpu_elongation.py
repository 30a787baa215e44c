"""LGS spot elongation (Eq. 3) switched through the parameters: alpha_eta = 0 gives the
plain noise model; turning it back on gives the elongated one (operators, diagonal and
frames against the FP64 oracle)."""
import numpy as np
import pytest

import oracle as O
import synth
from tests.gpu_common import TOL_FRAME, TOL_OP, assert_close, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


def test_alpha_eta_switches_the_noise_model():
    from paper_2202_11945_gb300 import Reconstructor
    wl = synth.tiny_mcao_elongated()
    geo_el, geo_plain = O.Geometry(wl), O.Geometry(synth.tiny_mcao())
    D = O.prior_diag(geo_el)
    R = Reconstructor(wl, precision=64, graph=False)
    s = np.random.default_rng(5).standard_normal(geo_el.n_s)
    for alpha_eta, geo in ((0.0, geo_plain), (0.2, geo_el)):
        R.update_params(alpha_eta=alpha_eta)
        w = np.concatenate([O.noise_weight(geo, g, s[W["soff"]:W["soff"] + W["ns"]])
                            for g, W in enumerate(geo.wfs)])
        assert_close(to_np(R.noise_weight(to_dev(s, 64))), w, TOL_OP[64], "C^-1")
        _, J = R.diagonals()
        assert_close(to_np(J), O.precond_diag(geo, D), 1e-12, "J")
    R.close()


def test_elongated_frames_differ_from_plain_and_match_oracle():
    from paper_2202_11945_gb300 import Reconstructor
    wl = synth.tiny_mcao_elongated()
    atm = synth.TruthAtmosphere(wl["truth"])
    ref_el, ref_plain = O.Reconstructor(wl), O.Reconstructor(synth.tiny_mcao())
    R = Reconstructor(wl, precision=64, graph=True)
    for t in range(4):
        s = synth.simulate_slopes(wl, t, atm=atm)
        a_el, a_plain = ref_el.frame(s), ref_plain.frame(s)
        a = to_np(R.reconstruct(to_dev(s, 64)))
        assert rel_l2(a, a_el) <= TOL_FRAME[64], t
        assert rel_l2(a_plain, a_el) > 1e3 * TOL_FRAME[64], t     # the model matters
    R.close()
