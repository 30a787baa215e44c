"""Pins of the oracle's whole frame (Algorithm 1, open loop)."""
import numpy as np

import oracle as O
import synth
from synth.sensor import true_phase_at


def test_zero_slopes_give_zero_commands():
    R = O.Reconstructor(synth.tiny_mcao())
    a = R.frame(np.zeros(R.geo.n_s))
    assert np.all(a == 0.0)


def test_cold_frame_is_linear_in_the_slopes():
    wl = synth.tiny_mcao()
    s1 = synth.simulate_slopes(wl, 0)
    s2 = synth.simulate_slopes(wl, 1)
    a1 = O.Reconstructor(wl).frame(s1)
    a2 = O.Reconstructor(wl).frame(s2)
    a12 = O.Reconstructor(wl).frame(2.0 * s1 - 0.5 * s2)
    # PCG is not linear in b (alpha_k depends on b), but scaling is exact up to rounding.
    # Rounding in a full-depth layer's piston coefficient (seen only by the prior, J =
    # alpha D_LL ~ 1e-5) is amplified ~1e5, hence 1e-8 rather than 1e-15.
    a3 = O.Reconstructor(wl).frame(3.0 * s1)
    assert np.linalg.norm(a3 - 3.0 * a1) / np.linalg.norm(3.0 * a1) < 1e-8
    assert np.linalg.norm(a12 - (2 * a1 - 0.5 * a2)) > 0  # documented non-linearity of fixed-k CG


def test_open_loop_gain():
    wl = synth.tiny_scao()
    wl["params"]["gain"] = 0.6
    R = O.Reconstructor(wl)
    s = synth.simulate_slopes(wl, 0)
    a1 = R.frame(s)
    c_after = R.c.copy()
    a_t1 = O.fit(R.geo, c_after)
    np.testing.assert_allclose(a1, 0.6 * a_t1, rtol=1e-14)
    a2 = R.frame(synth.simulate_slopes(wl, 1))
    np.testing.assert_allclose(a2, 0.4 * a1 + 0.6 * O.fit(R.geo, R.c), rtol=1e-13)


def test_warm_started_frames_follow_the_truth():
    """Physics sanity: the fitted on-axis DM shape correlates with the true phase."""
    wl = synth.tiny_scao()
    R = O.Reconstructor(wl)
    for t in range(6):
        a = R.frame(synth.simulate_slopes(wl, t))
    na = 17
    xa = (np.arange(na) - 8) * 0.5
    X, Y = np.meshgrid(xa, xa)
    tp = true_phase_at(wl, X, Y, 5)
    inside = np.hypot(X, Y) <= 4.0
    A = a.reshape(na, na)[inside]
    T = tp[inside]
    A, T = A - A.mean(), T - T.mean()
    assert (A @ T) / np.linalg.norm(A) / np.linalg.norm(T) > 0.9


def test_warm_residual_option_matches_explicit_residual():
    wl = synth.tiny_mcao()
    R1, R2 = O.Reconstructor(wl), O.Reconstructor(wl)
    for t in range(3):
        s = synth.simulate_slopes(wl, t)
        a1 = R1.frame(s)
        a2 = R2.frame(s, warm_residual=True)
    np.testing.assert_allclose(a2, a1, rtol=1e-8, atol=1e-8 * np.abs(a1).max())
