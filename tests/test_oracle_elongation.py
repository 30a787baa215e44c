"""Pins of the oracle's LGS spot-elongation noise model (Eq. 3, reading R28)."""
import numpy as np
import pytest

import oracle as O
import synth


def _dense_weight(geo, g):
    return np.stack([O.noise_weight(geo, g, e) for e in np.eye(geo.wfs[g]["ns"])], 1)


def _paper_blocks_weight(wl, geo, g):
    """(I - T) C_g^-1 (I - T) assembled from Eq. 3's 2x2 blocks, each inverted with
    numpy, and T of Sec. 3.2 as a dense matrix."""
    W, Wd = geo.wfs[g], wl["wfs"][g]
    k = W["n_active"]
    N, d = W["N"], W["d"]
    ii, jj = np.nonzero(W["mask"])                         # row-major = slope order
    x, y = -geo.D / 2 + (jj + 0.5) * d, -geo.D / 2 + (ii + 0.5) * d
    fw, H, f = Wd["na_fwhm"], Wd["H"], Wd["spot_fwhm"]
    a_eta = wl["params"]["alpha_eta"]
    Cinv = np.zeros((2 * k, 2 * k))
    for a in range(k):
        beta = fw / H ** 2 * np.array([x[a] - Wd["launch"][0], y[a] - Wd["launch"][1]])
        C = W["sigma"] ** 2 * (np.eye(2) + (a_eta / f) ** 2 * np.outer(beta, beta))
        Ci = np.linalg.inv(C)
        idx = [a, k + a]
        Cinv[np.ix_(idx, idx)] = Ci
    t = np.zeros((2 * k, 2))
    t[:k, 0] = 1.0
    t[k:, 1] = 1.0
    P = np.eye(2 * k) - t @ t.T / k
    return P @ Cinv @ P


@pytest.mark.parametrize("name", ["tiny_mcao_elongated", "paper_mcao"])
def test_weight_equals_the_inverted_blocks_of_eq3(name):
    wl = synth.workload_by_name(name)
    geo = O.Geometry(wl)
    g = 0 if name == "tiny_mcao_elongated" else 1
    if name == "paper_mcao":
        # a dense check on 74 x 74 subapertures is large: compare on random vectors
        ref = _paper_blocks_weight(wl, geo, g)
        rng = np.random.default_rng(2)
        for _ in range(3):
            v = rng.standard_normal(geo.wfs[g]["ns"])
            np.testing.assert_allclose(O.noise_weight(geo, g, v), ref @ v, rtol=1e-10,
                                       atol=1e-10 * np.abs(ref @ v).max())
        return
    np.testing.assert_allclose(_dense_weight(geo, g), _paper_blocks_weight(wl, geo, g),
                               rtol=1e-10, atol=1e-12 * np.abs(_dense_weight(geo, g)).max())


def test_elongation_changes_the_weight_and_off_is_the_plain_model():
    wl = synth.tiny_mcao_elongated()
    geo = O.Geometry(wl)
    plain = O.Geometry(synth.tiny_mcao())
    A, B = _dense_weight(geo, 0), _dense_weight(plain, 0)
    assert np.abs(A - B).max() > 0.05 * np.abs(B).max()          # the term is of order one
    O.set_elongation(geo, 0.0)
    np.testing.assert_array_equal(_dense_weight(geo, 0), B)


def test_elongated_weight_is_symmetric_psd_and_blind_to_tip_tilt():
    geo = O.Geometry(synth.tiny_mcao_elongated())
    for g in (0, 1):
        A = _dense_weight(geo, g)
        k = geo.wfs[g]["n_active"]
        np.testing.assert_allclose(A, A.T, atol=1e-12 * np.abs(A).max())
        assert np.linalg.eigvalsh(0.5 * (A + A.T))[0] > -1e-10 * np.abs(A).max()
        tx = np.r_[np.ones(k), np.zeros(k)]
        ty = np.r_[np.zeros(k), np.ones(k)]
        assert np.abs(A @ tx).max() < 1e-10 * np.abs(A).max()
        assert np.abs(A @ ty).max() < 1e-10 * np.abs(A).max()


def test_fast_diagonal_with_elongation_equals_bruteforce():
    geo = O.Geometry(synth.tiny_mcao_elongated())
    fast = O.data_diag(geo)
    np.testing.assert_allclose(fast, O.data_diag_bruteforce(geo), rtol=1e-11, atol=1e-12 * fast.max())
    plain = O.data_diag(O.Geometry(synth.tiny_mcao()))
    assert np.abs(fast - plain).max() > 1e-3 * plain.max()


def test_converged_solution_is_the_dense_map_with_elongated_noise():
    """Eq. 5 with the elongated C_eta: the oracle's M and b solve to the dense MAP of Eq. 4
    assembled from the forward model and the inverted blocks of Eq. 3."""
    wl = synth.tiny_mcao_elongated()
    geo = O.Geometry(wl)
    D = O.prior_diag(geo)
    s = synth.simulate_slopes(wl, 0)
    M = np.stack([O.apply_M(geo, e, D) for e in np.eye(geo.n_c)], 1)
    c = np.linalg.solve(M, O.rhs(geo, s))
    E = np.eye(geo.n_c)
    A = np.stack([O.forward_model(geo, geo.split(e)) for e in E], 1)
    Cinv = np.zeros((geo.n_s, geo.n_s))
    for g, W in enumerate(geo.wfs):
        sl = slice(W["soff"], W["soff"] + W["ns"])
        if W["el"] is not None:
            Cinv[sl, sl] = _paper_blocks_weight(wl, geo, g)
        else:
            Cinv[sl, sl] = _dense_weight(geo, g)
    Wm = np.stack([O.W_fwd(geo, geo.split(e)) for e in E], 1)
    lhs = A.T @ Cinv @ A + geo.alpha * Wm.T @ np.diag(D) @ Wm
    phi = np.linalg.solve(lhs, A.T @ Cinv @ s)
    np.testing.assert_allclose(Wm.T @ c, phi, rtol=1e-8, atol=1e-8 * np.abs(phi).max())
