"""Pins of the oracle's operator M, right-hand side, preconditioner and PCG (Sec. 3)."""
import numpy as np
import pytest

import oracle as O
import synth

TOL_KRYLOV = {"tiny_scao": 1e-12, "tiny_mcao": 1e-8}


def _setup(name):
    wl = synth.workload_by_name(name)
    geo = O.Geometry(wl)
    D = O.prior_diag(geo)
    M = np.stack([O.apply_M(geo, e, D) for e in np.eye(geo.n_c)], 1)
    return wl, geo, D, M


@pytest.fixture(scope="module", params=["tiny_scao", "tiny_mcao"])
def dense(request):
    return (request.param,) + _setup(request.param)


def test_M_symmetric_positive_definite(dense):
    name, wl, geo, D, M = dense
    assert np.abs(M - M.T).max() < 1e-12 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T))[0] > 0


def test_preconditioner_diagonal_equals_bruteforce(dense):
    name, wl, geo, D, M = dense
    fast = O.data_diag(geo)
    np.testing.assert_allclose(fast, O.data_diag_bruteforce(geo), rtol=1e-12, atol=1e-12 * fast.max())
    J = O.precond_diag(geo, D)
    np.testing.assert_allclose(J, np.diag(M), rtol=1e-12)          # tau = 0: J = diag(M)
    geo.tau = 1e-2
    Jt = O.precond_diag(geo, D)
    np.testing.assert_allclose(Jt, fast + geo.alpha * np.maximum(D, 1e-2), rtol=1e-15)
    geo.tau = 0.0


def test_pcg_first_iterate_closed_form(dense):
    name, wl, geo, D, M = dense
    rng = np.random.default_rng(5)
    b = rng.standard_normal(geo.n_c)
    c0 = rng.standard_normal(geo.n_c)
    Jinv = 1.0 / np.diag(M)
    r = b - M @ c0
    z = Jinv * r
    c1 = c0 + (r @ z) / (z @ M @ z) * z
    c, _ = O.pcg(geo, b, c0, Jinv, 1, D)
    np.testing.assert_allclose(c, c1, rtol=1e-10, atol=1e-12 * np.abs(c1).max())


@pytest.mark.parametrize("k", [2, 4, 6])
def test_pcg_iterate_is_krylov_minimiser(dense, k):
    """k-th PCG iterate = argmin of the M-norm error over c0 + K_k(J^-1 M, J^-1 r0)."""
    name, wl, geo, D, M = dense
    Ms = 0.5 * (M + M.T)
    b = O.rhs(geo, synth.simulate_slopes(wl, 0))
    Jinv = 1.0 / O.precond_diag(geo, D)
    c0 = np.random.default_rng(1).standard_normal(geo.n_c)
    r0 = b - Ms @ c0
    V = []
    v = Jinv * r0
    for _ in range(k):
        for _ in range(2):
            for u in V:
                v = v - (u @ v) * u
        v = v / np.linalg.norm(v)
        V.append(v)
        v = Jinv * (Ms @ v)
    V = np.array(V).T
    ck = c0 + V @ np.linalg.solve(V.T @ Ms @ V, V.T @ r0)
    c, r = O.pcg(geo, b, c0, Jinv, k, D)
    assert np.linalg.norm(c - ck) / np.linalg.norm(ck - c0) < TOL_KRYLOV[name]
    np.testing.assert_allclose(r, b - Ms @ c, atol=1e-9 * np.abs(b).max())


def test_pcg_zero_residual_stops(dense):
    name, wl, geo, D, M = dense
    x = np.random.default_rng(2).standard_normal(geo.n_c)
    b = O.apply_M(geo, x, D)
    c, r = O.pcg(geo, b, x, np.ones(geo.n_c), 3, D)
    assert np.all(np.isfinite(c))
    np.testing.assert_allclose(c, x, atol=1e-9 * np.abs(x).max())


def test_solution_is_discrete_map_estimate(dense):
    """Eq. (5) in wavelet space is Eq. (4) in FE space with C_phi^-1 = alpha W^T D W."""
    name, wl, geo, D, M = dense
    s = synth.simulate_slopes(wl, 0)
    b = O.rhs(geo, s)
    c = np.linalg.solve(M, b)
    n = geo.n_c
    # dense FE-domain assembly from the forward model A (Eq. 1) and C_hat^-1
    E = np.eye(n)
    A = np.stack([O.forward_model(geo, geo.split(e)) for e in E], 1)       # n_s x n_c
    Cinv = np.zeros((geo.n_s, geo.n_s))
    for g, W in enumerate(geo.wfs):
        sl = slice(W["soff"], W["soff"] + W["ns"])
        Cinv[sl, sl] = np.stack([O.noise_weight(geo, g, e) for e in np.eye(W["ns"])], 1)
    Wm = np.stack([O.W_fwd(geo, geo.split(e)) for e in E], 1)
    lhs = A.T @ Cinv @ A + geo.alpha * Wm.T @ np.diag(D) @ Wm
    phi = np.linalg.solve(lhs, A.T @ Cinv @ s)
    np.testing.assert_allclose(Wm.T @ c, phi, rtol=1e-8, atol=1e-8 * np.abs(phi).max())


def test_warm_residual_identity(dense):
    """Algorithm 1: (b_new - b_old) + r_old = b_new - M c_old."""
    name, wl, geo, D, M = dense
    Jinv = 1.0 / O.precond_diag(geo, D)
    b0 = O.rhs(geo, synth.simulate_slopes(wl, 0))
    b1 = O.rhs(geo, synth.simulate_slopes(wl, 1))
    c, r = O.pcg(geo, b0, np.zeros(geo.n_c), Jinv, 3, D)
    np.testing.assert_allclose((b1 - b0) + r, b1 - M @ c, atol=1e-9 * np.abs(b1).max())
