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


def _frame_dirs(wl, geo, D, k):
    """A cold k-iteration augmented solve of frame 0: its start, residual and directions."""
    Jinv = 1.0 / O.precond_diag(geo, D)
    b = O.rhs(geo, synth.simulate_slopes(wl, 0))
    c0 = np.zeros(geo.n_c)
    c, r, dirs = O.augmented_pcg(geo, b, c0, Jinv, k, D)
    return Jinv, b, c0, c, r, dirs


@pytest.mark.parametrize("k", [1, 4])
def test_augmented_deflation_reproduces_the_cg_iterate(dense, k):
    """Sec. 3.4 augmentation: deflating a start over the directions that CG generated
    from that start gives the CG iterate itself (the iterate minimises the M-norm error
    over c0 + span(P), and y_k = p_k.r0 / p_k.q_k equals CG's alpha_k)."""
    name, wl, geo, D, M = dense
    Jinv, b, c0, c, r, dirs = _frame_dirs(wl, geo, D, k)
    cd, rd, _ = O.augmented_pcg(geo, b, c0, Jinv, 0, D, r0=b - M @ c0, prev=dirs)
    tol = TOL_KRYLOV[name]
    assert np.linalg.norm(cd - c) <= tol * np.linalg.norm(c)
    assert np.linalg.norm(rd - r) <= tol * np.linalg.norm(b)


def test_augmented_directions_are_conjugate_images(dense):
    name, wl, geo, D, M = dense
    _, _, _, _, _, (P, Q, pq) = _frame_dirs(wl, geo, D, 4)
    assert len(P) == len(Q) == len(pq) == 4
    for i in range(4):
        np.testing.assert_allclose(Q[i], M @ P[i], rtol=0, atol=1e-12 * np.abs(Q[i]).max())
        assert abs(pq[i] - P[i] @ M @ P[i]) <= 1e-12 * pq[i]
        for j in range(i):
            assert abs(P[i] @ M @ P[j]) <= TOL_KRYLOV[name] * np.sqrt(pq[i] * pq[j])


def test_augmented_start_is_the_galerkin_projection(dense):
    """The deflated start of the next frame equals the M-orthogonal projection computed
    with the dense M and the full Gram matrix, and its residual is b - M c0'."""
    name, wl, geo, D, M = dense
    Jinv, b0, _, c, r, dirs = _frame_dirs(wl, geo, D, 4)
    b1 = O.rhs(geo, synth.simulate_slopes(wl, 1))
    P = np.array(dirs[0]).T
    ref = c + P @ np.linalg.solve(P.T @ M @ P, P.T @ (b1 - M @ c))
    r0 = (b1 - b0) + r                                     # the warm form of Algorithm 1
    cd, rd, _ = O.augmented_pcg(geo, b1, c, Jinv, 0, D, r0=r0, prev=dirs)
    tol = TOL_KRYLOV[name]
    assert np.linalg.norm(cd - ref) <= tol * np.linalg.norm(ref - c)
    np.testing.assert_allclose(rd, b1 - M @ cd, atol=1e-9 * np.abs(b1).max())
    assert np.abs(P.T @ rd).max() <= tol * np.linalg.norm(P, axis=0).max() * np.linalg.norm(r0)


@pytest.mark.parametrize("k", [2, 4])
def test_augmented_iterate_is_krylov_minimiser_of_the_projected_preconditioner(dense, k):
    """With the new directions M-conjugate to P, the augmented PCG is PCG from the
    deflated start with the preconditioner B = Pi J^-1 Pi^T, Pi = I - P (P^T M P)^-1 P^T M
    (dense, full Gram matrix): its k-th iterate minimises the M-norm error over
    c0' + K_k(B M, B r0')."""
    name, wl, geo, D, M = dense
    Ms = 0.5 * (M + M.T)
    Jinv, b0, _, c, r, dirs = _frame_dirs(wl, geo, D, 4)
    b1 = O.rhs(geo, synth.simulate_slopes(wl, 1))
    P = np.array(dirs[0]).T
    Pi = np.eye(geo.n_c) - P @ np.linalg.solve(P.T @ Ms @ P, P.T @ Ms)
    B = Pi @ np.diag(Jinv) @ Pi.T
    c0d = c + P @ np.linalg.solve(P.T @ Ms @ P, P.T @ (b1 - Ms @ c))
    r0d = b1 - Ms @ c0d
    V = []
    v = B @ r0d
    for _ in range(k):
        for _ in range(2):
            for u in V:
                v = v - (u @ v) * u
        v = v / np.linalg.norm(v)
        V.append(v)
        v = B @ (Ms @ v)
    V = np.array(V).T
    ck = c0d + V @ np.linalg.solve(V.T @ Ms @ V, V.T @ r0d)
    cg, _, new = O.augmented_pcg(geo, b1, c, Jinv, k, D, prev=dirs)
    assert np.linalg.norm(cg - ck) / np.linalg.norm(ck - c) < TOL_KRYLOV[name]
    assert len(new[0]) == k
    # the new directions are M-conjugate to the previous frame's
    for pn in new[0]:
        assert np.abs(P.T @ Ms @ pn).max() <= TOL_KRYLOV[name] * np.sqrt(pn @ Ms @ pn) * np.sqrt(
            np.diag(P.T @ Ms @ P)).max()


def test_augmented_frames_reduce_the_error_of_the_warm_start(dense):
    """Sec. 3.4: reusing the previous directions lowers the error of a fixed small
    iteration count.  Over a frozen-flow sequence at iter = 2, the mean M-norm error of
    the augmented frames (against the exact solve of each frame) is below that of the
    plain warm-started frames."""
    name, wl, geo, D, M = dense
    atm = synth.TruthAtmosphere(wl["truth"])
    seq = [synth.simulate_slopes(wl, t, atm=atm) for t in range(10)]
    err = {}
    for aug in (False, True):
        R = O.Reconstructor(wl)
        R.geo.iters = 2
        e = []
        for s in seq:
            R.frame(s, augmented=aug)
            b = O.rhs(R.geo, s)
            cs = np.linalg.solve(M, b)
            d = R.c - cs
            e.append(np.sqrt(d @ M @ d / (cs @ M @ cs)))
        err[aug] = np.mean(e[2:])
    assert err[True] < 0.9 * err[False], err
