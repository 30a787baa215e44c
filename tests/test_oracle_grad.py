"""Pins of the gradient oracle (oracle/fewha_grad.py) against definitions that do not use
its adjoint formulas: a dense finite-element-domain MAP solve, dense assembled operators,
and central finite differences of the converged map."""
import numpy as np
import pytest

import oracle as O
import synth
from oracle import fewha_grad as G

_cache = {}


def setup(name):
    if name not in _cache:
        wl = synth.workload_by_name(name)
        geo = O.Geometry(wl)
        Bd = G.data_matrix(geo)
        atm = synth.TruthAtmosphere(wl["truth"])
        s = synth.simulate_slopes(wl, 0, atm=atm)
        x, y = G.actuator_positions(geo)
        target = synth.true_phase_at(wl, x, y, 0, atm=atm)
        w = np.array([L["w"] for L in wl["layers"]])
        _cache[name] = (wl, geo, Bd, s, target, w)
    return _cache[name]


def objective(geo, Bd, s, alpha, w, target):
    _, a = G.converged_map(geo, Bd, s, alpha, w)
    return G.dm_error_objective(a, target)[0]


def columns(fn, n):
    e = np.zeros(n)
    cols = []
    for i in range(n):
        e[i] = 1.0
        cols.append(fn(e))
        e[i] = 0.0
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("name", ["tiny_scao", "tiny_mcao"])
def test_data_matrix_is_the_operator(name):
    wl, geo, Bd, s, target, w = setup(name)
    assert np.abs(Bd - Bd.T).max() <= 1e-12 * np.abs(Bd).max()
    rng = np.random.Generator(np.random.PCG64(7))
    c = rng.standard_normal(geo.n_c)
    D = O.prior_diag(geo)
    ref = O.apply_M(geo, c, D)
    got = Bd @ c + geo.alpha * D * c
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("name", ["tiny_scao", "tiny_mcao"])
def test_converged_map_is_the_fe_domain_map_estimate(name):
    """c* = W phi*, phi* minimising ||C_hat^-1/2 (s - A phi)||^2 + alpha ||D^1/2 W phi||^2,
    solved densely in the finite-element domain from the assembled A, C_hat^-1 and W."""
    wl, geo, Bd, s, target, w = setup(name)
    nphi = geo.n_c
    A = columns(lambda e: O.forward_model(geo, geo.split(e)), nphi)            # n_s x n_phi
    Ci = np.zeros((geo.n_s, geo.n_s))
    for g, W in enumerate(geo.wfs):
        sl = slice(W["soff"], W["soff"] + W["ns"])
        Ci[sl, sl] = columns(lambda e: O.noise_weight(geo, g, e), W["ns"])
    Wm = columns(lambda e: O.W_fwd(geo, geo.split(e)), nphi)                     # c = Wm phi
    D = O.prior_diag(geo, weights=w)
    H = A.T @ Ci @ A + geo.alpha * Wm.T @ np.diag(D) @ Wm
    phi = np.linalg.solve(H, A.T @ Ci @ s)
    c, a = G.converged_map(geo, Bd, s, geo.alpha, w)
    assert np.linalg.norm(Wm @ phi - c) <= 1e-8 * np.linalg.norm(c)


@pytest.mark.parametrize("name", ["tiny_scao", "tiny_mcao"])
def test_slope_gradient_equals_dense_chain(name):
    """dJ/ds = K^T M^-1 F_w^T g_a with K (the right-hand-side map) and F_w (the fit of
    coefficients) assembled column by column, not through the adjoint formulas."""
    wl, geo, Bd, s, target, w = setup(name)
    alpha = 0.4 * geo.alpha
    c, a = G.converged_map(geo, Bd, s, alpha, w)
    J, g_a = G.dm_error_objective(a, target)
    K = columns(lambda e: O.rhs(geo, e), geo.n_s)                    # n_c x n_s
    Fw = columns(lambda e: O.fit(geo, e), geo.n_c)                   # n_act x n_c
    M = Bd + alpha * np.diag(O.prior_diag(geo, weights=w))
    ref = K.T @ np.linalg.solve(M, Fw.T @ g_a)
    g_s, _, _ = G.map_gradients(geo, Bd, s, alpha, w, g_a)
    assert np.linalg.norm(g_s - ref) <= 1e-9 * np.linalg.norm(ref)


def richardson(f, x, h):
    """Central difference with one Richardson step: O(h^4) truncation, so a step large
    enough to keep the solve's rounding (cond(M) ~ 1e8) out of the difference."""
    d1 = (f(x + h) - f(x - h)) / (2 * h)
    d2 = (f(x + h / 2) - f(x - h / 2)) / h
    return (4 * d2 - d1) / 3


@pytest.mark.parametrize("name", ["tiny_scao", "tiny_mcao"])
def test_gradients_match_central_differences(name):
    wl, geo, Bd, s, target, w = setup(name)
    alpha = 2.5 * geo.alpha        # away from 1, so that a dropped alpha factor shows
    _, a = G.converged_map(geo, Bd, s, alpha, w)
    J, g_a = G.dm_error_objective(a, target)
    g_s, g_alpha, g_w = G.map_gradients(geo, Bd, s, alpha, w, g_a)
    # J is quadratic in s: central differences are exact up to rounding at any step
    rng = np.random.Generator(np.random.PCG64(11))
    for i in rng.choice(geo.n_s, 12, replace=False):
        h = 1.0
        sp, sm = s.copy(), s.copy()
        sp[i] += h
        sm[i] -= h
        fd = (objective(geo, Bd, sp, alpha, w, target) - objective(geo, Bd, sm, alpha, w, target)) / (2 * h)
        assert abs(fd - g_s[i]) <= 1e-8 * np.abs(g_s).max(), (i, fd, g_s[i])
    # alpha and the weights: the Cholesky solve of M (cond ~ 4e7) leaves ~1e-8 of rounding
    # in J, so these differences agree to ~1e-6..1e-5; a wrong term or sign is O(1)
    fd = richardson(lambda x: objective(geo, Bd, s, x, w, target), alpha, 1e-2 * alpha)
    assert abs(fd - g_alpha) <= 2e-5 * abs(g_alpha), (fd, g_alpha)
    for l in range(len(w)):
        def f(x, l=l):
            ww = w.copy()
            ww[l] = x
            return objective(geo, Bd, s, alpha, ww, target)
        fd = richardson(f, w[l], 1e-2 * w[l])
        assert abs(fd - g_w[l]) <= 2e-5 * np.abs(g_w).max(), (l, fd, g_w[l])


def test_prior_scales_inversely_with_the_weight():
    """The alpha and weight gradients rely on D_l proportional to 1 / w_l."""
    wl, geo, Bd, s, target, w = setup("tiny_mcao")
    D1 = O.prior_diag(geo, weights=w)
    w2 = w.copy()
    w2[1] *= 3.0
    D2 = O.prior_diag(geo, weights=w2)
    L = geo.layers[1]
    sl = slice(L["off"], L["off"] + L["n"] ** 2)
    assert np.allclose(D2[sl], D1[sl] / 3.0, rtol=1e-14)
    rest = np.ones(geo.n_c, bool)
    rest[sl] = False
    assert np.array_equal(D2[rest], D1[rest])


# -- reverse mode through the fixed-iteration frame -----------------------------------


@pytest.mark.parametrize("name,k", [("tiny_scao", 1), ("tiny_scao", 4), ("tiny_mcao", 4)])
def test_unrolled_vjp_matches_central_differences(name, k):
    """The reverse pass against central differences of the forward map (h = 1e-4 of the
    slopes' scale) in seeded random directions, warm start c0 != 0."""
    wl = synth.workload_by_name(name)
    geo = O.Geometry(wl)
    D = O.prior_diag(geo)
    s = synth.simulate_slopes(wl, 1)
    rng = np.random.default_rng(11)
    c0 = 0.1 * rng.standard_normal(geo.n_c)
    g_a = rng.standard_normal(geo.n_a)
    a, _, tape = G.unrolled_frame(geo, s, c0, k, D)
    gs = G.unrolled_frame_vjp(geo, tape, g_a)

    def J(x):
        return float(g_a @ G.unrolled_frame(geo, x, c0, k, D)[0])

    h = 1e-4 * np.abs(s).max()
    for _ in range(3):
        v = rng.standard_normal(geo.n_s)
        fd = (J(s + h * v) - J(s - h * v)) / (2 * h)
        assert abs(fd - gs @ v) <= 1e-6 * (abs(fd) + np.linalg.norm(gs) * np.linalg.norm(v) * 1e-3), (fd, gs @ v)


def test_unrolled_vjp_euler_identity():
    """From c0 = 0 every PCG iterate is homogeneous of degree one in b (alpha, beta are
    ratios of quadratic forms), so s . dJ/ds = J(s) exactly."""
    wl = synth.tiny_mcao()
    geo = O.Geometry(wl)
    s = synth.simulate_slopes(wl, 2)
    g_a = np.random.default_rng(4).standard_normal(geo.n_a)
    a, _, tape = G.unrolled_frame(geo, s, np.zeros(geo.n_c), 4)
    gs = G.unrolled_frame_vjp(geo, tape, g_a)
    assert abs(gs @ s - g_a @ a) <= 1e-7 * abs(g_a @ a)


def test_unrolled_frame_is_the_oracle_frame():
    """The differentiated map is the frame of Algorithm 1 (explicit r0, gain 1)."""
    wl = synth.tiny_mcao()
    ref = O.Reconstructor(wl)
    s0, s1 = synth.simulate_slopes(wl, 0), synth.simulate_slopes(wl, 1)
    ref.frame(s0)
    c0 = ref.c.copy()
    a = ref.frame(s1)
    a2, c2, _ = G.unrolled_frame(ref.geo, s1, c0, wl["params"]["iters"])
    np.testing.assert_allclose(a2, a, rtol=0, atol=1e-12 * np.abs(a).max())
