"""Pins of the oracle's forward-model operators (Sec. 2, Sec. 3.2)."""
import math

import numpy as np
import pytest

import oracle as O
import synth


def _geo(name):
    return O.Geometry(synth.workload_by_name(name))


def _rel(a, b):
    return abs(a - b) / max(abs(a), abs(b), 1e-300)


# ---------------------------------------------------------------- Shack-Hartmann
def _nodes(N, d, f):
    x = -N * d / 2 + np.arange(N + 1) * d
    X, Y = np.meshgrid(x, x)
    return f(X, Y)


def test_slopes_of_constant_and_waffle_vanish():
    sx, sy = O.fine_slopes(np.full((9, 9), 2.5))
    assert np.abs(sx).max() == 0 and np.abs(sy).max() == 0
    i, j = np.mgrid[0:9, 0:9]
    sx, sy = O.fine_slopes((-1.0) ** (i + j))
    assert np.abs(sx).max() < 1e-15 and np.abs(sy).max() < 1e-15


def test_slopes_of_tip_and_tilt_are_exact():
    d, N, t = 0.5, 8, 0.37
    sx, sy = O.fine_slopes(_nodes(N, d, lambda X, Y: t * X))
    np.testing.assert_allclose(sx, t * d, atol=1e-14)
    np.testing.assert_allclose(sy, 0.0, atol=1e-14)   # the literal printed y formula gives t*d/2
    sx, sy = O.fine_slopes(_nodes(N, d, lambda X, Y: t * Y))
    np.testing.assert_allclose(sy, t * d, atol=1e-14)
    np.testing.assert_allclose(sx, 0.0, atol=1e-14)


def test_slopes_of_bilinear_phase_are_average_gradients():
    """phi = x*y: mean of d(phi)/dx over a cell is its centre y; slope = that times d."""
    d, N = 0.5, 8
    sx, sy = O.fine_slopes(_nodes(N, d, lambda X, Y: X * Y))
    c = -N * d / 2 + (np.arange(N) + 0.5) * d
    np.testing.assert_allclose(sx, np.tile(c[:, None], (1, N)) * d, atol=1e-14)
    np.testing.assert_allclose(sy, np.tile(c[None, :], (N, 1)) * d, atol=1e-14)


def test_active_subaperture_counts():
    assert O.active_mask(16, 8.0, 0.0).sum() == 208
    assert O.active_mask(80, 39.0, 0.28).sum() == 4632
    m = O.active_mask(80, 39.0, 0.28)
    assert not m[40, 40] and not m[0, 0] and m[40, 5]


def test_coarse_sensor_measures_coarse_tilt():
    geo = _geo("tiny_mcao")
    g = 2
    W = geo.wfs[g]
    N, d, t = W["N"], W["d"], 0.21
    s = O.sh_slopes(geo, g, _nodes(N, d, lambda X, Y: t * X))
    k = W["n_active"]
    coarse = geo.D / W["n_sub"]
    # full blocks: every fine subaperture active -> exactly the coarse phase difference
    full = [K for K, (I, J) in enumerate(zip(*np.nonzero(W["cmask"])))
            if W["mask"][I * W["nb"]:(I + 1) * W["nb"], J * W["nb"]:(J + 1) * W["nb"]].all()]
    frac = np.array([W["mask"][I * 4:(I + 1) * 4, J * 4:(J + 1) * 4].mean()
                     for I, J in zip(*np.nonzero(W["cmask"]))])
    np.testing.assert_allclose(s[:k], t * coarse * frac, atol=1e-14)
    np.testing.assert_allclose(s[k:], 0.0, atol=1e-14)
    assert all(f <= 1 for f in frac) and len(full) + (frac < 1).sum() == k


# ---------------------------------------------------------------- adjoints
@pytest.mark.parametrize("name", ["tiny_scao", "tiny_mcao"])
def test_adjoint_identities(name):
    geo = _geo(name)
    rng = np.random.default_rng(7)
    phis = [rng.standard_normal((L["n"], L["n"])) for L in geo.layers]
    for g, W in enumerate(geo.wfs):
        v = rng.standard_normal((W["N"] + 1, W["N"] + 1))
        lhs = sum((a * b).sum() for a, b in zip(O.project_adj(geo, g, v), phis))
        assert _rel((O.project(geo, g, phis) * v).sum(), lhs) < 1e-12
        s = rng.standard_normal(W["ns"])
        assert _rel(O.sh_slopes(geo, g, v) @ s, (v * O.sh_slopes_adj(geo, g, s)).sum()) < 1e-12
        s2 = rng.standard_normal(W["ns"])
        assert _rel(O.noise_weight(geo, g, s) @ s2, s @ O.noise_weight(geo, g, s2)) < 1e-12
    s = rng.standard_normal(geo.n_s)
    lhs = O.forward_model(geo, phis) @ s
    rhs = sum((a * b).sum() for a, b in zip(phis, O.forward_model_adj(geo, s)))
    assert _rel(lhs, rhs) < 1e-12
    c = rng.standard_normal(geo.n_c)
    x = O.W_inv(geo, c)
    assert _rel(O.W_fwd(geo, phis) @ c, sum((a * b).sum() for a, b in zip(phis, x))) < 1e-12
    a = rng.standard_normal(geo.n_a)
    assert _rel(O.fit(geo, c) @ a, c @ O.fit_adj(geo, a)) < 1e-12


# ---------------------------------------------------------------- projection
def test_projection_of_constant_layers_is_their_sum():
    geo = _geo("tiny_mcao")
    consts = [1.5, -0.25, 4.0]
    phis = [np.full((L["n"], L["n"]), c) for c, L in zip(consts, geo.layers)]
    for g in range(len(geo.wfs)):
        np.testing.assert_allclose(O.project(geo, g, phis), sum(consts), atol=1e-13)


def test_projection_of_linear_layer_is_exact():
    """Layer phi(x, y) = a x + b y: P gives a (s x + theta_x h) + b (s y + theta_y h)."""
    wl = synth.tiny_mcao()
    geo = O.Geometry(wl)
    a, b = 0.3, -0.7
    for li, L in enumerate(geo.layers):
        n, dl = L["n"], L["delta"]
        xs = (np.arange(n) - n / 2) * dl
        X, Y = np.meshgrid(xs, xs)
        phis = [np.zeros((M["n"], M["n"])) for M in geo.layers]
        phis[li] = a * X + b * Y
        for g, W in enumerate(wl["wfs"]):
            s = 1 - L["h"] / W["H"] if W["lgs"] else 1.0
            N = geo.wfs[g]["N"]
            xa = -geo.D / 2 + np.arange(N + 1) * geo.wfs[g]["d"]
            XA, YA = np.meshgrid(xa, xa)
            expect = a * (s * XA + W["theta"][0] * L["h"]) + b * (s * YA + W["theta"][1] * L["h"])
            np.testing.assert_allclose(O.project(geo, g, phis), expect, atol=1e-12)


def test_ground_layer_projection_is_injection():
    """h = 0 and delta = d: P reads the layer nodes under the aperture unchanged."""
    geo = _geo("tiny_scao")
    rng = np.random.default_rng(3)
    phi0 = rng.standard_normal((32, 32))
    v = O.project(geo, 0, [phi0, np.zeros((16, 16))])
    np.testing.assert_array_equal(v, phi0[8:25, 8:25])


def test_footprint_outside_grid_is_rejected():
    wl = synth.tiny_scao()
    wl["layers"][1]["n"] = 8                   # 8 km layer: 9 nodes needed in an 8-node grid
    with pytest.raises(O.GeometryError):
        O.Geometry(wl)
    wl = synth.tiny_scao()
    wl["layers"][0]["n"] = 24                  # not a power of two
    with pytest.raises(O.GeometryError):
        O.Geometry(wl)


# ---------------------------------------------------------------- tip/tilt
def test_tiptilt_projector_properties():
    k = 7
    T = O.tiptilt_projector(k)
    np.testing.assert_allclose(T @ T, T, atol=1e-15)
    np.testing.assert_allclose(T, T.T, atol=0)
    tx = np.r_[np.ones(k), np.zeros(k)]
    ty = np.r_[np.zeros(k), np.ones(k)]
    np.testing.assert_allclose(T @ tx, tx, atol=1e-15)
    np.testing.assert_allclose(T @ ty, ty, atol=1e-15)
    assert abs(np.trace(T) - 2) < 1e-14


def test_lgs_noise_weight_is_projected_and_blind_to_tilt():
    geo = _geo("tiny_mcao")
    g = 0
    W = geo.wfs[g]
    k = W["n_active"]
    rng = np.random.default_rng(11)
    s = rng.standard_normal(2 * k)
    T = O.tiptilt_projector(k)
    I = np.eye(2 * k)
    Cinv = I / W["sigma"] ** 2
    np.testing.assert_allclose(O.noise_weight(geo, g, s), (I - T) @ Cinv @ (I - T) @ s, atol=1e-10)
    tilt = O.sh_slopes(geo, g, _nodes(W["N"], W["d"], lambda X, Y: 0.4 * X - 0.1 * Y))
    assert np.abs(O.noise_weight(geo, g, tilt)).max() < 1e-10
    ngs = geo.wfs[2]
    s = rng.standard_normal(ngs["ns"])
    np.testing.assert_allclose(O.noise_weight(geo, 2, s), s / ngs["sigma"] ** 2, rtol=1e-15)


# ---------------------------------------------------------------- fitting
def test_fitting_weights():
    w = O.fitting_weights([0.0, 2000.0, 4000.0, 8000.0, 12700.0, 20000.0], [0.0, 4000.0, 12700.0])
    np.testing.assert_allclose(w.sum(1), 1.0)
    np.testing.assert_allclose(w[0], [1, 0, 0])
    np.testing.assert_allclose(w[1], [0.5, 0.5, 0])
    np.testing.assert_allclose(w[2], [0, 1, 0])
    np.testing.assert_allclose(w[3], [0, 4700 / 8700, 4000 / 8700])
    np.testing.assert_allclose(w[4], [0, 0, 1])
    np.testing.assert_allclose(w[5], [0, 0, 1])


def test_fit_of_constant_layers():
    geo = _geo("tiny_mcao")
    consts = [1.0, 2.0, 3.0]
    c = O.W_fwd(geo, [np.full((L["n"], L["n"]), v) for v, L in zip(consts, geo.layers)])
    a = O.fit(geo, c)
    m0, m1 = geo.dms
    np.testing.assert_allclose(a[:81], 1.0 + 0.4 * 2.0, atol=1e-12)
    np.testing.assert_allclose(a[81:], 0.6 * 2.0 + 3.0, atol=1e-12)
    assert math.isclose(m0["w"].sum() + m1["w"].sum(), 3.0)
