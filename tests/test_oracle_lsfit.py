"""Pins of the oracle's least-squares DM fitting over fitting directions (reading R30)."""
import numpy as np
import pytest

import oracle as O
import synth

ARC = synth.arcsec(1.0)
DIRS = [(0.0, 0.0), (15 * ARC, 0.0), (-15 * ARC, 0.0), (0.0, 15 * ARC), (0.0, -15 * ARC)]


def _dense(geo, fg, k, n_fit):
    """A_k and L_k as dense matrices from unit vectors (pupil nodes x commands / layers)."""
    A = np.stack([O.dm_along(geo, fg, k, e).ravel() for e in np.eye(geo.n_a)], 1)
    cols = []
    for l, L in enumerate(geo.layers):
        for e in np.eye(L["n"] ** 2):
            phis = [np.zeros((Lq["n"], Lq["n"])) for Lq in geo.layers]
            phis[l] = e.reshape(L["n"], L["n"])
            cols.append(sum(Ly @ ph @ Lx.T for (Ly, Lx), ph in zip(fg["dirs"][k]["L"], phis)).ravel())
    return A, np.stack(cols, 1)


def test_ls_fit_equals_dense_least_squares():
    """CG on the normal equations against numpy's least squares on the stacked, weighted,
    piston-free system [sqrt(w_k) Pi A_k; sqrt(eps) I] a = [sqrt(w_k) Pi L_k phi; 0]."""
    wl = synth.tiny_mcao()
    geo = O.Geometry(wl)
    n_fit, eps = 8, 1e-3
    w = [1.0, 0.5, 0.5, 0.5, 0.5]
    fg = O.fitting_geometry(geo, DIRS, n_fit)
    rng = np.random.default_rng(8)
    phis = [rng.standard_normal((L["n"], L["n"])) for L in geo.layers]
    a = O.ls_fit(geo, phis, fg, w, eps)
    m = fg["mask"].ravel()
    rows, rhs = [], []
    phi_vec = np.concatenate([p.ravel() for p in phis])
    for k in range(len(DIRS)):
        A, L = _dense(geo, fg, k, n_fit)
        S = np.eye(m.size)[m]                               # selects the pupil nodes
        Pi = S - S.mean(axis=0, keepdims=True)             # ... without their mean
        rows.append(np.sqrt(w[k]) * Pi @ A)
        rhs.append(np.sqrt(w[k]) * Pi @ L @ phi_vec)
    rows.append(np.sqrt(eps) * np.eye(geo.n_a))
    rhs.append(np.zeros(geo.n_a))
    ref = np.linalg.lstsq(np.vstack(rows), np.concatenate(rhs), rcond=None)[0]
    np.testing.assert_allclose(a, ref, rtol=0, atol=1e-8 * np.abs(ref).max())


def test_representable_layers_are_fitted_exactly():
    """Layers at the DM altitudes on the DMs' own lattices (the paper's 3-layer case, where F
    is the identity): layers made of DM shapes leave no residual in any direction."""
    wl = synth.tiny_scao()
    wl["layers"] = [dict(h=0.0, w=1.0, delta=0.5, n=32, levels=3)]
    geo = O.Geometry(wl)
    n_fit = 16                                              # pupil nodes on the actuator lattice
    fg = O.fitting_geometry(geo, [(0.0, 0.0)], n_fit)
    rng = np.random.default_rng(9)
    a_true = rng.standard_normal(geo.n_a)
    # the layer holding the ground DM's bilinear surface: actuator k at layer node k + 8
    phi = np.zeros((32, 32))
    phi[8:25, 8:25] = a_true.reshape(17, 17)
    a = O.ls_fit(geo, [phi], fg, [1.0], 1e-10)
    res = O.pupil_centre(fg, O.dm_along(geo, fg, 0, a) - fg["dirs"][0]["L"][0][0] @ phi @ fg["dirs"][0]["L"][0][1].T)
    assert np.abs(res).max() <= 1e-8 * np.abs(a_true).max()


def test_fitting_directions_see_shifted_affine_surfaces():
    """Along direction theta the pupil node x sees a DM and a layer at x + theta h: affine
    surfaces come out exactly (where the stencils stay inside the lattices)."""
    wl = synth.tiny_mcao()
    geo = O.Geometry(wl)
    n_fit = 8
    th = (12 * ARC, -7 * ARC)
    fg = O.fitting_geometry(geo, [th], n_fit)
    xs = -geo.D / 2 + np.arange(n_fit + 1) * geo.D / n_fit
    c0, cx, cy = 0.3, -1.1, 0.7
    for mi, m in enumerate(geo.dms):
        na, sp = m["n_act"], m["spacing"]
        xa = (np.arange(na) - (na - 1) / 2.0) * sp
        a = np.zeros(geo.n_a)
        a[m["off"]:m["off"] + na * na] = (c0 + cx * xa[None, :] + cy * xa[:, None]).ravel()
        px, py = xs + th[0] * m["h"], xs + th[1] * m["h"]
        half = (na - 1) / 2.0 * sp
        inside = (np.abs(py)[:, None] <= half) & (np.abs(px)[None, :] <= half)
        want = c0 + cx * px[None, :] + cy * py[:, None]
        got = O.dm_along(geo, fg, 0, a)
        np.testing.assert_allclose(got[inside], want[inside], atol=1e-12)
    for l, L in enumerate(geo.layers):
        xl = (np.arange(L["n"]) - L["n"] / 2) * L["delta"]
        phis = [np.zeros((Lq["n"], Lq["n"])) for Lq in geo.layers]
        phis[l] = c0 + cx * xl[None, :] + cy * xl[:, None]
        Ly, Lx = fg["dirs"][0]["L"][l]
        px, py = xs + th[0] * L["h"], xs + th[1] * L["h"]
        want = c0 + cx * px[None, :] + cy * py[:, None]
        np.testing.assert_allclose(Ly @ phis[l] @ Lx.T, want, atol=1e-12)
