"""Pins of the oracle's closed-loop terms (Algorithm 1, reading R27): the DM projection
P_DM, the pseudo-open-loop slopes and the closed-loop control law."""
import numpy as np
import pytest

import oracle as O
import synth


def _affine_dm(m, c0, cx, cy):
    """Actuator values of the affine surface c0 + cx x + cy y on DM m's lattice."""
    na, sp = m["n_act"], m["spacing"]
    xa = (np.arange(na) - (na - 1) / 2.0) * sp
    return c0 + cx * xa[None, :] + cy * xa[:, None]


@pytest.mark.parametrize("name", ["tiny_mcao", "maory"])
def test_dm_projection_of_affine_surfaces(name):
    """A bilinear surface reproduces affine functions exactly: where sensor g's nodes fall
    inside DM m's actuator lattice it sees c0 + cx (s x + tx h) + cy (s y + ty h)."""
    wl = synth.workload_by_name(name)
    geo = O.Geometry(wl)
    rng = np.random.default_rng(7)
    for mi, m in enumerate(geo.dms):
        c0, cx, cy = rng.standard_normal(3)
        a = np.zeros(geo.n_a)
        a[m["off"]:m["off"] + m["n_act"] ** 2] = _affine_dm(m, c0, cx, cy).ravel()
        hm = float(wl["dms"][mi]["h"])
        half = (m["n_act"] - 1) / 2.0 * m["spacing"]
        for g, W in enumerate(wl["wfs"]):
            s = 1.0 - hm / W["H"] if W["lgs"] else 1.0
            tx, ty = W["theta"]
            N = geo.wfs[g]["N"]
            xs = -geo.D / 2 + np.arange(N + 1) * geo.D / N
            px, py = s * xs + tx * hm, s * xs + ty * hm
            inside = (np.abs(py)[:, None] <= half) & (np.abs(px)[None, :] <= half)
            want = c0 + cx * px[None, :] + cy * py[:, None]
            got = O.dm_project(geo, g, a)
            assert inside.sum() > 0
            np.testing.assert_allclose(got[inside], want[inside], rtol=0, atol=1e-12 * (1 + np.abs(want).max()))


def test_ground_dm_on_the_node_lattice_is_an_injection():
    """A ground DM whose actuators coincide with the aperture nodes (8 m SCAO: 17 x 17 at
    0.5 m) hands every actuator value to its node unchanged."""
    wl = synth.tiny_scao()
    geo = O.Geometry(wl)
    a = np.random.default_rng(3).standard_normal(geo.n_a)
    np.testing.assert_array_equal(O.dm_project(geo, 0, a), a.reshape(17, 17))


def test_surface_is_zero_beyond_the_outer_hats():
    """Outside the lattice the surface falls linearly to zero over one spacing: a node
    half a spacing beyond the last actuator sees half its value, one beyond sees none."""
    wl = synth.tiny_scao()
    wl["dms"] = [dict(h=0.0, spacing=0.5, n_act=15)]       # lattice [-3.5, 3.5], nodes [-4, 4]
    geo = O.Geometry(wl)
    a = np.ones(geo.n_a)
    v = O.dm_project(geo, 0, a)
    assert v[8, 8] == 1.0 and v[1, 1] == 1.0               # inside
    assert v[8, 0] == 0.0 and v[0, 8] == 0.0               # x = -4: one spacing beyond
    wl["dms"] = [dict(h=0.0, spacing=0.5, n_act=16)]       # lattice [-3.75, 3.75]
    geo = O.Geometry(wl)
    v = O.dm_project(geo, 0, np.ones(geo.n_a))
    assert v[8, 0] == 0.5 and v[0, 8] == 0.5 and v[0, 0] == 0.25   # half a spacing beyond
    assert v[8, 1] == 1.0 and v[8, 8] == 1.0


def test_dm_slopes_of_a_tilt():
    """A tilt c x on the ground DM gives every active subaperture the x-slope c d and no
    y-slope (8 m SCAO, every node inside the lattice)."""
    wl = synth.tiny_scao()
    geo = O.Geometry(wl)
    a = _affine_dm(geo.dms[0], 0.0, 0.3, 0.0).ravel()
    s = O.dm_slopes(geo, a)
    k = geo.wfs[0]["n_active"]
    np.testing.assert_allclose(s[:k], 0.3 * geo.wfs[0]["d"], rtol=1e-13)
    np.testing.assert_allclose(s[k:], 0.0, atol=1e-13)


@pytest.mark.parametrize("gain", [1.0, 0.5])
@pytest.mark.parametrize("name", ["tiny_scao", "tiny_mcao"])
def test_pseudo_open_loop_frames_follow_the_control_law(name, gain):
    """Residual slopes measured with the DM shape of two frames back (the two-step delay
    of Algorithm 1) become the open-loop slopes again, so the closed-loop commands obey
    a^(k+1) = a^(k) + gain (a~_k - a^(k-1)) with a~_k the open-loop reconstruction."""
    wl = synth.workload_by_name(name)
    wl["params"]["gain"] = gain
    atm = synth.TruthAtmosphere(wl["truth"])
    s_ol = [synth.simulate_slopes(wl, t, atm=atm) for t in range(6)]
    wl_open = synth.workload_by_name(name)
    wl_open["params"]["gain"] = 1.0
    ref = O.Reconstructor(wl_open)
    a_tilde = [ref.frame(s) for s in s_ol]                  # gain 1: a = a~
    cl = O.Reconstructor(wl)
    A = [np.zeros(cl.geo.n_a), np.zeros(cl.geo.n_a)]        # a^(-1), a^(0)
    for k, s in enumerate(s_ol):
        s_cl = s - O.dm_slopes(cl.geo, A[-2])               # the WFS saw a^(k-1)
        A.append(cl.frame(s_cl, closed_loop=True))
        want = A[-2] + gain * (a_tilde[k] - A[-3])
        # the layers' piston is unseen by the slopes (its coefficient is set by the prior
        # alone, ~1e5 times its rounding residue): compare each DM's commands without
        # their mean to 1e-10, the means to 1e-6
        np.testing.assert_allclose(A[-1], want, rtol=0, atol=1e-6 * np.abs(want).max())
        for m in cl.geo.dms:
            sl = slice(m["off"], m["off"] + m["n_act"] ** 2)
            d = A[-1][sl] - want[sl]
            assert np.abs(d - d.mean()).max() <= 1e-10 * np.abs(want).max()
