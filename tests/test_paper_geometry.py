"""The paper-geometry workload against the values printed in the paper's tables
(tests/golden/paper_geometry.txt, Sec. 4.1 Tables 1-5), reading R29 for what they leave
open (obstruction as an area fraction, star azimuths)."""
import math
import os

import numpy as np

import oracle as O
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_geometry.txt")


def _golden():
    out = {"layer": [], "dm": []}
    for line in open(GOLDEN):
        if not line.strip() or line.startswith("#"):
            continue
        k, *v = line.split()
        if k in ("layer", "dm"):
            out[k].append([float(x) for x in v])
        else:
            out[k] = [float(x) for x in v]
    return out


def test_workload_matches_the_printed_tables():
    g, wl = _golden(), synth.paper_mcao()
    assert wl["D"] == g["D"][0]
    assert math.isclose(wl["obs"] ** 2, g["obstruction_percent"][0] / 100.0)   # area fraction
    assert wl["truth"]["L0"] == g["L0"][0] and wl["params"]["L0"] == g["L0"][0]
    assert wl["params"]["alpha_eta"] == g["alpha_eta"][0]
    assert [(L["h"], L["w"], L["levels"], L["n"], L["delta"]) for L in wl["layers"]] == \
        [tuple([h, w, int(J), int(n), d]) for h, w, J, n, d in g["layer"]]
    assert [(m["n_act"], m["h"], m["spacing"]) for m in wl["dms"]] == \
        [(int(n), h, sp) for n, h, sp in g["dm"]]
    lgs = [W for W in wl["wfs"] if W["lgs"]]
    ngs = [W for W in wl["wfs"] if not W["lgs"]]
    count, nsub, diam = g["lgs"]
    assert len(lgs) == count and all(W["n_sub"] == nsub for W in lgs)
    for W in lgs:
        assert math.isclose(math.hypot(*W["theta"]), synth.arcsec(diam / 2), rel_tol=1e-12)
        assert W["H"] == g["na_height"][0] and W["na_fwhm"] == g["na_fwhm"][0]
    count, nsub, diam = g["ngs"]
    assert len(ngs) == count and all(W["n_sub"] == nsub for W in ngs)
    for W in ngs:
        assert math.isclose(math.hypot(*W["theta"]), synth.arcsec(diam / 2), rel_tol=1e-12)


def test_layers_at_the_dm_altitudes_make_the_fit_the_identity():
    """Sec. 4.1: with the 3 layers at the DM altitudes the fitting operator F is the
    identity on the actuators: a layer holding values v at the actuator nodes fits to v."""
    geo = O.Geometry(synth.paper_mcao())
    rng = np.random.default_rng(3)
    phis = []
    expect = []
    for L, m in zip(geo.layers, geo.dms):
        phi = rng.standard_normal((L["n"], L["n"]))
        phis.append(phi)
        na = m["n_act"]
        k0 = int(round(-(na - 1) / 2.0 * m["spacing"] / L["delta"] + L["n"] / 2))
        expect.append(phi[k0:k0 + na, k0:k0 + na].ravel())
    a = O.fit(geo, O.W_fwd(geo, phis))
    np.testing.assert_allclose(a, np.concatenate(expect), rtol=0, atol=1e-12)
