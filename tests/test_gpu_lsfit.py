"""Least-squares DM fitting over fitting directions on the GPU (fewha_fit_ls, Sec. 4.1)
against the oracle's CG on the same normal equations (oracle.ls_fit, itself pinned by
dense least squares, exact fits of representable layers and shifted affine surfaces).

Both sides solve a positive definite system (eps > 0) to a small relative residual, so
they agree up to that residual times the condition number: the double form is run to
1e-12 and compared at 1e-9 relative L2; the single form iterates in float (inner products
and CG scalars in double) to 1e-7, and its commands are compared at the FP32 frame bound
of 1e-4 relative L2."""
import numpy as np
import pytest

import oracle as O
import synth
from tests.gpu_common import TOL_FRAME, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

ARC = synth.arcsec(1.0)
DIRS5 = [(0.0, 0.0), (15 * ARC, 0.0), (-15 * ARC, 0.0), (0.0, 15 * ARC), (0.0, -15 * ARC)]
GRID9 = [(x * ARC, y * ARC) for y in (-20, 0, 20) for x in (-20, 0, 20)]
# name: directions, weights, n_fit, eps
CASES = {
    "tiny_scao": ([(0.0, 0.0), (5 * ARC, -3 * ARC)], [1.0, 2.0], 16, 1e-4),
    "tiny_mcao": (DIRS5, [1.0, 0.5, 0.5, 0.5, 0.5], 8, 1e-2),
    "maory": (GRID9, [1.0] * 9, 80, 1e-2),
    "paper_mcao": ([(x * ARC, y * ARC) for y in (-25, 0, 25) for x in (-25, 0, 25)], [1.0] * 9, 74, 1e-2),
}
SOLVE_TOL = {64: 1e-12, 32: 1e-7}
TOL = {64: 1e-9, 32: TOL_FRAME[32]}


def recon(wl, prec):
    from paper_2202_11945_gb300 import Reconstructor
    return Reconstructor(wl, precision=prec, graph=False)


def oracle_fit(geo, c, case):
    dirs, w, n_fit, eps = case
    return O.ls_fit(geo, O.W_inv(geo, c), O.fitting_geometry(geo, dirs, n_fit), w, eps)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", [64, 32])
def test_ls_fit_matches_oracle(name, prec):
    wl = synth.workload_by_name(name)
    geo = O.Geometry(wl)
    c = np.random.default_rng(11).standard_normal(geo.n_c)
    ref = oracle_fit(geo, c, CASES[name])
    R = recon(wl, prec)
    dirs, w, n_fit, eps = CASES[name]
    a, it, rel = R.fit_ls(to_dev(c, prec), dirs, w, n_fit, eps, tol=SOLVE_TOL[prec])
    assert 0 < it < 5000 and rel <= SOLVE_TOL[prec], (it, rel)
    assert rel_l2(to_np(a), ref) <= TOL[prec], rel_l2(to_np(a), ref)
    R.close()


@pytest.mark.parametrize("prec", [64, 32])
def test_configuration_changes_and_repeated_calls(prec):
    """Tables are rebuilt when the directions change (here to a larger set) and reused when
    they do not: a repeated call gives the same commands bit for bit."""
    wl = synth.tiny_mcao()
    geo = O.Geometry(wl)
    c = np.random.default_rng(12).standard_normal(geo.n_c)
    R = recon(wl, prec)
    small = ([(0.0, 0.0)], [1.0], 6, 1e-2)
    for case in (small, CASES["tiny_mcao"], small):
        a1, it1, _ = R.fit_ls(to_dev(c, prec), *case, tol=SOLVE_TOL[prec])
        a1 = to_np(a1)
        a2, it2, _ = R.fit_ls(to_dev(c, prec), *case, tol=SOLVE_TOL[prec])
        assert it1 == it2 and np.array_equal(a1, to_np(a2))
        assert rel_l2(a1, oracle_fit(geo, c, case)) <= TOL[prec]
    R.close()


def test_iteration_limit_and_zero_layers():
    wl = synth.tiny_mcao()
    geo = O.Geometry(wl)
    R = recon(wl, 64)
    dirs, w, n_fit, eps = CASES["tiny_mcao"]
    c = np.random.default_rng(13).standard_normal(geo.n_c)
    a, it, rel = R.fit_ls(to_dev(c, 64), dirs, w, n_fit, eps, max_iters=3)
    assert it == 3 and np.isfinite(rel) and rel > SOLVE_TOL[64]
    a, it, rel = R.fit_ls(to_dev(c, 64), dirs, w, n_fit, eps, max_iters=0)
    assert it == 0 and not to_np(a).any()
    a, it, rel = R.fit_ls(to_dev(np.zeros(geo.n_c), 64), dirs, w, n_fit, eps)
    assert it == 0 and rel == 0.0 and not to_np(a).any()
    R.close()


def test_bad_configurations_are_rejected():
    from paper_2202_11945_gb300.fewha import FewhaError
    wl = synth.tiny_mcao()
    geo = O.Geometry(wl)
    R = recon(wl, 32)
    c = to_dev(np.ones(geo.n_c), 32)
    bad = [
        (([(0.0, 0.0)], [0.0], 8, 1e-3), -1),              # no positive weight
        (([(0.0, 0.0)], [-1.0], 8, 1e-3), -1),             # negative weight
        (([(0.0, 0.0)], [1.0], 0, 1e-3), -1),              # n_fit out of range
        (([(0.0, 0.0)], [1.0], 257, 1e-3), -1),
        (([(0.0, 0.0)], [1.0], 8, -1.0), -1),              # negative eps
        (([(0.0, 0.0)] * 33, [1.0] * 33, 8, 1e-3), -1),    # too many directions
        (([(300 * ARC, 0.0)], [1.0], 8, 1e-3), -2),        # leaves the 8 km layer's grid
    ]
    for case, code in bad:
        with pytest.raises(FewhaError) as e:
            R.fit_ls(c, *case)
        assert e.value.code == code, (case, e.value.code)
    # the handle still works after the rejections
    a, it, rel = R.fit_ls(c, *CASES["tiny_mcao"])
    assert rel <= SOLVE_TOL[32]
    R.close()
