"""Operator-level parity: every C ABI operator against the FP64 oracle, element by element."""
import numpy as np
import pytest

import oracle as O
import tests.oracle_ops as OO
from tests.gpu_common import TOL_OP, assert_close, geometry, recon, to_dev, to_np

pytestmark = pytest.mark.gpu

CASES = [("tiny_scao", 64), ("tiny_scao", 32), ("tiny_mcao", 64), ("tiny_mcao", 32),
         ("maory", 32), ("maory", 64), ("tiny_mcao_elongated", 64), ("tiny_mcao_elongated", 32),
         ("paper_mcao", 32)]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: "%s-fp%d" % c)
def inst(request):
    name, prec = request.param
    geo, D = geometry(name)
    R = recon(name, prec)
    yield name, prec, geo, D, R
    R.close()


def _rng(seed):
    return np.random.default_rng(seed)


def test_sizes(inst):
    name, prec, geo, D, R = inst
    assert (R.n_coeffs, R.n_slopes, R.n_act, R.n_nodes) == (geo.n_c, geo.n_s, geo.n_a, OO.n_nodes(geo))


def test_wavelets(inst):
    name, prec, geo, D, R = inst
    x = _rng(1).standard_normal(geo.n_c)
    assert_close(to_np(R.dwt(to_dev(x, prec))), OO.dwt(geo, x), TOL_OP[prec], "W")
    assert_close(to_np(R.idwt(to_dev(x, prec))), OO.idwt(geo, x), TOL_OP[prec], "W^T")


def test_projection_and_adjoint(inst):
    name, prec, geo, D, R = inst
    x = _rng(2).standard_normal(geo.n_c)
    assert_close(to_np(R.project(to_dev(x, prec))), OO.project(geo, x), TOL_OP[prec], "P")
    v = _rng(3).standard_normal(R.n_nodes)
    assert_close(to_np(R.project_adj(to_dev(v, prec))), OO.project_adj(geo, v), TOL_OP[prec], "P^T")


def test_shack_hartmann_and_noise(inst):
    name, prec, geo, D, R = inst
    v = _rng(4).standard_normal(R.n_nodes)
    assert_close(to_np(R.slopes(to_dev(v, prec))), OO.slopes(geo, v), TOL_OP[prec], "Gamma")
    s = _rng(5).standard_normal(geo.n_s)
    assert_close(to_np(R.slopes_adj(to_dev(s, prec))), OO.slopes_adj(geo, s), TOL_OP[prec], "Gamma^T")
    assert_close(to_np(R.noise_weight(to_dev(s, prec))), OO.noise_weight(geo, s), TOL_OP[prec], "C^-1")


def test_forward_model_and_adjoint(inst):
    name, prec, geo, D, R = inst
    x = _rng(6).standard_normal(geo.n_c)
    assert_close(to_np(R.forward(to_dev(x, prec))), OO.forward(geo, x), TOL_OP[prec], "A")
    s = _rng(7).standard_normal(geo.n_s)
    assert_close(to_np(R.forward_adj(to_dev(s, prec))), OO.forward_adj(geo, s), TOL_OP[prec], "A^T")


def test_diagonals(inst):
    name, prec, geo, D, R = inst
    Dg, Jg = R.diagonals()
    assert_close(to_np(Dg), D, TOL_OP[prec], "D")
    J = O.precond_diag(geo, D)
    # J is built in double on the device for both forms
    assert_close(to_np(Jg), J, 1e-12 if prec == 64 else 1e-7, "J")


def test_operator_M_and_rhs(inst):
    name, prec, geo, D, R = inst
    c = _rng(8).standard_normal(geo.n_c)
    assert_close(to_np(R.apply_M(to_dev(c, prec))), O.apply_M(geo, c, D), TOL_OP[prec], "M")
    s = _rng(9).standard_normal(geo.n_s)
    assert_close(to_np(R.rhs(to_dev(s, prec))), O.rhs(geo, s), TOL_OP[prec], "b")


def test_fit_and_adjoint(inst):
    name, prec, geo, D, R = inst
    c = _rng(10).standard_normal(geo.n_c)
    assert_close(to_np(R.fit(to_dev(c, prec))), O.fit(geo, c), TOL_OP[prec], "F W^T")
    a = _rng(11).standard_normal(geo.n_a)
    assert_close(to_np(R.fit_adj(to_dev(a, prec))), O.fit_adj(geo, a), TOL_OP[prec], "(F W^T)^T")


def test_pcg_iterations(inst):
    name, prec, geo, D, R = inst
    import synth
    s = synth.simulate_slopes(synth.workload_by_name(name), 0)
    b = O.rhs(geo, s)
    Jinv = 1.0 / O.precond_diag(geo, D)
    c0 = _rng(12).standard_normal(geo.n_c)
    for k in (1, 4):
        ref, _ = O.pcg(geo, b, c0, Jinv, k, D)
        c = to_dev(c0, prec)
        R.pcg(to_dev(b, prec), c, k)
        err = np.linalg.norm(to_np(c) - ref) / np.linalg.norm(ref)
        assert err < (1e-9 if prec == 64 else 1e-4), (k, err)
