"""Differentiable reconstruction on the GPU: the converged map and its gradients (adjoint
PCG and adjoint operator kernels) against the FP64 gradient oracle, against central
finite differences of the GPU's own converged map, and through torch.autograd."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from oracle import fewha_grad as G
from tests.gpu_common import rel_l2, to_dev, to_np
from tests.test_oracle_grad import setup

pytestmark = pytest.mark.gpu

# The converged solve is PCG with the Jacobi preconditioner on M, whose preconditioned
# condition number is ~6e6 on these geometries: FP64 reaches a relative residual of 1e-11
# in ~8000 iterations, and the results then agree with the oracle's Cholesky solve as
# below.  The alpha gradient is -lambda^T D c, a sum with cancellation, so it is the least
# accurate.  The FP32 form iterates in float but refreshes its recurrence with the TRUE
# residual b - M x formed in double (reliable updates; x accumulated in double), and stops
# on that residual at the same 1e-11: its c* and lambda carry the FP64 form's error bound,
# and only the float outputs add a rounding of 6e-8 relative to the commands and the
# slope gradients.  So the FP32 bounds are the FP64 ones, with 1e-6 for the float outputs.
SOLVE_TOL = {64: 1e-11, 32: 1e-11}
TOL = {64: dict(dm=1e-7, gs=1e-8, ga=1e-4, gw=1e-6), 32: dict(dm=1e-6, gs=1e-6, ga=1e-4, gw=1e-6)}
MAX_IT = 20000


def demean(x):
    x = np.asarray(x, float)
    return x - x.mean()


def recon(wl, prec):
    from paper_2202_11945_gb300 import Reconstructor
    return Reconstructor(wl, precision=prec, graph=False)


def gpu_grads(R, s, target, prec, tol=None):
    dm, it, rel = R.reconstruct_converged(to_dev(s, prec), tol=SOLVE_TOL[prec] if tol is None else tol,
                                          max_iters=MAX_IT)
    a = to_np(dm)
    J, g_a = G.dm_error_objective(a, target)
    gs, ga, gw = R.backward(to_dev(g_a, prec))
    return a, J, to_np(gs), ga, np.array(gw), g_a, it, rel


@pytest.mark.parametrize("name", ["tiny_scao", "tiny_mcao"])
@pytest.mark.parametrize("prec", [64, 32])
def test_converged_map_and_gradients_match_oracle(name, prec):
    wl, geo, Bd, s, target, w = setup(name)
    R = recon(wl, prec)
    a, J, gs, ga, gw, g_a, it, rel = gpu_grads(R, s, target, prec)
    assert rel <= SOLVE_TOL[prec], (it, rel)
    _, a_ref = G.converged_map(geo, Bd, s, geo.alpha, w)
    # piston is unseen by the slopes: compare the commands without their mean
    assert rel_l2(demean(a), demean(a_ref)) <= TOL[prec]["dm"], rel_l2(demean(a), demean(a_ref))
    # gradients of the same objective, oracle evaluated with the GPU's own dJ/da~
    gs_ref, ga_ref, gw_ref = G.map_gradients(geo, Bd, s, geo.alpha, w, g_a)
    check_grads(prec, gs, ga, gw, gs_ref, ga_ref, gw_ref)
    R.close()


def check_grads(prec, gs, ga, gw, gs_ref, ga_ref, gw_ref, what=""):
    t = TOL[prec]
    assert rel_l2(gs, gs_ref) <= t["gs"], (what, rel_l2(gs, gs_ref))
    assert abs(ga - ga_ref) <= t["ga"] * abs(ga_ref), (what, ga, ga_ref)
    assert rel_l2(gw, gw_ref) <= t["gw"], (what, gw, gw_ref)


def test_central_differences_of_the_gpu_map():
    """FP64: the backward's alpha and weight gradients against central differences with a
    step of 1e-3 relative of the GPU's own converged map (solved to 1e-12)."""
    wl, geo, Bd, s, target, w = setup("tiny_mcao")
    R = recon(wl, 64)
    sd = to_dev(s, 64)

    def J(alpha, ww):
        R.update_params(alpha=alpha, cn2_weights=list(ww))
        dm, _, rel = R.reconstruct_converged(sd, tol=1e-12, max_iters=MAX_IT)
        return G.dm_error_objective(to_np(dm), target)[0]

    alpha = 2.5
    R.update_params(alpha=alpha, cn2_weights=list(w))
    _, _, gs, ga, gw, _, _, _ = gpu_grads(R, s, target, 64)
    h = 1e-3 * alpha
    fd = (J(alpha + h, w) - J(alpha - h, w)) / (2 * h)
    assert abs(fd - ga) <= 1e-4 * abs(ga), (fd, ga)
    for l in range(len(w)):
        h = 1e-3 * w[l]
        wp, wm = w.copy(), w.copy()
        wp[l] += h
        wm[l] -= h
        fd = (J(alpha, wp) - J(alpha, wm)) / (2 * h)
        assert abs(fd - gw[l]) <= 1e-4 * np.abs(gw).max(), (l, fd, gw[l])
    R.close()


def test_autograd_function_matches_oracle():
    from paper_2202_11945_gb300 import autograd as AG
    wl, geo, Bd, s, target, w = setup("tiny_mcao")
    R = recon(wl, 64)
    sl = torch.tensor(s, dtype=torch.float64, device="cuda", requires_grad=True)
    alpha = torch.tensor(1.7, dtype=torch.float64, requires_grad=True)
    cn2 = torch.tensor(w, dtype=torch.float64, requires_grad=True)
    a = AG.reconstruct(R, sl, alpha, cn2, tol=1e-11, max_iters=MAX_IT)
    t = torch.tensor(target, dtype=torch.float64, device="cuda")
    d = a - t
    J = ((d - d.mean()) ** 2).sum()
    J.backward()
    _, a_ref = G.converged_map(geo, Bd, s, 1.7, w)
    J_ref, _ = G.dm_error_objective(a_ref, target)
    assert abs(float(J.detach()) - J_ref) <= 1e-7 * J_ref
    # the oracle's gradients for the GPU's own dJ/da~ (isolates the backward)
    _, g_a = G.dm_error_objective(to_np(a.detach()), target)
    gs_ref, ga_ref, gw_ref = G.map_gradients(geo, Bd, s, 1.7, w, g_a)
    check_grads(64, to_np(sl.grad), float(alpha.grad), cn2.grad.numpy(), gs_ref, ga_ref, gw_ref)
    R.close()


def test_forward_model_function_is_adjoint():
    from paper_2202_11945_gb300 import autograd as AG
    wl = synth.tiny_mcao()
    R = recon(wl, 64)
    rng = np.random.Generator(np.random.PCG64(5))
    phi = torch.tensor(rng.standard_normal(R.n_coeffs), device="cuda", requires_grad=True)
    g = torch.tensor(rng.standard_normal(R.n_slopes), device="cuda")
    s = AG.forward_model(R, phi)
    (s * g).sum().backward()
    lhs = float((s * g).sum().detach())
    rhs = float((phi.detach() * phi.grad).sum())
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1.0)
    geo = O.Geometry(wl)
    s_ref = O.forward_model(geo, geo.split(phi.detach().cpu().numpy()))
    assert rel_l2(to_np(s), s_ref) <= 1e-12
    R.close()


def test_differentiable_workload_32_frames():
    """The 8 m geometry, 32 seeded frames of frozen flow: FP64 and FP32 gradients against
    the FP64 oracle (each frame's solves warm-started from the previous frame's).  The solves
    go to 1e-12: the alpha gradient -lambda^T D c cancels to ~1e-4 of its terms on some
    frames, so a 1e-11 residual leaves it near the 1e-4 bound."""
    wl = synth.differentiable()
    geo = O.Geometry(wl)
    Bd = G.data_matrix(geo)
    atm = synth.TruthAtmosphere(wl["truth"])
    x, y = G.actuator_positions(geo)
    w = np.array([L["w"] for L in wl["layers"]])
    R32, R64 = recon(wl, 32), recon(wl, 64)
    for t in range(32):
        s = synth.simulate_slopes(wl, t, atm=atm)
        target = synth.true_phase_at(wl, x, y, t, atm=atm)
        for prec, R in ((64, R64), (32, R32)):
            a, J, gs, ga, gw, g_a, it, rel = gpu_grads(R, s, target, prec, tol=1e-12)
            gs_ref, ga_ref, gw_ref = G.map_gradients(geo, Bd, s, geo.alpha, w, g_a)
            check_grads(prec, gs, ga, gw, gs_ref, ga_ref, gw_ref, (t, prec))
    R32.close()
    R64.close()


def test_maory_geometry_nine_weight_gradients():
    """The MAORY geometry (9 layers; ~4e4 iterations per cold FP64 solve): the alpha and
    ground-layer weight gradients against central differences (one Richardson step,
    step 1e-2 relative) of the GPU's converged map, solves warm-started."""
    wl = synth.maory()
    R = recon(wl, 64)
    atm = synth.TruthAtmosphere(wl["truth"])
    s = synth.simulate_slopes(wl, 0, atm=atm)
    geo = O.Geometry(wl)
    x, y = G.actuator_positions(geo)
    target = synth.true_phase_at(wl, x, y, 0, atm=atm)
    w = np.array([L["w"] for L in wl["layers"]])
    sd = to_dev(s, 64)
    dm, it, rel = R.reconstruct_converged(sd, tol=1e-10, max_iters=60000)
    assert rel <= 1e-10, (it, rel)
    J0, g_a = G.dm_error_objective(to_np(dm), target)
    _, ga, gw = R.backward(to_dev(g_a, 64))
    assert len(gw) == 9 and np.all(np.isfinite(gw))

    def J(alpha, ww):
        R.update_params(alpha=alpha, cn2_weights=list(ww))
        d, _, r = R.reconstruct_converged(sd, tol=1e-10, max_iters=60000)
        return G.dm_error_objective(to_np(d), target)[0]

    def rich(f, x0, h):
        d1 = (f(x0 + h) - f(x0 - h)) / (2 * h)
        d2 = (f(x0 + h / 2) - f(x0 - h / 2)) / h
        return (4 * d2 - d1) / 3

    fd = rich(lambda v: J(v, w), geo.alpha, 1e-2 * geo.alpha)
    assert abs(fd - ga) <= 1e-3 * abs(ga), (fd, ga)

    def f0(v):
        ww = w.copy()
        ww[0] = v
        return J(geo.alpha, ww)
    fd = rich(f0, w[0], 1e-2 * w[0])
    assert abs(fd - gw[0]) <= 1e-3 * np.abs(gw).max(), (fd, gw[0])
    R.close()


def test_maory_geometry_fp32_gradients_match_fp64():
    """The MAORY geometry, FP32 form: the converged commands and the slope, alpha and nine
    Cn2-weight gradients against the FP64 form's (which the test above checks against
    central differences), both solved to 1e-10."""
    wl = synth.maory()
    atm = synth.TruthAtmosphere(wl["truth"])
    s = synth.simulate_slopes(wl, 0, atm=atm)
    geo = O.Geometry(wl)
    x, y = G.actuator_positions(geo)
    target = synth.true_phase_at(wl, x, y, 0, atm=atm)
    out = {}
    for prec in (32, 64):
        R = recon(wl, prec)
        dm, it, rel = R.reconstruct_converged(to_dev(s, prec), tol=1e-10, max_iters=120000)
        assert rel <= 1e-10, (prec, it, rel)
        a = to_np(dm)
        if prec == 32:
            _, g_a = G.dm_error_objective(a, target)       # the same dJ/da~ for both forms
        gs, ga, gw = R.backward(to_dev(g_a, prec))
        out[prec] = (a, to_np(gs), ga, np.array(gw))
        R.close()
    a32, gs32, ga32, gw32 = out[32]
    a64, gs64, ga64, gw64 = out[64]
    assert rel_l2(demean(a32), demean(a64)) <= 1e-5, rel_l2(demean(a32), demean(a64))
    assert rel_l2(gs32, gs64) <= 1e-5, rel_l2(gs32, gs64)
    assert abs(ga32 - ga64) <= 1e-3 * abs(ga64), (ga32, ga64)
    assert rel_l2(gw32, gw64) <= 1e-4, (gw32, gw64)
