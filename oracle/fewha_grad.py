"""FP64 oracle of the differentiable reconstruction (a build addition; the paper has no
gradients).

TEST INFRASTRUCTURE ONLY, like the rest of this package.

The differentiable map is the CONVERGED reconstruction: c* solves M c = b exactly
(Eq. 6 with M = W B W^T + alpha D), so c* is the MAP estimate of the discretised model
(Sec. 3.1), and the fitted DM shape is a~ = F W^T c* (Algorithm 1, fitting step).  Here
the solve is a dense Cholesky factorisation of the assembled M (small geometries only).

The objective of the gradient checks is J = ||Pi (a~ - phi_true)||^2 over the actuators,
Pi removing the mean (piston).

Gradients of a scalar J(a~) with g_a = dJ/da~ (implicit differentiation of M c* = b):
  lambda   = M^-1 (F W^T)^T g_a          (M is symmetric)
  dJ/ds    = C_hat^-1 Gamma P W^T lambda  (b = W P^T Gamma^T C_hat^-1 s is linear in s)
  dJ/dalpha = -lambda^T D c*              (dM/dalpha = D)
  dJ/dw_l  = +alpha lambda_l^T (D_l / w_l) c*_l   (D_l is proportional to 1 / w_l, Sec. 3.1
                                                   prior with layer Cn2 weight w_l)

The fixed-iteration frame map (the map the real-time loop runs) is differentiated too, by
reverse mode through its recurrence: see unrolled_frame / unrolled_frame_vjp.
"""

import numpy as np

from .fewha_oracle import (W_fwd, W_inv, apply_M, data_operator, fit, fit_adj, noise_weight,
                           precond_diag, prior_diag, project, rhs, sh_slopes)


def data_matrix(geo):
    """W B W^T assembled column by column from unit vectors (dense)."""
    n = geo.n_c
    Bd = np.zeros((n, n))
    e = np.zeros(n)
    for i in range(n):
        e[i] = 1.0
        Bd[:, i] = W_fwd(geo, data_operator(geo, W_inv(geo, e)))
        e[i] = 0.0
    return 0.5 * (Bd + Bd.T)        # symmetric by construction; removes rounding asymmetry


def _system(geo, Bd, alpha, weights):
    D = prior_diag(geo, weights=weights)
    return Bd + alpha * np.diag(D), D


def _chol_solve(M, b):
    L = np.linalg.cholesky(M)
    return np.linalg.solve(L.T, np.linalg.solve(L, b))


def converged_map(geo, Bd, s, alpha, weights):
    """(c*, a~): the exact solution of M c = b and its fitted DM shape."""
    M, _ = _system(geo, Bd, alpha, weights)
    c = _chol_solve(M, rhs(geo, s))
    return c, fit(geo, c)


def slope_adjoint(geo, lam):
    """C_hat^-1 Gamma P W^T lambda, concatenated over the sensors."""
    phis = W_inv(geo, lam)
    return np.concatenate([noise_weight(geo, g, sh_slopes(geo, g, project(geo, g, phis)))
                           for g in range(len(geo.wfs))])


def map_gradients(geo, Bd, s, alpha, weights, g_a):
    """dJ/ds, dJ/dalpha and dJ/dw of J with dJ/da~ = g_a at the converged map."""
    M, D = _system(geo, Bd, alpha, weights)
    c = _chol_solve(M, rhs(geo, s))
    lam = _chol_solve(M, fit_adj(geo, g_a))
    g_s = slope_adjoint(geo, lam)
    g_alpha = -float(lam @ (D * c))
    g_w = np.array([alpha * float(lam[L["off"]:L["off"] + L["n"] ** 2] @
                                  (D * c)[L["off"]:L["off"] + L["n"] ** 2]) / w
                    for L, w in zip(geo.layers, weights)])
    return g_s, g_alpha, g_w


def dm_error_objective(a, target):
    """J = ||Pi (a~ - target)||^2 and its gradient 2 Pi (a~ - target), where Pi removes
    the mean over the actuators (piston: unseen by slopes and set to zero by the
    reconstruction, so it is left out of the error)."""
    d = np.asarray(a, float) - np.asarray(target, float)
    d = d - d.mean()
    return float(d @ d), 2.0 * d


def actuator_positions(geo):
    """(x, y) of every actuator, concatenated over the DMs (row-major per DM)."""
    xs, ys = [], []
    for m in geo.dms:
        k = (np.arange(m["n_act"]) - (m["n_act"] - 1) / 2.0) * m["spacing"]
        X, Y = np.meshgrid(k, k)
        xs.append(X.ravel())
        ys.append(Y.ravel())
    return np.concatenate(xs), np.concatenate(ys)


# ----------------------------------------------------------------------------
# Reverse mode through the fixed-iteration frame (build addition)
# ----------------------------------------------------------------------------


def unrolled_frame(geo, s, c0, iters, D=None):
    """The frame map of Algorithm 1 with the explicit initial residual r0 = b - M c0,
    `iters` PCG iterations (Sec. 3.3, R12) and the fit: returns (a~, c_k, tape), the
    tape holding every vector and scalar of the recurrence."""
    D = prior_diag(geo) if D is None else D
    Jinv = 1.0 / precond_diag(geo, D)
    b = rhs(geo, s)
    c = np.array(c0, float, copy=True)
    r = b - apply_M(geo, c, D)
    z = Jinv * r
    p = z.copy()
    rho = float(r @ z)
    t = dict(p=[], q=[], r=[r], z=[z], rho=[rho], sigma=[], alpha=[], beta=[], Jinv=Jinv, D=D)
    for _ in range(iters):
        q = apply_M(geo, p, D)
        sigma = float(p @ q)
        a = rho / sigma
        t["p"].append(p)
        t["q"].append(q)
        t["sigma"].append(sigma)
        t["alpha"].append(a)
        c = c + a * p
        r = r - a * q
        z = Jinv * r
        rho_new = float(r @ z)
        beta = rho_new / rho
        t["r"].append(r)
        t["z"].append(z)
        t["rho"].append(rho_new)
        t["beta"].append(beta)
        p = z + beta * p
        rho = rho_new
    return fit(geo, c), c, t


def unrolled_frame_vjp(geo, tape, g_a):
    """dJ/ds of J(a~(s)) through the fixed-iteration frame, g_a = dJ/da~.

    The recurrence of iteration i, statement by statement,
        q_i = M p_i,  sigma_i = p_i.q_i,  alpha_i = rho_i / sigma_i,
        c_(i+1) = c_i + alpha_i p_i,  r_(i+1) = r_i - alpha_i q_i,  z_(i+1) = J^-1 r_(i+1),
        rho_(i+1) = r_(i+1).z_(i+1),  beta_i = rho_(i+1) / rho_i,  p_(i+1) = z_(i+1) + beta_i p_i,
    is run backwards with the adjoint of each statement (M and J^-1 are symmetric); then
    p_0 = z_0, rho_0 = r_0.z_0, z_0 = J^-1 r_0, r_0 = b - M c0 give b_bar = r_bar_0, and
    dJ/ds = C_hat^-1 Gamma P W^T b_bar (b is linear in s)."""
    Jinv, D = tape["Jinv"], tape["D"]
    n = geo.n_c
    cbar = fit_adj(geo, g_a)
    rbar, zbar, pbar, rhobar = np.zeros(n), np.zeros(n), np.zeros(n), 0.0
    for i in reversed(range(len(tape["alpha"]))):
        p, q = tape["p"][i], tape["q"][i]
        r1, z1 = tape["r"][i + 1], tape["z"][i + 1]
        rho, rho1 = tape["rho"][i], tape["rho"][i + 1]
        sigma, a, beta = tape["sigma"][i], tape["alpha"][i], tape["beta"][i]
        # p_(i+1) = z_(i+1) + beta_i p_i
        zbar = zbar + pbar
        betabar = float(pbar @ p)
        pbar_i = beta * pbar
        # beta_i = rho_(i+1) / rho_i
        rhobar = rhobar + betabar / rho
        rhobar_i = -betabar * rho1 / rho ** 2
        # rho_(i+1) = r_(i+1) . z_(i+1)
        rbar = rbar + rhobar * z1
        zbar = zbar + rhobar * r1
        # z_(i+1) = J^-1 r_(i+1)
        rbar = rbar + Jinv * zbar
        # r_(i+1) = r_i - alpha_i q_i
        abar = -float(rbar @ q)
        qbar = -a * rbar
        # c_(i+1) = c_i + alpha_i p_i
        abar += float(cbar @ p)
        pbar_i = pbar_i + a * cbar
        # alpha_i = rho_i / sigma_i
        rhobar_i += abar / sigma
        sigmabar = -abar * rho / sigma ** 2
        # sigma_i = p_i . q_i
        pbar_i = pbar_i + sigmabar * q
        qbar = qbar + sigmabar * p
        # q_i = M p_i
        pbar_i = pbar_i + apply_M(geo, qbar, D)
        # the adjoint of the state before iteration i
        pbar, rhobar, zbar = pbar_i, rhobar_i, np.zeros(n)
    # p_0 = z_0, rho_0 = r_0 . z_0, z_0 = J^-1 r_0, r_0 = b - M c0
    zbar = zbar + pbar
    rbar = rbar + rhobar * tape["z"][0]
    zbar = zbar + rhobar * tape["r"][0]
    rbar = rbar + Jinv * zbar
    return slope_adjoint(geo, rbar)
