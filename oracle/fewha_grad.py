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
"""

import numpy as np

from .fewha_oracle import (W_fwd, W_inv, data_operator, fit, fit_adj, noise_weight,
                           prior_diag, project, rhs, sh_slopes)


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
