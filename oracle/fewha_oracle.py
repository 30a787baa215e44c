"""Plain FP64 CPU oracle of the FEWHA per-frame hot path (Stadler & Ramlau, MAORY).

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU baseline
of the benchmark; the product path never imports it.  Slow and literal on purpose:
every operator is written out from its definition in the paper, with numpy (and
small dense matrix products) as the only primitives, in float64 throughout.

Paper passages followed
  Sec. 2        layered atmosphere, A_g = Gamma_g P_g, Shack-Hartmann model, NGS/LGS
                propagation, noise covariance C_g = sigma^2 I (Eq. 2)
  Sec. 3.1      dual-domain discretisation, periodic Daubechies-3 wavelets W,
                diagonal prior D, operator M (Eq. 6), right-hand side b, Eq. (5)
  Sec. 3.2      LGS tip-tilt projector T and C_hat_g^-1 = (I - T) C_g^-1 (I - T)
  Sec. 3.3      modified Jacobi preconditioner (Eq. 7), warm restart
  Sec. 3.4      Algorithm 1 (RHS, initial residual, PCG, fitting, control law)
  Sec. 4.1      Tables 2 and 3 (layer grids, DM actuators, bilinear mirror shape)

Readings where the paper is silent or garbled:
  R1  the printed y-slope formula is garbled; the y-slope is the x-slope's mirror:
      s^y_ij = ((phi_{i+1,j} - phi_{i,j}) + (phi_{i+1,j+1} - phi_{i,j+1})) / 2
  R2  slopes are phase differences across a subaperture (rad), no 1/d factor
  R3  node (i, j) of an aperture grid sits at (x, y) = (-D/2 + j d, -D/2 + i d):
      index i runs along y (rows), j along x (columns)
  R4  a subaperture is active iff its centre radius r has obs*D/2 <= r <= D/2
  R5  layer grids are periodic n x n (n = 2^J), node (i, j) at ((j - n/2) delta,
      (i - n/2) delta); every projected footprint must lie inside the grid
  R6  W is orthonormal (c = W phi, W^-1 = W^T): the delta_l scaling is folded into D
  R7  db3 analysis a_k = sum_m h_m x_(2k+m mod n), d_k with g_m = (-1)^m h_(5-m);
      2-D: rows then columns, Mallat layout [LL LH; HL HH], recursion on LL
  R8  D: von Karman band average of the wavelet-coefficient variance (see
      prior_diag); constant per (layer, level)
  R9  coarse NGS sensors (nb > 1 fine subapertures per coarse one and side) live
      on the fine aperture grid; a coarse slope is (1/nb) * the sum of the fine
      slopes of the active fine subapertures in its block
  R10 C_g = sigma_g^2 I for every NGS and, with alpha_eta = 0, every LGS; T applies to
      LGS only
  R11 J uses the exact diagonal of W (sum_g P_g^T Gamma_g^T C_hat_g^-1 Gamma_g P_g)
      W^T; tau defaults to 0
  R12 PCG: left-preconditioned, Fletcher-Reeves beta, fixed iteration count, no
      early exit except r.z == 0 (then the iterate is final)
  R13 fitting F: a layer between two DM altitudes h_a <= h <= h_b is split
      linearly, (h_b - h)/(h_b - h_a) to DM a and the rest to DM b; above the top
      DM (or below the lowest) it goes wholly to that DM.  The shape is sampled
      bilinearly at the actuator positions, lateral coordinates unchanged.
  R14 open-loop control a = (1 - gain) a_prev + gain a_tilde (Algorithm 1)
  R26 augmented PCG (Sec. 3.4, Algorithm 1): the previous frame's directions P and
      Q = M P augment the Krylov space.  The start is corrected over span(P),
      c0 += P y, r0 -= Q y, y_k = p_k.r0 / p_k.q_k, and every new direction is made
      M-conjugate to P, p = z + beta p_old - P mu, mu_k = q_k.z / p_k.q_k (P^T Q is
      diagonal for the M-conjugate directions of one CG run).  At most 8 directions
      (iter <= 8); none on the first frame.
  R27 closed loop (Algorithm 1): the DM shape is bilinear between actuators (Sec. 4.1),
      i.e. sum_k a_k times the bilinear hat of actuator k, so it is zero beyond the
      outer actuators' hats; actuator (p, q) of a DM with n_act per side sits at
      ((q - (n_act-1)/2) spacing, (p - (n_act-1)/2) spacing).  Sensor g sees DM m like a
      layer, at s x + theta h_m (s = 1 - h_m/H for an LGS).  The pseudo-open-loop slopes
      are s + Gamma P_DM a^(i-1) (the residual slopes s measure phase minus DM shape)
      and the control law is a^(i+1) = a^(i) + gain (a_tilde - a^(i-1)), both as printed;
      a^(0) = a^(-1) = 0.
  R28 LGS spot elongation (Eq. 3): in subaperture (i, j) with midpoint (x, y) (R3),
      beta = (FWHM / H^2) ((x, y) - (x_LL, y_LL)), FWHM the sodium profile's, (x_LL, y_LL)
      the sensor's laser launch position; C_ij = sigma^2 (I + (alpha_eta^2 / f^2) beta
      beta^T), f the FWHM of the non-elongated spot [rad].  Its inverse (Sherman-Morrison)
      is sigma^-2 (I - gamma beta beta^T), gamma = c / (1 + c |beta|^2), c = alpha_eta^2
      / f^2, and C_hat^-1 = (I - T) C^-1 (I - T) no longer collapses to sigma^-2 (I - T).
      Elongation is on for an LGS when alpha_eta, FWHM and f are all > 0.
  R30 least-squares DM fitting (Sec. 4.1: more layers than DMs need a fit of their own): the
      commands minimise sum_k w_k ||Pi (A_k a - L_k phi)||^2 + eps ||a||^2, where along
      fitting direction theta_k the pupil nodes x (spacing D / n_fit, inside the annulus)
      see the layers at x + theta_k h_l (bilinear, R5) and the DMs at x + theta_k h_m
      (bilinear hats, R27), and Pi removes the mean over the pupil (piston is not fitted).
      Directions, weights, n_fit and eps are inputs.
"""

import math

import numpy as np

# ----------------------------------------------------------------------------
# Daubechies-3 wavelet filters (Sec. 3.1: "periodic Daubechies-N wavelets, N=3")
# ----------------------------------------------------------------------------


def db3_lowpass():
    """db3 scaling filter h_0..h_5 from Daubechies' closed form (sum h = sqrt 2)."""
    s10 = math.sqrt(10.0)
    r = math.sqrt(5.0 + 2.0 * s10)
    q = 16.0 * math.sqrt(2.0)
    return np.array([1.0 + s10 + r, 5.0 + s10 + 3.0 * r, 10.0 - 2.0 * s10 + 2.0 * r,
                     10.0 - 2.0 * s10 - 2.0 * r, 5.0 + s10 - 3.0 * r, 1.0 + s10 - r]) / q


def db3_filters():
    """(h, g): scaling and wavelet filters, g_m = (-1)^m h_(5-m) (reading R7)."""
    h = db3_lowpass()
    g = np.array([(-1.0) ** m * h[5 - m] for m in range(6)])
    return h, g


def _analysis_1d(x, axis):
    """One periodic analysis step along `axis` (length m even): [a | d]."""
    h, g = db3_filters()
    x = np.moveaxis(x, axis, -1)
    m = x.shape[-1]
    k = np.arange(m // 2)
    a = np.zeros(x.shape[:-1] + (m // 2,))
    d = np.zeros(x.shape[:-1] + (m // 2,))
    for t in range(6):
        idx = (2 * k + t) % m
        a += h[t] * x[..., idx]
        d += g[t] * x[..., idx]
    return np.moveaxis(np.concatenate([a, d], axis=-1), -1, axis)


def _synthesis_1d(y, axis):
    """Inverse of _analysis_1d: the transpose of the orthonormal analysis step."""
    h, g = db3_filters()
    y = np.moveaxis(y, axis, -1)
    m = y.shape[-1]
    k = np.arange(m // 2)
    a = y[..., : m // 2]
    d = y[..., m // 2:]
    x = np.zeros(y.shape)
    for t in range(6):
        idx = (2 * k + t) % m
        # x_(2k+t) receives h_t a_k + g_t d_k; within one t the indices are distinct
        x[..., idx] += h[t] * a + g[t] * d
    return np.moveaxis(x, -1, axis)


def dwt2(phi, levels):
    """Forward 2-D periodic db3 transform c = W phi of an n x n layer (R7)."""
    c = np.array(phi, dtype=np.float64, copy=True)
    n = c.shape[-1]
    for lev in range(levels):
        m = n >> lev
        blk = c[..., :m, :m]
        blk = _analysis_1d(blk, -1)      # rows (along x)
        blk = _analysis_1d(blk, -2)      # columns (along y)
        c[..., :m, :m] = blk
    return c


def idwt2(c, levels):
    """Inverse 2-D transform phi = W^T c (W orthonormal, R6)."""
    phi = np.array(c, dtype=np.float64, copy=True)
    n = phi.shape[-1]
    for lev in reversed(range(levels)):
        m = n >> lev
        blk = phi[..., :m, :m]
        blk = _synthesis_1d(blk, -2)
        blk = _synthesis_1d(blk, -1)
        phi[..., :m, :m] = blk
    return phi


def level_map(n, levels):
    """Level of every Mallat position: 1..levels for details, levels+1 for the LL band."""
    r = np.arange(n)
    mx = np.maximum(r[:, None], r[None, :])
    lev = np.full((n, n), levels + 1, dtype=np.int64)
    for j in range(1, levels + 1):
        lev[(mx >= (n >> j)) & (mx < (n >> (j - 1)))] = j
    return lev


def basis_1d(n, j, kind):
    """1-D level-j periodic basis functions (columns), kind 'a' (scaling) or 'd'.

    Column k is W_1d^T applied to the unit coefficient k of the level-j band, i.e.
    the synthesis of that unit vector through levels j, j-1, ..., 1.
    """
    nj = n >> j
    e = np.zeros((n, nj))
    off = 0 if kind == "a" else nj
    e[off + np.arange(nj), np.arange(nj)] = 1.0
    for lev in reversed(range(j)):
        m = n >> lev
        e[:m] = _synthesis_1d(e[:m], 0)
    return e


# ----------------------------------------------------------------------------
# Geometry (Sec. 2, Sec. 3.1, Sec. 4.1)
# ----------------------------------------------------------------------------


class GeometryError(ValueError):
    pass


def _interp_matrix(coord, n):
    """Bilinear (1-D linear) interpolation matrix from grid coordinates (R5)."""
    i0 = np.floor(coord).astype(np.int64)
    f = coord - i0
    if np.any(i0 < 0) or np.any(i0 + 1 > n - 1):
        raise GeometryError("footprint leaves the layer grid")
    R = np.zeros((coord.size, n))
    R[np.arange(coord.size), i0] += 1.0 - f
    R[np.arange(coord.size), i0 + 1] += f
    return R


def _hat_matrix(coord, n):
    """Bilinear hat-function sampling on a lattice of n nodes (R27): like the layer
    interpolation, but a stencil point outside [0, n-1] contributes nothing."""
    R = np.zeros((coord.size, n))
    for a, u in enumerate(coord):
        i0 = int(np.floor(u))
        f = u - i0
        if 0 <= i0 < n:
            R[a, i0] += 1.0 - f
        if 0 <= i0 + 1 < n:
            R[a, i0 + 1] += f
    return R


def active_mask(n, D, obs):
    """Active subapertures of an n x n lenslet array (R4)."""
    c = -D / 2 + (np.arange(n) + 0.5) * (D / n)
    r = np.hypot(c[None, :], c[:, None])
    return (r >= obs * D / 2) & (r <= D / 2)


def fitting_weights(layer_h, dm_h):
    """w[l, m]: share of layer l given to DM m (R13)."""
    order = np.argsort(dm_h)
    hs = np.asarray(dm_h, float)[order]
    w = np.zeros((len(layer_h), len(dm_h)))
    for l, h in enumerate(layer_h):
        if h >= hs[-1]:
            w[l, order[-1]] = 1.0
        elif h <= hs[0]:
            w[l, order[0]] = 1.0
        else:
            a = int(np.searchsorted(hs, h, side="right") - 1)
            t = (hs[a + 1] - h) / (hs[a + 1] - hs[a])
            w[l, order[a]] += t
            w[l, order[a + 1]] += 1.0 - t
    return w


class Geometry:
    """All static structure of one FEWHA instance, built from a workload dict."""

    def __init__(self, wl):
        self.D = float(wl["D"])
        self.obs = float(wl["obs"])
        p = wl["params"]
        self.alpha = float(p["alpha"])
        self.tau = float(p.get("tau", 0.0))
        self.gain = float(p.get("gain", 1.0))
        self.iters = int(p["iters"])
        self.r0 = float(p["r0"])
        self.L0 = float(p["L0"])
        # layers
        self.layers = []
        off = 0
        for L in wl["layers"]:
            n = int(L["n"])
            if n < 2 or n & (n - 1):
                raise GeometryError("layer grid side must be a power of two")
            if not (1 <= int(L["levels"]) <= int(round(math.log2(n)))):
                raise GeometryError("wavelet levels out of range")
            self.layers.append(dict(h=float(L["h"]), w=float(L["w"]), delta=float(L["delta"]),
                                    n=n, levels=int(L["levels"]), off=off))
            off += n * n
        self.n_c = off
        # sensors
        self.wfs = []
        soff = 0
        for W in wl["wfs"]:
            n_sub, nb = int(W["n_sub"]), int(W["nb"])
            N = n_sub * nb
            d = self.D / N
            lgs = bool(W["lgs"])
            if lgs and nb != 1:
                raise GeometryError("LGS sensors have no coarse blocks")
            fine = active_mask(N, self.D, self.obs)
            coarse = active_mask(n_sub, self.D, self.obs) if nb > 1 else fine
            if nb > 1:
                # fine subapertures only count inside active coarse blocks (R9)
                fine = fine & np.kron(coarse, np.ones((nb, nb), dtype=bool))
            n_act = int(coarse.sum())
            xs = -self.D / 2 + np.arange(N + 1) * d
            Ry, Rx = [], []
            for L in self.layers:
                s = 1.0 - L["h"] / float(W["H"]) if lgs else 1.0
                tx, ty = W["theta"]
                Rx.append(_interp_matrix((s * xs + tx * L["h"]) / L["delta"] + L["n"] / 2, L["n"]))
                Ry.append(_interp_matrix((s * xs + ty * L["h"]) / L["delta"] + L["n"] / 2, L["n"]))
            # the DMs seen by this sensor (R27), the same propagation as the layers
            Qx, Qy = [], []
            for m in wl["dms"]:
                hm, na = float(m["h"]), int(m["n_act"])
                s = 1.0 - hm / float(W["H"]) if lgs else 1.0
                tx, ty = W["theta"]
                Qx.append(_hat_matrix((s * xs + tx * hm) / float(m["spacing"]) + (na - 1) / 2.0, na))
                Qy.append(_hat_matrix((s * xs + ty * hm) / float(m["spacing"]) + (na - 1) / 2.0, na))
            self.wfs.append(dict(N=N, n_sub=n_sub, nb=nb, d=d, lgs=lgs, sigma=float(W["sigma"]),
                                 mask=fine, cmask=coarse, n_active=n_act, soff=soff,
                                 ns=2 * n_act, Rx=Rx, Ry=Ry, Qx=Qx, Qy=Qy,
                                 H=float(W["H"]), launch=tuple(W.get("launch", (0.0, 0.0))),
                                 na_fwhm=float(W.get("na_fwhm", 0.0)),
                                 spot_fwhm=float(W.get("spot_fwhm", 0.0))))
            soff += 2 * n_act
        self.n_s = soff
        # deformable mirrors and the fitting split (R13)
        self.dms = []
        aoff = 0
        fw = fitting_weights([L["h"] for L in self.layers], [float(m["h"]) for m in wl["dms"]])
        for mi, m in enumerate(wl["dms"]):
            na = int(m["n_act"])
            xa = (np.arange(na) - (na - 1) / 2.0) * float(m["spacing"])
            Rs = []
            for li, L in enumerate(self.layers):
                if fw[li, mi] != 0.0:
                    Rs.append(_interp_matrix(xa / L["delta"] + L["n"] / 2, L["n"]))
                else:
                    Rs.append(None)
            self.dms.append(dict(n_act=na, off=aoff, R=Rs, w=fw[:, mi], spacing=float(m["spacing"]),
                                 h=float(m["h"])))
            aoff += na * na
        self.n_a = aoff
        set_elongation(self, float(p.get("alpha_eta", 0.0)))

    # -- vector layout helpers ------------------------------------------------
    def split(self, c):
        return [np.asarray(c[L["off"]:L["off"] + L["n"] ** 2]).reshape(L["n"], L["n"])
                for L in self.layers]

    def join(self, blocks):
        return np.concatenate([np.asarray(b, float).ravel() for b in blocks])


def set_elongation(geo, alpha_eta):
    """The spot-elongation weights of every LGS (Eq. 3, reading R28) on its fine
    subaperture grid: beta_1, beta_2 and gamma = c / (1 + c |beta|^2), c = alpha_eta^2 /
    f^2, so that C_ij^-1 = sigma^-2 (I - gamma beta beta^T).  None where it is off."""
    geo.alpha_eta = alpha_eta
    for W in geo.wfs:
        W["el"] = None
        if not (W["lgs"] and alpha_eta > 0 and W["na_fwhm"] > 0 and W["spot_fwhm"] > 0):
            continue
        N, d = W["N"], W["d"]
        mid = -geo.D / 2 + (np.arange(N) + 0.5) * d
        k = W["na_fwhm"] / W["H"] ** 2
        b1 = k * (mid[None, :] - W["launch"][0]) * np.ones((N, 1))
        b2 = k * (mid[:, None] - W["launch"][1]) * np.ones((1, N))
        c = (alpha_eta / W["spot_fwhm"]) ** 2
        gam = c / (1.0 + c * (b1 ** 2 + b2 ** 2))
        W["el"] = dict(b1=b1, b2=b2, gamma=gam)


# ----------------------------------------------------------------------------
# Operators of the forward model (Sec. 2) in the finite-element domain
# ----------------------------------------------------------------------------


def project(geo, g, phis):
    """P_g phi: sum over layers of the bilinear layer values seen by sensor g.

    Sec. 2: phi_theta(x) = sum_l phi_l(s_l x + theta h_l), s_l = 1 - h_l/H for an LGS
    (cone effect) and 1 for an NGS.  Returned on the (N+1)^2 aperture node grid.
    """
    W = geo.wfs[g]
    out = np.zeros((W["N"] + 1, W["N"] + 1))
    for l, phi in enumerate(phis):
        out += W["Ry"][l] @ phi @ W["Rx"][l].T
    return out


def dm_project(geo, g, a):
    """The DM shapes seen by sensor g on its aperture nodes: sum over DMs of the
    bilinear mirror surface (Sec. 4.1) at s x + theta h_m (R27)."""
    W = geo.wfs[g]
    out = np.zeros((W["N"] + 1, W["N"] + 1))
    for mi, m in enumerate(geo.dms):
        A = np.asarray(a[m["off"]:m["off"] + m["n_act"] ** 2]).reshape(m["n_act"], m["n_act"])
        out += W["Qy"][mi] @ A @ W["Qx"][mi].T
    return out


def dm_slopes(geo, a):
    """Gamma P_DM a: the slopes every sensor would measure of the DM shapes a (the term
    of the pseudo-open-loop slopes of Algorithm 1)."""
    return np.concatenate([sh_slopes(geo, g, dm_project(geo, g, a)) for g in range(len(geo.wfs))])


def project_adj(geo, g, v):
    """P_g^T v: transpose of `project`, one array per layer."""
    W = geo.wfs[g]
    return [W["Ry"][l].T @ v @ W["Rx"][l] for l in range(len(geo.layers))]


def fine_slopes(v):
    """Shack-Hartmann x/y slopes of every fine subaperture (Sec. 2; R1, R2, R3)."""
    sx = 0.5 * ((v[:-1, 1:] - v[:-1, :-1]) + (v[1:, 1:] - v[1:, :-1]))
    sy = 0.5 * ((v[1:, :-1] - v[:-1, :-1]) + (v[1:, 1:] - v[:-1, 1:]))
    return sx, sy


def fine_slopes_adj(sx, sy):
    """Transpose of fine_slopes: node values from per-subaperture x/y weights."""
    n = sx.shape[0]
    v = np.zeros((n + 1, n + 1))
    v[:-1, 1:] += 0.5 * sx
    v[:-1, :-1] -= 0.5 * sx
    v[1:, 1:] += 0.5 * sx
    v[1:, :-1] -= 0.5 * sx
    v[1:, :-1] += 0.5 * sy
    v[:-1, :-1] -= 0.5 * sy
    v[1:, 1:] += 0.5 * sy
    v[:-1, 1:] -= 0.5 * sy
    return v


def _block_sum(a, n_sub, nb):
    return a.reshape(n_sub, nb, n_sub, nb).sum(axis=(1, 3))


def sh_slopes(geo, g, v):
    """Gamma_g v: slopes of the active subapertures, layout [s^x ; s^y] (Sec. 2)."""
    W = geo.wfs[g]
    sx, sy = fine_slopes(v)
    m = W["mask"]
    if W["nb"] == 1:
        return np.concatenate([sx[m], sy[m]])
    # coarse sensor (R9): (1/nb) * sum of active fine slopes in each block
    cx = _block_sum(np.where(m, sx, 0.0), W["n_sub"], W["nb"]) / W["nb"]
    cy = _block_sum(np.where(m, sy, 0.0), W["n_sub"], W["nb"]) / W["nb"]
    cm = W["cmask"]
    return np.concatenate([cx[cm], cy[cm]])


def sh_slopes_adj(geo, g, s):
    """Gamma_g^T s on the aperture node grid."""
    W = geo.wfs[g]
    k = W["n_active"]
    if W["nb"] == 1:
        m = W["mask"]
        sx = np.zeros(m.shape)
        sy = np.zeros(m.shape)
        sx[m] = s[:k]
        sy[m] = s[k:]
    else:
        cm = W["cmask"]
        cx = np.zeros(cm.shape)
        cy = np.zeros(cm.shape)
        cx[cm] = s[:k]
        cy[cm] = s[k:]
        ones = np.ones((W["nb"], W["nb"]))
        m = W["mask"]
        sx = np.where(m, np.kron(cx, ones), 0.0) / W["nb"]
        sy = np.where(m, np.kron(cy, ones), 0.0) / W["nb"]
    return fine_slopes_adj(sx, sy)


def tiptilt_projector(k):
    """T = (1/|M|) (t^x t^y)(t^x t^y)^T as a dense 2k x 2k matrix (Sec. 3.2)."""
    tx = np.concatenate([np.ones(k), np.zeros(k)])
    ty = np.concatenate([np.zeros(k), np.ones(k)])
    Tt = np.stack([tx, ty], axis=1)
    return (Tt @ Tt.T) / k


def noise_weight(geo, g, s):
    """C_hat_g^-1 s: (I - T) C_g^-1 (I - T) s for an LGS, C_g^-1 s for an NGS.

    C_g = sigma_g^2 I (Eq. 2, R10), or for an elongated LGS the 2x2 blocks of Eq. 3,
    inverted per subaperture as sigma^-2 (I - gamma beta beta^T) (R28); T from Sec. 3.2,
    applied through its rank-2 form T s = (1/|M|)(t^x (t^x . s) + t^y (t^y . s)).
    """
    W = geo.wfs[g]
    inv = 1.0 / W["sigma"] ** 2
    if not W["lgs"]:
        return inv * s
    k = W["n_active"]

    def i_minus_t(v):
        out = v.copy()
        out[:k] -= v[:k].sum() / k
        out[k:] -= v[k:].sum() / k
        return out

    def c_inv(v):
        if W["el"] is None:
            return inv * v
        m = W["mask"]
        b1, b2, gam = W["el"]["b1"][m], W["el"]["b2"][m], W["el"]["gamma"][m]
        bu = b1 * v[:k] + b2 * v[k:]
        return inv * np.concatenate([v[:k] - gam * b1 * bu, v[k:] - gam * b2 * bu])

    return i_minus_t(c_inv(i_minus_t(s)))


def forward_model(geo, phis):
    """s = A phi = (Gamma_g P_g phi)_g, concatenated over sensors (Eq. 1)."""
    return np.concatenate([sh_slopes(geo, g, project(geo, g, phis)) for g in range(len(geo.wfs))])


def forward_model_adj(geo, s):
    """A^T s, one array per layer."""
    out = [np.zeros((L["n"], L["n"])) for L in geo.layers]
    for g, W in enumerate(geo.wfs):
        sg = s[W["soff"]:W["soff"] + W["ns"]]
        for l, y in enumerate(project_adj(geo, g, sh_slopes_adj(geo, g, sg))):
            out[l] += y
    return out


def data_operator(geo, phis):
    """B phi = sum_g P_g^T Gamma_g^T C_hat_g^-1 Gamma_g P_g phi (FE domain)."""
    out = [np.zeros((L["n"], L["n"])) for L in geo.layers]
    for g in range(len(geo.wfs)):
        s = sh_slopes(geo, g, project(geo, g, phis))
        u = sh_slopes_adj(geo, g, noise_weight(geo, g, s))
        for l, y in enumerate(project_adj(geo, g, u)):
            out[l] += y
    return out


# ----------------------------------------------------------------------------
# Wavelet domain: W, D, M, b (Sec. 3.1)
# ----------------------------------------------------------------------------


def W_fwd(geo, phis):
    """Block-diagonal W: every layer transformed with its own level count."""
    return geo.join([dwt2(p, L["levels"]) for p, L in zip(phis, geo.layers)])


def W_inv(geo, c):
    return [idwt2(b, L["levels"]) for b, L in zip(geo.split(c), geo.layers)]


def von_karman_psd(kappa, r0, L0):
    """Phase PSD 0.023 r0^-5/3 (kappa^2 + L0^-2)^-11/6, kappa in cycles/m."""
    return 0.023 * r0 ** (-5.0 / 3.0) * (kappa ** 2 + L0 ** -2) ** (-11.0 / 6.0)


def prior_diag(geo, r0=None, L0=None, weights=None):
    """D: a diagonal stand-in for C_phi^-1 on the wavelet coefficients (Sec. 3.1, R8).

    For layer l (grid n, spacing delta, Cn2 weight w_l) and level band B (detail
    level j: FFT index box [-n/2^j, n/2^j)^2 minus [-n/2^(j+1), n/2^(j+1))^2; the LL
    band: [-n/2^(L+1), n/2^(L+1))^2), the coefficient variance is approximated by
    the band average of the DFT-domain variance n^2 dk^2 w_l Phi(|k| dk), dk = 1/(n
    delta), and D = 1 / variance.
    """
    r0 = geo.r0 if r0 is None else r0
    L0 = geo.L0 if L0 is None else L0
    out = []
    for li, L in enumerate(geo.layers):
        n, delta, lev = L["n"], L["delta"], L["levels"]
        w = L["w"] if weights is None else weights[li]
        dk = 1.0 / (n * delta)
        k = np.arange(-n // 2, n // 2)
        kap = dk * np.hypot(k[None, :], k[:, None])
        var = (n * dk) ** 2 * w * von_karman_psd(kap, r0, L0)

        def kin(m):
            """FFT indices of the half-open box [-m, m)^2 (m may be 1/2)."""
            ok = (k >= -m) & (k < m)
            return ok[None, :] & ok[:, None]

        Dl = np.zeros((n, n))
        lm = level_map(n, lev)
        for j in range(1, lev + 1):
            band = kin(n / 2.0 ** j) & ~kin(n / 2.0 ** (j + 1))
            Dl[lm == j] = 1.0 / var[band].mean()
        band = kin(n / 2.0 ** (lev + 1))      # half-width 1/2 at full depth: k = 0 only
        Dl[lm == lev + 1] = 1.0 / var[band].mean()
        out.append(Dl)
    return geo.join(out)


def apply_M(geo, c, D=None):
    """M c = W B W^T c + alpha D c (Eq. 6 with W orthonormal, R6)."""
    if D is None:
        D = prior_diag(geo)
    return W_fwd(geo, data_operator(geo, W_inv(geo, c))) + geo.alpha * D * c


def rhs(geo, s):
    """b = W sum_g P_g^T Gamma_g^T C_hat_g^-1 s_g (Sec. 3.1; Algorithm 1, RHS step)."""
    out = [np.zeros((L["n"], L["n"])) for L in geo.layers]
    for g, W in enumerate(geo.wfs):
        sg = np.asarray(s[W["soff"]:W["soff"] + W["ns"]], float)
        u = sh_slopes_adj(geo, g, noise_weight(geo, g, sg))
        for l, y in enumerate(project_adj(geo, g, u)):
            out[l] += y
    return W_fwd(geo, out)


# ----------------------------------------------------------------------------
# Preconditioner (Sec. 3.3, Eq. 7)
# ----------------------------------------------------------------------------


def data_diag_bruteforce(geo):
    """diag(W B W^T) by applying the data term to every unit vector (small cases)."""
    out = np.zeros(geo.n_c)
    for i in range(geo.n_c):
        e = np.zeros(geo.n_c)
        e[i] = 1.0
        out[i] = W_fwd(geo, data_operator(geo, W_inv(geo, e)))[i]
    return out


def data_diag(geo):
    """diag(W B W^T) exactly, from the separable structure of the basis.

    A wavelet basis function of layer l is an outer product f_y(i) f_x(j) of 1-D
    level-j functions, and bilinear projection onto a sensor's aperture grid is
    separable (Ry f_y)(Rx f_x)^T, so each slope of Gamma P psi is a product of
    1-D averages and differences.  Summing their squares over the mask (and, for
    an LGS, removing the tip/tilt means; for a coarse sensor, summing each block
    first) reduces to small matrix products per (sensor, layer, level, orientation).
    """
    out = [np.zeros((L["n"], L["n"])) for L in geo.layers]
    for li, L in enumerate(geo.layers):
        n, lev = L["n"], L["levels"]
        bands = []  # (level j, y-kind, x-kind, row offset, col offset)
        for j in range(1, lev + 1):
            h = n >> j
            bands += [(j, "a", "d", 0, h), (j, "d", "a", h, 0), (j, "d", "d", h, h)]
        bands.append((lev, "a", "a", 0, 0))
        funcs = {(j, k): basis_1d(n, j, k) for j in range(1, lev + 1) for k in "ad"}
        for W in geo.wfs:
            m = W["mask"].astype(float)
            inv = 1.0 / W["sigma"] ** 2
            Ry, Rx = W["Ry"][li], W["Rx"][li]
            for (j, ky, kx, r0_, c0_) in bands:
                Fy = Ry @ funcs[(j, ky)]
                Fx = Rx @ funcs[(j, kx)]
                ya, yd = 0.5 * (Fy[:-1] + Fy[1:]), Fy[1:] - Fy[:-1]
                xa, xd = 0.5 * (Fx[:-1] + Fx[1:]), Fx[1:] - Fx[:-1]
                # s^x = y-average * x-difference, s^y = y-difference * x-average
                if W["nb"] == 1:
                    val = (ya ** 2).T @ m @ (xd ** 2) + (yd ** 2).T @ m @ (xa ** 2)
                    if W["lgs"]:
                        tx = ya.T @ m @ xd
                        ty = yd.T @ m @ xa
                        val = val - (tx ** 2 + ty ** 2) / W["n_active"]
                        if W["el"] is not None:
                            # minus sum over the mask of gamma (beta . u)^2, u the slopes
                            # without their means mu = (tx, ty) / |M| (R28):
                            #   E - 2 mu . e + mu^T K mu
                            e = W["el"]
                            G11 = m * e["gamma"] * e["b1"] ** 2
                            G12 = m * e["gamma"] * e["b1"] * e["b2"]
                            G22 = m * e["gamma"] * e["b2"] ** 2
                            E = ((ya ** 2).T @ G11 @ (xd ** 2) + 2.0 * (ya * yd).T @ G12 @ (xd * xa)
                                 + (yd ** 2).T @ G22 @ (xa ** 2))
                            e1 = ya.T @ G11 @ xd + yd.T @ G12 @ xa
                            e2 = ya.T @ G12 @ xd + yd.T @ G22 @ xa
                            mx, my = tx / W["n_active"], ty / W["n_active"]
                            K11, K12, K22 = G11.sum(), G12.sum(), G22.sum()
                            val = val - (E - 2.0 * (mx * e1 + my * e2)
                                         + K11 * mx ** 2 + 2.0 * K12 * mx * my + K22 * my ** 2)
                else:
                    nb, ns = W["nb"], W["n_sub"]
                    val = 0.0
                    for I in range(ns):
                        for J in range(ns):
                            if not W["cmask"][I, J]:
                                continue
                            rs = slice(I * nb, (I + 1) * nb)
                            cs = slice(J * nb, (J + 1) * nb)
                            mb = m[rs, cs]
                            cx = ya[rs].T @ mb @ xd[cs] / nb
                            cy = yd[rs].T @ mb @ xa[cs] / nb
                            val = val + cx ** 2 + cy ** 2
                h = funcs[(j, ky)].shape[1]
                out[li][r0_:r0_ + h, c0_:c0_ + h] += inv * val
    return geo.join(out)


def precond_diag(geo, D=None, data=None):
    """J = diag(W B W^T) + alpha max(D, tau I) (Eq. 7; R11)."""
    if D is None:
        D = prior_diag(geo)
    if data is None:
        data = data_diag(geo)
    return data + geo.alpha * np.maximum(D, geo.tau)


# ----------------------------------------------------------------------------
# Solver and frame (Sec. 3.3, Sec. 3.4 / Algorithm 1)
# ----------------------------------------------------------------------------


def pcg(geo, b, c0, Jinv, iters, D=None, r0=None):
    """Preconditioned CG on M c = b, fixed iteration count (R12).

    Returns (c, r) after `iters` iterations started from c0 (r0 = b - M c0 unless
    an initial residual is supplied, the warm-restart form of Algorithm 1).
    """
    c = np.array(c0, float, copy=True)
    r = b - apply_M(geo, c, D) if r0 is None else np.array(r0, float, copy=True)
    z = Jinv * r
    p = z.copy()
    rz = float(r @ z)
    for _ in range(iters):
        if rz == 0.0:
            break
        q = apply_M(geo, p, D)
        a = rz / float(p @ q)
        c = c + a * p
        r = r - a * q
        z = Jinv * r
        rz_new = float(r @ z)
        beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
    return c, r


def augmented_pcg(geo, b, c0, Jinv, iters, D=None, r0=None, prev=None):
    """Augmented PCG of Algorithm 1 (Sec. 3.4, reading R26).

    `prev` = (P, Q, pq): the search directions p_k of the previous frame's PCG, their
    images q_k = M p_k and the inner products p_k . q_k.  The start is corrected over
    span(P), all coefficients from the same residual:
        y_k = (p_k . r0) / (p_k . q_k),   c0 <- c0 + sum_k y_k p_k,   r0 <- r0 - sum_k y_k q_k,
    and every direction of this frame is made M-conjugate to P:
        p = z + beta p_old - sum_k mu_k p_k,   mu_k = (q_k . z) / (p_k . q_k)
    (a previous direction with p_k . q_k <= 0 is left out).  Otherwise standard PCG for
    `iters` iterations; its directions, images and inner products are returned.

    Returns (c, r, (P, Q, pq)).
    """
    c = np.array(c0, float, copy=True)
    r = b - apply_M(geo, c, D) if r0 is None else np.array(r0, float, copy=True)
    P, Q, pq = prev if prev is not None else ([], [], [])
    use = [k for k in range(len(pq)) if pq[k] > 0.0]
    y = {k: float(P[k] @ r) / pq[k] for k in use}
    for k in use:
        c = c + y[k] * P[k]
        r = r - y[k] * Q[k]

    def conjugate_to_prev(v):
        mu = {k: float(Q[k] @ v) / pq[k] for k in use}
        for k in use:
            v = v - mu[k] * P[k]
        return v

    z = Jinv * r
    p = conjugate_to_prev(z)
    rz = float(r @ z)
    Ps, Qs, pqs = [], [], []
    for _ in range(iters):
        if rz == 0.0:
            break
        q = apply_M(geo, p, D)
        pq_k = float(p @ q)
        Ps.append(p.copy())
        Qs.append(q)
        pqs.append(pq_k)
        a = rz / pq_k
        c = c + a * p
        r = r - a * q
        z = Jinv * r
        rz_new = float(r @ z)
        p = conjugate_to_prev(z) + (rz_new / rz) * p
        rz = rz_new
    return c, r, (Ps, Qs, pqs)


def fit(geo, c):
    """a_tilde = F W^-1 c: layers back to the FE domain, then the DM fit (R13)."""
    phis = W_inv(geo, c)
    out = []
    for m in geo.dms:
        a = np.zeros((m["n_act"], m["n_act"]))
        for l, phi in enumerate(phis):
            if m["R"][l] is not None:
                a += m["w"][l] * (m["R"][l] @ phi @ m["R"][l].T)
        out.append(a.ravel())
    return np.concatenate(out)


def fitting_geometry(geo, directions, n_fit):
    """Pupil nodes and, per fitting direction, the layer and DM sampling matrices (R30)."""
    D = geo.D
    xs = -D / 2 + np.arange(n_fit + 1) * (D / n_fit)
    r = np.hypot(xs[None, :], xs[:, None])
    mask = (r >= geo.obs * D / 2) & (r <= D / 2)
    dirs = []
    for tx, ty in directions:
        L = [(_interp_matrix((xs + ty * Ly["h"]) / Ly["delta"] + Ly["n"] / 2, Ly["n"]),
              _interp_matrix((xs + tx * Ly["h"]) / Ly["delta"] + Ly["n"] / 2, Ly["n"]))
             for Ly in geo.layers]
        M = [(_hat_matrix((xs + ty * m["h"]) / m["spacing"] + (m["n_act"] - 1) / 2.0, m["n_act"]),
              _hat_matrix((xs + tx * m["h"]) / m["spacing"] + (m["n_act"] - 1) / 2.0, m["n_act"]))
             for m in geo.dms]
        dirs.append(dict(L=L, M=M))
    return dict(mask=mask, dirs=dirs)


def pupil_centre(fg, v):
    """Pi v: the pupil nodes' values without their mean, zero outside the pupil."""
    m = fg["mask"]
    out = np.where(m, v, 0.0)
    out[m] -= out[m].mean()
    return out


def dm_along(geo, fg, k, a):
    out = 0.0
    for mi, m in enumerate(geo.dms):
        A = np.asarray(a[m["off"]:m["off"] + m["n_act"] ** 2]).reshape(m["n_act"], m["n_act"])
        Qy, Qx = fg["dirs"][k]["M"][mi]
        out = out + Qy @ A @ Qx.T
    return out


def dm_along_adj(geo, fg, k, v):
    out = []
    for mi, m in enumerate(geo.dms):
        Qy, Qx = fg["dirs"][k]["M"][mi]
        out.append((Qy.T @ v @ Qx).ravel())
    return np.concatenate(out)


def ls_fit(geo, phis, fg, weights, eps, tol=1e-13, max_iters=100000):
    """Least-squares DM fit (R30) by CG on the normal equations
    (sum_k w_k A_k^T Pi A_k + eps I) a = sum_k w_k A_k^T Pi L_k phi."""
    K = len(fg["dirs"])

    def normal(a):
        out = eps * a
        for k in range(K):
            out = out + weights[k] * dm_along_adj(geo, fg, k, pupil_centre(fg, dm_along(geo, fg, k, a)))
        return out

    rhs_ = np.zeros(geo.n_a)
    for k in range(K):
        v = sum(Ly @ phi @ Lx.T for (Ly, Lx), phi in zip(fg["dirs"][k]["L"], phis))
        rhs_ = rhs_ + weights[k] * dm_along_adj(geo, fg, k, pupil_centre(fg, v))
    a = np.zeros(geo.n_a)
    r = rhs_.copy()
    p = r.copy()
    rr = float(r @ r)
    r0 = np.sqrt(rr)
    for _ in range(max_iters):
        if np.sqrt(rr) <= tol * r0 or rr == 0.0:
            break
        q = normal(p)
        al = rr / float(p @ q)
        a = a + al * p
        r = r - al * q
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
    return a


def fit_adj(geo, a):
    """(F W^-1)^T a, returned as a wavelet-coefficient vector."""
    phis = [np.zeros((L["n"], L["n"])) for L in geo.layers]
    for m in geo.dms:
        am = a[m["off"]:m["off"] + m["n_act"] ** 2].reshape(m["n_act"], m["n_act"])
        for l in range(len(phis)):
            if m["R"][l] is not None:
                phis[l] += m["w"][l] * (m["R"][l].T @ am @ m["R"][l])
    return W_fwd(geo, phis)


class Reconstructor:
    """One FEWHA instance across frames (Algorithm 1, open loop; augmented PCG on request)."""

    def __init__(self, wl):
        self.geo = Geometry(wl)
        self.D = prior_diag(self.geo)
        self.J = precond_diag(self.geo, self.D)
        self.Jinv = 1.0 / self.J
        self.c = np.zeros(self.geo.n_c)
        self.a = np.zeros(self.geo.n_a)
        self.b_prev = None
        self.r_prev = None
        self.dirs = None         # (P, Q, pq) of the previous augmented frame
        self.a_old = np.zeros(self.geo.n_a)   # a^(i-1) of the closed loop

    def frame(self, s, warm_residual=False, augmented=False, closed_loop=False):
        """One frame; with closed_loop, s are residual slopes and the pseudo-open-loop
        slopes and the closed-loop control law of Algorithm 1 apply (R27)."""
        geo = self.geo
        if closed_loop:
            s = np.asarray(s, float) + dm_slopes(geo, self.a_old)
        b = rhs(geo, s)
        r0 = None
        if warm_residual and self.b_prev is not None:
            r0 = (b - self.b_prev) + self.r_prev
        if augmented:
            self.c, r, self.dirs = augmented_pcg(geo, b, self.c, self.Jinv, geo.iters, self.D, r0,
                                                 self.dirs)
        else:
            self.c, r = pcg(geo, b, self.c, self.Jinv, geo.iters, self.D, r0)
        self.b_prev, self.r_prev = b, r
        a_tilde = fit(geo, self.c)
        if closed_loop:
            a_new = self.a + geo.gain * (a_tilde - self.a_old)
            self.a_old = self.a
            self.a = a_new
        else:
            self.a = (1.0 - geo.gain) * self.a + geo.gain * a_tilde
        return self.a.copy()
