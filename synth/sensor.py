"""Synthetic Shack-Hartmann measurements of the true atmosphere.

A subaperture measures the average phase gradient over its area times its size,
i.e. the phase difference across it (radians).  The simulation evaluates the true
phase on a grid at half the subaperture spacing and integrates the phase along the
two opposite subaperture edges with the trapezoid rule (3 points per fine edge,
2*nb + 1 per coarse edge), then adds i.i.d. Gaussian noise of the sensor's sigma
(seed 2000 + frame).  This is a measurement simulation of the truth, finer than
the reconstructor's own sensor model.

Illuminated subapertures: centre radius within [obs*D/2, D/2].
Slope layout per sensor: x-slopes of the illuminated subapertures in row-major
order (row = y), then the y-slopes in the same order; sensors concatenated.
"""

import numpy as np

from .atmosphere import TruthAtmosphere


def _illuminated(n, D, obs):
    c = -D / 2 + (np.arange(n) + 0.5) * (D / n)
    r = np.hypot(c[None, :], c[:, None])
    return (r >= obs * D / 2) & (r <= D / 2)


def slope_counts(wl):
    out = []
    for w in wl["wfs"]:
        out.append(2 * int(_illuminated(w["n_sub"], wl["D"], wl["obs"]).sum()))
    return out


def sensor_slopes(atm, wl, w, frame):
    """Noise-free synthetic slopes of one sensor (its slope layout)."""
    D = wl["D"]
    n_sub, nb = w["n_sub"], w["nb"]
    N = n_sub * nb
    xs = -D / 2 + np.arange(2 * N + 1) * (D / (2 * N))
    X, Y = np.meshgrid(xs, xs)                     # rows = y, cols = x
    H = w["H"] if w["lgs"] else 0.0
    ph = atm.phase(X, Y, w["theta"], H, frame)
    e = 2 * nb                                      # half-grid samples per subaperture edge
    wts = np.ones(e + 1)
    wts[0] = wts[-1] = 0.5
    wts /= wts.sum()
    span = n_sub * e
    left = np.zeros((n_sub, n_sub))
    right = np.zeros((n_sub, n_sub))
    bottom = np.zeros((n_sub, n_sub))
    top = np.zeros((n_sub, n_sub))
    for k in range(e + 1):
        # sample k along the edge: rows i*e + k (vertical edges), cols j*e + k (horizontal)
        left += wts[k] * ph[k:k + span:e, 0:span:e]
        right += wts[k] * ph[k:k + span:e, e:span + 1:e]
        bottom += wts[k] * ph[0:span:e, k:k + span:e]
        top += wts[k] * ph[e:span + 1:e, k:k + span:e]
    sx = right - left
    sy = top - bottom
    m = _illuminated(n_sub, D, wl["obs"])
    return np.concatenate([sx[m], sy[m]])


def simulate_slopes(wl, frame=0, atm=None, noise=True):
    """Full measurement vector of a workload at one frame (float64)."""
    if atm is None:
        atm = TruthAtmosphere(wl["truth"])
    parts = []
    rng = np.random.Generator(np.random.PCG64(2000 + frame))
    for w in wl["wfs"]:
        s = sensor_slopes(atm, wl, w, frame)
        if noise:
            s = s + w["sigma"] * rng.standard_normal(s.shape)
        parts.append(s)
    return np.concatenate(parts)


def true_phase_at(wl, x, y, frame=0, atm=None):
    """The true on-axis phase (star at infinity) at pupil points (x, y)."""
    if atm is None:
        atm = TruthAtmosphere(wl["truth"])
    return atm.phase(np.asarray(x, float), np.asarray(y, float), (0.0, 0.0), 0.0, frame)


def slope_sequence(wl, n_frames, atm=None, first=0):
    """Measurement vectors of frames first .. first + n_frames - 1 as rows (float64)."""
    if atm is None:
        atm = TruthAtmosphere(wl["truth"])
    return np.stack([simulate_slopes(wl, first + t, atm=atm) for t in range(n_frames)])
