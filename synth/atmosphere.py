"""Seeded von Karman phase screens with frozen flow (the synthetic true atmosphere).

Each true layer k is a periodic screen of screen_n^2 samples at spacing screen_dx,
drawn by the FFT method from the von Karman phase power spectrum

    Phi(f) = 0.023 * r0_k^(-5/3) * (f^2 + L0^-2)^(-11/6),   f in cycles/m,

with r0_k^(-5/3) = w_k * r0^(-5/3), phases in radians at 500 nm, seed 1000 + k.
Frozen flow translates layer k by its wind vector times the frame time.
"""

import numpy as np


def von_karman_screen(n, dx, r0, L0, seed):
    """One periodic screen (n x n, spacing dx) with the von Karman spectrum, zero mean."""
    rng = np.random.Generator(np.random.PCG64(seed))
    df = 1.0 / (n * dx)
    fx = np.fft.fftfreq(n, d=dx)
    f2 = fx[None, :] ** 2 + fx[:, None] ** 2
    psd = 0.023 * r0 ** (-5.0 / 3.0) * (f2 + 1.0 / L0 ** 2) ** (-11.0 / 6.0)
    psd[0, 0] = 0.0
    noise = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2.0)
    # phi(x) = sum_k a_k exp(2 pi i k.x), E|a_k|^2 = psd * df^2; real part, rescaled
    spec = noise * np.sqrt(psd) * df
    scr = np.fft.ifft2(spec) * (n * n)
    return np.ascontiguousarray(np.real(scr) * np.sqrt(2.0))


class TruthAtmosphere:
    """The true layered atmosphere of a workload; screens are drawn on first use."""

    def __init__(self, truth):
        self.h = list(truth["h"])
        self.w = list(truth["w"])
        self.r0 = float(truth["r0"])
        self.L0 = float(truth["L0"])
        self.n = int(truth["screen_n"])
        self.dx = float(truth["screen_dx"])
        self.wind = list(truth["wind"])
        self.rate = float(truth.get("frame_rate", 1000.0))
        self._screens = None

    @property
    def screens(self):
        if self._screens is None:
            self._screens = [
                von_karman_screen(self.n, self.dx, self.r0 * w ** (-3.0 / 5.0), self.L0, 1000 + k)
                for k, w in enumerate(self.w)
            ]
        return self._screens

    def sample(self, k, x, y, frame=0):
        """Layer k at metric points (x, y) at the given frame, periodic bilinear sampling."""
        vx, vy = self.wind[k]
        t = frame / self.rate
        u = (x - vx * t) / self.dx
        v = (y - vy * t) / self.dx
        j0 = np.floor(u)
        i0 = np.floor(v)
        fx = u - j0
        fy = v - i0
        n = self.n
        j0 = j0.astype(np.int64) % n
        i0 = i0.astype(np.int64) % n
        j1 = (j0 + 1) % n
        i1 = (i0 + 1) % n
        s = self.screens[k]
        return ((1 - fy) * ((1 - fx) * s[i0, j0] + fx * s[i0, j1])
                + fy * ((1 - fx) * s[i1, j0] + fx * s[i1, j1]))

    def phase(self, x, y, theta, H, frame=0):
        """Integrated phase seen from the pupil point (x, y) towards direction theta.

        H = 0 means a star at infinity; otherwise the cone of a source at height H.
        """
        out = np.zeros(np.broadcast(x, y).shape)
        for k, h in enumerate(self.h):
            s = 1.0 - h / H if H > 0 else 1.0
            out += self.sample(k, s * x + theta[0] * h, s * y + theta[1] * h, frame)
        return out
