"""Pins of the oracle's diagonal prior D (Sec. 3.1)."""
import numpy as np

import oracle as O
import synth
from synth.atmosphere import von_karman_screen


def _one_layer(n, delta, levels, w=1.0, r0=0.157, L0=25.0):
    wl = synth.tiny_scao()
    wl["layers"] = [dict(h=0.0, w=w, delta=delta, n=n, levels=levels)]
    wl["dms"] = [dict(h=0.0, spacing=0.5, n_act=5)]
    wl["params"]["r0"], wl["params"]["L0"] = r0, L0
    return O.Geometry(wl)


def test_band_boxes_count_like_coefficients():
    """The FFT band of every level holds exactly as many indices as that level has coefficients."""
    for n, lev in [(16, 2), (32, 5), (64, 6), (128, 7)]:
        k = np.arange(-n // 2, n // 2)

        def box(m):
            ok = (k >= -m) & (k < m)
            return ok[None, :] & ok[:, None]

        lm = O.level_map(n, lev)
        for j in range(1, lev + 1):
            band = box(n / 2 ** j) & ~box(n / 2 ** (j + 1))
            assert band.sum() == (lm == j).sum()
        assert box(n / 2 ** (lev + 1)).sum() == (lm == lev + 1).sum()


def test_prior_is_constant_per_level_and_scales_with_weight():
    geo = _one_layer(32, 0.5, 4)
    D = O.prior_diag(geo).reshape(32, 32)
    lm = O.level_map(32, 4)
    for j in range(1, 6):
        v = D[lm == j]
        assert np.ptp(v) == 0.0 and v[0] > 0
    D2 = O.prior_diag(_one_layer(32, 0.5, 4, w=0.25)).reshape(32, 32)
    np.testing.assert_allclose(D2, 4.0 * D, rtol=1e-14)
    D3 = O.prior_diag(_one_layer(32, 0.5, 4, r0=0.314)).reshape(32, 32)
    # D ~ r0^(5/3) for every band (the PSD scales with r0^-5/3)
    np.testing.assert_allclose(D3, 2 ** (5 / 3) * D, rtol=1e-12)


def test_inertial_range_scaling_is_eleven_thirds():
    """Pure power law (L0 -> infinity): D_j / D_(j+1) -> 2^(11/3) between detail levels."""
    geo = _one_layer(256, 0.5, 4, L0=1e9)
    D = O.prior_diag(geo).reshape(256, 256)
    lm = O.level_map(256, 4)
    for j in (1, 2, 3):
        ratio = D[lm == j][0] / D[lm == j + 1][0]
        assert abs(ratio / 2 ** (11 / 3) - 1) < 0.03


def test_prior_tracks_monte_carlo_wavelet_variances():
    """The band reading vs the empirical variance of db3 coefficients of von Karman screens.

    The band average is an approximation (wavelet spectra leak out of their boxes), so
    this is a loose physics check: every detail level within a factor 1.5.
    """
    n, delta, lev = 32, 0.5, 5
    geo = _one_layer(n, delta, lev)
    D = O.prior_diag(geo).reshape(n, n)
    lm = O.level_map(n, lev)
    acc = np.zeros((n, n))
    K = 200
    for s in range(K):
        acc += O.dwt2(von_karman_screen(n, delta, 0.157, 25.0, 50000 + s), lev) ** 2
    acc /= K
    for j in range(1, lev + 1):
        ratio = acc[lm == j].mean() * D[lm == j][0]
        assert 1 / 1.5 < ratio < 1.5, (j, ratio)
