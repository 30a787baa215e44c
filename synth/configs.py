"""Workload descriptions of the five FEWHA benchmark configurations.

A workload is a plain dict:

    D, obs            telescope diameter [m], central obstruction as a diameter ratio
    wfs[]             n_sub (subapertures per side), nb (fine subapertures per coarse
                      subaperture and side; 1 for an ordinary sensor), lgs (bool),
                      theta (x, y) [rad], H (sodium height [m], LGS only), sigma [rad]
    layers[]          reconstruction layers: h [m], w (Cn2 weight), delta (grid spacing
                      [m]), n (grid side, power of two), levels (wavelet scales)
    dms[]             h [m], spacing [m], n_act (actuators per side)
    params            alpha, tau, gain, iters, r0 [m at 500 nm], L0 [m]
    truth             the synthetic true atmosphere: h[], w[], r0, L0, screen_n,
                      screen_dx, wind (per-layer (vx, vy) [m/s]), frame_rate [Hz]

Geometry follows the paper's MAORY description (Sec. 4.1, Tables 1-4) where the
configuration names it; the rest is stated beside each value.
"""

import math

import numpy as np

ARCSEC = math.pi / (180.0 * 3600.0)
FOV_RAD = 60.0 * ARCSEC          # 1 arcmin field of view (Table 1)
NA_HEIGHT = 90e3                 # sodium layer height (Table 1)


def arcsec(x):
    return x * ARCSEC


def _ring(radius, azimuths_deg):
    return [(radius * math.cos(math.radians(a)), radius * math.sin(math.radians(a)))
            for a in azimuths_deg]


def _wind(n_layers, seed=3000, vmin=5.0, vmax=30.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    speed = rng.uniform(vmin, vmax, n_layers)
    ang = rng.uniform(0.0, 2.0 * math.pi, n_layers)
    return [(float(s * math.cos(a)), float(s * math.sin(a))) for s, a in zip(speed, ang)]


def _nearest_compress(truth_h, truth_w, recon_h):
    """Cn2 compression: every true layer goes to the nearest reconstruction altitude."""
    out = [0.0] * len(recon_h)
    for h, w in zip(truth_h, truth_w):
        k = min(range(len(recon_h)), key=lambda i: abs(recon_h[i] - h))
        out[k] += w
    return out


def _grid_side(D, nfine, wfs, h, delta, margin=2, nmax=128):
    """Smallest power-of-two layer grid holding every sensor footprint at height h."""
    half = 0.0
    for w in wfs:
        s = 1.0 - h / w["H"] if w["lgs"] else 1.0
        for t in w["theta"]:
            half = max(half, (s * D / 2.0 + abs(t) * h))
    need = half / delta + margin
    n = 8
    while n / 2 < need:
        n *= 2
    if n > nmax:
        raise ValueError("layer footprint needs a grid above %d" % nmax)
    return n


def tiny_scao():
    """Config 1: 8 m SCAO, one on-axis 16x16 NGS, two layers, one DM, FP64 plain."""
    layers = [dict(h=0.0, w=0.7, delta=0.5, n=32, levels=3),
              dict(h=8000.0, w=0.3, delta=1.0, n=16, levels=3)]
    return dict(
        name="tiny_scao_8m", D=8.0, obs=0.0,
        wfs=[dict(n_sub=16, nb=1, lgs=False, theta=(0.0, 0.0), H=0.0, sigma=0.05)],
        layers=layers,
        dms=[dict(h=0.0, spacing=0.5, n_act=17)],
        params=dict(alpha=1.0, tau=0.0, gain=1.0, iters=4, r0=0.157, L0=25.0),
        truth=dict(h=[0.0, 8000.0], w=[0.7, 0.3], r0=0.157, L0=25.0,
                   screen_n=256, screen_dx=0.125, wind=_wind(2), frame_rate=1000.0),
    )


MAORY_RECON_H = [0.0, 140.0, 280.0, 560.0, 1100.0, 2300.0, 4500.0, 9000.0, 18000.0]
MAORY_DM_H = [0.0, 4000.0, 12700.0]
MAORY_DM_NACT = [81, 49, 41]


def maory_truth_profile(n=35, h_max=25e3, h_min=50.0, scale_height=3000.0):
    """35-layer truth: ground plus 34 log-spaced altitudes, exponentially decaying Cn2."""
    h = [0.0] + list(np.geomspace(h_min, h_max, n - 1))
    w = np.exp(-np.asarray(h) / scale_height)
    w = w / w.sum()
    return [float(x) for x in h], [float(x) for x in w]


def maory():
    """Config 2: MAORY-size MCAO (39 m, 6 LGS 80x80 + 3 NGS 2x2, 9 layers, 3 DMs)."""
    D, nsub = 39.0, 80
    d = D / nsub
    lgs = [dict(n_sub=nsub, nb=1, lgs=True, theta=t, H=NA_HEIGHT, sigma=0.1)
           for t in _ring(arcsec(45.0), [0, 60, 120, 180, 240, 300])]
    ngs = [dict(n_sub=2, nb=40, lgs=False, theta=t, H=0.0, sigma=0.02)
           for t in _ring(arcsec(60.0), [60, 180, 300])]
    th, tw = maory_truth_profile()
    rw = _nearest_compress(th, tw, MAORY_RECON_H)
    layers = []
    for h, w in zip(MAORY_RECON_H, rw):
        if h <= 4500.0:
            layers.append(dict(h=h, w=w, delta=d, n=128, levels=7))
        else:
            layers.append(dict(h=h, w=w, delta=2 * d, n=64, levels=6))
    dms = [dict(h=h, spacing=(D + h * FOV_RAD) / (na - 1), n_act=na)
           for h, na in zip(MAORY_DM_H, MAORY_DM_NACT)]
    return dict(
        name="maory_39m_6lgs80_3ngs2_9L_3dm", D=D, obs=0.28, wfs=lgs + ngs,
        layers=layers, dms=dms,
        params=dict(alpha=1.0, tau=0.0, gain=1.0, iters=4, r0=0.157, L0=25.0),
        truth=dict(h=th, w=tw, r0=0.157, L0=25.0, screen_n=512, screen_dx=d / 2,
                   wind=_wind(len(th)), frame_rate=1000.0),
    )


NA_FWHM = 11.4e3                 # sodium profile FWHM [m] (Table 1)
SPOT_FWHM = arcsec(1.1)          # non-elongated LGS spot FWHM [rad]: not in the paper; a
                                 # value typical of an ELT LGS spot, stated as a choice


def with_elongation(wl, alpha_eta=0.2, na_fwhm=NA_FWHM, spot_fwhm=SPOT_FWHM):
    """Turn on the LGS spot-elongation noise model (Eq. 3; alpha_eta = 0.2 as in Table 5).

    Launch positions are not given in the paper: each laser is side-launched from the
    pupil edge at its guide star's azimuth, (D/2)(cos az, sin az)."""
    wl = dict(wl)
    wl["name"] = wl["name"] + "_elongated"
    wl["params"] = dict(wl["params"], alpha_eta=alpha_eta)
    wfs = []
    for W in wl["wfs"]:
        W = dict(W)
        if W["lgs"]:
            az = math.atan2(W["theta"][1], W["theta"][0])
            W.update(launch=(0.5 * wl["D"] * math.cos(az), 0.5 * wl["D"] * math.sin(az)),
                     na_fwhm=na_fwhm, spot_fwhm=spot_fwhm)
        wfs.append(W)
    wl["wfs"] = wfs
    return wl


def paper_mcao():
    """The paper's own MAORY simulation geometry (Sec. 4.1, Tables 1-5): 37 m, 11 % of the
    pupil area obstructed, 6 LGS 74x74 on a 90 arcsec diameter circle with spot
    elongation (alpha_eta = 0.2), 3 NGS 2x2 on a 110 arcsec circle, and 3 layers at the DM
    altitudes (128^2 @ 0.5 m, 64^2 @ 1 m, 64^2 @ 1 m) so that the fit F is the identity on
    the DM actuators (75^2 @ 0.5 m, 47^2 @ 1 m, 37^2 @ 1 m)."""
    D, nsub = 37.0, 74
    lgs = [dict(n_sub=nsub, nb=1, lgs=True, theta=t, H=NA_HEIGHT, sigma=0.1)
           for t in _ring(arcsec(45.0), [0, 60, 120, 180, 240, 300])]
    ngs = [dict(n_sub=2, nb=37, lgs=False, theta=t, H=0.0, sigma=0.02)
           for t in _ring(arcsec(55.0), [60, 180, 300])]
    layers = [dict(h=0.0, w=0.75, delta=0.5, n=128, levels=7),
              dict(h=4000.0, w=0.15, delta=1.0, n=64, levels=6),
              dict(h=12700.0, w=0.10, delta=1.0, n=64, levels=6)]
    dms = [dict(h=0.0, spacing=0.5, n_act=75), dict(h=4000.0, spacing=1.0, n_act=47),
           dict(h=12700.0, spacing=1.0, n_act=37)]
    th, tw = maory_truth_profile()
    wl = dict(
        name="paper_37m_6lgs74_3ngs2_3L_3dm", D=D, obs=math.sqrt(0.11), wfs=lgs + ngs,
        layers=layers, dms=dms,
        params=dict(alpha=1.0, tau=0.0, gain=1.0, iters=4, r0=0.157, L0=25.0),
        truth=dict(h=th, w=tw, r0=0.157, L0=25.0, screen_n=512, screen_dx=D / nsub / 2,
                   wind=_wind(len(th)), frame_rate=1000.0),
    )
    wl = with_elongation(wl)
    wl["name"] = "paper_37m_6lgs74_3ngs2_3L_3dm"
    return wl


def tiny_mcao_elongated():
    """The 4 m MCAO test geometry with the LGS spot-elongation noise model.  On a 4 m
    pupil the elongation is small; a 0.1 arcsec spot makes its term (alpha_eta |beta| /
    f)^2 of order one, so that the tests exercise it."""
    return with_elongation(tiny_mcao(), spot_fwhm=arcsec(0.1))


def realtime_loop():
    """Config 3: the config-1 geometry run as a 1 kHz frame loop with frozen flow."""
    wl = tiny_scao()
    wl["name"] = "realtime_8m_2000frames"
    wl["frames"] = 2000
    return wl


def differentiable():
    """Config 5: config-1 geometry used for gradients of the fitted-DM error."""
    wl = tiny_scao()
    wl["name"] = "differentiable_8m"
    return wl


def batched_instances(count=64, seed0=4000):
    """Config 4: independent tomography problems of uneven size."""
    out = []
    for i in range(count):
        rng = np.random.Generator(np.random.PCG64(seed0 + i))
        D = float(rng.choice([8.0, 16.0, 24.0, 39.0]))
        nfine = {8.0: 16, 16.0: 32, 24.0: 48, 39.0: 80}[D]
        d = D / nfine
        n_wfs = int(rng.integers(1, 7))
        sigma = float(rng.uniform(0.05, 0.15))
        if n_wfs == 1:
            wfs = [dict(n_sub=nfine, nb=1, lgs=False, theta=(0.0, 0.0), H=0.0, sigma=sigma)]
        else:
            az = [360.0 * k / (n_wfs - 1) for k in range(n_wfs - 1)]
            wfs = [dict(n_sub=nfine, nb=1, lgs=True, theta=t, H=NA_HEIGHT, sigma=sigma)
                   for t in _ring(arcsec(45.0), az)]
            wfs.append(dict(n_sub=nfine, nb=1, lgs=False, theta=(0.0, 0.0), H=0.0,
                            sigma=sigma))
        n_layers = int(rng.integers(2, 10))
        hs = [0.0] + sorted(rng.choice(MAORY_RECON_H[1:], n_layers - 1, replace=False).tolist())
        w = np.exp(-np.asarray(hs) / 3000.0) * rng.uniform(0.5, 1.5, n_layers)
        w = w / w.sum()
        layers = []
        for h, wl_ in zip(hs, w):
            delta = d if h <= 4500.0 else 2 * d
            n = _grid_side(D, nfine, wfs, h, delta)
            layers.append(dict(h=float(h), w=float(wl_), delta=delta, n=n,
                               levels=int(round(math.log2(n)))))
        n_dms = int(rng.integers(1, 4))
        dms = []
        for k, h in enumerate(MAORY_DM_H[:n_dms]):
            na = [nfine + 1, int(round(0.6 * nfine)) + 1, int(round(0.5 * nfine)) + 1][k]
            dms.append(dict(h=h, spacing=(D + h * FOV_RAD) / (na - 1), n_act=na))
        r0 = float(rng.uniform(0.1, 0.2))
        th = hs
        out.append(dict(
            name="instance_%02d" % i, D=D, obs=0.0 if D < 39.0 else 0.28, wfs=wfs,
            layers=layers, dms=dms,
            params=dict(alpha=1.0, tau=0.0, gain=1.0, iters=4, r0=r0, L0=25.0),
            truth=dict(h=list(th), w=[float(x) for x in w], r0=r0, L0=25.0,
                       screen_n=256 if D < 24 else 512, screen_dx=d / 2,
                       wind=_wind(len(th), seed=3000 + i), frame_rate=1000.0),
        ))
    return out


def tiny_mcao():
    """Test-size MCAO: 4 m, 20 % obstruction, 2 LGS 8x8, 1 coarse 2x2 NGS, 3 layers, 2 DMs.

    Small enough for dense assembly, and it exercises every sensor kind: the cone
    effect, LGS tip/tilt removal, coarse NGS blocks and a layer split between DMs.
    """
    D = 4.0
    lgs = [dict(n_sub=8, nb=1, lgs=True, theta=t, H=NA_HEIGHT, sigma=0.1)
           for t in _ring(arcsec(10.0), [0, 180])]
    ngs = [dict(n_sub=2, nb=4, lgs=False, theta=_ring(arcsec(15.0), [90])[0], H=0.0, sigma=0.02)]
    hs, ws = [0.0, 3000.0, 6000.0], [0.6, 0.25, 0.15]
    layers = [dict(h=h, w=w, delta=0.5, n=16, levels=4) for h, w in zip(hs, ws)]
    dms = [dict(h=0.0, spacing=0.5, n_act=9),
           dict(h=5000.0, spacing=(D + 5000.0 * FOV_RAD) / 6, n_act=7)]
    return dict(
        name="tiny_mcao_4m", D=D, obs=0.2, wfs=lgs + ngs, layers=layers, dms=dms,
        params=dict(alpha=1.0, tau=0.0, gain=1.0, iters=4, r0=0.157, L0=25.0),
        truth=dict(h=hs, w=ws, r0=0.157, L0=25.0, screen_n=128, screen_dx=0.125,
                   wind=_wind(3), frame_rate=1000.0),
    )


def workload_by_name(name):
    table = {"tiny_scao": tiny_scao, "maory": maory, "realtime": realtime_loop,
             "differentiable": differentiable, "tiny_mcao": tiny_mcao,
             "tiny_mcao_elongated": tiny_mcao_elongated, "paper_mcao": paper_mcao}
    return table[name]()
