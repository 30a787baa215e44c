"""Host logic of the GPU least-squares fit (no GPU needed): the stencil tables built by
build_lsfit and the per-node / per-actuator functions the fewha_fit_ls kernels call,
compiled for the CPU from the same sources (tests/host/lsfit_host.cu) and evaluated slice by
slice and actuator by actuator as the kernels do, against the oracle's sampling matrices
(Sec. 4.1, reading R30).  A wrong stencil index, weight, pupil mask or adjoint gather range
changes these results far beyond double rounding."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARC = synth.arcsec(1.0)
DIRS5 = [(0.0, 0.0), (15 * ARC, 0.0), (-15 * ARC, 0.0), (0.0, 15 * ARC), (0.0, -15 * ARC)]
CASES = [
    ("tiny_scao", [(0.0, 0.0), (5 * ARC, -3 * ARC)], [1.0, 2.0], 16, 1e-4),
    ("tiny_mcao", DIRS5, [1.0, 0.5, 0.0, 0.5, 0.5], 13, 1e-2),
    ("tiny_mcao", [(12 * ARC, -7 * ARC)], [1.0], 5, 0.0),
    ("maory", [(x * ARC, y * ARC) for y in (-20, 0, 20) for x in (-20, 0, 20)], [1.0] * 9, 80, 1e-2),
    ("paper_mcao", [(25 * ARC, 10 * ARC), (-20 * ARC, 0.0)], [1.0, 0.7], 37, 1e-3),
]


@pytest.fixture(scope="module")
def H(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    out = str(tmp_path_factory.mktemp("lsfit") / "lsfit_host.so")
    csrc = os.path.join(ROOT, "paper_2202_11945_gb300", "csrc")
    subprocess.run([nvcc, "-O1", "-std=c++17", "-x", "cu", "-Xcompiler", "-fPIC", "-shared",
                    os.path.join(ROOT, "tests", "host", "lsfit_host.cu"), os.path.join(csrc, "fewha_setup.cpp"),
                    "-o", out], check=True, capture_output=True)
    return ctypes.CDLL(out)


def _apply(H, wl, dirs, w, n_fit, eps, phi, a):
    from paper_2202_11945_gb300 import fewha
    tel, wfs, layers, dms, _ = fewha.structs_from_workload(wl, 64)
    D = ctypes.POINTER(ctypes.c_double)
    keep = [np.ascontiguousarray(x, float) for x in ([d[0] for d in dirs], [d[1] for d in dirs], w)]
    cfg = fewha.LsFit(len(dirs), *[x.ctypes.data_as(D) for x in keep], n_fit, eps)
    K, nf1 = len(dirs), n_fit + 1
    ul, ud = np.zeros((K, nf1, nf1)), np.zeros((K, nf1, nf1))
    ml, md, out = np.zeros(K), np.zeros(K), np.zeros(a.size)
    rc = H.lsfit_host_apply(ctypes.byref(tel), wfs, len(wfs), layers, len(layers), dms, len(dms),
                            ctypes.byref(cfg), phi.ctypes.data_as(D), a.ctypes.data_as(D),
                            *[x.ctypes.data_as(D) for x in (ul, ml, ud, md, out)])
    return rc, ul, ml, ud, md, out


@pytest.mark.parametrize("case", CASES, ids=["%s-%d" % (c[0], i) for i, c in enumerate(CASES)])
def test_sampling_and_adjoint_match_the_oracle(H, case):
    name, dirs, w, n_fit, eps = case
    wl = synth.workload_by_name(name)
    geo = O.Geometry(wl)
    fg = O.fitting_geometry(geo, dirs, n_fit)
    rng = np.random.default_rng(21)
    phis = [rng.standard_normal((L["n"], L["n"])) for L in geo.layers]
    phi = np.concatenate([p.ravel() for p in phis])
    a = rng.standard_normal(geo.n_a)
    rc, ul, ml, ud, md, out = _apply(H, wl, dirs, w, n_fit, eps, phi, a)
    assert rc == 0
    m = fg["mask"]
    assert not ul[:, ~m].any() and not ud[:, ~m].any()      # zero off the pupil
    ref_out = eps * a
    for k in range(len(dirs)):
        ref_l = O.pupil_centre(fg, sum(Ly @ p @ Lx.T for (Ly, Lx), p in zip(fg["dirs"][k]["L"], phis)))
        ref_d = O.pupil_centre(fg, O.dm_along(geo, fg, k, a))
        got_l = np.where(m, ul[k] - ml[k], 0.0)
        got_d = np.where(m, ud[k] - md[k], 0.0)
        assert np.abs(got_l - ref_l).max() <= 1e-12 * np.abs(ref_l).max(), k
        assert np.abs(got_d - ref_d).max() <= 1e-12 * np.abs(ref_d).max(), k
        ref_out = ref_out + w[k] * O.dm_along_adj(geo, fg, k, ref_d)
    assert np.abs(out - ref_out).max() <= 1e-12 * np.abs(ref_out).max()


def test_a_direction_leaving_a_layer_grid_is_a_geometry_error(H):
    wl = synth.tiny_mcao()
    geo = O.Geometry(wl)
    rc = _apply(H, wl, [(300 * ARC, 0.0)], [1.0], 8, 1e-3, np.zeros(geo.n_c), np.zeros(geo.n_a))[0]
    assert rc == -2
    with pytest.raises(O.GeometryError):
        O.fitting_geometry(geo, [(300 * ARC, 0.0)], 8)


@pytest.mark.parametrize("name,dirs,w,n_fit,eps", [
    ("tiny_mcao", DIRS5, [1.0, 0.5, 0.5, 0.5, 0.5], 8, 1e-2),
    ("paper_mcao", [(x * ARC, y * ARC) for y in (-25, 0, 25) for x in (-25, 0, 25)], [1.0] * 9, 74, 1e-2),
])
@pytest.mark.parametrize("prec,tol,bound", [(64, 1e-12, 1e-9), (32, 1e-7, 1e-4)])
def test_cg_arithmetic_reaches_the_oracle(H, name, dirs, w, n_fit, eps, prec, tol, bound):
    """The CG of the fit with the kernels' arithmetic (operators and vectors in the handle's
    type, inner products and scalars in double), run on the host: in double it meets the
    oracle's CG to 1e-9, in float to the FP32 frame bound 1e-4 (the accuracy the GPU tests
    hold the device to)."""
    from paper_2202_11945_gb300 import fewha
    wl = synth.workload_by_name(name)
    geo = O.Geometry(wl)
    c = np.random.default_rng(11).standard_normal(geo.n_c)
    phis = O.W_inv(geo, c)
    ref = O.ls_fit(geo, phis, O.fitting_geometry(geo, dirs, n_fit), w, eps)
    tel, wfs, layers, dms, _ = fewha.structs_from_workload(wl, prec)
    D = ctypes.POINTER(ctypes.c_double)
    keep = [np.ascontiguousarray(x, float) for x in ([d[0] for d in dirs], [d[1] for d in dirs], w)]
    cfg = fewha.LsFit(len(dirs), *[x.ctypes.data_as(D) for x in keep], n_fit, eps)
    phi = np.ascontiguousarray(np.concatenate([p.ravel() for p in phis]))
    a = np.zeros(geo.n_a)
    it, rel = ctypes.c_int(0), ctypes.c_double(0.0)
    rc = H.lsfit_host_solve(ctypes.byref(tel), wfs, len(wfs), layers, len(layers), dms, len(dms), ctypes.byref(cfg),
                            prec, phi.ctypes.data_as(D), a.ctypes.data_as(D), ctypes.c_double(tol), 5000,
                            ctypes.byref(it), ctypes.byref(rel))
    assert rc == 0 and 0 < it.value < 5000 and rel.value <= tol
    assert np.linalg.norm(a - ref) / np.linalg.norm(ref) <= bound
