"""Host set-up of the CUDA path (no GPU needed): the C++ tables every kernel reads
(fewha_setup.cpp: projection stencils of each (sensor, layer) pair and their adjoint gather
ranges, the slope index tables of fine and coarse sensors, the DM fitting stencils, shares
and gather ranges, the prior D and the db3 taps), compiled for the CPU from the same
sources (tests/host/setup_host.cpp) and compared with the oracle's matrices, which were
written separately from the paper (Sec. 2, Sec. 3.1, Sec. 4.1)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NAMES = ["tiny_scao", "tiny_mcao", "tiny_mcao_elongated", "maory", "paper_mcao"]
IP, DP = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)


@pytest.fixture(scope="module")
def H(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path_factory.mktemp("setup") / "setup_host.so")
    subprocess.run([cxx, "-O1", "-std=c++17", "-fPIC", "-shared", os.path.join(ROOT, "tests", "host", "setup_host.cpp"),
                    os.path.join(ROOT, "paper_2202_11945_gb300", "csrc", "fewha_setup.cpp"), "-o", out],
                   check=True, capture_output=True)
    return ctypes.CDLL(out)


_cache = {}


def tables(H, name):
    if name in _cache:
        return _cache[name]
    from paper_2202_11945_gb300 import fewha
    wl = synth.workload_by_name(name)
    tel, wfs, layers, dms, _ = fewha.structs_from_workload(wl, 64)
    args = (ctypes.byref(tel), wfs, len(wfs), layers, len(layers), dms, len(dms))
    sizes, lim = np.zeros(8, np.int64), np.zeros(6, np.int32)
    assert H.setup_sizes(*args, sizes.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), lim.ctypes.data_as(IP)) == 0
    MAXG, MAXL, MAXM, TAB, MAXN, MAXNACT = (int(x) for x in lim)
    n_c, n_s, n_nodes, n_act, n_sidx, n_cidx, n_tab, n_rng = (int(x) for x in sizes)
    t = dict(MAXL=MAXL, MAXM=MAXM, TAB=TAB, MAXN=MAXN, MAXNACT=MAXNACT)
    spec = [("pi0y", np.int32, n_tab), ("pi0x", np.int32, n_tab), ("pfy", float, n_tab), ("pfx", float, n_tab),
            ("ry_lo", np.int32, n_rng), ("ry_hi", np.int32, n_rng), ("rx_lo", np.int32, n_rng),
            ("rx_hi", np.int32, n_rng), ("sidx", np.int32, n_sidx), ("cidx", np.int32, max(n_cidx, 1)),
            ("di0", np.int32, MAXM * MAXL * MAXNACT), ("dfw", float, MAXM * MAXL * MAXNACT),
            ("dr_lo", np.int32, MAXM * MAXL * MAXN), ("dr_hi", np.int32, MAXM * MAXL * MAXN),
            ("fitw", float, MAXM * MAXL), ("D", float, n_c), ("taps", float, 12)]
    for k, dt, n in spec:
        t[k] = np.zeros(n, dt)
    p = wl["params"]
    rc = H.setup_tables(*args, ctypes.c_double(p["r0"]), ctypes.c_double(p["L0"]),
                        *[t[k].ctypes.data_as(IP if t[k].dtype == np.int32 else DP) for k, _, _ in spec])
    assert rc == 0
    t["n_c"], t["n_s"], t["n_nodes"], t["n_act"] = n_c, n_s, n_nodes, n_act
    _cache[name] = (wl, O.Geometry(wl), t)
    return _cache[name]


def dense(i0, f, rows, n):
    """The interpolation matrix of stencils (i0[a], i0[a] + 1) with weights (1 - f, f)."""
    R = np.zeros((rows, n))
    a = np.arange(rows)
    R[a, i0] += 1.0 - f
    R[a, i0 + 1] += f
    return R


def check_ranges(i0, lo, hi, R):
    """[lo, hi) of layer row i is exactly the rows whose stencil includes i, and holds
    every row with a non-zero weight on it."""
    for i in range(R.shape[1]):
        assert set(range(lo[i], hi[i])) == set(np.flatnonzero((i0 == i) | (i0 + 1 == i))), i
        assert set(np.flatnonzero(R[:, i])) <= set(range(lo[i], hi[i])), i


@pytest.mark.parametrize("name", NAMES)
def test_sizes_match_the_oracle(H, name):
    wl, geo, t = tables(H, name)
    assert (t["n_c"], t["n_s"], t["n_act"]) == (geo.n_c, geo.n_s, geo.n_a)
    assert t["n_nodes"] == sum((W["N"] + 1) ** 2 for W in geo.wfs)


@pytest.mark.parametrize("name", NAMES)
def test_projection_stencils_and_gather_ranges(H, name):
    wl, geo, t = tables(H, name)
    for g, W in enumerate(geo.wfs):
        for l, L in enumerate(geo.layers):
            base = (g * t["MAXL"] + l) * t["TAB"]
            rb = (g * t["MAXL"] + l) * t["MAXN"]
            for ax, Rm in (("y", W["Ry"][l]), ("x", W["Rx"][l])):
                i0 = t["pi0" + ax][base:base + W["N"] + 1]
                R = dense(i0, t["pf" + ax][base:base + W["N"] + 1], W["N"] + 1, L["n"])
                assert np.abs(R - Rm).max() <= 1e-13, (g, l, ax)
                check_ranges(i0, t["r%s_lo" % ax][rb:rb + L["n"]], t["r%s_hi" % ax][rb:rb + L["n"]], Rm)


@pytest.mark.parametrize("name", NAMES)
def test_slope_index_tables(H, name):
    """Fine sensors: the running index of each active subaperture in row-major order;
    coarse sensors: every active fine subaperture carries its coarse block's index."""
    wl, geo, t = tables(H, name)
    off = coff = 0
    for W in geo.wfs:
        N, nb = W["N"], W["nb"]
        sidx = t["sidx"][off:off + N * N].reshape(N, N)
        assert np.array_equal(sidx >= 0, W["mask"])
        if nb == 1:
            assert np.array_equal(sidx[W["mask"]], np.arange(W["n_active"]))
        else:
            ns = W["n_sub"]
            cidx = t["cidx"][coff:coff + ns * ns].reshape(ns, ns)
            assert np.array_equal(cidx >= 0, W["cmask"])
            assert np.array_equal(cidx[W["cmask"]], np.arange(W["n_active"]))
            blocks = np.kron(cidx, np.ones((nb, nb), dtype=np.int32))
            assert np.array_equal(sidx[W["mask"]], blocks[W["mask"]])
            coff += ns * ns
        off += N * N


@pytest.mark.parametrize("name", NAMES)
def test_dm_fitting_stencils_shares_and_ranges(H, name):
    wl, geo, t = tables(H, name)
    for m, dm in enumerate(geo.dms):
        na = dm["n_act"]
        for l, L in enumerate(geo.layers):
            assert t["fitw"][m * t["MAXL"] + l] == pytest.approx(dm["w"][l], abs=1e-15), (m, l)
            if dm["R"][l] is None:
                continue
            base = (m * t["MAXL"] + l) * t["MAXNACT"]
            i0 = t["di0"][base:base + na]
            R = dense(i0, t["dfw"][base:base + na], na, L["n"])
            assert np.abs(R - dm["R"][l]).max() <= 1e-13, (m, l)
            rb = (m * t["MAXL"] + l) * t["MAXN"]
            check_ranges(i0, t["dr_lo"][rb:rb + L["n"]], t["dr_hi"][rb:rb + L["n"]], dm["R"][l])


@pytest.mark.parametrize("name", NAMES)
def test_prior_matches_the_oracle(H, name):
    """D of the C++ set-up against the oracle's, two implementations of the same band rule
    (reading R8) written separately."""
    wl, geo, t = tables(H, name)
    ref = O.prior_diag(geo)
    assert np.abs(t["D"] - ref).max() <= 1e-12 * np.abs(ref).max()


def test_db3_taps_match_the_oracle(H):
    wl, geo, t = tables(H, "tiny_scao")
    h, g = O.db3_filters()
    assert np.abs(t["taps"][:6] - h).max() <= 1e-15
    assert np.abs(t["taps"][6:] - g).max() <= 1e-15


def extra(H, name):
    from paper_2202_11945_gb300 import fewha
    wl, geo, t = tables(H, name)
    tel, wfs, layers, dms, _ = fewha.structs_from_workload(wl, 64)
    n = len(t["pi0y"]) // t["MAXL"] * t["MAXM"]                # MAXG * MAXM * TAB
    q = {k: np.zeros(n, np.int32 if k.startswith("qi") else float) for k in ("qi0y", "qi0x", "qfy", "qfx")}
    el = np.zeros(10 * len(wl["wfs"]))
    rc = H.setup_extra(ctypes.byref(tel), wfs, len(wfs), layers, len(layers), dms, len(dms),
                       ctypes.c_double(wl["params"].get("alpha_eta", 0.0)),
                       *[q[k].ctypes.data_as(IP if k.startswith("qi") else DP) for k in ("qi0y", "qi0x", "qfy", "qfx")],
                       el.ctypes.data_as(DP))
    assert rc == 0
    return wl, geo, t, q, el.reshape(-1, 10)


@pytest.mark.parametrize("name", NAMES)
def test_closed_loop_dm_stencils(H, name):
    """The DM shapes each sensor sees (reading R27): bilinear hats, zero off the lattice."""
    wl, geo, t, q, _ = extra(H, name)
    for g, W in enumerate(geo.wfs):
        for m, dm in enumerate(geo.dms):
            base = (g * t["MAXM"] + m) * t["TAB"]
            for ax, Qm in (("y", W["Qy"][m]), ("x", W["Qx"][m])):
                i0 = q["qi0" + ax][base:base + W["N"] + 1]
                f = q["qf" + ax][base:base + W["N"] + 1]
                Q = np.zeros_like(Qm)
                for a in range(W["N"] + 1):
                    for col, wgt in ((i0[a], 1.0 - f[a]), (i0[a] + 1, f[a])):
                        if 0 <= col < dm["n_act"]:
                            Q[a, col] += wgt
                assert np.abs(Q - Qm).max() <= 1e-13, (g, m, ax)


@pytest.mark.parametrize("name", ["tiny_mcao_elongated", "paper_mcao", "tiny_mcao"])
def test_spot_elongation_constants(H, name):
    """Eq. 3 (reading R28): beta and gamma of every subaperture rebuilt from the per-sensor
    constants the kernels use, and the sums K of gamma beta beta^T over the active ones."""
    wl, geo, t, q, el = extra(H, name)
    for g, W in enumerate(geo.wfs):
        if W["el"] is None:
            assert el[g, 0] == 0
            continue
        on, k, c, lx, ly, x0, d = el[g, :7]
        assert on == 1
        N = W["N"]
        mid = x0 + np.arange(N) * d
        b1 = k * (mid[None, :] - lx) * np.ones((N, 1))
        b2 = k * (mid[:, None] - ly) * np.ones((1, N))
        gam = c / (1.0 + c * (b1 ** 2 + b2 ** 2))
        ref = W["el"]
        for got, want in ((b1, ref["b1"]), (b2, ref["b2"]), (gam, ref["gamma"])):
            assert np.abs(got - want).max() <= 1e-13 * max(np.abs(want).max(), 1e-300)
        m = W["mask"]
        K = [np.sum((ref["gamma"] * a * b)[m]) for a, b in ((ref["b1"], ref["b1"]), (ref["b1"], ref["b2"]),
                                                            (ref["b2"], ref["b2"]))]
        # K12 cancels to rounding on a symmetric geometry: compare against the largest K
        assert np.abs(el[g, 7:] - K).max() <= 1e-12 * np.abs(K).max()


def test_tail_matrix_is_the_oracles_three_level_transform(H):
    """The wavelet kernels apply the last three levels of a full decomposition (an 8 x 8 LL
    block down to 1 x 1) as one host-built 64 x 64 matrix: row k must be the oracle's
    three-level 2-D transform of the unit input k (Mallat layout), and its transpose the
    synthesis."""
    A = np.zeros(64 * 64)
    assert H.setup_tail(A.ctypes.data_as(DP)) == 0
    A = A.reshape(64, 64)
    for k in range(64):
        e = np.zeros(64)
        e[k] = 1.0
        assert np.abs(A[k] - O.dwt2(e.reshape(8, 8), 3).ravel()).max() <= 1e-14, k
        assert np.abs(A[:, k] - O.idwt2(e.reshape(8, 8), 3).ravel()).max() <= 1e-14, k


@pytest.mark.parametrize("name", ["tiny_mcao", "maory"])
def test_basis_tables_of_the_jacobi_diagonal(H, name):
    """The exact diagonal of W B W^T (Eq. 7) is built on the GPU from 1-D basis functions of
    each layer and level: the table holds the synthesis of the unit coefficient at shift 0
    of the level-j scaling (kind 0) and wavelet (kind 1) bands, i.e. column 0 of the oracle's
    basis matrices."""
    from paper_2202_11945_gb300 import fewha
    wl = synth.workload_by_name(name)
    geo = O.Geometry(wl)
    tel, wfs, layers, dms, _ = fewha.structs_from_workload(wl, 64)
    n_basis = sum(2 * L["levels"] * L["n"] for L in geo.layers)
    basis = np.zeros(n_basis)
    MAXL = tables(H, name)[2]["MAXL"]
    off = np.zeros(MAXL * 9 * 2, np.int32)
    maxlev = ctypes.c_int(0)
    assert H.setup_basis(ctypes.byref(tel), wfs, len(wfs), layers, len(layers), dms, len(dms),
                         basis.ctypes.data_as(DP), ctypes.c_long(n_basis), off.ctypes.data_as(IP),
                         ctypes.byref(maxlev)) == 0
    assert maxlev.value + 1 == 9
    for l, L in enumerate(geo.layers):
        n = L["n"]
        for j in range(1, L["levels"] + 1):
            for kind, name_k in ((0, "a"), (1, "d")):
                o = off[(l * 9 + j) * 2 + kind]
                ref = O.basis_1d(n, j, name_k)[:, 0]
                assert np.abs(basis[o:o + n] - ref).max() <= 1e-14, (l, j, kind)
