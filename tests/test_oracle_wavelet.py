"""Pins of the oracle's periodic Daubechies-3 transform (Sec. 3.1)."""
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "db3_taps.txt")


def _golden_taps():
    return np.array([float(x) for x in open(GOLDEN).read().split("\n")
                     if x.strip() and not x.startswith("#")])


def test_db3_taps_match_published_table():
    h, _ = O.db3_filters()
    np.testing.assert_allclose(h, _golden_taps(), atol=1e-11)


def test_db3_identities():
    h, g = O.db3_filters()
    assert abs(h.sum() - np.sqrt(2)) < 1e-15
    assert abs((h * h).sum() - 1) < 1e-15
    for m in (1, 2):                                   # double-shift orthogonality
        assert abs((h[:-2 * m] * h[2 * m:]).sum()) < 1e-15
    k = np.arange(6)
    for p in range(3):                                 # three vanishing moments of g
        assert abs((g * k ** p).sum()) < 1e-12
    assert abs((g * k ** 3).sum()) > 1e-3              # ... and not four
    assert abs(g @ h) < 1e-15


def test_db3_is_minimum_phase():
    """Daubechies' choice: the non-trivial zeros of H(z) = sum h_k z^-k lie inside |z| = 1."""
    h, _ = O.db3_filters()
    z = np.roots(h)                                    # roots of h0 z^5 + ... + h5
    far = z[np.abs(z + 1) > 1e-3]                      # drop the triple zero at z = -1
    assert len(far) == 2
    assert np.all(np.abs(far) < 1.0)


@pytest.mark.parametrize("n,levels", [(2, 1), (4, 2), (8, 3), (16, 4), (32, 3), (64, 6)])
def test_orthonormal_and_perfect_reconstruction(n, levels):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((n, n))
    c = O.dwt2(x, levels)
    np.testing.assert_allclose(O.idwt2(c, levels), x, atol=1e-12)
    assert abs((c ** 2).sum() - (x ** 2).sum()) < 1e-10 * (x ** 2).sum()
    if n <= 16:
        Wm = np.stack([O.dwt2(e.reshape(n, n), levels).ravel() for e in np.eye(n * n)], 1)
        np.testing.assert_allclose(Wm @ Wm.T, np.eye(n * n), atol=1e-12)


def test_constant_has_only_coarse_coefficient():
    n = 32
    c = O.dwt2(np.full((n, n), 3.0), 5)
    expect = np.zeros((n, n))
    expect[0, 0] = 3.0 * n                              # orthonormal: sum / sqrt(n*n) * ... = 3n
    np.testing.assert_allclose(c, expect, atol=1e-11)


@pytest.mark.parametrize("n", [16, 64, 128])
def test_piston_coefficient_synthesises_to_constant(n):
    """A unit full-depth LL coefficient is the constant 1/n on an n x n layer: the identity
    by which the fit adds a full layer's piston, w c_piston / n, to layers carried without it."""
    levels = int(np.log2(n))
    c = np.zeros((n, n))
    c[0, 0] = 1.0
    np.testing.assert_allclose(O.idwt2(c, levels), np.full((n, n), 1.0 / n), rtol=0, atol=1e-15)


def test_quadratics_have_no_interior_details():
    """Three vanishing moments: level-1 details of x^2 (away from the seam) are 0."""
    n = 32
    x = np.arange(n, dtype=float)
    row = 0.3 * x ** 2 - 2.0 * x + 1.0
    phi = np.tile(row, (n, 1))                          # varies along x only
    c = O.dwt2(phi, 1)
    d = c[: n // 2, n // 2:]                            # x-detail, y-approx block
    interior = d[:, : n // 2 - 3]                       # filters that do not wrap
    assert np.abs(interior).max() < 1e-10
    assert np.abs(d[:, -1]).max() > 1.0                 # the periodic seam does not vanish


def test_basis_functions_are_shifted_copies():
    n = 32
    for j in (1, 2, 3):
        for kind in "ad":
            F = O.basis_1d(n, j, kind)
            np.testing.assert_allclose(F.T @ F, np.eye(F.shape[1]), atol=1e-13)
            for k in range(F.shape[1]):
                np.testing.assert_allclose(F[:, k], np.roll(F[:, 0], k << j), atol=1e-13)


def test_two_d_basis_is_separable():
    n, lev = 16, 3
    lm = O.level_map(n, lev)
    for (r, c) in [(0, 0), (1, 3), (5, 2), (9, 12), (3, 7)]:
        e = np.zeros((n, n))
        e[r, c] = 1.0
        psi = O.idwt2(e, lev)
        j = min(int(lm[r, c]), lev)
        h = n >> j
        ky, kx = ("a" if r < h else "d"), ("a" if c < h else "d")
        fy = O.basis_1d(n, j, ky)[:, r % h]
        fx = O.basis_1d(n, j, kx)[:, c % h]
        np.testing.assert_allclose(psi, np.outer(fy, fx), atol=1e-13)


def test_level_map_counts():
    n, lev = 64, 6
    lm = O.level_map(n, lev)
    for j in range(1, lev + 1):
        assert (lm == j).sum() == 3 * (n >> j) ** 2
    assert (lm == lev + 1).sum() == (n >> lev) ** 2
