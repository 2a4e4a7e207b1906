"""Pins for the oracle's prox: Eq. "proxdef" (Sec. 2.1) with g = ||W.||_1,
W the orthonormal Haar wavelet, and Lemma "fne" (Sec. 2.2)."""
import itertools
import math

import numpy as np
import pytest

import synth
from oracle import pp_oracle as O


def test_soft_threshold_closed_form_cases():
    lam = 0.5
    v = np.array([0.0, 0.5, -0.5, 0.25j, 2.0, -3.0j, 3.0 + 4.0j], dtype=np.complex128)
    ref = np.array([0.0, 0.0, 0.0, 0.0, 1.5, -2.5j, (3.0 + 4.0j) * (1 - 0.5 / 5.0)])
    assert np.max(np.abs(O.soft_threshold(v, lam) - ref)) <= 1e-15
    assert np.array_equal(O.soft_threshold(v, 0.0), v)


@pytest.mark.parametrize("v", [0.3 + 0.1j, -1.2 + 0.7j, 0.05 - 0.02j, 2.0j])
def test_soft_threshold_is_the_scalar_prox_by_brute_force(v):
    # argmin_x 1/2 |x - v|^2 + lam |x| over a fine grid in the complex plane
    lam = 0.4
    g = np.linspace(-2.5, 2.5, 2001)
    X = g[None, :] + 1j * g[:, None]
    obj = 0.5 * np.abs(X - v) ** 2 + lam * np.abs(X)
    best = X.ravel()[np.argmin(obj)]
    assert abs(best - O.soft_threshold(np.array([v]), lam)[0]) <= 2 * (g[1] - g[0])


def _explicit_haar_basis_2level_4x4():
    """The 16 orthonormal 2-level 2-D Haar basis images of a 4x4 tile:
    level 2: approximation (constant 1/4) and three 4x4 details built from
    2x2-block patterns of +-1/4; level 1: in each 2x2 block, the three
    details [[1,1],[-1,-1]]/2, [[1,-1],[1,-1]]/2, [[1,-1],[-1,1]]/2."""
    out = []
    h2 = [np.array([[1, 1], [1, 1]]), np.array([[1, 1], [-1, -1]]),
          np.array([[1, -1], [1, -1]]), np.array([[1, -1], [-1, 1]])]
    for p in h2:
        out.append(np.kron(p, np.ones((2, 2))) / 4.0)
    for by, bx in itertools.product(range(2), range(2)):
        for p in h2[1:]:
            img = np.zeros((4, 4))
            img[2 * by:2 * by + 2, 2 * bx:2 * bx + 2] = p / 2.0
            out.append(img)
    return out


def test_haar_matches_explicit_basis():
    W = np.stack([O.haar_fwd(e.reshape(4, 4), 2).ravel() for e in np.eye(16)], axis=1)
    # orthonormal
    assert np.max(np.abs(W @ W.conj().T - np.eye(16))) <= 1e-15
    # rows of W are the basis images (up to order and sign)
    rows = [r.real.reshape(4, 4) for r in W]
    basis = _explicit_haar_basis_2level_4x4()
    for b in basis:
        assert any(np.max(np.abs(r - b)) < 1e-15 or np.max(np.abs(r + b)) < 1e-15 for r in rows)


@pytest.mark.parametrize("shape", [(8, 8), (16, 12), (8, 4, 12)])
def test_haar_norm_and_inverse(shape):
    x = synth.crandn(shape, 3).astype(np.complex128)
    c = O.haar_fwd(x, 2)
    assert abs(np.linalg.norm(c) - np.linalg.norm(x)) <= 1e-13 * np.linalg.norm(x)
    assert np.max(np.abs(O.haar_inv(c, 2) - x)) <= 1e-14 * np.max(np.abs(x))


@pytest.mark.parametrize("shape", [(8, 12), (4, 8, 8)])
def test_prox_is_tile_local(shape):
    # The 2-level Haar prox acts on independent 4x4 (4x4x4) tiles.
    x = synth.crandn(shape, 4).astype(np.complex128)
    lam = 0.3
    full = O.prox_l1_haar(x, lam, 2)
    tiled = np.empty_like(x)
    for idx in itertools.product(*[range(0, s, 4) for s in shape]):
        sl = tuple(slice(i, i + 4) for i in idx)
        tiled[sl] = O.prox_l1_haar(x[sl], lam, 2)
    assert np.max(np.abs(full - tiled)) <= 1e-14


def test_prox_optimality_conditions():
    # x = prox(v) iff, in the wavelet domain, (Wv - Wx)_i = lam * Wx_i/|Wx_i|
    # where Wx_i != 0 and |(Wv)_i| <= lam where Wx_i = 0.
    v = synth.crandn((16, 16), 9).astype(np.complex128)
    lam = 0.6
    x = O.prox_l1_haar(v, lam, 2)
    wv, wx = O.haar_fwd(v, 2), O.haar_fwd(x, 2)
    nz = np.abs(wx) > 1e-12   # exact zeros come back as rounding-level values
    assert nz.any() and (~nz).any()
    assert np.max(np.abs((wv - wx)[nz] - lam * wx[nz] / np.abs(wx[nz]))) <= 1e-13
    assert np.all(np.abs(wv[~nz]) <= lam + 1e-13)


def test_prox_non_expansive():
    lam = 0.2
    for s in range(10):
        a = synth.crandn((8, 8), 100 + s).astype(np.complex128)
        b = synth.crandn((8, 8), 200 + s).astype(np.complex128)
        lhs = np.linalg.norm(O.prox_l1_haar(a, lam) - O.prox_l1_haar(b, lam))
        assert lhs <= np.linalg.norm(a - b) + 1e-14


# ---- Daubechies-4 (the W of the paper's experiments, Sec. 5.1 / 5.2) ----


def test_db4_filter_defining_properties():
    # orthonormality to even shifts, unit DC gain sqrt 2, and two vanishing
    # moments of the high-pass (it annihilates constants and ramps)
    h, g = O.db4_filters()
    assert abs(np.sum(h) - math.sqrt(2.0)) <= 1e-15
    assert abs(np.sum(h * h) - 1.0) <= 1e-15
    assert abs(h[0] * h[2] + h[1] * h[3]) <= 1e-16
    k = np.arange(4)
    assert abs(np.sum(g)) <= 1e-15
    assert abs(np.sum(k * g)) <= 1e-14
    assert abs(np.sum(k * k * g)) > 1e-3          # exactly two moments vanish
    assert abs(np.sum(g * h)) <= 1e-16 and abs(g[0] * h[2] + g[1] * h[3]) <= 1e-16


def test_db4_one_level_matrix_is_orthogonal():
    n = 8
    M = np.stack([O.dwt1(np.eye(n)[:, j], 0) for j in range(n)], axis=1)
    assert np.max(np.abs(M.T @ M - np.eye(n))) <= 1e-14
    assert np.max(np.abs(M @ M.T - np.eye(n))) <= 1e-14
    # the inverse is the transpose
    Minv = np.stack([O.idwt1(np.eye(n)[:, j], 0) for j in range(n)], axis=1)
    assert np.max(np.abs(Minv - M.T)) <= 1e-14


def test_db4_detail_of_a_ramp_vanishes_away_from_the_wrap():
    n = 32
    x = 0.3 * np.arange(n) - 1.7
    c = O.dwt1(x, 0)
    d = c[n // 2:]
    assert np.max(np.abs(d[: n // 2 - 1])) <= 1e-13     # the last one straddles the wrap
    assert abs(d[-1]) > 1e-3


@pytest.mark.parametrize("shape,levels", [((16, 12), 1), ((16, 16), 2), ((32, 24), 3)])
def test_db4_norm_and_inverse(shape, levels):
    x = synth.crandn(shape, 3).astype(np.complex128)
    c = O.db4_fwd(x, levels)
    assert abs(np.linalg.norm(c) - np.linalg.norm(x)) <= 1e-13 * np.linalg.norm(x)
    assert np.max(np.abs(O.db4_inv(c, levels) - x)) <= 1e-13


def test_db4_differs_from_haar_and_keeps_constants_in_the_coarse_band():
    x = np.full((16, 16), 2.0 + 1.0j)
    c = O.db4_fwd(x, 2)
    mask = np.zeros((16, 16), bool)
    mask[:4, :4] = True
    assert np.max(np.abs(c[~mask])) <= 1e-13
    y = synth.crandn((16, 16), 4).astype(np.complex128)
    assert np.linalg.norm(O.db4_fwd(y, 1) - O.haar_fwd(y, 1)) > 0.1 * np.linalg.norm(y)


def test_db4_prox_optimality_and_non_expansiveness():
    lam = 0.3
    v = synth.crandn((16, 24), 5).astype(np.complex128)
    y = O.prox_l1_db4(v, lam, 2)
    cv, cy = O.db4_fwd(v, 2), O.db4_fwd(y, 2)
    on = np.abs(cy) > 1e-12     # zeros come back from the round trip at the 1e-16 level
    # v - y = lam W^T s with s_i = c_i/|c_i| where c_i != 0, |s_i| <= 1 elsewhere
    assert np.max(np.abs((cv - cy)[on] - lam * cy[on] / np.abs(cy[on]))) <= 1e-12
    assert np.max(np.abs(cv[~on])) <= lam + 1e-12
    w = synth.crandn((16, 24), 6).astype(np.complex128)
    assert np.linalg.norm(O.prox_l1_db4(v, lam, 2) - O.prox_l1_db4(w, lam, 2)) <= np.linalg.norm(v - w) + 1e-12
