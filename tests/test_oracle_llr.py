"""Pins for the oracle's locally-low-rank prox (the LLR regulariser of the MRF
experiment, Sec. 5.3): the block Casorati mapping, closed forms (one
coefficient image: group soft thresholding; a rank-one block), the
subgradient optimality conditions of the nuclear norm, unitary invariance
and non-expansiveness."""
import numpy as np
import pytest

import synth
from oracle import pp_oracle as O


def _x(shape, T, seed):
    return np.stack([synth.crandn(shape, seed + t).astype(np.complex128) for t in range(T)])


@pytest.mark.parametrize("shape,block", [((16, 8, 24), 8), ((8, 12), 4)])
def test_blocks_are_disjoint_tiles_and_the_map_inverts(shape, block):
    x = _x(shape, 3, 1)
    for shift in (None, (3, 5, 1)):
        M, back = O.llr_blocks(x, block, shift)
        assert M.shape == (int(np.prod(shape)) // block ** len(shape), block ** len(shape), 3)
        assert np.array_equal(back(M), x)
        # every voxel appears once: the Frobenius norms agree
        assert np.isclose(np.linalg.norm(M), np.linalg.norm(x))
    # the first block holds exactly the corner sub-volume, row = voxel, column = image
    M, _ = O.llr_blocks(x, block)
    corner = x[(slice(None),) + (slice(0, block),) * len(shape)]
    assert np.array_equal(np.sort_complex(M[0].ravel()), np.sort_complex(corner.ravel()))
    # a shift (x, y[, z]) moves the grid: the first block starts at voxel (.., sy, sx)
    sh = (1, 2, 3)[:len(shape)]
    M, _ = O.llr_blocks(x, block, sh)
    start = tuple(reversed(sh))
    idx = [(np.arange(block) + s0) % n for s0, n in zip(start, shape)]   # wraps circularly
    corner = x[np.ix_(range(3), *idx)]
    assert np.array_equal(np.sort_complex(M[0].ravel()), np.sort_complex(corner.ravel()))


def test_single_image_is_group_soft_thresholding():
    # T = 1: the nuclear norm of a column is its l2 norm, so each block is
    # scaled by max(0, 1 - lam / ||block||)
    shape, b = (16, 16, 8), 8
    x = _x(shape, 1, 3)
    lam = 0.8 * np.sqrt(b ** 3) * 0.7
    got = O.prox_llr(x, lam, b)
    for i in range(0, 16, b):
        for j in range(0, 16, b):
            sl = (slice(None), slice(i, i + b), slice(j, j + b), slice(0, 8))
            nrm = np.linalg.norm(x[sl])
            want = x[sl] * max(0.0, 1.0 - lam / nrm)
            assert np.allclose(got[sl], want, rtol=0, atol=1e-13)


def test_rank_one_block_closed_form():
    # M = s u v^H: the prox is max(s - lam, 0) u v^H
    rng = np.random.default_rng(4)
    u = rng.standard_normal(64) + 1j * rng.standard_normal(64)
    v = rng.standard_normal(4) + 1j * rng.standard_normal(4)
    u /= np.linalg.norm(u)
    v /= np.linalg.norm(v)
    s = 3.0
    M = s * np.outer(u, v.conj())                     # [64 voxels, 4 images]
    x = M.T.reshape(4, 8, 8)                          # one 8x8 block, 4 images
    for lam, keep in ((1.25, 1.75), (3.5, 0.0)):
        got = O.prox_llr(x, lam, 8)
        want = (keep * np.outer(u, v.conj())).T.reshape(4, 8, 8)
        assert np.allclose(got, want, rtol=0, atol=1e-13)


def test_optimality_conditions_of_the_nuclear_norm():
    # Y = prox(X) iff (X - Y)/lam is a subgradient of ||.||_* at Y:
    # (X - Y)/lam = U_r V_r^H + W, ||W|| <= 1, U_r^H W = 0, W V_r = 0
    shape, b, T = (8, 8, 16), 8, 5
    x = _x(shape, T, 7)
    lam = 22.6   # between the blocks' singular values (about 20 to 25 here)
    y = O.prox_llr(x, lam, b)
    MX, _ = O.llr_blocks(x, b)
    MY, _ = O.llr_blocks(y, b)
    ranks = []
    for mx, my in zip(MX, MY):
        G = (mx - my) / lam
        U, sv, Vh = np.linalg.svd(my, full_matrices=False)
        r = int(np.sum(sv > 1e-10 * max(sv.max(), 1e-300)))
        ranks.append(r)
        Ur, Vr = U[:, :r], Vh[:r].conj().T
        W = G - Ur @ Vr.conj().T
        assert np.linalg.norm(W, 2) <= 1 + 1e-10
        assert np.linalg.norm(Ur.conj().T @ W) <= 1e-10
        assert np.linalg.norm(W @ Vr) <= 1e-10
    assert 0 < min(ranks) and max(ranks) < T      # thresholding is active, not vacuous


def test_unitary_invariance_and_nonexpansiveness():
    shape, b, T = (8, 16, 8), 8, 4
    x = _x(shape, T, 9)
    z = _x(shape, T, 19)
    lam = 4.0
    rng = np.random.default_rng(2)
    Q, _ = np.linalg.qr(rng.standard_normal((T, T)) + 1j * rng.standard_normal((T, T)))
    xq = np.einsum("ts,s...->t...", Q.T, x)          # every voxel's T-vector times Q
    assert np.allclose(O.prox_llr(xq, lam, b), np.einsum("ts,s...->t...", Q.T, O.prox_llr(x, lam, b)),
                       atol=1e-12)
    px, pz = O.prox_llr(x, lam, b), O.prox_llr(z, lam, b)
    assert np.linalg.norm(px - pz) <= np.linalg.norm(x - z) * (1 + 1e-12)
    assert np.allclose(O.prox_llr(x, 0.0, b), x, atol=1e-12)
    assert np.all(O.prox_llr(x, 1e6, b) == 0)
    # the prox minimises lam LLR(y) + 1/2 ||y - x||^2: random perturbations do not beat it
    f = lambda y: lam * O.llr_norm(y, b) + 0.5 * np.linalg.norm(y - x) ** 2
    f0 = f(px)
    for s in range(5):
        d = _x(shape, T, 100 + s) * 1e-3
        assert f(px + d) >= f0 - 1e-9
