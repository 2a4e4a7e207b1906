"""Pins for the oracle's centred orthonormal FFT (Sec. 5.1 operator F)
against a direct DFT written from its definition."""
import math

import numpy as np
import pytest

from oracle import pp_oracle as O


def direct_centred_dft_matrix(n):
    # X[q] = n^-1/2 sum_p x[p] exp(-2 pi i (q - n//2)(p - n//2)/n)
    idx = np.arange(n) - n // 2
    return np.exp(-2j * math.pi * np.outer(idx, idx) / n) / math.sqrt(n)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 8, 9, 10, 12, 15, 16, 20, 25, 27, 32, 40, 45, 60, 64])
def test_cfft_matches_direct_dft_1d(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = direct_centred_dft_matrix(n) @ x
    got = O.cfft(x, axes=(0,))
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
    back = O.cifft(got, axes=(0,))
    assert np.max(np.abs(back - x)) <= 1e-12 * np.max(np.abs(x))


@pytest.mark.parametrize("shape", [(6, 10), (8, 12), (5, 4, 6)])
def test_cfft_matches_direct_dft_nd(shape):
    rng = np.random.default_rng(sum(shape))
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    ref = x
    for ax, n in enumerate(shape):
        ref = np.moveaxis(np.tensordot(direct_centred_dft_matrix(n), np.moveaxis(ref, ax, 0), axes=1), 0, ax)
    got = O.cfft(x, axes=tuple(range(len(shape))))
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    # unitary: Parseval
    assert abs(np.linalg.norm(got) - np.linalg.norm(x)) <= 1e-12 * np.linalg.norm(x)
