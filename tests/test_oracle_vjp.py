"""Pins for the oracle's reverse-mode gradient of the unrolled preconditioned
FISTA solve: FP64 central finite differences (h = 1e-6) on a tiny Cartesian
SENSE problem, for b (real and imaginary directions), lambda and every
polynomial coefficient."""
import numpy as np
import pytest

import synth
from oracle import pp_oracle as O


def tiny():
    shape, C = (8, 8), 2
    s = synth.coil_maps(shape, C, 3)
    m = synth.line_mask(shape, 2, 2, 3)
    nrm = lambda v: O.cart_normal(v, s, m)
    adj = lambda y: O.cart_adjoint(y, s, m)
    fwd = lambda x: O.cart_forward(x, s, m)
    x0 = synth.phantom(shape, 2).astype(np.complex128)
    b = fwd(x0) + 0.01 * synth.crandn((C,) + shape, 4) * m[None]
    L = O.power_iteration(nrm, shape, 1, iters=60)
    ybar = synth.crandn(shape, 5).astype(np.complex128)
    return nrm, adj, fwd, b, L, ybar, m


@pytest.mark.parametrize("d", [0, 1, 3])
def test_vjp_matches_central_differences(d):
    nrm, adj, fwd, b, L, ybar, m = tiny()
    lam, iters, h = 0.02, 6, 1e-6
    c = [float(v) for v in O.poly_coeffs_l2(d)]

    def loss(bb, ll, cc):
        y = O.pfista_unrolled(nrm, adj, bb, ll, cc, iters, L)
        return float(np.real(np.vdot(ybar, y)))

    b_bar, lam_bar, c_bar = O.pfista_unrolled_vjp(nrm, adj, fwd, b, lam, c, iters, L, ybar)
    # lambda
    fd = (loss(b, lam + h, c) - loss(b, lam - h, c)) / (2 * h)
    assert abs(fd - lam_bar) <= 1e-6 * max(1.0, abs(fd))
    # coefficients
    for i in range(d + 1):
        cp, cm = list(c), list(c)
        cp[i] += h
        cm[i] -= h
        fd = (loss(b, lam, cp) - loss(b, lam, cm)) / (2 * h)
        assert abs(fd - c_bar[i]) <= 1e-6 * max(1.0, abs(fd))
    # b along random real and imaginary directions (sampled entries)
    rng = np.random.default_rng(d)
    for _ in range(3):
        dirn = (rng.standard_normal(b.shape) + 1j * rng.standard_normal(b.shape)) * m[None]
        fd = (loss(b + h * dirn, lam, c) - loss(b - h * dirn, lam, c)) / (2 * h)
        an = float(np.real(np.vdot(b_bar, dirn)))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd))


def test_soft_threshold_vjp_is_the_jacobian_transpose():
    rng = np.random.default_rng(1)
    v = rng.standard_normal(50) + 1j * rng.standard_normal(50)
    g = rng.standard_normal(50) + 1j * rng.standard_normal(50)
    lam, h = 0.7, 1e-7
    jt, dl = O.soft_threshold_vjp(v, lam, g)
    for dv in (1.0, 1j):
        fd = (O.soft_threshold(v + h * dv, lam) - O.soft_threshold(v - h * dv, lam)) / (2 * h)
        # <g, J dv> (real) equals Re(conj(J^T g) dv) per entry
        assert np.allclose(np.real(np.conj(g) * fd), np.real(np.conj(jt) * dv), atol=1e-6)
    fd = np.sum(np.real(np.conj(g) * (O.soft_threshold(v, lam + h) - O.soft_threshold(v, lam - h)) / (2 * h)))
    assert abs(fd - dl) <= 1e-6 * max(1.0, abs(fd))
