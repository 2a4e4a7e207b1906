"""Pins for the oracle's SENSE operators (Sec. 5.1, 5.2): adjoint identity,
unitary limits, the exact NDFT, the Kaiser-Bessel pieces, and the readout
shortcut the CUDA path takes."""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.special

import synth
from oracle import pp_oracle as O


def _rel(a, b):
    return abs(a - b) / max(abs(a), abs(b))


@pytest.mark.parametrize("shape,coils", [((12, 10), 3), ((16, 16), 4), ((6, 8, 10), 2)])
def test_cartesian_adjoint_identity(shape, coils):
    x = synth.crandn(shape, 1).astype(np.complex128)
    y = synth.crandn((coils,) + shape, 2).astype(np.complex128)
    s = synth.coil_maps(shape, coils, 3)
    m = synth.line_mask(shape, 2, 4, 4)
    lhs = np.vdot(O.cart_forward(x, s, m), y)
    rhs = np.vdot(x, O.cart_adjoint(y, s, m))
    assert _rel(lhs, rhs) <= 1e-12


def test_cartesian_full_sampling_is_isometry():
    # sum_c |S_c|^2 = 1 and M = 1 => A^H A = I (up to the float32 rounding of S)
    shape = (16, 12)
    s = synth.coil_maps(shape, 4, 0).astype(np.complex128)
    s /= np.sqrt(np.sum(np.abs(s) ** 2, axis=0))
    x = synth.crandn(shape, 5).astype(np.complex128)
    nx = O.cart_normal(x, s, np.ones(shape))
    assert np.linalg.norm(nx - x) <= 1e-13 * np.linalg.norm(x)


def test_readout_shortcut_equals_full_fft():
    # M constant along x => F_x^H (F_y^H M F_y) F_x = F_y^H M F_y: the 1-D
    # (ky only, uncentred, mask moved to FFT order) normal operator equals the
    # oracle's full 2-D centred one.
    ny, nx, C = 16, 12, 3
    s = synth.coil_maps((ny, nx), C, 1).astype(np.complex128)
    m = synth.line_mask((ny, nx), 2, 4, 2)
    x = synth.crandn((ny, nx), 3).astype(np.complex128)
    mfo = np.fft.ifftshift(m[:, 0].astype(np.float64))
    out = np.zeros_like(x)
    for c in range(C):
        k = np.fft.fft(s[c] * x, axis=0, norm="ortho")
        out += np.conj(s[c]) * np.fft.ifft(mfo[:, None] * k, axis=0, norm="ortho")
    ref = O.cart_normal(x, s, m)
    assert np.linalg.norm(out - ref) <= 1e-14 * np.linalg.norm(ref)


@pytest.mark.parametrize("shape,mk", [((12, 16, 10), "poisson"), ((16, 12), "lines")])
def test_normal_columns_equal_full_fft(shape, mk):
    # columns of the readout-shortcut normal operator equal the same columns
    # of the full-FFT definition when the mask is constant along x
    C = 3
    s = synth.coil_maps(shape, C, 4).astype(np.complex128)
    m = (synth.poisson_disc_mask(shape, 2, 4, 5) if mk == "poisson" else
         synth.line_mask(shape, 2, 4, 5))
    x = synth.crandn(shape, 6).astype(np.complex128)
    ref = O.cart_normal(x, s, m)
    cols = [0, 3, shape[-1] - 1]
    got = O.cart_normal_columns(x, s, m, cols)
    assert np.linalg.norm(got - ref[..., cols]) <= 1e-14 * np.linalg.norm(ref[..., cols])
    # a mask that varies along x breaks the identity (the pin is not vacuous)
    m2 = m.copy()
    m2[..., 1::2] = 1 - m2[..., 1::2]
    bad = O.cart_normal_columns(x, s, m2, cols)
    assert np.linalg.norm(bad - O.cart_normal(x, s, m2)[..., cols]) > 1e-3 * np.linalg.norm(bad)


def test_bessel_i0_matches_scipy():
    x = np.linspace(0.0, 12.0, 97)
    got = O.bessel_i0(x)
    ref = scipy.special.i0(x)
    assert np.max(np.abs(got - ref) / ref) <= 1e-14


def test_kb_beta_value():
    # Beatty et al. formula at W = 4, sigma = 1.25
    assert abs(O.kb_beta(4, 1.25) - 6.996659) < 1e-5


@pytest.mark.parametrize("nu", [0.0, 0.1, 0.25, 0.4, 0.6])
def test_kb_transform_matches_quadrature(nu):
    W, beta = 4.0, O.kb_beta(4, 1.25)
    f = lambda u: float(O.kb_kernel(np.array([u]), W, beta)[0]) * math.cos(2 * math.pi * u * nu)
    ref, _ = scipy.integrate.quad(f, -W / 2, W / 2, epsabs=1e-13, epsrel=1e-13, limit=200)
    got = float(O.kb_transform(np.array([nu]), W, beta)[0])
    assert abs(got - ref) <= 1e-9 * abs(ref)


def test_nufft_adjoint_identity():
    shape = (24, 20)
    traj = synth.spiral_traj(4, 200, 2.0, 10.0)
    x = synth.crandn(shape, 1).astype(np.complex128)
    y = synth.crandn((len(traj),), 2).astype(np.complex128)
    lhs = np.vdot(O.nufft_forward(x, traj), y)
    rhs = np.vdot(x, O.nufft_adjoint(y, traj, shape))
    assert _rel(lhs, rhs) <= 1e-12
    s = synth.coil_maps(shape, 3, 4)
    yc = synth.crandn((3, len(traj)), 5).astype(np.complex128)
    lhs = np.vdot(O.nc_forward(x, s, traj), yc)
    rhs = np.vdot(x, O.nc_adjoint(yc, s, traj))
    assert _rel(lhs, rhs) <= 1e-12


def test_nufft_approximates_exact_ndft():
    # W = 4, sigma = 1.25 gridding: approximation error at the 1e-3 level for
    # smooth images, below 1e-2 for white noise.
    shape = (32, 32)
    traj = synth.spiral_traj(8, 512, 3.0, 16.0)
    for img, tol in ((synth.phantom(shape, 1), 5e-3), (synth.crandn(shape, 2), 1.5e-2)):
        img = img.astype(np.complex128)
        ref = O.ndft_forward(img, traj)
        got = O.nufft_forward(img, traj)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= tol


def test_nufft_on_grid_points_matches_cartesian():
    # kappa on the integer grid: the exact NDFT is the centred orthonormal DFT.
    n = 16
    ky, kx = np.meshgrid(np.arange(n) - n // 2, np.arange(n) - n // 2, indexing="ij")
    traj = np.stack([kx.ravel(), ky.ravel()], axis=1).astype(np.float32)
    x = synth.crandn((n, n), 7).astype(np.complex128)
    ref = O.cfft(x, axes=(0, 1)).ravel()
    assert np.linalg.norm(O.ndft_forward(x, traj) - ref) <= 1e-12 * np.linalg.norm(ref)


# ---- exact NDFT normal operator (evaluated on the GPU through the Toeplitz
# structure of F^H F: remark of Sec. 2, spiral experiment of Sec. 5.2) ----


def test_ndft_adjoint_identity():
    shape = (12, 10)
    traj = synth.spiral_traj(3, 40, 2.0, 5.0)
    x = synth.crandn(shape, 1).astype(np.complex128)
    y = synth.crandn((len(traj),), 2).astype(np.complex128)
    lhs = np.vdot(O.ndft_forward(x, traj), y)
    rhs = np.vdot(x, O.ndft_adjoint(y, traj, shape))
    assert _rel(lhs, rhs) <= 1e-12


def test_ndft_adjoint_on_grid_points_is_centred_inverse_dft():
    ny, nx = 8, 12
    ky, kx = np.meshgrid(np.arange(ny) - ny // 2, np.arange(nx) - nx // 2, indexing="ij")
    traj = np.stack([kx.ravel(), ky.ravel()], axis=1).astype(np.float32)
    Y = synth.crandn((ny, nx), 3).astype(np.complex128)
    ref = O.cifft(Y, axes=(0, 1))
    got = O.ndft_adjoint(Y.ravel(), traj, (ny, nx))
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_exact_normal_full_grid_is_identity():
    # every grid point sampled once and sum_c |S_c|^2 = 1  =>  A^H A = I
    ny, nx = 8, 10
    ky, kx = np.meshgrid(np.arange(ny) - ny // 2, np.arange(nx) - nx // 2, indexing="ij")
    traj = np.stack([kx.ravel(), ky.ravel()], axis=1).astype(np.float32)
    s = synth.coil_maps((ny, nx), 3, 0).astype(np.complex128)
    s /= np.sqrt(np.sum(np.abs(s) ** 2, axis=0))
    x = synth.crandn((ny, nx), 5).astype(np.complex128)
    got = O.nc_normal_exact(x, s, traj)
    assert np.linalg.norm(got - x) <= 1e-12 * np.linalg.norm(x)


def test_exact_normal_is_hermitian_and_close_to_gridding():
    shape = (24, 20)
    traj = synth.spiral_traj(4, 300, 3.0, 10.0)
    s = synth.coil_maps(shape, 3, 4)
    x = synth.phantom(shape, 1).astype(np.complex128)
    y = synth.crandn(shape, 6).astype(np.complex128)
    assert _rel(np.vdot(O.nc_normal_exact(x, s, traj), y), np.vdot(x, O.nc_normal_exact(y, s, traj))) <= 1e-12
    exact = O.nc_normal_exact(x, s, traj)
    grid = O.nc_normal(x, s, traj)
    # the W = 4, sigma = 1.25 gridding operator approximates it at the 1e-3 level
    assert np.linalg.norm(grid - exact) <= 1e-2 * np.linalg.norm(exact)


def test_gram_offsets_are_the_columns_of_the_brute_force_matrix():
    shape = (6, 8)
    ny, nx = shape
    traj = synth.spiral_traj(2, 15, 1.5, 3.0)
    h = O.ndft_gram_offsets(traj, shape)
    assert h.shape == (2 * ny - 1, 2 * nx - 1)
    # h(0) = K / n; h(-d) = conj(h(d))
    assert abs(h[ny - 1, nx - 1] - len(traj) / (ny * nx)) <= 1e-14
    assert np.max(np.abs(h[::-1, ::-1] - np.conj(h))) <= 1e-14
    for (r0, q0) in [(0, 0), (2, 5), (5, 7), (3, 0)]:
        e = np.zeros(shape, dtype=np.complex128)
        e[r0, q0] = 1.0
        col = O.ndft_adjoint(O.ndft_forward(e, traj), traj, shape)   # column r' = (r0, q0)
        for r in range(ny):
            for q in range(nx):
                assert abs(col[r, q] - h[r - r0 + ny - 1, q - q0 + nx - 1]) <= 1e-14


def test_sampled_exact_normal_matches_full():
    shape = (10, 12)
    traj = synth.spiral_traj(3, 60, 2.0, 5.0)
    s = synth.coil_maps(shape, 2, 1)
    x = synth.crandn(shape, 2).astype(np.complex128)
    full = O.nc_normal_exact(x, s, traj)
    pix = [(0, 0), (9, 11), (4, 7), (5, 0)]
    got = O.nc_normal_exact_at(x, s, traj, pix)
    ref = np.array([full[r, q] for r, q in pix])
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(full))
