"""FP64 CPU oracle for polynomial-preconditioned FISTA on multi-coil SENSE.

TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the benchmark's
CPU-baseline leg may import this module; the product path never does.  It
shares no code with the CUDA library: every function below restates the
paper's definitions in plain, slow numpy (complex128), with numpy's FFT as
the only library primitive.

Problem (Eq. "ucopt", Sec. 1):  min_x 1/2 ||A x - b||_2^2 + lambda ||W x||_1
  A = [M F S_1; ...; M F S_C]      Cartesian SENSE (Sec. 5.1 operator)
  A = [N S_1; ...; N S_C]          non-Cartesian SENSE with a Kaiser-Bessel
                                   gridding NUFFT N (Sec. 5.2 operator)
  A^H A with the exact NDFT F:     sum_c conj(S_c) F^H F S_c, the normal
                                   operator evaluated through the Toeplitz
                                   structure of F^H F (Sec. 2 remark, Sec. 5.2)
  W = orthonormal Haar wavelet (the paper's experiments use Daubechies-4;
      the workload here fixes a 2-level Haar).
Method: Algorithm "pfista" (Sec. 3.1) with p from Eq. "l2cost", evaluated by
the recursion of Listing "pcode" (Sec. 3.6), on the normalised problem of
Sec. 5 (A scaled to unit induced norm, b to unit l2 norm).

Readings where the paper is silent or ambiguous (each is listed in the design
notes of the repository):
  * FFT: orthonormal and centred (ifftshift -> FFT -> fftshift).
  * Momentum: z_{k+1} = y_{k+1} + beta_k (y_{k+1} - y_k), beta_k = k/(k+3)
    (the printed z_{k+1} = y_k + beta_k(y_k - y_{k-1}) is read as an index
    slip).
  * Soft threshold of a complex v: v * max(0, 1 - lambda/|v|), 0 at v = 0;
    every Haar coefficient, the coarsest approximation band included, is
    thresholded.
  * Induced norm: L = lambda_max(A^H A) from 50 power-iteration steps started
    from a SplitMix64 vector; L is the last Rayleigh quotient.
  * NUFFT: grid G = ceil(sigma*n) per axis, KB kernel of width W with
    beta = pi*sqrt((W/sigma)^2 (sigma-1/2)^2 - 0.8) (Beatty et al. 2005),
    taps m in (s - W/2, s + W/2] at grid coordinate s = kappa*G/n, and
    deapodisation by the kernel's continuous Fourier transform.

Parity unpinned: nothing.  Every function here is checked by the CPU tests
against closed forms, brute force or library routines (see tests/).
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

# --------------------------------------------------------------------------
# Fourier transforms (Sec. 5.1: "2D-Fourier transform"; reading: unitary,
# centred)
# --------------------------------------------------------------------------


def cfft(x, axes):
    """Centred orthonormal DFT over `axes`."""
    return np.fft.fftshift(np.fft.fftn(np.fft.ifftshift(x, axes=axes), axes=axes, norm="ortho"),
                           axes=axes)


def cifft(x, axes):
    """Inverse of cfft (its adjoint)."""
    return np.fft.fftshift(np.fft.ifftn(np.fft.ifftshift(x, axes=axes), axes=axes, norm="ortho"),
                           axes=axes)


# --------------------------------------------------------------------------
# Cartesian SENSE (Sec. 5.1): A_c = M F S_c
# --------------------------------------------------------------------------


def _img_axes(x):
    return tuple(range(-x.ndim, 0))


def cart_forward(x, sens, mask):
    """y_c = M * F(S_c * x); x [*img], sens [C, *img], mask [*img] (0/1)."""
    x = np.asarray(x, dtype=np.complex128)
    s = np.asarray(sens, dtype=np.complex128)
    m = np.asarray(mask).astype(np.float64)
    return m[None] * cfft(s * x[None], axes=_img_axes(x))


def cart_adjoint(y, sens, mask):
    """x = sum_c conj(S_c) * F^H(M * y_c)."""
    y = np.asarray(y, dtype=np.complex128)
    s = np.asarray(sens, dtype=np.complex128)
    m = np.asarray(mask).astype(np.float64)
    ax = tuple(range(-(y.ndim - 1), 0))
    return np.sum(np.conj(s) * cifft(m[None] * y, axes=ax), axis=0)


def cart_normal(x, sens, mask):
    """A^H A x with the full multi-dimensional FFT (no readout shortcut)."""
    return cart_adjoint(cart_forward(x, sens, mask), sens, mask)


def cart_normal_columns(x, sens, mask, cols):
    """Readout columns `cols` (indices along the last axis x) of cart_normal
    for a mask constant along x.  Then M commutes with the x transform and
    F^H M F = F_rest^H M F_rest with F_rest the transform over the other
    axes (F_x^H F_x = I), so every x column is its own problem:
    out[..., j] = sum_c conj(S_c[..., x_j]) F_rest^H M[..., x_j] F_rest (S_c x)[..., x_j].
    Returns [*img[:-1], len(cols)]; used to check single columns of large
    volumes without transforming the whole volume."""
    x = np.asarray(x, dtype=np.complex128)
    cols = list(cols)
    ax = tuple(range(-(x.ndim - 1), 0))
    out = np.zeros(x.shape[:-1] + (len(cols),), dtype=np.complex128)
    for j, q in enumerate(cols):
        m = np.asarray(mask)[..., q].astype(np.float64)
        xq = x[..., q]
        for c in range(np.shape(sens)[0]):
            sq = np.asarray(sens[c])[..., q].astype(np.complex128)
            out[..., j] += np.conj(sq) * cifft(m * cfft(sq * xq, axes=ax), axes=ax)
    return out


# --------------------------------------------------------------------------
# Kaiser-Bessel gridding NUFFT (Sec. 5.2 uses a NUFFT; parameters per the
# workload: width W, oversampling sigma)
# --------------------------------------------------------------------------


def kb_beta(width, oversamp):
    """Beatty et al. (2005) shape parameter for width W and oversampling sigma."""
    w, s = float(width), float(oversamp)
    return math.pi * math.sqrt((w / s) ** 2 * (s - 0.5) ** 2 - 0.8)


def bessel_i0(x):
    """Modified Bessel function I0 by its power series sum_k ((x/2)^k / k!)^2."""
    x = np.asarray(x, dtype=np.float64)
    q = (x / 2.0) ** 2
    term = np.ones_like(x)
    total = np.ones_like(x)
    for k in range(1, 80):
        term = term * q / (k * k)
        total = total + term
    return total


def kb_kernel(u, width, beta):
    """phi(u) = I0(beta * sqrt(1 - (2u/W)^2)) for |u| <= W/2, else 0."""
    u = np.asarray(u, dtype=np.float64)
    t = 1.0 - (2.0 * u / width) ** 2
    inside = t >= 0.0
    return np.where(inside, bessel_i0(beta * np.sqrt(np.where(inside, t, 0.0))), 0.0)


def kb_transform(nu, width, beta):
    """Continuous Fourier transform of kb_kernel at frequency nu (cycles per
    grid sample): W sinh(sqrt(a))/sqrt(a), a = beta^2 - (pi W nu)^2 (sin for
    a < 0, W at a = 0)."""
    nu = np.asarray(nu, dtype=np.float64)
    a = beta ** 2 - (math.pi * width * nu) ** 2
    out = np.empty_like(a)
    pos, neg = a > 0, a < 0
    out[pos] = width * np.sinh(np.sqrt(a[pos])) / np.sqrt(a[pos])
    out[neg] = width * np.sin(np.sqrt(-a[neg])) / np.sqrt(-a[neg])
    out[~(pos | neg)] = width
    return out


def _grid_size(n, oversamp):
    return int(math.ceil(oversamp * n))


def _nufft_taps(traj, shape, width, oversamp):
    """Per-sample taps: list over (ty, tx) of (grid row, grid col, weight),
    grid indices centred (index = m + G/2, wrapped mod G)."""
    ny, nx = shape
    gy, gx = _grid_size(ny, oversamp), _grid_size(nx, oversamp)
    beta = kb_beta(width, oversamp)
    t = np.asarray(traj, dtype=np.float64)
    sx = t[:, 0] * (gx / nx)
    sy = t[:, 1] * (gy / ny)
    mx0 = np.floor(sx - width / 2.0).astype(np.int64) + 1
    my0 = np.floor(sy - width / 2.0).astype(np.int64) + 1
    taps = []
    for b in range(width):
        my = my0 + b
        wy = kb_kernel(sy - my, width, beta)
        for a in range(width):
            mx = mx0 + a
            wx = kb_kernel(sx - mx, width, beta)
            taps.append(((my + gy // 2) % gy, (mx + gx // 2) % gx, wy * wx))
    return taps, (gy, gx), beta


def _apodisation(shape, grid, width, beta):
    ny, nx = shape
    gy, gx = grid
    ry = np.arange(ny) - ny // 2
    rx = np.arange(nx) - nx // 2
    return kb_transform(ry / gy, width, beta)[:, None] * kb_transform(rx / gx, width, beta)[None, :]


def nufft_forward(x, traj, width=4, oversamp=1.25):
    """Gridding approximation of y_k = 1/sqrt(n) sum_r x(r) exp(-2 pi i kappa_k.r/n):
    deapodise, zero-pad (centred) to the oversampled grid, centred unnormalised
    DFT, interpolate with the separable KB kernel.  x [ny, nx]; traj [K, 2]."""
    x = np.asarray(x, dtype=np.complex128)
    ny, nx = x.shape
    taps, (gy, gx), beta = _nufft_taps(traj, (ny, nx), width, oversamp)
    apod = _apodisation((ny, nx), (gy, gx), width, beta)
    xp = np.zeros((gy, gx), dtype=np.complex128)
    oy, ox = gy // 2 - ny // 2, gx // 2 - nx // 2
    xp[oy:oy + ny, ox:ox + nx] = x / apod
    X = np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(xp)))
    y = np.zeros(len(traj), dtype=np.complex128)
    for iy, ix, w in taps:
        y += w * X[iy, ix]
    return y / math.sqrt(ny * nx)


def nufft_adjoint(y, traj, shape, width=4, oversamp=1.25):
    """Exact adjoint of nufft_forward: spread, centred inverse DFT (unscaled),
    crop, deapodise."""
    y = np.asarray(y, dtype=np.complex128)
    ny, nx = shape
    taps, (gy, gx), beta = _nufft_taps(traj, (ny, nx), width, oversamp)
    apod = _apodisation((ny, nx), (gy, gx), width, beta)
    Xg = np.zeros((gy, gx), dtype=np.complex128)
    for iy, ix, w in taps:
        np.add.at(Xg, (iy, ix), w * y)
    xp = np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(Xg))) * (gy * gx)
    oy, ox = gy // 2 - ny // 2, gx // 2 - nx // 2
    return xp[oy:oy + ny, ox:ox + nx] / apod / math.sqrt(ny * nx)


def ndft_forward(x, traj):
    """Exact non-uniform DFT y_k = 1/sqrt(n) sum_r x(r) exp(-2 pi i (kx rx/nx + ky ry/ny)),
    r centred.  O(K n); for small pins only."""
    x = np.asarray(x, dtype=np.complex128)
    ny, nx = x.shape
    ry = (np.arange(ny) - ny // 2).astype(np.float64)
    rx = (np.arange(nx) - nx // 2).astype(np.float64)
    t = np.asarray(traj, dtype=np.float64)
    ey = np.exp(-2j * math.pi * np.outer(t[:, 1], ry) / ny)   # [K, ny]
    ex = np.exp(-2j * math.pi * np.outer(t[:, 0], rx) / nx)   # [K, nx]
    return np.einsum("ky,yx,kx->k", ey, x, ex) / math.sqrt(ny * nx)


def ndft_adjoint(y, traj, shape):
    """Exact adjoint of ndft_forward: x(r) = 1/sqrt(n) sum_k y_k exp(+2 pi i (kx rx/nx + ky ry/ny)),
    r centred.  O(K n); for small pins only."""
    y = np.asarray(y, dtype=np.complex128)
    ny, nx = shape
    ry = (np.arange(ny) - ny // 2).astype(np.float64)
    rx = (np.arange(nx) - nx // 2).astype(np.float64)
    t = np.asarray(traj, dtype=np.float64)
    ey = np.exp(2j * math.pi * np.outer(t[:, 1], ry) / ny)    # [K, ny]
    ex = np.exp(2j * math.pi * np.outer(t[:, 0], rx) / nx)    # [K, nx]
    return np.einsum("k,ky,kx->yx", y, ey, ex) / math.sqrt(ny * nx)


def nc_normal_exact(x, sens, traj):
    """A^H A with the exact non-uniform DFT F in place of the gridding NUFFT:
    sum_c conj(S_c) F^H F (S_c x).  This is the operator that the Toeplitz
    structure of F^H F (the remark of Sec. 2 and the spiral experiment of
    Sec. 5.2) evaluates exactly, without gridding.  O(C K n); small sizes."""
    s = np.asarray(sens, dtype=np.complex128)
    x = np.asarray(x, dtype=np.complex128)
    shape = s.shape[1:]
    out = np.zeros(shape, dtype=np.complex128)
    for c in range(s.shape[0]):
        out += np.conj(s[c]) * ndft_adjoint(ndft_forward(s[c] * x, traj), traj, shape)
    return out


def ndft_gram_offsets(traj, shape):
    """Entries of F^H F: (F^H F)[r, r'] = h(r - r') with
    h(dy, dx) = 1/n sum_k exp(2 pi i (kx dx/nx + ky dy/ny)), returned as
    h[dy + ny - 1, dx + nx - 1] for |dy| < ny, |dx| < nx.  The sum over k is
    separable per axis, so it is one matrix product (a library primitive)."""
    ny, nx = shape
    t = np.asarray(traj, dtype=np.float64)
    dy = np.arange(-(ny - 1), ny).astype(np.float64)
    dx = np.arange(-(nx - 1), nx).astype(np.float64)
    ey = np.exp(2j * math.pi * np.outer(t[:, 1], dy) / ny)    # [K, 2ny-1]
    ex = np.exp(2j * math.pi * np.outer(t[:, 0], dx) / nx)    # [K, 2nx-1]
    return (ey.T @ ex) / (ny * nx)


def nc_normal_exact_at(x, sens, traj, pixels, gram=None):
    """Selected outputs of nc_normal_exact, one by one from the entries of
    F^H F: out(r) = sum_c conj(S_c(r)) sum_r' h(r - r') S_c(r') x(r').
    pixels: list of (row, col); returns the values in that order."""
    s = np.asarray(sens, dtype=np.complex128)
    x = np.asarray(x, dtype=np.complex128)
    ny, nx = x.shape
    h = ndft_gram_offsets(traj, (ny, nx)) if gram is None else gram
    sx = s * x[None]
    out = []
    for (r, q) in pixels:
        # h(r - r') for every r': rows r - r' + ny - 1, columns q - q' + nx - 1
        hr = h[r + ny - 1 - np.arange(ny)][:, q + nx - 1 - np.arange(nx)]
        out.append(sum(np.conj(s[c, r, q]) * np.sum(hr * sx[c]) for c in range(s.shape[0])))
    return np.array(out)


def nc_forward(x, sens, traj, width=4, oversamp=1.25):
    """y_c = N(S_c x) for each coil; returns [C, K]."""
    s = np.asarray(sens, dtype=np.complex128)
    x = np.asarray(x, dtype=np.complex128)
    return np.stack([nufft_forward(s[c] * x, traj, width, oversamp) for c in range(s.shape[0])])


def nc_adjoint(y, sens, traj, width=4, oversamp=1.25):
    """x = sum_c conj(S_c) N^H y_c."""
    s = np.asarray(sens, dtype=np.complex128)
    shape = s.shape[1:]
    out = np.zeros(shape, dtype=np.complex128)
    for c in range(s.shape[0]):
        out += np.conj(s[c]) * nufft_adjoint(y[c], traj, shape, width, oversamp)
    return out


def nc_normal(x, sens, traj, width=4, oversamp=1.25):
    return nc_adjoint(nc_forward(x, sens, traj, width, oversamp), sens, traj, width, oversamp)


# --------------------------------------------------------------------------
# Orthonormal Haar wavelet and the l1 prox (Eq. "proxdef", Sec. 2.1)
# --------------------------------------------------------------------------

_R2 = math.sqrt(0.5)


def haar_fwd(x, levels):
    """Separable orthonormal Haar over every axis, `levels` levels, Mallat
    layout (approximation band in the low corner)."""
    out = np.array(x, dtype=np.complex128, copy=True)
    for lev in range(levels):
        region = tuple(slice(0, s >> lev) for s in out.shape)
        sub = out[region]
        for ax in range(out.ndim):
            a = np.take(sub, np.arange(0, sub.shape[ax], 2), axis=ax)
            b = np.take(sub, np.arange(1, sub.shape[ax], 2), axis=ax)
            sub = np.concatenate([(a + b) * _R2, (a - b) * _R2], axis=ax)
        out[region] = sub
    return out


def haar_inv(c, levels):
    """Inverse (transpose) of haar_fwd."""
    out = np.array(c, dtype=np.complex128, copy=True)
    for lev in reversed(range(levels)):
        region = tuple(slice(0, s >> lev) for s in out.shape)
        sub = out[region]
        for ax in reversed(range(out.ndim)):
            h = sub.shape[ax] // 2
            lo = np.take(sub, np.arange(0, h), axis=ax)
            hi = np.take(sub, np.arange(h, 2 * h), axis=ax)
            a = (lo + hi) * _R2
            b = (lo - hi) * _R2
            shp = list(sub.shape)
            res = np.empty(shp, dtype=np.complex128)
            idx_a = [slice(None)] * sub.ndim
            idx_b = [slice(None)] * sub.ndim
            idx_a[ax] = slice(0, None, 2)
            idx_b[ax] = slice(1, None, 2)
            res[tuple(idx_a)] = a
            res[tuple(idx_b)] = b
            sub = res
        out[region] = sub
    return out


def soft_threshold(v, lam):
    """prox of lam*|.| for complex entries: v * max(0, 1 - lam/|v|), 0 at v = 0."""
    v = np.asarray(v, dtype=np.complex128)
    mag = np.abs(v)
    safe = np.where(mag > 0, mag, 1.0)
    scale = np.where(mag > lam, 1.0 - lam / safe, 0.0)
    return v * scale


def prox_l1_haar(v, lam, levels=2):
    """prox_{lam ||W .||_1}(v) = W^T soft_lam(W v) for orthonormal W."""
    return haar_inv(soft_threshold(haar_fwd(v, levels), lam), levels)


# --------------------------------------------------------------------------
# Daubechies-4 wavelet (the W of the experiments, Sec. 5.1 and Sec. 5.2) and
# its l1 prox.  Reading: the four-coefficient orthonormal Daubechies filter
# (two vanishing moments), periodic boundary, Mallat layout, every
# coefficient thresholded.
# --------------------------------------------------------------------------


def db4_filters():
    """Analysis low-pass h[0..3] = ((1+s3), (3+s3), (3-s3), (1-s3)) / (4 sqrt 2),
    s3 = sqrt 3 (Daubechies' four-coefficient solution), and the high-pass
    g[k] = (-1)^k h[3-k]."""
    s3 = math.sqrt(3.0)
    h = np.array([1 + s3, 3 + s3, 3 - s3, 1 - s3]) / (4.0 * math.sqrt(2.0))
    g = np.array([(-1) ** k * h[3 - k] for k in range(4)])
    return h, g


def dwt1(x, axis):
    """One periodic analysis step along `axis` (even length n):
    a[i] = sum_k h[k] x[(2i+k) mod n], d[i] = sum_k g[k] x[(2i+k) mod n],
    returned as [a, d] concatenated along the axis."""
    h, g = db4_filters()
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, 0)
    n = x.shape[0]
    a = np.zeros((n // 2,) + x.shape[1:], dtype=np.complex128)
    d = np.zeros_like(a)
    for i in range(n // 2):
        for k in range(4):
            a[i] += h[k] * x[(2 * i + k) % n]
            d[i] += g[k] * x[(2 * i + k) % n]
    return np.moveaxis(np.concatenate([a, d], axis=0), 0, axis)


def idwt1(c, axis):
    """Transpose of dwt1: x[j] = sum_i h[j - 2i] a[i] + g[j - 2i] d[i] over the
    i with (j - 2i) mod n in 0..3."""
    h, g = db4_filters()
    c = np.moveaxis(np.asarray(c, dtype=np.complex128), axis, 0)
    n = c.shape[0]
    a, d = c[: n // 2], c[n // 2:]
    x = np.zeros_like(c)
    for i in range(n // 2):
        for k in range(4):
            x[(2 * i + k) % n] += h[k] * a[i] + g[k] * d[i]
    return np.moveaxis(x, 0, axis)


def db4_fwd(x, levels):
    """2-D separable Daubechies-4 transform, `levels` levels, Mallat layout:
    at each level rows (x) then columns (y) of the approximation band."""
    out = np.array(x, dtype=np.complex128, copy=True)
    for lev in range(levels):
        h, w = out.shape[0] >> lev, out.shape[1] >> lev
        out[:h, :w] = dwt1(dwt1(out[:h, :w], 1), 0)
    return out


def db4_inv(c, levels):
    """Inverse (transpose) of db4_fwd."""
    out = np.array(c, dtype=np.complex128, copy=True)
    for lev in reversed(range(levels)):
        h, w = out.shape[0] >> lev, out.shape[1] >> lev
        out[:h, :w] = idwt1(idwt1(out[:h, :w], 0), 1)
    return out


def prox_l1_db4(v, lam, levels=2):
    """prox_{lam ||W .||_1}(v) = W^T soft_lam(W v), W the orthonormal 2-D
    Daubechies-4 transform."""
    return db4_inv(soft_threshold(db4_fwd(v, levels), lam), levels)


def wavelet_prox(wavelet):
    """The prox of the chosen sparsifying transform (Eq. "proxdef")."""
    return prox_l1_db4 if wavelet == "db4" else prox_l1_haar


# --------------------------------------------------------------------------
# Locally-low-rank regulariser (the LLR term of the MRF experiment, Sec. 5.3,
# block size 8 x 8 x 8): LLR(x) = sum over blocks of the nuclear norm of the
# block's Casorati matrix (one row per voxel, one column per coefficient
# image).  Its prox is singular-value soft thresholding block by block.
# Reading: non-overlapping blocks tiling the volume after a circular shift
# (the shift lets a caller move the block grid between iterations).
# --------------------------------------------------------------------------


def llr_blocks(x, block, shift=None):
    """Casorati matrices of the blocks: returns [nblocks, block^ndim, T] for
    x of shape [T, *img] (every image axis a multiple of `block`), after
    rolling the image by -shift, and the inverse map.  shift is given in
    (x, y[, z]) order (readout axis first), as in the library's call."""
    x = np.asarray(x, dtype=np.complex128)
    T, img = x.shape[0], x.shape[1:]
    nd = len(img)
    sh = [0] * nd if shift is None else list(reversed([int(v) for v in shift][:nd]))
    xr = np.roll(x, [-v for v in sh], axis=tuple(range(1, nd + 1)))
    nb = [n // block for n in img]
    # [T, nb0, b, nb1, b, ...] -> [nb0, nb1, ..., b, b, ..., T]
    shp = [T]
    for n in nb:
        shp += [n, block]
    y = xr.reshape(shp)
    perm = [1 + 2 * i for i in range(nd)] + [2 + 2 * i for i in range(nd)] + [0]
    M = np.transpose(y, perm).reshape(int(np.prod(nb)), block ** nd, T)

    def back(Mb):
        z = Mb.reshape(nb + [block] * nd + [T])
        z = np.transpose(z, np.argsort(perm)).reshape(x.shape)
        return np.roll(z, sh, axis=tuple(range(1, nd + 1)))
    return M, back


def prox_llr(x, lam, block=8, shift=None):
    """prox_{lam LLR}(x): for every block's Casorati matrix M = U S V^H (SVD),
    U max(S - lam, 0) V^H."""
    M, back = llr_blocks(x, block, shift)
    out = np.empty_like(M)
    for i in range(M.shape[0]):
        U, sv, Vh = np.linalg.svd(M[i], full_matrices=False)
        out[i] = (U * np.maximum(sv - lam, 0.0)) @ Vh
    return back(out)


def llr_norm(x, block=8, shift=None):
    """LLR(x): the sum of the blocks' nuclear norms."""
    M, _ = llr_blocks(x, block, shift)
    return float(sum(np.linalg.svd(m, compute_uv=False).sum() for m in M))


# --------------------------------------------------------------------------
# Polynomial preconditioner: Eq. "l2cost" and the recursion of Listing "pcode"
# --------------------------------------------------------------------------


def poly_coeffs_l2(d):
    """Exact minimiser c[0..d] of int_0^1 (1 - z sum_i c_i z^i)^2 dz.

    Expanding the square, the cost is 1 - 2 sum_i c_i/(i+2)
    + sum_ij c_i c_j/(i+j+3); setting its gradient to zero gives the normal
    equations G c = h with G_ij = 1/(i+j+3) and h_i = 1/(i+2), solved here
    in exact rational arithmetic.  Returns a list of Fractions."""
    n = d + 1
    a = [[Fraction(1, i + j + 3) for j in range(n)] + [Fraction(1, i + 2)] for i in range(n)]
    for col in range(n):
        piv = next(r for r in range(col, n) if a[r][col] != 0)
        a[col], a[piv] = a[piv], a[col]
        for r in range(n):
            if r != col and a[r][col] != 0:
                f = a[r][col] / a[col][col]
                a[r] = [a[r][k] - f * a[col][k] for k in range(n + 1)]
    return [a[i][n] / a[i][i] for i in range(n)]


def poly_coeffs_wl2(d, moments):
    """Minimiser c[0..d] of the weighted cost of Eq. "wl2cost",
    int_0^1 w(z) (1 - z sum_i c_i z^i)^2 dz, from the weight's moments
    m_k = int_0^1 w(z) z^k dz (k = 0..2d+2).  Expanding the square, the
    normal equations are G c = h with G_ij = m_{i+j+2} and h_i = m_{i+1};
    with rational moments (Fractions) they are solved exactly."""
    n = d + 1
    m = list(moments)
    a = [[m[i + j + 2] for j in range(n)] + [m[i + 1]] for i in range(n)]
    for col in range(n):
        piv = max(range(col, n), key=lambda r: abs(a[r][col]))
        a[col], a[piv] = a[piv], a[col]
        for r in range(n):
            if r != col and a[r][col] != 0:
                f = a[r][col] / a[col][col]
                a[r] = [a[r][k] - f * a[col][k] for k in range(n + 1)]
    return [a[i][n] / a[i][i] for i in range(n)]


def poly_eval(c, z):
    """p(z) = sum_i c[i] z^i (coefficient order of Sec. 3.6)."""
    z = np.asarray(z, dtype=np.float64)
    out = np.zeros_like(z)
    for ci in reversed(list(c)):
        out = out * z + float(ci)
    return out


def poly_max_zp(c, samples=200001):
    """max over z in [0, 1] of z p(z) on a dense grid (the Lipschitz constant
    of the preconditioned step on a spectrum in (0, 1])."""
    z = np.linspace(0.0, 1.0, samples)
    return float(np.max(z * poly_eval(c, z)))


def horner_apply(c, normal, g):
    """p(N) g = c0 g + N(c1 g + N(c2 g + ...)) by the recursion of Listing
    "pcode": u = c_d g, then u = c_i g + N u for i = d-1 .. 0."""
    c = [float(ci) for ci in c]
    u = c[-1] * g
    for ci in reversed(c[:-1]):
        u = ci * g + normal(u)
    return u


# --------------------------------------------------------------------------
# Induced-norm estimate (Sec. 5: A normalised to unit induced norm)
# --------------------------------------------------------------------------

_SM_GAMMA = 0x9E3779B97F4A7C15
_SM_M1 = 0xBF58476D1CE4E5B9
_SM_M2 = 0x94D049BB133111EB
_MASK64 = (1 << 64) - 1


def splitmix64(seed, count):
    """SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) as a counter-based
    generator: output i mixes seed + (i+1)*gamma.  Returns uint64 array."""
    out = np.empty(count, dtype=np.uint64)
    for i in range(count):
        z = (int(seed) + (i + 1) * _SM_GAMMA) & _MASK64
        z = ((z ^ (z >> 30)) * _SM_M1) & _MASK64
        z = ((z ^ (z >> 27)) * _SM_M2) & _MASK64
        out[i] = z ^ (z >> 31)
    return out


def start_vector(seed, n):
    """Power-iteration start: entry i = (2u_{2i} - 1) + 1j (2u_{2i+1} - 1),
    u_j = (splitmix64_j >> 11) * 2^-53."""
    r = splitmix64(seed, 2 * n)
    u = (r >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return (2.0 * u[0::2] - 1.0) + 1j * (2.0 * u[1::2] - 1.0)


def power_iteration(normal, shape, seed, iters=50):
    """L = lambda_max(A^H A): v <- N v / ||N v|| from a unit SplitMix64 start;
    L is the Rayleigh quotient Re<v, N v> of the last step."""
    n = int(np.prod(shape))
    v = start_vector(seed, n).reshape(shape)
    v = v / np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = normal(v)
        lam = float(np.real(np.vdot(v, w)))
        v = w / np.linalg.norm(w)
    return lam


def mu_estimate(normal, shape, seed, L, iters=50):
    """Lower end mu of the spectrum of N_hat = A^H A / L for the Chebyshev
    design of Sec. 3.4: when A^H A is injective, power iteration on
    I - N_hat converges to its largest eigenvalue 1 - mu.  Start as
    power_iteration (unit SplitMix64 vector from `seed`); w = v - N_hat v,
    rho = Re<v, w>, v <- w / ||w||; returns mu = 1 - rho of the last step."""
    n = int(np.prod(shape))
    v = start_vector(seed, n).reshape(shape)
    v = v / np.linalg.norm(v)
    rho = 0.0
    for _ in range(iters):
        w = v - normal(v) / L
        rho = float(np.real(np.vdot(v, w)))
        v = w / np.linalg.norm(w)
    return 1.0 - rho


# --------------------------------------------------------------------------
# Algorithm "pfista" (and "fista" with p = 1; "ppgd"/"pgd" with beta = 0)
# --------------------------------------------------------------------------


def pfista(normal, adjoint, b, lam, coeffs, iters, L, levels=2, normalize_b=True,
           momentum=True, history=None, wavelet="haar"):
    """Polynomial-preconditioned FISTA on the normalised problem.

    A_hat = A/sqrt(L), b_hat = b/||b|| (when normalize_b), N_hat = A_hat^H A_hat.
    y_{-1} = y_0 = z_0 = 0; for k = 0..iters-1:
        g       = N_hat z_k - A_hat^H b_hat
        u       = p(N_hat) g            (coeffs None: p = 1)
        y_{k+1} = prox_{lam ||W.||_1}(z_k - u)
        beta_k  = k/(k+3)               (0 when momentum is False: Alg. "ppgd")
        z_{k+1} = y_{k+1} + beta_k (y_{k+1} - y_k)
    Returns y_iters.  `history`, if a list, receives every y_{k+1}.
    wavelet: "haar" (default) or "db4" for W in the prox."""
    b = np.asarray(b, dtype=np.complex128)
    bn = float(np.linalg.norm(b)) if normalize_b else 1.0
    ahb = adjoint(b) / (math.sqrt(L) * bn)

    def nhat(v):
        return normal(v) / L

    y = np.zeros_like(ahb)
    z = np.zeros_like(ahb)
    for k in range(iters):
        g = nhat(z) - ahb
        u = g if coeffs is None else horner_apply(coeffs, nhat, g)
        y_new = wavelet_prox(wavelet)(z - u, lam, levels)
        beta = k / (k + 3.0) if momentum else 0.0
        z = y_new + beta * (y_new - y)
        y = y_new
        if history is not None:
            history.append(y.copy())
    return y


def pfista_prox(normal, adjoint, b, v, sigma, lam, coeffs, iters, L, levels=2, momentum=True,
                history=None, wavelet="haar"):
    """Algorithm "pfista" for min_x 1/2 ||A x - b||^2 + (sigma/2) ||x - v||^2
    + lam ||W x||_1, in the problem's own units (b not normalised).  This is
    prox_{rho f}(v) with sigma = 1/rho for f(x) = 1/2 ||A x - b||^2
    + lam ||W x||_1, the subproblem of consensus ADMM (Algorithm "cadmm",
    Sec. 5.3).  The smooth part's Hessian is N' = A^H A + sigma I with
    Lipschitz constant L' = L + sigma; the iteration of Algorithm "pfista"
    runs with step 1/L' on N_hat' = N'/L', the gradient's constant term
    (A^H b + sigma v)/L' and the threshold lam/L'.  b or v may be None (0)."""
    Lp = L + sigma
    shape = None
    rhs = 0.0
    if b is not None:
        rhs = adjoint(np.asarray(b, dtype=np.complex128))
        shape = rhs.shape
    if v is not None:
        rhs = rhs + sigma * np.asarray(v, dtype=np.complex128)
        shape = np.shape(v)
    rhs = np.broadcast_to(np.asarray(rhs, dtype=np.complex128), shape) / Lp

    def nhat(x):
        return (normal(x) + sigma * x) / Lp

    y = np.zeros(shape, dtype=np.complex128)
    z = np.zeros(shape, dtype=np.complex128)
    for k in range(iters):
        g = nhat(z) - rhs
        u = g if coeffs is None else horner_apply(coeffs, nhat, g)
        y_new = wavelet_prox(wavelet)(z - u, lam / Lp, levels)
        beta = k / (k + 3.0) if momentum else 0.0
        z = y_new + beta * (y_new - y)
        y = y_new
        if history is not None:
            history.append(y.copy())
    return y


def consensus_admm(prox_list, shape, iters, history=None):
    """Global consensus ADMM (Algorithm "cadmm", Sec. 5.3) for
    min_x sum_i f_i(x): prox_list[i](v) returns prox_{rho f_i}(v).
    x_bar = x^i = u^i = 0; for k = 0..iters-1:
        x^i     = prox_{rho f_i}(x_bar - u^i)
        x_bar   = (1/N) sum_i x^i
        u^i     = u^i + x^i - x_bar        (reading of the update's stray
                                            superscript on x_bar)
    Returns x_bar; `history`, if a list, receives every x_bar."""
    n = len(prox_list)
    xbar = np.zeros(shape, dtype=np.complex128)
    u = [np.zeros(shape, dtype=np.complex128) for _ in range(n)]
    for _ in range(iters):
        xs = [prox_list[i](xbar - u[i]) for i in range(n)]
        xbar = sum(xs) / n
        for i in range(n):
            u[i] = u[i] + xs[i] - xbar
        if history is not None:
            history.append(xbar.copy())
    return xbar


# --------------------------------------------------------------------------
# Differentiable unrolled solve: Algorithm "pfista" run for a fixed number of
# iterations with b NOT normalised (L fixed), and its reverse-mode gradient.
# --------------------------------------------------------------------------


def pfista_unrolled(normal, adjoint, b, lam, coeffs, iters, L, levels=2, tape=None):
    """y_K of Algorithm "pfista" with A_hat = A/sqrt(L) and raw b:
    A_hat^H b = A^H b / sqrt(L).  `tape`, if a dict, receives z_k, g_k, w_k
    for every iteration (what the reverse pass needs)."""
    ahb = adjoint(np.asarray(b, dtype=np.complex128)) / math.sqrt(L)

    def nhat(v):
        return normal(v) / L

    y = np.zeros_like(ahb)
    z = np.zeros_like(ahb)
    if tape is not None:
        tape.update(z=[], g=[], w=[], ahb=ahb)
    for k in range(iters):
        g = nhat(z) - ahb
        u = horner_apply(coeffs, nhat, g)
        w = z - u
        y_new = prox_l1_haar(w, lam, levels)
        beta = k / (k + 3.0)
        if tape is not None:
            tape["z"].append(z)
            tape["g"].append(g)
            tape["w"].append(w)
        z = y_new + beta * (y_new - y)
        y = y_new
    return y


def soft_threshold_vjp(v, lam, gbar):
    """For s(v) = v max(0, 1 - lam/|v|) (a real-linear map on (Re, Im)):
    returns (J^T gbar, d/dlam of Re<gbar, s(v)>).  Where |v| > lam,
    J dv = (1 - lam/|v|) dv + (lam/|v|) vhat Re(conj(vhat) dv), vhat = v/|v|
    (symmetric), and ds/dlam = -vhat; elsewhere J = 0 and ds/dlam = 0."""
    v = np.asarray(v, dtype=np.complex128)
    mag = np.abs(v)
    on = mag > lam
    safe = np.where(on, mag, 1.0)
    vh = np.where(on, v / safe, 0.0)
    jt = np.where(on, (1.0 - lam / safe) * gbar + (lam / safe) * vh * np.real(np.conj(vh) * gbar), 0.0)
    dlam = float(np.sum(np.real(np.conj(gbar) * (-vh))))
    return jt, dlam


def pfista_unrolled_vjp(normal, adjoint, forward, b, lam, coeffs, iters, L, ybar, levels=2):
    """Gradient of the real loss Re<ybar, y_K> of pfista_unrolled with respect
    to b (as dLoss/dRe b + i dLoss/dIm b), lam and every coefficient c_i.
    Reverse pass of the iteration, step by step:
      z_{k+1} = (1+beta_k) y_{k+1} - beta_k y_k
      y_{k+1} = W^T s_lam(W w_k)
      w_k     = z_k - sum_i c_i N^i g_k,   g_k = N z_k - A_hat^H b
    with N = N_hat self-adjoint.  Returns (b_bar, lam_bar, c_bar)."""
    tape = {}
    pfista_unrolled(normal, adjoint, b, lam, coeffs, iters, L, levels, tape)
    c = [float(ci) for ci in coeffs]
    d = len(c) - 1

    def nhat(v):
        return normal(v) / L

    ybar_next = np.asarray(ybar, dtype=np.complex128).copy()   # adjoint of y_{k+1}
    zbar_next = np.zeros_like(ybar_next)                        # adjoint of z_{k+1}
    ybar_cur = np.zeros_like(ybar_next)                         # adjoint of y_k (partial)
    ahb_bar = np.zeros_like(ybar_next)
    c_bar = np.zeros(d + 1)
    lam_bar = 0.0
    for k in reversed(range(iters)):
        beta = k / (k + 3.0)
        ybar_next = ybar_next + (1.0 + beta) * zbar_next
        ybar_cur = -beta * zbar_next
        wc = haar_fwd(tape["w"][k], levels)
        jt, dl = soft_threshold_vjp(wc, lam, haar_fwd(ybar_next, levels))
        lam_bar += dl
        wbar = haar_inv(jt, levels)
        # v_j = N^j wbar, j = 0..d+1
        vs = [wbar]
        for _ in range(d + 1):
            vs.append(nhat(vs[-1]))
        g = tape["g"][k]
        for i in range(d + 1):
            c_bar[i] -= float(np.real(np.vdot(vs[i], g)))
        zbar = wbar - sum(c[i] * vs[i + 1] for i in range(d + 1))
        ahb_bar += sum(c[i] * vs[i] for i in range(d + 1))
        # step back
        zbar_next = zbar
        ybar_next = ybar_cur
    b_bar = forward(ahb_bar) / math.sqrt(L)
    return b_bar, lam_bar, c_bar


def poly_coeffs_cheb(d, mu):
    """Chebyshev minimax preconditioner of Sec. 3.4 (Eq. "linfcost"):
    r(z) = T_{d+1}((1 + mu - 2z)/(1 - mu)) / T_{d+1}((1 + mu)/(1 - mu)),
    p(z) = (1 - r(z))/z, built with numpy's Chebyshev series mapped from
    [mu, 1] onto [1, -1] and converted to the monomial basis."""
    T = np.polynomial.Chebyshev.basis(d + 1, domain=[mu, 1.0], window=[1.0, -1.0])
    r = T.convert(kind=np.polynomial.Polynomial).coef
    r = r / r[0]
    return [-float(v) for v in r[1:]]
