"""Seeded synthetic inputs for multi-coil SENSE reconstruction problems.

This module draws images, coil sensitivity maps, sampling patterns and noise.
It holds none of the reconstruction arithmetic (no FFT, no gridding, no
operator, no prox): the CUDA library and the CPU oracle both consume what it
returns, so both sides see bit-identical inputs.

The paper reconstructs measured knee, spiral-brain and MRF data (Sec. 5); those
datasets are not available, so these generators stand in for them with the
same shapes and structure: smooth multi-coil maps normalised so that
sum_c |S_c|^2 = 1, line masks that are constant along the readout axis,
variable-density Poisson-disc (ky, kz) masks and Archimedean spirals.

Array conventions (C order, readout axis x fastest):
  image  [ny, nx]          or [nz, ny, nx]           complex64
  sens   [C, ny, nx]       or [C, nz, ny, nx]        complex64
  mask   [ny, nx] uint8    or [nz, ny, nx] uint8     (centred k-space order)
  traj   [K, 2] float32    (kx, ky) in cycles/FOV, inside [-n/2, n/2)
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "crandn", "phantom", "coil_maps", "line_mask", "poisson_disc_mask",
    "spiral_traj", "cnoise", "batched_slices", "CONFIGS",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(int(seed))


def crandn(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Complex Gaussian array (Re, Im each N(0, scale^2/2)), complex64."""
    g = _rng(seed)
    s = scale / math.sqrt(2.0)
    out = g.standard_normal(shape) * s + 1j * (g.standard_normal(shape) * s)
    return out.astype(np.complex64)


def _norm_coords(shape):
    """Per-axis normalised coordinates (i - n/2)/n in [-1/2, 1/2), returned
    in array-axis order (z, y, x) or (y, x)."""
    axes = [(np.arange(n) - n // 2) / float(n) for n in shape]
    return np.meshgrid(*axes, indexing="ij")


def phantom(shape, seed: int, n_ellipses: int = 12) -> np.ndarray:
    """Sum of random ellipses (ellipsoids in 3-D) times a smooth phase.

    Centres lie in the inner 80 % of the field of view, semi-axes are
    U[0.05, 0.4] FOV, the in-plane rotation is U[0, pi) and amplitudes are
    U[0.1, 1].  The magnitude image is multiplied by
    exp(i*pi*(0.3*u_x + 0.2*u_y)) with u = 2*(i - n/2)/n in [-1, 1).
    """
    g = _rng(seed)
    shape = tuple(int(s) for s in shape)
    coords = _norm_coords(shape)
    if len(shape) == 2:
        y, x = coords
        z = None
    else:
        z, y, x = coords
    img = np.zeros(shape, dtype=np.float64)
    for _ in range(n_ellipses):
        cx, cy = g.uniform(-0.4, 0.4, size=2)
        ax, ay = g.uniform(0.05, 0.4, size=2)
        th = g.uniform(0.0, math.pi)
        amp = g.uniform(0.1, 1.0)
        xr = (x - cx) * math.cos(th) + (y - cy) * math.sin(th)
        yr = -(x - cx) * math.sin(th) + (y - cy) * math.cos(th)
        q = (xr / ax) ** 2 + (yr / ay) ** 2
        if z is not None:
            cz = g.uniform(-0.4, 0.4)
            az = g.uniform(0.05, 0.4)
            q = q + ((z - cz) / az) ** 2
        img += amp * (q <= 1.0)
    phase = np.exp(1j * math.pi * (0.3 * 2.0 * x + 0.2 * 2.0 * y))
    return (img * phase).astype(np.complex64)


def _sphere_points(n: int) -> np.ndarray:
    """n roughly uniform unit vectors (Fibonacci lattice), shape [n, 3]."""
    k = np.arange(n) + 0.5
    phi = np.arccos(1.0 - 2.0 * k / n)
    th = math.pi * (1.0 + math.sqrt(5.0)) * k
    return np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], axis=1)


def coil_maps(shape, coils: int, seed: int = 0) -> np.ndarray:
    """Smooth synthetic coil sensitivities, normalised so sum_c |S_c|^2 = 1.

    Coil c is a Gaussian bump exp(-|r - r_c|^2 / (2 * 0.5^2)) (r in FOV units)
    with phase 2*pi*c/C.  Centres lie on a circle (2-D) or a sphere (3-D) of
    radius 0.7 FOV.  A small seeded jitter of the centres makes the maps differ
    between seeds.
    """
    g = _rng(seed)
    shape = tuple(int(s) for s in shape)
    coords = _norm_coords(shape)
    maps = np.empty((coils,) + shape, dtype=np.complex128)
    if len(shape) == 2:
        y, x = coords
        for c in range(coils):
            th = 2.0 * math.pi * c / coils + g.uniform(-0.05, 0.05)
            cx, cy = 0.7 * math.cos(th), 0.7 * math.sin(th)
            d2 = (x - cx) ** 2 + (y - cy) ** 2
            maps[c] = np.exp(-d2 / (2 * 0.25)) * np.exp(1j * 2.0 * math.pi * c / coils)
    else:
        z, y, x = coords
        pts = _sphere_points(coils)
        for c in range(coils):
            cx, cy, cz = 0.7 * pts[c] + g.uniform(-0.02, 0.02, size=3)
            d2 = (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2
            maps[c] = np.exp(-d2 / (2 * 0.25)) * np.exp(1j * 2.0 * math.pi * c / coils)
    rss = np.sqrt(np.sum(np.abs(maps) ** 2, axis=0))
    maps /= rss
    return maps.astype(np.complex64)


def line_mask(shape, R: float, acs: int, seed: int) -> np.ndarray:
    """Variable-density random phase-encode line mask, constant along x.

    ny/R lines are kept: the `acs` centre lines (capped at ny/R) plus lines
    drawn without replacement with probability proportional to
    (1 - |2k/ny|)^2, k = ky - ny/2.  Returned in centred order, shape
    [ny, nx] (2-D) or [nz, ny, nx] with the same ky pattern for every kz.
    """
    g = _rng(seed)
    shape = tuple(int(s) for s in shape)
    ny, nx = shape[-2], shape[-1]
    n_keep = int(round(ny / R))
    n_acs = min(int(acs), n_keep)
    keep = np.zeros(ny, dtype=bool)
    c0 = ny // 2 - n_acs // 2
    keep[c0:c0 + n_acs] = True
    rest = np.flatnonzero(~keep)
    k = rest - ny // 2
    p = (1.0 - np.abs(2.0 * k / ny)) ** 2
    p = p / p.sum()
    n_draw = n_keep - n_acs
    if n_draw > 0:
        pick = g.choice(rest, size=n_draw, replace=False, p=p)
        keep[pick] = True
    m2 = np.repeat(keep[:, None], nx, axis=1).astype(np.uint8)
    if len(shape) == 3:
        m2 = np.repeat(m2[None], shape[0], axis=0)
    return m2


def _poisson_disc_ky_kz(ny: int, nz: int, r0: float, calib: int, g) -> np.ndarray:
    """Dart throwing over the (ky, kz) grid in random order: a point is kept
    when no kept point lies closer than r0 * (1 + 2*rho), rho = normalised
    radius of the candidate.  The centre calib x calib block is always kept."""
    ky = (np.arange(ny) - ny // 2) / (ny / 2.0)
    kz = (np.arange(nz) - nz // 2) / (nz / 2.0)
    KZ, KY = np.meshgrid(kz, ky, indexing="ij")
    rho = np.sqrt(KY ** 2 + KZ ** 2) / math.sqrt(2.0)
    rad = r0 * (1.0 + 2.0 * rho)
    order = g.permutation(ny * nz)
    mask = np.zeros((nz, ny), dtype=bool)
    cell = max(1, int(math.ceil(r0 * 3.0)))
    buckets: dict = {}
    for idx in order:
        iz, iy = divmod(int(idx), ny)
        r = rad[iz, iy]
        bz, by = iz // cell, iy // cell
        ok = True
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for (pz, py) in buckets.get((bz + dz, by + dy), ()):
                    if (pz - iz) ** 2 + (py - iy) ** 2 < r * r:
                        ok = False
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            mask[iz, iy] = True
            buckets.setdefault((bz, by), []).append((iz, iy))
    c = min(calib, ny, nz)
    mask[nz // 2 - c // 2: nz // 2 - c // 2 + c, ny // 2 - c // 2: ny // 2 - c // 2 + c] = True
    return mask


def poisson_disc_mask(shape, R: float, calib: int, seed: int, tol: float = 0.01) -> np.ndarray:
    """Variable-density Poisson-disc (ky, kz) mask with a fully sampled
    calib x calib centre, constant along the readout x.  The radius scale is
    bisected until the acceleration is R within `tol` (relative) or the
    bisection stalls.  Shape [nz, ny, nx], uint8, centred order."""
    nz, ny, nx = (int(s) for s in shape)
    target = ny * nz / float(R)
    lo, hi = 0.3, 8.0
    best = None
    for it in range(30):
        r0 = 0.5 * (lo + hi)
        m = _poisson_disc_ky_kz(ny, nz, r0, calib, _rng(seed + 7919 * it))
        cnt = m.sum()
        if best is None or abs(cnt - target) < abs(best.sum() - target):
            best = m
        if abs(cnt - target) <= tol * target:
            break
        if cnt > target:
            lo = r0
        else:
            hi = r0
    return np.repeat(best[:, :, None], nx, axis=2).astype(np.uint8)


def spiral_traj(interleaves: int = 16, samples: int = 4096, turns: float = 4.0,
                kmax: float = 128.0) -> np.ndarray:
    """Archimedean spiral k_l(t) = kmax*t*exp(i(2*pi*turns*t + 2*pi*l/L)),
    t = j/samples, j = 0..samples-1.  Returns [L*samples, 2] float32 with
    columns (kx, ky) in cycles/FOV, interleave-major order."""
    t = np.arange(samples, dtype=np.float64) / samples
    out = []
    for l in range(interleaves):
        k = kmax * t * np.exp(1j * (2.0 * math.pi * turns * t + 2.0 * math.pi * l / interleaves))
        out.append(np.stack([k.real, k.imag], axis=1))
    return np.concatenate(out, axis=0).astype(np.float32)


def cnoise(shape, sigma: float, seed: int) -> np.ndarray:
    """Complex Gaussian noise with Re, Im each N(0, sigma^2/2), complex64."""
    return crandn(shape, seed, scale=sigma)


def batched_slices(n_slices: int = 64, seed: int = 2207,
                   sizes=(128, 192, 256, 320, 384), coil_range=(8, 32), r_range=(3, 6)):
    """Uneven 2-D slice list: (ny, nx, coils, R) with ny, nx drawn
    independently from `sizes`, coils uniform on coil_range and R uniform on
    r_range (both inclusive)."""
    g = _rng(seed)
    out = []
    for _ in range(n_slices):
        ny = int(g.choice(sizes))
        nx = int(g.choice(sizes))
        c = int(g.integers(coil_range[0], coil_range[1] + 1))
        r = int(g.integers(r_range[0], r_range[1] + 1))
        out.append((ny, nx, c, r))
    return out


# The five synthetic workloads; seeds are 2204 + index.
CONFIGS = {
    "cart2d_128_c8": dict(kind="cart", shape=(128, 128), coils=8, R=4, acs=24, sigma=1e-3,
                          lam=1e-3, d=3, iters=40, seed=2204),
    "spiral2d_256_c32": dict(kind="noncart", shape=(256, 256), coils=32, interleaves=16,
                             samples=4096, turns=4.0, kb_width=4, oversamp=1.25, sigma=1e-3,
                             lam=5e-4, d=5, iters=100, seed=2205),
    "cart3d_256x256x128_c32": dict(kind="cart", shape=(128, 256, 256), coils=32, R=8, calib=24,
                                   sigma=1e-3, lam=2e-4, d=5, iters=60, seed=2206),
    "batched2d_64": dict(kind="batch", n_slices=64, acs=24, sigma=1e-3, lam=1e-3, d=3, iters=50,
                         seed=2207),
    "unrolled2d_8x256_c16": dict(kind="cart", batch=8, shape=(256, 256), coils=16, R=4, acs=24,
                                 sigma=1e-3, lam=1e-3, d=3, iters=20, checkpoint=5, seed=2208),
}
