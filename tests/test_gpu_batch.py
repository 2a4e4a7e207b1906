"""GPU parity of the batched uneven-slice path (many independent 2-D
Cartesian SENSE problems) against the FP64 oracle, slice by slice."""
import numpy as np
import pytest

import synth
from oracle import pp_oracle as O

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.complex128) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def pp():
    from paper_2204_10252_gb300.build import build_library
    build_library()
    import paper_2204_10252_gb300 as m
    m.lib()
    return m


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)).cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


# uneven slices: sizes, coil counts and accelerations all differ; includes
# lengths with factors 3 and 5 and a ragged column tile (nx = 20, 36)
SLICES = [((32, 48), 3, 3), ((48, 32), 2, 4), ((40, 20), 4, 2), ((24, 36), 1, 3), ((64, 64), 5, 5)]


@pytest.fixture(scope="module")
def batch(pp):
    shapes = [s for s, _, _ in SLICES]
    coils = [c for _, c, _ in SLICES]
    sens = [synth.coil_maps(s, c, 10 + i) for i, (s, c, _) in enumerate(SLICES)]
    masks = [synth.line_mask(s, R, 4, 20 + i) for i, (s, _, R) in enumerate(SLICES)]
    sens_t = [dev(x) for x in sens]
    b = pp.pp_batch_create(shapes, coils, sens_t, masks, seed=5, power_iters=50)
    b.np_sens, b.np_masks = sens, masks
    yield b
    b.destroy()


def split(flat, off, shapes):
    return [flat[off[i]:off[i + 1]].reshape(s) for i, s in enumerate(shapes)]


def test_batch_power_iteration(pp, batch):
    L = pp.pp_batch_scales(batch)
    for i, s in enumerate(batch.shapes):
        ref = O.power_iteration(lambda v: O.cart_normal(v, batch.np_sens[i], batch.np_masks[i]), s,
                                5 + i, iters=50)
        assert abs(L[i] - ref) <= 1e-5 * ref


def test_batch_normal_and_adjoint(pp, batch):
    import torch
    L = np.linspace(0.5, 1.5, batch.n)
    pp.pp_batch_set_scales(batch, L)
    xs = [synth.crandn(s, 30 + i) for i, s in enumerate(batch.shapes)]
    x = dev(np.concatenate([v.ravel() for v in xs]))
    y = torch.empty_like(x)
    pp.pp_batch_normal_apply(batch, x, y)
    got = split(host(y), batch.image_off, batch.shapes)
    for i in range(batch.n):
        ref = O.cart_normal(xs[i], batch.np_sens[i], batch.np_masks[i]) / L[i]
        assert rel(got[i], ref) <= 1e-5
    ks = [synth.crandn((c,) + s, 40 + i) * m[None] for i, (s, c, m) in
          enumerate(zip(batch.shapes, batch.coils, batch.np_masks))]
    k = dev(np.concatenate([v.ravel() for v in ks]))
    xa = torch.empty_like(x)
    pp.pp_batch_adjoint_apply(batch, k, xa)
    got = split(host(xa), batch.image_off, batch.shapes)
    for i in range(batch.n):
        assert rel(got[i], O.cart_adjoint(ks[i], batch.np_sens[i], batch.np_masks[i])) <= 1e-5


@pytest.mark.parametrize("d", [None, 3])
def test_batch_solve(pp, batch, d):
    import torch
    Ls = pp.pp_batch_scales(batch)
    xs = [synth.phantom(s, 50 + i) for i, s in enumerate(batch.shapes)]
    bs = [(O.cart_forward(xs[i], batch.np_sens[i], batch.np_masks[i]) +
           1e-3 * synth.crandn((batch.coils[i],) + batch.shapes[i], 60 + i) * batch.np_masks[i][None])
          .astype(np.complex64) for i in range(batch.n)]
    b = dev(np.concatenate([v.ravel() for v in bs]))
    out = torch.empty(int(batch.image_off[-1]), dtype=torch.complex64, device="cuda")
    lam, iters = 1e-3, 10
    c = None if d is None else [float(v) for v in O.poly_coeffs_l2(d)]
    r = pp.pp_batch_fista_solve(batch, b, lam, iters, c, 0 if d is None else d, out, history=True)
    got = split(host(out), batch.image_off, batch.shapes)
    tot = 0.0
    for i in range(batch.n):
        ref = O.pfista(lambda v: O.cart_normal(v, batch.np_sens[i], batch.np_masks[i]),
                       lambda yk: O.cart_adjoint(yk, batch.np_sens[i], batch.np_masks[i]),
                       bs[i].astype(np.complex128), lam, c, iters, Ls[i])
        assert rel(got[i], ref) <= 1e-4
        tot += np.linalg.norm(ref) ** 2
    assert abs(r.history[-1, 1] - tot) <= 1e-3 * tot


def test_batch_tile_is_one_of_the_candidates(pp, batch):
    t, grid = pp.pp_batch_tile(batch)
    assert t in (4, 8, 16, -8, -16, -32) and grid >= 1


# every slice length has a register FFT (16 x {8, 12, 16, 20, 24}); nx ragged
FAST = [((128, 24), 3, 3), ((192, 40), 2, 4), ((256, 16), 4, 3), ((320, 20), 2, 5), ((384, 12), 3, 4)]


@pytest.mark.parametrize("tile", [-8, -16, -32, 4, 8, 16])
def test_batch_variants_agree_with_oracle(pp, tile):
    import torch
    shapes = [s for s, _, _ in FAST]
    coils = [c for _, c, _ in FAST]
    sens = [synth.coil_maps(s, c, 70 + i) for i, (s, c, _) in enumerate(FAST)]
    masks = [synth.line_mask(s, R, 8, 80 + i) for i, (s, _, R) in enumerate(FAST)]
    b = pp.pp_batch_create(shapes, coils, [dev(x) for x in sens], masks, seed=1, power_iters=0)
    try:
        if tile == 16 and max(s[0] for s in shapes) > 256:
            with pytest.raises(pp.PPError):
                pp.pp_batch_set_tile(b, tile)
            return
        pp.pp_batch_set_tile(b, tile)
        assert pp.pp_batch_tile(b)[0] == tile
        L = np.linspace(0.7, 1.3, b.n)
        pp.pp_batch_set_scales(b, L)
        xs = [synth.crandn(s, 90 + i) for i, s in enumerate(shapes)]
        x = dev(np.concatenate([v.ravel() for v in xs]))
        y = torch.empty_like(x)
        pp.pp_batch_normal_apply(b, x, y)
        got = split(host(y), b.image_off, shapes)
        for i in range(b.n):
            assert rel(got[i], O.cart_normal(xs[i], sens[i], masks[i]) / L[i]) <= 1e-5
    finally:
        b.destroy()


@pytest.mark.parametrize("tile", [-8, -16, -32])
def test_uniform_length_batch(pp, tile):
    # every slice 256 rows (one register-FFT length): the uniform-length
    # kernels, one CTA per item (-8) or the coils split over 2 or 4 CTAs
    import torch
    shapes = [(256, 36), (256, 64), (256, 20)]
    coils = [4, 8, 2]
    sens = [synth.coil_maps(s, c, 170 + i) for i, (s, c) in enumerate(zip(shapes, coils))]
    masks = [synth.line_mask(s, 4, 8, 180 + i) for i, s in enumerate(shapes)]
    b = pp.pp_batch_create(shapes, coils, [dev(x) for x in sens], masks, seed=1, power_iters=0)
    try:
        pp.pp_batch_set_tile(b, tile)
        assert pp.pp_batch_tile(b)[0] == tile
        L = np.array([0.8, 1.1, 1.3])
        pp.pp_batch_set_scales(b, L)
        xs = [synth.crandn(s, 190 + i) for i, s in enumerate(shapes)]
        x = dev(np.concatenate([v.ravel() for v in xs]))
        y = torch.empty_like(x)
        for _ in range(2):
            pp.pp_batch_normal_apply(b, x, y)
            got = split(host(y), b.image_off, shapes)
            for i in range(b.n):
                assert rel(got[i], O.cart_normal(xs[i], sens[i], masks[i]) / L[i]) <= 1e-5
    finally:
        b.destroy()
