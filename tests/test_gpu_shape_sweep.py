"""Plans at the corners of what pp_plan_create accepts, each against the FP64
oracle (relative L2 <= 1e-5 for the forward, adjoint and normal applies):
more than 32 coils (the coil-innermost spiral pipeline and the Toeplitz
operator stop at 32, so these take the coil-major kernels) up to the
64-coil maximum, one coil, FFT lengths with factors 3 and 5, the smallest
gridding grid (40 points), every oversampling the gridding accepts from
1.125 to 2, a one-sample trajectory and samples on the -n/2 edge of the
k-space box; and batches of uneven slices at the same corners."""
import numpy as np
import pytest

import synth
from oracle import pp_oracle as O

pytestmark = pytest.mark.gpu

TOL_APPLY = 1e-5


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


def empty(shape):
    import torch
    return torch.zeros(tuple(shape), dtype=torch.complex64, device="cuda")


def edge_traj(n):
    # samples on the lower edge of [-n/2, n/2) in each axis, at a corner, and
    # one just inside the upper edge
    h = n / 2.0
    return np.array([[-h, 0.0], [0.0, -h], [-h, -h], [h - 0.01, 3.3], [1.7, h - 0.01]], np.float32)


# (id, kind, shape, coils, sampling); shapes are [ny, nx] or [nz, ny, nx]
CASES = [
    ("cart2d_60x100_c33", "cart", (60, 100), 33, dict(R=3, acs=8)),
    ("cart2d_256_c64", "cart", (256, 256), 64, dict(R=4, acs=24)),
    ("cart2d_8x4_c1", "cart", (8, 4), 1, dict(R=2, acs=2)),
    ("cart3d_12x20x8_c33", "cart", (12, 20, 8), 33, dict(R=3, calib=4)),
    ("cart3d_128x128x16_c64", "cart", (128, 128, 16), 64, dict(R=8, calib=12)),
    ("spiral_64_c33_s1.25", "noncart", (64, 64), 33, dict(oversamp=1.25, interleaves=4, samples=400)),
    ("spiral_96x128_c64_s1.5", "noncart", (96, 128), 64,
     dict(oversamp=1.5, interleaves=4, samples=500, turns=3.0, kmax=47.9)),
    ("spiral_32_c1_s1.25_grid40", "noncart", (32, 32), 1,
     dict(oversamp=1.25, interleaves=2, samples=300, turns=2.0, kmax=15.9)),
    ("spiral_64_c3_s1.125", "noncart", (64, 64), 3, dict(oversamp=1.125, interleaves=3, samples=400)),
    ("spiral_64x48_c5_s2_one_sample", "noncart", (64, 48), 5,
     dict(oversamp=2.0, traj=np.array([[3.3, -7.1]], np.float32))),
    ("spiral_64_c2_edge_samples", "noncart", (64, 64), 2, dict(oversamp=1.25, traj=edge_traj(64))),
    ("toeplitz_96x160_c1", "toeplitz", (96, 160), 1,
     dict(oversamp=1.25, interleaves=3, samples=500, turns=3.0, kmax=47.9)),
    ("toeplitz_192x64_c32", "toeplitz", (192, 64), 32,
     dict(oversamp=1.25, interleaves=4, samples=400, turns=3.0, kmax=31.9)),
]


@pytest.fixture(scope="module", params=list(range(len(CASES))), ids=[c[0] for c in CASES])
def case(request, pp):
    _, kind, shape, C, kw = CASES[request.param]
    seed = 900 + request.param
    sens = synth.coil_maps(shape, C, seed)
    if kind == "cart":
        mask = (synth.line_mask(shape, kw["R"], kw["acs"], seed) if len(shape) == 2 else
                synth.poisson_disc_mask(shape, kw["R"], kw["calib"], seed))
        plan = pp.pp_plan_create(shape, C, dev(sens), mask=mask, seed=seed, power_iters=0)
        fwd = lambda x: O.cart_forward(x, sens, mask)
        adj = lambda y: O.cart_adjoint(y, sens, mask)
        normal = lambda x: O.cart_normal(x, sens, mask)
        kshape = (C,) + tuple(shape)
        kmask = mask[None]
    else:
        sigma = kw["oversamp"]
        traj = kw.get("traj")
        if traj is None:
            traj = synth.spiral_traj(kw["interleaves"], kw["samples"], kw.get("turns", 4.0),
                                     kw.get("kmax", shape[0] / 2.0))
        plan = pp.pp_plan_create(shape, C, dev(sens), traj=traj, oversamp=sigma, seed=seed,
                                 power_iters=0, toeplitz=kind == "toeplitz")
        fwd = lambda x: O.nc_forward(x, sens, traj, oversamp=sigma)
        adj = lambda y: O.nc_adjoint(y, sens, traj, oversamp=sigma)
        # the Toeplitz plan's normal operator is the exact F^H F; its forward
        # and adjoint keep the gridding ones
        normal = ((lambda x: O.nc_normal_exact(x, sens, traj)) if kind == "toeplitz" else
                  (lambda x: O.nc_normal(x, sens, traj, oversamp=sigma)))
        kshape = (C, len(traj))
        kmask = 1.0
    yield dict(plan=plan, shape=tuple(shape), kshape=kshape, kmask=kmask, fwd=fwd, adj=adj,
               normal=normal)
    plan.destroy()


def test_forward(pp, case):
    x = synth.crandn(case["shape"], 1)
    y = empty(case["kshape"])
    pp.pp_forward_apply(case["plan"], dev(x), y)
    assert rel(host(y), case["fwd"](x)) <= TOL_APPLY


def test_adjoint(pp, case):
    yk = (synth.crandn(case["kshape"], 2) * case["kmask"]).astype(np.complex64)
    x = empty(case["shape"])
    pp.pp_adjoint_apply(case["plan"], dev(yk), x)
    assert rel(host(x), case["adj"](yk)) <= TOL_APPLY


def test_normal(pp, case):
    x = synth.crandn(case["shape"], 3)
    L = 1.37
    pp.pp_plan_set_scale(case["plan"], L)
    out = empty(case["shape"])
    pp.pp_normal_apply(case["plan"], dev(x), out)
    assert rel(host(out), case["normal"](x) / L) <= TOL_APPLY


# Batches at the same corners: a 4 x 4 slice, 512-point axes (no register FFT
# at that length), 33 to 64 coils per slice, a one-slice batch; each under
# every column tile the batch accepts
BATCHES = [
    ("generic_lengths", [((4, 4), 1, 2), ((12, 512), 33, 3), ((512, 20), 64, 4), ((60, 100), 17, 3)]),
    ("register_lengths", [((384, 384), 64, 6), ((128, 36), 33, 3), ((320, 256), 40, 5)]),
    ("one_slice", [((192, 192), 1, 4)]),
]


@pytest.mark.parametrize("which", range(len(BATCHES)), ids=[b[0] for b in BATCHES])
def test_batch_apply_at_the_limits(pp, which):
    import torch
    slices = BATCHES[which][1]
    shapes = [s for s, _, _ in slices]
    coils = [c for _, c, _ in slices]
    sens = [synth.coil_maps(s, c, 950 + i) for i, (s, c, _) in enumerate(slices)]
    masks = [synth.line_mask(s, R, 4, 960 + i) for i, (s, _, R) in enumerate(slices)]
    b = pp.pp_batch_create(shapes, coils, [dev(v) for v in sens], masks, seed=7, power_iters=0)
    try:
        L = np.linspace(0.7, 1.3, len(slices))
        pp.pp_batch_set_scales(b, L)
        xs = [synth.crandn(s, 970 + i) for i, s in enumerate(shapes)]
        ks = [synth.crandn((c,) + s, 980 + i) * m[None] for i, (s, c, m) in
              enumerate(zip(shapes, coils, masks))]
        ref_n = [O.cart_normal(xs[i], sens[i], masks[i]) / L[i] for i in range(len(slices))]
        ref_a = [O.cart_adjoint(ks[i], sens[i], masks[i]) for i in range(len(slices))]
        x = dev(np.concatenate([v.ravel() for v in xs]))
        k = dev(np.concatenate([v.ravel() for v in ks]))
        off = b.image_off
        tried = 0
        for tile in (4, 8, 16, -8, -16, -32):
            try:
                pp.pp_batch_set_tile(b, tile)
            except pp.PPError:
                continue
            tried += 1
            y = torch.empty_like(x)
            pp.pp_batch_normal_apply(b, x, y)
            got = host(y)
            for i, s in enumerate(shapes):
                assert rel(got[off[i]:off[i + 1]].reshape(s), ref_n[i]) <= TOL_APPLY, (tile, i)
            xa = torch.empty_like(x)
            pp.pp_batch_adjoint_apply(b, k, xa)
            got = host(xa)
            for i, s in enumerate(shapes):
                assert rel(got[off[i]:off[i + 1]].reshape(s), ref_a[i]) <= TOL_APPLY, (tile, i)
        assert tried >= 1
    finally:
        b.destroy()
