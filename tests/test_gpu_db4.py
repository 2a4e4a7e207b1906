"""GPU parity of the Daubechies-4 l1 prox (Eq. "proxdef" with the paper's
wavelet, Sec. 5.1 / 5.2) and of solves that use it, against the FP64 oracle.
Tolerances: relative L2 <= 1e-5 per prox, <= 1e-4 after a solve."""
import numpy as np
import pytest

import synth
from oracle import pp_oracle as O

pytestmark = pytest.mark.gpu

TOL_APPLY = 1e-5
TOL_SOLVE = 1e-4


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


# (ny, nx), levels: square and non-square, bands narrower than the 8-column
# CTA tile (ragged column groups), the deepest level 4, the 512 limit
SHAPES = [((64, 48), 1), ((64, 48), 2), ((256, 256), 2), ((256, 256), 3), ((96, 40), 3),
          ((32, 512), 4), ((512, 16), 2)]


@pytest.mark.parametrize("shape,levels", SHAPES, ids=["%dx%d_L%d" % (s[0], s[1], l) for s, l in SHAPES])
@pytest.mark.parametrize("inplace", [False, True])
def test_db4_prox_parity(pp, shape, levels, inplace):
    v = synth.crandn(shape, 7)
    lam = 0.6     # zeroes a large share of the unit-variance coefficients
    ref = O.prox_l1_db4(v.astype(np.complex128), lam, levels)
    assert np.count_nonzero(np.abs(O.db4_fwd(ref, levels)) < 1e-9) > 0.2 * v.size
    xin = dev(v)
    out = xin if inplace else empty(shape)
    pp.pp_prox_l1_db4(shape, levels, lam, xin, out)
    assert rel(host(out), ref) <= TOL_APPLY


def test_db4_prox_zero_threshold_is_identity(pp):
    v = synth.crandn((128, 96), 8)
    out = empty(v.shape)
    pp.pp_prox_l1_db4(v.shape, 3, 0.0, dev(v), out)
    assert rel(host(out), v.astype(np.complex128)) <= 1e-6


def test_db4_unsupported_raise(pp):
    with pytest.raises(pp.PPError) as e:
        pp.pp_prox_l1_db4((64, 40), 4, 0.1, empty((64, 40)), empty((64, 40)))   # 40 % 16
    assert e.value.status == 2
    with pytest.raises(pp.PPError) as e:
        pp.pp_prox_l1_db4((8, 16, 16), 2, 0.1, empty((8, 16, 16)), empty((8, 16, 16)))   # 3-D
    assert e.value.status == 2


def _cart_problem(pp, shape=(64, 48), coils=4, seed=12):
    sens = synth.coil_maps(shape, coils, seed)
    mask = synth.line_mask(shape, 3, 8, seed)
    plan = pp.pp_plan_create(shape, coils, dev(sens), mask=mask, seed=seed, power_iters=0)
    normal = lambda x: O.cart_normal(x, sens, mask)
    adj = lambda y: O.cart_adjoint(y, sens, mask)
    fwd = lambda x: O.cart_forward(x, sens, mask)
    return plan, normal, adj, fwd, (coils,) + shape, mask


def _spiral_problem(pp, shape=(64, 64), coils=5, seed=13):
    sens = synth.coil_maps(shape, coils, seed)
    traj = synth.spiral_traj(8, 300, 3.0, shape[0] / 2.0)
    plan = pp.pp_plan_create(shape, coils, dev(sens), traj=traj, seed=seed, power_iters=0)
    normal = lambda x: O.nc_normal(x, sens, traj)
    adj = lambda y: O.nc_adjoint(y, sens, traj)
    fwd = lambda x: O.nc_forward(x, sens, traj)
    return plan, normal, adj, fwd, (coils, len(traj)), None


@pytest.mark.parametrize("kind", ["cart", "spiral"])
@pytest.mark.parametrize("d,levels", [(None, 2), (3, 2), (3, 3)])
def test_db4_solve_parity(pp, kind, d, levels):
    shape = (64, 48) if kind == "cart" else (64, 64)
    plan, normal, adj, fwd, kshape, mask = (_cart_problem if kind == "cart" else _spiral_problem)(pp, shape)
    try:
        x0 = synth.phantom(shape, 5)
        noise = synth.crandn(kshape, 6) * 1e-3
        if mask is not None:
            noise = noise * mask[None]
        b = (fwd(x0) + noise).astype(np.complex64)
        L = float(O.power_iteration(normal, shape, 9, iters=30))
        pp.pp_plan_set_scale(plan, L)
        c = None if d is None else [float(v) for v in O.poly_coeffs_l2(d)]
        hist_ref = []
        ref = O.pfista(normal, adj, b.astype(np.complex128), 1e-3, c, 12, L, levels=levels,
                       history=hist_ref, wavelet="db4")
        out = empty(shape)
        r = pp.pp_fista_solve(plan, dev(b), 1e-3, 12, c, 0 if d is None else d, out, history=True,
                              levels=levels, wavelet="db4")
        assert rel(host(out), ref) <= TOL_SOLVE
        yy_ref = np.array([np.linalg.norm(h) ** 2 for h in hist_ref])
        assert np.max(np.abs(r.history[:, 1] - yy_ref) / yy_ref) <= 2 * TOL_SOLVE
        # the Haar solve of the same problem differs (the wavelet is really switched)
        out_h = empty(shape)
        pp.pp_fista_solve(plan, dev(b), 1e-3, 12, c, 0 if d is None else d, out_h, levels=2)
        assert rel(host(out_h), ref) > 10 * TOL_SOLVE
    finally:
        plan.destroy()


def test_db4_ppgd_without_momentum(pp):
    plan, normal, adj, fwd, kshape, mask = _cart_problem(pp)
    try:
        shape = (64, 48)
        b = (fwd(synth.phantom(shape, 8)) + synth.crandn(kshape, 9) * mask[None] * 1e-3).astype(np.complex64)
        L = float(O.power_iteration(normal, shape, 9, iters=30))
        pp.pp_plan_set_scale(plan, L)
        c = [float(v) for v in O.poly_coeffs_l2(3)]
        ref = O.pfista(normal, adj, b.astype(np.complex128), 1e-3, c, 8, L, momentum=False, wavelet="db4")
        out = empty(shape)
        pp.pp_fista_solve(plan, dev(b), 1e-3, 8, c, 3, out, momentum=False, wavelet="db4")
        assert rel(host(out), ref) <= TOL_SOLVE
    finally:
        plan.destroy()
