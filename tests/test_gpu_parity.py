"""GPU parity: every libpp entry point against the FP64 oracle on the same
seeded inputs.  Tolerances: relative L2 <= 1e-5 per operator apply, <= 1e-4
after a full solve (FP32 arithmetic throughout on the device, FP64
reductions)."""
import math

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


class Problem:
    """Oracle-side operator closures plus the GPU plan for one case."""

    def __init__(self, pp, kind, shape, coils, seed, **kw):
        self.kind, self.shape, self.C = kind, tuple(shape), coils
        self.sens = synth.coil_maps(shape, coils, seed)
        self.sens_t = dev(self.sens)
        if kind == "cart":
            if len(shape) == 2:
                self.mask = synth.line_mask(shape, kw.get("R", 4), kw.get("acs", 8), seed)
            else:
                self.mask = synth.poisson_disc_mask(shape, kw.get("R", 3), kw.get("calib", 4), seed)
            self.fwd = lambda x: O.cart_forward(x, self.sens, self.mask)
            self.adj = lambda y: O.cart_adjoint(y, self.sens, self.mask)
            self.kshape = (coils,) + self.shape
            self.plan = pp.pp_plan_create(shape, coils, self.sens_t, mask=self.mask, seed=seed,
                                          power_iters=0)
        else:
            self.traj = synth.spiral_traj(kw["interleaves"], kw["samples"], kw.get("turns", 4.0),
                                          kw.get("kmax", shape[0] / 2.0))
            self.fwd = lambda x: O.nc_forward(x, self.sens, self.traj)
            self.adj = lambda y: O.nc_adjoint(y, self.sens, self.traj)
            self.kshape = (coils, len(self.traj))
            self.plan = pp.pp_plan_create(shape, coils, self.sens_t, traj=self.traj, seed=seed,
                                          power_iters=0)
        self.normal = lambda x: self.adj(self.fwd(x))

    def ksp(self, seed):
        y = synth.crandn(self.kshape, seed)
        if self.kind == "cart":
            y = y * self.mask[None]
        return y.astype(np.complex64)


CASES = [
    ("cart", (64, 48), 3, dict(R=3, acs=6)),
    ("cart", (128, 128), 8, dict(R=4, acs=24)),
    ("cart", (16, 24, 20), 3, dict(R=3, calib=4)),
    ("noncart", (64, 64), 4, dict(interleaves=4, samples=512)),
    ("noncart", (72, 80), 2, dict(interleaves=3, samples=700, turns=3.0, kmax=35.9)),
    ("cart", (192, 256), 4, dict(R=3, acs=12)),
    ("cart", (384, 128), 5, dict(R=4, acs=16)),
    ("cart", (128, 192, 20), 2, dict(R=4, calib=8)),
    ("cart", (16, 24, 32), 2, dict(R=3, calib=4)),
]
IDS = ["cart2d_64x48", "cart2d_128", "cart3d_16x24x20", "spiral_64", "spiral_72x80_ragged",
       "cart2d_192x256", "cart2d_384x128", "cart3d_128x192x20", "cart3d_16x24x32"]


@pytest.fixture(scope="module", params=list(range(len(CASES))), ids=IDS)
def prob(request, pp):
    kind, shape, C, kw = CASES[request.param]
    p = Problem(pp, kind, shape, C, 100 + request.param, **kw)
    yield p
    p.plan.destroy()


SMALL_NC = [((64, 64), 5, dict(interleaves=4, samples=512)),
            ((72, 80), 2, dict(interleaves=3, samples=700, turns=3.0, kmax=35.9)),
            ((32, 40), 3, dict(interleaves=2, samples=300, turns=2.0, kmax=15.9))]


@pytest.mark.parametrize("case", range(len(SMALL_NC)), ids=["spiral64_c5", "spiral72x80_c2",
                                                            "spiral32x40_c3"])
def test_every_stencil_kind_small_grids(pp, case):
    # Grids that end inside a tile (32 x 40 -> 40 x 50: the smallest grid a
    # plan accepts) and coil counts that leave a coil group part empty.
    shape, C, kw = SMALL_NC[case]
    p = Problem(pp, "noncart", shape, C, 300 + case, **kw)
    try:
        x = synth.crandn(shape, 5)
        L = 2.5
        pp.pp_plan_set_scale(p.plan, L)
        ref = p.normal(x) / L
        for kind in range(7):
            for cpc in ((1, 3) if kind < 2 else (8,)):
                pp.pp_plan_set_tuning(p.plan, 1, kind, cpc)
                out = empty(shape)
                pp.pp_normal_apply(p.plan, dev(x), out)
                assert rel(host(out), ref) <= TOL_APPLY, (kind, cpc)
    finally:
        p.plan.destroy()


CI_CASES = [((64, 64), 5, 2.0, dict(interleaves=4, samples=512)),
            ((96, 128), 32, 2.0, dict(interleaves=4, samples=600, turns=3.0, kmax=47.9)),
            ((64, 64), 17, 2.0, dict(interleaves=3, samples=400, turns=3.0, kmax=31.9))]


@pytest.mark.parametrize("case", range(len(CI_CASES)), ids=["64_c5", "96x128_c32", "64_c17"])
def test_coil_innermost_pipeline(pp, case):
    # Oversampling 2 gives grids of register-FFT length (128, 192, 256); 32
    # coils run on the aliased workspaces, fewer on padded copies.
    shape, C, sigma, kw = CI_CASES[case]
    sens = synth.coil_maps(shape, C, 400 + case)
    traj = synth.spiral_traj(kw["interleaves"], kw["samples"], kw["turns"] if "turns" in kw else 4.0,
                             kw.get("kmax", shape[0] / 2.0))
    plan = pp.pp_plan_create(shape, C, dev(sens), traj=traj, oversamp=sigma, seed=1, power_iters=0)
    try:
        x = synth.crandn(shape, 6)
        normal = lambda v: O.nc_normal(v, sens, traj, oversamp=sigma)
        L = float(O.power_iteration(normal, shape, 9, iters=10))
        pp.pp_plan_set_scale(plan, L)
        ref = normal(x) / L
        for kind, rv in ((7, 1), (8, 1), (7, 4), (8, 4), (9, 1), (9, 4), (2, 1)):
            pp.pp_plan_set_tuning(plan, rv, kind, 8)
            out = empty(shape)
            pp.pp_normal_apply(plan, dev(x), out)
            assert rel(host(out), ref) <= TOL_APPLY, (kind, rv)
        # axpy epilogue of the Horner recursion goes through the same path
        pp.pp_plan_set_tuning(plan, 4, 7, 8)
        c = [float(v) for v in O.poly_coeffs_l2(3)]
        out = empty(shape)
        pp.pp_poly_apply(plan, c, 3, dev(x), out)
        ref = O.horner_apply(c, lambda v: normal(v) / L, x.astype(np.complex128))
        assert rel(host(out), ref) <= TOL_APPLY
    finally:
        plan.destroy()


C3_CASES = [((128, 128, 8), 3), ((128, 256, 12), 2), ((128, 192, 20), 5)]


@pytest.mark.parametrize("case", range(len(C3_CASES)), ids=["128x128x8_c3", "128x256x12_c2",
                                                           "128x192x20_c5"])
def test_cart3d_cluster_operator(pp, case):
    # nz = 128 and ny in {128, 192, 256}: the one-kernel cluster operator
    # (row variant 16) against the three-pass one (1), both against the oracle
    shape, C = C3_CASES[case]
    sens = synth.coil_maps(shape, C, 500 + case)
    mask = synth.poisson_disc_mask(shape, 4, 8, 500 + case)
    plan = pp.pp_plan_create(shape, C, dev(sens), mask=mask, seed=2, power_iters=0)
    try:
        x = synth.crandn(shape, 7)
        op = synth.crandn(shape, 8)
        L = 1.7
        pp.pp_plan_set_scale(plan, L)
        ref = O.cart_normal(x, sens, mask) / L
        for rv in (16, -16, 1):
            try:
                pp.pp_plan_set_tuning(plan, rv, 0, 8)
            except pp.PPError:
                assert rv in (16, -16)
                pytest.skip("no 16-CTA cluster fits this device")
            out = empty(shape)
            pp.pp_normal_apply(plan, dev(x), out)
            assert rel(host(out), ref) <= TOL_APPLY, rv
        # the Horner axpy epilogue (operand, alpha) through the cluster kernels
        c = [float(v) for v in O.poly_coeffs_l2(2)]
        refp = O.horner_apply(c, lambda v: O.cart_normal(v, sens, mask) / L, op.astype(np.complex128))
        for rv in (16, -16):
            pp.pp_plan_set_tuning(plan, rv, 0, 8)
            out = empty(shape)
            pp.pp_poly_apply(plan, c, 2, dev(op), out)
            assert rel(host(out), refp) <= TOL_APPLY, rv
    finally:
        plan.destroy()


DF_CASES = [((128, 256, 40), 5), ((128, 128, 8), 3), ((192, 192, 20), 9), ((128, 384, 16), 2),
            ((256, 128, 36), 7), ((128, 256, 4), 1)]


@pytest.mark.parametrize("case", range(len(DF_CASES)), ids=["128x256x40_c5", "128x128x8_c3",
                                                           "192x192x20_c9", "128x384x16_c2",
                                                           "256x128x36_c7", "128x256x4_c1"])
def test_cart3d_dataflow_operator(pp, case):
    # the 3-D persistent dataflow operator (row variant 3) for every coil
    # group size 1..8: full and ragged x-blocks (nx not a multiple of 16),
    # ragged last coil groups, nz and ny of 128 ... 384, and the Horner axpy
    # epilogue; against the oracle
    shape, C = DF_CASES[case]
    sens = synth.coil_maps(shape, C, 520 + case)
    mask = synth.poisson_disc_mask(shape, 4, 8, 520 + case)
    plan = pp.pp_plan_create(shape, C, dev(sens), mask=mask, seed=2, power_iters=0)
    try:
        x = synth.crandn(shape, 17)
        op = synth.crandn(shape, 18)
        L = 1.3
        pp.pp_plan_set_scale(plan, L)
        nrm = lambda v: O.cart_normal(v, sens, mask) / L
        ref = nrm(x)
        c = [float(v) for v in O.poly_coeffs_l2(2)]
        refp = O.horner_apply(c, nrm, op.astype(np.complex128))
        for cg, hi in [(g, h) for g in sorted({1, 2, 3, 4, 8, min(C, 8)}) for h in (0, 1, 2, 3, 4, 5)]:
            pp.pp_plan_set_tuning(plan, 3, hi, cg)
            assert pp.pp_plan_tuning(plan) == (3, hi, cg)
            out = empty(shape)
            pp.pp_normal_apply(plan, dev(x), out)
            assert rel(host(out), ref) <= TOL_APPLY, (cg, hi)
            out = empty(shape)
            pp.pp_poly_apply(plan, c, 2, dev(op), out)
            assert rel(host(out), refp) <= TOL_APPLY, (cg, hi)
        # the bounded waits never ran out: a synchronising call reports no timeout
        pp.pp_plan_mu(plan, 2, 1)
    finally:
        plan.destroy()


def test_bounded_wait_gives_up_and_the_device_stays_usable(pp):
    # a block waits on a counter nothing increments: the wait must give up
    # after its limit (50 ms), the call must report PP_ERR_TIMEOUT, and the
    # device must still run a normal apply correctly afterwards
    import time
    t0 = time.perf_counter()
    with pytest.raises(pp.PPError) as e:
        pp.pp_selftest_wait(50_000_000)
    assert e.value.status == 6
    assert time.perf_counter() - t0 < 5.0
    shape, C = (128, 128, 8), 2
    sens = synth.coil_maps(shape, C, 3)
    mask = synth.poisson_disc_mask(shape, 4, 8, 3)
    plan = pp.pp_plan_create(shape, C, dev(sens), mask=mask, power_iters=0)
    try:
        pp.pp_plan_set_tuning(plan, 3, 0, 2)
        x = synth.crandn(shape, 4)
        out = empty(shape)
        pp.pp_normal_apply(plan, dev(x), out)
        assert rel(host(out), O.cart_normal(x, sens, mask)) <= TOL_APPLY
    finally:
        plan.destroy()


C2_CASES = [((128, 128), 8), ((192, 256), 3), ((384, 128), 5), ((256, 36), 16)]


@pytest.mark.parametrize("case", range(len(C2_CASES)), ids=["128_c8", "192x256_c3", "384x128_c5",
                                                           "256x36_c16"])
def test_cart2d_coil_split_clusters(pp, case):
    # Coils split over 1, 2, 4 or 8 CTAs per 8-column group (cluster partial
    # sums); more CTAs than coils leaves some with no coil.  36 columns end
    # inside a column group.
    shape, C = C2_CASES[case]
    sens = synth.coil_maps(shape, C, 600 + case)
    mask = synth.line_mask(shape, 4, 8, 600 + case)
    plan = pp.pp_plan_create(shape, C, dev(sens), mask=mask, seed=3, power_iters=0)
    try:
        x = synth.crandn(shape, 9)
        op = synth.crandn(shape, 10)
        L = 0.9
        pp.pp_plan_set_scale(plan, L)
        ref = O.cart_normal(x, sens, mask) / L
        for cl in (1, 2, 4, 8):
            pp.pp_plan_set_tuning(plan, cl, 0, 8)
            assert pp.pp_plan_tuning(plan)[0] == cl
            out = empty(shape)
            pp.pp_normal_apply(plan, dev(x), out)
            assert rel(host(out), ref) <= TOL_APPLY, cl
            c = [float(v) for v in O.poly_coeffs_l2(2)]
            out = empty(shape)
            pp.pp_poly_apply(plan, c, 2, dev(op), out)
            refp = O.horner_apply(c, lambda v: O.cart_normal(v, sens, mask) / L, op.astype(np.complex128))
            assert rel(host(out), refp) <= TOL_APPLY, cl
    finally:
        plan.destroy()


def test_forward_parity(pp, prob):
    x = synth.crandn(prob.shape, 1)
    y = empty(prob.kshape)
    pp.pp_forward_apply(prob.plan, dev(x), y)
    assert rel(host(y), prob.fwd(x)) <= TOL_APPLY


def test_adjoint_parity(pp, prob):
    yk = prob.ksp(2)
    x = empty(prob.shape)
    pp.pp_adjoint_apply(prob.plan, dev(yk), x)
    assert rel(host(x), prob.adj(yk)) <= TOL_APPLY


def test_normal_parity_with_shared_scale(pp, prob):
    x = synth.crandn(prob.shape, 3)
    L = 0.731
    pp.pp_plan_set_scale(prob.plan, L)
    out = empty(prob.shape)
    pp.pp_normal_apply(prob.plan, dev(x), out)
    assert rel(host(out), prob.normal(x) / L) <= TOL_APPLY


@pytest.mark.parametrize("d", [0, 1, 3, 5])
def test_poly_apply_parity(pp, prob, d):
    x = synth.crandn(prob.shape, 4)
    L = float(O.power_iteration(prob.normal, prob.shape, 9, iters=10))
    pp.pp_plan_set_scale(prob.plan, L)
    c = [float(v) for v in O.poly_coeffs_l2(d)]
    out = empty(prob.shape)
    pp.pp_poly_apply(prob.plan, c, d, dev(x), out)
    ref = O.horner_apply(c, lambda v: prob.normal(v) / L, x.astype(np.complex128))
    assert rel(host(out), ref) <= TOL_APPLY


def test_power_iteration_matches_oracle(pp, prob):
    import torch
    L_ref = O.power_iteration(prob.normal, prob.shape, 77, iters=50)
    plan = pp.pp_plan_create(prob.shape, prob.C, prob.sens_t,
                             mask=getattr(prob, "mask", None) if prob.kind == "cart" else None,
                             traj=getattr(prob, "traj", None) if prob.kind != "cart" else None,
                             seed=77, power_iters=50)
    try:
        L = pp.pp_plan_scale(plan)
    finally:
        plan.destroy()
    assert abs(L - L_ref) <= 1e-5 * L_ref


@pytest.mark.parametrize("d", [None, 3])
def test_solve_parity(pp, prob, d):
    x0 = synth.phantom(prob.shape, 5)
    b = (prob.fwd(x0) + prob.ksp(6) * 1e-3).astype(np.complex64)
    L = float(O.power_iteration(prob.normal, prob.shape, 9, iters=30))
    pp.pp_plan_set_scale(prob.plan, L)
    lam, iters = 1e-3, 12
    c = None if d is None else [float(v) for v in O.poly_coeffs_l2(d)]
    hist_ref = []
    ref = O.pfista(prob.normal, prob.adj, b.astype(np.complex128), lam, c, iters, L,
                   history=hist_ref)
    out = empty(prob.shape)
    r = pp.pp_fista_solve(prob.plan, dev(b), lam, iters, c, 0 if d is None else d, out,
                          history=True, ref=dev(ref))
    assert r.L == L
    assert abs(r.bnorm - np.linalg.norm(b.astype(np.complex128))) <= 1e-9 * r.bnorm
    assert rel(host(out), ref) <= TOL_SOLVE
    # FP64 statistics per iteration: ||y_{k+1}||^2 and ||y_{k+1} - ref||^2
    yy_ref = np.array([np.linalg.norm(h) ** 2 for h in hist_ref])
    assert np.max(np.abs(r.history[:, 1] - yy_ref) / yy_ref) <= 2 * TOL_SOLVE
    dist_ref = np.array([np.linalg.norm(h - ref.astype(np.complex64)) ** 2 for h in hist_ref])
    assert abs(np.sqrt(r.history[-1, 2]) - np.sqrt(dist_ref[-1])) <= 2 * TOL_SOLVE * np.linalg.norm(ref)
    assert np.all(np.diff(np.sqrt(r.history[:, 2])) <= 0.5)   # well-formed, finite
    assert r.launches > iters


def test_safe_scale_divides_the_polynomial_by_its_step_bound(pp, prob):
    # pp_solve_info.safe_scale: the solve with c divided by max z p(z) on
    # [0, 1] (the reading that keeps FISTA's step rule); the same as passing
    # the divided coefficients, and equal to the oracle's solve with them
    x0 = synth.phantom(prob.shape, 5)
    b = (prob.fwd(x0) + prob.ksp(6) * 1e-3).astype(np.complex64)
    L = float(O.power_iteration(prob.normal, prob.shape, 9, iters=30))
    pp.pp_plan_set_scale(prob.plan, L)
    lam, iters, d = 1e-3, 12, 3
    c = [float(v) for v in O.poly_coeffs_l2(d)]
    m = pp.pp_poly_max_zp(c, d)
    assert abs(m - O.poly_max_zp(np.array(c))) <= 1e-9
    cs = [v / m for v in c]
    out_flag, out_div = empty(prob.shape), empty(prob.shape)
    pp.pp_fista_solve(prob.plan, dev(b), lam, iters, c, d, out_flag, safe_scale=True)
    pp.pp_fista_solve(prob.plan, dev(b), lam, iters, cs, d, out_div)
    if prob.kind == "cart":
        # the same coefficients, the same kernels: bit for bit (the
        # non-Cartesian adjoint accumulates each tile with shared-memory
        # atomics, whose order varies from call to call)
        assert np.array_equal(host(out_flag), host(out_div))
    ref = O.pfista(prob.normal, prob.adj, b.astype(np.complex128), lam, cs, iters, L)
    assert rel(host(out_flag), ref) <= TOL_SOLVE
    assert rel(host(out_div), ref) <= TOL_SOLVE


def test_mu_estimate_matches_oracle(pp, prob):
    # power iteration on I - N_hat (Sec. 3.4 remark) from the same seed and
    # L: the Rayleigh quotients 1 - mu agree to FP32-apply accuracy
    L = float(O.power_iteration(prob.normal, prob.shape, 9, iters=30))
    pp.pp_plan_set_scale(prob.plan, L)
    mu_ref = O.mu_estimate(prob.normal, prob.shape, 5, L, iters=40)
    mu = pp.pp_plan_mu(prob.plan, 40, 5)
    assert abs(mu - mu_ref) <= 1e-5
    assert mu < 1.0


def test_chebyshev_solve_with_estimated_mu(pp):
    # the Chebyshev design end to end, no caller-supplied mu: a 2-D
    # Cartesian problem with more coils than the acceleration (A^H A
    # injective), mu from pp_plan_mu, coefficients from pp_poly_coeffs_cheb,
    # 20 iterations against the oracle with the oracle's own mu estimate
    shape, C = (64, 64), 8
    p = Problem(pp, "cart", shape, C, 12, R=2, acs=16)
    try:
        x0 = synth.phantom(shape, 13)
        b = (p.fwd(x0) + p.ksp(14) * 1e-3).astype(np.complex64)
        L = float(O.power_iteration(p.normal, shape, 9, iters=30))
        pp.pp_plan_set_scale(p.plan, L)
        mu = pp.pp_plan_mu(p.plan, 200, 3)
        mu_ref = O.mu_estimate(p.normal, shape, 3, L, iters=200)
        assert 0.0 < mu < 1.0 and abs(mu - mu_ref) <= 1e-5
        c = [float(v) for v in pp.pp_poly_coeffs_cheb(3, mu)]
        c_ref = [float(v) for v in O.poly_coeffs_cheb(3, mu_ref)]
        assert np.max(np.abs(np.array(c) - c_ref)) <= 1e-3 * np.max(np.abs(c_ref))
        ref = O.pfista(p.normal, p.adj, b.astype(np.complex128), 1e-3, c, 20, L)
        out = empty(shape)
        pp.pp_fista_solve(p.plan, dev(b), 1e-3, 20, c, 3, out)
        assert rel(host(out), ref) <= TOL_SOLVE
    finally:
        p.plan.destroy()


@pytest.mark.parametrize("coeffs", ["l2", "cheb"])
def test_ppgd_without_momentum(pp, prob, coeffs):
    # Algorithm "ppgd" (beta_k = 0) with the l2 or the Chebyshev polynomial
    x0 = synth.phantom(prob.shape, 8)
    b = (prob.fwd(x0) + prob.ksp(9) * 1e-3).astype(np.complex64)
    L = float(O.power_iteration(prob.normal, prob.shape, 9, iters=30))
    pp.pp_plan_set_scale(prob.plan, L)
    c = [float(v) for v in (O.poly_coeffs_l2(3) if coeffs == "l2" else O.poly_coeffs_cheb(3, 0.05))]
    ref = O.pfista(prob.normal, prob.adj, b.astype(np.complex128), 1e-3, c, 8, L, momentum=False)
    out = empty(prob.shape)
    pp.pp_fista_solve(prob.plan, dev(b), 1e-3, 8, c, 3, out, momentum=False)
    assert rel(host(out), ref) <= TOL_SOLVE


@pytest.mark.parametrize("shape,levels", [((64, 48), 2), ((64, 48), 1), ((8, 16, 12), 2),
                                          ((6, 10, 14), 1), ((4, 4), 2), ((8, 12, 48), 2),
                                          ((16, 32, 64), 2), ((12, 8, 32), 1)])
@pytest.mark.parametrize("inplace", [False, True])
def test_prox_parity(pp, shape, levels, inplace):
    x = synth.crandn(shape, 7)
    lam = 0.4
    xin = dev(x)
    out = xin if inplace else empty(shape)
    pp.pp_prox_l1_haar(shape, levels, lam, xin, out)
    assert rel(host(out), O.prox_l1_haar(x, lam, levels)) <= TOL_APPLY


@pytest.mark.parametrize("shape", [(16, 32), (8, 16, 16)])
def test_prox_edge_cases(pp, shape):
    # an all-zero 4x4(x4) tile (|v| = 0: no division), a constant tile whose
    # coarsest Haar coefficient is exactly lambda (4 v in 2-D, 8 v in 3-D
    # with v = 1/4 resp. 1/8: the output is 0 there), one just above it;
    # lambda = 0 is the identity and a lambda above every |coefficient|
    # gives exactly 0
    x = synth.crandn(shape, 21)
    nd = len(shape)
    v = 0.25 if nd == 2 else 0.125
    t = lambda i: (slice(4 * i, 4 * i + 4),) * nd
    x[(slice(0, 4),) * nd] = 0.0
    x[t(1)] = v
    x[(slice(0, 4),) * (nd - 1) + (slice(8, 12),)] = v * (1 + 1e-3)
    lam = 1.0
    out = empty(shape)
    pp.pp_prox_l1_haar(shape, 2, lam, dev(x), out)
    got = host(out)
    ref = O.prox_l1_haar(x, lam, 2)
    assert np.all(np.isfinite(got))
    assert rel(got, ref) <= TOL_APPLY
    assert np.all(got[(slice(0, 4),) * nd] == 0)
    assert np.max(np.abs(got[t(1)])) <= 1e-6
    for lam_e, want in ((0.0, x.astype(np.complex128)), (1e6, np.zeros(shape))):
        pp.pp_prox_l1_haar(shape, 2, lam_e, dev(x), out)
        got = host(out)
        if lam_e == 0.0:
            assert rel(got, want) <= TOL_APPLY
        else:
            assert np.all(got == 0)


def test_solve_zero_and_nonfinite_b(pp):
    # b = 0: the solution is 0 (no NaN from the unit-norm scaling of b);
    # a NaN in b: the iterates are NaN (not silently zero), and a call
    # with a history reports PP_ERR_NONFINITE
    shape, C = (32, 32), 2
    p = Problem(pp, "cart", shape, C, 4, R=2, acs=8)
    try:
        pp.pp_plan_set_scale(p.plan, 1.5)
        c = [float(v) for v in O.poly_coeffs_l2(3)]
        out = empty(shape)
        r = pp.pp_fista_solve(p.plan, dev(np.zeros(p.kshape, np.complex64)), 1e-3, 5, c, 3, out,
                              history=True)
        assert np.all(host(out) == 0) and r.bnorm == 0.0
        b = p.ksp(5)
        b[1, 3, 7] = np.nan
        pp.pp_fista_solve(p.plan, dev(b), 1e-3, 5, c, 3, out)
        assert np.all(np.isnan(host(out)))
        with pytest.raises(pp.PPError) as e:
            pp.pp_fista_solve(p.plan, dev(b), 1e-3, 5, c, 3, out, history=True)
        assert e.value.status == 5
        # the plan still works afterwards
        b = p.ksp(6)
        pp.pp_fista_solve(p.plan, dev(b), 1e-3, 5, c, 3, out, history=True)
        assert np.all(np.isfinite(host(out)))
    finally:
        p.plan.destroy()


def test_solve_edge_cases(pp):
    shape, C = (32, 32), 1
    p = Problem(pp, "cart", shape, C, 3, R=2, acs=8)
    try:
        x0 = synth.phantom(shape, 1)
        b = (p.fwd(x0)).astype(np.complex64)
        L = float(O.power_iteration(p.normal, shape, 9, iters=30))
        pp.pp_plan_set_scale(p.plan, L)
        out = empty(shape)
        # zero iterations: y_0 = 0
        pp.pp_fista_solve(p.plan, dev(b), 1e-3, 0, None, 0, out)
        assert np.all(host(out) == 0)
        # lambda = 0, d = 0 with c0 != 1 (scaled gradient step)
        ref = O.pfista(p.normal, p.adj, b.astype(np.complex128), 0.0, [0.5], 6, L)
        pp.pp_fista_solve(p.plan, dev(b), 0.0, 6, [0.5], 0, out)
        assert rel(host(out), ref) <= TOL_SOLVE
        # rescale to the units of the original problem
        ref = O.pfista(p.normal, p.adj, b.astype(np.complex128), 1e-3, None, 5, L)
        ref = ref * np.linalg.norm(b.astype(np.complex128)) / math.sqrt(L)
        pp.pp_fista_solve(p.plan, dev(b), 1e-3, 5, None, 0, out, rescale=True)
        assert rel(host(out), ref) <= TOL_SOLVE
    finally:
        p.plan.destroy()


def test_unsupported_sizes_raise(pp):
    import torch
    sens = dev(synth.coil_maps((28, 28), 2, 0))
    with pytest.raises(pp.PPError) as e:   # 28 = 4 * 7: prime factor 7
        pp.pp_plan_create((28, 28), 2, sens, mask=np.ones((28, 28), np.uint8), power_iters=0)
    assert e.value.status == 2
    m = np.ones((32, 32), np.uint8)
    m[3, 5] = 0   # not constant along x
    sens = dev(synth.coil_maps((32, 32), 2, 0))
    with pytest.raises(pp.PPError) as e:
        pp.pp_plan_create((32, 32), 2, sens, mask=m, power_iters=0)
    assert e.value.status == 2
    traj = np.array([[40.0, 0.0]], np.float32)   # outside [-n/2, n/2)
    with pytest.raises(pp.PPError) as e:
        pp.pp_plan_create((64, 64), 2, dev(synth.coil_maps((64, 64), 2, 0)), traj=traj, power_iters=0)
    assert e.value.status == 1


@pytest.fixture(scope="module")
def full_spiral(pp):
    # 256^2, 32 coils, 16 x 4096 spiral: the workload the benchmark times.
    cfg = synth.CONFIGS["spiral2d_256_c32"]
    shape, C = cfg["shape"], cfg["coils"]
    sens = synth.coil_maps(shape, C, cfg["seed"])
    traj = synth.spiral_traj(cfg["interleaves"], cfg["samples"], cfg["turns"], 128.0)
    plan = pp.pp_plan_create(shape, C, dev(sens), traj=traj, power_iters=0)
    L = 123.0
    pp.pp_plan_set_scale(plan, L)
    x = synth.crandn(shape, 11)
    ref = O.nc_normal(x, sens, traj) / L
    yield plan, x, ref
    plan.destroy()


def test_full_size_spiral_normal_apply(pp, full_spiral):
    plan, x, ref = full_spiral
    out = empty(x.shape)
    pp.pp_normal_apply(plan, dev(x), out)
    assert rel(host(out), ref) <= TOL_APPLY


@pytest.mark.parametrize("row_variant,kind,cpc", [
    (1, 0, 8), (2, 0, 4), (4, 0, 16), (-1, 0, 32), (-1, 0, 2), (1, 1, 8), (2, 1, 3),
    (1, 2, 8), (-1, 3, 8), (2, 4, 8), (-1, 5, 8), (1, 6, 8), (-1, 6, 8), (1, 7, 8), (1, 8, 8), (4, 7, 8), (4, 8, 8), (1, 9, 8), (4, 9, 8)])
def test_full_size_spiral_every_launch_variant(pp, full_spiral, row_variant, kind, cpc):
    plan, x, ref = full_spiral
    tuned = pp.pp_plan_tuning(plan)
    try:
        pp.pp_plan_set_tuning(plan, row_variant, kind, cpc)
        assert pp.pp_plan_tuning(plan) == (row_variant, kind, cpc)
        out = empty(x.shape)
        pp.pp_normal_apply(plan, dev(x), out)
        assert rel(host(out), ref) <= TOL_APPLY
    finally:
        pp.pp_plan_set_tuning(plan, *tuned)
