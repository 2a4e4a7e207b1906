"""GPU parity of the Toeplitz-embedded normal operator: the exact F^H F of the
non-uniform DFT, evaluated through its Toeplitz structure (the remark on
Toeplitz normal operators in Sec. 2; the spiral experiment of Sec. 5.2),
against the oracle's exact-NDFT normal operator on the same seeded inputs.
Tolerances as for every operator: relative L2 <= 1e-5 per apply, <= 1e-4
after a solve."""
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


# (shape (ny, nx), coils, interleaves, samples): every supported side on rows
# and on columns, coil counts with a ragged last block of 8 and the full 32.
# Sides of register length (n = 128, 192, 256) run as two length-n halves,
# the others (n = 64, 96, 160) as one length-2n transform: both covered.
CASES = [((64, 64), 4, 8, 256), ((96, 128), 5, 8, 400), ((256, 160), 3, 8, 512),
         ((64, 256), 32, 6, 300), ((192, 96), 9, 8, 300), ((128, 192), 7, 6, 300)]
IDS = ["64_c4", "96x128_c5", "256x160_c3", "64x256_c32", "192x96_c9", "128x192_c7"]


class Case:
    def __init__(self, pp, shape, coils, inter, samples, seed=31):
        self.shape, self.C = shape, coils
        self.sens = synth.coil_maps(shape, coils, seed)
        self.traj = synth.spiral_traj(inter, samples, 3.0, min(shape) / 2.0)
        self.plan = pp.pp_plan_create(shape, coils, dev(self.sens), traj=self.traj, seed=seed,
                                      power_iters=0, toeplitz=True)
        self.normal = lambda v: O.nc_normal_exact(v, self.sens, self.traj)
        self.adj = lambda y: O.nc_adjoint(y, self.sens, self.traj)
        self.fwd = lambda x: O.nc_forward(x, self.sens, self.traj)


@pytest.fixture(scope="module", params=list(range(len(CASES))), ids=IDS)
def case(request, pp):
    c = Case(pp, *CASES[request.param])
    yield c
    c.plan.destroy()


def test_toeplitz_normal_parity(pp, case):
    x = synth.crandn(case.shape, 3)
    L = 0.731
    pp.pp_plan_set_scale(case.plan, L)
    out = empty(case.shape)
    pp.pp_normal_apply(case.plan, dev(x), out)
    assert rel(host(out), case.normal(x) / L) <= TOL_APPLY


def test_toeplitz_normal_is_hermitian(pp, case):
    x, y = synth.crandn(case.shape, 4), synth.crandn(case.shape, 5)
    pp.pp_plan_set_scale(case.plan, 1.0)
    nx_, ny_ = empty(case.shape), empty(case.shape)
    pp.pp_normal_apply(case.plan, dev(x), nx_)
    pp.pp_normal_apply(case.plan, dev(y), ny_)
    a = np.vdot(host(nx_), y.astype(np.complex128))
    b = np.vdot(x.astype(np.complex128), host(ny_))
    assert abs(a - b) <= 1e-5 * abs(a)


@pytest.mark.parametrize("d", [1, 3])
def test_toeplitz_poly_apply_parity(pp, d):
    c = Case(pp, *CASES[0])
    try:
        x = synth.crandn(c.shape, 6)
        L = float(O.power_iteration(c.normal, c.shape, 9, iters=10))
        pp.pp_plan_set_scale(c.plan, L)
        coef = [float(v) for v in O.poly_coeffs_l2(d)]
        out = empty(c.shape)
        pp.pp_poly_apply(c.plan, coef, d, dev(x), out)
        ref = O.horner_apply(coef, lambda v: c.normal(v) / L, x.astype(np.complex128))
        assert rel(host(out), ref) <= TOL_APPLY
    finally:
        c.plan.destroy()


def test_toeplitz_power_iteration_matches_oracle(pp):
    shape, coils, inter, samples = CASES[0]
    sens = synth.coil_maps(shape, coils, 31)
    traj = synth.spiral_traj(inter, samples, 3.0, min(shape) / 2.0)
    L_ref = O.power_iteration(lambda v: O.nc_normal_exact(v, sens, traj), shape, 77, iters=50)
    plan = pp.pp_plan_create(shape, coils, dev(sens), traj=traj, seed=77, power_iters=50,
                             toeplitz=True)
    try:
        L = pp.pp_plan_scale(plan)
    finally:
        plan.destroy()
    assert abs(L - L_ref) <= 1e-5 * L_ref


@pytest.mark.parametrize("d", [None, 3])
def test_toeplitz_solve_parity(pp, d):
    # the normal operator is the exact F^H F, A^H b the gridding adjoint (as
    # in the paper's Toeplitz experiment, Sec. 5.2)
    c = Case(pp, *CASES[0])
    try:
        x0 = synth.phantom(c.shape, 5)
        b = (c.fwd(x0) + synth.crandn((c.C, len(c.traj)), 6) * 1e-3).astype(np.complex64)
        L = float(O.power_iteration(c.normal, c.shape, 9, iters=30))
        pp.pp_plan_set_scale(c.plan, L)
        coef = None if d is None else [float(v) for v in O.poly_coeffs_l2(d)]
        ref = O.pfista(c.normal, c.adj, b.astype(np.complex128), 1e-3, coef, 12, L)
        out = empty(c.shape)
        pp.pp_fista_solve(c.plan, dev(b), 1e-3, 12, coef, 0 if d is None else d, out)
        assert rel(host(out), ref) <= TOL_SOLVE
    finally:
        c.plan.destroy()


def test_toeplitz_full_size_sampled_outputs(pp):
    # 256^2, 32 coils, 16 x 4096 spiral (the benchmark's workload): sampled
    # outputs, each computed one by one from the entries of F^H F
    cfg = synth.CONFIGS["spiral2d_256_c32"]
    shape, C = cfg["shape"], cfg["coils"]
    sens = synth.coil_maps(shape, C, cfg["seed"])
    traj = synth.spiral_traj(cfg["interleaves"], cfg["samples"], cfg["turns"], 128.0)
    plan = pp.pp_plan_create(shape, C, dev(sens), traj=traj, power_iters=0, toeplitz=True)
    grid_plan = pp.pp_plan_create(shape, C, dev(sens), traj=traj, power_iters=0)
    try:
        L = 123.0
        pp.pp_plan_set_scale(plan, L)
        pp.pp_plan_set_scale(grid_plan, L)
        x = synth.crandn(shape, 11)
        out, out_g = empty(shape), empty(shape)
        pp.pp_normal_apply(plan, dev(x), out)
        pp.pp_normal_apply(grid_plan, dev(x), out_g)
        got = host(out)
        g = np.random.default_rng(5)
        pix = [(0, 0), (0, 255), (255, 0), (255, 255), (128, 128), (127, 128)]
        pix += [tuple(int(v) for v in g.integers(0, 256, 2)) for _ in range(26)]
        ref = O.nc_normal_exact_at(x, sens, traj, pix) / L
        val = np.array([got[r, q] for r, q in pix])
        assert rel(val, ref) <= TOL_APPLY
        # the gridding operator approximates the exact one (W = 4, sigma = 1.25)
        assert rel(host(out_g), got) <= 1e-2
    finally:
        plan.destroy()
        grid_plan.destroy()
