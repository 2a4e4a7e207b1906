"""GPU parity of the consensus-ADMM pieces (Algorithm "cadmm", Sec. 5.3):
pp_fista_solve_prox (the subproblem prox_{rho f_i}: data term, proximal term
sigma/2 ||x - v||^2, Haar or Daubechies-4 l1) against the oracle's
pfista_prox, and consensus ADMM over two coil-group plans on one GPU
against the oracle's consensus_admm on the same subproblems."""
import numpy as np
import pytest

import synth
from oracle import pp_oracle as O

pytestmark = pytest.mark.gpu

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


def cart(shape, C, seed, R=3):
    s = synth.coil_maps(shape, C, seed)
    m = synth.line_mask(shape, R, 8, seed)
    b = (O.cart_forward(synth.phantom(shape, seed), s, m) +
         m[None] * synth.cnoise((C,) + shape, 1e-3, seed + 1)).astype(np.complex64)
    return s, m, b


@pytest.mark.parametrize("case", ["cart_d3", "cart_plain", "spiral_d5", "no_data", "no_v", "db4"])
def test_prox_subproblem_matches_oracle(pp, case):
    import torch
    shape = (64, 48) if case != "spiral_d5" else (64, 64)
    C = 4
    if case == "spiral_d5":
        s = synth.coil_maps(shape, C, 5)
        traj = synth.spiral_traj(4, 512, 4.0, 31.9)
        fwd = lambda x: O.nc_forward(x, s, traj)
        adj = lambda y: O.nc_adjoint(y, s, traj)
        b = (fwd(synth.phantom(shape, 5)) + synth.cnoise((C, len(traj)), 1e-3, 6)).astype(np.complex64)
        plan = pp.pp_plan_create(shape, C, dev(s), traj=traj, power_iters=0)
    else:
        s, m, b = cart(shape, C, 7)
        fwd = lambda x: O.cart_forward(x, s, m)
        adj = lambda y: O.cart_adjoint(y, s, m)
        plan = pp.pp_plan_create(shape, C, dev(s), mask=m, power_iters=0)
    nrm = lambda x: adj(fwd(x))
    try:
        L = O.power_iteration(nrm, shape, 3, iters=20)
        pp.pp_plan_set_scale(plan, L)
        sigma, lam, iters = 0.4 * L, 2e-3, 25
        d = {"cart_d3": 3, "cart_plain": 0, "spiral_d5": 5, "no_data": 3, "no_v": 3, "db4": 3}[case]
        c = None if case == "cart_plain" else [float(v) for v in O.poly_coeffs_l2(d)]
        v = (0.3 * synth.crandn(shape, 8)).astype(np.complex64)
        bb = None if case == "no_data" else b
        vv = None if case == "no_v" else v
        wav = "db4" if case == "db4" else "haar"
        ref = O.pfista_prox(nrm, adj, None if bb is None else bb.astype(np.complex128),
                            None if vv is None else vv.astype(np.complex128), sigma, lam, c, iters, L,
                            wavelet=wav)
        out = torch.empty(shape, dtype=torch.complex64, device="cuda")
        r = pp.pp_fista_solve_prox(plan, None if bb is None else dev(bb), None if vv is None else dev(vv),
                                   sigma, lam, iters, c, d, out, history=True, wavelet=wav)
        assert rel(host(out), ref) <= TOL_SOLVE
        assert np.all(np.isfinite(r.history))
        # the graph cache is shared with pp_fista_solve: a normal solve in
        # between and the subproblem again give the same result
        if bb is not None:
            pp.pp_fista_solve(plan, dev(bb), lam, 5, c, d if c else 0, out)
            pp.pp_fista_solve_prox(plan, dev(bb), None if vv is None else dev(vv), sigma, lam, iters, c, d,
                                   out, wavelet=wav)
            assert rel(host(out), ref) <= TOL_SOLVE
    finally:
        plan.destroy()


def test_consensus_admm_two_coil_groups_on_one_gpu(pp):
    # 8 coils split into two 4-coil groups (two plans), the whole-problem
    # lambda split evenly, sigma = 1/rho; six ADMM iterations with 30
    # preconditioned (d = 3) inner iterations, against the oracle
    import torch
    from paper_2204_10252_gb300.admm import coil_group_prox, consensus_admm
    shape, C = (64, 64), 8
    s, m, b = cart(shape, C, 31, R=2)
    groups = [list(range(0, 4)), list(range(4, 8))]
    lam, iters_in, admm_iters, d = 2e-3, 30, 6, 3
    c = [float(v) for v in O.poly_coeffs_l2(d)]
    L = O.power_iteration(lambda x: O.cart_normal(x, s, m), shape, 3, iters=20)
    sigma = 0.5 * L
    plans, gprox, oprox = [], [], []
    try:
        for g in groups:
            ni = lambda x, g=g: O.cart_normal(x, s[g], m)
            ai = lambda y, g=g: O.cart_adjoint(y, s[g], m)
            Li = O.power_iteration(ni, shape, 4, iters=20)
            plan = pp.pp_plan_create(shape, len(g), dev(s[g]), mask=m, power_iters=0)
            pp.pp_plan_set_scale(plan, Li)
            plans.append(plan)
            gprox.append(coil_group_prox(plan, dev(b[g]), sigma, lam / len(groups), iters_in, c, d))
            oprox.append(lambda v, ni=ni, ai=ai, bi=b[g].astype(np.complex128), Li=Li:
                         O.pfista_prox(ni, ai, bi, v, sigma, lam / len(groups), c, iters_in, Li))
        hist = []
        xbar = consensus_admm(gprox, len(groups), admm_iters,
                              torch.zeros(shape, dtype=torch.complex64, device="cuda"), history=hist)
        ref_hist = []
        ref = O.consensus_admm(oprox, shape, admm_iters, history=ref_hist)
        assert rel(host(xbar), ref) <= TOL_SOLVE
        for h, rh in zip(hist, ref_hist):
            assert rel(host(h), rh) <= TOL_SOLVE
    finally:
        for p in plans:
            p.destroy()
