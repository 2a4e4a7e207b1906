"""Plan set-up across plans of one process: a second plan with the same
geometry and sampling takes the launch shapes the first plan's tuner chose
(no timing runs) and computes the same operator as the oracle; a plan whose
trajectory differs is tuned on its own.  Parity of each plan's normal apply
against the FP64 oracle, relative L2 <= 1e-5."""
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


def apply_rel(pp, plan, x, ref):
    import torch
    out = torch.zeros(x.shape, dtype=torch.complex64, device="cuda")
    pp.pp_normal_apply(plan, dev(x), out)
    return rel(host(out), ref)


def test_second_plan_of_a_geometry_reuses_the_tuning(pp):
    shape, C, sigma = (96, 128), 32, 2.0
    sens = synth.coil_maps(shape, C, 701)
    traj = synth.spiral_traj(8, 1024, 4.0, 48.0)
    x = synth.crandn(shape, 702)
    ref = O.nc_normal(x, sens, traj, oversamp=sigma)
    plans = []
    try:
        for _ in range(2):
            plans.append(pp.pp_plan_create(shape, C, dev(sens), traj=traj, oversamp=sigma, power_iters=0))
        assert pp.pp_plan_tuning(plans[1]) == pp.pp_plan_tuning(plans[0])
        for p in plans:
            pp.pp_plan_set_scale(p, 1.0)
            assert apply_rel(pp, p, x, ref) <= TOL_APPLY
        # a caller's own launch shape on one plan leaves the other plan as tuned
        tuned = pp.pp_plan_tuning(plans[0])
        other = (1, 9, 8) if tuned != (1, 9, 8) else (4, 9, 8)
        pp.pp_plan_set_tuning(plans[0], *other)
        assert pp.pp_plan_tuning(plans[1]) == tuned
        assert apply_rel(pp, plans[0], x, ref) <= TOL_APPLY
        # a different trajectory is a different sampling: its plan is tuned
        # afresh and is still exact
        traj2 = synth.spiral_traj(8, 1024, 3.0, 48.0)
        ref2 = O.nc_normal(x, sens, traj2, oversamp=sigma)
        plans.append(pp.pp_plan_create(shape, C, dev(sens), traj=traj2, oversamp=sigma, power_iters=0))
        pp.pp_plan_set_scale(plans[2], 1.0)
        assert apply_rel(pp, plans[2], x, ref2) <= TOL_APPLY
    finally:
        for p in plans:
            p.destroy()


def test_second_3d_plan_reuses_the_tuning(pp):
    shape, C = (128, 128, 16), 3
    sens = synth.coil_maps(shape, C, 711)
    mask = synth.poisson_disc_mask(shape, 4, 8, 711)
    x = synth.crandn(shape, 712)
    ref = O.cart_normal(x, sens, mask)
    plans = []
    try:
        for _ in range(2):
            plans.append(pp.pp_plan_create(shape, C, dev(sens), mask=mask, power_iters=0))
        assert pp.pp_plan_tuning(plans[1]) == pp.pp_plan_tuning(plans[0])
        for p in plans:
            pp.pp_plan_set_scale(p, 1.0)
            assert apply_rel(pp, p, x, ref) <= TOL_APPLY
    finally:
        for p in plans:
            p.destroy()
