"""pp_adjoint_apply_static: the adjoint for callers that cannot allocate
device memory when they call (a plug-in whose host application owns all
device memory through its own pool, a real-time loop that forbids allocation
after start-up).  Its intermediates live in a fixed library-owned device
array; its output must equal the ordinary pp_adjoint_apply on the same
inputs, on two calls in a row (the array keeps the previous call's
contents), and calling it must leave the device's free memory unchanged.
This file is collected last so that a run stopping at the first failure has
run every other test before it."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL_APPLY = 1e-5


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


def cases(pp):
    out = []
    shape, C = (64, 48), 3
    sens = dev(synth.coil_maps(shape, C, 1))
    mask = synth.line_mask(shape, 3, 6, 1)
    out.append((pp.pp_plan_create(shape, C, sens, mask=mask, power_iters=0), sens,
                lambda s, C=C, shape=shape, mask=mask: synth.crandn((C,) + shape, s) * mask[None],
                shape))
    shape, C = (64, 64), 4
    sens = dev(synth.coil_maps(shape, C, 2))
    traj = synth.spiral_traj(4, 512, 4.0, 32.0)
    out.append((pp.pp_plan_create(shape, C, sens, traj=traj, power_iters=0), sens,
                lambda s, C=C, traj=traj: synth.crandn((C, len(traj)), s), shape))
    shape, C = (16, 24, 20), 2
    sens = dev(synth.coil_maps(shape, C, 3))
    mask = synth.poisson_disc_mask(shape, 3, 4, 3)
    out.append((pp.pp_plan_create(shape, C, sens, mask=mask, power_iters=0), sens,
                lambda s, C=C, shape=shape, mask=mask: synth.crandn((C,) + shape, s) * mask[None],
                shape))
    return out


def test_static_adjoint_matches_allocating_adjoint_twice(pp):
    import torch
    for plan, _sens, draw, shape in cases(pp):
        try:
            for call in range(2):
                y = dev(draw(100 + call))
                ref = torch.empty(shape, dtype=torch.complex64, device="cuda")
                got = torch.empty_like(ref)
                pp.pp_adjoint_apply(plan, y, ref)
                pp.pp_adjoint_apply_static(plan, y, got)
                torch.cuda.synchronize()
                r = ref.cpu().numpy().astype(np.complex128)
                g = got.cpu().numpy().astype(np.complex128)
                assert np.linalg.norm(g - r) <= TOL_APPLY * np.linalg.norm(r)
        finally:
            plan.destroy()


def test_static_adjoint_leaves_free_device_memory_unchanged(pp):
    # after one warm call (the first call on a device looks the array up and
    # may make the runtime commit it), further calls allocate nothing: the
    # device's free memory and torch's allocator are the same before and
    # after, while the output is still correct
    import torch
    for plan, _sens, draw, shape in cases(pp):
        try:
            y = dev(draw(7))
            ref = torch.empty(shape, dtype=torch.complex64, device="cuda")
            got = torch.empty_like(ref)
            pp.pp_adjoint_apply(plan, y, ref)
            pp.pp_adjoint_apply_static(plan, y, got)
            torch.cuda.synchronize()
            free0, _ = torch.cuda.mem_get_info()
            alloc0 = torch.cuda.memory_allocated()
            for _ in range(5):
                pp.pp_adjoint_apply_static(plan, y, got)
            torch.cuda.synchronize()
            free1, _ = torch.cuda.mem_get_info()
            assert free1 == free0
            assert torch.cuda.memory_allocated() == alloc0
            r = ref.cpu().numpy().astype(np.complex128)
            g = got.cpu().numpy().astype(np.complex128)
            assert np.linalg.norm(g - r) <= TOL_APPLY * np.linalg.norm(r)
        finally:
            plan.destroy()


def test_static_adjoint_rejects_plans_above_the_limit(pp):
    shape, C = (256, 256), 16         # 8 * 16 * 320 * (256 + 320) bytes = 23.6 MB > 16 MiB
    sens = dev(synth.coil_maps(shape, C, 4))
    traj = synth.spiral_traj(2, 256, 2.0, 100.0)
    plan = pp.pp_plan_create(shape, C, sens, traj=traj, power_iters=0)
    try:
        import torch
        y = dev(synth.crandn((C, len(traj)), 5))
        x = torch.empty(shape, dtype=torch.complex64, device="cuda")
        with pytest.raises(pp.PPError) as e:
            pp.pp_adjoint_apply_static(plan, y, x)
        assert e.value.status == 2 and "16 MiB" in str(e.value)
    finally:
        plan.destroy()
