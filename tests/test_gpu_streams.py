"""Every entry point on a caller's non-blocking stream.  Each call's inputs
(coil maps included, for plan creation) are written on that stream behind a
long device-side spin, so a step that the library ran on another stream
(the legacy default stream, or its own capture stream) would read them
before they exist.  Results equal those of the same calls on the default
stream (bit for bit where the path has a fixed summation order) and the FP64
oracle (relative L2 <= 1e-5 per apply)."""
import numpy as np
import pytest

import synth
from oracle import pp_oracle as O

pytestmark = pytest.mark.gpu

TOL_APPLY = 1e-5
SPIN = 50_000_000   # device clock cycles of the spin before each input write


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.complex128) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def pp():
    from paper_2204_10252_gb300.build import build_library
    build_library()
    import paper_2204_10252_gb300 as m
    m.lib()
    return m


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


def late(a, stream):
    """A device copy of `a` whose write is queued on `stream` after a spin."""
    import torch
    src = torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)).pin_memory()
    with torch.cuda.stream(stream):
        torch.cuda._sleep(SPIN)
        out = torch.empty(src.shape, dtype=src.dtype, device="cuda")
        out.copy_(src, non_blocking=True)
    return out


def on(stream, fn):
    import torch
    with torch.cuda.stream(stream):
        r = fn()
    stream.synchronize()
    return r


CASES = [
    ("cart2d", (64, 48), 3, dict(R=3, acs=6)),
    ("cart3d_dataflow", (128, 128, 8), 3, dict(R=4, calib=8)),
    ("spiral", (64, 64), 5, dict(oversamp=2.0)),
    ("toeplitz", (64, 64), 4, dict(oversamp=1.25)),
]


@pytest.mark.parametrize("case", range(len(CASES)), ids=[c[0] for c in CASES])
def test_plan_and_applies_on_a_side_stream(pp, case):
    import torch
    name, shape, C, kw = CASES[case]
    s = torch.cuda.Stream()
    sens = synth.coil_maps(shape, C, 1200 + case)
    x = synth.crandn(shape, 1210 + case)
    if name.startswith("cart"):
        mask = (synth.line_mask(shape, kw["R"], kw["acs"], 1220 + case) if len(shape) == 2 else
                synth.poisson_disc_mask(shape, kw["R"], kw["calib"], 1220 + case))
        mk = lambda st, sd: pp.pp_plan_create(shape, C, sd, mask=mask, seed=3, power_iters=20, stream=st)
        normal = lambda v: O.cart_normal(v, sens, mask)
        fwd = lambda v: O.cart_forward(v, sens, mask)
        kshape = (C,) + shape
        exact = True
    else:
        traj = synth.spiral_traj(4, 512, 3.0, shape[0] / 2.0 - 0.1)
        toep = name == "toeplitz"
        mk = lambda st, sd: pp.pp_plan_create(shape, C, sd, traj=traj, oversamp=kw["oversamp"], seed=3,
                                              power_iters=20, stream=st, toeplitz=toep)
        normal = ((lambda v: O.nc_normal_exact(v, sens, traj)) if toep else
                  (lambda v: O.nc_normal(v, sens, traj, oversamp=kw["oversamp"])))
        fwd = lambda v: O.nc_forward(v, sens, traj, oversamp=kw["oversamp"])
        kshape = (C, len(traj))
        exact = True
    # the plan made on the side stream from maps written there late, and a
    # reference plan on the default stream
    side = mk(s, late(sens, s))
    s.synchronize()
    ref_sens = torch.from_numpy(sens.astype(np.complex64)).cuda()
    base = mk(None, ref_sens)
    try:
        assert pp.pp_plan_scale(side) == pp.pp_plan_scale(base)
        L = pp.pp_plan_scale(base)
        want = normal(x) / L
        # normal apply
        y_side = torch.zeros(shape, dtype=torch.complex64, device="cuda")
        xs = late(x, s)
        on(s, lambda: pp.pp_normal_apply(side, xs, y_side))
        y_base = torch.zeros_like(y_side)
        pp.pp_normal_apply(base, torch.from_numpy(x.astype(np.complex64)).cuda(), y_base)
        got, ref = host(y_side), host(y_base)
        assert rel(got, want) <= TOL_APPLY
        if exact:
            assert np.array_equal(got, ref)
        # forward apply
        k_side = torch.zeros(kshape, dtype=torch.complex64, device="cuda")
        xs = late(x, s)
        on(s, lambda: pp.pp_forward_apply(side, xs, k_side))
        assert rel(host(k_side), fwd(x)) <= TOL_APPLY
        # Horner polynomial
        c = [float(v) for v in O.poly_coeffs_l2(3)]
        p_side = torch.zeros(shape, dtype=torch.complex64, device="cuda")
        xs = late(x, s)
        on(s, lambda: pp.pp_poly_apply(side, c, 3, xs, p_side))
        wantp = O.horner_apply(c, lambda v: normal(v) / L, x.astype(np.complex128))
        assert rel(host(p_side), wantp) <= TOL_APPLY
    finally:
        side.destroy()
        base.destroy()


@pytest.mark.parametrize("case", [0, 2], ids=["cart2d", "spiral"])
def test_solve_on_a_side_stream(pp, case):
    import torch
    name, shape, C, kw = CASES[case]
    s = torch.cuda.Stream()
    sens = synth.coil_maps(shape, C, 1300 + case)
    sens_t = torch.from_numpy(sens.astype(np.complex64)).cuda()
    if name == "cart2d":
        mask = synth.line_mask(shape, kw["R"], kw["acs"], 1310)
        plan = pp.pp_plan_create(shape, C, sens_t, mask=mask, seed=3, power_iters=30)
        b = (O.cart_forward(synth.phantom(shape, 1320), sens, mask) +
             1e-3 * synth.crandn((C,) + shape, 1321) * mask[None]).astype(np.complex64)
    else:
        traj = synth.spiral_traj(4, 512, 3.0, shape[0] / 2.0 - 0.1)
        plan = pp.pp_plan_create(shape, C, sens_t, traj=traj, oversamp=kw["oversamp"], seed=3,
                                 power_iters=30)
        b = (O.nc_forward(synth.phantom(shape, 1320), sens, traj, oversamp=kw["oversamp"]) +
             1e-3 * synth.crandn((C, len(traj)), 1321)).astype(np.complex64)
    try:
        c = [float(v) for v in O.poly_coeffs_l2(3)]
        out_side = torch.zeros(shape, dtype=torch.complex64, device="cuda")
        bs = late(b, s)
        r_side = on(s, lambda: pp.pp_fista_solve(plan, bs, 1e-3, 12, c, 3, out_side, history=True))
        out_base = torch.zeros_like(out_side)
        r_base = pp.pp_fista_solve(plan, torch.from_numpy(b).cuda(), 1e-3, 12, c, 3, out_base,
                                   history=True)
        got, ref = host(out_side), host(out_base)
        if name == "cart2d":
            # no atomics on the Cartesian path: the same bits on either stream
            assert np.array_equal(got, ref)
            assert np.array_equal(r_side.history, r_base.history)
        else:
            # the spiral adjoint spreads with shared-memory atomics
            assert rel(got, ref) <= 1e-5
            assert np.allclose(r_side.history, r_base.history, rtol=1e-4, atol=0)
    finally:
        plan.destroy()


def test_batch_and_prox_on_a_side_stream(pp):
    import torch
    s = torch.cuda.Stream()
    slices = [((32, 48), 3, 3), ((64, 64), 5, 4)]
    shapes = [sh for sh, _, _ in slices]
    coils = [cc for _, cc, _ in slices]
    sens = [synth.coil_maps(sh, cc, 1400 + i) for i, (sh, cc, _) in enumerate(slices)]
    masks = [synth.line_mask(sh, R, 4, 1410 + i) for i, (sh, _, R) in enumerate(slices)]
    b = on(s, lambda: pp.pp_batch_create(shapes, coils, [late(v, s) for v in sens], masks, seed=5,
                                         power_iters=20, stream=s))
    try:
        Ls = pp.pp_batch_scales(b)
        for i, sh in enumerate(shapes):
            ref = O.power_iteration(lambda v: O.cart_normal(v, sens[i], masks[i]), sh, 5 + i, iters=20)
            assert abs(Ls[i] - ref) <= 1e-5 * ref
        xs = [synth.crandn(sh, 1420 + i) for i, sh in enumerate(shapes)]
        x = late(np.concatenate([v.ravel() for v in xs]), s)
        y = torch.zeros(x.shape, dtype=torch.complex64, device="cuda")
        on(s, lambda: pp.pp_batch_normal_apply(b, x, y))
        got = host(y)
        off = b.image_off
        for i, sh in enumerate(shapes):
            ref = O.cart_normal(xs[i], sens[i], masks[i]) / Ls[i]
            assert rel(got[off[i]:off[i + 1]].reshape(sh), ref) <= TOL_APPLY
    finally:
        b.destroy()
    # the standalone proxes
    v = synth.crandn((64, 48), 1430)
    vin = late(v, s)
    out = torch.zeros((64, 48), dtype=torch.complex64, device="cuda")
    on(s, lambda: pp.pp_prox_l1_haar((64, 48), 2, 0.3, vin, out))
    assert rel(host(out), O.prox_l1_haar(v, 0.3, 2)) <= TOL_APPLY
    stack = synth.crandn((3, 16, 16, 16), 1440)
    sin = late(stack, s)
    out3 = torch.zeros((3, 16, 16, 16), dtype=torch.complex64, device="cuda")
    on(s, lambda: pp.pp_prox_llr((16, 16, 16), 3, 8, 2.0, sin, out3))
    assert rel(host(out3), O.prox_llr(stack, 2.0, 8)) <= TOL_APPLY


def test_plans_used_from_concurrent_host_threads(pp):
    # Three plans, each with its own stream: made and first solved one after
    # the other (the first solve captures the plan's CUDA graph, and CUDA
    # forbids a device-wide synchronisation in any thread while a capture
    # is open), then used by three host threads at once -- applies, solves
    # (graph replays) and second plans of the same geometry made while the
    # other threads compute.  Each thread synchronises only its own stream.
    # The results equal the serial run's bits (no atomics on this path).
    import threading
    import torch
    specs = [((64, 48), 3, 1500), ((48, 64), 4, 1501), ((64, 64), 2, 1502)]
    c = [float(v) for v in O.poly_coeffs_l2(3)]
    st = {}
    for shape, C, seed in specs:
        s = torch.cuda.Stream()
        sens = synth.coil_maps(shape, C, seed)
        mask = synth.line_mask(shape, 3, 6, seed)
        b = (O.cart_forward(synth.phantom(shape, seed), sens, mask) +
             1e-3 * synth.crandn((C,) + shape, seed + 1) * mask[None]).astype(np.complex64)
        with torch.cuda.stream(s):
            sd = torch.from_numpy(sens.astype(np.complex64)).cuda()
            plan = pp.pp_plan_create(shape, C, sd, mask=mask, seed=seed, power_iters=30)
            x = torch.from_numpy(synth.crandn(shape, seed + 2).astype(np.complex64)).cuda()
            bd = torch.from_numpy(b).cuda()
        st[seed] = dict(s=s, sd=sd, mask=mask, plan=plan, x=x, b=bd, shape=shape, C=C)

    def run(seed, out, errors, make_second):
        try:
            d = st[seed]
            s = d["s"]
            with torch.cuda.stream(s):
                y = torch.zeros_like(d["x"])
                for _ in range(20):
                    pp.pp_normal_apply(d["plan"], d["x"], y)
                xo = torch.zeros_like(d["x"])
                pp.pp_fista_solve(d["plan"], d["b"], 1e-3, 15, c, 3, xo)
                L2 = None
                if make_second:
                    second = pp.pp_plan_create(d["shape"], d["C"], d["sd"], mask=d["mask"], seed=seed,
                                               power_iters=30)
                    L2 = pp.pp_plan_scale(second)
                    d.setdefault("extra", []).append(second)
                s.synchronize()
                out[seed] = (y.cpu().numpy(), xo.cpu().numpy(), L2)
                s.synchronize()
        except Exception as e:   # reported by the main thread
            errors.append(repr(e))

    try:
        serial, errors = {}, []
        for _, _, seed in specs:
            run(seed, serial, errors, False)
        assert not errors, errors
        for rep in range(2):
            conc = {}
            threads = [threading.Thread(target=run, args=(seed, conc, errors, rep == 1))
                       for _, _, seed in specs]
            for t in threads:
                t.start()
            for t in threads:
                t.join()
            assert not errors, errors
            for _, _, seed in specs:
                y, xo, _ = serial[seed]
                y2, xo2, L2 = conc[seed]
                assert np.array_equal(y2, y) and np.array_equal(xo2, xo), (rep, seed)
                if L2 is not None:
                    assert L2 == pp.pp_plan_scale(st[seed]["plan"]), (rep, seed)
    finally:
        torch.cuda.synchronize()
        for d in st.values():
            for q in d.get("extra", []):
                q.destroy()
            d["plan"].destroy()
