"""Secondary benchmark lines (bench.py --workload ...): the Cartesian 128^2
solve, the 3-D Cartesian normal operator, the batch of 64 uneven slices and
the differentiable unrolled solve.  Same timing rules as bench.py: warm-up,
CUDA events on the launching stream, L2 flushed between timed steps, clocks
sampled during the timed region, max over ranks."""
from __future__ import annotations

import math
import time

import numpy as np
import torch

import bench
import synth


def _flush_buf(dev):
    return torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)


def _timed(fn, steps, dev, local):
    """Total ms over `steps` calls of fn(), L2 flushed before each (outside
    the events), clocks sampled throughout."""
    stream = torch.cuda.current_stream()
    flush = _flush_buf(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    torch.cuda.synchronize()
    with bench.ClockSampler(local) as clk:
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            fn()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev), clk.summary()


def _hbm_peak():
    return bench.hbm_peak_gbs()


def _base(args, world, metric, unit, value, ms_per_step, cfg, clocks, extra=None):
    out = {"metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded); no datasets", "config": cfg, "clocks": clocks}
    if extra:
        out.update(extra)
    return out


def cart2d(args, pp, rank, world, local):
    c = dict(synth.CONFIGS["cart2d_128_c8"])
    dev = torch.device("cuda", local)
    seed = bench.replica_seed(c["seed"], rank)
    shape, C = c["shape"], c["coils"]
    sens = torch.from_numpy(synth.coil_maps(shape, C, seed)).to(dev)
    mask = synth.line_mask(shape, c["R"], c["acs"], seed)
    plan = pp.pp_plan_create(shape, C, sens, mask=mask, seed=seed, power_iters=50)
    x0 = torch.from_numpy(synth.phantom(shape, seed)).to(dev)
    b = torch.empty((C,) + shape, dtype=torch.complex64, device=dev)
    pp.pp_forward_apply(plan, x0, b)
    b += torch.from_numpy(synth.cnoise((C,) + shape, c["sigma"], seed + 1) * mask[None]).to(dev)
    coeffs = [float(v) for v in pp.pp_poly_coeffs_l2(c["d"])]
    xo = torch.empty(shape, dtype=torch.complex64, device=dev)
    run = lambda: pp.pp_fista_solve(plan, b, c["lam"], c["iters"], coeffs, c["d"], xo)
    for _ in range(args.warmup):
        run()
    ms, clk = _timed(run, args.steps, dev, local)
    ms = bench.max_over_ranks(ms, world, dev)
    applies = c["iters"] * (c["d"] + 1)
    xin = torch.from_numpy(synth.crandn(shape, 3)).to(dev)
    stages = pp.pp_profile_normal(plan, xin, torch.empty_like(xin), reps=100)
    apply_ms = sum(stages.values())
    bytes_apply = 8.0 * (C * shape[0] * shape[1] + 3 * shape[0] * shape[1])
    ttt = bench.time_to_target(pp, plan, b, c, coeffs, 0.0, torch.cuda.current_stream())
    plan.destroy()
    return _base(args, world, "A^H A applies/s (preconditioned FISTA, d=3, 40 iterations)", "applies/s",
                 bench.job_throughput(args.steps * applies, world, ms / 1e3), ms / args.steps,
                 {"workload": "cart2d_128_c8", "image": list(shape), "coils": C, "R": c["R"],
                  "d": c["d"], "iters": c["iters"], "l2": "flushed between timed steps"}, clk,
                 {"normal_apply_us": apply_ms * 1e3, "stage_ms_per_apply": stages,
                  "l2_resident_gbs": bytes_apply / (apply_ms / 1e3) / 1e9, "time_to_nrmse": ttt})


def cart3d(args, pp, rank, world, local):
    c = dict(synth.CONFIGS["cart3d_256x256x128_c32"])
    dev = torch.device("cuda", local)
    seed = bench.replica_seed(c["seed"], rank)
    shape, C = c["shape"], c["coils"]          # (nz, ny, nx)
    t0 = time.perf_counter()
    maps = synth.coil_maps(shape, C, seed)
    sens = torch.from_numpy(maps).to(dev)
    del maps
    mask = synth.poisson_disc_mask(shape, c["R"], c["calib"], seed)
    gen_s = time.perf_counter() - t0
    plan = pp.pp_plan_create(shape, C, sens, mask=mask, seed=seed, power_iters=0)
    x = torch.from_numpy(synth.crandn(shape, 3)).to(dev)
    y = torch.empty_like(x)
    run = lambda: pp.pp_normal_apply(plan, x, y)
    for _ in range(args.warmup):
        run()
    ms, clk = _timed(run, args.steps, dev, local)
    ms = bench.max_over_ranks(ms, world, dev)
    n = int(np.prod(shape))
    bytes_apply = 8.0 * (C * n + 3 * n)
    gbs = bytes_apply / (ms / args.steps / 1e3) / 1e9
    peak, src = _hbm_peak()
    stages = pp.pp_profile_normal(plan, x, y, reps=2)
    # FFT work per apply: per coil and x column, nz length-ny transforms and
    # ny pairs of length-nz transforms each way (5 N log2 N per transform)
    nz, ny, nx = shape
    fft = lambda N: 5.0 * N * math.log2(N)
    flops_apply = C * nx * 2.0 * (nz * fft(ny) + ny * fft(nz))
    tflops = flops_apply / (ms / args.steps / 1e3) / 1e12
    fp32_peak, fp32_src = bench.fp32_peak(dev, clk)
    # the 3-D Haar prox of the solve (2 levels, 4x4x4 tiles): one read and one
    # write of a 67 MB volume per call, HBM-bound.  Calls alternate between two
    # (input, output) pairs, 268 MB in all (twice the L2), back to back.
    x2 = torch.from_numpy(synth.crandn(shape, 4)).to(dev)
    y2 = torch.empty_like(x2)
    pairs = [(x, y), (x2, y2)]
    prox_calls = 20 * args.steps

    def prox_run():
        for i in range(prox_calls):
            xi, yi = pairs[i & 1]
            pp.pp_prox_l1_haar(shape, 2, float(c["lam"]), xi, yi)

    prox_run()
    prox_ms, _ = _timed(prox_run, 1, dev, local)
    prox_bytes = 16.0 * n
    prox_gbs = prox_bytes * prox_calls / (prox_ms / 1e3) / 1e9
    # the locally-low-rank prox of Sec. 5.3 on T = 5 coefficient images of the
    # volume (8^3 blocks: 512 x 5 complex matrices), alternating over two
    # input/output pairs (4 x 335 MB); lambda near the blocks' middle singular
    # values, so the threshold keeps some and drops others
    T_llr, lam_llr = 5, 20.0
    del x2, y2, pairs
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed + 7)
    llr_pairs = [(torch.randn(T_llr * n, dtype=torch.complex64, device=dev, generator=gen),
                  torch.empty(T_llr * n, dtype=torch.complex64, device=dev)) for _ in range(2)]
    llr_calls = 2 * args.steps

    def llr_run():
        for i in range(llr_calls):
            xi, yi = llr_pairs[i & 1]
            pp.pp_prox_llr(shape, T_llr, 8, lam_llr, xi, yi)

    llr_run()
    llr_ms, _ = _timed(llr_run, 1, dev, local)
    llr_bytes = 2.0 * 8 * T_llr * n
    llr_gbs = llr_bytes * llr_calls / (llr_ms / 1e3) / 1e9
    del llr_pairs
    tuning = pp.pp_plan_tuning(plan)
    plan.destroy()
    return _base(args, world, "A^H A applies/s (3-D Cartesian normal operator)", "applies/s",
                 bench.job_throughput(args.steps, world, ms / 1e3), ms / args.steps,
                 {"workload": "cart3d_256x256x128_c32", "image": list(shape), "coils": C, "R": c["R"],
                  "l2": "inputs larger than L2 (2 GiB of coil maps) and flushed between steps",
                  "input_generation_s": gen_s,
                  "tuning": {"row_variant": tuning[0], "coils_per_group": tuning[2],
                             "meaning": "3 = persistent dataflow kernel, 16/-16 = cluster kernel, "
                                        "1 = three passes per coil"}}, clk,
                 {"roofline": {"bound": "hbm", "kernel": "whole normal apply", "achieved": gbs,
                               "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                               "traffic": bench.ncu_traffic("cart3d_normal", "ncu_traffic_3d.json"),
                               "peak_source": src,
                               "algorithmic_bytes_per_apply": bytes_apply,
                               "fft_flops_per_apply": flops_apply, "tflops": tflops,
                               "fp32_peak": fp32_peak, "fp32_frac": tflops / fp32_peak,
                               "fp32_peak_source": fp32_src},
                  "stage_ms_per_apply": stages,
                  "prox": {"kernel": "prox3q_kernel", "bound": "hbm", "achieved": prox_gbs, "peak": peak,
                           "unit": "GB/s", "frac": prox_gbs / peak, "bytes_per_call": prox_bytes,
                           "ms_per_call": prox_ms / prox_calls,
                           "timing": "back-to-back calls alternating over two 67 MB input/output "
                                     "pairs (268 MB, larger than L2)"},
                  "llr_prox": {"kernel": "llr_prox_kernel", "images": T_llr, "block": 8, "lambda": lam_llr,
                               "bound": "alu", "achieved_gbs": llr_gbs, "hbm_peak": peak,
                               "hbm_frac": llr_gbs / peak, "bytes_per_call": llr_bytes,
                               "ms_per_call": llr_ms / llr_calls,
                               "timing": "back-to-back calls alternating over two 335 MB input/output "
                                         "pairs (1.3 GB, larger than L2); one-sided Jacobi SVD per "
                                         "512 x 5 block, instruction bound"}})


def batched(args, pp, rank, world, local):
    c = dict(synth.CONFIGS["batched2d_64"])
    dev = torch.device("cuda", local)
    slices = synth.batched_slices(c["n_slices"], bench.replica_seed(c["seed"], rank))
    shapes = [(ny, nx) for ny, nx, _, _ in slices]
    coils = [C for _, _, C, _ in slices]
    sens, masks = [], []
    for i, (ny, nx, C, R) in enumerate(slices):
        sens.append(torch.from_numpy(synth.coil_maps((ny, nx), C, c["seed"] + i)).to(dev))
        masks.append(synth.line_mask((ny, nx), R, c["acs"], c["seed"] + i))
    t0 = time.perf_counter()
    batch = pp.pp_batch_create(shapes, coils, sens, masks, seed=c["seed"], power_iters=50)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    xs = torch.cat([torch.from_numpy(synth.phantom(s, c["seed"] + 100 + i)).reshape(-1)
                    for i, s in enumerate(shapes)]).to(dev)
    b = torch.empty(int(batch.kspace_off[-1]), dtype=torch.complex64, device=dev)
    pp.pp_batch_forward_apply(batch, xs, b)
    coeffs = [float(v) for v in pp.pp_poly_coeffs_l2(c["d"])]
    xo = torch.empty(int(batch.image_off[-1]), dtype=torch.complex64, device=dev)
    run = lambda: pp.pp_batch_fista_solve(batch, b, c["lam"], c["iters"], coeffs, c["d"], xo)
    for _ in range(args.warmup):
        run()
    ms, clk = _timed(run, args.steps, dev, local)
    ms = bench.max_over_ranks(ms, world, dev)
    # one batched normal apply, timed alone
    y = torch.empty_like(xo)
    apply_ms, _ = _timed(lambda: pp.pp_batch_normal_apply(batch, xs, y), 20, dev, local)
    apply_ms /= 20
    nimg = int(batch.image_off[-1])
    bytes_apply = 8.0 * (sum(C * s[0] * s[1] for C, s in zip(coils, shapes)) + 3 * nimg)
    gbs = bytes_apply / (apply_ms / 1e3) / 1e9
    peak, src = _hbm_peak()
    tile, grid = pp.pp_batch_tile(batch)
    batch.destroy()
    applies = c["iters"] * (c["d"] + 1) * len(slices)
    return _base(args, world, "slice A^H A applies/s (64 uneven slices, d=3, 50 iterations)",
                 "slice-applies/s", bench.job_throughput(args.steps * applies, world, ms / 1e3),
                 ms / args.steps,
                 {"workload": "batched2d_64", "slices": len(slices), "image_elems": nimg,
                  "coil_map_bytes": 8 * sum(C * s[0] * s[1] for C, s in zip(coils, shapes)),
                  "d": c["d"], "iters": c["iters"], "l2": "inputs larger than L2; flushed between steps",
                  "autotuned_cols_per_cta": tile, "persistent_ctas": grid, "setup_s": setup_s}, clk,
                 {"roofline": {"bound": "hbm", "kernel": "cart2d_batch_normal_kernel (one launch per apply)",
                               "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                               "traffic": bench.ncu_traffic("cart2d_batch_normal", "ncu_traffic_batched.json"),
                               "peak_source": src,
                               "algorithmic_bytes_per_apply": bytes_apply},
                  "batched_apply_ms": apply_ms})


def unrolled(args, pp, rank, world, local):
    c = dict(synth.CONFIGS["unrolled2d_8x256_c16"])
    dev = torch.device("cuda", local)
    shape, C, B = c["shape"], c["coils"], c["batch"]
    sens = [torch.from_numpy(synth.coil_maps(shape, C, c["seed"] + i)).to(dev) for i in range(B)]
    masks = [synth.line_mask(shape, c["R"], c["acs"], c["seed"] + i) for i in range(B)]
    batch = pp.pp_batch_create([shape] * B, [C] * B, sens, masks, seed=c["seed"], power_iters=50)
    xs = torch.cat([torch.from_numpy(synth.phantom(shape, c["seed"] + 10 + i)).reshape(-1)
                    for i in range(B)]).to(dev)
    b = torch.empty(int(batch.kspace_off[-1]), dtype=torch.complex64, device=dev)
    pp.pp_batch_forward_apply(batch, xs, b)
    lam = torch.tensor(c["lam"], dtype=torch.float64, requires_grad=True)
    coeffs = torch.tensor([float(v) for v in pp.pp_poly_coeffs_l2(c["d"])], dtype=torch.float64,
                          requires_grad=True)
    bq = b.clone().requires_grad_(True)
    ybar = torch.from_numpy(synth.crandn((int(batch.image_off[-1]),), 5)).to(dev)

    def step():
        y = pp.unrolled_pfista(batch, bq, lam, coeffs, c["iters"], c["checkpoint"])
        loss = torch.sum((torch.conj(ybar) * y).real)
        loss.backward()

    for _ in range(args.warmup):
        step()
    ms, clk = _timed(step, args.steps, dev, local)
    ms = bench.max_over_ranks(ms, world, dev)
    batch.destroy()
    return _base(args, world, "unrolled solves/s (forward + backward, batch 8 x 256^2, 16 coils, 20 iterations, d=3)",
                 "fwd+bwd/s", bench.job_throughput(args.steps, world, ms / 1e3), ms / args.steps,
                 {"workload": "unrolled2d_8x256_c16", "batch": B, "image": list(shape), "coils": C,
                  "iters": c["iters"], "d": c["d"], "checkpoint_every": c["checkpoint"],
                  "l2": "flushed between timed steps"}, clk)


def apply_only(args, pp, local):
    """Profiling aid (--apply-only K): the workload's operator K times, no
    bench line.  cart2d: K normal applies; cart3d: the workload's volume with
    --apply-coils of its coils (4 by default: a capture small enough for
    ncu), K normal applies, then K
    3-D Haar prox calls, then K locally-low-rank prox calls on 5 images of the
    volume; batched2d_64: K batched normal applies (--tuning T
    forces the batch tile code T)."""
    dev = torch.device("cuda", local)
    K = args.apply_only
    if args.workload == "batched2d_64":
        c = dict(synth.CONFIGS["batched2d_64"])
        slices = synth.batched_slices(c["n_slices"], c["seed"])
        shapes = [(ny, nx) for ny, nx, _, _ in slices]
        sens = [torch.from_numpy(synth.coil_maps((ny, nx), C, c["seed"] + i)).to(dev)
                for i, (ny, nx, C, _) in enumerate(slices)]
        masks = [synth.line_mask((ny, nx), R, c["acs"], c["seed"] + i)
                 for i, (ny, nx, _, R) in enumerate(slices)]
        batch = pp.pp_batch_create(shapes, [C for _, _, C, _ in slices], sens, masks, seed=c["seed"],
                                   power_iters=0)
        if args.tuning:   # force the tile the plan-time tuner picks without a profiler attached
            pp.pp_batch_set_tile(batch, int(args.tuning))
        x = torch.from_numpy(synth.crandn((int(batch.image_off[-1]),), 3)).to(dev)
        y = torch.empty_like(x)
        for _ in range(K):
            pp.pp_batch_normal_apply(batch, x, y)
        torch.cuda.synchronize()
        batch.destroy()
        return {"apply_only": K, "workload": args.workload}
    c = dict(synth.CONFIGS[args.workload])
    shape, C = c["shape"], c["coils"]
    if len(shape) == 3:
        C = min(C, max(1, args.apply_coils))
    sens = torch.from_numpy(synth.coil_maps(shape, C, c["seed"])).to(dev)
    mask = (synth.line_mask(shape, c["R"], c["acs"], c["seed"]) if len(shape) == 2 else
            synth.poisson_disc_mask(shape, c["R"], c["calib"], c["seed"]))
    plan = pp.pp_plan_create(shape, C, sens, mask=mask, seed=c["seed"], power_iters=0)
    if args.tuning:   # force a launch shape (row_variant,stencil_kind,stencil_coils)
        pp.pp_plan_set_tuning(plan, *[int(v) for v in args.tuning.split(",")])
    x = torch.from_numpy(synth.crandn(shape, 3)).to(dev)
    y = torch.empty_like(x)
    for _ in range(K):
        pp.pp_normal_apply(plan, x, y)
    if len(shape) == 3:
        for _ in range(K):
            pp.pp_prox_l1_haar(shape, 2, float(c["lam"]), x, y)
        # the bench line's LLR prox case: 5 coefficient images, 8^3 blocks
        gen = torch.Generator(device=dev)
        gen.manual_seed(c["seed"] + 7)
        xl = torch.randn(5 * x.numel(), dtype=torch.complex64, device=dev, generator=gen)
        yl = torch.empty_like(xl)
        for _ in range(K):
            pp.pp_prox_llr(shape, 5, 8, 20.0, xl, yl)
    torch.cuda.synchronize()
    plan.destroy()
    return {"apply_only": K, "workload": args.workload}


def run(args, pp, rank, world, local):
    if args.apply_only:
        return apply_only(args, pp, local)
    return {"cart2d_128_c8": cart2d, "cart3d_256x256x128_c32": cart3d, "batched2d_64": batched,
            "unrolled2d_8x256_c16": unrolled}[args.workload](args, pp, rank, world, local)
