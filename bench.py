#!/usr/bin/env python
"""Benchmark of polynomial-preconditioned FISTA (Algorithm "pfista").

Workload (2-D non-Cartesian SENSE): 256x256 complex64 image, 32 coils,
16-interleave Archimedean spiral with 4096 samples per interleave,
Kaiser-Bessel gridding (width 4, oversampling 1.25), 2-level Haar l1 with
lambda = 5e-4, degree-5 l2-optimal polynomial, 100 iterations.  Synthetic
seeded inputs (random-ellipse phantom, smooth coil maps, complex Gaussian
noise sigma = 1e-3).

One step = one pp_fista_solve call: A^H b, then 100 iterations of
(d+1) = 6 normal-operator applies, the fused Haar prox and the momentum
update, captured as one CUDA graph.  Metric: A^H A applies per second
(whole job).  The plan (coil maps, trajectory, the 50-step power iteration)
is built before the timed region and reported separately as setup time.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 run under torch.distributed.run: each rank solves its own
independent problem (a different seed); no collective touches the data path.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = "spiral2d_256_c32"
METRIC = "A^H A applies/s (preconditioned FISTA solve, d=5, 100 iterations)"
UNIT = "applies/s"
FP32_LANES_PER_SM = 128   # FP32 FMA lanes per SM on this architecture (4 x 32)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["pp", "reference"], default="pp")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip time-to-NRMSE, e2e, CPU baseline (quick runs)")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "cart2d_128_c8", "cart3d_256x256x128_c32", "batched2d_64",
                             "unrolled2d_8x256_c16"],
                    help="benchmark line to produce (the default is the headline workload)")
    ap.add_argument("--poly", choices=["l2", "cheb"], default="l2",
                    help="spiral workload: the preconditioner, Eq. l2cost (default) or the Chebyshev "
                         "minimax design of Sec. 3.4 with mu estimated by pp_plan_mu (set-up time "
                         "includes that estimate)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the 3-D and batched lines that the default run appends")
    ap.add_argument("--apply-only", type=int, default=0, metavar="K",
                    help="profiling aid: build the workload's plan (no power iteration), apply "
                         "its operator K times and exit without a bench line")
    ap.add_argument("--apply-coils", type=int, default=4, metavar="C",
                    help="with --apply-only on the 3-D workload: how many of its coils the "
                         "capture case keeps (default 4; 32 is the whole workload, 2 GiB of maps)")
    ap.add_argument("--tuning", default="",
                    help="with --apply-only: row_ifft_variant,stencil_kind,stencil_coils to force "
                         "(batched2d_64: the batch tile code)")
    ap.add_argument("--wavelet", choices=["haar", "db4"], default="haar",
                    help="spiral workload: W of the prox, the 2-level Haar or the Daubechies-4 "
                         "(the paper's choice)")
    ap.add_argument("--operator", choices=["gridding", "toeplitz"], default="gridding",
                    help="spiral workload: the gridding normal operator (G^T G stencil) or the "
                         "exact F^H F through its Toeplitz embedding")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cfg():
    return dict(synth.CONFIGS[WORKLOAD])


def replica_seed(base, rank):
    """Each rank solves an independent problem instance of the same shape."""
    return base + 1000 * rank


def max_over_ranks(value, world, device=None):
    """Largest `value` over all ranks (the job's time is its slowest rank)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, max_seconds):
    """Units all ranks processed divided by the slowest rank's time."""
    return world * units_per_rank / max_seconds


def make_inputs(c, rank):
    """Host-side synthetic inputs for one replica (seed offset by rank)."""
    seed = replica_seed(c["seed"], rank)
    shape, C = c["shape"], c["coils"]
    sens = synth.coil_maps(shape, C, seed)
    traj = synth.spiral_traj(c["interleaves"], c["samples"], c["turns"], shape[0] / 2.0)
    x_true = synth.phantom(shape, seed)
    noise = synth.cnoise((C, len(traj)), c["sigma"], seed + 1)
    return seed, sens, traj, x_true, noise


# ---------------------------------------------------------------------------
# clocks (nvidia-smi sampled during the timed region)
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline bookkeeping: algorithmic FLOPs per launch of each normal-operator
# kernel (conventional 5 N log2 N per complex FFT of length N)
# ---------------------------------------------------------------------------
def kernel_flops(c, K, toeplitz=False):
    ny, nx = c["shape"]
    C = c["coils"]
    G = int(math.ceil(c["oversamp"] * nx))
    n = nx * ny
    fft = lambda N: 5.0 * N * math.log2(N)
    W = c["kb_width"]
    if toeplitz:
        # rows: ny length-2nx FFTs per coil; columns: 2nx pairs of length-2ny
        # FFTs per coil plus the real spectrum product
        Mx, My = 2 * nx, 2 * ny
        return {
            "ci_rows_fwd_kernel": C * ny * fft(Mx) + 6.0 * C * n,
            "toep_cols_kernel": C * Mx * 2 * fft(My) + 2.0 * C * Mx * My,
            "ci_rows_inv_cl_kernel": C * ny * fft(Mx) + 8.0 * C * n + 4.0 * n,
            # the same rows as two length-nx halves (the algorithmic count stays that of
            # the length-2nx transform, so the two forms compare directly)
            "toep_rows_fwd_half_kernel": C * ny * fft(Mx) + 6.0 * C * n,
            "toep_cols_half_kernel": C * Mx * 2 * fft(My) + 2.0 * C * Mx * My,
            "toep_rows_inv_half_cl_kernel": C * ny * fft(Mx) + 8.0 * C * n + 4.0 * n,
        }
    return {
        "rows_fwd_kernel": C * ny * fft(G) + 8.0 * C * n,
        "cols_kernel": C * G * fft(G),
        # G^T G stencil: (2W-1)^2 complex-by-real multiply-adds per grid point and coil
        "gtg_stencil_kernel": 4.0 * (2 * W - 1) ** 2 * C * G * G,
        "gtg_stencil2_kernel": 4.0 * (2 * W - 1) ** 2 * C * G * G,
        "gtg_stencil_rb_kernel": 4.0 * (2 * W - 1) ** 2 * C * G * G,
        "gtg_stencil_cl_kernel": 4.0 * (2 * W - 1) ** 2 * C * G * G,
        "coil_sum_kernel": 2.0 * C * n,
        "ci_rows_fwd_kernel": C * ny * fft(G) + 8.0 * C * n,
        "ci_cols_kernel": C * G * fft(G),
        "ci_stencil_kernel": 4.0 * (2 * W - 1) ** 2 * C * G * G,
        "ci_rows_inv_kernel": C * ny * fft(G) + 10.0 * C * n,
        "ci_rows_inv_cl_kernel": C * ny * fft(G) + 10.0 * C * n,
        "ci_sum_kernel": 4.0 * 2.0 * n,
        "rows_adj_cb_kernel": C * ny * fft(G) + 10.0 * C * n,
        "rows_adj_kernel": C * ny * fft(G) + 10.0 * C * n,
        "rows4_fwd_kernel": C * ny * fft(G) + 8.0 * C * n,
        "cols4_kernel": C * G * fft(G),
        "rows4_adj_kernel": C * ny * fft(G) + 10.0 * C * n,
        "rows4_adj_cl_kernel": C * ny * fft(G) + 10.0 * C * n,
        "rows4_inv_kernel": C * ny * fft(G) + 8.0 * C * n,
    }


def fp32_peak(dev, clocks):
    """FP32 CUDA-core peak of this device: SMs (from the device) x 128 FMA
    lanes x 2 flop x the median SM clock sampled during the timed region
    (the maximum clock when no sample was taken)."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz")
    src = "median SM clock sampled during the timed region"
    if not mhz:
        mhz, src = 2070.0, "maximum SM clock (no clock samples)"
    peak = sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    return peak, "derived: %d SMs x %d FP32 lanes x 2 flop/FMA x %.0f MHz (%s)" % (
        sms, FP32_LANES_PER_SM, mhz, src)


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of this machine's GPUs, else the fallback."""
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s"


def csrc_digest(files=None):
    """Digest of the kernel sources: the named files of csrc/ (the kernel's
    translation unit and the headers it includes), or all of csrc/."""
    d = os.path.join(ROOT, "paper_2204_10252_gb300", "csrc")
    paths = ([os.path.join(d, f) for f in sorted(files)] if files else
             sorted(glob.glob(os.path.join(d, "*"))))
    h = hashlib.sha256()
    for f in paths:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, summary="ncu_traffic.json"):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, or
    None when missing or taken on different kernel sources (the digest covers
    the files the summary lists in csrc_files, else all of csrc/)."""
    p = os.path.join(ROOT, "profiles", summary)
    try:
        d = json.load(open(p))
    except Exception:
        return None
    e = d.get("kernels", {}).get(kernel)
    try:
        same = d.get("csrc_sha") == csrc_digest(d.get("csrc_files"))
    except OSError:
        same = False
    if not e or not same:
        return None
    return e.get("dram_bytes_per_launch")


EXACT_SAMPLES = 4096
_SAMPLE = {}


def _sample_init(seed_rank, exact):
    """Worker start-up: the replica's inputs, generated in the worker."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    c = cfg()
    _, sens, traj, _, _ = make_inputs(c, seed_rank)
    _SAMPLE.update(c=c, sens=sens, traj=traj, exact=exact)


def _sample_run(coils):
    return oracle_sample(_SAMPLE["c"], _SAMPLE["sens"], _SAMPLE["traj"], coils, _SAMPLE["exact"])


def oracle_sample(c, sens, traj, coils, exact=False):
    """One bounded sample of the workload on the FP64 oracle: the normal
    operator restricted to the first `coils` coils (a fraction coils/C of one
    full A^H A apply); for the exact (Toeplitz-evaluated) operator, one coil
    and the first EXACT_SAMPLES samples, whose direct sums cost a fraction
    (1/C)(EXACT_SAMPLES/K) of the full apply.  Returns (seconds, fraction)."""
    from oracle import pp_oracle as O
    x = synth.crandn(c["shape"], 3).astype(np.complex128)
    t0 = time.perf_counter()
    if exact:
        O.nc_normal_exact(x, sens[:1], traj[:EXACT_SAMPLES])
        return time.perf_counter() - t0, EXACT_SAMPLES / float(len(traj) * c["coils"])
    O.nc_normal(x, sens[:coils], traj, c["kb_width"], c["oversamp"])
    return time.perf_counter() - t0, coils / float(c["coils"])


class OraclePool:
    """The oracle as it stands on every host core: one spawned worker per
    core (numpy's FFT and scatter-add are single-threaded, so workers are the
    way to use the cores), each running bounded samples of the workload."""

    def __init__(self, exact=False, workers=None):
        import multiprocessing as mp
        self.cores = int(workers or os.cpu_count() or 1)
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_sample_init,
                                                 initargs=(0, exact))
        self.pool.map(_sample_run, [1] * self.cores)   # start-up and first touch, untimed

    def step(self, coils):
        """One concurrent sample per worker: (wall seconds, full applies done)."""
        t0 = time.perf_counter()
        res = self.pool.map(_sample_run, [coils] * self.cores)
        return time.perf_counter() - t0, sum(f for _, f in res)

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(c, budget_s=15.0, coils=2, exact=False):
    """The oracle as it stands, timed on all host cores on ~budget_s of
    bounded samples; reported in full-apply units."""
    op = OraclePool(exact)
    try:
        el, frac, n = 0.0, 0.0, 0
        while el < budget_s:
            t, f = op.step(coils)
            el += t
            frac += f
            n += 1
    finally:
        op.close()
    if exact:
        what = ("%d rounds of %d concurrent samples (one per host core), each the exact-NDFT A^H A "
                "of 1 of the 32 coils over the first %d of the 65536 spiral samples (256x256) on the "
                "numpy FP64 oracle (direct sums), scaled to full applies" % (n, op.cores, EXACT_SAMPLES))
    else:
        what = ("%d rounds of %d concurrent samples (one worker process per host core), each the "
                "A^H A apply of %d of the 32 coils (256x256, 65536-sample spiral) on the numpy FP64 "
                "oracle, scaled to full applies" % (n, op.cores, coils))
    return {"value": frac / el, "unit": UNIT, "cores": op.cores, "kind": "oracle", "sample": what}


# ---------------------------------------------------------------------------
# reference arm: the oracle as it stands, timed on the host cores
# ---------------------------------------------------------------------------
def run_reference(args, rank, world, coils=2):
    if rank != 0:
        return
    op = OraclePool()
    try:
        for _ in range(args.warmup):
            op.step(coils)
        el, frac = 0.0, 0.0
        for _ in range(args.steps):
            t, f = op.step(coils)
            el += t
            frac += f
    finally:
        op.close()
    v = frac / el
    sample = ("each step is one A^H A apply of %d of the 32 coils (256x256, 65536-sample spiral) per "
              "host core, %d worker processes running concurrently, on the numpy FP64 oracle, scaled "
              "to full applies" % (coils, op.cores))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": op.cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    rank, world, local = dist_env()
    import torch
    import torch.distributed as dist

    if world > 1:
        backend = "nccl" if (args.impl == "pp" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    if args.impl == "reference":
        run_reference(args, rank, world)
        if world > 1:
            dist.destroy_process_group()
        return

    import paper_2204_10252_gb300 as pp
    from paper_2204_10252_gb300.build import build_library
    build_library()
    pp.lib()
    torch.cuda.set_device(local)
    if args.workload != WORKLOAD:
        import bench_workloads
        out = bench_workloads.run(args, pp, rank, world, local)
        if rank == 0:
            print(json.dumps(out))
        if world > 1:
            dist.destroy_process_group()
        return
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    c = cfg()
    if args.apply_only:
        # one plan, a forced launch shape, K normal-operator applies: a small,
        # deterministic launch sequence for an ncu capture of one apply
        sens = synth.coil_maps(c["shape"], c["coils"], c["seed"])
        traj = synth.spiral_traj(c["interleaves"], c["samples"], c["turns"], c["shape"][1] / 2.0)
        plan = pp.pp_plan_create(c["shape"], c["coils"], torch.from_numpy(sens).to(dev), traj=traj,
                                 kb_width=c["kb_width"], oversamp=c["oversamp"], power_iters=0,
                                 toeplitz=args.operator == "toeplitz")
        if args.tuning:
            pp.pp_plan_set_tuning(plan, *[int(v) for v in args.tuning.split(",")])
        xa = torch.from_numpy(synth.crandn(c["shape"], 3)).to(dev)
        ya = torch.empty_like(xa)
        for _ in range(args.apply_only):
            pp.pp_normal_apply(plan, xa, ya)
        torch.cuda.synchronize()
        print(json.dumps({"apply_only": args.apply_only, "tuning": pp.pp_plan_tuning(plan)}))
        plan.destroy()
        return
    seed, sens, traj, x_true, noise = make_inputs(c, rank)
    shape, C, d, iters, lam = c["shape"], c["coils"], c["d"], c["iters"], c["lam"]
    K = len(traj)

    sens_t = torch.from_numpy(sens).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    toep = args.operator == "toeplitz"
    plan = pp.pp_plan_create(shape, C, sens_t, traj=traj, kb_width=c["kb_width"],
                             oversamp=c["oversamp"], seed=seed, power_iters=50, toeplitz=toep)
    torch.cuda.synchronize()
    setup_plan_s = time.perf_counter() - t0
    L = pp.pp_plan_scale(plan)
    # a second plan of the same geometry in the same process (the next frame
    # or slice of a series) reuses the first plan's launch-shape choices
    t0 = time.perf_counter()
    plan2 = pp.pp_plan_create(shape, C, sens_t, traj=traj, kb_width=c["kb_width"],
                              oversamp=c["oversamp"], seed=seed, power_iters=50, toeplitz=toep)
    torch.cuda.synchronize()
    setup_plan_warm_s = time.perf_counter() - t0
    plan2.destroy()

    # measurements b = A x_true + noise (input synthesis: the forward model runs in libpp)
    xt = torch.from_numpy(x_true).to(dev)
    b = torch.empty((C, K), dtype=torch.complex64, device=dev)
    pp.pp_forward_apply(plan, xt, b)
    b += torch.from_numpy(noise).to(dev)
    mu = None
    if args.poly == "cheb":
        # the Chebyshev interval [mu, 1]: mu by power iteration on I - N_hat
        t0 = time.perf_counter()
        mu = pp.pp_plan_mu(plan, 50, seed)
        setup_plan_s += time.perf_counter() - t0
        setup_plan_warm_s += time.perf_counter() - t0
        if not 0.0 < mu < 1.0:
            raise RuntimeError("the mu estimate %g leaves no Chebyshev interval" % mu)
        coeffs = [float(v) for v in pp.pp_poly_coeffs_cheb(d, mu)]
        # the minimax residual reaches -1/T_{d+1}(a) on [mu, 1], so z p(z) peaks
        # at 1 + 1/T_{d+1}(a) (near 2 here): scale p so the step keeps FISTA's
        # rule (max z p(z) = 1); unscaled, the momentum iteration diverges
        zp_max = pp.pp_poly_max_zp(coeffs, d)
        coeffs = [v / zp_max for v in coeffs]
    else:
        coeffs = [float(v) for v in pp.pp_poly_coeffs_l2(d)]
    x_out = torch.empty(shape, dtype=torch.complex64, device=dev)
    applies_per_step = iters * (d + 1)

    for _ in range(args.warmup):
        pp.pp_fista_solve(plan, b, lam, iters, coeffs, d, x_out, wavelet=args.wavelet)
    torch.cuda.synchronize()

    # L2 is 129 MB and the solve's working set (~80 MB) fits in it: flush it
    # between timed steps by writing a 256 MB buffer (outside the timed events).
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    launches = 0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            r = pp.pp_fista_solve(plan, b, lam, iters, coeffs, d, x_out, wavelet=args.wavelet)
            ev[i][1].record(stream)
            launches += r.launches
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    total_ms = sum(a.elapsed_time(bb) for a, bb in ev)
    max_ms = max_over_ranks(total_ms, world, dev)
    value = job_throughput(args.steps * applies_per_step, world, max_ms / 1e3)
    ms_per_step = max_ms / args.steps
    clocks = clk.summary()

    # --- per-kernel timing of the normal operator (CUDA events on the stream) ---
    xin = torch.from_numpy(synth.crandn(shape, 3)).to(dev)
    yout = torch.empty_like(xin)
    stages = pp.pp_profile_normal(plan, xin, yout, reps=50)
    apply_ms = sum(stages.values())
    flops = kernel_flops(c, K, toep)
    # cols_kernel runs twice per apply (forward and inverse): per-launch time is half
    launches_per_apply = {"cols_kernel": 2, "cols4_kernel": 2, "ci_cols_kernel": 2}
    per_launch_ms = {k: v / launches_per_apply.get(k, 1) for k, v in stages.items()}
    dom = max(stages, key=stages.get)
    peak_tflops, peak_src = fp32_peak(dev, clocks)
    ach = flops.get(dom, float("nan")) / (per_launch_ms[dom] / 1e3) / 1e12
    traffic = ncu_traffic(dom, "ncu_traffic_toeplitz.json" if toep else "ncu_traffic.json")
    hbm_peak, hbm_src = hbm_peak_gbs()
    roofline = {
        "bound": "alu", "kernel": dom, "achieved": ach, "peak": peak_tflops, "unit": "TFLOP/s",
        "frac": ach / peak_tflops, "traffic": traffic, "peak_source": peak_src,
        # the same launch against HBM: its DRAM bytes (ncu, cold cache) over
        # its live per-launch time, for reference (the working set is
        # L2-resident, so this is not the bound)
        "hbm_gbs_of_dominant": None if traffic is None else traffic / (per_launch_ms[dom] / 1e3) / 1e9,
        "hbm_frac_of_dominant": None if traffic is None else
        traffic / (per_launch_ms[dom] / 1e3) / 1e9 / hbm_peak,
        "hbm_peak_gbs": hbm_peak, "hbm_peak_source": hbm_src,
        "stage_ms_per_apply": {k: round(v, 5) for k, v in stages.items()},
        "stage_share": {k: round(v / apply_ms, 4) for k, v in stages.items()},
    }

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded phantom, coil maps, spiral, noise); no datasets",
        "config": {"workload": WORKLOAD + ("_toeplitz" if toep else "") +
                               ("_db4" if args.wavelet == "db4" else "") +
                               ("_cheb" if args.poly == "cheb" else ""), "image": list(shape),
                   "preconditioner": ("Chebyshev minimax on [mu, 1] (Sec. 3.4), mu = %.6g from 50 "
                                      "power-iteration steps on I - N_hat, scaled by 1/max z p(z) = "
                                      "1/%.4f" % (mu, zp_max)) if mu is not None
                   else "l2-optimal (Eq. l2cost)",
                   "wavelet": ("Daubechies-4, 2 levels" if args.wavelet == "db4" else "Haar, 2 levels"),
                   "coils": C, "samples": K,
                   "normal_operator": ("exact F^H F by its 2ny x 2nx Toeplitz embedding" if toep else
                                       "Kaiser-Bessel gridding, precomputed G^T G stencil"),
                   "kb_width": c["kb_width"], "oversamp": c["oversamp"], "lambda": lam, "d": d,
                   "iters": iters, "applies_per_step": applies_per_step,
                   "l2": "flushed between timed steps (256 MB write)", "parallelism":
                   "replicas" if world > 1 else "single GPU",
                   "setup_plan_s": setup_plan_s, "setup_plan_warm_s": setup_plan_warm_s, "L": L},
        "roofline": roofline, "clocks": clocks, "gpu_launches": launches,
    }

    if not args.no_extras:
        # --- end to end through the public API with host buffers ---
        b_host = b.cpu().pin_memory()
        x_host = torch.empty(shape, dtype=torch.complex64).pin_memory()
        b_dev = torch.empty_like(b)
        ee = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            ee[i][0].record(stream)
            b_dev.copy_(b_host, non_blocking=True)
            pp.pp_fista_solve(plan, b_dev, lam, iters, coeffs, d, x_out, wavelet=args.wavelet)
            x_host.copy_(x_out, non_blocking=True)
            ee[i][1].record(stream)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(sum(a.elapsed_time(bb) for a, bb in ee), world, dev)
        out["e2e"] = {"value": job_throughput(args.steps * applies_per_step, world, e2e_ms / 1e3),
                      "unit": UNIT, "h2d_bytes_per_step": b_host.numel() * 8,
                      "d2h_bytes_per_step": x_host.numel() * 8}
        # --- time to NRMSE <= 1e-3 against each method's own converged solution ---
        out["time_to_nrmse"] = time_to_target(pp, plan, b, c, coeffs, setup_plan_s, stream,
                                              wavelet=args.wavelet, setup_warm_s=setup_plan_warm_s)
        if rank == 0 and world == 1:
            out["cpu_baseline"] = cpu_baseline(c, exact=toep)
    plan.destroy()
    if world == 1 and not args.no_extras and not args.no_secondary:
        del sens_t, b, x_out, flush
        torch.cuda.empty_cache()
        out["secondary"] = secondary_lines(args, local)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


SECONDARY = (("cart3d_256x256x128_c32", 20), ("batched2d_64", 5))
SECONDARY_KEYS = ("metric", "value", "unit", "ms_per_step", "steps", "warmup", "config", "clocks",
                  "roofline", "prox", "llr_prox", "batched_apply_ms", "stage_ms_per_apply")


def secondary_lines(args, local):
    """The HBM-bound workloads, measured in the same run with the same timing
    rules (bench_workloads): the 256x256x128, 32-coil normal operator with
    the 3-D Haar and locally-low-rank proxes, and the 64-slice batched solve
    and apply."""
    import torch
    import paper_2204_10252_gb300 as pp
    import bench_workloads
    sec = {}
    for wl, steps in SECONDARY:
        a = argparse.Namespace(**vars(args))
        a.workload, a.steps, a.warmup, a.apply_only = wl, steps, max(3, min(args.warmup, 5)), 0
        r = bench_workloads.run(a, pp, 0, 1, local)
        sec[wl] = {k: r[k] for k in SECONDARY_KEYS if k in r}
        torch.cuda.empty_cache()
    return sec


def time_to_target(pp, plan, b, c, coeffs, setup_s, stream, target=1e-3, wavelet="haar", setup_warm_s=None):
    """Per method: converged y_inf (20x the iteration count), the first k
    with ||y_k - y_inf|| / ||y_inf|| <= target, per-iteration time from a
    timed graph replay, and time = setup + k * T_iter."""
    import torch
    shape, lam, d, iters = c["shape"], c["lam"], c["d"], c["iters"]
    res = {}
    for name, cc, dd in (("preconditioned_d%d" % d, coeffs, d), ("plain_fista", None, 0)):
        n_inf = 20 * iters
        y_inf = torch.empty(shape, dtype=torch.complex64, device=b.device)
        pp.pp_fista_solve(plan, b, lam, n_inf, cc, dd, y_inf, wavelet=wavelet)
        y = torch.empty_like(y_inf)
        r = pp.pp_fista_solve(plan, b, lam, n_inf, cc, dd, y, history=True, ref=y_inf, wavelet=wavelet)
        nrm = float(torch.linalg.vector_norm(y_inf.to(torch.complex128)).item())
        err = np.sqrt(np.maximum(r.history[:, 2], 0.0)) / nrm
        hit = np.flatnonzero(err <= target)
        k_star = int(hit[0]) + 1 if hit.size else None
        # per-iteration time: timed replay of `iters` iterations
        pp.pp_fista_solve(plan, b, lam, iters, cc, dd, y, wavelet=wavelet)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(5):
            pp.pp_fista_solve(plan, b, lam, iters, cc, dd, y, wavelet=wavelet)
        e1.record(stream)
        torch.cuda.synchronize()
        t_iter = e0.elapsed_time(e1) / 1e3 / (5 * iters)
        res[name] = {
            "iters_to_target": k_star,
            "applies_to_target": None if k_star is None else k_star * (dd + 1),
            "iter_ms": t_iter * 1e3,
            "seconds_without_setup": None if k_star is None else k_star * t_iter,
            "seconds_with_setup": None if k_star is None else setup_s + k_star * t_iter,
            "seconds_with_warm_setup": None if k_star is None or setup_warm_s is None
            else setup_warm_s + k_star * t_iter,
            "nrmse_at_config_iters": float(err[min(iters, len(err)) - 1]),
            "iters_run": n_inf,
        }
    a, p_ = res["preconditioned_d%d" % d], res["plain_fista"]
    if a["seconds_without_setup"] and p_["seconds_without_setup"]:
        res["speedup_without_setup"] = p_["seconds_without_setup"] / a["seconds_without_setup"]
        res["speedup_with_setup"] = p_["seconds_with_setup"] / a["seconds_with_setup"]
        if setup_warm_s is not None:
            res["speedup_with_warm_setup"] = p_["seconds_with_warm_setup"] / a["seconds_with_warm_setup"]
    res["target"] = target
    return res


if __name__ == "__main__":
    main()
