"""Writes tests/golden/spiral2d_256_c32_pfista100.npz: the FP64 oracle's
solution of the full spiral workload (256x256 image, 32 coils, 16-interleave
spiral with 4096 samples each, Kaiser-Bessel gridding W = 4, sigma = 1.25,
2-level Haar l1 with lambda = 5e-4, degree-5 l2-optimal polynomial) after
100 iterations of Algorithm "pfista", together with the induced-norm estimate
L from 50 power-iteration steps (seed 2205).

Inputs are the seeded synthetic ones of the benchmark (synth.CONFIGS
"spiral2d_256_c32"): b = N(S x_true) + noise, computed by the oracle's
forward model and rounded to complex64 (what the device path is given).
Every arithmetic step is the oracle's; this script only spreads the coil sum
of each normal-operator apply over worker processes, adding the per-group
oracle results in FP64.

Run:  python tests/golden/make_spiral_golden.py [workers]   (about 40 minutes
on 6 x86 cores)
"""
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import pp_oracle as O  # noqa: E402

OUT = os.path.join(HERE, "spiral2d_256_c32_pfista100.npz")
CFG = synth.CONFIGS["spiral2d_256_c32"]
_W = {}


def inputs():
    shape, C = CFG["shape"], CFG["coils"]
    sens = synth.coil_maps(shape, C, CFG["seed"])
    traj = synth.spiral_traj(CFG["interleaves"], CFG["samples"], CFG["turns"], shape[0] / 2.0)
    x_true = synth.phantom(shape, CFG["seed"])
    noise = synth.cnoise((C, len(traj)), CFG["sigma"], CFG["seed"] + 1)
    return sens, traj, x_true, noise


def measurements(sens, traj, x_true, noise):
    """b = A x_true + noise by the oracle's forward model, rounded to complex64."""
    b = O.nc_forward(x_true, sens, traj, CFG["kb_width"], CFG["oversamp"]) + noise
    return b.astype(np.complex64)


def _init(coils):
    sens, traj, _, _ = inputs()
    _W["sens"], _W["traj"] = sens[coils], traj


def _part(x):
    return O.nc_normal(x, _W["sens"], _W["traj"], CFG["kb_width"], CFG["oversamp"])


def main(workers):
    sens, traj, x_true, noise = inputs()
    C = sens.shape[0]
    groups = [list(range(C))[i::workers] for i in range(workers)]
    ctx = mp.get_context("spawn")
    pools = [ctx.Pool(1, initializer=_init, initargs=(g,)) for g in groups]
    calls = [0]

    def normal(x):
        rs = [p.apply_async(_part, (x,)) for p in pools]
        calls[0] += 1
        return sum(r.get() for r in rs)

    t0 = time.time()
    b = measurements(sens, traj, x_true, noise)
    L = O.power_iteration(normal, CFG["shape"], CFG["seed"], iters=50)
    print("L = %.17g (%.0f s)" % (L, time.time() - t0), flush=True)
    adjoint = lambda y: O.nc_adjoint(y, sens, traj, CFG["kb_width"], CFG["oversamp"])
    c = [float(v) for v in O.poly_coeffs_l2(CFG["d"])]
    y = O.pfista(normal, adjoint, b.astype(np.complex128), CFG["lam"], c, CFG["iters"], L)
    print("solve done: %d applies, %.0f s" % (calls[0], time.time() - t0), flush=True)
    for p in pools:
        p.close()
    np.savez(OUT, y=y.astype(np.complex64), L=np.float64(L), iters=CFG["iters"], d=CFG["d"],
             lam=CFG["lam"], seed=CFG["seed"])


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 6)
