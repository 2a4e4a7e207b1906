"""Consensus ADMM (Algorithm "cadmm", Sec. 5.3) split over two gloo ranks on
the CPU: each rank holds one coil group's subproblem, the only exchange is
the all-reduce of the group solutions, and the result equals the oracle's
single-process consensus ADMM on the same subproblems."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import pp_oracle as O


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem():
    """A small multi-coil Cartesian problem split into two coil groups."""
    import synth
    shape, C = (16, 16), 4
    s = synth.coil_maps(shape, C, 21)
    m = synth.line_mask(shape, 2, 4, 21)
    x0 = synth.phantom(shape, 21)
    b = O.cart_forward(x0, s, m) + m[None] * synth.cnoise((C,) + shape, 1e-3, 22)
    groups = [[0, 1], [2, 3]]
    lam, iters_in, admm_iters = 2e-3, 40, 6
    L = O.power_iteration(lambda x: O.cart_normal(x, s, m), shape, 3)
    sigma = 0.5 * L
    c = O.poly_coeffs_l2(3)
    proxes = []
    for g in groups:
        ni = lambda x, g=g: O.cart_normal(x, s[g], m)
        ai = lambda y, g=g: O.cart_adjoint(y, s[g], m)
        Li = O.power_iteration(ni, shape, 4)
        proxes.append(lambda v, ni=ni, ai=ai, bi=b[g], Li=Li:
                      O.pfista_prox(ni, ai, bi, v, sigma, lam / len(groups), c, iters_in, Li))
    return shape, proxes, admm_iters


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2204_10252_gb300.admm import consensus_admm, groups_of_rank
        shape, proxes, iters = _problem()
        mine = groups_of_rank(len(proxes), rank, world)
        local = [lambda v, p=proxes[i]: torch.from_numpy(p(v.numpy())) for i in mine]
        like = torch.zeros(shape, dtype=torch.complex128)
        xbar = consensus_admm(local, len(proxes), iters, like)
        q.put((rank, mine, xbar.numpy()))
    finally:
        dist.destroy_process_group()


def test_consensus_admm_two_gloo_ranks_matches_single_process_oracle():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shape, proxes, iters = _problem()
    ref = O.consensus_admm(proxes, shape, iters)
    assert sorted(g for _, mine, _ in out for g in mine) == [0, 1]   # each group on one rank
    for rank, mine, xbar in out:
        assert np.linalg.norm(xbar - ref) <= 1e-12 * np.linalg.norm(ref), rank


def test_consensus_admm_single_process_runs_every_group():
    # no process group: all groups run in this process, same result
    from paper_2204_10252_gb300.admm import consensus_admm
    shape, proxes, iters = _problem()
    local = [lambda v, p=p: torch.from_numpy(p(v.numpy())) for p in proxes]
    xbar = consensus_admm(local, len(proxes), iters, torch.zeros(shape, dtype=torch.complex128))
    ref = O.consensus_admm(proxes, shape, iters)
    assert np.linalg.norm(xbar.numpy() - ref) <= 1e-12 * np.linalg.norm(ref)
