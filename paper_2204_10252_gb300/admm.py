"""Global consensus ADMM over coil groups (Algorithm "cadmm", Sec. 5.3).

The paper splits a problem too large for one device by receiver coils: with
A = [A_1; ...; A_N] and b split alike into coil groups,
    f_i(x) = 1/2 ||A_i x - b_i||^2 + (lambda / N) ||W x||_1
sums to the whole objective.  Each iteration solves every group's
subproblem prox_{rho f_i}(x_bar - u_i) -- a regularised inverse problem,
solved here by preconditioned FISTA on that group's plan
(pp_fista_solve_prox with sigma = 1/rho) -- then averages the group
solutions into x_bar and updates the scaled duals u_i.  The average is the
only exchange between groups: one all-reduce of an image per iteration.

Groups are spread over the ranks of the default torch.distributed process
group (rank r holds groups r, r + W, ...); with no process group, or one
rank, every group runs in this process in turn.  The all-reduce runs over
whatever backend the group uses (NCCL between GPUs, gloo between hosts).
Tensors stay where the subproblem solver puts them; the averaging and dual
updates are elementwise tensor arithmetic around that collective.
"""
from __future__ import annotations

from typing import Callable, List, Optional, Sequence

import torch


def groups_of_rank(n_groups: int, rank: int, world: int) -> List[int]:
    """Coil groups handled by `rank`: r, r + world, r + 2 world, ..."""
    return list(range(rank, n_groups, world))


def consensus_admm(local_prox: Sequence[Callable[[torch.Tensor], torch.Tensor]], n_groups: int,
                   iters: int, like: torch.Tensor, history: Optional[list] = None) -> torch.Tensor:
    """x_bar after `iters` iterations of Algorithm "cadmm":
        x_i   = prox_{rho f_i}(x_bar - u_i)      for this rank's groups
        x_bar = (1/N) sum_i x_i                  (all-reduce over the ranks)
        u_i   = u_i + x_i - x_bar
    starting from x_bar = x_i = u_i = 0.  local_prox[j](v) returns
    prox_{rho f_i}(v) for this rank's j-th group; n_groups is N over all
    ranks; `like` gives the image's shape, dtype and device."""
    import torch.distributed as dist
    distributed = dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1
    xbar = torch.zeros_like(like)
    us = [torch.zeros_like(like) for _ in local_prox]
    for _ in range(iters):
        xs = [prox(xbar - u) for prox, u in zip(local_prox, us)]
        total = torch.zeros_like(like)
        for x in xs:
            total += x
        if distributed:
            dist.all_reduce(total, op=dist.ReduceOp.SUM)
        xbar = total / n_groups
        for u, x in zip(us, xs):
            u += x - xbar
        if history is not None:
            history.append(xbar.clone())
    return xbar


def coil_group_prox(plan, b_group: torch.Tensor, sigma: float, lam_group: float, iters: int,
                    coeffs, d: int, **solve_kw) -> Callable[[torch.Tensor], torch.Tensor]:
    """prox_{rho f_i} for one coil group on the GPU: `plan` is built on the
    group's coil maps, b_group its k-space; sigma = 1/rho; lam_group the
    group's share of lambda (lambda / N)."""
    from .binding import pp_fista_solve_prox

    def prox(v: torch.Tensor) -> torch.Tensor:
        out = torch.empty_like(v)
        pp_fista_solve_prox(plan, b_group, v.contiguous(), sigma, lam_group, iters, coeffs, d, out,
                            **solve_kw)
        return out
    return prox
