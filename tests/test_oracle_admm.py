"""Pins for the oracle's consensus ADMM (Algorithm "cadmm", Sec. 5.3) and its
subproblem prox_{rho f_i} (pfista_prox): the subproblem's fixed point and
closed forms, and consensus ADMM over coil groups reaching the solution of
the whole problem (the sum of the subproblems)."""
import math

import numpy as np
import pytest

import synth
from oracle import pp_oracle as O


def problem(shape=(16, 16), C=4, seed=3):
    s = synth.coil_maps(shape, C, seed)
    m = synth.line_mask(shape, 3, 4, seed)
    x0 = synth.phantom(shape, seed)
    b = O.cart_forward(x0, s, m) + m[None] * synth.cnoise((C,) + shape, 1e-3, seed + 1)
    return s, m, b


def test_prox_subproblem_closed_form_without_data_and_threshold():
    # b = None, lam = 0: argmin (sigma/2)||x - v||^2 is v itself
    v = synth.crandn((8, 8), 2).astype(np.complex128)
    nrm = lambda x: 0.0 * x
    # (the operator is 0, so L = 0 and L' = sigma: one step lands on the answer)
    got = O.pfista_prox(nrm, None, None, v, 0.7, 0.0, None, 3, 0.0)
    assert np.allclose(got, v, atol=1e-14)
    # ... and with a threshold: the prox of (lam/sigma)||W.||_1 at v
    got = O.pfista_prox(nrm, None, None, v, 0.7, 0.2, None, 3, 0.0)
    assert np.allclose(got, O.prox_l1_haar(v, 0.2 / 0.7), atol=1e-14)


@pytest.mark.parametrize("coeffs", [None, "l2_3"])
def test_prox_subproblem_fixed_point_and_least_squares(coeffs):
    # lam = 0: the solution of (A^H A + sigma I) x = A^H b + sigma v (dense solve);
    # lam > 0: a fixed point of the subproblem's proximal-gradient map
    s, m, b = problem()
    nrm = lambda x: O.cart_normal(x, s, m)
    adj = lambda y: O.cart_adjoint(y, s, m)
    L = O.power_iteration(nrm, (16, 16), 1)
    sigma = 0.3 * L
    v = synth.crandn((16, 16), 5).astype(np.complex128) * 0.1
    c = None if coeffs is None else O.poly_coeffs_l2(3)
    y = O.pfista_prox(nrm, adj, b, v, sigma, 0.0, c, 400, L)
    n = 256
    E = np.eye(n, dtype=np.complex128).reshape(n, 16, 16)
    H = np.stack([nrm(e).ravel() for e in E], axis=1) + sigma * np.eye(n)
    ref = np.linalg.solve(H, (adj(b) + sigma * v).ravel()).reshape(16, 16)
    assert np.linalg.norm(y - ref) <= 1e-10 * np.linalg.norm(ref)
    lam = 2e-3
    Lp = L + sigma
    y = O.pfista_prox(nrm, adj, b, v, sigma, lam, c, 1500, L)
    g = (nrm(y) + sigma * y - adj(b) - sigma * v) / Lp
    u = g if c is None else O.horner_apply(c, lambda x: (nrm(x) + sigma * x) / Lp, g)
    assert np.linalg.norm(O.prox_l1_haar(y - u, lam / Lp) - y) <= 1e-10 * np.linalg.norm(y)


def test_consensus_admm_reaches_the_whole_problem():
    # f(x) = 1/2 ||A x - b||^2 + lam ||W x||_1 split by rows (as the coil
    # groups split A): f_i = 1/2 ||A_i x - b_i||^2 + (lam/N) ||W x||_1, so
    # sum_i f_i = f.  Each A_i here has more rows than unknowns (every f_i
    # strongly convex), where consensus ADMM with accurate subproblem solves
    # converges linearly to argmin f.
    rng = np.random.default_rng(11)
    n, groups = 16, [range(0, 24), range(24, 48)]
    A = rng.standard_normal((48, n)) + 1j * rng.standard_normal((48, n))
    b = rng.standard_normal(48) + 1j * rng.standard_normal(48)
    lam = 0.5
    op = lambda M: ((lambda x: (M.conj().T @ (M @ x.ravel())).reshape(4, 4)),
                    (lambda y: (M.conj().T @ y).reshape(4, 4)))
    nrm, adj = op(A)
    L = float(np.linalg.eigvalsh(A.conj().T @ A).max())
    rho = 10.0 / L
    proxes = []
    for g in groups:
        Ai = A[list(g)]
        ni, ai = op(Ai)
        Li = float(np.linalg.eigvalsh(Ai.conj().T @ Ai).max())
        # plain FISTA inner solves: with lam > 0 the preconditioned iteration
        # stops at its own fixed point, near but not at the prox (Thm "err")
        proxes.append(lambda v, ni=ni, ai=ai, bi=b[list(g)], Li=Li:
                      O.pfista_prox(ni, ai, bi, v, 1.0 / rho, lam / len(groups), None, 1500, Li))
    hist = []
    xbar = O.consensus_admm(proxes, (4, 4), 80, history=hist)
    xs = O.pfista_prox(nrm, adj, b, None, 0.0, lam, None, 5000, L)
    g = (nrm(xs) - adj(b)) / L
    assert np.linalg.norm(O.prox_l1_haar(xs - g, lam / L) - xs) <= 1e-12 * np.linalg.norm(xs)
    assert np.linalg.norm(xbar - xs) <= 1e-8 * np.linalg.norm(xs)
    # the iterates settle geometrically
    e = [np.linalg.norm(h - xs) for h in hist]
    assert e[40] < 1e-4 * e[2]
    # a single group is the whole problem's prox: one step with v = 0 and
    # a huge rho is the subproblem solution itself
    one = O.consensus_admm([lambda v: O.pfista_prox(nrm, adj, b, v, 1e-12, lam, None, 5000, L)], (4, 4), 1)
    assert np.linalg.norm(one - xs) <= 1e-8 * np.linalg.norm(xs)
