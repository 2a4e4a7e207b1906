"""Pins for the oracle's solver: Algorithms "fista"/"pfista" (Sec. 2.1, 3.1),
Thm. "fp" (fixed point), Thms. "pgdbnd"/"ppgdbnd" (per-step bounds), Thm.
"err" (Sec. 3.5), the noise-colouring theorem at lambda = 0 (Sec. 3.7) and
the power-iteration norm estimate (Sec. 5)."""
import math

import numpy as np
import pytest

import synth
from oracle import pp_oracle as O


def dense_problem(m=40, shape=(4, 4), seed=0, cond=None):
    rng = np.random.default_rng(seed)
    n = int(np.prod(shape))
    A = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
    if cond is not None:
        U, s, Vh = np.linalg.svd(A, full_matrices=False)
        s = np.geomspace(1.0, 1.0 / cond, n)
        A = (U * s) @ Vh
    b = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    fwd = lambda x: A @ x.ravel()
    adj = lambda y: (A.conj().T @ y).reshape(shape)
    nrm = lambda x: adj(fwd(x))
    return A, b, fwd, adj, nrm


def test_splitmix64_reference_outputs():
    # First outputs of SplitMix64 from state 0 (Vigna's reference sequence).
    got = [int(v) for v in O.splitmix64(0, 3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_power_iteration_matches_dense_eigenvalue():
    A, b, fwd, adj, nrm = dense_problem(cond=20.0, seed=1)
    lmax = np.linalg.eigvalsh(A.conj().T @ A).max()
    L = O.power_iteration(nrm, (4, 4), seed=7, iters=50)
    assert L <= lmax * (1 + 1e-12)
    assert abs(L - lmax) <= 1e-6 * lmax


@pytest.mark.parametrize("coeffs", [None, "l2_3", "l2_5"])
def test_lambda_zero_reaches_least_squares(coeffs):
    # lambda = 0: both plain and preconditioned FISTA solve the normalised
    # least-squares problem; the solutions coincide (no noise colouring).
    A, b, fwd, adj, nrm = dense_problem(cond=5.0, seed=2)
    L = np.linalg.eigvalsh(A.conj().T @ A).max()
    c = None if coeffs is None else O.poly_coeffs_l2(int(coeffs[-1]))
    y = O.pfista(nrm, adj, b, 0.0, c, 1000 if c is None else 400, L, levels=2)
    Ah = A / math.sqrt(L)
    bh = b / np.linalg.norm(b)
    ref = np.linalg.lstsq(Ah, bh, rcond=None)[0].reshape(4, 4)
    assert np.linalg.norm(y - ref) <= 1e-8 * np.linalg.norm(ref)


def test_fixed_point_at_convergence():
    A, b, fwd, adj, nrm = dense_problem(cond=5.0, seed=3)
    L = np.linalg.eigvalsh(A.conj().T @ A).max()
    lam = 0.02
    x = O.pfista(nrm, adj, b, lam, None, 3000, L)
    ahb = adj(b) / (math.sqrt(L) * np.linalg.norm(b))
    step = O.prox_l1_haar(x - (nrm(x) / L - ahb), lam)
    assert np.linalg.norm(x - step) <= 1e-10 * np.linalg.norm(x)


@pytest.mark.parametrize("d", [None, 3])
def test_per_step_error_bounds(d):
    # ||e_{k+1}|| <= ||(I - p(N) N) e_k|| for PGD (p = 1) and PPGD.
    A, b, fwd, adj, nrm = dense_problem(cond=8.0, seed=4)
    L = np.linalg.eigvalsh(A.conj().T @ A).max()
    lam = 0.01
    c = None if d is None else O.poly_coeffs_l2(d)
    ystar = O.pfista(nrm, adj, b, lam, c, 5000, L, momentum=False)
    hist = []
    O.pfista(nrm, adj, b, lam, c, 30, L, momentum=False, history=hist)
    nhat = lambda v: nrm(v) / L
    prev = np.zeros_like(ystar)
    for yk in hist:
        e_prev = prev - ystar
        pe = e_prev if c is None else O.horner_apply(c, nhat, e_prev)
        bound = np.linalg.norm(e_prev - (nhat(pe) if c is None else O.horner_apply(c, nhat, nhat(e_prev))))
        assert np.linalg.norm(yk - ystar) <= bound * (1 + 1e-9) + 1e-13
        prev = yk


def test_solution_error_bound():
    # Thm "err": ||y_inf - x*|| <= delta/(1 - gamma) for injective N, lambda_p = lambda.
    A, b, fwd, adj, nrm = dense_problem(cond=3.0, seed=5)
    L = np.linalg.eigvalsh(A.conj().T @ A).max()
    lam = 0.05
    c = O.poly_coeffs_l2(3)
    xstar = O.pfista(nrm, adj, b, lam, None, 4000, L)
    ystar = O.pfista(nrm, adj, b, lam, c, 4000, L)
    Nh = (A.conj().T @ A) / L
    P = np.zeros_like(Nh)
    for ci in reversed([float(v) for v in c]):
        P = ci * np.eye(16) + Nh @ P
    gamma = np.linalg.norm(np.eye(16) - P @ Nh, 2)
    assert gamma < 1.0
    Ah = A / math.sqrt(L)
    bh = b / np.linalg.norm(b)
    resid = Ah.conj().T @ (Ah @ xstar.ravel() - bh)
    delta = np.linalg.norm((np.eye(16) - P) @ resid)
    assert np.linalg.norm(ystar - xstar) <= delta / (1 - gamma) + 1e-12
    # and the bound is not vacuous here
    assert delta / (1 - gamma) < np.linalg.norm(xstar)


def test_cartesian_pgd_objective_monotone_and_fixed_points():
    # Tiny Cartesian SENSE problem.  PGD with step 1/L (p = 1, beta = 0) never
    # increases the objective; plain and preconditioned FISTA both reach a
    # fixed point of their own update (Thm "fp" applied to Eq. "ppgd").
    shape, C = (16, 16), 4
    s = synth.coil_maps(shape, C, 1)
    m = synth.line_mask(shape, 3, 4, 1)
    x0 = synth.phantom(shape, 1)
    b = O.cart_forward(x0, s, m) + m[None] * synth.cnoise((C,) + shape, 1e-3, 2)
    nrm = lambda v: O.cart_normal(v, s, m)
    adj = lambda y: O.cart_adjoint(y, s, m)
    L = O.power_iteration(nrm, shape, 3)
    lam = 1e-3
    bh = b / np.linalg.norm(b)
    ahb = adj(b) / (math.sqrt(L) * np.linalg.norm(b))

    def obj(x):
        r = O.cart_forward(x, s, m) / math.sqrt(L) - bh
        return 0.5 * np.linalg.norm(r) ** 2 + lam * np.sum(np.abs(O.haar_fwd(x, 2)))

    hist = []
    O.pfista(nrm, adj, b, lam, None, 30, L, momentum=False, history=hist)
    objs = [obj(np.zeros(shape))] + [obj(h) for h in hist]
    assert all(b_ <= a_ + 1e-15 for a_, b_ in zip(objs, objs[1:]))
    nhat = lambda v: nrm(v) / L
    for c in (None, O.poly_coeffs_l2(3)):
        y = O.pfista(nrm, adj, b, lam, c, 3000, L)
        g = nhat(y) - ahb
        u = g if c is None else O.horner_apply(c, nhat, g)
        assert np.linalg.norm(O.prox_l1_haar(y - u, lam) - y) <= 1e-9 * np.linalg.norm(y)


def test_cartesian_pgd_with_db4_prox_is_monotone_and_reaches_a_fixed_point():
    # the same with W = Daubechies-4 (the paper's choice in Sec. 5): PGD never
    # increases the objective with the db4 l1 term, and preconditioned FISTA
    # stops at a fixed point of its own db4 update (Thm "fp")
    shape, C = (16, 16), 4
    s = synth.coil_maps(shape, C, 1)
    m = synth.line_mask(shape, 3, 4, 1)
    x0 = synth.phantom(shape, 1)
    b = O.cart_forward(x0, s, m) + m[None] * synth.cnoise((C,) + shape, 1e-3, 2)
    nrm = lambda v: O.cart_normal(v, s, m)
    adj = lambda y: O.cart_adjoint(y, s, m)
    L = O.power_iteration(nrm, shape, 3)
    lam = 1e-3
    bh = b / np.linalg.norm(b)
    ahb = adj(b) / (math.sqrt(L) * np.linalg.norm(b))

    def obj(x):
        r = O.cart_forward(x, s, m) / math.sqrt(L) - bh
        return 0.5 * np.linalg.norm(r) ** 2 + lam * np.sum(np.abs(O.db4_fwd(x, 2)))

    hist = []
    O.pfista(nrm, adj, b, lam, None, 30, L, momentum=False, history=hist, wavelet="db4")
    objs = [obj(np.zeros(shape))] + [obj(h) for h in hist]
    assert all(b_ <= a_ + 1e-15 for a_, b_ in zip(objs, objs[1:]))
    nhat = lambda v: nrm(v) / L
    c = O.poly_coeffs_l2(3)
    y = O.pfista(nrm, adj, b, lam, c, 3000, L, wavelet="db4")
    u = O.horner_apply(c, nhat, nhat(y) - ahb)
    assert np.linalg.norm(O.prox_l1_db4(y - u, lam) - y) <= 1e-9 * np.linalg.norm(y)
    # and it is not the Haar solution
    yh = O.pfista(nrm, adj, b, lam, c, 3000, L)
    assert np.linalg.norm(yh - y) > 1e-6 * np.linalg.norm(y)
