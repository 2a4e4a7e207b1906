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


# ---------------------------------------------------------------------------
# Momentum schedule of Algorithm "pfista" (Sec. 3.1), pinned by iterates
# derived by hand.  With lambda = 0 the prox is the identity (W orthonormal),
# and with a diagonal normal operator N_hat = diag(m) every pixel runs the
# scalar recursion y_{k+1} = q z_k + r, where p is the preconditioner,
# q = 1 - m p(m) and r = p(m) a (a = A_hat^H b_hat).  Unrolling by hand with
# beta_k = k/(k+3) (beta_0 = 0, beta_1 = 1/4, beta_2 = 2/5, beta_3 = 1/2) and
# z_{k+1} = y_{k+1} + beta_k (y_{k+1} - y_k), y_0 = z_0 = 0:
#   y_1 = r
#   y_2 = r (1 + q)
#   y_3 = r (1 + q + 5/4 q^2)                    (z_2 = r (1 + 5/4 q))
#   y_4 = r (1 + q + q^2 + 7/4 q^3)              (z_3 = r (1 + q + 7/4 q^2))
#   y_5 = r (1 + q + q^2 + 7/8 q^3 + 21/8 q^4)   (z_4 = r (1 + q + 7/8 q^2 + 21/8 q^3))
# and without momentum (Algorithm "ppgd") the geometric sums
#   y_k = r (1 + q + ... + q^(k-1)).
# A schedule shifted by one, (k-1)/(k+2), or the printed
# z_{k+1} = y_k + beta_k (y_k - y_{k-1}) each change y_2 or y_3.
# ---------------------------------------------------------------------------

_MOM = lambda q, r: [r,
                     r * (1 + q),
                     r * (1 + q + 1.25 * q ** 2),
                     r * (1 + q + q ** 2 + 1.75 * q ** 3),
                     r * (1 + q + q ** 2 + 0.875 * q ** 3 + 2.625 * q ** 4)]


def _diag_problem(seed=11):
    rng = np.random.default_rng(seed)
    m = rng.uniform(0.05, 0.95, (4, 4))                       # spectrum of N_hat
    b = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    normal = lambda v: m * v                                  # L = 1: N_hat = N
    adjoint = lambda y: np.asarray(y).reshape(4, 4)           # A^H b = b
    return m, b, normal, adjoint


@pytest.mark.parametrize("coeffs", [[4.0, -10.0 / 3.0], [1.5, 0.25]])
def test_momentum_schedule_matches_hand_derived_iterates(coeffs):
    m, b, normal, adjoint = _diag_problem()
    p = coeffs[0] + coeffs[1] * m
    q, r = 1.0 - m * p, p * b
    hist = []
    O.pfista(normal, adjoint, b, 0.0, coeffs, 5, 1.0, normalize_b=False, history=hist)
    for k, (got, want) in enumerate(zip(hist, _MOM(q, r))):
        assert np.max(np.abs(got - want)) <= 1e-14 * np.max(np.abs(want)), "y_%d" % (k + 1)
    # the same with b normalised to unit norm (Sec. 5): a = b / ||b||
    hist = []
    O.pfista(normal, adjoint, b, 0.0, coeffs, 5, 1.0, normalize_b=True, history=hist)
    rn = r / np.linalg.norm(b)
    for got, want in zip(hist, _MOM(q, rn)):
        assert np.max(np.abs(got - want)) <= 1e-14 * np.max(np.abs(want))


def test_plain_fista_momentum_and_ppgd_geometric_sums():
    # p = 1 (coeffs None, Algorithm "fista") follows the same closed forms
    # with q = 1 - m, r = a; beta = 0 (Algorithm "pgd") gives geometric sums
    m, b, normal, adjoint = _diag_problem(12)
    q, r = 1.0 - m, b
    hist = []
    O.pfista(normal, adjoint, b, 0.0, None, 5, 1.0, normalize_b=False, history=hist)
    for got, want in zip(hist, _MOM(q, r)):
        assert np.max(np.abs(got - want)) <= 1e-14 * np.max(np.abs(want))
    hist = []
    O.pfista(normal, adjoint, b, 0.0, [2.0, -1.0], 6, 1.0, normalize_b=False, momentum=False,
             history=hist)
    p = 2.0 - m
    q, r = 1.0 - m * p, p * b
    for k, got in enumerate(hist, start=1):
        want = r * sum(q ** j for j in range(k))
        assert np.max(np.abs(got - want)) <= 1e-14 * np.max(np.abs(want))


def test_unrolled_forward_follows_the_same_iterates():
    # the differentiable solve's forward (raw b, fixed L) runs the same
    # iteration: its y_K equals the hand-derived iterates for K = 1..5 ...
    m, b, normal, adjoint = _diag_problem(13)
    c = [4.0, -10.0 / 3.0]
    p = c[0] + c[1] * m
    want = _MOM(1.0 - m * p, p * b)
    for K in range(1, 6):
        got = O.pfista_unrolled(normal, adjoint, b, 0.0, c, K, 1.0)
        assert np.max(np.abs(got - want[K - 1])) <= 1e-14 * np.max(np.abs(want[K - 1]))


def test_unrolled_forward_equals_pfista_without_b_normalisation():
    # ... and, on a Cartesian SENSE problem with an active soft threshold,
    # every y_K equals pfista(..., normalize_b=False)
    shape, C = (16, 16), 4
    s = synth.coil_maps(shape, C, 5)
    msk = synth.line_mask(shape, 3, 4, 5)
    b = O.cart_forward(synth.phantom(shape, 5), s, msk)
    nrm = lambda v: O.cart_normal(v, s, msk)
    adj = lambda y: O.cart_adjoint(y, s, msk)
    L = O.power_iteration(nrm, shape, 5)
    c = O.poly_coeffs_l2(3)
    lam = 0.02 * float(np.max(np.abs(adj(b)))) / math.sqrt(L)
    hist = []
    O.pfista(nrm, adj, b, lam, c, 8, L, normalize_b=False, history=hist)
    for K in (1, 2, 5, 8):
        yk = O.pfista_unrolled(nrm, adj, b, lam, c, K, L)
        assert np.max(np.abs(yk - hist[K - 1])) <= 1e-14 * np.max(np.abs(hist[K - 1]))
    # the threshold is active: some Haar coefficients are set to zero
    wc = O.haar_fwd(hist[-1], 2)
    assert np.sum(np.abs(wc) == 0) > 0


# ---------------------------------------------------------------------------
# mu for the Chebyshev design (the Sec. 3.4 remark): power iteration on
# I - N_hat converges to 1 - mu when A^H A is injective.
# ---------------------------------------------------------------------------

def test_mu_estimate_diagonal_operator():
    # N = diag(m), L = max m: the smallest eigenvalue of N_hat is
    # min m / max m; a well-separated spectrum converges fast
    m = np.array([0.2, 0.9, 3.0, 5.0, 2.5, 4.0, 1.7, 0.6] * 2).reshape(4, 4)
    normal = lambda v: m * v
    mu = O.mu_estimate(normal, (4, 4), 3, float(m.max()), iters=400)
    assert abs(mu - 0.2 / 5.0) <= 1e-10
    # the iteration approaches from above: fewer steps never undershoot
    for k in (5, 20, 60):
        assert O.mu_estimate(normal, (4, 4), 3, float(m.max()), iters=k) >= 0.04 - 1e-15


def test_mu_estimate_matches_dense_smallest_eigenvalue():
    A, b, fwd, adj, nrm = dense_problem(cond=6.0, seed=8)
    ev = np.linalg.eigvalsh(A.conj().T @ A)
    L = float(ev.max())
    mu = O.mu_estimate(nrm, (4, 4), 9, L, iters=3000)
    assert abs(mu - ev.min() / L) <= 1e-8
    # with the Chebyshev polynomial on [mu, 1], |1 - z p(z)| <= 1/T_{d+1}(a)
    # at every eigenvalue of N_hat (the bound the remark's design minimises)
    c = O.poly_coeffs_cheb(3, mu)
    z = ev / L
    a = (1 + mu) / (1 - mu)
    bound = 1.0 / np.cosh(4 * np.arccosh(a))
    assert np.max(np.abs(1 - z * O.poly_eval(c, z))) <= bound * (1 + 1e-9)


def test_mu_estimate_of_a_singular_operator_is_zero():
    # a null space (fewer rows than unknowns): 1 is an eigenvalue of
    # I - N_hat and the estimate goes to 0 (no usable Chebyshev interval)
    A, b, fwd, adj, nrm = dense_problem(m=10, seed=10)
    ev = np.linalg.eigvalsh(A.conj().T @ A)
    L = float(ev.max())
    assert ev[ev > 1e-9 * L].min() / L > 1e-3        # the smallest non-zero one is far from 0
    assert abs(O.mu_estimate(nrm, (4, 4), 2, L, iters=300)) <= 1e-8
