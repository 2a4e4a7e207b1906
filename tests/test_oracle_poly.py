"""Pins for the polynomial preconditioner: Eq. "l2cost" (Sec. 3.1),
Thm. "ppos" (Sec. 3.4), the recursion of Listing "pcode" (Sec. 3.6),
Lemma "permute" (Sec. 3.3) and Fig. "complexity" (Sec. 3.6)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import pp_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_coeff_table():
    out = {}
    with open(os.path.join(GOLDEN, "l2_coeffs.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            d, rest = line.split(":")
            out[int(d)] = [Fraction(t) for t in rest.split()]
    return out


def cost_by_quadrature(c):
    # Gauss-Legendre on [0, 1] with 40 nodes is exact for degree <= 79.
    t, w = np.polynomial.legendre.leggauss(40)
    z = 0.5 * (t + 1.0)
    r = 1.0 - z * O.poly_eval(c, z)
    return 0.5 * float(np.sum(w * r * r))


@pytest.mark.parametrize("d", range(0, 9))
def test_golden_table_is_the_oracle(d):
    assert load_coeff_table()[d] == O.poly_coeffs_l2(d)


@pytest.mark.parametrize("d", range(0, 9))
def test_minimum_cost_closed_form(d):
    # the minimum of the l2 cost is 1/(d+2)^2
    c = O.poly_coeffs_l2(d)
    assert abs(cost_by_quadrature(c) - 1.0 / (d + 2) ** 2) <= 1e-12


@pytest.mark.parametrize("d", range(0, 6))
def test_coefficients_match_discretised_least_squares(d):
    # Independent route: weighted least squares on Gauss-Legendre nodes,
    # min sum_j w_j (1 - sum_i c_i z_j^{i+1})^2, which equals the integral.
    t, w = np.polynomial.legendre.leggauss(40)
    z = 0.5 * (t + 1.0)
    sw = np.sqrt(0.5 * w)
    V = np.stack([z ** (i + 1) for i in range(d + 1)], axis=1)
    c_ls, *_ = np.linalg.lstsq(sw[:, None] * V, sw, rcond=None)
    c = np.array([float(x) for x in O.poly_coeffs_l2(d)])
    assert np.max(np.abs(c - c_ls)) <= 1e-7 * np.max(np.abs(c))


@pytest.mark.parametrize("d", range(0, 9))
def test_positivity_on_unit_interval(d):
    z = np.linspace(1e-6, 1.0, 20001)
    assert np.all(O.poly_eval(O.poly_coeffs_l2(d), z) > 0.0)


def test_figure_complexity_regions():
    c3 = O.poly_coeffs_l2(3)
    with open(os.path.join(GOLDEN, "fig_complexity.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for z, region in rows:
        z = float(z)
        pgd = (1.0 - z) ** 4
        pp = abs(1.0 - z * O.poly_eval(c3, np.array([z]))[0])
        if region == "low":
            assert pp < pgd
        else:
            assert pp > pgd


@pytest.mark.parametrize("d", [0, 1, 3, 5])
def test_horner_on_diagonal_operator(d):
    # For N = diag(lam_i), p(N) g = p(lam_i) g_i, with exactly d applies of N.
    rng = np.random.default_rng(d)
    lam = rng.uniform(0.0, 1.0, 64)
    g = rng.standard_normal(64) + 1j * rng.standard_normal(64)
    calls = []

    def normal(v):
        calls.append(1)
        return lam * v

    c = O.poly_coeffs_l2(d)
    got = O.horner_apply(c, normal, g)
    ref = O.poly_eval(c, lam) * g
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert len(calls) == d


def test_permutability_lemma():
    # A^H p(A A^H) = p(A^H A) A^H for a dense A (Lemma "permute").
    rng = np.random.default_rng(0)
    A = rng.standard_normal((7, 5)) + 1j * rng.standard_normal((7, 5))
    A /= np.linalg.norm(A, 2)
    c = [float(x) for x in O.poly_coeffs_l2(3)]

    def pmat(M):
        out = c[-1] * np.eye(M.shape[0])
        for ci in reversed(c[:-1]):
            out = ci * np.eye(M.shape[0]) + M @ out
        return out

    AH = A.conj().T
    lhs = AH @ pmat(A @ AH)
    rhs = pmat(AH @ A) @ AH
    assert np.max(np.abs(lhs - rhs)) <= 1e-12 * np.max(np.abs(lhs))


@pytest.mark.parametrize("d,mu", [(1, 0.1), (3, 0.05), (5, 0.02), (3, 0.3)])
def test_chebyshev_equioscillates_on_mu_1(d, mu):
    # Sec. 3.4: r(z) = 1 - z p(z) is T_{d+1} on [mu, 1] scaled by 1/T_{d+1}(a),
    # a = (1+mu)/(1-mu): it takes +-1/T_{d+1}(a) alternately at the d+2
    # points where (1+mu-2z)/(1-mu) = cos(j pi/(d+1)), and r(0) = 1.
    c = O.poly_coeffs_cheb(d, mu)
    a = (1 + mu) / (1 - mu)
    Ta = np.cosh((d + 1) * np.arccosh(a))
    j = np.arange(d + 2)
    w = np.cos(j * np.pi / (d + 1))
    z = (1 + mu - w * (1 - mu)) / 2
    r = 1 - z * O.poly_eval(c, z)
    assert np.max(np.abs(r - (-1.0) ** j / Ta)) <= 1e-9
    zz = np.linspace(mu, 1, 4001)
    assert np.max(np.abs(1 - zz * O.poly_eval(c, zz))) <= 1 / Ta + 1e-9
    # p > 0 on (0, 1] (Thm "ppos")
    assert np.all(O.poly_eval(c, np.linspace(1e-6, 1, 4001)) > 0)


@pytest.mark.parametrize("d", [1, 3, 5])
def test_chebyshev_beats_l2_in_the_max_norm_on_mu_1(d):
    mu = 0.1
    zz = np.linspace(mu, 1, 4001)
    cheb = np.max(np.abs(1 - zz * O.poly_eval(O.poly_coeffs_cheb(d, mu), zz)))
    l2 = np.max(np.abs(1 - zz * O.poly_eval(O.poly_coeffs_l2(d), zz)))
    assert cheb < l2


# ---- weighted l2 design, Eq. "wl2cost" ----


def _moments(weight_terms, d):
    # w(z) = sum_t a_t z^e_t  ->  m_k = sum_t a_t / (k + e_t + 1), exact
    return [sum(Fraction(a) / (k + e + 1) for a, e in weight_terms) for k in range(2 * d + 3)]


@pytest.mark.parametrize("d", range(0, 9))
def test_wl2_with_unit_weight_is_the_l2_design(d):
    assert O.poly_coeffs_wl2(d, _moments([(1, 0)], d)) == O.poly_coeffs_l2(d)


@pytest.mark.parametrize("d", [1, 3, 5])
@pytest.mark.parametrize("terms", [[(1, 1)], [(1, 0), (3, 2)], [(2, 0), (-1, 1)]])
def test_wl2_matches_weighted_least_squares_by_quadrature(d, terms):
    # independent route: Gauss-Legendre nodes on [0, 1] (exact for these
    # polynomial integrands), weighted least squares on the discretised cost
    c = np.array([float(v) for v in O.poly_coeffs_wl2(d, _moments(terms, d))])
    xg, wg = np.polynomial.legendre.leggauss(40)
    z, wq = (xg + 1) / 2, wg / 2
    w = sum(a * z ** e for a, e in terms)
    assert np.all(w > 0)
    A = np.stack([z ** (i + 1) for i in range(d + 1)], axis=1) * np.sqrt(wq * w)[:, None]
    rhs = np.sqrt(wq * w)
    ref, *_ = np.linalg.lstsq(A, rhs, rcond=None)
    assert np.max(np.abs(c - ref)) <= 1e-7 * np.max(np.abs(ref))


def test_wl2_weight_shifts_the_residual_where_it_is_heavy():
    # a weight concentrated near z = 1 lowers |1 - z p(z)| there relative to
    # the unweighted design
    d = 3
    cw = [float(v) for v in O.poly_coeffs_wl2(d, _moments([(1, 6)], d))]
    cu = [float(v) for v in O.poly_coeffs_l2(d)]
    z = np.linspace(0.8, 1.0, 50)
    rw = np.abs(1 - z * O.poly_eval(cw, z))
    ru = np.abs(1 - z * O.poly_eval(cu, z))
    assert np.mean(rw) < np.mean(ru)


@pytest.mark.parametrize("mu", [1e-3, 0.05, 0.3])
@pytest.mark.parametrize("d", [1, 3, 5])
def test_max_zp_of_chebyshev_is_one_plus_reciprocal_t(d, mu):
    # on [mu, 1] the Chebyshev residual r = 1 - z p(z) equioscillates between
    # +-1/T_{d+1}(a), a = (1 + mu)/(1 - mu), and below mu it stays in (0, 1],
    # so max z p(z) = 1 + 1/T_{d+1}(a) (the step overshoot under FISTA)
    a = (1 + mu) / (1 - mu)
    want = 1 + 1 / math.cosh((d + 1) * math.acosh(a))
    assert abs(O.poly_max_zp(O.poly_coeffs_cheb(d, mu)) - want) <= 1e-6


def test_max_zp_of_the_l2_polynomials():
    # d = 0: z p(z) = 3z/2 peaks at z = 1; d = 1: z (4 - 10 z/3) peaks at z = 3/5
    assert abs(O.poly_max_zp([1.5]) - 1.5) <= 1e-12
    assert abs(O.poly_max_zp(O.poly_coeffs_l2(1)) - 1.2) <= 1e-9
