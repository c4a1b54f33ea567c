"""Pins of the FP64 oracle's implied-volatility formulas against what the
paper and the mathematics fix (values the paper prints, its closed forms,
limits that reduce to textbook models, high-precision evaluation).
None of these re-derives a value through the oracle's own code path."""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.optimize import brentq

import oracle as O
from helpers import Golden, bachelier_call, black_call

mpmath = pytest.importorskip("mpmath")


# --------------------------------------------------------------------------
# Printed worked examples: Sec. 6.2, DSabr_I tables (forward convention of
# Sec. 2: f = S0 exp((r - y) T); dynamic formula eq. vola_SABRd, Case I).
# --------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["dsabr1_eurostoxx50.txt", "dsabr1_eurusd.txt"])
def test_dynamic_case1_reproduces_printed_surface(name):
    g = Golden(name)
    p = g.floats("params")
    S0 = g.floats("spot")[0]
    frac = g.meta["strike"][0] == "fraction_of_spot"
    worst = 0.0
    worst_spot_fwd = 0.0
    for T, r, y, k, printed in g.rows:
        K = k * S0 if frac else k
        f = S0 * math.exp((r - y) * T)
        v = 100.0 * O.vol_dynamic(1, p, f, K, T)
        worst = max(worst, abs(v - printed))
        worst_spot_fwd = max(worst_spot_fwd, abs(100.0 * O.vol_dynamic(1, p, S0, K, T) - printed))
    # printed to 4 decimals from single precision: 1e-4 vol-% covers both
    assert worst <= 1e-4, worst
    # the forward convention matters: using the spot misses by far more
    assert worst_spot_fwd > 1e-3


# --------------------------------------------------------------------------
# Sec. 2.2: constant nu and rho reduce the dynamic model to the static one,
# i.e. eq. vola_SABRd collapses to eq. vola_SABR.
# --------------------------------------------------------------------------
def test_dynamic_reduces_to_expanded_static_form():
    rng = np.random.default_rng(11)
    for _ in range(40):
        a, b, r, n = rng.uniform(0.05, 1.0), rng.uniform(0, 1), rng.uniform(-0.95, 0.95), rng.uniform(0.05, 2.0)
        K, T = rng.uniform(0.5, 1.6), rng.uniform(0.05, 8.0)
        ref = O.vol_expanded(a, b, r, n, 1.0, K, T)
        d1 = O.vol_dynamic(1, [a, b, r, n, 0.0, 0.0], 1.0, K, T)
        d2 = O.vol_dynamic(2, [a, b, r, n, 0, 0, 0, 0, 0, 0], 1.0, K, T)
        assert abs(d1 - ref) <= 1e-13 * abs(ref)
        assert abs(d2 - ref) <= 1e-13 * abs(ref)
        co = O.dyn_coeffs(1, [a, b, r, n, 0.0, 0.0], T)
        np.testing.assert_allclose(co, [n * n, n * n, n * r, n * n * r * r], rtol=1e-13, atol=1e-15)


def test_case2_with_zero_extras_is_case1():
    rng = np.random.default_rng(12)
    for _ in range(20):
        p = [0.3, 0.8, rng.uniform(-0.9, 0.9), rng.uniform(0.1, 1.5), rng.uniform(0, 3), rng.uniform(0, 3)]
        T = rng.uniform(0.1, 10)
        np.testing.assert_allclose(O.dyn_coeffs(2, p + [0, 0, 0, 0], T), O.dyn_coeffs(1, p, T),
                                   rtol=1e-12, atol=1e-16)


# --------------------------------------------------------------------------
# Case I closed forms, Sec. 2.2 eq. exact-integral-expressions, in a range of
# (a+b)T and 2bT where they lose no more than a few digits.
# --------------------------------------------------------------------------
def case1_closed_forms(p, T):
    nu0, rho0, a, b = p[3], p[2], p[4], p[5]
    x = 2 * b * T
    y = (a + b) * T
    nu1 = 6 * nu0 ** 2 / x ** 3 * ((x * x / 2 - x + 1) - math.exp(-x))
    nu2 = 6 * nu0 ** 2 / x ** 3 * (2 * (math.exp(-x) - 1) + x * (math.exp(-x) + 1))
    eta1 = 2 * nu0 * rho0 / (T * T * (a + b) ** 2) * (math.exp(-y) - (1 - y))
    eta2 = 3 * nu0 ** 2 * rho0 ** 2 / (T ** 4 * (a + b) ** 4) * (
        math.exp(-2 * y) - 8 * math.exp(-y) + (7 + 2 * y * (-3 + y)))
    return np.array([nu1, nu2, eta1, eta2])


def test_case1_matches_paper_closed_forms():
    rng = np.random.default_rng(13)
    for _ in range(40):
        T = rng.uniform(0.2, 10)
        a, b = rng.uniform(0.5, 3) / T, rng.uniform(0.5, 3) / T
        p = [0.3, 0.6, rng.uniform(-1, 1), rng.uniform(0.1, 2), a, b]
        np.testing.assert_allclose(O.dyn_coeffs(1, p, T), case1_closed_forms(p, T), rtol=1e-9)


def test_case1_small_rate_limits():
    # as a, b -> 0 the four functions tend to nu0^2, nu0^2, nu0 rho0, nu0^2 rho0^2
    p = [0.3, 0.6, -0.7, 0.9, 1e-9, 2e-9]
    np.testing.assert_allclose(O.dyn_coeffs(1, p, 2.0), [0.81, 0.81, -0.63, 0.3969], rtol=1e-8)


# --------------------------------------------------------------------------
# Case II: the paper's Appendix A closed forms for nu1^2, nu2^2 and eta1.
# --------------------------------------------------------------------------
def appendix_a(p, T):
    _, _, r0, n0, a, b, dr, dn, qr, qn = p
    e = math.exp
    nu1 = (9 * qn ** 2 + 6 * b ** 4 * n0 * (4 * dn + n0) * T ** 2 + 4 * b ** 5 * dn ** 2 * T ** 3
           + 9 * b * qn * (16 * dn + n0 - qn * T)
           + 6 * b ** 3 * T * (-n0 * (8 * dn + n0) + (4 * dn + n0) * qn * T)
           + 3 * b ** 2 * (n0 * (16 * dn + n0) - 4 * (8 * dn + n0) * qn * T + qn ** 2 * T ** 2)
           - 3 * e(-2 * b * T) * (3 * qn ** 2 + 3 * b * qn * (16 * dn * e(b * T) + n0 + qn * T)
                                  + b ** 2 * (n0 + qn * T) * (16 * dn * e(b * T) + n0 + qn * T))
           ) / (4 * b ** 5 * T ** 3)
    inner = (-18 * qn ** 2 + 6 * b ** 3 * n0 * (8 * dn + n0) * T + 4 * b ** 5 * dn ** 2 * T ** 3
             + 9 * b * qn * (-32 * dn - 2 * n0 + qn * T)
             + 6 * b ** 2 * (-n0 * (16 * dn + n0) + 2 * (8 * dn + n0) * qn * T))
    nu2 = e(-2 * b * T) * (18 * qn ** 2 + 6 * b ** 3 * T * (n0 + qn * T) ** 2
                           + 6 * b ** 2 * (n0 + qn * T) * (n0 + 3 * qn * T)
                           + 9 * b * qn * (2 * n0 + 3 * qn * T) + e(2 * b * T) * inner
                           + 48 * b * dn * e(b * T) * (6 * qn + b * (n0 * (2 + b * T) + qn * T * (4 + b * T)))
                           ) / (4 * b ** 5 * T ** 3)
    s = a + b
    t1 = (-2 * dn * qr / a ** 3 - 2 * dr * qn / b ** 3 - 6 * qr * qn / s ** 4 + dr * n0 * T / b + dn * r0 * T / a
          + a ** 3 * n0 * r0 * T / s ** 4 + b ** 3 * n0 * r0 * T / s ** 4
          + dn * (-r0 + qr * T) / a ** 2 + dr * (-n0 + qn * T) / b ** 2
          + a ** 2 * (-n0 * r0 + n0 * qr * T + qn * r0 * T) / s ** 4
          - 2 * a * (n0 * qr + qn * (r0 - qr * T)) / s ** 4
          + b * (-2 * n0 * (qr + a * r0) + a * n0 * (2 * qr + 3 * a * r0) * T
                 + 2 * qn * (qr * T + r0 * (-1 + a * T))) / s ** 4
          + b ** 2 * (qn * r0 * T + n0 * (qr * T + r0 * (-1 + 3 * a * T))) / s ** 4)
    ebt, eat, est = e(b * T), e(a * T), e(s * T)
    big = (4 * b ** 7 * dn * ebt * qr + 8 * a ** 2 * b ** 5 * dn * ebt * (b * r0 + qr * (3 + b * T))
           + 2 * a * b ** 6 * dn * ebt * (b * r0 + qr * (8 + b * T))
           + a ** 7 * dr * eat * (4 * qn + b ** 3 * dn * ebt * T ** 2 + 2 * b * (n0 + qn * T))
           + 4 * a ** 6 * b * dr * eat * (4 * qn + b ** 3 * dn * ebt * T ** 2 + 2 * b * (n0 + qn * T))
           + 2 * a ** 5 * b ** 2 * (12 * dr * eat * qn + 3 * b ** 3 * dr * dn * est * T ** 2
                                    + 6 * b * dr * eat * (n0 + qn * T)
                                    + b * (r0 + qr * T) * (dn * ebt + n0 + qn * T))
           + 4 * a ** 4 * b ** 3 * (dn * ebt * qr + n0 * qr + 4 * dr * eat * qn + qn * r0 + 2 * qr * qn * T
                                    + b ** 3 * dr * dn * est * T ** 2 + 2 * b * dr * eat * (n0 + qn * T)
                                    + b * (r0 + qr * T) * (2 * dn * ebt + n0 + qn * T))
           + a ** 3 * b ** 3 * (12 * qr * qn + b ** 4 * dr * dn * est * T ** 2
                                + 4 * b * (4 * dn * ebt * qr + n0 * qr + qn * (dr * eat + r0 + 2 * qr * T))
                                + 2 * b ** 2 * (dr * eat * (n0 + qn * T) + (r0 + qr * T) * (6 * dn * ebt + n0 + qn * T))))
    eta1 = 2 / T ** 2 * (t1 + e(-s * T) * big / (2 * a ** 3 * b ** 3 * s ** 4))
    return nu1, nu2, eta1


def test_case2_matches_appendix_a_closed_forms():
    rng = np.random.default_rng(14)
    for _ in range(30):
        p = [0.3, 0.8, rng.uniform(-0.8, 0.2), rng.uniform(0.2, 1.0), rng.uniform(0.3, 2.0), rng.uniform(0.3, 2.0),
             rng.uniform(-0.2, 0.2), rng.uniform(0, 0.3), rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3)]
        T = rng.uniform(0.5, 5)
        co = O.dyn_coeffs(2, p, T)
        nu1, nu2, eta1 = appendix_a(p, T)
        assert abs(co[0] - nu1) <= 1e-11 * abs(nu1)
        assert abs(co[1] - nu2) <= 1e-11 * abs(nu2)
        assert abs(co[2] - eta1) <= 1e-11 * max(abs(eta1), 1e-3)


def test_eta2_matches_literal_triple_integral():
    # eta2^2 = 12/T^4 int_0^T int_0^t (int_0^s nu rho du)^2 ds dt, by scipy
    for case, p, T in [(1, [0.3, 0.8, -0.6, 0.8, 0.4, 0.9], 1.7),
                       (2, [0.3, 0.8, -0.5, 0.7, 1.1, 0.6, 0.1, 0.2, 0.25, -0.2], 2.3)]:
        nurho = lambda u: O.nu_t(case, p, u) * O.rho_t(case, p, u)
        G = lambda s: integrate.quad(nurho, 0, s, epsabs=1e-14, epsrel=1e-13)[0]
        inner = lambda t: integrate.quad(lambda s: G(s) ** 2, 0, t, epsabs=1e-14, epsrel=1e-12)[0]
        val = 12 / T ** 4 * integrate.quad(inner, 0, T, epsabs=1e-14, epsrel=1e-11)[0]
        assert abs(O.dyn_coeffs(case, p, T)[3] - val) <= 1e-9 * abs(val)


def test_dyn_coeffs_match_scipy_quadrature_of_definitions():
    rng = np.random.default_rng(15)
    for _ in range(6):
        case = 2
        p = [0.3, 0.8, rng.uniform(-0.8, 0.2), rng.uniform(0.2, 1.0), rng.uniform(0.0, 40.0), rng.uniform(0.0, 40.0),
             rng.uniform(-0.2, 0.2), rng.uniform(0, 0.3), rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3)]
        T = rng.uniform(0.1, 10)
        nu = lambda t: O.nu_t(case, p, t)
        rho = lambda t: O.rho_t(case, p, t)
        q = lambda fn: integrate.quad(fn, 0, T, epsabs=0, epsrel=1e-13, limit=400)[0]
        ref = [3 / T ** 3 * q(lambda t: (T - t) ** 2 * nu(t) ** 2),
               6 / T ** 3 * q(lambda t: (T - t) * t * nu(t) ** 2),
               2 / T ** 2 * q(lambda t: (T - t) * nu(t) * rho(t))]
        np.testing.assert_allclose(O.dyn_coeffs(case, p, T)[:3], ref, rtol=1e-10)


# --------------------------------------------------------------------------
# x(z), Sec. 2.1 eq. equis: 50-digit evaluation, and its integral form.
# --------------------------------------------------------------------------
def test_x_of_z_against_50_digit_evaluation():
    mpmath.mp.dps = 50
    for rho in [-0.999999, -0.9, -0.4, 0.0, 0.5, 0.95, 0.999]:
        for z in [1e-9, 3e-6, 9.9e-3, 1.01e-2, 0.3, 1.0, 4.0, 25.0]:
            for s in (1, -1):
                zz = s * z
                zm, rm = mpmath.mpf(zz), mpmath.mpf(rho)
                ref = mpmath.log((mpmath.sqrt(1 - 2 * rm * zm + zm * zm) + zm - rm) / (1 - rm))
                got = O.x_of_z(zz, rho)
                # the printed log form loses a few ulps where its argument nears 1
                assert abs(got - float(ref)) <= 1e-14 * abs(float(ref)), (rho, zz, got, float(ref))


def test_x_of_z_is_the_integral_of_the_legendre_kernel():
    for rho, z in [(-0.5, 0.7), (0.3, -1.5), (0.8, 2.0), (-0.9, -0.005)]:
        val = integrate.quad(lambda s: 1 / math.sqrt(1 - 2 * rho * s + s * s), 0, z, epsabs=0, epsrel=2e-14)[0]
        assert abs(O.x_of_z(z, rho) - val) <= 2e-13 * abs(val)


def test_z_over_x_is_continuous_at_the_series_switch():
    for rho in [-0.8, 0.0, 0.6]:
        a = O.z_over_x(0.01 * (1 - 1e-12), rho)
        b = O.z_over_x(0.01 * (1 + 1e-12), rho)
        assert abs(a - b) <= 1e-14
    assert O.z_over_x(0.0, 0.3) == 1.0


# --------------------------------------------------------------------------
# Static formulas: limits fixed by the model (Sec. 2, beta = 1 lognormal,
# beta = 0 normal) and relations between the three printed forms.
# --------------------------------------------------------------------------
def test_hagan_lognormal_limit_is_alpha():
    for alpha in [0.05, 0.2, 0.7]:
        for K in [0.5, 1.0, 1.7]:
            for T in [0.1, 1.0, 10.0]:
                for rho in [-0.5, 0.4]:
                    assert O.vol_hagan(alpha, 1.0, rho, 0.0, 1.0, K, T) == pytest.approx(alpha, rel=1e-15, abs=0)


def test_hagan_normal_limit_matches_bachelier_implied_black_vol():
    # beta = 0, nu = 0 is the normal model dF = alpha dW: the Black vol that
    # reprices the Bachelier call, up to the formula's truncation error.
    for a in [0.05, 0.1, 0.15]:
        for T in [0.5, 1.0, 2.0]:
            for K in np.linspace(0.8, 1.25, 10):
                price = bachelier_call(1.0, K, T, a)
                iv = brentq(lambda s: black_call(1.0, K, T, s) - price, 1e-4, 5, xtol=1e-15, rtol=1e-15)
                L = math.log(1.0 / K)
                bound = 0.02 * a * a * T * (L * L + a * a * T)
                assert abs(O.vol_hagan(a, 0.0, 0.0, 0.0, 1.0, K, T) - iv) <= bound * iv + 1e-12


def test_expanded_A1_is_the_first_taylor_coefficient_of_hagan_and_obloj():
    # eq. vola_SABR: sigma = (1/omega)(1 + A1 L + ...), L = ln(K/f); at T = 0
    # the slope of Hagan's and Oblój's sigma in L at the money is A1/omega.
    h = 1e-4
    for a, b, r, n in [(0.2, 0.7, -0.4, 0.5), (0.3, 0.5, 0.3, 1.2), (0.1, 0.9, -0.8, 0.3)]:
        w = 1.0 / a
        A1 = -0.5 * (1 - b - r * n * w)
        for fn in (O.vol_hagan, O.vol_obloj, O.vol_expanded):
            slope = (fn(a, b, r, n, 1.0, math.exp(h), 0.0) - fn(a, b, r, n, 1.0, math.exp(-h), 0.0)) / (2 * h)
            assert abs(slope * w - A1) <= 1e-6


def test_obloj_equals_hagan_at_beta_one_and_at_the_money():
    rng = np.random.default_rng(16)
    for _ in range(50):
        a, r, n = rng.uniform(0.05, 1), rng.uniform(-0.95, 0.95), rng.uniform(0.05, 2)
        K, T, b = rng.uniform(0.5, 1.6), rng.uniform(0.05, 5), rng.uniform(0, 1)
        assert O.vol_obloj(a, 1.0, r, n, 1.0, K, T) == pytest.approx(O.vol_hagan(a, 1.0, r, n, 1.0, K, T), rel=1e-14)
        assert O.vol_obloj(a, b, r, n, 1.3, 1.3, T) == pytest.approx(O.vol_hagan(a, b, r, n, 1.3, 1.3, T), rel=1e-14)


def test_obloj_is_continuous_in_beta_at_one():
    v1 = O.vol_obloj(0.2, 1.0, -0.3, 0.6, 1.0, 0.8, 1.0)
    v2 = O.vol_obloj(0.2, 1.0 - 1e-9, -0.3, 0.6, 1.0, 0.8, 1.0)
    assert abs(v1 - v2) <= 1e-8


def test_quadrature_is_exact_on_polynomials():
    rng = np.random.default_rng(17)
    for deg in [0, 3, 9, 19, 25]:
        c = rng.normal(size=deg + 1)
        a, b = -0.7, 2.3
        exact = sum(c[k] * (b ** (k + 1) - a ** (k + 1)) / (k + 1) for k in range(deg + 1))
        assert abs(O.integrate_poly(c, a, b) - exact) <= 1e-12 * max(1.0, abs(exact)) * (1 + deg)


def test_misfit_definition():
    assert O.misfit([1.0, 2.0], [2.0, 4.0]) == pytest.approx(0.5)


def test_feasibility_against_dense_sampling():
    rng = np.random.default_rng(18)
    agree = 0
    for _ in range(400):
        p = [0.3, 0.8, rng.uniform(-1, 1), rng.uniform(0.01, 1.5), rng.uniform(0, 3), rng.uniform(0, 3),
             rng.uniform(-0.6, 0.6), rng.uniform(-0.5, 0.5), rng.uniform(-2, 2), rng.uniform(-2, 2)]
        Tmax = rng.uniform(0.5, 10)
        t = np.linspace(0, Tmax, 20001)
        rho = (p[2] + p[8] * t) * np.exp(-p[4] * t) + p[6]
        nu = (p[3] + p[9] * t) * np.exp(-p[5] * t) + p[7]
        dense = bool(rho.min() >= -1 and rho.max() <= 1 and nu.min() > 0)
        margin = min(abs(rho.min() + 1), abs(rho.max() - 1), abs(nu.min()))
        if margin < 1e-5:
            continue
        assert O.feasible(4, p, Tmax) == dense, p
        agree += 1
    assert agree > 300
