"""Pins of the oracle's conditional-Bessel Monte Carlo step (the low-bias
scheme Sec. 4 names as the fallback for log-Euler) to what the mathematics
fixes, independently of the oracle itself:

* its Gamma sampler against the Gamma law (scipy's CDF, Kolmogorov-Smirnov);
* nu = 0, rho = 0: the step samples the absorbed CEV law exactly, at any step
  size, so one step to maturity must give the closed form (tests/helpers.py
  cev_call) and the probability of absorption must be Q(a, m), the
  regularised upper incomplete gamma function;
* beta = 1, nu = 0: Black's formula, at any step size;
* |rho| = 1, nu = 0 (the branch where the Bessel clock stops): the CEV law
  again, as the step shrinks;
* nu > 0: the same prices as the log-Euler scheme on a fine grid (the
  log-Euler oracle is pinned separately), for static and dynamic
  parameters, from 4 steps a year.
"""
import numpy as np
import pytest
from scipy import stats
from scipy.special import gammaincc

import oracle as O
from helpers import black_call, cev_call

K3 = np.array([0.7, 1.0, 1.4])


def _z(got, se, ref):
    return np.abs(got - ref) / se


@pytest.mark.parametrize("a", [0.5, 0.7, 1.0, 3.2, 50.0])
def test_gamma_sampler_follows_the_gamma_law(a):
    g = O.mb_gamma_draws(a, 100000, seed=3)
    assert stats.kstest(g, stats.gamma(a).cdf).pvalue > 1e-4
    assert abs(g.mean() - a) <= 5 * np.sqrt(a / g.size)


@pytest.mark.parametrize("alpha,beta,T", [(0.3, 0.5, 1.0), (0.6, 0.3, 2.0), (0.3, 0.0, 1.0), (0.4, 0.8, 0.5)])
@pytest.mark.parametrize("per_maturity", [1, 12])
def test_bessel_step_is_exact_for_cev(alpha, beta, T, per_maturity):
    # calls, and a put of strike 1e-6 whose price / strike is P(F_T = 0)
    K = np.append(K3, 1e-6)
    ic = np.array([1, 1, 1, 0], np.int8)
    n = 1 << 17
    got, se = O.mc_price(O.HAGAN, [alpha, beta, 0.0, 0.0], 1.0, np.full(4, T), K, is_call=ic, n_paths=n,
                         steps_per_year=per_maturity / T - 1e-9 if per_maturity == 1 else per_maturity, seed=5,
                         n_threads=8, scheme=O.MC_BESSEL)
    ref = np.array([cev_call(1.0, k, T, alpha, beta) for k in K3])
    assert np.all(_z(got[:3], se[:3], ref) <= 4.0), _z(got[:3], se[:3], ref)
    a = 0.5 + beta / (2 * (1 - beta))
    m = (1.0 / (1 - beta)) ** 2 / (2 * alpha * alpha * T)
    p_abs = gammaincc(a, m)
    assert abs(got[3] / 1e-6 - p_abs) <= 4 * np.sqrt(max(p_abs, 1.0 / n) / n)


@pytest.mark.parametrize("spy", [0.99, 12])
def test_bessel_lognormal_branch_is_black(spy):
    K = np.array([0.8, 1.0, 1.3])
    got, se = O.mc_price(O.HAGAN, [0.25, 1.0, 0.5, 0.0], 1.0, np.ones(3), K, n_paths=1 << 17, steps_per_year=spy,
                         seed=9, n_threads=8, scheme=O.MC_BESSEL)
    assert np.all(_z(got, se, black_call(1.0, K, 1.0, 0.25)) <= 4.0)


@pytest.mark.parametrize("rho", [1.0, -1.0])
def test_bessel_unit_correlation_branch_converges_to_cev(rho):
    got, se = O.mc_price(O.HAGAN, [0.3, 0.5, rho, 0.0], 1.0, np.ones(3), K3, n_paths=1 << 16, steps_per_year=200,
                         seed=11, n_threads=8, scheme=O.MC_BESSEL)
    ref = np.array([cev_call(1.0, k, 1.0, 0.3, 0.5) for k in K3])
    assert np.all(np.abs(got - ref) <= 4 * se + 2e-4), got - ref


@pytest.mark.parametrize("model,p", [(O.HAGAN, [0.5, 0.3, 0.3, 0.8]), (O.HAGAN, [0.3, 0.5, -0.6, 0.6]),
                                     (O.DYN_I, [0.3, 0.7, -0.6, 0.9, 0.5, 1.2])])
def test_bessel_agrees_with_fine_log_euler(model, p):
    # 4 steps a year against log-Euler at 400 (independent streams); the
    # allowance covers log-Euler's own first-order bias at that grid
    T = np.repeat([0.5, 1.0], 3)
    K = np.tile(K3, 2)
    pb, sb = O.mc_price(model, p, 1.0, T, K, n_paths=1 << 17, steps_per_year=4, seed=21, n_threads=8,
                        scheme=O.MC_BESSEL)
    pl, sl = O.mc_price(model, p, 1.0, T, K, n_paths=1 << 17, steps_per_year=400, seed=22, n_threads=8)
    assert np.all(np.abs(pb - pl) <= 4 * np.hypot(sb, sl) + 5e-4), pb - pl


def test_bessel_rejects_unknown_scheme_and_is_thread_count_free():
    T, K = np.ones(3), K3
    a = O.mc_price(O.HAGAN, [0.3, 0.5, -0.3, 0.4], 1.0, T, K, n_paths=5000, steps_per_year=10, seed=2, n_threads=1,
                   scheme=O.MC_BESSEL)
    b = O.mc_price(O.HAGAN, [0.3, 0.5, -0.3, 0.4], 1.0, T, K, n_paths=5000, steps_per_year=10, seed=2, n_threads=7,
                   scheme=O.MC_BESSEL)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    with pytest.raises(ValueError):
        O.mc_price(O.HAGAN, [0.3, 0.5, -0.3, 0.4], 1.0, T, K, n_paths=5000, scheme=7)
