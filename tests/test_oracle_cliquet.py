"""Pins of the oracle's cliquet pricer (Sec. 6.3, eqs. (eq_cliquet) and
(cliquet_global)).

With nu = 0 and beta = 1 the SABR forward is a geometric Brownian motion
with volatility alpha and the log-Euler step is exact, so the local returns
R_i = F(d_i)/F(d_{i-1}) - 1 are i.i.d. with 1 + R lognormal of mean 1:
  * without global limits the price is (n-1) E[max(min(R, C), F)] and
    E[max(min(R, C), F)] = F + C_B(1, 1+F) - C_B(1, 1+C), a call spread on
    the gross return (Black formula, unit forward);
  * with global limits the expectation of max(F_g, min(C_g, sum)) follows
    from the exact law of one clipped return (atoms at F and C, lognormal
    density between) convolved n-1 times on a fine grid.
"""
import pytest

import oracle as O
from helpers import black_call, exact_gbm_cliquet


def test_cliquet_without_global_limits_is_a_sum_of_call_spreads():
    a, T, n = 0.2, 1.0, 4
    dt = T / n
    fl, cl = -0.02, 0.02
    per = fl + black_call(1.0, 1.0 + fl, dt, a) - black_call(1.0, 1.0 + cl, dt, a)
    ref = (n - 1) * per
    # the convolution route agrees with the closed form
    assert exact_gbm_cliquet(a, T, n, fl, cl, -1.0, 1.0) == pytest.approx(ref, abs=1e-9)
    price, se = O.mc_cliquet(O.HAGAN, [a, 1.0, -0.3, 0.0], 1.0, T, n, fl, cl, -1e9, 1e9, n_paths=1 << 15,
                             steps_per_year=250, seed=4, n_threads=8)
    assert abs(price - ref) <= 4 * se + 1e-12


@pytest.mark.parametrize("fg,cg", [(-0.01, 0.02), (0.0, 0.2), (0.005, 0.03)])
def test_cliquet_global_limits_match_the_exact_law(fg, cg):
    a, T, n, fl, cl = 0.25, 1.0, 4, -0.02, 0.02
    ref = exact_gbm_cliquet(a, T, n, fl, cl, fg, cg)
    price, se = O.mc_cliquet(O.HAGAN, [a, 1.0, 0.2, 0.0], 1.0, T, n, fl, cl, fg, cg, n_paths=1 << 15,
                             steps_per_year=100, seed=9, n_threads=8)
    assert abs(price - ref) <= 4 * se + 1e-12
    # the limits in the printed order, max(C_g, min(F_g, .)), would be C_g
    # whenever F_g <= C_g: the reading must not be that constant
    assert abs(price - cg) > 10 * se


def test_cliquet_two_resets_is_one_clipped_return():
    a, T = 0.3, 0.5
    dt = T / 2
    fl, cl = -0.05, 0.04
    ref = fl + black_call(1.0, 1.0 + fl, dt, a) - black_call(1.0, 1.0 + cl, dt, a)
    price, se = O.mc_cliquet(O.HAGAN, [a, 1.0, 0.0, 0.0], 1.0, T, 2, fl, cl, -1e9, 1e9, n_paths=1 << 15,
                             steps_per_year=52, seed=5, n_threads=8)
    assert abs(price - ref) <= 4 * se + 1e-12


def test_cliquet_global_limits_and_discount():
    args = (O.HAGAN, [0.25, 0.7, -0.4, 0.6], 1.0, 1.0, 4, -0.02, 0.02)
    free, _ = O.mc_cliquet(*args, -1e9, 1e9, n_paths=8192, seed=2, n_threads=4)
    capped, _ = O.mc_cliquet(*args, -1e9, 0.01, n_paths=8192, seed=2, n_threads=4)
    floored, _ = O.mc_cliquet(*args, 0.0, 1e9, n_paths=8192, seed=2, n_threads=4)
    both, _ = O.mc_cliquet(*args, 0.0, 0.2, n_paths=8192, seed=2, n_threads=4)
    assert capped <= free <= floored and 0.0 <= both <= 0.2
    disc, _ = O.mc_cliquet(*args, 0.0, 0.2, disc=0.9, n_paths=8192, seed=2, n_threads=4)
    assert disc == pytest.approx(0.9 * both, rel=1e-15)


def test_cliquet_dynamic_models_with_zero_vol_of_vol_are_gbm():
    # DSabr_I with nu0 = 0 keeps alpha constant; Case II needs nu(t) > 0, and
    # nu(t) = 1e-9 moves alpha by about 1e-9 relative
    a, T, n, fl, cl, fg, cg = 0.15, 1.0, 4, -0.02, 0.02, 0.0, 0.2
    ref = exact_gbm_cliquet(a, T, n, fl, cl, fg, cg)
    for model, p in [(O.DYN_I, [a, 1.0, -0.5, 0.0, 1.0, 1.0]),
                     (O.DYN_II, [a, 1.0, -0.5, 0.0, 1.0, 1.0, 0.1, 1e-9, 0.2, 0.0])]:
        price, se = O.mc_cliquet(model, p, 1.0, T, n, fl, cl, fg, cg, n_paths=1 << 14, steps_per_year=100,
                                 seed=3, n_threads=8)
        assert abs(price - ref) <= 4 * se + 1e-12
