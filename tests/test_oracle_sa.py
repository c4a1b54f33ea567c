"""Pins of the oracle's synchronous parallel Simulated Annealing (Sec. 5):
brute-force search on a tiny two-parameter problem, invariants of the
proposal/acceptance bookkeeping, and agreement of Technique II's cost with a
direct Monte Carlo evaluation."""
import numpy as np

import oracle as O

K15 = 0.6 + 0.8 * np.arange(15) / 14
T15 = np.ones(15)
TRUTH = [0.2, 0.7, -0.4, 0.5]


def _market(noise=1e-4, seed=20240720):
    rng = np.random.default_rng(seed)
    return O.implied_vol(O.HAGAN, TRUTH, 1.0, T15, K15) + rng.normal(0, noise, 15)


def test_sa_agrees_with_brute_force_grid_on_rho_nu():
    mkt = _market()
    rho = np.linspace(-0.9, 0.5, 141)
    nu = np.linspace(0.1, 1.5, 141)
    best = (np.inf, None)
    for r in rho:
        for n in nu:
            m = O.misfit(O.implied_vol(O.HAGAN, [0.2, 0.7, r, n], 1.0, T15, K15), mkt)
            if m < best[0]:
                best = (m, (r, n))
    h = rho[1] - rho[0]
    lo = [0.2, 0.7, -0.9, 0.1]
    hi = [0.2, 0.7, 0.5, 1.5]
    res = O.sa_calibrate(O.HAGAN, 1.0, T15, K15, mkt, lo, hi, n_chains=64, seed=3, n_threads=4)
    assert res["misfit"] <= best[0] * (1 + 1e-9)
    assert abs(res["params"][2] - best[1][0]) <= h and abs(res["params"][3] - best[1][1]) <= h
    # fixed coordinates (lo == hi) never move
    assert res["params"][0] == 0.2 and res["params"][1] == 0.7
    # and the returned misfit is the cost of the returned point
    m = O.misfit(O.implied_vol(O.HAGAN, res["params"], 1.0, T15, K15), mkt)
    assert m == res["misfit"]


def test_sa_noise_free_two_parameter_recovery():
    mkt = _market(noise=0.0)
    lo = [0.2, 0.7, -0.99, 0.01]
    hi = [0.2, 0.7, 0.99, 3.0]
    res = O.sa_calibrate(O.HAGAN, 1.0, T15, K15, mkt, lo, hi, n_chains=64, factor=0.9, seed=1, n_threads=4)
    assert res["misfit"] < 1e-12
    np.testing.assert_allclose(res["params"][2:], TRUTH[2:], atol=2e-5)


def test_sa_bookkeeping_and_thread_independence():
    mkt = _market()
    lo = [1e-6, 0.0, -1 + 1e-6, 1e-6]
    hi = [2.0, 1.0, 1 - 1e-6, 3.0]
    kw = dict(n_chains=16, n_levels=12, chain_len=20, seed=42)
    r1 = O.sa_calibrate(O.HAGAN, 1.0, T15, K15, mkt, lo, hi, n_threads=1, trace=True, **kw)
    r4 = O.sa_calibrate(O.HAGAN, 1.0, T15, K15, mkt, lo, hi, n_threads=4, trace=True, **kw)
    for k in ("misfit", "n_evals", "n_accepts", "restart_misfit"):
        assert r1[k] == r4[k]
    assert np.array_equal(r1["params"], r4["params"]) and np.array_equal(r1["trace"], r4["trace"])
    assert 0 < r1["n_accepts"] <= r1["n_evals"] <= 16 * 12 * 20
    assert r1["misfit"] <= r1["restart_misfit"]
    assert np.all(np.asarray(r1["params"]) >= lo) and np.all(np.asarray(r1["params"]) <= hi)
    # the starting point is the box midpoint: the best can only improve on it
    f0 = O.misfit(O.implied_vol(O.HAGAN, [0.5 * (a + b) for a, b in zip(lo, hi)], 1.0, T15, K15), mkt)
    assert r1["misfit"] <= f0


def test_sa_rejects_infeasible_case2_proposals():
    # Case II constraints (Sec. 5.2): every returned point is feasible.
    T = np.repeat([0.5, 1.0, 2.0], 5)
    K = np.tile(np.linspace(0.8, 1.2, 5), 3)
    truth = [0.25, 0.8, -0.4, 0.6, 0.8, 0.9, 0.1, 0.15, 0.2, -0.1]
    mkt = O.implied_vol(O.DYN_II, truth, 1.0, T, K)
    lo = [0.05, 0.5, -1.0, 0.01, 0.0, 0.0, -0.5, -0.3, -1.0, -1.0]
    hi = [0.6, 1.0, 1.0, 1.5, 3.0, 3.0, 0.5, 0.5, 1.0, 1.0]
    res = O.sa_calibrate(O.DYN_II, 1.0, T, K, mkt, lo, hi, n_chains=8, n_levels=6, chain_len=10, seed=5)
    assert O.feasible(O.DYN_II, res["params"], 2.0)
    assert O.feasible(O.DYN_II, res["restart_params"], 2.0)


def test_sa_mc_cost_is_the_mc_price_misfit():
    # Technique II: the cost is eq. error_calibrate_relativo on MC prices with
    # common random numbers (the same paths for every evaluation).
    T = np.array([0.5, 0.5, 1.0, 1.0])
    K = np.array([0.9, 1.1, 0.9, 1.1])
    truth = [0.25, 0.6, -0.3, 0.5]
    mkt, _ = O.mc_price(O.HAGAN, truth, 1.0, T, K, n_paths=4096, steps_per_year=50, seed=77)
    lo = [0.25, 0.6, -0.9, 0.1]
    hi = [0.25, 0.6, 0.5, 1.5]
    res = O.sa_calibrate(O.HAGAN, 1.0, T, K, mkt, lo, hi, cost=O.COST_MC, n_chains=4, n_levels=3, chain_len=4,
                         mc_paths=1024, mc_steps_per_year=50, mc_seed=5, seed=9)
    price, _ = O.mc_price(O.HAGAN, res["params"], 1.0, T, K, n_paths=1024, steps_per_year=50, seed=5)
    assert res["misfit"] == O.misfit(price, mkt)
