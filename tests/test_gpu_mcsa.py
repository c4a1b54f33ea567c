"""GPU parity of Technique II (Sec. 5.2): SA whose cost is the misfit of
Monte Carlo prices on common random numbers, against the oracle."""
import os

import numpy as np
import pytest

import oracle as O
import paper_2407_20713_gb300 as sg

pytestmark = pytest.mark.gpu

T = np.array([0.5, 0.5, 1.0, 1.0, 1.5])
K = np.array([0.9, 1.1, 0.9, 1.1, 1.0])


def _problem(model, lo, hi, prec, truth, **kw):
    mkt, _ = O.mc_price(model, truth, 1.0, T, K, n_paths=8192, steps_per_year=50, seed=77)
    pb = sg.CalibrationProblem(model=model, T=T, K=K, market=mkt, lo=lo, hi=hi, prec=prec, cost=sg.COST_MC_PRICE,
                               mc_paths=2048, mc_steps_per_year=50, mc_seed=5, **kw)
    return pb, mkt


@pytest.mark.parametrize("model,truth,lo,hi", [
    (sg.HAGAN, [0.25, 0.6, -0.3, 0.5], [0.25, 0.6, -0.9, 0.1], [0.25, 0.6, 0.5, 1.5]),
    (sg.DYN_I, [0.25, 0.8, -0.4, 0.6, 0.5, 0.8], [0.1, 0.8, -0.9, 0.1, 0.0, 0.0], [0.5, 0.8, 0.5, 1.5, 2.0, 2.0]),
    # DSabr_II, the paper's Technique II model (Sec. 6.2): infeasible
    # proposals (rho(t) or nu(t) out of range) are rejected on both sides
    (sg.DYN_II, [0.25, 0.8, -0.4, 0.6, 0.5, 0.8, 0.05, 0.1, 0.1, 0.1],
     [0.1, 0.8, -0.8, 0.2, 0.0, 0.0, -0.2, 0.0, -0.3, -0.3], [0.5, 0.8, 0.3, 1.2, 2.0, 2.0, 0.2, 0.3, 0.3, 0.3]),
])
def test_fp64_mc_cost_trajectory_is_the_oracle_trajectory(model, truth, lo, hi):
    pb, mkt = _problem(model, lo, hi, sg.FP64, truth, n_chains=6, n_levels=3, chain_len=4, seed=9)
    g = sg.calibrate(pb)
    o = O.sa_calibrate(model, 1.0, T, K, mkt, lo, hi, cost=O.COST_MC, n_chains=6, n_levels=3, chain_len=4,
                       mc_paths=2048, mc_steps_per_year=50, mc_seed=5, seed=9, n_threads=8)
    assert g.status == 0
    assert g.n_evals == o["n_evals"] and g.n_accepts == o["n_accepts"]
    np.testing.assert_allclose(g.params, o["params"], rtol=1e-9, atol=1e-13)
    assert g.misfit == pytest.approx(o["misfit"], rel=1e-8)
    assert g.misfit_fp64 == pytest.approx(o["misfit"], rel=1e-8)


def test_fp32_mc_cost_stays_close_to_the_oracle():
    truth = [0.25, 0.6, -0.3, 0.5]
    lo, hi = [0.25, 0.6, -0.9, 0.1], [0.25, 0.6, 0.5, 1.5]
    pb, mkt = _problem(sg.HAGAN, lo, hi, sg.FP32, truth, n_chains=16, n_levels=6, chain_len=6, seed=3)
    g = sg.calibrate(pb)
    o = O.sa_calibrate(sg.HAGAN, 1.0, T, K, mkt, lo, hi, cost=O.COST_MC, n_chains=16, n_levels=6, chain_len=6,
                       mc_paths=2048, mc_steps_per_year=50, mc_seed=5, seed=3, n_threads=8)
    assert g.status == 0
    # FP32 prices move the misfit by ~1e-5 relative per quote; trajectories may
    # part ways late, so compare outcomes: both reach the same basin.
    assert abs(g.misfit_fp64 - o["misfit"]) <= 0.5 * o["misfit"] + 1e-6
    np.testing.assert_allclose(g.params[2:], o["params"][2:], atol=0.1)


def test_fp32_mc_surface_fixed_beta_within_one_percent_of_the_oracle():
    # Technique II on the MC surface's shape (8 maturities x 15 calls, Sec.
    # 5.2 with the price misfit of Sec. 3 eq. error_calibrate_relativo), beta
    # fixed at its true value and a box of about +-50% around the truth, so
    # that the SA reaches its minimum; common random numbers make the cost a
    # deterministic function of the parameters.  The paths per evaluation
    # (1024 at 50 steps a year) are fewer than the benchmark's so that the
    # FP64 oracle runs the same schedule in seconds.  FP32 paths must end
    # within 1% of the oracle's final misfit.
    from paper_2407_20713_gb300 import workloads
    w = workloads.mc_surface()
    a, b, r, n = w.truth
    mkt, _ = O.mc_price(O.HAGAN, w.truth, 1.0, w.T, w.K, n_paths=1 << 18, steps_per_year=50,
                        seed=w.meta["market_seed"] & 0xFFFFFFFF)
    lo = [0.5 * a, b, max(-0.95, r - 0.4), 0.5 * n]
    hi = [1.5 * a, b, min(0.95, r + 0.4), 1.5 * n]
    kw = dict(n_chains=64, n_levels=30, chain_len=10, factor=0.8)
    for seed in (1, 2):
        pb = sg.CalibrationProblem(model=sg.HAGAN, T=w.T, K=w.K, market=mkt, lo=lo, hi=hi, prec=sg.FP32,
                                   cost=sg.COST_MC_PRICE, mc_paths=1024, mc_steps_per_year=50, mc_seed=5, seed=seed,
                                   **kw)
        g = sg.calibrate(pb)
        o = O.sa_calibrate(O.HAGAN, 1.0, w.T, w.K, mkt, lo, hi, cost=O.COST_MC, mc_paths=1024,
                           mc_steps_per_year=50, mc_seed=5, seed=seed, n_threads=os.cpu_count() or 8, **kw)
        assert g.status == 0
        assert abs(g.misfit_fp64 - o["misfit"]) <= 0.01 * o["misfit"], (seed, g.misfit_fp64, o["misfit"])
