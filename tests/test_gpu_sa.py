"""GPU parity of sabr_calibrate / sabr_calibrate_batch (Sec. 5 synchronous
parallel SA) with the FP64 oracle.

FP64: the same Philox streams and operation order give the oracle's
trajectory, so best point, restart point and counters agree to rounding.
FP32: trajectories part ways, so the bar is the final misfit within 1% of the
oracle's on a problem the method solves to its minimum, and recovery of the
synthetic truth."""
import os

import numpy as np
import pytest

import oracle as O
import paper_2407_20713_gb300 as sg

pytestmark = pytest.mark.gpu

K15 = 0.6 + 0.8 * np.arange(15) / 14
T15 = np.ones(15)
TRUTH = [0.2, 0.7, -0.4, 0.5]
LO4 = [1e-6, 0.0, -1 + 1e-6, 1e-6]
HI4 = [2.0, 1.0, 1 - 1e-6, 3.0]


def market(model=O.HAGAN, truth=TRUTH, T=T15, K=K15, noise=1e-4, seed=20240720):
    rng = np.random.default_rng(seed)
    return O.implied_vol(model, truth, 1.0, T, K) + rng.normal(0, noise, len(T))


def run_both(model, T, K, mkt, lo, hi, prec=sg.FP64, **kw):
    pb = sg.CalibrationProblem(model=model, T=T, K=K, market=mkt, lo=lo, hi=hi, prec=prec, **kw)
    g = sg.calibrate(pb)
    o = O.sa_calibrate(model, 1.0, T, K, mkt, lo, hi, n_chains=pb.n_chains, T0=pb.T0, factor=pb.factor,
                       n_levels=pb.n_levels, chain_len=pb.chain_len, step0=pb.step0, step_min=pb.step_min,
                       seed=pb.seed, x0=pb.x0, n_threads=8)
    return g, o


def dyn_surface(model, n_mats=3, n_strikes=5):
    mats = np.array([0.25, 1.0, 3.0, 0.5, 2.0, 5.0][:n_mats])
    T = np.repeat(mats, n_strikes)
    K = np.tile(np.linspace(0.8, 1.25, n_strikes), n_mats)
    if model == O.DYN_I:
        truth = [0.25, 0.8, -0.5, 0.7, 0.6, 0.9]
        lo = [0.05, 0.5, -1.0, 0.01, 0.0, 0.0]
        hi = [0.6, 1.0, 1.0, 1.5, 3.0, 3.0]
    else:
        truth = [0.25, 0.8, -0.4, 0.6, 0.8, 0.9, 0.1, 0.15, 0.2, -0.1]
        lo = [0.05, 0.5, -1.0, 0.01, 0.0, 0.0, -0.5, -0.3, -1.0, -1.0]
        hi = [0.6, 1.0, 1.0, 1.5, 3.0, 3.0, 0.5, 0.5, 1.0, 1.0]
    return T, K, market(model, truth, T, K, seed=11), lo, hi


@pytest.mark.parametrize("model", [sg.HAGAN, sg.OBLOJ, sg.EXPANDED])
def test_fp64_static_trajectory_is_the_oracle_trajectory(model):
    mkt = market()
    g, o = run_both(model, T15, K15, mkt, LO4, HI4, n_chains=64, n_levels=20, chain_len=30, seed=5)
    assert g.status == 0
    assert g.n_evals == o["n_evals"] and g.n_accepts == o["n_accepts"]
    np.testing.assert_allclose(g.params, o["params"], rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(g.restart_params, o["restart_params"], rtol=1e-10, atol=1e-14)
    assert g.misfit == pytest.approx(o["misfit"], rel=1e-10)
    assert g.misfit_fp64 == pytest.approx(o["misfit"], rel=1e-10)


@pytest.mark.parametrize("model", [sg.DYN_I, sg.DYN_II])
def test_fp64_dynamic_trajectory_is_the_oracle_trajectory(model):
    T, K, mkt, lo, hi = dyn_surface(model)
    g, o = run_both(model, T, K, mkt, lo, hi, n_chains=16, n_levels=6, chain_len=12, seed=9)
    assert g.status == 0
    assert g.n_evals == o["n_evals"] and g.n_accepts == o["n_accepts"]
    np.testing.assert_allclose(g.params, o["params"], rtol=1e-9, atol=1e-13)
    assert g.misfit == pytest.approx(o["misfit"], rel=1e-9)


def test_fp32_two_parameter_fit_within_one_percent_of_oracle():
    mkt = market()
    lo = [0.2, 0.7, -1 + 1e-6, 1e-6]
    hi = [0.2, 0.7, 1 - 1e-6, 3.0]
    g, o = run_both(sg.HAGAN, T15, K15, mkt, lo, hi, prec=sg.FP32, n_chains=64, seed=3)
    assert abs(g.misfit_fp64 - o["misfit"]) <= 0.01 * o["misfit"]
    np.testing.assert_allclose(g.params[2:], o["params"][2:], atol=2e-3)


def test_fp32_recovers_the_synthetic_smile():
    # beta fixed (the paper's usual practice, Sec. 3); noise 1e-4 in vol
    mkt = market()
    lo = [1e-6, 0.7, -1 + 1e-6, 1e-6]
    hi = [2.0, 0.7, 1 - 1e-6, 3.0]
    pb = sg.CalibrationProblem(model=sg.HAGAN, T=T15, K=K15, market=mkt, lo=lo, hi=hi, prec=sg.FP32,
                               n_chains=256, seed=1)
    g = sg.calibrate(pb)
    fit = O.implied_vol(O.HAGAN, g.params, 1.0, T15, K15)
    true = O.implied_vol(O.HAGAN, TRUTH, 1.0, T15, K15)
    assert np.max(np.abs(fit - true)) <= 3e-4
    assert abs(g.params[2] - TRUTH[2]) <= 0.05 and abs(g.params[3] - TRUTH[3]) / TRUTH[3] <= 0.05


def test_fp32_full_smile_reports_error_against_oracle():
    mkt = market()
    g, o = run_both(sg.HAGAN, T15, K15, mkt, LO4, HI4, prec=sg.FP32, n_chains=64, seed=7)
    # the FP32 in-loop misfit and its FP64 re-score agree to FP32 rounding
    assert abs(g.misfit - g.misfit_fp64) <= 1e-3 * g.misfit_fp64 + 1e-9
    # both land in the same basin: the model fit is within a few noise levels
    for params in (g.params, o["params"]):
        fit = O.implied_vol(O.HAGAN, params, 1.0, T15, K15)
        assert np.sqrt(np.mean((fit - mkt) ** 2)) <= 2e-3


@pytest.mark.parametrize("prec", [sg.FP32, sg.FP64])
def test_result_is_the_same_alone_and_in_a_batch(prec):
    mkt = market()
    T, K, mk2, lo2, hi2 = dyn_surface(O.DYN_I)
    a = sg.CalibrationProblem(model=sg.HAGAN, T=T15, K=K15, market=mkt, lo=LO4, hi=HI4, prec=prec,
                              n_chains=300, n_levels=8, chain_len=20, seed=21)
    b = sg.CalibrationProblem(model=sg.DYN_I, T=T, K=K, market=mk2, lo=lo2, hi=hi2, prec=prec,
                              n_chains=40, n_levels=5, chain_len=10, seed=4)
    c = sg.CalibrationProblem(model=sg.HAGAN, T=T15[:7], K=K15[:7], market=mkt[:7], lo=LO4, hi=HI4,
                              prec=prec, n_chains=1000, n_levels=3, chain_len=5, seed=99)
    alone = sg.calibrate(a)
    batch = sg.calibrate_batch([c, a, b])
    assert np.array_equal(alone.params, batch[1].params)
    assert alone.misfit == batch[1].misfit and alone.n_evals == batch[1].n_evals
    assert alone.n_accepts == batch[1].n_accepts


def test_graph_replay_equals_direct_launches_and_repeats():
    mkt = market()
    pbs = [sg.CalibrationProblem(model=sg.HAGAN, T=T15, K=K15, market=mkt, lo=LO4, hi=HI4,
                                 n_chains=128, n_levels=10, chain_len=20, seed=s) for s in range(3)]
    direct = sg.calibrate_batch(pbs)
    plan = sg.Plan(pbs, use_graph=True)
    plan.run()
    r1 = plan.results()
    plan.run()
    r2 = plan.results()
    n_launch, ms = plan.stats()
    plan.close()
    for x, y, z in zip(direct, r1, r2):
        assert np.array_equal(x.params, y.params) and np.array_equal(y.params, z.params)
        assert x.misfit == y.misfit == z.misfit and x.n_evals == y.n_evals == z.n_evals
    # a level of this plan has fewer units than the GPU has resident blocks,
    # so it runs level by level: init, 10 levels, finalize
    assert n_launch == 1 + 10 + 1 and ms > 0


def test_ready_queue_equals_level_by_level_launches(monkeypatch):
    # the persistent ready-queue launch and one launch per level run the same
    # units; results are bitwise identical, also for a batch whose problems
    # have different level counts, chain counts and models
    mkt = market()
    T, K, mk2, lo2, hi2 = dyn_surface(O.DYN_I)
    pbs = [sg.CalibrationProblem(model=sg.HAGAN, T=T15, K=K15, market=mkt, lo=LO4, hi=HI4, prec=sg.FP32,
                                 n_chains=6000, n_levels=12, chain_len=20, seed=31),
           sg.CalibrationProblem(model=sg.HAGAN, T=T15[:9], K=K15[:9], market=mkt[:9], lo=LO4, hi=HI4,
                                 prec=sg.FP32, n_chains=700, n_levels=5, chain_len=20, seed=32),
           sg.CalibrationProblem(model=sg.DYN_I, T=T, K=K, market=mk2, lo=lo2, hi=hi2, prec=sg.FP64,
                                 n_chains=90, n_levels=7, chain_len=10, seed=33),
           sg.CalibrationProblem(model=sg.HAGAN, T=T15, K=K15, market=mkt, lo=LO4, hi=HI4, prec=sg.FP32,
                                 n_chains=64, n_levels=0, chain_len=20, seed=34)]
    # 21 and 20 strikes, enough chains for one lane per chain: the step
    # loops with a first chunk of ten pairs, odd and even quote counts
    K21 = 0.5 + 0.05 * np.arange(21)
    m21 = market(T=np.ones(21), K=K21, seed=5)
    pbs += [sg.CalibrationProblem(model=sg.HAGAN, T=np.ones(n), K=K21[:n], market=m21[:n], lo=LO4, hi=HI4,
                                  prec=sg.FP32, n_chains=20000, n_levels=6, chain_len=20, seed=35 + n)
            for n in (21, 20)]
    # and several maturities (22 and 23 quotes): the same loops without the
    # one-maturity numerator
    for Tm in (np.repeat([0.5, 2.0], 11), np.concatenate([np.repeat([0.5, 2.0], 8), np.full(7, 3.0)])):
        Km = np.tile(np.linspace(0.6, 1.4, 11), 3)[:len(Tm)]
        pbs.append(sg.CalibrationProblem(model=sg.HAGAN, T=Tm, K=Km, market=market(T=Tm, K=Km, seed=6), lo=LO4,
                                         hi=HI4, prec=sg.FP32, n_chains=20000, n_levels=6, chain_len=20,
                                         seed=60 + len(Tm)))
    plan = sg.Plan(pbs, use_graph=True)
    plan.run()
    queued = plan.results()
    n_launch, _ = plan.stats()
    plan.close()
    # FP32 Hagan group (three problems, more units per level than resident
    # blocks): init, queue reset, one persistent launch, finalize; the FP64
    # Case I group (one problem, two of whose levels fit in the persistent
    # grid): the same four launches
    assert n_launch == 2 + 2 + 2 + 2
    monkeypatch.setenv("SABR_PLAN_QUEUE", "0")
    plan = sg.Plan(pbs, use_graph=True)
    plan.run()
    levelwise = plan.results()
    n_launch, _ = plan.stats()
    plan.close()
    assert n_launch == 2 + (12 + 7) + 2
    for x, y in zip(queued, levelwise):
        assert x.status == y.status == 0
        assert np.array_equal(x.params, y.params) and np.array_equal(x.restart_params, y.restart_params)
        assert x.misfit == y.misfit and x.misfit_fp64 == y.misfit_fp64
        assert x.n_evals == y.n_evals and x.n_accepts == y.n_accepts


def test_edge_cases():
    mkt = market()
    # no levels: the start point comes back
    g = sg.calibrate(sg.CalibrationProblem(model=sg.HAGAN, T=T15, K=K15, market=mkt, lo=LO4, hi=HI4,
                                           n_levels=0, x0=TRUTH))
    np.testing.assert_allclose(g.params, TRUTH, rtol=1e-7)
    assert g.n_evals == 0
    # one chain, one quote, a chain count that leaves a ragged last block
    for nc in (1, 257):
        g, o = run_both(sg.HAGAN, T15[:1], K15[:1], mkt[:1], LO4, HI4, n_chains=nc, n_levels=3, chain_len=4,
                        seed=2)
        assert g.n_evals == o["n_evals"]
        np.testing.assert_allclose(g.params, o["params"], rtol=1e-10)
    # fixed coordinates never move
    lo = [0.2, 0.7, -0.9, 0.1]
    hi = [0.2, 0.7, 0.5, 1.5]
    g = sg.calibrate(sg.CalibrationProblem(model=sg.HAGAN, T=T15, K=K15, market=mkt, lo=lo, hi=hi,
                                           n_levels=5, chain_len=10, prec=sg.FP32))
    assert g.params[0] == np.float32(0.2) and g.params[1] == np.float32(0.7)
    # invalid input is refused before any launch
    with pytest.raises(sg.SabrError):
        sg.calibrate(sg.CalibrationProblem(model=sg.HAGAN, T=T15, K=K15, market=-mkt, lo=LO4, hi=HI4))
    with pytest.raises(sg.SabrError):
        sg.calibrate(sg.CalibrationProblem(model=sg.HAGAN, T=T15, K=K15, market=mkt, lo=HI4, hi=LO4))
    with pytest.raises(sg.SabrError):
        sg.calibrate(sg.CalibrationProblem(model=sg.HAGAN, T=T15, K=K15, market=mkt, lo=LO4, hi=HI4,
                                           n_chains=0))


def test_full_size_static_surface_in_the_benchmark_launch_configuration():
    # 10 smiles x 21 strikes, 4096 chains each, 200 levels x 100 proposals,
    # FP32, one device-resident plan replayed as a CUDA graph (as timed).
    # Per smile the oracle re-evaluates the returned point: its FP64 misfit
    # must equal the library's FP64 re-score and the in-loop FP32 misfit must
    # agree to FP32 rounding.  On these nearly degenerate smiles the SA's end
    # point depends on the trajectory: the oracle's own FP64 results on one
    # smile differ by up to 78% between seeds, so an FP32 run (a different
    # trajectory) is held to twice the oracle's misfit on three sampled
    # smiles; the exact comparison at this size is the FP64 one below.
    from paper_2407_20713_gb300 import workloads
    smiles = workloads.static_surface()
    mkts = [O.implied_vol(O.HAGAN, sm.truth, 1.0, sm.T, sm.K) + sm.noise for sm in smiles]
    pbs = [sg.CalibrationProblem(model=sg.HAGAN, T=sm.T, K=sm.K, market=m, lo=sm.lo, hi=sm.hi, prec=sg.FP32,
                                 n_chains=sm.n_chains, n_levels=200, chain_len=100, factor=0.95, seed=7 + i)
           for i, (sm, m) in enumerate(zip(smiles, mkts))]
    plan = sg.Plan(pbs, use_graph=True)
    plan.run()
    res = plan.results()
    plan.close()
    for sm, m, r in zip(smiles, mkts, res):
        assert r.status == 0
        assert r.n_evals > 0.9 * sm.n_chains * 200 * 100
        o_fit = O.misfit(O.implied_vol(O.HAGAN, r.params, 1.0, sm.T, sm.K), m)
        assert r.misfit_fp64 == pytest.approx(o_fit, rel=1e-7)
        assert abs(r.misfit - r.misfit_fp64) <= 2e-3 * r.misfit_fp64
    for i in (0, 4, 9):
        sm, m, r = smiles[i], mkts[i], res[i]
        o = O.sa_calibrate(O.HAGAN, 1.0, sm.T, sm.K, m, sm.lo, sm.hi, n_chains=sm.n_chains, factor=0.95,
                           n_levels=200, chain_len=100, seed=7 + i, n_threads=os.cpu_count() or 8)
        assert r.misfit_fp64 <= 2.0 * o["misfit"], (i, r.misfit_fp64, o["misfit"])


def test_full_size_fp32_fixed_beta_surface_within_one_percent_of_the_oracle():
    # The benchmark's launch configuration (10 smiles x 21 strikes, 4096
    # chains each, 200 levels x 100 proposals, FP32, one plan replayed as a
    # CUDA graph) on smiles whose SA reaches its minimum: beta is fixed at
    # each smile's true value (lo = hi, the paper's usual practice, Sec. 3),
    # so alpha, rho, nu are well determined.  Per smile the FP32 result's
    # FP64 misfit must lie within 1% of the oracle's (Sec. 3 eq.
    # error_calibrate_relativo; the oracle runs the same seeds in FP64), and
    # the recovered smile must lie within 3 noise levels of the true smile.
    from paper_2407_20713_gb300 import workloads
    smiles = workloads.static_surface()
    boxes = []
    for sm in smiles:
        lo, hi = list(sm.lo), list(sm.hi)
        lo[1] = hi[1] = float(sm.truth[1])
        boxes.append((lo, hi))
    mkts = [O.implied_vol(O.HAGAN, sm.truth, 1.0, sm.T, sm.K) + sm.noise for sm in smiles]
    pbs = [sg.CalibrationProblem(model=sg.HAGAN, T=sm.T, K=sm.K, market=m, lo=lo, hi=hi, prec=sg.FP32,
                                 n_chains=sm.n_chains, n_levels=200, chain_len=100, factor=0.95, seed=7 + i)
           for i, (sm, m, (lo, hi)) in enumerate(zip(smiles, mkts, boxes))]
    plan = sg.Plan(pbs, use_graph=True)
    plan.run()
    res = plan.results()
    plan.close()
    for i, (sm, m, (lo, hi), r) in enumerate(zip(smiles, mkts, boxes, res)):
        assert r.status == 0
        assert r.params[1] == np.float32(sm.truth[1])
        o = O.sa_calibrate(O.HAGAN, 1.0, sm.T, sm.K, m, lo, hi, n_chains=sm.n_chains, factor=0.95,
                           n_levels=200, chain_len=100, seed=7 + i, n_threads=os.cpu_count() or 8)
        o_fit = O.misfit(O.implied_vol(O.HAGAN, r.params, 1.0, sm.T, sm.K), m)
        assert r.misfit_fp64 == pytest.approx(o_fit, rel=1e-7)
        assert abs(r.misfit_fp64 - o["misfit"]) <= 0.01 * o["misfit"], (i, r.misfit_fp64, o["misfit"])
        fit = O.implied_vol(O.HAGAN, r.params, 1.0, sm.T, sm.K)
        true = O.implied_vol(O.HAGAN, sm.truth, 1.0, sm.T, sm.K)
        assert np.max(np.abs(fit - true)) <= 3e-4, (i, np.max(np.abs(fit - true)))


def test_full_size_fp64_smiles_follow_the_oracle_trajectory():
    # the FP64 form at the headline's size (4096 chains, 200 x 100) on two
    # sampled smiles of the surface: the same Philox streams give the
    # oracle's trajectory through all ~8e7 evaluations
    from paper_2407_20713_gb300 import workloads
    smiles = workloads.static_surface()
    for i in (0, 4):
        sm = smiles[i]
        m = O.implied_vol(O.HAGAN, sm.truth, 1.0, sm.T, sm.K) + sm.noise
        pb = sg.CalibrationProblem(model=sg.HAGAN, T=sm.T, K=sm.K, market=m, lo=sm.lo, hi=sm.hi, prec=sg.FP64,
                                   n_chains=sm.n_chains, n_levels=200, chain_len=100, factor=0.95, seed=7 + i)
        g = sg.calibrate(pb)
        o = O.sa_calibrate(O.HAGAN, 1.0, sm.T, sm.K, m, sm.lo, sm.hi, n_chains=sm.n_chains, factor=0.95,
                           n_levels=200, chain_len=100, seed=7 + i, n_threads=os.cpu_count() or 8)
        assert g.n_evals == o["n_evals"] and g.n_accepts == o["n_accepts"]
        np.testing.assert_allclose(g.params, o["params"], rtol=1e-9, atol=1e-12)
        assert g.misfit_fp64 == pytest.approx(o["misfit"], rel=1e-9)


def test_full_size_dynamic_surface_sampled_against_oracle():
    # cfg 3 shape: 12 maturities x 21 strikes, 8192 chains, Case I and II,
    # FP32 (20 of the 200 levels): the oracle re-evaluates the returned point
    from paper_2407_20713_gb300 import workloads
    for case, model in ((1, sg.DYN_I), (2, sg.DYN_II)):
        w = workloads.dynamic_surface(case=case, feasible=lambda x: O.feasible(O.DYN_II, x, 10.0))
        m = O.implied_vol(model, w.truth, 1.0, w.T, w.K) + w.noise
        pb = sg.CalibrationProblem(model=model, T=w.T, K=w.K, market=m, lo=w.lo, hi=w.hi, prec=sg.FP32,
                                   n_chains=w.n_chains, n_levels=20, chain_len=100, seed=3)
        r = sg.calibrate(pb)
        assert r.status == 0
        o_fit = O.misfit(O.implied_vol(model, r.params, 1.0, w.T, w.K), m)
        assert r.misfit_fp64 == pytest.approx(o_fit, rel=1e-7)
        assert abs(r.misfit - r.misfit_fp64) <= 2e-3 * r.misfit_fp64
        # the returned point is the best ever evaluated: no worse than x0
        x0 = 0.5 * (np.asarray(w.lo) + np.asarray(w.hi))
        o_x0 = O.misfit(O.implied_vol(model, x0, 1.0, w.T, w.K), m)
        assert r.misfit_fp64 < o_x0


@pytest.mark.parametrize("prec", [sg.FP32, sg.FP64])
def test_maximum_quote_and_maturity_counts(prec):
    # 64 maturities x 64 strikes = 4096 quotes, the largest problem the
    # library accepts, in both precisions (Case I: every maturity has its
    # own term structure); FP64 follows the oracle's trajectory
    mats = np.linspace(0.1, 10.0, 64)
    T = np.repeat(mats, 64)
    K = np.tile(np.linspace(0.6, 1.5, 64), 64)
    truth = [0.25, 0.8, -0.5, 0.7, 0.6, 0.9]
    lo = [0.05, 0.5, -1.0, 0.01, 0.0, 0.0]
    hi = [0.6, 1.0, 1.0, 1.5, 3.0, 3.0]
    m = market(O.DYN_I, truth, T, K, seed=5)
    g, o = run_both(sg.DYN_I, T, K, m, lo, hi, prec=prec, n_chains=3, n_levels=2, chain_len=3, seed=8)
    assert g.status == 0
    if prec == sg.FP64:
        assert g.n_evals == o["n_evals"] and g.n_accepts == o["n_accepts"]
        np.testing.assert_allclose(g.params, o["params"], rtol=1e-10)
    o_fit = O.misfit(O.implied_vol(O.DYN_I, g.params, 1.0, T, K), m)
    assert g.misfit_fp64 == pytest.approx(o_fit, rel=1e-7)
    # the in-loop cost of the returned point (every quote reading its own
    # maturity's polynomial, 64 of them) agrees with the FP64 re-score
    assert abs(g.misfit - g.misfit_fp64) <= 2e-3 * g.misfit_fp64
    # one quote more is refused
    with pytest.raises(sg.SabrError):
        sg.calibrate(sg.CalibrationProblem(model=sg.DYN_I, T=np.append(T, 1.0), K=np.append(K, 1.0),
                                           market=np.append(m, 0.2), lo=lo, hi=hi, prec=prec, n_chains=2,
                                           n_levels=1, chain_len=1))


def test_fp32_and_fp64_outcomes_have_the_same_distribution_over_seeds():
    # the end point of the SA on these smiles depends on the trajectory (the
    # spread over seeds is 2-20x within one precision), so FP32 is compared
    # with FP64 in distribution: 12 seeds each at the headline's size
    from paper_2407_20713_gb300 import workloads
    smiles = workloads.static_surface()
    for i in (0, 9):
        sm = smiles[i]
        m = O.implied_vol(O.HAGAN, sm.truth, 1.0, sm.T, sm.K) + sm.noise
        out = {}
        for prec in (sg.FP32, sg.FP64):
            pbs = [sg.CalibrationProblem(model=sg.HAGAN, T=sm.T, K=sm.K, market=m, lo=sm.lo, hi=sm.hi, prec=prec,
                                         n_chains=sm.n_chains, n_levels=200, chain_len=100, factor=0.95,
                                         seed=1000 + s) for s in range(12)]
            out[prec] = np.array([r.misfit_fp64 for r in sg.calibrate_batch(pbs)])
        med32, med64 = np.median(out[sg.FP32]), np.median(out[sg.FP64])
        assert 0.7 <= med32 / med64 <= 1.43, (i, med32, med64)
        assert out[sg.FP32].min() <= 1.1 * out[sg.FP64].min(), (i, out[sg.FP32].min(), out[sg.FP64].min())


CASE2_TRUTH = [0.25, 0.8, -0.4, 0.6, 0.8, 0.9, 0.1, 0.15, 0.2, -0.1]
CASE2_LO = [0.05, 0.5, -1.0, 0.01, 0.0, 0.0, -0.5, -0.5, -1.0, -1.0]


@pytest.mark.parametrize("model,truth,lo,hi,mats", [
    (sg.HAGAN, TRUTH, LO4, HI4, [0.1, 1.0, 5.0]),
    (sg.OBLOJ, TRUTH, LO4, HI4, [0.1, 1.0, 5.0]),
    (sg.EXPANDED, TRUTH, LO4, HI4, [0.1, 1.0, 5.0]),
    (sg.DYN_I, [0.25, 0.8, -0.5, 0.7, 0.6, 0.9], [0.05, 0.5, -1.0, 0.01, 0.0, 0.0], [0.6, 1.0, 1.0, 1.5, 5.0, 5.0],
     [0.1, 0.25, 0.5, 1.0, 2.0, 5.0, 10.0]),
    # Case II: the composite term-structure rule of the FP32 form, with the
    # cfg-3 box (rates up to 5), a box up to the paper's b = 150 (Sec. 6.2),
    # one long maturity, and 30 years
    (sg.DYN_II, CASE2_TRUTH, CASE2_LO,
     [0.6, 1.0, 1.0, 1.5, 5.0, 5.0, 0.5, 0.5, 1.0, 1.0], [0.1, 0.25, 0.5, 0.75, 1, 1.5, 2, 3, 4, 5, 7, 10]),
    (sg.DYN_II, [0.25, 0.8, -0.4, 0.6, 40.0, 120.0, 0.1, 0.15, 0.2, 0.3], CASE2_LO,
     [0.6, 1.0, 1.0, 1.5, 150.0, 150.0, 0.5, 0.5, 1.0, 1.0], [0.05, 0.5, 1.0, 5.0]),
    (sg.DYN_II, CASE2_TRUTH, CASE2_LO, [0.6, 1.0, 1.0, 1.5, 5.0, 5.0, 0.5, 0.5, 1.0, 1.0], [10.0]),
    (sg.DYN_II, [0.25, 0.8, -0.4, 0.6, 0.05, 0.1, 0.1, 0.15, 0.02, -0.01], CASE2_LO,
     [0.6, 1.0, 1.0, 1.5, 5.0, 5.0, 0.5, 0.5, 1.0, 1.0], [0.5, 2.0, 10.0, 30.0]),
])
def test_fp32_in_loop_cost_matches_the_oracle(model, truth, lo, hi, mats):
    # With no levels the returned misfit is the FP32 in-loop cost of x0
    # (init kernel, the same group_cost as every proposal).  On a noise-free
    # surface at the true point it is the sum of the squared FP32 relative
    # vol errors (eq. error_calibrate_relativo with market = oracle vols);
    # at a perturbed point it must equal the oracle's misfit.
    K1 = np.linspace(0.5, 1.6, 21)
    T = np.repeat(np.asarray(mats, dtype=float), K1.size)
    K = np.tile(K1, len(mats))
    ref = O.implied_vol(model, truth, 1.0, T, K)
    ok = ref > 0.02
    T, K, ref = T[ok], K[ok], ref[ok]
    base = dict(model=model, T=T, K=K, market=ref, lo=lo, hi=hi, prec=sg.FP32, n_chains=8, n_levels=0)
    g = sg.calibrate(sg.CalibrationProblem(x0=truth, **base))
    assert g.status == 0
    rms = np.sqrt(g.misfit / T.size)
    print("in-loop FP32 rms relative vol error", model, mats, rms)
    assert rms <= 3e-6, (model, rms)
    x1 = np.array(truth, dtype=float)
    x1[0] *= 1.03
    x1[2] = x1[2] + 0.05
    g1 = sg.calibrate(sg.CalibrationProblem(x0=x1, **base))
    # the FP32 form holds its points in FP32: the oracle evaluates the point
    # as returned (x1 rounded to FP32)
    o1 = O.misfit(O.implied_vol(model, g1.params, 1.0, T, K), ref)
    assert np.allclose(g1.params, x1[:len(g1.params)], rtol=1e-7)
    assert g1.misfit == pytest.approx(o1, rel=2e-4), (model, g1.misfit, o1)
    assert g1.misfit_fp64 == pytest.approx(o1, rel=1e-9)


@pytest.mark.parametrize("prec", [sg.FP32, sg.FP64])
def test_speculative_hagan_loop_equals_the_one_step_loop(prec, monkeypatch):
    # Hagan chains with several lanes evaluate step st and, as if each were
    # accepted, the next steps together; the results (best point, restart point,
    # misfits, counters) must be those of the one-step loop bit for bit,
    # for small problems whose lanes share the quotes (the large batch, one
    # lane per chain, runs the one-step loop either way)
    mkt = market()
    T, K = np.repeat([0.5, 2.0], 15), np.tile(K15, 2)
    m2 = market(T=T, K=K, seed=4)
    pbs = [sg.CalibrationProblem(model=sg.HAGAN, T=T, K=K, market=m2, lo=LO4, hi=HI4, prec=prec,
                                 n_chains=4000, n_levels=6, chain_len=31, seed=41 + i) for i in range(3)]
    small = sg.CalibrationProblem(model=sg.HAGAN, T=T15, K=K15, market=mkt, lo=LO4, hi=HI4, prec=prec,
                                  n_chains=48, n_levels=8, chain_len=40, seed=44)
    # chain lengths shorter than, and not a multiple of, the speculation depth
    short = [sg.CalibrationProblem(model=sg.HAGAN, T=T15[:8], K=K15[:8], market=mkt[:8], lo=LO4, hi=HI4,
                                   prec=prec, n_chains=20, n_levels=5, chain_len=cl, seed=45 + cl)
             for cl in (1, 2, 3, 5, 7)]
    spec = sg.calibrate_batch(pbs) + [sg.calibrate(small)] + [sg.calibrate(q) for q in short]
    monkeypatch.setenv("SABR_SPECULATE", "0")
    plain = sg.calibrate_batch(pbs) + [sg.calibrate(small)] + [sg.calibrate(q) for q in short]
    for a, b in zip(spec, plain):
        assert a.status == b.status == 0
        assert np.array_equal(a.params, b.params) and np.array_equal(a.restart_params, b.restart_params)
        assert a.misfit == b.misfit and a.misfit_fp64 == b.misfit_fp64
        assert a.n_evals == b.n_evals and a.n_accepts == b.n_accepts
