"""Serving: continuous batching of calibration requests (sabr_server_*).

Each result must be the same alone and in the mix (bit for bit, and the same
as sabr_calibrate), requests that arrive while others run must join them,
admission must respect the device-memory pool, and the host-side limits
(queue, timeouts, cancellation) must report their status codes."""
import time

import numpy as np
import pytest

import oracle as O
import paper_2407_20713_gb300 as sg
from paper_2407_20713_gb300 import workloads

pytestmark = pytest.mark.gpu


def formula_request(i, model=None, n_chains=256, n_levels=12, chain_len=20, prec=sg.FP32):
    rng = np.random.default_rng(1000 + i)
    n_mats = int(rng.integers(1, 5))
    n_strikes = int(rng.integers(5, 22))
    mats = np.sort(rng.choice([0.25, 0.5, 1.0, 2.0, 3.0, 5.0], n_mats, replace=False))
    T = np.repeat(mats, n_strikes)
    K = np.tile(np.linspace(0.7, 1.3, n_strikes), n_mats)
    model = model if model is not None else [sg.HAGAN, sg.HAGAN, sg.OBLOJ, sg.DYN_I, sg.DYN_II][i % 5]
    if model in (sg.HAGAN, sg.OBLOJ, sg.EXPANDED):
        truth, lo, hi = [0.25, 0.6, -0.3, 0.6], workloads.STATIC_LO, workloads.STATIC_HI
    elif model == sg.DYN_I:
        truth, lo, hi = [0.25, 0.8, -0.4, 0.6, 0.5, 0.8], workloads.DYN1_LO, workloads.DYN1_HI
    else:
        truth, lo, hi = [0.25, 0.8, -0.4, 0.6, 0.5, 0.8, 0.05, 0.1, 0.1, 0.05], workloads.DYN2_LO, workloads.DYN2_HI
    mkt = O.implied_vol(model, truth, 1.0, T, K) + rng.normal(0, 1e-4, T.size)
    return sg.CalibrationProblem(model=model, T=T, K=K, market=mkt, lo=lo, hi=hi, prec=prec, n_chains=n_chains,
                                 n_levels=n_levels, chain_len=chain_len, seed=77 + i)


def mc_request(i):
    T = np.array([0.5, 0.5, 1.0, 1.0])
    K = np.array([0.9, 1.1, 0.9, 1.1])
    mkt, _ = O.mc_price(O.HAGAN, [0.25, 0.6, -0.3, 0.5], 1.0, T, K, n_paths=4096, steps_per_year=50, seed=3)
    return sg.CalibrationProblem(model=sg.HAGAN, T=T, K=K, market=mkt, lo=[0.25, 0.6, -0.9, 0.1],
                                 hi=[0.25, 0.6, 0.5, 1.5], cost=sg.COST_MC_PRICE, n_chains=8, n_levels=3,
                                 chain_len=3, mc_paths=2048, mc_steps_per_year=50, mc_seed=5, seed=11 + i)


def same(a, b):
    return (np.array_equal(a.params, b.params) and a.misfit == b.misfit and a.n_evals == b.n_evals
            and a.n_accepts == b.n_accepts and a.misfit_fp64 == b.misfit_fp64)


@pytest.mark.parametrize("use_graph", [True, False])
def test_results_are_the_same_alone_and_in_the_mix(use_graph):
    probe = [formula_request(0), formula_request(3), mc_request(0)]
    ref = [sg.calibrate(p) for p in probe]
    # alone: one request at a time in a fresh server
    srv = sg.Server(device_bytes=256 << 20, use_graph=use_graph)
    alone = [srv.wait(srv.submit(p), timeout_ms=60000) for p in probe]
    srv.close()
    for a, r in zip(alone, ref):
        assert same(a, r)
    # in the mix: many other requests, arriving while the probes run
    srv = sg.Server(device_bytes=256 << 20, use_graph=use_graph)
    tickets, probe_t = [], []
    for i in range(40):
        if i in (5, 17, 29):
            probe_t.append(srv.submit(probe[len(probe_t)]))
        else:
            tickets.append(srv.submit(formula_request(100 + i) if i % 9 else mc_request(100 + i)))
        if i % 10 == 0:
            time.sleep(0.01)
    mixed = [srv.wait(t, timeout_ms=120000) for t in probe_t]
    for t in tickets:
        srv.wait(t, timeout_ms=120000)
    st = srv.stats()
    srv.close()
    for m, r in zip(mixed, ref):
        assert same(m, r)
    assert st["completed"] == 40 and st["steps"] > 0


def test_late_arrivals_join_running_requests():
    srv = sg.Server(device_bytes=256 << 20)
    # a request long enough to be resident for seconds
    long_t = srv.submit(formula_request(1, n_chains=16384, n_levels=4000, chain_len=200))
    time.sleep(0.1)
    short_t = srv.submit(formula_request(2, n_chains=64, n_levels=3, chain_len=5))
    short = srv.wait(short_t, timeout_ms=60000)
    # the short request finished while the long one was still resident
    assert short.status == 0
    assert srv.poll(long_t) is None
    assert srv.stats()["active"] >= 1
    srv.cancel(long_t)
    with pytest.raises(sg.SabrError) as e:
        srv.wait(long_t, timeout_ms=120000)
    assert e.value.status == sg.capi.ECANCELLED
    srv.close()


def test_admission_respects_the_device_pool():
    srv = sg.Server(device_bytes=4 << 20)   # room for only a few such requests at a time
    ts = [srv.submit(formula_request(4 + i, n_chains=4096)) for i in range(12)]
    peak = 0
    while True:
        st = srv.stats()
        peak = max(peak, st["pool_bytes_in_use"])
        if st["completed"] == 12:
            break
        time.sleep(0.002)
    for t in ts:
        assert srv.wait(t, timeout_ms=60000).status == 0
    srv.close()
    assert 0 < peak <= 4 << 20


@pytest.mark.parametrize("model", [sg.DYN_I, sg.DYN_II])
def test_dynamic_request_at_the_shared_memory_worst_case(model):
    # two maturities and few quotes give one lane per chain, and enough chains
    # keep it from widening: 256 chains of two maturity slices each per
    # block, with max_quotes leaving no slack in the quote staging
    T = np.repeat([0.5, 2.0], 21)
    K = np.tile(np.linspace(0.6, 1.4, 21), 2)
    if model == sg.DYN_I:
        truth, lo, hi = [0.25, 0.8, -0.4, 0.6, 0.5, 0.8], workloads.DYN1_LO, workloads.DYN1_HI
    else:
        truth, lo, hi = [0.25, 0.8, -0.4, 0.6, 0.5, 0.8, 0.05, 0.1, 0.1, 0.05], workloads.DYN2_LO, workloads.DYN2_HI
    mkt = O.implied_vol(model, truth, 1.0, T, K)
    pb = sg.CalibrationProblem(model=model, T=T, K=K, market=mkt, lo=lo, hi=hi, n_chains=152 * 256, n_levels=3,
                               chain_len=8, seed=5)
    srv = sg.Server(device_bytes=256 << 20, max_quotes=T.size)
    r = srv.wait(srv.submit(pb), timeout_ms=60000)
    srv.close()
    alone = sg.calibrate(pb)
    assert r.status == 0 and r.misfit_fp64 == alone.misfit_fp64 and np.array_equal(r.params, alone.params)


def test_host_side_limits_and_status_codes():
    srv = sg.Server(device_bytes=64 << 20, max_queue=2, max_active=1)
    t1 = srv.submit(formula_request(6, n_chains=16384, n_levels=4000, chain_len=200))
    time.sleep(0.05)
    t2 = srv.submit(formula_request(7))
    t3 = srv.submit(formula_request(8))
    with pytest.raises(sg.SabrError) as e:          # queue full
        srv.submit(formula_request(9))
    assert e.value.status == sg.capi.EBUSY
    srv.cancel(t3)                                   # cancel a queued request
    with pytest.raises(sg.SabrError) as e:
        srv.wait(t3, timeout_ms=1000)
    assert e.value.status == sg.capi.ECANCELLED
    with pytest.raises(sg.SabrError) as e:           # bounded wait runs out
        srv.wait(t1, timeout_ms=1)
    assert e.value.status == sg.capi.ETIMEOUT
    with pytest.raises(sg.SabrError) as e:
        srv.poll(987654321)
    assert e.value.status == sg.capi.ENOTFOUND
    srv.cancel(t1)                                   # cancel a resident request
    with pytest.raises(sg.SabrError) as e:
        srv.wait(t1, timeout_ms=60000)
    assert e.value.status == sg.capi.ECANCELLED
    assert srv.wait(t2, timeout_ms=60000).status == 0
    srv.close()
