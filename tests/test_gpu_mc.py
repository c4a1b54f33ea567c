"""GPU parity of sabr_mc_price (Sec. 4) with the FP64 oracle on identical
Philox streams: 1e-5 absolute in FP32 (forward 1), 1e-10 in FP64; and, at
2^24 paths where the oracle would take minutes, the properties that hold at
any size (Black limit, the absorbed-CEV closed form with the log-Euler bias
study, martingale, put-call identity)."""
import numpy as np
import pytest

import oracle as O
import paper_2407_20713_gb300 as sg
from helpers import Golden, black_call, cev_call

pytestmark = pytest.mark.gpu

TOL = {sg.FP32: 1e-5, sg.FP64: 1e-10}


def quotes():
    T = np.repeat([0.25, 0.5, 1.0, 1.37], 4)
    K = np.tile([0.8, 0.95, 1.05, 1.3], 4)
    ic = np.tile([1, 1, 0, 1], 4).astype(np.int8)
    return T, K, ic


PARAMS = {
    sg.HAGAN: [0.3, 0.6, -0.4, 0.7],
    sg.DYN_I: [0.3, 0.7, -0.6, 0.9, 0.5, 1.2],
    sg.DYN_II: [0.3, 0.8, -0.5, 0.7, 1.1, 0.6, 0.1, 0.2, 0.25, -0.2],
}


@pytest.mark.parametrize("prec", [sg.FP32, sg.FP64])
@pytest.mark.parametrize("model", [sg.HAGAN, sg.DYN_I, sg.DYN_II])
def test_mc_matches_oracle_on_the_same_streams(model, prec):
    T, K, ic = quotes()
    disc = np.linspace(0.99, 0.9, T.size)
    n_paths = 3 * 4096 + 77  # ragged against blocks and warps
    p = PARAMS[model]
    ref, rse = O.mc_price(model, p, 1.0, T, K, is_call=ic, disc=disc, n_paths=n_paths, steps_per_year=250,
                          seed=12345, n_threads=8)
    got, gse = sg.mc_price(model, p, 1.0, T, K, is_call=ic, discount=disc, n_paths=n_paths, steps_per_year=250,
                           seed=12345, prec=prec)
    got, gse = got.cpu().numpy(), gse.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= TOL[prec], np.abs(got - ref)
    assert np.max(np.abs(gse - rse)) <= TOL[prec]


@pytest.mark.parametrize("prec", [sg.FP32, sg.FP64])
def test_mc_absorption_heavy_case_matches_oracle(prec):
    # beta = 0 with a large alpha: many paths hit zero and are absorbed
    T = np.array([0.5, 1.0, 2.0, 2.0])
    K = np.array([0.5, 1.0, 1.0, 0.2])
    ic = np.array([1, 1, 0, 0], dtype=np.int8)
    p = [0.9, 0.0, -0.2, 0.5]
    ref, _ = O.mc_price(O.HAGAN, p, 1.0, T, K, is_call=ic, n_paths=5000, steps_per_year=100, seed=8, n_threads=8)
    got, _ = sg.mc_price(sg.HAGAN, p, 1.0, T, K, is_call=ic, n_paths=5000, steps_per_year=100, seed=8, prec=prec)
    assert np.max(np.abs(got.cpu().numpy() - ref)) <= TOL[prec]


def test_mc_full_size_black_limit_and_identities():
    n = 1 << 24
    T = np.array([0.5, 0.5, 1.0, 1.0, 1.0])
    K = np.array([1.0, 1.2, 1e-12, 0.9, 0.9])
    ic = np.array([1, 1, 1, 1, 0], dtype=np.int8)
    # nu = 0, beta = 1: geometric Brownian motion, exact under log-Euler
    p = [0.25, 1.0, -0.3, 0.0]
    got, se = sg.mc_price(sg.HAGAN, p, 1.0, T, K, is_call=ic, n_paths=n, steps_per_year=250, seed=1)
    got, se = got.cpu().numpy(), se.cpu().numpy()
    ref = black_call(1.0, K[:2], T[:2], 0.25)
    assert np.all(np.abs(got[:2] - ref) <= 4 * se[:2])
    assert abs(got[2] - 1.0) <= 4 * se[2]                      # martingale
    assert abs((got[3] - got[4]) - (got[2] - 0.9)) <= 1e-6     # put-call, pathwise
    # full SABR dynamics: martingale and put-call identity still hold
    got, se = sg.mc_price(sg.HAGAN, [0.3, 0.5, -0.5, 0.8], 1.0, T, K, is_call=ic, n_paths=n,
                          steps_per_year=250, seed=2)
    got, se = got.cpu().numpy(), se.cpu().numpy()
    assert abs(got[2] - 1.0) <= 4 * se[2]
    assert abs((got[3] - got[4]) - (got[2] - 0.9)) <= 1e-6


@pytest.mark.parametrize("a,b", [(0.3, 0.5), (0.6, 0.3)])
def test_mc_log_euler_bias_against_cev(a, b):
    # nu = 0: the absorbed CEV closed form (helpers.cev_call) against the
    # FP32 kernel at 2^24 paths, on step grids from 25 to 1000 steps a year.
    # The table printed (pytest -s) is the scheme's bias study; the bar: at
    # 1000 steps a year every price lies within 4 standard errors plus a
    # quarter of the largest bias seen at 25 steps (first-order decay of the
    # bias), and the bias never grows as the step shrinks by 40x.
    n = 1 << 24
    T = np.array([0.5, 1.0, 1.0, 1.0, 2.0])
    K = np.array([1.0, 0.7, 1.0, 1.4, 1.0])
    ref = np.array([cev_call(1.0, k, t, a, b) for k, t in zip(K, T)])
    bias = {}
    for spy in (25, 100, 250, 1000):
        got, se = sg.mc_price(sg.HAGAN, [a, b, 0.0, 0.0], 1.0, T, K, n_paths=n, steps_per_year=spy, seed=77)
        got, se = got.cpu().numpy(), se.cpu().numpy()
        bias[spy] = (got - ref, se)
        print("alpha %.2f beta %.2f steps/yr %4d bias %s se %s" % (a, b, spy, np.array2string(got - ref, precision=6),
                                                                 np.array2string(se, precision=6)))
    d25, _ = bias[25]
    d1000, se1000 = bias[1000]
    assert np.all(np.abs(d1000) <= 4 * se1000 + 0.25 * np.max(np.abs(d25)))
    assert np.max(np.abs(d1000)) <= np.max(np.abs(d25)) + 4 * np.max(se1000)


@pytest.mark.parametrize("prec", [sg.FP32, sg.FP64])
def test_mc_reproduces_the_papers_dsabr2_eurusd_prices(prec):
    # the paper's DSabr_II EUR/USD prices (Sec. 6.2.2) at its calibrated
    # parameters, through the C-ABI at 2^20 paths (the paper's count)
    g = Golden("dsabr2_eurusd.txt")
    p, S0 = g.floats("params"), g.floats("spot")[0]
    for T in sorted(set(g.rows[:, 0])):
        rows = g.rows[g.rows[:, 0] == T]
        r, y, K, V = rows[0, 1], rows[0, 2], rows[:, 3], rows[:, 4]
        F = S0 * np.exp((r - y) * T)
        got, se = sg.mc_price(sg.DYN_II, p, F, np.full(K.size, T), K, discount=np.full(K.size, np.exp(-r * T)),
                              n_paths=1 << 20, steps_per_year=250, seed=9, prec=prec)
        got, se = got.cpu().numpy(), se.cpu().numpy()
        assert np.all(np.abs(got - V) <= 4 * se + 0.005 * V), (T, (got - V) / V)


@pytest.mark.parametrize("prec", [sg.FP32, sg.FP64])
@pytest.mark.parametrize("name,model", [("DYN_I", sg.DYN_I), ("DYN_II", sg.DYN_II)])
def test_mc_reproduces_the_papers_european_call_table(name, model, prec):
    # Sec. 4's European call prices (2^20 paths, 123 steps of 1/250) through
    # the C-ABI at the paper's path count, so the two Monte Carlo noises are
    # alike and their difference has sqrt(2) SE; the bound is 5 of those
    g = Golden("table1_european_call.txt")
    S0, K, T = g.floats("spot")[0], g.floats("strike")[0], g.floats("maturity")[0]
    r, y = g.floats("rates")
    n_steps = int(g.floats("steps")[0])
    V, *p = g.floats(name)
    got, se = sg.mc_price(model, p, S0 * np.exp((r - y) * T), np.array([n_steps / 250.0]), np.array([K]),
                          discount=np.array([np.exp(-r * T)]), n_paths=1 << 20, steps_per_year=250, seed=4,
                          prec=prec)
    got, se = float(got.cpu()[0]), float(se.cpu()[0])
    assert abs(got - V) <= 5 * np.sqrt(2.0) * se, (got, V, se)


def test_mc_is_deterministic_and_validates():
    T, K, ic = quotes()
    a, _ = sg.mc_price(sg.HAGAN, PARAMS[sg.HAGAN], 1.0, T, K, is_call=ic, n_paths=10000, seed=5)
    b, _ = sg.mc_price(sg.HAGAN, PARAMS[sg.HAGAN], 1.0, T, K, is_call=ic, n_paths=10000, seed=5)
    assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
    got, _ = sg.mc_price(sg.HAGAN, PARAMS[sg.HAGAN], 1.0, [1.0], [1.0], n_paths=2, seed=5)
    ref, _ = O.mc_price(O.HAGAN, PARAMS[sg.HAGAN], 1.0, [1.0], [1.0], n_paths=2, seed=5)
    assert abs(got.item() - ref[0]) <= 1e-5
    with pytest.raises(sg.SabrError):   # rho(t) leaves [-1, 1]
        sg.mc_price(sg.DYN_II, [0.3, 0.8, 0.9, 0.7, 0.0, 0.6, 0.3, 0.2, 0.0, 0.0], 1.0, [1.0], [1.0])
    with pytest.raises(sg.SabrError):
        sg.mc_price(sg.HAGAN, PARAMS[sg.HAGAN], 1.0, np.ones(513), np.ones(513))
    with pytest.raises(sg.SabrError):
        sg.mc_price(sg.HAGAN, PARAMS[sg.HAGAN], 1.0, [1.0], [1.0], n_paths=1)


def test_mc_at_the_size_limits():
    # 64 maturities x 8 options = 512 (the limit) over 32 years at 250 steps a
    # year: 8000 steps; FP32 fits one block's shared memory and matches the
    # oracle on the same streams, FP64 (32 B a step) is refused
    mats = np.linspace(0.5, 32.0, 64)
    T = np.repeat(mats, 8)
    K = np.tile([0.5, 0.8, 0.95, 1.0, 1.05, 1.2, 1.6, 2.5], 64)
    ic = np.tile([1, 1, 0, 1, 0, 1, 1, 1], 64).astype(np.int8)
    p = [0.2, 0.7, -0.3, 0.3]
    ref, _ = O.mc_price(sg.HAGAN, p, 1.0, T, K, is_call=ic, n_paths=777, steps_per_year=250, seed=21, n_threads=8)
    got, _ = sg.mc_price(sg.HAGAN, p, 1.0, T, K, is_call=ic, n_paths=777, steps_per_year=250, seed=21, prec=sg.FP32)
    err = np.abs(got.cpu().numpy() - ref)
    # the FP32 log-state takes one rounding (2^-24 relative) per step, so its
    # error grows like sqrt(steps): 1e-5 up to 2 years (500 steps), 5e-5 at
    # 32 years (8000 steps)
    assert np.max(err[T <= 2.0]) <= TOL[sg.FP32]
    assert np.max(err) <= 5e-5
    with pytest.raises(sg.SabrError):
        sg.mc_price(sg.HAGAN, p, 1.0, T, K, is_call=ic, n_paths=777, steps_per_year=250, seed=21, prec=sg.FP64)
    with pytest.raises(sg.SabrError):  # one option more
        sg.mc_price(sg.HAGAN, p, 1.0, np.append(T, 1.0), np.append(K, 1.0), n_paths=777, prec=sg.FP32)
