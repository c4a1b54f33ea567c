"""GPU parity of the conditional-Bessel Monte Carlo step (sabr_mc_price_scheme
with SABR_MC_BESSEL, the low-bias scheme Sec. 4 names as the fallback for
log-Euler) against the oracle on identical Philox streams, its exactness for
the absorbed CEV law on the GPU, and its bias against log-Euler."""
import numpy as np
import pytest

import oracle as O
import paper_2407_20713_gb300 as sg
from helpers import cev_call

pytestmark = pytest.mark.gpu

TOL = {sg.FP32: 2e-5, sg.FP64: 1e-10}
T16 = np.repeat([0.25, 0.5, 1.0, 1.37], 4)
K16 = np.tile([0.8, 0.95, 1.05, 1.3], 4)
IC16 = np.tile([1, 1, 0, 1], 4).astype(np.int8)

CASES = {
    "hagan": (sg.HAGAN, [0.3, 0.6, -0.4, 0.7]),
    "dyn1": (sg.DYN_I, [0.3, 0.7, -0.6, 0.9, 0.5, 1.2]),
    "dyn2": (sg.DYN_II, [0.3, 0.8, -0.5, 0.7, 1.1, 0.6, 0.1, 0.2, 0.25, -0.2]),
    "normal": (sg.HAGAN, [0.25, 0.0, 0.3, 0.5]),             # beta = 0: Y = F
    "absorbing": (sg.HAGAN, [0.6, 0.3, -0.2, 0.4]),          # many paths reach 0
    "lognormal": (sg.HAGAN, [0.25, 1.0, -0.5, 0.6]),         # beta = 1 branch
    "unit_rho": (sg.DYN_I, [0.3, 0.5, 1.0, 0.5, 0.0, 0.3]),  # rho(t) = 1: the clock stops
}


def _both(model, p, T, K, ic, n_paths, spy, seed, prec, disc=None):
    ref, rse = O.mc_price(model, p, 1.0, T, K, is_call=ic, disc=disc, n_paths=n_paths, steps_per_year=spy, seed=seed,
                          n_threads=8, scheme=O.MC_BESSEL)
    got, gse = sg.mc_price(model, p, 1.0, T, K, is_call=ic, discount=disc, n_paths=n_paths, steps_per_year=spy,
                           seed=seed, prec=prec, scheme=sg.MC_BESSEL)
    return ref, rse, got.cpu().numpy(), gse.cpu().numpy()


@pytest.mark.parametrize("prec", [sg.FP32, sg.FP64])
@pytest.mark.parametrize("spy", [12, 250])
@pytest.mark.parametrize("case", sorted(CASES))
def test_bessel_matches_oracle_on_the_same_streams(case, spy, prec):
    model, p = CASES[case]
    n_paths = 3 * 4096 + 77  # ragged against blocks and warps
    disc = np.linspace(0.99, 0.9, T16.size)
    ref, rse, got, gse = _both(model, p, T16, K16, IC16, n_paths, spy, 4321, prec, disc)
    assert np.max(np.abs(got - ref)) <= TOL[prec], np.abs(got - ref)
    assert np.max(np.abs(gse - rse)) <= TOL[prec], np.abs(gse - rse)


@pytest.mark.parametrize("prec", [sg.FP32, sg.FP64])
def test_bessel_small_and_single_option_cases(prec):
    for n_paths in (2, 33):
        ref, rse, got, gse = _both(sg.HAGAN, [0.3, 0.5, -0.3, 0.5], np.array([0.7]), np.array([1.0]), None, n_paths,
                                   3, 9, prec)
        assert np.max(np.abs(got - ref)) <= TOL[prec] and np.max(np.abs(gse - rse)) <= TOL[prec]


def test_bessel_rejects_an_unknown_scheme():
    with pytest.raises(sg.SabrError):
        sg.mc_price(sg.HAGAN, [0.3, 0.5, -0.3, 0.5], 1.0, np.ones(1), np.ones(1), n_paths=64, scheme=7)


@pytest.mark.parametrize("alpha,beta,T", [(0.3, 0.5, 1.0), (0.6, 0.3, 2.0), (0.3, 0.0, 1.0)])
@pytest.mark.parametrize("spy", ["one step", 50])
def test_bessel_is_the_absorbed_cev_law_on_the_gpu(alpha, beta, T, spy):
    # nu = 0, rho = 0: exact at any step size, FP32, 2^22 paths
    K = np.array([0.7, 1.0, 1.4, 1e-6])
    ic = np.array([1, 1, 1, 0], np.int8)
    s = 0.99 / T if spy == "one step" else spy
    got, se = sg.mc_price(sg.HAGAN, [alpha, beta, 0.0, 0.0], 1.0, np.full(4, T), K, is_call=ic, n_paths=1 << 22,
                          steps_per_year=s, seed=17, scheme=sg.MC_BESSEL)
    got, se = got.cpu().numpy(), se.cpu().numpy()
    ref = np.array([cev_call(1.0, k, T, alpha, beta) for k in K[:3]])
    assert np.all(np.abs(got[:3] - ref) <= 4.5 * se[:3]), (got[:3] - ref) / se[:3]


def test_bessel_bias_against_log_euler():
    # SABR with vol of vol (no closed form): the Bessel scheme on grids of 1
    # to 64 steps a year against log-Euler at 2000 steps a year, 2^24 paths
    # each, independent streams.  The table printed (pytest -s) is the bias
    # study; the bar: from 4 steps a year every price lies within 4 combined
    # standard errors plus 1e-4 (log-Euler's own bias at 2000 steps a year
    # is below that) of the fine log-Euler price.
    n = 1 << 24
    T = np.array([0.5, 1.0, 1.0, 1.0, 2.0])
    K = np.array([1.0, 0.7, 1.0, 1.4, 1.0])
    for p in ([0.3, 0.5, -0.4, 0.6], [0.6, 0.3, 0.3, 0.8]):
        fine, fse = sg.mc_price(sg.HAGAN, p, 1.0, T, K, n_paths=n, steps_per_year=2000, seed=101)
        fine, fse = fine.cpu().numpy(), fse.cpu().numpy()
        for spy in (1, 4, 16, 64):
            got, se = sg.mc_price(sg.HAGAN, p, 1.0, T, K, n_paths=n, steps_per_year=spy, seed=102,
                                  scheme=sg.MC_BESSEL)
            got, se = got.cpu().numpy(), se.cpu().numpy()
            d = got - fine
            print("params %s bessel steps/yr %3d  minus log-Euler(2000) %s  se %s" % (
                p, spy, np.array2string(d, precision=6), np.array2string(np.hypot(se, fse), precision=6)))
            if spy >= 4:
                assert np.all(np.abs(d) <= 4 * np.hypot(se, fse) + 1e-4), d
        for spy in (4, 16, 64):
            le, lse = sg.mc_price(sg.HAGAN, p, 1.0, T, K, n_paths=n, steps_per_year=spy, seed=103)
            print("params %s log-Euler steps/yr %3d  minus log-Euler(2000) %s" % (
                p, spy, np.array2string(le.cpu().numpy() - fine, precision=6)))
