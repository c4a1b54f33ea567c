"""GPU parity of sabr_mc_cliquet (Sec. 6.3) with the FP64 oracle on identical
Philox streams (1e-5 absolute in FP32, 1e-10 in FP64, forward 1), and at the
full size of 2^22 paths the exact GBM law (nu = 0, beta = 1) within four
standard errors."""
import numpy as np
import pytest

import oracle as O
import paper_2407_20713_gb300 as sg
from helpers import exact_gbm_cliquet

pytestmark = pytest.mark.gpu

TOL = {sg.FP32: 1e-5, sg.FP64: 1e-10}

# Sec. 6.3 contract: one year, four resets, local limits -2% / +2%, global
# floor 0 and cap 0.2
CONTRACT = dict(T=1.0, n_resets=4, floor_local=-0.02, cap_local=0.02, floor_global=0.0, cap_global=0.2)

PARAMS = {
    sg.HAGAN: [0.3, 0.6, -0.4, 0.7],
    sg.DYN_I: [0.12, 0.8, -0.3, 0.6, 0.7, 1.1],
    sg.DYN_II: [0.12, 0.8, -0.3, 0.5, 1.1, 0.6, 0.1, 0.2, 0.25, -0.2],
}


def oracle_price(model, p, c, n_paths, spy, seed, disc=1.0, f=1.0):
    return O.mc_cliquet(model, p, f, c["T"], c["n_resets"], c["floor_local"], c["cap_local"], c["floor_global"],
                        c["cap_global"], disc=disc, n_paths=n_paths, steps_per_year=spy, seed=seed, n_threads=8)


def gpu_price(model, p, c, n_paths, spy, seed, prec, disc=1.0, f=1.0):
    pr, se = sg.mc_cliquet(model, p, f, c["T"], c["n_resets"], c["floor_local"], c["cap_local"], c["floor_global"],
                           c["cap_global"], discount=disc, n_paths=n_paths, steps_per_year=spy, seed=seed, prec=prec)
    return float(pr.item()), float(se.item())


@pytest.mark.parametrize("prec", [sg.FP32, sg.FP64])
@pytest.mark.parametrize("model", [sg.HAGAN, sg.DYN_I, sg.DYN_II])
def test_cliquet_matches_oracle_on_the_same_streams(model, prec):
    n_paths = 5 * 4096 + 37  # ragged against blocks and warps
    ref, rse = oracle_price(model, PARAMS[model], CONTRACT, n_paths, 250, 777, disc=0.97)
    got, gse = gpu_price(model, PARAMS[model], CONTRACT, n_paths, 250, 777, prec, disc=0.97)
    assert abs(got - ref) <= TOL[prec], (got, ref)
    assert abs(gse - rse) <= TOL[prec]


@pytest.mark.parametrize("prec", [sg.FP32, sg.FP64])
def test_cliquet_binding_limits_and_odd_grids(prec):
    # resets off the 1/spy grid, tight global limits, a forward != 1
    c = dict(T=0.83, n_resets=7, floor_local=-0.01, cap_local=0.015, floor_global=-0.005, cap_global=0.01)
    p = [0.4, 0.5, 0.3, 0.9]
    ref, _ = oracle_price(sg.HAGAN, p, c, 3000, 37, 5, f=1.7)
    got, _ = gpu_price(sg.HAGAN, p, c, 3000, 37, 5, prec, f=1.7)
    assert abs(got - ref) <= TOL[prec]


@pytest.mark.parametrize("prec", [sg.FP32, sg.FP64])
def test_cliquet_absorbed_paths_match_oracle(prec):
    # beta = 0 with a large alpha: paths hit zero between resets (R = -1)
    c = dict(T=2.0, n_resets=5, floor_local=-2.0, cap_local=0.5, floor_global=-1e300, cap_global=1e300)
    p = [0.9, 0.0, -0.2, 0.5]
    ref, _ = oracle_price(sg.HAGAN, p, c, 4000, 100, 8)
    got, _ = gpu_price(sg.HAGAN, p, c, 4000, 100, 8, prec)
    assert abs(got - ref) <= TOL[prec]


def test_cliquet_full_size_exact_gbm_law():
    a = 0.25
    ref = exact_gbm_cliquet(a, 1.0, 4, -0.02, 0.02, -0.01, 0.03)
    c = dict(T=1.0, n_resets=4, floor_local=-0.02, cap_local=0.02, floor_global=-0.01, cap_global=0.03)
    got, se = gpu_price(sg.HAGAN, [a, 1.0, 0.1, 0.0], c, 1 << 22, 250, 2024, sg.FP32)
    assert abs(got - ref) <= 4 * se, (got, ref, se)


def test_cliquet_rejects_bad_input():
    p = PARAMS[sg.HAGAN]
    bad = [dict(CONTRACT, n_resets=1), dict(CONTRACT, n_resets=65), dict(CONTRACT, floor_local=0.1),
           dict(CONTRACT, floor_global=0.3), dict(CONTRACT, T=0.0)]
    for c in bad:
        with pytest.raises(sg.SabrError):
            gpu_price(sg.HAGAN, p, c, 1000, 250, 1, sg.FP32)
    infeasible = [0.12, 0.8, -0.3, 0.5, 1.1, 0.6, 0.9, 0.2, 0.25, -0.2]  # rho(0) = 0.6 + ... > 1
    infeasible[2], infeasible[6] = 0.6, 0.6
    with pytest.raises(sg.SabrError):
        gpu_price(sg.DYN_II, infeasible, CONTRACT, 1000, 250, 1, sg.FP32)
