"""GPU parity of sabr_implied_vol (through the C-ABI) with the FP64 oracle,
element by element: 1e-12 relative in FP64 and 3e-5 relative in FP32."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2407_20713_gb300 as sg

pytestmark = pytest.mark.gpu

TOL = {sg.FP64: 1e-12, sg.FP32: 3e-5}


def _random_params(model, rng):
    if model in (sg.HAGAN, sg.OBLOJ, sg.EXPANDED):
        return [rng.uniform(0.05, 0.8), rng.uniform(0, 1), rng.uniform(-0.95, 0.95), rng.uniform(0.05, 2.5)]
    p = [rng.uniform(0.05, 0.8), rng.uniform(0, 1), rng.uniform(-0.95, 0.95), rng.uniform(0.05, 2.0),
         rng.uniform(0, 3), rng.uniform(0, 3)]
    if model == sg.DYN_II:
        while True:
            q = p + [rng.uniform(-0.2, 0.2), rng.uniform(0, 0.3), rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3)]
            if O.feasible(O.DYN_II, q, 10.0):
                return q
    return p


def _grid(rng, n):
    K = rng.uniform(0.5, 1.6, n)
    T = rng.choice([0.05, 0.1, 0.25, 0.5, 1.0, 2.0, 5.0, 10.0], n)
    K[:5] = [1.0, 1.0 + 1e-7, 1.0 - 1e-7, 1.0 + 1e-4, 0.999]   # at and next to the money
    return T, K


@pytest.mark.parametrize("prec", [sg.FP64, sg.FP32])
@pytest.mark.parametrize("model", [sg.HAGAN, sg.OBLOJ, sg.EXPANDED, sg.DYN_I, sg.DYN_II])
def test_implied_vol_matches_oracle(model, prec):
    rng = np.random.default_rng(100 + 10 * model + prec)
    n = 2 * 256 + 37  # several blocks and a ragged tail
    for trial in range(4):
        p = _random_params(model, rng)
        T, K = _grid(rng, n)
        got = sg.implied_vol(model, p, 1.0, T, K, prec=prec).cpu().numpy()
        ref = O.implied_vol(model, p, 1.0, T, K)
        rel = np.abs(got - ref) / np.abs(ref)
        assert rel.max() <= TOL[prec], (p, rel.argmax(), got[rel.argmax()], ref[rel.argmax()], rel.max())


@pytest.mark.parametrize("prec", [sg.FP64, sg.FP32])
def test_static_special_cases(prec):
    T = np.array([0.1, 1.0, 5.0, 1.0, 1.0])
    K = np.array([0.6, 1.0, 1.4, 1.0 + 1e-6, 0.9])
    cases = [
        (sg.HAGAN, [0.3, 1.0, -0.5, 0.0]),         # nu -> 0, beta = 1: sigma = alpha
        (sg.HAGAN, [0.02, 0.0, 0.0, 0.0]),         # normal model
        (sg.HAGAN, [0.2, 0.5, 0.999, 0.8]),        # rho near +1
        (sg.HAGAN, [0.2, 0.5, -0.999, 0.8]),       # rho near -1
        (sg.OBLOJ, [0.2, 1.0, -0.3, 0.6]),         # beta = 1 limit of z
        (sg.OBLOJ, [0.2, 0.999999, -0.3, 0.6]),
        (sg.HAGAN, [0.5, 0.3, -0.2, 3.0]),         # large z
    ]
    for model, p in cases:
        got = sg.implied_vol(model, p, 1.0, T, K, prec=prec).cpu().numpy()
        ref = O.implied_vol(model, p, 1.0, T, K)
        assert np.max(np.abs(got - ref) / ref) <= TOL[prec], (model, p)
    got = sg.implied_vol(sg.HAGAN, [0.3, 1.0, -0.5, 0.0], 1.0, T, K, prec=prec).cpu().numpy()
    assert np.allclose(got, 0.3, rtol=TOL[prec], atol=0)


def test_paper_printed_dsabr1_surface_on_gpu():
    from helpers import Golden
    g = Golden("dsabr1_eurostoxx50.txt")
    p = g.floats("params")
    S0 = g.floats("spot")[0]
    for T, r, y, k, printed in g.rows:
        f = S0 * np.exp((r - y) * T)
        for prec in (sg.FP64, sg.FP32):
            v = sg.implied_vol(sg.DYN_I, p, f, [T], [k * S0], prec=prec).cpu().numpy()[0]
            assert abs(100 * v - printed) <= 1e-4 + (3e-5 * printed if prec == sg.FP32 else 0)


def test_large_launch_sampled_against_oracle():
    rng = np.random.default_rng(7)
    n = (1 << 22) + 13
    T = torch.from_numpy(rng.choice([0.25, 1.0, 3.0], n)).cuda()
    K = torch.from_numpy(rng.uniform(0.5, 1.6, n)).cuda()
    p = [0.25, 0.6, -0.3, 0.7]
    out = sg.implied_vol(sg.HAGAN, p, 1.0, T, K, prec=sg.FP32)
    idx = np.concatenate([rng.integers(0, n, 2000), [0, n - 1]])
    ref = O.implied_vol(sg.HAGAN, p, 1.0, T.cpu().numpy()[idx], K.cpu().numpy()[idx])
    got = out.cpu().numpy()[idx]
    assert np.max(np.abs(got - ref) / ref) <= 3e-5


def test_empty_and_invalid_inputs():
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    out = sg.implied_vol(sg.HAGAN, [0.2, 0.5, 0.0, 0.5], 1.0, e, e)
    assert out.numel() == 0
    with pytest.raises(sg.SabrError):
        sg.implied_vol(sg.HAGAN, [-0.2, 0.5, 0.0, 0.5], 1.0, [1.0], [1.0])
    with pytest.raises(sg.SabrError):
        sg.implied_vol(sg.HAGAN, [0.2, 1.5, 0.0, 0.5], 1.0, [1.0], [1.0])
    with pytest.raises(sg.SabrError):
        sg.implied_vol(sg.HAGAN, [0.2, 0.5, 1.0, 0.5], 1.0, [1.0], [1.0])
    with pytest.raises(sg.SabrError):
        sg.implied_vol(sg.HAGAN, [0.2, 0.5, 0.0, 0.5], -1.0, [1.0], [1.0])


@pytest.mark.parametrize("prec", [sg.FP64, sg.FP32])
@pytest.mark.parametrize("model", [sg.HAGAN, sg.OBLOJ])
def test_static_formulas_on_an_extreme_grid(model, prec):
    # strikes from 5% to 20x the forward, maturities from 4 days to 30 years,
    # parameters at the edges of their ranges: the branch-free z/x(z) and the
    # SFU forms must hold their accuracy everywhere the formula is defined
    K = np.exp(np.linspace(np.log(0.05), np.log(20.0), 41))
    K = np.concatenate([K, [1.0, 1.0 + 1e-7, 1.0 - 1e-7, 1.0 + 1e-3]])
    T = np.array([0.01, 1.0, 30.0])
    TT, KK = np.repeat(T, K.size), np.tile(K, T.size)
    worst = 0.0
    for alpha in (0.01, 0.3, 2.0):
        for beta in (0.0, 0.5, 1.0):
            for rho in (-0.999, -0.5, 0.0, 0.5, 0.999):
                for nu in (0.01, 0.5, 3.0):
                    p = [alpha, beta, rho, nu]
                    ref = O.implied_vol(model, p, 1.0, TT, KK)
                    got = sg.implied_vol(model, p, 1.0, TT, KK, prec=prec).cpu().numpy()
                    ok = np.isfinite(ref) & (ref > 0)
                    assert np.all(np.isfinite(got[ok])), p
                    err = np.abs(got[ok] - ref[ok]) / ref[ok]
                    worst = max(worst, float(err.max()))
    assert worst <= TOL[prec], worst


@pytest.mark.parametrize("prec", [sg.FP64, sg.FP32])
@pytest.mark.parametrize("model", [sg.DYN_I, sg.DYN_II])
def test_dynamic_formulas_on_an_extreme_grid(model, prec):
    # maturities from 4 days to 30 years and decay rates a, b from 0 to 5
    # (a T, b T up to 150): the Case I series/closed-form switch and the
    # Case II eta2^2 rules must hold their accuracy
    K = np.exp(np.linspace(np.log(0.3), np.log(3.0), 15))
    T = np.array([0.01, 0.25, 1.0, 10.0, 30.0])
    TT, KK = np.repeat(T, K.size), np.tile(K, T.size)
    rng = np.random.default_rng(77 + model + 10 * prec)
    worst, n = 0.0, 0
    for a in (0.0, 1e-3, 1.0, 5.0):
        for b in (0.0, 1e-3, 1.0, 5.0):
            p = [0.25, 0.7, -0.5, 0.8, a, b]
            if model == sg.DYN_II:
                while True:
                    q = p + [rng.uniform(-0.2, 0.2), rng.uniform(0.0, 0.3), rng.uniform(-0.3, 0.3),
                             rng.uniform(-0.3, 0.3)]
                    if O.feasible(O.DYN_II, q, 30.0):
                        p = q
                        break
            ref = O.implied_vol(model, p, 1.0, TT, KK)
            got = sg.implied_vol(model, p, 1.0, TT, KK, prec=prec).cpu().numpy()
            ok = np.isfinite(ref) & (ref > 0)
            n += int(ok.sum())
            assert np.all(np.isfinite(got[ok])), p
            worst = max(worst, float((np.abs(got[ok] - ref[ok]) / ref[ok]).max()))
    assert n > 0.8 * 16 * TT.size and worst <= TOL[prec], (n, worst)
