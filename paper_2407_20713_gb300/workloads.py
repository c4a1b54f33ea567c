"""Seeded synthetic workloads shaped like the calibration problems of the
paper's experiments (Sec. 6 and Appendix B: a few maturities of 15-21
strikes around the money, vols of 13-34%).

This module only draws inputs: strikes, maturities, true parameters, noise
samples, boxes and schedules.  It contains none of the method's arithmetic;
market vols or prices are formed by the caller from the true parameters
(through the oracle in tests, through the library in the benchmark) plus the
noise drawn here.
"""
from dataclasses import dataclass, field
from typing import List

import numpy as np

from .capi import DYN_I, DYN_II, HAGAN

STATIC_LO = [1e-6, 0.0, -1.0 + 1e-6, 1e-6]
STATIC_HI = [2.0, 1.0, 1.0 - 1e-6, 3.0]
DYN1_LO = [1e-6, 0.0, -1.0, 1e-6, 0.0, 0.0]
DYN1_HI = [2.0, 1.0, 1.0, 3.0, 5.0, 5.0]
DYN2_LO = DYN1_LO + [-0.5, -0.5, -1.0, -1.0]
DYN2_HI = DYN1_HI + [0.5, 0.5, 1.0, 1.0]


@dataclass
class Smile:
    """Quotes of one calibration problem plus the truth that generates them."""
    model: int
    T: np.ndarray
    K: np.ndarray
    truth: np.ndarray
    noise: np.ndarray          # additive noise on the market value, drawn here
    lo: List[float]
    hi: List[float]
    n_chains: int
    fwd: float = 1.0
    meta: dict = field(default_factory=dict)


def one_smile(seed: int = 20240720) -> Smile:
    """T = 1, f = 1, 15 strikes K/f evenly in [0.6, 1.4] (ATM included),
    truth (0.2, 0.7, -0.4, 0.5), N(0, 1e-4) vol noise, 64 chains."""
    rng = np.random.default_rng(seed)
    K = 0.6 + 0.8 * np.arange(15) / 14
    return Smile(HAGAN, np.ones(15), K, np.array([0.2, 0.7, -0.4, 0.5]), rng.normal(0.0, 1e-4, 15),
                 STATIC_LO, STATIC_HI, 64)


SURFACE_MATURITIES = np.array([0.1, 0.25, 0.5, 0.75, 1.0, 1.5, 2.0, 3.0, 4.0, 5.0])


def static_surface(seed: int = 20240721, n_chains: int = 4096) -> List[Smile]:
    """10 maturities x 21 strikes K/f in [0.5, 1.5]; each maturity is its own
    smile with truths alpha~U[0.1,0.5], beta~U[0.3,1], rho~U[-0.8,0.2],
    nu~U[0.2,1.5] and N(0, 1e-4) vol noise."""
    rng = np.random.default_rng(seed)
    K = 0.5 + 0.05 * np.arange(21)
    out = []
    for T in SURFACE_MATURITIES:
        truth = np.array([rng.uniform(0.1, 0.5), rng.uniform(0.3, 1.0), rng.uniform(-0.8, 0.2),
                          rng.uniform(0.2, 1.5)])
        out.append(Smile(HAGAN, np.full(21, T), K.copy(), truth, rng.normal(0.0, 1e-4, 21), STATIC_LO, STATIC_HI,
                         n_chains, meta={"T": float(T)}))
    return out


DYN_MATURITIES = np.array([0.1, 0.25, 0.5, 0.75, 1.0, 1.5, 2.0, 3.0, 4.0, 5.0, 7.0, 10.0])


def dynamic_surface(seed: int = 20240722, case: int = 1, n_chains: int = 8192, feasible=None) -> Smile:
    """12 maturities in [0.1, 10] x 21 strikes K/f in [0.5, 1.5], one joint
    problem.  Case I truths: alpha~U[0.1,0.5], beta~U[0.5,1], rho0~U[-0.8,0],
    nu0~U[0.2,1], a,b~U[0,2]; Case II adds d_rho~U[-0.2,0.2], d_nu~U[0,0.3],
    q_rho, q_nu~U[-0.3,0.3], redrawn until `feasible(truth)` holds."""
    rng = np.random.default_rng(seed)
    T = np.repeat(DYN_MATURITIES, 21)
    K = np.tile(0.5 + 0.05 * np.arange(21), DYN_MATURITIES.size)
    base = [rng.uniform(0.1, 0.5), rng.uniform(0.5, 1.0), rng.uniform(-0.8, 0.0), rng.uniform(0.2, 1.0),
            rng.uniform(0.0, 2.0), rng.uniform(0.0, 2.0)]
    if case == 1:
        truth = np.array(base)
        return Smile(DYN_I, T, K, truth, rng.normal(0.0, 1e-4, T.size), DYN1_LO, DYN1_HI, n_chains)
    while True:
        truth = np.array(base + [rng.uniform(-0.2, 0.2), rng.uniform(0.0, 0.3), rng.uniform(-0.3, 0.3),
                                 rng.uniform(-0.3, 0.3)])
        if feasible is None or feasible(truth):
            break
    return Smile(DYN_II, T, K, truth, rng.normal(0.0, 1e-4, T.size), DYN2_LO, DYN2_HI, n_chains)


MC_MATURITIES = np.array([0.25, 0.5, 0.75, 1.0, 1.25, 1.5, 1.75, 2.0])


def mc_surface(seed: int = 20240723, n_chains: int = 256) -> Smile:
    """8 maturities x 15 strikes K/f evenly in [0.6, 1.4] of calls; truth
    drawn as in static_surface.  Prices come from 2^24 paths on a separate
    Philox key (meta['market_seed']); calibration uses 2^16 paths at 250
    steps a year (meta['cal_seed'])."""
    rng = np.random.default_rng(seed)
    T = np.repeat(MC_MATURITIES, 15)
    K = np.tile(0.6 + 0.8 * np.arange(15) / 14, MC_MATURITIES.size)
    truth = np.array([rng.uniform(0.1, 0.5), rng.uniform(0.3, 1.0), rng.uniform(-0.8, 0.2),
                      rng.uniform(0.2, 1.5)])
    return Smile(HAGAN, T, K, truth, np.zeros(T.size), STATIC_LO, STATIC_HI, n_chains,
                 meta={"market_paths": 1 << 24, "cal_paths": 1 << 16, "steps_per_year": 250.0,
                       "market_seed": int(rng.integers(1, 2 ** 63)), "cal_seed": int(rng.integers(1, 2 ** 63))})


@dataclass
class Request:
    arrival: float        # seconds after the start of the stream
    smile: Smile
    cost: int             # 0 = implied-vol misfit, 1 = MC price misfit
    mc_paths: int
    n_levels: int
    chain_len: int


def serving_stream(n: int = 10000, rate_hz: float = 100.0, seed: int = 20240724) -> List[Request]:
    """Poisson arrivals of calibration requests of uneven size: 1-12
    maturities x 5-41 strikes.  With probability 0.05 a request is a static
    MC-price calibration (2^14-2^16 paths, 64 chains, 10 x 10 schedule);
    otherwise it is a formula calibration (1024 chains, 100 x 50 schedule),
    Hagan with probability 0.8 and dynamic (Case I or II, evenly) otherwise."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for _ in range(n):
        t += rng.exponential(1.0 / rate_hz)
        n_mats = int(rng.integers(1, 13))
        n_strikes = int(rng.integers(5, 42))
        mats = np.sort(rng.choice(DYN_MATURITIES, n_mats, replace=False))
        K1 = np.linspace(0.7, 1.3, n_strikes)
        T = np.repeat(mats, n_strikes)
        K = np.tile(K1, n_mats)
        u = rng.uniform()
        if u < 0.05:
            truth = np.array([rng.uniform(0.1, 0.5), rng.uniform(0.3, 1.0), rng.uniform(-0.8, 0.2),
                              rng.uniform(0.2, 1.5)])
            sm = Smile(HAGAN, T, K, truth, np.zeros(T.size), STATIC_LO, STATIC_HI, 64)
            reqs.append(Request(t, sm, 1, int(2 ** rng.integers(14, 17)), 10, 10))
            continue
        if rng.uniform() < 0.8:
            truth = np.array([rng.uniform(0.1, 0.5), rng.uniform(0.3, 1.0), rng.uniform(-0.8, 0.2),
                              rng.uniform(0.2, 1.5)])
            sm = Smile(HAGAN, T, K, truth, rng.normal(0.0, 1e-4, T.size), STATIC_LO, STATIC_HI, 1024)
        else:
            case = 1 if rng.uniform() < 0.5 else 2
            base = [rng.uniform(0.1, 0.5), rng.uniform(0.5, 1.0), rng.uniform(-0.8, 0.0), rng.uniform(0.2, 1.0),
                    rng.uniform(0.0, 2.0), rng.uniform(0.0, 2.0)]
            if case == 1:
                sm = Smile(DYN_I, T, K, np.array(base), rng.normal(0.0, 1e-4, T.size), DYN1_LO, DYN1_HI, 1024)
            else:
                extra = [rng.uniform(-0.1, 0.1), rng.uniform(0.0, 0.2), rng.uniform(-0.1, 0.1),
                         rng.uniform(0.0, 0.1)]
                sm = Smile(DYN_II, T, K, np.array(base + extra), rng.normal(0.0, 1e-4, T.size), DYN2_LO,
                           DYN2_HI, 1024)
        reqs.append(Request(t, sm, 0, 0, 100, 50))
    return reqs
