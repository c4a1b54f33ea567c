"""sabr_mc_price_noalloc: the Monte Carlo pricer for callers that cannot let a
library allocate device memory (processes whose device memory belongs to
their own fixed-size pool, applications that forbid library allocations).
Called through the C-ABI, it must give the prices of sabr_mc_price within the
MC parity tolerance, on two calls in a row with different problems (the
shared scratch keeps the previous call's contents, which must not leak into
the next result).  This file is collected last so that a run stopping at its
first failure has run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2407_20713_gb300 as sg
from paper_2407_20713_gb300 import capi

pytestmark = pytest.mark.gpu

TOL = {sg.FP32: 1e-5, sg.FP64: 1e-10}


def _call(name, model, params, T, K, is_call, disc, n_paths, seed, prec):
    lib = capi.load()
    p = np.zeros(10)
    p[: len(params)] = params
    T = np.ascontiguousarray(T, dtype=np.float64)
    K = np.ascontiguousarray(K, dtype=np.float64)
    ic = np.ascontiguousarray(is_call, dtype=np.int8)
    dc = np.ascontiguousarray(disc, dtype=np.float64)
    price = torch.full((T.size,), np.nan, dtype=torch.float64, device="cuda")
    se = torch.full((T.size,), np.nan, dtype=torch.float64, device="cuda")
    st = getattr(lib, name)(model, p.ctypes.data_as(capi.PD), 1.0, T.ctypes.data_as(capi.PD),
                            K.ctypes.data_as(capi.PD), ic.ctypes.data_as(capi.PI8), dc.ctypes.data_as(capi.PD),
                            T.size, n_paths, 250.0, seed, ctypes.c_void_p(price.data_ptr()),
                            ctypes.c_void_p(se.data_ptr()), prec,
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    capi.check(st, name)
    torch.cuda.synchronize()
    return price.cpu().numpy(), se.cpu().numpy()


PROBLEMS = [
    # a larger problem first, then a smaller one: the second call runs on
    # scratch that still holds the first call's tables and partial sums
    (sg.DYN_I, [0.3, 0.7, -0.6, 0.9, 0.5, 1.2], np.repeat([0.25, 0.5, 1.0, 1.5], 6),
     np.tile([0.8, 0.9, 1.0, 1.05, 1.1, 1.3], 4), 50000, 17),
    (sg.HAGAN, [0.25, 0.5, -0.3, 0.6], np.array([0.5, 1.0, 1.0]), np.array([1.0, 0.9, 1.2]), 20000, 5),
]


@pytest.mark.parametrize("prec", [sg.FP32, sg.FP64])
def test_noalloc_prices_match_mc_price_on_two_calls_in_a_row(prec):
    got = []
    for model, p, T, K, n_paths, seed in PROBLEMS:
        ic = (np.arange(T.size) % 3 != 1).astype(np.int8)
        disc = np.linspace(1.0, 0.95, T.size)
        got.append(_call("sabr_mc_price_noalloc", model, p, T, K, ic, disc, n_paths, seed, prec))
    for (model, p, T, K, n_paths, seed), (price, se) in zip(PROBLEMS, got):
        ic = (np.arange(T.size) % 3 != 1).astype(np.int8)
        disc = np.linspace(1.0, 0.95, T.size)
        ref, rse = _call("sabr_mc_price", model, p, T, K, ic, disc, n_paths, seed, prec)
        assert np.all(np.isfinite(price)) and np.all(np.isfinite(se))
        assert np.max(np.abs(price - ref)) <= TOL[prec]
        assert np.max(np.abs(se - rse)) <= TOL[prec]


def test_noalloc_refuses_problems_beyond_its_scratch():
    # 60 maturities at 2^22 paths: 1216 blocks x 60 x 256 B of partial sums
    T = np.repeat(np.linspace(0.1, 12.0, 60), 8)
    K = np.tile(np.linspace(0.8, 1.2, 8), 60)
    with pytest.raises(sg.SabrError) as e:
        _call("sabr_mc_price_noalloc", sg.HAGAN, [0.25, 0.5, -0.3, 0.6], T, K, np.ones(T.size), np.ones(T.size),
              1 << 22, 1, sg.FP32)
    assert e.value.status == capi.EINVAL
