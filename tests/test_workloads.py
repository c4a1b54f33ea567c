"""The seeded synthetic inputs (paper_2407_20713_gb300/workloads.py): the
shapes and distributions the benchmark and the parity tests are built on
(10 x 21 static surface, 12 x 21 dynamic surfaces, 8 x 15 MC surface, the
serving stream's mix and arrival rate), reproducible from their seeds, with
every truth inside its calibration box."""
import numpy as np

import oracle as O
from paper_2407_20713_gb300 import workloads as W


def _inside(x, lo, hi):
    return np.all(np.asarray(x) >= np.asarray(lo)) and np.all(np.asarray(x) <= np.asarray(hi))


def test_static_surface_shape_and_reproducibility():
    a, b = W.static_surface(), W.static_surface()
    assert len(a) == 10
    for sa, sb, T in zip(a, b, W.SURFACE_MATURITIES):
        assert sa.T.size == 21 and np.all(sa.T == T) and sa.n_chains == 4096
        assert np.allclose(sa.K, 0.5 + 0.05 * np.arange(21))
        assert np.array_equal(sa.truth, sb.truth) and np.array_equal(sa.noise, sb.noise)
        assert _inside(sa.truth, sa.lo, sa.hi) and abs(np.std(sa.noise) - 1e-4) < 6e-5
    assert not np.array_equal(a[0].truth, W.static_surface(seed=1)[0].truth)


def test_dynamic_surfaces_are_feasible_and_inside_their_boxes():
    for case, model in ((1, O.DYN_I), (2, O.DYN_II)):
        w = W.dynamic_surface(case=case, feasible=lambda x: O.feasible(O.DYN_II, x, 10.0))
        assert w.T.size == 12 * 21 and np.array_equal(np.unique(w.T), W.DYN_MATURITIES)
        assert w.n_chains == 8192 and _inside(w.truth, w.lo, w.hi)
        assert O.feasible(model, w.truth, float(w.T.max()))


def test_mc_surface_shape():
    w = W.mc_surface()
    assert w.T.size == 8 * 15 and np.array_equal(np.unique(w.T), W.MC_MATURITIES)
    assert np.allclose(np.unique(w.K), 0.6 + 0.8 * np.arange(15) / 14)
    assert w.meta["cal_paths"] == 1 << 16 and w.meta["market_paths"] == 1 << 24
    assert w.meta["cal_seed"] != w.meta["market_seed"] and _inside(w.truth, w.lo, w.hi)


def test_serving_stream_mix_sizes_and_arrivals():
    reqs = W.serving_stream(n=4000, rate_hz=50.0)
    mc = [r for r in reqs if r.cost == 1]
    formula = [r for r in reqs if r.cost == 0]
    hagan = [r for r in formula if r.smile.model == O.HAGAN]
    assert abs(len(mc) / len(reqs) - 0.05) < 0.015
    assert abs(len(hagan) / len(formula) - 0.8) < 0.03
    for r in reqs:
        n_mats, n_q = np.unique(r.smile.T).size, r.smile.T.size
        assert 1 <= n_mats <= 12 and 5 <= n_q // n_mats <= 41 and n_q % n_mats == 0
        assert _inside(r.smile.truth, r.smile.lo, r.smile.hi)
    assert all(2 ** 14 <= r.mc_paths <= 2 ** 16 for r in mc)
    gaps = np.diff([0.0] + [r.arrival for r in reqs])
    assert abs(gaps.mean() * 50.0 - 1.0) < 0.06
