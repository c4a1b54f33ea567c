"""GPU parity of the multi-GPU forms (Sec. 5.1): a calibration whose chains
are split over shards (sabr_shard_*) and a Monte Carlo price whose grid is
split into block ranges (sabr_mc_shard_*) equal the one-GPU sabr_calibrate
and sabr_mc_price bit for bit.

One GPU stands in for several: the shards run one after another or side by
side on it, and exchange their per-level minima on the host (threads of one
process, or two processes over gloo).  No kernel waits on another."""
import os
import socket
import sys
import threading

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle as O
import paper_2407_20713_gb300 as sg
from paper_2407_20713_gb300 import shard as S

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
K21 = 0.5 + 0.05 * np.arange(21)
LO4 = [1e-6, 0.0, -1 + 1e-6, 1e-6]
HI4 = [2.0, 1.0, 1 - 1e-6, 3.0]
CASE2_LO = [0.05, 0.5, -1.0, 0.01, 0.0, 0.0, -0.5, -0.5, -1.0, -1.0]
CASE2_HI = [0.6, 1.0, 1.0, 1.5, 5.0, 5.0, 0.5, 0.5, 1.0, 1.0]


def _problem(model, prec, n_chains=1000, n_levels=12, chain_len=25, seed=5):
    if model == sg.HAGAN:
        T = np.repeat([0.5, 2.0], 21)
        K = np.tile(K21, 2)
        truth, lo, hi = [0.3, 0.6, -0.3, 0.8], LO4, HI4
    else:
        T = np.repeat([0.25, 1.0, 4.0], 21)
        K = np.tile(K21, 3)
        truth, lo, hi = [0.25, 0.8, -0.4, 0.6, 0.8, 0.9, 0.1, 0.15, 0.2, -0.1], CASE2_LO, CASE2_HI
    m = O.implied_vol(model, truth, 1.0, T, K) + np.random.default_rng(seed).normal(0, 1e-4, T.size)
    return sg.CalibrationProblem(model=model, T=T, K=K, market=m, lo=lo, hi=hi, prec=prec, n_chains=n_chains,
                                 n_levels=n_levels, chain_len=chain_len, seed=seed)


def _threaded_sharded(pb, world):
    """run_sharded on `world` shards of one GPU, one host thread each, the
    all-gather through a barrier."""
    box = [None] * world
    barrier = threading.Barrier(world)
    results = [None] * world
    errors = []

    def worker(r):
        try:
            torch.cuda.set_device(0)
            stream = torch.cuda.Stream()
            begin, count = S.chain_slice(pb.n_chains, r, world)
            shard = sg.Shard(pb, begin, count, stream=stream)

            def allgather(v):
                box[r] = v
                barrier.wait()
                out = list(box)
                barrier.wait()
                return out
            results[r] = S.run_sharded(S._CudaEngine(shard), pb.n_levels, allgather)
            shard.close()
        except Exception as e:  # report in the main thread
            errors.append(e)
            barrier.abort()

    ts = [threading.Thread(target=worker, args=(r,)) for r in range(world)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(600)
    assert not errors, errors
    return results


def _same(merged, ref, d):
    e = merged.extra
    assert merged.misfit == ref.misfit
    assert np.array_equal(merged.params[:d], ref.params)
    assert merged.n_evals == ref.n_evals and merged.n_accepts == ref.n_accepts
    assert e[0] == ref.misfit_fp64 and e[1] == ref.restart_misfit
    assert np.array_equal(e[3:3 + d], ref.restart_params)
    assert int(e[2]) == ref.status == 0


@pytest.mark.parametrize("model,prec,world", [(sg.HAGAN, sg.FP32, 2), (sg.HAGAN, sg.FP64, 3),
                                              (sg.DYN_II, sg.FP32, 2)])
def test_chain_shards_equal_the_one_gpu_calibration(model, prec, world):
    pb = _problem(model, prec, n_chains=1000 if model == sg.HAGAN else 300)
    ref = sg.calibrate(pb)
    out = _threaded_sharded(pb, world)
    d = sg.capi.N_PARAMS[model]
    for merged, _ in out:
        _same(merged, ref, d)
    if prec == sg.FP64:
        # and the FP64 form is the oracle's trajectory (Sec. 5 SA)
        o = O.sa_calibrate(model, 1.0, pb.T, pb.K, pb.market, pb.lo, pb.hi, n_chains=pb.n_chains,
                           n_levels=pb.n_levels, chain_len=pb.chain_len, seed=pb.seed, n_threads=8)
        assert out[0][0].n_evals == o["n_evals"]
        np.testing.assert_allclose(out[0][0].params[:d], o["params"], rtol=1e-10)


def test_shard_api_refuses_misuse():
    pb = _problem(sg.HAGAN, sg.FP32, n_chains=64, n_levels=2)
    with pytest.raises(sg.SabrError):
        sg.Shard(pb, 60, 10)                      # past the last chain
    mc = _problem(sg.HAGAN, sg.FP32, n_chains=64, n_levels=2)
    mc.cost = sg.COST_MC_PRICE
    with pytest.raises(sg.SabrError):
        sg.Shard(mc, 0, 32)                       # Technique II is not sharded
    sh = sg.Shard(pb, 0, 32)
    with pytest.raises(sg.SabrError):
        sh.level(1)                               # levels run in order
    with pytest.raises(sg.SabrError):
        sh.result()                               # not every level has run
    sh.close()


MC_T = np.repeat([0.25, 0.75, 1.5], 5)
MC_K = np.tile([0.8, 0.9, 1.0, 1.1, 1.25], 3)


@pytest.mark.parametrize("prec,world", [(sg.FP32, 2), (sg.FP32, 5), (sg.FP64, 3)])
def test_block_shards_equal_the_one_gpu_price(prec, world):
    p = [0.3, 0.7, -0.4, 0.6, 0.5, 1.2]
    kw = dict(is_call=(np.arange(15) % 4 != 1).astype(np.int8), discount=np.linspace(1.0, 0.97, 15),
              n_paths=300001, steps_per_year=100, seed=11, prec=prec)
    ref, rse = sg.mc_price(sg.DYN_I, p, 1.0, MC_T, MC_K, **kw)
    total, dpb = sg.mc_shard_layout(sg.DYN_I, p, 1.0, MC_T, MC_K, **kw)
    parts = [sg.mc_shard_partials(sg.DYN_I, p, 1.0, MC_T, MC_K, total, *S.chain_slice(total, r, world), **kw)
             for r in range(world)]
    full = torch.cat(parts)
    assert full.shape == (total, dpb)
    price, se = sg.mc_shard_reduce(sg.DYN_I, p, 1.0, MC_T, MC_K, total, full, **kw)
    assert torch.equal(price, ref) and torch.equal(se, rse)
    with pytest.raises(sg.SabrError):
        sg.mc_shard_partials(sg.DYN_I, p, 1.0, MC_T, MC_K, total, total - 1, 2, **kw)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _gloo_worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    pb = _problem(sg.HAGAN, sg.FP32)
    r = S.calibrate_sharded(pb)
    p = [0.3, 0.7, -0.4, 0.6, 0.5, 1.2]
    price, se = S.mc_price_sharded(sg.DYN_I, p, 1.0, MC_T, MC_K, n_paths=200000, steps_per_year=100, seed=3,
                                   prec=sg.FP32)
    out[rank] = (r.params.tolist(), r.misfit, r.misfit_fp64, r.n_evals, r.n_accepts, r.restart_params.tolist(),
                 price.cpu().numpy().tolist(), se.cpu().numpy().tolist())
    dist.destroy_process_group()


def test_two_processes_on_one_gpu_over_gloo():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(600)
        assert p.exitcode == 0
    ref = sg.calibrate(_problem(sg.HAGAN, sg.FP32))
    pr, se = sg.mc_price(sg.DYN_I, [0.3, 0.7, -0.4, 0.6, 0.5, 1.2], 1.0, MC_T, MC_K, n_paths=200000,
                         steps_per_year=100, seed=3, prec=sg.FP32)
    for r in range(2):
        params, misfit, m64, ne, na, restart, price, stderr = out[r]
        assert np.array_equal(params, ref.params) and misfit == ref.misfit and m64 == ref.misfit_fp64
        assert ne == ref.n_evals and na == ref.n_accepts and np.array_equal(restart, ref.restart_params)
        assert np.array_equal(price, pr.cpu().numpy()) and np.array_equal(stderr, se.cpu().numpy())
