"""The host side of the multi-GPU forms (Sec. 5.1): chain-sharded SA and
block-sharded Monte Carlo partials, run as gloo ranks on CPU.

The exchange logic of paper_2407_20713_gb300.shard (per-level all-gather of
the shards' minima, lexicographic restart point, merge of the shard results,
block-order gather of partial sums) is driven here by an engine that runs the
oracle's SA on a share of the chains; the sharded run must reproduce the
oracle's unsharded calibration bit for bit.  The GPU engine (the library's
sabr_shard_*) is checked against sabr_calibrate in tests/test_gpu_shard.py."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

K15 = 0.6 + 0.8 * np.arange(15) / 14
LO4 = [1e-6, 0.0, -1 + 1e-6, 1e-6]
HI4 = [2.0, 1.0, 1 - 1e-6, 3.0]
SA = dict(n_levels=6, chain_len=15, seed=17)


def _market():
    sys.path.insert(0, ROOT)
    import oracle as O
    T = np.repeat([0.5, 2.0], 15)
    K = np.tile(K15, 2)
    m = O.implied_vol(O.HAGAN, [0.2, 0.7, -0.4, 0.5], 1.0, T, K) + np.random.default_rng(3).normal(0, 1e-4, 30)
    return T, K, m


class OracleEngine:
    """The oracle's SA on chains c0 .. c0+nc-1, behind the engine interface."""

    def __init__(self, n_chains, c0, nc):
        import oracle as O
        from paper_2407_20713_gb300 import shard as S
        self.S = S
        T, K, m = _market()
        self.sh = O.SaShard(O.HAGAN, 1.0, T, K, m, LO4, HI4, n_chains=n_chains, c0=c0, nc=nc, **SA)

    def level(self, lv):
        return self.sh.level(lv)

    def restart(self, f, x):
        self.sh.restart(f, x)

    def result(self):
        f, c, x, ev, ac = self.sh.result()
        return self.S.ShardResult(f, c, x, ev, ac, np.array([self.sh.xs[0], self.sh.fs]))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _sa_worker(rank, world, port, n_chains, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2407_20713_gb300 import shard as S
    begin, count = S.chain_slice(n_chains, rank, world)
    merged, win = S.run_sharded(OracleEngine(n_chains, begin, count), SA["n_levels"], S.torch_allgather())
    out[rank] = (merged.misfit, merged.chain, merged.params.tolist(), merged.n_evals, merged.n_accepts,
                 merged.extra.tolist(), win)
    dist.destroy_process_group()


def _spawn(target, world, *args):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port) + args + (out,)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    return dict(out)


@pytest.mark.parametrize("world,n_chains", [(2, 37), (3, 64)])
def test_chain_sharded_sa_over_gloo_equals_the_unsharded_oracle(world, n_chains):
    sys.path.insert(0, ROOT)
    import oracle as O
    T, K, m = _market()
    ref = O.sa_calibrate(O.HAGAN, 1.0, T, K, m, LO4, HI4, n_chains=n_chains, **SA)
    out = _spawn(_sa_worker, world, n_chains)
    assert sorted(out) == list(range(world))
    for r in range(world):
        f, chain, params, ne, na, extra, win = out[r]
        assert out[r] == out[0]                         # every rank ends with the same result
        assert f == ref["misfit"]                        # bit for bit
        assert np.array_equal(np.array(params)[:4], ref["params"])
        assert ne == ref["n_evals"] and na == ref["n_accepts"]
        assert extra[1] == ref["restart_misfit"] and extra[0] == ref["restart_params"][0]


def test_slices_cover_the_range_in_order():
    from paper_2407_20713_gb300 import shard as S
    for total in (1, 7, 64, 1216):
        for world in (1, 2, 3, 8):
            if world > total:
                continue
            sl = [S.chain_slice(total, r, world) for r in range(world)]
            assert sl[0][0] == 0 and sum(c for _, c in sl) == total
            assert all(sl[i][0] + sl[i][1] == sl[i + 1][0] for i in range(world - 1))
            assert max(c for _, c in sl) - min(c for _, c in sl) <= 1
    # ties go to the lower chain, as the one-GPU block argmin does
    p = [(1.0, 5, np.zeros(10)), (0.5, 9, np.ones(10)), (0.5, 3, np.full(10, 2.0))]
    assert S.lexicographic_min(p)[1] == 3


def _gather_worker(rank, world, port, total, out):
    # the MC path: each rank owns a block range; the gathered partials,
    # trimmed per rank, are the full array in block order
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2407_20713_gb300 import shard as S
    begin, count = S.chain_slice(total, rank, world)
    part = torch.arange(begin * 4, (begin + count) * 4, dtype=torch.float64).reshape(count, 4)
    full = S.gather_blocks(part, total)
    out[rank] = full.numpy().ravel().tolist()
    dist.destroy_process_group()


def test_block_partials_gather_in_block_order():
    out = _spawn(_gather_worker, 3, 11)
    for r in range(3):
        assert out[r] == list(np.arange(44, dtype=float))
