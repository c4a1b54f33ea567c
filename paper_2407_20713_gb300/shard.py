"""Multi-GPU forms of the calibration and the pricer (Sec. 5.1, Sec. 5.2).

The paper runs the chains of one calibration on several GPUs and, at the end
of every temperature level, takes the minimum of the GPUs' minima on the host
as the common restart point of the next level (its OpenMP scheme, one host
thread per GPU).  Here one process drives one GPU; a shard (`api.Shard`, the
C-ABI's sabr_shard_*) holds a contiguous range of the chains, and the
per-level exchange of shard minima is an all-gather of a few doubles over
torch.distributed (gloo or NCCL).  The Monte Carlo pricer is split by blocks
of its grid; the shards' per-block FP64 partial sums are gathered in block
order and reduced on every rank.

Both forms reproduce the one-GPU results bit for bit: chains draw their
proposals from counters keyed by their global index and their lanes are
chosen from the total chain count, minima are lexicographic in (cost, global
chain), and the pricer's per-block partials do not depend on which device
computed them.

Only host logic lives here; every step of the method runs in the library's
kernels.  The exchange is written against a small engine interface (level,
restart, result) so that it can be driven by any engine that runs a share of
the chains.
"""
from dataclasses import dataclass
from typing import Callable, List, Sequence, Tuple

import numpy as np

Point = Tuple[float, int, np.ndarray]  # (cost, global chain, x[10])


def chain_slice(total: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous share (begin, count) of `total` chains (or blocks) for
    `rank` of `world`; the first total % world ranks take one more."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank outside [0, world)")
    base, extra = divmod(int(total), int(world))
    begin = rank * base + min(rank, extra)
    return begin, base + (1 if rank < extra else 0)


def lexicographic_min(points: Sequence[Point]) -> Point:
    """The point of lowest cost, lowest global chain on a tie (the order the
    one-GPU argmin over blocks of chains produces)."""
    return min(points, key=lambda p: (p[0], p[1]))


@dataclass
class ShardResult:
    """One shard's part of a calibration result."""
    misfit: float          # best cost evaluated by the shard's chains
    chain: int             # its global chain (-1 when no level ran)
    params: np.ndarray     # [10]
    n_evals: int
    n_accepts: int
    extra: np.ndarray      # engine-specific values carried with the winner

    def encode(self) -> np.ndarray:
        return np.concatenate([[self.misfit, float(self.chain)], self.params,
                               [float(self.n_evals), float(self.n_accepts)], self.extra]).astype(np.float64)

    @staticmethod
    def decode(v: np.ndarray, n_extra: int) -> "ShardResult":
        return ShardResult(float(v[0]), int(v[1]), v[2:12].copy(), int(v[12]), int(v[13]), v[14:14 + n_extra].copy())


def encode_point(p: Point) -> np.ndarray:
    f, c, x = p
    return np.concatenate([[f, float(c)], np.asarray(x, dtype=np.float64)[:10]])


def decode_point(v: np.ndarray) -> Point:
    return float(v[0]), int(v[1]), v[2:12].copy()


def run_sharded(engine, n_levels: int, allgather: Callable[[np.ndarray], List[np.ndarray]]):
    """The synchronous multi-device SA of Sec. 5.1 over one shard `engine`:
    per level, run the shard's chains, gather every shard's lowest final
    state, restart from the lexicographic minimum; then merge the shards'
    results (lowest (misfit, chain); counters summed).  `engine.level(lv)`
    returns a Point, `engine.restart(f, x)` sets the next start and
    `engine.result()` a ShardResult; `allgather(v)` returns every rank's
    vector v in rank order.  Returns (merged ShardResult, winner's rank)."""
    for lv in range(int(n_levels)):
        mine = engine.level(lv)
        pts = [decode_point(v) for v in allgather(encode_point(mine))]
        f, _, x = lexicographic_min(pts)
        engine.restart(f, x)
    r = engine.result()
    n_extra = r.extra.size
    allr = [ShardResult.decode(v, n_extra) for v in allgather(r.encode())]
    win = min(range(len(allr)), key=lambda i: (allr[i].misfit, allr[i].chain))
    w = allr[win]
    merged = ShardResult(w.misfit, w.chain, w.params, sum(a.n_evals for a in allr), sum(a.n_accepts for a in allr),
                         w.extra)
    return merged, win


def torch_allgather(group=None):
    """allgather(v) over torch.distributed: a float64 vector per rank, in rank
    order (CUDA tensors under NCCL, host tensors otherwise)."""
    import torch
    import torch.distributed as dist

    def gather(v: np.ndarray) -> List[np.ndarray]:
        dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else "cpu"
        t = torch.as_tensor(np.ascontiguousarray(v, dtype=np.float64), device=dev)
        out = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
        dist.all_gather(out, t, group=group)
        return [o.cpu().numpy() for o in out]
    return gather


class _CudaEngine:
    """The library's shard (sabr_shard_*) behind the engine interface."""

    def __init__(self, shard):
        self.shard = shard

    def level(self, lv):
        return self.shard.level(lv)

    def restart(self, f, x):
        self.shard.restart(f, x)

    def result(self):
        r, chain = self.shard.result()
        p = np.zeros(10)
        p[:r.params.size] = r.params
        rp = np.zeros(10)
        rp[:r.restart_params.size] = r.restart_params
        extra = np.concatenate([[r.misfit_fp64, r.restart_misfit, float(r.status)], rp])
        return ShardResult(r.misfit, chain, p, r.n_evals, r.n_accepts, extra)


def calibrate_sharded(problem, group=None, stream=None, allgather=None):
    """Calibrate `problem` with its chains split over the ranks of a
    torch.distributed group (one GPU per rank); every rank returns the same
    CalibrationResult, equal to api.calibrate(problem) on one GPU."""
    import torch.distributed as dist
    from . import api, capi

    rank, world = dist.get_rank(group), dist.get_world_size(group)
    begin, count = chain_slice(problem.n_chains, rank, world)
    shard = api.Shard(problem, begin, count, stream=stream)
    try:
        merged, _ = run_sharded(_CudaEngine(shard), problem.n_levels, allgather or torch_allgather(group))
    finally:
        shard.close()
    d = capi.N_PARAMS[problem.model]
    e = merged.extra
    return api.CalibrationResult(merged.params[:d].copy(), merged.misfit, float(e[0]), e[3:3 + d].copy(),
                                 float(e[1]), merged.n_evals, merged.n_accepts, int(e[2]))


def gather_blocks(part, total: int, group=None):
    """Every rank's block partials (rank r holds the blocks
    chain_slice(total, r, world), one row each), concatenated in block order
    on every rank.  Shares are padded to the largest for the all-gather and
    trimmed after it.  Device tensors go through NCCL as they are; under
    another backend they travel through host memory and come back to the
    device of `part`."""
    import torch
    import torch.distributed as dist

    rank, world = dist.get_rank(group), dist.get_world_size(group)
    count = chain_slice(total, rank, world)[1]
    if part.shape[0] != count:
        raise ValueError("partials do not match this rank's share of the blocks")
    nccl = dist.get_backend(group) == "nccl"
    width = chain_slice(total, 0, world)[1]  # the largest share
    buf = torch.zeros((width,) + tuple(part.shape[1:]), dtype=part.dtype, device=part.device if nccl else "cpu")
    buf[:count] = part if nccl else part.cpu()
    out = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(out, buf, group=group)
    return torch.cat([o[:chain_slice(total, r, world)[1]] for r, o in enumerate(out)]).to(part.device)


def mc_price_sharded(model, params, fwd, T, K, is_call=None, discount=None, n_paths=1 << 16, steps_per_year=250.0,
                     seed=0, prec=0, group=None, stream=None):
    """mc_price with the blocks of its grid split over the ranks of a
    torch.distributed group; every rank returns the prices and standard
    errors of the one-GPU pricer (bit for bit on devices of one kind)."""
    import torch.distributed as dist
    from . import api

    rank, world = dist.get_rank(group), dist.get_world_size(group)
    kw = dict(is_call=is_call, discount=discount, n_paths=n_paths, steps_per_year=steps_per_year, seed=seed,
              prec=prec)
    total, dpb = api.mc_shard_layout(model, params, fwd, T, K, **kw)
    # every rank uses rank 0's grid
    total = int(torch_allgather(group)(np.array([float(total)]))[0][0])
    begin, count = chain_slice(total, rank, world)
    part = api.mc_shard_partials(model, params, fwd, T, K, total, begin, count, stream=stream, **kw)
    full = gather_blocks(part, total, group)
    return api.mc_shard_reduce(model, params, fwd, T, K, total, full, stream=stream, **kw)
