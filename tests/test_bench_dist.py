"""The multi-rank path of bench.py: with world size 2 on the gloo backend
(CPU), the whole-job time is the maximum over ranks and the units and
end-to-end rates are summed over ranks."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    res = bench.aggregate(t_local=1.0 + rank, units_local=100.0 * (rank + 1), e2e_local=5.0 + rank, dist=dist)
    out[rank] = res
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        assert out[r]["time_s"] == 2.0          # max over ranks
        assert out[r]["units"] == 300.0         # summed
        assert out[r]["value"] == 150.0
        assert out[r]["e2e"] == 11.0


def test_aggregate_single_process():
    sys.path.insert(0, ROOT)
    import bench
    res = bench.aggregate(2.0, 10.0, 3.0, None)
    assert res == {"time_s": 2.0, "units": 10.0, "value": 5.0, "e2e": 3.0}


def test_profile_figures_are_read_only_while_the_kernel_is_unchanged(tmp_path, monkeypatch):
    # bench.py takes DRAM traffic and instructions per launch from the
    # committed ncu summary, and drops both once a source of the kernel no
    # longer matches the hash the summary records
    sys.path.insert(0, ROOT)
    import bench
    prof = ("| warp instructions (`smsp__inst_executed.sum`) | 1000.0 inst |\n"
            "| active lanes per warp instruction (`smsp__thread_inst_executed_per_inst_executed.ratio`) | 25.0  |\n"
            "traffic_bytes_per_launch: 4096\nsource_sha256 (k.cu): %s\n")
    import hashlib
    (tmp_path / "profiles").mkdir()
    (tmp_path / "paper_2407_20713_gb300" / "csrc").mkdir(parents=True)
    src = tmp_path / "paper_2407_20713_gb300" / "csrc" / "k.cu"
    src.write_bytes(b"kernel v1")
    (tmp_path / "profiles" / "k.md").write_text(prof % hashlib.sha256(b"kernel v1").hexdigest())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("k.md", ["k.cu"]) == 4096
    assert bench.profiled_thread_instructions("k.md", ["k.cu"]) == 25000.0
    assert abs(bench.issue_bound(50.0, 2000.0) - 152 * 128 * 2e9 / 50.0) < 1.0
    src.write_bytes(b"kernel v2")
    assert bench.profiled_traffic("k.md", ["k.cu"]) is None
    assert bench.profiled_thread_instructions("k.md", ["k.cu"]) is None
