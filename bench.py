#!/usr/bin/env python
"""Throughput benchmark of the SABR calibration hot path on GB300.

Workload (one "step"): Technique I calibration of a static SABR surface by
synchronous parallel Simulated Annealing -- 10 maturities T in {0.1 .. 5},
each its own smile of 21 strikes K/f in [0.5, 1.5], Hagan formula, FP32 bulk
arithmetic, 4096 chains per smile, geometric cooling 0.95, 200 levels x 100
proposals.  Inputs are synthetic (seeded truths + N(0, 1e-4) vol noise).

Metric: SA cost evaluations per second (one evaluation = the misfit of one
proposal over its 21 quotes), whole job over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank calibrates its own surface (distinct seeds) on its
own GPU; no data-path collective (weak scaling).  --impl reference times the
FP64 CPU oracle on a bounded sample of the same workload.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_LEVELS, CHAIN_LEN, N_CHAINS, FACTOR = 200, 100, 4096, 0.95
SFU_PER_QUOTE = 5    # Hagan quote: (Kf)^((1-b)/2), sqrt, log, two divisions
FP32_PER_QUOTE = 25  # the remaining FP32 arithmetic of eq. (haganf) + misfit
SMS = 152


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 form")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def surface_problems(smiles, market, prec, seed0):
    import paper_2407_20713_gb300 as sg
    out = []
    for i, (sm, mkt) in enumerate(zip(smiles, market)):
        out.append(sg.CalibrationProblem(model=sg.HAGAN, T=sm.T, K=sm.K, market=mkt, lo=sm.lo, hi=sm.hi,
                                         prec=prec, n_chains=sm.n_chains, factor=FACTOR, n_levels=N_LEVELS,
                                         chain_len=CHAIN_LEN, seed=seed0 + i))
    return out


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(smiles, market, n_levels=10):
    """The FP64 oracle, as it stands, on a bounded sample: smile 0 of the
    surface, all 4096 chains, n_levels of the 200 levels (x 100 proposals)."""
    import oracle as O
    sm, mkt = smiles[0], market[0]
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    r = O.sa_calibrate(O.HAGAN, 1.0, sm.T, sm.K, mkt, sm.lo, sm.hi, n_chains=sm.n_chains, factor=FACTOR,
                       n_levels=n_levels, chain_len=CHAIN_LEN, seed=1, n_threads=cores)
    dt = time.perf_counter() - t0
    return {"value": r["n_evals"] / dt, "unit": "cost-evals/s", "cores": cores, "kind": "oracle",
            "sample": "smile 1 of 10 (21 strikes), %d chains, %d of %d levels x %d proposals; %.1f s"
                      % (sm.n_chains, n_levels, N_LEVELS, CHAIN_LEN, dt)}


def oracle_market(smiles):
    import oracle as O
    return [O.implied_vol(O.HAGAN, sm.truth, 1.0, sm.T, sm.K) + sm.noise for sm in smiles]


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2407_20713_gb300 import workloads
    smiles = workloads.static_surface()
    market = oracle_market(smiles)
    for _ in range(args.warmup):
        cpu_baseline(smiles, market, n_levels=1)
    vals, dts = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(smiles, market, n_levels=4)
        dts.append(time.perf_counter() - t0)
        vals.append(cb["value"])
    value = float(np.mean(vals))
    cb["value"] = value
    cb["sample"] = "each step: smile 1 of 10, %d chains, 4 of %d levels x %d proposals" % (N_CHAINS, N_LEVELS,
                                                                                           CHAIN_LEN)
    line = {"impl": "reference", "metric": "SABR SA cost evals/s (static Hagan surface, 10x21, FP32 bulk)",
            "value": value, "unit": "cost-evals/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(dts)), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "static Hagan surface: 10 maturities x 21 strikes, 4096 chains/smile, "
                                   "200x100 SA", "sampled": True},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "cost-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    import paper_2407_20713_gb300 as sg
    from paper_2407_20713_gb300 import workloads

    smiles = workloads.static_surface(seed=20240721 + 1000 * rank, n_chains=N_CHAINS)
    # market vols from the true parameters (library, FP64) plus seeded noise
    market = [sg.implied_vol(sg.HAGAN, sm.truth, 1.0, sm.T, sm.K, prec=sg.FP64).cpu().numpy() + sm.noise
              for sm in smiles]
    problems = surface_problems(smiles, market, sg.FP32, seed0=7 + 100 * rank)
    stream = torch.cuda.current_stream()
    plan = sg.Plan(problems, use_graph=True)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    for _ in range(max(3, args.warmup)):
        plan.run(stream)
        plan.results()

    rates = None
    try:
        import ctypes
        buf = (ctypes.c_double * 8)()
        sg.capi.check(sg.capi.load().sabr_probe_pipe_rates(buf, 8, ctypes.c_void_p(stream.cuda_stream)),
                      "probe")
        rates = list(buf)
    except Exception:
        rates = None

    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    level_ms = []
    evals = []
    for k in range(args.steps):
        flush.zero_()                        # evict L2 between timed steps
        ev[k][0].record(stream)
        plan.run(stream)
        ev[k][1].record(stream)
        res = plan.results()
        evals.append(sum(r.n_evals for r in res))
        n_launch, lms = plan.stats()
        level_ms.append(lms)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_local = float(np.sum(step_ms)) / 1e3
    t = torch.tensor([t_local], dtype=torch.float64, device=dev)
    e = torch.tensor([float(np.sum(evals))], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(e, op=dist.ReduceOp.SUM)
    t_max, e_tot = float(t.item()), float(e.item())
    value = e_tot / t_max

    # end to end through the public API: host arrays in, results out
    res_bytes = 216 * len(problems)
    h2d = sum(3 * 8 * len(sm.T) + 8 * 20 + 40 for sm in smiles)
    sg.calibrate_batch(problems)
    torch.cuda.synchronize()
    e2e_t, e2e_ev = 0.0, 0
    for _ in range(max(1, min(args.steps, 3))):
        t0 = time.perf_counter()
        out = sg.calibrate_batch(problems)
        e2e_t += time.perf_counter() - t0
        e2e_ev += sum(r.n_evals for r in out)
    e2e_value_local = e2e_ev / e2e_t
    ee = torch.tensor([e2e_value_local], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(ee, op=dist.ReduceOp.SUM)

    # roofline of the dominant kernel: the SA level kernel (FP32 Hagan)
    lvl_ms = float(np.mean(level_ms))
    quote_evals_per_launch = (float(np.mean(evals)) / N_LEVELS) * 21
    achieved = quote_evals_per_launch / (lvl_ms / 1e3) / 1e9
    sm_mhz = clocks.get("sm_mhz") or 1920.0
    if rates:
        sfu_rate = min(rates[1], rates[3], rates[4])   # ex2/rsqrt/rcp ops per SM clock
        fp32_rate = rates[0]
        peak_sfu = SMS * sfu_rate * sm_mhz * 1e6 / SFU_PER_QUOTE / 1e9
        peak_fp32 = SMS * fp32_rate * sm_mhz * 1e6 / FP32_PER_QUOTE / 1e9
        peak = min(peak_sfu, peak_fp32)
        peak_note = "measured pipe rates (sabr_probe_pipe_rates) x 152 SMs x median SM clock"
    else:
        peak = SMS * 16 * sm_mhz * 1e6 / SFU_PER_QUOTE / 1e9
        peak_note = "nominal 16 SFU ops/clk/SM x 152 SMs x median SM clock"
    roofline = {"bound": "alu", "kernel": "sa_level_kernel<float,HAGAN>", "achieved": achieved, "peak": peak,
                "unit": "Gquote-eval/s", "frac": achieved / peak, "traffic": None,
                "launch_ms": lvl_ms, "quote_evals_per_launch": quote_evals_per_launch, "peak_from": peak_note,
                "pipe_rates_per_sm_clk": rates}

    line = {"metric": "SABR SA cost evals/s (static Hagan surface, 10x21, FP32 bulk)", "value": value,
            "unit": "cost-evals/s", "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "static Hagan surface: 10 maturities x 21 strikes (each its own smile), "
                                   "4096 SA chains/smile, 200 levels x 100 proposals, cooling 0.95",
                       "l2": "flushed (256 MB write) between timed steps", "precision": "FP32 bulk, FP64 sums"},
            "clocks": clocks, "gpu_launches": int(n_launch * args.steps),
            "e2e": {"value": float(ee.item()), "unit": "cost-evals/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": res_bytes},
            "roofline": roofline}

    if not args.no_fp64:
        p64 = sg.Plan(surface_problems(smiles, market, sg.FP64, seed0=7 + 100 * rank), use_graph=True)
        p64.run(stream)
        p64.results()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        a.record(stream)
        p64.run(stream)
        b.record(stream)
        r64 = p64.results()
        torch.cuda.synchronize()
        ms64 = a.elapsed_time(b)
        line["fp64_form"] = {"value": sum(r.n_evals for r in r64) / (ms64 / 1e3), "unit": "cost-evals/s",
                             "ms_per_step": ms64}
        p64.close()

    res = plan.results()
    errs = [abs(r.misfit - r.misfit_fp64) / max(r.misfit_fp64, 1e-300) for r in res]
    line["fp32_vs_fp64_misfit_rel_err_max"] = float(np.max(errs))
    plan.close()

    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(smiles, market)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
