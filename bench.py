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
METRIC = "SABR SA cost evals/s (static Hagan surface, 10x21, FP32 bulk)"
WORKLOAD = ("static Hagan surface: 10 maturities x 21 strikes (each its own smile), 4096 SA chains/smile, "
            "200 levels x 100 proposals, cooling 0.95")
# Algorithmic work of one Hagan quote evaluation (eq. haganf + the misfit
# term), by pipe: (K f)^((1-beta)/2) (one exp2 of a precomputed log; the
# formula's other powers of K f are its square and cube), one square root,
# one logarithm, two divisions (t = z/(1 + D) of z/x(z), and the formula's
# quotient), and about 30 FP32 adds/multiplies.
HAGAN_QUOTE_OPS = {"ex2": 1, "rsq": 1, "lg2": 1, "rcp": 2, "fp32": 30}
# One log-Euler path-step: Box-Muller (log, sqrt, sin, cos), the exp of
# nu-hat, ~12 FP32 operations, and half a Philox4x32-10 block (ten rounds of
# two 32x32 multiplies, each a low and a high half: 20 integer multiplies).
MC_STEP_OPS = {"lg2": 1, "rsq": 1, "sin": 2, "ex2": 1, "fp32": 12, "imad": 20}
# Algorithmic work of one dynamic-model proposal on the 12 x 21 joint
# surface.  Case I: per maturity the Case I functions (four short series of
# about 20 FMAs each, or their closed forms) and the polynomial of eq.
# (vola_SABRd) -- about 120 FP32 operations, one exp2 and a few
# reciprocals -- and per quote 4 FP32 (polynomial and misfit term).  Case
# II: per node of the shared rule (96 nodes) two exp2 and about 30 FP32
# operations; per maturity a recurrence step and the polynomial (about 41
# FP32, one exp2, five reciprocals); per quote 4 FP32.
DYN_PROPOSAL_OPS = {
    1: {"ex2": 12, "rcp": 60, "fp32": 12 * 120 + 252 * 4},
    2: {"ex2": 96 * 2 + 12, "rcp": 60, "fp32": 96 * 30 + 12 * 41 + 252 * 4},
}
SMS = 152


LEVEL_KERNEL_SOURCES = ["sa.cu", "engine.cuh", "sabr_math.cuh"]
LEVEL_PROFILE = "sa_queue_kernel_hagan_static_surface.md"


def _current_profile(profile, sources):
    """Text of a committed ncu summary under profiles/, or None when the
    kernel's sources have changed since that capture (the summary records
    their SHA-256)."""
    import hashlib
    import re
    try:
        text = open(os.path.join(ROOT, "profiles", profile)).read()
    except OSError:
        return None
    h = re.search(r"^source_sha256[^:]*: ([0-9a-f]{64})", text, re.M)
    if not h:
        return None
    d = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, "paper_2407_20713_gb300", "csrc", f), "rb") as fh:
            d.update(fh.read())
    return text if d.hexdigest() == h.group(1) else None


def _scale(text, units):
    """Factor from a capture's launch to a launch of `units` units: a summary
    that records `units_per_launch` (a capture of a shorter run of the same
    kernel) scales by units / units_per_launch, otherwise 1."""
    import re
    u = re.search(r"^units_per_launch: ([0-9.e+]+)", text, re.M)
    return units / float(u.group(1)) if (u and units) else 1.0


def profiled_traffic(profile, sources, units=None):
    """DRAM bytes (read + write) per launch from a committed ncu summary
    (scaled to a launch of `units` units when the capture records its own),
    or None when the kernel has changed since the capture."""
    import re
    text = _current_profile(profile, sources)
    t = re.search(r"^traffic_bytes_per_launch: (\d+)", text, re.M) if text else None
    return int(int(t.group(1)) * _scale(text, units)) if t else None


def profiled_thread_instructions(profile, sources, units=None):
    """Thread instructions per launch (warp instructions x active lanes per
    warp instruction) from a committed ncu summary (scaled like
    profiled_traffic), or None when the kernel has changed since the
    capture."""
    import re
    text = _current_profile(profile, sources)
    if not text:
        return None
    w = re.search(r"`smsp__inst_executed\.sum`\) \| ([0-9.]+)", text)
    lanes = re.search(r"`smsp__thread_inst_executed_per_inst_executed\.ratio`\) \| ([0-9.]+)", text)
    return float(w.group(1)) * float(lanes.group(1)) * _scale(text, units) if w and lanes else None


def issue_bound(thread_instr_per_unit, sm_mhz):
    """Units per second if every issue slot of the GPU (4 schedulers x 32
    lanes per SM clock) carried one of the unit's instructions."""
    return SMS * 4 * 32 * sm_mhz * 1e6 / thread_instr_per_unit


def pipe_bound(ops, rates, sm_mhz):
    """Units per second allowed by the busiest pipe: rates are operations per
    SM clock (sabr_probe_pipe_rates: fma, ex2, lg2, rsq, rcp, sin, imad, dfma)."""
    r = {"fp32": rates[0], "ex2": rates[1], "lg2": rates[2], "rsq": rates[3], "rcp": rates[4], "sin": rates[5],
         "imad": rates[6]}
    sfu = sum(n / r[k] for k, n in ops.items() if k in ("ex2", "lg2", "rsq", "rcp", "sin"))
    t = {"sfu": sfu, "fp32": ops.get("fp32", 0) / r["fp32"], "int": ops.get("imad", 0) / r["imad"]}
    pipe = max(t, key=t.get)
    return SMS * sm_mhz * 1e6 / t[pipe], pipe, t


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 form")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-extra", action="store_true", help="skip the MC, dynamic and serving measurements")
    ap.add_argument("--levels", type=int, default=None,
                    help="temperature levels of the headline surface (default 200; fewer for a short ncu capture)")
    ap.add_argument("--case", choices=["full", "small", "mc", "cliquet", "dynamic1", "dynamic2", "single"],
                    default="full",
                    help="small: 2 smiles x 10 levels, main measurement only; mc: one 2^20-path MC pricing "
                         "of the MC surface; cliquet: one 2^20-path cliquet; dynamic1 / dynamic2: two runs of "
                         "three levels of the joint Case I / Case II fit; single: two FP32 calibrations of the "
                         "one-smile configuration (the last six for profiler captures)")
    ap.add_argument("--serve-requests", type=int, default=400)
    ap.add_argument("--serve-loads", type=float, nargs="*", default=[0.5, 0.8, 0.95],
                    help="fractions of capacity for --serve-only (each with --serve-requests requests)")
    ap.add_argument("--serve-capacity", type=float, default=None,
                    help="for --serve-only: the capacity (calibrations/s) the loads are fractions of, from an "
                         "earlier run at the same request count, instead of measuring it again")
    ap.add_argument("--serve-only", action="store_true",
                    help="only the serving measurement (capacity and loads) at --serve-requests requests")
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


def cpu_baseline(smiles, market, n_levels=N_LEVELS):
    """The FP64 oracle, as it stands, on a bounded sample: smile 0 of the
    surface, all 4096 chains, n_levels of the 200 levels (x 100 proposals);
    by default one whole smile calibration (several seconds on 16 cores)."""
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


def cpu_baseline_single_smile():
    """The oracle (FP64, all host cores) on one whole cfg 1 calibration: one
    Hagan smile, 15 strikes, 64 chains, 200 levels x 100 proposals."""
    import oracle as O
    from paper_2407_20713_gb300 import workloads
    w = workloads.one_smile()
    mkt = O.implied_vol(O.HAGAN, w.truth, 1.0, w.T, w.K) + w.noise
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    o = O.sa_calibrate(O.HAGAN, 1.0, w.T, w.K, mkt, w.lo, w.hi, n_chains=w.n_chains, factor=FACTOR,
                       n_levels=N_LEVELS, chain_len=CHAIN_LEN, seed=1, n_threads=cores)
    dt = time.perf_counter() - t0
    return {"ms_per_calibration": 1e3 * dt, "cores": cores, "misfit": o["misfit"],
            "workload": "one Hagan smile, T = 1, 15 strikes, 64 chains, 200 levels x 100 proposals"}


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
        cb = cpu_baseline(smiles, market, n_levels=40)
        dts.append(time.perf_counter() - t0)
        vals.append(cb["value"])
    value = float(np.mean(vals))
    cb["value"] = value
    cb["sample"] = "each step: smile 1 of 10, %d chains, 40 of %d levels x %d proposals" % (N_CHAINS, N_LEVELS,
                                                                                            CHAIN_LEN)
    line = {"impl": "reference", "metric": METRIC,
            "value": value, "unit": "cost-evals/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(dts)), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sampled": "each step: smile 1 of 10, 40 of the 200 levels"},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "cost-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)



def grid_steps(maturities, spy):
    """Number of steps of the MC time grid (every multiple of 1/spy below the
    last maturity, with each maturity inserted)."""
    mats = sorted(set(float(t) for t in maturities))
    n, k = 0, 1
    for Tm in mats:
        while k / spy < Tm - 1e-10:
            n += 1
            k += 1
        n += 1
        if abs(k / spy - Tm) <= 1e-10:
            k += 1
    return n


def measure_mc(sg, torch, stream, rates, sm_mhz):
    """sabr_mc_price on the Monte Carlo surface shape: 8 maturities x 15
    strikes of calls, 2^22 paths, 250 steps a year (504 grid steps)."""
    from paper_2407_20713_gb300 import workloads
    w = workloads.mc_surface()
    n_paths = 1 << 22
    steps = grid_steps(w.T, 250.0)
    out = {}
    for prec, name in ((sg.FP32, "fp32"), (sg.FP64, "fp64")):
        sg.mc_price(sg.HAGAN, w.truth, 1.0, w.T, w.K, n_paths=1 << 16, steps_per_year=250, seed=1, prec=prec)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sg.mc_price(sg.HAGAN, w.truth, 1.0, w.T, w.K, n_paths=n_paths, steps_per_year=250, seed=1, prec=prec)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        out[name] = {"value": n_paths * steps / (ms / 1e3), "unit": "path-steps/s", "ms": ms}
    res = {"workload": "8 maturities x 15 strikes, 2^22 paths, %d steps, Hagan dynamics" % steps,
           "value": out["fp32"]["value"], "unit": "path-steps/s", "fp64_form": out["fp64"]}
    res["bessel"] = measure_mc_bessel(sg, torch, stream, w, n_paths)
    if rates:
        peak, pipe, _ = pipe_bound(MC_STEP_OPS, rates, sm_mhz)
        res["roofline"] = {"bound": "alu", "pipe": pipe, "ops_per_path_step": MC_STEP_OPS,
                           "achieved": res["value"], "peak": peak, "unit": "path-steps/s",
                           "frac": res["value"] / peak,
                           "traffic": profiled_traffic("mc_paths_kernel_mc_surface.md",
                                                       ["mc.cu", "mc.cuh", "sabr_math.cuh"]),
                           "traffic_note": "DRAM bytes per launch from the 2^20-path capture: the tables, "
                                           "independent of the path count"}
        ti = profiled_thread_instructions("mc_paths_kernel_mc_surface.md", ["mc.cu", "mc.cuh", "sabr_math.cuh"])
        if ti:
            per_unit = ti / ((1 << 20) * steps)   # the capture prices 2^20 paths on the same grid
            ib = issue_bound(per_unit, sm_mhz)
            res["roofline"]["issue_bound"] = {"thread_instructions_per_unit": per_unit, "peak": ib,
                                              "frac": res["value"] / ib,
                                              "from": "ncu warp instructions x active lanes of the committed "
                                                      "2^20-path capture"}
    return res


def measure_mc_bessel(sg, torch, stream, w, n_paths):
    """The conditional-Bessel scheme (sabr_mc_price_scheme, SABR_MC_BESSEL)
    on the same surface and paths, FP32: its path-step rate on the 250 steps
    a year grid, and, against a log-Euler reference at 2000 steps a year, the
    largest price bias of the Bessel scheme at 12 steps a year and of
    log-Euler at 250 with the time each takes (independent streams; the
    bias figures carry the reference's own noise, `reference_se_max`)."""
    def timed(spy, scheme, seed):
        sg.mc_price(sg.HAGAN, w.truth, 1.0, w.T, w.K, n_paths=1 << 16, steps_per_year=spy, seed=seed, scheme=scheme)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pr, se = sg.mc_price(sg.HAGAN, w.truth, 1.0, w.T, w.K, n_paths=n_paths, steps_per_year=spy, seed=seed,
                             scheme=scheme)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b), pr.cpu().numpy(), se.cpu().numpy()
    steps = grid_steps(w.T, 250.0)
    ms250, _, _ = timed(250, sg.MC_BESSEL, 1)
    _, ref, rse = timed(2000, None, 4)
    ms12, p12, s12 = timed(12, sg.MC_BESSEL, 2)
    msle, ple, sle = timed(250, None, 3)
    return {"value": n_paths * steps / (ms250 / 1e3), "unit": "path-steps/s", "ms": ms250,
            "workload": "the same surface and paths, %d steps (250 a year), FP32" % steps,
            "equal_accuracy": {
                "reference": "log-Euler at 2000 steps a year (%d steps)" % grid_steps(w.T, 2000.0),
                "reference_se_max": float(np.max(rse)),
                "bessel_12_per_year": {"steps": grid_steps(w.T, 12.0), "ms": ms12,
                                       "max_abs_bias": float(np.max(np.abs(p12 - ref))),
                                       "se_max": float(np.max(s12))},
                "log_euler_250_per_year": {"steps": steps, "ms": msle,
                                           "max_abs_bias": float(np.max(np.abs(ple - ref))),
                                           "se_max": float(np.max(sle))},
                "speedup": msle / ms12}}


def measure_cliquet(sg, torch, stream, rates, sm_mhz):
    """sabr_mc_cliquet on the Sec. 6.3 contract (one year, 4 resets, local
    limits -2%/+2%, global floor 0 and cap 0.2), 2^20 paths, 250 steps a
    year, DSabr_I dynamics with synthetic EUR/USD-like parameters."""
    n_paths, spy = 1 << 20, 250.0
    p = [0.11, 0.75, -0.25, 0.6, 0.9, 1.4]
    steps = grid_steps(np.array([0.25, 0.5, 0.75, 1.0]), spy)
    out = {}
    for prec, name in ((sg.FP32, "fp32"), (sg.FP64, "fp64")):
        sg.mc_cliquet(sg.DYN_I, p, 1.0, 1.0, 4, -0.02, 0.02, 0.0, 0.2, n_paths=1 << 14, steps_per_year=spy,
                      prec=prec)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pr, se = sg.mc_cliquet(sg.DYN_I, p, 1.0, 1.0, 4, -0.02, 0.02, 0.0, 0.2, n_paths=n_paths,
                               steps_per_year=spy, seed=11, prec=prec)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        out[name] = {"ms": ms, "value": n_paths * steps / (ms / 1e3), "unit": "path-steps/s",
                     "price": float(pr.item()), "stderr": float(se.item())}
    res = {"workload": "cliquet T=1y, 4 resets, 2^20 paths, %d steps, DSabr_I" % steps,
           "value": out["fp32"]["value"], "unit": "path-steps/s", "ms": out["fp32"]["ms"], "fp64_form": out["fp64"],
           "price": out["fp32"]["price"]}
    if rates:
        peak, pipe, _ = pipe_bound(MC_STEP_OPS, rates, sm_mhz)
        res["roofline"] = {"bound": "alu", "pipe": pipe, "ops_per_path_step": MC_STEP_OPS,
                           "achieved": res["value"], "peak": peak, "unit": "path-steps/s",
                           "frac": res["value"] / peak,
                           "traffic": profiled_traffic("cliquet_kernel_dsabr1_2p20.md",
                                                       ["cliquet.cu", "mc.cuh", "sabr_math.cuh"])}
        ti = profiled_thread_instructions("cliquet_kernel_dsabr1_2p20.md", ["cliquet.cu", "mc.cuh", "sabr_math.cuh"])
        if ti:
            per_unit = ti / (n_paths * steps)   # the capture is this workload
            ib = issue_bound(per_unit, sm_mhz)
            res["roofline"]["issue_bound"] = {"thread_instructions_per_unit": per_unit, "peak": ib,
                                              "frac": res["value"] / ib,
                                              "from": "ncu warp instructions x active lanes of the committed "
                                                      "capture (the cliquet kernel alone; the value includes "
                                                      "the call's table upload and reduction)"}
    return res


def measure_single_smile(sg, torch, stream):
    """cfg 1: one Hagan smile (T = 1, 15 strikes), 64 chains, 200 levels x 100
    proposals: the time of one whole calibration in FP64 and in FP32 on the
    GPU (the oracle's time on it is part of the CPU baseline)."""
    from paper_2407_20713_gb300 import workloads
    w = workloads.one_smile()
    mkt = sg.implied_vol(sg.HAGAN, w.truth, 1.0, w.T, w.K, prec=sg.FP64).cpu().numpy() + w.noise
    out = {}
    for prec, name in ((sg.FP64, "fp64"), (sg.FP32, "fp32")):
        pb = sg.CalibrationProblem(model=sg.HAGAN, T=w.T, K=w.K, market=mkt, lo=w.lo, hi=w.hi, prec=prec,
                                   n_chains=w.n_chains, n_levels=N_LEVELS, chain_len=CHAIN_LEN, factor=FACTOR,
                                   seed=1)
        plan = sg.Plan([pb], use_graph=True)
        for _ in range(3):
            plan.run(stream)
            plan.results()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.run(stream)
        b.record(stream)
        r = plan.results()[0]
        ms = a.elapsed_time(b)
        plan.close()
        out[name] = {"ms_per_calibration": ms, "cost_evals_per_s": r.n_evals / (ms / 1e3),
                     "misfit_fp64": r.misfit_fp64}
    out["workload"] = "one Hagan smile, T = 1, 15 strikes, 64 chains, 200 levels x 100 proposals"
    return out


def _case2_ok(x, tmax, n=2001):
    """rho(t) in [-1, 1] and nu(t) > 0 on [0, tmax] for Case II parameters
    (dense grid; host-side check of a synthetic truth)."""
    t = np.linspace(0.0, tmax, n)
    rho = (x[2] + x[8] * t) * np.exp(-x[4] * t) + x[6]
    nu = (x[3] + x[9] * t) * np.exp(-x[5] * t) + x[7]
    return bool(np.all(np.abs(rho) <= 0.999) and np.all(nu > 1e-3))


def measure_mc_calibration(sg, torch, stream, rates, sm_mhz):
    """Technique II (SA with the Monte Carlo price misfit) on the MC surface:
    8 maturities x 15 calls, 256 chains, 2^16 paths x 250 steps a year per
    cost evaluation (504 grid steps), FP32 paths.  Static Hagan (cfg 4): a
    sample of 20 levels x 10 proposals of the 200 x 100 schedule in FP32,
    1 level x 2 proposals in FP64.  DSabr_II (the paper's Technique II
    model): 2 levels x 5 proposals in FP32."""
    from paper_2407_20713_gb300 import workloads
    w = workloads.mc_surface()
    m = w.meta
    steps = grid_steps(w.T, m["steps_per_year"])
    dyn = workloads.dynamic_surface(case=2, feasible=lambda x: _case2_ok(x, float(w.T.max())))

    def run(model, truth, lo, hi, prec, levels, clen):
        mkt = sg.mc_price(model, truth, 1.0, w.T, w.K, n_paths=m["market_paths"], steps_per_year=250,
                          seed=m["market_seed"])[0].cpu().numpy()
        keep = mkt >= 1e-6  # quotes priced below 1e-6 f are left out
        pb = sg.CalibrationProblem(model=model, T=w.T[keep], K=w.K[keep], market=mkt[keep], lo=lo, hi=hi,
                                   prec=prec, cost=sg.COST_MC_PRICE, n_chains=w.n_chains, n_levels=levels,
                                   chain_len=clen, mc_paths=m["cal_paths"], mc_steps_per_year=m["steps_per_year"],
                                   mc_seed=m["cal_seed"], seed=5)
        plan = sg.Plan([pb], use_graph=True)
        plan.run(stream)
        plan.results()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.run(stream)
        b.record(stream)
        r = plan.results()[0]
        ms = a.elapsed_time(b)
        plan.close()
        evals = r.n_evals + 1  # the init evaluation of x0 is one more MC pricing
        return {"value": evals / (ms / 1e3), "unit": "cost-evals/s", "ms": ms, "levels": levels,
                "chain_len": clen, "quotes": int(keep.sum()),
                "path_steps_per_s": evals * m["cal_paths"] * steps / (ms / 1e3)}

    hag32 = run(sg.HAGAN, w.truth, w.lo, w.hi, sg.FP32, 20, 10)
    hag64 = run(sg.HAGAN, w.truth, w.lo, w.hi, sg.FP64, 1, 2)
    dyn32 = run(sg.DYN_II, dyn.truth, dyn.lo, dyn.hi, sg.FP32, 2, 5)
    res = {"workload": "Technique II, static Hagan, 8 x 15 calls, 256 chains, 2^16 paths x %d steps per cost "
                       "evaluation" % steps,
           "value": hag32["value"], "unit": "cost-evals/s", "path_steps_per_s": hag32["path_steps_per_s"],
           "ms": hag32["ms"], "sample": "20 of 200 levels x 10 of 100 proposals (FP32); 1 level x 2 proposals "
                                       "(FP64)",
           "fp64_form": hag64, "dsabr2_fp32": dict(dyn32, sample="2 levels x 5 proposals")}
    if rates:
        peak, pipe, _ = pipe_bound(MC_STEP_OPS, rates, sm_mhz)
        res["roofline"] = {"bound": "alu", "pipe": pipe, "unit": "path-steps/s", "peak": peak,
                           "achieved": res["path_steps_per_s"], "frac": res["path_steps_per_s"] / peak}
    return res


def measure_dynamic(sg, torch, stream, levels=N_LEVELS, rates=None, sm_mhz=None):
    """Joint dynamic fits on 12 maturities x 21 strikes, 8192 chains each, one
    Case I and one Case II surface, FP32; `levels` of the 200 levels."""
    from paper_2407_20713_gb300 import workloads
    res = {}
    for case, model in ((1, sg.DYN_I), (2, sg.DYN_II)):
        w = workloads.dynamic_surface(case=case, feasible=lambda x: _case2_ok(x, float(workloads.DYN_MATURITIES[-1])))
        mkt = sg.implied_vol(model, w.truth, 1.0, w.T, w.K, prec=sg.FP64).cpu().numpy() + w.noise
        pb = sg.CalibrationProblem(model=model, T=w.T, K=w.K, market=mkt, lo=w.lo, hi=w.hi, prec=sg.FP32,
                                   n_chains=w.n_chains, n_levels=levels, chain_len=CHAIN_LEN, seed=3)
        plan = sg.Plan([pb], use_graph=True)
        plan.run(stream)
        plan.results()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.run(stream)
        b.record(stream)
        r = plan.results()[0]
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        res["case%d" % case] = {"value": r.n_evals / (ms / 1e3), "unit": "cost-evals/s", "ms": ms,
                                "levels": levels, "quote_evals_per_s": r.n_evals * 252 / (ms / 1e3)}
        if rates and sm_mhz:
            peak, pipe, _ = pipe_bound(DYN_PROPOSAL_OPS[case], rates, sm_mhz)
            res["case%d" % case]["roofline"] = {
                "bound": "alu", "pipe": pipe, "unit": "cost-evals/s", "peak": peak,
                "achieved": r.n_evals / (ms / 1e3), "frac": r.n_evals / (ms / 1e3) / peak,
                "ops_per_proposal": DYN_PROPOSAL_OPS[case]}
            # the ceiling the kernel meets: issue slots, at the instructions
            # per proposal drawn (out-of-box and infeasible ones included)
            # of the committed one-level capture of the same surface
            ti = profiled_thread_instructions("sa_level_kernel_dyn%d_joint_surface.md" % case, LEVEL_KERNEL_SOURCES)
            if ti:
                per_unit = ti / (w.n_chains * CHAIN_LEN)
                ib = issue_bound(per_unit, sm_mhz)
                drawn = w.n_chains * CHAIN_LEN * levels / (ms / 1e3)
                res["case%d" % case]["roofline"]["issue_bound"] = {
                    "unit": "proposals drawn/s", "thread_instructions_per_unit": per_unit, "peak": ib,
                    "achieved": drawn, "frac": drawn / ib,
                    "from": "ncu warp instructions x active lanes of the committed one-level capture"}
        plan.close()
    return res


def measure_serving(sg, n_requests, rate_hz, formula_only=False):
    """Poisson stream of calibration requests of uneven size (1-12 maturities x
    5-41 strikes; 80% Hagan / 20% dynamic, 5% MC) through the server; with
    formula_only the MC requests of the stream are left out."""
    import threading
    from paper_2407_20713_gb300 import workloads
    reqs = workloads.serving_stream(n=n_requests, rate_hz=rate_hz)
    if formula_only:
        reqs = [q for q in reqs if q.cost == 0]
    probs = []
    for q in reqs:
        sm = q.smile
        if q.cost == 0:
            mkt = sg.implied_vol(sm.model, sm.truth, 1.0, sm.T, sm.K, prec=sg.FP64).cpu().numpy() + sm.noise
            # the asymptotic formulas can give a non-positive vol at extreme
            # synthetic truths (one Case II request of the 10 000-request
            # stream, 3 of its 55 quotes): such quotes are left out, as a
            # market would not quote them
            keep = np.isfinite(mkt) & (mkt > 0.0)
        else:
            mkt = sg.mc_price(sm.model, sm.truth, 1.0, sm.T, sm.K, n_paths=q.mc_paths, steps_per_year=250,
                              seed=99)[0].cpu().numpy()
            # quotes priced below 1e-6 f are left out of a price calibration
            keep = mkt >= 1e-6
        sm.T, sm.K, mkt = sm.T[keep], sm.K[keep], mkt[keep]
        probs.append(sg.CalibrationProblem(model=sm.model, T=sm.T, K=sm.K, market=mkt, lo=sm.lo, hi=sm.hi,
                                           cost=q.cost, prec=sg.FP32, n_chains=sm.n_chains, n_levels=q.n_levels,
                                           chain_len=q.chain_len, mc_paths=max(q.mc_paths, 2),
                                           mc_steps_per_year=250.0, mc_seed=7, seed=11))
    srv = sg.Server(device_bytes=8 << 30, max_active=512, max_quotes=512)
    arrive, done, tickets = {}, {}, {}
    lock = threading.Lock()
    t0 = time.perf_counter()

    errors = []

    def submitter():
        try:
            for i, q in enumerate(reqs):
                now = time.perf_counter() - t0
                if q.arrival > now:
                    time.sleep(q.arrival - now)
                a = time.perf_counter()
                t = srv.submit(probs[i])
                with lock:
                    arrive[i] = a
                    tickets[i] = t
        except Exception as exc:  # surfaced below instead of stalling the poll loop
            errors.append(exc)

    th = threading.Thread(target=submitter)
    th.start()
    deadline = time.perf_counter() + 600.0 + 0.5 * len(reqs)
    while len(done) < len(reqs) and time.perf_counter() < deadline and not errors:
        with lock:
            outstanding = [(i, t) for i, t in tickets.items() if i not in done]
        for i, t in outstanding:
            if srv.poll(t) is not None:
                done[i] = time.perf_counter()
        time.sleep(0.0005)
    th.join()
    if errors:
        srv.close()
        raise errors[0]
    lat = np.array([done[i] - arrive[i] for i in done])
    wall = max(done.values()) - t0
    st = srv.stats()
    srv.close()
    out = {"requests": len(reqs), "completed": len(done), "offered_rate_hz": rate_hz,
           "calibrations_per_s": len(done) / wall,
           "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
           "steps": st["steps"], "kernel_launches": st["kernel_launches"], "wall_s": wall}
    # latency per request class
    by = {}
    for i in done:
        by.setdefault(request_class(sg, reqs[i]), []).append(done[i] - arrive[i])
    out["by_class"] = {c: {"requests": len(v), "p50_ms": 1e3 * float(np.percentile(v, 50)),
                           "p99_ms": 1e3 * float(np.percentile(v, 99))} for c, v in sorted(by.items())}
    return out


def request_class(sg, q):
    """hagan / dynamic (formula cost, Case I or II) / mc (price cost)."""
    if q.cost != 0:
        return "mc"
    return "hagan" if q.smile.model == sg.HAGAN else "dynamic"


def measure_fp64_one_per_launch(sg, n_per_class=6):
    """The plain FP64 form, one request per launch (sabr_calibrate), on
    requests of each class drawn from the serving stream; its capacity on the
    stream's mix is 1 / sum_c p_c t_c (p_c the class fractions of the
    stream, t_c the mean time of one request).  An MC request runs 1 level x
    2 proposals and its time is scaled to its 10 x 10 schedule (FP64 paths
    take about a minute for a whole MC request)."""
    from paper_2407_20713_gb300 import workloads
    stream = workloads.serving_stream(n=2000, rate_hz=1.0)
    frac = {}
    for q in stream:
        c = request_class(sg, q)
        frac[c] = frac.get(c, 0) + 1.0 / len(stream)
    times = {}
    for c in ("hagan", "dynamic", "mc"):
        ts = []
        for q in [q for q in stream if request_class(sg, q) == c][:n_per_class]:
            sm = q.smile
            if q.cost == 0:
                mkt = sg.implied_vol(sm.model, sm.truth, 1.0, sm.T, sm.K, prec=sg.FP64).cpu().numpy() + sm.noise
                pb = sg.CalibrationProblem(model=sm.model, T=sm.T, K=sm.K, market=mkt, lo=sm.lo, hi=sm.hi,
                                           prec=sg.FP64, n_chains=sm.n_chains, n_levels=q.n_levels,
                                           chain_len=q.chain_len, seed=11)
                scale = 1.0
            else:
                mkt = sg.mc_price(sm.model, sm.truth, 1.0, sm.T, sm.K, n_paths=q.mc_paths, steps_per_year=250,
                                  seed=99)[0].cpu().numpy()
                keep = mkt >= 1e-6
                pb = sg.CalibrationProblem(model=sm.model, T=sm.T[keep], K=sm.K[keep], market=mkt[keep], lo=sm.lo,
                                           hi=sm.hi, cost=sg.COST_MC_PRICE, prec=sg.FP64, n_chains=sm.n_chains,
                                           n_levels=1, chain_len=2, mc_paths=q.mc_paths, mc_steps_per_year=250.0,
                                           mc_seed=7, seed=11)
                scale = (q.n_levels * q.chain_len) / 2.0
            t0 = time.perf_counter()
            sg.calibrate(pb)
            ts.append((time.perf_counter() - t0) * scale)
        times[c] = float(np.mean(ts))
    cap = 1.0 / sum(frac[c] * times[c] for c in times)
    return {"calibrations_per_s": cap, "seconds_per_request": times, "class_fractions": frac,
            "sample": "%d requests per class from the serving stream; MC scaled from 1 level x 2 proposals"
                      % n_per_class}

def measure_serving_loads(sg, n_requests, fractions=(0.5, 0.8, 0.95), load_requests=None, capacity=None):
    """Capacity (all requests at once; or `capacity` from an earlier run),
    then Poisson arrivals at the given fractions of it (half the requests
    each unless load_requests is given); beside it the plain FP64
    one-request-per-launch form on the same mix."""
    burst = measure_serving(sg, n_requests, rate_hz=1e9) if capacity is None else {
        "calibrations_per_s": capacity, "given": "from an earlier run at %d requests" % n_requests}
    cap = burst["calibrations_per_s"]
    n_load = load_requests or max(1, n_requests // 2)
    loads = {"load%d" % int(100 * f): measure_serving(sg, n_load, rate_hz=f * cap) for f in fractions}
    out = {"capacity": burst}
    out.update(loads)
    # the 5% MC requests take most of the GPU time of the mix; the formula
    # requests alone, all at once
    out["formula_only_capacity"] = measure_serving(sg, n_requests, rate_hz=1e9, formula_only=True)
    out["fp64_one_request_per_launch"] = measure_fp64_one_per_launch(sg)
    return out


def run_mc_case():
    """sabr_mc_price on the MC surface shape at 2^20 paths (profiling):
    log-Euler FP32 twice, FP64, then the conditional-Bessel scheme FP32."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2407_20713_gb300 as sg
    from paper_2407_20713_gb300 import workloads
    w = workloads.mc_surface()
    for prec in (sg.FP32, sg.FP32, sg.FP64):
        sg.mc_price(sg.HAGAN, w.truth, 1.0, w.T, w.K, n_paths=1 << 20, steps_per_year=250, seed=1, prec=prec)
    sg.mc_price(sg.HAGAN, w.truth, 1.0, w.T, w.K, n_paths=1 << 20, steps_per_year=250, seed=1, scheme=sg.MC_BESSEL)
    torch.cuda.synchronize()
    print(json.dumps({"case": "mc", "ok": True}))


def run_dynamic_case(case):
    """Three levels of the joint Case I or Case II fit (12 maturities x 21
    strikes, 8192 chains, FP32) as one plan, run twice (profiling)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2407_20713_gb300 as sg
    from paper_2407_20713_gb300 import workloads
    model = sg.DYN_I if case == 1 else sg.DYN_II
    w = workloads.dynamic_surface(case=case, feasible=lambda x: _case2_ok(x, float(workloads.DYN_MATURITIES[-1])))
    mkt = sg.implied_vol(model, w.truth, 1.0, w.T, w.K, prec=sg.FP64).cpu().numpy() + w.noise
    pb = sg.CalibrationProblem(model=model, T=w.T, K=w.K, market=mkt, lo=w.lo, hi=w.hi, prec=sg.FP32,
                               n_chains=w.n_chains, n_levels=3, chain_len=CHAIN_LEN, seed=3)
    plan = sg.Plan([pb], use_graph=True)
    for _ in range(2):
        plan.run(torch.cuda.current_stream())
        plan.results()
    plan.close()
    torch.cuda.synchronize()
    print(json.dumps({"case": "dynamic%d" % case, "ok": True}))


def run_single_case():
    """Two FP32 calibrations of one Hagan smile (15 strikes, 64 chains,
    200 levels x 100 proposals) as one plan (profiling)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2407_20713_gb300 as sg
    from paper_2407_20713_gb300 import workloads
    w = workloads.one_smile()
    mkt = sg.implied_vol(sg.HAGAN, w.truth, 1.0, w.T, w.K, prec=sg.FP64).cpu().numpy() + w.noise
    pb = sg.CalibrationProblem(model=sg.HAGAN, T=w.T, K=w.K, market=mkt, lo=w.lo, hi=w.hi, prec=sg.FP32,
                               n_chains=w.n_chains, n_levels=N_LEVELS, chain_len=CHAIN_LEN, factor=FACTOR, seed=1)
    plan = sg.Plan([pb], use_graph=True)
    for _ in range(2):
        plan.run(torch.cuda.current_stream())
        plan.results()
    n_launch, _ = plan.stats()
    plan.close()
    torch.cuda.synchronize()
    print(json.dumps({"case": "single", "ok": True, "launches_per_run": n_launch}))


def run_cliquet_case():
    """One sabr_mc_cliquet of the Sec. 6.3 contract at 2^20 paths (profiling)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2407_20713_gb300 as sg
    p = [0.11, 0.75, -0.25, 0.6, 0.9, 1.4]
    for _ in range(2):
        sg.mc_cliquet(sg.DYN_I, p, 1.0, 1.0, 4, -0.02, 0.02, 0.0, 0.2, n_paths=1 << 20, steps_per_year=250)
    torch.cuda.synchronize()
    print(json.dumps({"case": "cliquet", "ok": True}))


def aggregate(t_local, units_local, e2e_local, dist=None):
    """Whole-job numbers across ranks: time = max over ranks (all ranks start
    together after a barrier), units and end-to-end rates summed."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device()) if torch.cuda.is_available() else torch.device("cpu")
    v = torch.tensor([t_local, units_local, e2e_local], dtype=torch.float64, device=dev)
    t = v[0:1].clone()
    rest = v[1:].clone()
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(rest, op=dist.ReduceOp.SUM)
    t_max, units, e2e = float(t.item()), float(rest[0].item()), float(rest[1].item())
    return {"time_s": t_max, "units": units, "value": units / t_max, "e2e": e2e}


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
    global N_LEVELS
    if args.case == "small":
        smiles = smiles[:2]
        N_LEVELS = 10
    if args.levels:
        N_LEVELS = args.levels
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
    agg = aggregate(t_local, float(np.sum(evals)), e2e_ev / e2e_t, dist)
    t_max, value = agg["time_s"], agg["value"]

    # roofline of the dominant kernel: the persistent SA launch that runs
    # every level of the surface from its ready queue (FP32 Hagan); its time
    # is read from the plan's events around that launch (and the queue
    # reset before it) on the bench's stream
    lvl_ms = float(np.mean(level_ms))
    launch_ms = lvl_ms * N_LEVELS
    quote_evals_per_launch = float(np.mean(evals)) * 21
    achieved = quote_evals_per_launch / (launch_ms / 1e3) / 1e9
    sm_mhz = clocks.get("sm_mhz") or 1920.0
    if rates:
        peak_units, pipe, _ = pipe_bound(HAGAN_QUOTE_OPS, rates, sm_mhz)
        peak = peak_units / 1e9
        peak_note = ("measured pipe rates (sabr_probe_pipe_rates) x 152 SMs x median SM clock; binding pipe: %s"
                     % pipe)
    else:
        peak = SMS * sm_mhz * 1e6 / (1 / 32 + 4 / 16) / 1e9
        peak_note = "nominal SFU rates (ex2 32, others 16 per SM clock) x 152 SMs x median SM clock"
    roofline = {"bound": "alu", "kernel": "sa_queue_kernel<float,HAGAN>", "achieved": achieved, "peak": peak,
                "unit": "Gquote-eval/s", "frac": achieved / peak,
                "traffic": profiled_traffic(LEVEL_PROFILE, LEVEL_KERNEL_SOURCES, quote_evals_per_launch),
                "launch_ms": launch_ms, "level_ms": lvl_ms, "quote_evals_per_launch": quote_evals_per_launch,
                "peak_from": peak_note, "pipe_rates_per_sm_clk": rates}
    ti = profiled_thread_instructions(LEVEL_PROFILE, LEVEL_KERNEL_SOURCES, quote_evals_per_launch)
    if ti:
        # the ceiling the kernel actually meets: issue slots, at the
        # instructions per quote evaluation of the committed capture
        per_unit = ti / quote_evals_per_launch
        ib = issue_bound(per_unit, sm_mhz) / 1e9
        roofline["issue_bound"] = {"thread_instructions_per_unit": per_unit, "peak": ib, "frac": achieved / ib,
                                   "from": "ncu warp instructions x active lanes of the committed capture"}

    line = {"metric": METRIC, "value": value,
            "unit": "cost-evals/s", "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD,
                       "l2": "flushed (256 MB write) between timed steps",
                       "precision": ("FP32 quote arithmetic, chain state and best point; misfit summed across "
                                     "lanes in double-float (FP32 pairs); FP64 re-score of the returned point")},
            "clocks": clocks, "gpu_launches": int(n_launch * args.steps),
            "e2e": {"value": agg["e2e"], "unit": "cost-evals/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": res_bytes},
            "roofline": roofline}

    if not args.no_fp64 and args.case == "full":
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

    if rank == 0 and not args.no_extra and args.case == "full":
        for key, fn in (("mc", lambda: measure_mc(sg, torch, stream, rates, sm_mhz)),
                        ("single_smile", lambda: measure_single_smile(sg, torch, stream)),
                        ("mc_calibration", lambda: measure_mc_calibration(sg, torch, stream, rates, sm_mhz)),
                        ("cliquet", lambda: measure_cliquet(sg, torch, stream, rates, sm_mhz)),
                        ("dynamic", lambda: measure_dynamic(sg, torch, stream, rates=rates, sm_mhz=sm_mhz)),
                        ("serving", lambda: measure_serving_loads(sg, args.serve_requests))):
            try:
                line[key] = fn()
            except Exception as exc:  # report, keep the headline line
                line[key] = {"error": repr(exc)}
    if rank == 0 and not args.no_cpu and args.case == "full":
        line["cpu_baseline"] = cpu_baseline(smiles, market)
        line["cpu_baseline"]["single_smile"] = cpu_baseline_single_smile()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_serving_only(args):
    """The serving measurement alone, e.g. at the stream's full 10 000
    requests (capacity, then 50 / 80 / 95% of it with half the requests
    each), printed as one JSON line."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2407_20713_gb300 as sg
    torch.cuda.set_device(0)
    out = measure_serving_loads(sg, args.serve_requests, fractions=tuple(args.serve_loads),
                                load_requests=args.serve_requests, capacity=args.serve_capacity)
    print(json.dumps({"serving": out, "requests": args.serve_requests}), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.serve_only:
        run_serving_only(a)
    elif a.case == "mc":
        run_mc_case()
    elif a.case == "cliquet":
        run_cliquet_case()
    elif a.case == "single":
        run_single_case()
    elif a.case in ("dynamic1", "dynamic2"):
        run_dynamic_case(int(a.case[-1]))
    else:
        run_ours(a)
