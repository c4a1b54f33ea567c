"""Python binding of libsabr: the same entry points as include/sabr.h.

Only argument marshalling happens here; every step of the path runs in the
library's CUDA kernels.  PyTorch provides device memory and streams.
"""
import ctypes
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import capi
from .capi import COST_MC_PRICE, COST_VOL, FP32, FP64  # noqa: F401


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _params10(params, model):
    p = np.zeros(10, dtype=np.float64)
    a = np.asarray(params, dtype=np.float64).ravel()
    n = capi.N_PARAMS[model]
    p[: min(n, a.size)] = a[:n]
    return p


def _dev64(x, device):
    if isinstance(x, torch.Tensor):
        t = x.to(device=device, dtype=torch.float64)
    else:
        t = torch.as_tensor(np.asarray(x, dtype=np.float64), device=device)
    return t.contiguous()


def implied_vol(model, params, fwd, T, K, prec=FP32, out=None, stream=None, device="cuda"):
    """Model implied vols of options (T[i], K[i]); returns a float64 CUDA tensor."""
    lib = capi.load()
    Tt = _dev64(T, device)
    Kt = _dev64(K, device).expand_as(Tt).contiguous() if _dev64(K, device).numel() == 1 else _dev64(K, device)
    if out is None:
        out = torch.empty_like(Tt)
    p = _params10(params, model)
    st = lib.sabr_implied_vol(model, p.ctypes.data_as(capi.PD), float(fwd), ctypes.c_void_p(Tt.data_ptr()),
                              ctypes.c_void_p(Kt.data_ptr()), Tt.numel(), ctypes.c_void_p(out.data_ptr()),
                              prec, _stream_handle(stream))
    capi.check(st, "sabr_implied_vol")
    return out


def mc_price(model, params, fwd, T, K, is_call=None, discount=None, n_paths=1 << 16,
             steps_per_year=250.0, seed=0, prec=FP32, stream=None, device="cuda", scheme=None):
    """Monte Carlo prices and standard errors (float64 CUDA tensors).
    scheme None: sabr_mc_price (log-Euler); capi.MC_LOG_EULER or
    capi.MC_BESSEL: sabr_mc_price_scheme."""
    lib = capi.load()
    T = np.ascontiguousarray(T, dtype=np.float64).ravel()
    K = np.ascontiguousarray(np.broadcast_to(np.asarray(K, dtype=np.float64), T.shape))
    ic = None if is_call is None else np.ascontiguousarray(is_call, dtype=np.int8).ravel()
    dc = None if discount is None else np.ascontiguousarray(discount, dtype=np.float64).ravel()
    price = torch.empty(T.size, dtype=torch.float64, device=device)
    se = torch.empty(T.size, dtype=torch.float64, device=device)
    p = _params10(params, model)
    head = (model, p.ctypes.data_as(capi.PD), float(fwd), T.ctypes.data_as(capi.PD), K.ctypes.data_as(capi.PD),
            ic.ctypes.data_as(capi.PI8) if ic is not None else None,
            dc.ctypes.data_as(capi.PD) if dc is not None else None, T.size, int(n_paths), float(steps_per_year),
            int(seed) & 0xFFFFFFFFFFFFFFFF)
    tail = (ctypes.c_void_p(price.data_ptr()), ctypes.c_void_p(se.data_ptr()), prec, _stream_handle(stream))
    if scheme is None:
        capi.check(lib.sabr_mc_price(*head, *tail), "sabr_mc_price")
    else:
        capi.check(lib.sabr_mc_price_scheme(*head, int(scheme), *tail), "sabr_mc_price_scheme")
    return price, se


def mc_cliquet(model, params, fwd, T, n_resets, floor_local, cap_local, floor_global=-1e300, cap_global=1e300,
               discount=1.0, n_paths=1 << 20, steps_per_year=250.0, seed=0, prec=FP32, stream=None, device="cuda"):
    """Monte Carlo cliquet price and standard error (float64 CUDA tensors of one element)."""
    lib = capi.load()
    price = torch.empty(1, dtype=torch.float64, device=device)
    se = torch.empty(1, dtype=torch.float64, device=device)
    p = _params10(params, model)
    st = lib.sabr_mc_cliquet(model, p.ctypes.data_as(capi.PD), float(fwd), float(T), int(n_resets),
                             float(floor_local), float(cap_local), float(floor_global), float(cap_global),
                             float(discount), int(n_paths), float(steps_per_year), int(seed) & 0xFFFFFFFFFFFFFFFF,
                             ctypes.c_void_p(price.data_ptr()), ctypes.c_void_p(se.data_ptr()), prec,
                             _stream_handle(stream))
    capi.check(st, "sabr_mc_cliquet")
    return price, se


def _mc_host_args(model, params, T, K, is_call, discount):
    T = np.ascontiguousarray(T, dtype=np.float64).ravel()
    K = np.ascontiguousarray(np.broadcast_to(np.asarray(K, dtype=np.float64), T.shape))
    ic = None if is_call is None else np.ascontiguousarray(is_call, dtype=np.int8).ravel()
    dc = None if discount is None else np.ascontiguousarray(discount, dtype=np.float64).ravel()
    p = _params10(params, model)
    keep = (T, K, ic, dc, p)
    args = (model, p.ctypes.data_as(capi.PD), None, T.ctypes.data_as(capi.PD), K.ctypes.data_as(capi.PD),
            ic.ctypes.data_as(capi.PI8) if ic is not None else None,
            dc.ctypes.data_as(capi.PD) if dc is not None else None, T.size)
    return keep, args


def mc_shard_layout(model, params, fwd, T, K, is_call=None, discount=None, n_paths=1 << 16, steps_per_year=250.0,
                    seed=0, prec=FP32):
    """(total_blocks, doubles_per_block) of the path-sharded form of mc_price."""
    lib = capi.load()
    keep, a = _mc_host_args(model, params, T, K, is_call, discount)
    nb, dpb = ctypes.c_int32(), ctypes.c_int64()
    st = lib.sabr_mc_shard_layout(a[0], a[1], float(fwd), *a[3:], int(n_paths), float(steps_per_year),
                                  int(seed) & 0xFFFFFFFFFFFFFFFF, prec, ctypes.byref(nb), ctypes.byref(dpb))
    capi.check(st, "sabr_mc_shard_layout")
    return nb.value, dpb.value


def mc_shard_partials(model, params, fwd, T, K, total_blocks, block_begin, block_count, is_call=None,
                      discount=None, n_paths=1 << 16, steps_per_year=250.0, seed=0, prec=FP32, stream=None,
                      device="cuda"):
    """Per-block partial sums of blocks [block_begin, block_begin + block_count)
    of the mc_price grid (a float64 CUDA tensor, block_count x doubles_per_block)."""
    lib = capi.load()
    _, dpb = mc_shard_layout(model, params, fwd, T, K, is_call, discount, n_paths, steps_per_year, seed, prec)
    out = torch.empty((block_count, dpb), dtype=torch.float64, device=device)
    keep, a = _mc_host_args(model, params, T, K, is_call, discount)
    st = lib.sabr_mc_shard_partials(a[0], a[1], float(fwd), *a[3:], int(n_paths), float(steps_per_year),
                                    int(seed) & 0xFFFFFFFFFFFFFFFF, prec, int(total_blocks), int(block_begin),
                                    int(block_count), ctypes.c_void_p(out.data_ptr()), _stream_handle(stream))
    capi.check(st, "sabr_mc_shard_partials")
    return out


def mc_shard_reduce(model, params, fwd, T, K, total_blocks, partials, is_call=None, discount=None, n_paths=1 << 16,
                    steps_per_year=250.0, seed=0, prec=FP32, stream=None):
    """Prices and standard errors from the partials of all blocks, in block order."""
    lib = capi.load()
    partials = partials.contiguous()
    n = int(np.asarray(T).size)
    price = torch.empty(n, dtype=torch.float64, device=partials.device)
    se = torch.empty(n, dtype=torch.float64, device=partials.device)
    keep, a = _mc_host_args(model, params, T, K, is_call, discount)
    st = lib.sabr_mc_shard_reduce(a[0], a[1], float(fwd), *a[3:], int(n_paths), float(steps_per_year),
                                  int(seed) & 0xFFFFFFFFFFFFFFFF, prec, int(total_blocks),
                                  ctypes.c_void_p(partials.data_ptr()), ctypes.c_void_p(price.data_ptr()),
                                  ctypes.c_void_p(se.data_ptr()), _stream_handle(stream))
    capi.check(st, "sabr_mc_shard_reduce")
    return price, se


@dataclass
class CalibrationProblem:
    """One calibration problem: quotes, model and SA settings (host data)."""
    model: int
    T: np.ndarray
    K: np.ndarray
    market: np.ndarray
    lo: Sequence[float]
    hi: Sequence[float]
    fwd: float = 1.0
    cost: int = COST_VOL
    prec: int = FP32
    n_chains: int = 64
    T0: float = 0.0
    factor: float = 0.95
    n_levels: int = 200
    chain_len: int = 100
    step0: float = 0.1
    step_min: float = 1e-6
    seed: int = 0
    x0: Optional[Sequence[float]] = None
    is_call: Optional[np.ndarray] = None
    discount: Optional[np.ndarray] = None
    mc_paths: int = 1 << 16
    mc_steps_per_year: float = 250.0
    mc_seed: int = 0
    _keep: list = field(default_factory=list, repr=False)

    def to_c(self):
        T = np.ascontiguousarray(self.T, dtype=np.float64).ravel()
        K = np.ascontiguousarray(self.K, dtype=np.float64).ravel()
        M = np.ascontiguousarray(self.market, dtype=np.float64).ravel()
        if not (T.size == K.size == M.size):
            raise ValueError("T, K and market must have the same length")
        ic = None if self.is_call is None else np.ascontiguousarray(self.is_call, dtype=np.int8).ravel()
        dc = None if self.discount is None else np.ascontiguousarray(self.discount, dtype=np.float64).ravel()
        x0 = None if self.x0 is None else _params10(self.x0, self.model)
        self._keep = [T, K, M, ic, dc, x0]
        pr = capi.Problem()
        pr.model, pr.cost, pr.prec, pr.fwd = self.model, self.cost, self.prec, float(self.fwd)
        pr.n_quotes = T.size
        pr.T, pr.K, pr.market = T.ctypes.data_as(capi.PD), K.ctypes.data_as(capi.PD), M.ctypes.data_as(capi.PD)
        pr.is_call = ic.ctypes.data_as(capi.PI8) if ic is not None else None
        pr.discount = dc.ctypes.data_as(capi.PD) if dc is not None else None
        pr.n_chains = int(self.n_chains)
        pr.mc_paths = int(self.mc_paths)
        pr.mc_steps_per_year = float(self.mc_steps_per_year)
        pr.mc_seed = int(self.mc_seed) & 0xFFFFFFFFFFFFFFFF
        pr.x0 = x0.ctypes.data_as(capi.PD) if x0 is not None else None
        b = capi.Bounds()
        lo = _params10(self.lo, self.model)
        hi = _params10(self.hi, self.model)
        for i in range(10):
            b.lo[i], b.hi[i] = lo[i], hi[i]
        c = capi.Cooling(float(self.T0), float(self.factor), int(self.n_levels), int(self.chain_len),
                         float(self.step0), float(self.step_min))
        return pr, b, c, int(self.seed) & 0xFFFFFFFFFFFFFFFF


@dataclass
class CalibrationResult:
    params: np.ndarray
    misfit: float
    misfit_fp64: float
    restart_params: np.ndarray
    restart_misfit: float
    n_evals: int
    n_accepts: int
    status: int

    @staticmethod
    def from_c(r: capi.Result, model: int):
        d = capi.N_PARAMS[model]
        return CalibrationResult(np.array(r.params[:d]), r.misfit, r.misfit_fp64,
                                 np.array(r.restart_params[:d]), r.restart_misfit, r.n_evals, r.n_accepts,
                                 r.status)


def _marshal(problems: List[CalibrationProblem]):
    n = len(problems)
    P = (capi.Problem * n)()
    B = (capi.Bounds * n)()
    C = (capi.Cooling * n)()
    S = (ctypes.c_uint64 * n)()
    keep = []
    for i, pb in enumerate(problems):
        P[i], B[i], C[i], S[i] = pb.to_c()
        keep.append(pb._keep)  # arrays stay alive while the C structs point at them
    P._keep = keep
    return P, B, C, S


def calibrate_batch(problems: List[CalibrationProblem], stream=None) -> List[CalibrationResult]:
    """Calibrate independent problems together (blocking)."""
    lib = capi.load()
    P, B, C, S = _marshal(problems)
    R = (capi.Result * len(problems))()
    st = lib.sabr_calibrate_batch(len(problems), P, B, C, S, R, _stream_handle(stream))
    capi.check(st, "sabr_calibrate_batch")
    return [CalibrationResult.from_c(R[i], pb.model) for i, pb in enumerate(problems)]


def calibrate(problem: CalibrationProblem, stream=None) -> CalibrationResult:
    """Calibrate one problem (blocking)."""
    lib = capi.load()
    pr, b, c, seed = problem.to_c()
    r = capi.Result()
    st = lib.sabr_calibrate(ctypes.byref(pr), ctypes.byref(b), ctypes.byref(c), seed, ctypes.byref(r),
                            _stream_handle(stream))
    capi.check(st, "sabr_calibrate")
    return CalibrationResult.from_c(r, problem.model)


class Plan:
    """A device-resident batch whose whole calibration replays as one CUDA graph."""

    def __init__(self, problems: List[CalibrationProblem], use_graph=True, stream=None):
        self._lib = capi.load()
        self._problems = problems
        self._arrays = _marshal(problems)
        P, B, C, S = self._arrays
        h = ctypes.c_void_p()
        st = self._lib.sabr_plan_create(len(problems), P, B, C, S, 1 if use_graph else 0,
                                        _stream_handle(stream), ctypes.byref(h))
        capi.check(st, "sabr_plan_create")
        self._h = h

    def run(self, stream=None):
        capi.check(self._lib.sabr_plan_run(self._h, _stream_handle(stream)), "sabr_plan_run")

    def results(self) -> List[CalibrationResult]:
        R = (capi.Result * len(self._problems))()
        capi.check(self._lib.sabr_plan_results(self._h, R), "sabr_plan_results")
        return [CalibrationResult.from_c(R[i], pb.model) for i, pb in enumerate(self._problems)]

    def stats(self):
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        capi.check(self._lib.sabr_plan_stats(self._h, ctypes.byref(n), ctypes.byref(ms)), "sabr_plan_stats")
        return n.value, ms.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sabr_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Shard:
    """Chains [chain_begin, chain_begin + chain_count) of a problem on the
    current device (sabr_shard_* of include/sabr.h).  level(lv) returns the
    shard's lowest final state (f, global chain, x[10]); restart(f, x) sets
    the next level's start; result() returns (CalibrationResult, best global
    chain)."""

    def __init__(self, problem: CalibrationProblem, chain_begin: int, chain_count: int, stream=None):
        self._lib = capi.load()
        self._problem = problem
        pr, b, c, seed = problem.to_c()
        h = ctypes.c_void_p()
        self._stream = stream
        st = self._lib.sabr_shard_create(ctypes.byref(pr), ctypes.byref(b), ctypes.byref(c), seed,
                                         int(chain_begin), int(chain_count), _stream_handle(stream),
                                         ctypes.byref(h))
        capi.check(st, "sabr_shard_create")
        self._h = h

    def level(self, lv):
        p = capi.ChainPoint()
        capi.check(self._lib.sabr_shard_level(self._h, int(lv), ctypes.byref(p), _stream_handle(self._stream)),
                   "sabr_shard_level")
        return p.f, p.chain, np.array(p.x[:])

    def restart(self, f, x):
        p = capi.ChainPoint()
        p.f = float(f)
        p.chain = -1
        for i in range(10):
            p.x[i] = float(x[i])
        capi.check(self._lib.sabr_shard_restart(self._h, ctypes.byref(p), _stream_handle(self._stream)),
                   "sabr_shard_restart")

    def result(self):
        r = capi.Result()
        ch = ctypes.c_int64()
        capi.check(self._lib.sabr_shard_result(self._h, ctypes.byref(r), ctypes.byref(ch),
                                               _stream_handle(self._stream)), "sabr_shard_result")
        return CalibrationResult.from_c(r, self._problem.model), ch.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sabr_shard_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching calibration server (sabr_server_* of include/sabr.h)."""

    def __init__(self, device_bytes=1 << 30, max_queue=1 << 20, max_active=256, max_quotes=512, use_graph=True):
        self._lib = capi.load()
        cfg = capi.ServerConfig(int(device_bytes), int(max_queue), int(max_active), int(max_quotes),
                                1 if use_graph else 0)
        h = ctypes.c_void_p()
        capi.check(self._lib.sabr_server_create(ctypes.byref(cfg), ctypes.byref(h)), "sabr_server_create")
        self._h = h
        self._models = {}

    def submit(self, problem: CalibrationProblem) -> int:
        pr, b, c, seed = problem.to_c()
        t = ctypes.c_uint64()
        capi.check(self._lib.sabr_server_submit(self._h, ctypes.byref(pr), ctypes.byref(b), ctypes.byref(c), seed,
                                                ctypes.byref(t)), "sabr_server_submit")
        self._models[t.value] = problem.model
        return t.value

    def poll(self, ticket):
        r = capi.Result()
        st = self._lib.sabr_server_poll(self._h, ticket, ctypes.byref(r))
        if st == capi.EAGAIN:
            return None
        capi.check(st, "sabr_server_poll")
        return CalibrationResult.from_c(r, self._models.pop(ticket))

    def wait(self, ticket, timeout_ms=-1):
        r = capi.Result()
        capi.check(self._lib.sabr_server_wait(self._h, ticket, int(timeout_ms), ctypes.byref(r)), "sabr_server_wait")
        return CalibrationResult.from_c(r, self._models.pop(ticket))

    def cancel(self, ticket):
        capi.check(self._lib.sabr_server_cancel(self._h, ticket), "sabr_server_cancel")

    def stats(self):
        st = capi.ServerStats()
        capi.check(self._lib.sabr_server_get_stats(self._h, ctypes.byref(st)), "sabr_server_get_stats")
        return {name: getattr(st, name) for name, _ in capi.ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sabr_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
