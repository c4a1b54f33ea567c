"""ctypes declarations of the C-ABI in include/sabr.h (argument marshalling only).

Loading fails loudly when libsabr.so has not been built: there is no CPU or
Python fallback for any entry point.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsabr.so")

c_double = ctypes.c_double
c_int = ctypes.c_int
c_int8 = ctypes.c_int8
c_int32 = ctypes.c_int32
c_int64 = ctypes.c_int64
c_uint64 = ctypes.c_uint64
c_void_p = ctypes.c_void_p
PD = ctypes.POINTER(c_double)
PI8 = ctypes.POINTER(c_int8)
PU64 = ctypes.POINTER(c_uint64)

# enums (values as in include/sabr.h)
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EAGAIN, EBUSY, ECANCELLED, ENOTFOUND = range(9)
HAGAN, OBLOJ, EXPANDED, DYN_I, DYN_II = range(5)
COST_VOL, COST_MC_PRICE = 0, 1
FP32, FP64 = 0, 1
MC_LOG_EULER, MC_BESSEL = 0, 1
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ETIMEOUT", "EAGAIN", "EBUSY", "ECANCELLED",
                "ENOTFOUND"]
MODEL_NAMES = {"hagan": HAGAN, "obloj": OBLOJ, "expanded": EXPANDED, "dyn1": DYN_I, "dyn2": DYN_II}
N_PARAMS = {HAGAN: 4, OBLOJ: 4, EXPANDED: 4, DYN_I: 6, DYN_II: 10}


class Problem(ctypes.Structure):
    _fields_ = [("model", c_int), ("cost", c_int), ("prec", c_int), ("fwd", c_double),
                ("n_quotes", c_int64), ("T", PD), ("K", PD), ("market", PD), ("is_call", PI8),
                ("discount", PD), ("n_chains", c_int32), ("mc_paths", c_int64),
                ("mc_steps_per_year", c_double), ("mc_seed", c_uint64), ("x0", PD)]


class Bounds(ctypes.Structure):
    _fields_ = [("lo", c_double * 10), ("hi", c_double * 10)]


class Cooling(ctypes.Structure):
    _fields_ = [("T0", c_double), ("factor", c_double), ("n_levels", c_int32), ("chain_len", c_int32),
                ("step0", c_double), ("step_min", c_double)]


class Result(ctypes.Structure):
    _fields_ = [("params", c_double * 10), ("misfit", c_double), ("misfit_fp64", c_double),
                ("restart_params", c_double * 10), ("restart_misfit", c_double),
                ("n_evals", c_int64), ("n_accepts", c_int64), ("status", c_int)]


class ChainPoint(ctypes.Structure):
    _fields_ = [("f", c_double), ("chain", c_int64), ("x", c_double * 10)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("device_bytes", c_int64), ("max_queue", c_int32), ("max_active", c_int32),
                ("max_quotes", c_int32), ("use_graph", c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", c_int64), ("admitted", c_int64), ("completed", c_int64), ("cancelled", c_int64),
                ("steps", c_int64), ("kernel_launches", c_int64), ("queued", c_int32), ("active", c_int32),
                ("pool_bytes_in_use", c_int64)]


# name -> (restype, argtypes)
SIGNATURES = {
    "sabr_implied_vol": (c_int, [c_int, PD, c_double, c_void_p, c_void_p, c_int64, c_void_p, c_int,
                                 c_void_p]),
    "sabr_mc_price": (c_int, [c_int, PD, c_double, PD, PD, PI8, PD, c_int64, c_int64, c_double, c_uint64,
                              c_void_p, c_void_p, c_int, c_void_p]),
    "sabr_mc_price_scheme": (c_int, [c_int, PD, c_double, PD, PD, PI8, PD, c_int64, c_int64, c_double, c_uint64,
                                     c_int, c_void_p, c_void_p, c_int, c_void_p]),
    "sabr_mc_price_noalloc": (c_int, [c_int, PD, c_double, PD, PD, PI8, PD, c_int64, c_int64, c_double,
                                      c_uint64, c_void_p, c_void_p, c_int, c_void_p]),
    "sabr_mc_cliquet": (c_int, [c_int, PD, c_double, c_double, c_int32, c_double, c_double, c_double, c_double,
                                c_double, c_int64, c_double, c_uint64, c_void_p, c_void_p, c_int, c_void_p]),
    "sabr_calibrate": (c_int, [ctypes.POINTER(Problem), ctypes.POINTER(Bounds), ctypes.POINTER(Cooling),
                               c_uint64, ctypes.POINTER(Result), c_void_p]),
    "sabr_calibrate_batch": (c_int, [c_int32, ctypes.POINTER(Problem), ctypes.POINTER(Bounds),
                                     ctypes.POINTER(Cooling), PU64, ctypes.POINTER(Result), c_void_p]),
    "sabr_plan_create": (c_int, [c_int32, ctypes.POINTER(Problem), ctypes.POINTER(Bounds),
                                 ctypes.POINTER(Cooling), PU64, c_int32, c_void_p,
                                 ctypes.POINTER(c_void_p)]),
    "sabr_plan_run": (c_int, [c_void_p, c_void_p]),
    "sabr_plan_results": (c_int, [c_void_p, ctypes.POINTER(Result)]),
    "sabr_plan_stats": (c_int, [c_void_p, ctypes.POINTER(c_int64), ctypes.POINTER(c_double)]),
    "sabr_plan_destroy": (None, [c_void_p]),
    "sabr_probe_pipe_rates": (c_int, [PD, c_int32, c_void_p]),
    "sabr_server_create": (c_int, [ctypes.POINTER(ServerConfig), ctypes.POINTER(c_void_p)]),
    "sabr_server_submit": (c_int, [c_void_p, ctypes.POINTER(Problem), ctypes.POINTER(Bounds),
                                   ctypes.POINTER(Cooling), c_uint64, ctypes.POINTER(c_uint64)]),
    "sabr_server_poll": (c_int, [c_void_p, c_uint64, ctypes.POINTER(Result)]),
    "sabr_server_wait": (c_int, [c_void_p, c_uint64, c_int64, ctypes.POINTER(Result)]),
    "sabr_server_cancel": (c_int, [c_void_p, c_uint64]),
    "sabr_server_get_stats": (c_int, [c_void_p, ctypes.POINTER(ServerStats)]),
    "sabr_server_destroy": (None, [c_void_p]),
    "sabr_mc_shard_layout": (c_int, [c_int, PD, c_double, PD, PD, PI8, PD, c_int64, c_int64, c_double, c_uint64,
                                     c_int, ctypes.POINTER(c_int32), ctypes.POINTER(c_int64)]),
    "sabr_mc_shard_partials": (c_int, [c_int, PD, c_double, PD, PD, PI8, PD, c_int64, c_int64, c_double,
                                       c_uint64, c_int, c_int32, c_int32, c_int32, c_void_p, c_void_p]),
    "sabr_mc_shard_reduce": (c_int, [c_int, PD, c_double, PD, PD, PI8, PD, c_int64, c_int64, c_double, c_uint64,
                                     c_int, c_int32, c_void_p, c_void_p, c_void_p, c_void_p]),
    "sabr_shard_create": (c_int, [ctypes.POINTER(Problem), ctypes.POINTER(Bounds), ctypes.POINTER(Cooling),
                                  c_uint64, c_int32, c_int32, c_void_p, ctypes.POINTER(c_void_p)]),
    "sabr_shard_level": (c_int, [c_void_p, c_int32, ctypes.POINTER(ChainPoint), c_void_p]),
    "sabr_shard_restart": (c_int, [c_void_p, ctypes.POINTER(ChainPoint), c_void_p]),
    "sabr_shard_result": (c_int, [c_void_p, ctypes.POINTER(Result), ctypes.POINTER(c_int64), c_void_p]),
    "sabr_shard_destroy": (None, [c_void_p]),
    "sabr_last_error": (ctypes.c_char_p, []),
}

_lib = None


def load():
    """Load libsabr.so (built by paper_2407_20713_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libsabr.so is not built (run __graft_entry__.build() or "
                              "python -m paper_2407_20713_gb300.build); there is no fallback")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            if hasattr(lib, name):
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
        _lib = lib
    return _lib


class SabrError(RuntimeError):
    def __init__(self, status, where):
        msg = load().sabr_last_error().decode(errors="replace")
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__("%s failed: %s (%s)" % (where, name, msg))
        self.status = status


def check(status, where):
    if status != OK:
        raise SabrError(status, where)
