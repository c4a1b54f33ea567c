"""Plain FP64 CPU oracle of the SABR calibration hot path.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA
library and its binding never import, link or call it, and it shares no
code with them.  The arithmetic lives in ``sabr_oracle.c``; this module only
marshals numpy arrays through ctypes.

Model ids: 0 Hagan (Sec. 2.1 eq. haganf), 1 Oblój (eq. sigma-SABR),
2 expanded static form (eq. vola_SABR), 3 dynamic Case I, 4 dynamic Case II
(Sec. 2.2, eq. vola_SABRd with eq. el_fun_1 / el_fun_3).
Parameter layout p[10]: alpha, beta, rho0, nu0, a, b, d_rho, d_nu, q_rho, q_nu.
"""
import ctypes
import os

import numpy as np

from . import build_oracle

HAGAN, OBLOJ, EXPANDED, DYN_I, DYN_II = 0, 1, 2, 3, 4
COST_VOL, COST_MC = 0, 1
MC_LOG_EULER, MC_BESSEL = 0, 1
TAG_SA = 0x53410000
TAG_MC = 0x4D430000

_lib = None

_D = ctypes.c_double
_I64 = ctypes.c_int64
_PD = ctypes.POINTER(ctypes.c_double)
_PI8 = ctypes.POINTER(ctypes.c_int8)
_PU32 = ctypes.POINTER(ctypes.c_uint32)
_PI64 = ctypes.POINTER(ctypes.c_int64)


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = ctypes.CDLL(path)
        L.orc_n_params.argtypes = [ctypes.c_int]
        L.orc_n_params.restype = ctypes.c_int
        L.orc_x_of_z.argtypes = [_D, _D]
        L.orc_x_of_z.restype = _D
        L.orc_z_over_x.argtypes = [_D, _D]
        L.orc_z_over_x.restype = _D
        for name in ("orc_vol_hagan", "orc_vol_obloj", "orc_vol_expanded"):
            fn = getattr(L, name)
            fn.argtypes = [_D] * 7
            fn.restype = _D
        L.orc_rho_t.argtypes = [ctypes.c_int, _PD, _D]
        L.orc_rho_t.restype = _D
        L.orc_nu_t.argtypes = [ctypes.c_int, _PD, _D]
        L.orc_nu_t.restype = _D
        L.orc_dyn_coeffs.argtypes = [ctypes.c_int, _PD, _D, _PD]
        L.orc_dyn_coeffs.restype = None
        L.orc_vol_dynamic.argtypes = [ctypes.c_int, _PD, _D, _D, _D]
        L.orc_vol_dynamic.restype = _D
        L.orc_implied_vol.argtypes = [ctypes.c_int, _PD, _D, _D, _D]
        L.orc_implied_vol.restype = _D
        L.orc_implied_vol_batch.argtypes = [ctypes.c_int, _PD, _D, _PD, _PD, _I64, _PD]
        L.orc_implied_vol_batch.restype = None
        L.orc_feasible.argtypes = [ctypes.c_int, _PD, _D]
        L.orc_feasible.restype = ctypes.c_int
        L.orc_misfit.argtypes = [_PD, _PD, _I64]
        L.orc_misfit.restype = _D
        L.orc_integrate_poly.argtypes = [_PD, ctypes.c_int, _D, _D]
        L.orc_integrate_poly.restype = _D
        L.orc_philox4x32_10.argtypes = [_PU32, _PU32, _PU32]
        L.orc_philox4x32_10.restype = None
        L.orc_u01.argtypes = [ctypes.c_uint32]
        L.orc_u01.restype = _D
        L.orc_sa_uniforms.argtypes = [_PU32, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _PD]
        L.orc_sa_uniforms.restype = None
        L.orc_box_muller.argtypes = [_D, _D, _PD, _PD]
        L.orc_box_muller.restype = None
        L.orc_mc_grid.argtypes = [_PD, _I64, _D, _PD, _I64]
        L.orc_mc_grid.restype = _I64
        L.orc_mc_price.argtypes = [ctypes.c_int, _PD, _D, _PD, _PD, _PI8, _PD, _I64,
                                   _I64, _D, ctypes.c_uint64, ctypes.c_int, _PD, _PD]
        L.orc_mc_price.restype = ctypes.c_int
        L.orc_mc_price_scheme.argtypes = [ctypes.c_int, ctypes.c_int, _PD, _D, _PD, _PD, _PI8, _PD, _I64,
                                          _I64, _D, ctypes.c_uint64, ctypes.c_int, _PD, _PD]
        L.orc_mc_price_scheme.restype = ctypes.c_int
        L.orc_mb_gamma_draws.argtypes = [_D, ctypes.c_uint64, _I64, _PD]
        L.orc_mb_gamma_draws.restype = None
        L.orc_mc_cliquet.argtypes = [ctypes.c_int, _PD, _D, _D, ctypes.c_int, _D, _D, _D, _D, _D, _I64, _D,
                                     ctypes.c_uint64, ctypes.c_int, _PD, _PD]
        L.orc_mc_cliquet.restype = ctypes.c_int
        L.orc_sa_calibrate.argtypes = [
            ctypes.c_int, ctypes.c_int, _D, _I64, _PD, _PD, _PD, _PD, _PI8,
            ctypes.c_int, _I64, _D, ctypes.c_uint64, _PD, _PD, _PD,
            _D, _D, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_uint64, ctypes.c_int,
            _PD, _PD, _PD, _PD, _PI64, _PI64, _PD]
        L.orc_sa_calibrate.restype = ctypes.c_int
        L.orc_sa_shard_level.argtypes = [
            ctypes.c_int, ctypes.c_int, _D, _I64, _PD, _PD, _PD, _PD, _PI8,
            _I64, _D, ctypes.c_uint64, _PD, _PD, _D, _D, ctypes.c_int, ctypes.c_int, _D, _D,
            ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int, _PD, _D,
            _PD, _PD, _PD, _PD, _PI64, _PI64]
        L.orc_sa_shard_level.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_PD) if a is not None else None


def _params(p):
    q = np.zeros(10, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64).ravel()
    q[: p.size] = p
    return q


def n_params(model):
    return lib().orc_n_params(model)


def x_of_z(z, rho):
    return lib().orc_x_of_z(float(z), float(rho))


def z_over_x(z, rho):
    return lib().orc_z_over_x(float(z), float(rho))


def vol_hagan(alpha, beta, rho, nu, f, K, T):
    return lib().orc_vol_hagan(alpha, beta, rho, nu, f, K, T)


def vol_obloj(alpha, beta, rho, nu, f, K, T):
    return lib().orc_vol_obloj(alpha, beta, rho, nu, f, K, T)


def vol_expanded(alpha, beta, rho, nu, f, K, T):
    return lib().orc_vol_expanded(alpha, beta, rho, nu, f, K, T)


def rho_t(case, p, t):
    q = _params(p)
    return lib().orc_rho_t(case, _dp(q), float(t))


def nu_t(case, p, t):
    q = _params(p)
    return lib().orc_nu_t(case, _dp(q), float(t))


def dyn_coeffs(case, p, T):
    """(nu1^2, nu2^2, eta1, eta2^2) at maturity T, Sec. 2.2 eq. integrales_SABRd."""
    q = _params(p)
    out = np.zeros(4)
    lib().orc_dyn_coeffs(case, _dp(q), float(T), _dp(out))
    return out


def vol_dynamic(case, p, f, K, T):
    q = _params(p)
    return lib().orc_vol_dynamic(case, _dp(q), float(f), float(K), float(T))


def implied_vol(model, p, f, T, K):
    q = _params(p)
    T = np.ascontiguousarray(np.broadcast_arrays(np.asarray(T, float), np.asarray(K, float))[0],
                             dtype=np.float64).ravel()
    K = np.ascontiguousarray(np.broadcast_to(np.asarray(K, float), T.shape), dtype=np.float64).ravel()
    out = np.empty_like(T)
    lib().orc_implied_vol_batch(model, _dp(q), float(f), _dp(T), _dp(K), T.size, _dp(out))
    return out


def feasible(model, p, Tmax):
    q = _params(p)
    return bool(lib().orc_feasible(model, _dp(q), float(Tmax)))


def misfit(model_vals, mkt):
    a = np.ascontiguousarray(model_vals, dtype=np.float64)
    b = np.ascontiguousarray(mkt, dtype=np.float64)
    return lib().orc_misfit(_dp(a), _dp(b), a.size)


def integrate_poly(coeffs, a, b):
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    return lib().orc_integrate_poly(_dp(c), c.size - 1, float(a), float(b))


def philox(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def u01(w):
    return lib().orc_u01(int(w) & 0xFFFFFFFF)


def sa_uniforms(key, chain, level, step, d):
    """The d + 1 uniforms of SA proposal (chain, level, step): d moves, then
    the acceptance uniform."""
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    u = (ctypes.c_double * (d + 1))()
    lib().orc_sa_uniforms(k, int(chain), int(level), int(step), int(d), u)
    return np.array(u[:])


def box_muller(u1, u2):
    a, b = ctypes.c_double(), ctypes.c_double()
    lib().orc_box_muller(float(u1), float(u2), ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def mc_grid(T, steps_per_year):
    T = np.ascontiguousarray(T, dtype=np.float64).ravel()
    n = lib().orc_mc_grid(_dp(T), T.size, float(steps_per_year), None, 0)
    g = np.empty(n)
    lib().orc_mc_grid(_dp(T), T.size, float(steps_per_year), _dp(g), n)
    return g


def mc_price(model, p, f, T, K, is_call=None, disc=None, n_paths=1 << 12,
             steps_per_year=250.0, seed=0, n_threads=1, scheme=MC_LOG_EULER):
    """Sec. 4 Monte Carlo prices and standard errors: the log-Euler scheme
    (MC_LOG_EULER) or the conditional-Bessel step (MC_BESSEL)."""
    q = _params(p)
    T = np.ascontiguousarray(T, dtype=np.float64).ravel()
    K = np.ascontiguousarray(K, dtype=np.float64).ravel()
    ic = None if is_call is None else np.ascontiguousarray(is_call, dtype=np.int8).ravel()
    dc = None if disc is None else np.ascontiguousarray(disc, dtype=np.float64).ravel()
    price = np.empty(T.size)
    se = np.empty(T.size)
    rc = lib().orc_mc_price_scheme(int(scheme), model, _dp(q), float(f), _dp(T), _dp(K),
                            ic.ctypes.data_as(_PI8) if ic is not None else None,
                            _dp(dc), T.size, int(n_paths), float(steps_per_year),
                            int(seed) & 0xFFFFFFFFFFFFFFFF, int(n_threads),
                            _dp(price), _dp(se))
    if rc != 0:
        raise ValueError("orc_mc_price rejected its input")
    return price, se


def mb_gamma_draws(a, n, seed=0):
    """n Gamma(a) draws of the conditional-Bessel step's sampler."""
    out = np.empty(int(n))
    lib().orc_mb_gamma_draws(float(a), int(seed) & 0xFFFFFFFFFFFFFFFF, int(n), _dp(out))
    return out


def sa_calibrate(model, f, T, K, mkt, lo, hi, *, cost=COST_VOL, n_chains=64,
                 T0=0.0, factor=0.95, n_levels=200, chain_len=100, step0=0.1,
                 step_min=1e-6, seed=0, x0=None, is_call=None, disc=None,
                 mc_paths=1 << 12, mc_steps_per_year=250.0, mc_seed=0,
                 n_threads=1, trace=False):
    """Sec. 5 synchronous parallel SA; returns a dict of the result."""
    T = np.ascontiguousarray(T, dtype=np.float64).ravel()
    K = np.ascontiguousarray(K, dtype=np.float64).ravel()
    mkt = np.ascontiguousarray(mkt, dtype=np.float64).ravel()
    lo = _params(lo)
    hi = _params(hi)
    x0a = None if x0 is None else _params(x0)
    ic = None if is_call is None else np.ascontiguousarray(is_call, dtype=np.int8).ravel()
    dc = None if disc is None else np.ascontiguousarray(disc, dtype=np.float64).ravel()
    bx = np.zeros(10)
    rx = np.zeros(10)
    bf = ctypes.c_double()
    rf = ctypes.c_double()
    ne = ctypes.c_int64()
    na = ctypes.c_int64()
    tr = np.zeros(max(n_levels, 1)) if trace else None
    rc = lib().orc_sa_calibrate(
        model, cost, float(f), T.size, _dp(T), _dp(K), _dp(mkt), _dp(dc),
        ic.ctypes.data_as(_PI8) if ic is not None else None,
        int(n_chains), int(mc_paths), float(mc_steps_per_year),
        int(mc_seed) & 0xFFFFFFFFFFFFFFFF, _dp(x0a), _dp(lo), _dp(hi),
        float(T0), float(factor), int(n_levels), int(chain_len), float(step0),
        float(step_min), int(seed) & 0xFFFFFFFFFFFFFFFF, int(n_threads),
        _dp(bx), ctypes.byref(bf), _dp(rx), ctypes.byref(rf),
        ctypes.byref(ne), ctypes.byref(na), _dp(tr))
    if rc != 0:
        raise ValueError("orc_sa_calibrate rejected its input")
    d = n_params(model)
    out = dict(params=bx[:d].copy(), misfit=bf.value, restart_params=rx[:d].copy(),
               restart_misfit=rf.value, n_evals=ne.value, n_accepts=na.value)
    if trace:
        out["trace"] = tr[:n_levels].copy()
    return out


class SaShard:
    """The chains c0 .. c0+nc-1 of orc_sa_calibrate, one level at a time
    (Sec. 5.1, the multi-GPU form of Technique I): level() runs a level from
    the current restart point and returns this share's lowest final state
    (cost, chain, x), restart() sets the next level's start, result() the
    share's best-ever point (cost, chain, x) and counters.  Formula cost
    (Technique I) only."""

    def __init__(self, model, f, T, K, mkt, lo, hi, *, n_chains, c0, nc, T0=0.0, factor=0.95, n_levels=200,
                 chain_len=100, step0=0.1, step_min=1e-6, seed=0, x0=None, n_threads=1):
        self.model, self.f = model, float(f)
        self.T = np.ascontiguousarray(T, dtype=np.float64).ravel()
        self.K = np.ascontiguousarray(K, dtype=np.float64).ravel()
        self.mkt = np.ascontiguousarray(mkt, dtype=np.float64).ravel()
        self.lo, self.hi = _params(lo), _params(hi)
        self.d = n_params(model)
        xs = _params(x0) if x0 is not None else 0.5 * (self.lo + self.hi)
        xs[self.d:] = 0.0
        fs = misfit(implied_vol(model, xs, f, self.T, self.K), self.mkt)
        self.T0 = float(T0) if T0 > 0.0 else (fs if fs > 0.0 else 1.0)
        self.factor, self.chain_len, self.step0, self.step_min = factor, chain_len, step0, step_min
        self.seed, self.n_threads, self.c0, self.nc = seed, n_threads, c0, nc
        self.xs, self.fs = xs, fs
        self.cx = np.zeros(10 * nc)
        self.cf = np.zeros(nc)
        self.bx = np.tile(xs, nc)
        self.bf = np.full(nc, fs)
        self.ev = np.zeros(nc, dtype=np.int64)
        self.ac = np.zeros(nc, dtype=np.int64)

    def level(self, lev):
        rc = lib().orc_sa_shard_level(
            self.model, COST_VOL, self.f, self.T.size, _dp(self.T), _dp(self.K), _dp(self.mkt), None, None,
            0, 250.0, 0, _dp(self.lo), _dp(self.hi), self.T0, float(self.factor), int(lev), int(self.chain_len),
            float(self.step0), float(self.step_min), int(self.seed) & 0xFFFFFFFFFFFFFFFF, int(self.n_threads),
            int(self.c0), int(self.nc), _dp(self.xs), float(self.fs), _dp(self.cx), _dp(self.cf), _dp(self.bx),
            _dp(self.bf), self.ev.ctypes.data_as(_PI64), self.ac.ctypes.data_as(_PI64))
        if rc != 0:
            raise ValueError("orc_sa_shard_level rejected its input")
        i = int(np.argmin(self.cf))  # first of the lowest
        return float(self.cf[i]), self.c0 + i, self.cx[10 * i:10 * i + 10].copy()

    def restart(self, f, x):
        self.xs = np.asarray(x, dtype=np.float64).copy()
        self.fs = float(f)

    def result(self):
        i = int(np.argmin(self.bf))
        return (float(self.bf[i]), self.c0 + i, self.bx[10 * i:10 * i + 10].copy(), int(self.ev.sum()),
                int(self.ac.sum()))


def mc_cliquet(model, p, f, T, n_resets, floor_l, cap_l, floor_g, cap_g, disc=1.0, n_paths=1 << 12,
               steps_per_year=250.0, seed=0, n_threads=1):
    """Sec. 6.3 cliquet price and standard error."""
    q = _params(p)
    price, se = ctypes.c_double(), ctypes.c_double()
    rc = lib().orc_mc_cliquet(model, _dp(q), float(f), float(T), int(n_resets), float(floor_l), float(cap_l),
                              float(floor_g), float(cap_g), float(disc), int(n_paths), float(steps_per_year),
                              int(seed) & 0xFFFFFFFFFFFFFFFF, int(n_threads), ctypes.byref(price), ctypes.byref(se))
    if rc != 0:
        raise ValueError("orc_mc_cliquet rejected its input")
    return price.value, se.value
