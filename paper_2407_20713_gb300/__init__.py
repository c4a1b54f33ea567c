"""GB300-native (sm_103a) SABR calibration hot path.

Implements the data-parallel core of Fernandez, Ferreiro, Garcia, Leitao,
Lopez-Salas and Vazquez, "Static and dynamic SABR stochastic volatility
models: calibration and option pricing using GPUs": implied-vol formulas
(Sec. 2), Monte Carlo pricing (Sec. 4) and synchronous parallel Simulated
Annealing calibration (Sec. 5), behind the C-ABI of include/sabr.h.
"""
from . import capi  # noqa: F401
from .capi import (COST_MC_PRICE, COST_VOL, DYN_I, DYN_II, EXPANDED, FP32, FP64, HAGAN,  # noqa: F401
                   MC_BESSEL, MC_LOG_EULER, OBLOJ, SabrError)
from .api import (CalibrationProblem, CalibrationResult, Plan, Server, Shard, calibrate,  # noqa: F401
                  calibrate_batch, implied_vol, mc_cliquet, mc_price, mc_shard_layout, mc_shard_partials,
                  mc_shard_reduce)
