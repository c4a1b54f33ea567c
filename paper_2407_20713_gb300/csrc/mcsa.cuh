// mcsa.cuh -- Technique II (Sec. 5.2): synchronous parallel SA whose cost is
// the relative misfit of Monte Carlo prices (Sec. 3 eq.
// error_calibrate_relativo with Data = V).  Every evaluation of a problem
// uses the same paths (common random numbers), so the cost is a smooth
// deterministic function of the parameters.
//
// One proposal wave = (1) a propose kernel, one thread per chain: Philox
// uniforms, the move, the box and Case II checks; (2) the fused MC kernel
// over every chain's proposal (grid: path blocks x chains); (3) the
// fixed-order price reduction; (4) an accept kernel, one thread per chain:
// FP64 misfit, best-ever update, Metropolis.  Levels end with a one-block
// argmin that restarts every chain from the lowest final state.  The SA
// arithmetic is FP64 in both precisions (it is a few scalar operations per
// chain); the precision switch applies to the paths.
#pragma once
#include <cstdint>

#include "../../include/sabr.h"
#include "mc.cuh"

namespace sabr {

struct McSaDev {
  int model, d, n_chains, n_levels, chain_len, n_quotes;
  double lo[10], hi[10];
  double T0_given, step0, step_min, Tmax;
  uint32_t key0, key1;
  const double* ck;        // factor^k
  const double* x0;        // [10]
  const double* mkt;       // [n_quotes], caller order
  double* state;           // restart x[10], restart f, T0
  double* cx;              // [n_chains][10] current points
  double* cf;              // [n_chains]
  double* bx;              // [n_chains][10] best points
  double* bf;              // [n_chains]
  unsigned long long* ev;
  unsigned long long* ac;
  double* set_params;      // [n_chains][10] proposals of the wave
  int* set_valid;          // [n_chains]
  double* prices;          // [n_chains][n_quotes] MC prices of the wave
  double* one_params;      // [10] single evaluation (x0, re-score)
  double* one_prices;      // [n_quotes]
  sabr_result* result;
};

}  // namespace sabr
