// mcsa_host.h -- host side of Technique II calibration (see mcsa.cuh).
#pragma once
#include <vector>

#include "mc_host.h"
#include "mcsa.cuh"

namespace sabr {

struct McSaHost {
  int model = 0, n_chains = 0, n_levels = 0, chain_len = 0;
  double T0 = 0, step0 = 0, step_min = 0;
  uint64_t seed = 0;
  double lo[kMaxD], hi[kMaxD], x0[kMaxD];
  std::vector<double> mkt, ck;
  McHost mc;    // paths in the problem's precision
  McHost mc64;  // FP64 paths for the final re-score
  int bps = 1, bps1 = 1;
  // device image (filled by mcsa_layout)
  McSaDev dev;
  McDev dmc, dmc64;
  int *q_value = nullptr, *q_out = nullptr, *q_value64 = nullptr, *q_out64 = nullptr;
  double *disc = nullptr, *disc64 = nullptr;
  double *partial = nullptr, *partial1 = nullptr;
  size_t end = 0;
};

sabr_status mcsa_prepare(const sabr_problem& pr, const sabr_bounds& b, const sabr_cooling& c, uint64_t seed,
                         McSaHost& m);
size_t mcsa_arena_bytes(const McSaHost& m);
// Lays the problem out at [off0, ...) of the arena (host image img, device
// base); m.end receives the end offset.
void mcsa_layout(McSaHost& m, unsigned char* img, unsigned char* base, size_t off0, sabr_result* dres);
int64_t mcsa_enqueue(const McSaHost& m, cudaStream_t s);
// One piece: 0 start, 1 wave (level, step), 2 level restart, 3 final.
int64_t mcsa_enqueue_piece(const McSaHost& m, cudaStream_t s, int what, int level, int step);

}  // namespace sabr
