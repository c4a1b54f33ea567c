// engine_host.h -- host-side pieces of the formula-cost SA engine shared by
// plans (sa.cu) and the serving runtime (server.cu).
#pragma once
#include <cstdint>
#include <vector>

#include "common.h"
#include "engine.cuh"

namespace sabr {

// Validated, FP64-preprocessed problem (quotes sorted by maturity).
struct HostProblem {
  int model = 0, prec = 0, cost = 0, d = 0, n_quotes = 0, n_mats = 0, n_chains = 0, n_levels = 0,
      chain_len = 0;
  double fwd = 1.0, Tmax = 0.0;
  std::vector<double> lfk, l2kf, l2k, T, mkt, mT, ck;
  std::vector<int> mat;
  double x0[kMaxD], lo[kMaxD], hi[kMaxD];
  double T0 = 0.0, step0 = 0.0, step_min = 0.0;
  uint64_t seed = 0;
  int chain0 = 0;  // global index of chain 0 (chain-sharded problems)
  // FP32 Case II term-structure rule (case2_rule_build): per node (u, W,
  // tau, 0), per sub-panel (half width, sum of W, sum of tau W, 0), per
  // maturity (first sub-panel, sub-panel count)
  std::vector<float> c2_node, c2_sub;
  std::vector<int> c2_panel;
  int c2_nsub = 0;
};

sabr_status formula_prepare(const sabr_problem& pr, const sabr_bounds& b, const sabr_cooling& c, uint64_t seed,
                            HostProblem& h);
// Lanes per chain for a problem of a batch holding batch_chains chains.
// Tuning override: the environment variable SABR_LANES (a power of two in
// [1, 32]) sets it for every problem; results then differ only by the FP32
// rounding of the lane sums.
int choose_lanes(int n_quotes, int n_mats, int model, int prec, long long batch_chains);
// Dynamic shared memory of a level block (cpb chains) / of an init block;
// c2_nsub: sub-panels of the FP32 Case II rule (0 otherwise).
size_t level_smem_bytes(int prec, int model, int Q, int M, int cpb, int c2_nsub = 0);
// Most sub-panels an FP32 Case II rule may have (8 nodes each).
constexpr int kMaxC2Sub = 128;
size_t init_smem_bytes(const HostProblem& h);
// Lays out one problem's device region at [off0, end) of an arena: its
// quotes, schedule, start point, chain state and block partials, filling d.
// img == nullptr performs a dry run (offsets only).  Returns end.
// `block`: threads per level block (chains per block = block / G).
size_t formula_layout(const HostProblem& h, int G, unsigned char* img, unsigned char* base, size_t off0,
                      ProblemDev& d, sabr_result* dres, int block = kSaBlock);

// Kernel launches for (prec, model).
void set_engine_smem(int prec, int model, size_t bytes);
void launch_init(int prec, int model, const ProblemDev* probs, const int* plist, int n, size_t smem, cudaStream_t s);
void launch_level(int prec, int model, const ProblemDev* probs, const int4* bmap, int blocks, int level, size_t smem,
                  cudaStream_t s);
void launch_persistent(int prec, int model, const ProblemDev* probs, const int4* work, const int* n_work, int grid,
                       size_t smem, cudaStream_t s);
void launch_finalize(int prec, int model, const ProblemDev* probs, const int* plist, int n, cudaStream_t s,
                     const unsigned int* queue_err = nullptr);
// Resident 256-thread blocks per SM of the level kernel at `smem` (the
// server's grid-stride launches).
int persistent_blocks_per_sm(int prec, int model, size_t smem);

}  // namespace sabr
