// mc_host.h -- host-side description of a Monte Carlo pricing problem, shared
// by sabr_mc_price and the Technique II (MC-cost) calibration engine.
#pragma once
#include <cstdint>
#include <vector>

#include "common.h"
#include "mc.cuh"

namespace sabr {

struct McHost {
  int model = 0, prec = 0, n_quotes = 0, n_steps = 0, n_slots = 0;
  int scheme = SABR_MC_LOG_EULER;  // path scheme (sabr_mc_scheme)
  double fwd = 1.0, Tmax = 0.0;
  int64_t n_paths = 0;
  uint64_t seed = 0;
  size_t smem = 0;
  std::vector<double> mats, K, disc, step_t, step_h;
  std::vector<int> mat_q0, mat_nq, mat_slot, step_mat, q_out, q_value;
  std::vector<int8_t> call;
};

// Validates the option set and builds the step grid (options sorted by
// maturity; q_out maps the sorted position back to the caller's index).
sabr_status mc_prepare(int model, double fwd, const double* T, const double* K, const int8_t* is_call,
                       const double* discount, int64_t n, int64_t n_paths, double spy, uint64_t seed,
                       int prec, McHost& h);
size_t mc_image_bytes(const McHost& h);
// Writes the device image into host_img; pointers in d refer to dev_base.
void mc_fill_image(const McHost& h, unsigned char* host_img, unsigned char* dev_base, McDev& d, int** q_value,
                   int** q_out, double** disc);
int mc_blocks_per_set(const McHost& h, int n_sets);
// Enqueues the path kernel (grid blocks_per_set x n_sets) and the reduction.
sabr_status mc_launch(const McHost& h, const McDev& d, const double* set_params, const int* set_valid, int n_sets,
                      int blocks_per_set, double* partial, const int* q_value, const int* q_out,
                      const double* disc, double* price, double* se, int out_stride, cudaStream_t s);

}  // namespace sabr
