// common.h -- host-side status/error plumbing shared by the libsabr sources.
#pragma once
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <string>

#include "../../include/sabr.h"

namespace sabr {

// Thread-local message of the last failure (returned by sabr_last_error).
void set_error(const char* fmt, ...);
void clear_error();

inline sabr_status fail(sabr_status s, const char* msg) {
  set_error("%s", msg);
  return s;
}

inline sabr_status cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? SABR_ENOMEM : SABR_ECUDA;
}

#define SABR_CUDA(call)                                   \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return ::sabr::cuda_fail(e_, #call); \
  } while (0)

#define SABR_TRY(expr)                   \
  do {                                   \
    sabr_status s_ = (expr);             \
    if (s_ != SABR_OK) return s_;        \
  } while (0)

inline int n_params(int model) {
  switch (model) {
    case SABR_HAGAN:
    case SABR_OBLOJ:
    case SABR_EXPANDED: return 4;
    case SABR_DYN_I: return 6;
    case SABR_DYN_II: return 10;
    default: return -1;
  }
}

// Streaming multiprocessors of the current device (cached per device).
int device_sms();

// Range checks of a parameter vector common to every entry point.
sabr_status check_params(int model, const double* p);

constexpr int kMaxD = 10;
constexpr int kMaxQuotes = 4096;
constexpr int kMaxMats = 64;

}  // namespace sabr
