// api.cu -- error reporting and argument checks shared by the entry points.
#include <atomic>
#include <cmath>

#include "common.h"

namespace sabr {

static thread_local char g_error[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_error, sizeof(g_error), fmt, ap);
  va_end(ap);
}

void clear_error() { g_error[0] = '\0'; }

// SM count of the current device, queried once per device ordinal and
// cached (the grid sizes of the kernels are multiples of it).
int device_sms() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
  if (dev < 64) {
    const int c = cache[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return 1;
  if (dev < 64) cache[dev].store(sms, std::memory_order_relaxed);
  return sms;
}

sabr_status check_params(int model, const double* p) {
  if (n_params(model) < 0) return fail(SABR_EINVAL, "unknown model");
  if (!p) return fail(SABR_EINVAL, "params is NULL");
  const int d = n_params(model);
  for (int i = 0; i < d; ++i)
    if (!std::isfinite(p[i])) return fail(SABR_EINVAL, "non-finite parameter");
  if (!(p[0] > 0.0)) return fail(SABR_EINVAL, "alpha must be > 0");
  if (!(p[1] >= 0.0 && p[1] <= 1.0)) return fail(SABR_EINVAL, "beta must lie in [0, 1]");
  if (model <= SABR_EXPANDED) {
    if (!(p[2] > -1.0 && p[2] < 1.0)) return fail(SABR_EINVAL, "rho must lie in (-1, 1)");
    if (!(p[3] >= 0.0)) return fail(SABR_EINVAL, "nu must be >= 0");
  } else {
    if (!(p[2] >= -1.0 && p[2] <= 1.0)) return fail(SABR_EINVAL, "rho0 must lie in [-1, 1]");
    if (!(p[4] >= 0.0 && p[5] >= 0.0)) return fail(SABR_EINVAL, "a and b must be >= 0");
    if (model == SABR_DYN_I && !(p[3] >= 0.0)) return fail(SABR_EINVAL, "nu0 must be >= 0");
  }
  return SABR_OK;
}

}  // namespace sabr

extern "C" const char* sabr_last_error(void) { return sabr::g_error; }
