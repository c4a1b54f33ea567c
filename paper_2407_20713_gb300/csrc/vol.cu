// vol.cu -- sabr_implied_vol: one thread per option, grid-stride.
#include <cmath>

#include "common.h"
#include "sabr_math.cuh"

namespace sabr {

struct VolArgs {
  double p[kMaxD];
  double fwd;
};

template <class R, int MODEL>
__global__ void __launch_bounds__(256) implied_vol_kernel(VolArgs a, const double* __restrict__ T,
                                                          const double* __restrict__ K, int64_t n,
                                                          double* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  StaticConst<R> sc;
  if (MODEL == SABR_HAGAN || MODEL == SABR_OBLOJ) sc = static_setup<R>(a.p);
  const R l2f = (R)log2(a.fwd);
  const R fwd = (R)a.fwd;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double kd = K[i];
    const R t = (R)T[i], k = (R)kd;
    const R lfk = m_log(fwd / k);
    R v;
    if (MODEL == SABR_HAGAN) {
      v = vol_hagan<R>(sc, lfk, m_log2((R)(kd * a.fwd)), t);
    } else if (MODEL == SABR_OBLOJ) {
      v = vol_obloj<R>(sc, lfk, m_log2((R)(kd * a.fwd)), m_log2(k), t);
    } else if (MODEL == SABR_EXPANDED) {
      v = vol_poly<R>(expanded_coef<R>(a.p, l2f, t), lfk);
    } else {
      v = vol_poly<R>(dynamic_coef<R, MODEL == SABR_DYN_II>(a.p, l2f, t), lfk);
    }
    out[i] = (double)v;
  }
}

template <class R>
static void launch_vol(int model, const VolArgs& a, const double* T, const double* K, int64_t n,
                       double* out, cudaStream_t s) {
  int64_t blocks = (n + 255) / 256;
  const int64_t cap = (int64_t)device_sms() * 16;
  if (blocks > cap) blocks = cap;
  switch (model) {
    case SABR_HAGAN: implied_vol_kernel<R, SABR_HAGAN><<<blocks, 256, 0, s>>>(a, T, K, n, out); break;
    case SABR_OBLOJ: implied_vol_kernel<R, SABR_OBLOJ><<<blocks, 256, 0, s>>>(a, T, K, n, out); break;
    case SABR_EXPANDED: implied_vol_kernel<R, SABR_EXPANDED><<<blocks, 256, 0, s>>>(a, T, K, n, out); break;
    case SABR_DYN_I: implied_vol_kernel<R, SABR_DYN_I><<<blocks, 256, 0, s>>>(a, T, K, n, out); break;
    default: implied_vol_kernel<R, SABR_DYN_II><<<blocks, 256, 0, s>>>(a, T, K, n, out); break;
  }
}

}  // namespace sabr

extern "C" sabr_status sabr_implied_vol(sabr_model model, const double* params, double fwd,
                                        const double* T, const double* K, int64_t n,
                                        double* vol_out, sabr_precision prec, void* stream) {
  using namespace sabr;
  clear_error();
  SABR_TRY(check_params(model, params));
  if (!(fwd > 0.0) || !std::isfinite(fwd)) return fail(SABR_EINVAL, "fwd must be > 0");
  if (prec != SABR_FP32 && prec != SABR_FP64) return fail(SABR_EINVAL, "unknown precision");
  if (n < 0) return fail(SABR_EINVAL, "n < 0");
  if (n == 0) return SABR_OK;
  if (!T || !K || !vol_out) return fail(SABR_EINVAL, "NULL array");
  VolArgs a;
  for (int i = 0; i < kMaxD; ++i) a.p[i] = i < n_params(model) ? params[i] : 0.0;
  a.fwd = fwd;
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == SABR_FP32)
    launch_vol<float>(model, a, T, K, n, vol_out, s);
  else
    launch_vol<double>(model, a, T, K, n, vol_out, s);
  SABR_CUDA(cudaGetLastError());
  return SABR_OK;
}
