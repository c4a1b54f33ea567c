// cliquet.cu -- sabr_mc_cliquet: Monte Carlo price of the cliquet option of
// Sec. 6.3, eqs. (eq_cliquet) and (cliquet_global), on the paths of the
// Sec. 4 scheme: the same Philox streams, step coefficients, absorption and
// path_step as sabr_mc_price, with the reset dates inserted into the grid as
// landing points.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.h"
#include "mc.cuh"
#include "mc_host.h"

namespace sabr {

constexpr int kClqBlock = 128;

// Grid-stride over paths: thread t of the grid prices paths t, t + stride,
// ... and keeps FP64 sums of the payoff and its square; each block adds its
// threads' sums in thread order into partial[2 b], partial[2 b + 1].
template <class R>
__global__ void __launch_bounds__(kClqBlock) cliquet_kernel(McDev P, const double* __restrict__ params,
                                                           double floor_l, double cap_l, double floor_g,
                                                           double cap_g, double* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char smem[];
  StepCoef<R>* tab = (StepCoef<R>*)smem;
  int* land = (int*)(tab + P.n_steps);  // land[r] = the step ending at reset r
  __shared__ double red[2][kClqBlock];
  double p[kMaxD];
#pragma unroll
  for (int i = 0; i < kMaxD; ++i) p[i] = params[i];
  build_steps<R>(P, p, tab, land);
  __syncthreads();
  const R beta_m1 = (R)(p[1] - 1.0);
  const R lnf = (R)PathUnits<R>::logu(P.fwd), lna = (R)PathUnits<R>::logu(p[0]);
  const R log_abs = (R)(P.log_absorb * PathUnits<R>::kLogUnit);
  const R fl = (R)floor_l, cl = (R)cap_l;
  double s1 = 0.0, s2 = 0.0;
  // kMcPathsPerThread paths per thread (path, path + stride, ...) advance
  // together
  constexpr int NPT = kMcPathsPerThread;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p0 < P.n_paths; p0 += NPT * stride) {
    int64_t path[NPT];
    PathState<R> st[NPT];
    R prev[NPT], sum[NPT];
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      path[k] = p0 + k * stride;
      st[k] = PathState<R>{lnf, lna, false};
      prev[k] = (R)0;
      sum[k] = (R)0;
    }
    int reset = 0, i_land = land[0];
    auto at_reset = [&]() {
#pragma unroll
      for (int k = 0; k < NPT; ++k) {
        const R F = st[k].absorbed ? (R)0 : PathUnits<R>::expu(st[k].lnF);
        if (reset >= 1) {
          // R_i = F(d_i)/F(d_{i-1}) - 1; a path absorbed before d_{i-1}
          // adds R_i = 0 (0 to 0)
          const R ret = prev[k] > (R)0 ? F / prev[k] - (R)1 : (R)0;
          const R c = ret < cl ? ret : cl;
          sum[k] += c > fl ? c : fl;
        }
        prev[k] = F;
      }
      ++reset;
      i_land = reset < P.n_mats ? land[reset] : -1;
    };
    for (int i = 0; i < P.n_steps; i += 2) {
      uint4 w[NPT];
#pragma unroll
      for (int k = 0; k < NPT; ++k) w[k] = path_words<R>(P, path[k], i);
#pragma unroll
      for (int k = 0; k < NPT; ++k) path_step<R>(tab[i], w[k].x, w[k].y, beta_m1, log_abs, st[k]);
      if (i == i_land) at_reset();
      if (i + 1 < P.n_steps) {
#pragma unroll
        for (int k = 0; k < NPT; ++k) path_step<R>(tab[i + 1], w[k].z, w[k].w, beta_m1, log_abs, st[k]);
        if (i + 1 == i_land) at_reset();
      }
    }
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      if (path[k] < P.n_paths) {
        double g = (double)sum[k];
        g = g < cap_g ? g : cap_g;
        g = g > floor_g ? g : floor_g;
        s1 += g;
        s2 += g * g;
      }
    }
  }
  red[0][threadIdx.x] = s1;
  red[1][threadIdx.x] = s2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      a += red[0][t];
      b += red[1][t];
    }
    partial[2 * blockIdx.x] = a;
    partial[2 * blockIdx.x + 1] = b;
  }
}

// Block sums in block order -> discounted mean and its standard error.
__global__ void cliquet_reduce_kernel(const double* __restrict__ partial, int blocks, int64_t n_paths, double disc,
                                      double* __restrict__ price, double* __restrict__ se) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0, s2 = 0.0;
  for (int b = 0; b < blocks; ++b) {
    s += partial[2 * b];
    s2 += partial[2 * b + 1];
  }
  const double N = (double)n_paths, mean = s / N;
  double var = (s2 - s * mean) / (N - 1.0);
  if (var < 0.0) var = 0.0;
  *price = disc * mean;
  if (se) *se = disc * sqrt(var / N);
}

}  // namespace sabr

extern "C" sabr_status sabr_mc_cliquet(sabr_model model, const double* params, double fwd, double T,
                                       int32_t n_resets, double floor_local, double cap_local, double floor_global,
                                       double cap_global, double discount, int64_t n_paths, double steps_per_year,
                                       uint64_t seed, double* price_out, double* stderr_out, sabr_precision prec,
                                       void* stream) {
  using namespace sabr;
  clear_error();
  SABR_TRY(check_params(model, params));
  if (!price_out) return fail(SABR_EINVAL, "price_out is NULL");
  if (!(T > 0.0) || !std::isfinite(T)) return fail(SABR_EINVAL, "T must be finite and > 0");
  if (n_resets < 2 || n_resets > kMaxMats) return fail(SABR_EINVAL, "n_resets must lie in [2, 64]");
  if (!(floor_local <= cap_local) || !(floor_global <= cap_global) || !std::isfinite(discount))
    return fail(SABR_EINVAL, "need floor <= cap (local and global) and a finite discount");
  if (n_paths < 2) return fail(SABR_EINVAL, "n_paths must be >= 2");
  if (model == SABR_DYN_II && !case2_feasible<double, double>(params, T))
    return fail(SABR_EINVAL, "parameters violate rho(t) in [-1,1], nu(t) > 0");
  std::vector<double> resets(n_resets), K(n_resets, fwd);
  for (int i = 0; i < n_resets; ++i) resets[i] = (double)(i + 1) * T / n_resets;
  McHost h;
  SABR_TRY(mc_prepare(model, fwd, resets.data(), K.data(), nullptr, nullptr, n_resets, n_paths, steps_per_year, seed,
                      prec, h));
  const size_t smem = (size_t)h.n_steps * (prec == SABR_FP64 ? sizeof(StepCoef<double>) : sizeof(StepCoef<float>)) +
                      (size_t)n_resets * sizeof(int);
  if (smem > 200 * 1024) return fail(SABR_EINVAL, "too many time steps for one launch");
  // resident blocks of the GPU (grid-stride; no partly filled second wave),
  // and no more than the paths need at kMcPathsPerThread paths per thread
  int per_sm = 8;
  if (prec == SABR_FP64) {
    cudaFuncSetAttribute(cliquet_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cliquet_kernel<double>, kClqBlock, smem);
  } else {
    cudaFuncSetAttribute(cliquet_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cliquet_kernel<float>, kClqBlock, smem);
  }
  per_sm = std::min(std::max(per_sm, 1), 8);
  const int64_t per_block = (int64_t)kClqBlock * kMcPathsPerThread;
  const int blocks = (int)std::min<int64_t>(device_sms() * (int64_t)per_sm, (n_paths + per_block - 1) / per_block);
  const size_t img = mc_image_bytes(h);
  const size_t params_off = (img + 255) & ~(size_t)255;
  const size_t part_off = params_off + 256;
  const size_t bytes = part_off + sizeof(double) * 2 * blocks;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* dev = nullptr;
  SABR_CUDA(cudaMallocAsync((void**)&dev, bytes, s));
  std::vector<unsigned char> host(part_off, 0);
  McDev d;
  int *q_value, *q_out;
  double* disc;
  mc_fill_image(h, host.data(), dev, d, &q_value, &q_out, &disc);
  double p10[kMaxD];
  for (int i = 0; i < kMaxD; ++i) p10[i] = i < n_params(model) ? params[i] : 0.0;
  std::memcpy(host.data() + params_off, p10, sizeof(p10));
  // pageable source: the copy has consumed `host` when this returns
  cudaError_t e = cudaMemcpyAsync(dev, host.data(), part_off, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    cudaFreeAsync(dev, s);
    return cuda_fail(e, "cudaMemcpyAsync");
  }
  double* part = (double*)(dev + part_off);
  const double* dp = (const double*)(dev + params_off);
  if (prec == SABR_FP64) {
    e = cudaFuncSetAttribute(cliquet_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      cliquet_kernel<double><<<blocks, kClqBlock, smem, s>>>(d, dp, floor_local, cap_local, floor_global,
                                                            cap_global, part);
  } else {
    e = cudaFuncSetAttribute(cliquet_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      cliquet_kernel<float><<<blocks, kClqBlock, smem, s>>>(d, dp, floor_local, cap_local, floor_global,
                                                           cap_global, part);
  }
  if (e == cudaSuccess) {
    cliquet_reduce_kernel<<<1, 32, 0, s>>>(part, blocks, n_paths, discount, price_out, stderr_out);
    e = cudaGetLastError();
  }
  cudaFreeAsync(dev, s);
  if (e != cudaSuccess) return cuda_fail(e, "cliquet launch");
  return SABR_OK;
}
