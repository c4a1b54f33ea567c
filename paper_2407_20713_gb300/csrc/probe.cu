// probe.cu -- per-SM throughput of the arithmetic pipes the hot path uses
// (FP32 FMA, the SFU/MUFU operations, 32-bit integer multiply, FP64 FMA),
// in operations per SM clock.  Each thread runs 8 independent chains of one
// operation; SM clocks are read with clock64() so the rates do not depend on
// the clock frequency.  Used to state the ALU roofline the kernels are
// measured against.
#include <cstring>
#include <vector>

#include "common.h"

namespace sabr {

constexpr int kProbeChains = 8;
constexpr int kProbeUnroll = 32;

template <int OP>
__device__ __forceinline__ float probe_op_f(float x, float a, float b) {
  float y;
  if (OP == 0) {
    y = fmaf(x, a, b);
  } else if (OP == 1) {
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));
  } else if (OP == 2) {
    asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    y = fabsf(y) + 1.0f;
  } else if (OP == 3) {
    asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  } else if (OP == 4) {
    // x -> 1/(x + 1): a chain of reciprocals that cannot fold into identity
    asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x + 1.0f));
  } else {
    asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  }
  return y;
}

template <int OP>
__global__ void probe_f32_kernel(int iters, float a, float b, float* sink, long long* cycles) {
  float x[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) x[c] = 0.5f + 0.01f * c + 1e-6f * threadIdx.x;
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kProbeUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kProbeChains; ++c) x[c] = probe_op_f<OP>(x[c], a, b);
  }
  __syncthreads();
  const long long t1 = clock64();
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s += x[c];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

__global__ void probe_imad_kernel(int iters, unsigned a, unsigned b, unsigned* sink, long long* cycles) {
  unsigned x[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) x[c] = 0x9E3779B9u * (threadIdx.x + c);
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kProbeUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kProbeChains; ++c) x[c] = x[c] * a + b;
  }
  __syncthreads();
  const long long t1 = clock64();
  unsigned s = 0;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s ^= x[c];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

__global__ void probe_dfma_kernel(int iters, double a, double b, double* sink, long long* cycles) {
  double x[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) x[c] = 0.5 + 0.01 * c + 1e-9 * threadIdx.x;
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kProbeUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kProbeChains; ++c) x[c] = fma(x[c], a, b);
  }
  __syncthreads();
  const long long t1 = clock64();
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s += x[c];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace sabr

extern "C" sabr_status sabr_probe_pipe_rates(double* rates, int32_t n_rates, void* stream) {
  using namespace sabr;
  clear_error();
  if (!rates || n_rates < 8) return fail(SABR_EINVAL, "rates must hold 8 values");
  int dev = 0, sms = 0;
  SABR_CUDA(cudaGetDevice(&dev));
  SABR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int threads = 1024, blocks = sms;
  void* sink = nullptr;
  long long* cyc = nullptr;
  SABR_CUDA(cudaMalloc(&sink, sizeof(double) * threads * blocks));
  SABR_CUDA(cudaMalloc(&cyc, sizeof(long long) * blocks));
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<long long> hc(blocks);
  auto rate = [&](int op, int iters) -> double {
    switch (op) {
      case 0: probe_f32_kernel<0><<<blocks, threads, 0, s>>>(iters, 0.999f, 1e-3f, (float*)sink, cyc); break;
      case 1: probe_f32_kernel<1><<<blocks, threads, 0, s>>>(iters, 0.f, 0.f, (float*)sink, cyc); break;
      case 2: probe_f32_kernel<2><<<blocks, threads, 0, s>>>(iters, 0.f, 0.f, (float*)sink, cyc); break;
      case 3: probe_f32_kernel<3><<<blocks, threads, 0, s>>>(iters, 0.f, 0.f, (float*)sink, cyc); break;
      case 4: probe_f32_kernel<4><<<blocks, threads, 0, s>>>(iters, 0.f, 0.f, (float*)sink, cyc); break;
      case 5: probe_f32_kernel<5><<<blocks, threads, 0, s>>>(iters, 0.f, 0.f, (float*)sink, cyc); break;
      case 6: probe_imad_kernel<<<blocks, threads, 0, s>>>(iters, 0x9E3779B9u, 7u, (unsigned*)sink, cyc); break;
      default: probe_dfma_kernel<<<blocks, threads, 0, s>>>(iters, 0.999, 1e-3, (double*)sink, cyc); break;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1.0;
    cudaMemcpy(hc.data(), cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost);
    long long mx = 1;
    for (long long c : hc) mx = c > mx ? c : mx;
    return (double)threads * iters * kProbeUnroll * kProbeChains / (double)mx;
  };
  const int iters[8] = {2000, 400, 400, 400, 400, 400, 1000, 40};
  for (int op = 0; op < 8; ++op) {
    rate(op, iters[op] / 10);  // warm-up
    rates[op] = rate(op, iters[op]);
  }
  cudaFree(sink);
  cudaFree(cyc);
  SABR_CUDA(cudaGetLastError());
  return SABR_OK;
}
