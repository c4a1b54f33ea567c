// mc.cu -- sabr_mc_price: fused path simulation + deterministic reduction.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.h"
#include "mc.cuh"
#include "mc_bessel.cuh"
#include "mc_host.h"

namespace sabr {

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------
struct McSmem {
  size_t tab, land, q0, nq, slot, K, call, wacc, total;
};

template <class R>
__host__ __device__ inline McSmem mc_smem_layout(int n_steps, int n_quotes, int n_mats, int n_slots) {
  McSmem L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = (o + 15) & ~(size_t)15;
    o = r + bytes;
    return r;
  };
  L.wacc = take(sizeof(double) * kMcWarps * n_slots * 32);
  L.tab = take(sizeof(StepCoef<R>) * n_steps);
  L.K = take(sizeof(R) * n_quotes);
  L.land = take(sizeof(int) * n_mats);
  L.q0 = take(sizeof(int) * n_mats);
  L.nq = take(sizeof(int) * n_mats);
  L.slot = take(sizeof(int) * n_mats);
  L.call = take(n_quotes);
  L.total = (o + 15) & ~(size_t)15;
  return L;
}

// grid = (blocks_per_set, n_sets).  Set s prices with set_params[s][0..9];
// sets whose set_valid flag is 0 are skipped.  Writes, per block, the FP64
// sums of payoff and payoff^2 of every option to
// partial[(s * blocks_per_set + block) * n_slots * 32 + value].
// block0 / grid_total (path sharding): this launch runs blocks block0 ..
// block0 + gridDim.x - 1 of a grid of grid_total blocks -- each block takes
// the paths it would take in that grid -- and writes their partials at
// positions 0 .. gridDim.x - 1; grid_total = 0 means the launch is the
// whole grid.  SCHEME: SABR_MC_LOG_EULER (eq. (dis_SABRd)) or
// SABR_MC_BESSEL (the conditional-Bessel step of mc_bessel.cuh).
template <class R, int SCHEME>
__global__ void __launch_bounds__(kMcBlock) mc_paths_kernel(McDev P, const double* __restrict__ set_params,
                                                           const int* __restrict__ set_valid,
                                                           double* __restrict__ partial, int block0,
                                                           int grid_total) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int set = blockIdx.y;
  if (set_valid && !set_valid[set]) return;
  const McSmem L = mc_smem_layout<R>(P.n_steps, P.n_quotes, P.n_mats, P.n_slots);
  double* wacc = (double*)(smem + L.wacc);
  StepCoef<R>* tab = (StepCoef<R>*)(smem + L.tab);
  R* sK = (R*)(smem + L.K);
  int* land = (int*)(smem + L.land);
  int* s_q0 = (int*)(smem + L.q0);
  int* s_nq = (int*)(smem + L.nq);
  int* s_slot = (int*)(smem + L.slot);
  int8_t* scall = (int8_t*)(smem + L.call);
  double p[kMaxD];
#pragma unroll
  for (int i = 0; i < kMaxD; ++i) p[i] = set_params[(size_t)set * kMaxD + i];
  const int nv = P.n_slots * 32;
  for (int i = threadIdx.x; i < kMcWarps * nv; i += blockDim.x) wacc[i] = 0.0;
  if constexpr (SCHEME == SABR_MC_BESSEL) {
    build_steps_bessel<R>(P, p, (StepCoefB<R>*)tab, land);
  } else {
    build_steps<R>(P, p, tab, land);
  }
  for (int q = threadIdx.x; q < P.n_quotes; q += blockDim.x) {
    sK[q] = (R)P.K[q];
    scall[q] = P.is_call[q];
  }
  for (int m = threadIdx.x; m < P.n_mats; m += blockDim.x) {
    s_q0[m] = P.mat_q0[m];
    s_nq[m] = P.mat_nq[m];
    s_slot[m] = P.mat_slot[m];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  const int64_t gblocks = grid_total > 0 ? grid_total : gridDim.x;
  const int64_t path0 = (int64_t)(block0 + blockIdx.x) * blockDim.x + threadIdx.x;
  double* my_acc = wacc + (size_t)warp * nv;
  if constexpr (SCHEME == SABR_MC_BESSEL) {
    const StepCoefB<R>* tb = (const StepCoefB<R>*)tab;
    if (p[1] == 1.0) {
      simulate_paths_bessel<R, true>(P, p, tb, land, s_q0, s_nq, s_slot, sK, scall, path0, gblocks * blockDim.x,
                                     my_acc);
    } else {
      simulate_paths_bessel<R, false>(P, p, tb, land, s_q0, s_nq, s_slot, sK, scall, path0, gblocks * blockDim.x,
                                      my_acc);
    }
  } else {
    simulate_paths<R>(P, p, tab, land, s_q0, s_nq, s_slot, sK, scall, path0, gblocks * blockDim.x, my_acc);
  }
  __syncthreads();
  double* out = partial + ((size_t)set * gridDim.x + blockIdx.x) * nv;
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kMcWarps; ++w) s += wacc[(size_t)w * nv + v];
    out[v] = s;
  }
}

// One thread per (set, option): fixed-order sum over blocks, eq. (payoff).
__global__ void mc_reduce_kernel(McDev P, int n_sets, int blocks_per_set, const double* __restrict__ partial,
                                 const int* __restrict__ q_value, const int* __restrict__ q_out,
                                 const double* __restrict__ disc, const int* __restrict__ set_valid,
                                 double* __restrict__ price, double* __restrict__ se, int out_stride) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_sets * P.n_quotes) return;
  const int set = idx / P.n_quotes, q = idx % P.n_quotes;
  if (set_valid && !set_valid[set]) return;
  const int nv = P.n_slots * 32;
  const int v = q_value[q];
  double s = 0.0, s2 = 0.0;
  for (int b = 0; b < blocks_per_set; ++b) {
    const double* part = partial + ((size_t)set * blocks_per_set + b) * nv;
    s += part[v];
    s2 += part[v + 1];
  }
  const double N = (double)P.n_paths;
  const double mean = s / N;
  double var = (s2 - s * mean) / (N - 1.0);
  if (var < 0.0) var = 0.0;
  const double D = disc[q];
  price[(size_t)set * out_stride + q_out[q]] = D * mean;
  if (se) se[(size_t)set * out_stride + q_out[q]] = D * sqrt(var / N);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
sabr_status mc_prepare(int model, double fwd, const double* T, const double* K, const int8_t* is_call,
                       const double* discount, int64_t n, int64_t n_paths, double spy, uint64_t seed,
                       int prec, McHost& h) {
  if (n_params(model) < 0) return fail(SABR_EINVAL, "unknown model");
  if (prec != SABR_FP32 && prec != SABR_FP64) return fail(SABR_EINVAL, "unknown precision");
  if (!(fwd > 0.0) || !std::isfinite(fwd)) return fail(SABR_EINVAL, "fwd must be > 0");
  if (n < 1 || n > kMaxMcQuotes) return fail(SABR_EINVAL, "number of options must lie in [1, 512]");
  if (!T || !K) return fail(SABR_EINVAL, "NULL option array");
  if (n_paths < 2 || n_paths > ((int64_t)1 << 31)) return fail(SABR_EINVAL, "n_paths must lie in [2, 2^31]");
  if (!(spy > 0.0) || !std::isfinite(spy)) return fail(SABR_EINVAL, "steps_per_year must be > 0");
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) {
    if (!(T[i] > 0.0) || !std::isfinite(T[i])) return fail(SABR_EINVAL, "maturities must be > 0");
    if (!(K[i] >= 0.0) || !std::isfinite(K[i])) return fail(SABR_EINVAL, "strikes must be >= 0");
    if (discount && !std::isfinite(discount[i])) return fail(SABR_EINVAL, "non-finite discount");
    order[i] = i;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return T[a] < T[b]; });
  h.model = model;
  h.prec = prec;
  h.fwd = fwd;
  h.n_paths = n_paths;
  h.seed = seed;
  h.n_quotes = (int)n;
  h.K.resize(n);
  h.call.resize(n);
  h.disc.resize(n);
  h.q_out.resize(n);
  h.q_value.resize(n);
  h.mats.clear();
  h.mat_q0.clear();
  h.mat_nq.clear();
  h.mat_slot.clear();
  int slots = 0;
  for (int s = 0; s < n; ++s) {
    const int i = order[s];
    if (h.mats.empty() || T[i] != h.mats.back()) {
      if (!h.mats.empty()) slots += (2 * h.mat_nq.back() + 31) / 32;
      h.mats.push_back(T[i]);
      h.mat_q0.push_back(s);
      h.mat_nq.push_back(0);
      h.mat_slot.push_back(slots);
    }
    const int pos = h.mat_nq.back()++;
    h.K[s] = K[i];
    h.call[s] = is_call ? (is_call[i] != 0) : 1;
    h.disc[s] = discount ? discount[i] : 1.0;
    h.q_out[s] = i;
    h.q_value[s] = h.mat_slot.back() * 32 + 2 * pos;
  }
  slots += (2 * h.mat_nq.back() + 31) / 32;
  h.n_slots = slots;
  if ((int)h.mats.size() > kMaxMats) return fail(SABR_EINVAL, "more than 64 distinct maturities");
  // grid: multiples of 1/spy below the last maturity with every maturity
  // inserted; a multiple within 1e-10 of a maturity is that maturity.
  h.step_t.clear();
  h.step_h.clear();
  h.step_mat.clear();
  double prev = 0.0;
  int64_t k = 1;
  for (size_t m = 0; m < h.mats.size(); ++m) {
    const double Tm = h.mats[m];
    while ((double)k / spy < Tm - 1e-10) {
      const double t = (double)k / spy;
      h.step_t.push_back(t);
      h.step_h.push_back(t - prev);
      h.step_mat.push_back(-1);
      prev = t;
      ++k;
      if ((int64_t)h.step_t.size() > kMaxMcSteps) return fail(SABR_EINVAL, "more than 8192 time steps");
    }
    h.step_t.push_back(Tm);
    h.step_h.push_back(Tm - prev);
    h.step_mat.push_back((int)m);
    prev = Tm;
    if (std::fabs((double)k / spy - Tm) <= 1e-10) ++k;
  }
  h.n_steps = (int)h.step_t.size();
  if (h.n_steps > kMaxMcSteps) return fail(SABR_EINVAL, "more than 8192 time steps");
  h.Tmax = h.mats.back();
  const size_t smem = prec == SABR_FP64
                          ? mc_smem_layout<double>(h.n_steps, h.n_quotes, (int)h.mats.size(), h.n_slots).total
                          : mc_smem_layout<float>(h.n_steps, h.n_quotes, (int)h.mats.size(), h.n_slots).total;
  if (smem > 220 * 1024) return fail(SABR_EINVAL, "too many time steps and options for one launch");
  h.smem = smem;
  return SABR_OK;
}

// Device image of an McHost: sizes and offsets in one buffer.
size_t mc_image_bytes(const McHost& h) {
  const size_t Q = h.n_quotes, M = h.mats.size(), S = h.n_steps;
  return 16 * 12 + 8 * (2 * S + 2 * Q) + 4 * (S + 3 * M + 2 * Q) + Q + 256;
}

void mc_fill_image(const McHost& h, unsigned char* host_img, unsigned char* dev_base, McDev& d, int** q_value,
                   int** q_out, double** disc) {
  size_t o = 0;
  auto put = [&](const void* src, size_t bytes) {
    o = (o + 15) & ~(size_t)15;
    std::memcpy(host_img + o, src, bytes);
    unsigned char* p = dev_base + o;
    o += bytes;
    return p;
  };
  d.model = h.model;
  d.n_quotes = h.n_quotes;
  d.n_mats = (int)h.mats.size();
  d.n_steps = h.n_steps;
  d.n_slots = h.n_slots;
  d.n_paths = h.n_paths;
  d.fwd = h.fwd;
  d.log_absorb = std::log(1e-12 * h.fwd);
  d.key0 = (uint32_t)h.seed;
  d.key1 = (uint32_t)(h.seed >> 32);
  for (int r = 0; r < 10; ++r) {  // Philox round keys (key schedule of Salmon et al.)
    d.rk.k0[r] = d.key0 + (uint32_t)r * 0x9E3779B9u;
    d.rk.k1[r] = d.key1 + (uint32_t)r * 0xBB67AE85u;
  }
  d.step_t = (const double*)put(h.step_t.data(), 8 * h.step_t.size());
  d.step_h = (const double*)put(h.step_h.data(), 8 * h.step_h.size());
  d.step_mat = (const int*)put(h.step_mat.data(), 4 * h.step_mat.size());
  d.mat_q0 = (const int*)put(h.mat_q0.data(), 4 * h.mat_q0.size());
  d.mat_nq = (const int*)put(h.mat_nq.data(), 4 * h.mat_nq.size());
  d.mat_slot = (const int*)put(h.mat_slot.data(), 4 * h.mat_slot.size());
  d.K = (const double*)put(h.K.data(), 8 * h.K.size());
  d.is_call = (const int8_t*)put(h.call.data(), h.call.size());
  *q_value = (int*)put(h.q_value.data(), 4 * h.q_value.size());
  *q_out = (int*)put(h.q_out.data(), 4 * h.q_out.size());
  *disc = (double*)put(h.disc.data(), 8 * h.disc.size());
}

using McPathsFn = void (*)(McDev, const double*, const int*, double*, int, int);

// The path kernel of a problem's precision and scheme, with its dynamic
// shared memory allowance raised to what the problem needs.
static McPathsFn mc_paths_fn(const McHost& h) {
  McPathsFn fn;
  if (h.prec == SABR_FP64) {
    fn = h.scheme == SABR_MC_BESSEL ? mc_paths_kernel<double, SABR_MC_BESSEL> : mc_paths_kernel<double, SABR_MC_LOG_EULER>;
  } else {
    fn = h.scheme == SABR_MC_BESSEL ? mc_paths_kernel<float, SABR_MC_BESSEL> : mc_paths_kernel<float, SABR_MC_LOG_EULER>;
  }
  cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h.smem);
  return fn;
}

// Paths one thread takes at a time.
static int mc_thread_paths(const McHost& h) {
  return h.scheme == SABR_MC_BESSEL ? kBesselPathsPerThread : mc_paths_per_thread(h.prec);
}

// Blocks per parameter set.  Every block of a launch does the same work
// (n_paths / blocks-per-set paths), so with R resident blocks a launch of
// n_sets x p blocks takes ceil(n_sets p / R) rounds of a block's time, which
// is proportional to 1/p: p minimises ceil(n_sets p / R) / p over p up to
// what the paths need (each thread takes kMcPathsPerThread paths at a time)
// and up to 8 rounds.  One set: p = R, one round, grid-stride.  256 sets on
// 760 resident blocks: p = 8 (3 rounds, 0.375) instead of p = 2 (one round
// with a third of the GPU idle, 0.5).
int mc_blocks_per_set(const McHost& h, int n_sets) {
  int per_sm = 8;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mc_paths_fn(h), kMcBlock, h.smem);
  per_sm = std::min(std::max(per_sm, 1), 8);
  const int64_t resident = device_sms() * (int64_t)per_sm;
  const int64_t sets = std::max(1, n_sets);
  const int64_t per_block = (int64_t)kMcBlock * mc_thread_paths(h);
  const int64_t by_paths = (h.n_paths + per_block - 1) / per_block;
  const int64_t p_max = std::max<int64_t>(1, std::min(by_paths, 8 * resident / sets));
  int64_t best = 1;
  double best_cost = 1e300;
  for (int64_t p = 1; p <= p_max; ++p) {
    const double cost = (double)((sets * p + resident - 1) / resident) / (double)p;
    if (cost < best_cost * (1.0 - 1e-12)) {
      best_cost = cost;
      best = p;
    }
  }
  return (int)best;
}

static void launch_paths(const McHost& h, const McDev& d, const double* set_params, const int* set_valid,
                         dim3 grid, double* partial, int block0, int grid_total, cudaStream_t s) {
  mc_paths_fn(h)<<<grid, kMcBlock, h.smem, s>>>(d, set_params, set_valid, partial, block0, grid_total);
}

sabr_status mc_launch(const McHost& h, const McDev& d, const double* set_params, const int* set_valid, int n_sets,
                      int blocks_per_set, double* partial, const int* q_value, const int* q_out,
                      const double* disc, double* price, double* se, int out_stride, cudaStream_t s) {
  launch_paths(h, d, set_params, set_valid, dim3(blocks_per_set, n_sets), partial, 0, 0, s);
  const int total = n_sets * h.n_quotes;
  mc_reduce_kernel<<<(total + 127) / 128, 128, 0, s>>>(d, n_sets, blocks_per_set, partial, q_value, q_out, disc,
                                                       set_valid, price, se, out_stride);
  SABR_CUDA(cudaGetLastError());
  return SABR_OK;
}

// Library-owned scratch of sabr_mc_price, one per device, reused by every
// call on that device (calls are serialised by a mutex and by waiting for the
// previous call's kernels before the scratch is rewritten).
struct McWorkspace {
  void* dev = nullptr;
  size_t dev_bytes = 0;
  unsigned char* host = nullptr;
  size_t host_bytes = 0;
  cudaEvent_t done = nullptr;
};
static std::mutex g_mc_mutex;
static std::vector<McWorkspace> g_mc_ws;

static sabr_status ensure_ws(McWorkspace& w, size_t dev_bytes, size_t host_bytes) {
  if (!w.done) SABR_CUDA(cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming));
  SABR_CUDA(cudaEventSynchronize(w.done));
  if (w.dev_bytes < dev_bytes) {
    if (w.dev) cudaFree(w.dev);
    w.dev = nullptr;
    w.dev_bytes = 0;
    SABR_CUDA(cudaMalloc(&w.dev, dev_bytes));
    w.dev_bytes = dev_bytes;
  }
  if (w.host_bytes < host_bytes) {
    if (w.host) cudaFreeHost(w.host);
    w.host = nullptr;
    w.host_bytes = 0;
    SABR_CUDA(cudaMallocHost(&w.host, host_bytes));
    w.host_bytes = host_bytes;
  }
  return SABR_OK;
}

}  // namespace sabr

namespace sabr {

static sabr_status mc_price(sabr_model model, const double* params, double fwd, const double* T, const double* K,
                            const int8_t* is_call, const double* discount, int64_t n, int64_t n_paths,
                            double steps_per_year, uint64_t seed, int scheme, double* price_out, double* stderr_out,
                            sabr_precision prec, void* stream) {
  SABR_TRY(check_params(model, params));
  if (!price_out) return fail(SABR_EINVAL, "price_out is NULL");
  if (scheme != SABR_MC_LOG_EULER && scheme != SABR_MC_BESSEL) return fail(SABR_EINVAL, "unknown path scheme");
  McHost h;
  SABR_TRY(mc_prepare(model, fwd, T, K, is_call, discount, n, n_paths, steps_per_year, seed, prec, h));
  h.scheme = scheme;
  if (model == SABR_DYN_II && !case2_feasible<double, double>(params, h.Tmax))
    return fail(SABR_EINVAL, "parameters violate rho(t) in [-1,1], nu(t) > 0");
  const int bps = mc_blocks_per_set(h, 1);
  const size_t img = mc_image_bytes(h);
  const size_t params_off = (img + 255) & ~(size_t)255;
  const size_t part_off = params_off + 256;
  const size_t dev_bytes = part_off + sizeof(double) * (size_t)bps * h.n_slots * 32;
  std::lock_guard<std::mutex> lock(g_mc_mutex);
  int dev = 0;
  SABR_CUDA(cudaGetDevice(&dev));
  if ((int)g_mc_ws.size() <= dev) g_mc_ws.resize(dev + 1);
  McWorkspace& w = g_mc_ws[dev];
  SABR_TRY(ensure_ws(w, dev_bytes, part_off));
  McDev d;
  int* q_value;
  int* q_out;
  double* disc;
  unsigned char* base = (unsigned char*)w.dev;
  mc_fill_image(h, w.host, base, d, &q_value, &q_out, &disc);
  double p10[kMaxD];
  for (int i = 0; i < kMaxD; ++i) p10[i] = i < n_params(model) ? params[i] : 0.0;
  std::memcpy(w.host + params_off, p10, sizeof(p10));
  cudaStream_t s = (cudaStream_t)stream;
  SABR_CUDA(cudaMemcpyAsync(w.dev, w.host, part_off, cudaMemcpyHostToDevice, s));
  SABR_TRY(mc_launch(h, d, (const double*)(base + params_off), nullptr, 1, bps, (double*)(base + part_off), q_value,
                     q_out, disc, price_out, stderr_out, (int)n, s));
  SABR_CUDA(cudaEventRecord(w.done, s));
  return SABR_OK;
}

}  // namespace sabr

extern "C" sabr_status sabr_mc_price(sabr_model model, const double* params, double fwd, const double* T,
                                     const double* K, const int8_t* is_call, const double* discount, int64_t n,
                                     int64_t n_paths, double steps_per_year, uint64_t seed, double* price_out,
                                     double* stderr_out, sabr_precision prec, void* stream) {
  sabr::clear_error();
  return sabr::mc_price(model, params, fwd, T, K, is_call, discount, n, n_paths, steps_per_year, seed,
                        SABR_MC_LOG_EULER, price_out, stderr_out, prec, stream);
}

extern "C" sabr_status sabr_mc_price_scheme(sabr_model model, const double* params, double fwd, const double* T,
                                            const double* K, const int8_t* is_call, const double* discount,
                                            int64_t n, int64_t n_paths, double steps_per_year, uint64_t seed,
                                            sabr_mc_scheme scheme, double* price_out, double* stderr_out,
                                            sabr_precision prec, void* stream) {
  sabr::clear_error();
  return sabr::mc_price(model, params, fwd, T, K, is_call, discount, n, n_paths, steps_per_year, seed, (int)scheme,
                        price_out, stderr_out, prec, stream);
}

// ---------------------------------------------------------------------------
// Path sharding (the multi-GPU form of the Sec. 4 pricer): the grid of
// sabr_mc_price split into block ranges, one per device; the per-block FP64
// partial sums, gathered in block order, reduce to the unsharded prices bit
// for bit.
// ---------------------------------------------------------------------------
namespace sabr {

struct McShardCall {
  McHost h;
  int total_blocks = 0;
};

static sabr_status mc_shard_prepare(sabr_model model, const double* params, double fwd, const double* T,
                                    const double* K, const int8_t* is_call, const double* discount, int64_t n,
                                    int64_t n_paths, double spy, uint64_t seed, sabr_precision prec, McShardCall& c) {
  SABR_TRY(check_params(model, params));
  SABR_TRY(mc_prepare(model, fwd, T, K, is_call, discount, n, n_paths, spy, seed, prec, c.h));
  if (model == SABR_DYN_II && !case2_feasible<double, double>(params, c.h.Tmax))
    return fail(SABR_EINVAL, "parameters violate rho(t) in [-1,1], nu(t) > 0");
  c.total_blocks = mc_blocks_per_set(c.h, 1);
  return SABR_OK;
}

// Uploads the tables and parameters into the per-device workspace; returns
// the device image and the workspace (whose `done` event the caller records).
static sabr_status mc_shard_upload(const McShardCall& c, const double* params, cudaStream_t s, McDev& d,
                                   int** q_value, int** q_out, double** disc, const double** dparams,
                                   McWorkspace** ws) {
  const size_t img = mc_image_bytes(c.h);
  const size_t params_off = (img + 255) & ~(size_t)255;
  const size_t part_off = params_off + 256;
  int dev = 0;
  SABR_CUDA(cudaGetDevice(&dev));
  if ((int)g_mc_ws.size() <= dev) g_mc_ws.resize(dev + 1);
  McWorkspace& w = g_mc_ws[dev];
  SABR_TRY(ensure_ws(w, part_off, part_off));
  unsigned char* base = (unsigned char*)w.dev;
  mc_fill_image(c.h, w.host, base, d, q_value, q_out, disc);
  double p10[kMaxD];
  for (int i = 0; i < kMaxD; ++i) p10[i] = i < n_params(c.h.model) ? params[i] : 0.0;
  std::memcpy(w.host + params_off, p10, sizeof(p10));
  SABR_CUDA(cudaMemcpyAsync(w.dev, w.host, part_off, cudaMemcpyHostToDevice, s));
  *dparams = (const double*)(base + params_off);
  *ws = &w;
  return SABR_OK;
}

}  // namespace sabr

extern "C" sabr_status sabr_mc_shard_layout(sabr_model model, const double* params, double fwd, const double* T,
                                            const double* K, const int8_t* is_call, const double* discount,
                                            int64_t n, int64_t n_paths, double steps_per_year, uint64_t seed,
                                            sabr_precision prec, int32_t* total_blocks,
                                            int64_t* doubles_per_block) {
  using namespace sabr;
  clear_error();
  if (!total_blocks || !doubles_per_block) return fail(SABR_EINVAL, "NULL output");
  McShardCall c;
  SABR_TRY(mc_shard_prepare(model, params, fwd, T, K, is_call, discount, n, n_paths, steps_per_year, seed, prec, c));
  *total_blocks = c.total_blocks;
  *doubles_per_block = (int64_t)c.h.n_slots * 32;
  return SABR_OK;
}

extern "C" sabr_status sabr_mc_shard_partials(sabr_model model, const double* params, double fwd, const double* T,
                                              const double* K, const int8_t* is_call, const double* discount,
                                              int64_t n, int64_t n_paths, double steps_per_year, uint64_t seed,
                                              sabr_precision prec, int32_t total_blocks, int32_t block_begin,
                                              int32_t block_count, double* partials_out, void* stream) {
  using namespace sabr;
  clear_error();
  if (!partials_out) return fail(SABR_EINVAL, "partials_out is NULL");
  std::lock_guard<std::mutex> lock(g_mc_mutex);
  McShardCall c;
  SABR_TRY(mc_shard_prepare(model, params, fwd, T, K, is_call, discount, n, n_paths, steps_per_year, seed, prec, c));
  if (total_blocks < 1 || block_count < 1 || block_begin < 0 || (int64_t)block_begin + block_count > total_blocks)
    return fail(SABR_EINVAL, "block range outside [0, total_blocks)");
  cudaStream_t s = (cudaStream_t)stream;
  McDev d;
  int *q_value, *q_out;
  double* disc;
  const double* dp;
  McWorkspace* w;
  SABR_TRY(mc_shard_upload(c, params, s, d, &q_value, &q_out, &disc, &dp, &w));
  launch_paths(c.h, d, dp, nullptr, dim3(block_count, 1), partials_out, block_begin, total_blocks, s);
  SABR_CUDA(cudaGetLastError());
  SABR_CUDA(cudaEventRecord(w->done, s));
  return SABR_OK;
}

extern "C" sabr_status sabr_mc_shard_reduce(sabr_model model, const double* params, double fwd, const double* T,
                                            const double* K, const int8_t* is_call, const double* discount,
                                            int64_t n, int64_t n_paths, double steps_per_year, uint64_t seed,
                                            sabr_precision prec, int32_t total_blocks, const double* partials,
                                            double* price_out, double* stderr_out, void* stream) {
  using namespace sabr;
  clear_error();
  if (!partials || !price_out) return fail(SABR_EINVAL, "NULL partials or price_out");
  std::lock_guard<std::mutex> lock(g_mc_mutex);
  McShardCall c;
  SABR_TRY(mc_shard_prepare(model, params, fwd, T, K, is_call, discount, n, n_paths, steps_per_year, seed, prec, c));
  if (total_blocks < 1) return fail(SABR_EINVAL, "total_blocks must be >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  McDev d;
  int *q_value, *q_out;
  double* disc;
  const double* dp;
  McWorkspace* w;
  SABR_TRY(mc_shard_upload(c, params, s, d, &q_value, &q_out, &disc, &dp, &w));
  mc_reduce_kernel<<<(c.h.n_quotes + 127) / 128, 128, 0, s>>>(d, 1, total_blocks, partials, q_value, q_out, disc,
                                                               nullptr, price_out, stderr_out, (int)n);
  SABR_CUDA(cudaGetLastError());
  SABR_CUDA(cudaEventRecord(w->done, s));
  return SABR_OK;
}
