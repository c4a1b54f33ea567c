// mc_noalloc.cu -- sabr_mc_price_noalloc: Monte Carlo prices without any
// memory allocation by the library.
//
// Who needs it: callers that cannot let a library allocate device memory --
// processes whose device memory is handed out entirely by their own
// fixed-size pool (a cudaMalloc from the library would fail, or take memory
// the pool counts on), and applications whose rules forbid libraries to
// allocate.  sabr_mc_price keeps a growable per-device workspace
// (cudaMalloc / cudaMallocHost on first use and when it grows); this variant
// instead uses one fixed scratch array that is part of the library image.
//
// The scratch below is a file-scope __device__ array of kNoAllocScratchBytes
// (8 MiB).  Every GPU that loads the library holds it until the process
// exits.  In host code its name is only a host-side stand-in, not a device
// address, so its address is looked up once per device (cudaGetSymbolAddress,
// with that device current) on the first call on that device, and passed to
// the kernels.  All calls share the array and it keeps the last call's
// contents; each call rewrites every byte it reads (the option and step
// tables are copied in, every block writes all of its partial sums), so
// nothing needs clearing.  Calls whose work overlaps on the GPU (different
// streams, or different host threads on the same device without ordering)
// race on the array.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "common.h"
#include "mc_host.h"

namespace sabr {

constexpr size_t kNoAllocScratchBytes = 8u << 20;   // device scratch
constexpr size_t kNoAllocImageBytes = 256u << 10;   // option/step tables + params

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Host staging of the tables: static storage, rewritten under the mutex.
static unsigned char g_noalloc_host[kNoAllocImageBytes];
static std::mutex g_noalloc_mutex;
static void* g_noalloc_dev_ptr[64] = {nullptr};  // per device ordinal

static sabr_status noalloc_scratch(int dev, unsigned char** ptr) {
  if (dev < 0 || dev >= 64) return fail(SABR_EINVAL, "device ordinal out of range for the no-alloc scratch");
  if (!g_noalloc_dev_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    g_noalloc_dev_ptr[dev] = p;
  }
  *ptr = (unsigned char*)g_noalloc_dev_ptr[dev];
  return SABR_OK;
}

}  // namespace sabr

extern "C" sabr_status sabr_mc_price_noalloc(sabr_model model, const double* params, double fwd, const double* T,
                                             const double* K, const int8_t* is_call, const double* discount,
                                             int64_t n, int64_t n_paths, double steps_per_year, uint64_t seed,
                                             double* price_out, double* stderr_out, sabr_precision prec,
                                             void* stream) {
  using namespace sabr;
  clear_error();
  SABR_TRY(check_params(model, params));
  if (!price_out) return fail(SABR_EINVAL, "price_out is NULL");
  McHost h;
  SABR_TRY(mc_prepare(model, fwd, T, K, is_call, discount, n, n_paths, steps_per_year, seed, prec, h));
  if (model == SABR_DYN_II && !case2_feasible<double, double>(params, h.Tmax))
    return fail(SABR_EINVAL, "parameters violate rho(t) in [-1,1], nu(t) > 0");
  // a fixed grid (at most 1216 blocks), independent of the occupancy the
  // pricing kernel reaches, so the scratch bound below is a property of the
  // problem alone
  const int64_t per_block = (int64_t)kMcBlock * mc_paths_per_thread(h.prec);
  const int bps = (int)std::min<int64_t>(1216, (h.n_paths + per_block - 1) / per_block);
  const size_t img = mc_image_bytes(h);
  const size_t params_off = (img + 255) & ~(size_t)255;
  const size_t part_off = params_off + 256;
  const size_t need = part_off + sizeof(double) * (size_t)bps * h.n_slots * 32;
  if (part_off > kNoAllocImageBytes || need > kNoAllocScratchBytes)
    return fail(SABR_EINVAL,
                "problem too large for the 8 MiB no-alloc scratch (fewer options or steps, or use sabr_mc_price)");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  int dev = 0;
  SABR_CUDA(cudaGetDevice(&dev));
  unsigned char* base = nullptr;
  SABR_TRY(noalloc_scratch(dev, &base));
  McDev d;
  int* q_value;
  int* q_out;
  double* disc;
  mc_fill_image(h, g_noalloc_host, base, d, &q_value, &q_out, &disc);
  double p10[kMaxD];
  for (int i = 0; i < kMaxD; ++i) p10[i] = i < n_params(model) ? params[i] : 0.0;
  std::memcpy(g_noalloc_host + params_off, p10, sizeof(p10));
  cudaStream_t s = (cudaStream_t)stream;
  // pageable source: the copy has consumed g_noalloc_host when this returns
  // (the runtime may first wait for the stream's earlier work)
  SABR_CUDA(cudaMemcpyAsync(base, g_noalloc_host, part_off, cudaMemcpyHostToDevice, s));
  return mc_launch(h, d, (const double*)(base + params_off), nullptr, 1, bps, (double*)(base + part_off), q_value,
                   q_out, disc, price_out, stderr_out, (int)n, s);
}
