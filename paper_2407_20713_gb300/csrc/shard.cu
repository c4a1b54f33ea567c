// shard.cu -- chain-sharded calibration: the multi-GPU form of Technique I
// (Sec. 5.1).  The paper runs the chains of one calibration on several GPUs
// and, at the end of every temperature level, takes the minimum of the
// GPUs' minima on the host as the common restart point.  A shard here holds
// a contiguous range of a problem's chains on the current device; the
// caller exchanges each level's shard minima (any transport: a collective,
// host memory) and hands the overall minimum back.
//
// A sharded run equals the unsharded sabr_calibrate bit for bit:
//  * every chain draws its proposals from Philox counters keyed by its
//    global index;
//  * lanes per chain are chosen from the problem's total chain count, as
//    sabr_calibrate chooses them for the problem alone, so each chain's
//    misfit sums run in the same order;
//  * the level-end and best-ever minima are lexicographic in (cost, global
//    chain), which is what the unsharded block-then-grid argmin computes.
#include <cstring>

#include "common.h"
#include "engine.cuh"
#include "engine_host.h"

struct sabr_shard {
  int device = 0;
  sabr::HostProblem hp;
  sabr::ProblemDev pd{};
  void* arena = nullptr;
  sabr::ProblemDev* d_prob = nullptr;
  sabr_result* d_result = nullptr;
  int4* d_bmap = nullptr;
  int* d_plist = nullptr;
  size_t smem_level = 0, smem_init = 0;
  int next_level = 0;
  int finalized = 0;
};

namespace sabr {

static void free_shard(sabr_shard* s) {
  if (!s) return;
  if (s->arena) cudaFree(s->arena);
  delete s;
}

static sabr_status shard_create(const sabr_problem* pr, const sabr_bounds* b, const sabr_cooling* c, uint64_t seed,
                                int32_t chain_begin, int32_t chain_count, cudaStream_t st, sabr_shard** out) {
  if (!out) return fail(SABR_EINVAL, "out is NULL");
  *out = nullptr;
  if (!pr || !b || !c) return fail(SABR_EINVAL, "NULL argument");
  if (pr->cost != SABR_COST_VOL) return fail(SABR_EINVAL, "only implied-vol (Technique I) problems are sharded");
  if (chain_count < 1 || chain_begin < 0 || (int64_t)chain_begin + chain_count > pr->n_chains)
    return fail(SABR_EINVAL, "chain range outside [0, n_chains)");
  sabr_shard* s = new sabr_shard();
  cudaGetDevice(&s->device);
  sabr_status e = formula_prepare(*pr, *b, *c, seed, s->hp);
  if (e != SABR_OK) {
    free_shard(s);
    return e;
  }
  // lanes per chain as for the whole problem calibrated alone
  const int G = choose_lanes(s->hp.n_quotes, s->hp.n_mats, s->hp.model, s->hp.prec, s->hp.n_chains);
  s->hp.n_chains = chain_count;
  s->hp.chain0 = chain_begin;
  if (level_smem_bytes(s->hp.prec, s->hp.model, s->hp.n_quotes, s->hp.n_mats, kLevelBlock / G, s->hp.c2_nsub) >
      kMaxLevelSmem) {
    free_shard(s);
    return fail(SABR_EINVAL, "the quotes of the problem exceed one block's shared memory at its precision");
  }
  auto align = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t o_prob = 0, o_res = align(sizeof(ProblemDev));
  const size_t o_region = align(o_res + sizeof(sabr_result));
  ProblemDev dry;
  const size_t end = formula_layout(s->hp, G, nullptr, nullptr, o_region, dry, nullptr, kLevelBlock);
  const size_t o_bmap = align(end), o_plist = align(o_bmap + sizeof(int4) * dry.n_blocks);
  const size_t bytes = align(o_plist + sizeof(int));
  cudaError_t ce = cudaMalloc(&s->arena, bytes);
  if (ce != cudaSuccess) {
    free_shard(s);
    return cuda_fail(ce, "cudaMalloc(shard)");
  }
  unsigned char* base = (unsigned char*)s->arena;
  std::vector<unsigned char> img(bytes, 0);
  s->d_prob = (ProblemDev*)(base + o_prob);
  s->d_result = (sabr_result*)(base + o_res);
  formula_layout(s->hp, G, img.data(), base, o_region, s->pd, s->d_result, kLevelBlock);
  std::memcpy(img.data() + o_prob, &s->pd, sizeof(ProblemDev));
  std::vector<int4> bm(s->pd.n_blocks);
  for (int i = 0; i < s->pd.n_blocks; ++i) bm[i] = make_int4(0, i, 0, 0);
  std::memcpy(img.data() + o_bmap, bm.data(), sizeof(int4) * bm.size());
  s->d_bmap = (int4*)(base + o_bmap);
  s->d_plist = (int*)(base + o_plist);
  s->smem_level = level_smem_bytes(s->hp.prec, s->hp.model, s->hp.n_quotes, s->hp.n_mats, s->pd.cpb, s->hp.c2_nsub);
  s->smem_init = init_smem_bytes(s->hp);
  set_engine_smem(s->hp.prec, s->hp.model, std::max(s->smem_level, s->smem_init));
  ce = cudaMemcpyAsync(s->arena, img.data(), bytes, cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) {
    // f(x0) and T0, identical on every shard
    launch_init(s->hp.prec, s->hp.model, s->d_prob, s->d_plist, 1, s->smem_init, st);
    ce = cudaGetLastError();
  }
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) {
    free_shard(s);
    return cuda_fail(ce, "shard set-up");
  }
  *out = s;
  return SABR_OK;
}

static sabr_status read_point(sabr_shard* s, int chain_slot, sabr_chain_point* p, cudaStream_t st) {
  double state[kStateLen];
  SABR_CUDA(cudaMemcpyAsync(state, s->pd.state, sizeof(state), cudaMemcpyDeviceToHost, st));
  SABR_CUDA(cudaStreamSynchronize(st));
  p->f = state[kMaxD];
  p->chain = (int64_t)state[chain_slot];
  for (int i = 0; i < kMaxD; ++i) p->x[i] = state[i];
  return SABR_OK;
}

}  // namespace sabr

extern "C" {

sabr_status sabr_shard_create(const sabr_problem* problem, const sabr_bounds* bounds, const sabr_cooling* cooling,
                              uint64_t seed, int32_t chain_begin, int32_t chain_count, void* stream,
                              sabr_shard** out) {
  sabr::clear_error();
  return sabr::shard_create(problem, bounds, cooling, seed, chain_begin, chain_count, (cudaStream_t)stream, out);
}

sabr_status sabr_shard_level(sabr_shard* s, int32_t level, sabr_chain_point* local_min, void* stream) {
  using namespace sabr;
  clear_error();
  if (!s || !local_min) return fail(SABR_EINVAL, "NULL argument");
  if (level != s->next_level || level >= s->hp.n_levels || s->finalized)
    return fail(SABR_EINVAL, "levels run in order 0 .. n_levels-1, before the result");
  cudaStream_t st = (cudaStream_t)stream;
  launch_level(s->hp.prec, s->hp.model, s->d_prob, s->d_bmap, s->pd.n_blocks, level, s->smem_level, st);
  SABR_CUDA(cudaGetLastError());
  SABR_TRY(read_point(s, kStateArgChain, local_min, st));
  s->next_level = level + 1;
  return SABR_OK;
}

sabr_status sabr_shard_restart(sabr_shard* s, const sabr_chain_point* restart, void* stream) {
  using namespace sabr;
  clear_error();
  if (!s || !restart) return fail(SABR_EINVAL, "NULL argument");
  double head[kMaxD + 1];
  for (int i = 0; i < kMaxD; ++i) head[i] = restart->x[i];
  head[kMaxD] = restart->f;
  cudaStream_t st = (cudaStream_t)stream;
  SABR_CUDA(cudaMemcpyAsync(s->pd.state, head, sizeof(head), cudaMemcpyHostToDevice, st));
  SABR_CUDA(cudaStreamSynchronize(st));
  return SABR_OK;
}

sabr_status sabr_shard_result(sabr_shard* s, sabr_result* out, int64_t* best_chain, void* stream) {
  using namespace sabr;
  clear_error();
  if (!s || !out) return fail(SABR_EINVAL, "NULL argument");
  if (s->next_level != s->hp.n_levels) return fail(SABR_EINVAL, "not every level has run");
  cudaStream_t st = (cudaStream_t)stream;
  launch_finalize(s->hp.prec, s->hp.model, s->d_prob, s->d_plist, 1, st);
  SABR_CUDA(cudaGetLastError());
  SABR_CUDA(cudaMemcpyAsync(out, s->d_result, sizeof(sabr_result), cudaMemcpyDeviceToHost, st));
  sabr_chain_point bp;
  SABR_TRY(read_point(s, kStateBestChain, &bp, st));
  if (best_chain) *best_chain = bp.chain;
  s->finalized = 1;
  return SABR_OK;
}

void sabr_shard_destroy(sabr_shard* s) { sabr::free_shard(s); }

}  // extern "C"
