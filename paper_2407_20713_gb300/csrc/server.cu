// server.cu -- continuous-batching calibration server (see include/sabr.h).
//
// One worker thread runs steps.  A step (1) admits queued requests while the
// device pool and max_active allow, uploading each into its own pool region
// and computing f(x0); (2) writes a work table -- one entry (request, block,
// level) per 256-thread block of every resident formula request -- and
// launches one persistent SA-level kernel per (precision, model) over it;
// (3) advances every resident MC-cost request by one proposal wave on a
// second stream; (4) enqueues the final reduction of requests that ran their
// last level and releases those the GPU has finished.  Requests arriving
// while others run therefore share the next launches.  No device code waits
// on anything; all waiting is host-side with time limits.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.h"
#include "engine_host.h"
#include "mcsa_host.h"

namespace sabr {

constexpr int kGroups = 10;            // (precision, model) pairs
constexpr int kWorkPerGroup = 4096;    // work-table entries per group per step

static int group_of(int prec, int model) { return prec * 5 + model; }

// First-fit allocator over [0, size) in 256-byte units.
class PoolAlloc {
 public:
  void init(size_t n) {
    free_.clear();
    free_[0] = n;
    used_ = 0;
  }
  bool alloc(size_t n, size_t* off) {
    n = (n + 255) & ~(size_t)255;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const size_t rest = it->second - n, o = it->first + n;
        free_.erase(it);
        if (rest) free_[o] = rest;
        used_ += n;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = (n + 255) & ~(size_t)255;
    used_ -= n;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0;
};

enum { R_QUEUED, R_ACTIVE, R_FINISHING, R_DONE, R_CANCELLED };

struct Request {
  uint64_t ticket = 0;
  int state = R_QUEUED;
  bool is_mc = false;
  bool cancel = false;
  bool cancelled_resident = false;
  HostProblem hp;
  McSaHost mh;
  int G = 1, n_blocks = 0;
  size_t bytes = 0, off = 0;
  int slot = -1;
  ProblemDev pd;
  int level = 0;
  int mc_level = 0, mc_step = 0;
  bool mc_started = false;
  cudaEvent_t wave_ev = nullptr;  // last MC wave
  cudaEvent_t done_ev = nullptr;
  sabr_result result;
};

}  // namespace sabr

struct sabr_server {
  sabr_server_config cfg;
  int device = 0;
  cudaStream_t sf = nullptr, smc = nullptr;
  unsigned char* pool = nullptr;
  sabr::PoolAlloc alloc;
  sabr::ProblemDev* d_probs = nullptr;
  sabr_result* d_results = nullptr;
  sabr_result* h_results = nullptr;
  int* d_ident = nullptr;
  int4* d_work[2] = {nullptr, nullptr};
  int* d_nwork[2] = {nullptr, nullptr};
  int4* h_work[2] = {nullptr, nullptr};
  int* h_nwork[2] = {nullptr, nullptr};
  cudaEvent_t buf_ev[2] = {nullptr, nullptr};
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  size_t smem[sabr::kGroups] = {};
  int grid[sabr::kGroups] = {};
  std::vector<int> free_slots;

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<sabr::Request>> queue;
  std::vector<std::shared_ptr<sabr::Request>> active;
  std::unordered_map<uint64_t, std::shared_ptr<sabr::Request>> all;
  uint64_t next_ticket = 1;
  bool stop = false;
  sabr_server_stats stats;
  std::thread worker;
  int step_parity = 0;
};

namespace sabr {

static size_t server_smem(int prec, int model, int max_quotes) {
  // worst case over lane counts: 256 chains per block, and for the dynamic
  // models at most 512 maturity slices per block (G lanes per chain hold
  // its M maturities, with G >= M/2 rounded to a power of two, and G = 1
  // only for M <= 2)
  const size_t rs = prec == SABR_FP64 ? 8 : 4;
  size_t b = level_smem_bytes(prec, SABR_HAGAN, max_quotes, kMaxMats, 256);
  if (model == SABR_DYN_I || model == SABR_DYN_II) b += 512 * coef_stride(prec, model) * rs + 64;
  // the FP32 Case II term-structure rule at its largest
  if (model == SABR_DYN_II && prec == SABR_FP32) b += (size_t)kMaxC2Sub * (kC2Nodes + 1) * 16 + kMaxMats * 8 + 16;
  return b;
}

static void enqueue_step_launches(sabr_server* s, int par, cudaStream_t st) {
  cudaMemcpyAsync(s->d_nwork[par], s->h_nwork[par], sizeof(int) * kGroups, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(s->d_work[par], s->h_work[par], sizeof(int4) * kWorkPerGroup * kGroups, cudaMemcpyHostToDevice,
                  st);
  for (int g = 0; g < kGroups; ++g)
    launch_persistent(g / 5, g % 5, s->d_probs, s->d_work[par] + (size_t)g * kWorkPerGroup, s->d_nwork[par] + g,
                      s->grid[g], s->smem[g], st);
}

static sabr_status upload_formula(sabr_server* s, Request& r) {
  std::vector<unsigned char> img(r.bytes, 0);
  unsigned char* base = s->pool + r.off;
  formula_layout(r.hp, r.G, img.data(), base, 0, r.pd, s->d_results + r.slot);
  SABR_CUDA(cudaMemcpyAsync(base, img.data(), r.bytes, cudaMemcpyHostToDevice, s->sf));
  SABR_CUDA(cudaMemcpyAsync(s->d_probs + r.slot, &r.pd, sizeof(ProblemDev), cudaMemcpyHostToDevice, s->sf));
  launch_init(r.hp.prec, r.hp.model, s->d_probs, s->d_ident + r.slot, 1, init_smem_bytes(r.hp), s->sf);
  s->stats.kernel_launches += 1;
  SABR_CUDA(cudaGetLastError());
  return SABR_OK;
}

static sabr_status upload_mc(sabr_server* s, Request& r) {
  std::vector<unsigned char> img(r.bytes, 0);
  unsigned char* base = s->pool + r.off;
  mcsa_layout(r.mh, img.data(), base, 0, s->d_results + r.slot);
  SABR_CUDA(cudaMemcpyAsync(base, img.data(), r.bytes, cudaMemcpyHostToDevice, s->smc));
  return SABR_OK;
}

// One MC proposal wave (preceded by the start of the calibration on the
// first call); a level's last wave is followed by its restart.
static void mc_wave(sabr_server* s, Request& r) {
  const McSaHost& m = r.mh;
  if (!r.mc_started) {
    s->stats.kernel_launches += mcsa_enqueue_piece(m, s->smc, 0, 0, 0);
    r.mc_started = true;
  }
  if (r.mc_level < m.n_levels && m.chain_len > 0) {
    s->stats.kernel_launches += mcsa_enqueue_piece(m, s->smc, 1, r.mc_level, r.mc_step);
    if (++r.mc_step == m.chain_len) {
      s->stats.kernel_launches += mcsa_enqueue_piece(m, s->smc, 2, r.mc_level, 0);
      r.mc_step = 0;
      ++r.mc_level;
    }
  } else {
    r.mc_level = m.n_levels;
  }
  cudaEventRecord(r.wave_ev, s->smc);
}

static void release(sabr_server* s, Request& r) {
  if (r.slot >= 0) {
    s->alloc.release(r.off, r.bytes);
    s->free_slots.push_back(r.slot);
    r.slot = -1;
  }
  if (r.wave_ev) cudaEventDestroy(r.wave_ev);
  if (r.done_ev) cudaEventDestroy(r.done_ev);
  r.wave_ev = r.done_ev = nullptr;
}

static void worker_main(sabr_server* s) {
  cudaSetDevice(s->device);
  std::vector<std::shared_ptr<Request>> admitted;
  while (true) {
    admitted.clear();
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->queue.empty() && s->active.empty() && !s->stop)
        s->cv_work.wait_for(lk, std::chrono::milliseconds(2));
      if (s->stop) break;
      // admission by device memory and slots, in arrival order
      while (!s->queue.empty() && !s->free_slots.empty()) {
        auto r = s->queue.front();
        if (r->cancel) {
          s->queue.pop_front();
          r->state = R_CANCELLED;
          s->stats.cancelled++;
          s->cv_done.notify_all();
          continue;
        }
        size_t off;
        if (!s->alloc.alloc(r->bytes, &off)) break;
        s->queue.pop_front();
        r->off = off;
        r->slot = s->free_slots.back();
        s->free_slots.pop_back();
        r->state = R_ACTIVE;
        s->active.push_back(r);
        admitted.push_back(r);
        s->stats.admitted++;
      }
      s->stats.queued = (int32_t)s->queue.size();
      s->stats.active = (int32_t)s->active.size();
      s->stats.pool_bytes_in_use = (int64_t)s->alloc.used();
    }
    for (auto& r : admitted) {
      cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming);
      cudaEventCreateWithFlags(&r->wave_ev, cudaEventDisableTiming);
      if (r->is_mc)
        upload_mc(s, *r);
      else
        upload_formula(s, *r);
    }

    // ---- formula step ------------------------------------------------
    const int par = s->step_parity;
    cudaEventSynchronize(s->buf_ev[par]);  // the step that last used this buffer is done
    int counts[kGroups] = {0};
    std::vector<std::shared_ptr<Request>> snapshot;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      snapshot = s->active;
    }
    std::vector<Request*> to_finalize;
    bool any_formula = false;
    for (auto& rp : snapshot) {
      Request& r = *rp;
      if (r.is_mc || r.state != R_ACTIVE) continue;
      if (r.cancel) {
        r.cancelled_resident = true;
        to_finalize.push_back(&r);
        continue;
      }
      if (r.level < r.hp.n_levels) {
        const int g = group_of(r.hp.prec, r.hp.model);
        if (counts[g] + r.n_blocks > kWorkPerGroup) continue;  // waits for the next step
        for (int b = 0; b < r.n_blocks; ++b)
          s->h_work[par][(size_t)g * kWorkPerGroup + counts[g] + b] = make_int4(r.slot, b, r.level, 0);
        counts[g] += r.n_blocks;
        ++r.level;
        any_formula = true;
      }
      if (r.level >= r.hp.n_levels) to_finalize.push_back(&r);
    }
    if (any_formula) {
      for (int g = 0; g < kGroups; ++g) s->h_nwork[par][g] = counts[g];
      if (s->graph[par]) {
        cudaGraphLaunch(s->graph[par], s->sf);
        s->stats.kernel_launches += kGroups;
      } else {
        cudaMemcpyAsync(s->d_nwork[par], s->h_nwork[par], sizeof(int) * kGroups, cudaMemcpyHostToDevice, s->sf);
        for (int g = 0; g < kGroups; ++g) {
          if (!counts[g]) continue;
          cudaMemcpyAsync(s->d_work[par] + (size_t)g * kWorkPerGroup, s->h_work[par] + (size_t)g * kWorkPerGroup,
                          sizeof(int4) * counts[g], cudaMemcpyHostToDevice, s->sf);
          launch_persistent(g / 5, g % 5, s->d_probs, s->d_work[par] + (size_t)g * kWorkPerGroup,
                            s->d_nwork[par] + g, s->grid[g], s->smem[g], s->sf);
          s->stats.kernel_launches++;
        }
      }
      cudaEventRecord(s->buf_ev[par], s->sf);
      s->step_parity ^= 1;
      s->stats.steps++;
    }
    for (Request* r : to_finalize) {
      if (!r->cancelled_resident) {
        launch_finalize(r->hp.prec, r->hp.model, s->d_probs, s->d_ident + r->slot, 1, s->sf);
        s->stats.kernel_launches++;
        cudaMemcpyAsync(s->h_results + r->slot, s->d_results + r->slot, sizeof(sabr_result), cudaMemcpyDeviceToHost,
                        s->sf);
      }
      cudaEventRecord(r->done_ev, s->sf);
      r->state = R_FINISHING;
    }

    // ---- MC requests: one wave each, at most one wave in flight --------
    for (auto& rp : snapshot) {
      Request& r = *rp;
      if (!r.is_mc || r.state != R_ACTIVE) continue;
      if (cudaEventQuery(r.wave_ev) == cudaErrorNotReady) continue;
      if (r.cancel) {
        r.cancelled_resident = true;
        cudaEventRecord(r.done_ev, s->smc);
        r.state = R_FINISHING;
        continue;
      }
      if (r.mc_level < r.mh.n_levels) mc_wave(s, r);
      if (r.mc_level >= r.mh.n_levels) {
        if (!r.mc_started) mc_wave(s, r);
        s->stats.kernel_launches += mcsa_enqueue_piece(r.mh, s->smc, 3, 0, 0);
        cudaMemcpyAsync(s->h_results + r.slot, s->d_results + r.slot, sizeof(sabr_result), cudaMemcpyDeviceToHost,
                        s->smc);
        cudaEventRecord(r.done_ev, s->smc);
        r.state = R_FINISHING;
      }
    }

    // ---- retire finished requests -------------------------------------
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (size_t i = 0; i < s->active.size();) {
        Request& r = *s->active[i];
        if (r.state == R_FINISHING && cudaEventQuery(r.done_ev) == cudaSuccess) {
          if (r.cancelled_resident) {
            r.state = R_CANCELLED;
            s->stats.cancelled++;
          } else {
            r.result = s->h_results[r.slot];
            r.state = R_DONE;
            s->stats.completed++;
          }
          release(s, r);
          s->active.erase(s->active.begin() + i);
          s->cv_done.notify_all();
        } else {
          ++i;
        }
      }
      s->stats.active = (int32_t)s->active.size();
      s->stats.pool_bytes_in_use = (int64_t)s->alloc.used();
    }
    if (!any_formula) {
      // nothing to launch for the formula engine: avoid spinning while MC
      // waves or final reductions are in flight
      std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
  }
}

static void destroy_server(sabr_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  if (s->sf) cudaStreamSynchronize(s->sf);
  if (s->smc) cudaStreamSynchronize(s->smc);
  for (auto& kv : s->all) release(s, *kv.second);
  for (int p = 0; p < 2; ++p) {
    if (s->graph[p]) cudaGraphExecDestroy(s->graph[p]);
    if (s->buf_ev[p]) cudaEventDestroy(s->buf_ev[p]);
    if (s->h_work[p]) cudaFreeHost(s->h_work[p]);
    if (s->h_nwork[p]) cudaFreeHost(s->h_nwork[p]);
  }
  if (s->h_results) cudaFreeHost(s->h_results);
  if (s->pool) cudaFree(s->pool);
  if (s->sf) cudaStreamDestroy(s->sf);
  if (s->smc) cudaStreamDestroy(s->smc);
  delete s;
}

static sabr_status create_server(const sabr_server_config* cfg, sabr_server** out) {
  if (!cfg || !out) return fail(SABR_EINVAL, "NULL argument");
  *out = nullptr;
  if (cfg->device_bytes < (1 << 20)) return fail(SABR_EINVAL, "device_bytes must be >= 1 MiB");
  if (cfg->max_active < 1 || cfg->max_active > 4096) return fail(SABR_EINVAL, "max_active must lie in [1, 4096]");
  if (cfg->max_queue < 1) return fail(SABR_EINVAL, "max_queue must be >= 1");
  if (cfg->max_quotes < 1 || cfg->max_quotes > kMaxQuotes) return fail(SABR_EINVAL, "max_quotes must lie in [1, 4096]");
  sabr_server* s = new sabr_server();
  s->cfg = *cfg;
  std::memset(&s->stats, 0, sizeof(s->stats));
  cudaGetDevice(&s->device);
  const int A = cfg->max_active;
  const size_t tables = sizeof(ProblemDev) * A + sizeof(sabr_result) * A + sizeof(int) * A +
                        2 * (sizeof(int4) * kWorkPerGroup * kGroups + 256 * 2);
  cudaError_t e = cudaMalloc(&s->pool, (size_t)cfg->device_bytes + tables + 4096);
  if (e != cudaSuccess) {
    delete s;
    return cuda_fail(e, "cudaMalloc(server pool)");
  }
  unsigned char* t = s->pool + (((size_t)cfg->device_bytes + 255) & ~(size_t)255);
  auto carve = [&](size_t bytes) {
    unsigned char* r = t;
    t += (bytes + 255) & ~(size_t)255;
    return r;
  };
  s->d_probs = (ProblemDev*)carve(sizeof(ProblemDev) * A);
  s->d_results = (sabr_result*)carve(sizeof(sabr_result) * A);
  s->d_ident = (int*)carve(sizeof(int) * A);
  for (int p = 0; p < 2; ++p) {
    s->d_work[p] = (int4*)carve(sizeof(int4) * kWorkPerGroup * kGroups);
    s->d_nwork[p] = (int*)carve(sizeof(int) * kGroups);
  }
  s->alloc.init((size_t)cfg->device_bytes);
  std::vector<int> ident(A);
  for (int i = 0; i < A; ++i) ident[i] = i;
  e = cudaMemcpy(s->d_ident, ident.data(), sizeof(int) * A, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_results, sizeof(sabr_result) * A);
  for (int p = 0; p < 2 && e == cudaSuccess; ++p) {
    e = cudaMallocHost(&s->h_work[p], sizeof(int4) * kWorkPerGroup * kGroups);
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_nwork[p], sizeof(int) * kGroups);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->buf_ev[p], cudaEventDisableTiming);
    if (e == cudaSuccess) std::memset(s->h_nwork[p], 0, sizeof(int) * kGroups);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->sf, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->smc, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    destroy_server(s);
    return cuda_fail(e, "server set-up");
  }
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
  for (int g = 0; g < kGroups; ++g) {
    s->smem[g] = server_smem(g / 5, g % 5, cfg->max_quotes);
    set_engine_smem(g / 5, g % 5, s->smem[g]);
    s->grid[g] = sms * persistent_blocks_per_sm(g / 5, g % 5, s->smem[g]);
  }
  if (cfg->use_graph) {
    for (int p = 0; p < 2; ++p) {
      cudaGraph_t graph = nullptr;
      e = cudaStreamBeginCapture(s->sf, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        enqueue_step_launches(s, p, s->sf);
        e = cudaStreamEndCapture(s->sf, &graph);
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&s->graph[p], graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        destroy_server(s);
        return cuda_fail(e, "server graph capture");
      }
    }
  }
  for (int i = A - 1; i >= 0; --i) s->free_slots.push_back(i);
  s->worker = std::thread(worker_main, s);
  *out = s;
  return SABR_OK;
}

static sabr_status submit(sabr_server* s, const sabr_problem* pr, const sabr_bounds* b, const sabr_cooling* c,
                          uint64_t seed, uint64_t* ticket) {
  if (!s || !pr || !b || !c || !ticket) return fail(SABR_EINVAL, "NULL argument");
  auto r = std::make_shared<Request>();
  if (pr->cost == SABR_COST_MC_PRICE) {
    r->is_mc = true;
    SABR_TRY(mcsa_prepare(*pr, *b, *c, seed, r->mh));
    r->bytes = mcsa_arena_bytes(r->mh);
  } else {
    SABR_TRY(formula_prepare(*pr, *b, *c, seed, r->hp));
    if (r->hp.n_quotes > s->cfg.max_quotes) return fail(SABR_EINVAL, "request has more quotes than max_quotes");
    r->G = choose_lanes(r->hp.n_quotes, r->hp.n_mats, r->hp.model, r->hp.prec, r->hp.n_chains);
    ProblemDev tmp;
    r->bytes = formula_layout(r->hp, r->G, nullptr, nullptr, 0, tmp, nullptr) + 256;
    r->n_blocks = tmp.n_blocks;
    if (r->n_blocks > kWorkPerGroup) return fail(SABR_EINVAL, "request has too many chains for one step");
    const size_t need =
        level_smem_bytes(r->hp.prec, r->hp.model, r->hp.n_quotes, r->hp.n_mats, tmp.cpb, r->hp.c2_nsub);
    if (need > s->smem[group_of(r->hp.prec, r->hp.model)])
      return fail(SABR_EINVAL, "request needs more shared memory than the server reserves");
  }
  if (r->bytes > (size_t)s->cfg.device_bytes) return fail(SABR_EINVAL, "request larger than the server pool");
  std::lock_guard<std::mutex> lk(s->mu);
  if ((int)s->queue.size() >= s->cfg.max_queue) return fail(SABR_EBUSY, "server queue is full");
  r->ticket = s->next_ticket++;
  s->queue.push_back(r);
  s->all[r->ticket] = r;
  s->stats.submitted++;
  *ticket = r->ticket;
  s->cv_work.notify_one();
  return SABR_OK;
}

static sabr_status take_result(sabr_server* s, uint64_t ticket, sabr_result* out, bool* done) {
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return fail(SABR_ENOTFOUND, "unknown ticket");
  Request& r = *it->second;
  *done = false;
  if (r.state == R_DONE) {
    if (out) *out = r.result;
    s->all.erase(it);
    *done = true;
    return SABR_OK;
  }
  if (r.state == R_CANCELLED) {
    s->all.erase(it);
    *done = true;
    return fail(SABR_ECANCELLED, "request was cancelled");
  }
  return SABR_EAGAIN;
}

}  // namespace sabr

extern "C" {

sabr_status sabr_server_create(const sabr_server_config* config, sabr_server** out) {
  sabr::clear_error();
  return sabr::create_server(config, out);
}

sabr_status sabr_server_submit(sabr_server* server, const sabr_problem* problem, const sabr_bounds* bounds,
                               const sabr_cooling* cooling, uint64_t seed, uint64_t* ticket) {
  sabr::clear_error();
  return sabr::submit(server, problem, bounds, cooling, seed, ticket);
}

sabr_status sabr_server_poll(sabr_server* server, uint64_t ticket, sabr_result* out) {
  sabr::clear_error();
  if (!server) return sabr::fail(SABR_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(server->mu);
  bool done;
  return sabr::take_result(server, ticket, out, &done);
}

sabr_status sabr_server_wait(sabr_server* server, uint64_t ticket, int64_t timeout_ms, sabr_result* out) {
  sabr::clear_error();
  if (!server) return sabr::fail(SABR_EINVAL, "server is NULL");
  std::unique_lock<std::mutex> lk(server->mu);
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
  while (true) {
    bool done;
    sabr_status st = sabr::take_result(server, ticket, out, &done);
    if (st != SABR_EAGAIN) return st;
    if (timeout_ms >= 0) {
      if (server->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
        st = sabr::take_result(server, ticket, out, &done);
        if (st != SABR_EAGAIN) return st;
        return sabr::fail(SABR_ETIMEOUT, "request did not finish in time");
      }
    } else {
      server->cv_done.wait_for(lk, std::chrono::milliseconds(50));
    }
  }
}

sabr_status sabr_server_cancel(sabr_server* server, uint64_t ticket) {
  sabr::clear_error();
  if (!server) return sabr::fail(SABR_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(server->mu);
  auto it = server->all.find(ticket);
  if (it == server->all.end()) return sabr::fail(SABR_ENOTFOUND, "unknown ticket");
  sabr::Request& r = *it->second;
  if (r.state == sabr::R_QUEUED) {
    r.cancel = true;
    r.state = sabr::R_CANCELLED;
    for (size_t i = 0; i < server->queue.size(); ++i)
      if (server->queue[i]->ticket == ticket) {
        server->queue.erase(server->queue.begin() + i);
        break;
      }
    server->stats.cancelled++;
    server->cv_done.notify_all();
  } else if (r.state == sabr::R_ACTIVE) {
    r.cancel = true;
  }
  return SABR_OK;
}

sabr_status sabr_server_get_stats(sabr_server* server, sabr_server_stats* out) {
  sabr::clear_error();
  if (!server || !out) return sabr::fail(SABR_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(server->mu);
  *out = server->stats;
  return SABR_OK;
}

void sabr_server_destroy(sabr_server* server) { sabr::destroy_server(server); }

}  // extern "C"
