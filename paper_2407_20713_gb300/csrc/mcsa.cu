// mcsa.cu -- kernels and host enqueue of Technique II (see mcsa.cuh).
#include <cmath>
#include <cstring>

#include "common.h"
#include "mc_host.h"
#include "mcsa.cuh"
#include "mcsa_host.h"

namespace sabr {

__device__ __forceinline__ double misfit_prices(const double* __restrict__ price, const double* __restrict__ mkt,
                                                int n) {
  double s = 0.0;
  for (int q = 0; q < n; ++q) {
    const double r = (mkt[q] - price[q]) / mkt[q];
    s += r * r;
  }
  return s;
}

__device__ __forceinline__ bool feasible2(const double* x, double Tmax) {
  return case2_feasible<double, double>(x, Tmax);
}

// x0 -> one_params
__global__ void mcsa_start_kernel(McSaDev P) {
  if (threadIdx.x < kMaxD) P.one_params[threadIdx.x] = P.x0[threadIdx.x];
}

// f(x0), T0, and every chain's state.
__global__ void mcsa_init_kernel(McSaDev P) {
  __shared__ double f0s;
  if (threadIdx.x == 0) {
    const double f0 = misfit_prices(P.one_prices, P.mkt, P.n_quotes);
    f0s = f0;
    for (int i = 0; i < kMaxD; ++i) P.state[i] = P.x0[i];
    P.state[kMaxD] = f0;
    P.state[kMaxD + 1] = P.T0_given > 0.0 ? P.T0_given : (f0 > 0.0 ? f0 : 1.0);
    P.result->status = isfinite(f0) ? SABR_OK : SABR_EINVAL;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < P.n_chains; c += blockDim.x) {
    for (int i = 0; i < kMaxD; ++i) {
      P.cx[(size_t)c * kMaxD + i] = P.x0[i];
      P.bx[(size_t)c * kMaxD + i] = P.x0[i];
    }
    P.cf[c] = f0s;
    P.bf[c] = f0s;
    P.ev[c] = 0;
    P.ac[c] = 0;
  }
}

// u[0 .. d-1]: move uniforms, u[d]: acceptance uniform (sa_accept_word).
__device__ __forceinline__ void wave_uniforms(const McSaDev& P, int chain, int level, int st, double* u) {
  const int nb = sa_philox_blocks(P.d);
  uint32_t w0 = 0, w1 = 0, w2 = 0;
  for (int b = 0; b < nb; ++b) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)chain, (uint32_t)level, (uint32_t)st, kTagSA + (uint32_t)b),
                                  P.key0, P.key1);
    if (b == 0) {
      w0 = w.x;
      w1 = w.y;
      w2 = w.z;
    }
    u[4 * b + 0] = u01<double>(w.x);
    u[4 * b + 1] = u01<double>(w.y);
    u[4 * b + 2] = u01<double>(w.z);
    u[4 * b + 3] = u01<double>(w.w);
  }
  u[P.d] = u01<double>(sa_accept_word(w0, w1, w2));
}

__device__ __forceinline__ double level_step(const McSaDev& P, int level, double* Tk) {
  const double T0 = P.state[kMaxD + 1];
  *Tk = __dmul_rn(T0, P.ck[level]);
  double sk = __dmul_rn(P.step0, __dsqrt_rn(__ddiv_rn(*Tk, T0)));
  return sk < P.step_min ? P.step_min : sk;
}

// Proposal x' = x + s_k (hi - lo)(2u - 1) of every chain for (level, st).
__global__ void mcsa_propose_kernel(McSaDev P, int level, int st) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= P.n_chains) return;
  double Tk;
  const double sk = level_step(P, level, &Tk);
  double u[12];
  wave_uniforms(P, c, level, st, u);
  bool inside = true;
  double xp[kMaxD];
  for (int i = 0; i < kMaxD; ++i) {
    if (i < P.d) {
      const double step = __dmul_rn(sk, __dsub_rn(P.hi[i], P.lo[i]));
      xp[i] = __dadd_rn(P.cx[(size_t)c * kMaxD + i], __dmul_rn(step, __dsub_rn(__dmul_rn(2.0, u[i]), 1.0)));
      inside = inside && !(xp[i] < P.lo[i] || xp[i] > P.hi[i]);
    } else {
      xp[i] = 0.0;
    }
  }
  if (inside && P.model == SABR_DYN_II) inside = feasible2(xp, P.Tmax);
  for (int i = 0; i < kMaxD; ++i) P.set_params[(size_t)c * kMaxD + i] = xp[i];
  P.set_valid[c] = inside ? 1 : 0;
}

// Misfit of every evaluated proposal, best-ever update, Metropolis.
__global__ void mcsa_accept_kernel(McSaDev P, int level, int st) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= P.n_chains || !P.set_valid[c]) return;
  double Tk;
  level_step(P, level, &Tk);
  const double fp = misfit_prices(P.prices + (size_t)c * P.n_quotes, P.mkt, P.n_quotes);
  P.ev[c] += 1;
  if (!(fp == fp)) return;
  const double* xp = P.set_params + (size_t)c * kMaxD;
  if (fp < P.bf[c]) {
    P.bf[c] = fp;
    for (int i = 0; i < kMaxD; ++i) P.bx[(size_t)c * kMaxD + i] = xp[i];
  }
  const double delta = fp - P.cf[c];
  bool acc = delta <= 0.0;
  if (!acc) {
    double u[12];
    wave_uniforms(P, c, level, st, u);
    acc = u[P.d] < exp(-delta / Tk);
  }
  if (acc) {
    for (int i = 0; i < kMaxD; ++i) P.cx[(size_t)c * kMaxD + i] = xp[i];
    P.cf[c] = fp;
    P.ac[c] += 1;
  }
}

// Level end: every chain restarts from the lowest final state (lowest index
// on a tie).  One block.
__global__ void mcsa_restart_kernel(McSaDev P) {
  __shared__ double sf[256];
  __shared__ int si[256];
  __shared__ double win[kMaxD + 1];
  double f = INFINITY;
  int idx = 0x7fffffff;
  for (int c = threadIdx.x; c < P.n_chains; c += blockDim.x)
    if (P.cf[c] < f) {
      f = P.cf[c];
      idx = c;
    }
  sf[threadIdx.x] = f;
  si[threadIdx.x] = idx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double fb = INFINITY;
    int ib = 0x7fffffff;
    for (int t = 0; t < (int)blockDim.x; ++t)
      if (sf[t] < fb || (sf[t] == fb && si[t] < ib)) {
        fb = sf[t];
        ib = si[t];
      }
    for (int i = 0; i < kMaxD; ++i) win[i] = P.cx[(size_t)ib * kMaxD + i];
    win[kMaxD] = fb;
    for (int i = 0; i < kMaxD; ++i) P.state[i] = win[i];
    P.state[kMaxD] = fb;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < P.n_chains; c += blockDim.x) {
    for (int i = 0; i < kMaxD; ++i) P.cx[(size_t)c * kMaxD + i] = win[i];
    P.cf[c] = win[kMaxD];
  }
}

// Best over all chains -> result; the best point goes to one_params for the
// FP64 re-score.  One block.
__global__ void mcsa_final_kernel(McSaDev P) {
  __shared__ double sf[256];
  __shared__ int si[256];
  __shared__ unsigned long long se[256], sa[256];
  double f = INFINITY;
  int idx = 0x7fffffff;
  unsigned long long ev = 0, ac = 0;
  for (int c = threadIdx.x; c < P.n_chains; c += blockDim.x) {
    if (P.bf[c] < f) {
      f = P.bf[c];
      idx = c;
    }
    ev += P.ev[c];
    ac += P.ac[c];
  }
  sf[threadIdx.x] = f;
  si[threadIdx.x] = idx;
  se[threadIdx.x] = ev;
  sa[threadIdx.x] = ac;
  __syncthreads();
  if (threadIdx.x == 0) {
    double fb = INFINITY;
    int ib = 0x7fffffff;
    unsigned long long te = 0, ta = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      if (sf[t] < fb || (sf[t] == fb && si[t] < ib)) {
        fb = sf[t];
        ib = si[t];
      }
      te += se[t];
      ta += sa[t];
    }
    sabr_result* r = P.result;
    const bool none = P.n_levels == 0 || ib == 0x7fffffff;
    for (int i = 0; i < kMaxD; ++i) {
      const double v = none ? P.state[i] : P.bx[(size_t)ib * kMaxD + i];
      r->params[i] = v;
      P.one_params[i] = v;
      r->restart_params[i] = P.state[i];
    }
    r->misfit = none ? P.state[kMaxD] : fb;
    r->restart_misfit = P.state[kMaxD];
    r->n_evals = (int64_t)te;
    r->n_accepts = (int64_t)ta;
  }
}

__global__ void mcsa_rescore_kernel(McSaDev P) {
  if (threadIdx.x == 0) P.result->misfit_fp64 = misfit_prices(P.one_prices, P.mkt, P.n_quotes);
}

// ---------------------------------------------------------------------------
// Host
// ---------------------------------------------------------------------------
size_t mcsa_arena_bytes(const McSaHost& m) {
  // dry run of mcsa_layout from offset 0 (no image, no device base)
  McSaHost t = m;
  mcsa_layout(t, nullptr, nullptr, 0, nullptr);
  return t.end + 256;
}

void mcsa_layout(McSaHost& m, unsigned char* img, unsigned char* base, size_t off0, sabr_result* dres) {
  size_t o = off0;
  auto take = [&](size_t x) {
    o = (o + 255) & ~(size_t)255;
    size_t r = o;
    o += x;
    return r;
  };
  const size_t C = m.n_chains, Q = m.mc.n_quotes;
  const size_t nv = (size_t)m.mc.n_slots * 32;
  const bool write = img != nullptr;
  size_t o_mc = take(mc_image_bytes(m.mc));
  if (write) mc_fill_image(m.mc, img + o_mc, base + o_mc, m.dmc, &m.q_value, &m.q_out, &m.disc);
  size_t o_mc64 = take(mc_image_bytes(m.mc64));
  if (write) mc_fill_image(m.mc64, img + o_mc64, base + o_mc64, m.dmc64, &m.q_value64, &m.q_out64, &m.disc64);
  McSaDev& d = m.dev;
  std::memset(&d, 0, sizeof(d));
  d.model = m.model;
  d.d = n_params(m.model);
  d.n_chains = m.n_chains;
  d.n_levels = m.n_levels;
  d.chain_len = m.chain_len;
  d.n_quotes = m.mc.n_quotes;
  for (int i = 0; i < kMaxD; ++i) {
    d.lo[i] = m.lo[i];
    d.hi[i] = m.hi[i];
  }
  d.T0_given = m.T0;
  d.step0 = m.step0;
  d.step_min = m.step_min;
  d.Tmax = m.mc.Tmax;
  d.key0 = (uint32_t)m.seed;
  d.key1 = (uint32_t)(m.seed >> 32);
  size_t o_mkt = take(8 * Q);
  if (write) std::memcpy(img + o_mkt, m.mkt.data(), 8 * Q);
  d.mkt = (const double*)(base + o_mkt);
  size_t o_ck = take(8 * m.ck.size());
  if (write) std::memcpy(img + o_ck, m.ck.data(), 8 * m.ck.size());
  d.ck = (const double*)(base + o_ck);
  size_t o_x0 = take(8 * kMaxD);
  if (write) std::memcpy(img + o_x0, m.x0, 8 * kMaxD);
  d.x0 = (const double*)(base + o_x0);
  d.state = (double*)(base + take(8 * 12));
  d.cx = (double*)(base + take(8 * C * kMaxD));
  d.bx = (double*)(base + take(8 * C * kMaxD));
  d.cf = (double*)(base + take(8 * C));
  d.bf = (double*)(base + take(8 * C));
  d.ev = (unsigned long long*)(base + take(8 * C));
  d.ac = (unsigned long long*)(base + take(8 * C));
  d.set_params = (double*)(base + take(8 * C * kMaxD));
  d.set_valid = (int*)(base + take(4 * C));
  d.prices = (double*)(base + take(8 * C * Q));
  d.one_params = (double*)(base + take(8 * kMaxD));
  d.one_prices = (double*)(base + take(8 * Q));
  m.partial = (double*)(base + take(8 * C * (size_t)m.bps * nv));
  m.partial1 = (double*)(base + take(8 * (size_t)m.bps1 * nv));
  d.result = dres;
  m.end = o;
}

sabr_status mcsa_prepare(const sabr_problem& pr, const sabr_bounds& b, const sabr_cooling& c, uint64_t seed,
                         McSaHost& m) {
  m.model = pr.model;
  const int d = n_params(pr.model);
  if (d < 0) return fail(SABR_EINVAL, "unknown model");
  if (!pr.market) return fail(SABR_EINVAL, "NULL market array");
  if (pr.n_chains < 1 || pr.n_chains > (1 << 16)) return fail(SABR_EINVAL, "MC cost: n_chains must lie in [1, 65536]");
  if (!(c.factor > 0.0) || !std::isfinite(c.factor) || c.n_levels < 0 || c.chain_len < 0 || !(c.step0 >= 0.0) ||
      !(c.step_min >= 0.0) || !std::isfinite(c.T0))
    return fail(SABR_EINVAL, "bad cooling schedule");
  SABR_TRY(mc_prepare(pr.model, pr.fwd, pr.T, pr.K, pr.is_call, pr.discount, pr.n_quotes, pr.mc_paths,
                      pr.mc_steps_per_year, pr.mc_seed, pr.prec, m.mc));
  SABR_TRY(mc_prepare(pr.model, pr.fwd, pr.T, pr.K, pr.is_call, pr.discount, pr.n_quotes, pr.mc_paths,
                      pr.mc_steps_per_year, pr.mc_seed, SABR_FP64, m.mc64));
  m.mkt.assign(pr.market, pr.market + pr.n_quotes);
  for (double v : m.mkt)
    if (!(v != 0.0) || !std::isfinite(v)) return fail(SABR_EINVAL, "market prices must be finite and nonzero");
  m.n_chains = pr.n_chains;
  m.n_levels = c.n_levels;
  m.chain_len = c.chain_len;
  m.T0 = c.T0;
  m.step0 = c.step0;
  m.step_min = c.step_min;
  m.seed = seed;
  for (int i = 0; i < kMaxD; ++i) {
    m.lo[i] = i < d ? b.lo[i] : 0.0;
    m.hi[i] = i < d ? b.hi[i] : 0.0;
    if (!(m.lo[i] <= m.hi[i]) || !std::isfinite(m.lo[i]) || !std::isfinite(m.hi[i]))
      return fail(SABR_EINVAL, "bounds need finite lo <= hi");
    m.x0[i] = i < d ? (pr.x0 ? pr.x0[i] : 0.5 * (m.lo[i] + m.hi[i])) : 0.0;
    if (m.x0[i] < m.lo[i] || m.x0[i] > m.hi[i]) return fail(SABR_EINVAL, "x0 outside the box");
  }
  SABR_TRY(check_params(pr.model, m.x0));
  m.ck.resize(m.n_levels + 1);
  for (int k = 0; k < m.n_levels; ++k) m.ck[k] = std::pow(c.factor, (double)k);
  m.bps = mc_blocks_per_set(m.mc, m.n_chains);
  m.bps1 = mc_blocks_per_set(m.mc, 1);
  return SABR_OK;
}

// Pieces of a Technique II calibration: what = 0 start (f(x0) and chain
// state), 1 one proposal wave at (level, step), 2 the restart at a level's
// end, 3 the best point and its FP64 re-score.  Returns launches or -1.
int64_t mcsa_enqueue_piece(const McSaHost& m, cudaStream_t s, int what, int level, int step) {
  const McSaDev& P = m.dev;
  const int tb = 128, cb = (m.n_chains + tb - 1) / tb;
  if (what == 0) {
    mcsa_start_kernel<<<1, 32, 0, s>>>(P);
    if (mc_launch(m.mc, m.dmc, P.one_params, nullptr, 1, m.bps1, m.partial1, m.q_value, m.q_out, m.disc,
                  P.one_prices, nullptr, m.mc.n_quotes, s) != SABR_OK)
      return -1;
    mcsa_init_kernel<<<1, 256, 0, s>>>(P);
    return 4;
  }
  if (what == 1) {
    mcsa_propose_kernel<<<cb, tb, 0, s>>>(P, level, step);
    if (mc_launch(m.mc, m.dmc, P.set_params, P.set_valid, m.n_chains, m.bps, m.partial, m.q_value, m.q_out, m.disc,
                  P.prices, nullptr, m.mc.n_quotes, s) != SABR_OK)
      return -1;
    mcsa_accept_kernel<<<cb, tb, 0, s>>>(P, level, step);
    return 4;
  }
  if (what == 2) {
    mcsa_restart_kernel<<<1, 256, 0, s>>>(P);
    return 1;
  }
  mcsa_final_kernel<<<1, 256, 0, s>>>(P);
  if (mc_launch(m.mc64, m.dmc64, P.one_params, nullptr, 1, m.bps1, m.partial1, m.q_value64, m.q_out64, m.disc64,
                P.one_prices, nullptr, m.mc.n_quotes, s) != SABR_OK)
    return -1;
  mcsa_rescore_kernel<<<1, 32, 0, s>>>(P);
  return 4;
}

// Enqueues one whole Technique II calibration.  Returns launches or -1.
int64_t mcsa_enqueue(const McSaHost& m, cudaStream_t s) {
  int64_t n = 0, k;
  if ((k = mcsa_enqueue_piece(m, s, 0, 0, 0)) < 0) return -1;
  n += k;
  for (int lv = 0; lv < m.n_levels; ++lv) {
    for (int st = 0; st < m.chain_len; ++st) {
      if ((k = mcsa_enqueue_piece(m, s, 1, lv, st)) < 0) return -1;
      n += k;
    }
    if ((k = mcsa_enqueue_piece(m, s, 2, lv, 0)) < 0) return -1;
    n += k;
  }
  if ((k = mcsa_enqueue_piece(m, s, 3, 0, 0)) < 0) return -1;
  return n + k;
}

}  // namespace sabr
