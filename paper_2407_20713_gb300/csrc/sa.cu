// sa.cu -- synchronous parallel Simulated Annealing (Sec. 5) on the GPU.
//
// Work decomposition: a chain is a group of G lanes (G = 1..32, a power of
// two); lanes split the quotes of the cost function.  A block holds
// blockDim/G chains of one problem (64-thread blocks in plans, 256 in the
// server).  A unit of work is one temperature level (chain_len Metropolis
// steps per chain) of one block of chains; the chains' states live in
// registers for the whole unit.  At the end of the unit each block writes
// the argmin of its chains' final states, and the last block of a problem's
// level to finish (an atomic ticket) takes the argmin over the block minima
// (lowest block on a tie) and writes the restart point of the next level.
//
// Plans run every level of a launch group in one persistent launch: a grid
// of a few 64-thread blocks per SM takes units from a device-resident ready
// queue, and the block that closes a problem's level appends the units of
// that problem's next level.  Problems therefore move from level to level
// independently -- an SM that finishes early takes the next ready unit of
// any problem instead of waiting at a grid-wide barrier -- and the result
// of every unit depends only on its problem, level and block, never on which
// block of the grid ran it.  The server launches the same per-unit code over
// a work list, one level per step.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.h"
#include "engine.cuh"
#include "engine_host.h"
#include "mcsa_host.h"

namespace sabr {

// ---------------------------------------------------------------------------
// Shared-memory staging of a problem's quotes.
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ SmemQuotes<R> stage_quotes(const ProblemDev& P, unsigned char* base,
                                                      int nthreads, int tid, unsigned char** end) {
  const int Q = P.n_quotes, M = P.n_mats;
  // Q + 1 quote slots: the pair layout of an odd count needs one more
  QuotePack<R>* pack = (QuotePack<R>*)base;  // base is 16-byte aligned
  R* l2k = (R*)(pack + Q + 1);
  R* mT = l2k + Q;
  const bool dyn = P.model == SABR_DYN_I || P.model == SABR_DYN_II;
  if (sizeof(R) == 4 && P.model == SABR_HAGAN) {
    float4* pr = (float4*)base;
    const float* lfk = (const float*)P.q_lfk;
    const float* l2kf = (const float*)P.q_l2kf;
    const float* T = (const float*)P.q_T;
    const float* w = (const float*)P.q_w;
    for (int j = tid; j < (Q + 1) / 2; j += nthreads) {
      const int i0 = 2 * j, i1 = 2 * j + 1;
      const bool two = i1 < Q;
      pr[2 * j] = make_float4(lfk[i0], two ? lfk[i1] : 0.0f, l2kf[i0], two ? l2kf[i1] : 0.0f);
      pr[2 * j + 1] = make_float4(T[i0], two ? T[i1] : 0.0f, -w[i0], two ? -w[i1] : 0.0f);
    }
  } else {
    for (int i = tid; i < Q; i += nthreads) {
      QuotePack<R> qp;
      qp.lfk = ((const R*)P.q_lfk)[i];
      qp.l2kf = dyn ? mat_in_slot(P.q_mat[i], R{}) : ((const R*)P.q_l2kf)[i];
      qp.T = ((const R*)P.q_T)[i];
      qp.w = ((const R*)P.q_w)[i];
      pack[i] = qp;
      l2k[i] = ((const R*)P.q_l2k)[i];
    }
  }
  for (int j = tid; j < M; j += nthreads) mT[j] = ((const R*)P.m_T)[j];
  unsigned char* e = (unsigned char*)(((uintptr_t)(mT + M) + 15) & ~(uintptr_t)15);
  SmemQuotes<R> sq{pack, (const float4*)base, l2k, mT, nullptr, nullptr, nullptr};
  if (sizeof(R) == 4 && P.model == SABR_DYN_II) {
    // the Case II term-structure rule: nodes, sub-panels, maturity panels
    float4* nd = (float4*)e;
    float4* sb = nd + kC2Nodes * P.c2_nsub;
    int2* pn = (int2*)(sb + P.c2_nsub);
    for (int i = tid; i < kC2Nodes * P.c2_nsub; i += nthreads) nd[i] = P.c2_node[i];
    for (int i = tid; i < P.c2_nsub; i += nthreads) sb[i] = P.c2_sub[i];
    for (int i = tid; i < M; i += nthreads) pn[i] = P.c2_panel[i];
    sq.c2_node = nd;
    sq.c2_sub = sb;
    sq.c2_panel = pn;
    e = (unsigned char*)(((uintptr_t)(pn + M) + 15) & ~(uintptr_t)15);
  }
  *end = e;
  return sq;
}

// Lexicographic minimum of (f, i): the smaller f, then the smaller index, so
// the result does not depend on the order of merging.
__device__ __forceinline__ void argmin_merge(double& f, int& i, double f2, int i2) {
  if (f2 < f || (f2 == f && i2 < i)) {
    f = f2;
    i = i2;
  }
}
__device__ __forceinline__ void warp_argmin(double& f, int& i) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double f2 = __shfl_xor_sync(0xffffffffu, f, off);
    const int i2 = __shfl_xor_sync(0xffffffffu, i, off);
    argmin_merge(f, i, f2, i2);
  }
}

// Quote pairs per point the speculative Hagan loop keeps in flight (several
// points are evaluated at once, so fewer than QueuePairs), and the steps it
// evaluates at once: two (on one 15-strike smile, 64 chains, 8 lanes a
// chain, four measured 8% slower: 17.39 against 16.12 ms per calibration;
// the results do not depend on the depth).
template <class R> struct SpecPairs {
  static constexpr int value = 2;
};
constexpr int kSpecDepth = 2;
// First chunk of the one-lane FP32 Hagan step loop for problems of at least
// 20 quotes: ten pairs, measured against five on the 21-strike smiles
// (3.08e10 against 2.96e10 cost-evals/s).
constexpr int kBigChunk = 10;
template <int N> struct IntTag {
  static constexpr int value = N;
};

template <int MODEL> struct Dim {
  static constexpr int value = MODEL == SABR_DYN_II ? 10 : (MODEL == SABR_DYN_I ? 6 : 4);
};

__device__ __forceinline__ unsigned group_mask(int G) {
  if (G >= 32) return 0xffffffffu;
  const int lane32 = threadIdx.x & 31;
  return ((1u << G) - 1u) << (lane32 & ~(G - 1));
}

__device__ __forceinline__ void load_problem(const ProblemDev* probs, int pid, ProblemDev* P) {
  const int words = (int)(sizeof(ProblemDev) / 4);
  for (int i = threadIdx.x; i < words; i += blockDim.x)
    ((int*)P)[i] = ((const int*)(probs + pid))[i];
  __syncthreads();
}

// Proposal step: x' = x + step (2u - 1).  The FP64 form rounds each
// operation exactly as written (no contraction into an FMA).
__device__ __forceinline__ float propose(float x, float step, float u) {
  return x + step * (2.0f * u - 1.0f);
}
__device__ __forceinline__ double propose(double x, double step, double u) {
  return __dadd_rn(x, __dmul_rn(step, __dsub_rn(__dmul_rn(2.0, u), 1.0)));
}
// Metropolis acceptance of an uphill move (delta > 0) at temperature Tk.
// FP32 form: u < 2^(-delta log2(e)/Tk) by the SFU, with log2(e)/Tk formed
// once per level.
__device__ __forceinline__ bool metropolis(float u, float delta, float inv_Tk, double) {
  return u < ex2_approx(-delta * inv_Tk);
}
__device__ __forceinline__ bool metropolis(double u, double delta, float, double Tk) {
  return u < exp(-delta / Tk);
}

// Ready queue of a plan's launch group.  entry[u] names unit u as
// (problem, level, block) with the top bit set, or is 0 until the unit is
// appended; units are claimed in order by an atomic head and appended by an
// atomic tail.  The units of level 0 are placed before the launch; the block
// that closes level k of a problem appends that problem's level k + 1.
struct LevelQueue {
  unsigned long long* entry;  // [total]
  unsigned long long* head;
  unsigned long long* tail;
  unsigned int* err;          // nonzero once a wait has given up
  unsigned long long total;   // units of the whole run
  unsigned long long wait_ns; // longest wait for an entry before giving up
};
__host__ __device__ constexpr unsigned long long queue_entry(int p, int lv, int blk) {
  return (1ull << 63) | ((unsigned long long)p << 43) | ((unsigned long long)lv << 23) | (unsigned long long)blk;
}
constexpr int kQueueMaxProblems = 1 << 20, kQueueMaxLevels = 1 << 20, kQueueMaxBlocks = 1 << 23;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits (one thread) until entry u has been appended; 0 when the queue's
// error flag is set or the wait runs past q.wait_ns (which then sets it).
__device__ unsigned long long queue_wait(const LevelQueue& q, unsigned long long u) {
  volatile unsigned long long* slot = q.entry + u;
  volatile unsigned int* err = q.err;
  unsigned long long e = *slot;
  if (e == 0) {
    const unsigned long long t0 = global_ns();
    while (e == 0) {
      if (*err) return 0;
      if (global_ns() - t0 > q.wait_ns) {
        atomicExch(q.err, 1u);
        return 0;
      }
      __nanosleep(200);
      e = *slot;
    }
  }
  __threadfence();
  return e;
}

// ---------------------------------------------------------------------------
// f(x0) and the restart state of level 0.  One block of G threads per problem.
// ---------------------------------------------------------------------------
template <class R, int MODEL>
__global__ void sa_init_kernel(const ProblemDev* __restrict__ probs, const int* __restrict__ plist) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ ProblemDev P;
  load_problem(probs, plist[blockIdx.x], &P);
  unsigned char* rest;
  const SmemQuotes<R> sq = stage_quotes<R>(P, smem, blockDim.x, threadIdx.x, &rest);
  __syncthreads();
  R* coef = (R*)rest;
  const int G = P.G, lane = threadIdx.x;
  R x[kMaxD];
#pragma unroll
  for (int i = 0; i < kMaxD; ++i) x[i] = (R)P.x0[i];
  double f0 = 0.0;
  if (lane < G)
    f0 = cost_to_double(group_cost<R, MODEL>(x, P.n_quotes, P.n_mats, (R)P.l2f, sq, coef, lane, G, group_mask(G)));
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < kMaxD; ++i) P.state[i] = (double)x[i];
    P.state[kMaxD] = f0;
    P.state[kMaxD + 1] = P.T0_given > 0.0 ? P.T0_given : (f0 > 0.0 ? f0 : 1.0);
    P.result->status = isfinite(f0) ? SABR_OK : SABR_EINVAL;
  }
}

// ---------------------------------------------------------------------------
// One temperature level for every chain of a launch group.
// ---------------------------------------------------------------------------
// Block `blk` of problem P (staged in shared memory) runs level `level`.
// Every thread of the block calls this.
// Units of one problem may run on different blocks of one persistent launch,
// so the state another block wrote (restart point, per-chain best and
// counters, block minima) is read from L2 (ld.global.cg), never from a
// possibly stale L1 line.  `q` (plans only) receives the units of the next
// level when this block closes level `level` of problem `pid`.
template <class R, int MODEL, int PAIRS = 2, bool SEL = false>
__device__ __forceinline__ void sa_level_block(const ProblemDev& P, int pid, int blk, int level, unsigned char* smem,
                                               const LevelQueue* q) {
  unsigned char* rest;
  const SmemQuotes<R> sq = stage_quotes<R>(P, smem, blockDim.x, threadIdx.x, &rest);
  constexpr int D = Dim<MODEL>::value;
  const int G = P.G, cpb = P.cpb;
  const int g = threadIdx.x / G, lane = threadIdx.x % G;
  // per-maturity polynomial slices exist only for the dynamic models
  const int coef_m = (MODEL == SABR_DYN_I || MODEL == SABR_DYN_II) ? P.n_mats : 0;
  constexpr int CS = CoefStride<R, MODEL>::value;
  R* coef = (R*)rest + (size_t)g * CS * coef_m;
  double* red_f = (double*)((R*)rest + (size_t)cpb * CS * coef_m + 16);
  red_f = (double*)(((uintptr_t)red_f + 15) & ~(uintptr_t)15);
  R* red_x = (R*)(red_f + cpb);
  __syncthreads();

  const int chain = blk * cpb + g;
  const bool active = chain < P.n_chains;
  const uint32_t gchain = (uint32_t)(P.chain0 + chain);  // Philox counter word 0
  const unsigned gmask = group_mask(G);

  // temperature, step widths and box of this level, formed once by thread 0
  // (FP64 division and square root issue at a small fraction of the FP32
  // rate) and shared by the block's chains
  __shared__ R s_lo[kMaxD], s_hi[kMaxD], s_step[kMaxD];
  __shared__ double s_Tk;
  __shared__ float s_invTk;
  if (threadIdx.x == 0) {
    const double T0 = __ldcg(&P.state[kMaxD + 1]);
    const double Tk0 = __dmul_rn(T0, P.ck[level]);
    double sk = __dmul_rn(P.step0, __dsqrt_rn(__ddiv_rn(Tk0, T0)));
    if (sk < P.step_min) sk = P.step_min;
    for (int i = 0; i < D; ++i) {
      s_step[i] = (R)__dmul_rn(sk, __dsub_rn(P.hi[i], P.lo[i]));
      s_lo[i] = (R)P.lo[i];
      s_hi[i] = (R)P.hi[i];
    }
    s_Tk = Tk0;
    s_invTk = (float)(1.4426950408889634 / Tk0);  // log2(e) / T_k: FP32 Metropolis in base 2
  }
  __syncthreads();
  const double Tk = s_Tk;
  R x[D];
#pragma unroll
  for (int i = 0; i < D; ++i) x[i] = (R)__ldcg(&P.state[i]);
  using C = typename CostOf<R>::T;
  C fcur = cost_from(__ldcg(&P.state[kMaxD]), C{});
  C bf = fcur;
  const float inv_Tk = s_invTk;
  // the chain's best point lives in its chain_bx row (written by lane 0 on
  // each improvement), not in registers
  R* cbx = (R*)P.chain_bx + (size_t)chain * kMaxD;
  if (active) {
    if (level == 0) {
      if (lane == 0) {
#pragma unroll
        for (int i = 0; i < kMaxD; ++i) cbx[i] = i < D ? x[i] : (R)0;
      }
    } else {
      bf = cost_from(__ldcg(&P.chain_bf[chain]), C{});
    }
  }
  unsigned ev = 0, ac = 0;  // per level: at most chain_len each
  const R l2f = (R)P.l2f;
  const R Tmax = (R)P.Tmax;

  if (active) {
    // The FP32 static formulas draw one Philox block per proposal on one lane
    // and keep the ten round keys in registers; the other forms (whose
    // lanes share the draws, or whose register budget is tight) step the
    // key schedule in every block.
    constexpr bool kRoundKeys = sizeof(R) == 4 && (MODEL == SABR_HAGAN || MODEL == SABR_OBLOJ);
    PhiloxKeys pk;
    if constexpr (kRoundKeys) pk = philox_keys(P.key0, P.key1);
    const uint32_t key0 = P.key0, key1 = P.key1;
    auto draw = [&](uint4 c) {
      if constexpr (kRoundKeys) {
        return philox4x32_10(c, pk);
      } else {
        return philox4x32_10(c, key0, key1);
      }
    };
    bool ran_spec = false;
    if constexpr (MODEL == SABR_HAGAN) {
      if (P.spec) {
        // Speculative acceptance (Hagan, several lanes per chain).
        // Acceptance is the common outcome (about 96% of the evaluated
        // proposals on the benchmark smiles), so each iteration forms step
        // st's proposal from x and the proposal of each step st + k
        // (k < SD) from that of step st + k - 1, as if every earlier one
        // were accepted, and evaluates all SD points at once
        // (group_costn_hagan: per point the arithmetic and order of
        // group_cost).  The steps are then decided in order with these
        // costs until one is rejected (out of the box, NaN or by the
        // Metropolis test): that step still counts, the later points are
        // dropped, and the chain advances past it.  The trajectory,
        // counters and best point are those of the one-step loop below.
        ran_spec = true;
        constexpr int SD = kSpecDepth;
        auto words = [&](int s) { return draw(make_uint4(gchain, (uint32_t)level, (uint32_t)s, kTagSA)); };
        uint4 w[SD];
#pragma unroll
        for (int k = 0; k < SD; ++k) w[k] = words(k);
        int st = 0;
        while (st < P.chain_len) {
          // the words of the next SD steps, should all SD be taken (off the
          // critical path)
          uint4 wn[SD];
#pragma unroll
          for (int k = 0; k < SD; ++k) wn[k] = words(st + SD + k);
          R u[SD][D + 1];
          R xs[SD][4];
          bool in[SD];
#pragma unroll
          for (int k = 0; k < SD; ++k) {
            u[k][0] = u01<R>(w[k].x);
            u[k][1] = u01<R>(w[k].y);
            u[k][2] = u01<R>(w[k].z);
            u[k][3] = u01<R>(w[k].w);
            u[k][D] = u01<R>(sa_accept_word(w[k].x, w[k].y, w[k].z));
            in[k] = true;
#pragma unroll
            for (int i = 0; i < D; ++i) {
              xs[k][i] = propose(k == 0 ? x[i] : xs[k - 1][i], s_step[i], u[k][i]);
              in[k] = in[k] && !(xs[k][i] < s_lo[i] || xs[k][i] > s_hi[i]);
            }
          }
          int adv = 1;
          if (in[0]) {
            C f[SD];
            group_costn_hagan<R, SpecPairs<R>::value, SD>(xs, P.n_quotes, sq, lane, G, gmask, f);
            bool go = true;
#pragma unroll
            for (int k = 0; k < SD; ++k) {
              if constexpr (sizeof(R) == 4 && SEL) {
                // FP32, SEL: the decisions as selects (as in the one-step
                // loop), so that the chains of a warp, whose steps accept and
                // reject at different points, run the same instructions
                const bool take = go && st + k < P.chain_len;
                adv = take ? k + 1 : adv;
                const bool eval = take && in[k];
                ev += eval ? 1u : 0u;
                const bool better = eval && cost_less(f[k], bf);
                const float dk = cost_delta(f[k], fcur);
                const float pacc = ex2_approx(-dk * inv_Tk);
                const bool acc = eval && (dk <= 0.0f || u[k][D] < pacc);
                bf = better ? f[k] : bf;
                if (better && lane == 0) {
#pragma unroll
                  for (int i = 0; i < D; ++i) cbx[i] = xs[k][i];
                }
#pragma unroll
                for (int i = 0; i < D; ++i) x[i] = acc ? xs[k][i] : x[i];
                fcur = acc ? f[k] : fcur;
                ac += acc ? 1u : 0u;
                go = acc;
              } else if (go && st + k < P.chain_len) {
                adv = k + 1;
                bool acc = false;
                if (in[k]) {
                  ++ev;
                  if (!cost_is_nan(f[k])) {
                    if (cost_less(f[k], bf)) {
                      bf = f[k];
                      if (lane == 0) {
#pragma unroll
                        for (int i = 0; i < D; ++i) cbx[i] = xs[k][i];
                      }
                    }
                    const auto dk = cost_delta(f[k], fcur);
                    acc = dk <= 0 || metropolis(u[k][D], dk, inv_Tk, Tk);
                  }
                }
                if (acc) {
#pragma unroll
                  for (int i = 0; i < D; ++i) x[i] = xs[k][i];
                  fcur = f[k];
                  ++ac;
                } else {
                  go = false;
                }
              }
            }
          }
          // words of the next iteration's steps st + adv .. st + adv + SD - 1
          // from the current and the next window
#pragma unroll
          for (int k = 0; k < SD; ++k) {
            uint4 v = wn[k];  // adv == SD
#pragma unroll
            for (int a = 1; a < SD; ++a) {
              if (adv == a) v = k + a < SD ? w[k + a] : wn[k + a - SD];
            }
            w[k] = v;
          }
          st += adv;
        }
      }
    }
    // The step loop.  KIND 0: every model and lane count; KIND 1 + F (FP32
    // Hagan, one lane per chain, at least PAIRS pairs): hagan_cost_g1 with
    // F's bits for an odd quote count (1), a first chunk of kBigChunk pairs
    // (2) and one maturity (4).  The choice is made once per unit, outside
    // the loop, so the loop body holds no branch on it.
    auto step_loop = [&](auto kind) {
      constexpr int KIND = decltype(kind)::value;
      uint4 wbuf = make_uint4(0u, 0u, 0u, 0u);
      constexpr int NB = sa_philox_blocks(D);  // Philox blocks per step
      const int S = G >= NB ? G / NB : 1;  // steps per batch of Philox blocks
      int s_ctr = 0;                         // st mod S
      uint4 wnext = make_uint4(0u, 0u, 0u, 0u);
      if (NB == 1 && G == 1 && !ran_spec)
        wnext = draw(make_uint4(gchain, (uint32_t)level, 0u, kTagSA));
      for (int st = 0; st < (ran_spec ? 0 : P.chain_len); ++st) {
        // D Philox words of blocks 0, 1, ... with counter (chain, level, step,
        // tag + block): D move uniforms and, from their unused low bits, the
        // acceptance uniform (sa_accept_word).  With G >= NB lanes, the chain's
        // lanes compute the blocks of S = G/NB consecutive steps at once
        // (lane l: step st0 + l/NB, block l%NB) and every step gathers its
        // words by shuffles; otherwise each lane computes all NB blocks of
        // every step.
        uint32_t wv[4 * NB];
        if (NB == 1 && G == 1) {
          // one lane, one block: no exchange; the block of the next step is
          // formed here, off the critical path of this one (its counter does
          // not depend on this step's outcome)
          const uint4 w = wnext;
          wnext = draw(make_uint4(gchain, (uint32_t)level, (uint32_t)(st + 1), kTagSA));
          wv[0] = w.x;
          wv[1] = w.y;
          wv[2] = w.z;
          wv[3] = w.w;
        } else if (G >= NB) {
          const int s_in = s_ctr;
          s_ctr = s_ctr + 1 == S ? 0 : s_ctr + 1;
          if (s_in == 0) {
            const int l = lane < S * NB ? lane : 0;
            wbuf = draw(make_uint4(gchain, (uint32_t)level, (uint32_t)(st + l / NB), kTagSA + (uint32_t)(l % NB)));
          }
          const int base = ((threadIdx.x & 31) & ~(G - 1)) + s_in * NB;
#pragma unroll
          for (int i = 0; i < D; ++i) {
            const uint32_t word =
                (i & 3) == 0 ? wbuf.x : ((i & 3) == 1 ? wbuf.y : ((i & 3) == 2 ? wbuf.z : wbuf.w));
            wv[i] = __shfl_sync(gmask, word, base + (i >> 2));
          }
        } else {
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            const uint4 w = draw(make_uint4(gchain, (uint32_t)level, (uint32_t)st, kTagSA + (uint32_t)b));
            wv[4 * b + 0] = w.x;
            wv[4 * b + 1] = w.y;
            wv[4 * b + 2] = w.z;
            wv[4 * b + 3] = w.w;
          }
        }
        R u[D + 1];
#pragma unroll
        for (int i = 0; i < D; ++i) u[i] = u01<R>(wv[i]);
        u[D] = u01<R>(sa_accept_word(wv[0], wv[1], wv[2]));
        R xp[D];
        bool inside = true;
#pragma unroll
        for (int i = 0; i < D; ++i) {
          xp[i] = propose(x[i], s_step[i], u[i]);
          inside = inside && !(xp[i] < s_lo[i] || xp[i] > s_hi[i]);
        }
        if (MODEL == SABR_DYN_II && inside) inside = case2_feasible<R>(xp, Tmax);
        if (!inside) continue;
        C fp;
        if constexpr (KIND == 0) {
          fp = group_cost<R, MODEL, PAIRS>(xp, P.n_quotes, P.n_mats, l2f, sq, coef, lane, G, gmask);
        } else {
          constexpr int F = KIND - 1;  // bit 0: odd count, bit 1: big chunk, bit 2: one maturity
          fp = hagan_cost_g1<((F & 2) ? kBigChunk : PAIRS), (F & 1) != 0, (F & 4) != 0>(xp, P.n_quotes, sq);
        }
        ++ev;
        if constexpr (sizeof(R) == 4) {
          // FP32: the decision as selects (a NaN cost compares false, so it
          // is neither an improvement nor accepted), with the SFU 2^x of
          // the Metropolis test formed whatever the sign of delta, so lanes
          // that accept and lanes that reject run the same instructions
          const bool better = cost_less(fp, bf);
          const float delta = cost_delta(fp, fcur);
          const float pacc = ex2_approx(-delta * inv_Tk);
          const bool acc = delta <= 0.0f || u[D] < pacc;
          bf = better ? fp : bf;
          if (better && lane == 0) {
#pragma unroll
            for (int i = 0; i < D; ++i) cbx[i] = xp[i];
          }
#pragma unroll
          for (int i = 0; i < D; ++i) x[i] = acc ? xp[i] : x[i];
          fcur = acc ? fp : fcur;
          ac += acc ? 1u : 0u;
        } else {
          if (cost_is_nan(fp)) continue;
          if (cost_less(fp, bf)) {
            bf = fp;
            if (lane == 0) {
#pragma unroll
              for (int i = 0; i < D; ++i) cbx[i] = xp[i];
            }
          }
          const auto delta = cost_delta(fp, fcur);
          if (delta <= 0 || metropolis(u[D], delta, inv_Tk, Tk)) {
#pragma unroll
            for (int i = 0; i < D; ++i) x[i] = xp[i];
            fcur = fp;
            ++ac;
          }
        }
      }
    };
    if constexpr (MODEL == SABR_HAGAN && sizeof(R) == 4) {
      const bool one_lane = !ran_spec && G == 1;
      const int full = P.n_quotes >> 1;
      // (the big chunk only where the kernel's register budget holds it:
      // the persistent launch, whose PAIRS is 5)
      const bool big = PAIRS >= 5 && full >= kBigChunk;
      const int f = ((P.n_quotes & 1) ? 1 : 0) | (big ? 2 : 0) | (P.n_mats == 1 ? 4 : 0);
      if (!one_lane || full < PAIRS) {
        step_loop(IntTag<0>{});
      } else {
        switch (f) {
          case 0: step_loop(IntTag<1>{}); break;
          case 1: step_loop(IntTag<2>{}); break;
          case 2: step_loop(IntTag<3>{}); break;
          case 3: step_loop(IntTag<4>{}); break;
          case 4: step_loop(IntTag<5>{}); break;
          case 5: step_loop(IntTag<6>{}); break;
          case 6: step_loop(IntTag<7>{}); break;
          default: step_loop(IntTag<8>{}); break;
        }
      }
    } else {
      step_loop(IntTag<0>{});
    }
    if (lane == 0) {
      P.chain_bf[chain] = cost_to_double(bf);
      if (level == 0) {
        P.chain_ev[chain] = ev;
        P.chain_ac[chain] = ac;
      } else {
        P.chain_ev[chain] = __ldcg(&P.chain_ev[chain]) + ev;
        P.chain_ac[chain] = __ldcg(&P.chain_ac[chain]) + ac;
      }
      red_f[g] = cost_to_double(fcur);
#pragma unroll
      for (int i = 0; i < kMaxD; ++i) red_x[g * kMaxD + i] = i < D ? x[i] : (R)0;
    }
  } else if (lane == 0) {
    red_f[g] = INFINITY;
  }
  __syncthreads();

  // block argmin of the final states (lowest chain index on a tie), by warp 0
  __shared__ int s_last;
  if (threadIdx.x < 32) {
    double fb = INFINITY;
    int best = 0x7fffffff;
    for (int c = threadIdx.x; c < cpb; c += 32) argmin_merge(fb, best, red_f[c], c);
    warp_argmin(fb, best);
    if (threadIdx.x == 0) {
      P.part_f[blk] = fb;
      P.part_c[blk] = blk * cpb + best;
      for (int i = 0; i < kMaxD; ++i) P.part_x[(size_t)blk * kMaxD + i] = (double)red_x[best * kMaxD + i];
      __threadfence();
      const unsigned ticket = atomicAdd(P.arrive, 1u);
      s_last = ticket == (unsigned)(P.n_blocks - 1);
    }
  }
  __syncthreads();
  if (s_last) {
    // last block of this problem: the restart point of the next level is the
    // argmin over the block minima (lowest block on a tie), by every thread
    __shared__ double s_wf[kSaBlock / 32];
    __shared__ int s_wb[kSaBlock / 32];
    __threadfence();
    double f = INFINITY;
    int bb = 0x7fffffff;
    for (int b = threadIdx.x; b < P.n_blocks; b += blockDim.x) argmin_merge(f, bb, __ldcg(&P.part_f[b]), b);
    warp_argmin(f, bb);
    if ((threadIdx.x & 31) == 0) {
      s_wf[threadIdx.x >> 5] = f;
      s_wb[threadIdx.x >> 5] = bb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) argmin_merge(f, bb, s_wf[w], s_wb[w]);
      for (int i = 0; i < kMaxD; ++i) P.state[i] = __ldcg(&P.part_x[(size_t)bb * kMaxD + i]);
      P.state[kMaxD] = f;
      P.state[kStateArgChain] = (double)(P.chain0 + __ldcg(&P.part_c[bb]));
      *P.arrive = 0u;
    }
    if (q != nullptr && level + 1 < P.n_levels) {
      // append the next level's units of this problem, after the restart
      // point is visible device-wide
      __shared__ unsigned long long s_base;
      if (threadIdx.x == 0) {
        __threadfence();
        s_base = atomicAdd(q->tail, (unsigned long long)P.n_blocks);
      }
      __syncthreads();
      __threadfence();
      volatile unsigned long long* ent = q->entry;
      for (int b = threadIdx.x; b < P.n_blocks; b += blockDim.x) ent[s_base + b] = queue_entry(pid, level + 1, b);
    }
  }
}

// One temperature level for a list of (problem, block) work items.
// Plans launch one block per item with `level` >= 0 (the level of the
// launch); the server launches a fixed grid that strides over a work list
// read from device memory (n_work != nullptr), each item carrying its own
// level in .z (level < 0), so that one captured launch serves every step
// whatever its mix of requests.  Both use this one kernel, so a problem's
// arithmetic is the same machine code in a plan and in the server.
// Register budget: up to 128 registers for the static formulas' quote loop
// (pairs of quotes), the dynamic term structures (Case I closed forms, the
// Case II rule's eight node values and thirteen running sums per panel) and
// the chain state; the expanded form keeps 80.
template <class R, int MODEL> struct LevelMinBlocks {
  static constexpr int value = sizeof(R) == 8 ? 1 : (MODEL == SABR_EXPANDED ? 3 : 2);
};

template <class R, int MODEL>
__global__ void __launch_bounds__(kSaBlock, (LevelMinBlocks<R, MODEL>::value))
    sa_level_kernel(const ProblemDev* __restrict__ probs, const int4* __restrict__ work,
                    const int* __restrict__ n_work, int n_items, int level) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ ProblemDev P;
  const int nw = n_work ? *n_work : n_items;
  for (int w = blockIdx.x; w < nw; w += gridDim.x) {
    const int4 it = work[w];
    const int lv = level >= 0 ? level : it.z;
    load_problem(probs, it.x, &P);
    if (lv < P.n_levels) sa_level_block<R, MODEL, 2, true>(P, it.x, it.y, lv, smem, nullptr);
    __syncthreads();
  }
}

// Every level of a plan's launch group in one launch: each block takes units
// from the ready queue until all are claimed (or a wait gave up).
// Resident warps per SM the queue kernel is compiled for (in blocks of
// kLevelBlock threads): the FP32 static formulas eight (two warps a
// scheduler, up to 255 registers for the quote-pair loop), the FP32
// dynamic models sixteen (128 registers; their term structures are
// latency-bound and want more warps), the expanded form 24 at 80
// registers, the FP64 form eight.
template <class R, int MODEL> struct QueueBlocks {
  static constexpr int warps =
      sizeof(R) == 8 ? 8 : ((MODEL == SABR_HAGAN || MODEL == SABR_OBLOJ) ? 8 : (MODEL == SABR_EXPANDED ? 24 : 16));
  static constexpr int value = warps * 32 / kLevelBlock;
};
template <class R, int MODEL> struct QueuePairs {
  static constexpr int value = 5;
};

// SEL: the speculative Hagan loop takes its decisions as selects (the
// launches of single problems, whose chains have several lanes; in the
// kernel that also runs the one-lane step loop of large batches they
// measured 1.6% slower there, from its register allocation).
template <class R, int MODEL, bool SEL = false>
__global__ void __launch_bounds__(kLevelBlock, (QueueBlocks<R, MODEL>::value))
    sa_queue_kernel(const ProblemDev* __restrict__ probs, LevelQueue q) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ ProblemDev P;
  __shared__ unsigned long long s_e;
  for (;;) {
    if (threadIdx.x == 0) {
      unsigned long long e = 0;
      if (*(volatile unsigned int*)q.err == 0) {
        const unsigned long long u = atomicAdd(q.head, 1ull);
        if (u < q.total) e = queue_wait(q, u);
      }
      s_e = e;
    }
    __syncthreads();
    const unsigned long long e = s_e;
    if (e == 0) return;
    const int pid = (int)((e >> 43) & (kQueueMaxProblems - 1));
    const int lv = (int)((e >> 23) & (kQueueMaxLevels - 1));
    const int blk = (int)(e & (kQueueMaxBlocks - 1));
    load_problem(probs, pid, &P);
    sa_level_block<R, MODEL, QueuePairs<R, MODEL>::value, SEL>(P, pid, blk, lv, smem, &q);
    __syncthreads();
  }
}

// Before each run: head and error flag cleared, the units of level 0 (a
// list fixed when the plan was built) in place, every later entry empty.
__global__ void queue_reset_kernel(LevelQueue q, const unsigned long long* __restrict__ level0, unsigned long long n0) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < q.total; i += stride)
    q.entry[i] = i < n0 ? level0[i] : 0ull;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *q.head = 0ull;
    *q.tail = n0;
    *q.err = 0u;
  }
}

// ---------------------------------------------------------------------------
// Best point over all chains, FP64 re-score, counters -> result.
// One 256-thread block per problem.
// ---------------------------------------------------------------------------
// `queue_err` (plans): a ready-queue wait gave up, so the levels did not all
// run; the result then carries SABR_ETIMEOUT.
template <class R, int MODEL>
__global__ void __launch_bounds__(kSaBlock) sa_finalize_kernel(const ProblemDev* __restrict__ probs,
                                                              const int* __restrict__ plist,
                                                              const unsigned int* __restrict__ queue_err) {
  __shared__ ProblemDev P;
  __shared__ double s_f[kSaBlock];
  __shared__ int s_c[kSaBlock];
  __shared__ unsigned long long s_ev[kSaBlock], s_ac[kSaBlock];
  __shared__ double s_best[kMaxD];
  __shared__ double s_coef[3 * kMaxMats];
  load_problem(probs, plist[blockIdx.x], &P);
  const int tid = threadIdx.x;

  double fb = INFINITY;
  int cb = 0x7fffffff;
  unsigned long long ev = 0, ac = 0;
  if (P.n_levels > 0) {
    for (int c = tid; c < P.n_chains; c += blockDim.x) {
      const double v = P.chain_bf[c];
      if (v < fb) {
        fb = v;
        cb = c;
      }
      ev += P.chain_ev[c];
      ac += P.chain_ac[c];
    }
  }
  s_f[tid] = fb;
  s_c[tid] = cb;
  s_ev[tid] = ev;
  s_ac[tid] = ac;
  __syncthreads();
  if (tid == 0) {
    double f = INFINITY;
    int c = 0x7fffffff;
    unsigned long long te = 0, ta = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      if (s_f[t] < f || (s_f[t] == f && s_c[t] < c)) {
        f = s_f[t];
        c = s_c[t];
      }
      te += s_ev[t];
      ta += s_ac[t];
    }
    if (P.n_levels == 0 || c == 0x7fffffff) {
      f = P.state[kMaxD];
      for (int i = 0; i < kMaxD; ++i) s_best[i] = P.state[i];
      P.state[kStateBestChain] = -1.0;
    } else {
      const R* bx = (const R*)P.chain_bx + (size_t)c * kMaxD;
      for (int i = 0; i < kMaxD; ++i) s_best[i] = (double)bx[i];
      P.state[kStateBestChain] = (double)(P.chain0 + c);
    }
    sabr_result* r = P.result;
    for (int i = 0; i < kMaxD; ++i) {
      r->params[i] = s_best[i];
      r->restart_params[i] = P.state[i];
    }
    r->misfit = f;
    r->restart_misfit = P.state[kMaxD];
    if (queue_err != nullptr && *queue_err != 0u) r->status = SABR_ETIMEOUT;
    r->n_evals = (int64_t)te;
    r->n_accepts = (int64_t)ta;
  }
  __syncthreads();

  // FP64 re-score of the best point (Sec. 3 eq. error_calibrate_relativo).
  const double l2f = P.l2f;
  if (MODEL == SABR_DYN_I || MODEL == SABR_DYN_II) {
    for (int j = tid; j < P.n_mats; j += blockDim.x) {
      const PolyCoef<double> c = dynamic_coef<double, MODEL == SABR_DYN_II>(s_best, l2f, P.m64_T[j]);
      s_coef[3 * j] = c.c0;
      s_coef[3 * j + 1] = c.c1;
      s_coef[3 * j + 2] = c.c2;
    }
    __syncthreads();
  }
  double acc = 0.0;
  const StaticConst<double> sc = static_setup<double>(s_best);
  for (int q = tid; q < P.n_quotes; q += blockDim.x) {
    double v;
    if (MODEL == SABR_HAGAN) {
      v = vol_hagan<double>(sc, P.q64_lfk[q], P.q64_l2kf[q], P.q64_T[q]);
    } else if (MODEL == SABR_OBLOJ) {
      v = vol_obloj<double>(sc, P.q64_lfk[q], P.q64_l2kf[q], P.q64_l2k[q], P.q64_T[q]);
    } else if (MODEL == SABR_EXPANDED) {
      v = vol_poly<double>(expanded_coef<double>(s_best, l2f, P.q64_T[q]), P.q64_lfk[q]);
    } else {
      const int j = P.q_mat[q];
      PolyCoef<double> c;
      c.c0 = s_coef[3 * j];
      c.c1 = s_coef[3 * j + 1];
      c.c2 = s_coef[3 * j + 2];
      v = vol_poly<double>(c, P.q64_lfk[q]);
    }
    const double r = (P.q64_mkt[q] - v) / P.q64_mkt[q];
    acc += r * r;
  }
  __syncthreads();
  s_f[tid] = acc;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int t = 0; t < (int)blockDim.x; ++t) s += s_f[t];
    P.result->misfit_fp64 = s;
  }
}
// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Whether Hagan problems whose chains have several lanes use the
// speculative step loop (sa_level_block): the environment variable
// SABR_SPECULATE=0 selects the one-step loop (the same results; kept for
// comparison).
static bool speculate_enabled() {
  const char* e = std::getenv("SABR_SPECULATE");
  return !(e && e[0] == '0');
}

static int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// About 24 quotes per lane (a lane runs its quote loop three quotes at a
// time), widened while the batch has fewer than (SMs x 256) threads and quotes
// remain to split; the dynamic models take one lane per two maturities and
// per ~48 quotes.
int choose_lanes(int n_quotes, int n_mats, int model, int prec, long long batch_chains) {
  if (const char* e = std::getenv("SABR_LANES")) {
    int g = std::atoi(e);
    if (g >= 1 && g <= 32 && (g & (g - 1)) == 0) return g;
  }
  // fewer lanes repeat the per-proposal work (Philox, proposal,
  // Metropolis, lane sum) less often
  int G = next_pow2((n_quotes + 23) / 24);
  // The dynamic models: a quote is a few FMAs on its maturity's polynomial,
  // and the per-maturity functions dominate (closed forms for Case I; for
  // Case II also the eta2^2 quadrature, whose nodes the lanes share), so one
  // lane per two maturities and per ~48 quotes (measured on 12 maturities x
  // 21 strikes, 8192 chains: 8 lanes beat 4 and 16 for both cases)
  if (model == SABR_DYN_I || model == SABR_DYN_II)
    G = std::max(std::max(1, next_pow2(n_mats) / 2), next_pow2((n_quotes + 47) / 48));
  G = std::min(G, 32);
  // the FP32 Hagan form hands its lanes pairs of quotes (more lanes than
  // pairs would idle; on one 15-strike smile, 64 chains: 8 lanes 16.12 ms,
  // 16 lanes 16.50 ms per calibration)
  const int units = (model == SABR_HAGAN && prec == SABR_FP32) ? (n_quotes + 1) / 2 : n_quotes;
  const int cap = std::min(32, next_pow2(units));
  const long long fill = (long long)device_sms() * 256;
  while (G < cap && batch_chains * G < fill) G <<= 1;
  return G;
}

size_t level_smem_bytes(int prec, int model, int Q, int M, int cpb, int c2_nsub) {
  const size_t rs = prec == SABR_FP64 ? 8 : 4;
  const size_t cm = (model == SABR_DYN_I || model == SABR_DYN_II) ? (size_t)M : 0;
  size_t b = 4 * rs * ((size_t)Q + 1) + ((size_t)Q + M) * rs;  // pack (or pairs), l2k, mT
  b = align_up(b, 16);
  if (prec == SABR_FP32 && model == SABR_DYN_II)  // Case II rule: nodes, sub-panels, panels
    b = align_up(b + (size_t)c2_nsub * (kC2Nodes + 1) * 16 + (size_t)M * 8, 16);
  b += (size_t)cpb * coef_stride(prec, model) * cm * rs + 16 * rs;
  b = align_up(b, 16) + 16;
  b += (size_t)cpb * 8 + (size_t)cpb * kMaxD * rs;
  return align_up(b, 16) + 64;
}

size_t init_smem_bytes(const HostProblem& h) {
  return level_smem_bytes(h.prec, SABR_DYN_II, h.n_quotes, h.n_mats, 1, h.c2_nsub);
}

// The FP32 Case II term-structure rule of a problem: the maturities split
// [0, Tmax] into panels [T_{j-1}, T_j], and each panel into sub-panels no
// wider than max(start, 2/k) (k the largest exponential rate the box allows:
// 2b for nu^2, a + b for nu rho); an 8-point Gauss-Legendre rule on each
// sub-panel.  The widths grow geometrically away from t = 0, so e^{-k' t}
// is resolved for every rate k' <= k: where a sub-panel is wide (k' h
// large) the exponential is already negligible at its start.
static sabr_status case2_rule_build(HostProblem& h) {
  h.c2_node.clear();
  h.c2_sub.clear();
  h.c2_panel.clear();
  const double amax = std::max(std::fabs(h.lo[4]), std::fabs(h.hi[4]));
  const double bmax = std::max(std::fabs(h.lo[5]), std::fabs(h.hi[5]));
  const double kmax = std::max(2.0 * bmax, amax + bmax);
  const double w0 = kmax > 0.0 ? 2.0 / kmax : 1e300;
  constexpr GaussRule<kC2Nodes> gr = make_gauss<kC2Nodes>();
  double prev = 0.0;
  int nsub = 0;
  for (int j = 0; j < h.n_mats; ++j) {
    const double T = h.mT[j];
    h.c2_panel.push_back(nsub);
    int cnt = 0;
    double s0 = prev;
    for (;;) {
      double e = s0 + std::max(s0, w0);
      if (e >= T || T - e < 0.5 * std::max(e, w0)) e = T;
      const double hh = 0.5 * (e - s0);
      double sw = 0.0, stw = 0.0;
      for (int k = 0; k < kC2Nodes; ++k) {
        const double u = s0 + hh * (1.0 + gr.x[k]), W = hh * gr.w[k];
        h.c2_node.insert(h.c2_node.end(), {(float)u, (float)W, (float)(T - u), 0.0f});
        sw += W;
        stw += (T - u) * W;
      }
      h.c2_sub.insert(h.c2_sub.end(), {(float)hh, (float)sw, (float)stw, 0.0f});
      ++cnt;
      if (++nsub > kMaxC2Sub) return fail(SABR_EINVAL, "Case II rate bounds too wide for the FP32 term-structure rule");
      if (e >= T) break;
      s0 = e;
    }
    h.c2_panel.push_back(cnt);
    prev = T;
  }
  h.c2_nsub = nsub;
  return SABR_OK;
}

sabr_status formula_prepare(const sabr_problem& pr, const sabr_bounds& b, const sabr_cooling& c, uint64_t seed,
                            HostProblem& h) {
  h.model = pr.model;
  h.d = n_params(pr.model);
  if (h.d < 0) return fail(SABR_EINVAL, "unknown model");
  if (pr.cost != SABR_COST_VOL) return fail(SABR_EINVAL, "not an implied-vol cost");
  if (pr.prec != SABR_FP32 && pr.prec != SABR_FP64) return fail(SABR_EINVAL, "unknown precision");
  if (!(pr.fwd > 0.0) || !std::isfinite(pr.fwd)) return fail(SABR_EINVAL, "fwd must be > 0");
  if (pr.n_quotes < 1 || pr.n_quotes > kMaxQuotes) return fail(SABR_EINVAL, "n_quotes must lie in [1, 4096]");
  if (!pr.T || !pr.K || !pr.market) return fail(SABR_EINVAL, "NULL quote array");
  if (pr.n_chains < 1 || pr.n_chains > (1 << 24)) return fail(SABR_EINVAL, "n_chains must lie in [1, 2^24]");
  if (!(c.factor > 0.0) || !std::isfinite(c.factor) || c.n_levels < 0 || c.chain_len < 0 || !(c.step0 >= 0.0) ||
      !(c.step_min >= 0.0) || !std::isfinite(c.T0) || !std::isfinite(c.step0) || !std::isfinite(c.step_min))
    return fail(SABR_EINVAL, "bad cooling schedule");
  h.prec = pr.prec;
  h.cost = pr.cost;
  h.n_quotes = (int)pr.n_quotes;
  h.n_chains = pr.n_chains;
  h.n_levels = c.n_levels;
  h.chain_len = c.chain_len;
  h.fwd = pr.fwd;
  h.T0 = c.T0;
  h.step0 = c.step0;
  h.step_min = c.step_min;
  h.seed = seed;
  const int Q = h.n_quotes;
  std::vector<int> order(Q);
  for (int i = 0; i < Q; ++i) {
    if (!(pr.T[i] > 0.0) || !std::isfinite(pr.T[i])) return fail(SABR_EINVAL, "maturities must be > 0");
    if (!(pr.K[i] > 0.0) || !std::isfinite(pr.K[i])) return fail(SABR_EINVAL, "strikes must be > 0");
    if (!(pr.market[i] > 0.0) || !std::isfinite(pr.market[i])) return fail(SABR_EINVAL, "market vols must be > 0");
    order[i] = i;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int bb) { return pr.T[a] < pr.T[bb]; });
  h.lfk.resize(Q);
  h.l2kf.resize(Q);
  h.l2k.resize(Q);
  h.T.resize(Q);
  h.mkt.resize(Q);
  h.mat.resize(Q);
  h.mT.clear();
  for (int s = 0; s < Q; ++s) {
    const int i = order[s];
    if (h.mT.empty() || pr.T[i] != h.mT.back()) h.mT.push_back(pr.T[i]);
    h.mat[s] = (int)h.mT.size() - 1;
    h.lfk[s] = std::log(pr.fwd / pr.K[i]);
    h.l2kf[s] = std::log2(pr.K[i] * pr.fwd);
    h.l2k[s] = std::log2(pr.K[i]);
    h.T[s] = pr.T[i];
    h.mkt[s] = pr.market[i];
  }
  h.n_mats = (int)h.mT.size();
  if (h.n_mats > kMaxMats) return fail(SABR_EINVAL, "more than 64 distinct maturities");
  h.Tmax = h.mT.back();
  for (int i = 0; i < kMaxD; ++i) {
    h.lo[i] = i < h.d ? b.lo[i] : 0.0;
    h.hi[i] = i < h.d ? b.hi[i] : 0.0;
    if (!(h.lo[i] <= h.hi[i]) || !std::isfinite(h.lo[i]) || !std::isfinite(h.hi[i]))
      return fail(SABR_EINVAL, "bounds need finite lo <= hi");
    h.x0[i] = i < h.d ? (pr.x0 ? pr.x0[i] : 0.5 * (h.lo[i] + h.hi[i])) : 0.0;
    if (h.x0[i] < h.lo[i] || h.x0[i] > h.hi[i]) return fail(SABR_EINVAL, "x0 outside the box");
  }
  if (h.model == SABR_DYN_II && !case2_feasible<double, double>(h.x0, h.Tmax))
    return fail(SABR_EINVAL, "x0 violates the Case II constraints");
  if (h.model == SABR_DYN_II && h.prec == SABR_FP32) SABR_TRY(case2_rule_build(h));
  h.ck.resize(std::max(h.n_levels, 1));
  for (int k = 0; k < h.n_levels; ++k) h.ck[k] = std::pow(c.factor, (double)k);
  return SABR_OK;
}

size_t formula_layout(const HostProblem& h, int G, unsigned char* img, unsigned char* base, size_t off0,
                      ProblemDev& d, sabr_result* dres, int block) {
  size_t o = off0;
  auto take = [&](size_t bytes) {
    o = align_up(o, 256);
    const size_t r = o;
    o += bytes;
    return r;
  };
  const bool write = img != nullptr;
  auto put = [&](size_t at, const void* src, size_t bytes) {
    if (write) std::memcpy(img + at, src, bytes);
  };
  std::memset(&d, 0, sizeof(d));
  d.model = h.model;
  d.prec = h.prec;
  d.cost = h.cost;
  d.d = h.d;
  d.n_quotes = h.n_quotes;
  d.n_mats = h.n_mats;
  d.n_chains = h.n_chains;
  d.n_levels = h.n_levels;
  d.chain_len = h.chain_len;
  d.G = G;
  d.cpb = block / G;
  d.n_blocks = (h.n_chains + d.cpb - 1) / d.cpb;
  d.fwd = h.fwd;
  d.l2f = std::log2(h.fwd);
  d.Tmax = h.Tmax;
  for (int k = 0; k < kMaxD; ++k) {
    d.lo[k] = h.lo[k];
    d.hi[k] = h.hi[k];
  }
  d.T0_given = h.T0;
  d.step0 = h.step0;
  d.step_min = h.step_min;
  d.key0 = (uint32_t)h.seed;
  d.key1 = (uint32_t)(h.seed >> 32);
  const size_t rs = h.prec == SABR_FP64 ? 8 : 4;
  const size_t Q = h.n_quotes, M = h.n_mats, C = h.n_chains, B = d.n_blocks;
  const size_t o_lfk = take(Q * rs), o_l2kf = take(Q * rs), o_l2k = take(Q * rs), o_T = take(Q * rs),
               o_w = take(Q * rs), o_mat = take(Q * 4), o_mT = take(M * rs);
  const size_t o64_lfk = take(Q * 8), o64_l2kf = take(Q * 8), o64_l2k = take(Q * 8), o64_T = take(Q * 8),
               o64_mkt = take(Q * 8), o64_mT = take(M * 8);
  const size_t o_ck = take(h.ck.size() * 8), o_x0 = take(kMaxD * 8), o_state = take(kStateLen * 8);
  const size_t o_bf = take(C * 8), o_bx = take(C * kMaxD * rs), o_ev = take(C * 8), o_ac = take(C * 8);
  const size_t o_pf = take(B * 8), o_pc = take(B * 4), o_px = take(B * kMaxD * 8), o_arr = take(4);
  const size_t o_c2n = take(4 * h.c2_node.size()), o_c2s = take(4 * h.c2_sub.size()),
               o_c2p = take(4 * h.c2_panel.size());
  if (write) {
    if (h.prec == SABR_FP64) {
      put(o_lfk, h.lfk.data(), Q * 8);
      put(o_l2kf, h.l2kf.data(), Q * 8);
      put(o_l2k, h.l2k.data(), Q * 8);
      put(o_T, h.T.data(), Q * 8);
      put(o_w, h.mkt.data(), Q * 8);
      put(o_mT, h.mT.data(), M * 8);
    } else {
      std::vector<float> t(Q);
      for (size_t k = 0; k < Q; ++k) t[k] = (float)h.lfk[k];
      put(o_lfk, t.data(), Q * 4);
      for (size_t k = 0; k < Q; ++k) t[k] = (float)h.l2kf[k];
      put(o_l2kf, t.data(), Q * 4);
      for (size_t k = 0; k < Q; ++k) t[k] = (float)h.l2k[k];
      put(o_l2k, t.data(), Q * 4);
      for (size_t k = 0; k < Q; ++k) t[k] = (float)h.T[k];
      put(o_T, t.data(), Q * 4);
      for (size_t k = 0; k < Q; ++k) t[k] = (float)(1.0 / h.mkt[k]);
      put(o_w, t.data(), Q * 4);
      std::vector<float> tm(M);
      for (size_t k = 0; k < M; ++k) tm[k] = (float)h.mT[k];
      put(o_mT, tm.data(), M * 4);
    }
    put(o_mat, h.mat.data(), Q * 4);
    put(o64_lfk, h.lfk.data(), Q * 8);
    put(o64_l2kf, h.l2kf.data(), Q * 8);
    put(o64_l2k, h.l2k.data(), Q * 8);
    put(o64_T, h.T.data(), Q * 8);
    put(o64_mkt, h.mkt.data(), Q * 8);
    put(o64_mT, h.mT.data(), M * 8);
    put(o_ck, h.ck.data(), h.ck.size() * 8);
    put(o_x0, h.x0, kMaxD * 8);
    std::memset(img + o_arr, 0, 4);
    put(o_c2n, h.c2_node.data(), 4 * h.c2_node.size());
    put(o_c2s, h.c2_sub.data(), 4 * h.c2_sub.size());
    put(o_c2p, h.c2_panel.data(), 4 * h.c2_panel.size());
  }
  d.q_lfk = base + o_lfk;
  d.q_l2kf = base + o_l2kf;
  d.q_l2k = base + o_l2k;
  d.q_T = base + o_T;
  d.q_w = base + o_w;
  d.q_mat = (const int*)(base + o_mat);
  d.m_T = base + o_mT;
  d.q64_lfk = (const double*)(base + o64_lfk);
  d.q64_l2kf = (const double*)(base + o64_l2kf);
  d.q64_l2k = (const double*)(base + o64_l2k);
  d.q64_T = (const double*)(base + o64_T);
  d.q64_mkt = (const double*)(base + o64_mkt);
  d.m64_T = (const double*)(base + o64_mT);
  d.ck = (const double*)(base + o_ck);
  d.x0 = (const double*)(base + o_x0);
  d.state = (double*)(base + o_state);
  d.chain_bf = (double*)(base + o_bf);
  d.chain_bx = base + o_bx;
  d.chain_ev = (unsigned long long*)(base + o_ev);
  d.chain_ac = (unsigned long long*)(base + o_ac);
  d.part_f = (double*)(base + o_pf);
  d.part_c = (int*)(base + o_pc);
  d.part_x = (double*)(base + o_px);
  d.arrive = (unsigned int*)(base + o_arr);
  d.result = dres;
  d.c2_node = (const float4*)(base + o_c2n);
  d.c2_sub = (const float4*)(base + o_c2s);
  d.c2_panel = (const int2*)(base + o_c2p);
  d.c2_nsub = h.c2_nsub;
  d.chain0 = h.chain0;
  // speculation pays where a chain's lanes share its quotes (small,
  // latency-bound problems); with one lane per chain (large batches) the two
  // evaluations cost more issue slots than the latency they hide (measured
  // on the benchmark surface: 2.28e10 against 2.53e10 cost-evals/s)
  d.spec = (h.model == SABR_HAGAN && G > 1 && speculate_enabled()) ? 1 : 0;
  return o;
}

// ---- launch wrappers ------------------------------------------------------
template <class R, int MODEL>
static void set_smem_one(size_t bytes) {
  cudaFuncSetAttribute(sa_level_kernel<R, MODEL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(sa_init_kernel<R, MODEL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

#define SABR_DISPATCH(prec, model, CALL)                              \
  do {                                                                \
    if ((prec) == SABR_FP64) {                                        \
      using R = double;                                               \
      switch (model) {                                                \
        case SABR_HAGAN: { constexpr int M = SABR_HAGAN; CALL; } break;       \
        case SABR_OBLOJ: { constexpr int M = SABR_OBLOJ; CALL; } break;       \
        case SABR_EXPANDED: { constexpr int M = SABR_EXPANDED; CALL; } break; \
        case SABR_DYN_I: { constexpr int M = SABR_DYN_I; CALL; } break;       \
        default: { constexpr int M = SABR_DYN_II; CALL; } break;              \
      }                                                               \
    } else {                                                          \
      using R = float;                                                \
      switch (model) {                                                \
        case SABR_HAGAN: { constexpr int M = SABR_HAGAN; CALL; } break;       \
        case SABR_OBLOJ: { constexpr int M = SABR_OBLOJ; CALL; } break;       \
        case SABR_EXPANDED: { constexpr int M = SABR_EXPANDED; CALL; } break; \
        case SABR_DYN_I: { constexpr int M = SABR_DYN_I; CALL; } break;       \
        default: { constexpr int M = SABR_DYN_II; CALL; } break;              \
      }                                                               \
    }                                                                 \
  } while (0)

void set_engine_smem(int prec, int model, size_t bytes) { SABR_DISPATCH(prec, model, (set_smem_one<R, M>(bytes))); }

void launch_init(int prec, int model, const ProblemDev* probs, const int* plist, int n, size_t smem, cudaStream_t s) {
  SABR_DISPATCH(prec, model, (sa_init_kernel<R, M><<<n, 32, smem, s>>>(probs, plist)));
}

void launch_level(int prec, int model, const ProblemDev* probs, const int4* bmap, int blocks, int level, size_t smem,
                  cudaStream_t s) {
  SABR_DISPATCH(prec, model,
                (sa_level_kernel<R, M><<<blocks, kLevelBlock, smem, s>>>(probs, bmap, nullptr, blocks, level)));
}

void launch_persistent(int prec, int model, const ProblemDev* probs, const int4* work, const int* n_work, int grid,
                       size_t smem, cudaStream_t s) {
  SABR_DISPATCH(prec, model, (sa_level_kernel<R, M><<<grid, kSaBlock, smem, s>>>(probs, work, n_work, 0, -1)));
}

void launch_finalize(int prec, int model, const ProblemDev* probs, const int* plist, int n, cudaStream_t s,
                     const unsigned int* queue_err) {
  SABR_DISPATCH(prec, model, (sa_finalize_kernel<R, M><<<n, kSaBlock, 0, s>>>(probs, plist, queue_err)));
}

// single: the group is one problem (FP32 Hagan then takes the SEL kernel)
static bool queue_sel(int prec, int model, bool single) { return single && prec == SABR_FP32 && model == SABR_HAGAN; }

static void launch_queue(int prec, int model, const ProblemDev* probs, const LevelQueue& q, int grid, size_t smem,
                         bool single, cudaStream_t s) {
  if (queue_sel(prec, model, single)) {
    sa_queue_kernel<float, SABR_HAGAN, true><<<grid, kLevelBlock, smem, s>>>(probs, q);
    return;
  }
  SABR_DISPATCH(prec, model, (sa_queue_kernel<R, M><<<grid, kLevelBlock, smem, s>>>(probs, q)));
}

static int queue_blocks_per_sm(int prec, int model, size_t smem, bool single) {
  int nb = 1;
  if (queue_sel(prec, model, single)) {
    cudaFuncSetAttribute(sa_queue_kernel<float, SABR_HAGAN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sa_queue_kernel<float, SABR_HAGAN, true>, kLevelBlock, smem);
    return nb < 1 ? 1 : nb;
  }
  SABR_DISPATCH(prec, model, (cudaFuncSetAttribute(sa_queue_kernel<R, M>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                              cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sa_queue_kernel<R, M>, kLevelBlock,
                                                                            smem)));
  return nb < 1 ? 1 : nb;
}

int persistent_blocks_per_sm(int prec, int model, size_t smem) {
  int nb = 1;
  SABR_DISPATCH(prec, model,
                (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sa_level_kernel<R, M>, kSaBlock, smem)));
  return nb < 1 ? 1 : nb;
}

struct LaunchGroup {
  int prec = 0, model = 0;
  std::vector<int> problems;
  int total_blocks = 0;
  int max_levels = 0;
  size_t smem_level = 0, smem_init = 0;
  int4* d_bmap = nullptr;
  int* d_plist = nullptr;
  // ready queue (all levels in one persistent launch); per-level launches
  // when use_queue is false
  bool use_queue = false;
  LevelQueue q{};
  unsigned long long* d_level0 = nullptr;
  unsigned long long n0 = 0;
  int queue_grid = 0;
};

// Resident 64-thread blocks per SM that a plan's persistent level launch
// aims for: four give every SM scheduler two warps, so all schedulers carry
// the same load (the environment variable SABR_WORKERS_PER_SM overrides it
// for tuning).
static int workers_per_sm(int prec, int model) {
  if (const char* e = std::getenv("SABR_WORKERS_PER_SM")) {
    const int w = std::atoi(e);
    if (w >= 1 && w <= 32) return w;
  }
  int w = 4;
  SABR_DISPATCH(prec, model, (w = QueueBlocks<R, M>::value));
  return w;
}
// Whether plans may use the ready queue: the environment variable
// SABR_PLAN_QUEUE=0 makes them launch their levels one by one instead (the
// same units in a different launch shape; the results are identical).
static bool queue_enabled() {
  const char* e = std::getenv("SABR_PLAN_QUEUE");
  return !(e && e[0] == '0');
}
// A ready queue takes 8 bytes per unit; beyond this a plan launches its
// levels one by one instead.
constexpr unsigned long long kMaxQueueBytes = 512ull << 20;

}  // namespace sabr

struct sabr_plan {
  int device = 0;
  int n = 0;
  void* arena = nullptr;
  sabr::ProblemDev* d_probs = nullptr;
  sabr_result* d_results = nullptr;
  sabr_result* h_results = nullptr;
  std::vector<sabr::LaunchGroup> groups;
  int max_levels = 0;
  bool use_graph = false;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t own_stream = nullptr;
  cudaEvent_t ev_lv0 = nullptr, ev_lv1 = nullptr, ev_done = nullptr;
  int64_t launches = 0;
  int64_t level_launches = 0;
  bool ran = false;
  std::vector<sabr::McSaHost> mc;  // Technique II problems
  std::vector<int> mc_index;       // their batch index
};

namespace sabr {

// The whole calibration of a plan, enqueued on s.
static sabr_status enqueue_plan(sabr_plan* p, cudaStream_t s, bool capturing) {
  int64_t launches = 0, level_launches = 0;
  for (auto& g : p->groups) {
    launch_init(g.prec, g.model, p->d_probs, g.d_plist, (int)g.problems.size(), g.smem_init, s);
    ++launches;
  }
  if (capturing)
    SABR_CUDA(cudaEventRecordWithFlags(p->ev_lv0, s, cudaEventRecordExternal));
  else
    SABR_CUDA(cudaEventRecord(p->ev_lv0, s));
  for (auto& g : p->groups) {
    if (!g.use_queue || g.q.total == 0) continue;
    queue_reset_kernel<<<(int)std::min<unsigned long long>(1024, (g.q.total + 255) / 256), 256, 0, s>>>(
        g.q, g.d_level0, g.n0);
    launch_queue(g.prec, g.model, p->d_probs, g.q, g.queue_grid, g.smem_level, g.problems.size() == 1, s);
    launches += 2;
    ++level_launches;
  }
  for (int lv = 0; lv < p->max_levels; ++lv)
    for (auto& g : p->groups) {
      if (g.use_queue || lv >= g.max_levels) continue;
      launch_level(g.prec, g.model, p->d_probs, g.d_bmap, g.total_blocks, lv, g.smem_level, s);
      ++launches;
      ++level_launches;
    }
  if (capturing)
    SABR_CUDA(cudaEventRecordWithFlags(p->ev_lv1, s, cudaEventRecordExternal));
  else
    SABR_CUDA(cudaEventRecord(p->ev_lv1, s));
  for (auto& g : p->groups) {
    launch_finalize(g.prec, g.model, p->d_probs, g.d_plist, (int)g.problems.size(), s,
                    g.use_queue ? g.q.err : nullptr);
    ++launches;
  }
  for (auto& m : p->mc) {
    const int64_t k = mcsa_enqueue(m, s);
    if (k < 0) return SABR_ECUDA;
    launches += k;
  }
  SABR_CUDA(cudaGetLastError());
  SABR_CUDA(cudaMemcpyAsync(p->h_results, p->d_results, sizeof(sabr_result) * p->n, cudaMemcpyDeviceToHost, s));
  p->launches = launches;
  p->level_launches = level_launches;
  return SABR_OK;
}

static void free_plan(sabr_plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->ev_lv0) cudaEventDestroy(p->ev_lv0);
  if (p->ev_lv1) cudaEventDestroy(p->ev_lv1);
  if (p->ev_done) cudaEventDestroy(p->ev_done);
  if (p->own_stream) cudaStreamDestroy(p->own_stream);
  if (p->arena) cudaFree(p->arena);
  if (p->h_results) cudaFreeHost(p->h_results);
  delete p;
}

static sabr_status build_plan(int32_t n, const sabr_problem* problems, const sabr_bounds* bounds,
                              const sabr_cooling* cooling, const uint64_t* seeds, int use_graph, cudaStream_t stream,
                              sabr_plan** out) {
  if (!out) return fail(SABR_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || !problems || !bounds || !cooling || !seeds) return fail(SABR_EINVAL, "empty batch or NULL array");
  std::vector<HostProblem> hp;
  std::vector<int> fidx, midx;
  std::vector<McSaHost> mch;
  long long batch_chains = 0;
  for (int i = 0; i < n; ++i) {
    if (problems[i].cost == SABR_COST_MC_PRICE) {
      mch.emplace_back();
      SABR_TRY(mcsa_prepare(problems[i], bounds[i], cooling[i], seeds[i], mch.back()));
      midx.push_back(i);
    } else {
      hp.emplace_back();
      SABR_TRY(formula_prepare(problems[i], bounds[i], cooling[i], seeds[i], hp.back()));
      batch_chains += hp.back().n_chains;
      fidx.push_back(i);
    }
  }
  const int nf = (int)hp.size();
  sabr_plan* p = new sabr_plan();
  p->n = n;
  p->mc_index = midx;
  p->mc = std::move(mch);
  cudaGetDevice(&p->device);

  // arena: problem table, results, per-problem regions, launch maps
  std::vector<int> lanes(nf);
  std::vector<ProblemDev> pd(nf);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    o = align_up(o, 256);
    const size_t r = o;
    o += bytes;
    return r;
  };
  const size_t probs_off = take(sizeof(ProblemDev) * std::max(nf, 1));
  const size_t results_off = take(sizeof(sabr_result) * n);
  std::vector<size_t> f_off(nf), mc_off(p->mc.size());
  for (int i = 0; i < nf; ++i) {
    lanes[i] = choose_lanes(hp[i].n_quotes, hp[i].n_mats, hp[i].model, hp[i].prec, batch_chains);
    if (level_smem_bytes(hp[i].prec, hp[i].model, hp[i].n_quotes, hp[i].n_mats, kLevelBlock / lanes[i],
                         hp[i].c2_nsub) > kMaxLevelSmem) {
      free_plan(p);
      return fail(SABR_EINVAL, "the quotes of a problem exceed one block's shared memory at its precision");
    }
    f_off[i] = align_up(o, 256);
    o = formula_layout(hp[i], lanes[i], nullptr, nullptr, f_off[i], pd[i], nullptr, kLevelBlock);
  }
  for (size_t k = 0; k < p->mc.size(); ++k) mc_off[k] = take(mcsa_arena_bytes(p->mc[k]));
  for (int i = 0; i < nf; ++i) {
    LaunchGroup* g = nullptr;
    for (auto& gg : p->groups)
      if (gg.prec == hp[i].prec && gg.model == hp[i].model) g = &gg;
    if (!g) {
      p->groups.push_back(LaunchGroup());
      g = &p->groups.back();
      g->prec = hp[i].prec;
      g->model = hp[i].model;
    }
    g->problems.push_back(i);
    g->total_blocks += pd[i].n_blocks;
    g->max_levels = std::max(g->max_levels, hp[i].n_levels);
    g->smem_level = std::max(g->smem_level, level_smem_bytes(hp[i].prec, hp[i].model, hp[i].n_quotes, hp[i].n_mats,
                                                              pd[i].cpb, hp[i].c2_nsub));
    g->smem_init = std::max(g->smem_init, init_smem_bytes(hp[i]));
    p->max_levels = std::max(p->max_levels, hp[i].n_levels);
  }
  std::vector<size_t> bmap_off(p->groups.size()), plist_off(p->groups.size());
  std::vector<size_t> qent_off(p->groups.size()), qctl_off(p->groups.size()), ql0_off(p->groups.size());
  std::vector<std::vector<unsigned long long>> level0(p->groups.size());
  const int sms = device_sms();
  for (size_t gi = 0; gi < p->groups.size(); ++gi) {
    LaunchGroup& g = p->groups[gi];
    bmap_off[gi] = take(sizeof(int4) * g.total_blocks);
    plist_off[gi] = take(sizeof(int) * g.problems.size());
    // ready queue: one entry per (problem, level, block) of the run
    unsigned long long total = 0;
    double unit_ns = 0.0;  // generous bound on the duration of one unit
    for (int pi : g.problems) {
      total += (unsigned long long)hp[pi].n_levels * (unsigned long long)pd[pi].n_blocks;
      for (int b = 0; hp[pi].n_levels > 0 && b < pd[pi].n_blocks; ++b) level0[gi].push_back(queue_entry(pi, 0, b));
      const double per_step = (double)(hp[pi].n_quotes / lanes[pi] + 1) + 64.0 * hp[pi].n_mats + 64.0;
      unit_ns = std::max(unit_ns, 100.0 * per_step * (double)hp[pi].chain_len);
    }
    // The queue pays when a level of the group has more units than the
    // persistent grid has blocks and several problems can fill each
    // other's level ends.  A single problem (every unit of a level waits for
    // the same restart point) uses it only when two of its levels fit in the
    // persistent grid: the grid then holds the blocks of one level and, on
    // the queue, those of the next, which start as soon as the level closes
    // instead of after a kernel launch (a level's fixed cost on one smile of
    // 64 chains: 13.7 us with a launch per level); larger single problems
    // run level by level.
    const int per_sm = std::min(workers_per_sm(g.prec, g.model),
                                queue_blocks_per_sm(g.prec, g.model, g.smem_level, g.problems.size() == 1));
    int grid = std::max(1, std::min(g.total_blocks, sms * per_sm));
    const bool single_small = g.problems.size() == 1 && 2 * g.total_blocks <= sms * per_sm && p->max_levels > 1;
    if (single_small) grid = 2 * g.total_blocks;
    g.use_queue = queue_enabled() && ((g.problems.size() > 1 && g.total_blocks > grid) || single_small) &&
                  nf <= kQueueMaxProblems && p->max_levels < kQueueMaxLevels && total * 8 <= kMaxQueueBytes;
    for (int pi : g.problems) g.use_queue = g.use_queue && pd[pi].n_blocks <= kQueueMaxBlocks;
    if (g.use_queue) {
      g.q.total = total;
      g.q.wait_ns = (unsigned long long)std::min(6.0e11, 5.0e9 + 100.0 * unit_ns);
      g.n0 = level0[gi].size();
      qent_off[gi] = take(8 * std::max<unsigned long long>(total, 1));
      qctl_off[gi] = take(32);
      ql0_off[gi] = take(8 * std::max<size_t>(level0[gi].size(), 1));
      g.queue_grid = grid;
    }
  }
  const size_t arena_bytes = align_up(o, 256);

  std::vector<unsigned char> img(arena_bytes, 0);
  cudaError_t e = cudaMalloc(&p->arena, arena_bytes);
  if (e != cudaSuccess) {
    free_plan(p);
    return cuda_fail(e, "cudaMalloc(plan arena)");
  }
  unsigned char* base = (unsigned char*)p->arena;
  sabr_result* dres = (sabr_result*)(base + results_off);
  for (int i = 0; i < nf; ++i)
    formula_layout(hp[i], lanes[i], img.data(), base, f_off[i], pd[i], dres + fidx[i], kLevelBlock);
  for (size_t k = 0; k < p->mc.size(); ++k) mcsa_layout(p->mc[k], img.data(), base, mc_off[k], dres + p->mc_index[k]);
  if (nf > 0) std::memcpy(img.data() + probs_off, pd.data(), sizeof(ProblemDev) * nf);
  for (size_t gi = 0; gi < p->groups.size(); ++gi) {
    LaunchGroup& g = p->groups[gi];
    std::vector<int4> bm;
    for (int pi : g.problems)
      for (int b = 0; b < pd[pi].n_blocks; ++b) bm.push_back(make_int4(pi, b, 0, 0));
    std::memcpy(img.data() + bmap_off[gi], bm.data(), sizeof(int4) * bm.size());
    std::memcpy(img.data() + plist_off[gi], g.problems.data(), sizeof(int) * g.problems.size());
    g.d_bmap = (int4*)(base + bmap_off[gi]);
    g.d_plist = (int*)(base + plist_off[gi]);
    if (g.use_queue) {
      g.q.entry = (unsigned long long*)(base + qent_off[gi]);
      g.q.head = (unsigned long long*)(base + qctl_off[gi]);
      g.q.tail = g.q.head + 1;
      g.q.err = (unsigned int*)(g.q.head + 2);
      g.d_level0 = (unsigned long long*)(base + ql0_off[gi]);
      if (!level0[gi].empty())
        std::memcpy(img.data() + ql0_off[gi], level0[gi].data(), 8 * level0[gi].size());
    }
    set_engine_smem(g.prec, g.model, std::max(g.smem_level, g.smem_init));
  }
  p->d_probs = (ProblemDev*)(base + probs_off);
  p->d_results = dres;
  e = cudaMemcpy(p->arena, img.data(), arena_bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMallocHost(&p->h_results, sizeof(sabr_result) * n);
  if (e == cudaSuccess) e = cudaEventCreate(&p->ev_lv0);
  if (e == cudaSuccess) e = cudaEventCreate(&p->ev_lv1);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_done, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    free_plan(p);
    return cuda_fail(e, "plan set-up");
  }
  p->use_graph = use_graph != 0;
  if (p->use_graph) {
    cudaStream_t cs = stream;
    if (!cs) {
      e = cudaStreamCreateWithFlags(&p->own_stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) {
        free_plan(p);
        return cuda_fail(e, "cudaStreamCreate");
      }
      cs = p->own_stream;
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      free_plan(p);
      return cuda_fail(e, "cudaStreamBeginCapture");
    }
    sabr_status st = enqueue_plan(p, cs, true);
    e = cudaStreamEndCapture(cs, &graph);
    if (st != SABR_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      free_plan(p);
      return st != SABR_OK ? st : cuda_fail(e, "cudaStreamEndCapture");
    }
    e = cudaGraphInstantiate(&p->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      free_plan(p);
      return cuda_fail(e, "cudaGraphInstantiate");
    }
  }
  *out = p;
  return SABR_OK;
}

static sabr_status run_plan(sabr_plan* p, cudaStream_t s) {
  if (p->use_graph) {
    SABR_CUDA(cudaGraphLaunch(p->exec, s));
  } else {
    SABR_TRY(enqueue_plan(p, s, false));
  }
  SABR_CUDA(cudaEventRecord(p->ev_done, s));
  p->ran = true;
  return SABR_OK;
}

static sabr_status plan_results(sabr_plan* p, sabr_result* out) {
  if (!p->ran) return fail(SABR_EINVAL, "plan has not been run");
  SABR_CUDA(cudaEventSynchronize(p->ev_done));
  std::memcpy(out, p->h_results, sizeof(sabr_result) * p->n);
  return SABR_OK;
}

}  // namespace sabr

extern "C" {

sabr_status sabr_plan_create(int32_t n, const sabr_problem* problems, const sabr_bounds* bounds,
                             const sabr_cooling* cooling, const uint64_t* seeds, int32_t use_graph, void* stream,
                             sabr_plan** out) {
  sabr::clear_error();
  return sabr::build_plan(n, problems, bounds, cooling, seeds, use_graph, (cudaStream_t)stream, out);
}

sabr_status sabr_plan_run(sabr_plan* plan, void* stream) {
  sabr::clear_error();
  if (!plan) return sabr::fail(SABR_EINVAL, "plan is NULL");
  return sabr::run_plan(plan, (cudaStream_t)stream);
}

sabr_status sabr_plan_results(sabr_plan* plan, sabr_result* out) {
  sabr::clear_error();
  if (!plan || !out) return sabr::fail(SABR_EINVAL, "NULL argument");
  return sabr::plan_results(plan, out);
}

sabr_status sabr_plan_stats(sabr_plan* plan, int64_t* launches, double* level_ms) {
  sabr::clear_error();
  if (!plan) return sabr::fail(SABR_EINVAL, "plan is NULL");
  if (launches) *launches = plan->launches;
  if (level_ms) {
    *level_ms = 0.0;
    if (plan->ran && plan->level_launches > 0 && plan->max_levels > 0) {
      SABR_CUDA(cudaEventSynchronize(plan->ev_done));
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, plan->ev_lv0, plan->ev_lv1) == cudaSuccess)
        *level_ms = (double)ms / (double)plan->max_levels;
    }
  }
  return SABR_OK;
}

void sabr_plan_destroy(sabr_plan* plan) { sabr::free_plan(plan); }

sabr_status sabr_calibrate_batch(int32_t n, const sabr_problem* problems, const sabr_bounds* bounds,
                                 const sabr_cooling* cooling, const uint64_t* seeds, sabr_result* out, void* stream) {
  sabr::clear_error();
  if (!out) return sabr::fail(SABR_EINVAL, "out is NULL");
  sabr_plan* p = nullptr;
  SABR_TRY(sabr::build_plan(n, problems, bounds, cooling, seeds, 0, (cudaStream_t)stream, &p));
  sabr_status st = sabr::run_plan(p, (cudaStream_t)stream);
  if (st == SABR_OK) st = sabr::plan_results(p, out);
  sabr::free_plan(p);
  return st;
}

sabr_status sabr_calibrate(const sabr_problem* problem, const sabr_bounds* bounds, const sabr_cooling* cooling,
                           uint64_t seed, sabr_result* out, void* stream) {
  return sabr_calibrate_batch(1, problem, bounds, cooling, &seed, out, stream);
}

}  // extern "C"
