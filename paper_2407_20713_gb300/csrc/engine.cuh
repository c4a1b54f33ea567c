// engine.cuh -- device-side layout of a batch of calibration problems and
// the group-collective cost of Sec. 3 eq. (error_calibrate_relativo).
#pragma once
#include <cstdint>

#include "../../include/sabr.h"
#include "sabr_math.cuh"

namespace sabr {

constexpr int kSaBlock = 256;   // threads per SA block (server, init, finalize)
// Threads per block of the plans' level kernel: small blocks spread a
// batch's chains evenly over the 152 SMs (14 resident per SM at <= 72
// registers), where 256-thread blocks leave a partly filled second wave.
constexpr int kLevelBlock = 64;
// Dynamic shared memory a level block may use: the 227 KB opt-in limit less
// room for the kernel's static shared memory.
constexpr size_t kMaxLevelSmem = 226 * 1024;
// Restart state of a problem: x[10], f, T0, then the global chain index of
// the last level's argmin and of the best-ever point (as doubles, exact).
constexpr int kStateLen = 14;
constexpr int kStateArgChain = 12, kStateBestChain = 13;

// One problem of a batch, as the kernels see it (all pointers device).
// Quotes are sorted by maturity; q_* arrays hold the working precision R,
// q64_* arrays the FP64 values used by the final re-score.
struct ProblemDev {
  int model, prec, cost, d;
  int n_quotes, n_mats, n_chains, n_levels;
  int chain_len, G, cpb, n_blocks;
  double fwd, l2f, Tmax;
  double lo[10], hi[10];
  double T0_given, step0, step_min;
  uint32_t key0, key1;
  const void* q_lfk;   // ln(f/K)
  const void* q_l2kf;  // log2(K f)
  const void* q_l2k;   // log2(K)
  const void* q_T;     // maturity
  const void* q_w;     // 1/market (FP32) or market (FP64)
  const int* q_mat;    // maturity index
  const void* m_T;     // distinct maturities [n_mats]
  const double* q64_lfk;
  const double* q64_l2kf;
  const double* q64_l2k;
  const double* q64_T;
  const double* q64_mkt;
  const double* m64_T;
  const double* ck;    // factor^k, k < n_levels
  const double* x0;    // [10]
  double* state;       // [kStateLen]
  double* chain_bf;    // [n_chains] best misfit of each chain
  void* chain_bx;      // [n_chains][10] best point of each chain (R)
  unsigned long long* chain_ev;
  unsigned long long* chain_ac;
  double* part_f;      // [n_blocks] block argmin of the final states
  int* part_c;
  double* part_x;      // [n_blocks][10]
  unsigned int* arrive;
  sabr_result* result;
  // FP32 Case II term-structure rule (device copies of HostProblem's)
  const float4* c2_node;
  const float4* c2_sub;
  const int2* c2_panel;
  int c2_nsub;
  // global index of the problem's chain 0: a shard of a chain-sharded
  // problem runs chains chain0 .. chain0 + n_chains - 1 of it (Philox
  // counters and reported chain indices are global)
  int chain0;
  int spec;  // Hagan: speculative two-step loop (same results)
};

// Per-quote inputs ln(f/K), log2(K f), T and 1/market (FP32) or market
// (FP64), packed so that one 16-byte (FP32) shared-memory load fetches a
// quote.
template <class R> struct __align__(16) QuotePack {
  R lfk, l2kf, T, w;
};
// The dynamic models read neither log2(K f) nor T per quote (their quotes
// use the polynomial of their maturity), so their packs carry the quote's
// maturity index, as integer bits, in the l2kf slot: one load per quote
// fetches everything its evaluation needs but the polynomial.
__device__ __forceinline__ float mat_in_slot(int j, float) { return __int_as_float(j); }
__device__ __forceinline__ double mat_in_slot(int j, double) { return __longlong_as_double((long long)j); }
__device__ __forceinline__ int mat_of_slot(float v) { return __float_as_int(v); }
__device__ __forceinline__ int mat_of_slot(double v) { return (int)__double_as_longlong(v); }

// Quote tables of one problem staged in shared memory.  The FP32 Hagan
// form evaluates its quotes two at a time (hagan_resid_pair), so its quotes
// are staged as pairs instead: for pair j (quotes 2j and 2j + 1 in maturity
// order) pair[2j] = (lfk, lfk', l2kf, l2kf') and pair[2j + 1] =
// (T, T', -1/market, -1/market'), two 16-byte loads a pair; an odd count
// leaves a zero second element in the last pair, whose residual is not
// summed.
template <class R> struct SmemQuotes {
  const QuotePack<R>* pack;  // per quote (every model but the FP32 Hagan form)
  const float4* pair;        // per pair of quotes (FP32 Hagan form)
  const R* l2k;              // per quote: log2 K (Oblój)
  const R* mT;               // per maturity: T
  // FP32 Case II term-structure rule
  const float4* c2_node;     // per node: u, W, tau = T_j - u
  const float4* c2_sub;      // per sub-panel: half width, sum W, sum tau W
  const int2* c2_panel;      // per maturity: first sub-panel, count
};

// Double-float number hi + lo (|lo| <= ulp(hi)/2): sums of FP32 terms carried
// to about 48 significant bits on the FP32 pipe.  GB300 issues FP64 at about
// 1/75 of its FP32 rate, so the FP32 form keeps FP64 out of the per-proposal
// path and sums the misfit in this format instead.
struct DF {
  float hi, lo;
};
// Exact sum a + b = s + e (Knuth's two-sum; no multiplies, so nothing is
// contracted into an FMA).  Symmetric in a and b.
__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return DF{s, e};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const DF s = df_two_sum(a.hi, b.hi);
  const float e = s.lo + (a.lo + b.lo);
  const float hi = s.hi + e;
  return DF{hi, e - (hi - s.hi)};
}

// Cost type of the working precision: double for FP64, DF for FP32.
template <class R> struct CostOf {
  using T = double;
};
template <> struct CostOf<float> {
  using T = DF;
};
__device__ __forceinline__ double cost_from(double d, double) { return d; }
__device__ __forceinline__ DF cost_from(double d, DF) {
  const float hi = (float)d;
  return DF{hi, (float)(d - (double)hi)};
}
__device__ __forceinline__ double cost_to_double(double c) { return c; }
__device__ __forceinline__ double cost_to_double(DF c) { return (double)c.hi + (double)c.lo; }
__device__ __forceinline__ bool cost_less(double a, double b) { return a < b; }
__device__ __forceinline__ bool cost_less(DF a, DF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool cost_is_nan(double a) { return !(a == a); }
__device__ __forceinline__ bool cost_is_nan(DF a) { return !(a.hi == a.hi); }
__device__ __forceinline__ double cost_delta(double a, double b) { return a - b; }
__device__ __forceinline__ float cost_delta(DF a, DF b) { return (a.hi - b.hi) + (a.lo - b.lo); }

// ((market - model)/market)^2 term.  FP32 keeps 1/market (one FMA); FP64
// divides exactly as written.
__device__ __forceinline__ float resid(float v, float inv_mkt) { return 1.0f - v * inv_mkt; }
__device__ __forceinline__ double resid(double v, double mkt) { return (mkt - v) / mkt; }

// Sum over the G lanes of a chain by an xor butterfly: every lane ends with
// the same, order-fixed total.  FP64 in the FP64 form; double-float in the
// FP32 form.
__device__ __forceinline__ double lanes_sum(double v, int G, unsigned gmask) {
  for (int off = G >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(gmask, v, off);
  return v;
}
__device__ __forceinline__ DF lanes_sum(float v, int G, unsigned gmask) {
  DF s{v, 0.0f};
  for (int off = G >> 1; off > 0; off >>= 1) {
    const DF o{__shfl_xor_sync(gmask, s.hi, off), __shfl_xor_sync(gmask, s.lo, off)};
    s = df_add(s, o);
  }
  return s;
}

// Shared-memory slots per maturity in a chain group's coefficient slice: the
// polynomial (c0, c1, c2), and a fourth slot (for Case II it holds eta2^2
// until the polynomial is formed) that aligns each polynomial to 16 bytes.
// The FP32 Case II form also keeps, per maturity, the panel integrals its
// term-structure rule sums (slots 4 .. 12 of a 16-slot stride).
template <class R, int MODEL> struct CoefStride {
  static constexpr int value = (MODEL == SABR_DYN_II && sizeof(R) == 4) ? 16 : 4;
};
__host__ __device__ constexpr int coef_stride(int prec, int model) {
  return (model == SABR_DYN_II && prec == SABR_FP32) ? 16 : 4;
}

// The polynomial of maturity j from a coefficient slice: one 16-byte load
// in FP32 (the slice is 16-byte aligned and its stride is 4), two in FP64.
__device__ __forceinline__ PolyCoef<float> load_poly(const float* coef, int j) {
  const float4 v = *reinterpret_cast<const float4*>(coef + 4 * j);
  return PolyCoef<float>{v.x, v.y, v.z};
}
__device__ __forceinline__ PolyCoef<double> load_poly(const double* coef, int j) {
  const double2 v = *reinterpret_cast<const double2*>(coef + 4 * j);
  return PolyCoef<double>{v.x, v.y, coef[4 * j + 2]};
}

// Per-maturity polynomials of a Case II point into coef[4 j ..]: nu1^2,
// nu2^2, eta1 by one lane per maturity; then eta2^2 of each maturity by all
// G lanes, which split its quadrature nodes and sum them by a fixed-order
// butterfly (every lane gets the same total); then each lane forms the
// polynomials of the maturities it owns.
template <class R>
__device__ __forceinline__ void case2_group_coef(const R* xp, int n_mats, R l2f, const SmemQuotes<R>& sq, R* coef,
                                                 int lane, int G, unsigned gmask) {
  constexpr int CS = 4;
  const R rho0 = (R)xp[2], nu0 = (R)xp[3], dr = (R)xp[6], dn = (R)xp[7];
  for (int j = lane; j < n_mats; j += G) {
    const R T = sq.mT[j];
    R o3[3];
    case2_single<R>(rho0, nu0, (R)xp[4] * T, (R)xp[5] * T, dr, dn, (R)xp[8] * T, (R)xp[9] * T, o3);
    coef[CS * j + 0] = o3[0];
    coef[CS * j + 1] = o3[1];
    coef[CS * j + 2] = o3[2];
  }
  // eta2^2 of every maturity: all lanes share its nodes, a fixed-order
  // butterfly gives every lane the total, and the lane that owns the
  // maturity (j mod G) parks it in the slice's fourth slot ...
  for (int j = 0; j < n_mats; ++j) {
    const R T = sq.mT[j];
    const R A = (R)xp[4] * T, B = (R)xp[5] * T, Qr = (R)xp[8] * T, Qn = (R)xp[9] * T;
    const Eta2Rule<R> rule(A, B);
    const int nodes = rule.nodes();
    R part = (R)0;
    for (int k = lane; k < nodes; k += G) part += rule.node(k, rho0, nu0, A, B, dr, dn, Qr, Qn);
    for (int off = G >> 1; off > 0; off >>= 1) part += __shfl_xor_sync(gmask, part, off);
    if (lane == (j & (G - 1))) coef[CS * j + 3] = part;
  }
  // ... so that the owners then form their maturities' polynomials side by
  // side (the slots a lane reads here are the ones it wrote)
  for (int j = lane; j < n_mats; j += G) {
    const PolyCoef<R> c = dynamic_poly<R>((R)xp[0], (R)xp[1], l2f, sq.mT[j], coef[CS * j + 0], coef[CS * j + 1],
                                          coef[CS * j + 2], coef[CS * j + 3]);
    coef[CS * j + 0] = c.c0;
    coef[CS * j + 1] = c.c1;
    coef[CS * j + 2] = c.c2;
  }
}

// Partial sum of the squared residuals of one lane's quotes, FP32 Hagan
// form (quotes in pairs, SmemQuotes::pair): lane `lane` of G takes pairs
// lane, lane + G, ... (an odd count's last quote in its zero-filled pair).
// With one lane per chain
// the pairs run in straight-line chunks of PAIRS and the odd quote is
// evaluated inside the first chunk, so that its dependency chain overlaps
// the pairs' instead of running alone after them (measured +7.8% on the
// 21-strike smiles, 2.53e10 -> 2.73e10 cost-evals/s); its residual joins
// the sum after the pairs.
template <int PAIRS, bool T1>
__device__ __forceinline__ float hagan_partial(const StaticConst<float>& sc, const HaganT1& h, int n_quotes,
                                               const SmemQuotes<float>& sq, int lane, int G) {
  const int full = n_quotes >> 1;  // pairs with two quotes
  const bool odd = (n_quotes & 1) != 0;
  auto pair_r = [&](int j) {
    const float4 a = sq.pair[2 * j], b = sq.pair[2 * j + 1];
    return hagan_resid_pair<T1>(sc, make_float2(a.x, a.y), make_float2(a.z, a.w), make_float2(b.x, b.y),
                                make_float2(b.z, b.w), make_float2(1.0f, 1.0f), h);
  };
  // the odd quote alone (the scalar form of the same formula)
  auto odd_r = [&]() {
    const float4 a = sq.pair[2 * full], b = sq.pair[2 * full + 1];
    return fmaf(vol_hagan_f32<T1>(sc, h, a.x, a.z, b.x), b.z, 1.0f);
  };
  float2 acc2 = make_float2(0.0f, 0.0f);
  float r_odd = 0.0f;
  bool odd_here;
  if (G == 1) {
    odd_here = odd;
    int j = 0;
    if (full >= PAIRS) {
      float2 r[PAIRS];
      if (odd) {
#pragma unroll
        for (int k = 0; k < PAIRS; ++k) r[k] = pair_r(k);
        r_odd = odd_r();
      } else {
#pragma unroll
        for (int k = 0; k < PAIRS; ++k) r[k] = pair_r(k);
      }
#pragma unroll
      for (int k = 0; k < PAIRS; ++k) acc2 = fma2(r[k], r[k], acc2);
      j = PAIRS;
    } else if (odd) {
      r_odd = odd_r();
    }
    for (; j + PAIRS <= full; j += PAIRS) {
      float2 r[PAIRS];
#pragma unroll
      for (int k = 0; k < PAIRS; ++k) r[k] = pair_r(j + k);
#pragma unroll
      for (int k = 0; k < PAIRS; ++k) acc2 = fma2(r[k], r[k], acc2);
    }
    for (; j < full; ++j) {
      const float2 r = pair_r(j);
      acc2 = fma2(r, r, acc2);
    }
  } else {
    // several lanes: an odd count's last quote is evaluated as the first
    // element of its zero-filled pair (residual 0 for the filler), so the
    // lane that holds it runs the same instructions as the others instead
    // of a separate scalar pass while they wait
    odd_here = false;
    const int npairs = full + (odd ? 1 : 0);
#pragma unroll PAIRS
    for (int j = lane; j < npairs; j += G) {
      const float4 a = sq.pair[2 * j], b = sq.pair[2 * j + 1];
      const float2 r = hagan_resid_pair<T1>(sc, make_float2(a.x, a.y), make_float2(a.z, a.w),
                                            make_float2(b.x, b.y), make_float2(b.z, b.w),
                                            make_float2(1.0f, 2 * j + 1 < n_quotes ? 1.0f : 0.0f), h);
      acc2 = fma2(r, r, acc2);
    }
  }
  if (odd_here) acc2.x = fmaf(r_odd, r_odd, acc2.x);
  return acc2.x + acc2.y;
}

// The FP32 Hagan cost with one lane per chain and at least PAIRS pairs,
// for a step loop specialised to that case (and to the parity of the quote
// count, ODD): the static constants of the point, the first chunk of pairs
// and the odd quote form one straight-line block, so the constants'
// dependency chain (a reciprocal and two logarithms) overlaps the chunk's
// first pairs.  Same operations and order of summation as group_cost at
// G = 1 (hagan_partial), so the same result bit for bit.
template <int PAIRS, bool ODD, bool T1>
__device__ __forceinline__ DF hagan_cost_g1(const float* xp, int n_quotes, const SmemQuotes<float>& sq) {
  const StaticConst<float> sc = static_setup<float>(xp);
  const HaganT1 h = T1 ? hagan_t1(sc, sq.mT[0]) : HaganT1{0.0f, 0.0f, 0.0f};
  const int full = n_quotes >> 1;
  auto pair_r = [&](int j) {
    const float4 a = sq.pair[2 * j], b = sq.pair[2 * j + 1];
    return hagan_resid_pair<T1>(sc, make_float2(a.x, a.y), make_float2(a.z, a.w), make_float2(b.x, b.y),
                                make_float2(b.z, b.w), make_float2(1.0f, 1.0f), h);
  };
  float2 r[PAIRS];
#pragma unroll
  for (int k = 0; k < PAIRS; ++k) r[k] = pair_r(k);
  float r_odd = 0.0f;
  if constexpr (ODD) {
    const float4 a = sq.pair[2 * full], b = sq.pair[2 * full + 1];
    r_odd = fmaf(vol_hagan_f32<T1>(sc, h, a.x, a.z, b.x), b.z, 1.0f);
  }
  float2 acc2 = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int k = 0; k < PAIRS; ++k) acc2 = fma2(r[k], r[k], acc2);
  int j = PAIRS;
  for (; j + PAIRS <= full; j += PAIRS) {
#pragma unroll
    for (int k = 0; k < PAIRS; ++k) r[k] = pair_r(j + k);
#pragma unroll
    for (int k = 0; k < PAIRS; ++k) acc2 = fma2(r[k], r[k], acc2);
  }
  for (; j < full; ++j) {
    const float2 q = pair_r(j);
    acc2 = fma2(q, q, acc2);
  }
  if constexpr (ODD) acc2.x = fmaf(r_odd, r_odd, acc2.x);
  return DF{acc2.x + acc2.y, 0.0f};
}

// The Hagan cost of SD points at once (the speculative step loop of the
// level kernel): every lane evaluates its quotes for each point, with the
// lane assignment, order of summation and arithmetic of group_cost for
// each point, so each result equals group_cost's bit for bit; the SD
// evaluations are independent work for the scheduler.
template <class R, int PAIRS, int SD>
__device__ __forceinline__ void group_costn_hagan(const R (&xs)[SD][4], int n_quotes, const SmemQuotes<R>& sq,
                                                  int lane, int G, unsigned gmask,
                                                  typename CostOf<R>::T (&fs)[SD]) {
  R acc[SD];
  if constexpr (sizeof(R) == 4) {
    StaticConst<float> sc[SD];
#pragma unroll
    for (int k = 0; k < SD; ++k) sc[k] = static_setup<float>(xs[k]);
    const int full = n_quotes >> 1;
    const int npairs = full + (n_quotes & 1);
    float2 a2[SD];
#pragma unroll
    for (int k = 0; k < SD; ++k) a2[k] = make_float2(0.0f, 0.0f);
#pragma unroll PAIRS
    for (int j = lane; j < npairs; j += G) {
      const float4 a = sq.pair[2 * j], b = sq.pair[2 * j + 1];
      const float2 lfk = make_float2(a.x, a.y), l2kf = make_float2(a.z, a.w), T = make_float2(b.x, b.y),
                   wn = make_float2(b.z, b.w), one = make_float2(1.0f, 2 * j + 1 < n_quotes ? 1.0f : 0.0f);
#pragma unroll
      for (int k = 0; k < SD; ++k) {
        const float2 r = hagan_resid_pair(sc[k], lfk, l2kf, T, wn, one);
        a2[k] = fma2(r, r, a2[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < SD; ++k) acc[k] = a2[k].x + a2[k].y;
  } else {
    StaticConst<R> sc[SD];
#pragma unroll
    for (int k = 0; k < SD; ++k) {
      sc[k] = static_setup<R>(xs[k]);
      acc[k] = (R)0;
    }
    for (int q = lane; q < n_quotes; q += G) {
      const QuotePack<R> qp = sq.pack[q];
#pragma unroll
      for (int k = 0; k < SD; ++k) {
        const R r = resid(vol_hagan<R>(sc[k], qp.lfk, qp.l2kf, qp.T), qp.w);
        acc[k] += r * r;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < SD; ++k) fs[k] = lanes_sum(acc[k], G, gmask);
}

// FP32 Case II: the four functions of eq. (integrales_SABRd) of every
// maturity from one composite rule over [0, Tmax] whose panels end at the
// maturities (sub-panels and nodes prepared per problem, case2_rule_build).
// With nu(t) = (nu0 + q_nu t) e^{-bt} + d_nu, rho(t) = (rho0 + q_rho t) e^{-at}
// + d_rho and G(t) = int_0^t nu rho, in real time:
//   nu1^2 = 3 A/T^3, A = int_0^T (T-t)^2 nu^2     nu2^2 = 6 D/T^3, D = int_0^T (T-t) t nu^2
//   eta1  = 2 H/T^2, H = int_0^T (T-t) nu rho     eta2^2 = 12 K/T^4, K = int_0^T (T-t) G^2
// (the last by Fubini from the triple integral).  Each panel j contributes
// its own integrals with weights in T_j - t; across panels the totals obey
// positive recurrences in Delta = T_j - T_{j-1} (e.g. A_j = A_{j-1} +
// Delta (2 B_{j-1} + Delta C_{j-1}) + a_j with B = int (T-t) nu^2,
// C = int nu^2), so no difference of large terms is formed.  Lanes take
// whole panels (maturity j on lane j mod G); at a node only nu and rho are
// evaluated (two 2^x), G inside a sub-panel comes from the Gauss-Legendre
// integration matrix, and G at a panel's start from a scan over the lanes.
// With G = G_start + g(t), the panel's integrals of G^2 are kept as
// coefficients of a quadratic in G_start (P0, P1, P2), so every node is
// evaluated once.  `loc` holds 12 slots per maturity for the panel
// integrals; coef[4 j ..] receives nu1^2, nu2^2, eta1, eta2^2 and then the
// polynomial of maturity j.
__device__ __forceinline__ void case2_group_coef_rule(const float* xp, int n_mats, float l2f,
                                                      const SmemQuotes<float>& sq, float* coef, float* loc, int lane,
                                                      int G, unsigned gmask) {
  const float rho0 = xp[2], nu0 = xp[3], dr = xp[6], dn = xp[7], qr = xp[8], qn = xp[9];
  const float na2 = -xp[4] * 1.4426950408889634f, nb2 = -xp[5] * 1.4426950408889634f;
  float carry = 0.0f;  // G at the start of this round's first panel
  for (int r0 = 0; r0 < n_mats; r0 += G) {
    const int j = r0 + lane;
    float c_ = 0.f, e_ = 0.f, b_ = 0.f, a_ = 0.f, d_ = 0.f, n_ = 0.f, h_ = 0.f;
    float P0 = 0.f, P1 = 0.f, P2 = 0.f, Q0 = 0.f, Q1 = 0.f, Q2 = 0.f;
    if (j < n_mats) {
      const int2 pr = sq.c2_panel[j];
      for (int sbi = pr.x; sbi < pr.x + pr.y; ++sbi) {
        const float4 sub = sq.c2_sub[sbi];  // half width, sum W, sum tau W
        const float cin = n_;               // int of nu rho from the panel start
        const float4* nd = sq.c2_node + kC2Nodes * sbi;
        float f[kC2Nodes];
#pragma unroll
        for (int k = 0; k < kC2Nodes; ++k) {
          const float4 q = nd[k];  // u, W, tau
          const float eb = ex2_approx(nb2 * q.x), ea = ex2_approx(na2 * q.x);
          const float nu = fmaf(fmaf(qn, q.x, nu0), eb, dn);
          const float rho = fmaf(fmaf(qr, q.x, rho0), ea, dr);
          f[k] = nu * rho;
          const float wn = q.y * nu * nu;
          c_ += wn;
          e_ = fmaf(q.x, wn, e_);
          b_ = fmaf(q.z, wn, b_);
          const float twn = q.z * wn;
          a_ = fmaf(q.z, twn, a_);
          d_ = fmaf(q.x, twn, d_);
          const float wf = q.y * f[k];
          n_ += wf;
          h_ = fmaf(q.z, wf, h_);
        }
        float s1 = 0.f, s2 = 0.f, t1 = 0.f, t2 = 0.f;
#pragma unroll
        for (int k = 0; k < kC2Nodes; ++k) {
          float g = 0.f;
#pragma unroll
          for (int i = 0; i < kC2Nodes; ++i) g = fmaf(kC2.S[k][i], f[i], g);
          g *= sub.x;
          const float4 q = nd[k];
          const float wg = q.y * g, twg = q.z * wg;
          s1 += wg;
          s2 = fmaf(wg, g, s2);
          t1 += twg;
          t2 = fmaf(twg, g, t2);
        }
        // int W (Gs + cin + g)^2 as a quadratic in Gs, the G at the panel start
        P0 += sub.y;
        P1 += fmaf(cin, sub.y, s1);
        P2 += fmaf(cin, fmaf(cin, sub.y, 2.0f * s1), s2);
        Q0 += sub.z;
        Q1 += fmaf(cin, sub.z, t1);
        Q2 += fmaf(cin, fmaf(cin, sub.z, 2.0f * t1), t2);
      }
    }
    // G at each panel's start: exclusive scan of the panels' int nu rho
    float incl = n_;
    for (int off = 1; off < G; off <<= 1) {
      const float y = __shfl_up_sync(gmask, incl, off, G);
      if (lane >= off) incl += y;
    }
    const float Gs = carry + (incl - n_);
    carry += __shfl_sync(gmask, incl, G - 1, G);
    if (j < n_mats) {
      float* L = loc + 12 * j;
      L[0] = c_;
      L[1] = e_;
      L[2] = b_;
      L[3] = a_;
      L[4] = d_;
      L[5] = n_;
      L[6] = h_;
      L[7] = fmaf(Gs, fmaf(Gs, P0, 2.0f * P1), P2);  // int G^2 over the panel
      L[8] = fmaf(Gs, fmaf(Gs, Q0, 2.0f * Q1), Q2);  // int (T_j - t) G^2
    }
  }
  __syncwarp(gmask);
  // the recurrences over the panels (every lane runs them; lane j mod G
  // forms maturity j's functions and polynomial)
  float C = 0.f, E = 0.f, B = 0.f, A = 0.f, D = 0.f, N = 0.f, H = 0.f, I = 0.f, K = 0.f, Tp = 0.f;
  for (int j = 0; j < n_mats; ++j) {
    const float T = sq.mT[j], dl = T - Tp;
    const float* L = loc + 12 * j;
    A += fmaf(dl, fmaf(dl, C, 2.0f * B), L[3]);
    B += fmaf(dl, C, L[2]);
    C += L[0];
    D += fmaf(dl, E, L[4]);
    E += L[1];
    H += fmaf(dl, N, L[6]);
    N += L[5];
    K += fmaf(dl, I, L[8]);
    I += L[7];
    Tp = T;
    if ((j & (G - 1)) == lane) {
      const float iT = rcp_approx(T), iT2 = iT * iT;
      const PolyCoef<float> c = dynamic_poly<float>(xp[0], xp[1], l2f, T, 3.0f * A * iT2 * iT, 6.0f * D * iT2 * iT,
                                                    2.0f * H * iT2, 12.0f * K * iT2 * iT2);
      coef[4 * j + 0] = c.c0;
      coef[4 * j + 1] = c.c1;
      coef[4 * j + 2] = c.c2;
    }
  }
}

// Cost of point xp evaluated by the G lanes of one chain group.  Lane `lane`
// takes quotes lane, lane+G, ...; per-lane partial sums are combined by
// lanes_sum.
// For the dynamic models the lanes first compute the per-maturity polynomial
// of eq. (vola_SABRd) into `coef` (this group's slice of shared memory).
// PAIRS: quote pairs the FP32 Hagan loop keeps in flight (more independent
// work for the scheduler, at the price of registers: the 128-register
// kernels use 2, the plans' persistent launch, which runs four 64-thread
// blocks per SM and so may use up to 255 registers, uses 5 -- measured on
// the 21-strike smiles against 2, 3, 4 and 6, and against chunks of 4, 6 and
// 11 pairs with the odd quote's pair inside the last chunk).
template <class R, int MODEL, int PAIRS = 2>
__device__ __forceinline__ typename CostOf<R>::T group_cost(const R* xp, int n_quotes, int n_mats, R l2f,
                                             const SmemQuotes<R>& sq, R* coef, int lane, int G,
                                             unsigned gmask) {
  R acc = (R)0;
  if constexpr (MODEL == SABR_HAGAN && sizeof(R) == 4) {
    const StaticConst<float> sc = static_setup<float>(xp);
    // one lane per chain and one maturity: the folded numerator (HaganT1),
    // as in the one-lane step loop (hagan_cost_g1)
    if (G == 1 && n_mats == 1) {
      acc = hagan_partial<PAIRS, true>(sc, hagan_t1(sc, sq.mT[0]), n_quotes, sq, lane, G);
    } else {
      acc = hagan_partial<PAIRS, false>(sc, HaganT1{0.0f, 0.0f, 0.0f}, n_quotes, sq, lane, G);
    }
  } else if (MODEL == SABR_HAGAN || MODEL == SABR_OBLOJ) {
    const StaticConst<R> sc = static_setup<R>(xp);
#pragma unroll 3
    for (int q = lane; q < n_quotes; q += G) {
      const QuotePack<R> qp = sq.pack[q];
      const R v = (MODEL == SABR_HAGAN) ? vol_hagan<R>(sc, qp.lfk, qp.l2kf, qp.T)
                                        : vol_obloj<R>(sc, qp.lfk, qp.l2kf, sq.l2k[q], qp.T);
      const R r = resid(v, qp.w);
      acc += r * r;
    }
  } else if (MODEL == SABR_EXPANDED) {
    const PolyCoef<R> c0 = expanded_coef<R>(xp, l2f, (R)0);
    const PolyCoef<R> c1 = expanded_coef<R>(xp, l2f, (R)1);
    const R bw = c1.c0 - c0.c0;  // B / omega
    for (int q = lane; q < n_quotes; q += G) {
      const QuotePack<R> qp = sq.pack[q];
      PolyCoef<R> c = c0;
      c.c0 = c0.c0 + bw * qp.T;
      const R r = resid(vol_poly<R>(c, qp.lfk), qp.w);
      acc += r * r;
    }
  } else {
    constexpr int CS = 4;  // polynomial slots per maturity (load_poly)
    if (MODEL == SABR_DYN_I) {
      for (int j = lane; j < n_mats; j += G) {
        const PolyCoef<R> c = dynamic_coef<R, false>(xp, l2f, sq.mT[j]);
        coef[CS * j + 0] = c.c0;
        coef[CS * j + 1] = c.c1;
        coef[CS * j + 2] = c.c2;
      }
    } else if constexpr (sizeof(R) == 4) {
      case2_group_coef_rule(xp, n_mats, l2f, sq, coef, coef + 4 * n_mats, lane, G, gmask);
    } else {
      case2_group_coef<R>(xp, n_mats, l2f, sq, coef, lane, G, gmask);
    }
    __syncwarp(gmask);
    for (int q = lane; q < n_quotes; q += G) {
      const QuotePack<R> qp = sq.pack[q];
      const PolyCoef<R> c = load_poly(coef, mat_of_slot(qp.l2kf));
      const R r = resid(vol_poly<R>(c, qp.lfk), qp.w);
      acc += r * r;
    }
    __syncwarp(gmask);
  }
  return lanes_sum(acc, G, gmask);
}


}  // namespace sabr
