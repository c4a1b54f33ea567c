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
constexpr int kStateLen = 12;  // restart x[10], restart f, T0

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

// Quote tables of one problem staged in shared memory.
template <class R> struct SmemQuotes {
  const QuotePack<R>* pack;  // per quote
  const R* l2k;              // per quote: log2 K (Oblój)
  const R* mT;               // per maturity: T
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
template <int MODEL> struct CoefStride {
  static constexpr int value = 4;
};
__host__ __device__ constexpr int coef_stride(int) { return 4; }

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
  constexpr int CS = CoefStride<SABR_DYN_II>::value;
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

// Cost of point xp evaluated by the G lanes of one chain group.  Lane `lane`
// takes quotes lane, lane+G, ...; per-lane partial sums are combined by
// lanes_sum.
// For the dynamic models the lanes first compute the per-maturity polynomial
// of eq. (vola_SABRd) into `coef` (this group's slice of shared memory).
template <class R, int MODEL>
__device__ __forceinline__ typename CostOf<R>::T group_cost(const R* xp, int n_quotes, int n_mats, R l2f,
                                             const SmemQuotes<R>& sq, R* coef, int lane, int G,
                                             unsigned gmask) {
  R acc = (R)0;
  if (MODEL == SABR_HAGAN || MODEL == SABR_OBLOJ) {
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
    constexpr int CS = CoefStride<MODEL>::value;
    if (MODEL == SABR_DYN_I) {
      for (int j = lane; j < n_mats; j += G) {
        const PolyCoef<R> c = dynamic_coef<R, false>(xp, l2f, sq.mT[j]);
        coef[CS * j + 0] = c.c0;
        coef[CS * j + 1] = c.c1;
        coef[CS * j + 2] = c.c2;
      }
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
