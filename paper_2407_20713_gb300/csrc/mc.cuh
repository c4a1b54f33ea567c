// mc.cuh -- fused Monte Carlo pricer of Sec. 4: one thread per path, the
// log-Euler scheme of eq. (dis_SABRd) in log space, payoffs of every option
// of a maturity accumulated when the path lands on it, eq. (payoff).
#pragma once
#include <cstdint>

#include "../../include/sabr.h"
#include "sabr_math.cuh"

namespace sabr {

constexpr int kMcBlock = 128;         // threads per MC block (4 warps)
constexpr int kMcWarps = kMcBlock / 32;
constexpr int kMaxMcQuotes = 512;     // options per pricing call
constexpr int kMaxMcSteps = 8192;     // grid points per path

// One pricing problem (quotes sorted by maturity; all pointers device).
struct McDev {
  int model;          // static models use constant nu, rho
  int n_quotes, n_mats, n_steps, n_slots;
  int64_t n_paths;
  double fwd, log_absorb;  // ln(1e-12 f)
  uint32_t key0, key1;
  PhiloxKeys rk;           // the ten round keys of (key0, key1): kernel
                           // parameters, read as constants by the path loop
  const double* step_t;    // [n_steps] right end t_{i+1} of step i, where
                           // its nu(t), rho(t) are taken
  const double* step_h;    // [n_steps] length of step i
  const int* step_mat;     // [n_steps] maturity reached at the end of step i, or -1
  const int* mat_q0;       // [n_mats] first quote of each maturity
  const int* mat_nq;       // [n_mats] its number of quotes
  const int* mat_slot;     // [n_mats] first accumulator slot (32 values each)
  const double* K;         // [n_quotes]
  const int8_t* is_call;   // [n_quotes]
};

// Butterfly reduce-scatter across a warp: on entry every lane holds 32
// values v[0..31]; on exit lane l holds the warp sum of value l.  Five
// levels, 16+8+4+2+1 shuffles, fixed order (deterministic).
template <class R>
__device__ __forceinline__ R warp_reduce_scatter32(R (&v)[32], int lane) {
#pragma unroll
  for (int lvl = 0; lvl < 5; ++lvl) {
    const int half = 16 >> lvl;
    const bool upper = (lane & half) != 0;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const R keep = upper ? v[k + half] : v[k];
      const R send = upper ? v[k] : v[k + half];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, half);
    }
  }
  return v[0];
}

// Path state units: FP32 paths carry log2 F and log2 alpha, so that nu-hat =
// alpha F^(beta-1) and F come from one SFU exp2 each; FP64 paths carry the
// natural logarithms.  kLogUnit converts a natural-log increment.
template <class R> struct PathUnits;
template <> struct PathUnits<float> {
  static constexpr double kLogUnit = 1.4426950408889634;  // 1/ln 2
  __device__ static float expu(float x) { return ex2_approx(x); }
  __host__ __device__ static double logu(double x) { return log2(x); }
};
template <> struct PathUnits<double> {
  static constexpr double kLogUnit = 1.0;
  __device__ static double expu(double x) { return exp(x); }
  __host__ __device__ static double logu(double x) { return log(x); }
};

// Per-block step coefficients, in shared memory (one 16-byte load per step
// in FP32), scaled by the log unit u:
//   a_i = u nu_i sqrt(h_i)    (vol step; its drift -u nu_i^2 h_i / 2 is
//                              -a_i^2 / (2 u), formed in the step)
//   c_i = u rho_i sqrt(h_i)   d_i = u sqrt(1 - rho_i^2) sqrt(h_i)
//   e_i = -u h_i / 2
template <class R> struct __align__(16) StepCoef {
  R a, c, d, e;
};

// Also writes land[m] = the step whose end is maturity m.
template <class R>
__device__ __forceinline__ void build_steps(const McDev& P, const double* p, StepCoef<R>* tab,
                                            int* land) {
  for (int i = threadIdx.x; i < P.n_steps; i += blockDim.x) {
    const double h = P.step_h[i], t = P.step_t[i];
    double nu, rho;
    if (P.model == SABR_DYN_I) {
      rho = p[2] * exp(-p[4] * t);
      nu = p[3] * exp(-p[5] * t);
    } else if (P.model == SABR_DYN_II) {
      rho = (p[2] + p[8] * t) * exp(-p[4] * t) + p[6];
      nu = (p[3] + p[9] * t) * exp(-p[5] * t) + p[7];
    } else {
      rho = p[2];
      nu = p[3];
    }
    const double sh = sqrt(h);
    const double u = PathUnits<R>::kLogUnit;
    StepCoef<R> s;
    s.a = (R)(u * nu * sh);
    s.c = (R)(u * rho * sh);
    s.d = (R)(u * sqrt(fmax(0.0, (1.0 - rho) * (1.0 + rho))) * sh);
    s.e = (R)(-0.5 * u * h);
    tab[i] = s;
    const int m = P.step_mat[i];
    if (m >= 0) land[m] = i;
  }
}

// FP32: SFU forms.  -2 ln u1 = -2 ln 2 log2 u1 lies in (0, 34] for u1 in
// [2^-24, 1 - 2^-24], so sqrt = s rsqrt(s); the angle 2 pi u2 - pi lies in
// (-pi, pi), where the SFU sine and cosine keep an absolute error below
// 2^-21, and (cos, sin)(2 pi u2) = -(cos, sin)(2 pi u2 - pi).  Every operand
// is a normal number, so the flush-to-zero forms apply.
__device__ __forceinline__ void box_muller(float u1, float u2, float& z1, float& z2) {
  const float s2 = -1.38629436111989061f * lg2_approx(u1);
  const float r = s2 * rsqrt_approx(s2);
  const float ang = 6.28318530717958647692f * u2 - 3.14159265358979323846f;
  const float s = sin_approx(ang), c = cos_approx(ang);
  z1 = -r * c;
  z2 = -r * s;
}
__device__ __forceinline__ void box_muller(double u1, double u2, double& z1, double& z2) {
  const double r = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  z1 = r * c;
  z2 = r * s;
}

// State of one path in log units, and one step of the log-Euler scheme of
// eq. (dis_SABRd): the normals of steps 2m and 2m + 1 come, by Box-Muller,
// from words (x, y) and (z, w) of Philox block (path, m, 0, tag) -- see
// path_words; nu-hat uses the old alpha and the old F.  A path is absorbed
// once F < 1e-12 f (its F reads 0 from then on).
template <class R> struct PathState {
  R lnF, lnA;
  bool absorbed;
};

// The FP32 loops read the ten round keys as kernel parameters; the FP64 loop
// (register-heavy) steps the key schedule instead.  Same words either way.
template <class R = float>
__device__ __forceinline__ uint4 path_words(const McDev& P, int64_t path, int i) {
  const uint4 c = make_uint4((uint32_t)path, (uint32_t)(i >> 1), 0u, kTagMC);
  if constexpr (sizeof(R) == 4) {
    return philox4x32_10(c, P.rk);
  } else {
    return philox4x32_10(c, P.key0, P.key1);
  }
}

template <class R>
__device__ __forceinline__ void path_step(const StepCoef<R>& s, uint32_t wa, uint32_t wb, R beta_m1, R log_abs,
                                          PathState<R>& st) {
  R z1, z2;
  box_muller(u01<R>(wa), u01<R>(wb), z1, z2);
  const R nuhat = PathUnits<R>::expu(st.lnA + beta_m1 * st.lnF);
  st.lnF = st.lnF + nuhat * (s.c * z1 + s.d * z2) + nuhat * nuhat * s.e;
  const R b_over_a = s.a * (R)(-0.5 / PathUnits<R>::kLogUnit);  // b = a * b_over_a
  st.lnA = st.lnA + s.a * (z1 + b_over_a);
  st.absorbed = st.absorbed || !(st.lnF >= log_abs);
}

// Paths per thread: independent paths advance step by step together
// (independent dependency chains for the scheduler).  The cliquet kernel and
// the FP64 pricer take three (measured fastest against two and four in the
// scalar form); the FP32 pricer takes four, two pairs of paths stepped with
// the packed FP32x2 instructions (simulate_paths<float>).
constexpr int kMcPathsPerThread = 3;
template <class R> struct McPathsPerThread {
  static constexpr int value = sizeof(R) == 4 ? 4 : kMcPathsPerThread;
};
__host__ __device__ constexpr int mc_paths_per_thread(int prec) { return prec == SABR_FP32 ? 4 : kMcPathsPerThread; }

// Simulates, with every thread of the grid, the paths path0 + k pstride
// (k = 0 .. kMcPathsPerThread - 1), then the next kMcPathsPerThread
// pstride, ... of one parameter set and adds, per warp, the sums of payoff
// and payoff^2 of every option to wacc[warp][slot * 32 + lane] (FP64).
// Values of maturity m are laid out as (option j, kind k) -> value 2 j + k,
// in chunks of 32 starting at slot mat_slot[m].  Steps go in pairs: one
// Philox block per path feeds both.
template <class R>
__device__ __forceinline__ void simulate_paths_scalar(const McDev& P, const double* p,
                                               const StepCoef<R>* tab, const int* land,
                                               const int* s_q0, const int* s_nq, const int* s_slot,
                                               const R* sK, const int8_t* scall, int64_t path0,
                                               int64_t pstride, double* wacc) {
  constexpr int NPT = kMcPathsPerThread;
  const int lane = threadIdx.x & 31;
  const R beta_m1 = (R)(p[1] - 1.0);
  const R lnf = (R)PathUnits<R>::logu(P.fwd), lna = (R)PathUnits<R>::logu(p[0]);
  const R log_abs = (R)(P.log_absorb * PathUnits<R>::kLogUnit);
  const int64_t n_paths = P.n_paths;
  const int n_steps = P.n_steps;
  // every lane of the warp runs the same trip count (idle lanes pay 0)
  const int64_t warp_path0 = path0 - lane;
  for (int64_t wp = warp_path0; wp < n_paths; wp += NPT * pstride) {
    int64_t path[NPT];
    bool live[NPT];
    PathState<R> st[NPT];
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      path[k] = wp + k * pstride + lane;
      live[k] = path[k] < n_paths;
      st[k] = PathState<R>{lnf, lna, false};
    }
    int m = 0, i_land = land[0];  // next maturity and the step it ends
    // payoffs of maturity m on the NPT paths, summed into the warp rows
    auto pay_out = [&]() {
      R F[NPT];
#pragma unroll
      for (int k = 0; k < NPT; ++k) F[k] = st[k].absorbed || !live[k] ? (R)0 : PathUnits<R>::expu(st[k].lnF);
      const int q0 = s_q0[m], nq = s_nq[m], slot0 = s_slot[m];
      for (int c0 = 0; c0 < 2 * nq; c0 += 32) {
        R v[32];
#pragma unroll
        for (int kk = 0; kk < 32; kk += 2) {
          const int j = (c0 + kk) >> 1;
          R pay = (R)0, pay2 = (R)0;
          if (j < nq) {
            const R K = sK[q0 + j];
            const bool call = scall[q0 + j] != 0;
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
              const R x = call ? (F[k] > K ? F[k] - K : (R)0) : (K > F[k] ? K - F[k] : (R)0);
              const R y = live[k] ? x : (R)0;
              pay += y;
              pay2 += y * y;
            }
          }
          v[kk] = pay;
          v[kk + 1] = pay2;
        }
        const R tot = warp_reduce_scatter32<R>(v, lane);
        const int slot = slot0 + (c0 >> 5);
        wacc[slot * 32 + lane] += (double)tot;
      }
      ++m;
      i_land = m < P.n_mats ? land[m] : -1;
    };
    for (int i = 0; i < n_steps; i += 2) {
      uint4 w[NPT];
#pragma unroll
      for (int k = 0; k < NPT; ++k) w[k] = path_words<R>(P, path[k], i);
      {
        const StepCoef<R> s = tab[i];
#pragma unroll
        for (int k = 0; k < NPT; ++k) path_step<R>(s, w[k].x, w[k].y, beta_m1, log_abs, st[k]);
      }
      if (i == i_land) pay_out();
      if (i + 1 < n_steps) {
        const StepCoef<R> s = tab[i + 1];
#pragma unroll
        for (int k = 0; k < NPT; ++k) path_step<R>(s, w[k].z, w[k].w, beta_m1, log_abs, st[k]);
        if (i + 1 == i_land) pay_out();
      }
    }
  }
}

// Two FP32 paths of one log-Euler step (path_step<float>) with the packed
// FP32x2 instructions: the adds, multiplies and FMAs of both paths share an
// issue slot; the SFU operations and the absorption test stay per path.  The
// normals are z1 = -r cos, z2 = -r sin; with zr1 = r cos, zr2 = r sin the
// signs go into the step coefficients (nc = -c, nd = -d, passed negated).
__device__ __forceinline__ void path_step2(float a, float nc, float nd, float e, uint32_t wa0, uint32_t wb0,
                                           uint32_t wa1, uint32_t wb1, float beta_m1, float log_abs, float2& lnF,
                                           float2& lnA, bool& abs0, bool& abs1) {
  const float2 u1 = make_float2(u01<float>(wa0), u01<float>(wa1));
  const float2 u2 = make_float2(u01<float>(wb0), u01<float>(wb1));
  const float2 s2 = mul2(f2(-1.38629436111989061f), make_float2(lg2_approx(u1.x), lg2_approx(u1.y)));
  const float2 r = mul2(s2, make_float2(rsqrt_approx(s2.x), rsqrt_approx(s2.y)));
  const float2 ang = fma2(f2(6.28318530717958647692f), u2, f2(-3.14159265358979323846f));
  const float2 zr1 = mul2(r, make_float2(cos_approx(ang.x), cos_approx(ang.y)));
  const float2 zr2 = mul2(r, make_float2(sin_approx(ang.x), sin_approx(ang.y)));
  // nu-hat from the old alpha and the old F
  const float2 arg = fma2(f2(beta_m1), lnF, lnA);
  const float2 nuhat = make_float2(ex2_approx(arg.x), ex2_approx(arg.y));
  const float2 t = fma2(f2(nd), zr2, mul2(f2(nc), zr1));  // c z1 + d z2
  lnF = fma2(nuhat, fma2(nuhat, f2(e), t), lnF);
  const float b = a * (float)(-0.5 / PathUnits<float>::kLogUnit);
  lnA = fma2(f2(a), fma2(zr1, f2(-1.0f), f2(b)), lnA);  // a (z1 + b)
  abs0 = abs0 || !(lnF.x >= log_abs);
  abs1 = abs1 || !(lnF.y >= log_abs);
}

// The FP32 path loop: four paths per thread as two pairs (path_step2); the
// same path numbering, Philox counters, landing steps and payoff
// accumulation as simulate_paths_scalar.
__device__ __forceinline__ void simulate_paths_f32(const McDev& P, const double* p, const StepCoef<float>* tab,
                                                   const int* land, const int* s_q0, const int* s_nq,
                                                   const int* s_slot, const float* sK, const int8_t* scall,
                                                   int64_t path0, int64_t pstride, double* wacc) {
  constexpr int NPT = 4;
  const int lane = threadIdx.x & 31;
  const float beta_m1 = (float)(p[1] - 1.0);
  const float lnf = (float)PathUnits<float>::logu(P.fwd), lna = (float)PathUnits<float>::logu(p[0]);
  const float log_abs = (float)(P.log_absorb * PathUnits<float>::kLogUnit);
  const int64_t n_paths = P.n_paths;
  const int n_steps = P.n_steps;
  const int64_t warp_path0 = path0 - lane;
  for (int64_t wp = warp_path0; wp < n_paths; wp += NPT * pstride) {
    int64_t path[NPT];
    bool live[NPT], absd[NPT];
    float2 lnF[2], lnA[2];
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      path[k] = wp + k * pstride + lane;
      live[k] = path[k] < n_paths;
      absd[k] = false;
    }
    lnF[0] = lnF[1] = make_float2(lnf, lnf);
    lnA[0] = lnA[1] = make_float2(lna, lna);
    int m = 0, i_land = land[0];
    auto pay_out = [&]() {
      float F[NPT];
#pragma unroll
      for (int k = 0; k < NPT; ++k) {
        const float lf = (k & 1) ? lnF[k >> 1].y : lnF[k >> 1].x;
        F[k] = absd[k] || !live[k] ? 0.0f : PathUnits<float>::expu(lf);
      }
      const int q0 = s_q0[m], nq = s_nq[m], slot0 = s_slot[m];
      for (int c0 = 0; c0 < 2 * nq; c0 += 32) {
        float v[32];
#pragma unroll
        for (int kk = 0; kk < 32; kk += 2) {
          const int j = (c0 + kk) >> 1;
          float pay = 0.0f, pay2 = 0.0f;
          if (j < nq) {
            const float K = sK[q0 + j];
            const bool call = scall[q0 + j] != 0;
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
              const float x = call ? (F[k] > K ? F[k] - K : 0.0f) : (K > F[k] ? K - F[k] : 0.0f);
              const float y = live[k] ? x : 0.0f;
              pay += y;
              pay2 += y * y;
            }
          }
          v[kk] = pay;
          v[kk + 1] = pay2;
        }
        const float tot = warp_reduce_scatter32<float>(v, lane);
        wacc[(slot0 + (c0 >> 5)) * 32 + lane] += (double)tot;
      }
      ++m;
      i_land = m < P.n_mats ? land[m] : -1;
    };
    for (int i = 0; i < n_steps; i += 2) {
      uint4 w[NPT];
#pragma unroll
      for (int k = 0; k < NPT; ++k) w[k] = path_words(P, path[k], i);
      {
        const StepCoef<float> s = tab[i];
        path_step2(s.a, -s.c, -s.d, s.e, w[0].x, w[0].y, w[1].x, w[1].y, beta_m1, log_abs, lnF[0], lnA[0],
                   absd[0], absd[1]);
        path_step2(s.a, -s.c, -s.d, s.e, w[2].x, w[2].y, w[3].x, w[3].y, beta_m1, log_abs, lnF[1], lnA[1],
                   absd[2], absd[3]);
      }
      if (i == i_land) pay_out();
      if (i + 1 < n_steps) {
        const StepCoef<float> s = tab[i + 1];
        path_step2(s.a, -s.c, -s.d, s.e, w[0].z, w[0].w, w[1].z, w[1].w, beta_m1, log_abs, lnF[0], lnA[0],
                   absd[0], absd[1]);
        path_step2(s.a, -s.c, -s.d, s.e, w[2].z, w[2].w, w[3].z, w[3].w, beta_m1, log_abs, lnF[1], lnA[1],
                   absd[2], absd[3]);
        if (i + 1 == i_land) pay_out();
      }
    }
  }
}

// The pricer's path loop in the working precision R.
template <class R>
__device__ __forceinline__ void simulate_paths(const McDev& P, const double* p, const StepCoef<R>* tab,
                                               const int* land, const int* s_q0, const int* s_nq, const int* s_slot,
                                               const R* sK, const int8_t* scall, int64_t path0, int64_t pstride,
                                               double* wacc) {
  if constexpr (sizeof(R) == 4) {
    simulate_paths_f32(P, p, tab, land, s_q0, s_nq, s_slot, sK, scall, path0, pstride, wacc);
  } else {
    simulate_paths_scalar<R>(P, p, tab, land, s_q0, s_nq, s_slot, sK, scall, path0, pstride, wacc);
  }
}

}  // namespace sabr
