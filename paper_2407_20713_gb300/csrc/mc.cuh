// mc.cuh -- fused Monte Carlo pricer of Sec. 4: one thread per path, the
// log-Euler scheme of eq. (dis_SABRd) in log space, payoffs of every option
// of a maturity accumulated when the path lands on it, eq. (payoff).
#pragma once
#include <cstdint>

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

__device__ __forceinline__ uint4 path_words(const McDev& P, int64_t path, int i) {
  return philox4x32_10(make_uint4((uint32_t)path, (uint32_t)(i >> 1), 0u, kTagMC), P.rk);
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

// Paths per thread of the pricing kernel: independent paths advance step by
// step together (independent dependency chains for the scheduler; three
// measured fastest against two and four).
constexpr int kMcPathsPerThread = 3;

// Simulates, with every thread of the grid, the paths path0 + k pstride
// (k = 0 .. kMcPathsPerThread - 1), then the next kMcPathsPerThread
// pstride, ... of one parameter set and adds, per warp, the sums of payoff
// and payoff^2 of every option to wacc[warp][slot * 32 + lane] (FP64).
// Values of maturity m are laid out as (option j, kind k) -> value 2 j + k,
// in chunks of 32 starting at slot mat_slot[m].  Steps go in pairs: one
// Philox block per path feeds both.
template <class R>
__device__ __forceinline__ void simulate_paths(const McDev& P, const double* p,
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
      for (int k = 0; k < NPT; ++k) w[k] = path_words(P, path[k], i);
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

}  // namespace sabr
