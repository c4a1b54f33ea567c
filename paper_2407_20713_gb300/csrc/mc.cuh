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
  const double* step_t;    // [n_steps] left end t_i of step i
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
  __device__ static float expu(float x) { return exp2f(x); }
  __host__ __device__ static double logu(double x) { return log2(x); }
};
template <> struct PathUnits<double> {
  static constexpr double kLogUnit = 1.0;
  __device__ static double expu(double x) { return exp(x); }
  __host__ __device__ static double logu(double x) { return log(x); }
};

// Per-block step coefficients, in shared memory:
//   a_i = nu_i sqrt(h_i)      (vol step)    b_i = -nu_i^2 h_i / 2
//   c_i = rho_i sqrt(h_i)     d_i = sqrt(1 - rho_i^2) sqrt(h_i)
//   e_i = -h_i / 2
template <class R> struct StepCoef {
  R a, b, c, d, e;
};

template <class R>
__device__ __forceinline__ void build_steps(const McDev& P, const double* p, StepCoef<R>* tab,
                                            int* smat) {
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
    s.b = (R)(-0.5 * u * nu * nu * h);
    s.c = (R)(u * rho * sh);
    s.d = (R)(u * sqrt(fmax(0.0, (1.0 - rho) * (1.0 + rho))) * sh);
    s.e = (R)(-0.5 * u * h);
    tab[i] = s;
    smat[i] = P.step_mat[i];
  }
}

// FP32: SFU forms.  -2 ln u1 lies in (0, 34] for u1 in [2^-24, 1 - 2^-24], so
// sqrt = s rsqrt(s); the angle 2 pi u2 - pi lies in (-pi, pi), where the SFU
// sine and cosine keep an absolute error below 2^-21, and
// (cos, sin)(2 pi u2) = -(cos, sin)(2 pi u2 - pi).
__device__ __forceinline__ void box_muller(float u1, float u2, float& z1, float& z2) {
  const float s2 = -2.0f * __logf(u1);
  const float r = s2 * rsqrtf(s2);
  float s, c;
  __sincosf(6.28318530717958647692f * u2 - 3.14159265358979323846f, &s, &c);
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

// Simulates the paths path0, path0 + pstride, ... of one parameter set and
// adds, per warp, the sums of payoff and payoff^2 of every option to
// wacc[warp][slot * 32 + lane] (FP64).  Values of maturity m are laid out as
// (option j, kind k) -> value 2 j + k, in chunks of 32 starting at slot
// mat_slot[m].
template <class R>
__device__ __forceinline__ void simulate_paths(const McDev& P, const double* p,
                                               const StepCoef<R>* tab, const int* smat,
                                               const int* s_q0, const int* s_nq, const int* s_slot,
                                               const R* sK, const int8_t* scall, int64_t path0,
                                               int64_t pstride, double* wacc) {
  const int lane = threadIdx.x & 31;
  const R beta_m1 = (R)(p[1] - 1.0);
  const R lnf = (R)PathUnits<R>::logu(P.fwd), lna = (R)PathUnits<R>::logu(p[0]);
  const R log_abs = (R)(P.log_absorb * PathUnits<R>::kLogUnit);
  const int64_t n_paths = P.n_paths;
  // every lane of the warp runs the same trip count (idle lanes pay 0)
  const int64_t warp_path0 = path0 - lane;
  for (int64_t wp = warp_path0; wp < n_paths; wp += pstride) {
    const int64_t path = wp + lane;
    const bool live = path < n_paths;
    R lnF = lnf, lnA = lna;
    bool absorbed = false;
    uint4 w = make_uint4(0, 0, 0, 0);
    for (int i = 0; i < P.n_steps; ++i) {
      if ((i & 1) == 0)
        w = philox4x32_10(make_uint4((uint32_t)path, (uint32_t)(i >> 1), 0u, kTagMC), P.key0, P.key1);
      const uint32_t wa = (i & 1) ? w.z : w.x, wb = (i & 1) ? w.w : w.y;
      R z1, z2;
      box_muller(u01<R>(wa), u01<R>(wb), z1, z2);
      const StepCoef<R> s = tab[i];
      const R nuhat = PathUnits<R>::expu(lnA + beta_m1 * lnF);  // old alpha, old F
      lnF = lnF + nuhat * (s.c * z1 + s.d * z2) + nuhat * nuhat * s.e;
      lnA = lnA + s.a * z1 + s.b;
      absorbed = absorbed || !(lnF >= log_abs);
      const int m = smat[i];
      if (m >= 0) {
        const R F = absorbed || !live ? (R)0 : PathUnits<R>::expu(lnF);
        const int q0 = s_q0[m], nq = s_nq[m], slot0 = s_slot[m];
        for (int c0 = 0; c0 < 2 * nq; c0 += 32) {
          R v[32];
#pragma unroll
          for (int k = 0; k < 32; k += 2) {
            const int j = (c0 + k) >> 1;
            R pay = (R)0;
            if (j < nq && live) {
              const R K = sK[q0 + j];
              pay = scall[q0 + j] ? (F > K ? F - K : (R)0) : (K > F ? K - F : (R)0);
            }
            v[k] = pay;
            v[k + 1] = pay * pay;
          }
          const R tot = warp_reduce_scatter32<R>(v, lane);
          const int slot = slot0 + (c0 >> 5);
          wacc[slot * 32 + lane] += (double)tot;
        }
      }
    }
  }
}

}  // namespace sabr
