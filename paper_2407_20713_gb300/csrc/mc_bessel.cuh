// mc_bessel.cuh -- the conditional-Bessel path step: the low-bias
// alternative to the log-Euler scheme that Sec. 4 names as its fallback (the
// scheme of Chen, Oosterlee and van der Weide reduces the SABR forward, given
// the volatility path, to a time-changed CEV process; here that process is
// sampled exactly).
//
// Write dF = alpha F^beta (rho dW + sqrt(1 - rho^2) dB), dalpha = nu alpha dW
// with W, B independent.  One step [t, t + h] (nu, rho those of the step,
// taken at its right end as in the log-Euler scheme):
//  1. alpha' = alpha e^x, x = nu sqrt(h) Z_a - nu^2 h / 2 (exact);
//  2. rho int alpha dW = (rho / nu)(alpha' - alpha) exactly, formed as
//     alpha rho sqrt(h) expm1(x) / (nu sqrt(h)) (alpha rho sqrt(h) Z_a at
//     nu = 0) and applied at the start of the step:
//     Y0 = Y + shift, Y = F^(1-beta) / (1 - beta);
//  3. V = int alpha^2 ds by the trapezoidal rule, (h/2)(alpha^2 + alpha'^2);
//  4. given Y0, Y'^2 is a squared Bessel process of dimension
//     delta = 1 - beta / ((1 - beta)(1 - rho^2)) absorbed at 0, run for time
//     tau = (1 - rho^2) V.  With a = 1 - delta / 2 and m = Y0^2 / (2 tau):
//     G ~ Gamma(a); absorbed if G >= m, else
//     Y'^2 = tau ((N1 + sqrt(2 (m - G)))^2 + N2^2)
//     (the absorbed transition density is a Gamma(a)-then-Poisson mixture
//     of chi-square laws, i.e. a noncentral chi-square with 2 degrees and
//     noncentrality 2 (m - G) below the Gamma draw).  With rho^2 = 1 the
//     clock stops: Y'^2 = Y0^2 - beta / (1 - beta) V;
//  5. beta = 1: Y = ln F, Y' = Y + shift - V / 2 + sqrt((1 - rho^2) V) N1.
// At nu = 0, rho = 0 every step is exact (the absorbed CEV law itself).
//
// Random numbers of step i of path j: Philox blocks (j, i, b, kTagMB).
// Block 0: (Z_a, N1), (N2, X_0) by Box-Muller from words (0, 1), (2, 3);
// block 1: U_0 = word 0, U_b = word 1; block k + 1 (k = 1 .. 7, drawn only
// when trial k runs): X_k = first Box-Muller output of words (0, 1),
// U_k = word 2.  Gamma(a) by Marsaglia and Tsang's method (ACM TOMS 26(3),
// 2000) with shape a' = a (a >= 1) or a + 1 (a < 1, the draw then times
// U_b^(1/a)): d = a' - 1/3, c = 1/sqrt(9 d), trial k accepts d v,
// v = (1 + c X_k)^3 > 0, if U_k < 1 - 0.0331 X_k^4 or
// ln U_k < X_k^2 / 2 + d (1 - v + ln v).  After 8 rejected trials
// (probability below 1e-10) the draw is d.
#pragma once
#include "mc.cuh"

namespace sabr {

constexpr uint32_t kTagMB = 0x4D420000u;
constexpr int kBesselTrials = 8;
// Paths per thread of the conditional-Bessel loop (two independent
// dependency chains; the Gamma trials branch per path).
constexpr int kBesselPathsPerThread = 2;

// Per-step coefficients (same size as StepCoef, so the pricer's shared
// memory layout serves both schemes).
template <class R> struct __align__(16) StepCoefB {
  R kap;  // nu sqrt(h)
  R rsh;  // rho sqrt(h)
  R hh;   // h / 2
  R omr;  // 1 - rho^2
};
static_assert(sizeof(StepCoefB<float>) == sizeof(StepCoef<float>), "step table layout");
static_assert(sizeof(StepCoefB<double>) == sizeof(StepCoef<double>), "step table layout");

template <class R>
__device__ __forceinline__ void build_steps_bessel(const McDev& P, const double* p, StepCoefB<R>* tab, int* land) {
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
    StepCoefB<R> s;
    s.kap = (R)(nu * sh);
    s.rsh = (R)(rho * sh);
    s.hh = (R)(0.5 * h);
    s.omr = (R)fmax(0.0, (1.0 - rho) * (1.0 + rho));
    tab[i] = s;
    const int m = P.step_mat[i];
    if (m >= 0) land[m] = i;
  }
}

// The elementary functions of the step in each precision: FP32 takes the
// SFU forms where their error is far below the Monte Carlo noise (ln and the
// powers) and the library's expm1f and sqrtf; FP64 the library functions.
template <class R> struct BesselMath;
template <> struct BesselMath<float> {
  __device__ static float ln(float x) { return lg2_approx(x) * 0.69314718055994531f; }
  __device__ static float expm1_(float x) { return expm1f(x); }
  __device__ static float sqrt_(float x) { return sqrtf(x); }
  __device__ static float div(float a, float b) { return __fdividef(a, b); }
  __device__ static float pow_(float x, float y) { return ex2_approx(y * lg2_approx(x)); }
  __device__ static float exp_(float x) { return ex2_approx(x * 1.4426950408889634f); }
};
template <> struct BesselMath<double> {
  __device__ static double ln(double x) { return log(x); }
  __device__ static double expm1_(double x) { return expm1(x); }
  __device__ static double sqrt_(double x) { return sqrt(x); }
  __device__ static double div(double a, double b) { return a / b; }
  __device__ static double pow_(double x, double y) { return pow(x, y); }
  __device__ static double exp_(double x) { return exp(x); }
};

template <class R>
__device__ __forceinline__ uint4 bessel_words(const McDev& P, int64_t path, int i, uint32_t b) {
  const uint4 c = make_uint4((uint32_t)path, (uint32_t)i, b, kTagMB);
  if constexpr (sizeof(R) == 4) {
    return philox4x32_10(c, P.rk);
  } else {
    return philox4x32_10(c, P.key0, P.key1);
  }
}

// Per-step constants shared by every path of the step.
template <class R> struct BesselStep {
  StepCoefB<R> s;
  R inv_kap;        // 1 / kap, or 0 at nu = 0
  R a, d, c, inva;  // Gamma shape, Marsaglia-Tsang d and c, 1/a for a < 1 (else 0)
};

template <class R>
__device__ __forceinline__ BesselStep<R> bessel_step_setup(const StepCoefB<R>& s, R bb) {
  using M = BesselMath<R>;
  BesselStep<R> k;
  k.s = s;
  k.inv_kap = s.kap > (R)0 ? (R)1 / s.kap : (R)0;
  k.a = k.d = k.c = k.inva = (R)0;
  if (s.omr > (R)0) {
    k.a = (R)0.5 + (R)0.5 * bb / s.omr;
    const R ap = k.a >= (R)1 ? k.a : k.a + (R)1;
    k.d = ap - (R)(1.0 / 3.0);
    k.c = (R)1 / M::sqrt_((R)9 * k.d);
    k.inva = k.a < (R)1 ? (R)1 / k.a : (R)0;
  }
  return k;
}

template <class R>
__device__ __forceinline__ R bessel_gamma(const McDev& P, const BesselStep<R>& k, int64_t path, int i, R x0, R u0,
                                          R ub) {
  using M = BesselMath<R>;
  R g = k.d;
  for (int t = 0; t < kBesselTrials; ++t) {
    R x = x0, u = u0;
    if (t > 0) {
      const uint4 w = bessel_words<R>(P, path, i, (uint32_t)(t + 1));
      R unused;
      box_muller(u01<R>(w.x), u01<R>(w.y), x, unused);
      u = u01<R>(w.z);
    }
    const R tt = (R)1 + k.c * x;
    if (tt > (R)0) {
      const R v = tt * tt * tt;
      const R x2 = x * x;
      if (u < (R)1 - (R)0.0331 * x2 * x2 || M::ln(u) < (R)0.5 * x2 + k.d * ((R)1 - v + M::ln(v))) {
        g = k.d * v;
        break;
      }
    }
  }
  if (k.inva > (R)0) g = g * M::pow_(ub, k.inva);
  return g;
}

// State of one path: Y = F^(1-beta)/(1-beta) (ln F at beta = 1), alpha, and
// whether it is absorbed (or not a path of the problem).
template <class R> struct BesselPath {
  R Y, A;
  bool dead;
};

template <class R, bool LOGNORMAL>
__device__ __forceinline__ void bessel_step(const McDev& P, const BesselStep<R>& k, R bb, int64_t path, int i,
                                            BesselPath<R>& st) {
  using M = BesselMath<R>;
  if (st.dead) return;
  const StepCoefB<R>& s = k.s;
  const uint4 w0 = bessel_words<R>(P, path, i, 0u), w1 = bessel_words<R>(P, path, i, 1u);
  R za, n1, n2, x0;
  box_muller(u01<R>(w0.x), u01<R>(w0.y), za, n1);
  box_muller(u01<R>(w0.z), u01<R>(w0.w), n2, x0);
  const R em = M::expm1_(s.kap * za - (R)0.5 * s.kap * s.kap);
  const R a_new = st.A + st.A * em;
  const R shift = st.A * s.rsh * (s.kap > (R)0 ? em * k.inv_kap : za);
  const R V = s.hh * (st.A * st.A + a_new * a_new);
  st.A = a_new;
  if (LOGNORMAL) {
    st.Y = st.Y + shift - (R)0.5 * V + M::sqrt_(s.omr * V) * n1;
    return;
  }
  const R Y0 = st.Y + shift;
  if (!(Y0 > (R)0)) {
    st.dead = true;
    return;
  }
  const R tau = s.omr * V;
  if (!(tau > (R)0)) {
    const R y2 = Y0 * Y0 - bb * V;
    if (!(y2 > (R)0)) {
      st.dead = true;
    } else {
      st.Y = M::sqrt_(y2);
    }
    return;
  }
  const R m = M::div(Y0 * Y0, (R)2 * tau);
  const R G = bessel_gamma<R>(P, k, path, i, x0, u01<R>(w1.x), u01<R>(w1.y));
  if (!(G < m)) {
    st.dead = true;
    return;
  }
  const R q = n1 + M::sqrt_((R)2 * (m - G));
  st.Y = M::sqrt_(tau * (q * q + n2 * n2));
}

// The path loop of the conditional-Bessel scheme: the path numbering,
// landing steps and payoff accumulation of simulate_paths_scalar, one step
// at a time.
template <class R, bool LOGNORMAL>
__device__ __forceinline__ void simulate_paths_bessel(const McDev& P, const double* p, const StepCoefB<R>* tab,
                                                      const int* land, const int* s_q0, const int* s_nq,
                                                      const int* s_slot, const R* sK, const int8_t* scall,
                                                      int64_t path0, int64_t pstride, double* wacc) {
  using M = BesselMath<R>;
  constexpr int NPT = kBesselPathsPerThread;
  const int lane = threadIdx.x & 31;
  const double beta = p[1];
  const R b1 = (R)(1.0 - beta);
  const R inv_b1 = LOGNORMAL ? (R)0 : (R)(1.0 / (1.0 - beta));
  const R bb = LOGNORMAL ? (R)0 : (R)(beta / (1.0 - beta));
  const R y_start = LOGNORMAL ? (R)log(P.fwd) : (R)(pow(P.fwd, 1.0 - beta) / (1.0 - beta));
  const R a_start = (R)p[0];
  const int64_t n_paths = P.n_paths;
  const int n_steps = P.n_steps;
  const int64_t warp_path0 = path0 - lane;
  for (int64_t wp = warp_path0; wp < n_paths; wp += NPT * pstride) {
    int64_t path[NPT];
    bool live[NPT];
    BesselPath<R> st[NPT];
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      path[k] = wp + k * pstride + lane;
      live[k] = path[k] < n_paths;
      st[k] = BesselPath<R>{y_start, a_start, !live[k]};
    }
    int m = 0, i_land = land[0];
    auto pay_out = [&]() {
      R F[NPT];
#pragma unroll
      for (int k = 0; k < NPT; ++k)
        F[k] = st[k].dead ? (R)0 : (LOGNORMAL ? M::exp_(st[k].Y) : M::pow_(b1 * st[k].Y, inv_b1));
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
        wacc[(slot0 + (c0 >> 5)) * 32 + lane] += (double)tot;
      }
      ++m;
      i_land = m < P.n_mats ? land[m] : -1;
    };
    for (int i = 0; i < n_steps; ++i) {
      const BesselStep<R> k = bessel_step_setup<R>(tab[i], bb);
#pragma unroll
      for (int j = 0; j < NPT; ++j) bessel_step<R, LOGNORMAL>(P, k, bb, path[j], i, st[j]);
      if (i == i_land) pay_out();
    }
  }
}

}  // namespace sabr
