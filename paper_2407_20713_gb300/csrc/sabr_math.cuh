// sabr_math.cuh -- device arithmetic of the SABR hot path, templated on the
// working precision R (float = FP32 bulk, double = FP64 form).
//
//  * Philox4x32-10 counter-based generator and the (0,1) uniform map.
//  * z/x(z) of Sec. 2.1 eq. (equis) in a cancellation-free form.
//  * Static implied vols: eq. (haganf), eq. (sigma-SABR), eq. (vola_SABR).
//  * Dynamic coefficients nu1^2, nu2^2, eta1, eta2^2 of Sec. 2.2
//    eq. (integrales_SABRd) for Case I (eq. el_fun_1) and Case II
//    (eq. el_fun_3), and the per-maturity polynomial of eq. (vola_SABRd).
#pragma once
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

namespace sabr {

// ---------------------------------------------------------------------------
// Precision traits
// ---------------------------------------------------------------------------
template <class R> struct Tr;
template <> struct Tr<float> {
  static constexpr int kSeries = 12;          // phi_m series terms below kSeriesMax
  static constexpr double kSeriesMax = 2.0;   // (the recurrence above it)
  static constexpr int kCase1Series = 20;     // Case I series terms (argument < 2)
};
template <> struct Tr<double> {
  static constexpr int kSeries = 32;
  static constexpr double kSeriesMax = 5.0;
  static constexpr int kCase1Series = 32;
  static constexpr int kGauss = 16;
};

__device__ __forceinline__ float m_exp(float x) { return expf(x); }
__device__ __forceinline__ double m_exp(double x) { return exp(x); }
// FP32 2^x by the SFU instruction (PTX ex2.approx.ftz.f32, about 2 ulp;
// results below 2^-126 flush to zero, which no caller reaches).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float m_exp2(float x) { return ex2_approx(x); }
// The other SFU forms used by the FP32 hot loops, flush-to-zero (every
// operand they see is a normal number, so no denormal fix-up is needed):
// reciprocal (1 ulp), reciprocal square root, sine and cosine on (-pi, pi).
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sin_approx(float x) {
  float y;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float cos_approx(float x) {
  float y;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// e^x of the Case II quadrature nodes (x <= 0): in FP32 2^(x log2 e) by the
// SFU, whose relative error (a few 1e-7 for |x| < 1, growing like
// |x| 2^-24 from the rounded product) stays far inside the FP32 form's
// tolerance; in FP64 the library exp.
__device__ __forceinline__ float m_exp_node(float x) { return ex2_approx(x * 1.4426950408889634f); }
__device__ __forceinline__ double m_exp_node(double x) { return exp(x); }
__device__ __forceinline__ double m_exp2(double x) { return exp2(x); }
__device__ __forceinline__ float m_log(float x) { return logf(x); }
__device__ __forceinline__ double m_log(double x) { return log(x); }
__device__ __forceinline__ float m_log2(float x) { return log2f(x); }
__device__ __forceinline__ double m_log2(double x) { return log2(x); }
__device__ __forceinline__ float m_log1p(float x) { return log1pf(x); }
__device__ __forceinline__ double m_log1p(double x) { return log1p(x); }
__device__ __forceinline__ float m_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double m_expm1(double x) { return expm1(x); }
__device__ __forceinline__ float m_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }
// Hot-loop division and square root: in FP32 the SFU reciprocal / rsqrt
// forms (about 2 ulp), in FP64 the IEEE operations.
__device__ __forceinline__ float m_div(float a, float b) { return a * rcp_approx(b); }
__device__ __forceinline__ double m_div(double a, double b) { return a / b; }
__device__ __forceinline__ float m_sqrt_pos(float x) { return x * rsqrt_approx(x); }  // x > 0
__device__ __forceinline__ float m_rcp(float x) { return rcp_approx(x); }
__device__ __forceinline__ double m_rcp(double x) { return 1.0 / x; }
// Division by a constant: FP32 multiplies by the rounded reciprocal (one
// extra rounding), FP64 divides as written.
__device__ __forceinline__ float m_divc(float a, double c) { return a * (float)(1.0 / c); }
__device__ __forceinline__ double m_divc(double a, double c) { return a / c; }
__device__ __forceinline__ double m_sqrt_pos(double x) { return sqrt(x); }

// ---------------------------------------------------------------------------
// Compile-time tables: factorials and Gauss-Legendre rules (nodes found by
// Newton's method on P_n from cosine initial guesses, all constexpr).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr double cx_fact(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}
__host__ __device__ constexpr double cx_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 40; ++k) {
    term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    sum += term;
  }
  return sum;
}
template <int N> struct GaussRule {
  double x[N], w[N];  // nodes/weights on [-1, 1]
};
template <int N> __host__ __device__ constexpr GaussRule<N> make_gauss() {
  GaussRule<N> g{};
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < N; ++i) {
    double x = cx_cos(pi * (i + 0.75) / (N + 0.5));
    double p = 0, dp = 1;
    for (int it = 0; it < 60; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 1; k < N; ++k) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      p = p1;
      dp = N * (x * p1 - p0) / (x * x - 1.0);
      x -= p / dp;
    }
    double p0 = 1.0, p1 = x;
    for (int k = 1; k < N; ++k) {
      double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
      p0 = p1;
      p1 = p2;
    }
    dp = N * (x * p1 - p0) / (x * x - 1.0);
    g.x[i] = x;
    g.w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
  return g;
}
// Device copies of the rules, constant-initialised at compile time.
template <int N> __constant__ GaussRule<N> kGaussRule = make_gauss<N>();

// Integration matrix of the N-point Gauss-Legendre rule: S[k][i] is the
// integral over [-1, x_k] of the i-th Lagrange basis polynomial of the nodes,
// so that sum_i S[k][i] f(x_i) integrates the interpolant of f from -1 to
// node k.  Each basis polynomial has degree N - 1, so the N-point rule
// mapped to [-1, x_k] integrates it exactly.
template <int N> struct GaussIntMatrix {
  double S[N][N];
};
template <int N> __host__ __device__ constexpr GaussIntMatrix<N> make_gauss_int() {
  GaussIntMatrix<N> m{};
  const GaussRule<N> g = make_gauss<N>();
  for (int k = 0; k < N; ++k)
    for (int i = 0; i < N; ++i) {
      double acc = 0.0;
      for (int q = 0; q < N; ++q) {
        const double y = -1.0 + (g.x[q] + 1.0) * (g.x[k] + 1.0) * 0.5;
        double l = 1.0;
        for (int r = 0; r < N; ++r)
          if (r != i) l *= (y - g.x[r]) / (g.x[i] - g.x[r]);
        acc += g.w[q] * (g.x[k] + 1.0) * 0.5 * l;
      }
      m.S[k][i] = acc;
    }
  return m;
}
// FP32 copies for the Case II term-structure rule (8 nodes a sub-panel).
constexpr int kC2Nodes = 8;
struct C2Tables {
  float S[kC2Nodes][kC2Nodes];  // integration matrix
  float w[kC2Nodes];            // weights on [-1, 1]
};
__host__ __device__ constexpr C2Tables make_c2_tables() {
  C2Tables t{};
  const GaussIntMatrix<kC2Nodes> m = make_gauss_int<kC2Nodes>();
  const GaussRule<kC2Nodes> g = make_gauss<kC2Nodes>();
  for (int k = 0; k < kC2Nodes; ++k) {
    t.w[k] = (float)g.w[k];
    for (int i = 0; i < kC2Nodes; ++i) t.S[k][i] = (float)m.S[k][i];
  }
  return t;
}
__constant__ C2Tables kC2 = make_c2_tables();

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64
// multiplications, key bumped by the golden-ratio Weyl constants.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t ma = 0xD2511F53u, mb = 0xCD9E8D57u;
    // each 32 x 32 -> 64-bit product in one wide multiply
    const uint64_t pa = (uint64_t)ma * c.x, pb = (uint64_t)mb * c.z;
    const uint32_t ha = (uint32_t)(pa >> 32), la = (uint32_t)pa;
    const uint32_t hb = (uint32_t)(pb >> 32), lb = (uint32_t)pb;
    c = make_uint4(hb ^ c.y ^ k0, lb, ha ^ c.w ^ k1, la);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}
// The same generator with its ten round keys formed once (they depend on
// the key only): a caller drawing many blocks under one key keeps them in
// registers instead of stepping the key schedule in every block.
struct PhiloxKeys {
  uint32_t k0[10], k1[10];
};
__device__ __forceinline__ PhiloxKeys philox_keys(uint32_t k0, uint32_t k1) {
  PhiloxKeys pk;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    pk.k0[r] = k0;
    pk.k1[r] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return pk;
}
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKeys& pk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t ma = 0xD2511F53u, mb = 0xCD9E8D57u;
    const uint64_t pa = (uint64_t)ma * c.x, pb = (uint64_t)mb * c.z;
    const uint32_t ha = (uint32_t)(pa >> 32), la = (uint32_t)pa;
    const uint32_t hb = (uint32_t)(pb >> 32), lb = (uint32_t)pb;
    c = make_uint4(hb ^ c.y ^ pk.k0[r], lb, ha ^ c.w ^ pk.k1[r], la);
  }
  return c;
}
constexpr uint32_t kTagSA = 0x53410000u;
constexpr uint32_t kTagMC = 0x4D430000u;

// SA proposal (chain, level, step) of a d-parameter model draws words
// 0 .. d-1 of Philox blocks (chain, level, step, kTagSA + j/4), j = word:
// the high 23 bits of word i move parameter i, and the acceptance uniform is
// the 23 bits the moves leave unused in words 0, 1 and 2 (low 9, 9 and 5
// bits), packed as the high bits of one word.  A static model (d = 4) needs
// one Philox block per proposal.
constexpr int sa_philox_blocks(int d) { return (d + 3) / 4; }
__device__ __forceinline__ uint32_t sa_accept_word(uint32_t w0, uint32_t w1, uint32_t w2) {
  return ((w0 & 0x1FFu) << 23) | ((w1 & 0x1FFu) << 14) | ((w2 & 0x1Fu) << 9);
}

// 23 random bits + 1/2, scaled by 2^-23: exact in float, strictly in (0,1).
// Written as one fused multiply-add, (w >> 9) 2^-23 + 2^-24, whose product
// and sum are both exact, so the value is the same.
template <class R> __device__ __forceinline__ R u01(uint32_t w) {
  return fma((R)(w >> 9), (R)1.1920928955078125e-07, (R)5.9604644775390625e-08);
}
// FP32: the same value without an integer conversion.  The float with bits
// 0x3F800000 | (w >> 9) is 1 + (w >> 9) 2^-23 exactly, and subtracting
// 1 - 2^-24 from it is exact (Sterbenz: both lie in [1/2, 2]), leaving
// (w >> 9) 2^-23 + 2^-24.
template <> __device__ __forceinline__ float u01<float>(uint32_t w) {
  return __uint_as_float(0x3F800000u | (w >> 9)) - 0.99999994039535522f;
}

// ---------------------------------------------------------------------------
// z / x(z), eq. (equis):  x = ln u,  u = (D + z - rho)/(1 - rho),
// D = sqrt(1 - 2 rho z + z^2) = sqrt((z - rho)^2 + (1 - rho)(1 + rho)).
// Since (D + z - rho)(D - z + rho) = (1 - rho)(1 + rho), also
// u = (1 + rho)/(D - z + rho); the first form has no cancellation for
// z >= rho, the second none for z <= rho.  Both are D + |z - rho| over a
// constant or a constant over it.  The per-proposal constants of rho are
// kept in ZxConst.
// ---------------------------------------------------------------------------
template <class R> struct ZxConst {
  R rho, omr, opr, q0;  // rho, 1 - rho, 1 + rho, (1 - rho)(1 + rho)
  R ln_opr, ln_omr;     // ln(1 + rho), ln(1 - rho) (FP32 form only)
};
// omr = 1 - rho and opr = 1 + rho are formed from the FP64 parameter.
template <class R, class P> __device__ __forceinline__ ZxConst<R> zx_setup(P rho) {
  ZxConst<R> c;
  c.rho = (R)rho;
  c.omr = (R)(1.0 - (double)rho);
  c.opr = (R)(1.0 + (double)rho);
  c.q0 = c.omr * c.opr;
  c.ln_opr = c.ln_omr = (R)0;
  return c;
}

// FP64 form: u is one division of selected operands.  Near z = 0, ln u alone
// loses the relative accuracy of x, and Goldberg's identity
// ln(1 + w) = w ln(u)/(u - 1) (u the rounded 1 + w) is used with
// w = u - 1 = 2 z/(1 - z + D), i.e.
//     z / x = (u - 1)(1 - z + D) / (2 ln u)     (z/w = (1 - z + D)/2),
// and z / x = (1 - z + D)/2 when u rounds to 1.  Every lane runs the same
// instructions whatever the sign and size of z (selects, no branches).
// The result is returned as a quotient zn / xd so callers fold it into their
// own single division.
template <class R>
__device__ __forceinline__ void z_over_x_parts(R z, const ZxConst<R>& c, R& zn, R& xd) {
  const R zr = z - c.rho;
  const R D = m_sqrt_pos(zr * zr + c.q0);
  const bool low = z <= c.rho;
  const R u = m_div(low ? c.opr : D + zr, low ? D - zr : c.omr);
  const R L = m_log(u);
  const R um1 = u - (R)1;
  const R half_w_inv = ((R)1 - z + D) * (R)0.5;  // z / w
  const bool near = z > (R)-0.5 && z < (R)0.5;
  const bool one = um1 == (R)0;
  zn = one ? half_w_inv : (near ? um1 * half_w_inv : z);
  xd = one ? (R)1 : L;
}

// FP32 form.  With t = (u - 1)/(u + 1) = z/(1 + D) (|t| < 1; from the form
// of u above), x = ln u = 2 atanh t, so z/x = (1 + D)/(2 S(t^2)) where
// S(t^2) = atanh(t)/t = sum_k t^(2k)/(2k + 1).  For |t| < 1/5 (|x| < 0.41)
// the series to t^8 is exact to 1e-8 relative.  Elsewhere |x| > 0.40 and
// x = ln u = +-(ln(D + |z - rho|) - ln(1 -+ rho)), the first logarithm from
// the SFU log2 (absolute error about 2^-22) and the second a per-proposal
// constant, is accurate to a few 1e-7 relative.  Both are formed and one is
// selected, so no lane branches; FP32 emulation against the FP64 formula
// (with the SFU errors added) gives a worst relative error below 1e-6 over
// z in [-20, 20], rho in [-0.999999, 0.999999].
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
template <> __device__ __forceinline__ ZxConst<float> zx_setup<float, double>(double rho) {
  ZxConst<float> c;
  c.rho = (float)rho;
  c.omr = (float)(1.0 - rho);
  c.opr = (float)(1.0 + rho);
  c.q0 = c.omr * c.opr;
  c.ln_opr = lg2_approx(c.opr) * 0.69314718055994531f;
  c.ln_omr = lg2_approx(c.omr) * 0.69314718055994531f;
  return c;
}
// A float rho: 1 -+ rho rounded once in FP32 is the value the FP64 route
// gives (the exact difference rounded to float), without FP64 instructions.
template <> __device__ __forceinline__ ZxConst<float> zx_setup<float, float>(float rho) {
  ZxConst<float> c;
  c.rho = rho;
  c.omr = 1.0f - rho;
  c.opr = 1.0f + rho;
  c.q0 = c.omr * c.opr;
  c.ln_opr = lg2_approx(c.opr) * 0.69314718055994531f;
  c.ln_omr = lg2_approx(c.omr) * 0.69314718055994531f;
  return c;
}
template <>
__device__ __forceinline__ void z_over_x_parts<float>(float z, const ZxConst<float>& c, float& zn, float& xd) {
  const float zr = z - c.rho;
  const float D = m_sqrt_pos(zr * zr + c.q0);
  const float onepD = 1.0f + D;
  const float t = z * rcp_approx(onepD);
  const float t2 = t * t;
  float S2 = 2.0f / 9.0f;  // 2 S(t^2)
  S2 = S2 * t2 + 2.0f / 7.0f;
  S2 = S2 * t2 + 2.0f / 5.0f;
  S2 = S2 * t2 + 2.0f / 3.0f;
  S2 = S2 * t2 + 2.0f;
  // |x| = |lg ln 2 - ln(1 -+ rho)| (the sign of x is that of z, so
  // z/x = |z|/|x|; the near-branch values are positive)
  const float lg = lg2_approx(D + fabsf(zr));
  const float ax = fmaf(lg, 0.69314718055994531f, zr > 0.0f ? -c.ln_omr : -c.ln_opr);
  const bool near = fabsf(t) < 0.2f;
  zn = fabsf(near ? onepD : z);
  xd = fabsf(near ? S2 : ax);
}

// ---------------------------------------------------------------------------
// Per-quote inputs (parameter independent, formed in FP64 on the host):
//   lfk  = ln(f/K)        l2kf = log2(K f)       l2k = log2(K)      T
// ---------------------------------------------------------------------------
template <class R> struct StaticConst {
  R alpha, beta, rho, nu;
  R omb, half_omb, c2, c4, nu_over_alpha, br_a, br_b, br_c;
  R abr_a, abr_b, abr_c;  // alpha br_a, alpha br_b, alpha br_c
  ZxConst<R> zx;
};

// params: x[0..3] = alpha, beta, rho, nu (any real type)
template <class R, class P>
__device__ __forceinline__ StaticConst<R> static_setup(const P* x) {
  StaticConst<R> s;
  s.alpha = (R)x[0];
  s.beta = (R)x[1];
  s.rho = (R)x[2];
  s.nu = (R)x[3];
  s.omb = (R)1 - s.beta;
  s.half_omb = (R)0.5 * s.omb;
  s.c2 = m_divc(s.omb * s.omb, 24.0);
  s.c4 = m_divc(s.omb * s.omb * s.omb * s.omb, 1920.0);
  s.nu_over_alpha = m_div(s.nu, s.alpha);
  s.br_a = s.c2 * s.alpha * s.alpha;
  s.br_b = (R)0.25 * s.rho * s.beta * s.nu * s.alpha;
  s.br_c = m_divc((R)2 - (R)3 * s.rho * s.rho, 24.0) * s.nu * s.nu;
  s.abr_a = s.alpha * s.br_a;
  s.abr_b = s.alpha * s.br_b;
  s.abr_c = s.alpha * s.br_c;
  s.zx = zx_setup<R>(x[2]);
  return s;
}

// eq. (haganf) with z of eq. (zeta), fk = (K f)^{(1-beta)/2} = 2^(e) from
// log2(K f).  The bracket 1 + (br_a/fk^2 + br_b/fk + br_c) T times alpha/fk
// is written over fk^3, so one power of (K f) serves the whole formula:
//   sigma = (z/x) [fk^2 (alpha + alpha br_c T) + (alpha br_b fk + alpha br_a) T]
//           / (fk^3 den).
template <class R>
__device__ __forceinline__ R vol_hagan(const StaticConst<R>& s, R lfk, R l2kf, R T) {
  const R fk = m_exp2(s.half_omb * l2kf);
  const R L2 = lfk * lfk;
  const R den = (R)1 + L2 * (s.c2 + s.c4 * L2);
  const R z = s.nu_over_alpha * lfk * fk;
  R zn, xd;
  z_over_x_parts<R>(z, s.zx, zn, xd);
  const R fk2 = fk * fk;
  const R num = fk2 * (s.alpha + s.abr_c * T) + (s.abr_b * fk + s.abr_a) * T;
  return m_div(zn * num, fk2 * fk * den * xd);
}

// eq. (sigma-SABR): z = nu (f^{1-b} - K^{1-b}) / (alpha (1-b)); the
// difference is K^{1-b} expm1((1-b) ln(f/K)), its b -> 1 limit ln(f/K);
// nu ln(f/K)/x(z) = (alpha ln(f/K)/zd) (z/x(z)), alpha/K^{1-b} at K = f.
// ---------------------------------------------------------------------------
// Two quotes of eq. (haganf) at once, FP32.  GB300's packed FP32 forms
// (FFMA2 / FMUL2 / FADD2, __ffma2_rn and friends) do two lanes' worth of
// FP32 arithmetic in one issue slot, so the formula's ~30 adds and
// multiplies per quote take half the issue slots of the scalar form; the
// SFU operations and the branch selects stay per element.  Same operations,
// in the same order and contraction, as vol_hagan<float> with
// z_over_x_parts<float>; returns the residuals r = one + v * (-1/market) of
// both quotes (one = 1, or 0 for the zero-filled second element of an odd
// count's last pair, whose residual is then exactly 0).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// Per-proposal constants of eq. (haganf) for quotes of one maturity T (a
// problem whose quotes all share T, such as one smile): the bracket's T
// terms folded into the numerator, num = fk (fk A + B) + C with
// A = alpha + alpha br_c T, B = alpha br_b T, C = alpha br_a T (two FP32x2
// operations fewer per pair of quotes).
struct HaganT1 {
  float A, B, C;
};
__device__ __forceinline__ HaganT1 hagan_t1(const StaticConst<float>& s, float T) {
  return HaganT1{fmaf(s.abr_c, T, s.alpha), s.abr_b * T, s.abr_a * T};
}

// One quote of eq. (haganf) in FP32: vol_hagan<float>, or with the
// numerator of HaganT1 when T1 (T is then not read).
template <bool T1>
__device__ __forceinline__ float vol_hagan_f32(const StaticConst<float>& s, const HaganT1& h, float lfk, float l2kf,
                                               float T) {
  if constexpr (!T1) {
    return vol_hagan<float>(s, lfk, l2kf, T);
  } else {
    const float fk = ex2_approx(s.half_omb * l2kf);
    const float L2 = lfk * lfk;
    const float den = 1.0f + L2 * (s.c2 + s.c4 * L2);
    const float z = s.nu_over_alpha * lfk * fk;
    float zn, xd;
    z_over_x_parts<float>(z, s.zx, zn, xd);
    const float fk2 = fk * fk;
    const float num = fmaf(fk, fmaf(fk, h.A, h.B), h.C);
    return m_div(zn * num, fk2 * fk * den * xd);
  }
}

template <bool T1 = false>
__device__ __forceinline__ float2 hagan_resid_pair(const StaticConst<float>& s, float2 lfk, float2 l2kf, float2 T,
                                                   float2 wneg, float2 one = make_float2(1.0f, 1.0f),
                                                   const HaganT1& h = HaganT1{0.0f, 0.0f, 0.0f}) {
  const float2 e = mul2(f2(s.half_omb), l2kf);
  const float2 fk = make_float2(ex2_approx(e.x), ex2_approx(e.y));
  const float2 L2 = mul2(lfk, lfk);
  const float2 den = fma2(L2, fma2(f2(s.c4), L2, f2(s.c2)), f2(1.0f));
  const float2 z = mul2(mul2(f2(s.nu_over_alpha), lfk), fk);
  // z / x(z): near branch (|t| < 0.2) by the atanh series, far branch by
  // the logarithm, both formed and one selected per element
  const float2 zr = add2(z, f2(-s.zx.rho));
  const float2 y = fma2(zr, zr, f2(s.zx.q0));
  const float2 D = mul2(y, make_float2(rsqrt_approx(y.x), rsqrt_approx(y.y)));
  const float2 onepD = add2(D, f2(1.0f));
  const float2 t = mul2(z, make_float2(rcp_approx(onepD.x), rcp_approx(onepD.y)));
  const float2 t2 = mul2(t, t);
  float2 S2 = fma2(f2(2.0f / 9.0f), t2, f2(2.0f / 7.0f));
  S2 = fma2(S2, t2, f2(2.0f / 5.0f));
  S2 = fma2(S2, t2, f2(2.0f / 3.0f));
  S2 = fma2(S2, t2, f2(2.0f));
  const float2 lg = make_float2(lg2_approx(D.x + fabsf(zr.x)), lg2_approx(D.y + fabsf(zr.y)));
  const float2 cs = make_float2(zr.x > 0.0f ? -s.zx.ln_omr : -s.zx.ln_opr, zr.y > 0.0f ? -s.zx.ln_omr : -s.zx.ln_opr);
  const float2 ax = fma2(lg, f2(0.69314718055994531f), cs);
  const bool nx = fabsf(t.x) < 0.2f, ny = fabsf(t.y) < 0.2f;
  const float2 zn = make_float2(fabsf(nx ? onepD.x : z.x), fabsf(ny ? onepD.y : z.y));
  const float2 xd = make_float2(fabsf(nx ? S2.x : ax.x), fabsf(ny ? S2.y : ax.y));
  // sigma = (z/x) [fk^2 (alpha + alpha br_c T) + (alpha br_b fk + alpha br_a) T] / (fk^3 den)
  const float2 fk2 = mul2(fk, fk);
  float2 num;
  if constexpr (T1) {
    num = fma2(fk, fma2(fk, f2(h.A), f2(h.B)), f2(h.C));
  } else {
    num = fma2(fk2, fma2(f2(s.abr_c), T, f2(s.alpha)), mul2(fma2(f2(s.abr_b), fk, f2(s.abr_a)), T));
  }
  const float2 dd = mul2(mul2(mul2(fk2, fk), den), xd);
  const float2 v = mul2(mul2(zn, num), make_float2(rcp_approx(dd.x), rcp_approx(dd.y)));
  return fma2(v, wneg, one);
}

template <class R>
__device__ __forceinline__ R vol_obloj(const StaticConst<R>& s, R lfk, R l2kf, R l2k, R T) {
  const R kpow = m_exp2(s.omb * l2k);  // K^{1-beta}
  const R zd = (s.omb == (R)0) ? lfk : m_div(kpow * m_expm1(s.omb * lfk), s.omb);
  const R z = s.nu_over_alpha * zd;
  // lead = alpha lfk / zd, or alpha / K^{1-beta} at the money
  const R ln = (lfk == (R)0) ? s.alpha : s.alpha * lfk;
  const R ld = (lfk == (R)0) ? kpow : zd;
  const R fkinv = m_exp2(-s.half_omb * l2kf);
  const R L2 = lfk * lfk;
  const R den = (R)1 + L2 * (s.c2 + s.c4 * L2);
  const R brk = (R)1 + (s.br_a * fkinv * fkinv + s.br_b * fkinv + s.br_c) * T;
  R zn, xd;
  z_over_x_parts<R>(z, s.zx, zn, xd);
  return m_div(ln * zn * brk, ld * xd * den);
}

// ---------------------------------------------------------------------------
// Polynomial form sigma = c0 + c1 L + c2 L^2 with L = ln(K/f) = -lfk, used
// by eq. (vola_SABR) (c0 carries B T) and by eq. (vola_SABRd) per maturity.
// ---------------------------------------------------------------------------
template <class R> struct PolyCoef {
  R c0, c1, c2;
};

// eq. (vola_SABR): omega = f^{1-beta}/alpha (log2 f given).
template <class R, class P>
__device__ __forceinline__ PolyCoef<R> expanded_coef(const P* x, R l2f, R T) {
  const R alpha = (R)x[0], beta = (R)x[1], rho = (R)x[2], nu = (R)x[3];
  const R omb = (R)1 - beta;
  const R w = m_div(m_exp2(omb * l2f), alpha);
  const R rnw = rho * nu * w;
  const R A1 = (R)-0.5 * (omb - rnw);
  const R A2 = m_divc(omb * omb + (R)3 * (omb - rnw) + ((R)2 - (R)3 * rho * rho) * nu * nu * w * w, 12.0);
  const R B = m_div(omb * omb, (R)24 * w * w) + m_div(beta * rho * nu, (R)4 * w) +
              m_divc((R)2 - (R)3 * rho * rho, 24.0) * nu * nu;
  PolyCoef<R> c;
  c.c0 = m_div((R)1 + B * T, w);
  c.c1 = m_div(A1, w);
  c.c2 = m_div(A2, w);
  return c;
}

// eq. (vola_SABRd) from the four functions at T.
template <class R>
__device__ __forceinline__ PolyCoef<R> dynamic_poly(R alpha, R beta, R l2f, R T, R nu1sq,
                                                    R nu2sq, R eta1, R eta2sq) {
  const R omb = (R)1 - beta;
  const R w = m_div(m_exp2(omb * l2f), alpha);
  const R A1 = m_divc(beta - (R)1, 2.0) + m_divc(eta1 * w, 2.0);
  const R A2 = m_divc(omb * omb, 12.0) + m_divc(omb - eta1 * w, 4.0) +
               m_divc((R)4 * nu1sq + (R)3 * (eta2sq - (R)3 * eta1 * eta1), 24.0) * w * w;
  const R B = m_div(m_divc(omb * omb, 24.0) + m_divc(w * beta * eta1, 4.0) +
                        m_divc((R)2 * nu2sq - (R)3 * eta2sq, 24.0) * w * w,
                    w * w);
  PolyCoef<R> c;
  c.c0 = m_div((R)1 + B * T, w);
  c.c1 = m_div(A1, w);
  c.c2 = m_div(A2, w);
  return c;
}

template <class R>
__device__ __forceinline__ R vol_poly(const PolyCoef<R>& c, R lfk) {
  const R L = -lfk;
  return c.c0 + L * (c.c1 + L * c.c2);
}

// ---------------------------------------------------------------------------
// Case I, eq. (exact-integral-expressions), each function written as
// (constant) x g(argument) with g evaluated by its Taylor series for
// argument < 2 (where the printed closed forms cancel) and by the closed form
// otherwise:
//   nu1^2 = 6 nu0^2 g1(2bT),  g1(x) = (x^2/2 - x + 1 - e^-x)/x^3
//         = sum_{k>=0} (-x)^k / (k+3)!
//   nu2^2 = 6 nu0^2 g2(2bT),  g2(x) = (2(e^-x - 1) + x(e^-x + 1))/x^3
//         = sum_{k>=0} (-x)^k (k+1)/(k+3)!
//   eta1  = 2 nu0 rho0 g3(y), g3(y) = (e^-y - 1 + y)/y^2
//         = sum_{k>=0} (-y)^k / (k+2)!,            y = (a+b)T
//   eta2^2 = 3 nu0^2 rho0^2 g4(y),
//         g4(y) = (e^-2y - 8 e^-y + 7 + 2y(y-3))/y^4
//         = sum_{k>=0} (-y)^k (2^{k+4} - 8)/(k+4)!
// ---------------------------------------------------------------------------
__host__ __device__ constexpr double g1c(int k) { return 1.0 / cx_fact(k + 3); }
__host__ __device__ constexpr double g2c(int k) { return (k + 1.0) / cx_fact(k + 3); }
__host__ __device__ constexpr double g3c(int k) { return 1.0 / cx_fact(k + 2); }
__host__ __device__ constexpr double g4c(int k) {
  double p = 1.0;
  for (int i = 0; i < k + 4; ++i) p *= 2.0;
  return (p - 8.0) / cx_fact(k + 4);
}

template <class R>
__device__ __forceinline__ void case1_coeffs(R nu0, R rho0, R a, R b, R T, R out[4]) {
  constexpr int N = Tr<R>::kCase1Series;
  const R x = (R)2 * b * T, y = (a + b) * T;
  R g1, g2, g3, g4;
  if (x < (R)2) {
    const R mx = -x;
    R s1 = (R)g1c(N), s2 = (R)g2c(N);
#pragma unroll
    for (int k = N - 1; k >= 0; --k) {
      s1 = s1 * mx + (R)g1c(k);
      s2 = s2 * mx + (R)g2c(k);
    }
    g1 = s1;
    g2 = s2;
  } else {
    const R e = m_exp(-x), ix = m_rcp(x), ix3 = ix * ix * ix;
    g1 = ((x * x * (R)0.5 - x + (R)1) - e) * ix3;
    g2 = ((R)2 * (e - (R)1) + x * (e + (R)1)) * ix3;
  }
  if (y < (R)2) {
    const R my = -y;
    R s3 = (R)g3c(N), s4 = (R)g4c(N);
#pragma unroll
    for (int k = N - 1; k >= 0; --k) {
      s3 = s3 * my + (R)g3c(k);
      s4 = s4 * my + (R)g4c(k);
    }
    g3 = s3;
    g4 = s4;
  } else {
    const R e = m_exp(-y), iy = m_rcp(y), iy2 = iy * iy;
    g3 = (e - (R)1 + y) * iy2;
    g4 = (m_exp(-(R)2 * y) - (R)8 * e + ((R)7 + (R)2 * y * (y - (R)3))) * iy2 * iy2;
  }
  out[0] = (R)6 * nu0 * nu0 * g1;
  out[1] = (R)6 * nu0 * nu0 * g2;
  out[2] = (R)2 * nu0 * rho0 * g3;
  out[3] = (R)3 * nu0 * nu0 * rho0 * rho0 * g4;
}

// ---------------------------------------------------------------------------
// Case II.  In scaled time tau = t/T every integrand is a polynomial in tau
// times e^{-x tau}, x in {A+B, B, 2B, A} (A = aT, B = bT), so each function is
// a combination of phi_m(x) = int_0^1 tau^m e^{-x tau} dtau.  Below
// x = kSeriesMax (5 in FP64, 2 in FP32), phi_m(x) = m! e^{-x} S_m(x) with
// S_m(x) = sum_n x^n/(m+n+1)! (positive terms; S_{m-1} = 1/m! + x S_m
// downwards); above it the upward recurrence phi_m = (m phi_{m-1} - e^{-x})/x
// is used (for m <= 4 in FP32 emulation against quadrature: relative error
// at most 1.6e-6 with 12 series terms below 2).
// ---------------------------------------------------------------------------
// phi_0..phi_M at x >= 0, given e = e^{-x}.
template <class R, int M>
__device__ __forceinline__ void phi_vec_e(R x, R e, R* phi) {
  if constexpr (sizeof(R) == 4) {
    // FP32: both forms, then a select per phi_m -- the lanes of a chain hold
    // different quadrature nodes, and a branch on x would run both forms
    // one after the other whenever they disagree
    constexpr int N = Tr<R>::kSeries;
    R S = (R)(1.0 / cx_fact(M + N + 1));
#pragma unroll
    for (int n = N - 1; n >= 0; --n) S = S * x + (R)(1.0 / cx_fact(M + n + 1));
    R ser[M + 1];
    ser[M] = (R)cx_fact(M) * e * S;
#pragma unroll
    for (int m = M - 1; m >= 0; --m) {
      S = (R)(1.0 / cx_fact(m + 1)) + x * S;
      ser[m] = (R)cx_fact(m) * e * S;
    }
    const bool use_series = x < (R)Tr<R>::kSeriesMax;
    const R ix = m_rcp(x);
    R rec = ((R)1 - e) * ix;
    phi[0] = use_series ? ser[0] : rec;
#pragma unroll
    for (int m = 1; m <= M; ++m) {
      rec = ((R)m * rec - e) * ix;
      phi[m] = use_series ? ser[m] : rec;
    }
  } else if (x < (R)Tr<R>::kSeriesMax) {
    constexpr int N = Tr<R>::kSeries;
    // S_M(x) = sum_{n=0..N} x^n/(M+n+1)! by Horner's rule, one FMA a term
    R S = (R)(1.0 / cx_fact(M + N + 1));
#pragma unroll
    for (int n = N - 1; n >= 0; --n) S = S * x + (R)(1.0 / cx_fact(M + n + 1));
    phi[M] = (R)cx_fact(M) * e * S;
#pragma unroll
    for (int m = M - 1; m >= 0; --m) {
      S = (R)(1.0 / cx_fact(m + 1)) + x * S;
      phi[m] = (R)cx_fact(m) * e * S;
    }
  } else {
    const R ix = m_rcp(x);
    phi[0] = ((R)1 - e) * ix;
#pragma unroll
    for (int m = 1; m <= M; ++m) phi[m] = ((R)m * phi[m - 1] - e) * ix;
  }
}

template <class R, int M>
__device__ __forceinline__ void phi_vec(R x, R* phi) {
  phi_vec_e<R, M>(x, m_exp(-x), phi);
}

// nu1^2 = 3 int_0^1 (1-tau)^2 nu^2,  nu2^2 = 6 int_0^1 (1-tau) tau nu^2,
// eta1 = 2 int_0^1 (1-tau) nu rho, with nu = (nu0 + Qn tau) e^{-B tau} + dn,
// rho = (rho0 + Qr tau) e^{-A tau} + dr: polynomial coefficients expanded by
// hand below.
template <class R>
__device__ __forceinline__ void case2_single(R rho0, R nu0, R A, R B, R dr, R dn, R Qr,
                                             R Qn, R out3[3]) {
  R f2B[5], fB[5], fA[5], fAB[5];
  phi_vec<R, 4>((R)2 * B, f2B);
  phi_vec<R, 3>(B, fB);
  phi_vec<R, 2>(A, fA);
  phi_vec<R, 3>(A + B, fAB);
  // P = (nu0 + Qn t)^2 = p0 + p1 t + p2 t^2 ; Rn = nu0 + Qn t
  const R p0 = nu0 * nu0, p1 = (R)2 * nu0 * Qn, p2 = Qn * Qn;
  // (1-t)^2 P
  const R a0 = p0, a1 = p1 - (R)2 * p0, a2 = p2 - (R)2 * p1 + p0, a3 = p1 - (R)2 * p2, a4 = p2;
  // (1-t)^2 Rn
  const R b0 = nu0, b1 = Qn - (R)2 * nu0, b2 = nu0 - (R)2 * Qn, b3 = Qn;
  const R nu1 = (R)3 * (a0 * f2B[0] + a1 * f2B[1] + a2 * f2B[2] + a3 * f2B[3] + a4 * f2B[4] +
                        (R)2 * dn * (b0 * fB[0] + b1 * fB[1] + b2 * fB[2] + b3 * fB[3]) +
                        m_divc(dn * dn, 3.0));
  // (1-t) t P = p0 t + (p1 - p0) t^2 + (p2 - p1) t^3 - p2 t^4
  // (1-t) t Rn = nu0 t + (Qn - nu0) t^2 - Qn t^3
  const R nu2 = (R)6 * (p0 * f2B[1] + (p1 - p0) * f2B[2] + (p2 - p1) * f2B[3] - p2 * f2B[4] +
                        (R)2 * dn * (nu0 * fB[1] + (Qn - nu0) * fB[2] - Qn * fB[3]) +
                        m_divc(dn * dn, 6.0));
  // nu rho = Kp(t) e^{-(A+B)t} + dr Rn e^{-Bt} + dn (rho0 + Qr t) e^{-At} + dn dr
  // Kp = k0 + k1 t + k2 t^2
  const R k0 = nu0 * rho0, k1 = nu0 * Qr + Qn * rho0, k2 = Qn * Qr;
  // (1-t) Kp = k0 + (k1-k0) t + (k2-k1) t^2 - k2 t^3 ; (1-t) Rn ; (1-t)(rho0 + Qr t)
  const R eta1 = (R)2 * (k0 * fAB[0] + (k1 - k0) * fAB[1] + (k2 - k1) * fAB[2] - k2 * fAB[3] +
                         dr * (nu0 * fB[0] + (Qn - nu0) * fB[1] - Qn * fB[2]) +
                         dn * (rho0 * fA[0] + (Qr - rho0) * fA[1] - Qr * fA[2]) +
                         m_divc(dn * dr, 2.0));
  out3[0] = nu1;
  out3[1] = nu2;
  out3[2] = eta1;
}

// G(s) = int_0^s nu(Tu) rho(Tu) du at one node s, from
// int_0^s u^m e^{-xu} du = s^{m+1} phi_m(x s).
template <class R>
__device__ __forceinline__ R case2_G(R s, R rho0, R nu0, R A, R B, R dr, R dn, R Qr, R Qn) {
  R pAB[3], pB[2], pA[2];
  const R eA = m_exp_node(-A * s), eB = m_exp_node(-B * s);  // e^{-(A+B)s} = eA eB
  phi_vec_e<R, 2>((A + B) * s, eA * eB, pAB);
  phi_vec_e<R, 1>(B * s, eB, pB);
  phi_vec_e<R, 1>(A * s, eA, pA);
  const R k0 = nu0 * rho0, k1 = nu0 * Qr + Qn * rho0, k2 = Qn * Qr;
  const R s2 = s * s;
  return s * (k0 * pAB[0] + s * k1 * pAB[1] + s2 * k2 * pAB[2]) +
         dr * s * (nu0 * pB[0] + s * Qn * pB[1]) + dn * s * (rho0 * pA[0] + s * Qr * pA[1]) +
         dn * dr * s;
}

// Number of geometric panels [4^-(P-1) .. 1] the eta2^2 rule uses: enough
// that the boundary layer of width 1/(A+B) at s = 0 spans whole panels.
template <class R>
__device__ __forceinline__ int case2_panels(R A, R B) {
  const R x = A + B;
  int p = 1;
  R edge = (R)1;
  while (p < 7 && edge * x > (R)1) {
    edge *= (R)0.25;
    ++p;
  }
  return p;
}

// Node k of the eta2^2 rule on panel k / NG (the k % NG-th Gauss point):
// its term 12 h w (1 - s) G(s)^2, so that eta2^2 is the sum over all
// k < npanels * NG of these terms (lanes may share the nodes of one
// maturity).
template <class R>
__device__ __forceinline__ R case2_eta2_node(int k, int npanels, R rho0, R nu0, R A, R B, R dr, R dn, R Qr,
                                             R Qn) {
  constexpr int NG = Tr<R>::kGauss;
  const int panel = k / NG, i = k % NG;
  R hi = (R)1;
  for (int q = npanels - 1; q > panel; --q) hi *= (R)0.25;
  const R lo = panel > 0 ? hi * (R)0.25 : (R)0;
  const R c = (R)0.5 * (lo + hi), h = (R)0.5 * (hi - lo);
  const R s = c + h * (R)kGaussRule<NG>.x[i];
  const R G = case2_G<R>(s, rho0, nu0, A, B, dr, dn, Qr, Qn);
  return (R)12 * h * (R)kGaussRule<NG>.w[i] * ((R)1 - s) * G * G;
}

// The eta2^2 rule of one maturity as a list of nodes, so that the lanes of a
// chain can share them: nodes() terms, term k by node(k).
//  * FP64: the graded panels above (16 Gauss-Legendre nodes per panel).
//  * FP32: one 16-node Gauss-Legendre rule in u after the exponential map
//    s = expm1(lam u)/expm1(lam), lam = log1p(A + B)/2, which clusters the
//    nodes in the boundary layer of width 1/(A + B) at s = 0; over 40 random
//    parameter sets (T in {0.1, 1, 5, 10}, rates up to 5) its relative error
//    on eta2^2 is below 1e-11 (16 nodes; 8e-8 with 12), against 8e-6 for
//    graded panels of 6 nodes, which need 18 nodes on average.
template <class R> struct Eta2Rule;
template <> struct Eta2Rule<double> {
  int np;
  __device__ Eta2Rule(double A, double B) : np(case2_panels<double>(A, B)) {}
  __device__ int nodes() const { return np * Tr<double>::kGauss; }
  __device__ double node(int k, double rho0, double nu0, double A, double B, double dr, double dn, double Qr,
                         double Qn) const {
    return case2_eta2_node<double>(k, np, rho0, nu0, A, B, dr, dn, Qr, Qn);
  }
};
template <> struct Eta2Rule<float> {
  static constexpr int kNodes = 16;
  float lam, inv_em;
  bool flat;  // A + B ~ 0: plain Gauss-Legendre on [0, 1]
  __device__ Eta2Rule(float A, float B) {
    lam = 0.5f * lg2_approx(1.0f + (A + B)) * 0.69314718055994531f;
    flat = lam < 1e-6f;
    inv_em = flat ? 0.0f : rcp_approx(expm1f(lam));
  }
  __device__ int nodes() const { return kNodes; }
  __device__ float node(int k, float rho0, float nu0, float A, float B, float dr, float dn, float Qr,
                        float Qn) const {
    const float u = 0.5f * ((float)kGaussRule<kNodes>.x[k] + 1.0f);
    const float w = 0.5f * (float)kGaussRule<kNodes>.w[k];
    float sv = u, ds = 1.0f;
    if (!flat) {
      const float em = expm1f(lam * u);
      sv = em * inv_em;
      ds = lam * (em + 1.0f) * inv_em;
    }
    const float G = case2_G<float>(sv, rho0, nu0, A, B, dr, dn, Qr, Qn);
    return 12.0f * w * ds * (1.0f - sv) * G * G;
  }
};

// All four Case II functions at T (single thread).
template <class R, class P>
__device__ __forceinline__ void case2_coeffs(const P* x, R T, R out[4]) {
  const R rho0 = (R)x[2], nu0 = (R)x[3], A = (R)x[4] * T, B = (R)x[5] * T;
  const R dr = (R)x[6], dn = (R)x[7], Qr = (R)x[8] * T, Qn = (R)x[9] * T;
  case2_single<R>(rho0, nu0, A, B, dr, dn, Qr, Qn, out);
  const Eta2Rule<R> rule(A, B);
  R e2 = (R)0;
  for (int k = 0; k < rule.nodes(); ++k) e2 += rule.node(k, rho0, nu0, A, B, dr, dn, Qr, Qn);
  out[3] = e2;
}

// Per-maturity polynomial for DYN_I / DYN_II (single thread).
template <class R, bool CASE2, class P>
__device__ __forceinline__ PolyCoef<R> dynamic_coef(const P* x, R l2f, R T) {
  R c[4];
  if constexpr (CASE2) {
    case2_coeffs<R, P>(x, T, c);
  } else {
    case1_coeffs<R>((R)x[3], (R)x[2], (R)x[4], (R)x[5], T, c);
  }
  return dynamic_poly<R>((R)x[0], (R)x[1], l2f, T, c[0], c[1], c[2], c[3]);
}

// Case II feasibility: rho(t) in [-1, 1], nu(t) > 0 on [0, Tmax] (extremes
// at the ends or at the stationary point t* = 1/k - c/q of
// g(t) = (c + q t) e^{-k t} + d).  Host and device: the library checks x0
// and the parameters of its pricers on the host with the same code the
// kernels use to reject proposals.
template <class R> __host__ __device__ __forceinline__ R hd_exp(R x) {
#ifdef __CUDA_ARCH__
  return m_exp(x);
#else
  return std::exp(x);
#endif
}
template <class R>
__host__ __device__ __forceinline__ void g_range(R c, R q, R k, R d, R Tmax, R& gmin, R& gmax) {
  const R g0 = c + d;
  const R g1 = (c + q * Tmax) * hd_exp(-k * Tmax) + d;
  gmin = g0 < g1 ? g0 : g1;
  gmax = g0 < g1 ? g1 : g0;
  if (k != (R)0 && q != (R)0) {
    const R ts = (R)1 / k - c / q;
    if (ts > (R)0 && ts < Tmax) {
      const R gs = (c + q * ts) * hd_exp(-k * ts) + d;
      gmin = gs < gmin ? gs : gmin;
      gmax = gs > gmax ? gs : gmax;
    }
  }
}
template <class R, class P>
__host__ __device__ __forceinline__ bool case2_feasible(const P* x, R Tmax) {
  R rmin, rmax, nmin, nmax;
  g_range<R>((R)x[2], (R)x[8], (R)x[4], (R)x[6], Tmax, rmin, rmax);
  g_range<R>((R)x[3], (R)x[9], (R)x[5], (R)x[7], Tmax, nmin, nmax);
  return rmin >= (R)-1 && rmax <= (R)1 && nmin > (R)0;
}

}  // namespace sabr
