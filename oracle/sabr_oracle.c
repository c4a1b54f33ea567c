/*
 * sabr_oracle.c -- plain FP64 CPU oracle.  TEST INFRASTRUCTURE ONLY: see the
 * header.  Compiled with -ffp-contract=off so that every product and sum is
 * rounded exactly as written.
 */
#include "sabr_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

int orc_n_params(int model) {
  switch (model) {
    case ORC_HAGAN:
    case ORC_OBLOJ:
    case ORC_EXPANDED: return 4;
    case ORC_DYN_I: return 6;
    case ORC_DYN_II: return 10;
    default: return -1;
  }
}

/* ------------------------------------------------------------------------ */
/* Quadrature: 10-point Gauss-Legendre rule, nodes found by Newton's method  */
/* on P_10 (three-term Legendre recurrence), applied adaptively by bisection */
/* until the two halves agree with the whole.                               */
/* ------------------------------------------------------------------------ */
#define GL_N 10
static double gl_x[GL_N], gl_w[GL_N];
static int gl_ready = 0;

static void legendre_pd(int n, double x, double* p, double* dp) {
  double p0 = 1.0, p1 = x;
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *p = p1;
  *dp = n * (x * p1 - p0) / (x * x - 1.0);
}

__attribute__((constructor)) static void gl_init(void) {
  for (int i = 0; i < GL_N; ++i) {
    double x = cos(M_PI * (i + 0.75) / (GL_N + 0.5));
    double p, dp;
    for (int it = 0; it < 100; ++it) {
      legendre_pd(GL_N, x, &p, &dp);
      double dx = p / dp;
      x -= dx;
      if (fabs(dx) < 1e-17) break;
    }
    legendre_pd(GL_N, x, &p, &dp);
    gl_x[i] = x;
    gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
  gl_ready = 1;
}

static double gl10(orc_fn f, void* ctx, double a, double b, double* absint) {
  double c = 0.5 * (a + b), h = 0.5 * (b - a), s = 0.0, sa = 0.0;
  for (int i = 0; i < GL_N; ++i) {
    double v = f(c + h * gl_x[i], ctx);
    s += gl_w[i] * v;
    sa += gl_w[i] * fabs(v);
  }
  if (absint) *absint = fabs(h) * sa;
  return s * h;
}

/* Bisect until the two halves agree with the whole to tol, or to within the
 * rounding noise of the sums themselves (a few ulps of the integral of |f|
 * over the subinterval), beyond which bisection cannot improve anything. */
static double adapt(orc_fn f, void* ctx, double a, double b, double whole,
                    double tol, int depth) {
  double m = 0.5 * (a + b);
  double al, ar;
  double l = gl10(f, ctx, a, m, &al), r = gl10(f, ctx, m, b, &ar);
  double noise = 16.0 * 2.220446049250313e-16 * (al + ar);
  double diff = fabs(l + r - whole);
  if (depth <= 0 || diff <= tol || diff <= noise) return l + r;
  return adapt(f, ctx, a, m, l, 0.5 * tol, depth - 1) +
         adapt(f, ctx, m, b, r, 0.5 * tol, depth - 1);
}

double orc_integrate(orc_fn f, void* ctx, double a, double b, double rtol) {
  if (!gl_ready) gl_init();
  if (a == b) return 0.0;
  double scale;
  double whole = gl10(f, ctx, a, b, &scale);
  double tol = rtol * scale;
  if (tol < 1e-300) tol = 1e-300;
  return adapt(f, ctx, a, b, whole, tol, 48);
}

typedef struct { const double* c; int deg; } poly_ctx;
static double poly_eval(double t, void* vctx) {
  const poly_ctx* pc = (const poly_ctx*)vctx;
  double s = 0.0;
  for (int k = pc->deg; k >= 0; --k) s = s * t + pc->c[k];
  return s;
}
double orc_integrate_poly(const double* c, int deg, double a, double b) {
  poly_ctx pc = {c, deg};
  return orc_integrate(poly_eval, &pc, a, b, 1e-15);
}

/* ------------------------------------------------------------------------ */
/* x(z), Sec. 2.1 eq. (equis).                                               */
/* ------------------------------------------------------------------------ */
/* Near z = 0 the quotient z/x(z) is 0/0.  There x(z) is evaluated from its
 * integral form x(z) = int_0^z (1 - 2 rho s + s^2)^(-1/2) ds (the derivative
 * of the log in eq. (equis)), whose integrand is the Legendre generating
 * function: x(z) = sum_n P_n(rho) z^(n+1)/(n+1), P_n by the three-term
 * recurrence.  For |z| < 1e-2 fourteen terms leave < 1e-28 relative. */
static double x_series(double z, double rho) {
  double pm1 = 1.0, p = rho; /* P_0, P_1 */
  double zp = z;             /* z^(n+1) */
  double s = z;              /* n = 0 term: P_0 z / 1 */
  for (int n = 1; n < 14; ++n) {
    zp *= z;
    s += p * zp / (n + 1.0);
    double pn1 = ((2.0 * n + 1.0) * rho * p - n * pm1) / (n + 1.0);
    pm1 = p;
    p = pn1;
  }
  return s;
}

double orc_x_of_z(double z, double rho) {
  if (fabs(z) < 1e-2) return x_series(z, rho);
  /* 1 - 2 rho z + z^2 = (z - rho)^2 + (1 - rho)(1 + rho): no cancellation. */
  double D = sqrt((z - rho) * (z - rho) + (1.0 - rho) * (1.0 + rho));
  if (z < 1.0) {
    /* The log argument u = (D + z - rho)/(1 - rho) satisfies
     * u - 1 = 2 z / (1 - z + D), because (D + z - 1)(D - z + 1) =
     * D^2 - (z - 1)^2 = 2 z (1 - rho).  For z < 1 every term of 1 - z + D is
     * positive, so x = log1p(u - 1) keeps full relative accuracy. */
    double w = 2.0 * z / (1.0 - z + D);
    if (w >= -0.5) return log1p(w);
    /* u < 1/2: form u itself, rationalised, since
     * (D + (z - rho)) (D - (z - rho)) = (1 - rho)(1 + rho). */
    return log((1.0 + rho) / (D - (z - rho)));
  }
  return log((D + z - rho) / (1.0 - rho)); /* eq. (equis) as printed */
}

double orc_z_over_x(double z, double rho) {
  if (z == 0.0) return 1.0;
  return z / orc_x_of_z(z, rho);
}

/* ------------------------------------------------------------------------ */
/* Static implied volatilities, Sec. 2.1                                     */
/* ------------------------------------------------------------------------ */
/* The bracket {1 + [ ... ] T} shared by eqs. (haganf) and (sigma-SABR). */
static double hagan_bracket(double alpha, double beta, double rho, double nu,
                            double f, double K, double T) {
  double omb = 1.0 - beta;
  double fk = pow(K * f, 0.5 * omb); /* (K f)^((1-beta)/2) */
  double term = omb * omb / 24.0 * alpha * alpha / (fk * fk) +
                0.25 * rho * beta * nu * alpha / fk +
                (2.0 - 3.0 * rho * rho) / 24.0 * nu * nu;
  return 1.0 + term * T;
}

/* The denominator series 1 + (1-beta)^2/24 ln^2 + (1-beta)^4/1920 ln^4. */
static double log_series(double beta, double lfk) {
  double omb = 1.0 - beta;
  double l2 = lfk * lfk;
  return 1.0 + omb * omb / 24.0 * l2 + omb * omb * omb * omb / 1920.0 * l2 * l2;
}

/* Sec. 2.1, eq. (haganf) with z of eq. (zeta). */
double orc_vol_hagan(double alpha, double beta, double rho, double nu,
                     double f, double K, double T) {
  double omb = 1.0 - beta;
  double lfk = log(f / K);
  double fk = pow(K * f, 0.5 * omb);
  double z = nu / alpha * fk * lfk;
  double lead = alpha / (fk * log_series(beta, lfk));
  return lead * orc_z_over_x(z, rho) *
         hagan_bracket(alpha, beta, rho, nu, f, K, T);
}

/* Sec. 2.1, eq. (sigma-SABR) with z = nu (f^(1-beta) - K^(1-beta)) /
 * (alpha (1-beta)).  The difference f^(1-beta) - K^(1-beta) is formed as
 * K^(1-beta) expm1((1-beta) ln(f/K)) (an identity: f^(1-beta) =
 * K^(1-beta) e^((1-beta) ln(f/K))) and its beta -> 1 limit ln(f/K).
 * nu ln(f/K)/x(z) = (alpha ln(f/K)/zd) (z/x(z)) with zd = z alpha/nu, which
 * stays finite as nu -> 0; at K = f the first factor is alpha/K^(1-beta). */
double orc_vol_obloj(double alpha, double beta, double rho, double nu,
                     double f, double K, double T) {
  double omb = 1.0 - beta;
  double lfk = log(f / K);
  double zd = (omb == 0.0) ? lfk : pow(K, omb) * expm1(omb * lfk) / omb;
  double z = nu * zd / alpha;
  double lead = (lfk == 0.0) ? alpha / pow(K, omb) : alpha * lfk / zd;
  return lead * orc_z_over_x(z, rho) / log_series(beta, lfk) *
         hagan_bracket(alpha, beta, rho, nu, f, K, T);
}

/* Sec. 2.1, eq. (vola_SABR), omega = f^(1-beta)/alpha, L = ln(K/f). */
double orc_vol_expanded(double alpha, double beta, double rho, double nu,
                        double f, double K, double T) {
  double omb = 1.0 - beta;
  double w = pow(f, omb) / alpha;
  double L = log(K / f);
  double A1 = -0.5 * (omb - rho * nu * w);
  double A2 = (omb * omb + 3.0 * (omb - rho * nu * w) +
               (2.0 - 3.0 * rho * rho) * nu * nu * w * w) / 12.0;
  double B = omb * omb / 24.0 / (w * w) + beta * rho * nu / 4.0 / w +
             (2.0 - 3.0 * rho * rho) / 24.0 * nu * nu;
  return (1.0 + A1 * L + A2 * L * L + B * T) / w;
}

/* ------------------------------------------------------------------------ */
/* Dynamic SABR, Sec. 2.2                                                    */
/* ------------------------------------------------------------------------ */
/* eq. (el_fun_1): rho(t) = rho0 e^{-a t}, nu(t) = nu0 e^{-b t};
 * eq. (el_fun_3): rho(t) = (rho0 + q_rho t) e^{-a t} + d_rho,
 *                 nu(t)  = (nu0 + q_nu t) e^{-b t} + d_nu. */
double orc_rho_t(int dyn_case, const double* p, double t) {
  if (dyn_case == 1) return p[2] * exp(-p[4] * t);
  return (p[2] + p[8] * t) * exp(-p[4] * t) + p[6];
}
double orc_nu_t(int dyn_case, const double* p, double t) {
  if (dyn_case == 1) return p[3] * exp(-p[5] * t);
  return (p[3] + p[9] * t) * exp(-p[5] * t) + p[7];
}

typedef struct { int dyn_case; const double* p; double T; int npan; } dyn_ctx;

static double ig_nu1(double t, void* v) { /* (T-t)^2 nu(t)^2 */
  const dyn_ctx* c = (const dyn_ctx*)v;
  double n = orc_nu_t(c->dyn_case, c->p, t);
  return (c->T - t) * (c->T - t) * n * n;
}
static double ig_nu2(double t, void* v) { /* (T-t) t nu(t)^2 */
  const dyn_ctx* c = (const dyn_ctx*)v;
  double n = orc_nu_t(c->dyn_case, c->p, t);
  return (c->T - t) * t * n * n;
}
static double ig_nurho(double u, void* v) { /* nu(u) rho(u) */
  const dyn_ctx* c = (const dyn_ctx*)v;
  return orc_nu_t(c->dyn_case, c->p, u) * orc_rho_t(c->dyn_case, c->p, u);
}
static double ig_eta1(double t, void* v) { /* (T-t) nu(t) rho(t) */
  const dyn_ctx* c = (const dyn_ctx*)v;
  return (c->T - t) * ig_nurho(t, v);
}
/* G(s) = int_0^s nu(u) rho(u) du by the composite 10-point rule on c->npan
 * equal panels of [0, s].  A fixed rule makes G a smooth function of s, so
 * the outer adaptive integral below converges (an adaptive inner rule would
 * change its subdivision with s and leave non-smooth rounding noise). */
static double G_fixed(const dyn_ctx* c, double s, double* absint) {
  const double h = s / c->npan;
  double g = 0.0, a = 0.0;
  for (int k = 0; k < c->npan; ++k) {
    double ak;
    g += gl10(ig_nurho, (void*)c, k * h, (k + 1) * h, &ak);
    a += ak;
  }
  if (absint) *absint = a;
  return g;
}

/* Panels for G_fixed: the fewest (a power of two) for which doubling them
 * changes G(T) by no more than 1e-15 of int_0^T |nu rho|, or by no more than
 * the rounding of the 10n-term sum itself (8 sqrt(10 n) eps of it): with
 * fast decay rates (a T, b T of order 100) the change never gets below
 * 1e-15 once rounding dominates, and the search would otherwise run to 2^16
 * panels. */
static int choose_panels(dyn_ctx* c) {
  c->npan = 1;
  double a, g = G_fixed(c, c->T, &a);
  for (int n = 2; n <= (1 << 16); n *= 2) {
    c->npan = n;
    double a2, g2 = G_fixed(c, c->T, &a2);
    const double noise = 8.0 * sqrt(10.0 * n) * DBL_EPSILON;
    if (fabs(g2 - g) <= (noise > 1e-15 ? noise : 1e-15) * a2 + 1e-300) return n;
    g = g2;
  }
  return c->npan;
}

/* eta2^2 = (12/T^4) int_0^T int_0^t G(s)^2 ds dt with G(s) = int_0^s nu rho.
 * Exchanging the order of the two outer integrals over 0 <= s <= t <= T
 * (Fubini) gives (12/T^4) int_0^T (T - s) G(s)^2 ds. */
static double ig_eta2(double s, void* v) {
  const dyn_ctx* c = (const dyn_ctx*)v;
  double G = G_fixed(c, s, NULL);
  return (c->T - s) * G * G;
}

void orc_dyn_coeffs(int dyn_case, const double* p, double T, double out[4]) {
  dyn_ctx c = {dyn_case, p, T, 1};
  choose_panels(&c);
  double T2 = T * T, T3 = T2 * T, T4 = T3 * T;
  out[0] = 3.0 / T3 * orc_integrate(ig_nu1, &c, 0.0, T, 1e-15);
  out[1] = 6.0 / T3 * orc_integrate(ig_nu2, &c, 0.0, T, 1e-15);
  out[2] = 2.0 / T2 * orc_integrate(ig_eta1, &c, 0.0, T, 1e-15);
  out[3] = 12.0 / T4 * orc_integrate(ig_eta2, &c, 0.0, T, 1e-14);
}

/* eq. (vola_SABRd) with A1(T), A2(T), B(T) as printed below it. */
double orc_vol_dynamic(int dyn_case, const double* p, double f, double K,
                       double T) {
  double co[4];
  orc_dyn_coeffs(dyn_case, p, T, co);
  double nu1sq = co[0], nu2sq = co[1], eta1 = co[2], eta2sq = co[3];
  double alpha = p[0], beta = p[1], omb = 1.0 - beta;
  double w = pow(f, omb) / alpha;
  double L = log(K / f);
  double A1 = (beta - 1.0) / 2.0 + eta1 * w / 2.0;
  double A2 = omb * omb / 12.0 + (omb - eta1 * w) / 4.0 +
              (4.0 * nu1sq + 3.0 * (eta2sq - 3.0 * eta1 * eta1)) / 24.0 * w * w;
  double B = (omb * omb / 24.0 + w * beta * eta1 / 4.0 +
              (2.0 * nu2sq - 3.0 * eta2sq) / 24.0 * w * w) / (w * w);
  return (1.0 + A1 * L + A2 * L * L + B * T) / w;
}

double orc_implied_vol(int model, const double* p, double f, double K,
                       double T) {
  switch (model) {
    case ORC_HAGAN: return orc_vol_hagan(p[0], p[1], p[2], p[3], f, K, T);
    case ORC_OBLOJ: return orc_vol_obloj(p[0], p[1], p[2], p[3], f, K, T);
    case ORC_EXPANDED: return orc_vol_expanded(p[0], p[1], p[2], p[3], f, K, T);
    case ORC_DYN_I: return orc_vol_dynamic(1, p, f, K, T);
    case ORC_DYN_II: return orc_vol_dynamic(2, p, f, K, T);
    default: return NAN;
  }
}

void orc_implied_vol_batch(int model, const double* p, double f,
                           const double* T, const double* K, int64_t n,
                           double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = orc_implied_vol(model, p, f, K[i], T[i]);
}

/* Feasibility.  A continuous function on [0, Tmax] attains its extremes at
 * the end points or where its derivative vanishes.  For
 * g(t) = (c + q t) e^{-k t} + d, g'(t) = (q - k (c + q t)) e^{-k t} has the
 * single root t* = 1/k - c/q when k != 0 and q != 0. */
static void extremes(double c, double q, double k, double d, double Tmax,
                     double* gmin, double* gmax) {
  double g0 = c + d;
  double g1 = (c + q * Tmax) * exp(-k * Tmax) + d;
  double lo = g0 < g1 ? g0 : g1, hi = g0 < g1 ? g1 : g0;
  if (k != 0.0 && q != 0.0) {
    double ts = 1.0 / k - c / q;
    if (ts > 0.0 && ts < Tmax) {
      double gs = (c + q * ts) * exp(-k * ts) + d;
      if (gs < lo) lo = gs;
      if (gs > hi) hi = gs;
    }
  }
  *gmin = lo;
  *gmax = hi;
}

int orc_feasible(int model, const double* p, double Tmax) {
  if (model != ORC_DYN_II) return 1; /* the box already bounds rho and nu */
  double rmin, rmax, nmin, nmax;
  extremes(p[2], p[8], p[4], p[6], Tmax, &rmin, &rmax);
  extremes(p[3], p[9], p[5], p[7], Tmax, &nmin, &nmax);
  return (rmin >= -1.0 && rmax <= 1.0 && nmin > 0.0) ? 1 : 0;
}

/* Sec. 3, eq. (error_calibrate_relativo). */
double orc_misfit(const double* model_vals, const double* mkt, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double r = (mkt[i] - model_vals[i]) / mkt[i];
    s += r * r;
  }
  return s;
}

/* ------------------------------------------------------------------------ */
/* Random numbers                                                            */
/* ------------------------------------------------------------------------ */
/* Philox4x32-10 as published: per round the two 32x32 -> 64 products
 * M0*c0 and M1*c2 are formed, the new block is
 * (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
 * and the key is bumped by the Weyl constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

double orc_u01(uint32_t w) { return ((double)(w >> 9) + 0.5) * 0x1p-23; }

void orc_box_muller(double u1, double u2, double* z1, double* z2) {
  double r = sqrt(-2.0 * log(u1));
  *z1 = r * cos(2.0 * M_PI * u2);
  *z2 = r * sin(2.0 * M_PI * u2);
}

/* ------------------------------------------------------------------------ */
/* Monte Carlo, Sec. 4                                                       */
/* ------------------------------------------------------------------------ */
static int cmp_dbl(const void* a, const void* b) {
  double x = *(const double*)a, y = *(const double*)b;
  return (x > y) - (x < y);
}

/* Grid: every k/steps_per_year below the last maturity, with each maturity
 * inserted; a grid multiple within 1e-10 of a maturity is that maturity. */
int64_t orc_mc_grid(const double* T, int64_t n, double spy, double* grid,
                    int64_t cap) {
  double* mats = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  memcpy(mats, T, sizeof(double) * n);
  qsort(mats, n, sizeof(double), cmp_dbl);
  int64_t cnt = 0, k = 1;
  for (int64_t m = 0; m < n; ++m) {
    if (m > 0 && mats[m] == mats[m - 1]) continue;
    double Tm = mats[m];
    while ((double)k / spy < Tm - 1e-10) {
      if (cnt < cap) grid[cnt] = (double)k / spy;
      ++cnt;
      ++k;
    }
    if (cnt < cap) grid[cnt] = Tm;
    ++cnt;
    if (fabs((double)k / spy - Tm) <= 1e-10) ++k;
  }
  free(mats);
  return cnt;
}

/* State of one path of the log-Euler scheme. */
typedef struct {
  double F, alpha, t;
  int absorbed;
  uint32_t w[4];
} mc_state;

static void mc_start(const double* p, double f, mc_state* s) {
  s->F = f;
  s->alpha = p[0];
  s->t = 0.0;
  s->absorbed = 0;
  s->w[0] = s->w[1] = s->w[2] = s->w[3] = 0;
}

/* Step i of path `path` (from s->t to grid[i]) of the log-Euler scheme,
 * eq. (dis_SABRd), with the OLD alpha_i in nu-hat.  The time-dependent
 * nu(t), rho(t) of the step are taken at its right end, grid[i] (a reading:
 * the equation prints nu(t_i), but the paper's DSabr_II results of Sec. 6.2
 * -- its EUR/USD prices, and EURO STOXX 50 parameters with rho(0) < -1 --
 * are those of the scheme whose first step uses t_1, not t_0).  The normals
 * of steps 2m and 2m+1 come from Philox block (path, m, 0, tag) by
 * Box-Muller.  Absorption (a reading; the paper is silent): once
 * F < 1e-12 f the path is frozen at F = 0. */
static void mc_step(int model, const double* p, double absorb_at, const double* grid, int64_t i,
                    uint32_t path, const uint32_t key[2], mc_state* s) {
  int dyn = (model == ORC_DYN_I) ? 1 : (model == ORC_DYN_II ? 2 : 0);
  double beta = p[1];
  double h = grid[i] - s->t;
  if ((i & 1) == 0) {
    uint32_t ctr[4] = {path, (uint32_t)(i >> 1), 0u, ORC_TAG_MC};
    orc_philox4x32_10(ctr, key, s->w);
  }
  uint32_t wa = (i & 1) ? s->w[2] : s->w[0], wb = (i & 1) ? s->w[3] : s->w[1];
  double z1, z2;
  orc_box_muller(orc_u01(wa), orc_u01(wb), &z1, &z2);
  double nu = dyn ? orc_nu_t(dyn, p, grid[i]) : p[3];
  double rho = dyn ? orc_rho_t(dyn, p, grid[i]) : p[2];
  double sh = sqrt(h);
  if (!s->absorbed) {
    double nuhat = s->alpha * pow(s->F, beta - 1.0);
    double Fn = s->F * exp(nuhat * (rho * z1 + sqrt(1.0 - rho * rho) * z2) * sh -
                           nuhat * nuhat * h / 2.0);
    if (!(Fn >= absorb_at)) {
      s->absorbed = 1;
      s->F = 0.0;
    } else {
      s->F = Fn;
    }
  }
  s->alpha = s->alpha * exp(nu * z1 * sh - nu * nu * h / 2.0);
  s->t = grid[i];
}

/* Path j of the scheme; at each grid point that is a maturity the payoffs
 * of the options of that maturity are added to sum[] and sumsq[]. */
static void mc_path(int model, const double* p, double f, const double* grid,
                    int64_t n_steps, const double* T, const double* K,
                    const int8_t* is_call, const int64_t* qorder, int64_t n,
                    uint32_t path, const uint32_t key[2], double* sum,
                    double* sumsq) {
  mc_state st;
  mc_start(p, f, &st);
  int64_t qi = 0;
  for (int64_t i = 0; i < n_steps; ++i) {
    mc_step(model, p, 1e-12 * f, grid, i, path, key, &st);
    /* quotes sorted by maturity: pay those that mature at this grid point */
    while (qi < n && fabs(T[qorder[qi]] - st.t) <= 1e-10) {
      int64_t q = qorder[qi++];
      int call = is_call ? is_call[q] != 0 : 1;
      double F = st.F;
      double pay = call ? (F > K[q] ? F - K[q] : 0.0) : (K[q] > F ? K[q] - F : 0.0);
      sum[q] += pay;
      sumsq[q] += pay * pay;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* The conditional-Bessel step (the low-bias fallback Sec. 4 names)          */
/* ------------------------------------------------------------------------ */
/* Write the SDE as dF = alpha F^beta (rho dW + sqrt(1-rho^2) dB),
 * dalpha = nu alpha dW, with W and B independent.  Over one step [t, t+h]
 * (nu, rho those of the step):
 *  1. alpha is a geometric Brownian motion: alpha' = alpha e^{x},
 *     x = nu sqrt(h) Z_a - nu^2 h / 2 (exact).
 *  2. The part of the forward's noise driven by W integrates exactly:
 *     rho int alpha dW = (rho/nu)(alpha' - alpha).  For beta < 1 put
 *     Y = F^{1-beta}/(1-beta); by Ito dY = rho alpha dW + sqrt(1-rho^2) alpha dB
 *     - beta alpha^2 / (2 (1-beta) Y) dt.  The W part is applied at the start
 *     of the step (Y0 = Y + (rho/nu)(alpha' - alpha), the one approximation
 *     besides step 3), and with the clock tau = (1-rho^2) int alpha^2 ds the
 *     rest is dY = dB_tau + (delta - 1)/(2 Y) dtau, a Bessel process of
 *     dimension delta = 1 - beta / ((1-beta)(1-rho^2)) < 2, absorbed at 0
 *     (Chen, Oosterlee and van der Weide reduce the forward the same way).
 *  3. int alpha^2 ds over the step by the trapezoidal rule,
 *     (h/2)(alpha^2 + alpha'^2).
 *  4. Y'^2 given Y0^2 is a squared Bessel process of dimension delta absorbed
 *     at 0, run for time tau.  Its transition is sampled exactly: with
 *     a = 1 - delta/2 and m = Y0^2 / (2 tau), draw G ~ Gamma(a); the path is
 *     absorbed if G >= m, else Y'^2 = tau ((N1 + sqrt(2 (m - G)))^2 + N2^2).
 *     (Expanding the Bessel function of the absorbed transition density
 *     gives weights e^{-m} m^{n+a} / Gamma(n+a+1) times the density of
 *     2 tau Gamma(n+1); these are the law of a Gamma(a) variable G below m
 *     followed by a Poisson(m - G) count n, and a Poisson(lambda/2) mixture
 *     of chi-square laws with 2 + 2n degrees is the noncentral chi-square
 *     with 2 degrees and noncentrality lambda = 2 (m - G): the square of a
 *     normal of mean sqrt(lambda) plus the square of a standard normal.  The
 *     total weight, the probability of not being absorbed, is
 *     P(G < m) = P(a, m), the regularised lower incomplete gamma function.)
 *     With rho^2 = 1 the clock stops and the drift integrates alone:
 *     Y'^2 = Y0^2 - beta/(1-beta) int alpha^2 ds (absorbed if <= 0).
 *  5. beta = 1: Y = ln F, Y' = Y + (rho/nu)(alpha' - alpha) - V/2
 *     + sqrt((1-rho^2) V) N1 with V the integral of step 3; no absorption.
 * The shift (rho/nu)(alpha' - alpha) is formed as alpha rho sqrt(h) expm1(x)
 * / (nu sqrt(h)), which is alpha rho sqrt(h) Z_a at nu = 0.
 * With nu = 0 and rho = 0 every step is exact: the scheme then samples the
 * absorbed CEV law itself, at any step size.
 *
 * Random numbers of step i (grid index) of path j, Philox blocks with
 * counter (j, i, b, ORC_TAG_MB):
 *   block 0: (Z_a, N1) = BoxMuller(u(w0), u(w1)), (N2, X_0) = BoxMuller(u(w2), u(w3))
 *   block 1: U_0 = u(w0), U_b = u(w1)
 *   block k + 1 (k = 1 .. 7, drawn only when needed): X_k = first output of
 *            BoxMuller(u(w0), u(w1)), U_k = u(w2)
 * Gamma(a) by Marsaglia and Tsang's method (ACM TOMS 26(3), 2000): with
 * a' = a (a >= 1) or a + 1 (a < 1), d = a' - 1/3, c = 1/sqrt(9 d), trial k
 * forms v = (1 + c X_k)^3 and accepts d v when v > 0 and either
 * U_k < 1 - 0.0331 X_k^4 or ln U_k < X_k^2/2 + d (1 - v + ln v); for a < 1
 * the draw is multiplied by U_b^{1/a}.  A reading where the method has no
 * bound: after 8 rejected trials (probability below 1e-10) the draw is d. */
#define MB_TRIALS 8

static void mb_block(uint32_t path, int64_t i, uint32_t b, const uint32_t key[2], uint32_t w[4]) {
  uint32_t ctr[4] = {path, (uint32_t)i, b, ORC_TAG_MB};
  orc_philox4x32_10(ctr, key, w);
}

static double mb_gamma(double a, double x0, double u0, double ub, uint32_t path, int64_t i,
                       const uint32_t key[2]) {
  double ap = a >= 1.0 ? a : a + 1.0;
  double d = ap - 1.0 / 3.0;
  double c = 1.0 / sqrt(9.0 * d);
  double g = d;
  for (int k = 0; k < MB_TRIALS; ++k) {
    double x = x0, u = u0;
    if (k > 0) {
      uint32_t w[4];
      double unused;
      mb_block(path, i, (uint32_t)(k + 1), key, w);
      orc_box_muller(orc_u01(w[0]), orc_u01(w[1]), &x, &unused);
      u = orc_u01(w[2]);
    }
    double t = 1.0 + c * x;
    if (!(t > 0.0)) continue;
    double v = t * t * t;
    if (u < 1.0 - 0.0331 * (x * x) * (x * x) || log(u) < 0.5 * x * x + d * (1.0 - v + log(v))) {
      g = d * v;
      break;
    }
  }
  if (a < 1.0) g = g * pow(ub, 1.0 / a);
  return g;
}

void orc_mb_gamma_draws(double a, uint64_t seed, int64_t n, double* out) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int64_t j = 0; j < n; ++j) {
    uint32_t w0[4], w1[4];
    double za, n1, n2, x0;
    mb_block((uint32_t)j, 0, 0u, key, w0);
    mb_block((uint32_t)j, 0, 1u, key, w1);
    orc_box_muller(orc_u01(w0[0]), orc_u01(w0[1]), &za, &n1);
    orc_box_muller(orc_u01(w0[2]), orc_u01(w0[3]), &n2, &x0);
    out[j] = mb_gamma(a, x0, orc_u01(w1[0]), orc_u01(w1[1]), (uint32_t)j, 0, key);
  }
}

/* State of one path of the conditional-Bessel scheme: Y = F^{1-beta}/(1-beta)
 * (beta < 1) or ln F (beta = 1). */
typedef struct {
  double Y, alpha, t;
  int absorbed;
} mb_state;

static void mb_start(const double* p, double f, mb_state* s) {
  double beta = p[1];
  s->Y = beta == 1.0 ? log(f) : pow(f, 1.0 - beta) / (1.0 - beta);
  s->alpha = p[0];
  s->t = 0.0;
  s->absorbed = 0;
}

static double mb_forward(const double* p, const mb_state* s) {
  double beta = p[1];
  if (s->absorbed) return 0.0;
  return beta == 1.0 ? exp(s->Y) : pow((1.0 - beta) * s->Y, 1.0 / (1.0 - beta));
}

/* Step i of path `path` (from s->t to grid[i]); nu(t), rho(t) of the step at
 * its right end, as in mc_step. */
static void mc_step_bessel(int model, const double* p, const double* grid, int64_t i, uint32_t path,
                           const uint32_t key[2], mb_state* s) {
  int dyn = (model == ORC_DYN_I) ? 1 : (model == ORC_DYN_II ? 2 : 0);
  double beta = p[1];
  double h = grid[i] - s->t;
  double nu = dyn ? orc_nu_t(dyn, p, grid[i]) : p[3];
  double rho = dyn ? orc_rho_t(dyn, p, grid[i]) : p[2];
  s->t = grid[i];
  if (s->absorbed) return;
  uint32_t w0[4], w1[4];
  mb_block(path, i, 0u, key, w0);
  mb_block(path, i, 1u, key, w1);
  double za, n1, n2, x0;
  orc_box_muller(orc_u01(w0[0]), orc_u01(w0[1]), &za, &n1);
  orc_box_muller(orc_u01(w0[2]), orc_u01(w0[3]), &n2, &x0);
  double u0 = orc_u01(w1[0]), ub = orc_u01(w1[1]);
  /* step 1: the volatility */
  double sh = sqrt(h);
  double kap = nu * sh;
  double em = expm1(kap * za - 0.5 * kap * kap);
  double alpha_new = s->alpha + s->alpha * em;
  /* step 2: (rho/nu)(alpha' - alpha) */
  double shift = s->alpha * rho * sh * (kap > 0.0 ? em / kap : za);
  /* step 3: int alpha^2 ds */
  double V = 0.5 * h * (s->alpha * s->alpha + alpha_new * alpha_new);
  double omr = (1.0 - rho) * (1.0 + rho);
  s->alpha = alpha_new;
  if (beta == 1.0) { /* step 5 */
    s->Y = s->Y + shift - 0.5 * V + sqrt(omr * V) * n1;
    return;
  }
  double Y0 = s->Y + shift;
  if (!(Y0 > 0.0)) {
    s->absorbed = 1;
    return;
  }
  double tau = omr * V;
  if (!(tau > 0.0)) { /* rho^2 = 1 */
    double y2 = Y0 * Y0 - beta / (1.0 - beta) * V;
    if (!(y2 > 0.0)) {
      s->absorbed = 1;
      return;
    }
    s->Y = sqrt(y2);
    return;
  }
  /* step 4 */
  double a = 0.5 + 0.5 * (beta / (1.0 - beta)) / omr;
  double m = Y0 * Y0 / (2.0 * tau);
  double G = mb_gamma(a, x0, u0, ub, path, i, key);
  if (!(G < m)) {
    s->absorbed = 1;
    return;
  }
  double q = n1 + sqrt(2.0 * (m - G));
  s->Y = sqrt(tau * (q * q + n2 * n2));
}

static void mc_path_bessel(int model, const double* p, double f, const double* grid,
                           int64_t n_steps, const double* T, const double* K,
                           const int8_t* is_call, const int64_t* qorder, int64_t n,
                           uint32_t path, const uint32_t key[2], double* sum,
                           double* sumsq) {
  mb_state st;
  mb_start(p, f, &st);
  int64_t qi = 0;
  for (int64_t i = 0; i < n_steps; ++i) {
    mc_step_bessel(model, p, grid, i, path, key, &st);
    while (qi < n && fabs(T[qorder[qi]] - st.t) <= 1e-10) {
      int64_t q = qorder[qi++];
      int call = is_call ? is_call[q] != 0 : 1;
      double F = mb_forward(p, &st);
      double pay = call ? (F > K[q] ? F - K[q] : 0.0) : (K[q] > F ? K[q] - F : 0.0);
      sum[q] += pay;
      sumsq[q] += pay * pay;
    }
  }
}

int orc_mc_price(int model, const double* p, double f, const double* T,
                 const double* K, const int8_t* is_call, const double* disc,
                 int64_t n, int64_t n_paths, double spy, uint64_t seed,
                 int n_threads, double* price, double* se) {
  return orc_mc_price_scheme(ORC_MC_LOG_EULER, model, p, f, T, K, is_call, disc, n, n_paths, spy, seed,
                             n_threads, price, se);
}

int orc_mc_price_scheme(int scheme, int model, const double* p, double f, const double* T,
                        const double* K, const int8_t* is_call, const double* disc,
                        int64_t n, int64_t n_paths, double spy, uint64_t seed,
                        int n_threads, double* price, double* se) {
  if (scheme != ORC_MC_LOG_EULER && scheme != ORC_MC_BESSEL) return -1;
  if (n <= 0 || n_paths <= 1 || !(spy > 0.0) || !(f > 0.0)) return -1;
  for (int64_t q = 0; q < n; ++q)
    if (!(T[q] > 0.0)) return -1;
  double Tmax = 0.0;
  for (int64_t q = 0; q < n; ++q) Tmax = T[q] > Tmax ? T[q] : Tmax;
  if (!orc_feasible(model, p, Tmax)) return -1;
  int64_t n_steps = orc_mc_grid(T, n, spy, NULL, 0);
  double* grid = (double*)malloc(sizeof(double) * n_steps);
  orc_mc_grid(T, n, spy, grid, n_steps);
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  int64_t* qorder = (int64_t*)malloc(sizeof(int64_t) * n);
  for (int64_t q = 0; q < n; ++q) qorder[q] = q;
  for (int64_t a = 1; a < n; ++a) /* insertion sort by maturity, stable */
    for (int64_t b = a; b > 0 && T[qorder[b - 1]] > T[qorder[b]]; --b) {
      int64_t tmp = qorder[b];
      qorder[b] = qorder[b - 1];
      qorder[b - 1] = tmp;
    }
  /* Fixed blocks of paths, summed in block order: the result does not
   * depend on the number of threads. */
  const int64_t BLK = 4096;
  int64_t nblk = (n_paths + BLK - 1) / BLK;
  double* part = (double*)calloc((size_t)nblk * 2 * n, sizeof(double));
  if (n_threads < 1) n_threads = 1;
#pragma omp parallel for schedule(dynamic) num_threads(n_threads)
  for (int64_t b = 0; b < nblk; ++b) {
    double* s = part + b * 2 * n;
    double* s2 = s + n;
    int64_t j1 = (b + 1) * BLK < n_paths ? (b + 1) * BLK : n_paths;
    for (int64_t j = b * BLK; j < j1; ++j) {
      if (scheme == ORC_MC_BESSEL)
        mc_path_bessel(model, p, f, grid, n_steps, T, K, is_call, qorder, n, (uint32_t)j, key, s, s2);
      else
        mc_path(model, p, f, grid, n_steps, T, K, is_call, qorder, n, (uint32_t)j, key, s, s2);
    }
  }
  for (int64_t q = 0; q < n; ++q) {
    double s = 0.0, s2 = 0.0;
    for (int64_t b = 0; b < nblk; ++b) {
      s += part[b * 2 * n + q];
      s2 += part[b * 2 * n + n + q];
    }
    double N = (double)n_paths;
    double mean = s / N;
    double var = (s2 - s * mean) / (N - 1.0);
    if (var < 0.0) var = 0.0;
    double D = disc ? disc[q] : 1.0;
    price[q] = D * mean; /* eq. (payoff) */
    if (se) se[q] = D * sqrt(var / N);
  }
  free(part);
  free(grid);
  free(qorder);
  return 0;
}

/* Cliquet of Sec. 6.3 on one path: F is recorded at the reset dates
 * d_1 < ... < d_n (grid points), R_i = F(d_i)/F(d_{i-1}) - 1 for i = 2..n,
 * eq. (eq_cliquet) sums max(min(R_i, cap_l), floor_l), and the global limits
 * give max(floor_g, min(cap_g, sum)) (eq. (cliquet_global) with its two
 * limits in the order that makes floor_g a floor).  A path absorbed before
 * d_{i-1} has F(d_{i-1}) = 0 and contributes R_i = 0 (0 to 0); absorbed
 * between d_{i-1} and d_i it contributes R_i = -1. */
static double cliquet_path(int model, const double* p, double f, const double* grid,
                           int64_t n_steps, const double* resets, int n_resets,
                           double floor_l, double cap_l, double floor_g, double cap_g,
                           uint32_t path, const uint32_t key[2]) {
  mc_state st;
  mc_start(p, f, &st);
  int ri = 0;
  double prev = 0.0, sum = 0.0;
  for (int64_t i = 0; i < n_steps; ++i) {
    mc_step(model, p, 1e-12 * f, grid, i, path, key, &st);
    if (ri < n_resets && fabs(resets[ri] - st.t) <= 1e-10) {
      if (ri >= 1) {
        double R = prev > 0.0 ? st.F / prev - 1.0 : 0.0;
        double c = R < cap_l ? R : cap_l;
        sum += c > floor_l ? c : floor_l;
      }
      prev = st.F;
      ++ri;
    }
  }
  double g = sum < cap_g ? sum : cap_g;
  return g > floor_g ? g : floor_g;
}

int orc_mc_cliquet(int model, const double* p, double f, double T, int n_resets,
                   double floor_l, double cap_l, double floor_g, double cap_g,
                   double disc, int64_t n_paths, double spy, uint64_t seed,
                   int n_threads, double* price, double* se) {
  if (!(T > 0.0) || n_resets < 2 || n_paths <= 1 || !(spy > 0.0) || !(f > 0.0)) return -1;
  if (!orc_feasible(model, p, T)) return -1;
  double* resets = (double*)malloc(sizeof(double) * n_resets);
  for (int i = 0; i < n_resets; ++i) resets[i] = (double)(i + 1) * T / n_resets;
  int64_t n_steps = orc_mc_grid(resets, n_resets, spy, NULL, 0);
  double* grid = (double*)malloc(sizeof(double) * n_steps);
  orc_mc_grid(resets, n_resets, spy, grid, n_steps);
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  const int64_t BLK = 4096;
  int64_t nblk = (n_paths + BLK - 1) / BLK;
  double* part = (double*)calloc((size_t)nblk * 2, sizeof(double));
  if (n_threads < 1) n_threads = 1;
#pragma omp parallel for schedule(dynamic) num_threads(n_threads)
  for (int64_t b = 0; b < nblk; ++b) {
    int64_t j1 = (b + 1) * BLK < n_paths ? (b + 1) * BLK : n_paths;
    for (int64_t j = b * BLK; j < j1; ++j) {
      double v = cliquet_path(model, p, f, grid, n_steps, resets, n_resets, floor_l, cap_l,
                              floor_g, cap_g, (uint32_t)j, key);
      part[2 * b] += v;
      part[2 * b + 1] += v * v;
    }
  }
  double s = 0.0, s2 = 0.0;
  for (int64_t b = 0; b < nblk; ++b) {
    s += part[2 * b];
    s2 += part[2 * b + 1];
  }
  double N = (double)n_paths, mean = s / N, var = (s2 - s * mean) / (N - 1.0);
  if (var < 0.0) var = 0.0;
  *price = disc * mean;
  if (se) *se = disc * sqrt(var / N);
  free(part);
  free(grid);
  free(resets);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Simulated Annealing, Sec. 5                                               */
/* ------------------------------------------------------------------------ */
typedef struct {
  int model, cost;
  double f;
  int64_t n;
  const double *T, *K, *mkt, *disc;
  const int8_t* is_call;
  int64_t mc_paths;
  double mc_spy;
  uint64_t mc_seed;
  double Tmax;
  double* scratch; /* 2n doubles per thread */
} sa_ctx;

/* Cost of x: eq. (error_calibrate_relativo) with Data = vols (Technique I)
 * or MC prices (Technique II).  NaN marks an evaluation that failed. */
static double sa_cost(const sa_ctx* c, const double* x, double* scratch) {
  if (c->cost == ORC_COST_VOL) {
    orc_implied_vol_batch(c->model, x, c->f, c->T, c->K, c->n, scratch);
  } else {
    if (orc_mc_price(c->model, x, c->f, c->T, c->K, c->is_call, c->disc, c->n,
                     c->mc_paths, c->mc_spy, c->mc_seed, 1, scratch, NULL) != 0)
      return NAN;
  }
  return orc_misfit(scratch, c->mkt, c->n);
}

/* The uniforms of proposal (chain, level, step) of a d-parameter model.
 * Word j (j < d) is word j%4 of the Philox block with counter
 * (chain, level, step, TAG_SA + j/4); u[j] = orc_u01(word j) moves
 * parameter j.  orc_u01 keeps the top 23 bits of a word, so words 0, 1, 2
 * carry 9 + 9 + 9 unused low bits; the acceptance uniform u[d] is the 23-bit
 * integer whose bits, high to low, are the low 9 bits of word 0, the low 9
 * of word 1 and the low 5 of word 2, mapped like any other 23-bit draw. */
void orc_sa_uniforms(const uint32_t key[2], int chain, int level, int step,
                     int d, double* u) {
  uint32_t w[4], spare[3] = {0u, 0u, 0u};
  for (int j = 0; j < d; ++j) {
    if ((j & 3) == 0) {
      uint32_t ctr[4] = {(uint32_t)chain, (uint32_t)level, (uint32_t)step,
                         ORC_TAG_SA + (uint32_t)(j >> 2)};
      orc_philox4x32_10(ctr, key, w);
    }
    u[j] = orc_u01(w[j & 3]);
    if (j < 3) spare[j] = w[j & 3] % 512u; /* the bits below the top 23 */
  }
  uint32_t bits = spare[0] * 16384u + spare[1] * 32u + spare[2] % 32u;
  u[d] = ((double)bits + 0.5) * 0x1p-23;
}

/* Temperature and step scale of level lev: geometric cooling
 * T_k = T0 c^k and s_k = max(s_min, s0 sqrt(T_k / T0)). */
static void sa_level_schedule(double T0, double factor, int lev, double step0,
                              double step_min, double* Tk, double* sk) {
  *Tk = T0 * pow(factor, (double)lev);
  *sk = step0 * sqrt(*Tk / T0);
  if (*sk < step_min) *sk = step_min;
}

/* chain_len Metropolis steps of level lev for the nc chains c0 .. c0+nc-1:
 * state i (chain c0 + i) is x = cx + 10 i with cost cf[i], its best-ever
 * point bx + 10 i, bf[i], and its counters ev[i], ac[i]. */
static void sa_level_chains(const sa_ctx* c, int d, const double* lo,
                            const double* hi, const uint32_t key[2], double Tk,
                            double sk, int lev, int chain_len, int c0, int nc,
                            double* cx, double* cf, double* bx, double* bf,
                            int64_t* ev, int64_t* ac, double* scratch,
                            int n_threads) {
#pragma omp parallel for schedule(static) num_threads(n_threads)
  for (int i = 0; i < nc; ++i) {
    const int ch = c0 + i;
    double* x = cx + 10 * i;
    double* scr = scratch + c->n * i;
    double u[11], xp[10];
    for (int st = 0; st < chain_len; ++st) {
      orc_sa_uniforms(key, ch, lev, st, d, u);
      int inside = 1;
      for (int j = 0; j < 10; ++j) xp[j] = 0.0;
      for (int j = 0; j < d; ++j) {
        double step = sk * (hi[j] - lo[j]);
        xp[j] = x[j] + step * (2.0 * u[j] - 1.0);
        if (xp[j] < lo[j] || xp[j] > hi[j]) inside = 0;
      }
      if (!inside || !orc_feasible(c->model, xp, c->Tmax)) continue;
      double fp = sa_cost(c, xp, scr);
      ev[i]++;
      if (!(fp == fp)) continue;
      if (fp < bf[i]) { /* best-ever over every evaluated point */
        bf[i] = fp;
        memcpy(bx + 10 * i, xp, sizeof(xp));
      }
      double delta = fp - cf[i];
      if (delta <= 0.0 || u[d] < exp(-delta / Tk)) { /* Metropolis */
        memcpy(x, xp, sizeof(xp));
        cf[i] = fp;
        ac[i]++;
      }
    }
  }
}

int orc_sa_calibrate(int model, int cost, double f, int64_t n,
                     const double* T, const double* K, const double* mkt,
                     const double* disc, const int8_t* is_call, int n_chains,
                     int64_t mc_paths, double mc_spy, uint64_t mc_seed,
                     const double* x0, const double* lo, const double* hi,
                     double T0, double factor, int n_levels, int chain_len,
                     double step0, double step_min, uint64_t seed,
                     int n_threads, double* best_x, double* best_f,
                     double* restart_x, double* restart_f, int64_t* n_evals,
                     int64_t* n_accepts, double* trace) {
  int d = orc_n_params(model);
  if (d < 0 || n <= 0 || n_chains <= 0 || n_levels < 0 || chain_len < 0)
    return -1;
  for (int64_t q = 0; q < n; ++q)
    if (!(mkt[q] != 0.0) || !(T[q] > 0.0) || !(K[q] > 0.0)) return -1;
  for (int i = 0; i < d; ++i)
    if (!(lo[i] <= hi[i])) return -1;
  sa_ctx c = {model, cost, f, n, T, K, mkt, disc, is_call, mc_paths, mc_spy,
              mc_seed, 0.0, NULL};
  for (int64_t q = 0; q < n; ++q) c.Tmax = T[q] > c.Tmax ? T[q] : c.Tmax;
  if (n_threads < 1) n_threads = 1;

  /* Level 0: every chain starts from x0 (the box midpoint if none given). */
  double xs[10], fs;
  for (int i = 0; i < 10; ++i) xs[i] = 0.0;
  for (int i = 0; i < d; ++i) xs[i] = x0 ? x0[i] : 0.5 * (lo[i] + hi[i]);
  for (int i = 0; i < d; ++i)
    if (xs[i] < lo[i] || xs[i] > hi[i]) return -1;
  if (!orc_feasible(model, xs, c.Tmax)) return -1;
  double* scr0 = (double*)malloc(sizeof(double) * n);
  fs = sa_cost(&c, xs, scr0);
  free(scr0);
  if (!(fs == fs)) return -1;
  if (!(T0 > 0.0)) T0 = fs > 0.0 ? fs : 1.0;

  double* cx = (double*)malloc(sizeof(double) * 10 * n_chains);
  double* cf = (double*)malloc(sizeof(double) * n_chains);
  double* bx = (double*)malloc(sizeof(double) * 10 * n_chains);
  double* bf = (double*)malloc(sizeof(double) * n_chains);
  int64_t* ev = (int64_t*)calloc(n_chains, sizeof(int64_t));
  int64_t* ac = (int64_t*)calloc(n_chains, sizeof(int64_t));
  double* scratch = (double*)malloc(sizeof(double) * n * n_chains);
  for (int ch = 0; ch < n_chains; ++ch) {
    memcpy(cx + 10 * ch, xs, sizeof(xs));
    memcpy(bx + 10 * ch, xs, sizeof(xs));
    cf[ch] = fs;
    bf[ch] = fs;
  }
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};

  for (int lev = 0; lev < n_levels; ++lev) {
    double Tk, sk;
    sa_level_schedule(T0, factor, lev, step0, step_min, &Tk, &sk);
    sa_level_chains(&c, d, lo, hi, key, Tk, sk, lev, chain_len, 0, n_chains,
                    cx, cf, bx, bf, ev, ac, scratch, n_threads);
    /* Level end: the chain with the lowest final cost (lowest index on a
     * tie) gives the common start of the next level. */
    int arg = 0;
    for (int ch = 1; ch < n_chains; ++ch)
      if (cf[ch] < cf[arg]) arg = ch;
    memcpy(xs, cx + 10 * arg, sizeof(xs));
    fs = cf[arg];
    for (int ch = 0; ch < n_chains; ++ch) {
      memcpy(cx + 10 * ch, xs, sizeof(xs));
      cf[ch] = fs;
    }
    if (trace) trace[lev] = fs;
  }

  int barg = 0;
  for (int ch = 1; ch < n_chains; ++ch)
    if (bf[ch] < bf[barg]) barg = ch;
  if (best_x) memcpy(best_x, bx + 10 * barg, sizeof(double) * 10);
  if (best_f) *best_f = bf[barg];
  if (restart_x) memcpy(restart_x, xs, sizeof(double) * 10);
  if (restart_f) *restart_f = fs;
  int64_t te = 0, ta = 0;
  for (int ch = 0; ch < n_chains; ++ch) {
    te += ev[ch];
    ta += ac[ch];
  }
  if (n_evals) *n_evals = te;
  if (n_accepts) *n_accepts = ta;
  free(cx);
  free(cf);
  free(bx);
  free(bf);
  free(ev);
  free(ac);
  free(scratch);
  return 0;
}

/* One level of orc_sa_calibrate for the chains c0 .. c0+nc-1 only (the
 * multi-GPU form of Sec. 5.1: each device runs a share of the chains and the
 * host takes the minimum of the shares' minima at every level).  Every
 * chain starts from the restart point (xs, fs); on return cx/cf hold the
 * chains' final states (the caller takes the argmin over all shares, lowest
 * chain on a tie) and bx/bf/ev/ac (indexed by chain - c0) are updated.
 * T0 is the first level's temperature (f(x0) when the caller's schedule
 * says so). */
int orc_sa_shard_level(int model, int cost, double f, int64_t n,
                       const double* T, const double* K, const double* mkt,
                       const double* disc, const int8_t* is_call,
                       int64_t mc_paths, double mc_spy, uint64_t mc_seed,
                       const double* lo, const double* hi, double T0,
                       double factor, int lev, int chain_len, double step0,
                       double step_min, uint64_t seed, int n_threads, int c0,
                       int nc, const double* xs, double fs, double* cx,
                       double* cf, double* bx, double* bf, int64_t* ev,
                       int64_t* ac) {
  int d = orc_n_params(model);
  if (d < 0 || n <= 0 || nc <= 0 || c0 < 0 || lev < 0 || chain_len < 0 ||
      !(T0 > 0.0))
    return -1;
  sa_ctx c = {model, cost, f, n, T, K, mkt, disc, is_call, mc_paths, mc_spy,
              mc_seed, 0.0, NULL};
  for (int64_t q = 0; q < n; ++q) c.Tmax = T[q] > c.Tmax ? T[q] : c.Tmax;
  if (n_threads < 1) n_threads = 1;
  for (int i = 0; i < nc; ++i) {
    memcpy(cx + 10 * i, xs, sizeof(double) * 10);
    cf[i] = fs;
  }
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  double Tk, sk;
  sa_level_schedule(T0, factor, lev, step0, step_min, &Tk, &sk);
  double* scratch = (double*)malloc(sizeof(double) * n * nc);
  sa_level_chains(&c, d, lo, hi, key, Tk, sk, lev, chain_len, c0, nc, cx, cf,
                  bx, bf, ev, ac, scratch, n_threads);
  free(scratch);
  return 0;
}
