/*
 * sabr_oracle.h -- plain FP64 CPU oracle for the SABR calibration hot path of
 * Fernandez, Ferreiro, Garcia, Leitao, Lopez-Salas, Vazquez, "Static and
 * dynamic SABR stochastic volatility models: calibration and option pricing
 * using GPUs".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library
 * and its Python binding) may include, link or call this code; only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg do.  It shares
 * no code, header, table or constant generator with the CUDA path.
 *
 * Every routine is written for a reader checking it against the paper by eye:
 * straight FP64 arithmetic, no blocking, no fusion.  Where the paper is
 * silent the reading taken is stated beside the code.
 *
 * Parameter vector layout (all models), double p[10]:
 *   p[0]=alpha p[1]=beta p[2]=rho0 p[3]=nu0 p[4]=a p[5]=b
 *   p[6]=d_rho p[7]=d_nu p[8]=q_rho p[9]=q_nu
 * Static models read p[0..3] with rho=rho0, nu=nu0; dynamic Case I reads
 * p[0..5]; dynamic Case II reads all ten.
 */
#ifndef SABR_ORACLE_H
#define SABR_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Model identifiers. */
enum {
  ORC_HAGAN = 0,    /* Sec. 2.1, eq. (haganf): Hagan et al. implied vol      */
  ORC_OBLOJ = 1,    /* Sec. 2.1, eq. (sigma-SABR): Oblój correction          */
  ORC_EXPANDED = 2, /* Sec. 2.1, eq. (vola_SABR): expanded static form       */
  ORC_DYN_I = 3,    /* Sec. 2.2, eqs. (vola_SABRd) + (el_fun_1), Case I      */
  ORC_DYN_II = 4    /* Sec. 2.2, eqs. (vola_SABRd) + (el_fun_3), Case II     */
};
enum { ORC_COST_VOL = 0, ORC_COST_MC = 1 };

/* Number of calibrated coordinates for a model: 4, 6 or 10. */
int orc_n_params(int model);

/* Adaptive Gauss-Legendre quadrature of f over [a,b] to relative tolerance
 * rtol (of the integral of |f|).  Exposed so the tests can pin it. */
typedef double (*orc_fn)(double t, void* ctx);
double orc_integrate(orc_fn f, void* ctx, double a, double b, double rtol);
/* Integrates p(t)=sum_k c[k] t^k; used by the tests to pin the rule. */
double orc_integrate_poly(const double* c, int deg, double a, double b);

/* Sec. 2.1, eq. (equis): x(z) = ln((sqrt(1-2 rho z + z^2) + z - rho)/(1-rho)).
 * Returns z/x(z) (=1 at z=0). */
double orc_x_of_z(double z, double rho);
double orc_z_over_x(double z, double rho);

/* Static implied volatilities, Sec. 2.1. */
double orc_vol_hagan(double alpha, double beta, double rho, double nu,
                     double f, double K, double T);
double orc_vol_obloj(double alpha, double beta, double rho, double nu,
                     double f, double K, double T);
double orc_vol_expanded(double alpha, double beta, double rho, double nu,
                        double f, double K, double T);

/* Sec. 2.2: rho(t), nu(t) of Case I (eq. el_fun_1) or Case II (eq. el_fun_3).
 * dyn_case is 1 or 2. */
double orc_rho_t(int dyn_case, const double* p, double t);
double orc_nu_t(int dyn_case, const double* p, double t);

/* Sec. 2.2, eq. (integrales_SABRd): out = {nu1^2, nu2^2, eta1, eta2^2} at T,
 * by adaptive quadrature of the definitions. */
void orc_dyn_coeffs(int dyn_case, const double* p, double T, double out[4]);

/* Sec. 2.2, eq. (vola_SABRd) with the coefficients above. */
double orc_vol_dynamic(int dyn_case, const double* p, double f, double K,
                       double T);

/* Dispatch on the model id; p as in the layout above. */
double orc_implied_vol(int model, const double* p, double f, double K, double T);
void orc_implied_vol_batch(int model, const double* p, double f,
                           const double* T, const double* K, int64_t n,
                           double* out);

/* Sec. 2.2 (after eq. el_fun_3) and Sec. 5.2: rho(t) in [-1,1] and
 * nu(t) > 0 for t in (0, Tmax].  1 = feasible, 0 = not. */
int orc_feasible(int model, const double* p, double Tmax);

/* Sec. 3, eq. (error_calibrate_relativo): sum ((mkt - model)/mkt)^2. */
double orc_misfit(const double* model_vals, const double* mkt, int64_t n);

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), one block. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]);
/* 32-bit word -> uniform in (0,1): ((w >> 9) + 0.5) * 2^-23. */
double orc_u01(uint32_t w);
/* The d + 1 uniforms of SA proposal (chain, level, step) of a d-parameter
 * model: u[0..d-1] move the parameters, u[d] decides acceptance. */
void orc_sa_uniforms(const uint32_t key[2], int chain, int level, int step,
                     int d, double* u);
/* Box-Muller: two uniforms -> two independent standard normals. */
void orc_box_muller(double u1, double u2, double* z1, double* z2);

/* Counter tags (counter word 3) that keep the SA and MC streams apart. */
#define ORC_TAG_SA 0x53410000u
#define ORC_TAG_MC 0x4D430000u

/* Sec. 4, eqs. (dis_SABRd), (payoff): Monte Carlo prices of n European
 * options sharing one forward f.  Static models use the constant-parameter
 * SDE (eqs. model_staticSABR1/2), DYN_I/DYN_II use nu(t), rho(t) at each
 * step's right end (see mc_step).
 * disc may be NULL (=1), is_call may be NULL (=all calls).
 * Returns 0 on success, -1 on invalid input. */
int orc_mc_price(int model, const double* p, double f, const double* T,
                 const double* K, const int8_t* is_call, const double* disc,
                 int64_t n, int64_t n_paths, double steps_per_year,
                 uint64_t seed, int n_threads, double* price, double* stderr_out);

/* Path schemes of the Monte Carlo pricer.  ORC_MC_LOG_EULER is the paper's
 * scheme (Sec. 4, eq. (dis_SABRd)); ORC_MC_BESSEL is the low-bias variant
 * the paper names as the fallback for log-Euler (Sec. 4, the scheme of Chen,
 * Oosterlee and van der Weide): the volatility is stepped exactly, the
 * forward is mapped, given the volatility path, to a squared Bessel process
 * absorbed at zero, and that process is sampled exactly (see mc_step_bessel). */
enum { ORC_MC_LOG_EULER = 0, ORC_MC_BESSEL = 1 };
/* Counter tag of the conditional-Bessel step's Philox blocks. */
#define ORC_TAG_MB 0x4D420000u
/* orc_mc_price with a choice of scheme (same arguments and result). */
int orc_mc_price_scheme(int scheme, int model, const double* p, double f,
                        const double* T, const double* K, const int8_t* is_call,
                        const double* disc, int64_t n, int64_t n_paths,
                        double steps_per_year, uint64_t seed, int n_threads,
                        double* price, double* stderr_out);
/* n Gamma(a) draws of the conditional-Bessel step's sampler, draw j from the
 * words of path j, step 0 (the sampler exactly as the step uses it). */
void orc_mb_gamma_draws(double a, uint64_t seed, int64_t n, double* out);

/* Sec. 6.3, eqs. (eq_cliquet), (cliquet_global): a cliquet on the forward
 * with reset dates d_i = i T / n_resets (i = 1 .. n_resets), paying
 * sum_{i=2..n} max(min(R_i, cap_l), floor_l), R_i = F(d_i)/F(d_{i-1}) - 1,
 * then max(floor_g, min(cap_g, .)) (the printed global formula has the two
 * limits swapped; with floor_g = 0 < cap_g it would be constant), times
 * disc.  Same paths as orc_mc_price (grid with the reset dates inserted). */
int orc_mc_cliquet(int model, const double* p, double f, double T, int n_resets,
                   double floor_l, double cap_l, double floor_g, double cap_g,
                   double disc, int64_t n_paths, double steps_per_year,
                   uint64_t seed, int n_threads, double* price, double* se);

/* The step grid the MC walks: multiples of 1/steps_per_year with every
 * maturity inserted.  Writes up to cap points; returns the count. */
int64_t orc_mc_grid(const double* T, int64_t n, double steps_per_year,
                    double* grid, int64_t cap);

/* Sec. 5, synchronous parallel Simulated Annealing (Technique I when
 * cost == ORC_COST_VOL, Technique II when cost == ORC_COST_MC).
 * trace (may be NULL) receives the restart misfit after every level. */
int orc_sa_calibrate(int model, int cost, double f, int64_t n,
                     const double* T, const double* K, const double* mkt,
                     const double* disc, const int8_t* is_call,
                     int n_chains, int64_t mc_paths, double mc_steps_per_year,
                     uint64_t mc_seed, const double* x0,
                     const double* lo, const double* hi,
                     double T0, double factor, int n_levels, int chain_len,
                     double step0, double step_min,
                     uint64_t seed, int n_threads,
                     double* best_x, double* best_f,
                     double* restart_x, double* restart_f,
                     int64_t* n_evals, int64_t* n_accepts, double* trace);

/* One level of orc_sa_calibrate for chains c0 .. c0+nc-1 from the restart
 * point (xs, fs): the share of one device in the multi-GPU form of Sec. 5.1.
 * cx[10 nc], cf[nc] receive the final states; bx, bf, ev, ac (indexed by
 * chain - c0) carry the best-ever points and counters across levels. */
int orc_sa_shard_level(int model, int cost, double f, int64_t n,
                       const double* T, const double* K, const double* mkt,
                       const double* disc, const int8_t* is_call,
                       int64_t mc_paths, double mc_spy, uint64_t mc_seed,
                       const double* lo, const double* hi, double T0,
                       double factor, int lev, int chain_len, double step0,
                       double step_min, uint64_t seed, int n_threads, int c0,
                       int nc, const double* xs, double fs, double* cx,
                       double* cf, double* bx, double* bf, int64_t* ev,
                       int64_t* ac);

#ifdef __cplusplus
}
#endif
#endif /* SABR_ORACLE_H */
