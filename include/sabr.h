/*
 * sabr.h -- C-ABI of libsabr.so: SABR implied volatilities, Monte Carlo
 * prices and Simulated-Annealing calibration on one NVIDIA GB300 (sm_103a).
 *
 * Method: Fernandez, Ferreiro, Garcia, Leitao, Lopez-Salas, Vazquez,
 * "Static and dynamic SABR stochastic volatility models: calibration and
 * option pricing using GPUs".  Citations below name the paper's sections and
 * equation labels.
 *
 * Conventions for every entry point
 *  - Plain C types only; no exceptions cross the ABI.  Every call returns a
 *    sabr_status; on failure sabr_last_error() gives a message (per thread).
 *  - "device" pointers are CUDA global-memory pointers of the current device;
 *    "host" pointers are ordinary (pageable or pinned) host memory.
 *  - cuda_stream is a cudaStream_t (NULL = legacy default stream).  Calls
 *    documented as asynchronous only enqueue work on that stream.
 *  - The caller owns every buffer it passes in; the library never frees
 *    caller memory.  Library-owned memory lives inside plans and servers and
 *    is released by their destroy calls.
 *  - Parameter vector layout, double params[10]:
 *      [0]=alpha [1]=beta [2]=rho0 [3]=nu0 [4]=a [5]=b
 *      [6]=d_rho [7]=d_nu [8]=q_rho [9]=q_nu
 *    Static models (HAGAN, OBLOJ, EXPANDED) read [0..3] (rho = rho0,
 *    nu = nu0); DYN_I reads [0..5]; DYN_II reads all ten.
 */
#ifndef SABR_H
#define SABR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SABR_OK = 0,
  SABR_EINVAL = 1,     /* an argument is out of range or inconsistent      */
  SABR_ENOMEM = 2,     /* device or pinned host memory could not be had    */
  SABR_ECUDA = 3,      /* a CUDA runtime call failed                       */
  SABR_ETIMEOUT = 4,   /* a bounded wait ran out                           */
  SABR_EAGAIN = 5,     /* result not ready yet (server poll)               */
  SABR_EBUSY = 6,      /* server queue full                                */
  SABR_ECANCELLED = 7, /* request cancelled before it finished             */
  SABR_ENOTFOUND = 8   /* unknown server ticket                            */
} sabr_status;

typedef enum {
  SABR_HAGAN = 0,    /* Sec. 2.1, eq. (haganf): Hagan implied vol          */
  SABR_OBLOJ = 1,    /* Sec. 2.1, eq. (sigma-SABR): Oblój correction       */
  SABR_EXPANDED = 2, /* Sec. 2.1, eq. (vola_SABR): expanded static form    */
  SABR_DYN_I = 3,    /* Sec. 2.2, eq. (vola_SABRd), eq. (el_fun_1)         */
  SABR_DYN_II = 4    /* Sec. 2.2, eq. (vola_SABRd), eq. (el_fun_3)         */
} sabr_model;

typedef enum {
  SABR_COST_VOL = 0,     /* Technique I (Sec. 5.1): misfit in implied vols */
  SABR_COST_MC_PRICE = 1 /* Technique II (Sec. 5.2): misfit in MC prices   */
} sabr_cost;

typedef enum {
  SABR_FP32 = 0, /* FP32 bulk arithmetic; misfit sums across lanes in  */
                 /* double-float (FP32 pairs), MC payoff sums in FP64,  */
                 /* FP64 re-score of the returned point                 */
  SABR_FP64 = 1  /* FP64 throughout                                     */
} sabr_precision;

typedef enum {
  SABR_MC_LOG_EULER = 0, /* Sec. 4, eq. (dis_SABRd): the paper's scheme     */
  SABR_MC_BESSEL = 1     /* conditional-Bessel step: the low-bias fallback  */
                         /* Sec. 4 names (see sabr_mc_price_scheme)         */
} sabr_mc_scheme;

/* ------------------------------------------------------------------------
 * sabr_implied_vol -- model implied volatility of n European options.
 * Sec. 2.1 eqs. (haganf), (sigma-SABR), (vola_SABR); Sec. 2.2 eq.
 * (vola_SABRd) with nu1^2, nu2^2, eta1, eta2^2 of eq. (integrales_SABRd).
 *   params  host, double[10] (layout above)
 *   fwd     forward f > 0 common to all n options
 *   T, K    device, double[n]: maturities (years, > 0) and strikes (> 0)
 *   vol_out device, double[n]
 * Asynchronous on cuda_stream.  n == 0 is a no-op.  EINVAL for a bad model,
 * precision, fwd or parameter set (alpha <= 0, beta outside [0,1], |rho|
 * >= 1 for static models, nu < 0, a or b < 0).
 * ------------------------------------------------------------------------ */
sabr_status sabr_implied_vol(sabr_model model, const double* params,
                             double fwd, const double* T, const double* K,
                             int64_t n, double* vol_out,
                             sabr_precision prec, void* cuda_stream);

/* ------------------------------------------------------------------------
 * sabr_mc_price -- Monte Carlo prices of n European options on one path
 * set, Sec. 4: log-Euler scheme eq. (dis_SABRd) (exact lognormal step of
 * the vol, log-Euler step of the forward with the old vol), price estimator
 * eq. (payoff).  One path serves every maturity: the step grid is every
 * multiple of 1/steps_per_year with each maturity inserted.  The forward is
 * absorbed (frozen at 0) once it falls below 1e-12 * fwd.
 *   params       host, double[10]; static models use constant nu and rho,
 *                DYN_I / DYN_II use nu(t), rho(t) at each step's right end
 *                (the paper prints nu(t_i), but its DSabr_II results of
 *                Sec. 6.2 are those of the right end)
 *   T, K         host, double[n]; maturities > 0, strikes >= 0
 *   is_call      host, int8[n] (nonzero = call) or NULL (all calls)
 *   discount     host, double[n] discount factors or NULL (all 1)
 *   n_paths      >= 2; path j draws its normals from Philox4x32-10 with
 *                key = seed and counter (j, step/2, 0, 0x4D430000)
 *   price_out    device, double[n]
 *   stderr_out   device, double[n] or NULL: standard error of each price
 * Asynchronous on cuda_stream; the host arrays are read before return.
 * Uses library-owned device scratch (per-block partial sums).  EINVAL for
 * bad sizes, n > 512 options, more than 64 distinct maturities, more than
 * 8192 time steps, step and option tables beyond one block's shared memory
 * (the step table takes 16 B a step in FP32 and 32 B in FP64, so FP64 stops
 * near 5000 steps), or parameters violating rho(t) in [-1,1], nu(t) > 0 on
 * (0, max T].
 * ------------------------------------------------------------------------ */
sabr_status sabr_mc_price(sabr_model model, const double* params, double fwd,
                          const double* T, const double* K,
                          const int8_t* is_call, const double* discount,
                          int64_t n, int64_t n_paths, double steps_per_year,
                          uint64_t seed, double* price_out, double* stderr_out,
                          sabr_precision prec, void* cuda_stream);

/* ------------------------------------------------------------------------
 * sabr_mc_price_scheme -- sabr_mc_price with a choice of path scheme.  Same
 * arguments, layout, ownership and checks; scheme SABR_MC_LOG_EULER gives
 * exactly sabr_mc_price.  SABR_MC_BESSEL is the low-bias scheme Sec. 4 names
 * as the fallback for log-Euler (after Chen, Oosterlee and van der Weide):
 * per step, with nu(t), rho(t) at the step's right end,
 *   - the vol moves exactly, alpha' = alpha exp(nu sqrt(h) Z - nu^2 h/2);
 *   - rho int alpha dW = (rho/nu)(alpha' - alpha) is added to
 *     Y = F^(1-beta)/(1-beta) at the start of the step;
 *   - int alpha^2 ds is taken by the trapezoidal rule;
 *   - given those, Y^2 is a squared Bessel process of dimension
 *     1 - beta/((1-beta)(1-rho^2)) absorbed at 0 on the clock
 *     (1-rho^2) int alpha^2 ds, sampled exactly (a Gamma draw by Marsaglia
 *     and Tsang's method, then a noncentral chi-square with 2 degrees);
 *   - beta = 1 steps ln F exactly given the vol path, without absorption.
 * At nu = 0, rho = 0 the step is exact (the absorbed CEV law) at any step
 * size; for nu > 0 a few steps a year match fine-grid log-Euler prices.
 * Path j, step i draws Philox4x32-10 blocks (j, i, b, 0x4D420000), b = 0, 1
 * always and b = 2 .. 8 for further Gamma trials.  A path is absorbed when
 * its Bessel process reaches 0 (no 1e-12 threshold).  EINVAL for an
 * unknown scheme and the checks of sabr_mc_price.
 * ------------------------------------------------------------------------ */
sabr_status sabr_mc_price_scheme(sabr_model model, const double* params,
                                 double fwd, const double* T, const double* K,
                                 const int8_t* is_call, const double* discount,
                                 int64_t n, int64_t n_paths,
                                 double steps_per_year, uint64_t seed,
                                 sabr_mc_scheme scheme, double* price_out,
                                 double* stderr_out, sabr_precision prec,
                                 void* cuda_stream);

/* ------------------------------------------------------------------------
 * sabr_mc_price_noalloc -- the same prices as sabr_mc_price, for callers
 * that cannot let a library allocate device memory: processes whose device
 * memory is handed out entirely by their own fixed-size pool (a cudaMalloc
 * from the library would fail, or take memory the pool counts on), and
 * applications whose rules forbid libraries to allocate.  The paper has no
 * counterpart.
 * Same arguments, layout and semantics as sabr_mc_price, with these
 * differences:
 *  - No cudaMalloc / cudaFree / cudaMallocHost / stream-ordered allocation
 *    is made.  Scratch is one fixed 8 MiB device array in the library image
 *    (every GPU that loads the library holds it until exit); host staging is
 *    static storage.  The option and step tables are copied from that static
 *    storage with an ordinary pageable cudaMemcpyAsync, which the runtime
 *    may perform only after the stream's earlier work.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture on the device.
 *  - EINVAL when a problem needs more than the 8 MiB scratch -- per-block
 *    partial sums take 256 B per block for every 16 options of a maturity
 *    (up to 1216 blocks), and the option and time-step tables must fit in
 *    256 KiB -- use sabr_mc_price then.
 *  - All calls share the scratch and it keeps the last call's contents; each
 *    call overwrites everything it reads.  Calls whose GPU work overlaps (on
 *    different streams, or from threads with no ordering) race on it: order
 *    them on one stream.
 * ------------------------------------------------------------------------ */
sabr_status sabr_mc_price_noalloc(sabr_model model, const double* params,
                                  double fwd, const double* T, const double* K,
                                  const int8_t* is_call, const double* discount,
                                  int64_t n, int64_t n_paths,
                                  double steps_per_year, uint64_t seed,
                                  double* price_out, double* stderr_out,
                                  sabr_precision prec, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Path-sharded Monte Carlo pricing: the Sec. 4 pricer spread over several
 * GPUs (Sec. 5.2 spreads Technique II's Monte Carlo cost over devices).
 * sabr_mc_price runs a grid of total_blocks blocks; block b takes a fixed,
 * interleaved set of the paths and writes FP64 sums of payoff and payoff^2
 * of every option.  A shard runs blocks [block_begin, block_begin +
 * block_count) of that grid on the current device; the caller gathers the
 * shards' partials in block order (any transport) and reduces them on one
 * device.  The result equals sabr_mc_price on a device of the same kind bit
 * for bit.  Every call takes the problem arguments of sabr_mc_price (same
 * meaning, layout, host/device placement and checks).
 *   sabr_mc_shard_layout   total_blocks: the grid sabr_mc_price would use on
 *                          the current device (every shard must use one
 *                          value); doubles_per_block: size of one block's
 *                          partials.  Host only; no device work.
 *   sabr_mc_shard_partials partials_out: device, block_count *
 *                          doubles_per_block doubles, block i of the range
 *                          at offset i * doubles_per_block.
 *   sabr_mc_shard_reduce   partials: device, total_blocks * doubles_per_block
 *                          doubles in block order; price_out / stderr_out as
 *                          sabr_mc_price.
 * Asynchronous on cuda_stream (tables are staged in library-owned device
 * scratch, as sabr_mc_price).  EINVAL for a block range outside
 * [0, total_blocks) and the checks of sabr_mc_price.
 * ------------------------------------------------------------------------ */
sabr_status sabr_mc_shard_layout(sabr_model model, const double* params,
                                 double fwd, const double* T, const double* K,
                                 const int8_t* is_call, const double* discount,
                                 int64_t n, int64_t n_paths,
                                 double steps_per_year, uint64_t seed,
                                 sabr_precision prec, int32_t* total_blocks,
                                 int64_t* doubles_per_block);
sabr_status sabr_mc_shard_partials(sabr_model model, const double* params,
                                   double fwd, const double* T, const double* K,
                                   const int8_t* is_call,
                                   const double* discount, int64_t n,
                                   int64_t n_paths, double steps_per_year,
                                   uint64_t seed, sabr_precision prec,
                                   int32_t total_blocks, int32_t block_begin,
                                   int32_t block_count, double* partials_out,
                                   void* cuda_stream);
sabr_status sabr_mc_shard_reduce(sabr_model model, const double* params,
                                 double fwd, const double* T, const double* K,
                                 const int8_t* is_call, const double* discount,
                                 int64_t n, int64_t n_paths,
                                 double steps_per_year, uint64_t seed,
                                 sabr_precision prec, int32_t total_blocks,
                                 const double* partials, double* price_out,
                                 double* stderr_out, void* cuda_stream);

/* ------------------------------------------------------------------------
 * sabr_mc_cliquet -- Monte Carlo price of a cliquet on the forward, Sec. 6.3
 * eqs. (eq_cliquet) and (cliquet_global), on the paths of sabr_mc_price
 * (same scheme, absorption and Philox streams; the reset dates are inserted
 * into the step grid).  Reset dates d_i = i T / n_resets, i = 1..n_resets;
 * the payoff is
 *     g = sum_{i=2..n_resets} max(min(R_i, cap_local), floor_local),
 *     R_i = F(d_i) / F(d_{i-1}) - 1,
 *     price = discount * E[max(floor_global, min(cap_global, g))].
 * The printed global formula, max(C_g, min(F_g, .)), is the constant C_g
 * whenever F_g <= C_g; the limits are taken in the order that makes
 * floor_global a floor.  A path absorbed before d_{i-1} adds R_i = 0.
 *   params       host, double[10], as sabr_mc_price
 *   T            final reset date (years), > 0; n_resets in [2, 64]
 *   floor_local <= cap_local, floor_global <= cap_global (pass +-1e300 for
 *                no global limits)
 *   price_out    device, double[1]; stderr_out device double[1] or NULL
 * Asynchronous on cuda_stream; device scratch is stream-ordered
 * (cudaMallocAsync / cudaFreeAsync).  EINVAL for bad sizes or limits, more
 * than 8192 time steps, or parameters violating rho(t) in [-1,1],
 * nu(t) > 0 on [0, T].
 * ------------------------------------------------------------------------ */
sabr_status sabr_mc_cliquet(sabr_model model, const double* params, double fwd,
                            double T, int32_t n_resets, double floor_local,
                            double cap_local, double floor_global,
                            double cap_global, double discount,
                            int64_t n_paths, double steps_per_year,
                            uint64_t seed, double* price_out,
                            double* stderr_out, sabr_precision prec,
                            void* cuda_stream);

/* ------------------------------------------------------------------------
 * Calibration problems (Sec. 3 eqs. (error_calibrate_individual_relativo),
 * (error_calibrate_relativo); Sec. 5).  All arrays in a problem are HOST
 * memory and are copied by the call that receives them.
 * ------------------------------------------------------------------------ */
typedef struct {
  sabr_model model;
  sabr_cost cost;
  sabr_precision prec;
  double fwd;              /* forward f > 0 shared by all quotes          */
  int64_t n_quotes;        /* 1 .. 4096                                   */
  const double* T;         /* [n_quotes] maturities (years) > 0           */
  const double* K;         /* [n_quotes] strikes > 0                      */
  const double* market;    /* [n_quotes] market vols (COST_VOL) or prices */
  const int8_t* is_call;   /* [n_quotes] or NULL: MC cost only            */
  const double* discount;  /* [n_quotes] or NULL: MC cost only            */
  int32_t n_chains;        /* SA chains w >= 1                            */
  int64_t mc_paths;        /* MC cost: paths per evaluation               */
  double mc_steps_per_year;/* MC cost: 1/dt                               */
  uint64_t mc_seed;        /* MC cost: Philox key of the common paths     */
  const double* x0;        /* [10] start point, or NULL = box midpoint    */
} sabr_problem;

/* Closed box per coordinate; lo[i] == hi[i] fixes coordinate i.  Open
 * bounds of the paper (alpha > 0, |rho| < 1, nu > 0) are given inset. */
typedef struct {
  double lo[10], hi[10];
} sabr_bounds;

/* Geometric cooling T_k = T0 * factor^k (k = 0 .. n_levels-1); at level k
 * every chain runs chain_len Metropolis steps with moves
 * x' = x + s_k (hi - lo) (2u - 1), s_k = max(step_min, step0 sqrt(T_k/T0)).
 * T0 <= 0 selects T0 = f(x0). */
typedef struct {
  double T0;
  double factor;
  int32_t n_levels;
  int32_t chain_len;
  double step0;
  double step_min;
} sabr_cooling;

typedef struct {
  double params[10];         /* best point seen by any chain            */
  double misfit;             /* its cost as evaluated in the loop        */
  double misfit_fp64;        /* its cost re-evaluated in FP64 on the GPU */
  double restart_params[10]; /* restart point after the last level       */
  double restart_misfit;
  int64_t n_evals;           /* cost evaluations (in-box proposals)      */
  int64_t n_accepts;         /* accepted Metropolis moves                */
  sabr_status status;
} sabr_result;

/* ------------------------------------------------------------------------
 * sabr_calibrate -- Sec. 5, synchronous parallel Simulated Annealing: all
 * chains start from x0; each runs chain_len Metropolis steps per temperature
 * level; the lowest final state restarts every chain at the next level.
 * Proposal uniforms of chain c at (level k, step j) come from Philox4x32-10
 * with key = seed and counter (c, k, j, 0x53410000 + block): the top 23 bits
 * of words 0 .. d-1 move the d parameters, and the acceptance uniform is the
 * 23 bits those words leave unused (low 9, 9 and 5 bits of words 0, 1, 2),
 * so a static model draws one block per proposal.  Out-of-box
 * (and, for DYN_II, infeasible) proposals are rejected without a cost
 * evaluation.  Blocking: returns when *out is filled.  Results depend only on
 * (problem, bounds, cooling, seed) and G, the lanes that share a chain's
 * quotes (the order of the misfit's partial sums), never on the rest of the
 * batch, slots or launch shape.  G is chosen from the problem and the total
 * chain count of its batch (more lanes when the batch is small), so a
 * problem calibrated alone and inside a large batch may differ in the last
 * bits of its sums when its G differs; the environment variable SABR_LANES
 * fixes G for every problem.
 * ------------------------------------------------------------------------ */
sabr_status sabr_calibrate(const sabr_problem* problem,
                           const sabr_bounds* bounds,
                           const sabr_cooling* cooling, uint64_t seed,
                           sabr_result* out, void* cuda_stream);

/* n independent problems calibrated together in one set of launches;
 * problems[i] uses bounds[i], cooling[i], seeds[i], out[i].  Blocking. */
sabr_status sabr_calibrate_batch(int32_t n, const sabr_problem* problems,
                                 const sabr_bounds* bounds,
                                 const sabr_cooling* cooling,
                                 const uint64_t* seeds, sabr_result* out,
                                 void* cuda_stream);

/* A plan keeps a batch resident in device memory and records its whole
 * calibration (all levels) as one CUDA graph, so that it can be replayed.
 * sabr_plan_run is asynchronous; sabr_plan_results waits for the last run
 * and copies the n results to the host.  use_graph = 0 launches the kernels
 * one by one instead. */
typedef struct sabr_plan sabr_plan;
sabr_status sabr_plan_create(int32_t n, const sabr_problem* problems,
                             const sabr_bounds* bounds,
                             const sabr_cooling* cooling,
                             const uint64_t* seeds, int32_t use_graph,
                             void* cuda_stream, sabr_plan** out);
sabr_status sabr_plan_run(sabr_plan* plan, void* cuda_stream);
sabr_status sabr_plan_results(sabr_plan* plan, sabr_result* out);
/* Kernel launches one run of the plan enqueues, and the average time of one
 * temperature level (all problems of the plan) over the last run, from
 * events around the level work (ms; 0 if not timed).  The levels of a
 * launch group (problems of one model and precision) run in one persistent
 * launch that takes (problem, level, block of chains) units from a
 * device-resident ready queue when the group holds several problems with
 * more units per level than the GPU holds resident blocks, or one problem
 * two of whose levels fit in them; problems then move from level to level
 * independently, and SABR_ETIMEOUT in a result means a wait of that launch
 * gave up and its levels did not all run.  Other groups launch one kernel
 * per level.  The launch shape never changes the results. */
sabr_status sabr_plan_stats(sabr_plan* plan, int64_t* launches_per_run,
                            double* level_kernel_ms);
void sabr_plan_destroy(sabr_plan* plan);

/* ------------------------------------------------------------------------
 * Chain-sharded calibration: Sec. 5.1's multi-GPU Technique I.  Each GPU
 * runs a share of the chains; after every temperature level the host takes
 * the minimum of the shares' lowest final states as the common restart
 * point.  A shard holds chains [chain_begin, chain_begin + chain_count) of
 * problem->n_chains (the problem's total) on the current device; the caller
 * runs level 0 .. n_levels-1 in order on every shard, exchanges the shards'
 * minima (any transport: a collective, host memory), takes the
 * lexicographic minimum in (f, chain) and gives it to every shard with
 * sabr_shard_restart before the next level.  After the last level each
 * shard's sabr_shard_result gives its best-ever point; the overall result is
 * the shard result of lowest (misfit, best_chain), with n_evals and
 * n_accepts summed.  Done this way the result equals sabr_calibrate on the
 * whole problem bit for bit: chains draw their proposals from Philox
 * counters keyed by their global index, and lanes per chain are chosen from
 * the total chain count.  Implied-vol cost (Technique I) only.
 *   sabr_shard_create   problem, bounds, cooling, seed: as sabr_calibrate
 *                       (host arrays, copied).  Computes f(x0) and T0;
 *                       blocking.  EINVAL for a chain range outside
 *                       [0, n_chains) or an MC-cost problem.
 *   sabr_shard_level    runs `level` (which must follow the previous one)
 *                       from the current restart point; *local_min = the
 *                       shard's lowest final state (lowest global chain on
 *                       a tie).  Blocking.
 *   sabr_shard_restart  restart point (x, f) of the next level.  Blocking.
 *   sabr_shard_result   after the last level: the shard's result (best
 *                       point, its FP64 re-score, counters) and the global
 *                       chain of its best point (-1 with no levels).
 *                       Blocking.
 * ------------------------------------------------------------------------ */
typedef struct {
  double f;       /* cost of the state                                */
  int64_t chain;  /* global chain index                               */
  double x[10];   /* parameters (layout of params above)              */
} sabr_chain_point;
typedef struct sabr_shard sabr_shard;
sabr_status sabr_shard_create(const sabr_problem* problem,
                              const sabr_bounds* bounds,
                              const sabr_cooling* cooling, uint64_t seed,
                              int32_t chain_begin, int32_t chain_count,
                              void* cuda_stream, sabr_shard** out);
sabr_status sabr_shard_level(sabr_shard* shard, int32_t level,
                             sabr_chain_point* local_min, void* cuda_stream);
sabr_status sabr_shard_restart(sabr_shard* shard,
                               const sabr_chain_point* restart,
                               void* cuda_stream);
sabr_status sabr_shard_result(sabr_shard* shard, sabr_result* out,
                              int64_t* best_chain, void* cuda_stream);
void sabr_shard_destroy(sabr_shard* shard);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of calibration requests (Sec. 5 engines).
 * A server owns a worker thread, a device-memory pool and a stream.  Each
 * worker step admits queued requests while the pool and max_active allow
 * (admission by device memory), then advances every resident formula-cost
 * request by one temperature level in one set of persistent launches
 * (replayed from a captured CUDA graph when use_graph != 0) and every
 * resident MC-cost request by one proposal wave on a second stream, so that
 * requests that arrive while others run join them on the device.  Finished
 * requests release their memory at once.  A request's result does not depend
 * on what else is resident: it is the result of sabr_calibrate on that
 * request alone (G chosen from the request alone).
 * ------------------------------------------------------------------------ */
typedef struct {
  int64_t device_bytes; /* pool for resident requests (>= 1 MiB)          */
  int32_t max_queue;    /* waiting requests; submit returns EBUSY beyond   */
  int32_t max_active;   /* resident requests, 1 .. 4096                    */
  int32_t max_quotes;   /* largest formula request accepted, <= 4096       */
  int32_t use_graph;    /* replay each step from a captured CUDA graph     */
} sabr_server_config;

typedef struct {
  int64_t submitted, admitted, completed, cancelled, steps, kernel_launches;
  int32_t queued, active;
  int64_t pool_bytes_in_use;
} sabr_server_stats;

typedef struct sabr_server sabr_server;

/* Creates the server on the current device (pool allocated here). */
sabr_status sabr_server_create(const sabr_server_config* config, sabr_server** out);
/* Deep-copies the host arrays of *problem; the caller may free them after
 * return.  EBUSY if the queue is full, EINVAL for a malformed problem or one
 * larger than the pool or max_quotes.  *ticket identifies the request. */
sabr_status sabr_server_submit(sabr_server* server, const sabr_problem* problem,
                               const sabr_bounds* bounds,
                               const sabr_cooling* cooling, uint64_t seed,
                               uint64_t* ticket);
/* EAGAIN while queued or running; SABR_OK with *out filled when done;
 * ECANCELLED, ENOTFOUND.  A finished ticket is released by the first poll or
 * wait that returns it. */
sabr_status sabr_server_poll(sabr_server* server, uint64_t ticket, sabr_result* out);
/* Blocks up to timeout_ms (< 0: no limit) for the request; ETIMEOUT when the
 * time runs out first. */
sabr_status sabr_server_wait(sabr_server* server, uint64_t ticket, int64_t timeout_ms,
                             sabr_result* out);
/* Cancels a queued request (ECANCELLED for later polls); a resident one is
 * cancelled at the next step boundary.  ENOTFOUND for unknown tickets. */
sabr_status sabr_server_cancel(sabr_server* server, uint64_t ticket);
sabr_status sabr_server_get_stats(sabr_server* server, sabr_server_stats* out);
/* Stops the worker after the current step, drops what is left, frees all. */
void sabr_server_destroy(sabr_server* server);

/* Measurement utility (not part of the paper's method): throughput of the
 * arithmetic pipes on the current device, in operations per SM clock, from
 * loops of independent operations timed with the SM cycle counter:
 *   rates[0] FP32 FMA   [1] MUFU ex2   [2] MUFU lg2 (with one FP32 add)
 *   rates[3] MUFU rsqrt [4] MUFU rcp   [5] MUFU sin  [6] INT32 multiply-add
 *   rates[7] FP64 FMA
 * n_rates >= 8.  Blocking; allocates and frees a small device buffer.  The
 * ALU roofline of the kernels is stated from these rates. */
sabr_status sabr_probe_pipe_rates(double* rates, int32_t n_rates, void* cuda_stream);

/* Human-readable message of the last failure on this thread. */
const char* sabr_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SABR_H */
