/*
 * gvegas.h -- C ABI of the GB300 (sm_103a) VEGAS / BASES library.
 *
 * The library runs the per-iteration loop of "Monte Carlo integration on
 * GPU" (Kanzaki, arXiv 1010.2107), Sec. 2.1 steps 2-6, entirely on one GPU:
 *   step 2  point generation (counter-based Philox4x32-10 in registers,
 *           integer-exact grid bins, the adaptive-grid map x = g(y), J),
 *   step 3  the integrand (a fixed registry: Genz families, two-peak
 *           Gaussian, massless RAMBO phase space with a Breit-Wigner),
 *   step 4  accumulation of w = f J into per-bin sums of w and w^2 on every
 *           axis, per-hypercube sums (BASES), and the iteration estimate,
 *   step 5  grid optimisation (smoothing, log-compression, rebinning) in FP64,
 *   step 6  inverse-variance combination of iterations, chi^2, ACC test.
 * The paper moved only steps 2-3 to the GPU and copied NCALL function values
 * back every iteration (Sec. 2.2); here nothing but the small result
 * structure crosses to the host, and only when asked.
 *
 * Conventions
 *  - Every entry point returns a vegas_status; no exception or abort crosses
 *    the ABI.  On failure vegas_last_error(ctx) (or vegas_last_error(NULL)
 *    for failures before a context exists) gives a message.
 *  - The context owns every device buffer it uses (cudaMalloc at creation,
 *    cudaFree at vegas_destroy).  All pointers passed in or out are HOST
 *    pointers owned by the caller, unless an argument says "device".
 *  - Work is ordered on the context's CUDA stream (config.stream, or a
 *    stream the context creates when that is NULL).  Calls that fill host
 *    outputs synchronise that stream before returning; the others do not.
 *  - The integration domain is the unit hypercube [0,1)^ndim.
 *  - A context is not thread-safe: one host thread at a time.
 *
 * Random numbers: the j-th random word of sample s (0 <= s < NCALL) in
 * iteration `it` of instance `inst` is output word j mod 4 of
 * Philox4x32-10(counter = (s, floor(j/4), it, inst), key = (seed mod 2^32,
 * seed >> 32)).  `it` counts every iteration the context has run, from 0.
 * With ybits = 24 axis a uses word a (y_a = (word >> 8) / 2^24); with
 * ybits = 53 it uses words 2a and 2a+1 (27 + 26 bits).  Grid bins are
 * computed from those bits in integer arithmetic, so they do not depend on
 * the floating-point precision of the rest of the path.
 */
#ifndef GVEGAS_H
#define GVEGAS_H

#ifndef __CUDACC_RTC__ /* the run-time compiled kernels see no C library */
#include <stddef.h>
#include <stdint.h>
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define GVEGAS_MAXDIM 32      /* largest ndim a context accepts            */
#define GVEGAS_MAXBINS 256    /* largest nbins (grid bins per axis)         */
#define GVEGAS_MAXHIST 4096   /* iterations kept in one combination window  */
#define GVEGAS_MAXUSERPARAMS 120 /* parameters of a run-time compiled integrand */

typedef struct vegas_ctx vegas_ctx;

typedef enum {
  VEGAS_OK = 0,
  VEGAS_EINVAL = 1,     /* an argument is out of range                      */
  VEGAS_ENOMEM = 2,     /* a device or pinned-host allocation failed        */
  VEGAS_ECUDA = 3,      /* a CUDA call failed (message has the CUDA error)  */
  VEGAS_ETIMEOUT = 4,   /* a bounded device-side wait gave up               */
  VEGAS_ENONFINITE = 5, /* reserved: non-finite weights are counted, not fatal */
  VEGAS_ESTATE = 6      /* call not valid for this context (e.g. batch ctx) */
} vegas_status;

/* Integrand registry (step 3).  Parameter layouts, with d = ndim:
 *  VG_GENZ_GAUSSIAN      a[d], u[d]:  f = exp(-sum_i a_i^2 (x_i - u_i)^2)
 *  VG_GENZ_PRODUCT_PEAK  a[d], u[d]:  f = prod_i (a_i^-2 + (x_i - u_i)^2)^-1
 *  VG_GENZ_CORNER_PEAK   a[d]:        f = (1 + sum_i a_i x_i)^-(d+1)
 *  VG_GENZ_OSCILLATORY   a[d], u1:    f = cos(2 pi u1 + sum_i a_i x_i)
 *  VG_DOUBLE_GAUSSIAN    c1, c2, w:   f = 1/2 sum_{c in {c1,c2}}
 *                                          (w sqrt pi)^-d exp(-sum_i ((x_i-c)/w)^2)
 *  VG_GENZ_CONTINUOUS    a[d], u[d]:  f = exp(-sum_i a_i |x_i - u_i|)
 *  VG_GENZ_DISCONTINUOUS a[d], u[min(d,2)]:  f = exp(sum_i a_i x_i) where
 *                                          x_1 <= u_1 and x_2 <= u_2, else 0
 *  VG_RAMBO_BW           10 slots (VG_RB_*), d = 4 n:  n massless partons
 *      from RAMBO (4 numbers each), f = V_n * cut(p) * BW(s_12) *
 *      prod_{i} 1/s_{i,i+1 mod n}, with BW(s) = M G / ((s-M^2)^2 + M^2 G^2),
 *      V_n = (pi/2)^(n-1) s^(n-2) / ((n-1)!(n-2)!), cut = hard pT > ptmin
 *      or prod_i sigmoid((pT_i - T)/wc), and Delta R_ij > drmin for all
 *      pairs.  Units GeV.  (Stand-in for the W + n-gluon processes of
 *      Sec. 4, eq. 1, with the jet cuts of eqs. 2-3.)
 *  VG_W_MUNU             15 slots (VG_W_*), d = 5:  u dbar -> W+ -> mu+ nu_mu
 *      in pp collisions (Sec. 4, the process with n = 0 gluons, and the mu+
 *      cuts |eta| < ETAMAX, pT > PTMIN), f in pb.  y1 -> shat = M^2 +
 *      M Gamma tan(rho), rho uniform between the images of [SMIN, S];
 *      y2 -> W rapidity uniform in [ln(tau)/2, -ln(tau)/2]; y3 -> cos theta
 *      of the mu+ against the u (which comes from the proton along +z) in
 *      the partonic frame; y4 -> its azimuth; y5 -> one of 16 helicity
 *      combinations, weight 16 (Sec. 4: one variable sums the helicities).
 *      |M|^2 = g^4 |V_ud|^2 uhat^2 / ((shat - M^2)^2 + M^2 Gamma^2) for
 *      u(-) dbar(+) -> nu(-) mu+(+), zero for the others, averaged over
 *      spins and colours (1/12); g^2 = 8 M^2 G_F / sqrt 2.  Parton densities
 *      A x^a (1 - x)^b per flavour (a stand-in for a PDF table). */
typedef enum {
  VG_GENZ_GAUSSIAN = 0,
  VG_GENZ_PRODUCT_PEAK = 1,
  VG_GENZ_CORNER_PEAK = 2,
  VG_GENZ_OSCILLATORY = 3,
  VG_DOUBLE_GAUSSIAN = 4,
  VG_RAMBO_BW = 5,
  VG_GENZ_CONTINUOUS = 6,
  VG_GENZ_DISCONTINUOUS = 7,
  VG_W_MUNU = 8,
  VG_USER = 64          /* run-time compiled (vegas_create_user); not valid
                           for vegas_create or the batched and no-alloc calls */
} vegas_integrand_kind;

enum {
  VG_W_SQRTS = 0, VG_W_M = 1, VG_W_GAMMA = 2, VG_W_GF = 3, VG_W_VUD = 4,
  VG_W_PTMIN = 5, VG_W_ETAMAX = 6,
  VG_W_SMIN = 7,   /* lower end of the shat range, GeV^2                  */
  VG_W_CUTS = 8,   /* 1: apply the mu+ cuts, 0: none                      */
  VG_W_AU = 9, VG_W_ALU = 10, VG_W_BU = 11,   /* u density A, a, b         */
  VG_W_AD = 12, VG_W_ALD = 13, VG_W_BD = 14,  /* dbar density A, a, b      */
  VG_W_NPARAMS = 15
};

enum {
  VG_RB_N = 0, VG_RB_SQRTS = 1, VG_RB_M = 2, VG_RB_GAMMA = 3,
  VG_RB_PTMIN = 4, VG_RB_DRMIN = 5,
  VG_RB_CUT = 6,   /* 0 hard pT cut, 1 sigmoid pT cut, 2 no cuts          */
  VG_RB_T = 7, VG_RB_WC = 8,
  VG_RB_OBS = 9,   /* 0 full integrand, 1 f = 1, 2 f = s12, 3 f = BW(s12) */
  VG_RB_NPARAMS = 10
};

/* Arithmetic of the hot path.  Grid refinement and the combination of
 * iterations are FP64 in every form.
 *  VG_FP64          map, integrand and sums in FP64.
 *  VG_FP32_ACC64    map and integrand in FP32; every weight is added to
 *                   FP64 sums (per-bin histograms, totals, cube sums).
 *  VG_FP32_ACCCOMP  map and integrand in FP32; per-thread and per-warp sums
 *                   in compensated FP32 (hi, lo) pairs, per-bin histograms
 *                   in FP32 shared memory flushed into FP64 every few
 *                   thousand points; FP64 from the CTA level up. */
typedef enum {
  VG_FP64 = 0,
  VG_FP32_ACC64 = 1,
  VG_FP32_ACCCOMP = 2
} vegas_precision;

typedef struct {
  int kind;              /* vegas_integrand_kind                          */
  int ndim;              /* must equal vegas_config.ndim                  */
  const double* params;  /* host array, copied at creation                */
  int nparams;
} vegas_integrand;

/* Sec. 5.1 parameters (NCALL, ITMX, ACC) plus the grid and the sampler. */
typedef struct {
  int ndim;              /* 1..GVEGAS_MAXDIM                               */
  int nbins;             /* grid bins per axis N, 2..GVEGAS_MAXBINS (50)   */
  int64_t ncall;         /* points per iteration NCALL, 2..2^32            */
  int itmx;              /* default iteration count for bases/iterate (>0) */
  double acc;            /* stop when sigma/|I| < acc (<= 0: never)        */
  double alpha;          /* grid damping exponent (1.5)                    */
  int nstrat;            /* hypercube divisions per axis g; 0/1 = none.
                            NCALL must be a multiple of g^ndim with at
                            least 2 points per cube.                       */
  uint64_t seed;         /* Philox key                                     */
  uint32_t instance;     /* Philox counter word 3                          */
  int precision;         /* vegas_precision                                */
  int ybits;             /* 24 or 53; 0 = 53 for VG_FP64, 24 otherwise     */
  void* stream;          /* cudaStream_t to order work on, or NULL         */
} vegas_config;

typedef struct {
  double I;              /* combined estimate of the current window       */
  double sigma;          /* its standard error                             */
  double chi2_dof;       /* chi^2 per degree of freedom (0 for 1 iteration) */
  int iters_done;        /* iterations in the current window              */
  int stopped;           /* 1 if the ACC test ended the last call early    */
  int64_t nonfinite;     /* non-finite weights seen (counted as 0)         */
  int64_t samples;       /* points evaluated in the current window        */
} vegas_result;

#ifndef __CUDACC_RTC__ /* the run-time compiled kernels take the types only */

/* Create a context: copies config and integrand, allocates device buffers,
 * sets the uniform grid e_a[k] = k/N (step 1).  Errors: VEGAS_EINVAL for
 * out-of-range sizes or parameter counts, VEGAS_ENOMEM, VEGAS_ECUDA. */
vegas_status vegas_create(const vegas_config* config,
                          const vegas_integrand* integrand, vegas_ctx** out);

/* End of a run (Sec. 2.1: step 6 ends the loop; the sample main program of
 * Appendix A runs one integration and exits): waits for the context stream,
 * then frees every device and pinned buffer and cached graph of the
 * context.  NULL is ignored. */
void vegas_destroy(vegas_ctx* ctx);

/* Steps 2-6, n_iter times (Sec. 2.1, step 6): each iteration evaluates NCALL
 * points, reduces the per-bin sums, refines the grid if refine != 0, and
 * adds its estimate to the combination window; stops early (device-side)
 * when sigma/|I| < config.acc.  out (nullable) receives the combined result
 * and forces a stream synchronisation. */
vegas_status vegas_iterate(vegas_ctx* ctx, int n_iter, int refine,
                           vegas_result* out);

/* Start a new combination window (the grid and the iteration counter are
 * kept).  Stream-ordered, no synchronisation. */
vegas_status vegas_reset_results(vegas_ctx* ctx);

/* Put back the uniform grid e_a[k] = k/N of step 1 (device-side,
 * stream-ordered, no synchronisation). */
vegas_status vegas_reset_grid(vegas_ctx* ctx);

/* BASES (Sec. 2.1 and Sec. 5.1): a grid-optimisation phase of up to itmx1
 * refining iterations (stopping at acc1), then an integration phase of up
 * to itmx2 iterations on the frozen grid (stopping at acc2).  Both phases
 * run as one CUDA graph with the ACC tests on the device.  out receives the
 * integration phase alone, phase1 the first phase; when both are NULL the
 * call returns without synchronising (results stay readable through
 * vegas_iterate(ctx, 0, 0, &r) or vegas_get_history). */
vegas_status bases_integrate(vegas_ctx* ctx, int itmx1, double acc1,
                             int itmx2, double acc2, vegas_result* out,
                             vegas_result* phase1);

/* Copy the grid edges [ndim][nbins+1] and, if bin_sums is not NULL, the
 * per-bin sums [2][ndim][nbins] (sum w, sum w^2) of the last pass that
 * formed them: a refining iteration or vegas_eval.  Passes that leave the
 * grid unchanged (vegas_iterate with refine = 0, the integration phase of
 * bases_integrate) skip them, since only the grid optimisation (step 5)
 * reads them; their estimates, cube sums and maxima are complete. */
vegas_status vegas_get_grid(vegas_ctx* ctx, double* edges, double* bin_sums);

/* Replace the grid (step 5's output, Sec. 2.1).  BASES keeps the grid of its
 * optimisation phase for the integration phase and for SPRING (Sec. 2.1);
 * this puts a saved grid back, which with vegas_set_iteration resumes a run
 * exactly where vegas_get_grid / vegas_get_iteration left it.  edges is a
 * host array [ndim][nbins+1]; every axis must start at 0, end at 1 and
 * increase strictly, else VEGAS_EINVAL (the grid is then unchanged).
 * Stream-ordered (the tables are rebuilt on the device). */
vegas_status vegas_set_grid(vegas_ctx* ctx, const double* edges);

/* The iteration history of the current window: hist[i] = (I_i, sigma_i^2),
 * up to max_iters rows; *n_out receives the number of rows. */
vegas_status vegas_get_history(vegas_ctx* ctx, double* hist, int max_iters,
                               int* n_out);

/* Per-hypercube sums of the last stratified iteration, [g^ndim][2]
 * (sum w, sum w^2); VEGAS_ESTATE without stratification. */
vegas_status vegas_get_cube_sums(vegas_ctx* ctx, double* sums);

/* The Philox iteration counter (iterations run so far; synchronises the
 * stream) and a setter for exact resume together with vegas_set_grid
 * (stream-ordered on the device, no synchronisation; the next iteration
 * draws iteration `it`'s points). */
vegas_status vegas_get_iteration(vegas_ctx* ctx, uint32_t* it);
vegas_status vegas_set_iteration(vegas_ctx* ctx, uint32_t it);

/* Create a context for an integrand given as CUDA C++ source, compiled at
 * run time (NVRTC, sm_103a) into the same sampling, dump and SPRING kernels
 * the built-in integrands use (step 3 of Sec. 2.1 with the user's f; the
 * paper's users likewise write their integrand as device code).  `source`
 * must define, at namespace scope,
 *
 *   template <typename T>
 *   __device__ T vegas_user_f(const T* x, int d, const T* p);
 *
 * returning f(x) for the point x[0..d) in (0,1)^d, with p[0..nparams) the
 * parameters converted to T.  T is double for VG_FP64 and float for the two
 * FP32 forms.  The source sees the CUDA device built-ins and this library's
 * device helpers (namespace gv), no C or C++ library headers.  The kernels
 * are compiled with ndim as their exact dimension; a compiled program is
 * cached, keyed by (source, precision, ybits, ndim, kernel shape), for the
 * life of the process.  No adjoint kernel (vegas_grad) is built.  Errors:
 * VEGAS_EINVAL with the compiler's log in vegas_last_error(NULL) when the
 * source does not compile, or for bad sizes; VEGAS_ECUDA when the run-time
 * compiler (libnvrtc) cannot be loaded or the module does not load. */
vegas_status vegas_create_user(const vegas_config* config, const char* source,
                               const double* params, int nparams,
                               vegas_ctx** out);

/* Compile `source` as vegas_create_user would for `config`, without
 * loading it (needs no device); the program is cached for a later
 * vegas_create_user.  Errors as there. */
vegas_status vegas_user_compile(const vegas_config* config, const char* source);

/* Replace the integrand parameters (step 3 of Sec. 2.1; the paper compiles
 * its integrand's constants into the user's gVegasFunc.cu, Appendix A, so a
 * change means a rebuild).  Here they are device data read at run time: the
 * same count and layout as at creation (host array), checked as there
 * (VEGAS_EINVAL, context unchanged); captured graphs stay valid. */
vegas_status vegas_set_params(vegas_ctx* ctx, const double* params,
                              int nparams);

/* One evaluation pass at Philox iteration `it` on the current grid without
 * refinement and without touching the window or the counter: the
 * estimate I and its variance.  Two calls with the same `it` use common
 * random numbers. */
vegas_status vegas_eval(vegas_ctx* ctx, uint32_t it, double* I, double* var);

/* No counterpart in the paper, which computes integrals only (Sec. 5.2):
 * the derivative of the iteration estimate of Sec. 2.1 step 4 with respect
 * to integrand parameters theta, for fits of a resonance mass, width or cut
 * threshold by gradient.  On the frozen grid with the random numbers of
 * iteration `it` (common random numbers):
 *   dI/dtheta = (1/NCALL) sum_s J_s df/dtheta(x_s).
 * theta = (M, Gamma, T) for VG_RAMBO_BW, (c1, c2, w) for
 * VG_DOUBLE_GAUSSIAN, (u[d], a[d]) for VG_GENZ_GAUSSIAN; VEGAS_EINVAL for
 * the other kinds.  grad has vegas_ntheta(ctx) entries; I (nullable) gets
 * the estimate itself. */
vegas_status vegas_grad(vegas_ctx* ctx, uint32_t it, double* grad, double* I);
int vegas_ntheta(const vegas_ctx* ctx);

/* Step 2-3 for a list of sample indices at iteration `it` on the current
 * grid (host arrays of n entries; any output may be NULL): words [n][W]
 * (W = ndim or 2 ndim), bins [n][ndim], x [n][ndim], jac [n], f [n].
 * x, jac and f are in the context's precision, widened to double. */
vegas_status vegas_sample_dump(vegas_ctx* ctx, uint32_t it, const uint64_t* s,
                               int64_t n, uint32_t* words, int32_t* bins,
                               double* x, double* jac, double* f);

/* SPRING (Sec. 2.1: the results of the BASES integration phase drive event
 * generation; the steps follow Kawabata's SPRING, with integer cube choice).
 * Every bases_integrate records, during its integration phase, the largest
 * weight M_c = max(0, f J) seen in each hypercube c.
 * vegas_get_cube_max copies those maxima (in the integrand's units, like
 * vegas_get_cube_sums; G = nstrat^ndim values, 1 without stratification).
 * spring_generate runs trials t = trial0 .. trial0 + n_trials - 1 on the
 * frozen grid: each picks cube c with probability q_c / Q, q_c =
 * ceil(M_c 2^24 / max M) (Q the sum), places a point in it as the sampling
 * step does, and keeps it with probability w / (q_c max M 2^-24); a weight
 * above that bound is kept and counted in *n_overflow, a non-positive one
 * dropped and counted in *n_nonpos.  The Philox words of trial t come from
 * counter (t, word group, 0xFFFFFFFF, instance).  Kept points go to
 * x_out[k][ndim] and trial_out[k] (host arrays with room for n_trials rows;
 * either may be NULL to leave the events on the device) in trial order;
 * *n_events = k.  VEGAS_ESTATE before any bases_integrate or when every
 * maximum is zero; EINVAL when trial0 + n_trials exceeds 2^32. */
vegas_status vegas_get_cube_max(vegas_ctx* ctx, double* cmax);
/* Measurement: mean milliseconds of the SPRING trial kernel alone (CUDA
 * events on the context stream around it) over `reps` spring_generate calls
 * of n_trials trials from trial 0, events left on the device. */
vegas_status spring_profile(vegas_ctx* ctx, uint32_t n_trials, int reps, double* ms);
vegas_status spring_generate(vegas_ctx* ctx, uint64_t trial0, uint32_t n_trials,
                             double* x_out, uint64_t* trial_out, uint32_t* n_events,
                             uint32_t* n_overflow, uint32_t* n_nonpos);

/* Launch shape of the sampling kernel: threads per CTA (multiple of 32,
 * from 64 up to the kernel's limit: 512 for the specialised kernels, 256
 * otherwise) and CTAs per SM (0 = as many as fit).  Used by the
 * autotuner; takes effect on the next iteration.  EINVAL outside those
 * ranges. */
vegas_status vegas_set_launch(vegas_ctx* ctx, int threads, int ctas_per_sm);
vegas_status vegas_get_launch(vegas_ctx* ctx, int* threads, int* ctas,
                              int* ctas_per_sm);

/* Histogram tile of the sampling kernel (no counterpart in the paper, whose
 * host code sums the bins): each thread evaluates `points_per_thread`
 * points (1..8; 0 = automatic) between two gathers of the CTA's
 * (axis, bin) buckets; kernels that evaluate two points per thread at a
 * time round it up to even.  Changes only speed and the summation order
 * inside a CTA, never which points are drawn.  get_tile returns the points per
 * thread and the bucket capacity per (axis, bin) in use.  EINVAL outside
 * the range or when the tile does not fit in shared memory (the previous
 * shape then stays). */
vegas_status vegas_set_tile(vegas_ctx* ctx, int points_per_thread);
vegas_status vegas_get_tile(vegas_ctx* ctx, int* points_per_thread, int* cap);

/* Launch-shape autotuner (the paper tunes nBlockSize by hand, Appendix A):
 * times evaluation passes (as vegas_profile_pass: no refinement, window
 * untouched) for threads per CTA in {128, 256, 384, 512} and histogram
 * tiles in {automatic, 1, 2, 4} points per thread, each with the largest
 * and with the smallest bucket capacity that reaches the tile's best
 * occupancy, skipping shapes the kernel cannot take; the three fastest are
 * timed again in three
 * interleaved rounds of five passes, and the one with the best round is
 * kept.  Returns its threads, points
 * per thread and the pass time in ms (any output may be NULL).  The
 * specialised kernels (d = the compiled bound, 24-bit words, power-of-two
 * strata) accept up to 512 threads, the general ones 256.  Synchronises the
 * stream. */
vegas_status vegas_autotune(vegas_ctx* ctx, int* threads, int* points_per_thread, double* ms);

/* Measurement (the paper times whole programs, Sec. 3.3; this times each
 * kernel): runs n_pass evaluation passes at the current iteration index
 * (no refinement, window untouched) with CUDA events recorded on the
 * context stream around each kernel, and returns the mean milliseconds per
 * launch of ms[0] the sampling kernel, ms[1] the finishing kernel (the
 * fixed-order reduction of the per-CTA partials, then refinement and
 * combination when a pass asks for them), ms[2] the two together.
 * Synchronises the stream. */
vegas_status vegas_profile_pass(vegas_ctx* ctx, int n_pass, double* ms);

/* The same for the passes that leave the grid unchanged (vegas_iterate with
 * refine = 0, the integration phase of bases_integrate): no per-bin
 * histogram, their own launch shape. */
vegas_status vegas_profile_frozen_pass(vegas_ctx* ctx, int n_pass, double* ms);

/* ------------------------------------------------------------------------
 * Batched integration: n independent VEGAS integrations iterated together,
 * each iteration one persistent kernel over all instances plus one
 * finalisation kernel (the loop of Sec. 2.1, steps 2-6, for every
 * instance), a whole call captured in one CUDA graph.
 *
 * Instances share precision (VG_FP64 or VG_FP32_ACCCOMP), ybits, nbins and
 * seed; each has its own integrand (any kind but VG_RAMBO_BW and VG_W_MUNU), ndim
 * (1..16), ncall (< 2^32), alpha and `instance` id (Philox counter word 3,
 * so instance i draws the points a standalone context with the same id
 * draws).  No stratification and no ACC stop.  The stream of cfgs[0] (or a
 * stream the batch creates) orders all work.  Shared memory: the FP32 form
 * with 24-bit words runs one kernel per dimension and takes every nbins up
 * to GVEGAS_MAXBINS; the other forms run one kernel sized for the widest
 * instance, so nbins times the widest ndim is limited to about 2750
 * (256 bins up to 10 axes, 172 bins at 16 axes), VEGAS_EINVAL beyond.
 * ------------------------------------------------------------------------ */
typedef struct vegas_batch vegas_batch;

/* The paper runs one integration per program and sizes one kernel call per
 * iteration (Sec. 5.3: NCALL points in one call, 256 threads per block);
 * the batch extends that call over many independent integrations of
 * different dimension and NCALL.  Copies the n configs and integrands
 * (host arrays), allocates the batch's device buffers and sets uniform
 * grids (step 1 of Sec. 2.1 per instance).  VEGAS_EINVAL for a rule above
 * broken, VEGAS_ENOMEM, VEGAS_ECUDA; vegas_batch_last_error(NULL) says
 * which. */
vegas_status vegas_batch_create(int n, const vegas_config* cfgs, const vegas_integrand* integrands,
                                vegas_batch** out);
void vegas_batch_destroy(vegas_batch* batch);

/* Steps 2-6 of Sec. 2.1 for every instance, n_iter times (0..64): per
 * iteration the persistent sampling kernels (the FP32 form with 24-bit
 * words: one per dimension present, run concurrently; otherwise one) and
 * one finalisation kernel, the whole call one CUDA graph; refining after each iteration when
 * refine != 0.  out (nullable, host array of n) receives one result per
 * instance (combined over the instance's window) and forces a
 * synchronisation.  No ACC stop (every instance runs n_iter). */
vegas_status vegas_batch_iterate(vegas_batch* batch, int n_iter, int refine, vegas_result* out);

/* Uniform grids, empty windows and iteration counters back to zero. */
vegas_status vegas_batch_reset(vegas_batch* batch);

/* Replace the integrand parameters of instances first .. first+count-1
 * (Sec. 2.1 step 3, the integrand each instance's loop samples; the
 * batched form of vegas_set_params).  params: host array; instance
 * first + j reads its parameter block (the layout and count of
 * vegas_create) from params + j * stride, so stride must be at least the
 * largest count in the range.  The derived constants are formed on the
 * host and uploaded in one stream-ordered copy from pinned memory; grids,
 * histories and captured graphs are kept (the kernels read the constants
 * at run time).  VEGAS_EINVAL, with nothing changed, for a range outside
 * the batch, a short stride or parameters the instance's kind rejects. */
vegas_status vegas_batch_set_params(vegas_batch* batch, int first, int count, const double* params, int stride);

/* Grid edges [ndim_i][nbins+1] and (nullable) per-bin sums of the last
 * iteration [2][ndim_i][nbins] of instance i; its history (I_j, sigma_j^2). */
vegas_status vegas_batch_get_grid(vegas_batch* batch, int i, double* edges, double* bin_sums);
vegas_status vegas_batch_get_history(vegas_batch* batch, int i, double* hist, int max_iters, int* n_out);

/* Launch shape: threads per CTA (64..256, multiple of 32) and rounds per
 * work item (an item is threads * rounds points of one instance). */
vegas_status vegas_batch_set_launch(vegas_batch* batch, int threads, int rounds);
vegas_status vegas_batch_get_launch(vegas_batch* batch, int* threads, int* rounds, int* ctas, int* items);

/* Histogram tile of the batched sampling kernels (as vegas_set_tile; no
 * counterpart in the paper): the points each thread evaluates between two
 * gathers of the CTA's buckets, 0 = automatic.  The FP32 form with 24-bit
 * words runs one kernel per dimension (d = 1..16), where this is 1 or 2,
 * the points a thread keeps in flight; the other forms take 0..4.  EINVAL
 * outside the range or when the tile does not fit (the previous tile then
 * stays).  get_tile returns the points per thread and the bucket capacity
 * (of the widest dimension's kernel for the per-dimension kernels).
 * Changes only speed and the summation order inside a CTA. */
vegas_status vegas_batch_set_tile(vegas_batch* batch, int points_per_thread);
vegas_status vegas_batch_get_tile(vegas_batch* batch, int* points_per_thread, int* cap);

/* Autotuner: times every (threads, rounds) candidate, each with the largest
 * and the smallest bucket capacity that reach its occupancy, on the batch's
 * own workload (an evaluation pass, nothing recorded), times the three fastest
 * again in three interleaved rounds and keeps the one with the best round;
 * returns it and its sampling-kernel milliseconds. */
vegas_status vegas_batch_autotune(vegas_batch* batch, int* threads, int* rounds, double* ms);

/* Mean milliseconds of the sampling kernel (ms[0]) and the finalisation
 * (ms[1]) over n_pass evaluation passes (nothing recorded, no refinement). */
vegas_status vegas_batch_profile(vegas_batch* batch, int n_pass, double* ms);

const char* vegas_batch_last_error(const vegas_batch* batch);

/* Measured issue rate of one instruction class on the current device, in
 * thread-operations per second summed over all SMs (no counterpart in the
 * paper; these are the denominators of the ALU roofline).  op: 0 FP32 FMA,
 * 1 32x32->64 integer multiply pair (mul.hi + mul.lo, counted as one),
 * 2 FP64 FMA, 3 exp2 on the special-function unit, 4 u32->f32 conversion,
 * 5 Philox4x32-10 blocks, 6 shared-memory float atomicAdd into one
 * 50-bin histogram per CTA, 7 the same with one histogram per warp,
 * 8 32-bit integer shared atomicAdd, 9 double shared atomicAdd,
 * 10 Philox blocks with 64-bit products, 11 warp shuffles, 12 bin
 * updates by warp ownership (8 axes, 50 bins, shuffles, no atomics),
 * 13 64-bit integer shared atomicAdd (one histogram per CTA), 14 the same
 * with one histogram per warp, 15 32-bit integer atomicAdd per warp.
 * Launches its own kernels on the legacy default stream and synchronises. */
vegas_status vegas_microbench(int op, double* rate);

/* One evaluation pass that allocates no device memory (the paper has no
 * counterpart; this exists for callers that cannot call cudaMalloc, such as
 * code living inside another runtime's fixed memory pool or a
 * latency-critical loop where an allocation, which may synchronise the
 * device or fail under fragmentation, is not allowed after start-up).
 * Same pass as vegas_eval, without a context: `config` and `integrand` as
 * for vegas_create (config->stream orders the work; NULL means the legacy
 * default stream), `edges` a DEVICE array [ndim][nbins+1] holding the grid,
 * `it` the Philox iteration index (< 2^31), `out` a DEVICE array of
 * 2 ndim nbins + 5 doubles receiving the per-bin sums (sum w, then sum w^2,
 * as vegas_get_grid) followed by I, its variance, sum w, sum w^2 and the
 * count of non-finite weights.  Asynchronous: `out` is ready when the stream
 * reaches it.  Every intermediate lives in one static 8 MiB device array of
 * the library (held by every GPU that loads it until the process exits).
 * Every shape vegas_create accepts fits: the array holds the grid tables
 * and one row of partial sums (16 ndim nbins + 40 bytes) per CTA, and where
 * one row per resident CTA would not fit the pass runs fewer CTAs (about
 * 60 at ndim nbins = 32 x 256), which is slower but not an error.  The first call on a device
 * looks up that array's device address, so make it before any stream
 * capture.  All calls share the array and each call overwrites it: calls
 * that overlap on the GPU (other streams, other host threads) race and give
 * wrong results. */
vegas_status vegas_eval_noalloc(const vegas_config* config, const vegas_integrand* integrand,
                                const double* edges, uint32_t it, double* out);

/* Failure injection for tests (no counterpart in the paper).  Every device
 * and pinned-host allocation the library makes goes through one wrapper.
 * After vegas_fail_alloc_after(n) with n >= 0 the next n allocations
 * succeed and the one after fails as an exhausted device would
 * (cudaErrorMemoryAllocation, without calling the allocator); the hook then
 * disarms itself.  n < 0 disarms it.  The failing call returns
 * VEGAS_ENOMEM and frees what it had allocated.  Process-wide; any thread.
 * vegas_alloc_count returns the number of allocations attempted so far
 * (monotonic), so a test can count those a constructor makes. */
void vegas_fail_alloc_after(int64_t n);
uint64_t vegas_alloc_count(void);

/* No counterpart in the paper (its programs print and stop).  Message of
 * the last failure on ctx (or of the calling thread when ctx is NULL),
 * owned by the library and valid until the next call on that context or
 * thread.  Never NULL. */
const char* vegas_last_error(const vegas_ctx* ctx);

#endif /* __CUDACC_RTC__ */

#ifdef __cplusplus
}
#endif
#endif
