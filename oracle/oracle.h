/*
 * oracle.h -- plain single-threaded FP64 CPU oracle of the VEGAS / BASES
 * iteration described in Sec. 2.1 of "Monte Carlo integration on GPU"
 * (Kanzaki, arXiv 1010.2107): steps 2 (point generation), 3 (integrand),
 * 4 (accumulation), 5 (grid optimisation) and 6 (iteration / stopping),
 * plus the BASES two-phase split of Sec. 2.1 and Sec. 5.1.
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA library
 * against.  Only the test suite, the package entry's smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or constant with the CUDA library and never calls it.
 *
 * Precision: every value is computed in IEEE binary64 (double); sums use
 * Neumaier-compensated accumulation.  Built with -ffp-contract=off so that
 * x86-64 and aarch64 give identical results.
 *
 * Parity unpinned: the full RAMBO integrand with its cuts (kind 5, obs 0)
 * for n >= 3 partons has no closed form.  Its building blocks are pinned
 * (phase-space volume, momentum conservation, <s12>, the s12 density,
 * hand-built cut cases and Lorentz / azimuthal invariances) and so is the
 * complete product for n = 2, with both cut forms, against its closed
 * form; for n >= 3 the product is checked only against the CUDA path and
 * by statistical consistency.
 */
#ifndef GVEGAS_ORACLE_H
#define GVEGAS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAXDIM 64
#define ORC_MAXBINS 1024

/* Integrand kinds.  The numbering is a convention that the test suite maps
 * to the CUDA library's own enumeration. */
enum {
  ORC_GENZ_GAUSSIAN = 0,     /* params: a[d], u[d]                          */
  ORC_GENZ_PRODUCT_PEAK = 1, /* params: a[d], u[d]                          */
  ORC_GENZ_CORNER_PEAK = 2,  /* params: a[d]                                */
  ORC_GENZ_OSCILLATORY = 3,  /* params: a[d], u1                            */
  ORC_DOUBLE_GAUSSIAN = 4,   /* params: c1, c2, w                           */
  ORC_RAMBO_BW = 5,          /* params: see ORC_RB_* below, d = 4 n         */
  ORC_GENZ_CONTINUOUS = 6,   /* params: a[d], u[d]                          */
  ORC_GENZ_DISCONTINUOUS = 7, /* params: a[d], u[min(d, 2)]                 */
  ORC_W_MUNU = 8              /* params: see ORC_W_* below, d = 5             */
};

/* u dbar -> W+ -> mu+ nu_mu in pp collisions (Sec. 4, the process with
 * n = 0 gluons and the lepton cuts |eta| < 2.5, pT > 20 GeV), total cross
 * section in pb.  The five variables: y1 -> shat through the Breit-Wigner
 * mapping shat = M^2 + M Gamma tan(rho), rho uniform between the images of
 * [SHAT_MIN, S]; y2 -> the W rapidity, uniform in [ln(tau)/2, -ln(tau)/2];
 * y3 -> cos(theta) of the mu+ against the u direction in the partonic
 * frame; y4 -> its azimuth; y5 -> one of 16 helicity combinations (Sec. 4:
 * one variable sums the helicities).  The u comes from the proton moving
 * along +z, the dbar from the other.  Parton densities are a stand-in with
 * the shape f(x) = A x^a (1 - x)^b (no CTEQ6L1 table is available). */
enum {
  ORC_W_SQRTS = 0,   /* hadronic centre-of-mass energy sqrt(S), GeV    */
  ORC_W_M = 1,       /* W mass, GeV                                    */
  ORC_W_GAMMA = 2,   /* W width, GeV                                   */
  ORC_W_GF = 3,      /* Fermi constant, GeV^-2                         */
  ORC_W_VUD = 4,     /* |V_ud|                                         */
  ORC_W_PTMIN = 5,   /* mu+ transverse momentum cut, GeV               */
  ORC_W_ETAMAX = 6,  /* mu+ pseudorapidity cut                         */
  ORC_W_SMIN = 7,    /* lower end of the shat range, GeV^2             */
  ORC_W_CUTS = 8,    /* 1: apply the two cuts, 0: none                 */
  ORC_W_AU = 9, ORC_W_ALU = 10, ORC_W_BU = 11,  /* u density A, a, b    */
  ORC_W_AD = 12, ORC_W_ALD = 13, ORC_W_BD = 14, /* dbar density A, a, b */
  ORC_W_NPARAMS = 15
};

/* RAMBO + Breit-Wigner parameter slots. */
enum {
  ORC_RB_N = 0,      /* number of massless final-state partons n >= 2     */
  ORC_RB_SQRTS = 1,  /* partonic centre-of-mass energy, GeV              */
  ORC_RB_M = 2,      /* Breit-Wigner mass, GeV                           */
  ORC_RB_GAMMA = 3,  /* Breit-Wigner width, GeV                          */
  ORC_RB_PTMIN = 4,  /* hard transverse-momentum cut, GeV                */
  ORC_RB_DRMIN = 5,  /* Delta R separation cut                           */
  ORC_RB_CUT = 6,    /* 0 hard pT cut, 1 sigmoid pT cut, 2 no cuts       */
  ORC_RB_T = 7,      /* sigmoid threshold, GeV                           */
  ORC_RB_WC = 8,     /* sigmoid width, GeV                               */
  ORC_RB_OBS = 9,    /* 0 full integrand, 1 unit, 2 s12, 3 BW(s12) only  */
  ORC_RB_NPARAMS = 10
};

typedef struct {
  int kind;
  int ndim;
  const double* params;
  int nparams;
} orc_fn;

/* One VEGAS / BASES context: NCALL points per iteration in ndim
 * dimensions, nbins grid bins per axis, nstrat hypercube divisions per
 * axis (0 or 1 = no stratification), ybits = 24 (one Philox word per axis)
 * or 53 (two words per axis). */
typedef struct {
  int ndim;
  int nbins;
  int64_t ncall;
  int nstrat;
  int ybits;
  uint64_t seed;
  uint32_t instance;
  double alpha;
} orc_cfg;

/* Per-iteration outputs.  S1, S2: [ndim][nbins]; C1, C2: [nstrat^ndim]
 * (may be NULL).  tot: {sum w, sum w^2, I_j, sigma_j^2}.  Cmax (may be
 * NULL): [nstrat^ndim], per hypercube max(0, largest w), for SPRING. */
typedef struct {
  double* S1;
  double* S2;
  double* C1;
  double* C2;
  double tot[4];
  int64_t nonfinite;
  double* Cmax;
} orc_iter_out;

/* Philox4x32-10 block: out = Philox(ctr, key). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]);

/* The random words of sample s in iteration it (ndim or 2 ndim words). */
int orc_sample_words(const orc_cfg* cfg, uint32_t it, uint64_t s,
                     uint32_t* words);

/* Step 2: bins[a], frac[a], x[a] and the Jacobian of sample s. */
int orc_sample_point(const orc_cfg* cfg, const double* edges, uint32_t it,
                     uint64_t s, int32_t* bins, double* frac, double* x,
                     double* jac);

/* Step 2 from given words: the point of a sample in hypercube `cube`. */
int orc_point_from_words(const orc_cfg* cfg, const double* edges,
                         uint64_t cube, const uint32_t* words, int32_t* bins,
                         double* frac, double* x, double* jac);
int orc_points_from_words(const orc_cfg* cfg, const double* edges,
                          const uint64_t* cube, const uint32_t* words,
                          int64_t n, int32_t* bins, double* frac, double* x,
                          double* jac);

/* Step 2 for a list of sample indices; any output pointer may be NULL.
 * words: [n][W], bins: [n][ndim], frac, x: [n][ndim], jac: [n]. */
int orc_sample_batch(const orc_cfg* cfg, const double* edges, uint32_t it,
                     const uint64_t* s, int64_t n, uint32_t* words,
                     int32_t* bins, double* frac, double* x, double* jac);

/* Step 3: the integrand at n points x[n][ndim]. */
int orc_integrand(const orc_fn* fn, int64_t n, const double* x, double* f);

/* d f / d theta at n points; theta = (M, Gamma, T) for RAMBO_BW and
 * (u[d], a[d]) for GENZ_GAUSSIAN.  grad: [n][ntheta]. */
int orc_integrand_grad(const orc_fn* fn, int64_t n, const double* x,
                       double* grad);
int orc_ntheta(const orc_fn* fn);

/* Cut margins (test infrastructure): m[i] = the smallest relative distance
 * |q - e| / |e| from its edge e of any quantity q that the integrand at
 * x[i] compares with a cut or a discontinuity (RAMBO: each pT against the
 * hard cut, each Delta R against its cut; discontinuous Genz: x_1, x_2
 * against u_1, u_2; W: pT, |eta|, x1, x2 and the helicity-cell edge of
 * 16 y5); INFINITY where it compares none.  A point with a small margin
 * may fall on either side of its edge under rounding. */
int orc_cut_margin(const orc_fn* fn, int64_t n, const double* x, double* m);

/* RAMBO: n massless momenta (E, px, py, pz) from 4n numbers in (0, 1]. */
int orc_rambo(int n, double sqrt_s, const double* rho, double* p);
/* The RAMBO_BW integrand without the phase-space weight, from momenta. */
double orc_rambo_f_momenta(const double* params, const double* p);
/* Phase-space volume of n massless particles at energy sqrt_s. */
double orc_rambo_volume(int n, double sqrt_s);

/* Step 4: one full iteration over NCALL points. */
int orc_iteration(const orc_cfg* cfg, const orc_fn* fn, const double* edges,
                  uint32_t it, orc_iter_out* out);

/* Step 5: grid optimisation from the per-bin sums of squares. */
int orc_refine(int ndim, int nbins, double alpha, const double* S2,
               double* edges);

/* Step 6: combination of m iteration estimates.  out = {I, sigma, chi2/dof}. */
void orc_combine(int m, const double* I, const double* var, double out[3]);

/* VEGAS loop: up to itmx iterations starting at Philox iteration it0,
 * refining after each if refine != 0, stopping when sigma/|I| < acc.
 * hist: [itmx][2] (I_j, sigma_j^2).  Returns the number of iterations run. */
int orc_vegas(const orc_cfg* cfg, const orc_fn* fn, double* edges,
              uint32_t it0, int itmx, int refine, double acc, double* hist,
              double out[3]);

/* BASES: phase 1 (itmx1 iterations, refining) then phase 2 (itmx2
 * iterations, frozen grid); out combines phase 2 only.  n_done: {n1, n2}. */
int orc_bases(const orc_cfg* cfg, const orc_fn* fn, double* edges,
              uint32_t it0, int itmx1, double acc1, int itmx2, double acc2,
              double* hist, double out[3], int n_done[2]);

/* SPRING (unweighted events from the BASES integration phase; Sec. 2.1
 * names it, Kawabata's BASES/SPRING defines it; the steps below follow it,
 * with an integer cube choice).  orc_spring_table: integer hypercube weights
 * q_c = ceil(M_c * scale), scale = 2^24 / max_c M_c, from the per-cube
 * maxima M_c; returns -1 when every M_c is 0.  orc_spring: trials
 * t = t0 .. t0 + n - 1, each from the Philox words of counter
 * (t, word group, 0xFFFFFFFF, instance): words 0..W-1 place a point in the
 * chosen cube as the sampling step does (W = ndim, or 2 ndim for 53-bit
 * words), words W and W+1 form U = 2^32 w_W + w_{W+1} and pick the cube c
 * with P_c <= floor(U Q / 2^64) < P_{c+1} (P the prefix sums of q, Q the
 * total), and the next word (two for 53-bit) gives v in [0, 1).  With
 * w = f J and Mt = q_c / scale: w <= 0 is dropped (*nonpos), w > Mt is kept
 * (*overflow), otherwise kept iff v Mt < w.  Kept points go to x_out[k][ndim]
 * and trial_out[k] in trial order; *n_events = k. */
int orc_spring_table(int64_t G, const double* cmax, uint64_t* q, double* scale);
int orc_spring(const orc_cfg* cfg, const orc_fn* fn, const double* edges,
               const double* cmax, uint64_t t0, int64_t n, double* x_out,
               uint64_t* trial_out, int64_t* n_events, int64_t* overflow,
               int64_t* nonpos);

/* Estimator gradient on a frozen grid: dI/dtheta = (1/n) sum J df/dtheta. */
int orc_gradient(const orc_cfg* cfg, const orc_fn* fn, const double* edges,
                 uint32_t it, double* grad, double* I);

#ifdef __cplusplus
}
#endif
#endif
