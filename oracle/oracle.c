/*
 * oracle.c -- plain single-threaded FP64 CPU oracle of the VEGAS / BASES
 * iteration of "Monte Carlo integration on GPU" (Kanzaki, arXiv 1010.2107).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the package entry's
 * smoke check and the benchmark's CPU-baseline leg; never by the library.
 * It shares no code with the CUDA library.
 *
 * The paper fixes the structure of the method (Sec. 2.1, steps 1-6; BASES
 * phases in Sec. 2.1 and Sec. 5.1) and defers the formulas to VEGAS
 * (Lepage) and BASES (Kawabata).  Each function below follows one step and
 * states the published method it restates.  Everything is binary64 with
 * Neumaier-compensated sums; no blocking, fusion or reordering beyond the
 * order of the steps.
 *
 * Parity unpinned: the full RAMBO integrand with cuts for n >= 3 partons
 * (see oracle.h).  The cut margins (orc_cut_margin) are pinned by bisection
 * on the integrand's own cut decisions.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ */
/* Neumaier compensated summation.                                     */
/* ------------------------------------------------------------------ */
typedef struct {
  double s, c;
} ksum;

static void kadd(ksum* k, double v) {
  double t = k->s + v;
  if (fabs(k->s) >= fabs(v))
    k->c += (k->s - t) + v;
  else
    k->c += (v - t) + k->s;
  k->s = t;
}

static double kval(const ksum* k) { return k->s + k->c; }

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of    */
/* two 32x32->64 multiplications and a key-dependent XOR permutation,  */
/* with a Weyl-sequence key schedule between rounds.  Stands in for     */
/* the per-thread xorshift generator of Appendix A (step 2).           */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]) {
  const uint32_t mul0 = 0xD2511F53u, mul1 = 0xCD9E8D57u;
  const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += weyl0;
      k1 += weyl1;
    }
    uint64_t p0 = (uint64_t)mul0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)mul1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

static int words_per_sample(const orc_cfg* cfg) {
  return cfg->ybits == 53 ? 2 * cfg->ndim : cfg->ndim;
}

/* Counter layout: (sample index within the iteration, word group
 * floor(j/4), iteration index, instance id); key = (seed low, seed high).
 * Word j of a sample is output word j mod 4 of its group. */
int orc_sample_words(const orc_cfg* cfg, uint32_t it, uint64_t s,
                     uint32_t* words) {
  if (s > 0xFFFFFFFFull) return -1;
  int W = words_per_sample(cfg);
  uint32_t key[2] = {(uint32_t)cfg->seed, (uint32_t)(cfg->seed >> 32)};
  for (int q = 0; 4 * q < W; ++q) {
    uint32_t ctr[4] = {(uint32_t)s, (uint32_t)q, it, cfg->instance};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    for (int r = 0; r < 4 && 4 * q + r < W; ++r) words[4 * q + r] = out[r];
  }
  return 0;
}

static int cfg_valid(const orc_cfg* cfg) {
  if (cfg->ndim < 1 || cfg->ndim > ORC_MAXDIM) return 0;
  if (cfg->nbins < 1 || cfg->nbins > ORC_MAXBINS) return 0;
  if (cfg->ybits != 24 && cfg->ybits != 53) return 0;
  if (cfg->ncall < 2 || cfg->ncall > 0x100000000ll) return 0;
  int g = cfg->nstrat < 1 ? 1 : cfg->nstrat;
  if (cfg->ybits == 53 && (int64_t)g * cfg->nbins >= 2048) return 0;
  return 1;
}

/* Number of hypercubes g^d, or -1 if it overflows NCALL. */
static int64_t n_cubes(const orc_cfg* cfg) {
  int g = cfg->nstrat < 1 ? 1 : cfg->nstrat;
  int64_t G = 1;
  for (int a = 0; a < cfg->ndim; ++a) {
    G *= g;
    if (G > cfg->ncall) return -1;
  }
  return G;
}

/* Step 2: a space point from d random numbers.  y_a in [0,1) comes from
 * the top bits of the Philox words (24 bits: word a >> 8; 53 bits: 27
 * bits of word 2a then 26 bits of word 2a+1).  With g divisions per axis
 * the sample's hypercube fixes the integer part of g*y_a (stratified
 * sampling of BASES).  The grid bin k_a and the position inside it are
 * computed from y_a*N in integer arithmetic; the point is then mapped
 * through the piecewise-linear VEGAS grid (Lepage 1978):
 *     x_a = e_a[k] + frac (e_a[k+1] - e_a[k]),  J = prod_a N (e_a[k+1] - e_a[k]). */
int orc_point_from_words(const orc_cfg* cfg, const double* edges,
                         uint64_t cube, const uint32_t* w, int32_t* bins,
                         double* frac, double* x, double* jac) {
  if (!cfg_valid(cfg)) return -1;
  int d = cfg->ndim, N = cfg->nbins, b = cfg->ybits;
  int g = cfg->nstrat < 1 ? 1 : cfg->nstrat;
  double J = 1.0;
  uint64_t cube_rest = cube;
  for (int a = 0; a < d; ++a) {
    uint64_t m;
    if (b == 24)
      m = (uint64_t)(w[a] >> 8);
    else
      m = ((uint64_t)(w[2 * a] >> 5) << 26) | (uint64_t)(w[2 * a + 1] >> 6);
    uint64_t ca = cube_rest % (uint64_t)g;
    cube_rest /= (uint64_t)g;
    uint64_t Y = (ca << b) | m;                 /* g y_a = ca + m / 2^b  */
    uint64_t T = Y * (uint64_t)N;               /* g 2^b y_a N           */
    uint64_t Gb = (uint64_t)g << b;
    uint64_t k = T / Gb;
    uint64_t r = T % Gb;
    double fr = (double)r / (double)Gb;
    const double* e = edges + (size_t)a * (N + 1);
    double lo = e[k], hi = e[k + 1];
    double xa = lo + fr * (hi - lo);
    J *= (double)N * (hi - lo);
    if (bins) bins[a] = (int32_t)k;
    if (frac) frac[a] = fr;
    if (x) x[a] = xa;
  }
  if (jac) *jac = J;
  return 0;
}

int orc_sample_point(const orc_cfg* cfg, const double* edges, uint32_t it,
                     uint64_t s, int32_t* bins, double* frac, double* x,
                     double* jac) {
  if (!cfg_valid(cfg)) return -1;
  if ((int64_t)s >= cfg->ncall) return -1;
  int64_t G = n_cubes(cfg);
  if (G < 0) return -1;
  int64_t nc = cfg->ncall / G;
  uint32_t w[2 * ORC_MAXDIM];
  if (orc_sample_words(cfg, it, s, w)) return -1;
  return orc_point_from_words(cfg, edges, s / (uint64_t)nc, w, bins, frac, x,
                              jac);
}

/* Word -> point map for n word vectors (cube index per vector). */
int orc_points_from_words(const orc_cfg* cfg, const double* edges,
                          const uint64_t* cube, const uint32_t* w, int64_t n,
                          int32_t* bins, double* frac, double* x, double* jac) {
  int d = cfg->ndim, W = words_per_sample(cfg);
  for (int64_t i = 0; i < n; ++i)
    if (orc_point_from_words(cfg, edges, cube[i], w + i * W,
                             bins ? bins + i * d : NULL,
                             frac ? frac + i * d : NULL, x ? x + i * d : NULL,
                             jac ? jac + i : NULL))
      return -1;
  return 0;
}

int orc_sample_batch(const orc_cfg* cfg, const double* edges, uint32_t it,
                     const uint64_t* s, int64_t n, uint32_t* words,
                     int32_t* bins, double* frac, double* x, double* jac) {
  int d = cfg->ndim, W = words_per_sample(cfg);
  for (int64_t i = 0; i < n; ++i) {
    if (words && orc_sample_words(cfg, it, s[i], words + i * W)) return -1;
    if (orc_sample_point(cfg, edges, it, s[i], bins ? bins + i * d : NULL,
                         frac ? frac + i * d : NULL, x ? x + i * d : NULL,
                         jac ? jac + i : NULL))
      return -1;
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Step 3: integrands on [0,1]^d.                                      */
/* Genz (1984) test families, the two-peak Gaussian of Lepage's tests, */
/* and a massless RAMBO phase space (Kleiss, Stirling, Ellis 1986)     */
/* with a W-like Breit-Wigner and the jet cuts of Sec. 4 (pT and       */
/* Delta R of eqs. 2-3, simplified to plain Delta R).                  */
/* ------------------------------------------------------------------ */

double orc_rambo_volume(int n, double sqrt_s) {
  /* (pi/2)^(n-1) s^(n-2) / ((n-1)! (n-2)!) */
  double s = sqrt_s * sqrt_s;
  double v = pow(M_PI / 2.0, n - 1) * pow(s, n - 2);
  for (int i = 2; i <= n - 1; ++i) v /= (double)i;
  for (int i = 2; i <= n - 2; ++i) v /= (double)i;
  return v;
}

/* RAMBO: isotropic massless momenta q_i with energy density q0 e^{-q0},
 * then the conformal transformation (boost + scaling) that brings the
 * total momentum to (sqrt s, 0, 0, 0). */
int orc_rambo(int n, double sqrt_s, const double* rho, double* p) {
  double Q[4] = {0, 0, 0, 0};
  double* q = (double*)malloc(sizeof(double) * 4 * (size_t)n);
  if (!q) return -1;
  for (int i = 0; i < n; ++i) {
    const double* r = rho + 4 * i;
    double q0 = -log(r[0] * r[1]);
    double c = 2.0 * r[2] - 1.0;
    double sn = sqrt(1.0 - c * c);
    double phi = 2.0 * M_PI * r[3];
    q[4 * i + 0] = q0;
    q[4 * i + 1] = q0 * sn * cos(phi);
    q[4 * i + 2] = q0 * sn * sin(phi);
    q[4 * i + 3] = q0 * c;
    for (int mu = 0; mu < 4; ++mu) Q[mu] += q[4 * i + mu];
  }
  double MQ = sqrt(Q[0] * Q[0] - Q[1] * Q[1] - Q[2] * Q[2] - Q[3] * Q[3]);
  double bx = -Q[1] / MQ, by = -Q[2] / MQ, bz = -Q[3] / MQ;
  double gam = Q[0] / MQ;
  double A = 1.0 / (1.0 + gam);
  double X = sqrt_s / MQ;
  for (int i = 0; i < n; ++i) {
    double* qi = q + 4 * i;
    double bq = bx * qi[1] + by * qi[2] + bz * qi[3];
    p[4 * i + 0] = X * (gam * qi[0] + bq);
    p[4 * i + 1] = X * (qi[1] + bx * qi[0] + A * bq * bx);
    p[4 * i + 2] = X * (qi[2] + by * qi[0] + A * bq * by);
    p[4 * i + 3] = X * (qi[3] + bz * qi[0] + A * bq * bz);
  }
  free(q);
  return 0;
}

static double sinv(const double* pi, const double* pj) {
  /* s_ij = (p_i + p_j)^2 = 2 p_i . p_j for massless momenta */
  return 2.0 * (pi[0] * pj[0] - pi[1] * pj[1] - pi[2] * pj[2] - pi[3] * pj[3]);
}

static double breit_wigner(double s, double M, double G) {
  double t = s - M * M;
  return M * G / (t * t + M * M * G * G);
}

static double sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }

/* Integrand value (without phase-space weight) from n momenta, and
 * optionally its derivatives with respect to (M, Gamma, T). */
static double rambo_f_grad(const double* P, const double* p, double* grad) {
  int n = (int)P[ORC_RB_N];
  double M = P[ORC_RB_M], Gam = P[ORC_RB_GAMMA];
  int cut = (int)P[ORC_RB_CUT];
  int obs = (int)P[ORC_RB_OBS];
  if (grad) grad[0] = grad[1] = grad[2] = 0.0;
  double s12 = sinv(p, p + 4);
  if (obs == 2) return s12;
  if (obs == 3) return breit_wigner(s12, M, Gam);
  double pt[ORC_MAXDIM], eta[ORC_MAXDIM], phi[ORC_MAXDIM];
  for (int i = 0; i < n; ++i) {
    const double* pi = p + 4 * i;
    double pabs = sqrt(pi[1] * pi[1] + pi[2] * pi[2] + pi[3] * pi[3]);
    pt[i] = sqrt(pi[1] * pi[1] + pi[2] * pi[2]);
    eta[i] = atanh(pi[3] / pabs);
    phi[i] = atan2(pi[2], pi[1]);
  }
  double cutw = 1.0, dlogcut_dT = 0.0;
  if (cut == 0) {
    for (int i = 0; i < n; ++i)
      if (!(pt[i] > P[ORC_RB_PTMIN])) return 0.0;
  } else if (cut == 1) {
    double T = P[ORC_RB_T], wc = P[ORC_RB_WC];
    for (int i = 0; i < n; ++i) {
      double sg = sigmoid((pt[i] - T) / wc);
      cutw *= sg;
      dlogcut_dT += -(1.0 - sg) / wc;
    }
  }
  if (cut == 0 || cut == 1) {
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) {
        double de = eta[i] - eta[j];
        double dp = phi[i] - phi[j];
        while (dp > M_PI) dp -= 2.0 * M_PI;
        while (dp < -M_PI) dp += 2.0 * M_PI;
        double dR = sqrt(de * de + dp * dp);
        if (!(dR > P[ORC_RB_DRMIN])) return 0.0;
      }
  }
  double prod = 1.0;
  for (int i = 0; i < n; ++i) prod *= 1.0 / sinv(p + 4 * i, p + 4 * ((i + 1) % n));
  double bw = breit_wigner(s12, M, Gam);
  double f = prod * bw * cutw;
  if (grad) {
    double t = s12 - M * M;
    double D = t * t + M * M * Gam * Gam;
    double dD_dM = -4.0 * M * t + 2.0 * M * Gam * Gam;
    double dD_dG = 2.0 * M * M * Gam;
    double dbw_dM = Gam / D - M * Gam * dD_dM / (D * D);
    double dbw_dG = M / D - M * Gam * dD_dG / (D * D);
    grad[0] = prod * cutw * dbw_dM;
    grad[1] = prod * cutw * dbw_dG;
    grad[2] = (cut == 1) ? f * dlogcut_dT : 0.0;
  }
  return f;
}

double orc_rambo_f_momenta(const double* params, const double* p) {
  return rambo_f_grad(params, p, NULL);
}

int orc_ntheta(const orc_fn* fn) {
  switch (fn->kind) {
    case ORC_GENZ_GAUSSIAN: return 2 * fn->ndim;
    case ORC_DOUBLE_GAUSSIAN: return 3;
    case ORC_RAMBO_BW: return 3;
    default: return 0;
  }
}

static int fn_valid(const orc_fn* fn) {
  int d = fn->ndim;
  if (d < 1 || d > ORC_MAXDIM) return 0;
  switch (fn->kind) {
    case ORC_GENZ_GAUSSIAN:
    case ORC_GENZ_PRODUCT_PEAK: return fn->nparams >= 2 * d;
    case ORC_GENZ_CORNER_PEAK: return fn->nparams >= d;
    case ORC_GENZ_OSCILLATORY: return fn->nparams >= d + 1;
    case ORC_DOUBLE_GAUSSIAN: return fn->nparams >= 3;
    case ORC_GENZ_CONTINUOUS: return fn->nparams >= 2 * d;
    case ORC_GENZ_DISCONTINUOUS: return fn->nparams >= d + (d < 2 ? d : 2);
    case ORC_W_MUNU: return d == 5 && fn->nparams >= ORC_W_NPARAMS;
    case ORC_RAMBO_BW: {
      if (fn->nparams < ORC_RB_NPARAMS) return 0;
      int n = (int)fn->params[ORC_RB_N];
      return n >= 2 && 4 * n == d && n <= ORC_MAXDIM / 4;
    }
    default: return 0;
  }
}

/* u dbar -> W+ -> mu+ nu_mu (see oracle.h for the variables).  Written as
 * the textbook pieces, in this order: the mapping of y to (shat, y_W,
 * cos theta, phi, h) with its Jacobian, the parton luminosity, the flux
 * 1/(2 shat), the two-body phase space dPhi_2 = dcos(theta) dphi / (32
 * pi^2), and the helicity amplitude squared, sampled over the 16
 * helicity combinations with weight 16.  For massless V - A couplings only
 * u(-) dbar(+) -> nu(-) mu+(+) is non-zero:
 *   |M|^2 = g^4 |V_ud|^2 uhat^2 / ((shat - M^2)^2 + M^2 Gamma^2),
 *   uhat = (p_u - p_mu)^2,  g^2 = 8 M^2 G_F / sqrt(2),
 * averaged over the initial spins (1/4) and colours (3 / 9). */
static double w_munu(const double* P, const double* y) {
  const double S = P[ORC_W_SQRTS] * P[ORC_W_SQRTS], M = P[ORC_W_M], G = P[ORC_W_GAMMA];
  const double rho_lo = atan((P[ORC_W_SMIN] - M * M) / (M * G)), rho_hi = atan((S - M * M) / (M * G));
  const double rho = rho_lo + (rho_hi - rho_lo) * y[0];
  const double shat = M * M + M * G * tan(rho);
  const double dshat = (rho_hi - rho_lo) * M * G / (cos(rho) * cos(rho)); /* dshat/dy1 */
  const double tau = shat / S;
  if (!(tau > 0.0 && tau < 1.0)) return 0.0;
  const double L = -log(tau);
  const double yw = (y[1] - 0.5) * L; /* dyw/dy2 = L */
  const double x1 = sqrt(tau) * exp(yw), x2 = sqrt(tau) * exp(-yw);
  if (!(x1 < 1.0 && x2 < 1.0)) return 0.0;
  const double c = 2.0 * y[2] - 1.0; /* dc/dy3 = 2 */
  /* phi = 2 pi y4: nothing depends on it; dphi/dy4 = 2 pi */
  int h = (int)floor(16.0 * y[4]);
  if (h > 15) h = 15;
  if (P[ORC_W_CUTS] != 0.0) {
    const double pt = 0.5 * sqrt(shat) * sqrt(1.0 - c * c);
    const double eta = atanh(c) + yw; /* partonic rapidity of the mu+ plus the boost */
    if (!(pt > P[ORC_W_PTMIN] && fabs(eta) < P[ORC_W_ETAMAX])) return 0.0;
  }
  /* helicity bits: u, dbar, nu, mu+ (1 = positive helicity) */
  double msq = 0.0;
  if (h == (0 | 2 | 0 | 8)) {
    const double g2 = 8.0 * M * M * P[ORC_W_GF] / sqrt(2.0);
    const double uhat = -0.5 * shat * (1.0 - c);
    const double den = (shat - M * M) * (shat - M * M) + M * M * G * G;
    msq = g2 * g2 * P[ORC_W_VUD] * P[ORC_W_VUD] * uhat * uhat / den;
  }
  const double avg = 1.0 / 4.0 * 3.0 / 9.0;
  const double fu = P[ORC_W_AU] * pow(x1, P[ORC_W_ALU]) * pow(1.0 - x1, P[ORC_W_BU]);
  const double fd = P[ORC_W_AD] * pow(x2, P[ORC_W_ALD]) * pow(1.0 - x2, P[ORC_W_BD]);
  const double jac = dshat / S * L * 2.0 * 2.0 * M_PI; /* dtau dyw dc dphi per dy1..dy4 */
  const double dphi2 = 1.0 / (32.0 * M_PI * M_PI);
  const double pb = 0.3893793721e9; /* GeV^-2 -> pb */
  return fu * fd * jac * dphi2 / (2.0 * shat) * 16.0 * avg * msq * pb;
}

/* One point: f(x) and, when grad != NULL, df/dtheta. */
static double eval_point(const orc_fn* fn, const double* x, double* grad) {
  const double* P = fn->params;
  int d = fn->ndim;
  switch (fn->kind) {
    case ORC_GENZ_GAUSSIAN: {
      /* f = exp(-sum_i a_i^2 (x_i - u_i)^2) */
      const double *a = P, *u = P + d;
      double q = 0.0;
      for (int i = 0; i < d; ++i) q += a[i] * a[i] * (x[i] - u[i]) * (x[i] - u[i]);
      double f = exp(-q);
      if (grad)
        for (int i = 0; i < d; ++i) {
          grad[i] = f * 2.0 * a[i] * a[i] * (x[i] - u[i]);
          grad[d + i] = -f * 2.0 * a[i] * (x[i] - u[i]) * (x[i] - u[i]);
        }
      return f;
    }
    case ORC_GENZ_PRODUCT_PEAK: {
      /* f = prod_i 1 / (a_i^-2 + (x_i - u_i)^2) */
      const double *a = P, *u = P + d;
      double f = 1.0;
      for (int i = 0; i < d; ++i)
        f *= 1.0 / (1.0 / (a[i] * a[i]) + (x[i] - u[i]) * (x[i] - u[i]));
      return f;
    }
    case ORC_GENZ_CORNER_PEAK: {
      /* f = (1 + sum_i a_i x_i)^-(d+1) */
      double t = 1.0;
      for (int i = 0; i < d; ++i) t += P[i] * x[i];
      return pow(t, -(double)(d + 1));
    }
    case ORC_GENZ_CONTINUOUS: {
      /* f = exp(-sum_i a_i |x_i - u_i|)  (Genz 1984, "continuous") */
      const double *a = P, *u = P + d;
      double q = 0.0;
      for (int i = 0; i < d; ++i) q += a[i] * fabs(x[i] - u[i]);
      return exp(-q);
    }
    case ORC_GENZ_DISCONTINUOUS: {
      /* f = exp(sum_i a_i x_i) if x_1 <= u_1 and x_2 <= u_2, else 0
       * (Genz 1984, "discontinuous"; only x_1 for d = 1) */
      const double *a = P, *u = P + d;
      if (x[0] > u[0] || (d > 1 && x[1] > u[1])) return 0.0;
      double t = 0.0;
      for (int i = 0; i < d; ++i) t += a[i] * x[i];
      return exp(t);
    }
    case ORC_GENZ_OSCILLATORY: {
      /* f = cos(2 pi u_1 + sum_i a_i x_i) */
      double t = 2.0 * M_PI * P[d];
      for (int i = 0; i < d; ++i) t += P[i] * x[i];
      return cos(t);
    }
    case ORC_DOUBLE_GAUSSIAN: {
      /* f = 1/2 sum_{c in {c1,c2}} (w sqrt(pi))^-d exp(-sum_i ((x_i-c)/w)^2) */
      double c[2] = {P[0], P[1]}, w = P[2];
      double K = pow(w * sqrt(M_PI), -(double)d);
      double f = 0.0, g0 = 0.0, g1 = 0.0, gw = 0.0;
      for (int p = 0; p < 2; ++p) {
        double q = 0.0, lin = 0.0;
        for (int i = 0; i < d; ++i) {
          q += ((x[i] - c[p]) / w) * ((x[i] - c[p]) / w);
          lin += x[i] - c[p];
        }
        double E = exp(-q);
        f += 0.5 * K * E;
        double dc = 0.5 * K * E * 2.0 * lin / (w * w);
        if (p == 0) g0 = dc; else g1 = dc;
        gw += 0.5 * K * E * (-(double)d / w + 2.0 * q / w);
      }
      if (grad) {
        grad[0] = g0;
        grad[1] = g1;
        grad[2] = gw;
      }
      return f;
    }
    case ORC_W_MUNU:
      return w_munu(P, x);
    case ORC_RAMBO_BW: {
      int n = (int)P[ORC_RB_N];
      double sqrt_s = P[ORC_RB_SQRTS];
      double V = orc_rambo_volume(n, sqrt_s);
      int obs = (int)P[ORC_RB_OBS];
      if (grad) grad[0] = grad[1] = grad[2] = 0.0;
      if (obs == 1) return V;
      for (int i = 0; i < n; ++i)
        if (!(x[4 * i] * x[4 * i + 1] > 0.0)) return 0.0;
      double p[4 * (ORC_MAXDIM / 4)];
      if (orc_rambo(n, sqrt_s, x, p)) return NAN;
      double g3[3];
      double f = rambo_f_grad(P, p, grad ? g3 : NULL);
      if (grad)
        for (int t = 0; t < 3; ++t) grad[t] = V * g3[t];
      return V * f;
    }
  }
  return NAN;
}

int orc_integrand(const orc_fn* fn, int64_t n, const double* x, double* f) {
  if (!fn_valid(fn)) return -1;
  for (int64_t i = 0; i < n; ++i) f[i] = eval_point(fn, x + i * fn->ndim, NULL);
  return 0;
}

int orc_integrand_grad(const orc_fn* fn, int64_t n, const double* x,
                       double* grad) {
  if (!fn_valid(fn)) return -1;
  int nt = orc_ntheta(fn);
  if (nt == 0) return -1;
  for (int64_t i = 0; i < n; ++i)
    eval_point(fn, x + i * fn->ndim, grad + i * nt);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Cut margins (test infrastructure): how close each quantity that an  */
/* integrand compares with an edge lies to that edge, as the smallest  */
/* relative distance |q - e| / |e| over those quantities (INFINITY for */
/* an integrand that compares none).  A point whose margin is below    */
/* the rounding error of a computation of q may be cut on one side and */
/* kept on the other; every other point must agree.                    */
/* ------------------------------------------------------------------ */
static double rel_gap(double q, double e) {
  double den = fabs(e) > 0.0 ? fabs(e) : 1.0;
  return fabs(q - e) / den;
}

static double margin_point(const orc_fn* fn, const double* x) {
  const double* P = fn->params;
  int d = fn->ndim;
  double m = INFINITY;
  switch (fn->kind) {
    case ORC_GENZ_DISCONTINUOUS: {
      const double* u = P + d;
      m = rel_gap(x[0], u[0]);
      if (d > 1) m = fmin(m, rel_gap(x[1], u[1]));
      return m;
    }
    case ORC_W_MUNU: {
      /* the quantities w_munu tests, in its own arithmetic */
      const double S = P[ORC_W_SQRTS] * P[ORC_W_SQRTS], M = P[ORC_W_M], G = P[ORC_W_GAMMA];
      const double rho_lo = atan((P[ORC_W_SMIN] - M * M) / (M * G)), rho_hi = atan((S - M * M) / (M * G));
      const double shat = M * M + M * G * tan(rho_lo + (rho_hi - rho_lo) * x[0]);
      const double tau = shat / S;
      if (!(tau > 0.0 && tau < 1.0)) return rel_gap(tau, tau > 0.5 ? 1.0 : 0.0);
      const double L = -log(tau), yw = (x[1] - 0.5) * L;
      m = fmin(rel_gap(sqrt(tau) * exp(yw), 1.0), rel_gap(sqrt(tau) * exp(-yw), 1.0));
      const double k = floor(16.0 * x[4] + 0.5); /* nearest helicity-cell edge */
      if (k >= 1.0 && k <= 15.0) m = fmin(m, rel_gap(16.0 * x[4], k));
      if (P[ORC_W_CUTS] != 0.0) {
        const double c = 2.0 * x[2] - 1.0;
        const double pt = 0.5 * sqrt(shat) * sqrt(1.0 - c * c);
        const double eta = atanh(c) + yw;
        m = fmin(m, fmin(rel_gap(pt, P[ORC_W_PTMIN]), rel_gap(fabs(eta), P[ORC_W_ETAMAX])));
      }
      return m;
    }
    case ORC_RAMBO_BW: {
      int n = (int)P[ORC_RB_N], cut = (int)P[ORC_RB_CUT], obs = (int)P[ORC_RB_OBS];
      if (obs != 0 || cut == 2) return m;
      for (int i = 0; i < n; ++i)
        if (!(x[4 * i] * x[4 * i + 1] > 0.0)) return m;
      double p[4 * (ORC_MAXDIM / 4)], pt[ORC_MAXDIM], eta[ORC_MAXDIM], phi[ORC_MAXDIM];
      if (orc_rambo(n, P[ORC_RB_SQRTS], x, p)) return NAN;
      for (int i = 0; i < n; ++i) {
        const double* pi = p + 4 * i;
        double pabs = sqrt(pi[1] * pi[1] + pi[2] * pi[2] + pi[3] * pi[3]);
        pt[i] = sqrt(pi[1] * pi[1] + pi[2] * pi[2]);
        eta[i] = atanh(pi[3] / pabs);
        phi[i] = atan2(pi[2], pi[1]);
        if (cut == 0) m = fmin(m, rel_gap(pt[i], P[ORC_RB_PTMIN]));
      }
      for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
          double de = eta[i] - eta[j], dp = phi[i] - phi[j];
          while (dp > M_PI) dp -= 2.0 * M_PI;
          while (dp < -M_PI) dp += 2.0 * M_PI;
          m = fmin(m, rel_gap(sqrt(de * de + dp * dp), P[ORC_RB_DRMIN]));
        }
      return m;
    }
    default:
      return m;
  }
}

int orc_cut_margin(const orc_fn* fn, int64_t n, const double* x, double* m) {
  if (!fn_valid(fn)) return -1;
  for (int64_t i = 0; i < n; ++i) m[i] = margin_point(fn, x + i * fn->ndim);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Step 4: one iteration -- NCALL points, weights w = f J, per-bin     */
/* sums of w and w^2 on every axis, per-hypercube sums, and the        */
/* iteration estimate (VEGAS: sample mean and its variance; BASES      */
/* stratified: sum over hypercubes of volume-weighted cube means and   */
/* cube-mean variances).                                               */
/* ------------------------------------------------------------------ */
int orc_iteration(const orc_cfg* cfg, const orc_fn* fn, const double* edges,
                  uint32_t it, orc_iter_out* out) {
  if (!cfg_valid(cfg) || !fn_valid(fn) || fn->ndim != cfg->ndim) return -1;
  int d = cfg->ndim, N = cfg->nbins;
  int64_t n = cfg->ncall;
  int64_t G = n_cubes(cfg);
  if (G < 0 || n % G != 0) return -1;
  int64_t nc = n / G;
  int strat = G > 1;
  if (strat && nc < 2) return -1;
  size_t nb = (size_t)d * N;
  ksum* k1 = (ksum*)calloc(nb, sizeof(ksum));
  ksum* k2 = (ksum*)calloc(nb, sizeof(ksum));
  if (!k1 || !k2) {
    free(k1);
    free(k2);
    return -1;
  }
  ksum tw = {0, 0}, tw2 = {0, 0}, tI = {0, 0}, tV = {0, 0};
  ksum cw = {0, 0}, cw2 = {0, 0};
  double cmax = 0.0;
  int32_t bins[ORC_MAXDIM];
  double x[ORC_MAXDIM], J;
  out->nonfinite = 0;
  for (int64_t s = 0; s < n; ++s) {
    orc_sample_point(cfg, edges, it, (uint64_t)s, bins, NULL, x, &J);
    double f = eval_point(fn, x, NULL);
    double w = f * J;
    if (!isfinite(w)) {
      out->nonfinite++;
      w = 0.0;
    }
    double w2 = w * w;
    for (int a = 0; a < d; ++a) {
      kadd(&k1[(size_t)a * N + bins[a]], w);
      kadd(&k2[(size_t)a * N + bins[a]], w2);
    }
    kadd(&tw, w);
    kadd(&tw2, w2);
    if (w > cmax) cmax = w;
    if (out->Cmax && (s + 1) % nc == 0) {
      out->Cmax[s / nc] = cmax;
      cmax = 0.0;
    }
    if (strat) {
      kadd(&cw, w);
      kadd(&cw2, w2);
      if ((s + 1) % nc == 0) {
        int64_t c = s / nc;
        double s1 = kval(&cw), s2 = kval(&cw2);
        double m = s1 / (double)nc;
        double v = (s2 / (double)nc - m * m) / (double)(nc - 1);
        if (v < 0.0) v = 0.0;
        kadd(&tI, m);
        kadd(&tV, v);
        if (out->C1) out->C1[c] = s1;
        if (out->C2) out->C2[c] = s2;
        cw.s = cw.c = cw2.s = cw2.c = 0.0;
      }
    }
  }
  for (size_t i = 0; i < nb; ++i) {
    if (out->S1) out->S1[i] = kval(&k1[i]);
    if (out->S2) out->S2[i] = kval(&k2[i]);
  }
  free(k1);
  free(k2);
  out->tot[0] = kval(&tw);
  out->tot[1] = kval(&tw2);
  if (strat) {
    out->tot[2] = kval(&tI) / (double)G;
    out->tot[3] = kval(&tV) / ((double)G * (double)G);
  } else {
    double I = out->tot[0] / (double)n;
    double v = (out->tot[1] / (double)n - I * I) / (double)(n - 1);
    out->tot[2] = I;
    out->tot[3] = v < 0.0 ? 0.0 : v;
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Step 5: grid optimisation (Lepage 1978).  Per axis: smooth the      */
/* per-bin sums of (f J)^2 over neighbours, compress them with the     */
/* damping exponent alpha, r_k = ((1 - d_k/D) / ln(D/d_k))^alpha, and  */
/* place the new edges so that every new bin holds an equal share of   */
/* sum r, with r spread uniformly inside each old bin.                 */
/* ------------------------------------------------------------------ */
int orc_refine(int ndim, int nbins, double alpha, const double* S2,
               double* edges) {
  int N = nbins;
  if (ndim < 1 || N < 1 || N > ORC_MAXBINS) return -1;
  double dsm[ORC_MAXBINS], r[ORC_MAXBINS], enew[ORC_MAXBINS + 1];
  for (int a = 0; a < ndim; ++a) {
    const double* dd = S2 + (size_t)a * N;
    double* e = edges + (size_t)a * (N + 1);
    if (N == 1) continue;
    if (N == 2) {
      dsm[0] = dsm[1] = (dd[0] + dd[1]) / 2.0;
    } else {
      dsm[0] = (dd[0] + dd[1]) / 2.0;
      for (int k = 1; k < N - 1; ++k) dsm[k] = (dd[k - 1] + dd[k] + dd[k + 1]) / 3.0;
      dsm[N - 1] = (dd[N - 2] + dd[N - 1]) / 2.0;
    }
    double D = 0.0;
    for (int k = 0; k < N; ++k) D += dsm[k];
    if (!(D > 0.0) || !isfinite(D)) continue;
    double R = 0.0;
    for (int k = 0; k < N; ++k) {
      if (dsm[k] <= 0.0)
        r[k] = 0.0;
      else if (dsm[k] >= D)
        r[k] = 1.0;
      else
        r[k] = pow((1.0 - dsm[k] / D) / log(D / dsm[k]), alpha);
      R += r[k];
    }
    enew[0] = 0.0;
    enew[N] = 1.0;
    int k = 0;
    double acc = 0.0;
    for (int j = 1; j < N; ++j) {
      double tau = (double)j * R / (double)N;
      while (k < N - 1 && acc + r[k] < tau) {
        acc += r[k];
        ++k;
      }
      enew[j] = e[k] + (tau - acc) / r[k] * (e[k + 1] - e[k]);
    }
    for (int j = 0; j <= N; ++j) e[j] = enew[j];
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Step 6: combination of iterations (Lepage): inverse-variance        */
/* weighted mean, its error, and chi^2 per degree of freedom.          */
/* ------------------------------------------------------------------ */
void orc_combine(int m, const double* I, const double* var, double out[3]) {
  out[0] = out[1] = out[2] = 0.0;
  if (m <= 0) return;
  int nzero = 0;
  ksum z = {0, 0};
  for (int j = 0; j < m; ++j)
    if (!(var[j] > 0.0)) {
      kadd(&z, I[j]);
      ++nzero;
    }
  if (nzero > 0) {
    out[0] = kval(&z) / (double)nzero;
    return;
  }
  ksum sw = {0, 0}, swi = {0, 0};
  for (int j = 0; j < m; ++j) {
    kadd(&sw, 1.0 / var[j]);
    kadd(&swi, I[j] / var[j]);
  }
  double Ibar = kval(&swi) / kval(&sw);
  out[0] = Ibar;
  out[1] = 1.0 / sqrt(kval(&sw));
  if (m > 1) {
    ksum c2 = {0, 0};
    for (int j = 0; j < m; ++j) kadd(&c2, (I[j] - Ibar) * (I[j] - Ibar) / var[j]);
    out[2] = kval(&c2) / (double)(m - 1);
  }
}

/* Steps 2-6 repeated: the VEGAS loop.  The grid is refined after every
 * iteration when refine != 0; the loop stops early when the combined
 * relative error falls below acc (Sec. 5.1: ACC). */
int orc_vegas(const orc_cfg* cfg, const orc_fn* fn, double* edges,
              uint32_t it0, int itmx, int refine, double acc, double* hist,
              double out[3]) {
  int d = cfg->ndim, N = cfg->nbins;
  double* S1 = (double*)malloc(sizeof(double) * (size_t)d * N);
  double* S2 = (double*)malloc(sizeof(double) * (size_t)d * N);
  double* I = (double*)malloc(sizeof(double) * (size_t)(itmx > 0 ? itmx : 1));
  double* V = (double*)malloc(sizeof(double) * (size_t)(itmx > 0 ? itmx : 1));
  int done = 0, rc = 0;
  out[0] = out[1] = out[2] = 0.0;
  if (!S1 || !S2 || !I || !V) rc = -1;
  for (int i = 0; rc == 0 && i < itmx; ++i) {
    orc_iter_out o;
    memset(&o, 0, sizeof o);
    o.S1 = S1;
    o.S2 = S2;
    if (orc_iteration(cfg, fn, edges, it0 + (uint32_t)i, &o)) {
      rc = -1;
      break;
    }
    I[i] = o.tot[2];
    V[i] = o.tot[3];
    if (hist) {
      hist[2 * i] = I[i];
      hist[2 * i + 1] = V[i];
    }
    orc_combine(i + 1, I, V, out);
    if (refine) orc_refine(d, N, cfg->alpha, S2, edges);
    ++done;
    if (acc > 0.0 && out[1] < acc * fabs(out[0])) break;
  }
  free(S1);
  free(S2);
  free(I);
  free(V);
  return rc ? rc : done;
}

/* BASES (Sec. 2.1): a grid-optimisation phase of ITMX1 iterations, then
 * an integration phase of ITMX2 iterations on the frozen grid whose
 * estimates alone form the result (Sec. 5.1: ITMX1, ACC1, ITMX2, ACC2). */
int orc_bases(const orc_cfg* cfg, const orc_fn* fn, double* edges,
              uint32_t it0, int itmx1, double acc1, int itmx2, double acc2,
              double* hist, double out[3], int n_done[2]) {
  double tmp[3];
  int n1 = orc_vegas(cfg, fn, edges, it0, itmx1, 1, acc1, hist, tmp);
  if (n1 < 0) return n1;
  int n2 = orc_vegas(cfg, fn, edges, it0 + (uint32_t)n1, itmx2, 0, acc2,
                     hist ? hist + 2 * n1 : NULL, out);
  if (n2 < 0) return n2;
  n_done[0] = n1;
  n_done[1] = n2;
  return n1 + n2;
}

/* ------------------------------------------------------------------ */
/* SPRING: unweighted events on the frozen grid of the BASES           */
/* integration phase (see oracle.h for the reading).                   */
/* ------------------------------------------------------------------ */

#define ORC_SPRING_IT 0xFFFFFFFFu

int orc_spring_table(int64_t G, const double* cmax, uint64_t* q, double* scale) {
  double mx = 0.0;
  for (int64_t c = 0; c < G; ++c)
    if (cmax[c] > mx) mx = cmax[c];
  if (!(mx > 0.0) || !isfinite(mx)) return -1;
  *scale = 16777216.0 / mx; /* 2^24 / max M */
  for (int64_t c = 0; c < G; ++c) {
    double v = cmax[c] > 0.0 ? ceil(cmax[c] * *scale) : 0.0;
    q[c] = (uint64_t)v;
  }
  return 0;
}

/* floor(U Q / 2^64) in 64-bit pieces: U Q = (Uh 2^32 + Ul)(Qh 2^32 + Ql). */
static uint64_t mul_hi64(uint64_t U, uint64_t Q) {
  uint64_t Uh = U >> 32, Ul = U & 0xFFFFFFFFull;
  uint64_t Qh = Q >> 32, Ql = Q & 0xFFFFFFFFull;
  uint64_t ll = Ul * Ql, lh = Ul * Qh, hl = Uh * Ql, hh = Uh * Qh;
  uint64_t mid = (ll >> 32) + (lh & 0xFFFFFFFFull) + (hl & 0xFFFFFFFFull);
  return hh + (lh >> 32) + (hl >> 32) + (mid >> 32);
}

int orc_spring(const orc_cfg* cfg, const orc_fn* fn, const double* edges,
               const double* cmax, uint64_t t0, int64_t n, double* x_out,
               uint64_t* trial_out, int64_t* n_events, int64_t* overflow,
               int64_t* nonpos) {
  if (!cfg_valid(cfg) || !fn_valid(fn) || fn->ndim != cfg->ndim) return -1;
  if (n < 0 || t0 + (uint64_t)n > 0x100000000ull) return -1;
  int d = cfg->ndim, W = words_per_sample(cfg), V = cfg->ybits == 24 ? 1 : 2;
  int64_t G = n_cubes(cfg);
  if (G < 0) return -1;
  uint64_t* q = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)G);
  uint64_t* P = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(G + 1));
  if (!q || !P) {
    free(q);
    free(P);
    return -1;
  }
  double scale;
  if (orc_spring_table(G, cmax, q, &scale)) {
    free(q);
    free(P);
    return -1;
  }
  P[0] = 0;
  for (int64_t c = 0; c < G; ++c) P[c + 1] = P[c] + q[c];
  uint64_t Q = P[G];
  uint32_t key[2] = {(uint32_t)cfg->seed, (uint32_t)(cfg->seed >> 32)};
  uint32_t w[2 * ORC_MAXDIM + 8];
  int nw = W + 2 + V;
  int64_t k = 0, ov = 0, np = 0;
  double x[ORC_MAXDIM], J;
  for (int64_t i = 0; i < n; ++i) {
    uint64_t t = t0 + (uint64_t)i;
    for (int g4 = 0; 4 * g4 < nw; ++g4) {
      uint32_t ctr[4] = {(uint32_t)t, (uint32_t)g4, ORC_SPRING_IT, cfg->instance};
      uint32_t out[4];
      orc_philox4x32_10(ctr, key, out);
      for (int r = 0; r < 4 && 4 * g4 + r < nw; ++r) w[4 * g4 + r] = out[r];
    }
    /* the cube: the last c with P[c] <= u, by bisection over P[0..G] */
    uint64_t U = ((uint64_t)w[W] << 32) | (uint64_t)w[W + 1];
    uint64_t u = mul_hi64(U, Q);
    int64_t lo = 0, hi = G; /* P[lo] <= u < P[hi] */
    while (hi - lo > 1) {
      int64_t mid = lo + (hi - lo) / 2;
      if (P[mid] <= u)
        lo = mid;
      else
        hi = mid;
    }
    int64_t c = lo;
    orc_point_from_words(cfg, edges, (uint64_t)c, w, NULL, NULL, x, &J);
    double f = eval_point(fn, x, NULL);
    double wt = f * J;
    double v = V == 1 ? (double)(w[W + 2] >> 8) / 16777216.0
                      : ((double)(w[W + 2] >> 5) * 67108864.0 + (double)(w[W + 3] >> 6)) /
                            9007199254740992.0;
    double Mt = (double)q[c] / scale;
    int keep;
    if (!(wt > 0.0)) {
      ++np;
      keep = 0;
    } else if (wt > Mt) {
      ++ov;
      keep = 1;
    } else {
      keep = v * Mt < wt;
    }
    if (keep) {
      if (x_out)
        for (int a = 0; a < d; ++a) x_out[(size_t)k * d + a] = x[a];
      if (trial_out) trial_out[k] = t;
      ++k;
    }
  }
  free(q);
  free(P);
  *n_events = k;
  if (overflow) *overflow = ov;
  if (nonpos) *nonpos = np;
  return 0;
}

/* Gradient of the iteration estimate with respect to integrand
 * parameters on a frozen grid and fixed random numbers:
 * dI/dtheta = (1/NCALL) sum_s J_s df/dtheta(x_s).  With equal samples per
 * hypercube the stratified estimate has the same form. */
int orc_gradient(const orc_cfg* cfg, const orc_fn* fn, const double* edges,
                 uint32_t it, double* grad, double* I) {
  if (!cfg_valid(cfg) || !fn_valid(fn) || fn->ndim != cfg->ndim) return -1;
  int nt = orc_ntheta(fn);
  if (nt == 0) return -1;
  int64_t G = n_cubes(cfg);
  if (G < 0 || cfg->ncall % G != 0) return -1;
  ksum* kg = (ksum*)calloc((size_t)nt, sizeof(ksum));
  double* g = (double*)malloc(sizeof(double) * (size_t)nt);
  if (!kg || !g) {
    free(kg);
    free(g);
    return -1;
  }
  ksum kI = {0, 0};
  double x[ORC_MAXDIM], J;
  for (int64_t s = 0; s < cfg->ncall; ++s) {
    orc_sample_point(cfg, edges, it, (uint64_t)s, NULL, NULL, x, &J);
    double f = eval_point(fn, x, g);
    double w = f * J;
    if (isfinite(w)) kadd(&kI, w);
    for (int t = 0; t < nt; ++t)
      if (isfinite(g[t] * J)) kadd(&kg[t], g[t] * J);
  }
  for (int t = 0; t < nt; ++t) grad[t] = kval(&kg[t]) / (double)cfg->ncall;
  if (I) *I = kval(&kI) / (double)cfg->ncall;
  free(kg);
  free(g);
  return 0;
}
