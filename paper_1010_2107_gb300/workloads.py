"""Seeded synthetic workloads: shapes, sizes and integrand parameter vectors.

This module holds no arithmetic of the integration method.  It only states the
workloads (sizes, seeds, parameter vectors) and draws the parameters of the
batched Genz workload from numpy's PCG64 generator.  Both the CUDA library's
callers and the CPU oracle's tests take their inputs from here.

Workloads (after Sec. 5.1's conventions: NCALL points per iteration, ITMX
iterations, BASES split ITMX1 = ITMX2 with ITMX1 + ITMX2 = ITMX):

* ``gauss4``   VEGAS, FP64, d=4 Genz Gaussian exp(-sum 100 (x_i - 0.5)^2),
               50 bins, 5 iterations x 1e5 points, seed 1.
* ``dgauss8``  BASES, hypercube-stratified (4 divisions per axis, 65 536 cubes
               x 64 points), FP32 integrand, d=8 two-peak Gaussian (centres
               1/3 and 2/3, width 0.05), 50 bins, 5 + 5 iterations x 2^22.
* ``rambo5``   VEGAS on massless 2->5 RAMBO phase space at sqrt(s) = 1 TeV
               (20 dims), cyclic 1/s_{i,i+1} x Breit-Wigner(s12), pT > 20 GeV
               and Delta R > 0.4 cuts, FP32, 12 iterations x 2^24.
* ``rambo4_adjoint``  2->4 RAMBO (16 dims), sigmoid pT cut (T = 20 GeV,
               width 1 GeV); gradient in (M, Gamma, T) on 2^24 points after a
               5-iteration grid warm-up.
* ``user_dgauss8``  ``dgauss8`` with the integrand given as CUDA source
               (``DGAUSS_USER_SOURCE``) and compiled at run time.
* ``wmunu``    BASES, hypercube-stratified (8 divisions per axis, 32 768 cubes
               x 128 points), FP32, u dbar -> W+ -> mu+ nu at sqrt(S) = 14 TeV
               with the mu+ cuts (5 dims), 32 bins, 5 + 5 iterations x 2^22.
* ``genz256``  256 Genz integrands (product peak, corner peak, oscillatory),
               d uniform in 2..16, points per instance log-uniform in
               2^16..2^22, 8 iterations each.
"""
from __future__ import annotations

import math

import numpy as np

# Integrand kinds, in the numbering of include/gvegas.h.
GENZ_GAUSSIAN = 0
GENZ_PRODUCT_PEAK = 1
GENZ_CORNER_PEAK = 2
GENZ_OSCILLATORY = 3
DOUBLE_GAUSSIAN = 4
RAMBO_BW = 5
GENZ_CONTINUOUS = 6
GENZ_DISCONTINUOUS = 7
W_MUNU = 8
USER = 64  # run-time compiled source

# Parameter slots of RAMBO_BW.
RB_N, RB_SQRTS, RB_M, RB_GAMMA, RB_PTMIN, RB_DRMIN, RB_CUT, RB_T, RB_WC, RB_OBS = range(10)
RB_NPARAMS = 10

# Genz "difficulty" sums sum_i a_i per family (values customary in the
# Genz test-function literature).
GENZ_DIFFICULTY = {GENZ_OSCILLATORY: 9.0, GENZ_PRODUCT_PEAK: 7.25,
                   GENZ_CORNER_PEAK: 1.85}


def genz_gaussian_params(d: int, a: float = 10.0, u: float = 0.5) -> np.ndarray:
    """[a_1..a_d, u_1..u_d] for f = exp(-sum a_i^2 (x_i - u_i)^2)."""
    return np.concatenate([np.full(d, a), np.full(d, u)]).astype(np.float64)


def double_gaussian_params(c1: float = 1.0 / 3.0, c2: float = 2.0 / 3.0,
                           w: float = 0.05) -> np.ndarray:
    return np.array([c1, c2, w], dtype=np.float64)


# Parameter slots of W_MUNU (include/gvegas.h).
(W_SQRTS, W_M, W_GAMMA, W_GF, W_VUD, W_PTMIN, W_ETAMAX, W_SMIN, W_CUTS,
 W_AU, W_ALU, W_BU, W_AD, W_ALD, W_BD) = range(15)
W_NPARAMS = 15


def w_munu_params(sqrt_s: float = 14000.0, M: float = 80.4, Gamma: float = 2.1,
                  GF: float = 1.16639e-5, Vud: float = 0.974, ptmin: float = 20.0,
                  etamax: float = 2.5, smin: float | None = None, cuts: int = 1,
                  u_pdf=(2.0, -0.5, 3.0), dbar_pdf=(0.15, -1.15, 7.0)) -> np.ndarray:
    """u dbar -> W+ -> mu+ nu at the LHC energy of Sec. 5 with the lepton cuts
    of Sec. 4.  The parton densities are a stand-in, A x^a (1 - x)^b for u
    (valence-like) and dbar (sea-like), since no PDF table is available.
    The shat range starts at smin, by default (2 ptmin)^2, below which no
    mu+ passes the pT cut."""
    p = np.zeros(W_NPARAMS)
    p[W_SQRTS], p[W_M], p[W_GAMMA], p[W_GF], p[W_VUD] = sqrt_s, M, Gamma, GF, Vud
    p[W_PTMIN], p[W_ETAMAX], p[W_CUTS] = ptmin, etamax, cuts
    p[W_SMIN] = (2.0 * ptmin) ** 2 if smin is None else smin
    p[W_AU], p[W_ALU], p[W_BU] = u_pdf
    p[W_AD], p[W_ALD], p[W_BD] = dbar_pdf
    return p


# The two-peak Gaussian as a user integrand.  Its parameter vector holds the
# constants the source reads: p = (c1, c2, 1/w^2, (w sqrt(pi))^-d / 2).
DGAUSS_USER_SOURCE = r"""
template <typename T>
__device__ T vegas_user_f(const T* x, int d, const T* p) {
  T q1 = T(0), q2 = T(0);
  for (int i = 0; i < d; ++i) {
    const T t1 = x[i] - p[0], t2 = x[i] - p[1];
    q1 += t1 * t1;
    q2 += t2 * t2;
  }
  return p[3] * (gv::gexp(-q1 * p[2]) + gv::gexp(-q2 * p[2]));
}
"""


def double_gaussian_user_params(d: int = 8, c1: float = 1.0 / 3.0, c2: float = 2.0 / 3.0,
                                w: float = 0.05) -> np.ndarray:
    return np.array([c1, c2, 1.0 / (w * w), 0.5 * (w * math.sqrt(math.pi)) ** (-d)], dtype=np.float64)


def rambo_params(n: int, sqrt_s: float = 1000.0, M: float = 80.4,
                 Gamma: float = 2.1, ptmin: float = 20.0, drmin: float = 0.4,
                 cut: int = 0, T: float = 20.0, wc: float = 1.0,
                 obs: int = 0) -> np.ndarray:
    p = np.zeros(RB_NPARAMS)
    p[RB_N], p[RB_SQRTS], p[RB_M], p[RB_GAMMA] = n, sqrt_s, M, Gamma
    p[RB_PTMIN], p[RB_DRMIN], p[RB_CUT] = ptmin, drmin, cut
    p[RB_T], p[RB_WC], p[RB_OBS] = T, wc, obs
    return p


WORKLOADS = {
    "gauss4": dict(kind=GENZ_GAUSSIAN, ndim=4, params=genz_gaussian_params(4),
                   nbins=50, ncall=100_000, itmx=5, nstrat=0, seed=1,
                   precision="fp64", ybits=53, mode="vegas"),
    "dgauss8": dict(kind=DOUBLE_GAUSSIAN, ndim=8, params=double_gaussian_params(),
                    nbins=50, ncall=1 << 22, itmx1=5, itmx2=5, nstrat=4, seed=1,
                    precision="fp32", ybits=24, mode="bases"),
    "rambo5": dict(kind=RAMBO_BW, ndim=20, params=rambo_params(5), nbins=50,
                   ncall=1 << 24, itmx=12, nstrat=0, seed=1, precision="fp32",
                   ybits=24, mode="vegas"),
    "rambo4_adjoint": dict(kind=RAMBO_BW, ndim=16, params=rambo_params(4, cut=1),
                           nbins=50, ncall=1 << 24, warmup_iters=5, nstrat=0,
                           seed=1, precision="fp32", ybits=24, mode="adjoint"),
    # dgauss8 with the integrand compiled at run time from DGAUSS_USER_SOURCE
    "user_dgauss8": dict(kind=USER, source=DGAUSS_USER_SOURCE, ndim=8, params=double_gaussian_user_params(8),
                         oracle_kind=DOUBLE_GAUSSIAN, oracle_params=double_gaussian_params(),
                         nbins=50, ncall=1 << 22, itmx1=5, itmx2=5, nstrat=4, seed=1,
                         precision="fp32", ybits=24, mode="bases"),
    # the physics workload of Sec. 4 with n = 0 gluons (stand-in densities)
    "wmunu": dict(kind=W_MUNU, ndim=5, params=w_munu_params(), nbins=32, ncall=1 << 22, itmx1=5, itmx2=5,
                  nstrat=8, seed=1, precision="fp32", ybits=24, mode="bases"),
    # SPRING on the dgauss8 BASES run: 2^24 trials per step on its frozen grid
    "spring_dgauss8": dict(kind=DOUBLE_GAUSSIAN, ndim=8, params=double_gaussian_params(),
                           nbins=50, ncall=1 << 22, itmx1=5, itmx2=5, nstrat=4, seed=1,
                           precision="fp32", ybits=24, mode="spring", ntrials=1 << 24),
}


def genz_batch(count: int = 256, seed: int = 2, dmin: int = 2, dmax: int = 16,
               log2n_min: float = 16.0, log2n_max: float = 22.0):
    """Parameters of `count` Genz integrands drawn from PCG64(seed).

    Returns a list of dicts with kind, ndim, ncall and the parameter vector in
    the layout of include/gvegas.h:
      product peak: a[d], u[d];  corner peak: a[d];  oscillatory: a[d], u_1.
    a_i are uniform draws rescaled so that sum_i a_i equals the family's
    difficulty; u_i are uniform in [0, 1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    families = (GENZ_PRODUCT_PEAK, GENZ_CORNER_PEAK, GENZ_OSCILLATORY)
    out = []
    for i in range(count):
        kind = families[int(rng.integers(0, 3))]
        d = int(rng.integers(dmin, dmax + 1))
        n = int(math.floor(2.0 ** (log2n_min + (log2n_max - log2n_min) * rng.random())))
        a = rng.random(d)
        a = a * (GENZ_DIFFICULTY[kind] / a.sum())
        u = rng.random(d)
        if kind == GENZ_PRODUCT_PEAK:
            params = np.concatenate([a, u])
        elif kind == GENZ_CORNER_PEAK:
            params = a.copy()
        else:
            params = np.concatenate([a, u[:1]])
        out.append(dict(instance=i, kind=kind, ndim=d, ncall=n,
                        params=params.astype(np.float64)))
    return out


GENZ256 = dict(count=256, seed=2, nbins=50, itmx=8, sample_seed=1,
               precision="fp32", ybits=24, mode="batched")
