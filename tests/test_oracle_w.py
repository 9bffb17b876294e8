"""Pins of the oracle's u dbar -> W+ -> mu+ nu integrand (Sec. 4, the process
with n = 0 gluons and the mu+ cuts) against what physics and mathematics fix
independently of its code:

* integrated over the mu+ angles and the helicity variable, the integrand is
  the textbook partonic cross section
      sigma(shat) = G_F^2 M^4 |V_ud|^2 shat / (18 pi ((shat - M^2)^2 + M^2 Gamma^2))
  times the parton luminosity and the (shat, y_W) Jacobian;
* integrated over all five variables without cuts, it equals the same cross
  section folded with the densities by direct adaptive quadrature in
  (shat, y_W), with no Breit-Wigner mapping;
* helicity conservation: the right-handed mu+ follows the dbar, so the
  angular shape is (1 - cos theta)^2 against the u direction;
* the cut acceptance at fixed (shat, y_W) is the closed-form integral of
  (1 - c)^2 over the interval the pT and eta cuts leave;
* only one of the 16 helicity combinations contributes; the azimuth drops out.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_1010_2107_gb300 import workloads as wl

from closed_forms import gauss_legendre_split

pytestmark = pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")


def _f(p, y):
    return oracle.integrand(oracle.Integrand(oracle.W_MUNU, 5, p), np.atleast_2d(y))


def _mapping(p, y1, y2):
    """shat, y_W, x1, x2 and dtau/dy1 * dy_W/dy2 from the variable definitions."""
    S = p[wl.W_SQRTS] ** 2
    M, G = p[wl.W_M], p[wl.W_GAMMA]
    lo, hi = math.atan((p[wl.W_SMIN] - M * M) / (M * G)), math.atan((S - M * M) / (M * G))
    rho = lo + (hi - lo) * y1
    shat = M * M + M * G * math.tan(rho)
    tau = shat / S
    L = -math.log(tau)
    yw = (y2 - 0.5) * L
    dtau = (hi - lo) * M * G * (1.0 + math.tan(rho) ** 2) / S
    return shat, yw, math.sqrt(tau) * math.exp(yw), math.sqrt(tau) * math.exp(-yw), dtau * L


def _pdf(A, a, b, x):
    return A * x ** a * (1.0 - x) ** b


def _sigma_hat(p, shat):
    M, G = p[wl.W_M], p[wl.W_GAMMA]
    return (p[wl.W_GF] ** 2 * M ** 4 * p[wl.W_VUD] ** 2 * shat
            / (18.0 * math.pi * ((shat - M * M) ** 2 + M * M * G * G)))


PB = 0.3893793721e9


def _angular_integral(p, y1, y2, c_splits=()):
    """(1/16) sum_h int dy3 f at fixed (y1, y2, y4): Gauss-Legendre in y3 on
    panels split where the cuts act (c = 2 y3 - 1), exact midpoint sum over
    the 16 helicity cells."""
    t, w = gauss_legendre_split([(c + 1.0) / 2.0 for c in c_splits], 12, 2)
    tot = 0.0
    for h in range(16):
        y = np.column_stack([np.full_like(t, y1), np.full_like(t, y2), t,
                             np.full_like(t, 0.3), np.full_like(t, (h + 0.5) / 16.0)])
        tot += np.sum(w * _f(p, y)) / 16.0
    return tot


@pytest.mark.parametrize("y1,y2", [(0.5, 0.5), (0.2, 0.9), (0.97, 0.3), (0.05, 0.1), (0.6, 0.02)])
def test_angular_integral_is_the_partonic_cross_section(y1, y2):
    p = wl.w_munu_params(cuts=0)
    shat, yw, x1, x2, jac = _mapping(p, y1, y2)
    ref = (_pdf(p[wl.W_AU], p[wl.W_ALU], p[wl.W_BU], x1) * _pdf(p[wl.W_AD], p[wl.W_ALD], p[wl.W_BD], x2)
           * jac * _sigma_hat(p, shat) * PB)
    got = _angular_integral(p, y1, y2)
    assert got == pytest.approx(ref, rel=1e-12)


def test_total_without_cuts_matches_direct_quadrature():
    """The Breit-Wigner and rapidity mappings against plain quadrature in
    (shat, y_W): sigma = int dshat / S int dy f_u(x1) f_dbar(x2) sigma(shat)."""
    p = wl.w_munu_params(cuts=0, smin=400.0, sqrt_s=2000.0)
    S, M = p[wl.W_SQRTS] ** 2, p[wl.W_M]

    def inner(shat):
        tau = shat / S
        h = -0.5 * math.log(tau)
        g = lambda yw: (_pdf(p[wl.W_AU], p[wl.W_ALU], p[wl.W_BU], math.sqrt(tau) * math.exp(yw))
                        * _pdf(p[wl.W_AD], p[wl.W_ALD], p[wl.W_BD], math.sqrt(tau) * math.exp(-yw)))
        return integrate.quad(g, -h, h, epsabs=0, epsrel=1e-12, limit=200)[0] * _sigma_hat(p, shat) / S

    direct = integrate.quad(inner, p[wl.W_SMIN], S, points=[M * M], epsabs=0, epsrel=1e-11, limit=400)[0] * PB
    # the oracle over [0,1]^5: Gauss-Legendre panels in y1 (geometric at both
    # ends, where the tan mapping compresses the off-peak shat range) and y2,
    # exact in y3 (a quadratic), y4 (absent) and y5 (16 cells)
    t1, w1 = gauss_legendre_split([10.0 ** -j for j in range(1, 7)] + [1 - 10.0 ** -j for j in range(1, 7)], 12, 4)
    t2, w2 = gauss_legendre_split([], 12, 8)
    c = np.array([-math.sqrt(3 / 5), 0.0, math.sqrt(3 / 5)])
    wc = np.array([5 / 9, 8 / 9, 5 / 9])
    Y1, Y2, C, H = np.meshgrid(t1, t2, c, np.arange(16), indexing="ij")
    W = (w1[:, None, None, None] * w2[None, :, None, None] * wc[None, None, :, None] / 2.0 / 16.0
         * np.ones_like(H))
    y = np.column_stack([Y1.ravel(), Y2.ravel(), (C.ravel() + 1) / 2, np.full(Y1.size, 0.7),
                         (H.ravel() + 0.5) / 16])
    got = float(np.sum(W.ravel() * _f(p, y)))
    assert got == pytest.approx(direct, rel=1e-12)


def test_mu_plus_follows_the_dbar():
    """(1 - cos theta)^2 against the u direction, from helicity conservation:
    u(-) dbar(+) carry J_z = -1 along the u; nu(-) mu+(+) along the nu
    direction as well, so the amplitude is d^1_{-1,-1} = (1 + cos theta_nu) / 2."""
    p = wl.w_munu_params(cuts=0)
    h = 10.5 / 16
    for c1, c2 in [(0.5, -0.5), (0.9, -0.2), (-0.99, 0.0)]:
        f1, f2 = _f(p, [0.5, 0.5, (c1 + 1) / 2, 0.1, h])[0], _f(p, [0.5, 0.5, (c2 + 1) / 2, 0.1, h])[0]
        assert f1 / f2 == pytest.approx(((1 - c1) / (1 - c2)) ** 2, rel=1e-13)


@pytest.mark.parametrize("y1,y2", [(0.5, 0.5), (0.5, 0.85), (0.5, 0.1), (0.03, 0.5), (0.8, 0.95), (0.3, 0.7)])
def test_cut_acceptance_is_the_closed_form(y1, y2):
    p = wl.w_munu_params(cuts=1)
    q = wl.w_munu_params(cuts=0)
    shat, yw, *_ = _mapping(p, y1, y2)
    eta, ptmin = p[wl.W_ETAMAX], p[wl.W_PTMIN]
    cpt = math.sqrt(max(0.0, 1.0 - 4.0 * ptmin ** 2 / shat))
    lo, hi = max(-cpt, math.tanh(-eta - yw)), min(cpt, math.tanh(eta - yw))
    frac = max(0.0, ((1 - lo) ** 3 - (1 - hi) ** 3) / 8.0) if hi > lo else 0.0
    full = _angular_integral(q, y1, y2)
    got = _angular_integral(p, y1, y2, c_splits=(lo, hi))
    assert got == pytest.approx(frac * full, rel=1e-12, abs=1e-300)


def test_one_helicity_and_no_azimuth():
    p = wl.w_munu_params()
    rng = np.random.default_rng(5)
    y = rng.random((2000, 5))
    f = _f(p, y)
    h = np.minimum((16 * y[:, 4]).astype(int), 15)
    assert np.all(f[h != 10] == 0.0) and np.any(f[h == 10] > 0.0)
    y2 = y.copy()
    y2[:, 3] = rng.random(len(y))
    np.testing.assert_array_equal(_f(p, y2), f)


def test_wrong_dimension_or_parameter_count_is_rejected():
    p = wl.w_munu_params()
    with pytest.raises(ValueError):
        oracle.integrand(oracle.Integrand(oracle.W_MUNU, 4, p), np.full((1, 4), 0.5))
    with pytest.raises(ValueError):
        oracle.integrand(oracle.Integrand(oracle.W_MUNU, 5, p[:-1]), np.full((1, 5), 0.5))
