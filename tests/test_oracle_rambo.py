"""Pins of the oracle's RAMBO phase space (Kleiss, Stirling, Ellis 1986) and of
the W-like integrand built on it (Breit-Wigner in s12, cyclic 1/s_{i,i+1},
pT and Delta R cuts after eqs. 2-3 of Sec. 4)."""
import math

import numpy as np
import pytest

import closed_forms as cf
from paper_1010_2107_gb300 import workloads as wl

SQRTS = 1000.0


def test_volume_closed_form(orc):
    assert orc.rambo_volume(5, SQRTS) == pytest.approx(4.227825132e16, rel=1e-9)
    assert orc.rambo_volume(4, SQRTS) == pytest.approx(3.229820488e11, rel=1e-9)
    for n in (2, 3, 4, 5, 6):
        assert orc.rambo_volume(n, SQRTS) == pytest.approx(cf.rambo_volume(n, SQRTS), rel=1e-14)
    # two-body massless phase space volume is pi/2 (no 2 pi factors)
    assert orc.rambo_volume(2, 91.0) == pytest.approx(math.pi / 2, rel=1e-15)


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_momentum_conservation_and_masslessness(orc, n):
    rng = np.random.default_rng(n)
    for _ in range(200):
        rho = rng.random(4 * n)
        p = orc.rambo(n, SQRTS, rho)
        tot = p.sum(0)
        assert abs(tot[0] - SQRTS) < 1e-12 * SQRTS
        assert np.all(np.abs(tot[1:]) < 1e-12 * SQRTS)
        m2 = p[:, 0] ** 2 - np.sum(p[:, 1:] ** 2, 1)
        assert np.all(np.abs(m2) < 1e-11 * p[:, 0] ** 2 + 1e-9)
        assert np.all(p[:, 0] > 0)


def _fn(orc, n, **kw):
    return orc.Integrand(orc.RAMBO_BW, 4 * n, wl.rambo_params(n, **kw))


def test_unit_observable_gives_volume_with_zero_variance(orc):
    """f = 1 with no cuts: every weight is V_n at the uniform grid, so the
    iteration estimate is V_n with zero variance."""
    n = 5
    fn = _fn(orc, n, obs=1)
    cfg = orc.make_cfg(4 * n, nbins=50, ncall=4096, ybits=24)
    r = orc.iteration(cfg, fn, orc.uniform_grid(4 * n, 50), 0)
    V = cf.rambo_volume(n, SQRTS)
    assert r["I"] == pytest.approx(V, rel=1e-13)
    assert r["var"] <= (1e-13 * V) ** 2


@pytest.mark.parametrize("n", [3, 4, 5])
def test_mean_s12(orc, n):
    """sum_{i<j} s_ij = s and all pairs are equivalent, so <s12> = 2 s/(n(n-1))."""
    fn = _fn(orc, n, obs=2)
    cfg = orc.make_cfg(4 * n, nbins=50, ncall=1 << 16, ybits=53, seed=3)
    r = orc.iteration(cfg, fn, orc.uniform_grid(4 * n, 50), 0)
    V = cf.rambo_volume(n, SQRTS)
    mean, sig = r["I"] / V, math.sqrt(r["var"]) / V
    exact = 2 * SQRTS ** 2 / (n * (n - 1))
    assert abs(mean - exact) < 5 * sig
    assert sig < 0.02 * exact
    # the closed-form density reproduces the same mean
    assert cf.s12_density_moment(n, lambda x: x, npts=300) == pytest.approx(2 / (n * (n - 1)), rel=1e-6)


@pytest.mark.parametrize("n", [4, 5])
def test_breit_wigner_moment_against_s12_density(orc, n):
    """<BW(s12)> over flat phase space equals int rho(x) BW(x s) dx with the
    factorised s12 density; a wide resonance keeps the Monte Carlo error small."""
    M, G = 300.0, 150.0
    fn = _fn(orc, n, obs=3, M=M, Gamma=G)
    cfg = orc.make_cfg(4 * n, nbins=50, ncall=1 << 17, ybits=24, seed=5)
    r = orc.iteration(cfg, fn, orc.uniform_grid(4 * n, 50), 0)
    V = cf.rambo_volume(n, SQRTS)
    mean, sig = r["I"] / V, math.sqrt(r["var"]) / V
    s = SQRTS ** 2
    exact = cf.s12_density_moment(n, lambda x: M * G / ((x * s - M * M) ** 2 + M * M * G * G), npts=600)
    assert abs(mean - exact) < 5 * sig
    assert sig < 0.03 * exact


def _mom(pt, eta, phi):
    return np.array([[p * math.cosh(e), p * math.cos(f), p * math.sin(f), p * math.sinh(e)]
                     for p, e, f in zip(pt, eta, phi)])


BASE = dict(pt=[60.0, 45.0, 80.0, 30.0], eta=[0.3, -1.2, 2.0, -0.1], phi=[0.2, 2.0, -2.5, 1.1])


def test_hand_built_cut_cases(orc):
    """Hard cuts: every parton needs pT > 20 GeV and every pair Delta R > 0.4,
    with Delta phi taken across the +-pi branch cut."""
    P = wl.rambo_params(4, cut=0)
    assert orc.rambo_f_momenta(P, _mom(**BASE)) > 0
    for ptv, expect in ((19.9, False), (20.1, True)):
        b = {k: list(v) for k, v in BASE.items()}
        b["pt"][3] = ptv
        assert (orc.rambo_f_momenta(P, _mom(**b)) > 0) == expect
    for deta, expect in ((0.39, False), (0.41, True)):
        b = {k: list(v) for k, v in BASE.items()}
        b["eta"][1] = b["eta"][0] + deta
        b["phi"][1] = b["phi"][0]
        assert (orc.rambo_f_momenta(P, _mom(**b)) > 0) == expect
    # phi = pi - 0.1 and -pi + 0.1 are 0.2 apart, not 2 pi - 0.2
    b = {k: list(v) for k, v in BASE.items()}
    b["phi"][0], b["phi"][2] = math.pi - 0.1, -math.pi + 0.1
    b["eta"][2] = b["eta"][0] + 0.3
    assert orc.rambo_f_momenta(P, _mom(**b)) == 0.0
    b["eta"][2] = b["eta"][0] + 0.4
    assert orc.rambo_f_momenta(P, _mom(**b)) > 0
    # no cuts: soft partons pass
    b = {k: list(v) for k, v in BASE.items()}
    b["pt"][0] = 1.0
    assert orc.rambo_f_momenta(wl.rambo_params(4, cut=2), _mom(**b)) > 0


def test_cyclic_product_and_breit_wigner(orc):
    """Without cuts f = BW(s_12) prod_i 1/s_{i,i+1 mod n}: each s_ij is built
    from the construction's own (pT, eta, phi): s_ij = 2 pT_i pT_j (cosh deta - cos dphi)."""
    pt, eta, phi = BASE["pt"], BASE["eta"], BASE["phi"]
    n = 4

    def s(i, j):
        return 2 * pt[i] * pt[j] * (math.cosh(eta[i] - eta[j]) - math.cos(phi[i] - phi[j]))
    M, G = 80.4, 2.1
    bw = M * G / ((s(0, 1) - M * M) ** 2 + M * M * G * G)
    expect = bw / (s(0, 1) * s(1, 2) * s(2, 3) * s(3, 0))
    got = orc.rambo_f_momenta(wl.rambo_params(n, cut=2), _mom(pt, eta, phi))
    assert got == pytest.approx(expect, rel=1e-12)
    assert orc.rambo_f_momenta(wl.rambo_params(n, cut=2, obs=2), _mom(pt, eta, phi)) == pytest.approx(s(0, 1), rel=1e-13)


def _boost(p, beta, axis):
    g = 1 / math.sqrt(1 - beta ** 2)
    q = p.copy()
    q[:, 0] = g * (p[:, 0] + beta * p[:, axis])
    q[:, axis] = g * (p[:, axis] + beta * p[:, 0])
    return q


def _rotz(p, ang):
    q = p.copy()
    c, s = math.cos(ang), math.sin(ang)
    q[:, 1] = c * p[:, 1] - s * p[:, 2]
    q[:, 2] = s * p[:, 1] + c * p[:, 2]
    return q


@pytest.mark.parametrize("cut", [0, 1])
def test_longitudinal_invariance(orc, cut):
    """pT, Delta eta, Delta phi and s_ij are unchanged by z boosts and
    rotations about z, so the integrand with cuts is too."""
    rng = np.random.default_rng(cut)
    P = wl.rambo_params(5, cut=cut)
    hits = 0
    for _ in range(300):
        p = orc.rambo(5, SQRTS, rng.random(20))
        f0 = orc.rambo_f_momenta(P, p)
        if f0 > 0:
            hits += 1
        for q in (_boost(p, 0.6, 3), _boost(p, -0.9, 3), _rotz(p, 2.7), _rotz(p, -1.3)):
            assert orc.rambo_f_momenta(P, q) == pytest.approx(f0, rel=1e-9, abs=0)
    assert hits > 20


def test_lorentz_invariance_without_cuts(orc):
    """Without cuts the integrand depends on invariants only: arbitrary boosts
    leave it unchanged."""
    rng = np.random.default_rng(9)
    P = wl.rambo_params(5, cut=2)
    for _ in range(100):
        p = orc.rambo(5, SQRTS, rng.random(20))
        f0 = orc.rambo_f_momenta(P, p)
        q = _boost(_rotz(_boost(p, 0.5, 1), 0.7), -0.3, 2)
        assert orc.rambo_f_momenta(P, q) == pytest.approx(f0, rel=1e-8)


def test_rambo_gradient_matches_finite_differences(orc):
    """df/d(M, Gamma, T) with the sigmoid cut against central differences."""
    rng = np.random.default_rng(12)
    n = 4
    base = dict(cut=1)
    X = rng.random((400, 4 * n))
    g = orc.integrand_grad(_fn(orc, n, **base), X)
    f0 = orc.integrand(_fn(orc, n, **base), X)
    assert np.count_nonzero(f0) > 20
    for j, (name, h) in enumerate((("M", 1e-4), ("Gamma", 1e-5), ("T", 1e-4))):
        kp, km = dict(base), dict(base)
        kp[name] = dict(M=80.4, Gamma=2.1, T=20.0)[name] + h
        km[name] = dict(M=80.4, Gamma=2.1, T=20.0)[name] - h
        fd = (orc.integrand(_fn(orc, n, **kp), X) - orc.integrand(_fn(orc, n, **km), X)) / (2 * h)
        scale = np.max(np.abs(fd))
        np.testing.assert_allclose(g[:, j], fd, rtol=1e-5, atol=1e-7 * scale)


def test_zero_random_number_gives_zero_weight(orc):
    """A point with rho_1 rho_2 = 0 would give an infinite energy: it carries
    zero weight (a set of measure zero)."""
    n = 4
    x = np.full(4 * n, 0.5)
    x[4] = 0.0
    assert orc.integrand(_fn(orc, n, cut=2), x)[0] == 0.0


@pytest.mark.parametrize("cut", [0, 1])
def test_two_body_integrand_against_its_closed_form(orc, cut):
    """n = 2 pins the whole RAMBO integrand, cuts included: the partons are
    back to back with s12 = s21 = s and cos(theta) uniform, so
    f = V_2 cut BW(s) / s^2 with V_2 = pi/2, both transverse momenta equal
    (sqrt(s)/2) sin(theta), and Delta R >= pi passes any Delta R cut.  Hard
    cut: the mean of the cut is sqrt(1 - (2 ptmin / sqrt s)^2); sigmoid cut:
    the mean of sigmoid((pT - T)/w)^2 over cos(theta), by quadrature."""
    from scipy import integrate
    s = SQRTS ** 2
    p = wl.rambo_params(2, cut=cut, ptmin=150.0, T=150.0, wc=20.0)
    M, G = p[wl.RB_M], p[wl.RB_GAMMA]
    bw = M * G / ((s - M * M) ** 2 + M * M * G * G)
    if cut == 0:
        acc = math.sqrt(1.0 - (2.0 * p[wl.RB_PTMIN] / SQRTS) ** 2)
    else:
        sig = lambda c: 1.0 / (1.0 + math.exp(-((SQRTS / 2) * math.sqrt(1 - c * c) - p[wl.RB_T]) / p[wl.RB_WC]))
        acc = 0.5 * integrate.quad(lambda c: sig(c) ** 2, -1.0, 1.0, epsabs=0, epsrel=1e-12, limit=200)[0]
    expect = math.pi / 2 * bw / s ** 2 * acc
    fn = orc.Integrand(orc.RAMBO_BW, 8, p)
    cfg = orc.make_cfg(8, nbins=50, ncall=1 << 18, ybits=53, seed=11)
    r = orc.iteration(cfg, fn, orc.uniform_grid(8, 50), 0)
    assert abs(r["I"] - expect) < 5.0 * math.sqrt(r["var"])
    assert math.sqrt(r["var"]) < 0.01 * expect
