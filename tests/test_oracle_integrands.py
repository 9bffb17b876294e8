"""Pins of the oracle's integrands (step 3) against closed forms, by tensor
Gauss-Legendre quadrature at d <= 3 and by separability."""
import math

import numpy as np
import pytest

import closed_forms as cf


def _quad(orc, fn, d, nodes=12, intervals=40):
    X, W = cf.gauss_legendre_tensor(d, nodes, intervals)
    return float(np.sum(W * orc.integrand(fn, X)))


@pytest.mark.parametrize("d", [1, 2, 3])
def test_genz_gaussian_quadrature(orc, d):
    rng = np.random.default_rng(d)
    a = rng.uniform(2, 12, d)
    u = rng.uniform(0.1, 0.9, d)
    fn = orc.Integrand(orc.GENZ_GAUSSIAN, d, np.concatenate([a, u]))
    iv = 60 if d < 3 else 24
    assert _quad(orc, fn, d, 10, iv) == pytest.approx(cf.genz_gaussian(a, u), rel=1e-10)


def test_genz_gaussian_config_value_and_separability(orc):
    """The d=4 workload: f(x) = prod_i f_1(x_i) (so its integral is the 4th
    power of the 1-D one, pinned by quadrature above) and the closed form
    (sqrt(pi)/10 erf 5)^4 = 9.8696044010286631e-4."""
    a, u = [10.0] * 4, [0.5] * 4
    assert cf.genz_gaussian(a, u) == pytest.approx(9.8696044010286631e-4, rel=1e-15)
    f4 = orc.Integrand(orc.GENZ_GAUSSIAN, 4, a + u)
    f1 = orc.Integrand(orc.GENZ_GAUSSIAN, 1, [10.0, 0.5])
    X = np.random.default_rng(0).random((500, 4))
    prod = np.prod(np.stack([orc.integrand(f1, X[:, i]) for i in range(4)], 1), 1)
    np.testing.assert_allclose(orc.integrand(f4, X), prod, rtol=1e-13, atol=1e-300)
    one = orc.Integrand(orc.GENZ_GAUSSIAN, 1, [10.0, 0.5])
    assert _quad(orc, one, 1, 10, 100) ** 4 == pytest.approx(9.8696044010286631e-4, rel=1e-12)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_genz_product_peak_quadrature(orc, d):
    rng = np.random.default_rng(10 + d)
    a = rng.uniform(1, 6, d)
    u = rng.uniform(0, 1, d)
    fn = orc.Integrand(orc.GENZ_PRODUCT_PEAK, d, np.concatenate([a, u]))
    assert _quad(orc, fn, d, 10, 20) == pytest.approx(cf.genz_product_peak(a, u), rel=1e-10)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_genz_corner_peak_quadrature(orc, d):
    rng = np.random.default_rng(20 + d)
    a = rng.uniform(0.2, 1.5, d)
    fn = orc.Integrand(orc.GENZ_CORNER_PEAK, d, a)
    assert _quad(orc, fn, d, 10, 8) == pytest.approx(cf.genz_corner_peak(a), rel=1e-11)


def test_genz_corner_peak_closed_form_d1():
    """d = 1: int (1+ax)^-2 = 1/(1+a), a check of the inclusion-exclusion sum."""
    for a in (0.3, 1.85, 7.0):
        assert cf.genz_corner_peak([a]) == pytest.approx(1 / (1 + a), rel=1e-15)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_genz_oscillatory_quadrature(orc, d):
    rng = np.random.default_rng(30 + d)
    a = rng.uniform(0.5, 4.0, d)
    u1 = rng.random()
    fn = orc.Integrand(orc.GENZ_OSCILLATORY, d, np.concatenate([a, [u1]]))
    got = _quad(orc, fn, d, 10, 8)
    assert abs(got - cf.genz_oscillatory(a, u1)) < 1e-12


@pytest.mark.parametrize("d", [1, 2, 3])
def test_genz_continuous_quadrature(orc, d):
    """Kinks at u_i: a rule whose pieces end there integrates each smooth
    piece to rounding, against the closed form."""
    rng = np.random.default_rng(40 + d)
    a = rng.uniform(1, 8, d)
    u = rng.uniform(0.1, 0.9, d)
    fn = orc.Integrand(orc.GENZ_CONTINUOUS, d, np.concatenate([a, u]))
    n = 16 if d < 3 else 8
    X, W = cf.tensor_rule([cf.gauss_legendre_split([u[i]], n, 4) for i in range(d)])
    assert float(np.sum(W * orc.integrand(fn, X))) == pytest.approx(cf.genz_continuous(a, u), rel=1e-12)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_genz_discontinuous_quadrature(orc, d):
    """Jumps at u_1 (and u_2): rules with pieces ending there; the integrand
    is zero beyond them and exp(sum a_i x_i) before."""
    rng = np.random.default_rng(50 + d)
    a = rng.uniform(0.5, 4, d)
    u = rng.uniform(0.2, 0.8, min(d, 2))
    fn = orc.Integrand(orc.GENZ_DISCONTINUOUS, d, np.concatenate([a, u]))
    n = 16 if d < 3 else 8
    X, W = cf.tensor_rule([cf.gauss_legendre_split([u[i]] if i < 2 else [], n, 4) for i in range(d)])
    assert float(np.sum(W * orc.integrand(fn, X))) == pytest.approx(cf.genz_discontinuous(a, u), rel=1e-12)


def test_genz_discontinuous_edges_and_separability(orc):
    a, u = np.array([1.5, 2.0, 0.7]), np.array([0.4, 0.6])
    fn = orc.Integrand(orc.GENZ_DISCONTINUOUS, 3, np.concatenate([a, u]))
    x = np.array([[0.4, 0.6, 0.3], [0.4000001, 0.1, 0.1], [0.1, 0.6000001, 0.9], [0.1, 0.2, 0.99]])
    f = orc.integrand(fn, x)
    assert f[0] == pytest.approx(math.exp(a @ x[0]), rel=1e-15)  # the boundary point belongs to the region
    assert f[1] == 0.0 and f[2] == 0.0
    assert f[3] == pytest.approx(math.exp(a @ x[3]), rel=1e-15)
    fc = orc.Integrand(orc.GENZ_CONTINUOUS, 3, np.concatenate([a, [0.3, 0.5, 0.7]]))
    X = np.random.default_rng(0).random((200, 3))
    one = [orc.Integrand(orc.GENZ_CONTINUOUS, 1, [a[i], [0.3, 0.5, 0.7][i]]) for i in range(3)]
    prod = np.prod(np.stack([orc.integrand(one[i], X[:, i]) for i in range(3)], 1), 1)
    np.testing.assert_allclose(orc.integrand(fc, X), prod, rtol=1e-14)


@pytest.mark.parametrize("d", [1, 2])
def test_double_gaussian_quadrature(orc, d):
    c1, c2, w = 1 / 3, 2 / 3, 0.05
    fn = orc.Integrand(orc.DOUBLE_GAUSSIAN, d, [c1, c2, w])
    got = _quad(orc, fn, d, 10, 150 if d == 1 else 60)
    assert got == pytest.approx(cf.double_gaussian(c1, c2, w, d), rel=1e-10)
    # shifted centres make the erf tails visible
    fn2 = orc.Integrand(orc.DOUBLE_GAUSSIAN, d, [0.05, 0.9, 0.1])
    got2 = _quad(orc, fn2, d, 10, 150 if d == 1 else 60)
    assert got2 == pytest.approx(cf.double_gaussian(0.05, 0.9, 0.1, d), rel=1e-10)


def test_double_gaussian_d8_normalisation():
    """With centres 1/3, 2/3 and width 0.05 the erf tails are below 1e-20, so
    the normalised two-peak integral is 1 to double precision."""
    assert cf.double_gaussian(1 / 3, 2 / 3, 0.05, 8) == pytest.approx(1.0, abs=1e-15)
    assert 0.5 * sum((0.05 * math.sqrt(math.pi) / 2 * (math.erf((1 - c) / 0.05) + math.erf(c / 0.05))) ** 8
                     for c in (1 / 3, 2 / 3)) == pytest.approx(3.8050426185157195e-9, rel=1e-13)


@pytest.mark.parametrize("kind,extra", [(0, "gauss"), (4, "dgauss")])
def test_gradients_match_finite_differences(orc, kind, extra):
    """Pointwise df/dtheta against central differences of f in theta."""
    rng = np.random.default_rng(40 + kind)
    d = 3
    if kind == 0:
        theta = np.concatenate([rng.uniform(2, 5, d), rng.uniform(0.3, 0.7, d)])

        def params(t):
            return np.concatenate([t[d:], t[:d]])  # theta = (u, a); params = (a, u)
        t0 = np.concatenate([theta[d:], theta[:d]])
    else:
        t0 = np.array([0.3, 0.6, 0.2])

        def params(t):
            return t
    X = rng.random((50, d))
    fn = orc.Integrand(kind, d, params(t0))
    g = orc.integrand_grad(fn, X)
    for j in range(len(t0)):
        h = 1e-6
        tp, tm = t0.copy(), t0.copy()
        tp[j] += h
        tm[j] -= h
        fd = (orc.integrand(orc.Integrand(kind, d, params(tp)), X)
              - orc.integrand(orc.Integrand(kind, d, params(tm)), X)) / (2 * h)
        np.testing.assert_allclose(g[:, j], fd, rtol=2e-6, atol=1e-9 * np.max(np.abs(fd)) + 1e-300)


def test_gaussian_gradient_quadrature_matches_closed_form_derivative(orc):
    """int df/du and int df/da by quadrature equal the derivatives of the erf
    closed form (central differences of the closed form)."""
    d = 2
    a = np.array([4.0, 7.0])
    u = np.array([0.4, 0.65])
    fn = orc.Integrand(orc.GENZ_GAUSSIAN, d, np.concatenate([a, u]))
    X, W = cf.gauss_legendre_tensor(d, 10, 40)
    g = orc.integrand_grad(fn, X)
    q = W @ g
    h = 1e-6
    for i in range(d):
        up, um = u.copy(), u.copy()
        up[i] += h
        um[i] -= h
        assert q[i] == pytest.approx((cf.genz_gaussian(a, up) - cf.genz_gaussian(a, um)) / (2 * h), rel=1e-6)
        ap, am = a.copy(), a.copy()
        ap[i] += h
        am[i] -= h
        assert q[d + i] == pytest.approx((cf.genz_gaussian(ap, u) - cf.genz_gaussian(am, u)) / (2 * h), rel=1e-6)
