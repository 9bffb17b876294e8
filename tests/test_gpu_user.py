"""Run-time compiled user integrands (vegas_create_user) on the GPU.

* A user source that restates the Genz Gaussian runs the same kernels as the
  built-in kind: the same Philox words, bins, points and Jacobians bit for
  bit, f to rounding, and the whole VEGAS loop against the oracle with the
  bars of the built-in parity tests (FP64: 1e-12; compensated FP32: 1e-5
  relative and 0.1 sigma); SPRING draws the oracle's events.
* A user-only integrand (a product of truncated exponentials, integral 1):
  words, bins, points and Jacobians against the oracle's sampling step, f
  against the same formula in numpy at the dumped points, the iteration
  estimate against the mean of w = f J over all samples, and BASES against
  the closed form.
"""
import math

import numpy as np
import pytest

from paper_1010_2107_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

GAUSS = r"""
// Genz Gaussian: p = (a_1..a_d, u_1..u_d)
template <typename T>
__device__ T vegas_user_f(const T* x, int d, const T* p) {
  T q = T(0);
  for (int i = 0; i < d; ++i) {
    const T t = x[i] - p[d + i];
    q += p[i] * p[i] * t * t;
  }
  return exp(-q);
}
"""

# f = prod_i c_i exp(-c_i x_i) / (1 - exp(-c_i)): each factor integrates to 1
TRUNC_EXP = r"""
template <typename T>
__device__ T vegas_user_f(const T* x, int d, const T* p) {
  T f = T(1);
  for (int i = 0; i < d; ++i) f *= p[i] * exp(-p[i] * x[i]) / (T(1) - exp(-p[i]));
  return f;
}
"""


def trunc_exp_np(x, c):
    return np.prod(c * np.exp(-c * x) / (1.0 - np.exp(-c)), axis=1)


@pytest.fixture(scope="module")
def gv():
    from paper_1010_2107_gb300 import _build, gvegas
    _build.build()
    return gvegas


@pytest.mark.parametrize("d,precision,ybits,nstrat,ncall", [
    (4, 0, 53, 0, 3001),
    (4, 2, 24, 4, 4 ** 4 * 6),   # specialised kernel, two points in flight
    (5, 1, 53, 0, 3001),
    (12, 2, 24, 0, 3001),
])
def test_user_gauss_dump_equals_builtin(gv, d, precision, ybits, nstrat, ncall):
    params = wl.genz_gaussian_params(d)
    kw = dict(ncall=ncall, nstrat=nstrat, precision=precision, ybits=ybits)
    with gv.vegas_create_user(GAUSS, d, params, **kw) as u, \
            gv.vegas_create(wl.GENZ_GAUSSIAN, d, params, **kw) as b:
        s = np.unique(np.concatenate([[0, 1, ncall - 1], np.random.default_rng(2).integers(0, ncall, 400)]))
        for it in (0, 5):
            gu, gb = gv.vegas_sample_dump(u, it, s), gv.vegas_sample_dump(b, it, s)
            for k in ("words", "bins", "x", "jac"):
                assert np.array_equal(gu[k], gb[k]), k
            if precision == 0:
                np.testing.assert_allclose(gu["f"], gb["f"], rtol=1e-13, atol=1e-300)
            else:  # FP32: another summation order and exp form than the built-in's
                np.testing.assert_allclose(gu["f"], gb["f"], rtol=1e-4, atol=1e-7 * np.max(gb["f"]))


def test_user_gauss_fp64_vegas_loop_matches_the_oracle(gv, orc):
    d, N, n = 4, 50, 20011
    params = wl.genz_gaussian_params(d)
    with gv.vegas_create_user(GAUSS, d, params, nbins=N, ncall=n, precision=0, seed=3) as ctx:
        r = gv.vegas_iterate(ctx, 3, refine=True)
        edges = gv.vegas_get_grid(ctx)
        hist = gv.vegas_get_history(ctx)
    cfg = orc.make_cfg(d, nbins=N, ncall=n, ybits=53, seed=3)
    fn = orc.Integrand(wl.GENZ_GAUSSIAN, d, params)
    e = orc.uniform_grid(d, N)
    ref = orc.vegas(cfg, fn, e, 0, 3)
    assert r["iters_done"] == 3
    assert abs(r["I"] - ref["I"]) <= 1e-12 * abs(ref["I"])
    np.testing.assert_allclose(hist, ref["hist"], rtol=1e-11, atol=0)
    assert np.max(np.abs(edges - e)) < 1e-12


def test_user_gauss_fp32_strat_matches_the_oracle(gv, orc):
    d, g, N = 4, 4, 50
    ncall = g ** d * 64 + 0
    params = wl.genz_gaussian_params(d)
    with gv.vegas_create_user(GAUSS, d, params, nbins=N, ncall=ncall, nstrat=g, precision=2, ybits=24) as ctx:
        I, var = gv.vegas_eval(ctx, 2)
    cfg = orc.make_cfg(d, nbins=N, ncall=ncall, nstrat=g, ybits=24)
    o = orc.iteration(cfg, orc.Integrand(wl.GENZ_GAUSSIAN, d, params), orc.uniform_grid(d, N), 2)
    sig = math.sqrt(o["var"])
    assert abs(I - o["I"]) <= 1e-5 * abs(o["I"])
    assert abs(I - o["I"]) <= 0.1 * sig
    assert abs(math.sqrt(var) - sig) <= 1e-3 * sig


def test_user_gauss_spring_matches_the_oracle(gv, orc):
    d, g, N, nc = 3, 4, 20, 40
    params = wl.genz_gaussian_params(d, a=4.0)
    ncall = g ** d * nc
    with gv.vegas_create_user(GAUSS, d, params, nbins=N, ncall=ncall, nstrat=g, precision=0, ybits=24) as ctx:
        gv.bases_integrate(ctx, 2, 0.0, 2, 0.0)
        edges = gv.vegas_get_grid(ctx)
        cmax = gv.vegas_get_cube_max(ctx)
        cfg = orc.make_cfg(d, nbins=N, ncall=ncall, nstrat=g, ybits=24)
        fn = orc.Integrand(wl.GENZ_GAUSSIAN, d, params)
        ref = np.zeros_like(cmax)
        for it in (2, 3):
            ref = np.maximum(ref, orc.iteration(cfg, fn, edges, it, cubes=True)["Cmax"])
        np.testing.assert_allclose(cmax, ref, rtol=1e-12, atol=0)
        r = gv.spring_generate(ctx, 0, 30000)
        o = orc.spring(cfg, fn, edges, cmax, 0, 30000)
    np.testing.assert_array_equal(r["trial"], o["trial"])
    np.testing.assert_allclose(r["x"], o["x"], rtol=0, atol=1e-14)
    assert (r["overflow"], r["nonpos"]) == (o["overflow"], o["nonpos"])


@pytest.mark.parametrize("precision,ybits", [(0, 53), (2, 24)])
def test_user_only_integrand(gv, orc, precision, ybits):
    d, N, n = 5, 50, 20011
    c = np.array([12.0, 3.0, 20.0, 7.0, 1.5])
    with gv.vegas_create_user(TRUNC_EXP, d, c, nbins=N, ncall=n, precision=precision, ybits=ybits) as ctx:
        s = np.arange(n, dtype=np.uint64)
        dump = gv.vegas_sample_dump(ctx, 0, s)
        I, var = gv.vegas_eval(ctx, 0)
        cfg = orc.make_cfg(d, nbins=N, ncall=n, ybits=ybits)
        o = orc.sample_batch(cfg, orc.uniform_grid(d, N), 0, s)
        assert np.array_equal(dump["words"], o["words"]) and np.array_equal(dump["bins"], o["bins"])
        fx = trunc_exp_np(dump["x"], c)
        if precision == 0:
            assert np.array_equal(dump["jac"], o["jac"])
            np.testing.assert_allclose(dump["f"], fx, rtol=1e-13)
        else:
            np.testing.assert_allclose(dump["x"], o["x"], rtol=0, atol=3e-7)
            np.testing.assert_allclose(dump["f"], fx, rtol=2e-5)
        w = dump["f"] * dump["jac"]
        Iw = w.mean()
        vw = (np.mean(w * w) - Iw * Iw) / (n - 1)
        tol = 1e-12 if precision == 0 else 1e-6
        assert abs(I - Iw) <= tol * abs(Iw)
        assert abs(var - vw) <= (1e-9 if precision == 0 else 1e-5) * vw
        res, _ = gv.bases_integrate(ctx, 6, 0.0, 4, 0.0)
        assert abs(res["I"] - 1.0) <= 4.0 * res["sigma"] and res["sigma"] < 1e-2


def test_user_params_and_errors(gv):
    d = 3
    p1, p2 = wl.genz_gaussian_params(d), wl.genz_gaussian_params(d, a=2.0)
    with gv.vegas_create_user(GAUSS, d, p1, ncall=5000) as u, \
            gv.vegas_create_user(GAUSS, d, p2, ncall=5000) as v:
        gv.vegas_set_params(u, p2)
        assert gv.vegas_eval(u, 1) == gv.vegas_eval(v, 1)
        with pytest.raises(gv.VegasError):
            gv.vegas_set_params(u, p2[:-1])
        with pytest.raises(gv.VegasError):
            gv.vegas_grad(u, 0)
    with pytest.raises(gv.VegasError) as e:
        gv.vegas_create_user(GAUSS.replace("exp(-q)", "exp(-q) + oops"), d, p1)
    assert e.value.status == gv.EINVAL and "oops" in str(e.value)
    with pytest.raises(gv.VegasError) as e:
        gv.vegas_create_user(GAUSS, d, np.ones(gv.MAXUSERPARAMS + 1))
    assert e.value.status == gv.EINVAL


def test_zero_parameter_integrand(gv):
    src = "template <typename T> __device__ T vegas_user_f(const T* x, int d, const T*) " \
          "{ T s = T(0); for (int i = 0; i < d; ++i) s += x[i]; return s; }"
    with gv.vegas_create_user(src, 6, [], ncall=100003, precision=2) as ctx:
        r = gv.vegas_iterate(ctx, 3)
    assert abs(r["I"] - 3.0) <= 5 * r["sigma"]


def test_user_dgauss8_workload_source_matches_the_oracle(gv, orc):
    """The benchmarked user source (two-peak Gaussian, d = 8) at a reduced NCALL
    (65 536 cubes x 2 points) against the oracle's built-in twin."""
    w = wl.WORKLOADS["user_dgauss8"]
    d, g, N = w["ndim"], w["nstrat"], w["nbins"]
    ncall = g ** d * 2
    with gv.vegas_create_user(w["source"], d, w["params"], nbins=N, ncall=ncall, nstrat=g, precision=2,
                              ybits=24) as ctx:
        I, var = gv.vegas_eval(ctx, 1)
    cfg = orc.make_cfg(d, nbins=N, ncall=ncall, nstrat=g, ybits=24)
    o = orc.iteration(cfg, orc.Integrand(w["oracle_kind"], d, w["oracle_params"]), orc.uniform_grid(d, N), 1)
    sig = math.sqrt(o["var"])
    assert abs(I - o["I"]) <= 1e-5 * abs(o["I"]) and abs(I - o["I"]) <= 0.1 * sig
    assert abs(math.sqrt(var) - sig) <= 1e-3 * sig
