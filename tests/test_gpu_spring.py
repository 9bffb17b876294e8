"""SPRING on the GPU against the oracle, through the C ABI.  The GPU's own
per-cube maxima (recorded by bases_integrate's integration phase) are
checked against the oracle's maxima on the same grid, then given to the
oracle so that both sides draw from the same bounds:

* FP64 form: the same kept trials, bit for bit in their indices, the points
  to rounding, the same overflow and non-positive counts;
* FP32 form (FP32 weights and keep decision on the GPU, FP64 in the oracle):
  at most 0.5 % of trials decided differently, points to FP32 rounding.
"""
import numpy as np
import pytest

from paper_1010_2107_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gv():
    from paper_1010_2107_gb300 import _build, gvegas
    _build.build()
    return gvegas


def _run(gv, orc, kind, d, params, precision, *, g=4, N=20, nc=40, n1=2, n2=2):
    ncall = g ** d * nc
    ctx = gv.vegas_create(kind, d, params, nbins=N, ncall=ncall, nstrat=g, precision=precision, ybits=24)
    cfg = orc.make_cfg(d, nbins=N, ncall=ncall, nstrat=g, ybits=24)
    fn = orc.Integrand(kind, d, params)
    gv.bases_integrate(ctx, n1, 0.0, n2, 0.0)
    edges = gv.vegas_get_grid(ctx)
    cmax = gv.vegas_get_cube_max(ctx)
    # the oracle's maxima over the integration phase's iterations on this grid
    ref = np.zeros_like(cmax)
    for it in range(n1, n1 + n2):
        ref = np.maximum(ref, orc.iteration(cfg, fn, edges, it, cubes=True)["Cmax"])
    return ctx, cfg, fn, edges, cmax, ref


@pytest.mark.parametrize("precision", [0, 2])
def test_cube_maxima_match_the_oracle(gv, orc, precision):
    ctx, cfg, fn, edges, cmax, ref = _run(gv, orc, wl.GENZ_PRODUCT_PEAK, 2, np.array([5.0, 3.0, 0.3, 0.6]),
                                          precision)
    with ctx:
        tol = 1e-12 if precision == 0 else 1e-5
        np.testing.assert_allclose(cmax, ref, rtol=tol, atol=0)


@pytest.mark.parametrize("kind,d,params", [
    (wl.GENZ_PRODUCT_PEAK, 2, np.array([5.0, 3.0, 0.3, 0.6])),
    (wl.DOUBLE_GAUSSIAN, 4, wl.double_gaussian_params(w=0.15)),
    (wl.GENZ_GAUSSIAN, 3, wl.genz_gaussian_params(3, a=4.0)),
    (wl.W_MUNU, 5, wl.w_munu_params()),
], ids=["pp2", "dg4", "gauss3", "wmunu"])
def test_spring_fp64_matches_the_oracle(gv, orc, kind, d, params):
    ctx, cfg, fn, edges, cmax, ref = _run(gv, orc, kind, d, params, 0)
    with ctx:
        n = 30000
        r = gv.spring_generate(ctx, 0, n)
        o = orc.spring(cfg, fn, edges, cmax, 0, n)
        np.testing.assert_array_equal(r["trial"], o["trial"])
        np.testing.assert_allclose(r["x"], o["x"], rtol=0, atol=1e-14)
        assert (r["overflow"], r["nonpos"]) == (o["overflow"], o["nonpos"])
        assert r["n_events"] > n // 20


def test_spring_fp32_matches_the_oracle_up_to_boundary_flips(gv, orc):
    d, params = 4, wl.double_gaussian_params(w=0.15)
    ctx, cfg, fn, edges, cmax, ref = _run(gv, orc, wl.DOUBLE_GAUSSIAN, d, params, 2)
    with ctx:
        n = 30000
        r = gv.spring_generate(ctx, 0, n)
        o = orc.spring(cfg, fn, edges, cmax, 0, n)
        a, b = set(r["trial"].tolist()), set(o["trial"].tolist())
        assert len(a ^ b) <= 0.005 * n
        common = np.array(sorted(a & b), dtype=np.uint64)
        xi = r["x"][np.searchsorted(r["trial"], common)]
        xo = o["x"][np.searchsorted(o["trial"], common)]
        np.testing.assert_allclose(xi, xo, rtol=0, atol=3e-7)


def test_spring_is_counter_based_on_the_gpu(gv, orc):
    ctx, *_ = _run(gv, orc, wl.GENZ_PRODUCT_PEAK, 2, np.array([5.0, 3.0, 0.3, 0.6]), 2)
    with ctx:
        full = gv.spring_generate(ctx, 0, 20000)
        head = gv.spring_generate(ctx, 0, 7000)
        tail = gv.spring_generate(ctx, 7000, 13000)
        np.testing.assert_array_equal(full["trial"], np.concatenate([head["trial"], tail["trial"]]))
        np.testing.assert_array_equal(full["x"], np.concatenate([head["x"], tail["x"]]))
        counts = gv.spring_generate(ctx, 0, 20000, events=False)
        assert counts["n_events"] == full["n_events"] and counts["x"] is None


def test_spring_rambo_fp64_uses_the_scaled_maxima(gv, orc):
    d, params = 16, wl.rambo_params(4, cut=1)
    ctx, cfg, fn, edges, cmax, ref = _run(gv, orc, wl.RAMBO_BW, d, params, 0, g=1, N=50, nc=50000, n1=2, n2=1)
    with ctx:
        np.testing.assert_allclose(cmax, ref, rtol=1e-9)
        n = 20000
        r = gv.spring_generate(ctx, 0, n)
        o = orc.spring(cfg, fn, edges, cmax, 0, n)
        a, b = set(r["trial"].tolist()), set(o["trial"].tolist())
        assert len(a ^ b) <= 0.001 * n + 1


def test_spring_rejects_bad_calls(gv):
    ctx = gv.vegas_create(wl.GENZ_PRODUCT_PEAK, 2, np.array([5.0, 3.0, 0.3, 0.6]), ncall=4000, nstrat=2)
    with ctx:
        with pytest.raises(gv.VegasError):
            gv.spring_generate(ctx, 0, 10)  # no integration phase yet
        with pytest.raises(gv.VegasError):
            gv.vegas_get_cube_max(ctx)
        gv.bases_integrate(ctx, 1, 0.0, 1, 0.0)
        with pytest.raises(gv.VegasError):
            gv.spring_generate(ctx, 2 ** 32 - 5, 10)
        assert gv.spring_generate(ctx, 0, 0)["n_events"] == 0
