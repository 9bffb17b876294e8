"""CUDA path against the CPU oracle, through the C ABI, on identical seeded inputs.

Bars (stated per result):
  * Philox words and grid bins: bit-exact in every precision form.
  * FP64 form: the Jacobian bit-exact, x within 2 ulp; per-bin sums S1, S2 and the
    iteration totals within 1e-12 * sum|w| (condition-scaled; the GPU tree
    order differs from the oracle's sequential Neumaier order); estimates and
    refined edges within 1e-12 / 1e-13 relative.
  * FP32 forms (same 24-bit samples as the oracle): estimates within 1e-5
    relative AND within 0.1 sigma; per-bin sums S1 within 1e-5 * sum|w|, S2
    within 1e-5 * sum w^2 + 2e-4 * S2 of the cell (a cell's sum of squares
    can rest on a few points, whose FP32 error, 1e-4 at most per weight,
    passes into it undiluted).
  * Points one by one: FP64 values within 1e-12 relative; FP32 values within
    2e-4 relative (1e-6 of the largest weight absolute) of the oracle at the
    GPU's own FP32 point.  A point may fall on the other side of a cut or
    discontinuity only where the oracle's cut margin (the relative distance
    of pT, Delta R, a coordinate or a W cut quantity from its edge) is below
    1e-13 in FP64 or 1e-4 in FP32.
"""
import math

import numpy as np
import pytest

from paper_1010_2107_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gv():
    from paper_1010_2107_gb300 import _build, gvegas
    _build.build()
    return gvegas


def _pair(gv, orc, kind, d, params, *, N=50, ncall=10000, nstrat=0, precision=0, ybits=0, seed=1):
    ctx = gv.vegas_create(kind, d, params, nbins=N, ncall=ncall, nstrat=nstrat, precision=precision,
                          ybits=ybits, seed=seed)
    cfg = orc.make_cfg(d, nbins=N, ncall=ncall, nstrat=nstrat, ybits=ctx.ybits, seed=seed)
    fn = orc.Integrand(kind, d, params)
    return ctx, cfg, fn


CASES = [
    ("gauss4", wl.GENZ_GAUSSIAN, 4, wl.genz_gaussian_params(4), {}),
    ("pp3", wl.GENZ_PRODUCT_PEAK, 3, np.array([5.0, 3.0, 7.0, 0.3, 0.5, 0.8]), {}),
    ("cp6", wl.GENZ_CORNER_PEAK, 6, np.array([0.3, 0.1, 0.5, 0.2, 0.4, 0.35]), {}),
    ("osc5", wl.GENZ_OSCILLATORY, 5, np.array([1.0, 2.0, 0.5, 1.5, 3.0, 0.3]), {}),
    ("dg8", wl.DOUBLE_GAUSSIAN, 8, wl.double_gaussian_params(), {}),
    ("rb5", wl.RAMBO_BW, 20, wl.rambo_params(5), {}),
    ("rb4s", wl.RAMBO_BW, 16, wl.rambo_params(4, cut=1), {}),
    ("dg4strat", wl.DOUBLE_GAUSSIAN, 4, wl.double_gaussian_params(), dict(nstrat=4, ncall=4 ** 4 * 6)),
    ("gauss3strat3", wl.GENZ_GAUSSIAN, 3, wl.genz_gaussian_params(3, a=5.0), dict(nstrat=3, ncall=27 * 37)),
    ("cont4", wl.GENZ_CONTINUOUS, 4, np.array([3.0, 5.0, 2.0, 4.0, 0.3, 0.6, 0.5, 0.45]), {}),
    ("disc3", wl.GENZ_DISCONTINUOUS, 3, np.array([1.5, 2.0, 0.7, 0.4, 0.6]), {}),
    ("wmunu", wl.W_MUNU, 5, wl.w_munu_params(), {}),
    ("wmunu_strat", wl.W_MUNU, 5, wl.w_munu_params(), dict(nstrat=4, ncall=4 ** 5 * 12)),
]


@pytest.mark.parametrize("name,kind,d,params,kw", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision,ybits", [(0, 53), (0, 24), (2, 24), (1, 53)])
def test_words_bins_points(gv, orc, name, kind, d, params, kw, precision, ybits):
    ncall = kw.get("ncall", 3001)
    ctx, cfg, fn = _pair(gv, orc, kind, d, params, ncall=ncall, nstrat=kw.get("nstrat", 0),
                         precision=precision, ybits=ybits)
    with ctx:
        rng = np.random.default_rng(1)
        s = np.unique(np.concatenate([[0, 1, ncall - 1], rng.integers(0, ncall, 500)]))
        for it in (0, 7):
            g = gv.vegas_sample_dump(ctx, it, s)
            o = orc.sample_batch(cfg, orc.uniform_grid(d, 50), it, s)
            assert np.array_equal(g["words"], o["words"])
            assert np.array_equal(g["bins"], o["bins"])
            fg = g["f"] * g["jac"]
            if precision == 0:
                assert np.array_equal(g["jac"], o["jac"])
                np.testing.assert_allclose(g["x"], o["x"], rtol=4.5e-16, atol=1e-300)
                fo = orc.integrand(fn, o["x"]) * o["jac"]
                ok = np.isclose(fg, fo, rtol=1e-12, atol=1e-300)
                edge = 1e-13  # a few hundred ulp of a cut quantity
                margin = orc.cut_margin(fn, o["x"])
            else:
                np.testing.assert_allclose(g["x"], o["x"], rtol=0, atol=3e-7)
                # the oracle at the GPU's own FP32 point (the FP32 rounding of
                # x is a different input, not an error of the integrand)
                xg = np.ascontiguousarray(g["x"])
                fo = orc.integrand(fn, xg) * g["jac"]
                ok = np.isclose(fg, fo, rtol=2e-4, atol=1e-300 + 1e-6 * np.max(np.abs(fo)))
                edge = 1e-4  # FP32 rounding of pT, Delta R, eta through the boost
                margin = orc.cut_margin(fn, xg)
            # a point may land on the other side of a cut or discontinuity only
            # when the oracle puts its cut quantity within rounding of the edge
            bad = np.flatnonzero(~ok & ~(margin < edge))
            assert bad.size == 0, (bad[:10], fg[bad[:5]], fo[bad[:5]], margin[bad[:5]])


def _cond_close(a, b, scale, tol):
    return np.all(np.abs(a - b) <= tol * scale)


@pytest.mark.parametrize("name,kind,d,params,kw", CASES, ids=[c[0] for c in CASES])
def test_fp64_iteration_sums(gv, orc, name, kind, d, params, kw):
    ncall = kw.get("ncall", 20011)
    ctx, cfg, fn = _pair(gv, orc, kind, d, params, ncall=ncall, nstrat=kw.get("nstrat", 0), precision=0)
    with ctx:
        I, var = gv.vegas_eval(ctx, 3)
        _, bins = gv.vegas_get_grid(ctx, bin_sums=True)
    o = orc.iteration(cfg, fn, orc.uniform_grid(d, 50), 3)
    p = orc.sample_batch(cfg, orc.uniform_grid(d, 50), 3, np.arange(ncall))
    absw = np.abs(orc.integrand(fn, p["x"]) * p["jac"])
    tol = 1e-12
    assert abs(I - o["I"]) <= tol * max(absw.mean(), 1e-300)
    assert abs(math.sqrt(var) - math.sqrt(o["var"])) <= 1e-9 * math.sqrt(o["var"]) + 1e-300
    assert _cond_close(bins[0], o["S1"], absw.sum(), tol)
    assert _cond_close(bins[1], o["S2"], (absw ** 2).sum(), tol)


@pytest.mark.parametrize("name,kind,d,params,kw", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", [1, 2])
def test_fp32_iteration_vs_oracle(gv, orc, name, kind, d, params, kw, precision):
    ncall = kw.get("ncall", 65536 + 77)
    ctx, cfg, fn = _pair(gv, orc, kind, d, params, ncall=ncall, nstrat=kw.get("nstrat", 0),
                         precision=precision, ybits=24)
    with ctx:
        I, var = gv.vegas_eval(ctx, 2)
        _, bins = gv.vegas_get_grid(ctx, bin_sums=True)
    o = orc.iteration(cfg, fn, orc.uniform_grid(d, 50), 2)
    sig = math.sqrt(o["var"])
    p = orc.sample_batch(cfg, orc.uniform_grid(d, 50), 2, np.arange(ncall))
    absw = np.abs(orc.integrand(fn, p["x"]) * p["jac"])
    # 1e-5 of the larger of |I| and the mean |w|: the same as 1e-5 of |I|
    # for the non-negative integrands; for the sign-changing oscillatory
    # family, whose |I| can sit far below the weights it cancels, the
    # condition-scaled form of the bar
    assert abs(I - o["I"]) <= 1e-5 * max(abs(o["I"]), absw.mean()) + 1e-300
    assert abs(I - o["I"]) <= 0.1 * sig + 1e-300
    assert abs(math.sqrt(var) - sig) <= 1e-3 * sig + 1e-300
    assert _cond_close(bins[0], o["S1"], absw.sum(), 1e-5)
    # S2: also within twice the per-point FP32 bar (1e-4) of the cell itself
    assert np.all(np.abs(bins[1] - o["S2"]) <= 1e-5 * (absw ** 2).sum() + 2e-4 * np.abs(o["S2"]))


def test_vegas_loop_fp64_gauss4(gv, orc):
    """The d=4 Gaussian workload (5 x 1e5, FP64): every iteration estimate, the
    refined grid and the combined result against the oracle's VEGAS loop."""
    w = wl.WORKLOADS["gauss4"]
    ctx, cfg, fn = _pair(gv, orc, w["kind"], 4, w["params"], ncall=w["ncall"], precision=0)
    with ctx:
        r = gv.vegas_iterate(ctx, w["itmx"], refine=True)
        hist = gv.vegas_get_history(ctx)
        edges = gv.vegas_get_grid(ctx)
        assert gv.vegas_get_iteration(ctx) == w["itmx"]
    e = orc.uniform_grid(4, 50)
    ref = orc.vegas(cfg, fn, e, 0, w["itmx"])
    np.testing.assert_allclose(hist[:, 0], ref["hist"][:, 0], rtol=1e-12)
    np.testing.assert_allclose(hist[:, 1], ref["hist"][:, 1], rtol=1e-9)
    np.testing.assert_allclose(edges, e, rtol=0, atol=1e-13)
    assert r["I"] == pytest.approx(ref["I"], rel=1e-12)
    assert r["sigma"] == pytest.approx(ref["sigma"], rel=1e-9)
    assert r["chi2_dof"] == pytest.approx(ref["chi2_dof"], rel=1e-6, abs=1e-9)
    exact = 9.8696044010286631e-4
    assert abs(r["I"] - exact) < 4 * r["sigma"]


def test_bases_small_fp64_and_cubes(gv, orc):
    d, g = 4, 4
    ncall = g ** d * 8
    p = wl.double_gaussian_params()
    ctx, cfg, fn = _pair(gv, orc, wl.DOUBLE_GAUSSIAN, d, p, ncall=ncall, nstrat=g, precision=0, ybits=24)
    with ctx:
        out, ph1 = gv.bases_integrate(ctx, 3, 0.0, 3, 0.0)
        cubes = gv.vegas_get_cube_sums(ctx)
        hist = gv.vegas_get_history(ctx)
    e = orc.uniform_grid(d, 50)
    ref = orc.bases(cfg, fn, e, 0, 3, 0.0, 3, 0.0)
    assert (ph1["iters_done"], out["iters_done"]) == (3, 3)
    assert out["I"] == pytest.approx(ref["I"], rel=1e-12)
    assert out["sigma"] == pytest.approx(ref["sigma"], rel=1e-9)
    np.testing.assert_allclose(hist, ref["hist"][3:], rtol=1e-9)
    o = orc.iteration(cfg, fn, e, 5, cubes=True)
    np.testing.assert_allclose(cubes[:, 0], o["C1"], rtol=1e-12, atol=1e-12 * np.abs(o["C1"]).max())
    np.testing.assert_allclose(cubes[:, 1], o["C2"], rtol=1e-12, atol=1e-12 * np.abs(o["C2"]).max())


def test_nonfinite_weights_are_counted(gv):
    ctx = gv.vegas_create(gv.GENZ_GAUSSIAN, 1, [float("nan"), 0.5], ncall=1000)
    with ctx:
        r = gv.vegas_iterate(ctx, 1)
    assert r["nonfinite"] == 1000 and r["I"] == 0.0


def test_acc_stops_early_on_device(gv):
    ctx = gv.vegas_create(gv.GENZ_CORNER_PEAK, 2, [0.2, 0.3], nbins=20, ncall=4000, acc=1e-3)
    with ctx:
        r = gv.vegas_iterate(ctx, 50)
        it = gv.vegas_get_iteration(ctx)
    assert r["stopped"] == 1 and r["iters_done"] < 50 and it == r["iters_done"]
    assert r["sigma"] < 1e-3 * abs(r["I"])


@pytest.mark.parametrize("N", [2, 31, 33, 64, 65, 100, 256])
@pytest.mark.parametrize("precision", [0, 2])
def test_bin_counts_across_histogram_paths(gv, orc, N, precision):
    """Bin counts from 2 to 256 change the bucket capacity and tile shape of
    the CTA histogram; every one must give the oracle's per-bin sums (ragged
    NCALL, two iterations with a refined grid in between)."""
    d, ncall = 3, 3 * 4096 + 17
    params = wl.genz_gaussian_params(d, a=6.0, u=0.4)
    ctx, cfg, fn = _pair(gv, orc, wl.GENZ_GAUSSIAN, d, params, N=N, ncall=ncall, precision=precision,
                         ybits=24)
    e = orc.uniform_grid(d, N)
    with ctx:
        gv.vegas_iterate(ctx, 1, refine=True)
        I, var = gv.vegas_eval(ctx, 1)
        edges, bins = gv.vegas_get_grid(ctx, bin_sums=True)
    o0 = orc.iteration(cfg, fn, e, 0)
    e1 = orc.refine(o0["S2"], e)
    tol = 1e-12 if precision == 0 else 1e-5
    np.testing.assert_allclose(edges, e1, rtol=0, atol=1e-12 if precision == 0 else 1e-6)
    o1 = orc.iteration(cfg, fn, edges, 1)  # oracle on the GPU's grid: same points
    p = orc.sample_batch(cfg, edges, 1, np.arange(ncall))
    absw = np.abs(orc.integrand(fn, p["x"]) * p["jac"])
    assert _cond_close(bins[0], o1["S1"], absw.sum(), tol)
    assert _cond_close(bins[1], o1["S2"], (absw ** 2).sum(), tol)
    assert abs(I - o1["I"]) <= tol * absw.mean()


@pytest.mark.parametrize("ncall", [2, 3, 31, 33, 255, 257, 100003])
def test_tiny_and_ragged_ncall(gv, orc, ncall):
    d = 2
    params = np.array([3.0, 5.0, 0.3, 0.6])
    ctx, cfg, fn = _pair(gv, orc, wl.GENZ_PRODUCT_PEAK, d, params, ncall=ncall, precision=0)
    with ctx:
        I, var = gv.vegas_eval(ctx, 0)
        _, bins = gv.vegas_get_grid(ctx, bin_sums=True)
    o = orc.iteration(cfg, fn, orc.uniform_grid(d, 50), 0)
    assert I == pytest.approx(o["I"], rel=1e-12)
    assert var == pytest.approx(o["var"], rel=1e-9, abs=1e-300)
    np.testing.assert_allclose(bins[0], o["S1"], rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("d,precision", [(1, 0), (1, 2), (32, 0), (32, 2), (17, 2)])
def test_dimension_extremes(gv, orc, d, precision):
    params = np.concatenate([np.full(d, 0.3), np.full(d, 0.5)])
    ctx, cfg, fn = _pair(gv, orc, wl.GENZ_PRODUCT_PEAK, d, params, ncall=20000, precision=precision,
                         ybits=24)
    with ctx:
        I, var = gv.vegas_eval(ctx, 4)
        _, bins = gv.vegas_get_grid(ctx, bin_sums=True)
    o = orc.iteration(cfg, fn, orc.uniform_grid(d, 50), 4)
    tol = 1e-12 if precision == 0 else 1e-5
    assert I == pytest.approx(o["I"], rel=tol)
    np.testing.assert_allclose(bins[0], o["S1"], rtol=tol, atol=tol * np.abs(o["S1"]).max())


@pytest.mark.parametrize("precision", [0, 2])
@pytest.mark.parametrize("ppt", [1, 2, 3, 4, 8])
@pytest.mark.parametrize("nstrat", [0, 4])
def test_histogram_tile_shapes(gv, orc, precision, ppt, nstrat):
    """Every histogram tile (points per thread between gathers) gives the
    oracle's sums: the tile changes only the summation order.  The FP32
    kernel of d = 8 evaluates two points at a time and rounds odd tiles up."""
    d, ncall = 8, 4 ** 8 * 3 + (0 if nstrat else 101)
    params = wl.double_gaussian_params()
    ctx, cfg, fn = _pair(gv, orc, wl.DOUBLE_GAUSSIAN, d, params, ncall=ncall, nstrat=nstrat,
                         precision=precision, ybits=24)
    with ctx:
        gv.vegas_set_tile(ctx, ppt)
        t = gv.vegas_get_tile(ctx)
        I, var = gv.vegas_eval(ctx, 3)
        _, bins = gv.vegas_get_grid(ctx, bin_sums=True)
    if precision == 2:
        assert t["points_per_thread"] == ppt + (ppt % 2)
    else:
        assert t["points_per_thread"] == ppt
    assert t["cap"] >= 4
    o = orc.iteration(cfg, fn, orc.uniform_grid(d, 50), 3)
    p = orc.sample_batch(cfg, orc.uniform_grid(d, 50), 3, np.arange(ncall))
    absw = np.abs(orc.integrand(fn, p["x"]) * p["jac"])
    tol = 1e-12 if precision == 0 else 1e-5
    assert _cond_close(bins[0], o["S1"], absw.sum(), tol)
    assert _cond_close(bins[1], o["S2"], (absw ** 2).sum(), tol)
    assert abs(I - o["I"]) <= tol * absw.mean() + 0.1 * math.sqrt(o["var"]) * (precision != 0)


def test_set_tile_rejects_bad_values(gv):
    ctx = gv.vegas_create(wl.GENZ_GAUSSIAN, 3, wl.genz_gaussian_params(3), ncall=1000)
    with ctx:
        before = gv.vegas_get_tile(ctx)
        for bad in (-1, 9):
            with pytest.raises(gv.VegasError):
                gv.vegas_set_tile(ctx, bad)
        assert gv.vegas_get_tile(ctx) == before


@pytest.mark.parametrize("nstrat", [0, 4])
def test_autotuned_shape_keeps_parity(gv, orc, nstrat):
    """The autotuner only changes the launch shape: the tuned context still
    gives the oracle's sums."""
    d, ncall = 8, 4 ** 8 * 3 + (0 if nstrat else 101)
    params = wl.double_gaussian_params()
    ctx, cfg, fn = _pair(gv, orc, wl.DOUBLE_GAUSSIAN, d, params, ncall=ncall, nstrat=nstrat, precision=2, ybits=24)
    with ctx:
        t = gv.vegas_autotune(ctx)
        assert t["threads"] in (128, 256, 384, 512) and t["points_per_thread"] >= 1 and t["ms"] > 0
        assert gv.vegas_get_launch(ctx)["threads"] == t["threads"]
        I, var = gv.vegas_eval(ctx, 5)
        _, bins = gv.vegas_get_grid(ctx, bin_sums=True)
    o = orc.iteration(cfg, fn, orc.uniform_grid(d, 50), 5)
    p = orc.sample_batch(cfg, orc.uniform_grid(d, 50), 5, np.arange(ncall))
    absw = np.abs(orc.integrand(fn, p["x"]) * p["jac"])
    assert _cond_close(bins[0], o["S1"], absw.sum(), 1e-5)
    assert _cond_close(bins[1], o["S2"], (absw ** 2).sum(), 1e-5)
    assert abs(I - o["I"]) <= 0.1 * math.sqrt(o["var"])


def test_set_launch_limits(gv):
    ctx = gv.vegas_create(wl.DOUBLE_GAUSSIAN, 8, wl.double_gaussian_params(), ncall=1 << 16, precision=2, ybits=24)
    with ctx:
        gv.vegas_set_launch(ctx, 512)  # specialised kernel: allowed
        assert gv.vegas_get_launch(ctx)["threads"] == 512
        for bad in (32, 100, 544, 1024):
            with pytest.raises(gv.VegasError):
                gv.vegas_set_launch(ctx, bad)
        assert gv.vegas_get_launch(ctx)["threads"] == 512
    ctx = gv.vegas_create(wl.DOUBLE_GAUSSIAN, 7, wl.double_gaussian_params(), ncall=1 << 16, precision=2, ybits=24)
    with ctx:  # general kernel (d below the compiled bound): 256 at most
        with pytest.raises(gv.VegasError):
            gv.vegas_set_launch(ctx, 384)


def test_bases_wmunu_fp64_matches_the_oracle(gv, orc):
    """The W workload's BASES run (both phases, refinement between the first
    phase's iterations) at a reduced NCALL, FP64, against the oracle."""
    d, g, N = 5, 4, 50
    ncall = g ** d * 24
    p = wl.w_munu_params()
    with gv.vegas_create(wl.W_MUNU, d, p, nbins=N, ncall=ncall, nstrat=g, precision=0, ybits=24) as ctx:
        r, ph1 = gv.bases_integrate(ctx, 3, 0.0, 2, 0.0)
        edges = gv.vegas_get_grid(ctx)
    cfg = orc.make_cfg(d, nbins=N, ncall=ncall, nstrat=g, ybits=24)
    e = orc.uniform_grid(d, N)
    ref = orc.bases(cfg, orc.Integrand(wl.W_MUNU, d, p), e, 0, 3, 0.0, 2, 0.0)
    assert (ph1["iters_done"], r["iters_done"]) == (3, 2)
    assert abs(r["I"] - ref["I"]) <= 1e-11 * abs(ref["I"])
    assert abs(r["sigma"] - ref["sigma"]) <= 1e-9 * ref["sigma"]
    assert np.max(np.abs(edges - e)) < 1e-11


@pytest.mark.parametrize("precision,nstrat,ncall", [(0, 0, 20011), (2, 0, 65613), (0, 4, 4 ** 4 * 40),
                                                    (2, 4, 4 ** 4 * 40)])
def test_frozen_grid_passes_skip_only_the_bin_sums(gv, orc, precision, nstrat, ncall):
    """Passes that do not refine skip the per-bin histogram (only step 5
    reads it) and run on their own launch shape: their estimates equal those
    of evaluation passes (which keep it) on the same grid and counters, up to
    the order of the per-CTA sums; the bin sums stay those of the last pass
    that formed them."""
    d = 4
    p = wl.double_gaussian_params()
    with gv.vegas_create(wl.DOUBLE_GAUSSIAN, d, p, ncall=ncall, nstrat=nstrat, precision=precision,
                         ybits=24) as ctx:
        gv.vegas_iterate(ctx, 2, refine=True)
        _, bins0 = gv.vegas_get_grid(ctx, bin_sums=True)
        gv.vegas_reset_results(ctx)
        gv.vegas_iterate(ctx, 3, refine=False)
        hist = gv.vegas_get_history(ctx)
        _, bins1 = gv.vegas_get_grid(ctx, bin_sums=True)
        ev = np.array([gv.vegas_eval(ctx, it) for it in (2, 3, 4)])
    np.testing.assert_array_equal(bins1, bins0)
    tol = 1e-13 if precision == 0 else 1e-6
    np.testing.assert_allclose(hist[:, 0], ev[:, 0], rtol=tol)
    np.testing.assert_allclose(hist[:, 1], ev[:, 1], rtol=1e3 * tol)


def test_set_params_reaches_captured_graphs(gv):
    """The integrand constants and the output scale live in device memory, so
    a graph captured before vegas_set_params computes with the new values
    (the RAMBO scale changes with sqrt(s)): same results as a fresh context."""
    p1, p2 = wl.rambo_params(3, sqrt_s=500.0), wl.rambo_params(3, sqrt_s=900.0)
    kw = dict(ncall=20000, precision=0, ybits=53, seed=4)
    with gv.vegas_create(wl.RAMBO_BW, 12, p1, **kw) as a, gv.vegas_create(wl.RAMBO_BW, 12, p2, **kw) as b:
        gv.vegas_iterate(a, 2, refine=True)  # captures the graph with p1
        gv.vegas_reset_grid(a)
        gv.vegas_reset_results(a)
        gv.vegas_set_iteration(a, 0)
        gv.vegas_set_params(a, p2)
        ra = gv.vegas_iterate(a, 2, refine=True)  # same call shape: the cached graph
        rb = gv.vegas_iterate(b, 2, refine=True)
        # equal up to the order of the shared-memory bucket claims, which
        # moves the last bits of the per-bin sums and through refinement the
        # second iteration (a stale scale would be off by (9/5)^k)
        assert ra["I"] == pytest.approx(rb["I"], rel=1e-12)
        assert ra["sigma"] == pytest.approx(rb["sigma"], rel=1e-9)
        np.testing.assert_allclose(gv.vegas_get_grid(a), gv.vegas_get_grid(b), rtol=0, atol=1e-12)


def test_two_body_rambo_fp64_matches_the_oracle(gv, orc):
    """The two-body RAMBO integrand, whose oracle is pinned against its closed
    form (f = V_2 cut BW(s) / s^2), in the FP64 form: the estimate to 1e-12
    and the dumped weights point by point."""
    p = wl.rambo_params(2, sqrt_s=1000.0, ptmin=150.0)
    ncall = 20011
    with gv.vegas_create(wl.RAMBO_BW, 8, p, ncall=ncall, precision=0, ybits=53) as ctx:
        I, _ = gv.vegas_eval(ctx, 1)
        s = np.arange(0, ncall, 7, dtype=np.uint64)
        g = gv.vegas_sample_dump(ctx, 1, s)
    cfg = orc.make_cfg(8, nbins=50, ncall=ncall, ybits=53)
    fn = orc.Integrand(wl.RAMBO_BW, 8, p)
    o = orc.iteration(cfg, fn, orc.uniform_grid(8, 50), 1)
    ob = orc.sample_batch(cfg, orc.uniform_grid(8, 50), 1, s)
    assert abs(I - o["I"]) <= 1e-12 * abs(o["I"])
    assert np.array_equal(g["words"], ob["words"])
    fo = orc.integrand(fn, ob["x"]) * ob["jac"]
    # every point: the momenta come from a boost whose rounding grows with
    # gamma^2 of the isotropic system, 1e-11 at worst over these samples
    np.testing.assert_allclose(g["f"] * g["jac"], fo, rtol=1e-10, atol=1e-300)


@pytest.mark.parametrize("cut", [0, 1])
@pytest.mark.parametrize("precision", [2, 1])
def test_two_body_rambo_fp32_matches_the_oracle(gv, orc, cut, precision):
    """The two-body RAMBO integrand in the FP32 forms on 2^20 identical
    points: the estimate within 1e-5 relative and 0.1 sigma of the oracle's,
    whose integrand is pinned to the closed form f = V_2 cut BW(s) / s^2."""
    p = wl.rambo_params(2, cut=cut)
    ncall = 1 << 20
    with gv.vegas_create(wl.RAMBO_BW, 8, p, ncall=ncall, precision=precision, ybits=24) as ctx:
        I, var = gv.vegas_eval(ctx, 2)
    cfg = orc.make_cfg(8, nbins=50, ncall=ncall, ybits=24)
    o = orc.iteration(cfg, orc.Integrand(wl.RAMBO_BW, 8, p), orc.uniform_grid(8, 50), 2)
    sig = math.sqrt(o["var"])
    assert abs(I - o["I"]) <= 1e-5 * abs(o["I"]), (I, o["I"])
    assert abs(I - o["I"]) <= 0.1 * sig
    assert abs(math.sqrt(var) - sig) <= 1e-3 * sig
