"""Pins of the oracle's steps 4-6 (Sec. 2.1): accumulation, grid
optimisation, combination of iterations, the VEGAS loop and the BASES phases."""
import math

import numpy as np
import pytest

import closed_forms as cf
from paper_1010_2107_gb300 import workloads as wl

# --------------------------------------------------------------- step 4


@pytest.mark.parametrize("g,ybits", [(0, 24), (0, 53), (2, 24), (3, 53)])
def test_iteration_brute_force(orc, g, ybits):
    """Tiny iteration recomputed from the per-sample points: per-bin sums with
    np.add.at, sample mean / variance with numpy, and stratified cube means and
    variances from a reshape (cubes hold consecutive samples)."""
    d, N = 2, 7
    G = max(g, 1) ** d
    nc = 6
    n = G * nc if g > 1 else 40
    cfg = orc.make_cfg(d, nbins=N, ncall=n, nstrat=g, ybits=ybits, seed=17)
    e = np.array([[0, .1, .15, .3, .6, .7, .95, 1.0], [0, .2, .3, .4, .5, .6, .8, 1.0]])
    fn = orc.Integrand(orc.GENZ_PRODUCT_PEAK, d, [3.0, 5.0, 0.3, 0.6])
    r = orc.iteration(cfg, fn, e, 4, cubes=g > 1)
    p = orc.sample_batch(cfg, e, 4, np.arange(n))
    w = orc.integrand(fn, p["x"]) * p["jac"]
    for a in range(d):
        S1 = np.zeros(N)
        S2 = np.zeros(N)
        np.add.at(S1, p["bins"][:, a], w)
        np.add.at(S2, p["bins"][:, a], w * w)
        np.testing.assert_allclose(r["S1"][a], S1, rtol=1e-14)
        np.testing.assert_allclose(r["S2"][a], S2, rtol=1e-14)
    assert r["sum_w"] == pytest.approx(w.sum(), rel=1e-14)
    if g > 1:
        wc = w.reshape(G, nc)
        m = wc.mean(1)
        v = wc.var(1, ddof=1) / nc
        assert r["I"] == pytest.approx(m.mean(), rel=1e-13)
        assert r["var"] == pytest.approx(v.sum() / G ** 2, rel=1e-10)
        np.testing.assert_allclose(r["C1"], wc.sum(1), rtol=1e-14)
        np.testing.assert_allclose(r["C2"], (wc ** 2).sum(1), rtol=1e-14)
        # cubes partition y-space: cube c's samples have floor(g y_a) = digit a of c
        for c in range(G):
            ys = (p["bins"][c * nc:(c + 1) * nc] + p["frac"][c * nc:(c + 1) * nc]) / N
            for a in range(d):
                assert np.all(np.floor(max(g, 1) * ys[:, a] + 1e-12) == (c // g ** a) % g)
    else:
        assert r["I"] == pytest.approx(w.mean(), rel=1e-14)
        assert r["var"] == pytest.approx(w.var(ddof=1) / n, rel=1e-9)


def test_bin_sums_are_consistent_across_axes(orc):
    """Every axis partitions the same samples: sum_k S1[a][k] = sum w for all a."""
    d = 5
    cfg = orc.make_cfg(d, nbins=50, ncall=20000, ybits=24)
    fn = orc.Integrand(orc.GENZ_CORNER_PEAK, d, [0.3, 0.2, 0.5, 0.1, 0.4])
    r = orc.iteration(cfg, fn, orc.uniform_grid(d, 50), 0)
    np.testing.assert_allclose(r["S1"].sum(1), r["sum_w"], rtol=1e-13)
    np.testing.assert_allclose(r["S2"].sum(1), r["sum_w2"], rtol=1e-13)


def test_nonfinite_weights_are_counted_and_dropped(orc):
    cfg = orc.make_cfg(1, nbins=10, ncall=1000, ybits=24)
    fn = orc.Integrand(orc.GENZ_GAUSSIAN, 1, [float("nan"), 0.5])
    r = orc.iteration(cfg, fn, orc.uniform_grid(1, 10), 0)
    assert r["nonfinite"] == 1000 and r["sum_w"] == 0.0 and r["I"] == 0.0


def test_stratified_with_one_division_equals_plain(orc):
    fn = orc.Integrand(orc.GENZ_GAUSSIAN, 3, wl.genz_gaussian_params(3, a=4.0))
    e = orc.uniform_grid(3, 20)
    a = orc.iteration(orc.make_cfg(3, nbins=20, ncall=5000, nstrat=0), fn, e, 1)
    b = orc.iteration(orc.make_cfg(3, nbins=20, ncall=5000, nstrat=1), fn, e, 1)
    assert a["I"] == b["I"] and a["var"] == b["var"]

# --------------------------------------------------------------- step 5


def test_refine_fixed_point_and_scale_invariance(orc):
    N = 50
    e0 = orc.uniform_grid(3, N)
    np.testing.assert_allclose(orc.refine(np.ones((3, N)), e0), e0, atol=2e-16)
    rng = np.random.default_rng(2)
    S2 = rng.random((3, N)) ** 4
    a = orc.refine(S2, e0)
    b = orc.refine(S2 * 1024.0, e0)
    np.testing.assert_array_equal(a, b)
    assert np.all(np.diff(a, axis=1) > 0) and np.all(a[:, 0] == 0) and np.all(a[:, -1] == 1)


@pytest.mark.parametrize("k", [2, 17, 47])
def test_refine_single_bin_delta(orc, k):
    """S2 nonzero in one interior old bin: smoothing spreads it as d/3 over that
    bin and its two neighbours, equal smoothed values get equal compressed
    weights, so the N new bins split those three old bins evenly -- whatever
    the compression function."""
    N = 50
    e0 = orc.uniform_grid(1, N)
    S2 = np.zeros((1, N))
    S2[0, k] = 3.7
    lo, hi = k - 1, k + 2
    e = orc.refine(S2, e0)[0]
    expect = lo / N + (hi - lo) / N * np.arange(N + 1) / N
    expect[0], expect[-1] = 0.0, 1.0
    np.testing.assert_allclose(e, expect, atol=1e-15)


@pytest.mark.parametrize("k", [0, 1, 48, 49])
def test_refine_single_bin_delta_at_ends(orc, k):
    """Near an end the end-bin rule averages two bins (d/2) and the inner rule
    three (d/3): the new interior edges stay inside the smoothed support."""
    N = 50
    S2 = np.zeros((1, N))
    S2[0, k] = 1.0
    e = orc.refine(S2, orc.uniform_grid(1, N))[0]
    lo, hi = max(k - 1, 0) / N, (min(k + 1, N - 1) + 1) / N
    assert np.all(e[1:-1] >= lo - 1e-15) and np.all(e[1:-1] <= hi + 1e-15)
    assert np.all(np.diff(e) > 0)


def test_refine_alpha_zero_keeps_positive_grid(orc):
    """alpha = 0 makes every positive bin weigh 1: a grid whose smoothed sums are
    all positive is left where it is."""
    rng = np.random.default_rng(8)
    e0 = np.sort(np.concatenate([[0, 1], rng.random(19)]))[None, :]
    S2 = rng.random((1, 20)) + 0.1
    np.testing.assert_allclose(orc.refine(S2, e0, alpha=0.0), e0, atol=1e-15)


def test_refine_moves_bins_towards_large_weights(orc):
    N = 50
    S2 = np.ones((1, N))
    S2[0, N // 2:] = 100.0
    e = orc.refine(S2, orc.uniform_grid(1, N))[0]
    assert np.count_nonzero(e[1:-1] >= 0.5) > N // 2


def test_refine_hand_example(orc):
    """N = 3, S2 = (1, 2, 4), uniform grid, alpha = 1.5, worked by hand:
    smoothed d' = (3/2, 7/3, 3), D = 41/6; r_k = ((1 - d'_k/D)/ln(D/d'_k))^1.5;
    then the edges at the 1/3 and 2/3 quantiles of the piecewise-uniform r."""
    d = [1.5, 7 / 3, 3.0]
    D = sum(d)
    r = [((1 - x / D) / math.log(D / x)) ** 1.5 for x in d]
    R = sum(r)
    e_old = [0, 1 / 3, 2 / 3, 1]
    cum = [0, r[0], r[0] + r[1], R]
    expect = [0.0]
    for j in (1, 2):
        t = j * R / 3
        k = max(i for i in range(3) if cum[i] < t)
        expect.append(e_old[k] + (t - cum[k]) / r[k] * (e_old[k + 1] - e_old[k]))
    expect.append(1.0)
    got = orc.refine(np.array([[1.0, 2.0, 4.0]]), np.array([e_old]))[0]
    np.testing.assert_allclose(got, expect, rtol=1e-14)


def test_refine_zero_axis_is_left_unchanged(orc):
    e0 = np.array([[0, .3, .5, 1.0], [0, .1, .2, 1.0]])
    S2 = np.array([[0.0, 0.0, 0.0], [1.0, 2.0, 3.0]])
    e = orc.refine(S2, e0)
    np.testing.assert_array_equal(e[0], e0[0])
    assert not np.array_equal(e[1], e0[1])

# --------------------------------------------------------------- step 6


def test_combine_identical_and_weighted(orc):
    r = orc.combine([2.0] * 4, [0.25] * 4)
    assert r["I"] == 2.0 and r["sigma"] == pytest.approx(0.5 / 2) and r["chi2_dof"] == 0.0
    rng = np.random.default_rng(1)
    I = rng.normal(1.0, 0.1, 7)
    var = rng.uniform(0.001, 0.02, 7)
    r = orc.combine(I, var)
    assert r["I"] == pytest.approx(np.average(I, weights=1 / var), rel=1e-14)
    assert r["sigma"] == pytest.approx(np.sum(1 / var) ** -0.5, rel=1e-14)
    # two measurements: chi^2 = (I1 - I2)^2 / (var1 + var2)
    r2 = orc.combine(I[:2], var[:2])
    assert r2["chi2_dof"] == pytest.approx((I[0] - I[1]) ** 2 / (var[0] + var[1]), rel=1e-12)
    assert orc.combine([3.0], [0.5])["chi2_dof"] == 0.0
    z = orc.combine([1.0, 5.0, 5.0], [0.1, 0.0, 0.0])
    assert z["I"] == 5.0 and z["sigma"] == 0.0

# --------------------------------------------------------------- loops


def test_vegas_gaussian_d4_workload(orc):
    """The d=4 Gaussian workload (5 x 1e5, 53-bit, seed 1) is within 4 sigma of
    the erf closed form, with a sane chi^2 and an error that falls as the grid
    adapts."""
    w = wl.WORKLOADS["gauss4"]
    cfg = orc.make_cfg(4, nbins=50, ncall=w["ncall"], ybits=53, seed=1)
    fn = orc.Integrand(w["kind"], 4, w["params"])
    e = orc.uniform_grid(4, 50)
    r = orc.vegas(cfg, fn, e, 0, w["itmx"])
    exact = cf.genz_gaussian([10.0] * 4, [0.5] * 4)
    assert r["iters"] == 5
    assert abs(r["I"] - exact) < 4 * r["sigma"]
    assert r["sigma"] < 2e-3 * exact
    assert r["chi2_dof"] < 5
    h = r["hist"]
    assert math.sqrt(h[-1, 1]) < 0.5 * math.sqrt(h[0, 1])


def test_vegas_one_dimensional_convergence(orc):
    """f(x) = (1 - x/2)^-2 (corner peak with a = -1/2, rising fourfold): the
    grid moves towards the zero-variance map and the relative error of a
    single iteration drops by more than 5x over 5 iterations."""
    cfg = orc.make_cfg(1, nbins=50, ncall=20000, ybits=53, seed=4)
    fn = orc.Integrand(orc.GENZ_CORNER_PEAK, 1, [-0.5])  # (1 - x/2)^-2: smooth, rising
    e = orc.uniform_grid(1, 50)
    r = orc.vegas(cfg, fn, e, 0, 5)
    h = r["hist"]
    rel = np.sqrt(h[:, 1]) / h[:, 0]
    assert rel[-1] < rel[0] / 5
    assert r["I"] == pytest.approx(cf.genz_corner_peak([-0.5]), abs=5 * r["sigma"])


def test_vegas_accuracy_stop(orc):
    cfg = orc.make_cfg(2, nbins=20, ncall=4000, seed=2)
    fn = orc.Integrand(orc.GENZ_CORNER_PEAK, 2, [0.2, 0.3])
    r = orc.vegas(cfg, fn, orc.uniform_grid(2, 20), 0, 50, acc=1e-3)
    assert r["iters"] < 50 and r["sigma"] < 1e-3 * abs(r["I"])


def test_bases_phases(orc):
    """BASES: phase 1 refines, phase 2 runs on the frozen grid and alone forms
    the result; iteration indices continue across phases."""
    d, g = 4, 4
    cfg = orc.make_cfg(d, nbins=50, ncall=g ** d * 64, nstrat=g, ybits=24, seed=1)
    fn = orc.Integrand(orc.DOUBLE_GAUSSIAN, d, wl.double_gaussian_params())
    e = orc.uniform_grid(d, 50)
    r = orc.bases(cfg, fn, e, 0, 5, 0.0, 5, 0.0)
    assert (r["n1"], r["n2"]) == (5, 5)
    assert abs(r["I"] - 1.0) < 4 * r["sigma"]
    c = orc.combine(r["hist"][5:, 0], r["hist"][5:, 1])
    assert r["I"] == c["I"] and r["sigma"] == c["sigma"]
    # phase 2 left the grid alone: re-running iteration 9 on it reproduces hist[9]
    again = orc.iteration(cfg, fn, e, 9)
    assert again["I"] == r["hist"][9, 0]


def test_independent_seeds_agree(orc):
    fn = orc.Integrand(orc.GENZ_PRODUCT_PEAK, 3, [5.0, 5.0, 5.0, 0.3, 0.5, 0.7])
    exact = cf.genz_product_peak([5.0] * 3, [0.3, 0.5, 0.7])
    res = []
    for seed in (1, 2, 3):
        cfg = orc.make_cfg(3, nbins=50, ncall=20000, seed=seed)
        res.append(orc.vegas(cfg, fn, orc.uniform_grid(3, 50), 0, 4))
    for r in res:
        assert abs(r["I"] - exact) < 4 * r["sigma"]


def test_gradient_estimator_matches_common_random_number_differences(orc):
    """On a frozen grid with the same random numbers, the estimator gradient
    equals the central difference of the estimator itself (truncation O(h^2))."""
    n = 4
    P = wl.rambo_params(n, cut=1)
    cfg = orc.make_cfg(4 * n, nbins=50, ncall=20000, ybits=24, seed=1)
    e = orc.uniform_grid(4 * n, 50)
    g, I0 = orc.gradient(cfg, orc.Integrand(orc.RAMBO_BW, 4 * n, P), e, 0)
    for j, (slot, h) in enumerate(((wl.RB_M, 1e-3), (wl.RB_GAMMA, 1e-3), (wl.RB_T, 1e-2))):
        pp, pm = P.copy(), P.copy()
        pp[slot] += h
        pm[slot] -= h
        Ip = orc.iteration(cfg, orc.Integrand(orc.RAMBO_BW, 4 * n, pp), e, 0)["I"]
        Im = orc.iteration(cfg, orc.Integrand(orc.RAMBO_BW, 4 * n, pm), e, 0)["I"]
        assert g[j] == pytest.approx((Ip - Im) / (2 * h), rel=1e-3)
    assert I0 == pytest.approx(orc.iteration(cfg, orc.Integrand(orc.RAMBO_BW, 4 * n, P), e, 0)["I"], rel=1e-13)


def test_vegas_and_bases_agree_on_the_same_integrand(orc):
    """The paper's own check, agreement of independent methods within their
    errors: an unstratified VEGAS run and a stratified BASES run of the same
    integrand (disjoint Philox instances) agree within the combined sigma,
    and both agree with the closed form."""
    import closed_forms as cf
    d = 3
    p = wl.genz_gaussian_params(d, a=6.0, u=0.45)
    fn = orc.Integrand(orc.GENZ_GAUSSIAN, d, p)
    exact = cf.genz_gaussian(p[:d], p[d:])
    cv = orc.make_cfg(d, nbins=50, ncall=20000, ybits=53, seed=5, instance=1)
    rv = orc.vegas(cv, fn, orc.uniform_grid(d, 50), 0, 8)
    cb = orc.make_cfg(d, nbins=50, ncall=4 ** d * 300, nstrat=4, ybits=53, seed=5, instance=2)
    rb = orc.bases(cb, fn, orc.uniform_grid(d, 50), 0, 4, 0.0, 4, 0.0)
    comb = math.sqrt(rv["sigma"] ** 2 + rb["sigma"] ** 2)
    assert abs(rv["I"] - rb["I"]) < 4 * comb
    assert abs(rv["I"] - exact) < 4 * rv["sigma"] and abs(rb["I"] - exact) < 4 * rb["sigma"]
