"""Pins of the oracle's SPRING (event generation on the frozen grid of the
BASES integration phase; Sec. 2.1 names it, the steps follow Kawabata's
SPRING with an integer cube choice) against what the mathematics fixes:

* the integer cube table is the stated ceiling, recomputed in numpy;
* per-cube maxima are the brute-force maxima of the weights;
* with a constant integrand every trial is kept and the chosen cube is the
  one Python big-integer arithmetic picks from the same Philox words;
* with exact per-cube bounds SPRING is exact rejection sampling: the kept
  points follow f / I (chi-square over bins, closed-form bin masses) and
  the acceptance rate is I / (sum of bounds / G);
* trials are counter-based: any sub-range reproduces the same events.
"""
import math

import numpy as np
import pytest

import oracle as orc


def test_cube_table_is_the_stated_ceiling():
    rng = np.random.default_rng(5)
    M = rng.uniform(0, 3, 257)
    M[[3, 50, 99]] = 0.0
    q, scale = orc.spring_table(M)
    assert scale == 2.0 ** 24 / M.max()
    ref = np.where(M > 0, np.ceil(M * scale), 0).astype(np.uint64)
    np.testing.assert_array_equal(q, ref)
    assert q.max() == 2 ** 24 and q[3] == 0
    with pytest.raises(ValueError):
        orc.spring_table(np.zeros(4))


def test_cube_maxima_are_brute_force_maxima():
    d, g, nc = 2, 4, 37
    cfg = orc.make_cfg(d, nbins=10, ncall=g ** d * nc, nstrat=g, ybits=53)
    fn = orc.Integrand(orc.GENZ_PRODUCT_PEAK, d, np.array([5.0, 3.0, 0.3, 0.6]))
    e = orc.uniform_grid(d, 10)
    r = orc.iteration(cfg, fn, e, 3, cubes=True)
    p = orc.sample_batch(cfg, e, 3, np.arange(g ** d * nc))
    w = orc.integrand(fn, p["x"]) * p["jac"]
    np.testing.assert_array_equal(r["Cmax"], np.maximum(w.reshape(-1, nc).max(axis=1), 0.0))


def _words(cfg, t, nw):
    key = [cfg.seed & 0xFFFFFFFF, cfg.seed >> 32]
    out = []
    for q in range((nw + 3) // 4):
        out += list(orc.philox([t, q, 0xFFFFFFFF, cfg.instance], key))
    return [int(v) for v in out[:nw]]


@pytest.mark.parametrize("ybits", [24, 53])
def test_constant_integrand_keeps_every_trial_in_the_chosen_cube(ybits):
    d, g = 3, 3
    # 8 bins: edges k/8 exact, so J = 1 exactly and every weight is 1
    cfg = orc.make_cfg(d, nbins=8, ncall=g ** d * 2, nstrat=g, ybits=ybits, seed=7)
    fn = orc.Integrand(orc.GENZ_CORNER_PEAK, d, np.zeros(d))  # (1 + 0)^-(d+1) = 1
    e = orc.uniform_grid(d, 8)
    M = np.ones(g ** d)
    n = 400
    r = orc.spring(cfg, fn, e, M, 0, n)
    assert len(r["x"]) == n and r["overflow"] == 0 and r["nonpos"] == 0
    np.testing.assert_array_equal(r["trial"], np.arange(n))
    W = d if ybits == 24 else 2 * d
    Q = g ** d * 2 ** 24
    for t in range(0, n, 37):
        w = _words(cfg, t, W + 4)
        U = (w[W] << 32) | w[W + 1]
        c = ((U * Q) >> 64) // 2 ** 24
        digits = [(c // g ** a) % g for a in range(d)]
        np.testing.assert_array_equal(np.floor(r["x"][t] * g).astype(int), digits)


def _pp_exact_max(a, u, lo, hi):
    x = min(max(u, lo), hi)  # closest point of [lo, hi] to the peak
    return 1.0 / (a ** -2 + (x - u) ** 2)


@pytest.mark.parametrize("ybits", [24, 53])
def test_exact_bounds_give_exact_rejection_sampling(ybits):
    a, u, g = 5.0, 0.3, 8
    cfg = orc.make_cfg(1, nbins=4, ncall=g * 2, nstrat=g, ybits=ybits, seed=3)
    fn = orc.Integrand(orc.GENZ_PRODUCT_PEAK, 1, np.array([a, u]))
    e = orc.uniform_grid(1, 4)  # J = 1, x = y
    M = np.array([_pp_exact_max(a, u, c / g, (c + 1) / g) for c in range(g)])
    # rounding the bounds up keeps them bounds: no overflow can occur
    n = 200_000
    r = orc.spring(cfg, fn, e, M, 0, n)
    assert r["overflow"] == 0 and r["nonpos"] == 0
    F = lambda x: a * math.atan(a * (x - u))  # antiderivative of f
    I = F(1.0) - F(0.0)
    q, scale = orc.spring_table(M)
    Mt = q.astype(float) / scale
    p_acc = I / (Mt.sum() / g)
    k = len(r["x"])
    assert abs(k / n - p_acc) < 5 * math.sqrt(p_acc * (1 - p_acc) / n)
    edges = np.linspace(0, 1, 21)
    obs = np.histogram(r["x"][:, 0], edges)[0]
    exp = k * np.array([(F(edges[j + 1]) - F(edges[j])) / I for j in range(20)])
    chi2 = ((obs - exp) ** 2 / exp).sum()
    assert chi2 < 19 + 6 * math.sqrt(2 * 19)  # 19 degrees of freedom, far tail


def test_trials_are_counter_based():
    d, g = 2, 2
    cfg = orc.make_cfg(d, nbins=6, ncall=g ** d * 50, nstrat=g, ybits=24)
    fn = orc.Integrand(orc.GENZ_GAUSSIAN, d, np.array([4.0, 4.0, 0.4, 0.5]))
    e = orc.uniform_grid(d, 6)
    M = orc.iteration(cfg, fn, e, 0, cubes=True)["Cmax"]
    full = orc.spring(cfg, fn, e, M, 0, 3000)
    head = orc.spring(cfg, fn, e, M, 0, 1200)
    tail = orc.spring(cfg, fn, e, M, 1200, 1800)
    k = len(head["x"])
    np.testing.assert_array_equal(full["trial"], np.concatenate([head["trial"], tail["trial"]]))
    np.testing.assert_array_equal(full["x"][:k], head["x"])
    np.testing.assert_array_equal(full["x"][k:], tail["x"])
    assert full["overflow"] == head["overflow"] + tail["overflow"]


def test_non_positive_weights_are_dropped():
    d = 2
    cfg = orc.make_cfg(d, nbins=5, ncall=400, ybits=24)
    fn = orc.Integrand(orc.GENZ_OSCILLATORY, d, np.array([0.0, 9.0, 9.0]))  # cos(9 x1 + 9 x2)
    e = orc.uniform_grid(d, 5)
    r = orc.spring(cfg, fn, e, np.array([1.0]), 0, 5000)
    f = orc.integrand(fn, r["x"])
    assert r["nonpos"] > 1000 and np.all(f > 0)
