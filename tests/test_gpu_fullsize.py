"""Parity at the full workload sizes, in the launch configuration bench.py
times (the default launch shape of a context).

dgauss8 (BASES, 2^22 points, FP32 compensated): one iteration against the
oracle's full iteration on the same points (I within 1e-5 relative and
0.1 sigma, per-bin sums within 1e-5 sum|w|), sampled hypercube sums and
points one by one, and the whole 5 + 5 BASES run (within 0.1 sigma and
1e-4 relative: the FP32 and FP64 grids drift apart at the 1e-6 level over
five refinements).
rambo5 (VEGAS, 2^24 points, 20 dims): sampled points one by one on the
refined grid; the full-iteration estimate against the oracle on the first
2^16 of the same points (statistical); per-axis consistency of the bin sums.
rambo4_adjoint (2^24 points): the FP64 gradient against common-random-number
central differences of the FP64 estimate (1e-3; FP32 cannot resolve
M^2/s to the step size), and the FP32 gradient against the FP64 one on
the same points and grid within 1e-4 of the mean |J df/dtheta| (the
condition-scaled FP32 bar of the small-case gradient parity: the M and
Gamma derivatives change sign across the Breit-Wigner peak, so their sums
cancel).  A point within the FP32 cut margin may be cut by one arithmetic
and kept by the other (the reading of the point parity); such points are
found by dumping every point inside the margin, and their terms (J
df/dtheta without the hard Delta R cut) are moved to the FP32 side before
the comparison.  The oracle scans all 2^24 points."""
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


def _ctx(gv, w, **kw):
    return gv.vegas_create(w["kind"], w["ndim"], w["params"], nbins=w["nbins"], ncall=w["ncall"],
                           nstrat=w["nstrat"], seed=w["seed"], ybits=w["ybits"],
                           precision=gv.PRECISIONS[w["precision"]], **kw)


def _near_cut(orc, cfg, fn, edges, it, n, chunk=1 << 20):
    """Indices of the points whose oracle cut margin is below 1e-4, the FP32
    bar of the point parity: only these may be cut in one arithmetic and
    kept in the other."""
    near = []
    for c0 in range(0, n, chunk):
        idx = np.arange(c0, min(c0 + chunk, n))
        near.append(idx[orc.cut_margin(fn, orc.sample_batch(cfg, edges, it, idx)["x"]) < 1e-4])
    return np.concatenate(near)


def test_dgauss8_full_iteration(gv, orc):
    w = wl.WORKLOADS["dgauss8"]
    d, N, n = w["ndim"], w["nbins"], w["ncall"]
    with _ctx(gv, w) as ctx:
        I, var = gv.vegas_eval(ctx, 0)
        _, bins = gv.vegas_get_grid(ctx, bin_sums=True)
        cubes = gv.vegas_get_cube_sums(ctx)
        rng = np.random.default_rng(8)
        s = np.unique(rng.integers(0, n, 2000))
        dump = gv.vegas_sample_dump(ctx, 0, s)
    cfg = orc.make_cfg(d, nbins=N, ncall=n, nstrat=w["nstrat"], ybits=w["ybits"], seed=w["seed"])
    fn = orc.Integrand(w["kind"], d, w["params"])
    e = orc.uniform_grid(d, N)
    o = orc.iteration(cfg, fn, e, 0, cubes=True)
    sig = math.sqrt(o["var"])
    assert abs(I - o["I"]) <= 1e-5 * abs(o["I"]) and abs(I - o["I"]) <= 0.1 * sig
    assert abs(math.sqrt(var) - sig) <= 1e-3 * sig
    tot1, tot2 = np.abs(o["S1"]).sum(axis=1, keepdims=True), o["S2"].sum(axis=1, keepdims=True)
    assert np.all(np.abs(bins[0] - o["S1"]) <= 1e-5 * tot1)
    assert np.all(np.abs(bins[1] - o["S2"]) <= 1e-5 * tot2)
    # the cube sums the kernel reported for the vegas_eval pass above
    pick = np.unique(rng.integers(0, len(o["C1"]), 300))
    np.testing.assert_allclose(cubes[pick, 0], o["C1"][pick], rtol=1e-5, atol=1e-5 * np.abs(o["C1"]).max())
    # sampled points one by one
    p = orc.sample_batch(cfg, e, 0, s)
    assert np.array_equal(dump["words"], p["words"]) and np.array_equal(dump["bins"], p["bins"])
    fo = orc.integrand(fn, p["x"]) * p["jac"]
    np.testing.assert_allclose(dump["f"] * dump["jac"], fo, rtol=2e-5, atol=1e-6 * np.abs(fo).max())


def test_dgauss8_full_bases_run(gv, orc):
    w = wl.WORKLOADS["dgauss8"]
    d, N = w["ndim"], w["nbins"]
    with _ctx(gv, w) as ctx:
        out, ph1 = gv.bases_integrate(ctx, w["itmx1"], 0.0, w["itmx2"], 0.0)
    cfg = orc.make_cfg(d, nbins=N, ncall=w["ncall"], nstrat=w["nstrat"], ybits=w["ybits"], seed=w["seed"])
    fn = orc.Integrand(w["kind"], d, w["params"])
    ref = orc.bases(cfg, fn, orc.uniform_grid(d, N), 0, w["itmx1"], 0.0, w["itmx2"], 0.0)
    assert abs(out["I"] - ref["I"]) <= 0.1 * ref["sigma"]
    assert abs(out["I"] - ref["I"]) <= 1e-4 * abs(ref["I"])
    assert out["sigma"] == pytest.approx(ref["sigma"], rel=1e-2)
    assert abs(out["I"] - 1.0) < 5 * out["sigma"]  # the normalised two-peak integral


def test_rambo5_full_size(gv, orc):
    w = wl.WORKLOADS["rambo5"]
    d, N, n = w["ndim"], w["nbins"], w["ncall"]
    with _ctx(gv, w) as ctx:
        gv.vegas_iterate(ctx, 3, refine=True)
        edges = gv.vegas_get_grid(ctx)
        I, var = gv.vegas_eval(ctx, 3)
        _, bins = gv.vegas_get_grid(ctx, bin_sums=True)
        rng = np.random.default_rng(9)
        s = np.unique(rng.integers(0, n, 3000))
        dump = gv.vegas_sample_dump(ctx, 3, s)
    cfg = orc.make_cfg(d, nbins=N, ncall=n, ybits=w["ybits"], seed=w["seed"])
    fn = orc.Integrand(w["kind"], d, w["params"])
    p = orc.sample_batch(cfg, edges, 3, s)
    assert np.array_equal(dump["words"], p["words"]) and np.array_equal(dump["bins"], p["bins"])
    fo = orc.integrand(fn, p["x"]) * p["jac"]
    ok = np.isclose(dump["f"] * dump["jac"], fo, rtol=2e-4, atol=1e-300)
    assert np.mean(ok) >= 0.99
    # every axis partitions the same points
    S1 = bins[0].sum(axis=1)
    np.testing.assert_allclose(S1, S1[0], rtol=1e-6)
    # the first 2^16 points of this iteration through the oracle: same estimate
    sub = orc.iteration(orc.make_cfg(d, nbins=N, ncall=1 << 16, ybits=w["ybits"], seed=w["seed"]), fn, edges, 3)
    assert abs(I - sub["I"]) <= 5 * math.sqrt(sub["var"] + var)


def test_rambo5_full_iteration_in_the_tuned_shape(gv, orc):
    """rambo5 at full size (2^24 points, 20 dims) in the launch shape the
    autotuner picks (the one bench.py times), on a refined grid: sampled
    words and bins bit-exact, then the whole iteration against the oracle's
    on the same points and grid: I within 1e-5 relative and 0.1 sigma,
    per-bin sums S1 within 1e-5 of sum |w|, S2 within 1e-5 of sum w^2 plus
    2 eps of the cell itself (eps = 1e-4, the FP32 bar on one weight: a few
    points can carry most of a cell's sum of squares, and their FP32 error
    passes into it undiluted).  A point within the FP32 cut margin that the
    GPU cuts and the oracle keeps, or the reverse, is found by dumping every
    point inside the margin, and the oracle's sums take the GPU's decision
    for it before the comparison."""
    w = wl.WORKLOADS["rambo5"]
    d, N, n = w["ndim"], w["nbins"], w["ncall"]
    cfg = orc.make_cfg(d, nbins=N, ncall=n, ybits=w["ybits"], seed=w["seed"])
    fn = orc.Integrand(w["kind"], d, w["params"])
    with _ctx(gv, w) as ctx:
        gv.vegas_iterate(ctx, 2, refine=True)
        gv.vegas_autotune(ctx)
        edges = gv.vegas_get_grid(ctx)
        I, var = gv.vegas_eval(ctx, 2)
        _, bins = gv.vegas_get_grid(ctx, bin_sums=True)
        s = np.unique(np.concatenate([[0, n - 1], np.random.default_rng(12).integers(0, n, 4000)]))
        dump = gv.vegas_sample_dump(ctx, 2, s)
        near = _near_cut(orc, cfg, fn, edges, 2, n)
        dn = gv.vegas_sample_dump(ctx, 2, near)
    p = orc.sample_batch(cfg, edges, 2, s)
    assert np.array_equal(dump["words"], p["words"]) and np.array_equal(dump["bins"], p["bins"])
    o = orc.iteration(cfg, fn, edges, 2)
    pn = orc.sample_batch(cfg, edges, 2, near)
    wo, wg = orc.integrand(fn, pn["x"]) * pn["jac"], dn["f"] * dn["jac"]
    flip = (wg != 0) != (wo != 0)
    d1, d2 = np.where(flip, wg - wo, 0.0), np.where(flip, wg * wg - wo * wo, 0.0)
    S1, S2 = o["S1"].copy(), o["S2"].copy()
    for a in range(d):
        np.add.at(S1[a], pn["bins"][:, a], d1)
        np.add.at(S2[a], pn["bins"][:, a], d2)
    Io = o["I"] + d1.sum() / n
    sig = math.sqrt(o["var"])
    assert abs(I - Io) <= 1e-5 * abs(Io), (I, Io, int(flip.sum()))
    assert abs(I - Io) <= 0.1 * sig
    tot1, tot2 = np.abs(S1).sum(axis=1, keepdims=True), S2.sum(axis=1, keepdims=True)
    assert np.all(np.abs(bins[0] - S1) <= 1e-5 * tot1)
    assert np.all(np.abs(bins[1] - S2) <= 1e-5 * tot2 + 2e-4 * S2)


def test_rambo4_adjoint_full_size(gv, orc):
    w = wl.WORKLOADS["rambo4_adjoint"]
    params = np.asarray(w["params"], dtype=np.float64)
    n = w["ncall"]
    cfg = orc.make_cfg(w["ndim"], nbins=w["nbins"], ncall=n, ybits=w["ybits"], seed=w["seed"])
    fn = orc.Integrand(w["kind"], w["ndim"], params)
    with _ctx(gv, w) as c32:
        gv.vegas_iterate(c32, w["warmup_iters"], refine=True)
        edges = gv.vegas_get_grid(c32)
        g32, _ = gv.vegas_grad(c32, 100)
        # the same points by the oracle: mean |J df/dtheta| and the points
        # inside the FP32 cut margin, whose FP32 values are dumped
        total, near = np.zeros(3), []
        for c0 in range(0, n, 1 << 20):
            idx = np.arange(c0, min(c0 + (1 << 20), n))
            p = orc.sample_batch(cfg, edges, 100, idx)
            total += np.abs(orc.integrand_grad(fn, p["x"]) * p["jac"][:, None]).sum(axis=0)
            near.append(idx[orc.cut_margin(fn, p["x"]) < 1e-4])
        near = np.concatenate(near)
        dn = gv.vegas_sample_dump(c32, 100, near)
    scale = total / n
    # a point that FP32 keeps and the oracle (like the FP64 form) cuts, or
    # the reverse, moves the FP32 sum by its term without the hard cut
    pn = orc.sample_batch(cfg, edges, 100, near)
    kept32, kept = dn["f"] != 0, orc.integrand(fn, pn["x"]) != 0
    flip = kept32 != kept
    corr = np.zeros(3)
    if flip.any():
        free = params.copy()
        free[wl.RB_DRMIN] = 0.0
        t = orc.integrand_grad(orc.Integrand(w["kind"], w["ndim"], free), pn["x"][flip]) * pn["jac"][flip, None]
        corr = (np.where(kept32[flip], 1.0, -1.0)[:, None] * t).sum(axis=0) / n
    with _ctx(gv, dict(w, precision="fp64")) as ctx:
        gv.vegas_set_grid(ctx, edges)
        g, I = gv.vegas_grad(ctx, 100)
        assert np.all(np.abs(g32 - (g + corr)) <= 1e-4 * scale), (g32, g, corr, scale, int(flip.sum()))
        for j, (slot, h) in enumerate(((wl.RB_M, 1e-3), (wl.RB_GAMMA, 1e-3), (wl.RB_T, 1e-2))):
            pp, pm = params.copy(), params.copy()
            pp[slot] += h
            pm[slot] -= h
            gv.vegas_set_params(ctx, pp)
            Ip, _ = gv.vegas_eval(ctx, 100)
            gv.vegas_set_params(ctx, pm)
            Im, _ = gv.vegas_eval(ctx, 100)
            gv.vegas_set_params(ctx, params)
            fd = (Ip - Im) / (2 * h)
            assert g[j] == pytest.approx(fd, rel=1e-3), (j, g[j], fd)
