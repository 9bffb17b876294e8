"""Batched integration (vegas_batch_*) against standalone contexts with the
same Philox instance id, against the oracle, and on the 256-instance Genz
workload against closed forms.

Bars: FP64, iteration estimates within 1e-12 relative of the standalone
context and refined grids within 1e-12; compensated FP32, within 1e-5
relative and 0.1 sigma; the oracle loop on the same points (FP64) within
1e-12; every Genz instance within 5 sigma of its closed form.  The FP32
per-dimension kernels against the oracle's first iteration, instance by
instance (d = 1..16, every family, 2 to 256 bins, one or two points in
flight, and sampled instances of the full 256-instance batch in the
benchmarked shape): I within 1e-5 of max(|I|, mean |w|) and 0.1 sigma,
S1 within 1e-5 sum|w|, S2 within 1e-5 sum w^2 + 2e-4 of the cell, with
the weights of points within FP32 rounding of a discontinuity (oracle cut
margin below 1e-4) allowed on top."""
import math

import numpy as np
import pytest

import closed_forms as cf
from paper_1010_2107_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gv():
    from paper_1010_2107_gb300 import _build, gvegas
    _build.build()
    return gvegas


SMALL = [
    dict(kind=wl.GENZ_PRODUCT_PEAK, ndim=3, params=[5.0, 3.0, 7.0, 0.3, 0.5, 0.8], ncall=40_000, instance=3),
    dict(kind=wl.GENZ_CORNER_PEAK, ndim=6, params=[0.3, 0.1, 0.5, 0.2, 0.4, 0.35], ncall=70_001, instance=9),
    dict(kind=wl.GENZ_OSCILLATORY, ndim=2, params=[1.0, 2.0, 0.3], ncall=5_000, instance=0),
    dict(kind=wl.GENZ_GAUSSIAN, ndim=16, params=list(np.full(16, 2.0)) + list(np.full(16, 0.5)), ncall=123_457,
         instance=1),
    dict(kind=wl.DOUBLE_GAUSSIAN, ndim=5, params=[0.3, 0.7, 0.1], ncall=65_536, instance=77),
    dict(kind=wl.GENZ_PRODUCT_PEAK, ndim=1, params=[4.0, 0.2], ncall=3, instance=5),
]


@pytest.mark.parametrize("precision,ybits,tol", [(0, 53, 1e-12), (0, 24, 1e-12), (2, 24, 1e-5), (2, 53, 1e-5)])
def test_batch_matches_standalone_contexts(gv, precision, ybits, tol):
    iters = 3
    with gv.vegas_batch_create(SMALL, precision=precision, ybits=ybits, seed=4) as b:
        gv.vegas_batch_set_launch(b, 128, 16)
        res = gv.vegas_batch_iterate(b, iters)
        for i, ins in enumerate(SMALL):
            with gv.vegas_create(ins["kind"], ins["ndim"], ins["params"], ncall=ins["ncall"], precision=precision,
                                 ybits=ybits, seed=4, instance=ins["instance"]) as ctx:
                r = gv.vegas_iterate(ctx, iters)
                h = gv.vegas_get_history(ctx)
                e = gv.vegas_get_grid(ctx)
            hb = gv.vegas_batch_get_history(b, i)
            eb = gv.vegas_batch_get_grid(b, i)
            assert len(hb) == iters
            sig = np.sqrt(h[:, 1])
            np.testing.assert_allclose(hb[:, 0], h[:, 0], rtol=tol, atol=0.1 * sig.max() if tol > 1e-9 else 1e-300)
            assert np.all(np.abs(hb[:, 0] - h[:, 0]) <= 0.1 * sig + 1e-300)
            np.testing.assert_allclose(eb, e, rtol=0, atol=1e-12 if tol < 1e-9 else 1e-5)
            assert res[i]["I"] == pytest.approx(r["I"], rel=tol, abs=1e-300)
            assert res[i]["iters_done"] == iters


def test_batch_matches_oracle_fp64(gv, orc):
    with gv.vegas_batch_create(SMALL[:3], precision=0, seed=4) as b:
        gv.vegas_batch_iterate(b, 2)
        for i, ins in enumerate(SMALL[:3]):
            cfg = orc.make_cfg(ins["ndim"], nbins=50, ncall=ins["ncall"], ybits=53, seed=4, instance=ins["instance"])
            fn = orc.Integrand(ins["kind"], ins["ndim"], ins["params"])
            e = orc.uniform_grid(ins["ndim"], 50)
            ref = orc.vegas(cfg, fn, e, 0, 2)
            hb = gv.vegas_batch_get_history(b, i)
            np.testing.assert_allclose(hb[:, 0], ref["hist"][:, 0], rtol=1e-12)
            np.testing.assert_allclose(gv.vegas_batch_get_grid(b, i), e, rtol=0, atol=1e-12)


def _closed_form(ins):
    d, p = ins["ndim"], np.asarray(ins["params"])
    if ins["kind"] == wl.GENZ_PRODUCT_PEAK:
        return cf.genz_product_peak(p[:d], p[d:])
    if ins["kind"] == wl.GENZ_OSCILLATORY:
        return cf.genz_oscillatory(p[:d], p[d])
    if ins["kind"] == wl.GENZ_CORNER_PEAK and d <= 10:
        return cf.genz_corner_peak(p[:d], digits=60)
    return None


def test_genz256_workload_against_closed_forms(gv):
    """The batched workload at full size (256 instances, about 2.5e8 points per
    iteration, 8 iterations): every instance with a cheap closed form lies
    within 5 sigma of it; the autotuner picks a valid launch shape."""
    spec = wl.GENZ256
    insts = wl.genz_batch(spec["count"], spec["seed"])
    with gv.vegas_batch_create(insts, precision=2, seed=spec["sample_seed"]) as b:
        tuned = gv.vegas_batch_autotune(b)
        assert tuned["threads"] in (128, 256) and tuned["ms"] > 0
        res = gv.vegas_batch_iterate(b, spec["itmx"])
    checked = 0
    for ins, r in zip(insts, res):
        assert r["iters_done"] == spec["itmx"] and r["nonfinite"] == 0
        exact = _closed_form(ins)
        if exact is None:
            continue
        checked += 1
        assert abs(r["I"] - exact) <= 5 * r["sigma"] + 1e-12 * abs(exact), (ins["kind"], ins["ndim"], r, exact)
    assert checked > 150


def _family_params(kind, d, rng):
    """Parameters of one Genz-family (or two-peak Gaussian) instance: the
    layouts of vegas_create's parameter block."""
    a = rng.uniform(0.5, 3.0, d)
    u = rng.uniform(0.2, 0.8, d)
    if kind in (wl.GENZ_GAUSSIAN, wl.GENZ_PRODUCT_PEAK, wl.GENZ_CONTINUOUS):
        return list(np.concatenate([a, u]))
    if kind == wl.GENZ_CORNER_PEAK:
        return list(a / d)
    if kind == wl.GENZ_OSCILLATORY:
        return list(np.concatenate([a, u[:1]]))
    if kind == wl.GENZ_DISCONTINUOUS:
        return list(np.concatenate([a / d, u[:2]]))
    return [0.3, 0.7, 0.1]  # two-peak Gaussian: centres and width


def _weights_abs(orc, cfg, fn, edges, it, n, chunk=1 << 18):
    """Sum of |w| over the n points of an iteration, and the sums of |w| and
    w^2 over the points within FP32 rounding of a discontinuity (cut margin
    below 1e-4), which may fall on its other side (the oracle, in chunks)."""
    tot, near1, near2 = 0.0, 0.0, 0.0
    for s0 in range(0, n, chunk):
        p = orc.sample_batch(cfg, edges, it, np.arange(s0, min(n, s0 + chunk)))
        w = orc.integrand(fn, p["x"]) * p["jac"]
        tot += np.abs(w).sum()
        near = orc.cut_margin(fn, p["x"]) < 1e-4
        near1 += np.abs(w[near]).sum()
        near2 += (w[near] ** 2).sum()
    return tot, near1, near2


def _check_first_iteration(gv, orc, b, i, ins, N, seed):
    """Instance i of a batch after one refining iteration against the
    oracle's iteration 0 on the uniform grid (FP32 bars: I within 1e-5 of
    max(|I|, mean |w|) and 0.1 sigma, S1 within 1e-5 sum|w|, S2 within
    1e-5 sum w^2 + 2e-4 of the cell)."""
    d = ins["ndim"]
    cfg = orc.make_cfg(d, nbins=N, ncall=ins["ncall"], ybits=24, seed=seed, instance=ins["instance"])
    fn = orc.Integrand(ins["kind"], d, ins["params"])
    e0 = orc.uniform_grid(d, N)
    o = orc.iteration(cfg, fn, e0, 0)
    absw, near1, near2 = _weights_abs(orc, cfg, fn, e0, 0, ins["ncall"])
    hist = gv.vegas_batch_get_history(b, i)
    _, bins = gv.vegas_batch_get_grid(b, i, bin_sums=True)
    I, var = hist[0]
    sig = math.sqrt(o["var"])
    n = ins["ncall"]
    assert abs(I - o["I"]) <= 1e-5 * max(abs(o["I"]), absw / n) + near1 / n + 1e-300, (ins, I, o["I"])
    assert abs(I - o["I"]) <= 0.1 * sig + near1 / n + 1e-300, (ins, I, o["I"], sig)
    assert np.all(np.abs(bins[0] - o["S1"]) <= 1e-5 * absw + near1), ins
    sw2 = o["S2"][0].sum()  # every point lands in one bin of an axis
    assert np.all(np.abs(bins[1] - o["S2"]) <= 1e-5 * sw2 + 2e-4 * np.abs(o["S2"]) + near2), ins


FAMILIES = [wl.GENZ_GAUSSIAN, wl.GENZ_PRODUCT_PEAK, wl.GENZ_CORNER_PEAK, wl.GENZ_OSCILLATORY,
            wl.GENZ_CONTINUOUS, wl.GENZ_DISCONTINUOUS, wl.DOUBLE_GAUSSIAN]


@pytest.mark.parametrize("N", [2, 37, 256])
@pytest.mark.parametrize("pif", [1, 2])
def test_batch_dimension_kernels_against_the_oracle(gv, orc, N, pif):
    """The FP32 batched pass (one kernel per exact dimension, d = 1..16, every
    family, ragged point counts, 2 to 256 bins: tiles from heavy bucket
    overflow to sparse) against the oracle's first iteration, instance by
    instance."""
    rng = np.random.default_rng(100 + N + pif)
    insts = []
    for d in range(1, 17):
        kind = FAMILIES[d % len(FAMILIES)]
        if kind == wl.GENZ_DISCONTINUOUS and d < 2:
            kind = wl.GENZ_GAUSSIAN
        insts.append(dict(kind=kind, ndim=d, params=_family_params(kind, d, rng), ncall=3001 + 977 * d + (d % 3),
                          instance=10 + d))
    with gv.vegas_batch_create(insts, nbins=N, precision=2, ybits=24, seed=6) as b:
        gv.vegas_batch_set_launch(b, 128, 8)
        gv.vegas_batch_set_tile(b, pif)
        gv.vegas_batch_iterate(b, 1)
        for i, ins in enumerate(insts):
            _check_first_iteration(gv, orc, b, i, ins, N, 6)


def test_genz256_first_iteration_against_the_oracle_in_the_benchmarked_shape(gv, orc):
    """The full 256-instance batch (about 2.5e8 points) in the launch shape the
    benchmark times (256 threads, 64 rounds, two points in flight): the first
    iteration of sampled instances, one of every dimension present with at
    most 2^20 points and the largest one, against the oracle."""
    spec = wl.GENZ256
    insts = wl.genz_batch(spec["count"], spec["seed"])
    pick = {}
    for i, ins in enumerate(insts):
        if ins["ncall"] <= 1 << 20 and ins["ndim"] not in pick:
            pick[ins["ndim"]] = i
    big = max(range(len(insts)), key=lambda i: insts[i]["ncall"] * insts[i]["ndim"])
    chosen = sorted(set(pick.values()) | {big})
    with gv.vegas_batch_create(insts, nbins=spec["nbins"], precision=2, ybits=24, seed=spec["sample_seed"]) as b:
        gv.vegas_batch_set_launch(b, 256, 64)
        gv.vegas_batch_set_tile(b, 2)
        gv.vegas_batch_iterate(b, 1)
        for i in chosen:
            _check_first_iteration(gv, orc, b, i, insts[i], spec["nbins"], spec["sample_seed"])
    assert len(chosen) >= 10


@pytest.mark.parametrize("precision,ybits", [(0, 53), (2, 24)])
def test_batch_set_params_matches_a_batch_created_with_them(gv, precision, ybits):
    """vegas_batch_set_params on a batch whose iteration graph is already
    captured, for a range of instances, gives the run of a batch created
    with the new parameters (first iteration identical, the next within the
    run-to-run reproducibility of the per-bin sums); a short stride or a
    range outside the batch is refused with nothing changed."""
    new = [dict(ins) for ins in SMALL]
    for ins in new[1:4]:
        p = np.asarray(ins["params"], dtype=float)
        ins["params"] = list(p * 1.1) if ins["kind"] != wl.GENZ_OSCILLATORY else list(p + 0.05)
    with gv.vegas_batch_create(SMALL, precision=precision, ybits=ybits, seed=4) as b1, \
            gv.vegas_batch_create(new, precision=precision, ybits=ybits, seed=4) as b2:
        for b in (b1, b2):
            gv.vegas_batch_set_launch(b, 128, 16)
        gv.vegas_batch_iterate(b1, 2)  # captures the two-iteration graph
        rows = [ins["params"] for ins in new[1:4]]
        with pytest.raises(gv.VegasError):
            gv.vegas_batch_set_params(b1, rows, first=len(SMALL) - 2)  # runs past the end
        short = np.zeros((3, 1))
        with pytest.raises(gv.VegasError):
            gv.vegas_batch_set_params(b1, short, first=1)
        gv.vegas_batch_set_params(b1, rows, first=1)
        for b in (b1, b2):
            gv.vegas_batch_reset(b)
            gv.vegas_batch_iterate(b, 2)
        tol = 1e-12 if precision == 0 else 1e-5
        for i in range(len(SMALL)):
            h1, h2 = gv.vegas_batch_get_history(b1, i), gv.vegas_batch_get_history(b2, i)
            assert h1[0, 0] == h2[0, 0] and h1[0, 1] == h2[0, 1], i
            np.testing.assert_allclose(h1[1], h2[1], rtol=tol)
            np.testing.assert_allclose(gv.vegas_batch_get_grid(b1, i), gv.vegas_batch_get_grid(b2, i), rtol=0,
                                       atol=1e-12 if precision == 0 else 1e-5)


def test_general_batch_kernel_layout_is_sized_for_the_widest_instance(gv, orc):
    """The FP64 form (one kernel for every instance) sizes its shared memory
    for the batch's widest instance: 256 bins fit up to ten axes (checked
    against the oracle's first iteration, FP64 bars), while sixteen axes at
    256 bins do not fit and the batch is refused at creation."""
    rng = np.random.default_rng(7)
    insts = [dict(kind=wl.GENZ_GAUSSIAN if d != 5 else wl.GENZ_CORNER_PEAK, ndim=d,
                  params=_family_params(wl.GENZ_GAUSSIAN if d != 5 else wl.GENZ_CORNER_PEAK, d, rng),
                  ncall=20_011 + d, instance=40 + d) for d in (2, 5, 10)]
    with gv.vegas_batch_create(insts, nbins=256, precision=0, ybits=53, seed=3) as b:
        gv.vegas_batch_iterate(b, 1)
        for i, ins in enumerate(insts):
            d = ins["ndim"]
            cfg = orc.make_cfg(d, nbins=256, ncall=ins["ncall"], ybits=53, seed=3, instance=ins["instance"])
            fn = orc.Integrand(ins["kind"], d, ins["params"])
            o = orc.iteration(cfg, fn, orc.uniform_grid(d, 256), 0)
            I, _ = gv.vegas_batch_get_history(b, i)[0]
            _, bins = gv.vegas_batch_get_grid(b, i, bin_sums=True)
            assert I == pytest.approx(o["I"], rel=1e-12)
            assert np.all(np.abs(bins[0] - o["S1"]) <= 1e-12 * o["S1"][0].sum())
            assert np.all(np.abs(bins[1] - o["S2"]) <= 1e-12 * o["S2"][0].sum())
    wide = [dict(kind=wl.GENZ_GAUSSIAN, ndim=16, params=_family_params(wl.GENZ_GAUSSIAN, 16, rng), ncall=5000,
                 instance=1)]
    with pytest.raises(gv.VegasError):
        gv.vegas_batch_create(wide, nbins=256, precision=0, ybits=53, seed=3)
