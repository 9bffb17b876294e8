"""The allocation-free evaluation pass (vegas_eval_noalloc) against the
context-based one (vegas_eval), through the C ABI.

Callers that cannot call cudaMalloc (a fixed memory pool owned by another
runtime, a loop that must not allocate after start-up) use this entry point
with their own device buffers; its intermediates live in a static array of
the library.  This file is collected last so that a failure here stops a
``-x`` run only after every other test has run; it passes on its own too.
"""
import numpy as np
import pytest

from paper_1010_2107_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

CASES = [
    # kind, ndim, params, nbins, ncall, nstrat, precision, ybits, tolerance
    (wl.GENZ_GAUSSIAN, 4, wl.genz_gaussian_params(4), 50, 100_000, 0, 0, 53, 1e-12),
    (wl.DOUBLE_GAUSSIAN, 8, wl.double_gaussian_params(), 50, 4 ** 8 * 8, 4, 2, 24, 1e-5),
    (wl.RAMBO_BW, 20, wl.rambo_params(5), 50, 1 << 16, 0, 2, 24, 1e-5),
]


@pytest.mark.parametrize("kind,d,params,N,ncall,g,prec,ybits,tol", CASES,
                         ids=["gauss4_fp64", "dgauss8_strat_fp32", "rambo5_fp32"])
def test_noalloc_pass_matches_context_pass(orc, kind, d, params, N, ncall, g, prec, ybits, tol):
    torch = pytest.importorskip("torch")
    from paper_1010_2107_gb300 import _build
    from paper_1010_2107_gb300 import gvegas as gv
    _build.build()
    kw = dict(nbins=N, ncall=ncall, nstrat=g, precision=prec, ybits=ybits, seed=7)
    edges = np.tile(np.arange(N + 1, dtype=np.float64) / N, (d, 1))
    d_edges = torch.tensor(edges, dtype=torch.float64, device="cuda")
    d_out = torch.full((2 * d * N + 5,), float("nan"), dtype=torch.float64, device="cuda")
    with gv.vegas_create(kind, d, params, **kw) as ctx:
        for it in (3, 4):  # two calls in a row, each against the context pass
            I_ref, var_ref = gv.vegas_eval(ctx, it)
            _, bins_ref = gv.vegas_get_grid(ctx, bin_sums=True)
            torch.cuda.synchronize()
            gv.vegas_eval_noalloc(kind, d, params, d_edges.data_ptr(), it, d_out.data_ptr(), **kw)
            torch.cuda.synchronize()
            out = d_out.cpu().numpy()
            bins = out[:2 * d * N].reshape(2, d, N)
            I, var = out[2 * d * N], out[2 * d * N + 1]
            scale1 = np.abs(bins_ref[0]).sum(axis=1, keepdims=True)
            scale2 = np.abs(bins_ref[1]).sum(axis=1, keepdims=True)
            assert np.all(np.abs(bins[0] - bins_ref[0]) <= tol * scale1)
            assert np.all(np.abs(bins[1] - bins_ref[1]) <= tol * scale2)
            assert abs(I - I_ref) <= tol * abs(I_ref)
            assert abs(var - var_ref) <= max(tol, 1e-6) * var_ref
            assert out[2 * d * N + 4] == 0.0
            # and directly against the oracle's iteration on the same points
            cfg = orc.make_cfg(d, nbins=N, ncall=ncall, nstrat=g, ybits=ctx.ybits, seed=7)
            o = orc.iteration(cfg, orc.Integrand(kind, d, params), edges, it)
            s1 = np.abs(o["S1"]).sum(axis=1, keepdims=True)  # sum |w| (w >= 0 here)
            s2 = np.abs(o["S2"]).sum(axis=1, keepdims=True)
            assert np.all(np.abs(bins[0] - o["S1"]) <= tol * s1)
            # S2 also within twice the FP32 bar on one weight (1e-4) of the
            # cell: a single point can carry most of a cell's sum of squares
            s2cell = 0.0 if prec == 0 else 2e-4 * np.abs(o["S2"])
            assert np.all(np.abs(bins[1] - o["S2"]) <= tol * s2 + s2cell)
            assert abs(I - o["I"]) <= tol * abs(o["I"])
            if prec != 0:
                assert abs(I - o["I"]) <= 0.1 * np.sqrt(o["var"])


def test_noalloc_between_context_passes_with_another_shape(orc):
    """A context's captured VEGAS and BASES graphs replay correctly after a
    no-allocation pass of the same compiled kernel with fewer bins (a
    smaller shared-memory tile) ran in between; every result against the
    oracle."""
    torch = pytest.importorskip("torch")
    from paper_1010_2107_gb300 import _build
    from paper_1010_2107_gb300 import gvegas as gv
    _build.build()
    d, kind, params = 4, wl.GENZ_GAUSSIAN, wl.genz_gaussian_params(4)
    fn = orc.Integrand(kind, d, params)

    def small_noalloc(it):
        n_small = 10
        e = np.tile(np.arange(n_small + 1, dtype=np.float64) / n_small, (d, 1))
        d_e = torch.tensor(e, dtype=torch.float64, device="cuda")
        d_o = torch.zeros(2 * d * n_small + 5, dtype=torch.float64, device="cuda")
        gv.vegas_eval_noalloc(kind, d, params, d_e.data_ptr(), it, d_o.data_ptr(), nbins=n_small,
                              ncall=30_000, precision=0, seed=3)
        torch.cuda.synchronize()
        out = d_o.cpu().numpy()
        cfg = orc.make_cfg(d, nbins=n_small, ncall=30_000, ybits=53, seed=3)
        o = orc.iteration(cfg, fn, e, it)
        assert abs(out[2 * d * n_small] - o["I"]) <= 1e-12 * abs(o["I"])

    # VEGAS: 2 iterations (graph captured), the small pass, 2 more (replayed)
    kw = dict(nbins=50, ncall=20_000, precision=0, seed=5)
    with gv.vegas_create(kind, d, params, **kw) as ctx:
        gv.vegas_iterate(ctx, 2, refine=True)
        small_noalloc(1)
        r = gv.vegas_iterate(ctx, 2, refine=True)
        hist = gv.vegas_get_history(ctx)
    cfg = orc.make_cfg(d, nbins=50, ncall=20_000, ybits=53, seed=5)
    ref = orc.vegas(cfg, fn, orc.uniform_grid(d, 50), 0, 4)
    np.testing.assert_allclose(hist[:, 0], ref["hist"][:, 0], rtol=1e-12)
    assert r["I"] == pytest.approx(ref["I"], rel=1e-12)

    # BASES: a run (graph captured), the small pass, the same run again from
    # the uniform grid (replayed) on the next Philox iterations
    kw = dict(nbins=50, ncall=2 ** 4 * 500, nstrat=2, precision=0, seed=5)
    with gv.vegas_create(kind, d, params, **kw) as ctx:
        gv.bases_integrate(ctx, 2, 0.0, 2, 0.0)
        small_noalloc(2)
        gv.vegas_reset_grid(ctx)
        out, _ = gv.bases_integrate(ctx, 2, 0.0, 2, 0.0)
    cfg = orc.make_cfg(d, nbins=50, ncall=2 ** 4 * 500, nstrat=2, ybits=53, seed=5)
    ref = orc.bases(cfg, fn, orc.uniform_grid(d, 50), 4, 2, 0.0, 2, 0.0)
    assert out["I"] == pytest.approx(ref["I"], rel=1e-12)
    assert out["sigma"] == pytest.approx(ref["sigma"], rel=1e-9)


def test_noalloc_rejects_bad_arguments():
    """Host-side checks that fail before any launch: NULL device buffers, an
    iteration index beyond 2^31 - 1 and an out-of-range shape.  Only NULL or
    real device addresses are ever passed."""
    torch = pytest.importorskip("torch")
    from paper_1010_2107_gb300 import _build
    from paper_1010_2107_gb300 import gvegas as gv
    _build.build()
    d, N = 4, 50
    p = wl.genz_gaussian_params(d)
    d_edges = torch.zeros((d, N + 1), dtype=torch.float64, device="cuda")
    d_out = torch.zeros(2 * d * N + 5, dtype=torch.float64, device="cuda")
    with pytest.raises(gv.VegasError) as e:
        gv.vegas_eval_noalloc(wl.GENZ_GAUSSIAN, d, p, 0, 0, d_out.data_ptr(), ncall=1000)
    assert e.value.status == gv.EINVAL
    with pytest.raises(gv.VegasError) as e:
        gv.vegas_eval_noalloc(wl.GENZ_GAUSSIAN, d, p, d_edges.data_ptr(), 0, 0, ncall=1000)
    assert e.value.status == gv.EINVAL
    with pytest.raises(gv.VegasError) as e:
        gv.vegas_eval_noalloc(wl.GENZ_GAUSSIAN, d, p, d_edges.data_ptr(), 1 << 31, d_out.data_ptr(),
                              ncall=1000)
    assert e.value.status == gv.EINVAL
    with pytest.raises(gv.VegasError) as e:
        gv.vegas_eval_noalloc(wl.GENZ_GAUSSIAN, d, p, d_edges.data_ptr(), 0, d_out.data_ptr(),
                              ncall=1000, nbins=1000)
    assert e.value.status == gv.EINVAL
    torch.cuda.synchronize()
