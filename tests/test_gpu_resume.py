"""Exact resume: the grid (vegas_get_grid / vegas_set_grid) and the Philox
iteration counter (vegas_get_iteration / vegas_set_iteration) carry a run
into a fresh context, which then continues as if never interrupted.  BASES
keeps its optimised grid for the integration phase and for SPRING (Sec. 2.1);
this is the same hand-over between contexts."""
import numpy as np
import pytest

from paper_1010_2107_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gv():
    from paper_1010_2107_gb300 import _build, gvegas
    _build.build()
    return gvegas


CASES = [
    # kind, ndim, params, create kwargs, total iterations, split
    ("gauss4_fp64", wl.GENZ_GAUSSIAN, 4, wl.genz_gaussian_params(4), dict(ncall=50_000, precision=0), 6, 3),
    ("dgauss4_strat_fp32", wl.DOUBLE_GAUSSIAN, 4, wl.double_gaussian_params(),
     dict(ncall=4 ** 4 * 40, nstrat=4, precision=2, ybits=24), 5, 2),
    ("rambo3_fp64", wl.RAMBO_BW, 12, wl.rambo_params(3), dict(ncall=40_000, precision=0), 3, 1),
]


@pytest.mark.parametrize("name,kind,d,params,kw,total,split", CASES, ids=[c[0] for c in CASES])
def test_resume_in_a_fresh_context_matches_the_uninterrupted_run(gv, orc, name, kind, d, params, kw, total,
                                                                 split):
    """Context a runs `split` refining iterations, hands its grid and counter
    to a fresh context b, and runs on; b resumes from the hand-over.  The
    iteration estimates and cube sums are fixed-order sums, so b's first
    iteration equals a's bit for bit, and so does every iteration on a
    frozen grid.  The per-bin sums that drive refinement are summed in the
    order the histogram buckets were claimed (shared-memory atomics), which
    varies from run to run in the last bits; a refined grid therefore
    carries those bits on.  Refining FP64 runs agree to 1e-12 over two
    refinements; every further refinement amplifies the difference (about
    a hundredfold for the heavy-tailed RAMBO weights)."""
    kw = dict(kw, nbins=50, seed=11)
    rest = total - split
    with gv.vegas_create(kind, d, params, **kw) as a:
        gv.vegas_iterate(a, split, refine=True)
        edges_mid = gv.vegas_get_grid(a)
        it_mid = gv.vegas_get_iteration(a)
        gv.vegas_iterate(a, rest, refine=True)
        hist_a = gv.vegas_get_history(a)[split:]
        edges_a = gv.vegas_get_grid(a)
        gv.vegas_set_grid(a, edges_mid)  # and the same hand-over on a frozen grid
        gv.vegas_set_iteration(a, it_mid)
        gv.vegas_reset_results(a)
        gv.vegas_iterate(a, rest, refine=False)
        frozen_a = gv.vegas_get_history(a)
    assert it_mid == split
    with gv.vegas_create(kind, d, params, **kw) as b:
        gv.vegas_set_grid(b, edges_mid)
        gv.vegas_set_iteration(b, it_mid)
        r = gv.vegas_iterate(b, rest, refine=True)
        hist_b = gv.vegas_get_history(b)
        edges_b = gv.vegas_get_grid(b)
        assert gv.vegas_get_iteration(b) == total
        gv.vegas_set_grid(b, edges_mid)
        gv.vegas_set_iteration(b, it_mid)
        gv.vegas_reset_results(b)
        gv.vegas_iterate(b, rest, refine=False)
        frozen_b = gv.vegas_get_history(b)
    assert r["iters_done"] == rest
    assert np.array_equal(hist_b[0], hist_a[0])
    assert np.array_equal(frozen_b, frozen_a)
    if kw["precision"] == 0:
        np.testing.assert_allclose(hist_b, hist_a, rtol=1e-12, atol=0)
        np.testing.assert_allclose(edges_b, edges_a, rtol=0, atol=1e-12)
    if kind == wl.GENZ_GAUSSIAN:  # and the oracle's own uninterrupted loop
        cfg = orc.make_cfg(d, nbins=50, ncall=kw["ncall"], nstrat=kw.get("nstrat", 0), ybits=53, seed=11)
        e = orc.uniform_grid(d, 50)
        o = orc.vegas(cfg, orc.Integrand(kind, d, params), e, 0, total)
        np.testing.assert_allclose(hist_b[:, 0], o["hist"][split:, 0], rtol=1e-12)
        np.testing.assert_allclose(edges_b, e, rtol=0, atol=1e-12)


def test_frozen_grid_hand_over_after_bases(gv):
    """The grid a BASES run optimised, moved into a fresh context at the
    iteration index where its integration phase began, gives that
    integration phase again: the same per-iteration estimates, bit for bit
    (the phase does not refine, and its sums are fixed-order)."""
    d, g = 4, 4
    kw = dict(nbins=50, ncall=g ** d * 32, nstrat=g, precision=0, ybits=24, seed=3)
    p = wl.double_gaussian_params()
    with gv.vegas_create(wl.DOUBLE_GAUSSIAN, d, p, **kw) as a:
        gv.bases_integrate(a, 3, 0.0, 2, 0.0)
        hist_a = gv.vegas_get_history(a)  # the integration phase (2 rows)
        edges = gv.vegas_get_grid(a)      # its frozen grid
    with gv.vegas_create(wl.DOUBLE_GAUSSIAN, d, p, **kw) as c:
        gv.vegas_set_grid(c, edges)
        gv.vegas_set_iteration(c, 3)
        gv.vegas_iterate(c, 2, refine=False)
        hist_c = gv.vegas_get_history(c)
    assert np.array_equal(hist_c, hist_a)
