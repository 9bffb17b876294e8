"""Pins of the oracle's cut margins (the distance of a point's cut and
discontinuity quantities from their edges), which the parity tests use to
decide which points may fall on either side of an edge under rounding.

The pin is independent of the margin's own arithmetic: along a segment from
a point the integrand keeps to one it cuts, bisection on the integrand's
value (zero or not) locates the edge; there the margin must vanish, and away
from every edge it must be large."""
import numpy as np
import pytest

from paper_1010_2107_gb300 import workloads as wl


def _edge_by_bisection(orc, fn, xa, xb, steps=60):
    """A point within 2^-steps of the segment's zero/non-zero transition,
    with xa kept (f != 0) and xb cut (f == 0)."""
    fa = orc.integrand(fn, xa)[0]
    fb = orc.integrand(fn, xb)[0]
    assert fa != 0.0 and fb == 0.0
    for _ in range(steps):
        xm = 0.5 * (xa + xb)
        if orc.integrand(fn, xm)[0] != 0.0:
            xa = xm
        else:
            xb = xm
    return xa, xb


def _pairs(orc, fn, d, n=4000, seed=5):
    """Kept and cut points of the integrand from a seeded uniform sample."""
    x = np.random.default_rng(seed).uniform(0.02, 0.98, (n, d))
    f = orc.integrand(fn, x)
    return x[f != 0.0], x[f == 0.0]


@pytest.mark.parametrize("case", ["rambo_hard", "rambo_sigmoid", "disc3", "wmunu"])
def test_margin_vanishes_at_every_cut_edge(orc, case):
    if case == "rambo_hard":
        fn = orc.Integrand(orc.RAMBO_BW, 12, wl.rambo_params(3))
    elif case == "rambo_sigmoid":  # only the Delta R cut is an edge
        fn = orc.Integrand(orc.RAMBO_BW, 12, wl.rambo_params(3, cut=1))
    elif case == "disc3":
        fn = orc.Integrand(orc.GENZ_DISCONTINUOUS, 3, [1.5, 2.0, 0.7, 0.4, 0.6])
    else:
        fn = orc.Integrand(orc.W_MUNU, 5, wl.w_munu_params())
    kept, cut = _pairs(orc, fn, fn.ndim)
    assert len(kept) > 20 and len(cut) > 20
    found = 0
    for i in range(12):
        xa, xb = _edge_by_bisection(orc, fn, kept[i], cut[i])
        ma, mb = orc.cut_margin(fn, np.stack([xa, xb]))
        # 2^-60 of the segment: the edge quantity moves by far less than 1e-9
        assert min(ma, mb) < 1e-9, (case, i, ma, mb)
        found += 1
    assert found == 12
    # a kept point far inside, and the margin of the sample as a whole:
    # finite, non-negative, and mostly well away from zero
    m = orc.cut_margin(fn, kept)
    assert np.all(m >= 0.0) and np.all(np.isfinite(m))
    assert np.median(m) > 1e-3


def test_margin_is_infinite_without_edges(orc):
    x = np.random.default_rng(1).random((50, 4))
    for fn in (orc.Integrand(orc.GENZ_GAUSSIAN, 4, wl.genz_gaussian_params(4)),
               orc.Integrand(orc.RAMBO_BW, 8, wl.rambo_params(2, cut=2)),
               orc.Integrand(orc.RAMBO_BW, 8, wl.rambo_params(2, obs=3))):
        assert np.all(np.isinf(orc.cut_margin(fn, x)))


def test_margin_of_the_discontinuous_family_is_the_coordinate_gap(orc):
    """Genz discontinuous: margin = min(|x1 - u1| / u1, |x2 - u2| / u2)."""
    u1, u2 = 0.4, 0.6
    fn = orc.Integrand(orc.GENZ_DISCONTINUOUS, 3, [1.5, 2.0, 0.7, u1, u2])
    x = np.array([[0.39, 0.5, 0.3], [0.1, 0.61, 0.9], [0.4, 0.6, 0.5]])
    m = orc.cut_margin(fn, x)
    np.testing.assert_allclose(m, [0.01 / u1, 0.01 / u2, 0.0], rtol=1e-12, atol=1e-15)
