"""Pins of the oracle's step 2 (Sec. 2.1): random words -> y -> grid bin,
position in the bin, mapped point x and Jacobian J."""
from fractions import Fraction

import numpy as np
import pytest


def test_bins_exhaustive_24bit(orc):
    """All 2^24 values of the 24-bit mantissa m (y = m / 2^24) at N = 50:
    k = floor(y N) and frac = y N - k exactly, and x = y at the uniform grid to
    within rounding.  The low 8 bits of the word must be ignored."""
    N = 50
    cfg = orc.make_cfg(1, nbins=N, ncall=1 << 24, ybits=24)
    e = orc.uniform_grid(1, N)
    rng = np.random.default_rng(3)
    chunk = 1 << 22
    for lo in range(0, 1 << 24, chunk):
        m = np.arange(lo, lo + chunk, dtype=np.uint64)
        junk = rng.integers(0, 256, chunk, dtype=np.uint64)
        words = ((m << np.uint64(8)) | junk).astype(np.uint32).reshape(-1, 1)
        r = orc.points_from_words(cfg, e, 0, words)
        k = r["bins"][:, 0].astype(np.int64)
        prod = m.astype(np.int64) * N
        assert np.all(k * (1 << 24) <= prod) and np.all(prod < (k + 1) * (1 << 24))
        assert np.array_equal(r["frac"][:, 0] * float(1 << 24), (prod - k * (1 << 24)).astype(np.float64))
        y = m.astype(np.float64) / float(1 << 24)
        assert np.max(np.abs(r["x"][:, 0] - y)) <= 4e-16
        # edges k/50 are rounded, so N (e[k+1] - e[k]) = 1 to within 50 ulp(1)
        assert np.all(np.abs(r["jac"] - 1.0) <= 1.2e-14)


def _m53(w_hi, w_lo):
    return ((int(w_hi) >> 5) << 26) | (int(w_lo) >> 6)


@pytest.mark.parametrize("g", [1, 3, 4])
def test_bins_rational_53bit_and_stratified(orc, g):
    """53-bit mode and hypercube stratification: y_a = (c_a + m/2^53)/g with
    c_a the a-th base-g digit of the cube index; k = floor(y N) exactly and
    frac = y N - k after one round-to-nearest (exact when g = 1)."""
    d, N = 3, 50
    G = g ** d
    cfg = orc.make_cfg(d, nbins=N, ncall=G * 16, nstrat=g, ybits=53)
    e = orc.uniform_grid(d, N)
    rng = np.random.default_rng(5 + g)
    n = 3000
    words = rng.integers(0, 1 << 32, (n, 2 * d), dtype=np.uint64).astype(np.uint32)
    words[:5] = 0
    words[5:10] = 0xFFFFFFFF
    cube = rng.integers(0, G, n, dtype=np.uint64)
    r = orc.points_from_words(cfg, e, cube, words)
    for i in range(n):
        c = int(cube[i])
        for a in range(d):
            ca = (c // g ** a) % g
            y = (ca + Fraction(_m53(words[i, 2 * a], words[i, 2 * a + 1]), 1 << 53)) / g
            k = int(y * N)
            assert r["bins"][i, a] == k
            exact = y * N - k
            assert abs(Fraction(r["frac"][i, a]) - exact) <= Fraction(1, 1 << 53)
            if g == 1:
                assert Fraction(r["frac"][i, a]) == exact


def test_bins_stratified_24bit(orc):
    d, N, g = 2, 50, 4
    cfg = orc.make_cfg(d, nbins=N, ncall=16 * 64, nstrat=g, ybits=24)
    rng = np.random.default_rng(9)
    words = rng.integers(0, 1 << 32, (2000, d), dtype=np.uint64).astype(np.uint32)
    cube = rng.integers(0, g ** d, 2000, dtype=np.uint64)
    r = orc.points_from_words(cfg, orc.uniform_grid(d, N), cube, words)
    for i in range(2000):
        for a in range(d):
            ca = (int(cube[i]) // g ** a) % g
            y = (ca + Fraction(int(words[i, a]) >> 8, 1 << 24)) / g
            k = int(y * N)
            assert r["bins"][i, a] == k
            assert Fraction(r["frac"][i, a]) == y * N - k


def _random_grid(rng, d, N):
    w = rng.random((d, N)) ** 3 + 1e-3
    e = np.zeros((d, N + 1))
    e[:, 1:] = np.cumsum(w, axis=1) / w.sum(axis=1, keepdims=True)
    e[:, -1] = 1.0
    return e


def test_map_is_inverse_cdf(orc):
    """The map x(y) with Jacobian J is the inverse CDF of a piecewise-constant
    density, so E_y[g(x(y)) J(y)] = int_0^1 g(x) dx.  With one-point-per-bin
    midpoints and Gauss-Legendre nodes inside each y-bin this is exact for
    polynomials (x is linear and J constant inside a bin)."""
    N = 10
    rng = np.random.default_rng(1)
    e = _random_grid(rng, 1, N)
    cfg = orc.make_cfg(1, nbins=N, ncall=1 << 20, ybits=53)
    xg, wg = np.polynomial.legendre.leggauss(6)
    ys, ws = [], []
    for k in range(N):
        ys.append((k + 0.5 * (xg + 1)) / N)
        ws.append(0.5 * wg / N)
    ys, ws = np.concatenate(ys), np.concatenate(ws)
    m = np.round(ys * 2.0 ** 53).astype(np.uint64)
    words = np.zeros((len(m), 2), np.uint32)
    words[:, 0] = ((m >> np.uint64(26)) << np.uint64(5)).astype(np.uint32)
    words[:, 1] = ((m & np.uint64((1 << 26) - 1)) << np.uint64(6)).astype(np.uint32)
    r = orc.points_from_words(cfg, e, 0, words)
    x, J = r["x"][:, 0], r["jac"]
    for p in range(6):
        est = float(np.sum(ws * x ** p * J))
        assert abs(est - 1.0 / (p + 1)) < 1e-13
    assert np.all(np.diff(x) > 0)
    # int J dy = sum of bin widths = 1
    assert abs(float(np.sum(ws * J)) - 1.0) < 1e-14


def test_bin_occupancy_uniform(orc):
    """Bins depend only on y, so their counts are multinomial with p = 1/N on
    any grid (chi-square per axis, 49 dof)."""
    d, N, n = 4, 50, 200_000
    cfg = orc.make_cfg(d, nbins=N, ncall=n, ybits=24, seed=21)
    e = _random_grid(np.random.default_rng(4), d, N)
    b = orc.sample_batch(cfg, e, 2, np.arange(n))["bins"]
    for a in range(d):
        c = np.bincount(b[:, a], minlength=N)
        chi2 = float(np.sum((c - n / N) ** 2 / (n / N)))
        assert 20 < chi2 < 90
