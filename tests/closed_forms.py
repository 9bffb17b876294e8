"""Closed forms and reference quadratures used to pin the oracle.

Each function states the mathematics it evaluates.  Nothing here calls the
oracle or the CUDA library."""
from __future__ import annotations

import math
from decimal import Decimal, getcontext
from fractions import Fraction
from itertools import combinations

import numpy as np


def genz_gaussian(a, u):
    """int_[0,1]^d exp(-sum a_i^2 (x_i-u_i)^2) dx
       = prod_i sqrt(pi)/(2 a_i) [erf(a_i (1-u_i)) + erf(a_i u_i)]."""
    return math.prod(math.sqrt(math.pi) / (2 * ai) * (math.erf(ai * (1 - ui)) + math.erf(ai * ui))
                     for ai, ui in zip(a, u))


def genz_product_peak(a, u):
    """int prod_i (a_i^-2 + (x_i-u_i)^2)^-1 dx = prod_i a_i [atan(a_i(1-u_i)) + atan(a_i u_i)]."""
    return math.prod(ai * (math.atan(ai * (1 - ui)) + math.atan(ai * ui)) for ai, ui in zip(a, u))


def genz_corner_peak(a, digits: int = 80):
    """int (1 + a.x)^-(d+1) dx = (d! prod a)^-1 sum_{S subset [d]} (-1)^|S| (1 + sum_S a)^-1,
    evaluated in decimal arithmetic with the a_i converted exactly from binary64."""
    getcontext().prec = digits
    A = [Decimal(Fraction(float(x)).numerator) / Decimal(Fraction(float(x)).denominator) for x in a]
    d = len(A)
    total = Decimal(0)
    for k in range(d + 1):
        for S in combinations(range(d), k):
            total += (-1) ** k / (Decimal(1) + sum((A[i] for i in S), Decimal(0)))
    norm = Decimal(math.factorial(d))
    for x in A:
        norm *= x
    return float(total / norm)


def genz_oscillatory(a, u1):
    """int cos(2 pi u1 + a.x) dx = Re[e^{i 2 pi u1} prod_i (e^{i a_i} - 1)/(i a_i)]."""
    z = complex(math.cos(2 * math.pi * u1), math.sin(2 * math.pi * u1))
    for ai in a:
        z *= (complex(math.cos(ai), math.sin(ai)) - 1) / complex(0, ai)
    return z.real


def genz_continuous(a, u):
    """int exp(-sum a_i |x_i - u_i|) dx = prod_i (2 - e^{-a_i u_i} - e^{-a_i (1 - u_i)}) / a_i."""
    return math.prod((2 - math.exp(-ai * ui) - math.exp(-ai * (1 - ui))) / ai for ai, ui in zip(a, u))


def genz_discontinuous(a, u):
    """int_{x_1 <= u_1, x_2 <= u_2} exp(sum a_i x_i) dx
       = prod_{i < min(d,2)} (e^{a_i u_i} - 1)/a_i * prod_{i >= 2} (e^{a_i} - 1)/a_i."""
    out = 1.0
    for i, ai in enumerate(a):
        top = u[i] if i < 2 else 1.0
        out *= math.expm1(ai * top) / ai
    return out


def gauss_legendre_split(breaks, nodes_per_piece=16, pieces=8):
    """1-D composite Gauss-Legendre rule on [0, 1] whose pieces never straddle
    a point of `breaks` (kinks and jumps of the integrand sit on piece ends)."""
    xg, wg = np.polynomial.legendre.leggauss(nodes_per_piece)
    pts = sorted({0.0, 1.0, *[b for b in breaks if 0.0 < b < 1.0]})
    xs, ws = [], []
    for lo, hi in zip(pts[:-1], pts[1:]):
        edges = np.linspace(lo, hi, pieces + 1)
        for a, b in zip(edges[:-1], edges[1:]):
            xs.append(a + (b - a) * 0.5 * (xg + 1))
            ws.append(0.5 * (b - a) * wg)
    return np.concatenate(xs), np.concatenate(ws)


def tensor_rule(rules):
    """Tensor product of 1-D rules [(x, w), ...]: nodes [n][d] and weights [n]."""
    grids = np.meshgrid(*[r[0] for r in rules], indexing="ij")
    wgrids = np.meshgrid(*[r[1] for r in rules], indexing="ij")
    X = np.stack([g.ravel() for g in grids], axis=1)
    W = np.prod(np.stack([g.ravel() for g in wgrids], axis=1), axis=1)
    return X, W


def double_gaussian(c1, c2, w, d):
    """int 1/2 sum_c (w sqrt pi)^-d exp(-sum ((x_i-c)/w)^2) dx
       = 1/2 sum_c prod_i 1/2 [erf((1-c)/w) + erf(c/w)]."""
    return 0.5 * sum((0.5 * (math.erf((1 - c) / w) + math.erf(c / w))) ** d for c in (c1, c2))


def rambo_volume(n, sqrt_s):
    """Massless n-body phase-space volume (pi/2)^(n-1) s^(n-2) / ((n-1)! (n-2)!)."""
    s = sqrt_s ** 2
    return (math.pi / 2) ** (n - 1) * s ** (n - 2) / (math.factorial(n - 1) * math.factorial(n - 2))


def _kallen(a, b, c):
    return a * a + b * b + c * c - 2 * a * b - 2 * a * c - 2 * b * c


def s12_density_moment(n, g, npts=4000):
    """E[g(x)] for x = s12/s of two of n massless particles in flat phase space.

    Phase-space factorisation: the pair (1,2) has invariant mass^2 x s, the
    other n-2 particles mass^2 q s; massless two-body phase space is constant,
    the massless (n-2)-body volume grows like q^(n-4), and the decay of the
    total momentum into the two systems carries lambda^(1/2)(1, x, q).  So
    rho(x) is proportional to int_0^{(1-sqrt x)^2} q^(n-4) lambda^(1/2)(1,x,q) dq
    (n = 3: a delta at q = 0, rho(x) = 1 - x).  Composite Gauss-Legendre."""
    xg, wg = np.polynomial.legendre.leggauss(64)

    def inner(x):
        if n == 3:
            return 1.0 - x
        qmax = (1 - math.sqrt(x)) ** 2
        # substitute q = qmax t^2 to soften the square-root end point
        t = 0.5 * (xg + 1)
        q = qmax * t * t
        lam = np.maximum(_kallen(1.0, x, q), 0.0)
        return float(np.sum(0.5 * wg * q ** (n - 4) * np.sqrt(lam) * 2 * qmax * t))

    edges = np.linspace(0, 1, npts + 1) ** 2  # finer near x = 0
    num = den = 0.0
    for lo, hi in zip(edges[:-1], edges[1:]):
        xs = lo + (hi - lo) * 0.5 * (xg + 1)
        ws = 0.5 * (hi - lo) * wg
        r = np.array([inner(x) for x in xs])
        num += float(np.sum(ws * r * np.array([g(x) for x in xs])))
        den += float(np.sum(ws * r))
    return num / den


def gauss_legendre_tensor(d, nodes_per_interval, intervals):
    """Nodes and weights of a composite tensor Gauss-Legendre rule on [0,1]^d."""
    xg, wg = np.polynomial.legendre.leggauss(nodes_per_interval)
    edges = np.linspace(0, 1, intervals + 1)
    x1 = np.concatenate([lo + (hi - lo) * 0.5 * (xg + 1) for lo, hi in zip(edges[:-1], edges[1:])])
    w1 = np.concatenate([0.5 * (hi - lo) * wg for lo, hi in zip(edges[:-1], edges[1:])])
    grids = np.meshgrid(*([x1] * d), indexing="ij")
    wgrids = np.meshgrid(*([w1] * d), indexing="ij")
    X = np.stack([g.ravel() for g in grids], axis=1)
    W = np.prod(np.stack([g.ravel() for g in wgrids], axis=1), axis=1)
    return X, W
