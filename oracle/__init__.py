"""Plain FP64 CPU oracle of the VEGAS / BASES iteration (Sec. 2.1, steps 2-6).

TEST INFRASTRUCTURE ONLY.  The C source ``oracle.c`` is compiled with gcc into
``_build/liboracle.so`` and wrapped here with ctypes.  Only the test suite, the
package entry's ``smoke()`` check and the benchmark's CPU-baseline leg may import
this module.  It imports nothing from the CUDA library and the CUDA library
imports nothing from it.

Every function mirrors one C entry point of ``oracle.h``; see there for the
passage of the paper (or the published method it defers to) that each follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

# Integrand kinds (same numbers as the enumeration in oracle.h).
GENZ_GAUSSIAN = 0
GENZ_PRODUCT_PEAK = 1
GENZ_CORNER_PEAK = 2
GENZ_OSCILLATORY = 3
DOUBLE_GAUSSIAN = 4
RAMBO_BW = 5
GENZ_CONTINUOUS = 6
GENZ_DISCONTINUOUS = 7
W_MUNU = 8
# slots of the W_MUNU parameter vector (oracle.h)
(W_SQRTS, W_M, W_GAMMA, W_GF, W_VUD, W_PTMIN, W_ETAMAX, W_SMIN, W_CUTS,
 W_AU, W_ALU, W_BU, W_AD, W_ALD, W_BD) = range(15)
W_NPARAMS = 15

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (binary64, no FP contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB_PATH) for p in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call([
            "gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Cfg(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nbins", ctypes.c_int),
                ("ncall", ctypes.c_int64), ("nstrat", ctypes.c_int),
                ("ybits", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("instance", ctypes.c_uint32), ("alpha", ctypes.c_double)]


class Fn(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("ndim", ctypes.c_int),
                ("params", ctypes.POINTER(ctypes.c_double)),
                ("nparams", ctypes.c_int)]


class IterOut(ctypes.Structure):
    _fields_ = [("S1", ctypes.POINTER(ctypes.c_double)),
                ("S2", ctypes.POINTER(ctypes.c_double)),
                ("C1", ctypes.POINTER(ctypes.c_double)),
                ("C2", ctypes.POINTER(ctypes.c_double)),
                ("tot", ctypes.c_double * 4),
                ("nonfinite", ctypes.c_int64),
                ("Cmax", ctypes.POINTER(ctypes.c_double))]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _i32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _u64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


class Integrand:
    """An integrand of the registry: kind, dimension and parameter vector."""

    def __init__(self, kind: int, ndim: int, params):
        self.kind = int(kind)
        self.ndim = int(ndim)
        self.params = np.ascontiguousarray(params, dtype=np.float64)
        self._fn = Fn(self.kind, self.ndim, _dp(self.params), len(self.params))

    @property
    def fn(self):
        return ctypes.byref(self._fn)


def make_cfg(ndim, nbins=50, ncall=100000, nstrat=0, ybits=53, seed=1,
             instance=0, alpha=1.5):
    return Cfg(int(ndim), int(nbins), int(ncall), int(nstrat), int(ybits),
               int(seed), int(instance), float(alpha))


def uniform_grid(ndim: int, nbins: int) -> np.ndarray:
    """Edges e_a[k] = k / N of the initial grid, shape (ndim, nbins + 1)."""
    e = np.arange(nbins + 1, dtype=np.float64) / nbins
    return np.ascontiguousarray(np.tile(e, (ndim, 1)))


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_u32p(c), _u32p(k), _u32p(out))
    return out


def sample_batch(cfg: Cfg, edges: np.ndarray, it: int, s):
    """Words, bins, frac, x and Jacobian of the samples with indices s."""
    s = np.ascontiguousarray(s, dtype=np.uint64)
    n, d = len(s), cfg.ndim
    W = 2 * d if cfg.ybits == 53 else d
    words = np.zeros((n, W), np.uint32)
    bins = np.zeros((n, d), np.int32)
    frac = np.zeros((n, d))
    x = np.zeros((n, d))
    jac = np.zeros(n)
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    rc = lib().orc_sample_batch(ctypes.byref(cfg), _dp(edges), ctypes.c_uint32(it),
                                _u64p(s), ctypes.c_int64(n), _u32p(words),
                                _i32p(bins), _dp(frac), _dp(x), _dp(jac))
    if rc:
        raise ValueError("orc_sample_batch failed")
    return dict(words=words, bins=bins, frac=frac, x=x, jac=jac)


def points_from_words(cfg: Cfg, edges: np.ndarray, cube, words):
    """Step 2 from given Philox words (one row per sample) and cube indices."""
    words = np.ascontiguousarray(words, dtype=np.uint32)
    n, d = len(words), cfg.ndim
    cube = np.ascontiguousarray(np.broadcast_to(np.asarray(cube, np.uint64), (n,)))
    bins = np.zeros((n, d), np.int32)
    frac = np.zeros((n, d))
    x = np.zeros((n, d))
    jac = np.zeros(n)
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    rc = lib().orc_points_from_words(ctypes.byref(cfg), _dp(edges), _u64p(cube),
                                     _u32p(words), ctypes.c_int64(n), _i32p(bins),
                                     _dp(frac), _dp(x), _dp(jac))
    if rc:
        raise ValueError("orc_points_from_words failed")
    return dict(bins=bins, frac=frac, x=x, jac=jac)


def integrand(fn: Integrand, x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, fn.ndim)
    f = np.zeros(len(x))
    if lib().orc_integrand(fn.fn, ctypes.c_int64(len(x)), _dp(x), _dp(f)):
        raise ValueError("orc_integrand failed")
    return f


def ntheta(fn: Integrand) -> int:
    return lib().orc_ntheta(fn.fn)


def integrand_grad(fn: Integrand, x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, fn.ndim)
    nt = ntheta(fn)
    g = np.zeros((len(x), nt))
    if lib().orc_integrand_grad(fn.fn, ctypes.c_int64(len(x)), _dp(x), _dp(g)):
        raise ValueError("orc_integrand_grad failed")
    return g


def cut_margin(fn: Integrand, x) -> np.ndarray:
    """Smallest relative distance of each point's cut or discontinuity
    quantities from their edges (inf where the integrand has none)."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, fn.ndim)
    m = np.zeros(len(x))
    if lib().orc_cut_margin(fn.fn, ctypes.c_int64(len(x)), _dp(x), _dp(m)):
        raise ValueError("orc_cut_margin failed")
    return m


def rambo(n: int, sqrt_s: float, rho) -> np.ndarray:
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    p = np.zeros((n, 4))
    if lib().orc_rambo(ctypes.c_int(n), ctypes.c_double(sqrt_s), _dp(rho), _dp(p)):
        raise ValueError("orc_rambo failed")
    return p


def rambo_f_momenta(params, p) -> float:
    params = np.ascontiguousarray(params, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64)
    L = lib()
    L.orc_rambo_f_momenta.restype = ctypes.c_double
    return L.orc_rambo_f_momenta(_dp(params), _dp(p))


def rambo_volume(n: int, sqrt_s: float) -> float:
    L = lib()
    L.orc_rambo_volume.restype = ctypes.c_double
    return L.orc_rambo_volume(ctypes.c_int(n), ctypes.c_double(sqrt_s))


def iteration(cfg: Cfg, fn: Integrand, edges, it: int, cubes: bool = False):
    """Step 4 over one iteration; returns S1, S2, totals (and cube sums)."""
    d, N = cfg.ndim, cfg.nbins
    S1 = np.zeros((d, N))
    S2 = np.zeros((d, N))
    out = IterOut()
    out.S1, out.S2 = _dp(S1), _dp(S2)
    C1 = C2 = Cmax = None
    if cubes:
        g = max(cfg.nstrat, 1)
        C1 = np.zeros(g ** d)
        C2 = np.zeros(g ** d)
        Cmax = np.zeros(g ** d)
        out.C1, out.C2, out.Cmax = _dp(C1), _dp(C2), _dp(Cmax)
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    if lib().orc_iteration(ctypes.byref(cfg), fn.fn, _dp(edges), ctypes.c_uint32(it),
                           ctypes.byref(out)):
        raise ValueError("orc_iteration failed")
    res = dict(S1=S1, S2=S2, sum_w=out.tot[0], sum_w2=out.tot[1], I=out.tot[2],
               var=out.tot[3], nonfinite=out.nonfinite)
    if cubes:
        res.update(C1=C1, C2=C2, Cmax=Cmax)
    return res


def spring_table(cmax):
    """Integer hypercube weights q_c and the scale 2^24 / max M (SPRING)."""
    cmax = np.ascontiguousarray(cmax, dtype=np.float64)
    q = np.zeros(len(cmax), dtype=np.uint64)
    scale = ctypes.c_double()
    if lib().orc_spring_table(ctypes.c_int64(len(cmax)), _dp(cmax),
                              q.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), ctypes.byref(scale)):
        raise ValueError("orc_spring_table: no positive maximum")
    return q, scale.value


def spring(cfg: Cfg, fn: Integrand, edges, cmax, t0: int, n: int):
    """SPRING trials t0 .. t0+n-1 on a frozen grid with per-cube maxima cmax;
    returns kept points x [k][ndim], their trial indices, and the numbers of
    bound overflows and non-positive weights."""
    d = cfg.ndim
    x = np.zeros((n, d))
    t = np.zeros(n, dtype=np.uint64)
    k, ov, npos = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    cmax = np.ascontiguousarray(cmax, dtype=np.float64)
    if lib().orc_spring(ctypes.byref(cfg), fn.fn, _dp(edges), _dp(cmax), ctypes.c_uint64(t0),
                        ctypes.c_int64(n), _dp(x), t.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                        ctypes.byref(k), ctypes.byref(ov), ctypes.byref(npos)):
        raise ValueError("orc_spring failed")
    return dict(x=x[:k.value], trial=t[:k.value], overflow=ov.value, nonpos=npos.value)


def refine(S2, edges, alpha=1.5) -> np.ndarray:
    """Step 5 on a copy of edges; returns the new edges."""
    S2 = np.ascontiguousarray(S2, dtype=np.float64)
    e = np.array(edges, dtype=np.float64, copy=True, order="C")
    d, N1 = e.shape
    if lib().orc_refine(ctypes.c_int(d), ctypes.c_int(N1 - 1), ctypes.c_double(alpha),
                        _dp(S2), _dp(e)):
        raise ValueError("orc_refine failed")
    return e


def combine(I, var):
    I = np.ascontiguousarray(I, dtype=np.float64)
    var = np.ascontiguousarray(var, dtype=np.float64)
    out = np.zeros(3)
    lib().orc_combine(ctypes.c_int(len(I)), _dp(I), _dp(var), _dp(out))
    return dict(I=out[0], sigma=out[1], chi2_dof=out[2])


def vegas(cfg: Cfg, fn: Integrand, edges, it0: int, itmx: int, refine: bool = True,
          acc: float = 0.0):
    """Steps 2-6 repeated; edges are updated in place when refine is set."""
    hist = np.zeros((max(itmx, 1), 2))
    out = np.zeros(3)
    n = lib().orc_vegas(ctypes.byref(cfg), fn.fn, _dp(edges), ctypes.c_uint32(it0),
                        ctypes.c_int(itmx), ctypes.c_int(int(refine)),
                        ctypes.c_double(acc), _dp(hist), _dp(out))
    if n < 0:
        raise ValueError("orc_vegas failed")
    return dict(I=out[0], sigma=out[1], chi2_dof=out[2], iters=n, hist=hist[:n])


def bases(cfg: Cfg, fn: Integrand, edges, it0: int, itmx1: int, acc1: float,
          itmx2: int, acc2: float):
    hist = np.zeros((max(itmx1 + itmx2, 1), 2))
    out = np.zeros(3)
    nd = (ctypes.c_int * 2)()
    n = lib().orc_bases(ctypes.byref(cfg), fn.fn, _dp(edges), ctypes.c_uint32(it0),
                        ctypes.c_int(itmx1), ctypes.c_double(acc1), ctypes.c_int(itmx2),
                        ctypes.c_double(acc2), _dp(hist), _dp(out), nd)
    if n < 0:
        raise ValueError("orc_bases failed")
    return dict(I=out[0], sigma=out[1], chi2_dof=out[2], n1=nd[0], n2=nd[1],
                hist=hist[:n])


def gradient(cfg: Cfg, fn: Integrand, edges, it: int):
    nt = ntheta(fn)
    g = np.zeros(nt)
    I = ctypes.c_double()
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    if lib().orc_gradient(ctypes.byref(cfg), fn.fn, _dp(edges), ctypes.c_uint32(it),
                          _dp(g), ctypes.byref(I)):
        raise ValueError("orc_gradient failed")
    return g, I.value
