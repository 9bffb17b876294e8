"""Thin Python binding of the C ABI in include/gvegas.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does nothing
but convert arguments and results; all steps of the integration run in the CUDA
library ``_build/libgvegas.so``.  There is no CPU fallback: if the library is
missing or fails to load, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgvegas.so")

# vegas_status
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENONFINITE, ESTATE = range(7)
# vegas_integrand_kind
(GENZ_GAUSSIAN, GENZ_PRODUCT_PEAK, GENZ_CORNER_PEAK, GENZ_OSCILLATORY, DOUBLE_GAUSSIAN, RAMBO_BW,
 GENZ_CONTINUOUS, GENZ_DISCONTINUOUS, W_MUNU) = range(9)
USER = 64  # run-time compiled integrand (vegas_create_user)
MAXUSERPARAMS = 120
# vegas_precision
FP64, FP32_ACC64, FP32_ACCCOMP = range(3)
PRECISIONS = {"fp64": FP64, "fp32_acc64": FP32_ACC64, "fp32": FP32_ACCCOMP,
              "fp32_acccomp": FP32_ACCCOMP}

_lock = threading.Lock()
_lib = None


class VegasError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"gvegas status {status}: {message}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nbins", ctypes.c_int), ("ncall", ctypes.c_int64),
                ("itmx", ctypes.c_int), ("acc", ctypes.c_double), ("alpha", ctypes.c_double),
                ("nstrat", ctypes.c_int), ("seed", ctypes.c_uint64), ("instance", ctypes.c_uint32),
                ("precision", ctypes.c_int), ("ybits", ctypes.c_int), ("stream", ctypes.c_void_p)]


class IntegrandDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("ndim", ctypes.c_int),
                ("params", ctypes.POINTER(ctypes.c_double)), ("nparams", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("I", ctypes.c_double), ("sigma", ctypes.c_double), ("chi2_dof", ctypes.c_double),
                ("iters_done", ctypes.c_int), ("stopped", ctypes.c_int),
                ("nonfinite", ctypes.c_int64), ("samples", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_SIGS = {
    "vegas_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(IntegrandDesc),
                                    ctypes.POINTER(_P)]),
    "vegas_create_user": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_char_p, _DP, ctypes.c_int,
                                         ctypes.POINTER(_P)]),
    "vegas_user_compile": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_char_p]),
    "vegas_destroy": (None, [_P]),
    "vegas_iterate": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Result)]),
    "vegas_reset_results": (ctypes.c_int, [_P]),
    "vegas_reset_grid": (ctypes.c_int, [_P]),
    "bases_integrate": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_double, ctypes.POINTER(Result),
                                       ctypes.POINTER(Result)]),
    "vegas_get_grid": (ctypes.c_int, [_P, _DP, _DP]),
    "vegas_set_grid": (ctypes.c_int, [_P, _DP]),
    "vegas_get_history": (ctypes.c_int, [_P, _DP, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "vegas_get_cube_sums": (ctypes.c_int, [_P, _DP]),
    "vegas_get_iteration": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint32)]),
    "vegas_set_iteration": (ctypes.c_int, [_P, ctypes.c_uint32]),
    "vegas_set_params": (ctypes.c_int, [_P, _DP, ctypes.c_int]),
    "vegas_eval": (ctypes.c_int, [_P, ctypes.c_uint32, _DP, _DP]),
    "vegas_grad": (ctypes.c_int, [_P, ctypes.c_uint32, _DP, _DP]),
    "vegas_ntheta": (ctypes.c_int, [_P]),
    "vegas_sample_dump": (ctypes.c_int, [_P, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64),
                                         ctypes.c_int64, ctypes.POINTER(ctypes.c_uint32),
                                         ctypes.POINTER(ctypes.c_int32), _DP, _DP, _DP]),
    "vegas_set_launch": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "vegas_get_launch": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "vegas_set_tile": (ctypes.c_int, [_P, ctypes.c_int]),
    "vegas_get_cube_max": (ctypes.c_int, [_P, _DP]),
    "spring_profile": (ctypes.c_int, [_P, ctypes.c_uint32, ctypes.c_int, _DP]),
    "spring_generate": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_uint32, _DP,
                                       ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint32),
                                       ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32)]),
    "vegas_autotune": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _DP]),
    "vegas_get_tile": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "vegas_profile_pass": (ctypes.c_int, [_P, ctypes.c_int, _DP]),
    "vegas_profile_frozen_pass": (ctypes.c_int, [_P, ctypes.c_int, _DP]),
    "vegas_microbench": (ctypes.c_int, [ctypes.c_int, _DP]),
    "vegas_eval_noalloc": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(IntegrandDesc),
                                          ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p]),
    "vegas_last_error": (ctypes.c_char_p, [_P]),
    "vegas_fail_alloc_after": (None, [ctypes.c_int64]),
    "vegas_alloc_count": (ctypes.c_uint64, []),
    "vegas_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(Config), ctypes.POINTER(IntegrandDesc),
                                          ctypes.POINTER(_P)]),
    "vegas_batch_destroy": (None, [_P]),
    "vegas_batch_iterate": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Result)]),
    "vegas_batch_reset": (ctypes.c_int, [_P]),
    "vegas_batch_get_grid": (ctypes.c_int, [_P, ctypes.c_int, _DP, _DP]),
    "vegas_batch_get_history": (ctypes.c_int, [_P, ctypes.c_int, _DP, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "vegas_batch_set_launch": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "vegas_batch_get_launch": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "vegas_batch_autotune": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _DP]),
    "vegas_batch_set_tile": (ctypes.c_int, [_P, ctypes.c_int]),
    "vegas_batch_set_params": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _DP, ctypes.c_int]),
    "vegas_batch_get_tile": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "vegas_batch_profile": (ctypes.c_int, [_P, ctypes.c_int, _DP]),
    "vegas_batch_last_error": (ctypes.c_char_p, [_P]),
}


def lib() -> ctypes.CDLL:
    """Load libgvegas.so (built by __graft_entry__.build()); raise if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"CUDA library not built: {LIB_PATH} is missing "
                                  "(run __graft_entry__.build())")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def _check(st: int, handle=None):
    if st != OK:
        msg = lib().vegas_last_error(handle)
        raise VegasError(st, msg.decode() if msg else "")


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # a torch.cuda.Stream


class Context:
    """Owner of one vegas_ctx handle."""

    def __init__(self, handle, ndim, nbins, ncall, nstrat, ybits):
        self.handle = handle
        self.ndim, self.nbins, self.ncall, self.nstrat, self.ybits = ndim, nbins, ncall, nstrat, ybits

    def close(self):
        if self.handle:
            lib().vegas_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def vegas_create(kind: int, ndim: int, params, *, nbins: int = 50, ncall: int = 100_000,
                 itmx: int = 5, acc: float = 0.0, alpha: float = 1.5, nstrat: int = 0,
                 seed: int = 1, instance: int = 0, precision=FP64, ybits: int = 0,
                 stream=None) -> Context:
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    p = np.ascontiguousarray(params, dtype=np.float64)
    cfg = Config(int(ndim), int(nbins), int(ncall), int(itmx), float(acc), float(alpha),
                 int(nstrat), int(seed), int(instance), int(precision), int(ybits),
                 _stream_handle(stream))
    fn = IntegrandDesc(int(kind), int(ndim), _dp(p), len(p))
    h = _P()
    _check(lib().vegas_create(ctypes.byref(cfg), ctypes.byref(fn), ctypes.byref(h)))
    yb = ybits or (53 if precision == FP64 else 24)
    return Context(h, int(ndim), int(nbins), int(ncall), int(nstrat), yb)


def _config(ndim, nbins, ncall, itmx, acc, alpha, nstrat, seed, instance, precision, ybits, stream):
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    return Config(int(ndim), int(nbins), int(ncall), int(itmx), float(acc), float(alpha),
                  int(nstrat), int(seed), int(instance), int(precision), int(ybits),
                  _stream_handle(stream))


def vegas_create_user(source: str, ndim: int, params=(), *, nbins: int = 50, ncall: int = 100_000,
                      itmx: int = 5, acc: float = 0.0, alpha: float = 1.5, nstrat: int = 0,
                      seed: int = 1, instance: int = 0, precision=FP64, ybits: int = 0,
                      stream=None) -> Context:
    """Context for an integrand given as CUDA source defining
    ``template <typename T> __device__ T vegas_user_f(const T* x, int d, const T* p)``,
    compiled at run time (see include/gvegas.h)."""
    cfg = _config(ndim, nbins, ncall, itmx, acc, alpha, nstrat, seed, instance, precision, ybits, stream)
    p = np.ascontiguousarray(params, dtype=np.float64)
    h = _P()
    _check(lib().vegas_create_user(ctypes.byref(cfg), source.encode(), _dp(p) if len(p) else None, len(p),
                                   ctypes.byref(h)))
    yb = ybits or (53 if cfg.precision == FP64 else 24)
    return Context(h, int(ndim), int(nbins), int(ncall), int(nstrat), yb)


def vegas_user_compile(source: str, ndim: int, *, nbins: int = 50, ncall: int = 100_000, nstrat: int = 0,
                       precision=FP64, ybits: int = 0) -> None:
    """Compile a user integrand for this shape without a device; raises VegasError
    (EINVAL, with the compiler's log) when the source does not compile."""
    cfg = _config(ndim, nbins, ncall, 5, 0.0, 1.5, nstrat, 1, 0, precision, ybits, None)
    _check(lib().vegas_user_compile(ctypes.byref(cfg), source.encode()))


def vegas_destroy(ctx: Context):
    ctx.close()


def vegas_iterate(ctx: Context, n_iter: int, refine: bool = True, result: bool = True):
    r = Result()
    _check(lib().vegas_iterate(ctx.handle, int(n_iter), int(bool(refine)),
                               ctypes.byref(r) if result else None), ctx.handle)
    return r.as_dict() if result else None


def vegas_reset_results(ctx: Context):
    _check(lib().vegas_reset_results(ctx.handle), ctx.handle)


def vegas_reset_grid(ctx: Context):
    _check(lib().vegas_reset_grid(ctx.handle), ctx.handle)


def bases_integrate(ctx: Context, itmx1: int, acc1: float, itmx2: int, acc2: float,
                    result: bool = True):
    out, ph1 = Result(), Result()
    _check(lib().bases_integrate(ctx.handle, int(itmx1), float(acc1), int(itmx2), float(acc2),
                                 ctypes.byref(out) if result else None,
                                 ctypes.byref(ph1) if result else None), ctx.handle)
    return (out.as_dict(), ph1.as_dict()) if result else None


def vegas_get_grid(ctx: Context, bin_sums: bool = False):
    e = np.zeros((ctx.ndim, ctx.nbins + 1))
    b = np.zeros((2, ctx.ndim, ctx.nbins)) if bin_sums else None
    _check(lib().vegas_get_grid(ctx.handle, _dp(e), _dp(b) if bin_sums else None), ctx.handle)
    return (e, b) if bin_sums else e


def vegas_set_grid(ctx: Context, edges):
    e = np.ascontiguousarray(edges, dtype=np.float64)
    if e.shape != (ctx.ndim, ctx.nbins + 1):
        raise ValueError(f"edges must have shape {(ctx.ndim, ctx.nbins + 1)}")
    _check(lib().vegas_set_grid(ctx.handle, _dp(e)), ctx.handle)


def vegas_get_history(ctx: Context, max_iters: int = 4096):
    h = np.zeros((max_iters, 2))
    n = ctypes.c_int()
    _check(lib().vegas_get_history(ctx.handle, _dp(h), int(max_iters), ctypes.byref(n)), ctx.handle)
    return h[:min(n.value, max_iters)]


def vegas_get_cube_sums(ctx: Context):
    G = max(ctx.nstrat, 1) ** ctx.ndim
    c = np.zeros((G, 2))
    _check(lib().vegas_get_cube_sums(ctx.handle, _dp(c)), ctx.handle)
    return c


def vegas_get_iteration(ctx: Context) -> int:
    it = ctypes.c_uint32()
    _check(lib().vegas_get_iteration(ctx.handle, ctypes.byref(it)), ctx.handle)
    return it.value


def vegas_set_iteration(ctx: Context, it: int):
    _check(lib().vegas_set_iteration(ctx.handle, int(it)), ctx.handle)


def vegas_set_params(ctx: Context, params):
    p = np.ascontiguousarray(params, dtype=np.float64)
    _check(lib().vegas_set_params(ctx.handle, _dp(p), len(p)), ctx.handle)


def vegas_eval(ctx: Context, it: int):
    I, v = ctypes.c_double(), ctypes.c_double()
    _check(lib().vegas_eval(ctx.handle, int(it), ctypes.byref(I), ctypes.byref(v)), ctx.handle)
    return I.value, v.value


def vegas_ntheta(ctx: Context) -> int:
    return lib().vegas_ntheta(ctx.handle)


def vegas_grad(ctx: Context, it: int):
    g = np.zeros(max(vegas_ntheta(ctx), 1))
    I = ctypes.c_double()
    _check(lib().vegas_grad(ctx.handle, int(it), _dp(g), ctypes.byref(I)), ctx.handle)
    return g[:vegas_ntheta(ctx)], I.value


def vegas_sample_dump(ctx: Context, it: int, s):
    s = np.ascontiguousarray(s, dtype=np.uint64)
    n, d = len(s), ctx.ndim
    W = d if ctx.ybits == 24 else 2 * d
    words = np.zeros((n, W), np.uint32)
    bins = np.zeros((n, d), np.int32)
    x = np.zeros((n, d))
    jac = np.zeros(n)
    f = np.zeros(n)
    _check(lib().vegas_sample_dump(ctx.handle, int(it), s.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                   n, words.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                   bins.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   _dp(x), _dp(jac), _dp(f)), ctx.handle)
    return dict(words=words, bins=bins, x=x, jac=jac, f=f)


def vegas_set_launch(ctx: Context, threads: int, ctas_per_sm: int = 0):
    _check(lib().vegas_set_launch(ctx.handle, int(threads), int(ctas_per_sm)), ctx.handle)


def vegas_get_launch(ctx: Context):
    t, c, o = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().vegas_get_launch(ctx.handle, ctypes.byref(t), ctypes.byref(c), ctypes.byref(o)), ctx.handle)
    return dict(threads=t.value, ctas=c.value, occupancy=o.value)


def vegas_get_cube_max(ctx: Context):
    """Per-hypercube maxima of the last integration phase (SPRING bounds)."""
    g = max(ctx.nstrat, 1)
    out = np.zeros(g ** ctx.ndim)
    _check(lib().vegas_get_cube_max(ctx.handle, _dp(out)), ctx.handle)
    return out


def spring_generate(ctx: Context, trial0: int, n_trials: int, events: bool = True, out_x=None, out_t=None):
    """SPRING trials trial0 .. trial0 + n_trials - 1; returns the kept points
    (host copies when `events`), their trial indices, and the counts.
    out_x ([n_trials][ndim] float64) and out_t ([n_trials] uint64) may be
    given, e.g. in pinned memory; the results are views of their heads."""
    n_ev, n_ov, n_np = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    x = t = None
    if events:
        x = out_x if out_x is not None else np.empty((n_trials, ctx.ndim))
        t = out_t if out_t is not None else np.empty(n_trials, dtype=np.uint64)
        if x.shape != (n_trials, ctx.ndim) or x.dtype != np.float64 or not x.flags.c_contiguous:
            raise ValueError("out_x must be a C-contiguous float64 array [n_trials][ndim]")
        if t.shape != (n_trials,) or t.dtype != np.uint64 or not t.flags.c_contiguous:
            raise ValueError("out_t must be a C-contiguous uint64 array [n_trials]")
    _check(lib().spring_generate(ctx.handle, int(trial0), int(n_trials), _dp(x) if events else None,
                                 t.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)) if events else None,
                                 ctypes.byref(n_ev), ctypes.byref(n_ov), ctypes.byref(n_np)), ctx.handle)
    k = n_ev.value
    return dict(x=x[:k] if events else None, trial=t[:k] if events else None, n_events=k,
                overflow=n_ov.value, nonpos=n_np.value)


def spring_profile(ctx: Context, n_trials: int, reps: int = 5):
    """Mean ms of the SPRING trial kernel over `reps` calls of n_trials."""
    ms = ctypes.c_double()
    _check(lib().spring_profile(ctx.handle, int(n_trials), int(reps), ctypes.byref(ms)), ctx.handle)
    return ms.value


def vegas_set_tile(ctx: Context, points_per_thread: int = 0):
    _check(lib().vegas_set_tile(ctx.handle, int(points_per_thread)), ctx.handle)


def vegas_autotune(ctx: Context):
    """Time the launch shapes and keep the fastest; returns the choice."""
    t, p, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(lib().vegas_autotune(ctx.handle, ctypes.byref(t), ctypes.byref(p), ctypes.byref(ms)), ctx.handle)
    return dict(threads=t.value, points_per_thread=p.value, ms=ms.value)


def vegas_get_tile(ctx: Context):
    p, c = ctypes.c_int(), ctypes.c_int()
    _check(lib().vegas_get_tile(ctx.handle, ctypes.byref(p), ctypes.byref(c)), ctx.handle)
    return dict(points_per_thread=p.value, cap=c.value)


def vegas_profile_pass(ctx: Context, n_pass: int = 10):
    """Mean milliseconds per pass of the sampling kernel, the finishing kernel
    (reduction of the partials) and the two together."""
    ms = np.zeros(3)
    _check(lib().vegas_profile_pass(ctx.handle, int(n_pass), _dp(ms)), ctx.handle)
    return dict(sample=ms[0], finish=ms[1], passes=ms[2])


def vegas_profile_frozen_pass(ctx: Context, n_pass: int = 10):
    """As vegas_profile_pass for the passes that leave the grid unchanged (no
    per-bin histogram, their own launch shape)."""
    ms = np.zeros(3)
    _check(lib().vegas_profile_frozen_pass(ctx.handle, int(n_pass), _dp(ms)), ctx.handle)
    return dict(sample=ms[0], finish=ms[1], passes=ms[2])


def vegas_eval_noalloc(kind: int, ndim: int, params, edges_ptr: int, it: int, out_ptr: int, *,
                       nbins: int = 50, ncall: int = 100_000, nstrat: int = 0, seed: int = 1,
                       instance: int = 0, precision=FP64, ybits: int = 0, alpha: float = 1.5,
                       stream=None):
    """One evaluation pass on caller-owned device buffers (edges_ptr, out_ptr are
    device addresses) without any device allocation; see include/gvegas.h."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    p = np.ascontiguousarray(params, dtype=np.float64)
    cfg = Config(int(ndim), int(nbins), int(ncall), 1, 0.0, float(alpha), int(nstrat), int(seed),
                 int(instance), int(precision), int(ybits), _stream_handle(stream))
    fn = IntegrandDesc(int(kind), int(ndim), _dp(p), len(p))
    _check(lib().vegas_eval_noalloc(ctypes.byref(cfg), ctypes.byref(fn), ctypes.c_void_p(int(edges_ptr)),
                                    int(it), ctypes.c_void_p(int(out_ptr))))


MICROBENCH_OPS = {0: "ffma", 1: "imad_wide", 2: "dfma", 3: "mufu_ex2", 4: "i2f", 5: "philox_block",
                  6: "smem_atomic_f32_cta", 7: "smem_atomic_f32_warp", 8: "smem_atomic_i32",
                  9: "smem_atomic_f64", 10: "philox_block_wide", 11: "shfl",
                  12: "owner_bin_update", 13: "smem_atomic_u64_cta", 14: "smem_atomic_u64_warp",
                  15: "smem_atomic_i32_warp"}


def vegas_microbench(op: int) -> float:
    """Thread-operations per second of one instruction class (see the header)."""
    r = ctypes.c_double()
    _check(lib().vegas_microbench(int(op), ctypes.byref(r)))
    return r.value


class Batch:
    """Owner of one vegas_batch handle."""

    def __init__(self, handle, ndims, nbins):
        self.handle, self.ndims, self.nbins = handle, list(ndims), int(nbins)

    @property
    def n(self):
        return len(self.ndims)

    def close(self):
        if self.handle:
            lib().vegas_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _bcheck(st: int, handle=None):
    if st != OK:
        msg = lib().vegas_batch_last_error(handle)
        raise VegasError(st, msg.decode() if msg else "")


def vegas_batch_create(instances, *, nbins: int = 50, seed: int = 1, precision=FP32_ACCCOMP,
                       ybits: int = 0, alpha: float = 1.5, stream=None) -> Batch:
    """instances: sequence of dicts with kind, ndim, params, ncall and
    optionally instance (Philox id, default: position)."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    n = len(instances)
    cfgs = (Config * n)()
    fns = (IntegrandDesc * n)()
    keep = []
    for i, ins in enumerate(instances):
        p = np.ascontiguousarray(ins["params"], dtype=np.float64)
        keep.append(p)
        cfgs[i] = Config(int(ins["ndim"]), int(nbins), int(ins["ncall"]), 1, 0.0, float(alpha), 0, int(seed),
                         int(ins.get("instance", i)), int(precision), int(ybits), _stream_handle(stream))
        fns[i] = IntegrandDesc(int(ins["kind"]), int(ins["ndim"]), _dp(p), len(p))
    h = _P()
    _bcheck(lib().vegas_batch_create(n, cfgs, fns, ctypes.byref(h)))
    return Batch(h, [ins["ndim"] for ins in instances], nbins)


def vegas_batch_destroy(b: Batch):
    b.close()


def vegas_batch_iterate(b: Batch, n_iter: int, refine: bool = True, result: bool = True):
    out = (Result * b.n)()
    _bcheck(lib().vegas_batch_iterate(b.handle, int(n_iter), int(bool(refine)), out if result else None), b.handle)
    return [r.as_dict() for r in out] if result else None


def vegas_batch_reset(b: Batch):
    _bcheck(lib().vegas_batch_reset(b.handle), b.handle)


def vegas_batch_set_params(b: Batch, params, first: int = 0):
    """New parameter blocks for instances first, first+1, ...: a 2-D array
    (one row per instance, rows at least as long as each block) or a list
    of 1-D blocks."""
    if isinstance(params, np.ndarray) and params.ndim == 2:
        a = np.ascontiguousarray(params, dtype=np.float64)
    else:
        rows = [np.asarray(p, dtype=np.float64).ravel() for p in params]
        a = np.zeros((len(rows), max((len(r) for r in rows), default=0)))
        for j, r in enumerate(rows):
            a[j, :len(r)] = r
    _bcheck(lib().vegas_batch_set_params(b.handle, int(first), int(a.shape[0]), _dp(a), int(a.shape[1])), b.handle)


def vegas_batch_get_grid(b: Batch, i: int, bin_sums: bool = False):
    d = b.ndims[i]
    e = np.zeros((d, b.nbins + 1))
    s = np.zeros((2, d, b.nbins)) if bin_sums else None
    _bcheck(lib().vegas_batch_get_grid(b.handle, int(i), _dp(e), _dp(s) if bin_sums else None), b.handle)
    return (e, s) if bin_sums else e


def vegas_batch_get_history(b: Batch, i: int, max_iters: int = 64):
    h = np.zeros((max_iters, 2))
    n = ctypes.c_int()
    _bcheck(lib().vegas_batch_get_history(b.handle, int(i), _dp(h), int(max_iters), ctypes.byref(n)), b.handle)
    return h[:min(n.value, max_iters)]


def vegas_batch_set_launch(b: Batch, threads: int, rounds: int):
    _bcheck(lib().vegas_batch_set_launch(b.handle, int(threads), int(rounds)), b.handle)


def vegas_batch_get_launch(b: Batch):
    t, r, c, it = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _bcheck(lib().vegas_batch_get_launch(b.handle, ctypes.byref(t), ctypes.byref(r), ctypes.byref(c),
                                         ctypes.byref(it)), b.handle)
    return dict(threads=t.value, rounds=r.value, ctas=c.value, items=it.value)


def vegas_batch_set_tile(b: Batch, points_per_thread: int = 0):
    _bcheck(lib().vegas_batch_set_tile(b.handle, int(points_per_thread)), b.handle)


def vegas_batch_get_tile(b: Batch):
    p, c = ctypes.c_int(), ctypes.c_int()
    _bcheck(lib().vegas_batch_get_tile(b.handle, ctypes.byref(p), ctypes.byref(c)), b.handle)
    return dict(points_per_thread=p.value, cap=c.value)


def vegas_batch_autotune(b: Batch):
    t, r, m = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _bcheck(lib().vegas_batch_autotune(b.handle, ctypes.byref(t), ctypes.byref(r), ctypes.byref(m)), b.handle)
    return dict(threads=t.value, rounds=r.value, ms=m.value)


def vegas_batch_profile(b: Batch, n_pass: int = 5):
    ms = np.zeros(2)
    _bcheck(lib().vegas_batch_profile(b.handle, int(n_pass), _dp(ms)), b.handle)
    return dict(sample=ms[0], finalize=ms[1])


def vegas_batch_last_error(b: Batch | None = None) -> str:
    m = lib().vegas_batch_last_error(b.handle if b else None)
    return m.decode() if m else ""


def vegas_fail_alloc_after(n: int) -> None:
    """Let the next n device / pinned allocations succeed and fail the one
    after (n < 0: disarm); see include/gvegas.h."""
    lib().vegas_fail_alloc_after(int(n))


def vegas_alloc_count() -> int:
    """Allocations the library has attempted so far (monotonic)."""
    return int(lib().vegas_alloc_count())


def vegas_last_error(ctx: Context | None = None) -> str:
    m = lib().vegas_last_error(ctx.handle if ctx else None)
    return m.decode() if m else ""
