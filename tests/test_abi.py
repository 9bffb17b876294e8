"""The C ABI library loads and exports every entry point include/gvegas.h
declares; argument validation answers with status codes (no GPU needed: the
checks run before any CUDA call)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gvlib():
    from paper_1010_2107_gb300 import _build, gvegas
    _build.build()
    return gvegas


def _declared():
    text = open(os.path.join(ROOT, "include", "gvegas.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b((?:vegas|bases)_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(gvlib):
    names = _declared()
    assert "vegas_create" in names and "bases_integrate" in names and "vegas_get_grid" in names
    L = gvlib.lib()
    for n in names:
        assert hasattr(L, n), n


def test_binding_covers_the_header(gvlib):
    for n in _declared():
        assert callable(getattr(gvlib, n, None)), n


def _cfg(gv, **kw):
    base = dict(ndim=4, nbins=50, ncall=1000, itmx=5, acc=0.0, alpha=1.5, nstrat=0, seed=1,
                instance=0, precision=0, ybits=0, stream=None)
    base.update(kw)
    return gv.Config(**base)


@pytest.mark.parametrize("bad,msg", [
    (dict(ndim=0), "ndim"), (dict(ndim=33), "ndim"), (dict(nbins=1), "nbins"),
    (dict(nbins=257), "nbins"), (dict(ncall=1), "ncall"), (dict(precision=7), "precision"),
    (dict(ybits=32), "ybits"), (dict(nstrat=4, ncall=1000), "multiple"),
    (dict(nstrat=4, ncall=256), "2 points"), (dict(alpha=-1.0), "alpha"),
])
def test_invalid_config_is_rejected(gvlib, bad, msg):
    gv = gvlib
    import numpy as np
    p = np.zeros(2 * 33)
    cfg = _cfg(gv, **bad)
    fn = gv.IntegrandDesc(gv.GENZ_GAUSSIAN, cfg.ndim, p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          2 * cfg.ndim)
    h = ctypes.c_void_p()
    st = gv.lib().vegas_create(ctypes.byref(cfg), ctypes.byref(fn), ctypes.byref(h))
    assert st == gv.EINVAL
    assert not h.value
    assert msg in gv.vegas_last_error(None)


@pytest.mark.parametrize("kind,ndim,np_,msg", [
    (0, 4, 7, "parameters"), (5, 20, 10, None), (5, 18, 10, "4 n"), (9, 4, 4, "kind"),
    (8, 4, 15, "ndim 5"), (8, 5, 14, "parameters"), (8, 5, 15, "CUTS"), (8, 5, 15, "SMIN"),
])
def test_invalid_integrand_is_rejected(gvlib, kind, ndim, np_, msg):
    gv = gvlib
    import numpy as np
    from paper_1010_2107_gb300 import workloads as wl
    p = wl.rambo_params(5) if kind == 5 else np.ones(np_)
    if kind == 5 and ndim == 20:
        p = p.copy()
        p[wl.RB_CUT] = 7
        msg = "cut"
    if kind == 8 and np_ == 15:
        p = wl.w_munu_params()
        if msg == "CUTS":
            p[wl.W_CUTS] = 2
        if msg == "SMIN":
            p[wl.W_SMIN] = p[wl.W_SQRTS] ** 2
    cfg = _cfg(gv, ndim=ndim)
    fn = gv.IntegrandDesc(kind, ndim, p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(p))
    h = ctypes.c_void_p()
    st = gv.lib().vegas_create(ctypes.byref(cfg), ctypes.byref(fn), ctypes.byref(h))
    assert st == gv.EINVAL and not h.value
    assert msg in gv.vegas_last_error(None)


def test_null_arguments(gvlib):
    gv = gvlib
    L = gv.lib()
    assert L.vegas_create(None, None, None) == gv.EINVAL
    assert L.vegas_iterate(None, 1, 1, None) == gv.EINVAL
    assert L.vegas_get_grid(None, None, None) == gv.EINVAL
    assert L.bases_integrate(None, 1, 0.0, 1, 0.0, None, None) == gv.EINVAL
    assert L.vegas_batch_set_params(None, 0, 1, None, 1) == gv.EINVAL
    L.vegas_destroy(None)
    assert isinstance(gv.vegas_last_error(None), str)


@pytest.mark.parametrize("kind,ndim,params", [
    (8, 5, None),          # W -> mu nu: a single-context workload
    (5, 8, None),          # RAMBO
    (64, 4, [1.0, 2.0]),   # run-time compiled kinds have no batched kernel
])
def test_batch_rejects_unbatched_kinds(gvlib, kind, ndim, params):
    gv = gvlib
    import numpy as np
    from paper_1010_2107_gb300 import workloads as wl
    if params is None:
        params = wl.w_munu_params() if kind == 8 else wl.rambo_params(2)
    with pytest.raises(gv.VegasError) as e:
        gv.vegas_batch_create([dict(kind=kind, ndim=ndim, ncall=1000, params=np.asarray(params, float))])
    assert e.value.status == gv.EINVAL


def test_user_kind_needs_its_own_constructor(gvlib):
    gv = gvlib
    import numpy as np
    with pytest.raises(gv.VegasError) as e:
        gv.vegas_create(gv.USER, 4, np.ones(3))
    assert e.value.status == gv.EINVAL and "kind" in str(e.value)
    with pytest.raises(gv.VegasError) as e:
        gv.vegas_create_user("template <typename T> __device__ T vegas_user_f(const T* x, int d, const T* p)"
                             " { return x[0]; }", 4, np.ones(gv.MAXUSERPARAMS + 1))
    assert e.value.status == gv.EINVAL


def test_allocation_hook_is_host_only(gvlib):
    """vegas_fail_alloc_after / vegas_alloc_count run without a device: the
    counter is monotonic and arming or disarming it calls nothing on a GPU."""
    gv = gvlib
    c0 = gv.vegas_alloc_count()
    gv.vegas_fail_alloc_after(3)
    gv.vegas_fail_alloc_after(-1)
    assert gv.vegas_alloc_count() >= c0 >= 0
