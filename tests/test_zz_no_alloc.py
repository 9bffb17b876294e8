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
def test_noalloc_pass_matches_context_pass(kind, d, params, N, ncall, g, prec, ybits, tol):
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
