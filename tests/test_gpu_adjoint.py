"""Adjoint pass (vegas_grad) against the oracle's estimator gradient on the
same points, against central differences of the GPU's own estimate with
common random numbers, and through torch.autograd.

Bars: FP64 form, |dI_gpu - dI_oracle| <= 1e-9 * (1/n) sum |J df/dtheta|
(condition-scaled: the Breit-Wigner derivatives change sign across the
peak); FP32 form, the same with 1e-4; central differences of the FP64
estimate within 1e-3 relative (h chosen so truncation is below that).
A point whose oracle cut margin is below the form's rounding (1e-13 in
FP64, 1e-4 in FP32) may be cut in one arithmetic and kept in the other:
every point is dumped, and where the GPU and the oracle decide a point
inside that margin differently the oracle's sums take the GPU's decision
(the point's terms without the hard cuts) before the comparison."""
import numpy as np
import pytest

from paper_1010_2107_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gv():
    from paper_1010_2107_gb300 import _build, gvegas
    _build.build()
    return gvegas


def _theta_slots(kind, d):
    from paper_1010_2107_gb300.autograd import theta_slots
    return theta_slots(kind, d)


CASES = [
    ("rambo4_sigmoid", wl.RAMBO_BW, 16, wl.rambo_params(4, cut=1), 1 << 15),
    ("rambo5_hard", wl.RAMBO_BW, 20, wl.rambo_params(5, cut=0), 1 << 15),
    ("dgauss4", wl.DOUBLE_GAUSSIAN, 4, np.array([0.3, 0.7, 0.1]), 1 << 15),
    ("gauss3", wl.GENZ_GAUSSIAN, 3, np.array([4.0, 6.0, 3.0, 0.4, 0.5, 0.6]), 1 << 15),
]


@pytest.mark.parametrize("name,kind,d,params,n", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision,ybits,tol", [(0, 53, 1e-9), (2, 24, 1e-4)])
def test_gradient_matches_oracle(gv, orc, name, kind, d, params, n, precision, ybits, tol):
    with gv.vegas_create(kind, d, params, ncall=n, precision=precision, ybits=ybits, seed=3) as ctx:
        gv.vegas_iterate(ctx, 2, refine=True)  # a non-uniform frozen grid
        edges = gv.vegas_get_grid(ctx)
        g, I = gv.vegas_grad(ctx, 5)
        I_eval, _ = gv.vegas_eval(ctx, 5)
        dump = gv.vegas_sample_dump(ctx, 5, np.arange(n))
    cfg = orc.make_cfg(d, nbins=50, ncall=n, ybits=ybits, seed=3)
    fn = orc.Integrand(kind, d, params)
    go, Io = orc.gradient(cfg, fn, edges, 5)
    p = orc.sample_batch(cfg, edges, 5, np.arange(n))
    gp = orc.integrand_grad(fn, p["x"]) * p["jac"][:, None]
    scale = np.abs(gp).mean(axis=0)
    # RAMBO's hard cuts: points inside the cut margin that the GPU and the
    # oracle decide differently take the GPU's decision in the oracle's sums
    flip = np.zeros(n, dtype=bool)
    if kind == wl.RAMBO_BW:
        near = orc.cut_margin(fn, p["x"]) < (1e-13 if precision == 0 else 1e-4)
        kept_gpu, kept = dump["f"] != 0, orc.integrand(fn, p["x"]) != 0
        flip = near & (kept_gpu != kept)
        assert not np.any((kept_gpu != kept) & ~near), "a cut decided differently outside the margin"
    if flip.any():
        q = np.asarray(params, dtype=np.float64).copy()
        q[wl.RB_DRMIN] = 0.0
        if q[wl.RB_CUT] == 0:
            q[wl.RB_PTMIN] = 0.0
        free = orc.Integrand(kind, d, q)
        sign = np.where(kept_gpu[flip], 1.0, -1.0)
        go = go + (sign[:, None] * orc.integrand_grad(free, p["x"][flip]) * p["jac"][flip, None]).sum(axis=0) / n
        Io = Io + float((sign * orc.integrand(free, p["x"][flip]) * p["jac"][flip]).sum()) / n
    assert np.all(np.abs(g - go) <= tol * scale + 1e-300), (g, go, scale, int(flip.sum()))
    assert I == pytest.approx(Io, rel=tol * 10, abs=1e-300)
    assert I == pytest.approx(I_eval, rel=max(tol, 1e-12) * 10, abs=1e-300)


@pytest.mark.parametrize("name,kind,d,params,n", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_gradient_matches_crn_central_differences(gv, name, kind, d, params, n):
    slots = _theta_slots(kind, d)
    with gv.vegas_create(kind, d, params, ncall=n, precision=0, seed=5) as ctx:
        gv.vegas_iterate(ctx, 2, refine=True)
        g, _ = gv.vegas_grad(ctx, 9)
        for j, slot in enumerate(slots):
            # M, Gamma: 1e-3 GeV and T: 1e-2 GeV keep the O(h^2) truncation
            # below 1e-3 against the 2.1 GeV width and the 1 GeV cut width
            h = {wl.RB_M: 1e-3, wl.RB_GAMMA: 1e-3, wl.RB_T: 1e-2}[slot] if kind == wl.RAMBO_BW else 1e-6
            pp, pm = params.copy(), params.copy()
            pp[slot] += h
            pm[slot] -= h
            gv.vegas_set_params(ctx, pp)
            Ip, _ = gv.vegas_eval(ctx, 9)
            gv.vegas_set_params(ctx, pm)
            Im, _ = gv.vegas_eval(ctx, 9)
            gv.vegas_set_params(ctx, params)
            fd = (Ip - Im) / (2 * h)
            if kind == wl.RAMBO_BW and slot == wl.RB_T and params[wl.RB_CUT] == 0:
                continue
            assert g[j] == pytest.approx(fd, rel=1e-3, abs=1e-9 * abs(g).max()), (j, g[j], fd)


def test_autograd_function(gv):
    torch = pytest.importorskip("torch")
    from paper_1010_2107_gb300.autograd import vegas_estimate
    kind, d, params = wl.RAMBO_BW, 16, wl.rambo_params(4, cut=1)
    with gv.vegas_create(kind, d, params, ncall=1 << 15, precision=2, seed=2) as ctx:
        gv.vegas_iterate(ctx, 2)
        theta = torch.tensor([80.4, 2.1, 20.0], dtype=torch.float64, requires_grad=True)
        I = vegas_estimate(theta, ctx, 11, params, kind)
        (2.0 * I).backward()
        g, I_ref = gv.vegas_grad(ctx, 11)
    assert float(I.detach()) == pytest.approx(I_ref, rel=1e-12)
    np.testing.assert_allclose(theta.grad.numpy(), 2.0 * g, rtol=1e-12)


def test_gradient_rejects_kinds_without_adjoint(gv):
    with gv.vegas_create(wl.GENZ_CORNER_PEAK, 3, [0.1, 0.2, 0.3], ncall=1000) as ctx:
        with pytest.raises(gv.VegasError):
            gv.vegas_grad(ctx, 0)
