"""Allocation failures, injected on the host: the library's allocation
wrapper fails the chosen call before the allocator runs
(vegas_fail_alloc_after), so no GPU fault is involved.  Every constructor
must answer VEGAS_ENOMEM and free what it had allocated: device memory is
unchanged over 100 failing constructions, and the library works afterwards."""
import numpy as np
import pytest

from paper_1010_2107_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

MIB = 1 << 20


@pytest.fixture(scope="module")
def gv():
    from paper_1010_2107_gb300 import _build, gvegas
    _build.build()
    return gvegas


def _allocs_of(gv, make):
    c0 = gv.vegas_alloc_count()
    h = make()
    n = gv.vegas_alloc_count() - c0
    h.close()
    return n


def _cycles(gv, make, n_allocs, cycles=100):
    import torch
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for i in range(cycles):
        gv.vegas_fail_alloc_after(i % n_allocs)
        with pytest.raises(gv.VegasError) as e:
            make()
        assert e.value.status == gv.ENOMEM, str(e.value)
    gv.vegas_fail_alloc_after(-1)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert abs(free0 - free1) <= MIB, (free0, free1)


def test_context_creation_frees_everything_on_failure(gv, orc):
    pytest.importorskip("torch")
    d, N = 16, 64  # large buffers (partial rows of 2 d N per CTA): a leak shows
    p = wl.genz_gaussian_params(d, a=2.0)
    kw = dict(nbins=N, ncall=1 << 20, precision=2, ybits=24, seed=1)
    make = lambda: gv.vegas_create(gv.GENZ_GAUSSIAN, d, p, **kw)
    with make() as warm:  # loads the kernels and sizes the driver's pools
        gv.vegas_iterate(warm, 1)
    n = _allocs_of(gv, make)
    assert n >= 10
    _cycles(gv, make, n)
    # the library still works, and on the oracle's numbers
    kw2 = dict(nbins=50, ncall=20_000, precision=0, seed=1)
    with gv.vegas_create(gv.GENZ_GAUSSIAN, 4, wl.genz_gaussian_params(4), **kw2) as ctx:
        I, _ = gv.vegas_eval(ctx, 0)
    cfg = orc.make_cfg(4, nbins=50, ncall=20_000, ybits=53, seed=1)
    o = orc.iteration(cfg, orc.Integrand(gv.GENZ_GAUSSIAN, 4, wl.genz_gaussian_params(4)),
                      orc.uniform_grid(4, 50), 0)
    assert I == pytest.approx(o["I"], rel=1e-12)


def test_batch_creation_frees_everything_on_failure(gv):
    pytest.importorskip("torch")
    insts = wl.genz_batch(24, seed=5, log2n_min=14, log2n_max=16)
    make = lambda: gv.vegas_batch_create(insts, nbins=50, seed=1, precision=gv.FP32_ACCCOMP, ybits=24)
    with make() as warm:
        gv.vegas_batch_iterate(warm, 1, refine=True)
    n = _allocs_of(gv, make)
    assert n >= 10
    _cycles(gv, make, n)


def test_failure_in_a_later_allocation_keeps_the_context_usable(gv):
    """An allocation that fails inside a call on a live context (the SPRING
    buffers, grown on first use) answers VEGAS_ENOMEM and leaves the context
    usable: the next call allocates and succeeds."""
    d, g = 4, 4
    kw = dict(nbins=50, ncall=g ** d * 32, nstrat=g, precision=0, ybits=24, seed=3)
    with gv.vegas_create(gv.DOUBLE_GAUSSIAN, d, wl.double_gaussian_params(), **kw) as ctx:
        gv.bases_integrate(ctx, 2, 0.0, 2, 0.0)
        gv.vegas_fail_alloc_after(0)
        with pytest.raises(gv.VegasError) as e:
            gv.spring_generate(ctx, 0, 4096, events=False)
        assert e.value.status == gv.ENOMEM
        gv.vegas_fail_alloc_after(-1)
        r = gv.spring_generate(ctx, 0, 4096, events=False)
        assert r["n_events"] > 0


def test_failed_parameter_staging_keeps_the_batch_usable(gv):
    """vegas_batch_set_params allocates its pinned staging on first use: when
    that allocation fails the call answers VEGAS_ENOMEM with the batch's
    parameters unchanged, and the next call succeeds."""
    insts = wl.genz_batch(8, seed=5, log2n_min=12, log2n_max=13)
    with gv.vegas_batch_create(insts, nbins=50, seed=1, precision=gv.FP32_ACCCOMP, ybits=24) as b:
        r0 = gv.vegas_batch_iterate(b, 1)
        gv.vegas_fail_alloc_after(0)
        with pytest.raises(gv.VegasError) as e:
            gv.vegas_batch_set_params(b, [ins["params"] for ins in insts])
        assert e.value.status == gv.ENOMEM
        gv.vegas_fail_alloc_after(-1)
        gv.vegas_batch_reset(b)
        r1 = gv.vegas_batch_iterate(b, 1)
        assert [r["I"] for r in r1] == [r["I"] for r in r0]  # parameters unchanged
        gv.vegas_batch_set_params(b, [ins["params"] for ins in insts])
        gv.vegas_batch_reset(b)
        r2 = gv.vegas_batch_iterate(b, 1)
        assert [r["I"] for r in r2] == [r["I"] for r in r0]
