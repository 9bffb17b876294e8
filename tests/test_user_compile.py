"""Run-time compilation of user integrands without a device (vegas_user_compile):
the library's embedded kernel headers compile under NVRTC for sm_103a in every
precision form and kernel shape, and a faulty source comes back as
VEGAS_EINVAL with the compiler's log pointing at the user's own lines."""
import pytest

GAUSS = r"""
template <typename T>
__device__ T vegas_user_f(const T* x, int d, const T* p) {
  T q = T(0);
  for (int i = 0; i < d; ++i) {
    const T t = x[i] - p[d + i];
    q += p[i] * p[i] * t * t;
  }
  return exp(-q);
}
"""


@pytest.fixture(scope="module")
def gv():
    from paper_1010_2107_gb300 import _build, gvegas
    _build.build()
    return gvegas


@pytest.mark.parametrize("d,precision,ybits,nstrat,ncall", [
    (4, 0, 53, 0, 10000),      # FP64, general kernels
    (4, 0, 24, 4, 4 ** 4 * 8),  # FP64, specialised kernels
    (8, 2, 24, 2, 2 ** 8 * 8),  # compensated FP32, specialised, two points in flight
    (9, 2, 24, 0, 10000),      # compensated FP32, general
    (3, 1, 53, 0, 10000),      # FP32 with FP64 sums
    (32, 2, 24, 0, 10000),     # largest dimension
])
def test_user_source_compiles(gv, d, precision, ybits, nstrat, ncall):
    gv.vegas_user_compile(GAUSS, d, ncall=ncall, nstrat=nstrat, precision=precision, ybits=ybits)


def test_compile_error_reports_the_users_line(gv):
    bad = GAUSS.replace("return exp(-q);", "return exp(-q) + not_declared;")
    with pytest.raises(gv.VegasError) as e:
        gv.vegas_user_compile(bad, 4)
    assert e.value.status == gv.EINVAL
    msg = str(e.value)
    assert "not_declared" in msg and "vegas_user_f(9)" in msg


def test_missing_entry_point_is_rejected(gv):
    with pytest.raises(gv.VegasError) as e:
        gv.vegas_user_compile("__device__ float g(float x) { return x; }", 2)
    assert e.value.status == gv.EINVAL and "vegas_user_f" in str(e.value)


def test_bad_shapes_are_rejected_before_compiling(gv):
    for kw in (dict(ndim=0), dict(ndim=33), dict(ndim=4, precision=7), dict(ndim=4, ybits=30)):
        d = kw.pop("ndim")
        with pytest.raises(gv.VegasError) as e:
            gv.vegas_user_compile(GAUSS, d, **kw)
        assert e.value.status == gv.EINVAL


def test_library_helpers_are_visible_to_user_code(gv):
    """The embedded kernel headers come with their device helpers (namespace
    gv): the benchmarked two-peak Gaussian source uses gv::gexp."""
    from paper_1010_2107_gb300 import workloads as wl
    gv.vegas_user_compile(wl.DGAUSS_USER_SOURCE, 8, ncall=4 ** 8 * 2, nstrat=4, precision=2, ybits=24)
    src = ("template <typename T> __device__ T vegas_user_f(const T* x, int d, const T* p) "
           "{ return gv::qsqrt(x[0]) * gv::vexp(-x[1]); }")
    for precision in (0, 2):
        gv.vegas_user_compile(src, 2, precision=precision)


def test_embedded_kernel_headers_are_current(gv):
    """The build embeds the kernel headers in the library as text for the
    run-time compiler; the generated table holds every header as it is on
    disk (checked on a distinctive line of each)."""
    import os
    from paper_1010_2107_gb300 import _build
    inc = open(_build.RTC_INC).read()
    for name, path in _build.RTC_HEADERS:
        assert '{"' + name + '",' in inc
        lines = [l for l in open(path).read().splitlines() if len(l.strip()) > 40 and ")gvrtc" not in l]
        assert lines and lines[len(lines) // 2] in inc, path
    assert os.path.getmtime(_build.RTC_INC) >= max(os.path.getmtime(p) for _, p in _build.RTC_HEADERS) - 1
