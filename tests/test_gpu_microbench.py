"""The measured-rate microbenchmarks run and return finite positive rates."""
import math

import pytest

pytestmark = pytest.mark.gpu


def test_microbench_rates():
    from paper_1010_2107_gb300 import _build, gvegas as gv
    _build.build()
    for op in gv.MICROBENCH_OPS:
        r = gv.vegas_microbench(op)
        assert math.isfinite(r) and r > 0, (op, r)
    with pytest.raises(gv.VegasError):
        gv.vegas_microbench(99)
