"""Host-side launch-shape logic of kernels.h (choose_tile, choose_lanes),
compiled for the host and run without a GPU against a model of occupancy:

* tiles: points per thread a multiple of the kernel's minimum (a forced
  request rounded up to it), bucket capacity a multiple of 4 in 4..64, the
  reported occupancy the model's for that capacity, and with the small
  policy no smaller capacity of the searched range reaching the same
  occupancy; the large policy never takes a smaller capacity than the
  small one for the same tile; the dense floor never loses occupancy
  against the small policy;
* lanes: a power of two, at most 32 and at most the points per hypercube,
  the smallest that gives four rounds of work (or the bound).
"""
import json
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("host") / "tile_chooser")
    src = os.path.join(HERE, "host", "tile_chooser.cu")
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-o", exe, src],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    js, lanes = out.split("LANES")
    return json.loads(js), [tuple(int(v) for v in t.split(",")) for t in lanes.split()]


def test_tile_invariants(run):
    tiles, _ = run
    assert len(tiles) > 1000
    for t in tiles:
        assert t["ppt"] % t["ppt_min"] == 0 or t["ppt_req"] > 0, t
        if t["ppt_req"] > 0:
            want = -(-t["ppt_req"] // t["ppt_min"]) * t["ppt_min"]
            assert t["ppt"] == want, t
        else:
            assert t["ppt"] in (1, 2, 4) and t["ppt"] >= t["ppt_min"], t
        assert t["cap"] % 4 == 0 and 4 <= t["cap"] <= 64, t
        if t["occ"] > 0:
            assert t["occ"] == t["occ_check"], t


def test_small_policy_takes_the_smallest_capacity_of_equal_occupancy(run):
    tiles, _ = run
    key = lambda t: (t["threads"], t["N"], t["dN"], t["reg_cap"], t["ppt_req"], t["ppt_min"])
    by = {}
    for t in tiles:
        by.setdefault(key(t), {})[t["small"]] = t
    for k, pair in by.items():
        big, small = pair[0], pair[1]
        if big["ppt"] == small["ppt"] and big["occ"] == small["occ"] and big["occ"] > 0:
            assert small["cap"] <= big["cap"], (big, small)


def test_dense_floor_never_loses_occupancy(run):
    """The dense floor extends the small policy's range downwards: for the
    same tile it reaches at least the small policy's occupancy, and where
    the small policy found its capacity inside its own range (not by the
    halving fallback of a forced tile), never a larger one."""
    import math
    tiles, _ = run
    key = lambda t: (t["threads"], t["N"], t["dN"], t["reg_cap"], t["ppt_req"], t["ppt_min"])
    ceil4 = lambda v: (int(v) + 1 + 3) & ~3
    by = {}
    for t in tiles:
        by.setdefault(key(t), {})[t["small"]] = t
    checked = 0
    for k, trio in by.items():
        small, dense = trio[1], trio[2]
        if small["ppt"] == dense["ppt"] and small["occ"] > 0:
            assert dense["occ"] >= small["occ"], (small, dense)
            m = small["threads"] * small["ppt"] / small["N"]
            lo_small = min(ceil4(m + 2 * math.sqrt(m) + 1), min(ceil4(m + 4 * math.sqrt(m) + 2), 64))
            if dense["occ"] == small["occ"] and small["cap"] >= lo_small:
                assert dense["cap"] <= small["cap"], (small, dense)
            checked += 1
    assert checked > 100


def test_lanes(run):
    _, lanes = run
    assert lanes
    for G, nc, threads, ctas, L in lanes:
        assert L & (L - 1) == 0 and 1 <= L <= 32
        assert L == 1 or 2 * (L // 2) <= nc and L <= nc
        if L < 32 and 2 * L <= nc:
            assert G * L >= 4 * ctas * threads
        if L > 1:
            assert G * (L // 2) < 4 * ctas * threads
