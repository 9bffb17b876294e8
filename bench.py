#!/usr/bin/env python
"""Benchmark of the GB300 VEGAS / BASES hot path.

Default workload (``genz256``, the largest configuration): 256 independent
Genz integrands (product peak, corner peak, oscillatory; d from 2 to 16;
2^16..2^22 points each, about 2.5e8 points per iteration), FP32 map and
integrand with compensated FP32 sums, 50 bins per axis, 8 refining VEGAS
iterations of every instance from the uniform grid per step, as one batch.

Metric: points (samples) per second through the iteration loop, whole job.
Also reported: the plain FP64 GPU path on the same points (speed-up, and the
largest difference of the two estimates in units of sigma), the roofline of
the sampling pass, the CPU oracle timed on the host, the end-to-end rate
through the C ABI with host buffers, and (one GPU) the same figures for the
dgauss8 BASES, rambo5 and rambo4_adjoint workloads under ``workloads``.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own replica (different Philox instance word,
so different points) and the rates add up: weak scaling, no collective on the
data path; a barrier and a max-reduction of the elapsed time only.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "samples/sec per VEGAS/BASES iteration vs plain FP64 GPU path; % FP32 peak"
UNIT = "samples/s"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2

# Algorithmic FP32-pipe operations per point of the sampling kernel:
# Philox, word->bin/position, map, integrand, sums (the roofline's unit of
# work; the peak is the FP32 issue rate of all SMs at the maximum clock).
ALGO_OPS = {
    "dgauss8": dict(philox=2 * 10 * 6, bins=8 * 8, map=8 * 3, integrand=8 * 4 + 8, histogram=8 * 2, sums=2 + 12),
    "gauss4": dict(philox=2 * 10 * 6, bins=4 * 7, map=4 * 3, integrand=4 * 3 + 2, histogram=4 * 2, sums=4),
    "rambo5": dict(philox=5 * 10 * 6, bins=20 * 6, map=20 * 3, integrand=5 * 60 + 10 * 8 + 5 * 14 + 10,
                   histogram=20 * 2, sums=14),
    "rambo4_adjoint": dict(philox=4 * 10 * 6, bins=16 * 6, map=16 * 3,
                           integrand=4 * 60 + 6 * 8 + 4 * 14 + 10 + 4 * 6 + 20, sums=5 * 7),
    # per SPRING trial: three Philox blocks (8 point words, 2 cube words,
    # 1 acceptance word), a 16-step bisection over the cube table, bins,
    # map, integrand and the keep decision
    "spring_dgauss8": dict(philox=3 * 10 * 6, cube_search=16 * 3, bins=8 * 6, map=8 * 3,
                           integrand=8 * 4 + 8, keep=10),
    # the W integrand counted for the points of the coupling helicity cell
    # (the adapted grid sends nearly all points there): tan, three logs,
    # two exponentials for x1 and x2, the eta cut, the density exponent
    "wmunu": dict(philox=2 * 10 * 6, bins=5 * 8, map=5 * 3, integrand=90, histogram=5 * 2, sums=2 + 12),
    "user_dgauss8": dict(philox=2 * 10 * 6, bins=8 * 8, map=8 * 3, integrand=8 * 4 + 8, histogram=8 * 2,
                         sums=2 + 12),
}
# (`histogram`: the per-bin scatter, 2 per axis, which the passes that leave
# the grid unchanged skip.)
# DRAM bytes per launch of the sampling kernel from the committed ncu
# capture (profiles/), per pass kind (refining, frozen grid); a workload
# whose kernel changed since its capture has no entry.
TRAFFIC = {"dgauss8": (83968, 614528), "rambo5": (108032,), "wmunu": (80896, 352512),
           "rambo4_adjoint": (45504,), "spring_dgauss8": (1017088 + 3060992,),
           # one batched pass: the sum over its fifteen dimension kernels
           "genz256": (3620992,)}


def _workload(name):
    from paper_1010_2107_gb300 import workloads as wl
    return wl.WORKLOADS[name]


def _oracle_integrand(w):
    """The oracle's integrand of a workload (a user source's built-in twin)."""
    import oracle
    return oracle.Integrand(w.get("oracle_kind", w["kind"]), w["ndim"], w.get("oracle_params", w["params"]))


def _measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.p = None
        return self

    def __exit__(self, *exc):
        if self.p:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                self.out = ""
        else:
            self.out = ""

    def summary(self):
        rows = [r.split(",") for r in (self.out or "").strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i]
                          and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0, None
    import torch.distributed as dist
    dist.init_process_group(backend="nccl" if _cuda() else "gloo")
    return dist.get_rank(), dist.get_world_size(), int(os.environ.get("LOCAL_RANK", "0")), dist


def max_over_ranks(x, dist):
    """The largest value of x over all ranks (x itself on one rank): the
    job's elapsed time is the slowest rank's."""
    if not dist:
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_step, steps, seconds):
    """Units per second of the whole job: every rank processes
    units_per_step per step (weak scaling), in the slowest rank's time."""
    return world * units_per_step * steps / seconds


def rank_instance(base, rank, mode):
    """Philox instance word of a rank's replica: the context's instance is
    the rank; a batch's instances are offset by 1024 per rank (a batch holds
    fewer than 1024 instances), so no two ranks draw the same points."""
    return base + 1024 * rank if mode == "batched" else rank


def _cuda():
    import torch
    return torch.cuda.is_available()


# --------------------------------------------------------------------- oracle


def oracle_rate(name: str, iters_refine: int, iters_frozen: int):
    """The CPU oracle as it stands, single-threaded, on full-NCALL BASES
    iterations of the workload; returns (points/s, points, seconds)."""
    import oracle
    w = _workload(name)
    d = w["ndim"]
    cfg = oracle.make_cfg(d, nbins=w["nbins"], ncall=w["ncall"], nstrat=w["nstrat"], ybits=w["ybits"],
                          seed=w["seed"])
    fn = _oracle_integrand(w)
    e = oracle.uniform_grid(d, w["nbins"])
    t = time.perf_counter()
    if w.get("mode") == "bases":
        oracle.bases(cfg, fn, e, 0, iters_refine, 0.0, iters_frozen, 0.0)
    else:
        oracle.vegas(cfg, fn, e, 0, iters_refine + iters_frozen)
    dt = time.perf_counter() - t
    n = w["ncall"] * (iters_refine + iters_frozen)
    return n / dt, n, dt


def oracle_spring_rate(R, h, n=1 << 20):
    """The oracle's SPRING on the context's own grid and cube maxima."""
    import oracle
    oracle.build()
    gv, w = R.gv, R.w
    d = w["ndim"]
    cfg = oracle.make_cfg(d, nbins=w["nbins"], ncall=w["ncall"], nstrat=w["nstrat"], ybits=w["ybits"],
                          seed=w["seed"])
    fn = _oracle_integrand(w)
    edges, cmax = gv.vegas_get_grid(h), gv.vegas_get_cube_max(h)
    t = time.perf_counter()
    oracle.spring(cfg, fn, edges, cmax, 0, n)
    dt = time.perf_counter() - t
    return n / dt, n, dt


def _oracle_worker(job):
    """One process of the all-core CPU baseline: the oracle on its own
    instance word (a disjoint Philox counter range), timed inside."""
    name, instance = job
    import oracle
    oracle.build()
    w = _workload(name)
    d = w["ndim"]
    cfg = oracle.make_cfg(d, nbins=w["nbins"], ncall=w["ncall"], nstrat=w["nstrat"], ybits=w["ybits"],
                          seed=w["seed"], instance=instance)
    fn = _oracle_integrand(w)
    oracle.vegas(cfg, fn, oracle.uniform_grid(d, w["nbins"]), 0, 1)  # untimed warm-up
    e = oracle.uniform_grid(d, w["nbins"])
    t = time.perf_counter()
    oracle.vegas(cfg, fn, e, 0, 1)
    return w["ncall"], time.perf_counter() - t


def oracle_rate_allcores(name: str):
    """The oracle as it stands, one full-NCALL iteration in each of P
    independent processes (P = the cores this process may use), each on
    disjoint counter ranges: points of all processes over the slowest
    process's time.  Spawned processes (no fork after CUDA is up)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    P = len(os.sched_getaffinity(0))
    # a worker that dies makes the executor raise instead of waiting forever
    with ProcessPoolExecutor(max_workers=P, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_oracle_worker, [(name, 1 + p) for p in range(P)], timeout=600))
    n = sum(r[0] for r in res)
    dt = max(r[1] for r in res)
    return n / dt, n, dt, P


def _genz_sample(budget=1 << 22, stride=1, start=0):
    """Instances start, start + stride, ... of the batched workload, taken in
    order until they hold about `budget` points."""
    from paper_1010_2107_gb300 import workloads as wl
    insts = wl.genz_batch(wl.GENZ256["count"], wl.GENZ256["seed"])
    chosen, tot = [], 0
    for ins in insts[start::stride]:
        chosen.append(ins)
        tot += ins["ncall"]
        if tot >= budget:
            break
    return chosen, tot


def _oracle_genz(insts):
    """One iteration of each instance on its uniform grid through the oracle
    as it stands; returns (points, seconds)."""
    import oracle
    from paper_1010_2107_gb300 import workloads as wl
    t = time.perf_counter()
    for ins in insts:
        cfg = oracle.make_cfg(ins["ndim"], nbins=wl.GENZ256["nbins"], ncall=ins["ncall"], ybits=24,
                              seed=wl.GENZ256["sample_seed"], instance=ins["instance"])
        fn = oracle.Integrand(ins["kind"], ins["ndim"], ins["params"])
        oracle.iteration(cfg, fn, oracle.uniform_grid(ins["ndim"], wl.GENZ256["nbins"]), 0)
    return sum(i["ncall"] for i in insts), time.perf_counter() - t


def oracle_rate_batched():
    """The oracle, single-threaded, on the leading instances of the batch
    (about 2^22 points): (points/s, points, seconds, instances)."""
    import oracle
    oracle.build()
    chosen, _ = _genz_sample()
    n, dt = _oracle_genz(chosen)
    return n / dt, n, dt, len(chosen)


def _oracle_genz_worker(job):
    start, stride = job
    import oracle
    oracle.build()
    chosen, _ = _genz_sample(1 << 21, stride, start)
    return _oracle_genz(chosen)


def oracle_rate_batched_allcores():
    """One oracle process per core, each on its own instances of the batch
    (every P-th, about 2^21 points): points of all over the slowest time."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    P = len(os.sched_getaffinity(0))
    with ProcessPoolExecutor(max_workers=P, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_oracle_genz_worker, [(p, P) for p in range(P)], timeout=600))
    n = sum(r[0] for r in res)
    dt = max(r[1] for r in res)
    return n / dt, n, dt, P


def _reference_step(name):
    """One step of the reference arm (the oracle as it stands): returns a
    callable giving (points, seconds, description of the sample)."""
    import oracle
    if name == "genz256":
        chosen, tot = _genz_sample()  # the leading instances, about 2^22 points in all

        def step():
            n, dt = _oracle_genz(chosen)
            return n, dt, f"one iteration of the first {len(chosen)} instances ({n} points)"
        return step
    w = _workload(name)
    if w.get("mode") == "spring":
        d = w["ndim"]
        cfg = oracle.make_cfg(d, nbins=w["nbins"], ncall=w["ncall"], nstrat=w["nstrat"], ybits=w["ybits"],
                              seed=w["seed"])
        fn = _oracle_integrand(w)
        e = oracle.uniform_grid(d, w["nbins"])
        cmax = oracle.iteration(cfg, fn, e, 0, cubes=True)["Cmax"]  # bounds from one iteration
        n = 1 << 20

        def step():
            t = time.perf_counter()
            oracle.spring(cfg, fn, e, cmax, 0, n)
            return n, time.perf_counter() - t, f"{n} SPRING trials on the uniform grid"
        return step

    def step():
        _, n, dt = oracle_rate(name, 1, 0)
        return n, dt, f"one grid-optimising iteration of NCALL={w['ncall']}"
    return step


def run_reference(args):
    rank, world, _, dist = _dist()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    name = args.workload
    step = _reference_step(name)
    for _ in range(args.warmup):
        step()
    times, npts = [], 0
    for _ in range(args.steps):
        n, dt, sample = step()
        times.append(dt)
        npts += n
    total = sum(times)
    value = npts / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config(name),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{sample} per step, single-threaded FP64 C oracle"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def _config(name):
    if name == "genz256":
        from paper_1010_2107_gb300 import workloads as wl
        insts = wl.genz_batch(wl.GENZ256["count"], wl.GENZ256["seed"])
        return {"workload": name, "instances": len(insts), "ndim": "2..16", "nbins": wl.GENZ256["nbins"],
                "ncall_total": sum(i["ncall"] for i in insts), "integrand": "genz product/corner/oscillatory",
                "precision": wl.GENZ256["precision"], "ybits": wl.GENZ256["ybits"],
                "iterations": wl.GENZ256["itmx"], "l2": "flushed between steps (512 MiB write)"}
    w = _workload(name)
    c = {"workload": name, "ndim": w["ndim"], "nbins": w["nbins"], "ncall": w["ncall"],
         "integrand": {0: "genz_gaussian", 4: "double_gaussian", 5: "rambo_bw",
                       8: "u dbar -> W+ -> mu+ nu (stand-in densities)",
                       64: "double_gaussian as run-time compiled CUDA source"}[w["kind"]],
         "precision": w["precision"], "ybits": w["ybits"], "nstrat": w["nstrat"],
         "l2": "flushed between steps (512 MiB write)"}
    if w.get("mode") == "spring":
        c["iterations"] = (f"{w['ntrials']} SPRING trials per step on the frozen grid of a "
                           f"{w['itmx1']}+{w['itmx2']} BASES run")
    elif w.get("mode") == "bases":
        c["iterations"] = f"{w['itmx1']}+{w['itmx2']} (BASES)"
    elif w.get("mode") == "adjoint":
        c["iterations"] = f"one gradient pass on the grid of {w['warmup_iters']} refining iterations"
    else:
        c["iterations"] = w.get("itmx")
    return c


# ------------------------------------------------------------------------ ours


def _genz_ops(ins):
    """Algorithmic FP32-pipe operations per point of one Genz instance:
    Philox blocks, per-axis bin / map / integrand / histogram work, and the
    per-point sums."""
    d = ins["ndim"]
    # bins 6 + map 3 + histogram 2, plus the family's per-axis work
    # (product peak 3, corner peak and oscillatory 1)
    per_axis = {1: 14, 2: 12, 3: 12}.get(ins["kind"], 14)
    return ((d + 3) // 4) * 60 + per_axis * d + 20


class Runner:
    """One benchmarked workload: how to build it, run one step, time its
    dominant kernel and run one end-to-end step through the C ABI."""

    def __init__(self, name, gv, stream, rank, precision_override, autotune=True, launch=None):
        self.name, self.gv, self.stream, self.rank = name, gv, stream, rank
        self.autotune = autotune  # False: the library's default launch shape (profiling runs)
        self.fixed_launch = launch  # (threads, points per thread) to set instead of tuning
        self.tuned = None  # launch shape the autotuner chose for the benchmarked context
        if name == "genz256":
            from paper_1010_2107_gb300 import workloads as wl
            self.w = dict(wl.GENZ256)
            self.insts = wl.genz_batch(self.w["count"], self.w["seed"])
            for ins in self.insts:
                ins["instance"] = rank_instance(ins["instance"], rank, "batched")
            self.mode = "batched"
        else:
            self.w = _workload(name)
            self.mode = self.w.get("mode", "vegas")
        self.prec_name = precision_override or self.w["precision"]

    def precision(self, name=None):
        gv = self.gv
        return {"fp32": gv.FP32_ACCCOMP, "fp32_acc64": gv.FP32_ACC64, "fp64": gv.FP64}[name or self.prec_name]

    # ---------------------------------------------------------------- setup
    def make(self, prec):
        gv, w = self.gv, self.w
        if self.mode == "batched":
            h = gv.vegas_batch_create(self.insts, nbins=w["nbins"], seed=w["sample_seed"], precision=prec,
                                      ybits=w["ybits"], stream=self.stream)
            if self.fixed_launch:  # threads, points in flight per thread[, rounds per item]
                fl = self.fixed_launch
                gv.vegas_batch_set_launch(h, fl[0], fl[2] if len(fl) > 2 else 64)
                gv.vegas_batch_set_tile(h, fl[1])
            elif self.autotune:
                tuned = gv.vegas_batch_autotune(h)
                self.tuned = self.tuned or tuned
            return h
        kw = dict(nbins=w["nbins"], ncall=w["ncall"], nstrat=w["nstrat"], seed=w["seed"],
                  instance=rank_instance(0, self.rank, self.mode), precision=prec, ybits=w["ybits"],
                  stream=self.stream)
        if w.get("source"):
            h = gv.vegas_create_user(w["source"], w["ndim"], w["params"], **kw)
        else:
            h = gv.vegas_create(w["kind"], w["ndim"], w["params"], **kw)
        if self.mode == "adjoint":  # the grid the gradient is taken on
            gv.vegas_iterate(h, w["warmup_iters"], refine=True)
        elif self.mode == "spring":  # the BASES run whose integration phase bounds the cubes
            import numpy as np
            import torch
            n = w["ntrials"]  # pinned event buffers for the end-to-end steps, made once
            self._pinned = (torch.empty((n, w["ndim"]), dtype=torch.float64, pin_memory=True).numpy(),
                            torch.empty(n, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64))
            if self.autotune:
                tuned = gv.vegas_autotune(h)
                self.tuned = self.tuned or tuned
            gv.bases_integrate(h, w["itmx1"], 0.0, w["itmx2"], 0.0, result=False)
        elif self.fixed_launch:
            gv.vegas_set_launch(h, self.fixed_launch[0], 0)
            gv.vegas_set_tile(h, self.fixed_launch[1])
        elif self.autotune:
            tuned = gv.vegas_autotune(h)
            self.tuned = self.tuned or tuned
        return h

    @property
    def points_per_step(self):
        w = self.w
        if self.mode == "batched":
            return sum(i["ncall"] for i in self.insts) * w["itmx"]
        if self.mode == "bases":
            return w["ncall"] * (w["itmx1"] + w["itmx2"])
        if self.mode == "adjoint":
            return w["ncall"]
        if self.mode == "spring":
            return w["ntrials"]
        return w["ncall"] * w["itmx"]

    @property
    def launches_per_step(self):
        w = self.w
        # kernels of this library per step (memset nodes not counted):
        # batched: one reset, then per iteration the sampling kernels (FP32
        # form: one per dimension present; otherwise one) and k_batch_finalize;
        # BASES: grid reset (2), iteration set (1), control (2), then k_sample
        # + k_finish per pass; VEGAS: grid reset (2), window reset (1),
        # iteration set (1), control (1), then the passes; adjoint: k_grad +
        # k_colsum
        if self.mode == "batched":
            per_it = len({i["ndim"] for i in self.insts}) if self.prec_name == "fp32" else 1
            return 1 + (per_it + 1) * w["itmx"]
        if self.mode == "bases":
            return 2 + 1 + 2 + 2 * (w["itmx1"] + w["itmx2"])
        if self.mode == "adjoint":
            return 2
        if self.mode == "spring":  # cube table and guide (5 kernels), trials, compaction
            return 7
        return 2 + 1 + 1 + 1 + 2 * w["itmx"]

    def estimates(self, h):
        """The results the step produced, as (I, sigma) pairs: one per
        instance (batched), one for a VEGAS or BASES run; the adjoint's
        estimate and gradient components with sigma None."""
        gv = self.gv
        if self.mode == "batched":
            return [(r["I"], r["sigma"]) for r in gv.vegas_batch_iterate(h, 0)]
        if self.mode == "adjoint":
            g, I = gv.vegas_grad(h, 1000)
            return [(I, None)] + [(v, None) for v in g]
        if self.mode == "spring":
            return []
        r = gv.vegas_iterate(h, 0, refine=False)
        return [(r["I"], r["sigma"])]

    def step(self, h):
        gv, w = self.gv, self.w
        if self.mode == "batched":
            gv.vegas_batch_reset(h)
            gv.vegas_batch_iterate(h, w["itmx"], refine=True, result=False)
        elif self.mode == "bases":  # every step from iteration 0: the same points
            gv.vegas_reset_grid(h)
            gv.vegas_set_iteration(h, 0)
            gv.bases_integrate(h, w["itmx1"], 0.0, w["itmx2"], 0.0, result=False)
        elif self.mode == "adjoint":
            gv.vegas_grad(h, 1000)
        elif self.mode == "spring":
            gv.spring_generate(h, 0, w["ntrials"], events=False)
        else:
            gv.vegas_reset_grid(h)
            gv.vegas_reset_results(h)
            gv.vegas_set_iteration(h, 0)
            gv.vegas_iterate(h, w["itmx"], refine=True, result=False)

    def result(self, h):
        gv = self.gv
        if self.mode == "batched":
            res = gv.vegas_batch_iterate(h, 0)
            return {"instances": len(res), "max_chi2_dof": max(r["chi2_dof"] for r in res),
                    "nonfinite": sum(r["nonfinite"] for r in res)}
        if self.mode == "adjoint":
            g, I = gv.vegas_grad(h, 1000)
            return {"I": I, "dI_dM": g[0], "dI_dGamma": g[1], "dI_dT": g[2]}
        if self.mode == "spring":
            r = gv.spring_generate(h, 0, self.w["ntrials"], events=False)
            return {"events": r["n_events"], "acceptance": r["n_events"] / self.w["ntrials"],
                    "overflow": r["overflow"], "nonpos": r["nonpos"]}
        r = gv.vegas_iterate(h, 0, refine=False)
        return {"I": r["I"], "sigma": r["sigma"], "chi2_dof": r["chi2_dof"], "nonfinite": r["nonfinite"]}

    # --------------------------------------------------- kernel-level timing
    def kernel_ms(self, h):
        """(dominant kernel name, ms per launch, points per launch, other timings)."""
        gv = self.gv
        if self.mode == "batched":
            p = gv.vegas_batch_profile(h, 5)
            name = ("k_batch_dim (one kernel per dimension, concurrent)" if self.prec_name == "fp32"
                    else "k_batch_sample")
            return name, p["sample"], sum(i["ncall"] for i in self.insts), {"finalize_ms": p["finalize"]}
        if self.mode == "adjoint":
            import torch
            gv.vegas_grad(h, 1000)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(self.stream)
            for _ in range(5):
                gv.vegas_grad(h, 1000)
            b.record(self.stream)
            torch.cuda.synchronize()
            return "k_grad", a.elapsed_time(b) / 5, self.w["ncall"], {}
        if self.mode == "spring":
            return "k_spring", gv.spring_profile(h, self.w["ntrials"], 5), self.w["ntrials"], {}
        p = gv.vegas_profile_pass(h, 20)
        other = {"finish_ms": p["finish"]}
        if self.mode == "bases":
            # the step's mix: ITMX1 refining passes with the per-bin histogram,
            # ITMX2 frozen-grid passes without it
            q = gv.vegas_profile_frozen_pass(h, 20)
            n1, n2 = self.w["itmx1"], self.w["itmx2"]
            ops = ALGO_OPS.get(self.name, {})
            on, off = sum(ops.values()), sum(v for k, v in ops.items() if k != "histogram")
            other["launch_kinds"] = [
                {"kind": "refining pass", "launches_per_step": n1, "ms_per_launch": p["sample"], "ops_per_point": on},
                {"kind": "frozen-grid pass", "launches_per_step": n2, "ms_per_launch": q["sample"],
                 "ops_per_point": off}]
            other["finish_ms_frozen"] = q["finish"]
            return "k_sample", (n1 * p["sample"] + n2 * q["sample"]) / (n1 + n2), self.w["ncall"], other
        return "k_sample", p["sample"], self.w["ncall"], other

    def ops_per_point(self):
        if self.mode == "batched":
            tot = sum(i["ncall"] for i in self.insts)
            return sum(_genz_ops(i) * i["ncall"] for i in self.insts) / tot
        ops = ALGO_OPS.get(self.name)
        if not ops:
            return None
        if self.mode == "bases":  # launch-weighted over the step's refining and frozen-grid passes
            n1, n2 = self.w["itmx1"], self.w["itmx2"]
            on, off = sum(ops.values()), sum(v for k, v in ops.items() if k != "histogram")
            return (n1 * on + n2 * off) / (n1 + n2)
        return sum(ops.values())

    def launch(self, h):
        gv = self.gv
        if self.mode == "batched":
            return dict(gv.vegas_batch_get_launch(h), **gv.vegas_batch_get_tile(h))
        return dict(gv.vegas_get_launch(h), **gv.vegas_get_tile(h))

    # ------------------------------------------------------------ end to end
    def e2e_step(self, h):
        """One step through the public API with host buffers: inputs uploaded
        from host memory, the result read back; returns (h2d, d2h) bytes."""
        import numpy as np
        gv, w = self.gv, self.w
        if self.mode == "batched":
            # every instance's parameter block from host memory (the library
            # derives the integrand constants and uploads them, 120 doubles
            # per instance), then the run from uniform grids
            if getattr(self, "_param_rows", None) is None:
                width = max(len(i["params"]) for i in self.insts)
                self._param_rows = np.zeros((len(self.insts), width))
                for j, ins in enumerate(self.insts):
                    self._param_rows[j, :len(ins["params"])] = ins["params"]
            gv.vegas_batch_set_params(h, self._param_rows)
            gv.vegas_batch_reset(h)
            gv.vegas_batch_iterate(h, w["itmx"], refine=True, result=True)
            return 8 * (3 * 32 + 24) * len(self.insts), 48 * len(self.insts) + 1200 * len(self.insts)
        d, N = w["ndim"], w["nbins"]
        if self.mode == "spring":  # events copied to pinned host memory; the frozen grid stays
            r = gv.spring_generate(h, 0, w["ntrials"], events=True, out_x=self._pinned[0], out_t=self._pinned[1])
            return 0, r["n_events"] * (8 * d + 8)
        edges0 = np.tile(np.arange(N + 1, dtype=np.float64) / N, (d, 1))
        gv.vegas_set_grid(h, edges0)
        gv.vegas_set_params(h, np.asarray(w["params"], dtype=np.float64))
        h2d = edges0.nbytes + 8 * (3 * 32 + 24)
        if self.mode in ("bases", "vegas"):
            gv.vegas_set_iteration(h, 0)
        if self.mode == "bases":
            gv.bases_integrate(h, w["itmx1"], 0.0, w["itmx2"], 0.0)
            return h2d, 160
        if self.mode == "adjoint":
            gv.vegas_grad(h, 1000)
            return h2d, 8 * 5
        gv.vegas_reset_results(h)
        gv.vegas_iterate(h, w["itmx"], refine=True)
        return h2d, 160

    def close(self, h):
        h.close()


def timed_steps(R, h, k, warm, flush, stream, dist=None):
    """W untimed steps, then k steps each timed by CUDA events on the
    library's stream, L2 flushed before each; barriers around (ranks)."""
    import torch
    for _ in range(warm):
        R.step(h)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
    for a, b in evs:
        flush.zero_()
        a.record(stream)
        R.step(h)
        b.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    return [a.elapsed_time(b) for a, b in evs]


def roofline_of(R, h, peaks, peak_src, sms, workload):
    """The roofline object of the dominant kernel (ALU-bound: algorithmic
    operations per point x points per launch / its CUDA-event time, against
    the FP32 lane-issue peak) and the other kernel timings."""
    gv = R.gv
    kname, kms, units, other = R.kernel_ms(h)
    ops_pt = R.ops_per_point()
    if not ops_pt:
        return None, other
    achieved = ops_pt * units / (kms * 1e-3) / 1e12
    mhz = peaks.get("sm_max_mhz", 2070.0)
    peak = sms * 128 * mhz * 1e6 / 1e12
    traffic = TRAFFIC.get(workload)
    if traffic is not None and R.mode == "bases":  # launch-weighted like the time
        traffic = (R.w["itmx1"] * traffic[0] + R.w["itmx2"] * traffic[1]) / (R.w["itmx1"] + R.w["itmx2"])
    elif traffic is not None:
        traffic = traffic[0]
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": kname, "ops_per_point": round(ops_pt, 1),
            "points_per_launch": units, "ms_per_launch": kms,
            "peak_basis": f"{sms} SMs x 128 FP32 lanes x {mhz:.0f} MHz ({peak_src} max clock)"}
    if R.precision() == gv.FP64:
        roof["note"] = "FP64 form: bound by the FP64 pipe, see fp64_rate"
    if "launch_kinds" in other:
        roof["launch_kinds"] = other["launch_kinds"]
    return roof, other


def fp64_leg(R, h, flush, stream, rate32, steps):
    """The plain FP64 GPU path of the same workload on the same points
    (24-bit words, the same Philox iterations and, for the adjoint, the same
    grid): its rate, the speed-up, and the largest difference of the two
    forms' estimates in units of the FP64 sigma (relative for the adjoint)."""
    gv = R.gv
    h64 = R.make(gv.FP64)
    if R.mode == "adjoint":
        gv.vegas_set_grid(h64, gv.vegas_get_grid(h))
    ms64 = timed_steps(R, h64, steps, 2, flush, stream)
    e32, e64 = R.estimates(h), R.estimates(h64)
    out = {"value": R.points_per_step * steps / (sum(ms64) / 1e3), "unit": UNIT, "steps": steps,
           "same_points": True, "result": R.result(h64)}
    out["speedup"] = rate32 / out["value"]
    sig = [abs(a[0] - b[0]) / b[1] for a, b in zip(e32, e64) if b[1]]
    rel = [abs(a[0] - b[0]) / abs(b[0]) for a, b in zip(e32, e64) if b[0]]
    out["max_dI_over_sigma"] = max(sig) if sig else None
    out["max_rel_dI"] = max(rel) if rel else None
    if R.mode in ("bases", "vegas"):
        # Each form refines its own grid from its own per-bin sums, and for
        # integrands with cuts refinement amplifies the FP32 rounding from
        # iteration to iteration (a point that crosses a cut edge moves its
        # bins' sums by its whole weight), so after the first refinement the
        # two runs place their points differently.  The comparison on the
        # same points is therefore made in lockstep: every iteration of the
        # FP32 run is evaluated again by the FP64 form on the grid that
        # iteration used, with the same Philox iteration.
        brief = lambda r: {k: r[k] for k in ("I", "sigma", "chi2_dof") if k in r}
        out["independent_runs"] = {"max_dI_over_sigma": out["max_dI_over_sigma"], "max_rel_dI": out["max_rel_dI"],
                                   "fp32": brief(R.result(h)), "fp64": brief(out["result"]),
                                   "note": "each form refining its own grid; for heavy-tailed weights the "
                                           "iterations' sigmas are unreliable (chi2/dof well above 1), so two "
                                           "refinement histories can end many nominal sigmas apart"}
        out.update(lockstep(R, h, h64))
    R.close(h64)
    return out


def lockstep(R, h, h64):
    """The FP32 run's iterations, each evaluated again by the FP64 form on
    the same grid and Philox iteration: the largest per-iteration
    difference of the estimates in FP64 sigmas and relative."""
    gv, w = R.gv, R.w
    n_ref, n_all = (w["itmx1"], w["itmx1"] + w["itmx2"]) if R.mode == "bases" else (w["itmx"], w["itmx"])
    gv.vegas_reset_grid(h)
    gv.vegas_reset_results(h)
    gv.vegas_set_iteration(h, 0)
    sig, rel = [], []
    for i in range(n_all):
        grid = gv.vegas_get_grid(h)
        gv.vegas_iterate(h, 1, refine=i < n_ref, result=False)
        I32, _ = gv.vegas_get_history(h)[-1]
        gv.vegas_set_grid(h64, grid)
        I64, v64 = gv.vegas_eval(h64, i)
        if v64 > 0:
            sig.append(abs(I32 - I64) / v64 ** 0.5)
        if I64:
            rel.append(abs(I32 - I64) / abs(I64))
    return {"max_dI_over_sigma": max(sig) if sig else None, "max_rel_dI": max(rel) if rel else None,
            "same_points": "lockstep: each FP32 iteration's grid and Philox iteration, evaluated by both forms",
            "iterations": n_all}


EXTRA_WORKLOADS = ("dgauss8", "rambo5", "rambo4_adjoint")


def extra_line(name, gv, stream, flush, peaks, peak_src, sms, steps=10):
    """Value, roofline fraction and FP64 speed-up of one more workload,
    timed in the same run as the headline one."""
    R = Runner(name, gv, stream, 0, None)
    h = R.make(R.precision())
    ms = timed_steps(R, h, steps, 3, flush, stream)
    value = R.points_per_step * steps / (sum(ms) / 1e3)
    roof, _ = roofline_of(R, h, peaks, peak_src, sms, name)
    line = {"value": value, "unit": UNIT, "ms_per_step": sum(ms) / steps, "steps": steps,
            "roofline_frac": roof["frac"] if roof else None, "dominant_kernel": roof["kernel"] if roof else None,
            "kernel_ms_per_launch": roof["ms_per_launch"] if roof else None,
            "launch": R.launch(h), "autotuned": R.tuned}
    f = fp64_leg(R, h, flush, stream, value, 3)
    line["fp64"] = {k: f[k] for k in ("value", "speedup", "max_dI_over_sigma", "max_rel_dI", "same_points",
                                      "independent_runs") if k in f}
    line["result"] = R.result(h)
    R.close(h)
    return line


def run_ours(args):
    import torch

    from paper_1010_2107_gb300 import _build
    from paper_1010_2107_gb300 import gvegas as gv

    rank, world, local, dist = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the library has no CPU path)")
    torch.cuda.set_device(local)
    _build.build()
    # A dedicated stream: the library orders its work on it and the events
    # below are recorded on it (torch's default stream has handle 0, which
    # the library would replace by a stream of its own).
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    launch = tuple(int(v) for v in args.launch.split(",")) if args.launch else None
    R = Runner(args.workload, gv, stream, rank, args.precision, autotune=not args.no_autotune, launch=launch)
    prec = R.precision()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    h = R.make(prec)
    with ClockSampler(local) as clk:
        step_ms = timed_steps(R, h, args.steps, args.warmup, flush, stream, dist)
    total_ms = max_over_ranks(sum(step_ms), dist)
    pps = R.points_per_step
    value = whole_job_rate(world, pps, args.steps, total_ms / 1e3)
    res = R.result(h)

    # roofline of the dominant kernel, timed by CUDA events on its stream
    peaks, peak_src = _measured_peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    roof, other = roofline_of(R, h, peaks, peak_src, sms, args.workload)
    extra = dict(other)
    if R.mode in ("bases", "vegas"):
        launch = gv.vegas_get_launch(h)
        d, N = R.w["ndim"], R.w["nbins"]
        red_bytes = 8 * (2 * d * N + 5) * launch["ctas"] + 8 * (2 * d * N + 5)
        extra = {"reduction": {"kernel": "k_finish", "bytes_per_launch": red_bytes,
                               "ms_per_launch": other["finish_ms"],
                               "achieved_gbs": red_bytes / (other["finish_ms"] * 1e-3) / 1e9,
                               "peak_gbs": peaks.get("hbm_gbs"),
                               "note": "launch latency included; the partials are read from L2"}}

    # the plain FP64 GPU path on the same points (speed-up denominator)
    fp64 = None
    if not args.no_fp64 and prec != gv.FP64:
        fp64 = fp64_leg(R, h, flush, stream, value / world, max(3, args.steps // 4))

    # end to end through the C ABI with host buffers
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ke = max(3, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(ke):
        h2d, d2h = R.e2e_step(h)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist)
    e2e = {"value": whole_job_rate(world, pps, ke, e2e_s), "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "steps": ke}

    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu and R.mode == "spring":
        rate, n, dt = oracle_spring_rate(R, h)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{n} SPRING trials on the same frozen grid and cube maxima, {dt:.1f} s "
                         "single-threaded FP64 C oracle"}
    if rank == 0 and world == 1 and not args.no_cpu and R.mode == "batched":
        rate, n, dt, k = oracle_rate_batched()
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{n} points: one iteration of each of the first {k} instances of the batch on their "
                         f"uniform grids, {dt:.1f} s single-threaded FP64 C oracle"}
        try:
            rate_p, n_p, dt_p, P = oracle_rate_batched_allcores()
            cpu_all = {"value": rate_p, "unit": UNIT, "cores": P, "kind": "oracle, one process per core",
                       "sample": f"{n_p} points: each of {P} processes one iteration of its own instances "
                                 f"(every {P}th, about 2^21 points), slowest {dt_p:.1f} s"}
        except Exception as e:  # the single-threaded line above stands on its own
            cpu_all = {"unavailable": f"{type(e).__name__}: {e}"}
    if rank == 0 and world == 1 and not args.no_cpu and R.mode in ("bases", "vegas"):
        bases = R.mode == "bases"
        rate, n, dt = oracle_rate(args.workload, 3, 3) if bases else oracle_rate(args.workload, 1, 0)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{n} points: full-NCALL iterations of the same workload "
                         f"({'3+3 BASES' if bases else '1 VEGAS'}), {dt:.1f} s single-threaded FP64 C oracle"}
        try:
            rate_p, n_p, dt_p, P = oracle_rate_allcores(args.workload)
            cpu_all = {"value": rate_p, "unit": UNIT, "cores": P, "kind": "oracle, one process per core",
                       "sample": f"{n_p} points: one full-NCALL iteration in each of {P} processes on "
                                 f"disjoint counter ranges, slowest {dt_p:.1f} s"}
        except Exception as e:  # the single-threaded line above stands on its own
            cpu_all = {"unavailable": f"{type(e).__name__}: {e}"}

    # more workloads in the same run (one GPU)
    workloads = None
    if world == 1 and not args.no_extras and args.workload == "genz256":
        workloads = {}
        for name in EXTRA_WORKLOADS:
            try:
                workloads[name] = extra_line(name, gv, stream, flush, peaks, peak_src, sms)
            except Exception as e:  # one failing extra does not hide the headline
                workloads[name] = {"error": f"{type(e).__name__}: {e}"}

    clocks = clk.summary()
    if rank == 0:
        accumulation = {"fp32": "fp32_compensated", "fp32_acc64": "fp32_values_fp64_sums",
                        "fp64": "fp64"}[R.prec_name]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec != gv.FP64 else "f64",
            "data": "synthetic", "config": dict(_config(args.workload), accumulation=accumulation,
                                                launch=R.launch(h)),
            "roofline": roof, **extra, "fp64_path": fp64, "cpu_baseline": cpu,
            "cpu_baseline_allcores": cpu_all,
            "e2e": e2e, "gpu_launches": R.launches_per_step * args.steps, "clocks": clocks,
            "result": res,
            "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms)},
        }
        if workloads is not None:
            line["workloads"] = workloads
        if R.tuned:
            line["config"]["autotuned"] = R.tuned
        print(json.dumps(line))
    R.close(h)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_microbench():
    import torch

    from paper_1010_2107_gb300 import _build
    from paper_1010_2107_gb300 import gvegas as gv
    _build.build()
    props = torch.cuda.get_device_properties(0)
    out = {"device": props.name, "sms": props.multi_processor_count, "unit": "thread-ops/s"}
    for op, name in gv.MICROBENCH_OPS.items():
        out[name] = gv.vegas_microbench(op)
    per_sm_clk = {}
    with ClockSampler(0) as clk:
        for op, name in gv.MICROBENCH_OPS.items():
            gv.vegas_microbench(op)
    c = clk.summary()
    mhz = c.get("sm_mhz") or 2070.0
    for op, name in gv.MICROBENCH_OPS.items():
        per_sm_clk[name] = out[name] / (props.multi_processor_count * mhz * 1e6)
    out["per_sm_per_clock"] = per_sm_clk
    out["clocks"] = c
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="genz256",
                    choices=["dgauss8", "gauss4", "rambo5", "rambo4_adjoint", "genz256", "spring_dgauss8",
                             "user_dgauss8", "wmunu"])
    ap.add_argument("--precision", default=None, choices=[None, "fp32", "fp32_acc64", "fp64"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="time only the chosen workload (the default genz256 run also times dgauss8, rambo5 and "
                         "rambo4_adjoint)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shape (profiler runs, where the autotuner's timings are skewed)")
    ap.add_argument("--launch", default=None, metavar="THREADS,PPT[,ROUNDS]",
                    help="set this launch shape instead of tuning (profiler runs of a tuned shape); ROUNDS "
                         "(rounds per work item, default 64) applies to genz256")
    ap.add_argument("--microbench", action="store_true",
                    help="print the measured instruction-class rates (ALU roofline denominators)")
    args = ap.parse_args()
    if args.microbench:
        return run_microbench()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
