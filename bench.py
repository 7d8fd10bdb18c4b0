#!/usr/bin/env python
"""Throughput of the fused D2V16 MRT-FD step on GB300.

Headline workload: the shock-bubble interaction of Sec. V.C on a 2048 x 1024
grid (dx = dy = 1e-3, dt = 1e-5): a Mach-1.22 planar shock (gamma = 2
post-shock state (1.28, -0.3774, 0, p = 1.6512) held on the right) running
into a light circular bubble (rho = 0.1358, p = 1, radius 128 nodes) in gas
at rest, reflecting top and bottom, linear extrapolation on the left. One
benchmark step is one time step of the whole hot path over the grid (boundary
ghosts, moments, Eq. 14 equilibria, relaxation, back-map, Lax-Wendroff update
of Eq. A.1, watchdog and, every ``--audit-every`` steps, the conservation
audit), in the paper's arithmetic: FP64.

Timing: the K timed steps follow W warm-up steps and are bracketed by CUDA
events on the launching stream, with a barrier and a device synchronisation
on both sides; the job's time is the maximum over ranks. Each FP64
population buffer is 268 MB, twice the 129 MB L2, so consecutive steps do
not find their inputs in L2 (no flush is needed). The FP64 step is bound by
the FP64 units, not by memory: its roofline is arithmetic ("alu"), against
the FP64 fused multiply-add rate measured in this run
(include/lbm_probe.h), with the HBM fraction beside it.

Lines printed (rank 0): one JSON object. Besides the contract keys:
``df64_large_grid`` is the double-word step (FP32 pairs, ~48-bit
arithmetic on the FP32 units), ``fp32_large_grid``,
``fp32_dwmom_large_grid`` (double-word conserved moments and equilibria),
``tensor_core_tf32x3`` and ``fp32_two_steps_per_launch`` the FP32 steps, all on the same grid
(64-step CUDA-graph replays back to back) with their errors against an FP64
GPU run; ``reflection_600x200`` the 600 x 200 regular shock reflection
(Sec. V.B.a geometry) in FP64 and FP32, each step timed alone with the L2
flushed before it, and as a long run (graph replays, L2-resident);
``tubes`` the batch of 4096 quasi-1D Riemann problems (stable and unstable
tubes counted apart); ``von_neumann`` a stability map of Sec. IV's example;
``corrector`` the wall time of the learned coarse-grid corrector's use
against the fine run it stands in for;
``peaks`` the measured FMA rates; ``cpu_baseline`` the FP64 numpy oracle on
the host cores (all cores, and one) over a bounded sample of the headline
workload; ``e2e`` the headline step through the C ABI with host buffers;
``clocks`` nvidia-smi samples around the headline's timed region.

``--impl reference`` times the CPU oracle instead (the only reference
implementation this method has) on the same workload, on all host cores,
rank 0 only.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

if "--cpu-sample" in sys.argv or "--cpu-sample-tubes" in sys.argv:
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"

import numpy as np  # noqa: E402

METRIC = ("D2V16 MRT cell-updates/s at stated error vs FP64 oracle; "
          "% of HBM roofline")
UNIT = "cell-updates/s"
# Algorithmic traffic per cell-update: 16 populations read once and written once.
BYTES_PER_CELL = {"fp64": 256, "fp32": 128}
# Algorithmic FP64 operations per cell-update of the factorised step (FMA = 2):
# transform 28, conserved moments 24, equilibria 40, deviations 77,
# back-map 64, inverse transform 28, Lax-Wendroff update 128.
FLOPS_PER_CELL = 389
# FP64-pipe instructions per node update of k_step<double>, counted by ncu
# (sm__inst_executed_pipe_fp64, profiles/k_step_f64_bubble_2048x1024.md):
# the FP64 units retire one instruction per lane slot whether it is an add,
# a multiply or a fused multiply-add, so this count over the measured FMA
# rate is the step's time on those units.
FP64_INSTR_PER_CELL = 265
L2_FLUSH_BYTES = 256 << 20


class L2Flush:
    """Evicts the L2: writes one buffer larger than L2, then reads another
    (the read leaves clean lines, so the next kernel pays no write-back)."""

    def __init__(self, torch):
        n = L2_FLUSH_BYTES // 4
        self.w = torch.empty(n, dtype=torch.float32, device="cuda")
        self.r = torch.zeros(n, dtype=torch.float32, device="cuda")

    def __call__(self):
        self.w.zero_()
        self.r.sum()


def workload():
    import workloads as W
    return W.shock_bubble()


def config_json(w):
    """The workload, the same in both arms' lines; how an arm computes it is
    in the line's ``path``."""
    return {"workload": "shock_bubble_%dx%d" % (w.nx, w.ny),
            "nx": w.nx, "ny": w.ny, "dx": w.dx, "dt": w.dt, "shock_mach": 1.22,
            "bubble_rho": 0.1358, "bubble_radius_nodes": 128,
            "l2": "inputs larger than L2: 268 MB per FP64 population buffer (L2 129 MB), "
                  "no flush"}


# ----------------------------------------------------------------------------
# CPU oracle timing
# ----------------------------------------------------------------------------
def slab_workload(k, nslabs):
    """Rows [k h, (k+1) h) of the headline grid (h = ny / nslabs, the last
    slab taking the remainder) as a grid of its own with the full grid's
    sides (reflecting top and bottom): one host core's share of a sample."""
    import workloads as W
    w = workload()
    h = w.ny // nslabs
    y0, y1 = k * h, (w.ny if k == nslabs - 1 else (k + 1) * h)
    f = [np.ascontiguousarray(a[y0:y1]) for a in w.fields()]
    return W.Workload(w.name + "_slab", w.nx, y1 - y0, w.dx, w.dy, w.dt, w.s, w.bc, *f)


def oracle_steps(k, nslabs, seconds=None, steps=None, warmup=0):
    """Times oracle steps of slab k of nslabs; returns (cells, steps, seconds)."""
    from oracle import scheme
    w = slab_workload(k, nslabs)
    f = scheme.init_populations(*w.fields())
    cfg = w.cfg()
    for _ in range(max(1, warmup)):   # the first step also builds the oracle's matrices
        f = scheme.step(f, cfg)
    n, t0 = 0, time.perf_counter()
    while True:
        f = scheme.step(f, cfg)
        n += 1
        el = time.perf_counter() - t0
        if (steps is not None and n >= steps) or (seconds is not None and el >= seconds):
            return w.nx * w.ny, n, el


def _run_slabs(nslabs, seconds=None, steps=None, warmup=1):
    """Runs oracle_steps on nslabs host processes at once (fresh
    single-threaded interpreters, started by fork + exec: no GPU state is
    inherited); returns the list of (cells, steps, seconds)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    args = []
    if seconds is not None:
        args += ["--cpu-seconds", str(seconds)]
    if steps is not None:
        args += ["--steps", str(steps)]
    procs = [subprocess.Popen([sys.executable, os.path.abspath(__file__), "--cpu-sample", str(k),
                               str(nslabs), "--warmup", str(warmup)] + args,
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)
             for k in range(nslabs)]
    out = []
    for p in procs:
        so, se = p.communicate(timeout=900)
        if p.returncode != 0:
            raise RuntimeError("oracle sample failed: " + se[-300:])
        out.append(tuple(json.loads(so.strip().splitlines()[-1])))
    return out


def cpu_baseline(seconds):
    """The FP64 numpy oracle on the host: one process per core, each
    stepping one horizontal slab of the headline grid for about ``seconds``
    (aggregate rate), and one process stepping the whole grid (one core)."""
    cores = os.cpu_count() or 1
    try:
        res = _run_slabs(cores, seconds=seconds)
        value = sum(c * n / el for c, n, el in res)
        one = _run_slabs(1, seconds=seconds)[0]
    except (RuntimeError, subprocess.TimeoutExpired, ValueError) as e:
        return {"value": None, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": "failed: %s" % e}
    w = workload()
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d host processes, one per core, each stepping one %d-row slab of the "
                      "%dx%d grid as a grid of its own (FP64 numpy oracle, %.0f s each, %d to %d "
                      "steps per slab)" % (cores, w.ny // cores, w.nx, w.ny, seconds,
                                           min(n for _, n, _ in res), max(n for _, n, _ in res)),
            "single_core": {"value": one[0] * one[1] / one[2], "cores": 1,
                            "sample": "%d steps of the whole %dx%d grid, one process (%.1f s)"
                                      % (one[1], w.nx, w.ny, one[2])}}


def oracle_tube_steps(seconds):
    """Times oracle steps of a seeded 64-tube subset of the tube batch (each
    tube a one-node-deep grid, stepped in turn); returns (node-updates,
    seconds)."""
    import workloads
    from oracle import scheme
    B = workloads.tube_batch()
    pick = np.random.default_rng(64).choice(len(B["nx"]), 64, replace=False)
    tubes = []
    for t in pick:
        n = int(B["nx"][t])
        x = (np.arange(n) + 0.5) / n
        fields = [np.where(x <= 0.5, B["left"][t, q], B["right"][t, q])[None, :] for q in range(4)]
        bc = (("eq", tuple(B["left"][t])), ("eq", tuple(B["right"][t])),
              ("periodic", None), ("periodic", None))
        w = workloads.Workload("tube", n, 1, B["dx"][t], B["dx"][t], B["dt"], tuple(B["s"][t]), bc,
                               *fields)
        tubes.append([scheme.init_populations(*w.fields()), w.cfg(), n])
    updates, t0 = 0, time.perf_counter()
    while True:
        for tb in tubes:
            tb[0] = scheme.step(tb[0], tb[1])
            updates += tb[2]
        el = time.perf_counter() - t0
        if el >= seconds:
            return updates, el


def tubes_cpu_baseline(seconds):
    """oracle_tube_steps in a fresh single-threaded process."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    res = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample-tubes",
                          str(seconds)], capture_output=True, text=True, timeout=600, env=env)
    if res.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": "failed: " + res.stderr[-200:]}
    n, el = json.loads(res.stdout.strip().splitlines()[-1])
    return {"value": n / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d node-updates of a seeded 64-tube subset, FP64 numpy oracle (%.1f s, 1 thread)"
                      % (n, el)}


# ----------------------------------------------------------------------------
# GPU measurement
# ----------------------------------------------------------------------------
class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi every 100 ms from
    a reader thread that stamps each sample with the host clock, so that the
    samples taken inside a timed region can be picked out afterwards."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, device_uuid=None):
        import threading
        cmd = ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits", "-lms", "100"]
        if device_uuid:
            cmd += ["-i", device_uuid]
        self.samples = []          # (host time, sm MHz, max MHz, reasons)
        try:
            self.p = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()
        t0 = time.perf_counter()
        while not self.samples and time.perf_counter() - t0 < 5.0:   # running before timing starts
            time.sleep(0.02)

    def _read(self):
        for line in self.p.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm, mx = float(parts[1]), float(parts[2])
            except ValueError:
                continue
            reasons = {n for n, v in zip(self.NAMES, parts[5:9]) if v.lower() == "active"}
            self.samples.append((time.perf_counter(), sm, mx, reasons))

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            self.t.join(timeout=5)

    def summary(self, t0=None, t1=None):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sel = [x for x in self.samples if (t0 is None or x[0] >= t0) and (t1 is None or x[0] <= t1)]
        return {"sm_mhz": statistics.median(x[1] for x in sel) if sel else None,
                "sm_max_mhz": sel[-1][2] if sel else None, "samples": len(sel),
                "reasons": sorted(set().union(*[x[3] for x in sel])) if sel else []}


def device_uuid(torch):
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
    except Exception:
        return None


def max_over_ranks(dist, values, device):
    """Element-wise maximum of ``values`` (floats) over all ranks of the
    process group (``dist`` None: one process, the values themselves). The
    slowest rank's time is the job's time."""
    if dist is None:
        return list(values)
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def whole_job_rate(world, units_per_rank, seconds):
    """Units processed by all ranks (each rank the same work: weak scaling,
    independent replicas) per second of the slowest rank."""
    return world * units_per_rank / seconds


def time_steps(torch, lbm, ctx, stream, flush, K, W, per=1):
    """Per-step CUDA-event times (ms) of K steps after W warm-up steps, timed
    in iterations of `per` steps (one lbm_step call each; the L2 is flushed
    between iterations). Each iteration's time is listed once per step it
    advanced, divided by `per`."""
    with torch.cuda.stream(stream):
        for _ in range(W):
            lbm.lbm_step(ctx, per)
            flush()
        stream.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(K // per)]
        torch.cuda._sleep(200_000_000)   # keep the GPU busy while the loop is enqueued
        for a, b in ev:
            a.record(stream)
            lbm.lbm_step(ctx, per)
            b.record(stream)
            flush()
        stream.synchronize()
    return [a.elapsed_time(b) / per for a, b in ev for _ in range(per)]


def time_graph_steps(torch, lbm, ctx, stream, n, reps):
    """Mean ms per step of `reps` timed calls of lbm_step(ctx, n) (n a
    multiple of 64: CUDA-graph replays back to back), after one warm-up call.
    Consecutive steps are not flushed: a grid smaller than L2 stays there."""
    with torch.cuda.stream(stream):
        lbm.lbm_step(ctx, n)
        stream.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(reps)]
        for a, b in ev:
            a.record(stream)
            lbm.lbm_step(ctx, n)
            b.record(stream)
        stream.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / (reps * n)


def field_error(lbm, ctx, ref):
    """Relative L-infinity error per field of ctx's moments against `ref`
    (rho and T relative to their maxima, u and v to the maximum speed)."""
    m = [np.empty_like(ref[0]) for _ in range(4)]
    lbm.lbm_moments(ctx, *m)
    speed = np.sqrt(ref[1] ** 2 + ref[2] ** 2).max()
    return {"rho": float(np.abs(m[0] - ref[0]).max() / np.abs(ref[0]).max()),
            "u": float(np.abs(m[1] - ref[1]).max() / speed),
            "v": float(np.abs(m[2] - ref[2]).max() / speed),
            "T": float(np.abs(m[3] - ref[3]).max() / np.abs(ref[3]).max())}


def make_ctx(lbm, w, precision, audit_every, stream, tune=True):
    cfg = lbm.make_config(w.nx, w.ny, w.dx, w.dy, w.dt, w.s, w.bc, precision, audit_every)
    ctx = lbm.lbm_create(cfg, stream)
    lbm.lbm_set_init(ctx, *[np.ascontiguousarray(a) for a in w.fields()])
    if tune:
        lbm.lbm_autotune(ctx, 20)
    return ctx


def large_grid_measure(torch, lbm, stream, audit_every, hbm_peak):
    """The reduced-precision steps on the headline grid (268 MB of FP32
    traffic per step, larger than L2): FP32, tensor-core (3xTF32) and
    two-steps-per-launch FP32 steps timed as back-to-back graph replays, each
    compared with an FP64 GPU run after the same number of steps."""
    wl = workload()
    cl = wl.nx * wl.ny
    out = {}
    nsteps = 256
    c64 = make_ctx(lbm, wl, "fp64", 0, stream, tune=False)   # reference run: shape irrelevant
    lbm.lbm_step(c64, nsteps)
    ref = [np.empty((wl.ny, wl.nx)) for _ in range(4)]
    lbm.lbm_moments(c64, *ref)
    lbm.lbm_destroy(c64)
    for prec, key, fused in (("df64", "df64_large_grid", False),
                             ("fp32", "fp32_large_grid", False),
                             ("fp32_dwmom", "fp32_dwmom_large_grid", False),
                             ("tc_tf32x3", "tensor_core_tf32x3", False),
                             ("fp32", "fp32_two_steps_per_launch", True)):
        ctx = make_ctx(lbm, wl, prec, 0, stream, tune=False)   # the error run
        try:
            if fused:
                lbm.lbm_set_fused_steps(ctx, 2)
            lbm.lbm_step(ctx, nsteps)
            err = field_error(lbm, ctx, ref)
            st = lbm.lbm_status(ctx)
            ctx2 = make_ctx(lbm, wl, prec, audit_every, stream, tune=not fused)
            try:
                if fused:
                    lbm.lbm_set_fused_steps(ctx2, 2)
                ms = time_graph_steps(torch, lbm, ctx2, stream, 64, 10)
                blocks = lbm.lbm_step_blocks(ctx2)
            finally:
                lbm.lbm_destroy(ctx2)
            ms_na = None
            if audit_every > 0 and prec in ("fp32", "tc_tf32x3") and not fused:
                ctx3 = make_ctx(lbm, wl, prec, 0, stream, tune=not fused)   # the same step, no audits
                try:
                    ms_na = time_graph_steps(torch, lbm, ctx3, stream, 64, 10)
                finally:
                    lbm.lbm_destroy(ctx3)
        finally:
            lbm.lbm_destroy(ctx)
        gbs = BYTES_PER_CELL["fp64" if prec == "df64" else "fp32"] * cl / (ms * 1e-3) / 1e9
        out[key] = {"workload": "shock_bubble_%dx%d" % (wl.nx, wl.ny), "value": cl / (ms * 1e-3),
                    "unit": UNIT, "ms_per_step": ms, "achieved_gbs": gbs,
                    "frac_of_hbm": gbs / hbm_peak, "step_blocks": blocks,
                    "timing": "64-step CUDA-graph replays back to back (inputs larger than L2)",
                    "error_vs_fp64_gpu_after_%d_steps" % nsteps: err, "status": list(st),
                    "audit_every": audit_every}
        if ms_na is not None:
            out[key]["ms_per_step_no_audit"] = ms_na
            out[key]["frac_of_hbm_no_audit"] = (BYTES_PER_CELL["fp32"] * cl / (ms_na * 1e-3) / 1e9
                                                / hbm_peak)
        if prec == "fp32_dwmom":
            out[key]["note"] = ("FP32 step with the conserved moments, Eq. 14 equilibria and "
                                "temperature in double-word arithmetic (LBM_FP32_DWMOM)")
        if prec == "df64":
            out[key]["dtype"] = "f32 double-word (h + l)"
            out[key]["fp64_equivalent_tflops"] = FLOPS_PER_CELL * cl / (ms * 1e-3) / 1e12
            out[key]["note"] = ("populations as FP32 pairs (8 B), every step operation in "
                                "double-word arithmetic on the FP32 units; 256 B per node-update")
        if fused:
            out[key]["note"] = ("two time steps per launch (temporal blocking): the populations "
                                "cross HBM once per two steps, so achieved_gbs counts the "
                                "single-step algorithmic 128 B per node-update")
    return out


def reflection_measure(torch, lbm, stream, flush, audit_every, hbm_peak, K, W):
    """The 600 x 200 regular shock reflection (15 MB in FP32, smaller than
    L2): each step timed alone with the L2 flushed before it (the latency of
    a cold one-wave launch), and as a long run issues it (autotuned launch,
    64-step graph replays back to back, L2-resident)."""
    import workloads
    w = workloads.regular_reflection()
    cells = w.nx * w.ny
    out = {"workload": "regular_shock_reflection_%dx%d" % (w.nx, w.ny), "unit": UNIT,
           "flushed": "each step timed alone, L2 flushed (256 MiB write + 256 MiB read) before it"}
    for prec in ("fp32", "fp64"):
        ctx = make_ctx(lbm, w, prec, audit_every, stream, tune=False)
        try:
            t = time_steps(torch, lbm, ctx, stream, flush, K, W)
            ms = sum(t) / K
            out[prec + "_flushed"] = {"value": cells / (ms * 1e-3), "ms_per_step": ms,
                                      "step_blocks": lbm.lbm_step_blocks(ctx),
                                      "status": list(lbm.lbm_status(ctx))}
        finally:
            lbm.lbm_destroy(ctx)
        ctx = make_ctx(lbm, w, prec, audit_every, stream)
        try:
            ms = time_graph_steps(torch, lbm, ctx, stream, 640, 5)
            out[prec + "_long_run"] = {"value": cells / (ms * 1e-3), "ms_per_step": ms,
                                       "step_blocks": lbm.lbm_step_blocks(ctx)}
        finally:
            lbm.lbm_destroy(ctx)
    out["fp32_flushed"]["hbm_frac"] = (BYTES_PER_CELL["fp32"] * cells
                                       / (out["fp32_flushed"]["ms_per_step"] * 1e-3) / 1e9 / hbm_peak)
    return out


def traffic_record(kernel):
    """DRAM bytes per launch of ``kernel`` from the committed ncu summary, or
    None when the CUDA sources changed after it was taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))[kernel]
    except (OSError, KeyError, ValueError):
        return None
    return rec["dram_bytes_per_launch"] if rec.get("source_hash") == source_hash() else None


# The sources that define the one-step grid kernels (their DRAM counts in
# profiles/traffic.json are valid while these files are unchanged; host code
# that launches them is not among them).
STEP_SOURCES = ("lbm_step_kernels.cuh", "lbm_step.cuh", "d2v16.cuh", "tma.cuh", "coeffs.h",
                "dw.cuh", "lbm_dw_step.cuh")


def source_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_0908_3749_gb300", "csrc")
    for fn in STEP_SOURCES:
        h.update(open(os.path.join(d, fn), "rb").read())
    return h.hexdigest()[:16]


def e2e_steps(torch, lbm, ctx, w, K, W):
    """Steps through the C ABI with host buffers: each step copies the
    populations in from pinned host memory, runs one step and reads the
    moments back into pinned host memory. Wall-clock seconds per step."""
    es = lbm.lbm_element_size(ctx)
    f = torch.empty((16, w.ny, w.nx), dtype=torch.float64 if es == 8 else torch.float32).pin_memory()
    outs = torch.empty((4, w.ny, w.nx), dtype=torch.float64).pin_memory()  # rho, u, v, T
    fn = f.numpy()
    on = list(outs.numpy())
    lbm.lbm_get_populations(ctx, fn)
    times = []
    for k in range(W + K):
        t0 = time.perf_counter()
        lbm.lbm_set_populations(ctx, fn, k)
        lbm.lbm_step(ctx, 1)
        lbm.lbm_moments(ctx, *on)
        if k >= W:
            times.append(time.perf_counter() - t0)
    return times, f.numel() * f.element_size(), outs.numel() * 8


def tubes_measure(torch, lbm, stream, args, hbm_peak):
    """4096 seeded quasi-1D Riemann problems (Nx ~ U[128, 2048]) in one
    persistent launch per call: the autotuned tiling, then timed calls of
    ``--tube-steps`` steps each (inputs larger than L2). The watchdog's
    per-tube status after the timed calls splits the tubes into stable and
    unstable ones; a second batch then runs the configuration's whole 10 000
    steps (t = 0.1) and is counted the same way."""
    import workloads
    B = workloads.tube_batch()
    nt = len(B["nx"])
    nx = np.asarray(B["nx"])
    b = lbm.lbm_batch_create(B["nx"], B["dx"], B["dt"], B["s"], B["left"], B["right"], stream)
    try:
        lbm.lbm_batch_set_init(b, *workloads.tube_fields(B))
        chosen = lbm.lbm_batch_autotune(b, 20, None)
        n = args.tube_steps
        lbm.lbm_batch_step(b, n)               # capture + warm-up
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        times = []
        with torch.cuda.stream(stream):
            for k in range(3):
                ev[0].record(stream)
                lbm.lbm_batch_step(b, n)
                ev[1].record(stream)
                stream.synchronize()
                times.append(ev[0].elapsed_time(ev[1]))
        steps_run = lbm.lbm_batch_step_count(b)
        rc, bad, nbad, to = lbm.lbm_batch_status(b, nt)
        total = lbm.lbm_batch_total_nodes(b)
    finally:
        lbm.lbm_batch_destroy(b)
    ms = min(times) / n
    stable_nodes = int(nx[bad < 0].sum())
    out = {"workload": "4096_tubes_nx_128_2048", "nodes": total, "steps_per_launch": n,
           "value": total / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
           "achieved_gbs": BYTES_PER_CELL["fp32"] * total / (ms * 1e-3) / 1e9,
           "frac_of_hbm": BYTES_PER_CELL["fp32"] * total / (ms * 1e-3) / 1e9 / hbm_peak,
           "tiling": list(chosen), "timeout": to, "graph": True, "launches_per_call": 1,
           "steps_run": steps_run, "unstable_tubes": nbad, "stable_tubes": nt - nbad,
           "value_stable": stable_nodes / (ms * 1e-3),
           "value_stable_note": "node-updates of the tubes that stayed physical, per second of "
                                "the whole batch's step"}
    # the configuration's whole run, counted
    b = lbm.lbm_batch_create(B["nx"], B["dx"], B["dt"], B["s"], B["left"], B["right"], stream)
    try:
        lbm.lbm_batch_set_init(b, *workloads.tube_fields(B))
        lbm.lbm_batch_set_tiling(b, chosen[0], chosen[1])
        lbm.lbm_batch_step(b, B["nsteps"])
        rc, bad, nbad, to = lbm.lbm_batch_status(b, nt)
        out["full_run"] = {"steps": B["nsteps"], "unstable_tubes": nbad, "stable_tubes": nt - nbad,
                           "unstable_by_step": {str(s): int(((bad >= 0) & (bad <= s)).sum())
                                                for s in (100, 1000, 10000)}}
    finally:
        lbm.lbm_batch_destroy(b)
    return out


def vn_measure(torch, lbm, stream):
    """Stability map of the Sec. IV example: u = 0 .. 10 in 32 steps for the
    MRT and the SRT rates (64 cases) x 4096 wave numbers k dx in [0, pi] along
    x = 262 144 matrices G per sweep; eigenvalues on the device (FP64,
    compute-bound: the 4 KB of inputs stay in L2 and are not flushed)."""
    import workloads
    ex = workloads.vn_example(nk=4096)
    us = np.linspace(0.0, 10.0, 32)
    states = np.array([[2.0, u, 0.0, 2.0] for _ in range(2) for u in us])
    rates = np.repeat(ex["rates"], len(us), axis=0)
    cases = torch.from_numpy(lbm.vn_cases(states, rates)).cuda()
    k = torch.from_numpy(np.ascontiguousarray(ex["k"])).cuda()
    n = cases.shape[0] * k.shape[0]
    radius = torch.empty(n, dtype=torch.float64, device="cuda")

    def sweep():
        lbm.lbm_vn_spectrum(cases, k, ex["dx"], ex["dy"], ex["dt"], radius=radius, stream=stream,
                            count_nonconverged=False)

    for _ in range(3):
        sweep()
    stream.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    times = []
    for _ in range(5):
        ev[0].record(stream)
        sweep()
        ev[1].record(stream)
        stream.synchronize()
        times.append(ev[0].elapsed_time(ev[1]))
    r = radius.cpu().numpy().reshape(2, len(us), -1).max(axis=2)
    stable = {name: float(us[np.nonzero(r[c] <= 1.0 + 1e-9)[0]].max()) if (r[c] <= 1.0 + 1e-9).any()
              else None for c, name in enumerate(ex["names"])}
    ms = statistics.median(times)
    return {"workload": "Sec. IV example (rho, T) = (2, 2), u = 0..10 (32 values) x {MRT, SRT} "
                        "x 4096 k dx in [0, pi]",
            "matrices": n, "ms_per_sweep": ms, "matrices_per_s": n / (ms * 1e-3),
            "largest_stable_u": stable,
            "max_radius_at_u10": {name: float(r[c, -1]) for c, name in enumerate(ex["names"])},
            "launches_per_sweep": 2, "dtype": "f64"}


def corrector_measure(torch):
    """Wall time of the learned coarse-grid corrector's use against the fine
    run it stands in for (configuration of the learned part: 512 x 512
    coarse, 4x finer reference, t_end 0.02, FP32 steps): one held-out
    quadrant problem run fine (2048 x 2048, dt / 4) and coarse, plus one
    network inference (lbm_cnn_correct). The inference time does not depend
    on the weights, so an untrained network (identity output) is timed; the
    trained network's accuracy gain is the GPU test
    test_gpu_corrector.test_training_gains_at_full_scale."""
    import workloads
    from paper_0908_3749_gb300 import corrector, lbm
    n, r, t_end, dt = 512, 4, 0.02, 1e-5
    nc = int(round(t_end / dt))
    wf = workloads.corrector_quadrant(10001, n * r, dt / r)
    wc = workloads.corrector_quadrant(10001, n, dt)
    corrector.run_fields(wc, 10)                      # warm-up (library, graphs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, ok_f = corrector.run_fields(wf, nc * r)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    coarse, ok_c = corrector.run_fields(wc, nc)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    net = lbm.lbm_cnn_create(n, n)
    try:
        lbm.lbm_cnn_set_params(net, corrector.init_params(0))
        out = torch.empty_like(coarse)
        lbm.lbm_cnn_correct(net, coarse, out)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        for _ in range(5):
            lbm.lbm_cnn_correct(net, coarse, out)
        torch.cuda.synchronize()
        t4 = time.perf_counter()
    finally:
        lbm.lbm_cnn_destroy(net)
    inf = (t4 - t3) / 5
    return {"workload": "2D Riemann quadrant (seed 10001), coarse %dx%d / fine %dx%d, t_end %g, FP32"
                        % (n, n, n * r, n * r, t_end),
            "fine_run_s": t1 - t0, "coarse_run_s": t2 - t1, "inference_s": inf,
            "speedup_vs_fine": (t1 - t0) / (t2 - t1 + inf), "runs_physical": bool(ok_f and ok_c)}


def measure_peaks(lbm, stream):
    """FMA rates of this device (lane operations per second), measured now."""
    return {"fp64_fma_per_s": lbm.lbm_probe_fma_rate("fp64", 50.0, stream),
            "fp32_fma_per_s": lbm.lbm_probe_fma_rate("fp32", 50.0, stream),
            "fp32x2_fma_per_s": lbm.lbm_probe_fma_rate("fp32x2", 50.0, stream),
            "how": "independent FMA chains (8 per thread, 8 x 256 threads per SM), best of 3 "
                   "launches of ~50 ms (include/lbm_probe.h)"}


def run_ours(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_0908_3749_gb300 import lbm
    lbm.load()
    w = workload()
    cells = w.nx * w.ny
    stream = torch.cuda.Stream()
    clocks = Clocks(device_uuid(torch))
    K, W = args.steps, args.warmup
    peaks_file = {}
    try:
        peaks_file = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks_file.get("hbm_gbs", 6800.0)

    # Headline: FP64 step on the 2048 x 1024 grid, one block per 32 x 2 node
    # tile (k_step<double>; the autotuner's persistent candidates measure
    # within 0.1 % of it here, so the timed kernel is fixed, the one whose
    # DRAM counters profiles/traffic.json holds).
    ctx = make_ctx(lbm, w, "fp64", args.audit_every, stream, tune=False)
    blocks = lbm.lbm_step_blocks(ctx)
    tiles = -(-w.nx // 32) * -(-w.ny // 2)
    kname = "k_step<double>" if blocks >= tiles else "k_step_pipe<double>"
    peaks = measure_peaks(lbm, stream)     # the FP64 units at full clock before the region
    with torch.cuda.stream(stream):
        lbm.lbm_step(ctx, W)
        stream.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        h0 = time.perf_counter()
        ev0.record(stream)
        lbm.lbm_step(ctx, K)
        ev1.record(stream)
        torch.cuda.synchronize()
        h1 = time.perf_counter()
        if dist:
            dist.barrier()
    total_ms = max_over_ranks(dist, [ev0.elapsed_time(ev1)], "cuda")[0]
    status = lbm.lbm_status(ctx)
    e2e_t, h2d, d2h = e2e_steps(torch, lbm, ctx, w, max(5, K), 2)
    lbm.lbm_destroy(ctx)

    flush = L2Flush(torch)
    large = None if args.no_large else large_grid_measure(torch, lbm, stream, args.audit_every, hbm_peak)
    refl = None if args.no_small else reflection_measure(torch, lbm, stream, flush, args.audit_every,
                                                         hbm_peak, max(K, 20), W)
    tubes = None if args.no_tubes else tubes_measure(torch, lbm, stream, args, hbm_peak)
    vn = None if args.no_vn else vn_measure(torch, lbm, stream)
    corr = None if args.no_corrector else corrector_measure(torch)
    clocks.stop()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    ms = total_ms / K
    tflops = FLOPS_PER_CELL * cells / (ms * 1e-3) / 1e12
    peak_tflops = 2.0 * peaks["fp64_fma_per_s"] / 1e12
    line = {
        "metric": METRIC,
        "value": whole_job_rate(world, cells * K, total_ms * 1e-3),
        "unit": UNIT,
        "n_gpus": world,
        "steps": K,
        "warmup": W,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": config_json(w),
        "path": {"precision": "fp64", "audit_every": args.audit_every, "step_blocks": blocks,
                 "kernel": "%s (32 x 2 node tiles, %d blocks)" % (kname, blocks),
                 "timing": "CUDA events around the K steps on the launching stream"},
        "roofline": {"bound": "alu", "achieved": tflops, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": tflops / peak_tflops, "traffic": traffic_record(kname),
                     "kernel": kname,
                     "peak_source": "measured in this run: 2 x FP64 FMA rate (lbm_probe_fma_rate)",
                     "flops_per_cell_update": FLOPS_PER_CELL,
                     "fp64_pipe_frac": FP64_INSTR_PER_CELL * cells / (ms * 1e-3) / peaks["fp64_fma_per_s"],
                     "fp64_instructions_per_cell_update": FP64_INSTR_PER_CELL,
                     "hbm_frac": BYTES_PER_CELL["fp64"] * cells / (ms * 1e-3) / 1e9 / hbm_peak,
                     "hbm_peak_gbs": hbm_peak,
                     "bytes_per_cell_update": BYTES_PER_CELL["fp64"]},
        "status": list(status),
        "peaks": peaks,
        "e2e": {"value": cells / statistics.mean(e2e_t), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "path": "lbm_set_populations(pinned host) + lbm_step(1) + lbm_moments(pinned host), "
                        "FP64, headline grid"},
        "clocks": dict(clocks.summary(h0 - 0.5, h1 + 0.1),
                       window="0.5 s before the timed region (the FMA probes and warm-up at "
                              "full load) to its end",
                       whole_run=clocks.summary()),
        "gpu_launches": K,
    }
    if large:
        line.update(large)
        d = large.get("df64_large_grid")
        if d:
            d["speedup_vs_fp64_headline"] = ms / d["ms_per_step"]
            d["fp64_equivalent_frac_of_fp64_peak"] = d["fp64_equivalent_tflops"] / peak_tflops
            d["fp32_fma_per_s_peak"] = peaks["fp32_fma_per_s"]
    line["reflection_600x200"] = refl
    line["tubes"] = tubes
    line["von_neumann"] = vn
    line["corrector"] = corr
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        if tubes:
            tubes["cpu_baseline"] = tubes_cpu_baseline(min(args.cpu_seconds, 6.0))
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def run_reference(args):
    """The CPU oracle timed as the reference arm (rank 0 only): one process
    per host core, each stepping one slab of the workload's grid; W warm-up
    steps, then K timed steps per slab; the job's time is the slowest slab's."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    w = workload()
    cores = os.cpu_count() or 1
    res = _run_slabs(cores, steps=args.steps, warmup=args.warmup)
    cells = sum(c for c, _, _ in res)
    el = max(e for _, _, e in res)
    value = cells * args.steps / el
    sample = ("%d host processes, one per core, each stepping one %d-row slab of the %dx%d grid "
              "as a grid of its own (FP64 numpy oracle): %d warm-up + %d timed steps per slab"
              % (cores, w.ny // cores, w.nx, w.ny, args.warmup, args.steps))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_json(w), "impl": "reference",
        "path": {"precision": "fp64", "audit_every": 0,
                 "kernel": "numpy oracle, %d host processes" % cores},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--audit-every", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--no-small", action="store_true")
    ap.add_argument("--no-tubes", action="store_true")
    ap.add_argument("--no-vn", action="store_true")
    ap.add_argument("--no-corrector", action="store_true")
    ap.add_argument("--tube-steps", type=int, default=200)
    ap.add_argument("--cpu-seconds", type=float, default=8.0)
    ap.add_argument("--cpu-sample", type=int, nargs=2, default=None, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-sample-tubes", type=float, default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_sample is not None:
        k, nslabs = args.cpu_sample
        secs = None if "--steps" in sys.argv else args.cpu_seconds
        steps = args.steps if "--steps" in sys.argv else None
        print(json.dumps(oracle_steps(k, nslabs, seconds=secs, steps=steps, warmup=args.warmup)))
        return
    if args.cpu_sample_tubes is not None:
        print(json.dumps(oracle_tube_steps(args.cpu_sample_tubes)))
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
