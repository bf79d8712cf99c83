#!/usr/bin/env python
"""Benchmark of the ES adaptive moving-mesh hot path on one GB300 (or N, one process each).

A step is one full time step of the method: mesh redistribution (CFL time step,
monitor + filter, Jacobi sweeps, limiter, mesh velocity) followed by one SSP-RK3
step (three residual evaluations with metrics, sixth-order EC flux, WENO-MR
dissipation, divergence and the stage update; in 2D one fused launch per stage
covers both directions).  The metric is cell-stage updates per second:
cells x 3 stages x steps / time, summed over all ranks.

Default workload: the 2D two-component stiffened-gas shock-bubble instance,
400 x 200 cells on [0, 2] x [0, 1], adaptive moving mesh with 5 Jacobi sweeps
and 3 filter passes per step, in the mixed FP32/FP64 form; the FP64 form and the
batched form (64 uneven instances, one launch per kernel per stage) are timed
beside it.  Inputs are synthetic and seeded; they are resident in HBM before
the timed region starts.  L2 is flushed (a 256 MiB buffer is rewritten) before
every timed step, outside the events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank advances its own copy of the workload (independent
instances, no collective on the data path) and rank 0 prints one JSON line.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-stage updates/s on 1 GB300 (mixed/batched vs FP64 form) at stated L1 error"
UNIT = "cell-stage updates/s"
WORKLOAD = ("2D two-component stiffened-gas shock-bubble, 400x200 cells on [0,2]x[0,1], Ms 1.22, bubble r 0.2 "
            "(Gamma2 1.648, density ratio 0.138), adaptive moving mesh (monitor sqrt(1+alpha|grad rho|^2/max), "
            "alpha 100, 3 filter passes, 5 Jacobi sweeps per step), sixth-order EC + WENO-MR ES flux, SSP-RK3, CFL 0.4")

# nominal peaks, for context beside the measured ones: FP32 from the SM count and maximum clock
# (152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz); FP64 as stated for GB300 (1.25 TFLOP/s)
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_NOMINAL_TFLOPS = 1.25


def measure_alu_peaks(torch, seconds=0.6):
    """Fused multiply-add throughput of the FP32 (FFMA, paired FFMA2) and FP64 (DFMA) pipes from
    the library's microbenchmark (es_alu_peak), timed with CUDA events on the launch stream:
    launches of about 10 ms repeated for `seconds` per kind; the best launch counts.  The SM
    clock is sampled meanwhile (median under load reported; no clock is set)."""
    from paper_2202_07989_gb300 import es
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    grid = sms * 8
    sink = torch.empty(grid * 256, dtype=torch.float64, device="cuda")
    iters = {0: 40000, 1: 20000, 2: 600}
    out = {"grid_ctas": grid, "threads_per_cta": 256, "chains_per_thread": 16}
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for kind, name in enumerate(es.ALU_KINDS):
        es.es_alu_peak(kind, grid, iters[kind], sink)
        torch.cuda.synchronize()
        best, t_end = float("inf"), time.perf_counter() + seconds
        while time.perf_counter() < t_end:
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            flops = es.es_alu_peak(kind, grid, iters[kind], sink)
            b.record()
            b.synchronize()
            best = min(best, a.elapsed_time(b) / 1e3)
        out[name + "_tflops"] = flops / best / 1e12
    out["clocks"] = clocks.stop()
    out["fp32_tflops"] = max(out["fp32_ffma_tflops"], out["fp32_ffma2_tflops"])
    out["fp64_tflops"] = out["fp64_dfma_tflops"]
    return out


def hbm_peak_gbs():
    """The measured copy bandwidth of the GB300s (MEASURED_PEAKS.json), else the fallback."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum, cold cache) per fused 2D stage launch
# of the 400x200 mixed step: the mean of the three stage launches of a step in one ncu capture of
# the current kernel (stage 1 10.53 MB; stages 2 and 3, which also read M(xdot) and the step-start
# state, 18.31 MB each); the capture and its command are in profiles/.  The per-direction launches
# have no current capture (traffic null when the tuner picks them).
FLUX2D_TRAFFIC_BYTES = 15.72e6


def flux_flops_per_interface(D, NS, es=True):
    """Algorithmic flops of one interface of the flux kernel (each +, -, x, /, sqrt counted once;
    the per-term counts are those of the contracted two-point flux, the GCL stencil, the
    interface averages and the WENO-MR evaluations: EC pair 26 + 18D + 21N (six pairs), GCL
    10 + 11D, dissipation set-up 3D + 2D^2 + 4 + (2 in 2D, 15 in 3D) + (12 for N = 1, 45 for
    N = 2), per column of R 8 + 15 n_c + 2D^2 + 192 (the projection and two WENO-MR
    evaluations of 96), and n_c for the flux difference)."""
    NC = NS + D + 1
    pair = 26 + 18 * D + 21 * NS
    ec = 6 * pair
    gcl = 8 + 8 * D + 3 * D + 2
    if not es:
        return ec + gcl + NC
    setup = (2 if D == 2 else 15) + 3 * D + 2 * D * D + (12 if NS == 1 else 45) + 4
    weno = 96
    column = 8 + NC + 2 * D * D + 12 * NC + 2 * weno + 2 * NC
    return ec + gcl + setup + NC * column + NC


def oracle_flops_per_interface(D, NS):
    """Flops per interface of the residual without its metrics pass, counted on the FP64 oracle
    by its operation-counting build (tests/golden/op_counts.json, written by python -m
    oracle.opcount): the method as the paper writes it, every pair of every interface formed
    from scratch.  Returns (flops, {class: count}) or (None, None) when the file is missing."""
    path = os.path.join(ROOT, "tests", "golden", "op_counts.json")
    try:
        with open(path) as f:
            c = json.load(f)["cases"]["%dd%d" % (D, NS)]["per_interface_flux"]
        return float(c["flops"]), c
    except (OSError, KeyError, ValueError):
        return None, None


def launches_per_step(pb, mixed=True, fused=False):
    """Kernel launches of one es_step.  The mesh step: the metrics of x^n (with the reduction
    reset; 2D one launch, 3D three), CFL + gradients, then the monitor, nf filter passes and mu
    sweeps (the mixed 2D form runs them as one launch for mu 1..8, nf <= 4; otherwise one
    launch each plus the limiter when mu = 0), and the velocity pass; a fixed mesh stops after
    CFL with the velocity pass.  Then d flux launches per stage (one with the fused 2D stage
    launch); 3D stages 2 and 3 form their metrics, 2D stages use M + s dt M(xdot) from the
    velocity pass."""
    m = 1 if pb.d == 2 else 3
    per_stage = 1 if (fused and pb.d == 2) else pb.d
    if pb.fixed_mesh:
        return m + 2 + 3 * per_stage
    if mixed and pb.d == 2 and 1 <= pb.mu <= 8 and pb.nf <= 4:
        mesh = m + 1 + 1 + 1
    else:
        mesh = m + 1 + 1 + pb.nf + pb.mu + (pb.mu == 0) + 1
    return mesh + 3 * per_stage + (0 if pb.d == 2 else 2 * m)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons, pw = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                pw.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "power_w_max": max(pw) if pw else None, "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def _dev(a, torch):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


class Single:
    """One instance: device state, one full step, a CUDA graph of it."""

    def __init__(self, pb, U, x, precision, torch):
        from paper_2202_07989_gb300 import es
        self.torch = torch
        self.pb = pb
        self.ctx = es.Context(pb, precision)
        self.x = _dev(x, torch)
        self.J = self.ctx.es_init_mesh(self.x)
        self.JU = (_dev(U, torch) * self.J).contiguous()
        self.xdot = torch.zeros_like(self.x)
        self.dd = torch.zeros(2, dtype=torch.float64, device="cuda")
        self.state0 = (self.JU.clone(), self.J.clone(), self.x.clone())
        self.graph = None

    def reset(self):
        self.JU.copy_(self.state0[0])
        self.J.copy_(self.state0[1])
        self.x.copy_(self.state0[2])

    def step(self):
        self.ctx.es_step(self.JU, self.J, self.x, 0.0, self.xdot, self.dd)

    def capture(self):
        torch = self.torch
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step()
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.step()
        self.graph = g

    def run(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self.step()

    @property
    def cells(self):
        return self.pb.ncell


class RkOnly(Single):
    """Residual + SSP-RK3 stage updates only (no mesh redistribution): the mesh velocity is
    zero (it changes the values of the VCL metrics, not the work) and Delta t comes from one
    CFL evaluation at the initial state."""

    def __init__(self, pb, U, x, precision, torch):
        super().__init__(pb, U, x, precision, torch)
        xd, self.dd = self.ctx.mesh_redistribute(self.JU, self.J, self.x)
        self.xdot.zero_()
        torch.cuda.synchronize()

    def step(self):
        self.ctx.es_rk_step(self.JU, self.J, self.x, self.xdot, self.dd)


class EntropyLogged(Single):
    """A full step followed by the entropy diagnostics of the new state (total entropy; the
    production needs a residual and is not formed), captured together."""

    def __init__(self, pb, U, x, precision, torch):
        super().__init__(pb, U, x, precision, torch)
        self.ent = torch.zeros(2, dtype=torch.float64, device="cuda")

    def step(self):
        super().step()
        self.ctx.entropy_production(self.JU, self.J, None, None, self.ent)


FORM5 = "mixed_3d_stiffened_shock_bubble_800x160x160_um"


class Batch:
    """Independent instances advanced by one launch per kernel per stage."""

    def __init__(self, insts, precision, torch):
        from paper_2202_07989_gb300 import es
        self.torch = torch
        self.probs = [p for p, _, _ in insts]
        self.ctx = es.Context(self.probs, precision)
        self.JU, self.J, self.x, self.xd, self.dd = [], [], [], [], []
        for p, U, x in insts:
            c1 = es.Context(p, precision)
            xx = _dev(x, torch)
            J = c1.es_init_mesh(xx)
            self.x.append(xx)
            self.J.append(J)
            self.JU.append((_dev(U, torch) * J).contiguous())
            self.xd.append(torch.zeros_like(xx))
            self.dd.append(torch.zeros(2, dtype=torch.float64, device="cuda"))
            del c1
        self.ctx.es_bind_batch(self.JU, self.J, self.x, self.xd, self.dd)
        self.graph = None

    def step(self):
        self.ctx.es_step_batch()

    def capture(self):
        torch = self.torch
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step()
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.step()
        self.graph = g

    def run(self):
        self.graph.replay() if self.graph is not None else self.step()

    @property
    def cells(self):
        return sum(p.ncell for p in self.probs)


def tune(runner, batched=False):
    """Run the library's autotuner on the runner's state; returns the choice per direction as
    "S x WT tile, grid CTAs, ms per launch" and, in 2D, the fused stage launch ("fused TX x TY
    tile ..." when chosen, else "fused off" with its best time) and, on a mixed 2D moving mesh,
    the tile of the fused mesh-step launch."""
    if batched:
        t = runner.ctx.es_autotune()
    else:
        t = runner.ctx.es_autotune(runner.JU, runner.J, runner.x, runner.xdot)
    out = ["%dx%d tile, %d CTAs, %.3f ms" % (S, WT, grid, ms) for _, S, WT, grid, ms in t]
    if len(t) == 2:
        sh, TX, TY, grid, ms = runner.ctx.es_get_fusion()
        out.append("fused %dx%d tile, %d CTAs, %.3f ms" % (TX, TY, grid, ms) if sh >= 0 else "fused off (best %.3f ms)" % ms)
        sh, TX, TY, thr, ms = runner.ctx.es_get_mesh_tiles()
        if sh >= 0:
            out.append("mesh step %dx%d tile, %d threads, %.3f ms" % (TX, TY, thr, ms))
    return out


def is_fused(runner):
    return runner.ctx.pb.d == 2 and runner.ctx.es_get_fusion()[0] >= 0


def time_steps(runner, steps, warmup, torch, flush, after=None):
    """Device time (s) of exactly `steps` steps after `warmup` untimed ones, each step bracketed
    by CUDA events on the launch stream, L2 rewritten before each; `after(i)` runs after step i,
    outside the events."""
    for _ in range(warmup):
        runner.run()
    torch.cuda.synchronize()
    total = 0.0
    for i in range(steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        runner.run()
        b.record()
        b.synchronize()
        total += a.elapsed_time(b)
        if after is not None:
            after(i)
    torch.cuda.synchronize()
    return total / 1000.0


def time_span(runner, min_seconds, torch, flush):
    """Steps timed as time_steps does until their device time reaches min_seconds: (steps, s)."""
    total, n = 0.0, 0
    while total < min_seconds:
        total += time_steps(runner, 1, 0, torch, flush)
        n += 1
    return n, total


def kernel_profile(runner, steps, torch):
    """Per-class kernel time from CUDA events the library records on its launch stream."""
    ctx = runner.ctx
    ctx.es_profile(True)
    ctx.es_profile_read()
    g = runner.graph
    runner.graph = None
    for _ in range(steps):
        runner.run()
    torch.cuda.synchronize()
    prof = ctx.es_profile_read()
    ctx.es_profile(False)
    runner.graph = g
    return prof


def errors_vs(ref_JU, ref_J, pb, JU, J):
    """L1 (cell mean) and Linf errors of rho, p and the total entropy of (JU, J) against the reference."""
    def prims(JU_, J_):
        U = JU_ / J_
        rho = U[: pb.N].sum(0)
        v2 = sum((U[pb.N + m] / rho) ** 2 for m in range(pb.d))
        cvr = sum(pb.cv[l] * U[l] for l in range(pb.N))
        rr = sum(pb.R(l) * U[l] for l in range(pb.N))
        pinf = sum(pb.pinf[: pb.N])
        T = (U[pb.N + pb.d] - 0.5 * rho * v2 - pinf) / cvr
        p = rr * T - pinf
        eta = -sum(U[l] * (pb.cv[l] * np.log(T) - pb.R(l) * np.log(U[l])) for l in range(pb.N))
        return rho, p, (J_ * eta).sum() * np.prod(pb.dxi[: pb.d])
    r0, p0, s0 = prims(ref_JU, ref_J)
    r1, p1, s1 = prims(JU, J)
    return {"rho_l1": float(np.abs(r1 - r0).mean()), "rho_linf": float(np.abs(r1 - r0).max()),
            "p_l1": float(np.abs(p1 - p0).mean()), "p_linf": float(np.abs(p1 - p0).max()),
            "total_entropy_abs": float(abs(s1 - s0)), "total_entropy_rel": float(abs(s1 - s0) / abs(s0))}


def oracle_one_step(pb, U, x):
    """One full oracle step (mesh redistribution + SSP-RK3; on a fixed mesh the CFL step and
    SSP-RK3) of (U, x) from t = 0: (JU, J, x)."""
    from oracle.oracle import Oracle
    o = Oracle(pb)
    J = o.init_J(x)
    JU = U * J
    if pb.fixed_mesh:
        return o.rk_step(JU, J, x, np.zeros_like(x), o.cfl_dt(JU, J, x))
    xd, dt, dtau = o.mesh_redistribute(JU, J, x)
    return o.rk_step(JU, J, x, xd, dt)


def oracle_steps(pb, U, x, marks):
    """Full oracle steps (mesh redistribution + SSP-RK3; on a fixed mesh the CFL step and SSP-RK3)
    of (U, x) from t = 0: {k: (JU, J)} after each step count k in marks."""
    from oracle.oracle import Oracle
    o = Oracle(pb)
    J = o.init_J(x)
    JU = U * J
    out = {}
    for k in range(1, max(marks) + 1):
        if pb.fixed_mesh:
            JU, J, x = o.rk_step(JU, J, x, np.zeros_like(x), o.cfl_dt(JU, J, x))
        else:
            xd, dt, dtau = o.mesh_redistribute(JU, J, x)
            JU, J, x = o.rk_step(JU, J, x, xd, dt)
        if k in marks:
            out[k] = (JU.copy(), J.copy())
    return out


def cpu_baseline_leg(pb, U, x, gpu_after_one, budget_s=20.0):
    """The oracle as it stands, single-threaded on the host: full steps of the same workload
    until about budget_s of CPU time; returns its throughput and its one-step state."""
    from oracle.oracle import Oracle
    o = Oracle(pb)
    J = o.init_J(x)
    JU = U * J
    t0 = time.perf_counter()
    steps = 0
    first = None
    while True:
        xd, dt, dtau = o.mesh_redistribute(JU, J, x)
        JU, J, x = o.rk_step(JU, J, x, xd, dt)
        steps += 1
        if first is None:
            first = (JU.copy(), J.copy(), x.copy())
        if time.perf_counter() - t0 >= budget_s:
            break
    el = time.perf_counter() - t0
    val = pb.ncell * 3 * steps / el
    return {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d full steps (mesh redistribution + SSP-RK3) of the 400x200 workload from t = 0, %.1f s" % (steps, el)}, first


def cpu_model():
    """The host CPU's model as /proc/cpuinfo states it (x86: model name; Arm: the implementer and
    part codes), and the number of logical cores."""
    fields = {}
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ":" in ln:
                    k, v = [t.strip() for t in ln.split(":", 1)]
                    fields.setdefault(k, v)
    except OSError:
        pass
    name = fields.get("model name") or fields.get("Model") or (
        "CPU implementer %s part %s" % (fields.get("CPU implementer", "?"), fields.get("CPU part", "?")))
    return {"model": name, "logical_cores": os.cpu_count()}


def _oracle_batch_step(i):
    """One full oracle step from t = 0 of instance i of the 64-instance batch (a worker process)."""
    sys.path.insert(0, ROOT)
    from oracle.oracle import Oracle
    from paper_2202_07989_gb300 import workloads as W
    pb, U, x = W.batched_instance(W.batched_params(64)[i])
    o = Oracle(pb)
    J = o.init_J(x)
    JU = U * J
    t0 = time.perf_counter()
    xd, dt, dtau = o.mesh_redistribute(JU, J, x)
    o.rk_step(JU, J, x, xd, dt)
    return pb.ncell, time.perf_counter() - t0


def cpu_baseline_all_cores():
    """The oracle as it stands on every host core at once: one full step of each of the 64
    instances of the batched workload, the instances spread over a process pool (spawn) of one
    worker per logical core.  Value = the batch's cells x 3 stages / wall time of the pool."""
    import multiprocessing as mp
    n = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(n) as pool:
        pool.map(_oracle_batch_step, [0] * n)          # start-up and imports, outside the timing
        t0 = time.perf_counter()
        res = pool.map(_oracle_batch_step, sorted(range(64), key=lambda i: -W_batched_cells(i)), chunksize=1)
        wall = time.perf_counter() - t0
    cells = sum(c for c, _ in res)
    return {"value": cells * 3 / wall, "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": "one full step (mesh redistribution + SSP-RK3) from t = 0 of each of the 64 instances of "
                      "the batched workload (%d cells), one worker process per core, %.1f s wall, %.1f s CPU"
                      % (cells, wall, sum(t for _, t in res))}


def W_batched_cells(i):
    from paper_2202_07989_gb300 import workloads as W
    return W.batched_params(64)[i]["n"] ** 2


def rank_env():
    """(rank, world size, local rank) of this process from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value, device):
    """The maximum of a host scalar over all ranks (the value itself without a process group),
    followed by a barrier, so that every rank leaves the timed bracket together."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def main_ours(args):
    import torch
    rank, world, local = rank_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2202_07989_gb300 import build as B
    B.build()
    from paper_2202_07989_gb300 import es, workloads as W

    pb, U, x = W.shock_bubble_2d(400, 200)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    forms = {}
    runners = {}
    tiles = {}
    for name, prec in (("mixed", es.MIXED), ("fp64", es.FP64)):
        r = Single(pb, U, x, prec, torch)
        r.step()                      # first call on the context, outside capture
        r.reset()
        tiles[name] = tune(r)
        r.capture()
        r.reset()
        runners[name] = r

    # headline: mixed form, CUDA graph per step
    main = runners["mixed"]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    t_main = time_steps(main, args.steps, args.warmup, torch, flush)
    # a sustained span of at least args.min_seconds of the same steps right after the timed
    # ones, so that the clock record covers a stretch longer than the sampling period
    n_sus, t_sus = time_span(main, args.min_seconds, torch, flush)
    clk = clocks.stop()
    t_main = max_over_ranks(t_main, "cuda")
    value = pb.ncell * 3 * args.steps * world / t_main
    # the status word after every timed run: 0 = no non-physical state met by any kernel
    forms["mixed"] = {"value": pb.ncell * 3 * args.steps / t_main, "ms_per_step": 1e3 * t_main / args.steps,
                      "status": main.ctx.es_poll_status(), "steps_run": args.warmup + args.steps + n_sus}
    forms["mixed_sustained"] = {"value": pb.ncell * 3 * n_sus / t_sus, "ms_per_step": 1e3 * t_sus / n_sus,
                                "steps": n_sus, "seconds": t_sus,
                                "what": "the headline step repeated for at least %.1f s of device time right after "
                                        "the timed steps (clocks sampled over both)" % args.min_seconds}

    # FP64 form
    r64 = runners["fp64"]
    k64 = max(3, min(args.steps, 10))
    t64 = time_steps(r64, k64, 2, torch, flush)
    forms["fp64"] = {"value": pb.ncell * 3 * k64 / t64, "ms_per_step": 1e3 * t64 / k64, "status": r64.ctx.es_poll_status()}

    # residual + stage updates only (the first way the metric is quoted), mixed form
    rk = RkOnly(pb, U, x, es.MIXED, torch)
    rk.step()
    rk.reset()
    tune(rk)
    rk.capture()
    rk.reset()
    krk = max(3, min(args.steps, 200))
    trk = time_steps(rk, krk, 3, torch, flush)
    forms["mixed_rk_only"] = {"value": pb.ncell * 3 * krk / trk, "ms_per_step": 1e3 * trk / krk,
                              "status": rk.ctx.es_poll_status(),
                              "what": "residual + SSP-RK3 stage updates only, no mesh redistribution"}
    del rk

    # uniform-mesh mode (the paper's UM-WENOMR runs): the same instance on its uniform mesh,
    # fixed (no redistribution, metrics once per step); the paper compares MM and UM costs
    um = Single(pb.with_(fixed_mesh=True), U, x, es.MIXED, torch)
    um.step()
    um.reset()
    tiles["uniform_mesh_mixed"] = tune(um)
    um.capture()
    um.reset()
    kum = max(3, min(args.steps, 200))
    tum = time_steps(um, kum, 3, torch, flush)
    forms["uniform_mesh_mixed"] = {"value": pb.ncell * 3 * kum / tum, "ms_per_step": 1e3 * tum / kum,
                                   "mm_over_um_cost": (t_main / args.steps) / (tum / kum), "status": um.ctx.es_poll_status(),
                                   "what": "fixed uniform mesh: CFL step + SSP-RK3, metrics once per step"}
    del um

    # the MM-WENOJS comparison: the same moving-mesh step with the classical WENO-JS
    # dissipation (the paper reports WENO-MR 7.6..12% dearer on CPUs)
    js = Single(pb.with_(weno=1), U, x, es.MIXED, torch)
    js.step()
    js.reset()
    tiles["mm_wenojs_mixed"] = tune(js)
    js.capture()
    js.reset()
    kjs = max(3, min(args.steps, 200))
    tjs = time_steps(js, kjs, 3, torch, flush)
    forms["mm_wenojs_mixed"] = {"value": pb.ncell * 3 * kjs / tjs, "ms_per_step": 1e3 * tjs / kjs,
                                "wenomr_over_wenojs_cost": (t_main / args.steps) / (tjs / kjs),
                                "status": js.ctx.es_poll_status(),
                                "what": "moving-mesh step with the WENO-JS dissipation"}
    del js

    # kernel profile (dominant kernel = flux) of both forms
    prof_m = kernel_profile(main, args.steps, torch)
    prof_d = kernel_profile(r64, k64, torch)

    # batched form: 64 uneven instances, mixed
    batched = None
    prof_b = None
    kb = 1
    if not args.no_batched:
        # the 64 instances are split across the ranks (no data-path communication: instances
        # share nothing); each rank advances its share in one batched launch per kernel
        insts = W.batched_2d(64)
        total_cells = sum(p.ncell for p, _, _ in insts)
        mine = W.shard([p.ncell for p, _, _ in insts], world, rank)
        bt = Batch([insts[i] for i in mine], es.MIXED, torch)
        bt.step()
        torch.cuda.synchronize()
        tiles["batched_mixed"] = tune(bt, batched=True)
        bt.capture()
        kb = max(3, min(args.steps, 10))
        if world > 1:
            torch.distributed.barrier()
        tb = max_over_ranks(time_steps(bt, kb, 2, torch, flush), "cuda")
        batched = {"value": total_cells * 3 * kb / tb, "ms_per_step": 1e3 * tb / kb, "instances": len(insts),
                   "cells": total_cells, "instances_this_rank": len(mine), "cells_this_rank": bt.cells,
                   "status": bt.ctx.es_poll_status(),
                   "scaling": "strong",
                   "split": "the 64 instances split across %d rank(s) by cells (largest first to the least "
                            "loaded rank); time = slowest rank" % world}
        forms["batched_mixed"] = batched
        prof_b = kernel_profile(bt, kb, torch)

    # 3D forms (mixed): octant Riemann problem 128^3 (N = 1) and shock-bubble 128 x 64 x 64 (N = 2)
    if not args.no_3d:
        for name, (p3, U3, x3) in (("mixed_3d_riemann_128^3", W.riemann_3d(128)),
                                   ("mixed_3d_shock_bubble_128x64x64", W.shock_bubble_3d(64))):
            r3 = Single(p3, U3, x3, es.MIXED, torch)
            r3.step()
            r3.reset()
            tiles[name] = tune(r3)
            r3.capture()
            r3.reset()
            k3 = max(3, min(args.steps, 8))
            t3 = time_steps(r3, k3, 2, torch, flush)
            forms[name] = {"value": p3.ncell * 3 * k3 / t3, "ms_per_step": 1e3 * t3 / k3, "cells": p3.ncell,
                           "status": r3.ctx.es_poll_status()}
            del r3
        # the two-component stiffened 3D case (Example 5.11, p_inf = 100 around an ideal-gas
        # bubble, Mach 10), uniform-mesh form at the paper's finest grid, 800 x 160 x 160, with the
        # total entropy formed after every step (inside the timed step)
        p5, U5, x5 = W.shock_bubble_3d_stiffened(160)
        r5 = EntropyLogged(p5, U5, x5, es.MIXED, torch)
        del U5, x5
        r5.step()
        r5.reset()
        tiles[FORM5] = tune(r5)
        r5.capture()
        r5.reset()
        k5 = max(3, min(args.steps, 6))
        log = []
        t5 = time_steps(r5, k5, 1, torch, flush, after=lambda i: log.append(float(r5.ent[1])))
        forms[FORM5] = {"value": p5.ncell * 3 * k5 / t5, "ms_per_step": 1e3 * t5 / k5, "cells": p5.ncell,
                        "total_entropy_per_step": log, "status": r5.ctx.es_poll_status(),
                        "what": "Example 5.11 (stiffened gas Gamma 3, p_inf 100; ideal-gas bubble; Mach 10), "
                                "uniform-mesh form (the paper's UM-WENOMR), 800x160x160 cells, mixed; "
                                "total entropy formed after every step inside the timed step"}
        del r5

    # end to end: C-ABI call on pinned host buffers, copies inside the timed region
    e2e = None
    if rank == 0:
        c = es.Context(pb, es.MIXED)
        # the state in one pinned host block (JU, J, x consecutive): one transfer each way
        n0 = pb.ncell
        hbuf = torch.empty((pb.nc + 1 + pb.d) * n0, dtype=torch.float64).pin_memory()
        hJU, hJ, hx = hbuf[: pb.nc * n0], hbuf[pb.nc * n0: (pb.nc + 1) * n0], hbuf[(pb.nc + 1) * n0:]
        for h, dv in zip((hJU, hJ, hx), runners["mixed"].state0):
            h.copy_(dv.reshape(-1).cpu())
        c.es_run_host(hJU, hJ, hx, 1)
        torch.cuda.synchronize()
        ke = max(3, min(args.steps, 10))
        t0 = time.perf_counter()
        for _ in range(ke):
            c.es_run_host(hJU, hJ, hx, 1)
        te = time.perf_counter() - t0
        nb = (pb.nc + 1 + pb.d) * pb.ncell * 8
        e2e = {"value": pb.ncell * 3 * ke / te, "unit": UNIT, "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb + 8,
               "steps": ke, "call": "es_run_host (one pinned host block holding JU, J, x; 1 step per call; the library replays its CUDA graph of a step)"}

    # roofline of the dominant kernel (flux + divergence + RK stage) in the headline form:
    # the flops of every interface of a step over the time of the step's flux launches
    FLUX = ("flux_k1", "flux_k2", "flux_k3", "flux_2d")
    flux_ms = sum(prof_m[k][0] for k in FLUX)
    flux_n = sum(prof_m[k][1] for k in FLUX)
    hand_iface = flux_flops_per_interface(pb.d, pb.N, pb.es)
    oracle_iface, oracle_classes = oracle_flops_per_interface(pb.d, pb.N)
    # the algorithmic flops per interface: the oracle's counted work (operation-counting build); the hand count
    # of the kernel's contracted arithmetic is reported beside it
    per_iface = oracle_iface if oracle_iface else hand_iface
    # interfaces of one stage: (n_k + 1) per grid line of each direction
    ifaces_stage = sum((pb.n[k] + 1) * pb.ncell // pb.n[k] for k in range(pb.d))
    fused_m = is_fused(main)
    flops_launch = per_iface * ifaces_stage / (1 if fused_m else pb.d)
    avg_s = flux_ms / flux_n / 1e3 if flux_n else float("nan")
    ach = flops_launch / avg_s / 1e12
    ach_hand = hand_iface * ifaces_stage / (1 if fused_m else pb.d) / avg_s / 1e12
    peaks = measure_alu_peaks(torch)
    fp32_peak, fp64_peak = peaks["fp32_tflops"], peaks["fp64_tflops"]
    roofline = {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach / fp32_peak,
                "traffic": FLUX2D_TRAFFIC_BYTES if fused_m else None, "traffic_unit": "bytes per launch",
                "kernel": "flux2d_kernel (fused stage, mixed form)" if fused_m else "flux_kernel (mixed form)", "flops_per_launch": flops_launch,
                "avg_launch_ms": avg_s * 1e3,
                "flops_per_interface": per_iface,
                "flops_source": ("FP64 oracle, operation-counting build (tests/golden/op_counts.json), per interface "
                                 "of the residual without metrics" if oracle_iface else "hand count"),
                "oracle_op_classes_per_interface": oracle_classes,
                "mufu_share": ((oracle_classes["div"] + oracle_classes["sqrt"] + oracle_classes["log"] + oracle_classes["exp"])
                               / oracle_classes["flops"]) if oracle_classes else None,
                "hand_count_flops_per_interface": hand_iface,
                "achieved_hand_count": ach_hand, "frac_hand_count": None,
                "peak_source": "measured FP32 fused multiply-add throughput (es_alu_peak, best of FFMA and paired "
                               "FFMA2) in this run, of measured; nominal %.1f TFLOP/s" % FP32_NOMINAL_TFLOPS}
    roofline["frac_hand_count"] = ach_hand / fp32_peak
    # DRAM side of the same kernel: the captured bytes per launch over the live launch time,
    # against the measured copy bandwidth (the kernel is not HBM-bound)
    traffic = roofline["traffic"]
    hbm, hbm_src = hbm_peak_gbs()
    if traffic:
        roofline["dram_gbs"] = traffic / avg_s / 1e9
        roofline["dram_frac"] = roofline["dram_gbs"] / hbm
        roofline["hbm_peak_gbs"] = hbm
        roofline["hbm_peak_source"] = hbm_src
    flux64_ms = sum(prof_d[k][0] for k in FLUX)
    flux64_n = sum(prof_d[k][1] for k in FLUX)
    avg64 = flux64_ms / flux64_n / 1e3 if flux64_n else float("nan")
    fused_d = is_fused(r64)
    flops64 = per_iface * ifaces_stage / (1 if fused_d else pb.d)
    ach64 = flops64 / avg64 / 1e12
    roofline_fp64 = {"bound": "alu", "achieved": ach64, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": ach64 / fp64_peak, "avg_launch_ms": avg64 * 1e3,
                     "peak_source": "measured FP64 fused multiply-add throughput (es_alu_peak, DFMA) in this run, "
                                    "of measured; nominal %.2f TFLOP/s" % FP64_NOMINAL_TFLOPS,
                     "kernel": "flux2d_kernel (fused stage, FP64 form)" if fused_d else "flux_kernel (FP64 form)"}

    # the same kernel at the batched size (the 64-instance batch, or this rank's share of it)
    if prof_b is not None:
        fb_ms = sum(prof_b[k][0] for k in FLUX)
        fb_n = sum(prof_b[k][1] for k in FLUX)
        if fb_n:
            fused_b = is_fused(bt)
            bprobs = bt.probs
            iface_b = sum(sum((p.n[k] + 1) * p.ncell // p.n[k] for k in range(p.d)) for p in bprobs)
            flops_b = per_iface * iface_b / (1 if fused_b else 2)
            avg_b = fb_ms / fb_n / 1e3
            hand_b = hand_iface * iface_b / (1 if fused_b else 2) / avg_b / 1e12
            roofline["batched"] = {"achieved": flops_b / avg_b / 1e12, "frac": flops_b / avg_b / 1e12 / fp32_peak,
                                   "avg_launch_ms": avg_b * 1e3, "flops_per_launch": flops_b, "cells": bt.cells,
                                   "achieved_hand_count": hand_b, "frac_hand_count": hand_b / fp32_peak}

    # CPU baseline (rank 0 only): the oracle on a bounded sample, and the errors after one step
    cpu = None
    errs = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, ref1 = cpu_baseline_leg(pb, U, x, None, budget_s=args.cpu_seconds)
        cpu["cpu"] = cpu_model()
        if not args.no_batched:
            cpu["all_cores_batched"] = cpu_baseline_all_cores()
        errs = {}
        for name in ("fp64", "mixed"):
            r = runners[name]
            r.reset()
            r.step()
            torch.cuda.synchronize()
            errs[name] = errors_vs(ref1[0], ref1[1], pb, r.JU.cpu().numpy(), r.J.cpu().numpy())
            errs[name]["vs"] = "FP64 oracle after one full step from t = 0"
        # the mixed form against the FP64 GPU form over a longer run (the FP64 form matches the
        # oracle at 1e-12 per step; the oracle itself takes about a second a step), both with one
        # fixed Delta t so that they stay at the same time levels; the meshes move with each
        # form's own monitor, so x is compared too
        rm, rd = runners["mixed"], runners["fp64"]
        rm.reset()
        rd.reset()
        _, dd0 = rd.ctx.mesh_redistribute(rd.JU, rd.J, rd.x)
        dtf = 0.8 * float(dd0[0])
        done = 0
        for k_long in (100, 500):
            while done < k_long:
                rm.ctx.es_step(rm.JU, rm.J, rm.x, dtf, rm.xdot, rm.dd)
                rd.ctx.es_step(rd.JU, rd.J, rd.x, dtf, rd.xdot, rd.dd)
                done += 1
            torch.cuda.synchronize()
            e = errors_vs(rd.JU.cpu().numpy(), rd.J.cpu().numpy(), pb, rm.JU.cpu().numpy(), rm.J.cpu().numpy())
            e["x_linf"] = float((rm.x - rd.x).abs().max())
            e["t"] = k_long * dtf
            e["status"] = [rm.ctx.es_poll_status(), rd.ctx.es_poll_status()]
            e["vs"] = "FP64 GPU form after %d full steps of one fixed Delta t from t = 0" % k_long
            errs["mixed_vs_fp64_gpu_%d_steps" % k_long] = e
        # the batched launch: a fresh batch of the same 64 instances, one step, and the
        # oracle on its three smallest instances and its largest
        if not args.no_batched:
            insts = W.batched_2d(64)
            bt1 = Batch(insts, es.MIXED, torch)
            bt1.step()
            torch.cuda.synchronize()
            order = sorted(range(len(insts)), key=lambda i: insts[i][0].ncell)
            eb = {"vs": "FP64 oracle after one full step from t = 0, per sampled instance of the 64-instance batch"}
            for i in order[:3] + order[-1:]:
                p_, U_, x_ = insts[i]
                o1 = oracle_one_step(p_, U_, x_)
                eb["instance_%d_%dx%d" % (i, p_.n[0], p_.n[1])] = errors_vs(
                    o1[0], o1[1], p_, bt1.JU[i].cpu().numpy(), bt1.J[i].cpu().numpy())
            errs["batched_mixed"] = eb
            del bt1
        # the 3D path at sizes the oracle steps in seconds (the timed 3D forms are 128^3 and
        # 128 x 64 x 64; the kernels and launch shapes are the same at every size)
        if not args.no_3d:
            for name, (p3, U3, x3) in (("3d_shock_bubble_48x24x24", W.shock_bubble_3d(24)),
                                       ("3d_stiffened_shock_bubble_80x16x16_um", W.shock_bubble_3d_stiffened(16))):
                o1 = oracle_one_step(p3, U3, x3)
                for prec, tag in ((es.MIXED, "mixed"), (es.FP64, "fp64")):
                    r3 = Single(p3, U3, x3, prec, torch)
                    r3.step()
                    torch.cuda.synchronize()
                    e3 = errors_vs(o1[0], o1[1], p3, r3.JU.cpu().numpy(), r3.J.cpu().numpy())
                    e3["vs"] = "FP64 oracle after one full step from t = 0"
                    errs["%s_%s" % (tag, name)] = e3
                    del r3
            # the octant Riemann problem (the 128^3 form's workload) at 32^3: errors after 1 and
            # after 10 full steps
            p3, U3, x3 = W.riemann_3d(32)
            states = oracle_steps(p3, U3, x3, (1, 10))
            for prec, tag in ((es.MIXED, "mixed"), (es.FP64, "fp64")):
                r3 = Single(p3, U3, x3, prec, torch)
                done = 0
                for k, (JUo, Jo) in states.items():
                    while done < k:
                        r3.step()
                        done += 1
                    torch.cuda.synchronize()
                    e3 = errors_vs(JUo, Jo, p3, r3.JU.cpu().numpy(), r3.J.cpu().numpy())
                    e3["vs"] = "FP64 oracle after %d full steps from t = 0" % k
                    errs["%s_3d_riemann_32^3_%d_steps" % (tag, k)] = e3
                del r3

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_main / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": pb.ncell, "stages_per_step": 3, "form": "mixed FP32/FP64",
                   "graph": "one CUDA graph per full step", "l2": "256 MiB buffer rewritten before every timed step",
                   "instances_per_rank": 1, "flux_tiles": tiles.get("mixed")},
        "flux_tiles": tiles,
        "forms": forms, "errors": errs, "roofline": roofline, "roofline_fp64": roofline_fp64,
        "kernel_ms": {"mixed": {k: v[0] / args.steps for k, v in prof_m.items()},
                      "fp64": {k: v[0] / k64 for k, v in prof_d.items()},
                      "batched_mixed": ({k: v[0] / kb for k, v in prof_b.items()} if batched else None)},
        "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "alu_peaks": peaks,
        "gpu_launches": launches_per_step(pb, True, fused_m) * args.steps,
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle, as it stands, on the host cores
# ---------------------------------------------------------------------------

def main_reference(args):
    rank, world, _ = rank_env()
    if rank != 0:
        return
    from oracle.oracle import Oracle
    from paper_2202_07989_gb300 import workloads as W
    pb, U, x = W.shock_bubble_2d(400, 200)
    o = Oracle(pb)
    J = o.init_J(x)
    JU = U * J
    for _ in range(args.warmup):
        xd, dt, dtau = o.mesh_redistribute(JU, J, x)
        JU, J, x = o.rk_step(JU, J, x, xd, dt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        xd, dt, dtau = o.mesh_redistribute(JU, J, x)
        JU, J, x = o.rk_step(JU, J, x, xd, dt)
    el = time.perf_counter() - t0
    val = pb.ncell * 3 * args.steps / el
    sample = "%d full steps of the 400x200 workload after %d warm-up steps, single-threaded oracle" % (args.steps, args.warmup)
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "cells": pb.ncell, "stages_per_step": 3, "form": "FP64 CPU oracle"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main_kernel_case(args):
    """A few eager full steps of the shock-bubble instance at the given size (for ncu captures)."""
    import torch
    from paper_2202_07989_gb300 import build as B
    B.build()
    from paper_2202_07989_gb300 import es, workloads as W
    if args.kernel_case.startswith("3d:"):
        # 3D octant Riemann problem (single component), shock-bubble (two components, 2n x n x n) or
        # the stiffened shock-bubble of Example 5.11 (uniform-mesh form, 5n x n x n)
        kind, n = args.kernel_case[3:].split(":")
        pb, U, x = {"riemann": W.riemann_3d, "sb": W.shock_bubble_3d, "sb2": W.shock_bubble_3d_stiffened}[kind](int(n))
    else:
        nx, ny = [int(v) for v in args.kernel_case.split("x")]
        pb, U, x = W.shock_bubble_2d(nx, ny, length=(2.0, 1.0))
    r = Single(pb, U, x, es.MIXED if args.kernel_form == "mixed" else es.FP64, torch)
    tiles = tune(r) if args.kernel_tune else None
    if args.kernel_shapes:
        for k, sh in enumerate(int(v) for v in args.kernel_shapes.split(",")):
            r.ctx.es_set_tuning(k, sh, 0)
        tiles = r.ctx.es_get_tuning()
    if args.kernel_mesh_tiles is not None:
        r.ctx.es_set_mesh_tiles(args.kernel_mesh_tiles)
        tiles = [tiles, r.ctx.es_get_mesh_tiles()]
    if args.kernel_fusion is not None or (args.kernel_shapes and pb.d == 2):
        # fixed per-direction shapes in 2D mean the per-direction launches unless a fused shape is given
        r.ctx.es_set_fusion(args.kernel_fusion if args.kernel_fusion is not None else -1)
        tiles = [tiles, r.ctx.es_get_fusion()]
    for _ in range(args.kernel_steps):
        r.step()
    torch.cuda.synchronize()
    assert r.ctx.es_poll_status() == 0
    out = {"case": args.kernel_case, "form": args.kernel_form, "steps": args.kernel_steps, "flux_tiles": tiles}
    if args.kernel_time:
        r.reset()
        prof = kernel_profile(r, args.kernel_time, torch)
        out["kernel_ms_per_step"] = {k: v[0] / args.kernel_time for k, v in prof.items() if v[1]}
        out["launches_per_step"] = {k: v[1] / args.kernel_time for k, v in prof.items() if v[1]}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-3d", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--min-seconds", type=float, default=1.0,
                    help="device time of the sustained span of headline steps after the timed ones")
    ap.add_argument("--kernel-case", default=None, help="NXxNY | 3d:riemann:N | 3d:sb:N | 3d:sb2:N: only run a few steps of that grid (profiling)")
    ap.add_argument("--kernel-form", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--kernel-steps", type=int, default=2)
    ap.add_argument("--kernel-time", type=int, default=0, help="also time this many eager steps per kernel class")
    ap.add_argument("--kernel-tune", action="store_true", help="run the flux autotuner before the steps")
    ap.add_argument("--kernel-mesh-tiles", type=int, default=None,
                    help="tile shape 0..3 of the fused mixed 2D mesh-step launch (es_set_mesh_tiles)")
    ap.add_argument("--kernel-shapes", default=None, help="fix the flux tile shape per direction, e.g. 2,1")
    ap.add_argument("--kernel-fusion", type=int, default=None, help="2D: fix the fused stage shape (0..4, -1 off)")
    args = ap.parse_args()
    if args.kernel_case:
        return main_kernel_case(args)
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        main_reference(args)
    else:
        main_ours(args)


if __name__ == "__main__":
    main()
