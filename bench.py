"""Benchmark of the RAM step on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload disk|disk_large|batched] [--no-e2e] [--no-cpu]

One step = one full RAM step (shift by v0 dt with the PPM remap, then the
sub-cycled van Leer residual step) of every ring of a synthetic Keplerian disk
(1024 rings x 4096 phi cells, FP32 cells, FP64 shifts).  One disk's data fits
in L2, so the timed loop steps several copies of the disk in turn (each its own
disk advancing step by step), enough that a copy's data has left L2 before its
next step; the K steps run back to back between one pair of CUDA events on the
launching stream.  The same step timed on its own (L2 flushed before it, events
around it) is reported beside it as `isolated_step`.  With
N GPUs (torchrun, one rank per GPU) every rank advances its own disk (weak
scaling, no data exchange); the time is the max over ranks.

Prints ONE JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "RAM step Gcell-updates/s & % HBM roofline, FP32/batched vs plain FP64 at 1e-5 L1"
UNIT = "Gcell-updates/s"


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _workload(name, rank, disk=None):
    from paper_2305_05362_gb300 import workloads as wl
    if name == "disk":
        n_r, n_phi = (1024, 4096) if disk is None else disk
        return wl.disk(n_r=n_r, n_phi=n_phi, seed_dv=4 + rank, dtype=np.float32)
    if name == "disk_large":
        return wl.disk(n_r=8192, n_phi=16384, seed_dv=4 + rank, dtype=np.float32)
    if name == "batched":
        return wl.batched(n_rows=512, seed_len=6 + 100 * rank)
    if name == "batched_large":
        return wl.batched(n_rows=8192, seed_len=6 + 100 * rank)
    if name == "batched_dv":
        return wl.batched(n_rows=512, seed_len=6 + 100 * rank, with_dv=True)
    if name == "line":
        return wl.line_nonuniform()
    raise SystemExit("unknown workload %s" % name)


def _bytes_per_cell(w, es):
    """Algorithmic bytes of one step per cell: read Q, write Q, read dv when the
    residual step runs, and read the mesh (one 8-byte node per mesh cell) when it
    is not uniform: every row's own mesh, or one shared non-uniform mesh once."""
    b = 2 * es
    if w.dv is not None:
        b += es
    if not w.shared_mesh:
        b += 8
    else:
        x = np.asarray(w.row_nodes(0), dtype=np.float64)
        dx = np.diff(x)
        if not np.allclose(dx, dx.mean(), rtol=1e-9, atol=0.0):
            b += 8.0 * dx.size / w.n_cells
    return b


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="ram_bench_clocks_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.f = open(self.path, "w")
            cmd = ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                   "-lms", "50"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            self._remove()
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            lines = f.readlines()
        self._remove()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}

    def _remove(self):
        try:
            os.remove(self.path)
        except OSError:
            pass


def _traffic(kernel_key):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is
    unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        ent = d[kernel_key]
    except Exception:
        return None
    h = hashlib.sha256()
    for rel in ent["sources"]:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    if h.hexdigest() != ent["sha256"]:
        return None
    return ent


def _kernel_name(tuning):
    """The FP32 uniform-row kernel (order 3) the tuning selects, as ncu names it."""
    k = tuning["uniform_kernel_f32"]
    if k == 0:
        return "k_rows<float,3,%d>" % tuning["rows_cells_per_thread_f32"]
    if k == 1:
        return {1: "k_useg_pf<3,true,true>", 2: "k_useg_ring<3,8,true,true>"}.get(
            tuning["seg_variant_f32"], "k_useg<float,3,8,true,true>")
    return "k_stream<3,%d>" % tuning["stream_cells_per_lane_f32"]


def cpu_baseline(w, budget_s=10.0):
    """The FP64 oracle (C, OpenMP over rows) on the host cores: whole-disk steps
    until the time budget is spent."""
    import oracle
    shifts = np.array([oracle.shift_from_velocity(v, w.dt) for v in w.v0])
    q = np.asarray(w.q0, dtype=np.float64)
    dv = None if w.dv is None else np.asarray(w.dv, dtype=np.float64)
    steps = 0
    t0 = time.perf_counter()
    while True:
        q = oracle.step_rows(w.row_offset, w.nodes, w.shared_mesh, w.order, w.limiter,
                             shifts, q, dv=dv, dt=w.dt, scheme=w.scheme, nsub=w.nsub)
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    return {"value": w.n_cells * steps / el / 1e9, "unit": UNIT,
            "cores": int(oracle.num_threads()), "kind": "oracle",
            "sample": "%d full steps of the %s workload (%d cells) in %.1f s, FP64 C oracle, "
                      "OpenMP over rows" % (steps, w.name, w.n_cells, el)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = _workload(args.workload, 0,
                  tuple(int(x) for x in args.disk.split(",")) if args.disk else None)
    res = cpu_baseline(w, budget_s=max(2.0, 20.0 / max(1, args.steps)))
    steps = args.steps
    # each timed step is a bounded sample: the same oracle steps as cpu_baseline
    import oracle
    shifts = np.array([oracle.shift_from_velocity(v, w.dt) for v in w.v0])
    rows = max(1, min(w.n_rows, int(w.n_rows * 2.0 / max(1e-9, w.n_cells / (res["value"] * 1e9)))))
    ro = w.row_offset[:rows + 1]
    n = int(ro[-1])
    q = np.asarray(w.q0[:n], dtype=np.float64)
    dv = None if w.dv is None else np.asarray(w.dv[:n], dtype=np.float64)
    for _ in range(args.warmup):
        oracle.step_rows(ro, w.nodes, w.shared_mesh, w.order[:rows], w.limiter, shifts[:rows],
                         q, dv=dv, dt=w.dt, scheme=w.scheme, nsub=w.nsub[:rows])
    t0 = time.perf_counter()
    for _ in range(steps):
        q = oracle.step_rows(ro, w.nodes, w.shared_mesh, w.order[:rows], w.limiter,
                             shifts[:rows], q, dv=dv, dt=w.dt, scheme=w.scheme,
                             nsub=w.nsub[:rows])
    el = time.perf_counter() - t0
    value = n * steps / el / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "sample_rows": rows, "sample_cells": n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": int(oracle.num_threads()),
                             "kind": "oracle",
                             "sample": "%d of %d rings per step (%d cells), FP64 C oracle"
                                       % (rows, w.n_rows, n)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _dominant_kernel(info, w, tuning):
    """The kernel that takes the step's time, as ncu names it: the uniform-row
    kernel the tuning selects, else the non-uniform rows' kernel."""
    if info.n_tiles_general == 0:
        return _kernel_name(tuning)
    if tuning.get("nonuniform_kernel_f32", 0) == 1 and info.n_nseg_rows == info.n_rows - info.n_uniform_rows:
        return "k_nseg<%s,%s>" % ("true" if w.limiter else "false",
                                  "false" if w.dv is None else "true")
    return "k_gwarp<float>" if w.dv is None else "k_general<float>"


class Runner:
    """One workload on this rank's GPU: its plan, device tensors and the timed
    loop (CUDA events on the launching stream; copies of the workload stepped in
    turn so that every step reads inputs that are not in L2)."""

    def __init__(self, w, dev, world, args, tuning=None, autotune=True):
        import torch
        from paper_2305_05362_gb300 import ram
        self.torch, self.ram = torch, ram
        self.w, self.dev, self.world, self.args = w, dev, world, args
        self.plan = ram.Plan.from_workload(w, device=dev.index)
        self.info = self.plan.info()
        self.v0 = torch.tensor(w.v0, dtype=torch.float64, device=dev)
        self.nsub = torch.tensor(w.nsub, dtype=torch.int32, device=dev)
        if tuning:
            t = self.plan.tuning()
            for k, v in tuning.items():
                setattr(t, k, int(v))
            self.plan.set_tuning(t)
        elif autotune:
            for dt_ in (torch.float64, torch.float32):
                q_, _, dv_ = self.tensors(dt_)
                ram.autotune(self.plan, q_, torch.empty_like(q_), self.v0, w.dt, dv=dv_,
                             scheme=w.scheme, nsub=self.nsub, reps=10)
                del q_, dv_
        props = torch.cuda.get_device_properties(dev)
        l2 = int(getattr(props, "L2_cache_size", 0) or 0)
        self.l2 = max(l2, 128 << 20)
        self.flush_buf = torch.empty(max(2 * l2, 256 << 20) // 4, dtype=torch.float32, device=dev)
        self.flush_buf.fill_(1.0)

    def tensors(self, dtype):
        torch, w = self.torch, self.w
        q = torch.tensor(np.asarray(w.q0), dtype=dtype, device=self.dev)
        dv = None if w.dv is None else torch.tensor(np.asarray(w.dv), dtype=dtype, device=self.dev)
        return q, torch.empty_like(q), dv

    def n_sets(self):
        """Copies of the workload stepped in turn, so that the data of one step has
        left L2 (3 x L2 of algorithmic traffic in between) before its next step."""
        per_step = self.w.n_cells * _bytes_per_cell(self.w, 4)
        return int(min(16, max(1, math.ceil(3 * self.l2 / per_step))))

    def step(self, q, out, dv):
        w = self.w
        self.ram.step(self.plan, q, out, self.v0, w.dt, dv=dv, scheme=w.scheme, nsub=self.nsub)

    def _hold(self, host_per_step, steps):
        # hold the GPU while the timed loop is queued, so that the events time the
        # kernels, not the Python launch path
        if not self.args.no_hold:
            self.torch.cuda._sleep(int(min(20.0, 2.0 * host_per_step * steps + 0.05) * 2.1e9))

    def timed(self, dtype, steps, warm):
        """K steps back to back between one pair of CUDA events on the launching
        stream.  The workload's R copies (n_sets) are stepped in turn, each its own
        disk or batch advancing step by step (input and output swap), so every
        step reads inputs that are not in L2.  Returns copy 0's state and the
        mean time per step in ms."""
        torch = self.torch
        import torch.distributed as dist
        sets = [list(self.tensors(dtype)) for _ in range(self.n_sets())]

        def one(k):
            s = sets[k % len(sets)]
            self.step(s[0], s[1], s[2])
            s[0], s[1] = s[1], s[0]

        for k in range(warm):
            one(k)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(5):
            one(warm + k)
        host_per_step = (time.perf_counter() - t0) / 5
        # copy 0 has taken the same number of steps in every call with the same
        # (steps, warm): bring the counter back to a whole number of rounds
        k0 = warm + 5
        k0 += (-k0) % len(sets)
        for k in range(warm + 5, k0):
            one(k)
        torch.cuda.synchronize()
        if self.world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        self._hold(host_per_step, steps)
        e0.record()
        for k in range(steps):
            one(k0 + k)
        e1.record()
        torch.cuda.synchronize()
        if self.world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        q0 = sets[0][0]
        del sets
        return q0, ms

    def timed_flushed(self, dtype, steps, warm):
        """The step on its own: L2 flushed (a read of 2 x L2 bytes) before every
        step and a pair of CUDA events around each step.  Per step this adds the
        launch and drain of an isolated kernel to the step's own time."""
        torch = self.torch
        q, out, dv = self.tensors(dtype)
        for _ in range(warm):
            self.step(q, out, dv)
            q, out = out, q
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            self.flush_buf.sum()
            self.step(q, out, dv)
            q, out = out, q
        host_per_step = (time.perf_counter() - t0) / 5
        torch.cuda.synchronize()
        self._hold(host_per_step, steps)
        for k in range(steps):
            self.flush_buf.sum()
            ev[k][0].record()
            self.step(q, out, dv)
            ev[k][1].record()
            q, out = out, q
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(b) for a, b in ev)

    def refine_uniform(self):
        """The autotuner times warm-cache repeats of one step; the timed steps read
        cold inputs back to back, which can rank the warp-segment launch shapes
        differently.  Refine them under the timed loop's own protocol (200 steps
        each)."""
        if self.info.n_uniform_rows != self.w.n_rows:
            return
        torch = self.torch
        base = self.plan.tuning()
        cands = [None] + [(v, g) for v in (0, 1, 2) for g in (3, 4, 6, 8)]
        best, best_ms = None, float("inf")
        for c in cands:
            t = self.plan.tuning()
            for f, _ in t._fields_:
                setattr(t, f, getattr(base, f))
            if c is not None:
                t.uniform_kernel_f32, t.seg_variant_f32, t.seg_warps = 1, c[0], c[1]
            self.plan.set_tuning(t)
            _, med = self.timed(torch.float32, 200, 3)
            if med < best_ms:
                best, best_ms = c, med
        t = self.plan.tuning()
        for f, _ in t._fields_:
            setattr(t, f, getattr(base, f))
        if best is not None:
            t.uniform_kernel_f32, t.seg_variant_f32, t.seg_warps = 1, best[0], best[1]
        self.plan.set_tuning(t)

    def launches_per_step(self):
        """Kernels of this library per step: the parameter kernel (none when every
        row is a warp-segment row of the shared-memory ring kernel, which forms its
        own), one launch per order present among the uniform rows, and the
        non-uniform rows' launch."""
        w, info, t = self.w, self.info, self.plan.tuning().as_dict()
        uniform_orders = {int(o) for o in w.order} if info.n_uniform_rows else set()
        lens = np.diff(np.asarray(w.row_offset))
        all_seg = (info.n_uniform_rows == w.n_rows and bool(np.all(lens >= 512))
                   and bool(np.all(lens % 4 == 0))
                   and bool(np.all(np.asarray(w.row_offset) % 4 == 0)))
        nonuni = w.n_rows - info.n_uniform_rows
        nseg = t.get("nonuniform_kernel_f32", 0) == 1 and nonuni > 0
        nseg_all = nseg and info.n_nseg_rows == nonuni
        own = ((info.n_uniform_rows == 0 or
                (all_seg and t["uniform_kernel_f32"] == 1 and t["seg_variant_f32"] == 2))
               and (nonuni == 0 or nseg_all))
        if nseg_all:
            general = 1
        else:
            orders = {int(o) for o in w.order} if info.n_tiles_general else set()
            per_order = 1 if w.dv is None else 2  # the tiled kernel: whole-row and windowed
            general = (1 if nseg else 0) + per_order * len(orders)
        return (0 if own else 1) + len(uniform_orders) + general

    def record(self, steps, warmup, rank, with_fp64=True, fp64_steps=50):
        """Timed FP32 run with its clock sample and roofline; the FP64 form of the
        same step and the FP32-vs-FP64 relative L1 after the same steps."""
        torch, w, world = self.torch, self.w, self.world
        sampler = ClockSampler(_uuid(self.dev) if rank == 0 else None)
        if rank == 0:
            sampler.start()
        per_step = w.n_cells * _bytes_per_cell(w, 4)
        small = self.n_sets() * per_step < 2 * self.l2
        if small:
            # copies of a workload this small cannot leave L2 between their steps:
            # each step is timed on its own after an L2 flush instead
            q32 = None
            ms32 = self.timed_flushed(torch.float32, steps, warmup)
        else:
            q32, ms32 = self.timed(torch.float32, steps, warmup)
        clocks = sampler.stop() if rank == 0 else None
        st = self.plan.check_errors()
        from paper_2305_05362_gb300 import shard
        total_s = ms32 * steps / 1e3
        total_max = shard.global_max(total_s)
        value = w.n_cells * world * steps / total_max / 1e9
        bpc = _bytes_per_cell(w, 4)
        step_s = total_s / steps
        achieved = w.n_cells * bpc / step_s / 1e9
        peak, peak_kind = _peaks()
        tuning = self.plan.tuning().as_dict()
        kernel_key = _dominant_kernel(self.info, w, tuning)
        tr = _traffic(kernel_key + ":" + w.name)
        rec = {"workload": w.name, "rows": w.n_rows, "cells": w.n_cells, "value": value,
               "unit": UNIT, "steps": steps, "ms_per_step": 1e3 * total_max / steps,
               "gpu_launches": int(steps * self.launches_per_step()),
               "roofline": {"bound": "hbm", "kernel": kernel_key, "achieved": achieved,
                            "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                            "peak_kind": peak_kind, "bytes_per_cell": bpc,
                            "traffic": None if tr is None else tr["dram_bytes_per_launch"]},
               "clocks": clocks, "device_status": st, "tuning": tuning,
               "l2": ("L2 flushed (read of 2x L2) before each step, CUDA events around "
                      "each step, median of the steps: the workload is too small for "
                      "copies of it to exceed L2" if small else
                      "inputs larger than L2: %d copies of the workload stepped in turn "
                      "(%.0f MB of step traffic between two steps of one copy); the K steps "
                      "back to back between one pair of CUDA events"
                      % (self.n_sets(), (self.n_sets() - 1) * w.n_cells * bpc / 1e6))}
        # the same step on its own, L2 flushed before it: an isolated launch
        fl_ms = self.timed_flushed(torch.float32, 50, 3)
        rec["isolated_step"] = {
            "ms_per_step": fl_ms, "value": w.n_cells * world / (fl_ms / 1e3) / 1e9,
            "unit": UNIT, "roofline_frac": w.n_cells * bpc / (fl_ms / 1e3) / 1e9 / peak,
            "protocol": "L2 flushed (read of 2x L2) before each step, CUDA events around "
                        "each step, median of 50: adds an isolated kernel's launch and "
                        "drain to every step"}
        if with_fp64:
            n64 = min(fp64_steps, steps)
            q64, ms64 = self.timed(torch.float64, n64, 3)
            q32b, _ = self.timed(torch.float32, n64, 3)
            if small:
                ms64 = self.timed_flushed(torch.float64, n64, 3)
            a, b = q32b.double(), q64
            rec["fp64_same_launch"] = {
                "value": w.n_cells * n64 / (ms64 * n64 / 1e3) / 1e9, "unit": UNIT, "steps": n64,
                "form": "the same step in FP64 (cells and arithmetic), autotuned",
                "rel_l1_fp32_vs_fp64": float((a - b).abs().sum() / b.abs().sum())}
            del q64, q32b
        return rec, q32

    def close(self):
        self.plan.destroy()
        del self.flush_buf


def _uuid(dev):
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


def fp64_single_problem(w, dev, steps=10):
    """The plain FP64 single-problem form: every row is its own problem with its
    own plan, and every problem is its own launch, one after another, FP64
    cells and arithmetic (no batching).  Returns Gcell-updates/s."""
    import torch
    from paper_2305_05362_gb300 import ram
    plans, bufs = [], []
    for r in range(w.n_rows):
        x = w.row_nodes(r)
        n = x.size - 1
        p = ram.Plan([0, n], x, order=int(w.order[r]), limiter=w.limiter, device=dev.index)
        q = torch.tensor(np.asarray(w.q0[w.row_slice(r)]), dtype=torch.float64, device=dev)
        dv = (None if w.dv is None else
              torch.tensor(np.asarray(w.dv[w.row_slice(r)]), dtype=torch.float64, device=dev))
        v0 = torch.tensor([w.v0[r]], dtype=torch.float64, device=dev)
        ns = torch.tensor([w.nsub[r]], dtype=torch.int32, device=dev)
        plans.append(p)
        bufs.append((q, torch.empty_like(q), dv, v0, ns))

    def one_step():
        for p, (q, out, dv, v0, ns) in zip(plans, bufs):
            ram.step(p, q, out, v0, w.dt, dv=dv, scheme=w.scheme, nsub=ns)

    for _ in range(3):
        one_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        one_step()
    e1.record()
    torch.cuda.synchronize()
    s = e0.elapsed_time(e1) / 1e3
    for p in plans:
        p.destroy()
    return {"value": w.n_cells * steps / s / 1e9, "unit": UNIT, "steps": steps,
            "launches_per_step": int(w.n_rows),
            "form": "one FP64 plan and one launch per problem (row), problems one after "
                    "another on one stream"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="disk",
                    choices=["disk", "disk_large", "batched", "batched_large", "batched_dv", "line"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the extra records (batched rows, the large disk)")
    ap.add_argument("--fp64-steps", type=int, default=50)
    ap.add_argument("--tuning", default=None,
                    help="launch shapes as JSON (the tuning dict of an earlier line) instead of "
                         "running the autotuner, e.g. to profile the exact kernels of a run")
    ap.add_argument("--disk", default=None,
                    help="rings,cells of the disk workload (default 1024,4096), e.g. for a "
                         "profiling case above L2 but far below the large disk")
    ap.add_argument("--no-hold", action="store_true",
                    help="do not hold the GPU while the timed loop is queued (profiling only)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    from paper_2305_05362_gb300 import ram

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    disk = tuple(int(x) for x in args.disk.split(",")) if args.disk else None
    w = _workload(args.workload, rank, disk)
    tuning_arg = json.loads(args.tuning) if args.tuning else None
    run = Runner(w, dev, world, args, tuning=tuning_arg)
    if not tuning_arg:
        run.refine_uniform()
    head, _ = run.record(args.steps, args.warmup, rank, fp64_steps=args.fp64_steps)

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        es = 4
        qh = torch.tensor(np.asarray(w.q0), dtype=torch.float32).pin_memory()
        dvh = None if w.dv is None else torch.tensor(np.asarray(w.dv),
                                                     dtype=torch.float32).pin_memory()
        outh = torch.empty_like(qh).pin_memory()
        qd, outd, dvd = run.tensors(torch.float32)
        e_steps = max(10, min(200, args.steps // 10))

        def e2e_step():
            qd.copy_(qh, non_blocking=True)
            if dvh is not None:
                dvd.copy_(dvh, non_blocking=True)
            run.step(qd, outd, dvd)
            outh.copy_(outd, non_blocking=True)

        for _ in range(3):
            e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e_steps):
            e2e_step()
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        h2d = w.n_cells * es * (2 if w.dv is not None else 1)
        e2e = {"value": w.n_cells * world * e_steps / el / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(w.n_cells * es),
               "steps": e_steps,
               "note": "one step per host round trip: the host-device copies of Q (and dv) "
                       "bound it, not the kernel"}
        del qh, dvh, outh, qd, outd, dvd
    run.close()
    del run
    torch.cuda.empty_cache()

    # extra records, each with its own timing and clock sample: the batched rows
    # (512 and 8192 uneven rows) and the large disk (the roofline case)
    extra = {}
    if not args.no_extra and args.workload == "disk" and disk is None:
        for key, name, steps in (("batched", "batched", 2000),
                                 ("batched_large", "batched_large", 300),
                                 ("batched_dv", "batched_dv", 1000),
                                 ("line_nonuniform", "line", 200),
                                 ("roofline_R", "disk_large", 1000)):
            wx = _workload(name, rank)
            rx = Runner(wx, dev, world, args)
            if key == "roofline_R":
                rx.refine_uniform()
            rec, _ = rx.record(steps, args.warmup, rank, with_fp64=(key != "roofline_R"),
                               fp64_steps=50)
            rx.close()
            del rx
            torch.cuda.empty_cache()
            if key in ("batched", "batched_dv") and world == 1:
                rec["fp64_single_problem"] = fp64_single_problem(wx, dev)
            extra[key] = rec
            del wx

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(_workload(args.workload, 0, disk))

    if rank == 0:
        line = {
            "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "rows": w.n_rows, "cells": w.n_cells,
                       "order": sorted({int(o) for o in w.order}), "limiter": w.limiter,
                       "residual": "van Leer, sub-cycled per ring" if w.dv is not None else "none",
                       "l2": head["l2"],
                       "parallelism": "dp%d (independent disks per GPU)" % world,
                       "tuning": head["tuning"]},
            "gpu_launches": head["gpu_launches"],
            "roofline": head["roofline"],
            "isolated_step": head.get("isolated_step"),
            "fp64_single": head.get("fp64_same_launch"),
            "e2e": e2e, "cpu_baseline": cpu, "clocks": head["clocks"],
            "device_status": head["device_status"],
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
