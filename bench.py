#!/usr/bin/env python3
"""Throughput benchmark of the fused DUGKS time step on GB300.

Workload: the D3Q19 lid-driven cube, 256^3 cells, Re = 1000 (lid u = 0.1 along x on the
+y face, NEQ velocity walls on all six faces; lattice units dx = 1, RT = 1/3, dt = 0.5),
started from rest. One benchmark step = one time step of the whole hot path (the fused
step kernel; the FP64 residual/conservation reduction runs every RESIDUAL_EVERY steps
inside the timed region). The 2.5 GB of state is far larger than the 129 MB L2, so no
flush is needed between steps.

Reported (one JSON line on rank 0): MLUPS (million cell updates per second) for FP32
storage, the roofline of the fused kernel against the measured HBM copy bandwidth, the
BF16-storage and F16-storage forms beside it, the end-to-end MLUPS through the C ABI with
host buffers, the clocks seen during the timed region, and the FP64 CPU oracle on a
bounded sample of the same workload.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 (launched by torchrun) every rank runs an independent replica on its own GPU
(the workload is one domain; the path is not sharded): weak scaling, value = sum over
ranks.
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "D3Q19 256³ MLUPS + % HBM roofline (fp32 vs bf16-store); adjoint MLUPS"
N = 256
RE = 1000.0
LID = 0.1
RESIDUAL_EVERY = 100
Q = 19
BYTES_PER_VALUE = {0: 4, 1: 2, 2: 2, 3: 8}


def workload(q=Q):
    from paper_1411_6121_gb300 import workloads as W
    return W.cavity3d(n=N, re=RE, lid_u=LID, q=q)


def config_json(extra=None):
    c = {"workload": "D3Q19 lid-driven cube %d^3, Re=1000, lid u=0.1, NEQ walls, from rest" % N,
         "cells": N ** 3, "lattice": "D3Q19", "global_batch": 1, "seq_len": None,
         "parallelism": "replicas", "l2": "state 2.5 GB per buffer pair >> 129 MB L2 (no flush needed)",
         "residual_every": RESIDUAL_EVERY}
    if extra:
        c.update(extra)
    return c


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def strip_comments(src):
    """C/C++ source without its comments and blank lines (string and character literals kept)."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        elif c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        else:
            out.append(c)
            i += 1
    lines = (l.rstrip() for l in "".join(out).splitlines())
    return "\n".join(l for l in lines if l)


def kernel_source_hash():
    """Hash of the step kernels' code (comments excluded), to tell whether the DRAM counters of
    the committed profile were taken on this code."""
    h = hashlib.sha1()
    for name in ("dugks_step3d.cuh", "dugks_step3d_ws.cuh", "tma.cuh", "dugks_step.cuh", "dugks_device.cuh",
                 "step3d_q19.cu"):
        with open(os.path.join(ROOT, "paper_1411_6121_gb300", "csrc", name), encoding="utf-8") as f:
            h.update(strip_comments(f.read()).encode())
    return h.hexdigest()[:12]


def kernel_name(store, rows):
    """Name of the dominant kernel of the main leg (the D3Q19 throughput kernel; the cube
    has no body force, so its force-free instantiation)."""
    t = {0: "float", 1: "__nv_bfloat16", 2: "__half", 3: "double"}[store]
    if store == 3:
        return "fused_step<19,double,16,8>"
    if not rows:  # the library default for D3Q19: the warp-specialised kernel
        return "fused_step3d_ws<19,%s,false>" % t
    return "fused_step3d<19,%s,%d,false>" % (t, rows)


def profiled_traffic():
    """DRAM bytes per launch of the fused D3Q19 FP32 kernel from the committed ncu summary,
    if it was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "fused_step_d3q19_256.md")
    try:
        kv = {}
        for line in open(path):
            if ":" in line and line.strip().startswith("- "):
                k, v = line.strip()[2:].split(":", 1)
                kv[k.strip()] = v.strip().strip("`")
        if kv.get("kernel_source_sha1") != kernel_source_hash():
            return None
        return float(kv["dram_bytes_per_launch_256"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = sorted(v for v in (num(r[1]) for r in rows) if v is not None)
        mx = max((v for v in (num(r[2]) for r in rows) if v is not None), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = []
        for i, n in enumerate(names):
            if any(r[5 + i].lower() == "active" for r in rows):
                reasons.append(n)
        # median over samples taken under load (top half of the clock samples' power)
        pw = [num(r[3]) or 0.0 for r in rows]
        thr = sorted(pw)[len(pw) // 2]
        load = sorted(num(r[1]) for r in rows if (num(r[3]) or 0.0) >= thr and num(r[1]) is not None)
        med = load[len(load) // 2] if load else (sm[len(sm) // 2] if sm else None)
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": reasons, "samples": len(rows),
                "power_w_max": max(pw) if pw else None}


def run_form(torch, store, steps, warmup, dev, tile=None, q=Q, kernel=0):
    """Times `steps` fused steps of the 256^3 cube (storage `store`, velocity set q, kernel
    selector `kernel`) after `warmup`. Returns (ms per step, mean fused-kernel ms, launches of
    our kernels in the region, the last residual)."""
    from paper_1411_6121_gb300 import dugks
    cfg = workload(q)
    stream = torch.cuda.Stream(device=dev)
    sim = dugks.Sim(store=store, stream=stream.cuda_stream, use_graph=False, tile=tile, kernel=kernel, **cfg)
    sim.init()
    sim.residual()
    for i in range(warmup):
        sim.step(1)
    torch.cuda.synchronize(dev)
    n_ev = steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_ev)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    l0 = sim.launch_count()
    res = None
    t0.record(stream)
    for i in range(steps):
        ev[i][0].record(stream)
        sim.step(1)
        ev[i][1].record(stream)
        if (i + 1) % RESIDUAL_EVERY == 0:
            res = sim.residual()  # FP64 residual + conservation (a10), synchronous
    t1.record(stream)
    torch.cuda.synchronize(dev)
    l1 = sim.launch_count()
    total_ms = t0.elapsed_time(t1)
    kern = [a.elapsed_time(b) for a, b in ev]
    if res is None:
        res = sim.residual()
    sim.close()
    del sim
    return total_ms / steps, sum(kern) / len(kern), l1 - l0, res


def parse_cpulist(text):
    """The CPU set of a sysfs cpulist such as "0-71,144-215"."""
    cpus = set()
    for part in text.strip().split(","):
        if part:
            lo, _, hi = part.partition("-")
            cpus.update(range(int(lo), int(hi or lo) + 1))
    return cpus


def gpu_local_cpus(torch, dev):
    """CPUs local to the GPU (the sysfs local_cpulist of its PCI function), or None. Pinned
    host buffers are placed on the NUMA node of the thread that allocates them, and copies from
    a remote node cross the CPU-to-CPU link."""
    try:
        pr = torch.cuda.get_device_properties(dev)
        path = "/sys/bus/pci/devices/%04x:%02x:%02x.0/local_cpulist" % (pr.pci_domain_id, pr.pci_bus_id,
                                                                         pr.pci_device_id)
        return parse_cpulist(open(path).read()) & os.sched_getaffinity(0) or None
    except Exception:
        return None


def run_e2e(torch, steps, dev, trials=3, handles=2):
    """End to end through the C ABI with host buffers: every step uploads the state from
    pinned host memory, advances one step and reads the moments back to pinned host memory.
    `handles` independent simulations of the workload, each driven by a host thread of its own
    with the synchronous calls, so one handle's upload overlaps another's step and read-back.
    The process runs on the GPU's local CPUs meanwhile (so the pinned buffers sit on the GPU's
    NUMA node). Returns the median over `trials` timed runs of the wall time per step (all
    handles' steps counted), the bytes copied per step each way, and whether the local CPUs
    were found."""
    import ctypes as C
    from paper_1411_6121_gb300 import dugks
    old_aff = os.sched_getaffinity(0)
    local = gpu_local_cpus(torch, dev)
    try:
        if local:
            os.sched_setaffinity(0, local)
        cfg = workload()
        streams = [torch.cuda.Stream(device=dev) for _ in range(handles)]
        sims = [dugks.Sim(store=0, stream=st.cuda_stream, use_graph=False, **cfg) for st in streams]
        for sim in sims:
            sim.init()
        nb = sims[0].state_bytes()
        host_state = torch.empty(nb // 4, dtype=torch.float32, pin_memory=True)  # every step's input
        host_mom = [torch.empty((4, N ** 3), dtype=torch.float32, pin_memory=True) for _ in range(handles)]
        dptr = C.c_void_p(host_state.data_ptr())
        mptr = [C.c_void_p(m.data_ptr()) for m in host_mom]
        assert sims[0].lib.dugks_get_state(sims[0].h, dptr, nb, 0) == 0
        errors = []

        def drive(i, n):
            sim, lib = sims[i], sims[i].lib
            try:
                for _ in range(n):
                    rc = lib.dugks_set_state(sim.h, dptr, nb, 0)
                    if rc == 0:
                        rc = lib.dugks_step(sim.h, 1)
                    if rc == 0:
                        rc = lib.dugks_moments(sim.h, mptr[i], 0)
                    if rc != 0:
                        raise RuntimeError("handle %d: code %d" % (i, rc))
            except Exception as ex:  # reported after the join
                errors.append(ex)

        for i in range(handles):  # warm pass, one handle after another
            drive(i, 2)
        torch.cuda.synchronize(dev)
        per = []
        for _ in range(trials):
            threads = [threading.Thread(target=drive, args=(i, steps)) for i in range(handles)]
            t = time.perf_counter()
            for th in threads:
                th.start()
            for th in threads:
                th.join()
            per.append((time.perf_counter() - t) / (steps * handles))
            if errors:
                raise errors[0]
        for sim in sims:
            sim.close()
    finally:
        os.sched_setaffinity(0, old_aff)
    return sorted(per)[len(per) // 2], nb, 4 * 4 * N ** 3, local is not None


def run_batched(torch, steps, warmup, dev):
    """The batched form: 64 force-driven D2Q9 channels of uneven sizes (32x16 to 512x256,
    Re 10-500, seeded) with per-cell acceleration fields, one persistent launch per step,
    CUDA-graph replay, autotuned tile."""
    from paper_1411_6121_gb300 import dugks
    from paper_1411_6121_gb300 import workloads as W
    specs = W.batched_channels(64, seed=0x1411)
    ins = []
    for i, sp in enumerate(specs):
        fld = torch.tensor(W.force_field(sp["shape"], sp["g"][0], seed=1000 + i, rel=0.1), dtype=torch.float32,
                           device=dev)
        ins.append(dict(shape=sp["shape"], nu=sp["nu"], bcs=sp["bcs"], field=fld))
    stream = torch.cuda.Stream(device=dev)
    b = dugks.Batch(ins, dt=specs[0]["dt"], stream=stream.cuda_stream)
    for i in range(len(ins)):
        b.init(i)
    tile = b.tune()
    b.step(warmup)
    b.sync()
    cells = sum(sp["shape"][0] * sp["shape"][1] for sp in specs)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    b.step(steps)
    t1.record(stream)
    torch.cuda.synchronize(dev)
    ms = t0.elapsed_time(t1) / steps
    b.close()
    # algorithmic bytes per cell update: the FP32 D2Q9 state read and written (2 x 9 x 4) and the
    # per-cell acceleration field read (2 x 4)
    bpc = 2 * 9 * 4 + 2 * 4
    peak, src = hbm_peak()
    ach = bpc * cells / (ms * 1e-3) / 1e9
    return {"value": cells / (ms * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": ms, "instances": len(specs),
            "cells": cells, "tile": list(tile), "steps": steps,
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                         "bytes_per_cell_update": bpc, "peak_source": src,
                         "note": "events around the graph replay of all steps (one persistent launch each)"},
            "note": "64 D2Q9 channels, one persistent launch per step replayed as a CUDA graph"}


ADJ_STEPS, ADJ_EVERY = 2000, 100
ADJ_BYTES = 132  # algorithmic bytes per adjoint cell update (FP32 D2Q9): 3 x 36 state/adjoint + 8 G + 16 dL/dG


def run_adjoint(torch, dev, count=64):
    """Differentiable form: 64 uneven FP32 channels, loss ||u(T) - u_target||^2
    (u_target = 1.1 x the analytic channel profile) over T = 2000 steps with a checkpoint
    every 100 steps; gradient w.r.t. the per-cell acceleration field through dugks_record +
    dugks_adjoint_async. Each instance runs on its own CUDA stream; the reverse sweeps of all
    instances are enqueued back to back and run concurrently, timed with CUDA events on a
    stream that waits for all of them. The whole forward + reverse pass runs twice: the first
    captures each instance's segment graphs, the second (reported) replays them, as repeated
    gradient evaluations do."""
    import numpy as np
    from paper_1411_6121_gb300 import dugks
    from paper_1411_6121_gb300 import workloads as W
    specs = W.batched_channels(64, seed=0x1411)[:count]
    sims, seeds, streams = [], [], []
    cells_total = 0
    for i, sp in enumerate(specs):
        nx, ny = sp["shape"]
        n = nx * ny
        fld = torch.tensor(W.force_field(sp["shape"], sp["g"][0], seed=1000 + i, rel=0.1), dtype=torch.float32,
                           device=dev)
        st = torch.cuda.Stream(device=dev)
        sim = dugks.Sim(shape=sp["shape"], q=9, nu=sp["nu"], dt=sp["dt"], g=sp["g"], bcs=sp["bcs"], field=fld,
                        store=dugks.STORE_F32, stream=st.cuda_stream)
        sim._keep = fld
        sims.append(sim)
        streams.append(st)
        cells_total += n
    master = torch.cuda.Stream(device=dev)
    grads = [torch.empty((2, sp["shape"][0] * sp["shape"][1]), dtype=torch.float32, device=dev) for sp in specs]

    def sweep():
        """Forward rollouts with checkpoints of all instances, then their reverse sweeps,
        each instance on its own stream; returns the two device times (ms)."""
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        torch.cuda.synchronize(dev)
        ev[0].record(master)
        for sim, st in zip(sims, streams):
            st.wait_event(ev[0])
            sim.init()
            sim.record(ADJ_STEPS, ADJ_EVERY)
        for st in streams:
            master.wait_stream(st)
        ev[1].record(master)
        torch.cuda.synchronize(dev)
        seeds.clear()
        for sim, sp in zip(sims, specs):
            nx, ny = sp["shape"]
            m = torch.empty((3, nx * ny), dtype=torch.float32, device=dev)
            sim.moments(m)
            yc = np.repeat(np.arange(ny) + 0.5, nx)
            ut = torch.zeros((2, nx * ny), dtype=torch.float32, device=dev)
            ut[0] = torch.tensor(1.1 * sp["g"][0] * yc * (ny - yc) / (2.0 * sp["nu"]), dtype=torch.float32,
                                 device=dev)
            seed = torch.zeros_like(m)
            seed[1:] = 2.0 * (m[1:] - ut)
            seeds.append(seed)
        torch.cuda.synchronize(dev)
        ev[2].record(master)
        for st in streams:
            st.wait_event(ev[2])
        for sim, seed, gr in zip(sims, seeds, grads):
            sim.adjoint_async(seed, dfield=gr)
        for st in streams:
            master.wait_stream(st)
        ev[3].record(master)
        torch.cuda.synchronize(dev)
        for sim in sims:
            sim.sync()
        return ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])

    # the first sweep captures each instance's segment graphs (the library keeps them while
    # the buffers and parameters are unchanged); the second is the reported, repeated use
    _, cold_bwd_ms = sweep()
    l0 = sum(s.launch_count() for s in sims)
    fwd_ms, bwd_ms = sweep()
    launches = sum(s.launch_count() for s in sims) - l0
    # the largest instance alone (kernel-level figure at 132 algorithmic bytes per update)
    big = max(range(len(specs)), key=lambda k: specs[k]["shape"][0] * specs[k]["shape"][1])
    nb = specs[big]["shape"][0] * specs[big]["shape"][1]
    sims[big].init()
    sims[big].record(ADJ_STEPS, ADJ_EVERY)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(streams[big])
    sims[big].adjoint(seeds[big])
    e1.record(streams[big])
    torch.cuda.synchronize(dev)
    b_ms = e0.elapsed_time(e1)
    for sim in sims:
        sim.close()
    upd = cells_total * ADJ_STEPS
    big_mlups = nb * ADJ_STEPS / (b_ms * 1e-3) / 1e6
    peak, _ = hbm_peak()
    return {"value": upd / (bwd_ms * 1e-3) / 1e6, "unit": "MLUPS",
            "forward_with_checkpoints_mlups": upd / (fwd_ms * 1e-3) / 1e6,
            "forward_plus_adjoint_mlups": upd / ((fwd_ms + bwd_ms) * 1e-3) / 1e6,
            "reverse_ms": bwd_ms, "forward_ms": fwd_ms,
            "first_sweep_reverse_mlups": upd / (cold_bwd_ms * 1e-3) / 1e6,
            "instances": len(specs), "cells": cells_total,
            "steps": ADJ_STEPS, "checkpoint_every": ADJ_EVERY, "dtype": "f32", "gpu_launches": launches,
            "largest_instance": {"shape": list(specs[big]["shape"]), "adjoint_mlups": big_mlups,
                                 "bytes_per_cell_update": ADJ_BYTES,
                                 "roofline": {"bound": "hbm", "achieved": ADJ_BYTES * big_mlups * 1e6 / 1e9,
                                              "peak": peak, "unit": "GB/s",
                                              "frac": ADJ_BYTES * big_mlups * 1e6 / 1e9 / peak}},
            "note": "reverse sweep = recompute of each 100-step segment from its checkpoint + 2000 "
                    "transposed steps, per instance on its own stream, all instances concurrently; "
                    "second forward + reverse pass (the first captures the segment graphs, "
                    "first_sweep_reverse_mlups)"}


def run_case(torch, case, size, steps, warmup, dev):
    """One workload alone, for profiling (prints its own short JSON line, not the benchmark
    line). `cavity2d`: the D2Q9 lid-driven cavity of size x size cells at Re = 1000, FP32
    storage, `steps` timed steps after `warmup`, no graph (one launch per step). `adjoint`: the
    largest of the 64 uneven channels with a per-cell force field, `steps` recorded steps with
    a checkpoint every 10, then one reverse sweep, timed with CUDA events."""
    from paper_1411_6121_gb300 import dugks
    from paper_1411_6121_gb300 import workloads as W
    st = torch.cuda.Stream(device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if case == "cavity2d":
        cfg = W.cavity2d(n=size, re=RE)
        s = dugks.Sim(store=dugks.STORE_F32, stream=st.cuda_stream, use_graph=False, **cfg)
        s.init()
        s.step(warmup)
        s.sync()
        e0.record(st)
        s.step(steps)
        e1.record(st)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        s.close()
        return {"case": case, "shape": [size, size], "steps": steps, "ms_per_step": ms,
                "mlups": size * size / ms / 1e3, "gbs_at_72B": size * size * 72 / ms / 1e6}
    specs = W.batched_channels(64, seed=0x1411)
    sp = max(specs, key=lambda c: c["shape"][0] * c["shape"][1])
    nx, ny = sp["shape"]
    fld = torch.tensor(W.force_field(sp["shape"], sp["g"][0], seed=1, rel=0.1), dtype=torch.float32, device=dev)
    s = dugks.Sim(shape=sp["shape"], q=9, nu=sp["nu"], dt=sp["dt"], g=sp["g"], bcs=sp["bcs"], field=fld,
                  store=dugks.STORE_F32, stream=st.cuda_stream)
    s.init()
    s.record(steps, 10)
    seed = torch.ones((3, nx * ny), dtype=torch.float32, device=dev)
    torch.cuda.synchronize(dev)
    e0.record(st)
    s.adjoint(seed)
    e1.record(st)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    s.close()
    return {"case": case, "shape": [nx, ny], "steps": steps, "every": 10, "ms_per_step": ms,
            "mlups": nx * ny / ms / 1e3, "gbs_at_132B": nx * ny * ADJ_BYTES / ms / 1e6}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or "unknown"."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _oracle_rate(args):
    """One oracle process: MLUPS of the twin (q, n) over about `seconds` (worker of the
    CPU baseline; runs in a spawned process)."""
    q, n, seconds = args
    from oracle import Oracle
    from paper_1411_6121_gb300 import workloads as W
    cfg = W.cavity3d(n=n, re=RE, lid_u=LID, q=q) if q != 9 else W.cavity2d(n=n, re=RE, lid_u=LID)
    cfg = {k: v for k, v in cfg.items() if k not in ("rt", "rho0")}
    o = Oracle(**cfg)
    o.init()
    o.step(1)
    cells = n ** (3 if q != 9 else 2)
    steps, t = 0, time.perf_counter()
    while True:
        o.step(1)
        steps += 1
        el = time.perf_counter() - t
        if el > seconds:
            return cells * steps / el / 1e6, steps


def cpu_baseline(seconds=6.0):
    """The FP64 oracle as it stands on bounded samples of the workload's twins (the cube at the
    same Reynolds number, nu scaled with the size), on the host cores:
      * the 64^3 D3Q19 twin on one thread, and on all cores as one independent oracle process
        per core (spawned; the oracle itself is serial), whose summed rate is `value`;
      * the 128^2 D2Q9 cavity twin (Re = 1000) on one thread.
    About 3 x `seconds` of wall time."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    r1, s1 = _oracle_rate((Q, 64, seconds))
    r2, s2 = _oracle_rate((9, 128, seconds))
    ctx = mp.get_context("spawn")  # the GPU is initialised in this process: never fork
    with ctx.Pool(cores) as pool:
        res = pool.map_async(_oracle_rate, [(Q, 64, seconds)] * cores).get(timeout=30.0 + 10.0 * seconds)
    rall = sum(r for r, _ in res)
    return {"value": rall, "unit": "MLUPS", "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": "D3Q19 cube 64^3 at Re=1000 (lid 0.1, nu=0.1*64/1000), FP64: %d independent oracle "
                      "processes, one per core, %.0f s each (%d to %d steps)" % (
                          cores, seconds, min(s for _, s in res), max(s for _, s in res)),
            "single_thread": {"value": r1, "unit": "MLUPS", "cores": 1,
                              "sample": "the same 64^3 cube, %d steps, one thread" % s1},
            "cavity2d_128_single_thread": {"value": r2, "unit": "MLUPS", "cores": 1,
                                           "sample": "D2Q9 cavity 128^2 at Re=1000, %d steps, one thread" % s2}}


def max_over_ranks(torch, dist, x, device):
    """The maximum of a per-rank float over all ranks (the slowest rank sets the job time)."""
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world_size, cells_per_rank, ms_step):
    """Whole-job throughput: every rank advances its own replica of `cells_per_rank` cells
    per step; the job's step time is the slowest rank's."""
    return world_size * cells_per_rank / (ms_step * 1e-3) / 1e6


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the BF16/F16/e2e/CPU legs")
    ap.add_argument("--size", type=int, default=256, help="cube edge (256 for the benchmark; smaller for ncu)")
    ap.add_argument("--store", type=int, default=0, help="storage of the main leg (0 f32, 1 bf16, 2 f16, 3 f64)")
    ap.add_argument("--rows", type=int, default=0, help="thread-block rows of the 3D kernel (0: library default)")
    ap.add_argument("--case", default="", choices=["", "cavity2d", "adjoint"],
                    help="run one other workload alone for profiling (D2Q9 cavity of --size cells per side, "
                         "or the adjoint of the largest channel over --steps steps) and print its own line")
    args = ap.parse_args()
    global N
    N = args.size
    ws, rank, local = dist_env()
    warmup = max(3, args.warmup)

    if args.impl == "reference":
        # The reference arm is the FP64 CPU oracle, as it stands, on the host cores; rank 0
        # alone runs it. Each step is one oracle step of a 32^3 sample of the workload.
        if rank != 0:
            return 0
        from oracle import Oracle
        from paper_1411_6121_gb300 import workloads as W
        n = 32
        cfg = W.cavity3d(n=n, re=RE, lid_u=LID, q=Q)
        o = Oracle(**cfg)
        o.init()
        o.step(warmup)
        t = time.perf_counter()
        o.step(args.steps)
        el = time.perf_counter() - t
        v = n ** 3 * args.steps / el / 1e6
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": warmup, "ms_per_step": el / args.steps * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": config_json({"sample": "oracle on a %d^3 cube (same Re and lid), per step" % n}),
                "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                                 "sample": "D3Q19 cube %d^3, %d steps, FP64, 1 thread" % (n, args.steps)},
                "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0

    import torch
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_1411_6121_gb300 import dugks
    dugks.load()
    if args.case:
        if rank == 0:
            print(json.dumps(run_case(torch, args.case, args.size, args.steps, warmup, dev)), flush=True)
        return 0

    sampler = ClockSampler(local)
    if ws > 1:
        dist.barrier()
    sampler.start()
    ms_step, ms_kernel, launches, res = run_form(torch, args.store, args.steps, warmup, dev,
                                                 tile=(32, args.rows) if args.rows else None)
    clocks = sampler.stop()
    if ws > 1:
        ms_step = max_over_ranks(torch, dist, ms_step, dev)
    cells = N ** 3
    value = whole_job_mlups(ws, cells, ms_step)
    peak, peak_kind = hbm_peak()
    alg_bytes = 2 * Q * BYTES_PER_VALUE[args.store] * cells
    achieved = alg_bytes / (ms_kernel * 1e-3) / 1e9
    traffic = profiled_traffic() if (N == 256 and args.store == 0) else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_source": peak_kind, "kernel": kernel_name(args.store, args.rows),
                "bytes_per_cell_update": 2 * Q * BYTES_PER_VALUE[args.store], "kernel_ms": ms_kernel}
    extras = {}
    if not args.no_extras and rank == 0:
        for store, name in ((1, "bf16_store"), (2, "f16_store")):
            try:
                ms_s, ms_k, _, _ = run_form(torch, store, max(20, args.steps // 4), warmup, dev)
                ach = 2 * Q * BYTES_PER_VALUE[store] * cells / (ms_k * 1e-3) / 1e9
                extras[name] = {"value": cells / (ms_s * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": ms_s,
                                "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                                             "frac": ach / peak, "bytes_per_cell_update": 2 * Q * BYTES_PER_VALUE[store]}}
            except Exception as ex:  # reported, not hidden
                extras[name] = {"error": str(ex)}
    if not args.no_extras and rank == 0:
        # the paper's own 3D set (D3Q27, 216 B per cell update in FP32) on the same cube, through
        # the throughput kernel and the reference kernel
        try:
            d27 = {"unit": "MLUPS", "bytes_per_cell_update": 2 * 27 * 4}
            for kern, name in ((0, "throughput"), (1, "reference")):
                ms_s, ms_k, _, _ = run_form(torch, 0, max(20, args.steps // 4), warmup, dev, q=27, kernel=kern)
                ach = 2 * 27 * 4 * cells / (ms_k * 1e-3) / 1e9
                d27[name] = {"value": cells / (ms_s * 1e-3) / 1e6, "ms_per_step": ms_s,
                             "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                                          "frac": ach / peak}}
            extras["d3q27"] = d27
        except Exception as ex:
            extras["d3q27"] = {"error": str(ex)}
    if not args.no_extras and rank == 0:
        try:
            extras["batched"] = run_batched(torch, max(50, args.steps), warmup, dev)
        except Exception as ex:
            extras["batched"] = {"error": str(ex)}
    if not args.no_extras and rank == 0:
        try:
            extras["adjoint"] = run_adjoint(torch, dev)
        except Exception as ex:
            extras["adjoint"] = {"error": str(ex)}
    e2e = None
    if rank == 0 and not args.no_extras:
        sec, bi, bo, pinned_local = run_e2e(torch, max(3, min(10, args.steps // 20)), dev)
        e2e = {"value": cells / sec / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
               "note": "per step: state upload from pinned host, one step, moments to pinned host, via the C ABI; "
                       "two independent simulations of the workload, each driven by its own host thread, so one's "
                       "upload overlaps the other's step and read-back; median of 3 runs"
                       + ("; on the GPU's local CPUs" if pinned_local else "")}
    cpu = cpu_baseline() if (rank == 0 and ws == 1 and not args.no_extras) else None
    if ws > 1:
        dist.barrier()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
                "warmup": warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config_json(),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks, "residual": {"rel_du": res[0], "mass": res[1]}}
        line.update(extras)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
