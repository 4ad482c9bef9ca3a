#!/usr/bin/env python
"""Benchmark of the per-patch SRHD fluid update on GB300 (cell updates/s).

Workload: the 3-D periodic smooth-advection problem at 256^3 cells
(rho = 1 + 0.5 sin(2 pi (x+y+z)), p = 1, gamma = 10 along the diagonal),
tiled into 32768 patches of 8^3 cells with 2 ghost cells. One step is one
srhd_advance_patches launch over the whole batch: con2pri, PLM, the
MUSCL-Hancock half step, HLLC, the conservative update with the unphysical
check and retry, and the fused CFL minimum (plus its one-block finalize).
The ghosted inputs (1.13 GB mixed, 2.26 GB FP64) are resident in HBM and
larger than L2, so no flush is needed between steps.

The headline is the float path "mixed_cf" (float storage and arithmetic;
the cancellation-critical A of the con2pri equation by error-free float
products and a compensated sum, so no FP64 instruction at all). The mixed
path with A in double ("mixed", the design that keeps FP64 inside con2pri)
and the FP64 path are measured in the same run and reported under their
names. Multi-GPU (torchrun): every rank advances its own
copy of the batch (weak scaling, no data-path collective); the value is
all cells updated / max time over ranks.

--impl reference times the FP64 CPU oracle on the host cores instead (a
bounded sample of the same workload per step).
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_GRID = 256
CELLS_PER_PATCH = 512
METRIC = "cell updates/sec on 1 GB300 (mixed vs FP64) at stated L1 error; % HBM roofline"
UNIT = "cell updates/s"
WORKLOAD = ("3-D periodic smooth advection 256^3 (rho=1+0.5 sin(2pi(x+y+z)), p=1, gamma=10 "
            "along (1,1,1)); 32768 patches of 8^3 + 2 ghost cells; one fused MUSCL-Hancock/HLLC "
            "step with limiter retry and CFL min-reduction per step")

# Patch tile of one CTA: one 8^3 patch (tiles of 2, 4 and 8 face-adjacent
# patches as thread-block clusters cost more in lockstep than they save in
# halo work on GB300, so the tuner's tile dimension has this one value).
TILE_SHAPE = "1x1x1 patches of 8^3 per CTA"

# Algorithmic work per cell update, counted by the oracle's op-counting
# instantiation (oracle/count_flops.py): adds+subs, muls, divs, sqrts of one
# MUSCL-Hancock step of the benchmark state in the large-block limit, plus
# the CFL bound of the updated cell.
FLOPS_PER_CELL_UPDATE = 4583.2
# The same count for the VL integrator and for MUSCL-Hancock under the
# polytropic EoS with Gamma = 4/3 on the same state (oracle/count_flops.py,
# keys "vl" and "polytropic_gamma_4_3").
FLOPS_PER_CELL_UPDATE_VL = 3105.9
FLOPS_PER_CELL_UPDATE_POLY = 2778.0
# Algorithmic bytes per cell update: 5 conserved values read + 5 written.
BYTES_PER_CELL_UPDATE = {"mixed_cf": 40, "mixed": 40, "fp64": 80}
# The same with the halo a ghosted batch carries: 12^3 tile cells read and
# 8^3 written per 8^3 cell updates, five variables (87.5 B float, 175 B double).
HALO_BYTES_PER_CELL_UPDATE = {q: b / 2 * (1728 + 512) / 512 for q, b in
                              BYTES_PER_CELL_UPDATE.items()}
# Peaks: FP32 from the unit counts (152 SMs x 128 FP32 lanes x 2 flops x
# 2070 MHz); FP64 at the nominal 1.25 TFLOP/s of GB300; HBM measured.
PEAK_FP32_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
PEAK_FP64_TFLOPS = 1.25
# DRAM traffic per launch of the patch kernel from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), keyed by precision, valid
# only for the kernel sources with the recorded hash.
# Captured at 128^3 (4096 patches) and scaled by 8 to the 32768-patch launch
# (profiles/patch_kernel_advection128.md).
NCU_TRAFFIC = {"sources_sha": "58f24a62548a8eec",
               "mixed_cf": 8 * (141.724416e6 + 23.045632e6),
               "mixed": 8 * (141.782016e6 + 24.145664e6),
               "fp64": 8 * (283.940096e6 + 67.366144e6)}


# The sources that make the patch kernel's device code (its translation units
# and the headers its code comes from); host-side files (srhd_api.cu,
# srhd_noalloc.cu) and the headers of the other kernels that the launch file
# also includes (srhd_vl.cuh: the VL kernel; srhd_prolong.cuh: the AMR
# prolongation) do not change it.
KERNEL_SOURCES = ("srhd_amr.cuh", "srhd_fp64.cu", "srhd_kernels.cuh", "srhd_launch.inl",
                  "srhd_mixed.cu", "srhd_mixed_cf.cu", "srhd_physics.cuh")


def _code_only(text: str) -> str:
    """C/C++/CUDA source without comments and with whitespace collapsed, so
    that editing a comment does not count as a change of the kernels."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_sources_sha() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2012_11130_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(_code_only(open(os.path.join(csrc, f)).read()).encode())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, flag in zip(names, f[5:9]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# distributed helpers (torchrun)
# ---------------------------------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def job_throughput(local_ms: float, units_per_rank: int, steps: int, device=None):
    """Whole-job throughput of a weak-scaled run: every rank processed
    units_per_rank units per step for `steps` steps; the job took the
    slowest rank's time. Returns (units/s, max ms over ranks). Uses an
    all-reduce(MAX) when a process group is initialised (nccl on the GPU,
    gloo on the CPU), which is the only collective of the benchmark."""
    import torch
    world = 1
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    try:
        import torch.distributed as dist
        if dist.is_available() and dist.is_initialized():
            world = dist.get_world_size()
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
    except ImportError:
        pass
    max_ms = float(t.item())
    return world * units_per_rank * steps / (max_ms * 1e-3), max_ms


# ---------------------------------------------------------------------------
# workload on the device
# ---------------------------------------------------------------------------
def build_workload(torch, srhd, ctx, prec, n=N_GRID, ghost=2):
    from paper_2012_11130_gb300 import workloads
    W = workloads.advection_prims(n)                       # float64 [5][n][n][n]
    Wd = torch.from_numpy(W).to("cuda")
    del W
    C = ctx.prim2con(Wd.reshape(5, -1)).reshape(5, n, n, n)
    del Wd
    npx = n // 8
    P = C.reshape(5, npx, 8, npx, 8, npx, 8).permute(1, 3, 5, 0, 2, 4, 6).reshape(-1, 5, 8, 8, 8)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    P = P.to(dtype).contiguous()
    del C
    G = (ctx.fill_ghosts_uniform3 if ghost == 3 else ctx.fill_ghosts_uniform)(P, npx, npx, npx)
    del P
    npatch = G.shape[0]
    dh = 1.0 / n
    dt_dh = torch.tensor([[0.4 * dh, dh]], dtype=torch.float64, device="cuda").repeat(npatch, 1)
    return G, dt_dh


def time_device(torch, ctx, G, dt_dh, steps, warmup, barrier, prec, vl=False):
    npatch = G.shape[0]
    step = ctx.advance_patches_vl if vl else ctx.advance_patches
    out = torch.empty((npatch, 5, 8, 8, 8), dtype=G.dtype, device="cuda")
    dn = torch.empty(1, dtype=torch.float64, device="cuda")
    st = torch.empty(npatch, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        step(G, dt_dh, cons_out=out, dt_next=dn, patch_status=st, prec=prec)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for e0, e1 in evs:
        e0.record(stream)
        step(G, dt_dh, cons_out=out, dt_next=dn, patch_status=st, prec=prec)
        e1.record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    total_ms = t0.elapsed_time(t1)
    per = [e0.elapsed_time(e1) for e0, e1 in evs]
    status_max = int(st.abs().max().item())
    return total_ms, per, dn.item(), status_max


def time_uniform_loop(torch, ctx, G, dt_dh, steps, warmup, barrier, prec, cached):
    """A time loop on the device-resident uniform grid: each step advances
    the whole grid from the previous step's output (state ping-pong), with
    the fused CFL bound and the patch status. cached: srhd_advance_uniform_prim
    (the tiles' primitives gathered from the previous step's cache, which is
    seeded once by srhd_con2pri_patches before the loop); otherwise
    srhd_advance_uniform (every tile cell converted). The grid (0.34 GB
    float state, 0.40 GB cache, twice) exceeds L2, so no flush."""
    npatch = G.shape[0]
    npx = round(npatch ** (1 / 3))
    U = G[:, :, 2:10, 2:10, 2:10].contiguous()
    V = torch.empty_like(U)
    dn = torch.empty(1, dtype=torch.float64, device="cuda")
    st = torch.empty(npatch, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    if cached:
        P = ctx.con2pri_patches(U, prec=prec)
        Q = torch.empty_like(P)

    def step():
        nonlocal U, V, P, Q
        if cached:
            ctx.advance_uniform_prim(U, P, npx, npx, npx, dt_dh, cons_out=V, prim_out=Q,
                                     dt_next=dn, patch_status=st, prec=prec)
            P, Q = Q, P
        else:
            ctx.advance_uniform(U, npx, npx, npx, dt_dh, cons_out=V, dt_next=dn,
                                patch_status=st, prec=prec)
        U, V = V, U
    if not cached:
        P = Q = None
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for e0, e1 in evs:
        e0.record(stream)
        step()
        e1.record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    total_ms = t0.elapsed_time(t1)
    per = [e0.elapsed_time(e1) for e0, e1 in evs]
    status_max = int(st.abs().max().item())
    del U, V, P, Q
    return total_ms, per, dn.item(), status_max


def measure_link(torch, nbytes: int, reps: int = 5):
    """Host link bandwidth of this run (GB/s): a pinned host buffer of
    `nbytes` copied to the device, back, and both at once on two streams
    (best of `reps`, CUDA events). Recorded beside the end-to-end figure,
    whose copies move the same number of bytes per step."""
    n = nbytes // 4
    h_in = torch.empty(n, dtype=torch.float32, pin_memory=True)
    h_out = torch.empty(n, dtype=torch.float32, pin_memory=True)
    h_in.fill_(1.0)
    d_a = torch.empty(n, dtype=torch.float32, device="cuda")
    d_b = torch.empty(n, dtype=torch.float32, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    best = {"h2d": 0.0, "d2h": 0.0, "both": 0.0}
    for _ in range(reps):
        for kind in ("h2d", "d2h", "both"):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s1)
            s2.wait_event(e0)
            if kind in ("h2d", "both"):
                with torch.cuda.stream(s1):
                    d_a.copy_(h_in, non_blocking=True)
            if kind in ("d2h", "both"):
                with torch.cuda.stream(s2):
                    h_out.copy_(d_b, non_blocking=True)
            s1.wait_stream(s2)
            e1.record(s1)
            torch.cuda.synchronize()
            moved = nbytes * (2 if kind == "both" else 1)
            best[kind] = max(best[kind], moved / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    del h_in, h_out, d_a, d_b
    return {"h2d_gbs": best["h2d"], "d2h_gbs": best["d2h"], "both_directions_gbs": best["both"],
            "bytes": nbytes, "how": "pinned host <-> device copy of the interior grid's size, "
                                     "best of %d, CUDA events" % reps}


def host_numa():
    """NUMA placement of GPU 0 and of this process (Linux sysfs), for the
    record of the end-to-end figure."""
    out = {}
    try:
        import torch
        p = torch.cuda.get_device_properties(0)
        bus = f"{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
        out["gpu_pci"] = bus
        path = f"/sys/bus/pci/devices/{bus}/numa_node"
        if os.path.exists(path):
            out["gpu_numa_node"] = int(open(path).read().strip())
    except Exception as e:  # noqa: BLE001
        out["gpu_numa_error"] = str(e)[:120]
    try:
        out["cpus_allowed"] = len(os.sched_getaffinity(0))
        out["host_numa_nodes"] = len([d for d in os.listdir("/sys/devices/system/node")
                                      if re.fullmatch(r"node\d+", d)])
    except Exception:  # noqa: BLE001
        pass
    return out


def time_e2e(torch, ctx, G, dt_dh, steps, warmup, prec):
    """Headline end-to-end number: the uniform grid lives in pinned host
    memory and each step is one srhd_advance_uniform_host call, which copies
    the interiors in, gathers the ghost zones, steps and copies the updated
    interiors, the patch status and the next time step out (chunked over
    four streams). Successive steps ping-pong between two host arrays, so
    each step's input is the previous step's output. The call is
    synchronous, so each step's wall time is taken on the host around it.
    Returns (total seconds, per-step seconds, H2D bytes, D2H bytes)."""
    npatch = G.shape[0]
    npx = round(npatch ** (1 / 3))
    dh = float(dt_dh[0, 1])
    dt = float(dt_dh[0, 0])
    A = torch.empty((npatch, 5, 8, 8, 8), dtype=G.dtype, pin_memory=True)
    A.copy_(G[:, :, 2:10, 2:10, 2:10])
    B = torch.empty_like(A, pin_memory=True)
    st = torch.empty(npatch, dtype=torch.int32, pin_memory=True)
    for _ in range(warmup):
        ctx.advance_uniform_host(A, npx, npx, npx, dt, dh, cons_out=B, patch_status=st, prec=prec)
        A, B = B, A
    torch.cuda.synchronize()
    per = []
    # the interpreter's cyclic garbage collector runs before the timed
    # steps, not inside them (a full collection of the harness's heap can
    # stall the calling thread for milliseconds)
    gc.collect()
    gc.disable()
    try:
        t = time.perf_counter()
        for _ in range(steps):
            t1 = time.perf_counter()
            _, dn = ctx.advance_uniform_host(A, npx, npx, npx, dt, dh, cons_out=B,
                                             patch_status=st, prec=prec)
            per.append(time.perf_counter() - t1)
            A, B = B, A
        torch.cuda.synchronize()
        secs = time.perf_counter() - t
    finally:
        gc.enable()
    h2d = A.numel() * A.element_size()
    d2h = B.numel() * B.element_size() + st.numel() * 4 + 8
    del A, B
    return secs, per, h2d, d2h


def time_e2e_ghosted(torch, ctx, G, dt_dh, steps, warmup, prec):
    """Ghosted patch batch in host memory (srhd_advance_patches on host
    tensors, chunked over three streams): every step copies the 12^3 tiles
    in, 3.4 times the interior bytes."""
    Gh = torch.empty(G.shape, dtype=G.dtype, pin_memory=True)
    Gh.copy_(G)
    dth = dt_dh.cpu().pin_memory()
    outh = torch.empty((G.shape[0], 5, 8, 8, 8), dtype=G.dtype, pin_memory=True)
    dnh = torch.empty(1, dtype=torch.float64, pin_memory=True)
    for _ in range(warmup):
        ctx.advance_patches(Gh, dth, cons_out=outh, dt_next=dnh, prec=prec)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(steps):
        ctx.advance_patches(Gh, dth, cons_out=outh, dt_next=dnh, prec=prec)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t
    h2d = Gh.numel() * Gh.element_size() + dth.numel() * 8
    d2h = outh.numel() * outh.element_size() + 8
    del Gh, outh
    return secs, h2d, d2h


def l1_one_period(torch, srhd, prec, n=64, params=None, vl=False, with_drift=False):
    """L1 error of rho (Eq. relative L1 error) after one period of the
    diagonal wave at n^3, evolved on the GPU with the fused CFL (uniform p
    and velocity: the wave is translated exactly, whatever the EoS).
    with_drift: also the largest relative change over the period of the
    domain sums of D, M and Etilde (periodic: conserved to round-off)."""
    import numpy as np
    from paper_2012_11130_gb300 import workloads
    ctx = srhd.Context(params or srhd.Params())
    W = torch.from_numpy(workloads.advection_prims(n)).to("cuda")
    C = ctx.prim2con(W.reshape(5, -1)).reshape(5, n, n, n)
    npx = n // 8
    dtype = torch.float64 if prec == "fp64" else torch.float32
    U = C.reshape(5, npx, 8, npx, 8, npx, 8).permute(1, 3, 5, 0, 2, 4, 6).reshape(
        -1, 5, 8, 8, 8).to(dtype).contiguous()
    v = math.sqrt(99.0 / 3.0) / math.sqrt(100.0)
    t_end = 1.0 / (3 * v)
    dh = 1.0 / n
    dd = torch.empty((U.shape[0], 2), dtype=torch.float64, device="cuda")
    dn = torch.empty(1, dtype=torch.float64, device="cuda")
    out = torch.empty_like(U)
    sums0 = U.double().sum(dim=(0, 2, 3, 4))
    dt = ctx.cfl_dt(U, dh, prec=prec).item()
    t = 0.0
    steps = 0
    while t < t_end and steps < 100000:
        dt = min(dt, t_end - t)
        dd[:, 0] = dt
        dd[:, 1] = dh
        if vl:
            G = ctx.fill_ghosts_uniform3(U, npx, npx, npx)
            ctx.advance_patches_vl(G, dd, cons_out=out, dt_next=dn, prec=prec)
        else:
            G = ctx.fill_ghosts_uniform(U, npx, npx, npx)
            ctx.advance_patches(G, dd, cons_out=out, dt_next=dn, prec=prec)
        U, out = out, U
        t += dt
        steps += 1
        dt = dn.item()
    Pd = ctx.con2pri(U.permute(1, 0, 2, 3, 4).reshape(5, -1).contiguous(), prec=prec)
    rho = Pd[0].double().reshape(npx, npx, npx, 8, 8, 8).permute(0, 3, 1, 4, 2, 5).reshape(
        n, n, n).cpu().numpy()
    exact = workloads.advection_prims(n, t=t_end)[0]
    l1 = float(np.mean(np.abs(1.0 - rho / exact)))
    if with_drift:
        sums1 = U.double().sum(dim=(0, 2, 3, 4))
        drift = float(((sums1 - sums0).abs() / sums0.abs()).max())
        return l1, steps, drift
    return l1, steps


def bench_amr(torch, srhd, steps: int, warmup: int, prec: str = "mixed_cf"):
    """Batched AMR blast (5 levels, ~38k patches of uneven level): one fused
    launch per level substep (31 per coarse step), eager and from a CUDA
    graph of the whole coarse step."""
    from paper_2012_11130_gb300 import amr, autotune
    ctx = srhd.Context(srhd.Params())
    batch, lev = amr.blast_batch(ctx, prec=prec)
    best, times = autotune.tune(batch.G, batch.dt_dh, prec=prec, steps=2)
    batch.ctx = srhd.Context(best)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        batch.step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        batch.step()
    e1.record(stream)
    torch.cuda.synchronize()
    eager_ms = e0.elapsed_time(e1) / steps
    batch.capture()
    for _ in range(warmup):
        batch.replay()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        batch.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    graph_ms = e0.elapsed_time(e1) / steps
    upd = batch.cell_updates_per_step
    out = {
        "workload": ("off-centre relativistic blast, [0,1]^3, base 64^3, 5 levels of 8^3 "
                     "patches refined around the shell, static ghost zones; level l takes "
                     "2^l substeps per coarse step, one fused launch per level substep"),
        "precision": prec, "patches_per_level": batch.counts, "patches": sum(batch.counts),
        "launches_per_coarse_step": batch.launches_per_step,
        "cell_updates_per_coarse_step": upd,
        "value_graph": upd / (graph_ms * 1e-3), "value_eager": upd / (eager_ms * 1e-3),
        "unit": UNIT, "ms_per_coarse_step_graph": graph_ms, "ms_per_coarse_step_eager": eager_ms,
        "patch_status_max": int(batch.status.abs().max().item()),
        "autotune": {"chosen_variant": best.patch_variant,
                     "ms_per_variant": {str(k): v for k, v in times.items()}},
    }
    del batch
    torch.cuda.empty_cache()
    return out


def alu_roofline(flops_per_cell: float, cells: int, launch_ms: float, prec: str):
    """ALU roofline of a fused step (as the headline's): algorithmic flops per
    launch over the mean launch time, against the FP32 peak derived from
    unit counts and clocks (float paths) or the nominal FP64 peak."""
    achieved = flops_per_cell * cells / (launch_ms * 1e-3) / 1e12
    peak = PEAK_FP64_TFLOPS if prec == "fp64" else PEAK_FP32_TFLOPS
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "flops_per_cell_update": flops_per_cell}


def bench_polytropic(torch, srhd, steps: int, warmup: int, precs=("mixed_cf", "fp64"),
                     gamma=4.0 / 3.0, variants=None, n=N_GRID):
    """The 256^3 advection batch with the polytropic EoS (Gamma = 4/3, the
    ultra-relativistic gas the paper keeps it for), HLLC and the HLLE-only
    path: cell updates/s of the fused step and the one-period L1 of rho at
    64^3 (the same exact translation as for TM)."""
    out = {"workload": f"{n}^3 periodic advection (as the headline) with the polytropic EoS, "
                       f"Gamma = {gamma:g}", "gamma": gamma, "runs": {}}
    for prec in precs:
        for riemann in ("hllc", "hlle"):
            ctx = srhd.Context(srhd.Params(eos="polytropic", gamma=gamma, riemann=riemann))
            G, dt_dh = build_workload(torch, srhd, ctx, prec, n)
            total_ms, per, dt_next, smax = time_device(torch, ctx, G, dt_dh, steps, warmup,
                                                       lambda: None, prec)
            cells = G.shape[0] * CELLS_PER_PATCH
            r = {"value": cells * steps / (total_ms * 1e-3), "unit": UNIT,
                 "ms_per_step": total_ms / steps, "patch_status_max": smax}
            if abs(gamma - 4.0 / 3.0) < 1e-12:
                r["roofline"] = alu_roofline(FLOPS_PER_CELL_UPDATE_POLY, cells,
                                             statistics.mean(per), prec)
            if riemann == "hllc":
                r["l1_rho_64"], _ = l1_one_period(torch, srhd, prec, params=srhd.Params(
                    eos="polytropic", gamma=gamma))
            out["runs"][f"{prec}_{riemann}"] = r
            del G, dt_dh
            torch.cuda.empty_cache()
    return out


def bench_vl(torch, srhd, steps: int, warmup: int, precs=("mixed_cf", "fp64"), n=N_GRID):
    """The 256^3 advection batch advanced with the VL integrator (14^3 tiles,
    three ghost cells): cell updates/s of srhd_advance_patches_vl and the
    one-period L1 of rho at 64^3."""
    out = {"workload": f"{n}^3 periodic advection (as the headline), VL integrator, "
                       f"{(n // 8) ** 3} patches of 8^3 + 3 ghost cells", "runs": {}}
    for prec in precs:
        ctx = srhd.Context(srhd.Params())
        G, dt_dh = build_workload(torch, srhd, ctx, prec, n, ghost=3)
        total_ms, per, dt_next, smax = time_device(torch, ctx, G, dt_dh, steps, warmup,
                                                   lambda: None, prec, vl=True)
        cells = G.shape[0] * CELLS_PER_PATCH
        r = {"value": cells * steps / (total_ms * 1e-3), "unit": UNIT,
             "ms_per_step": total_ms / steps, "patch_status_max": smax,
             "roofline": alu_roofline(FLOPS_PER_CELL_UPDATE_VL, cells, statistics.mean(per), prec)}
        r["l1_rho_64"], _ = l1_one_period(torch, srhd, prec, vl=True)
        out["runs"][prec] = r
        del G, dt_dh
        torch.cuda.empty_cache()
    return out


def bench_jet(torch, srhd, steps: int, gammas=(10.0, 20.0, 50.0, 100.0),
              precs=("mixed_cf", "fp64"), variants=None):
    """Relativistic jet on a static 4-level AMR hierarchy (configuration 5):
    [0,1] x [0,1] x [0,2], base 64 x 64 x 128 cells (8 x 8 x 16 patches),
    levels 1-3 refined around the beam and cocoon, finest-equivalent
    512 x 512 x 1024; beam radius 16 finest cells injected through z = 0
    with Lorentz factor gamma, density contrast 1e-3, T_jet = 10 into a cold
    static ambient (T = 1e-6); outflow elsewhere; dt_l = 0.4 dh_l. Every
    coarse step: per level substep ghost fill + update, then restriction and
    coarse-fine flux correction (amr.AmrRun), as one CUDA graph. Reports,
    over the same `steps` coarse steps from the same initial state, cell
    updates/s of the update launches alone (CUDA events around them, eager
    steps), of the whole eager step and of the whole step replayed from the
    graph, the cells whose flux correction was skipped (Section 3.3 (4)), and
    the L1 difference of rho between each float run and the FP64 run after
    `steps` steps."""
    from paper_2012_11130_gb300 import amr, workloads
    base, dh0 = (8, 8, 16), 1.0 / 64
    lev = workloads.jet_hierarchy(base=base)
    inflow = dict(axis=2, side=0, center=(32.0, 32.0), radius=2.0, index=0)
    h = amr.Hierarchy(base, lev, bc=("outflow",) * 3, inflow=inflow, prolong="linear")
    c64 = srhd.Context(srhd.Params())
    out = {"workload": ("relativistic jet, [0,1]x[0,1]x[0,2], base 64x64x128, 4 levels of 8^3 "
                        "patches (finest-equivalent 512x512x1024) refined around beam and "
                        "cocoon; beam radius 16 finest cells through z = 0, density contrast "
                        "1e-3, T_jet = 10, ambient T = 1e-6; ghost fill (limited linear "
                        "prolongation with the primitive-variable fallback), restriction and "
                        "flux correction (skipped on cells it leaves unphysical) on the GPU; "
                        "one CUDA graph per coarse step"),
           "patches_per_level": h.counts, "patches": h.ntotal,
           "cell_updates_per_coarse_step": None, "coarse_steps": steps, "runs": {}}
    dev = torch.device("cuda")
    for g in gammas:
        amb, jet = workloads.jet_states(gamma_jet=g)
        Ca = c64.prim2con(torch.tensor(amb, dtype=torch.float64, device=dev).reshape(5, 1))
        Cj = c64.prim2con(torch.tensor(jet, dtype=torch.float64, device=dev).reshape(5, 1))
        finals = {}
        for prec in precs:
            dt = torch.float64 if prec == "fp64" else torch.float32
            C0 = Ca[:, 0].reshape(1, 5, 1, 1, 1).expand(h.ntotal, 5, 8, 8, 8).to(dt).contiguous()
            v = (variants or {}).get(prec, 0)
            ctx = srhd.Context(srhd.Params(patch_variant=v))
            run = amr.AmrRun(ctx, h, C0, dh0, prec=prec, special=Cj.t().to(dt))
            out["cell_updates_per_coarse_step"] = run.cell_updates_per_step
            start = (run.cur.clone(), run.prev.clone())

            def restore():
                run.cur.copy_(start[0])
                run.prev.copy_(start[1])
                run.status.zero_()
                run.skipped.zero_()
                run.prolong_fallbacks.zero_()
            run.step()                      # warm-up (one coarse step), then the initial state
            torch.cuda.synchronize()
            restore()
            # eager: `steps` coarse steps, CUDA events around every update launch
            run.timer = []
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                run.step()
            e1.record()
            torch.cuda.synchronize()
            upd_ms = sum(a.elapsed_time(b) for a, b in run.timer) / steps
            eager_ms = e0.elapsed_time(e1) / steps
            run.timer = None
            st = run.status.cpu()
            skipped = int(run.skipped.item())
            fallbacks = int(run.prolong_fallbacks.item())
            eager_final = run.cur.clone()
            # graph replay of the same `steps` coarse steps from the same
            # initial state (float paths; the FP64 step is long enough that
            # launch overhead does not matter)
            graph_ms = graph_equal = None
            if prec != "fp64":
                restore()
                run.capture(warmup=0)
                e0.record()
                for _ in range(steps):
                    run.replay()
                e1.record()
                torch.cuda.synchronize()
                graph_ms = e0.elapsed_time(e1) / steps
                graph_equal = bool(torch.equal(run.cur, eager_final))
            del eager_final
            upd = run.cell_updates_per_step
            out["runs"][f"{prec}_gamma{g:g}"] = {
                "cell_updates_per_s_update_only": upd / (upd_ms * 1e-3),
                "cell_updates_per_s_whole_step": upd / ((graph_ms or eager_ms) * 1e-3),
                "ms_update_per_coarse_step": upd_ms, "ms_whole_step_graph": graph_ms,
                "ms_whole_step_eager": eager_ms, "graph_equals_eager": graph_equal,
                "timed_steps": f"the same {steps} coarse steps for all three figures",
                "patches_unphysical": int(((st >> 8) & 1).sum()),
                "patches_retried_last_step": int(((st & 255) > 0).sum()),
                "flux_corrections_skipped": skipped,
                "prolongation_primitive_fallbacks": fallbacks,
            }
            o, n = h.offsets[0], h.counts[0]
            lo, ln = h.offsets[-1], h.counts[-1]
            finals[prec] = (run.cur[o:o + n].to(torch.float64).clone(),
                            run.cur[lo:lo + ln].to(torch.float64).clone())
            del run, C0
            torch.cuda.empty_cache()
        if "fp64" in finals:
            def rho(C):
                return c64.con2pri(C.permute(1, 0, 2, 3, 4).reshape(5, -1).contiguous())[0]
            r0, r3 = rho(finals["fp64"][0]), rho(finals["fp64"][1])
            for prec in precs:
                if prec == "fp64":
                    continue
                q0, q3 = rho(finals[prec][0]), rho(finals[prec][1])
                out["runs"][f"{prec}_gamma{g:g}"]["l1_rho_vs_fp64"] = {
                    "level0": float((1 - q0 / r0).abs().mean()),
                    "finest": float((1 - q3 / r3).abs().mean())}
    return out


def bench_con2pri_stress(torch, srhd, prec: str, log2n: int = 26, reps: int = 5):
    """The con2pri stress batch (2^26 cells; rho 1e-6..1e2, T 1e-8..1e4,
    gamma 1..1e6, random direction): cells/s of srhd_con2pri and the
    round-trip error |1 - htilde0/htilde2| of prim -> cons -> prim, maximum
    over the cells whose conditioning 1 + Mach^2 keeps it meaningful
    (kappa eps_A <= 1e-3) and binned by Mach number."""
    from paper_2012_11130_gb300 import workloads
    n = 1 << log2n
    ctx = srhd.Context(srhd.Params())
    W = workloads.stress_batch_prims_torch(n, seed=12345)           # float64 on the device
    dtype = torch.float64 if prec == "fp64" else torch.float32
    C = ctx.prim2con(W).to(dtype)                                   # FP64 conversion, then stored
    P = torch.empty_like(C)
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.con2pri(C, P, st, prec=prec)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        ctx.con2pri(C, P, st, prec=prec)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    T0 = W[4] / W[0]
    ht = lambda T: 2.5 * T + 2.25 * T * T / (1 + torch.sqrt(2.25 * T * T + 1))  # Eq. T_to_HTilde
    Pd = P.double()
    err = (1 - ht(T0) / ht(Pd[4] / Pd[0])).abs()
    h0 = 1 + ht(T0)
    cs2 = T0 * (5 * h0 - 8 * T0) / (3 * h0 * (h0 - T0))               # Eq. sound_speed
    mach2 = (W[1] ** 2 + W[2] ** 2 + W[3] ** 2) / (cs2 / (1 - cs2))
    eps_a = 2.2e-16 if prec != "mixed_cf" else 2.3e-13
    ok = (st == 0) & ((1 + mach2) * eps_a <= 1e-3)
    if prec != "fp64":  # float storage: the stored state itself is exact only to float
        ok = ok & ((1 + mach2) * 6e-8 <= 1e-3)
    bins = {}
    lm = 0.5 * torch.log10(mach2.clamp(min=1e-30))
    for lo in range(-4, 10, 2):
        sel = ok & (lm >= lo) & (lm < lo + 2)
        if int(sel.sum()) > 0:
            bins[f"1e{lo}..1e{lo + 2}"] = float(err[sel].max())
    accepted = int((st == 0).sum())
    out = {"cells": n, "cells_per_s": n / (ms * 1e-3), "ms": ms,
           "unphysical_fraction": float((st == 1).double().mean()),
           "accepted_cells": accepted,
           "cells_per_s_accepted": accepted / (ms * 1e-3),
           "accepted_note": ("cells the conversion returns as physical (status 0); the others "
                             "fail Eq. (Unphysical result) on their stored state: rounding the "
                             "conserved state to the storage type perturbs A by about "
                             "(1 + Mach^2) eps of that type, which in float storage reaches A "
                             "itself for cold gas moving relativistically"),
           "max_roundtrip_error_by_mach": bins}
    del W, C, P, st, Pd, err, T0, h0, cs2, mach2, lm, ok
    torch.cuda.empty_cache()
    return out


def shock_tube_l1(torch, srhd, prec: str, n: int = 1024):
    """Configuration 1 on the GPU: the 1-D shock tube to t = 0.4 (1024 cells,
    (1, 0, 1e3) | (1, 0, 1e-2), PLM + MUSCL-Hancock + HLLC, CFL 0.5, outflow)
    as 128 x 1 x 1 patches; returns the number of steps. The L1 error against
    the exact solution is computed by the caller."""
    from paper_2012_11130_gb300 import workloads
    W, x = workloads.shock_tube_prims(n)
    ctx = srhd.Context(srhd.Params(ndim=1))
    Wd = torch.from_numpy(W).to("cuda")
    C = ctx.prim2con(Wd).reshape(5, 1, 1, n).expand(5, 8, 8, n)
    npx = n // 8
    dtype = torch.float64 if prec == "fp64" else torch.float32
    U = C.reshape(5, 8, 8, npx, 8).permute(3, 0, 1, 2, 4).to(dtype).contiguous()
    dh = 1.0 / n
    dd = torch.empty((npx, 2), dtype=torch.float64, device="cuda")
    dn = torch.empty(1, dtype=torch.float64, device="cuda")
    out = torch.empty_like(U)
    dt = ctx.cfl_dt(U, dh, prec=prec).item()
    t, steps = 0.0, 0
    while t < 0.4 and steps < 100000:
        dt = min(dt, 0.4 - t)
        dd[:, 0] = dt
        dd[:, 1] = dh
        G = ctx.fill_ghosts_uniform(U, npx, 1, 1, bc=("outflow", "periodic", "periodic"))
        ctx.advance_patches(G, dd, cons_out=out, dt_next=dn, prec=prec)
        U, out = out, U
        t += dt
        steps += 1
        dt = dn.item()
    row = U[:, :, 0, 0, :].permute(1, 0, 2).reshape(5, n).contiguous()
    rho = ctx.con2pri(row, prec=prec)[0].double().cpu().numpy()
    return rho, x, steps


def bench_mixed_limits(torch, srhd, prec: str = "mixed_cf", schemes=("reduced", "total"),
                       n: int = 102400, t_end: float = 80.0, chunk: int = 2048,
                       max_seconds: float = 600.0):
    """The mixed-limits Riemann problem of Section 4.2.2 on the paper's grid
    (Table "tb:IC_RiemannProblems", second row: (rho, U, p) = (1e2, 1e-3,
    1e-4) | (1e-12, -1e2, 1e-10) at x = 5e-2; 102 400 cells of [0, 100];
    t = 80; single precision as in the paper), once per scheme: the paper's
    reduced energy and the original total energy. A row of 8 x 8 patches
    along y and z carries the 1-D problem (periodic y and z, outflow x); each
    step is one srhd_advance_uniform launch whose fused CFL bound (the 1-D
    signal speed, CFL 0.5) gives the next time step on the device, clipped
    to t_end there, so the host synchronises only every `chunk` steps. The
    exact solution at the cell centres is tests/golden/mixed_limits_cells_t80.txt
    (the cold state, the fan, the left plateau and the contact) and, beyond
    x = 0.3, its right plateau up to the shock and the right state. Reports
    per scheme the L1 error of rho (Eq. relative L1 error) between the head
    of the rarefaction and the initial discontinuity, where the paper
    measures 23 % for the original scheme, and over the whole fan, the mean
    density error of the shocked right plateau (a domain-wide relative L1
    would be set by the few smeared cells of the contact, across which the
    density jumps by 4e10), the largest pressure error of the cold left
    state, the shock position and its width in cells, and the time taken.
    A run stops early, with the time it reached, after max_seconds or once a
    patch's input is unphysical (the status code CODE_BAD_INPUT)."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", "mixed_limits_cells_t80.txt")
    cells = np.loadtxt(path)
    keys = {}
    for line in open(path):
        if line.startswith("# key "):
            k, v = line[6:].split("=")
            keys[k.strip()] = float(v)
    length = 100.0
    dh = length / n
    npx = n // 8
    x = (np.arange(n) + 0.5) * dh
    m = cells.shape[0]
    rho_ex = np.where(x < keys["x_shock"], keys["rho_right_plateau"], 1e-12)
    rho_ex[:m] = cells[:, 1]
    left = x < 5e-2
    W = np.zeros((5, n))
    W[0] = np.where(left, 1e2, 1e-12)
    W[1] = np.where(left, 1e-3, -1e2)
    W[4] = np.where(left, 1e-4, 1e-10)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    region = (x > 2.67e-2) & (x < 5e-2)   # rarefaction head .. initial discontinuity
    cold = x < 2e-2                        # the undisturbed cold left state
    fan = (x > 2.67e-2) & (x < 0.2093)     # the whole rarefaction fan
    plateau = (x > 0.3) & (x < keys["x_shock"] - 0.1)  # shocked right plateau
    res = {"workload": "mixed-limits Riemann problem (Section 4.2.2): (1e2, 1e-3, 1e-4) | "
                       "(1e-12, -1e2, 1e-10) at x = 5e-2, 102400 cells of [0,100] as 12800 "
                       "patches of 8^3 (y, z uniform), t = 80, CFL 0.5, outflow",
           "precision": prec, "runs": {}}
    for scheme in schemes:
        ctx = srhd.Context(srhd.Params(ndim=1, scheme=scheme))
        C = ctx.prim2con(torch.from_numpy(W).to("cuda")).reshape(5, 1, 1, n).expand(5, 8, 8, n)
        U = C.reshape(5, 8, 8, npx, 8).permute(3, 0, 1, 2, 4).to(dtype).contiguous()
        V = torch.empty_like(U)
        dd = torch.empty((npx, 2), dtype=torch.float64, device="cuda")
        dd[:, 1] = dh
        dn = ctx.cfl_dt(U, dh, prec=prec).reshape(1).to(torch.float64)
        st = torch.empty(npx, dtype=torch.int32, device="cuda")
        t = torch.zeros(1, dtype=torch.float64, device="cuda")
        nsteps = torch.zeros(1, dtype=torch.int64, device="cuda")
        # largest patch status seen (code << 8 | retries) and the sum of all
        # statuses (the retries while no code is set)
        worst = torch.zeros((), dtype=torch.int32, device="cuda")
        ssum = torch.zeros((), dtype=torch.int64, device="cuda")
        bc = ("outflow", "periodic", "periodic")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        while True:
            for _ in range(chunk):
                dtv = torch.minimum(dn, t_end - t)
                dd[:, 0] = dtv
                t += dtv
                nsteps += dtv > 0
                ctx.advance_uniform(U, npx, 1, 1, dd, bc=bc, cons_out=V, dt_next=dn,
                                    patch_status=st, prec=prec)
                torch.maximum(worst, st.max(), out=worst)
                ssum += st.sum()
                U, V = V, U
            tn, wn = t.item(), int(worst.item())
            secs = time.perf_counter() - t0
            print(f"mixed limits {scheme}: t = {tn:.4f}, {int(nsteps.item())} steps, "
                  f"status max {wn:#x}, {secs:.0f} s", file=sys.stderr, flush=True)
            if tn >= t_end or (wn >> 8) & 2 or secs > max_seconds:
                break
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        row = U[:, :, 0, 0, :].permute(1, 0, 2).reshape(5, n).contiguous()
        P = ctx.con2pri(row, prec=prec).double().cpu().numpy()
        rho, p = P[0], P[4]
        err = np.abs(1.0 - rho / rho_ex)
        steps = int(nsteps.item())
        # shock: cells between 10 % and 90 % of the jump from the right state
        # to the right plateau, around the exact position
        lo, hi = 1e-12, keys["rho_right_plateau"]
        near = np.abs(x - keys["x_shock"]) < 0.05
        frac = (rho[near] - lo) / (hi - lo)
        mid = x[near][np.argmin(np.abs(frac - 0.5))]
        res["runs"][scheme] = {
            "t_reached": float(t.item()), "steps": steps, "seconds": secs,
            "cell_updates_per_s_1d": n * steps / secs,
            "cell_updates_per_s_kernel": 64 * n * steps / secs,
            "l1_rho_rarefaction_head_to_x0": float(np.mean(err[region])),
            "cells_in_that_region": int(region.sum()),
            "l1_rho_fan": float(np.mean(err[fan])),
            "mean_rel_err_rho_right_plateau": float(np.mean(err[plateau])),
            "max_rel_err_p_cold_left_state": float(np.max(np.abs(p[cold] / 1e-4 - 1))),
            "shock_x_half_jump": float(mid), "shock_x_exact": keys["x_shock"],
            "shock_width_cells_10_90": int(np.sum((frac > 0.1) & (frac < 0.9))),
            "retries": int(ssum.item()) if int(worst.item()) < 256 else None,
            "worst_status_code": int(worst.item()) >> 8}
        del U, V, C
        torch.cuda.empty_cache()
    return res


# ---------------------------------------------------------------------------
# CPU oracle baseline (host cores)
# ---------------------------------------------------------------------------
def _oracle_chunk(args):
    start, count = args
    import numpy as np
    from oracle import oracle as O
    from paper_2012_11130_gb300 import workloads
    idx = np.arange(start, start + count)
    Wp = workloads.advection_ghosted_patch_prims(N_GRID, idx)
    C, _ = O.prim2con(Wp.transpose(1, 0, 2, 3, 4).reshape(5, -1))
    C = C.reshape(5, count, 12, 12, 12).transpose(1, 0, 2, 3, 4).copy()
    dh = 1.0 / N_GRID
    dt_dh = np.tile([0.4 * dh, dh], (count, 1))
    t = time.perf_counter()
    r = O.advance_patches(C, dt_dh)
    for q in range(count):
        O.cfl_dt(r["out"][q].reshape(5, -1), dh)  # the fused CFL of the step
    return time.perf_counter() - t


class OracleSampler:
    """Times the FP64 oracle on bounded samples of the workload's patches,
    spread over a persistent pool of spawned processes (one per host core)."""

    def __init__(self, cores: int):
        import multiprocessing as mp
        from oracle import oracle as O
        O.build()
        self.cores = cores
        self.pool = mp.get_context("spawn").Pool(cores)
        self.pool.map(_oracle_chunk, [(c, 1) for c in range(cores)])  # import + warm
        self.per_patch = max(_oracle_chunk((0, 8)) / 8, 1e-5)

    def sample(self, npatch_total: int, target_s: float, offset: int = 0):
        """Returns (cells/s, patches, wall seconds) of one sample."""
        per_core = max(1, int(target_s / self.per_patch))
        span = max(1, npatch_total - per_core)
        chunks = [((offset + c * per_core) % span, per_core) for c in range(self.cores)]
        t = time.perf_counter()
        self.pool.map(_oracle_chunk, chunks)
        wall = time.perf_counter() - t
        n = per_core * self.cores
        return n * CELLS_PER_PATCH / wall, n, wall

    def close(self):
        self.pool.close()
        self.pool.join()


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    npatch = (N_GRID // 8) ** 3
    per_step = max(2.0, min(8.0, 150.0 / max(1, args.steps + args.warmup)))
    sampler = OracleSampler(cores)
    for w in range(args.warmup):
        sampler.sample(npatch, per_step / 4, offset=97 * w)
    walls, ns = [], []
    for s in range(args.steps):
        _, n, wall = sampler.sample(npatch, per_step, offset=1013 * (s + 1))
        walls.append(wall)
        ns.append(n)
    sampler.close()
    value = sum(ns) * CELLS_PER_PATCH / sum(walls)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(walls) / len(walls), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "reference": "FP64 CPU oracle (the paper's method "
                   "restated, test infrastructure), host cores", "sample_patches_per_step":
                   int(statistics.median(ns))},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{int(statistics.median(ns))} of 32768 patches per step "
                                   f"(one step each with CFL, FP64, {cores} spawned processes)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        barrier = lambda: dist.barrier(device_ids=[local])  # noqa: E731
    else:
        torch.cuda.set_device(0)
        barrier = lambda: None  # noqa: E731
    from paper_2012_11130_gb300 import build as b
    if rank == 0 or world == 1:
        b.build()
    if world > 1:
        barrier()
    from paper_2012_11130_gb300 import srhd
    ctx = srhd.Context(srhd.Params())
    npatch = (args.grid // 8) ** 3
    cells = npatch * CELLS_PER_PATCH
    peaks = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6789.3))
    sha = kernel_sources_sha()

    results = {}
    precs = ("mixed_cf", "mixed", "fp64") if args.prec == "all" else (args.prec,)
    from paper_2012_11130_gb300 import autotune
    for prec in precs:
        G, dt_dh = build_workload(torch, srhd, ctx, prec, args.grid)
        torch.cuda.synchronize()
        tuned = None
        if args.variant is not None:
            ctx = srhd.Context(srhd.Params(patch_variant=args.variant))
            tuned = {"chosen_variant": args.variant, "ms_per_variant": None,
                     "tile": TILE_SHAPE}
        elif not args.no_tune:
            best, times = autotune.tune(G, dt_dh, prec=prec, steps=2 if prec == "fp64" else 3)
            ctx = srhd.Context(best)
            tuned = {"chosen_variant": best.patch_variant,
                     "ms_per_variant": {str(k): v for k, v in times.items()},
                     "tile": TILE_SHAPE}
        else:
            ctx = srhd.Context(srhd.Params())
        with ClockSampler(local) as clk:
            total_ms, per, dt_next, smax = time_device(torch, ctx, G, dt_dh, args.steps,
                                                       args.warmup, barrier, prec)
        clocks = clk.summary()
        value, total_ms = job_throughput(total_ms, cells, args.steps, device="cuda")
        loop = None
        if not args.no_loop:
            loop = {}
            for cached in (True, False):
                lt, lper, ldn, lsmax = time_uniform_loop(torch, ctx, G, dt_dh, args.steps,
                                                         args.warmup, barrier, prec, cached)
                lv, lt = job_throughput(lt, cells, args.steps, device="cuda")
                loop["cached" if cached else "uncached"] = {
                    "value": lv, "ms_per_step": lt / args.steps,
                    "launch_ms_mean": statistics.mean(lper), "dt_next": ldn,
                    "patch_status_max": lsmax,
                    "api": ("srhd_advance_uniform_prim (primitive cache)" if cached
                            else "srhd_advance_uniform")}
        e2e = None
        if not args.no_e2e:
            # five times the device steps in the float paths (about 0.26 s): a
            # rare slow host step (10-20 ms) then moves the mean by a few per
            # cent instead of a quarter
            ne = max(3, args.steps if prec == "fp64" else 5 * args.steps)
            secs, eper, h2d, d2h = time_e2e(torch, ctx, G, dt_dh, ne, max(3, args.warmup), prec)
            med = statistics.median(eper)
            e2e = {"value": world * cells * ne / secs, "unit": UNIT,
                   "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                   "steps": ne, "ms_per_step_median": 1e3 * med,
                   "ms_per_step_min": 1e3 * min(eper), "ms_per_step_max": 1e3 * max(eper),
                   "steps_over_twice_median": sum(1 for x in eper if x > 2 * med),
                   "value_at_median_step": world * cells / statistics.median(eper),
                   "link": measure_link(torch, h2d), "numa": host_numa(),
                   "api": "srhd_advance_uniform_host (interiors in pinned host memory)"}
            if prec == precs[0]:
                secs, h2d, d2h = time_e2e_ghosted(torch, ctx, G, dt_dh, 3, 1, prec)
                e2e["ghosted_batch"] = {
                    "value": world * cells * 3 / secs, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "api": "srhd_advance_patches on host tensors (12^3 ghosted tiles in)"}
        launch_ms = statistics.mean(per)
        flops = FLOPS_PER_CELL_UPDATE * cells
        peak_alu = PEAK_FP64_TFLOPS if prec == "fp64" else PEAK_FP32_TFLOPS
        achieved = flops / (launch_ms * 1e-3) / 1e12
        traffic = NCU_TRAFFIC.get(prec) if NCU_TRAFFIC.get("sources_sha") == sha else None
        alg_bytes = BYTES_PER_CELL_UPDATE[prec] * cells
        results[prec] = {
            "value": value,
            "ms_per_step": total_ms / args.steps,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_alu,
                         "unit": "TFLOP/s", "frac": achieved / peak_alu, "traffic": traffic,
                         "peak_source": ("nominal GB300 FP64 1.25 TFLOP/s" if prec == "fp64" else
                                         "derived: 152 SM x 128 FP32 lanes x 2 x 2070 MHz"),
                         "flops_per_cell_update": FLOPS_PER_CELL_UPDATE},
            "hbm_roofline": {"bound": "hbm", "achieved": alg_bytes / (launch_ms * 1e-3) / 1e9,
                             "peak": hbm_peak, "unit": "GB/s",
                             "frac": alg_bytes / (launch_ms * 1e-3) / 1e9 / hbm_peak,
                             "bytes_per_cell_update": BYTES_PER_CELL_UPDATE[prec],
                             "halo_bytes_per_cell_update": HALO_BYTES_PER_CELL_UPDATE[prec],
                             "halo_frac": (HALO_BYTES_PER_CELL_UPDATE[prec] * cells
                                           / (launch_ms * 1e-3) / 1e9 / hbm_peak),
                             "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"},
            "clocks": clocks, "e2e": e2e, "dt_next": dt_next, "patch_status_max": smax,
            "autotune": tuned,
            "launch_ms_mean": launch_ms, "launch_ms_min": min(per),
            "uniform_loop": loop,
        }
        del G, dt_dh
        torch.cuda.empty_cache()

    amr_res = None
    if not args.no_amr and args.grid == N_GRID:
        amr_res = bench_amr(torch, srhd, max(3, args.steps // 4), 2, precs[0] if precs[0] != "fp64"
                            else "mixed_cf")

    poly_res = None
    if not args.no_poly and rank == 0:
        poly_res = bench_polytropic(torch, srhd, max(3, args.steps // 2), 3,
                                    precs=tuple(q for q in ("mixed_cf", "fp64") if q in precs),
                                    n=args.grid)

    ml_res = None
    if args.mixed_limits and rank == 0:
        ml_res = bench_mixed_limits(torch, srhd)

    vl_res = None
    if not args.no_vl and rank == 0:
        vl_res = bench_vl(torch, srhd, max(3, args.steps // 2), 3,
                          precs=tuple(q for q in ("mixed_cf", "fp64") if q in precs), n=args.grid)

    jet_res = None
    if not args.no_jet and args.grid == N_GRID and rank == 0:
        vs = {q: results[q]["autotune"]["chosen_variant"] for q in precs
              if results[q].get("autotune")}
        jet_res = bench_jet(torch, srhd, args.jet_steps, variants=vs,
                            gammas=tuple(float(g) for g in args.jet_gammas.split(",")),
                            precs=tuple(q for q in ("mixed_cf", "fp64") if q in precs))

    l1 = {}
    l1_conv = {}
    stress = {}
    if not args.no_l1 and rank == 0:
        for prec in precs:
            # configuration 3: one period at 64^3, 128^3 and 256^3 (about 35 s
            # of the FP64 path at 256^3)
            runs = {}
            for n in (64, 128, 256):
                e, nsteps, drift = l1_one_period(torch, srhd, prec, n=n, with_drift=True)
                runs[str(n)] = {"l1_rho": e, "steps": nsteps, "conservation_drift": drift}
            ns = sorted(runs, key=int)
            l1_conv[prec] = {"runs": runs, "order": [
                math.log2(runs[a]["l1_rho"] / runs[b]["l1_rho"]) for a, b in zip(ns, ns[1:])]}
            l1[prec] = runs["64"]["l1_rho"]
        l1["grid"] = "64^3, one period, fused CFL 0.5"
        for prec in precs:
            stress[prec] = bench_con2pri_stress(torch, srhd, prec)

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0

    cpu = None
    if world == 1 and not args.no_cpu:
        sampler = OracleSampler(os.cpu_count() or 1)
        v, n, wall = sampler.sample(npatch, args.cpu_seconds)
        sampler.close()
        cpu = {"value": v, "unit": UNIT, "cores": os.cpu_count() or 1, "kind": "oracle",
               "sample": f"{n} of 32768 patches (one FP64 oracle step each, with CFL), "
                         f"{os.cpu_count()} spawned processes, {wall:.1f} s",
               "value_1core": 8 * CELLS_PER_PATCH / _oracle_chunk((0, 8))}
    st_l1 = None
    if rank == 0 and not args.no_l1:
        # configuration 1: shock-tube L1 of rho against the exact TM solution
        # (stored by tests/golden/make_shock_tube_exact.py), per precision
        import numpy as np
        ex = np.loadtxt(os.path.join(ROOT, "tests", "golden", "shock_tube_exact_1024.txt"))
        st_l1 = {}
        for prec in precs:
            rho, x, steps = shock_tube_l1(torch, srhd, prec)
            st_l1[prec] = float(np.mean(np.abs(1 - rho / ex[:, 1])))
        st_l1["steps"] = steps
        st_l1["grid"] = "1024 cells, t = 0.4, CFL 0.5"
    m = results[precs[0]]
    line = {
        "metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"mixed_cf": "f32", "mixed": "f32+f64", "fp64": "f64"}[precs[0]],
        "data": "synthetic",
        "config": {"workload": WORKLOAD if args.grid == N_GRID else
                   WORKLOAD.replace("256^3", f"{args.grid}^3").replace("32768", str(npatch)),
                   "cells": cells, "patches": npatch,
                   "precision": {"mixed_cf": "mixed_cf: float storage and arithmetic, con2pri A "
                                             "by error-free float products + compensated sum",
                                 "mixed": "mixed: float storage/arithmetic, con2pri A in double",
                                 "fp64": "fp64"}[precs[0]],
                   "l2": "inputs larger than L2 (ghosted batch resident in HBM), no flush",
                   "parallelism": f"replicas x{world}"},
        "roofline": m["roofline"], "hbm_roofline": m["hbm_roofline"],
        "clocks": m["clocks"], "e2e": m["e2e"], "cpu_baseline": cpu,
        "gpu_launches": 2 * args.steps,
        "autotune": m["autotune"],
        "uniform_loop": m["uniform_loop"],
        "other_precisions": {q: {k: results[q][k] for k in ("value", "ms_per_step", "roofline",
                                                             "hbm_roofline", "clocks", "e2e",
                                                             "autotune", "uniform_loop")}
                             for q in precs[1:]} or None,
        "l1_rho": l1 or None,
        "l1_convergence": l1_conv or None,
        "l1_shock_tube": st_l1,
        "con2pri_stress": stress or None,
        "amr_blast": amr_res,
        "amr_jet": jet_res,
        "polytropic": poly_res,
        "vl": vl_res,
        "mixed_limits": ml_res,
        "kernel_sources_sha": sha,
    }
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-loop", action="store_true",
                    help="skip the uniform-grid time loops (cached and uncached primitives)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-l1", action="store_true")
    ap.add_argument("--no-amr", action="store_true")
    ap.add_argument("--no-jet", action="store_true", help="skip the AMR jet (configuration 5)")
    ap.add_argument("--no-poly", action="store_true", help="skip the polytropic-EoS workload")
    ap.add_argument("--no-vl", action="store_true", help="skip the VL-integrator workload")
    ap.add_argument("--jet-steps", type=int, default=100, help="coarse steps of each jet run")
    ap.add_argument("--jet-gammas", default="10,20,50,100",
                    help="comma-separated beam Lorentz factors of the jet runs")
    ap.add_argument("--mixed-limits", action="store_true",
                    help="also run the mixed-limits Riemann problem of Section 4.2.2 on the "
                         "paper's 102400-cell grid to t = 80, both schemes (a few minutes)")
    ap.add_argument("--no-tune", action="store_true", help="skip the launch-variant autotuner")
    ap.add_argument("--variant", type=int, default=None,
                    help="use this launch variant of the patch kernel (no autotuning)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--grid", type=int, default=N_GRID,
                    help="cells per axis of the advection grid (multiple of 8)")
    ap.add_argument("--prec", choices=["all", "mixed_cf", "mixed", "fp64"], default="all")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)  # at least 3 untimed warm-up steps
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
