#!/usr/bin/env python
"""Throughput of the fused RK3 MHD substep on GB300, in Gcell-updates/s per substep.

A step is one pass of the whole hot path over the synthetic state: the
forcing draw and its phase tables, the three fused RHS + Runge-Kutta substeps
(sixth-order stencils with the periodic map applied on load) and the max
CFL speed of the step's input state (folded into substep 0, read back each
step).  Default workload: 256^3 periodic, FP64, forced at
|k| = 2-3 with a seeded phase each step, noise of amplitude 1e-5 on u and A,
nu = eta = 5e-3, c_s = 1, gamma = 5/3, dt = 1e-3.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on the
host cores instead (a bounded sample of the same workload per step).
Multi-GPU (torchrun): every rank integrates its own replica (weak scaling, no
data-path collective); the elapsed time is the max over ranks.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Gcell-updates/s per RK3 substep"
UNIT = "Gcell-updates/s"

# FP64 flops per cell-substep of the fused formulation (FMA = 2 flops; exp and
# the one division are not counted): 564 in the 54 derivative stencils, 155 in
# the physics of Eqs. B.1-B.4 with forcing, 40 in the Runge-Kutta update
# (24 at substep 0, where w is not read).
FLOPS_PER_CELL = {0: 743, 1: 759, 2: 759}


# The same count at stencil order 2r: a first derivative takes 3r - 1 flops, a
# second 3r + 1, a mixed one 5r - 1, so the 54 stencils take 186 r - 18.
def flops_per_cell(order, s):
    return 186 * (order // 2) - 18 + 24 + 155 + (24 if s == 0 else 40)
# Algorithmic bytes per cell-substep: read f and w, write f and w, eight fields
# each (w not read at s = 0).
def bytes_per_cell(elem_f, elem_w, s):
    return 8 * (2 * elem_f + (2 if s else 1) * elem_w)

# Nominal dense FP64 rate of one GB300 (no measured FP64 peak is provided).
FP64_NOMINAL_TFLOPS = 1.25
# DRAM bytes per cell of one launch of the integer-sum FP64 substep kernel
# (ncu, 128^3, substep-1/2 variant, over 2,097,152 cells): group scales (forced
# noise state) 424.2 MB read + 236.7 MB written, per-field scales (u_z scaled by
# 1e-3) 429.3 + 236.7 MB.
FX_TRAFFIC_PER_CELL = {"group": (424206592 + 236677888) / 2097152,
                       "field": (429260800 + 236704256) / 2097152}
# FP64-pipe thread instructions per cell of that kernel (ncu
# sm__inst_executed_pipe_fp64 x 32 / cells, 128^3 forced; the instruction stream
# does not depend on the grid), per mode: substep-0 (CFL) and substep-1/2 variants.
FX_FP64_PIPE_INST_PER_CELL = {"group": (206.3125, 179.3125), "field": (236.3125, 209.3125)}
# DRAM bytes per cell of one launch of the binary32 tiled substep, the mean over
# substeps 0, 1, 2 (ncu, 256^3 forced, one step: 1970.1 MB read + written per
# launch on average over 16,777,216 cells; algorithmic 96, 128, 128 B/cell)
TILED_TRAFFIC_PER_CELL = 1970099882.7 / 16777216
# The same for one launch of the 64-box ensemble kernel with its tuned split (ncu:
# 3260.7 MB per launch on average over its 27,340,800 cells; 1.6% above the
# algorithmic bytes: the halo cells of small boxes)
BATCH_TRAFFIC_PER_CELL = 3260725930.7 / 27340800

WORKLOADS = {
    "forced256_fp64": dict(n=(256, 256, 256), precision="fp64", force_amp=0.05, seed=2,
                           dt=1e-3, init="noise",
                           desc="256^3 periodic FP64 non-ideal MHD, 6th-order stencils, RK3, "
                                "forced |k|=2-3, noise 1e-5 on u and A"),
    "paper256_fp64": dict(n=(256, 256, 256), precision="fp64", force_amp=0.0, seed=0,
                          dt=1.19209e-7, init="uniform", vs=1.36,
                          desc="256^3 periodic FP64, all fields U[0,1], dt=1.19209e-7 "
                               "(the paper's own benchmark setup, Sec. 5)"),
    "forced512_fp32": dict(n=(512, 512, 512), precision="fp32", force_amp=0.05, seed=3,
                           dt=1e-3, init="noise",
                           desc="512^3 periodic FP32 forced non-ideal MHD (FP64 reductions)"),
    "closure128": dict(n=(128, 128, 128), precision="fp32", force_amp=0.05, seed=5, dt=1e-3,
                       init="turbulent", closure=True,
                       desc="learned closure: 128^3 FP32 coarse grid + 3-layer 3-D conv "
                            "(8-32-32-8, k=3, BF16 weights, FP32 accumulation) applied every "
                            "step, trained on 256^3 FP64 forced runs restricted 2x"),
    "closure_forward256": dict(n=(256, 256, 256), precision="fp32", force_amp=0.0, seed=7,
                               init="turbulent", closure_forward=True,
                               desc="learned-closure inference on a 256^3 FP32 state: input "
                                    "pack, 3-D conv 8-32-32-8 (k=3, circular, BF16 operands, "
                                    "FP32 accumulation, tcgen05) and output scaling"),
    "decomp256_fp64": dict(n=(256, 256, 256), precision="fp64", force_amp=0.05, seed=2,
                           dt=1e-3, init="noise", decomp=(2, 2, 2),
                           desc="256^3 periodic FP64 forced MHD split into 2x2x2 subdomains of "
                                "128^3 with radius-3 halos: pack sides and edges, exchange, "
                                "unpack, outer update, inner update overlapping the exchange "
                                "(Sec. 3.3), all subdomains on one GPU"),
    "ensemble64_fp32": dict(n=None, precision="fp32", force_amp=0.0, seed=4, dt=1e-3,
                            init="noise", ensemble=True,
                            desc="64 periodic boxes, per-axis sizes from {32,48,64,96,128}, "
                                 "nu and eta log-uniform in [1e-3,1e-2] (seed 4), FP32, one "
                                 "persistent launch per substep under a CUDA graph, tuned "
                                 "work items"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="forced256_fp64", choices=sorted(WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--stencil-order", type=int, default=6, choices=[2, 4, 6, 8],
                    help="central-difference order of the substep (the paper's is 6)")
    ap.add_argument("--full-entropy", action="store_true",
                    help="switch on conduction, bulk viscosity, heating and cooling "
                         "(K = zeta = 1e-3, H = 0.02, C = 0.01)")
    ap.add_argument("--closure-pairs", type=int, default=24)
    ap.add_argument("--closure-iters", type=int, default=800)
    ap.add_argument("--closure-rollout", type=int, default=20)
    ap.add_argument("--no-compare", action="store_true",
                    help="ensemble: skip the separate-launch and FP64 comparisons")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--fp64-peak", action="store_true",
                    help="also time a cuBLAS FP64 GEMM as a measured FP64 reference rate")
    ap.add_argument("--grid", type=int, default=0,
                    help="override the cube edge (small cases for profiling)")
    ap.add_argument("--init", default=None, choices=["noise", "uniform", "weak_uz"],
                    help="initial state (default: the workload's); weak_uz: noise with u_z "
                         "scaled by 1e-3 (the integer-sum path then takes per-field scales)")
    ap.add_argument("--no-workloads", action="store_true",
                    help="default workload only: skip the other workloads of the table")
    ap.add_argument("--fp64-compare-steps", type=int, default=0,
                    help="binary32 workloads: steps of a binary64 run from the same state "
                         "for the per-field error")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, bus_id):
        # torch gives the PCI bus number (an int); nvidia-smi prints the full
        # domain:bus:device.function address
        self.bus = bus_id if isinstance(bus_id, int) else None
        self.lines = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        rows, addrs = {}, set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 10:
                continue
            try:
                row = (float(parts[2]), float(parts[3]), parts[6:10])
                bus = int(parts[1].split(":")[-2], 16)
            except (IndexError, ValueError):
                continue
            addrs.add(parts[1])
            rows.setdefault(bus, []).append(row)
        if self.bus in rows:
            rows = rows[self.bus]
        elif len(addrs) == 1:  # only this process's GPU is visible
            rows = next(iter(rows.values()))
        else:
            return None
        reasons = sorted({self.NAMES[i] for _, _, r in rows for i in range(4)
                          if r[i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# inputs
# ---------------------------------------------------------------------------
def make_state(wl):
    from paper_2103_01597_gb300 import synthetic
    if wl["init"] == "uniform":
        return synthetic.uniform_state(wl["n"], wl["seed"])
    f = synthetic.noise_state(wl["n"], wl["seed"])
    if wl["init"] == "weak_uz":
        f[3] *= 1e-3
    return f


def dist_setup(args):
    """(world size, rank, local rank) from the launcher's environment (torchrun
    sets WORLD_SIZE, RANK, LOCAL_RANK; a plain launch is rank 0 of 1)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def timed_region_max(elapsed, dist, device):
    """Seconds of the timed region for the whole job: the largest over the ranks
    (the job ends with its slowest rank); unchanged without a process group."""
    if dist is None:
        return elapsed
    import torch
    t = torch.tensor([elapsed], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def pipeline_schedule(ne, H):
    """Order of the end-to-end loop over H handles taking turns: ("issue", j)
    loads step j's input into handle j mod H and queues the step, ("store", j)
    copies its result out and waits for it.  Steps 0 .. H-2 are issued first;
    then each store of step k follows the issue of step k + H - 1, whose handle
    last held step k - 1, already stored."""
    ops = [("issue", j) for j in range(min(H - 1, ne))]
    for k in range(ne):
        if k + H - 1 < ne:
            ops.append(("issue", k + H - 1))
        ops.append(("store", k))
    return ops


def job_rate(units_per_rank, ws, elapsed):
    """Whole-job throughput: the units every rank processed (the same number on
    each replica) over the slowest rank's time."""
    return ws * units_per_rank / elapsed


# ---------------------------------------------------------------------------
# the oracle arm / CPU baseline: a bounded sample of the same workload
# ---------------------------------------------------------------------------
def oracle_sample(wl, f, planes, nthreads=None):
    """One RK3 step (3 substeps) of the oracle at the cells of `planes` z-planes
    of the full-size state (the substeps read the full arrays)."""
    from oracle import core
    nx, ny, nz = wl["n"]
    k, j, i = np.meshgrid(np.arange(planes), np.arange(ny), np.arange(nx), indexing="ij")
    cells = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.int64)
    frc = None
    if wl["force_amp"]:
        fr = core.forcing_draw(wl["seed"], 0, wl["force_amp"])
        frc = fr
    p = core.Params(n=wl["n"], forcing=frc, order=wl.get("order", 6), **wl.get("entropy", {}))
    w = np.zeros_like(f)
    t0 = time.perf_counter()
    for s in range(3):
        core.substep_cells(f, w, p, wl["dt"], s, cells, nthreads=nthreads or os.cpu_count())
    return time.perf_counter() - t0, 3 * cells.shape[0]


def cpu_baseline(wl, f, seconds):
    """The oracle on the host cores, all threads (OpenMP) and one thread, each on
    a slab of z-planes of the workload's state sized for about `seconds`."""
    import oracle
    oracle.build_oracle()
    out = {}
    for nth in (os.cpu_count(), 1):
        planes = 1
        dt, cu = oracle_sample(wl, f, planes, nth)
        planes = max(1, min(wl["n"][2], int(planes * seconds / max(dt, 1e-3))))
        dt, cu = oracle_sample(wl, f, planes, nth)
        out[nth] = {"value": cu / dt / 1e9, "unit": UNIT, "cores": nth, "kind": "oracle",
                    "sample": "one RK3 step (3 substeps) at the %d cells of %d z-planes of the "
                              "%s state, FP64 C oracle, OpenMP over %d thread%s"
                              % (cu // 3, planes, "x".join(map(str, wl["n"])), nth,
                                 "s" if nth > 1 else ""),
                    "seconds": dt}
    line = dict(out[os.cpu_count()])
    line["single_thread"] = out[1]
    return line


def _sample_cells(n, count, seed):
    g = np.random.default_rng(seed)
    return np.stack([g.integers(0, n[0], count), g.integers(0, n[1], count),
                     g.integers(0, n[2], count)], axis=1).astype(np.int64)


def _rel_per_field(g, o):
    return [float(np.max(np.abs(g[q] - o[q])) / np.max(np.abs(o[q])))
            if np.max(np.abs(o[q])) > 0 else float(np.max(np.abs(g[q] - o[q])))
            for q in range(g.shape[0])]


def sampled_parity(sim, wl, order, count=2000):
    """One more RK3 step of the GPU state after the timed region, each substep
    checked against the FP64 oracle at `count` sampled cells (computed from the
    GPU's own input state of that substep): per-field max-norm relative error of
    f and w, and the paper's ulp metric on f."""
    from oracle import core
    from paper_2103_01597_gb300 import ac
    n = wl["n"]
    cells = _sample_cells(n, count, 11)
    idx = (cells[:, 2], cells[:, 1], cells[:, 0])
    step, _ = ac.ac_get_step(sim.h)
    forcing = core.forcing_draw(wl["seed"], step, wl["force_amp"]) if wl["force_amp"] else None
    p = core.Params(n=n, forcing=forcing, order=order, **wl.get("entropy", {}))
    f, w = sim.store(), sim.store_w()
    ef, ew, ulp = np.zeros(8), np.zeros(8), 0.0
    for s in range(3):
        fo, wo = core.substep_cells(f, w if s else None, p, wl["dt"], s, cells,
                                    nthreads=os.cpu_count())
        sim.substep(wl["dt"], s)
        f, w = sim.store(), sim.store_w()
        gs = np.stack([f[q][idx] for q in range(8)])
        gw = np.stack([w[q][idx] for q in range(8)])
        ef = np.maximum(ef, _rel_per_field(gs, fo))
        ew = np.maximum(ew, _rel_per_field(gw, wo))
        nz = fo != 0
        e = np.ldexp(1.0, (np.floor(np.log2(np.abs(fo[nz]))) - 52).astype(int))
        ulp = max(ulp, float(np.max(np.abs(gs[nz] - fo[nz]) / e)))
    return {"cells": count, "substeps": 3, "rel_err_f": ef.tolist(), "rel_err_w": ew.tolist(),
            "max_ulp_f": ulp, "bound": 1e-12,
            "how": "substeps 0-2 of the step after the timed region, oracle from the GPU's "
                   "own input state of each substep"}


def fp32_against_fp64(sim, wl, f0, steps, stream):
    """Per-field error of the binary32 state against a binary64 run of the same
    workload from the same initial state after `steps` steps (forcing draws
    identical: both handles restart at step 0)."""
    from paper_2103_01597_gb300 import ac
    ref = ac.Simulation(wl["n"], precision=ac.AC_FP64, force_amp=wl["force_amp"],
                        seed=wl["seed"], stream=stream.cuda_stream)
    ref.load(f0)
    sim.load(f0)
    ac.ac_set_step(sim.h, 0, 0)
    for _ in range(steps):
        ref.step(wl["dt"])
        sim.step(wl["dt"])
    r = ref.store()
    modes = ac.ac_get_stencil_modes(ref.h)
    ref.close()
    g = sim.store()
    return {"steps": steps, "rel_err_per_field": _rel_per_field(g, r),
            "fields": ["lnrho", "ux", "uy", "uz", "ss", "ax", "ay", "az"],
            "fp64_stencil_modes": list(modes),
            "how": "max|f32 - f64| / max|f64| per field after the same steps from the same "
                   "state (binary64 run: the default integer-sum path)"}


def run_reference(args, wl):
    ws, rank, _ = dist_setup(args)
    if rank != 0:
        return 0
    import oracle
    oracle.build_oracle()
    f = make_state(wl)
    nx, ny, _ = wl["n"]
    planes = max(1, int(2e5 // (nx * ny)) + 1)
    for _ in range(args.warmup):
        oracle_sample(wl, f, planes)
    tot, cu = 0.0, 0
    for _ in range(args.steps):
        dt, c = oracle_sample(wl, f, planes)
        tot += dt
        cu += c
    value = cu / tot / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["desc"], "grid": list(wl["n"]),
                       "sample_per_step": "%d z-planes (%d cells) x 3 substeps"
                                          % (planes, planes * nx * ny)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": "per step: one RK3 step at the cells of %d z-planes"
                                       % planes},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def fp64_dgemm_tflops(torch):
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    for _ in range(2):
        torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    del a, b
    return 2 * n ** 3 / best / 1e12


def host_link_gbs(host):
    """Rate of one copy of the pinned host buffer `host` to the device and back (GB/s,
    best of three each way, CUDA events on the current stream): the bound that the
    machine's host link puts on the end-to-end figures.  `host` is overwritten with
    its own contents."""
    import torch
    flat = host.view(-1)
    dev = torch.empty_like(flat, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    nb = flat.numel() * flat.element_size()
    best = [0.0, 0.0]
    for _ in range(3):
        ev[0].record()
        dev.copy_(flat, non_blocking=True)
        ev[1].record()
        flat.copy_(dev, non_blocking=True)
        ev[2].record()
        ev[2].synchronize()
        best[0] = max(best[0], nb / ev[0].elapsed_time(ev[1]) / 1e6)
        best[1] = max(best[1], nb / ev[1].elapsed_time(ev[2]) / 1e6)
    del dev
    return {"h2d_gbs": round(best[0], 1), "d2h_gbs": round(best[1], 1), "bytes": nb}


def run_ours(args, wl):
    import torch
    ws, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2103_01597_gb300 import ac, build
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    prec = {"fp64": ac.AC_FP64, "fp32": ac.AC_FP32, "fp32_w64": ac.AC_FP32_W64}[wl["precision"]]
    elem_f = 8 if prec == ac.AC_FP64 else 4
    elem_w = 4 if prec == ac.AC_FP32 else 8
    n = wl["n"]
    ncell = n[0] * n[1] * n[2]
    stream = torch.cuda.current_stream()
    order = wl.get("order", 6)
    sim = ac.Simulation(n, precision=prec, force_amp=wl["force_amp"], seed=wl["seed"],
                        device="cuda:%d" % local, stream=stream.cuda_stream, order=order,
                        **wl.get("entropy", {}))
    f0 = make_state(wl)
    host_in = torch.from_numpy(f0.reshape(-1)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    ac.ac_load(sim.h, ac.AC_ALL, host_in)
    dt = wl["dt"]

    def step(ev=None):
        for s in range(3):
            if ev is not None:
                ev[s][0].record(stream)
            ac.ac_integrate_substep(sim.h, dt, s)
            if ev is not None:
                ev[s][1].record(stream)
        # max CFL speed of the step's input state, computed inside substep 0
        return ac.ac_last_cfl(sim.h)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    bus = None
    try:
        bus = torch.cuda.get_device_properties(local).pci_bus_id
    except Exception:
        bus = None
    sampler = ClockSampler(bus) if rank == 0 else None
    time.sleep(0.3 if sampler else 0)
    evs = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(3)]
           for _ in range(args.steps)]
    launches0 = ac.ac_launch_count(sim.h)
    modes0 = ac.ac_get_stencil_modes(sim.h)
    # CUDA events around the substep kernel itself (and its preparation kernels),
    # recorded by the library on its stream over the timed region
    ac.ac_set_kernel_timing(sim.h, True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    cfl = 0.0
    for it in range(args.steps):
        cfl = step(evs[it])
    t1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    elapsed = t0.elapsed_time(t1) / 1e3
    launches = ac.ac_launch_count(sim.h) - launches0
    prep_ms, kern_ms, _ = ac.ac_kernel_timings(sim.h)
    ac.ac_set_kernel_timing(sim.h, False)
    clocks = sampler.stop() if sampler else None
    elapsed = timed_region_max(elapsed, dist, "cuda")
    per_sub = [[evs[it][s][0].elapsed_time(evs[it][s][1]) / 1e3 for it in range(args.steps)]
               for s in range(3)]
    value = job_rate(ncell * 3 * args.steps, ws, elapsed) / 1e9

    # per substep index: the whole substep (all its launches) and the substep
    # kernel alone (the dominant kernel: library events around its launch)
    avg = {s: statistics.mean(per_sub[s]) for s in range(3)}
    kern = {s: kern_ms[s] / 1e3 for s in range(3)}
    avg_all = statistics.mean(kern.values())
    modes = [m1 - m0 for m0, m1 in zip(modes0, ac.ac_get_stencil_modes(sim.h))]
    if wl["precision"] == "fp64":
        flops = {s: flops_per_cell(order, s) * ncell for s in range(3)}
        equiv = statistics.mean(flops[s] / kern[s] for s in range(3)) / 1e12
        dg = fp64_dgemm_tflops(torch) if (rank == 0 and args.fp64_peak) else None
        fixed = ac.ac_get_stencil_path(sim.h)
        # measured denominator: the library's DFMA-chain probe (2 flops per FMA)
        dfma = ac.ac_diag_fma_rate(ac.AC_FP64, stream.cuda_stream)
        peak = 2 * dfma / 1e12
        # the count per cell weighted by the modes the timed substeps ran (none
        # for plain binary64 stencils, which this table does not cover)
        inst = None
        traffic = None
        if fixed and order == 6 and sum(modes) and not modes[2] and not wl.get("entropy"):
            fg = modes[0] / sum(modes)
            G, F = FX_FP64_PIPE_INST_PER_CELL["group"], FX_FP64_PIPE_INST_PER_CELL["field"]
            inst = [fg * G[v] + (1 - fg) * F[v] for v in range(2)]
            traffic = (fg * FX_TRAFFIC_PER_CELL["group"] +
                       (1 - fg) * FX_TRAFFIC_PER_CELL["field"]) * ncell
        achieved = None
        if inst is not None:
            # FP64-pipe thread instructions of each launch, as DFMA-equivalent flops
            achieved = statistics.mean(2 * inst[min(s, 1)] * ncell / kern[s]
                                       for s in range(3)) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved is not None else None,
                "what": "FP64 pipe: FP64-pipe thread instructions per launch (ncu count per "
                        "cell x cells) x 2 flops / CUDA-event launch time, against the "
                        "measured DFMA rate",
                "fp64_pipe_inst_per_cell": inst,
                "peak_source": "measured: ac_diag_fma_rate(AC_FP64), the library's own DFMA "
                               "chains, x 2 flops (nominal: %.2f TFLOP/s)" % FP64_NOMINAL_TFLOPS,
                # dram read + write per launch of the substep-1/2 variant, from the
                # 128^3 ncu captures of the same kernels scaled by cells, weighted by
                # the modes the timed substeps ran
                "traffic": traffic,
                "kernel": ("fx_stats + fx_plan + fx_quantize + substep_fx_kernel (int64 "
                           "stencil sums)" if fixed else
                           "substep_kernel<double,double,IdxPeriodicR<%d>>" % (order // 2)),
                "prep_ms": {str(s): prep_ms[s] for s in range(3)},
                "method_flops_equiv": {
                    "achieved": equiv, "frac_of_peak": equiv / peak,
                    "alg_flops_per_cell_substep": {s: flops_per_cell(order, s)
                                                   for s in range(3)},
                    "note": ("the method's binary64 flops per cell-substep over the launch "
                             "time; on the integer-sum path the 540 stencil flops run as "
                             "exact int64 operations on the integer pipes, so this rate can "
                             "exceed the FP64 peak" if fixed else
                             "all arithmetic on the FP64 pipe")},
                "fp64_dgemm_measured_tflops": dg,
                "fma_peaks_tflops": {"fp64": peak,
                                     "fp32": 2 * ac.ac_diag_fma_rate(ac.AC_FP32,
                                                                     stream.cuda_stream) / 1e12},
                "avg_launch_ms": 1e3 * avg_all}
    else:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        bytes_s = {s: bytes_per_cell(elem_f, elem_w, s) * ncell for s in range(3)}
        achieved = statistics.mean(bytes_s[s] / kern[s] for s in range(3)) / 1e9
        tiled = order == 6 and not wl.get("entropy")
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"],
                # dram read + write per launch, mean over the three substeps (ncu at
                # 256^3, scaled by cells)
                "traffic": TILED_TRAFFIC_PER_CELL * ncell if tiled else None,
                "kernel": ("substep_tiled_kernel<float,true> (shared-memory plane ring)"
                           if order == 6 else
                           "substep_kernel<float,float,IdxPeriodicR<%d>>" % (order // 2)),
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)",
                "avg_launch_ms": 1e3 * avg_all}

    roof["kernel_ms"] = {str(s): 1e3 * kern[s] for s in range(3)}

    # end to end through the C ABI with host buffers: every step loads its whole
    # input state from pinned host memory and stores its whole result, in the
    # state's own precision (binary64 through ac_load / ac_store, binary32
    # through ac_load_f32 / ac_store_f32)
    e2e = None
    if args.e2e_steps > 0:
        ne = max(16, args.e2e_steps)  # the first load and the last store are not overlapped
        hb = elem_f  # host bytes per value
        if hb == 4:
            e_in = torch.from_numpy(f0.reshape(-1).astype(np.float32)).pin_memory()
            load, store = ac.ac_load_f32, ac.ac_store_f32
        else:
            e_in = host_in
            load, store = ac.ac_load, ac.ac_store
        # H handles on H streams take turns; up to H - 1 steps are queued ahead of
        # the store being waited on, so a short stall of the host thread does not
        # leave the GPU idle
        H = 3
        outs = [torch.empty_like(e_in).pin_memory() for _ in range(H)]
        e_out = outs[0]
        link = host_link_gbs(e_out)
        streams = [stream] + [torch.cuda.Stream(device=local) for _ in range(H - 1)]
        sims = [sim] + [ac.Simulation(n, precision=prec, force_amp=wl["force_amp"],
                                      seed=wl["seed"], device="cuda:%d" % local,
                                      stream=st.cuda_stream, order=order, **wl.get("entropy", {}))
                        for st in streams[1:]]
        h2d = 8 * ncell * hb
        d2h = 8 * ncell * hb + 16
        # untimed warm-up of the host side: the first copies through freshly pinned
        # pages run several times slower than the later ones on these machines
        for _ in range(max(3, args.warmup)):
            for hs, hout in zip(sims, outs):
                load(hs.h, ac.AC_ALL, e_in)
                ac.ac_integrate_step(hs.h, dt)
                store(hs.h, ac.AC_ALL, hout)
        torch.cuda.synchronize()
        # (a) one handle, serially: load -> step (+ CFL read) -> store
        phase = [[], []]  # per step: load + step + CFL read (host sync), store
        tt0 = time.perf_counter()
        for _ in range(ne):
            ta = time.perf_counter()
            load(sim.h, ac.AC_ALL, e_in)
            step()
            tb = time.perf_counter()
            store(sim.h, ac.AC_ALL, e_out)
            phase[0].append(tb - ta)
            phase[1].append(time.perf_counter() - tb)
        serial = ncell * 3 * ne * ws / (time.perf_counter() - tt0) / 1e9
        # (b) the handles take turns: step j runs on handle j mod H, loads its whole
        # input and stores its whole result; it waits on an event recorded after
        # step j - 1, so two steps never share the SMs and only the copies run
        # beside a step
        done = [torch.cuda.Event() for _ in range(H)]

        def issue(j):
            hs, st = sims[j % H], streams[j % H]
            load(hs.h, ac.AC_ALL, e_in)
            if j > 0:
                st.wait_event(done[(j - 1) % H])
            ac.ac_integrate_step(hs.h, dt)
            done[j % H].record(st)

        torch.cuda.synchronize()
        t_store = []
        tt0 = time.perf_counter()
        for op, j in pipeline_schedule(ne, H):
            if op == "issue":
                issue(j)
            else:
                store(sims[j % H].h, ac.AC_ALL, outs[j % H])
                t_store.append(time.perf_counter())
        tt = time.perf_counter() - tt0
        torch.cuda.synchronize()
        for hs in sims[1:]:
            hs.close()
        gaps = [b2 - a2 for a2, b2 in zip(t_store, t_store[1:])]
        e2e = {"value": ncell * 3 * ne * ws / tt / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h - 16, "steps": ne,
               "warmup": max(3, args.warmup),
               "host_format": "binary32" if hb == 4 else "binary64",
               "how": "%d handles on %d streams take turns (load, ac_integrate_step, store "
                      "each step); each step waits on an event after the previous one, and "
                      "the copies of the others overlap a step" % (H, H),
               "ms_between_stores": {"median": 1e3 * statistics.median(gaps),
                                     "max": 1e3 * max(gaps)} if gaps else None,
               "serial_one_handle": {"value": serial, "d2h_bytes_per_step": d2h,
                                     "how": "load, three ac_integrate_substep calls, CFL read, store "
                                            "in sequence",
                                     "median_ms": {
                                         "load_step_cfl": 1e3 * statistics.median(phase[0]),
                                         "store": 1e3 * statistics.median(phase[1])},
                                     "max_ms": {"load_step_cfl": 1e3 * max(phase[0]),
                                                "store": 1e3 * max(phase[1])}},
               "host_link": link}

    parity = None
    fp32_err = None
    if rank == 0 and ws == 1:
        if wl["precision"] == "fp64":
            parity = sampled_parity(sim, wl, order)
        elif args.fp64_compare_steps > 0:
            fp32_err = fp32_against_fp64(sim, wl, f0, args.fp64_compare_steps, stream)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, f0, args.cpu_seconds)
    sim.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": (value / ws / wl["vs"]) if "vs" in wl else None,
                "dtype": "f64" if wl["precision"] == "fp64" else "f32", "data": "synthetic",
                "config": {"workload": wl["desc"], "grid": list(n), "dt": dt,
                           "precision": wl["precision"], "layout": "periodic (wrap on load)",
                           "stencil_order": order,
                           "entropy_terms": wl.get("entropy"),
                           "parallelism": "replicas" if ws > 1 else "single GPU",
                           "l2": "inputs larger than L2 (%.1f GB of state resident)"
                                 % (ncell * (16 * elem_f + 8 * elem_w) / 1e9),
                           "step": "forcing draw + 3 fused substeps (substep 0 also reduces the "
                                   "max CFL speed) + 8-byte read of that max"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clocks,
                "stencil_modes": ({"group_scales": modes[0], "field_scales": modes[1],
                                   "plain_binary64": modes[2]} if sum(modes) else None),
                "parity_sampled": parity, "fp32_vs_fp64": fp32_err,
                "last_cfl_speed": cfl,
                "substep_ms": {str(s): 1e3 * avg[s] for s in range(3)}}
    if dist:
        dist.destroy_process_group()
    return line if rank == 0 else None


def run_ensemble(args, wl):
    """The batched ensemble: aggregate throughput of the graph-captured
    persistent launch, beside 64 separate binary32 and binary64 launches and the
    per-field binary32 error against binary64 after a few steps."""
    import torch
    from paper_2103_01597_gb300 import ac, build, synthetic
    ws, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    spec = synthetic.ensemble(wl["seed"])
    boxes = [(n, (2 * math.pi,) * 3, nu, eta) for n, nu, eta in spec]
    ncell = sum(n[0] * n[1] * n[2] for n, _, _, _ in boxes)
    states = [synthetic.noise_state(n, 100 + i) for i, (n, _, _, _) in enumerate(boxes)]
    stream = torch.cuda.current_stream()
    b = ac.Batch(boxes, stream=stream.cuda_stream)
    for i, f in enumerate(states):
        b.load(i, f)
    dt = wl["dt"]
    zc = ac.ac_batch_tune(b.b, dt)
    _, shapes, tune_ms = ac.ac_batch_get_tiling(b.b, len(boxes))
    cls16 = sorted({tuple(n[:2]) for (n, _, _, _), sh in zip(boxes, shapes) if sh == ac.AC_TILE_16X16})
    tuning = {"item_z_extent": zc,
              "boxes_per_tile_shape": {"32x8": shapes.count(ac.AC_TILE_32X8),
                                       "16x16": shapes.count(ac.AC_TILE_16X16)},
              "classes_on_16x16_(nx,ny)": [list(c) for c in cls16],
              "step_ms_default_split": tune_ms[0], "step_ms_tuned": tune_ms[1],
              "gain": tune_ms[0] / tune_ms[1] if tune_ms[1] > 0 else None,
              "note": "whole steps (3 substeps) timed by ac_batch_tune from the same state; "
                      "default split = z extent 64, every box on 32x8 tiles"}
    ac.ac_batch_set_graph(b.b, True)
    for _ in range(args.warmup):
        b.step(dt)
    torch.cuda.synchronize()
    bus = None
    try:
        bus = torch.cuda.get_device_properties(local).pci_bus_id
    except Exception:
        pass
    sampler = ClockSampler(bus) if rank == 0 else None
    time.sleep(0.3 if sampler else 0)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    l0 = ac.ac_batch_info(b.b)["launches"]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for it in range(args.steps):
        evs[it][0].record(stream)
        b.step(dt)
        evs[it][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    elapsed = t0.elapsed_time(t1) / 1e3
    launches = ac.ac_batch_info(b.b)["launches"] - l0
    clocks = sampler.stop() if sampler else None
    elapsed = timed_region_max(elapsed, dist, "cuda")
    value = job_rate(ncell * 3 * args.steps, ws, elapsed) / 1e9
    step_s = statistics.mean(e[0].elapsed_time(e[1]) / 1e3 for e in evs)
    launch_s = step_s / 3
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    alg = statistics.mean(bytes_per_cell(4, 4, s) for s in range(3)) * ncell
    achieved = alg / launch_s / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"],
            # dram read + write per launch, mean over the three substeps (ncu)
            "traffic": BATCH_TRAFFIC_PER_CELL * ncell,
            "kernel": "batch_substep_kernel<float> (persistent, graph-captured)",
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)",
            "avg_launch_ms": 1e3 * launch_s}

    # 64 separate launches per substep: binary32 and binary64 single-box handles.
    def separate(precision, steps=2):
        sims = []
        for i, (n, L, nu, eta) in enumerate(boxes):
            sim = ac.Simulation(n, L=L, precision=precision, nu=nu, eta=eta,
                                stream=stream.cuda_stream)
            sim.load(states[i])
            sims.append(sim)
        for sim in sims:
            sim.step(dt)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            for s in range(3):
                for sim in sims:
                    sim.substep(dt, s)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        return sims, ncell * 3 * steps / t / 1e9

    compare = {}
    err = None
    if rank == 0 and not args.no_compare:
        s32, v32 = separate(ac.AC_FP32)
        for sim in s32:
            sim.close()
        s64, v64 = separate(ac.AC_FP64)
        compare = {"separate_fp32_launches_gcell_s": v32, "separate_fp64_launches_gcell_s": v64,
                   "speedup_vs_separate_fp32": value / ws / v32,
                   "speedup_vs_separate_fp64": value / ws / v64}
        # binary32 batch vs binary64 handles after the same number of steps from the same state
        nsteps = 5
        for sim in s64:
            sim.close()
        bb = ac.Batch(boxes, stream=stream.cuda_stream)
        errs = np.zeros(8)
        for i, f in enumerate(states):
            bb.load(i, f)
        for _ in range(nsteps):
            bb.step(dt)
        for i, (n, L, nu, eta) in enumerate(boxes):
            sim = ac.Simulation(n, L=L, precision=ac.AC_FP64, nu=nu, eta=eta,
                                stream=stream.cuda_stream)
            sim.load(states[i])
            for _ in range(nsteps):
                sim.step(dt)
            r = sim.store()
            g = bb.store(i)
            sim.close()
            for q in range(8):
                den = np.max(np.abs(r[q]))
                errs[q] = max(errs[q], np.max(np.abs(g[q] - r[q])) / den if den else 0.0)
        bb.close()
        err = {"steps": nsteps, "max_over_boxes_rel_err_per_field": errs.tolist()}

    e2e = None
    if args.e2e_steps > 0:
        torch.cuda.synchronize()
        # the boxes' binary32 states in binary32 host buffers (one copy per box each way)
        ins = [torch.from_numpy(f.reshape(-1).astype(np.float32)).pin_memory() for f in states]
        outs = [torch.empty_like(t).pin_memory() for t in ins]
        outs2 = [torch.empty_like(t).pin_memory() for t in ins]
        link = host_link_gbs(outs[int(np.argmax([t.numel() for t in outs]))])
        # a second ensemble with the same boxes and split, on its own stream
        s2 = torch.cuda.Stream(device=local)
        b2 = ac.Batch(boxes, stream=s2.cuda_stream)
        ac.ac_batch_set_tiling(b2.b, zc, shapes)
        ac.ac_batch_set_graph(b2.b, True)
        pairs = [(b, outs), (b2, outs2)]
        ne = max(8, args.e2e_steps)

        def load_all(bb):
            for i, t in enumerate(ins):
                ac.ac_batch_load_f32(bb.b, i, ac.AC_ALL, t)

        def store_all(bb, hout):
            for i in range(len(boxes)):
                ac.ac_batch_store_f32(bb.b, i, ac.AC_ALL, hout[i])

        for _ in range(max(3, args.warmup)):  # untimed: first copies through new pinned pages
            for bb, hout in pairs:
                load_all(bb)
                bb.step(dt)
                store_all(bb, hout)
        torch.cuda.synchronize()
        # (a) one ensemble: load every box, step, store every box, in sequence
        tt0 = time.perf_counter()
        for _ in range(ne):
            load_all(b)
            b.step(dt)
            store_all(b, outs)
        serial = ncell * 3 * ne * ws / (time.perf_counter() - tt0) / 1e9
        # (b) the two ensembles take alternate steps; each step waits on an event
        # after the previous one, so only the copies run beside a step
        streams = [stream, s2]
        done = [torch.cuda.Event(), torch.cuda.Event()]
        torch.cuda.synchronize()
        tt0 = time.perf_counter()
        load_all(b)
        b.step(dt)
        for k in range(ne):
            cur, hout = pairs[k % 2]
            if k + 1 < ne:
                nxt = pairs[(k + 1) % 2][0]
                load_all(nxt)
                done[k % 2].record(streams[k % 2])
                streams[(k + 1) % 2].wait_event(done[k % 2])
                nxt.step(dt)
            store_all(cur, hout)
        tt = time.perf_counter() - tt0
        torch.cuda.synchronize()
        b2.close()
        e2e = {"value": ncell * 3 * ne * ws / tt / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": 8 * ncell * 4, "d2h_bytes_per_step": 8 * ncell * 4,
               "host_format": "binary32", "steps": ne, "warmup": max(3, args.warmup),
               "how": "two ensembles on two streams take alternate steps (64 box loads, "
                      "ac_batch_integrate_step, 64 box stores each); each step waits on an "
                      "event after the previous one, and one ensemble's copies overlap the "
                      "other's step",
               "serial_one_batch": {"value": serial}, "host_link": link}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        n0 = boxes[0][0]
        wl0 = dict(wl, n=n0, force_amp=0.0)
        cpu = cpu_baseline(wl0, states[0], args.cpu_seconds)
        cpu["sample"] += " (box 0 of the ensemble)"
    b.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": wl["desc"], "boxes": len(boxes), "cells": ncell,
                           "dt": dt, "tuned_item_z_extent": zc, "tuning": tuning,
                           "parallelism": "replicas" if ws > 1 else "single GPU",
                           "l2": "inputs larger than L2 (%.1f GB of state resident)"
                                 % (ncell * 24 * 4 / 1e9),
                           "step": "3 persistent substep launches (graph replay)"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks, "compare": compare, "fp32_vs_fp64": err}
    if dist:
        dist.destroy_process_group()
    return line if rank == 0 else None


def _spectra(f, n):
    """Kinetic (u) and magnetic (B = curl A, spectral) shell spectra on the host."""
    from oracle import closure as oc
    u = f[1:4]
    A = f[5:8]
    k = [np.fft.fftfreq(m, 1.0 / m) for m in (n[2], n[1], n[0])]
    KZ, KY, KX = np.meshgrid(*k, indexing="ij")
    Ah = [np.fft.fftn(A[a]) for a in range(3)]
    Bh = [1j * (KY * Ah[2] - KZ * Ah[1]), 1j * (KZ * Ah[0] - KX * Ah[2]),
          1j * (KX * Ah[1] - KY * Ah[0])]
    B = np.array([np.real(np.fft.ifftn(b)) for b in Bh])
    return oc.energy_spectrum(u), oc.energy_spectrum(B)


def run_closure(args, wl):
    """Coarse 128^3 FP32 grid with the learned closure applied every step."""
    import torch
    from paper_2103_01597_gb300 import ac, build, synthetic
    from paper_2103_01597_gb300 import closure as cl
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    nc = wl["n"]
    nf = tuple(2 * v for v in nc)
    cells = nc[0] * nc[1] * nc[2]
    dtf = wl["dt"]
    t0 = time.perf_counter()
    f0 = synthetic.turbulent_state(nf, wl["seed"], kmax=48, amp=0.3)
    npairs = args.closure_pairs
    pairs = cl.make_pairs(f0, nf, npairs + 4, dtf, seed=wl["seed"], force_amp=wl["force_amp"])
    t_data = time.perf_counter() - t0
    train, held = pairs[:npairs], pairs[npairs:]
    ins = cl.channel_rms([p[0] for p in train])
    outs = cl.channel_rms([p[1] for p in train])
    c = cl.Closure(nc, seed=wl["seed"])
    c.set_scales(ins, outs)
    base = float(np.mean([c.loss(x, t) for x, t in held]))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for it in range(args.closure_iters):
        x, t = train[it % len(train)]
        c.train_step(x, t, lr=2e-3 if it < 0.7 * args.closure_iters else 5e-4)
    e1.record(stream)
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1) / args.closure_iters
    after = float(np.mean([c.loss(x, t) for x, t in held]))
    defect = []
    for x, t in held:
        corr = c.correction(x)
        defect.append(float(torch.linalg.vector_norm(t - corr) / torch.linalg.vector_norm(t)))
    # the backward pass alone (forward, loss, input and weight gradients; no host
    # sync, parameters unchanged) on each convolution path
    lib = ac.load_library()
    bx, bt = ac._ptr8(cl._rows(held[0][0])), ac._ptr8(cl._rows(held[0][1]))
    bwd_ms = {}
    for path, name in ((ac.AC_CONV_MMA_SYNC, "mma_sync"), (ac.AC_CONV_TCGEN05_PAIR, "tcgen05_pair"),
                       (ac.AC_CONV_TCGEN05, "tcgen05")):
        ac.ac_closure_set_conv_path(c.c, path)
        for _ in range(2):
            assert lib.ac_closure_backward(c.c, bx, bt, None) == 0
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(10):
            lib.ac_closure_backward(c.c, bx, bt, None)
        e1.record(stream)
        torch.cuda.synchronize()
        bwd_ms[name] = e0.elapsed_time(e1) / 10
    c.status()

    # timed region: coarse steps with the closure applied after each step
    sim = ac.Simulation(nc, precision=ac.AC_FP32, force_amp=wl["force_amp"], seed=wl["seed"])
    cl.current_state(sim).copy_(held[0][0])
    for _ in range(args.warmup):
        sim.step(2 * dtf)
        c.apply(sim, 1e3)
    torch.cuda.synchronize()
    conv_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    ta, tb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = ac.ac_launch_count(sim.h) + ac.ac_closure_launch_count(c.c)
    lib = ac.load_library()
    bus = None
    try:
        bus = torch.cuda.get_device_properties(0).pci_bus_id
    except Exception:
        pass
    sampler = ClockSampler(bus)
    time.sleep(0.3)
    ta.record(stream)
    for it in range(args.steps):
        sim.step(2 * dtf)
        rc = lib.ac_closure_apply(c.c, sim.h, 1e3, None)  # forward + guard + add, no host sync
        assert rc == 0, ac.ac_strerror(rc)
    tb.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    elapsed = ta.elapsed_time(tb) / 1e3
    launches = ac.ac_launch_count(sim.h) + ac.ac_closure_launch_count(c.c) - l0
    # end to end through the public calls with host binary32 buffers (the coarse
    # state's own precision): load the coarse state, step, apply the guarded
    # closure, store the state
    hstate = torch.from_numpy(sim.store().reshape(-1).astype(np.float32)).pin_memory()
    hout = torch.empty_like(hstate).pin_memory()
    ne = max(2, args.e2e_steps)
    link = host_link_gbs(hout)

    def e2e_step():
        ac.ac_load_f32(sim.h, ac.AC_ALL, hstate)
        sim.step(2 * dtf)
        rc = lib.ac_closure_apply(c.c, sim.h, 1e3, None)
        assert rc == 0, ac.ac_strerror(rc)
        ac.ac_store_f32(sim.h, ac.AC_ALL, hout)

    for _ in range(3):  # untimed: first copies through new pinned pages
        e2e_step()
    torch.cuda.synchronize()
    tt0 = time.perf_counter()
    for _ in range(ne):
        e2e_step()
    tt = time.perf_counter() - tt0
    e2e = {"value": cells * 3 * ne / tt / 1e9, "unit": UNIT,
           "h2d_bytes_per_step": 8 * cells * 4, "d2h_bytes_per_step": 8 * cells * 4,
           "host_format": "binary32", "steps": ne, "warmup": 3, "host_link": link}
    # the forward pass (input pack + three convolution launches), timed alone on
    # the same state, on both convolution paths
    xs = cl._rows(cl.current_state(sim))
    fwd_s = {}
    for path, name in ((ac.AC_CONV_MMA_SYNC, "mma_sync"), (ac.AC_CONV_TCGEN05_PAIR, "tcgen05_pair"),
                       (ac.AC_CONV_TCGEN05, "tcgen05")):
        ac.ac_closure_set_conv_path(c.c, path)
        for it in range(args.steps):
            conv_ev[it][0].record(stream)
            ac.ac_closure_forward(c.c, xs, None)
            conv_ev[it][1].record(stream)
        torch.cuda.synchronize()
        fwd_s[name] = statistics.mean(e[0].elapsed_time(e[1]) for e in conv_ev) / 1e3
    c.status()
    conv_s = fwd_s["tcgen05"]
    value = cells * 3 * args.steps / elapsed / 1e9
    flops = 2 * 27 * (8 * 32 + 32 * 32 + 32 * 8) * cells
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    roof = {"bound": "tensor", "achieved": flops / conv_s / 1e12, "peak": peaks["bf16_tflops"],
            "unit": "TFLOP/s", "frac": flops / conv_s / 1e12 / peaks["bf16_tflops"],
            "traffic": None,
            "kernel": "conv_tc_kernel x3 (closure forward, tcgen05.mma BF16, TMEM accumulator)",
            "peak_source": "measured (MEASURED_PEAKS.json bf16_tflops, burst)",
            "avg_launch_ms": 1e3 * conv_s / 3,
            "forward_ms": {k: 1e3 * v for k, v in fwd_s.items()},
            "note": "algorithmic flops (8 real input and output channels)"}

    # spectra after M coarse steps: plain, with closure, and the restricted fine run
    M = args.closure_rollout
    fine = ac.Simulation(nf, precision=ac.AC_FP64, force_amp=wl["force_amp"], seed=wl["seed"])
    fine.load(f0)
    plain = ac.Simulation(nc, precision=ac.AC_FP32, force_amp=wl["force_amp"], seed=wl["seed"])
    corr = ac.Simulation(nc, precision=ac.AC_FP32, force_amp=wl["force_amp"], seed=wl["seed"])
    x0 = torch.empty((8, cells), dtype=torch.float32, device="cuda")
    fptrs, _, _, _ = ac.ac_get_state(fine.h)
    ac.ac_restrict(fptrs, ac.AC_FP64, nf, cl._rows(x0))
    cl.current_state(plain).copy_(x0)
    cl.current_state(corr).copy_(x0)
    applied = 0
    for m in range(M):
        frc = ac.ac_forcing_draw(wl["seed"], 1000 + m)
        for sm in (fine, plain, corr):
            ac.ac_set_forcing(sm.h, *frc)
        fine.step(dtf)
        fine.step(dtf)
        plain.step(2 * dtf)
        corr.step(2 * dtf)
        applied += int(c.apply(corr, 1e3))
    ref = torch.empty((8, cells), dtype=torch.float32, device="cuda")
    fptrs, _, _, _ = ac.ac_get_state(fine.h)
    ac.ac_restrict(fptrs, ac.AC_FP64, nf, cl._rows(ref))
    shape = (8, nc[2], nc[1], nc[0])
    R = ref.double().cpu().numpy().reshape(shape)
    P = cl.current_state(plain).double().cpu().numpy().reshape(shape)
    C = cl.current_state(corr).double().cpu().numpy().reshape(shape)
    kmax = nc[0] // 3
    def dist(a, b):
        return float(np.sqrt(np.sum((np.log(a[1:kmax]) - np.log(b[1:kmax])) ** 2) / (kmax - 1)))
    eR, mR = _spectra(R, nc)
    eP, mP = _spectra(P, nc)
    eC, mC = _spectra(C, nc)
    state_err = {"plain": float(np.sqrt(np.mean((P - R) ** 2) / np.mean(R ** 2))),
                 "closure": float(np.sqrt(np.mean((C - R) ** 2) / np.mean(R ** 2)))}
    quality = {"rollout_steps": M, "closure_applied": applied,
               "kinetic_log_spectrum_rms_distance": {"plain": dist(eP, eR), "closure": dist(eC, eR)},
               "magnetic_log_spectrum_rms_distance": {"plain": dist(mP, mR), "closure": dist(mC, mR)},
               "state_rel_l2_error_vs_restricted_fine": state_err,
               "heldout_loss_before_after": [base, after],
               "heldout_relative_defect_after": float(np.mean(defect)),
               "train_ms_per_iter": train_ms, "train_iters": args.closure_iters,
               "backward_ms_per_path": bwd_ms,
               "pairs": npairs, "data_gen_s": t_data}
    for sm in (fine, plain, corr, sim):
        sm.close()
    c.close()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16",
            "data": "synthetic",
            "config": {"workload": wl["desc"], "grid": list(nc), "fine_grid": list(nf),
                       "dt_coarse": 2 * dtf,
                       "step": "coarse RK3 step (3 fused substeps) + closure forward "
                               "(3 conv layers) + guarded correction"},
            "roofline": roof, "cpu_baseline": None, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks, "closure": quality}
    return line


# ---------------------------------------------------------------------------
# learned-closure inference
# ---------------------------------------------------------------------------
CF_METRIC = "closure forward throughput"
CF_UNIT = "Gcell/s"
# algorithmic flops per cell of the three layers (real channels: 8 -> 32 -> 32
# -> 8; the tensor cores also multiply padding, which is not counted)
CF_FLOPS = {1: 2 * 27 * 8 * 32, 2: 2 * 27 * 32 * 32, 3: 2 * 27 * 32 * 8}
# algorithmic flops per cell (8 real input channels, 8 real output channels)
CF_ALGO_FLOPS = 2 * 27 * (8 * 32 + 32 * 32 + 32 * 8)
# DRAM bytes per cell of one launch of the 32 -> 32 tcgen05 layer (ncu, 128^3:
# 144.9 MB read + 89.0 MB written over 2,097,152 cells)
CF_TRAFFIC_PER_CELL = (144.937728e6 + 89.045248e6) / 2097152


def _closure_oracle_sample(params, n, seed):
    from oracle import closure as oc
    net = oc.Net.unflat(np.asarray(params, dtype=np.float64))
    x = np.random.default_rng(seed).standard_normal((8, n, n, n))
    t0 = time.perf_counter()
    net.forward(x, bf16="config")
    return time.perf_counter() - t0, n ** 3


def run_closure_forward(args, wl):
    """Inference throughput of the learned closure (ac_closure_forward: input
    pack, three convolution launches, output scaling) on a 256^3 state; the
    dominant kernel is the 32 -> 32 layer."""
    import torch
    from paper_2103_01597_gb300 import ac, build, synthetic
    from paper_2103_01597_gb300 import closure as cl
    ws, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    n = wl["n"]
    cells = n[0] * n[1] * n[2]
    f = synthetic.turbulent_state(n, wl["seed"], kmax=48, amp=0.3).astype(np.float32).reshape(8, -1)
    rms = np.sqrt(np.mean(f.astype(np.float64) ** 2, axis=1))
    ins = np.maximum(rms, 1e-6).astype(np.float32)
    outs = (1e-2 * ins).astype(np.float32)
    stream = torch.cuda.current_stream()
    xs = torch.from_numpy(f).cuda()
    out = torch.empty_like(xs)
    c = cl.Closure(n, seed=wl["seed"], stream=stream.cuda_stream)
    c.set_scales(ins, outs)
    rin, rout = cl._rows(xs), cl._rows(out)
    lib = ac.load_library()
    pin, pout = ac._ptr8(rin), ac._ptr8(rout)
    for _ in range(args.warmup):
        assert lib.ac_closure_forward(c.c, pin, pout) == 0
    torch.cuda.synchronize()
    bus = None
    try:
        bus = torch.cuda.get_device_properties(local).pci_bus_id
    except Exception:
        pass
    sampler = ClockSampler(bus) if rank == 0 else None
    time.sleep(0.3 if sampler else 0)
    l0 = ac.ac_closure_launch_count(c.c)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ta, tb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ta.record(stream)
    for _ in range(args.steps):
        rc = lib.ac_closure_forward(c.c, pin, pout)
        assert rc == 0, ac.ac_strerror(rc)
    tb.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    elapsed = ta.elapsed_time(tb) / 1e3
    clocks = sampler.stop() if sampler else None
    launches = ac.ac_closure_launch_count(c.c) - l0
    c.status()
    elapsed = timed_region_max(elapsed, dist, "cuda")
    value = job_rate(cells * args.steps, ws, elapsed) / 1e9

    # per-launch device times (events around each launch, on the closure's stream)
    per = {}
    for path, name in ((ac.AC_CONV_TCGEN05, "tcgen05"), (ac.AC_CONV_TCGEN05_PAIR, "tcgen05_pair"),
                       (ac.AC_CONV_MMA_SYNC, "mma_sync")):
        ac.ac_closure_set_conv_path(c.c, path)
        ac.ac_closure_forward_timings(c.c, rin, rout)
        rows = [ac.ac_closure_forward_timings(c.c, rin, rout) for _ in range(max(3, args.steps))]
        per[name] = [statistics.mean(r[i] for r in rows) for i in range(5)]
    ac.ac_closure_set_conv_path(c.c, ac.AC_CONV_TCGEN05)
    ms2 = per["tcgen05"][2]
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    ach = CF_FLOPS[2] * cells / (ms2 / 1e3) / 1e12
    layers = {name: {"ms": {k: v for k, v in zip(("pack", "conv1", "conv2", "conv3", "scale"),
                                                 per[name])},
                     "conv_tflops": {"conv%d" % l: CF_FLOPS[l] * cells / (per[name][l] / 1e3) / 1e12
                                     for l in (1, 2, 3)}}
              for name in per}
    roof = {"bound": "tensor", "achieved": ach, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
            "frac": ach / peaks["bf16_tflops"], "traffic": CF_TRAFFIC_PER_CELL * cells,
            "traffic_note": "dram read + write bytes per launch, ncu at 128^3 scaled by cells",
            "kernel": "conv_tc_kernel<32,32> (layer 2, tcgen05.mma BF16, TMEM accumulators)",
            "per_unit": "2*27*32*32 = 55296 flops per cell", "units_per_launch": cells,
            "avg_launch_ms": ms2,
            "peak_source": "measured (MEASURED_PEAKS.json bf16_tflops, burst)",
            "launches": layers}

    # end to end through the public call: every forward copies its whole input
    # state in from pinned host memory and its whole correction out
    hin = torch.from_numpy(f).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ne = max(8, args.e2e_steps)
    link = host_link_gbs(hout)
    for _ in range(3):  # untimed: first copies through new pinned pages
        xs.copy_(hin, non_blocking=True)
        assert lib.ac_closure_forward(c.c, pin, pout) == 0
        hout.copy_(out, non_blocking=True)
    torch.cuda.synchronize()
    # (a) one closure on one stream: copy in, forward, copy out in sequence
    e0.record(stream)
    for _ in range(ne):
        xs.copy_(hin, non_blocking=True)
        assert lib.ac_closure_forward(c.c, pin, pout) == 0
        hout.copy_(out, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    serial = ws * cells * ne / (e0.elapsed_time(e1) / 1e3) / 1e9
    # (b) two closures with their own buffers on two streams take alternate
    # forwards, so that one's copies run while the other computes
    s2 = torch.cuda.Stream()
    c2 = cl.Closure(n, seed=wl["seed"], stream=s2.cuda_stream)
    c2.set_scales(ins, outs)
    with torch.cuda.stream(s2):
        xs2 = torch.empty_like(xs)
        out2 = torch.empty_like(out)
    hout2 = torch.empty_like(hin).pin_memory()
    lanes = [(c, stream, xs, out, pin, pout, hout),
             (c2, s2, xs2, out2, ac._ptr8(cl._rows(xs2)), ac._ptr8(cl._rows(out2)), hout2)]

    fdone = [torch.cuda.Event(), torch.cuda.Event()]

    def lane_step(k):
        # each forward waits on an event after the previous one, so that only the
        # copies run beside a forward
        cc, st, xk, ok, pk_in, pk_out, hk = lanes[k % 2]
        with torch.cuda.stream(st):
            xk.copy_(hin, non_blocking=True)
            if k > 0:
                st.wait_event(fdone[(k - 1) % 2])
            assert lib.ac_closure_forward(cc.c, pk_in, pk_out) == 0
            fdone[k % 2].record(st)
            hk.copy_(ok, non_blocking=True)

    for k in range(6):  # untimed
        lane_step(k)
    torch.cuda.synchronize()
    tt0 = time.perf_counter()
    for k in range(ne):
        lane_step(k)
    torch.cuda.synchronize()
    tt = time.perf_counter() - tt0
    c2.close()
    e2e = {"value": ws * cells * ne / tt / 1e9, "unit": CF_UNIT,
           "h2d_bytes_per_step": 8 * cells * 4, "d2h_bytes_per_step": 8 * cells * 4,
           "steps": ne, "warmup": 3,
           "how": "two closures on two streams take alternate forwards (copy in, "
                  "ac_closure_forward, copy out each); each forward waits on an event after "
                  "the previous one, and one's copies overlap the other's forward",
           "serial_one_stream": {"value": serial}, "host_link": link}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        params = ac.ac_closure_get_params(c.c)
        dt, cu = _closure_oracle_sample(params, 48, 1)
        cpu = {"value": cu / dt / 1e9, "unit": CF_UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": "closure forward of a 48^3 state (numpy FP64 oracle, BF16-rounded "
                         "operands, BLAS threads as numpy sets them)", "seconds": dt}
    c.close()
    if rank == 0:
        line = {"metric": CF_METRIC, "value": value, "unit": CF_UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "bf16 x bf16 -> f32",
                "data": "synthetic",
                "config": {"workload": wl["desc"], "grid": list(n),
                           "parallelism": "replicas" if ws > 1 else "single GPU",
                           "l2": "inputs larger than L2 (state 0.54 GB, each activation "
                                 "0.5-1.1 GB)",
                           "algorithmic_flops_per_cell": CF_ALGO_FLOPS,
                           "step": "one ac_closure_forward (pack + 3 conv + scale)"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks}
    if dist:
        dist.destroy_process_group()
    return line if rank == 0 else None


def run_closure_forward_reference(args, wl):
    """The oracle arm of the closure-inference workload: the numpy FP64 forward
    on a 32^3 sample per step."""
    ws, rank, _ = dist_setup(args)
    if rank != 0:
        return 0
    from paper_2103_01597_gb300 import closure as cl
    params = cl.init_params(wl["seed"])
    for _ in range(args.warmup):
        _closure_oracle_sample(params, 32, 0)
    tot, cu = 0.0, 0
    for i in range(args.steps):
        dt, c = _closure_oracle_sample(params, 32, i)
        tot += dt
        cu += c
    value = cu / tot / 1e9
    line = {"impl": "reference", "metric": CF_METRIC, "value": value, "unit": CF_UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["desc"], "grid": list(wl["n"]),
                       "sample_per_step": "closure forward of a 32^3 state"},
            "cpu_baseline": {"value": value, "unit": CF_UNIT, "cores": os.cpu_count(),
                             "kind": "oracle", "sample": "per step: a 32^3 forward"},
            "e2e": {"value": value, "unit": CF_UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    wl = dict(WORKLOADS[args.workload])
    if args.full_entropy:
        wl["entropy"] = dict(K=1e-3, zeta=1e-3, heat=0.02, cool=0.01)
        wl["desc"] += " + conduction, bulk viscosity, heating, cooling"
        wl.pop("vs", None)
    if args.stencil_order != 6:
        wl["order"] = args.stencil_order
        wl["desc"] = wl["desc"].replace("6th-order", "%dth-order" % args.stencil_order) + \
            " (stencil order %d)" % args.stencil_order
        wl.pop("vs", None)
    if args.init:
        wl["init"] = args.init
        wl["desc"] += " (initial state: %s)" % args.init
        wl.pop("vs", None)
    if args.grid and not wl.get("ensemble") and not wl.get("closure"):
        g = args.grid
        wl["n"] = (g, g, g)
        wl["desc"] = wl["desc"].replace("256^3", "%d^3" % g).replace("512^3", "%d^3" % g)
        wl.pop("vs", None)
    if args.impl == "reference":
        if wl.get("ensemble"):
            from paper_2103_01597_gb300 import synthetic
            n0 = synthetic.ensemble(wl["seed"])[0][0]
            wl = dict(wl, n=n0, desc=wl["desc"] + " (oracle sample: box 0)")
        if wl.get("closure_forward"):
            return run_closure_forward_reference(args, wl)
        return run_reference(args, wl)
    line = run_workload(args, wl)
    if line is None:
        return 0
    ws, _, _ = dist_setup(args)
    if args.workload == "forced256_fp64" and ws == 1 and not args.no_workloads and \
            not args.grid and args.stencil_order == 6 and not args.full_entropy and \
            not args.init:
        line["workloads"] = run_other_workloads(args)
    print(json.dumps(line))
    return 0


def run_decomp(args, wl):
    """The decomposed substep (Sec. 3.3) on one GPU, with and without the inner
    update overlapping the exchange, beside the undecomposed padded-layout run
    of the same arithmetic (plain binary64 stencils); result checked bitwise."""
    import torch
    from paper_2103_01597_gb300 import ac, build
    build.build()
    torch.cuda.set_device(0)
    n, p = wl["n"], wl["decomp"]
    ncell = n[0] * n[1] * n[2]
    stream = torch.cuda.current_stream()
    f0 = make_state(wl)
    dec = ac.Decomp(n, p, force_amp=wl["force_amp"], seed=wl["seed"], stream=stream.cuda_stream)
    ref = ac.Simulation(n, layout=ac.AC_LAYOUT_PADDED, force_amp=wl["force_amp"],
                        seed=wl["seed"], stream=stream.cuda_stream)
    dec.load(f0)
    ref.load(f0)
    dt = wl["dt"]
    dec.step(dt)
    ref.step(dt)
    bitwise = bool(np.array_equal(dec.store(), ref.store()))

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    bus = None
    try:
        bus = torch.cuda.get_device_properties(0).pci_bus_id
    except Exception:
        pass
    sampler = ClockSampler(bus)
    time.sleep(0.3)
    l0 = dec.info()["launches"]
    dec.set_overlap(True)
    t_ov = timed(lambda: dec.step(dt), args.steps)
    launches = (dec.info()["launches"] - l0) * args.steps // (args.steps + args.warmup)
    clocks = sampler.stop()
    dec.set_overlap(False)
    t_seq = timed(lambda: dec.step(dt), args.steps)
    t_ref = timed(lambda: ref.step(dt), args.steps)
    dec.close()
    ref.close()
    value = ncell * 3 * args.steps / t_ov / 1e9
    dfma = ac.ac_diag_fma_rate(ac.AC_FP64, stream.cuda_stream)
    flops = statistics.mean(flops_per_cell(6, s) for s in range(3)) * ncell * 3 * args.steps
    roof = {"bound": "alu", "achieved": flops / t_ov / 1e12, "peak": 2 * dfma / 1e12,
            "unit": "TFLOP/s", "frac": flops / t_ov / (2 * dfma),
            "what": "the method's binary64 flops per cell-substep (all on the FP64 pipe on the "
                    "plain stencils: a lower bound on the pipe's work) over the decomposed "
                    "substep's time, against the measured DFMA rate",
            "traffic": None, "kernel": "substep_box_kernel<double> (inner and outer segments)",
            "peak_source": "measured: ac_diag_fma_rate(AC_FP64) x 2"}
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_ov / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": wl["desc"], "grid": list(n), "subdomains": list(p)},
            "roofline": roof, "clocks": clocks, "gpu_launches": launches,
            "compare": {"no_overlap_gcell_s": ncell * 3 * args.steps / t_seq / 1e9,
                        "undecomposed_padded_gcell_s": ncell * 3 * args.steps / t_ref / 1e9,
                        "bitwise_equal_to_undecomposed": bitwise}}


def run_workload(args, wl):
    if wl.get("decomp"):
        return run_decomp(args, wl)
    if wl.get("closure_forward"):
        return run_closure_forward(args, wl)
    if wl.get("ensemble"):
        return run_ensemble(args, wl)
    if wl.get("closure"):
        return run_closure(args, wl)
    return run_ours(args, wl)


# The other workloads of the measurement table, run after the headline in the
# same process with fewer steps; each keeps its own roofline, clocks and error
# against binary64.
OTHER_WORKLOADS = {
    "paper256_fp64": dict(steps=10, warmup=3),
    "forced512_fp32": dict(steps=10, warmup=3, fp64_compare_steps=50),
    "ensemble64_fp32": dict(steps=10, warmup=3),
    "closure_forward256": dict(steps=10, warmup=3),
    "closure128": dict(steps=10, warmup=3, closure_pairs=12, closure_iters=400,
                       closure_rollout=20),
    "decomp256_fp64": dict(steps=5, warmup=3),
}
SUMMARY_KEYS = ("metric", "value", "unit", "ms_per_step", "steps", "warmup", "dtype",
                "roofline", "clocks", "gpu_launches", "substep_ms", "fp32_vs_fp64",
                "parity_sampled", "compare", "stencil_modes", "config", "closure")


def run_other_workloads(args):
    import torch
    out = {}
    for name, over in OTHER_WORKLOADS.items():
        sub = argparse.Namespace(**vars(args))
        sub.workload = name
        sub.e2e_steps = 0
        sub.no_cpu_baseline = True
        sub.fp64_compare_steps = 0
        for k, v in over.items():
            setattr(sub, k, v)
        t0 = time.perf_counter()
        line = run_workload(sub, dict(WORKLOADS[name]))
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        out[name] = {k: line[k] for k in SUMMARY_KEYS if k in line and line[k] is not None}
        out[name]["wall_s"] = round(time.perf_counter() - t0, 1)
    return out


if __name__ == "__main__":
    sys.exit(main())
