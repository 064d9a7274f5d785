#!/usr/bin/env python
"""Benchmark of the droplet time step (Mcell-steps/s) on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

One step = one pass of the whole segregated step (thermodynamics, evaporation
flux, alpha source and advection, properties, energy, species, momentum,
pressure projection, diagnostics) over one droplet grid.  Default workload:
the 3D Cartesian 256^3 case (forced inflow 1 m/s at 773 K, 20 bar,
Peng-Robinson equilibrium, seeded 1 % temperature perturbation) in plain FP64.
Under torchrun every rank runs an independent replica (the single-droplet path
does not shard), and value is the cells x steps of all ranks over the slowest
rank's time.

The reference arm (--impl reference) times the plain FP64 CPU oracle on the
host cores; no GPU is used there.  The oracle solves every linear system with
a sparse direct factorisation, which cannot hold a 256^3 grid: for the 3D
workloads each of its steps is a bounded sample, one oracle step of the same
case on 20^3 cells (same domain, physics and time step), counted as the cells
it advanced.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

if "--impl" in sys.argv and "reference" in sys.argv:
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"

import numpy as np  # noqa: E402

from paper_2005_02867_gb300 import workloads as W  # noqa: E402

WORKLOADS = {
    "cfg2_axisym_256x512": lambda: W.cfg2_axisym_256x512(),
    "cfg2_axisym_256x512_fp64": lambda: W.cfg2_axisym_256x512(precision=0),
    "cfg3_cart3d_256": lambda: W.cfg3_cart3d(),
    "cfg3_cart3d_256_fp64": lambda: W.cfg3_cart3d(precision=0),
    "cfg3_cart3d_128_fp64": lambda: W.cfg3_cart3d(nc=128, precision=0),
    "cfg3_cart3d_256_fp64_geometric": lambda: W.cfg3_cart3d(precision=0, adv_scheme=1),
    "cfg2_axisym_256x512_geometric": lambda: W.cfg2_axisym_256x512(adv_scheme=1),
    # the droplet placed around the spherical fibre (fiber_radius 0.05 mm)
    "cfg2_axisym_256x512_fibre": lambda: W.cfg2_axisym_256x512(fiber=1),
    "cfg3_cart3d_256_fp64_fibre": lambda: W.cfg3_cart3d(precision=0, fiber=1),
    # the 3D launched path (more than 2^22 cells) at ~2.5 GB on the device: the size of
    # the full ncu captures of its kernels
    "cfg3_cart3d_176": lambda: W.cfg3_cart3d(nc=176),
    "cfg3_cart3d_176_fp64": lambda: W.cfg3_cart3d(nc=176, precision=0),
    "cfg4_batch64": lambda: W.cfg4_batch(),
    "cfg4_batch64_fp64": lambda: [dict(c, precision=0) for c in W.cfg4_batch()],
    "cfg4_serial64_fp64": lambda: [dict(c, precision=0) for c in W.cfg4_batch()],
    "cfg1_axisym_64x128": lambda: W.cfg1_axisym_64x128(cg_rtol=1e-12, helm_rtol=1e-13),
    "cfg5_axisym_128x256": lambda: W.cfg5_axisym_128x256(cg_rtol=1e-12, helm_rtol=1e-13),
}
DEFAULT = "cfg3_cart3d_256_fp64"
ORACLE_3D_CELLS = 20      # cells per axis of the oracle's sample of a 3D workload
METRIC = "Mcell-steps/s"
FLUSH_BYTES = 512 << 20      # larger than the 129 MB L2


# DRAM traffic of the dominant kernel from a committed ncu capture: profiles/ncu_traffic.json
# maps a workload to {class, kernel, dram_bytes_per_launch, sources, sources_sha256, ...};
# the value is reported only while the sources that define the kernel (its translation
# unit and the headers it includes, listed in the record) hash as they did when the
# counters were taken (else null: the kernel has changed since).
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ncu_traffic.json")
# Binary64 instructions per unit (face / cell) of the FP64 assembly kernels as issued,
# from a committed ncu capture (profiles/ncu_fp64_inst.json), used while their sources
# hash as recorded: those kernels carry no algorithmic FP64 count in the library.
FP64_INST_FILE = os.path.join(ROOT, "profiles", "ncu_fp64_inst.json")
SOLVER_SOURCES = ["paper_2005_02867_gb300/csrc/solver.cu", "paper_2005_02867_gb300/csrc/common.cuh",
                  "paper_2005_02867_gb300/csrc/kernels.h", "include/droplet.h"]


def sources_sha256(files=SOLVER_SOURCES):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def captured_traffic(workload, kclass):
    try:
        with open(TRAFFIC_FILE) as fh:
            rec = json.load(fh).get(workload)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("class") != kclass:
        return None
    try:
        if rec.get("sources_sha256") != sources_sha256(rec.get("sources", SOLVER_SOURCES)):
            return None
    except OSError:
        return None
    return rec


def captured_fp64_inst(workload, kclass):
    """Binary64 instructions per unit of kclass on workload from the committed record,
    or None (no record, or the kernel's sources changed since the capture)."""
    try:
        with open(FP64_INST_FILE) as fh:
            rec = json.load(fh).get(workload)
    except (OSError, ValueError):
        return None
    if not rec or kclass not in rec:
        return None
    try:
        if rec.get("sources_sha256") != sources_sha256(rec["sources"]):
            return None
    except (OSError, KeyError):
        return None
    return rec[kclass]["inst_per_unit"]


def cells_of(cfg):
    if isinstance(cfg, list):
        return sum(cells_of(c) for c in cfg)
    return int(np.prod(cfg["n"][:2])) if cfg["geom"] == 0 else int(np.prod(cfg["n"]))


def describe(name, cfg):
    if isinstance(cfg, list):
        c0 = cfg[0]
        return {
            "workload": name, "droplets": len(cfg), "cells": cells_of(cfg),
            "grids": sorted({tuple(c["n"][:2]) for c in cfg}),
            "precision": "fp64" if c0["precision"] == 0 else "fp64 CG + fp32 multigrid / fp32 Helmholtz defect correction",
            "cg_rtol": c0["cg_rtol"], "helm_rtol": c0["helm_rtol"],
            "execution": "one graph launch per step, one branch per droplet",
            "l2": "flushed between timed steps (512 MiB device write outside the step events)",
        }
    n = list(cfg["n"][:2]) if cfg["geom"] == 0 else list(cfg["n"])
    return {
        "workload": name,
        "geometry": "axisymmetric r-z" if cfg["geom"] == 0 else "3D Cartesian",
        "grid": n,
        "cells": int(np.prod(n)),
        "dt_s": cfg["dt"],
        "gravity": list(cfg["g"]),
        "equilibrium": "Raoult" if cfg["eq_model"] == 0 else "Peng-Robinson",
        "pressure_Pa": cfg["P"],
        "precision": "fp64" if cfg["precision"] == 0 else "fp64 CG + fp32 multigrid / fp32 Helmholtz defect correction",
        "cg_rtol": cfg["cg_rtol"],
        "helm_rtol": cfg["helm_rtol"],
        "l2": "flushed between timed steps (512 MiB device write outside the step events)",
    }


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBps", "hbm"):
                if k in d:
                    return float(d[k]), "measured (MEASURED_PEAKS.json)"
        except Exception:
            pass
    return 6800.0, "fallback (6.8 TB/s)"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, gpu):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.f.name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "samples": len(sm), "reasons": sorted(reasons)}


ORACLE_SNIPPET = r"""
import sys, time, json
sys.path.insert(0, {root!r})
from oracle import step as O
cfg = json.loads({cfg!r})
cfg["n"] = tuple(cfg["n"]); cfg["L"] = tuple(cfg["L"]); cfg["xc"] = tuple(cfg["xc"]); cfg["g"] = tuple(cfg["g"])
st = O.init_state(cfg)
st = O.step(cfg, st)
t0 = time.perf_counter()
n = 0
while n < {nmax} and (n < {nmin} or time.perf_counter() - t0 < {budget}):
    st = O.step(cfg, st)
    n += 1
print(json.dumps(dict(steps=n, seconds=time.perf_counter() - t0)))
"""


def oracle_sample(cfg):
    """The case the oracle steps for a workload, and what it is: the workload itself
    (the first droplet of a batch), or for a 3D grid beyond the oracle's direct
    solver the same case on ORACLE_3D_CELLS^3 cells."""
    c = cfg[0] if isinstance(cfg, list) else cfg
    note = "first droplet of the batch" if isinstance(cfg, list) else "the workload itself"
    if c["geom"] == W.GEOM_CART3D and cells_of(c) > ORACLE_3D_CELLS ** 3:
        n = ORACLE_3D_CELLS
        c = dict(c, n=(n, n, n), precision=0)
        note = (f"the same case (domain, physics, time step) on {n}^3 cells: the oracle's sparse direct "
                f"solves cannot hold the full grid")
    return c, note


def cpu_oracle(cfg, nmin=2, nmax=50, budget=15.0):
    """Time the oracle on the host in a fresh single-threaded process (a bounded sample)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ORACLE_SNIPPET.format(root=ROOT, cfg=json.dumps(cfg), nmin=nmin, nmax=nmax, budget=budget)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1200)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["steps"], d["seconds"]


class SerialDroplets:
    """Single-droplet contexts driven one after the other (the unbatched form)."""

    def __init__(self, D, cfgs, stream):
        self.D = D
        self.sims = [D.Droplet(c, stream=stream) for c in cfgs]
        self.h = self.sims[0].h

    def step(self, n=1):
        rc = 0
        for s in self.sims:
            rc = rc or s.step(n)
        return rc

    def diag(self, droplet=0):
        return self.sims[droplet].diag()

    def close(self):
        for s in self.sims:
            s.close()


def step_model_bytes(cfg, its):
    """Algorithmic HBM bytes of one step of one droplet (the whole step, not one kernel),
    with its = {"p", "T", "w", "u"} the step's iteration counts (u summed over the
    velocity components): the stage sweeps (32 + 14 d + d^2) w_s per cell, the
    Jacobi-PCG 11 w_s per cell and iteration of each Helmholtz system, and per MG-PCG
    iteration (d + 12) 8 + c (5 d + 18) w_s per cell (c = 4/3 in 2D, 8/7 in 3D: the level
    sum), w_s = 8 in FP64 and 4 in mixed precision (the stencil word)."""
    d = 3 if cfg["geom"] == 1 else 2
    ws = 8.0 if cfg["precision"] == 0 else 4.0
    c = 4.0 / 3.0 if d == 2 else 8.0 / 7.0
    per_cell = (32 + 14 * d + d * d) * ws + (its["T"] + its["w"] + its["u"]) * 11.0 * ws \
        + its["p"] * ((d + 12) * 8.0 + c * (5 * d + 18) * ws)
    return per_cell * cells_of(cfg)


def replica_throughput(t_ms, ncell, steps):
    """Whole-job throughput of independent replicas: every rank advanced ncell
    cells by `steps` steps in its own t_ms; the job's time is the slowest
    rank's.  Returns (Mcell-steps/s over all ranks, max t_ms)."""
    import torch
    import torch.distributed as dist
    world = 1
    if dist.is_available() and dist.is_initialized():
        world = dist.get_world_size()
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(t_ms)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_ms = float(t.item())
    return ncell * steps * world / (t_ms / 1e3) / 1e6, t_ms


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    name = args.workload
    full = WORKLOADS[name]()
    cfg, note = oracle_sample(full)     # cells counted for the case the oracle steps
    ncell = cells_of(cfg)
    from oracle import step as O
    st = O.init_state(cfg)
    for _ in range(args.warmup):
        st = O.step(cfg, st)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st = O.step(cfg, st)
    el = time.perf_counter() - t0
    value = ncell * args.steps / el / 1e6
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "impl": "reference", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": describe(name, full),
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} oracle steps after {args.warmup} warm-up steps, single thread, of "
                                   f"{note} ({ncell} cells)"},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2005_02867_gb300 import _build, droplet as D

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or not os.path.exists(D.LIBPATH):
        _build.build_library()
    if world > 1:
        dist.barrier()
    D.load_library()

    name = args.workload
    cfg = WORKLOADS[name]()
    ncell = cells_of(cfg)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    if name.endswith("_serial64_fp64"):
        # the plain form: one single-droplet context per droplet, stepped one after the other
        sim = SerialDroplets(D, cfg, stream.cuda_stream)
    else:
        sim = D.Droplet(cfg, stream=stream.cuda_stream)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    fp64_peak = D.droplet_fp64_rate()

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        sim.step(1)
    torch.cuda.synchronize()

    # ---- device-timed region: inputs resident in HBM, L2 flushed before every step;
    # each step is one launch of the captured step graph
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks(local)
    status = 0
    barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record(stream)
        rc = sim.step(1)
        status = status or rc
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    ck = clocks.stop()
    t_ms_local = sum(a.elapsed_time(b) for a, b in evs)

    # ---- per-kernel timing: the same steps launched kernel by kernel with a CUDA event
    # pair around every launch of the timed classes (library stream), L2 flushed per step
    kprof = max(1, min(args.steps, 5))
    serial = isinstance(sim, SerialDroplets)
    D.droplet_profile(sim.h, 1)
    n0 = D.droplet_launch_count(sim.h)
    for k in range(kprof):
        flush.zero_()
        sim.step(1)
    torch.cuda.synchronize()
    launches_per_step = (D.droplet_launch_count(sim.h) - n0) / kprof
    # (serial form: every context's launches count, the event timing covers the first context)
    prof = {k: D.droplet_profile_read(sim.h, k) for k in D.KCLASS}
    D.droplet_profile(sim.h, 0)
    diag_run = sim.diag()   # solver iterations of a step of the run (the e2e leg restarts from uploads)
    cl_run = cfg if isinstance(cfg, list) else [cfg]
    model_b = 0.0
    for di, cd in enumerate(cl_run):
        dd = diag_run if di == 0 else sim.diag(di)
        model_b += step_model_bytes(cd, {"p": dd["its_p"], "T": dd["its_T"], "w": dd["its_w"], "u": dd["its_u"]})
    launches = int(round(launches_per_step * args.steps))
    value, t_ms = replica_throughput(t_ms_local, ncell, args.steps)

    # ---- end to end through the C ABI with host buffers: upload the state from
    # pinned host memory, one step, read the state back, every step
    cl = cfg if isinstance(cfg, list) else [cfg]
    bufs = {}
    def handle(di):
        return (sim.sims[di].h, 0) if serial else (sim.h, di)
    for di, cd in enumerate(cl):
        fields = ["alpha", "T", "omega", "p", "rhoG"] + ["u%d" % a for a in range(3 if cd["geom"] == 1 else 2)]
        h, k = handle(di)
        for f in fields:
            n = D.droplet_field_size(h, f, droplet=k)
            bufs[(di, f)] = torch.empty(n, dtype=torch.float64, pin_memory=True)
            D.droplet_get_field_ptr(h, f, bufs[(di, f)].data_ptr(), n, droplet=k)
    nbytes = sum(b.numel() * 8 for b in bufs.values())
    e2e_steps = max(1, min(args.steps, 10))
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for (di, f), b in bufs.items():
            h, k = handle(di)
            D.droplet_set_field_ptr(h, f, b.data_ptr(), b.numel(), droplet=k)
        sim.step(1)
        for (di, f), b in bufs.items():
            h, k = handle(di)
            D.droplet_get_field_ptr(h, f, b.data_ptr(), b.numel(), droplet=k)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value, _ = replica_throughput(e2e_s * 1e3, ncell, e2e_steps)
    sim.close()

    if rank == 0:
        dom = max(prof, key=lambda k: prof[k][0])
        peak, src = load_peaks()
        # binary64 pipe: one instruction per FMA slot, so its instruction rate is half the
        # measured FMA flop rate (about 2 per SM clock on GB300)
        inst_peak = fp64_peak * 1e12 / 2.0
        d0 = 3 if cl[0]["geom"] == 1 else 2

        def class_rates(k):
            """(HBM GB/s, binary64 instructions/s, where the count came from) of class k."""
            ms, nl, by, fl = prof[k]
            if ms <= 0:
                return 0.0, 0.0, None
            how = "algorithmic count of the library"
            if k in ("mom_assemble", "scalar_assemble"):
                per = captured_fp64_inst(name, k) if cl[0]["precision"] == 0 else None
                units = by / ((12 + 2 * d0) * 8.0)     # faces / cells: the bytes are (12 + 2d) 8 per unit
                fl = per * units if per else 0.0
                how = "issued count per unit from profiles/ncu_fp64_inst.json" if per else None
            return by / (ms / 1e3) / 1e9, fl / (ms / 1e3), how

        ms, nl, by, _ = prof[dom]
        hbm_gbs, inst_s, how = class_rates(dom)
        # GB300's binary64 pipe is the tighter roof for FP64 stencils: report the bound
        # with the larger fraction, against the FMA rate measured on this device
        if inst_s / inst_peak > hbm_gbs / peak:
            roof = {"bound": "alu", "achieved": inst_s / 1e9, "peak": inst_peak / 1e9,
                    "unit": "G binary64 instructions/s", "frac": inst_s / inst_peak,
                    "peak_source": "measured binary64 FMA rate of this GPU (droplet_fp64_rate), one instruction "
                                   "per FMA slot", "achieved_source": how,
                    "hbm_achieved_GBps": hbm_gbs, "hbm_frac": hbm_gbs / peak}
        else:
            roof = {"bound": "hbm", "achieved": hbm_gbs, "peak": peak, "unit": "GB/s", "frac": hbm_gbs / peak,
                    "peak_source": src, "fp64_Ginst_s": inst_s / 1e9, "fp64_frac": inst_s / inst_peak}
        tr = captured_traffic(name, dom)
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64" if cl[0]["precision"] == 0 else "f64 state, f32 stencil solves (multigrid, Helmholtz increments)",
            "data": "synthetic", "config": describe(name, cfg),
            "roofline": dict(roof, kernel=dom, traffic=(tr or {}).get("dram_bytes_per_launch"),
                             traffic_source=({k: tr[k] for k in ("kernel", "summary", "scaled_from") if k in tr}
                                             if tr else None),
                             launches=nl, kernel_ms_total=ms, profiled_steps=kprof,
                             share_of_graph_step=(ms / kprof) / (t_ms / args.steps) if t_ms > 0 else None),
            "kernel_classes": {k: {"ms": v[0], "launches": v[1], "GBps": class_rates(k)[0],
                                   "hbm_frac": class_rates(k)[0] / peak,
                                   "fp64_Ginst_s": class_rates(k)[1] / 1e9,
                                   "fp64_frac": class_rates(k)[1] / inst_peak}
                               for k, v in prof.items()},
            "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                    "steps": e2e_steps},
            "gpu_launches": launches,
            "gpu_launches_note": "kernel nodes per step counted on the directly launched profiling steps x timed steps",
            "solver_iterations_last_step": {"p": diag_run["its_p"], "T": diag_run["its_T"],
                                            "omega": diag_run["its_w"], "u": diag_run["its_u"]},
            # the whole step against HBM: algorithmic bytes of the step's model (stage sweeps,
            # Helmholtz and MG-PCG iterations as counted) over the device-timed step
            "step_model": {"bytes_per_step": model_b,
                           "GBps": model_b / (t_ms / args.steps / 1e3) / 1e9 if t_ms > 0 else 0.0,
                           "frac": (model_b / (t_ms / args.steps / 1e3) / 1e9) / peak if t_ms > 0 else 0.0,
                           "peak_GBps": peak},
            "status": status,
            "fp64_peak_TFs_measured": fp64_peak,
            "clocks": ck,
        }
        if world == 1 and not args.no_cpu_baseline:
            try:
                c0, note = oracle_sample(cfg)
                n, sec = cpu_oracle(c0)
                line["cpu_baseline"] = {"value": cells_of(c0) * n / sec / 1e6, "unit": METRIC, "cores": 1,
                                        "kind": "oracle",
                                        "sample": f"{n} oracle steps (single thread, after one untimed step) of "
                                                  f"{note} ({cells_of(c0)} cells)"}
            except Exception as e:  # the GPU number stands on its own
                line["cpu_baseline"] = {"value": None, "unit": METRIC, "cores": 1, "kind": "oracle",
                                        "sample": f"failed: {str(e)[-200:]}"}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
