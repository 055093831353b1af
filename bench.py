#!/usr/bin/env python3
"""Throughput of the fused LBM-PIBM-DEM lattice step on one GB300 per rank.

Default workload: 3-D thermosensitive sedimentation of 10 000 spheres
(diameter 6 lattice units) in a 384^3 walled box, D3Q19 + D3Q7 with FP32
population storage, Hertz / Mindlin-Deresiewicz DEM with 10 substeps per
lattice step (the largest single-GPU configuration).  One "step" = one
lattice step: fused collide-and-stream, DEM substeps (concurrent branch),
PIBM coupling.  The metric is fluid+thermal lattice-node updates per second
(MLUPS), plus particle-steps/s; L2 is flushed (256 MB write) before every
timed step and each step is timed on its own with CUDA events.  The 16-bit
storage forms, the 256x256x512 and 2-D cases, the batched ensemble and the
learned surrogate are reported as extra keys of the same line.

Under torchrun each rank runs an independent replica on its own GPU (the
method does not shard here: replicas only); value = all ranks' node updates /
the slowest rank's time.

--impl reference times the FP64 CPU oracle on the workload's bounded sample
(the 64^3 crop of the 384^3 case at its number density; rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fluid+thermal MLUPS and particle-steps/s at 1 GB300; % HBM peak; speedup vs plain FP32 at error"
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 256 << 20


def bytes_per_node(case) -> int:
    """Algorithmic bytes of one node update of the fused kernel: every flow and
    thermal population read once and written once (A-A in place)."""
    q = (9 + 5) if case["dim"] == 2 else (19 + 7)
    es = {"f64": 8, "f16": 2, "bf16": 2}.get(case.get("storage", "f32"), 4)
    return 2 * q * es


HEAT_CAP_D6 = 1.2 * 4.0 / 3.0 * np.pi * 27.0  # rho_p V_p of a sphere of diameter 6 (specific heat ratio 1)
STORAGE_NAME = {"f32": "FP32", "f16": "FP16-deviation storage (FP32 arithmetic)",
                "bf16": "BF16-deviation storage (FP32 arithmetic)", "f64": "FP64"}


def workload(name: str, storage: str = "f32"):
    """(case dict, description) of a named workload; every placement is seeded."""
    import workloads as W
    st = STORAGE_NAME[storage]
    if name == "sed3d384":
        case = W.sed3d(nx=384, ny=384, nz=384, n_p=10000, d=6.0, config_index=4, heat_cap=HEAT_CAP_D6,
                       T_p_random=True)
        desc = (f"sed3d384: 3-D thermosensitive sedimentation, 384^3 lattice, 10000 spheres d=6, "
                f"D3Q19+D3Q7 {st}, Hertz/Mindlin, 10 DEM substeps")
    elif name == "sed3d384_crop":
        case = W.sed3d(nx=64, ny=64, nz=64, n_p=46, d=6.0, config_index=4, heat_cap=HEAT_CAP_D6, T_p_random=True)
        desc = (f"sed3d384 crop: 64^3 lattice, 46 spheres d=6 (the 384^3 case's number density), thermosensitive, "
                f"D3Q19+D3Q7 {st}, Hertz/Mindlin, 10 DEM substeps")
    elif name == "sed2d":
        case = W.sed2d()
        desc = f"sed2d: 2-D sedimentation, 512x1024 lattice, 500 heated disks d=10, D2Q9+D2Q5 {st}, spring-dashpot, 10 DEM substeps"
    elif name == "sed3d":
        case = W.sed3d()
        desc = f"sed3d: 3-D sedimentation, 256x256x512 lattice, 2000 heated spheres d=8, D3Q19+D3Q7 {st}, Hertz/Mindlin, 10 DEM substeps"
    elif name == "sed3d_crop":
        case = W.sed3d(nx=64, ny=64, nz=128, n_p=62, config_index=2)
        desc = f"sed3d crop: 64x64x128 lattice, 62 heated spheres d=8 (the 256x256x512 case's number density), D3Q19+D3Q7 {st}, Hertz/Mindlin"
    elif name == "sed3d_mid":
        case = W.sed3d(nx=128, ny=128, nz=256, n_p=250)
        desc = f"sed3d_mid: 3-D sedimentation, 128x128x256 lattice, 250 heated spheres d=8, D3Q19+D3Q7 {st}, Hertz/Mindlin (profiling size)"
    elif name == "sed3d384_mid":
        case = W.sed3d(nx=192, ny=192, nz=192, n_p=1250, d=6.0, config_index=4, heat_cap=HEAT_CAP_D6, T_p_random=True)
        desc = f"sed3d384_mid: 192^3 lattice, 1250 thermosensitive spheres d=6, D3Q19+D3Q7 {st} (profiling size)"
    else:
        raise SystemExit(f"unknown workload {name}")
    case["storage"] = storage
    return case, desc


# bounded CPU sample of each workload (the oracle runs FP64 on one core)
CROP = {"sed3d384": "sed3d384_crop", "sed3d": "sed3d_crop", "sed3d384_mid": "sed3d384_crop",
        "sed3d_mid": "sed3d_crop", "sed2d": "sed2d"}


def cpu_info() -> dict:
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform
    return {"cpu_model": model or platform.processor() or platform.machine(), "nproc": os.cpu_count(),
            "machine": platform.machine()}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def kernel_source_sha(source: str, region_end: str | None) -> str:
    """sha256 of a kernel's source: the file, or its text up to the line that
    starts with region_end (the part of the file that holds the kernel and its
    launcher, so that other kernels of the file can change)."""
    text = open(os.path.join(ROOT, "paper_1502_01159_gb300", "csrc", source), "rb").read()
    if region_end:
        cut = text.find(b"\n" + region_end.encode())
        text = text[:cut] if cut >= 0 else text
    return hashlib.sha256(text).hexdigest()


def traffic_record(kernel: str, workload_name: str):
    """DRAM bytes per launch from a committed ncu summary, valid only while the
    kernel source is unchanged since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        rec = json.load(fh)
    entry = rec.get(kernel, {}).get(workload_name)
    if not entry:
        return None
    sha = kernel_source_sha(entry["source"], entry.get("region_end"))
    return entry["bytes_per_launch"] if sha == entry["source_sha256"] else None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"pibm_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        self.proc.wait()
        self.fh.close()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            if self.uuid and self.uuid not in parts[1]:
                continue
            try:
                sm.append(float(parts[2]))
                smax = max(smax, float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[6:10]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(value: float, dist, device) -> float:
    """Slowest rank's value (the job finishes when the last replica does)."""
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, units_per_rank: float, ms_step: float) -> float:
    """Whole-job throughput in millions of units per second: every rank runs an
    independent replica of the same workload."""
    return world * units_per_rank / (ms_step * 1e-3) / 1e6


def oracle_run(case, steps, warmup):
    import oracle
    o = oracle.Oracle(case)
    o.step(warmup)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    o.close()
    nodes = case["shape"][0] * case["shape"][1] * case["shape"][2]
    n_p = len(case["particles"]["R"]) if case.get("particles") else 0
    return nodes * steps / dt / 1e6, n_p * steps / dt, dt


def oracle_baselines() -> dict:
    """The FP64 single-threaded oracle on the bounded CPU samples of every
    workload family: the cavity in full (2000 steps), 200 steps of the 2-D
    sedimentation case, the 64x64x128 crop of the 3-D case (100 steps), one
    64^3 box of the ensemble (100 steps) and the 64^3 crop of the 384^3 case
    (100 steps).  Run in its own process beside the GPU measurements."""
    import workloads as W
    runs = []
    cav = W.cavity(n=128, Ar=2.5, storage="f64")
    runs.append(("cavity 128^2 (Ra 1e4, Ar 2.5, 8235 static points), in full", cav, 2000))
    runs.append(("sed2d 512x1024, 500 disks", workload("sed2d")[0], 200))
    runs.append(("sed3d crop 64x64x128, 62 spheres", workload("sed3d_crop")[0], 100))
    box = next(c for c in W.ensemble() if c["shape"][0] == 64)
    runs.append((f"ensemble box {box['name']}", box, 100))
    runs.append(("sed3d384 crop 64^3, 46 thermosensitive spheres", workload("sed3d384_crop")[0], 100))
    out = []
    for what, case, steps in runs:
        mlups, psps, dt = oracle_run(case, steps, 1)
        out.append({"case": what, "steps": steps, "MLUPS": round(mlups, 4), "particle_steps_per_s": round(psps, 1),
                    "seconds": round(dt, 2)})
    return {"cores": 1, "kind": "oracle", "precision": "f64", **cpu_info(), "runs": out}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    case, desc = workload(args.workload, args.storage)
    crop, crop_desc = workload(CROP[args.workload], args.storage)
    mlups, psps, dt = oracle_run(crop, args.steps, args.warmup)
    sample = (f"{args.steps} lattice steps (after {args.warmup} untimed) of {crop_desc}, the bounded CPU sample of "
              f"{args.workload}")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(mlups, 4), "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "implementation": "FP64 single-threaded C oracle on the host", "sample": crop_desc},
        "particle_steps_per_s": round(psps, 2),
        "cpu_baseline": {"value": round(mlups, 4), "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": sample,
                         **cpu_info()},
        "e2e": {"value": round(mlups, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def measure_gpu(case, steps, warmup, torch, flush):
    """Device time per lattice step (graph replay), L2 flushed before each step."""
    from paper_1502_01159_gb300 import Simulation
    sim = Simulation(case)
    s = sim.stream
    sim.step(warmup)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        with torch.cuda.stream(s):
            flush.fill_(k & 0xFF)
        ev[k][0].record(s)
        sim.step(1)
        ev[k][1].record(s)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    return sim, ms


def kernel_times(sim, steps, torch, flush):
    """Per-kernel-group device times: step-graph replays with CUDA event-record nodes around each
    kernel group on its own stream (pibm_step_timed)."""
    out = []
    for k in range(steps):
        with torch.cuda.stream(sim.stream):
            flush.fill_((k + 7) & 0xFF)
        out.append(sim.step_timed())
    return {key: statistics.mean(o[key] for o in out) for key in out[0]}


def e2e_run(case, steps, torch):
    """Whole job through the public API with host buffers: create the context
    (lattice at rest equilibrium, walls, contact law) and upload the particle
    set from pinned host memory; then per step: one lattice step and a
    read-back of the particle state (positions, velocities, spins,
    temperatures); finally the temperature field."""
    from paper_1502_01159_gb300 import Simulation
    parts = {}
    for k, v in case["particles"].items():
        a = np.ascontiguousarray(np.asarray(v, dtype=np.uint8 if k == "fixed" else np.float64))
        pin = torch.empty(a.shape, dtype=torch.uint8 if k == "fixed" else torch.float64, pin_memory=True).numpy()
        pin[...] = a
        parts[k] = pin
    c2 = dict(case)
    c2["particles"] = parts
    n_p = len(case["particles"]["R"])
    nodes = case["shape"][0] * case["shape"][1] * case["shape"][2]

    def pinned(shape):
        return torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
    # pinned host buffers for the read-backs, as for the uploads
    pout = {"X": pinned((n_p, 3)), "U": pinned((n_p, 3)), "W": pinned((n_p, 3)), "T_p": pinned((n_p,))}
    Tout = pinned((nodes,))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim = Simulation(c2)
    d2h = 0
    for _ in range(steps):
        sim.step(1)
        p = sim.read_particles(out=pout)
        d2h += sum(v.nbytes for v in p.values())
    T = sim.read_field("T", out=Tout)
    d2h += T.nbytes
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    h2d = sum(v.nbytes for v in parts.values())
    sim.close()
    return {"value": round(nodes * steps / dt / 1e6, 3), "unit": "MLUPS", "steps": steps, "seconds": round(dt, 4),
            "particles": n_p, "h2d_bytes_per_step": int(h2d // steps), "d2h_bytes_per_step": int(d2h // steps),
            "what": "create (device allocation, lattice at rest equilibrium) + upload of the particle set from pinned "
                    "host memory, then per step: pibm_step + particle state read-back; final temperature field "
                    "read-back (read-backs into pinned host buffers)"}


def _crop_errors(crop, storages, steps=50):
    """Relative L2 error per field and largest particle offset of the GPU path
    in each storage form against the FP64 oracle after `steps` steps."""
    import oracle
    from paper_1502_01159_gb300 import Simulation
    orc = oracle.Oracle(crop)
    orc.step(steps)
    ref = {k: orc.field(k) for k in ("rho", "T", "ux", "uy", "uz")}
    refP = orc.particles()
    orc.close()

    def rl2(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))
    out = {}
    for storage in storages:
        c2 = dict(crop)
        c2["storage"] = storage
        s2 = Simulation(c2)
        s2.step(steps)
        p = s2.read_particles()
        err = {"rho": rl2(s2.read_field("rho"), ref["rho"]), "T": rl2(s2.read_field("T"), ref["T"]),
               "u": rl2(np.stack([s2.read_field(c) for c in ("ux", "uy", "uz")]),
                        np.stack([ref[c] for c in ("ux", "uy", "uz")])),
               "X_max_abs": float(np.max(np.abs(p["X"] - refP["X"]))),
               "T_p_max_abs": float(np.max(np.abs(p["T_p"] - refP["T_p"])))}
        s2.close()
        out[storage] = {k: float(f"{v:.3g}") for k, v in err.items()}
    return out


def precision_study(torch, flush, head=None):
    """Reduced-precision storage (FP16 / BF16 deviations, FP32 arithmetic) against
    the plain FP32 form: step and lattice-kernel throughput on the full 384^3
    case (whose FP32 numbers are the headline's) and on the 256x256x512 case,
    and the error against the FP64 oracle on each case's crop (64^3 with 46
    spheres; 64x64x128 with 31 spheres) after 50 steps with the same recipe."""
    from paper_1502_01159_gb300 import TUNE_LATTICE_ROW_TILES
    out = {}
    for wl, crop_name in (("sed3d384", "sed3d384_crop"), ("sed3d", "sed3d_crop")):
        res = {}
        nodes = None
        for storage in ("f32", "f16", "bf16"):
            if storage == "f32" and wl == "sed3d384" and head is not None:
                res["f32"] = dict(head)
                continue
            case, _ = workload(wl, storage)
            nodes = case["shape"][0] * case["shape"][1] * case["shape"][2]
            sim, ms = measure_gpu(case, 8, 3, torch, flush)
            kt = kernel_times(sim, 6, torch, flush)
            # the same kernel with blocks that divide the row, for comparison
            sim.set_tuning(TUNE_LATTICE_ROW_TILES, 1)
            kt_np = kernel_times(sim, 6, torch, flush)["stream_collide"]
            sim.close()
            step = statistics.mean(ms)
            bpn = bytes_per_node(case)
            res[storage] = {"step_ms": round(step, 4), "MLUPS": round(nodes / (step * 1e-3) / 1e6, 1),
                            "stream_collide_ms": round(kt["stream_collide"], 4),
                            "stream_collide_GBs": round(nodes * bpn / (kt["stream_collide"] * 1e-3) / 1e9, 1),
                            "bytes_per_node": bpn}
            res[storage]["stream_collide_ms_row_tiles"] = round(kt_np, 4)
        crop, _ = workload(crop_name)
        if crop_name == "sed3d_crop":
            import workloads as W
            crop = W.sed3d(nx=64, ny=64, nz=128, n_p=31, config_index=2)
        crop["g_particle"] = [0.0, 0.0, -2e-4]
        errs = _crop_errors(crop, ("f32", "f16", "bf16"))
        for storage in ("f32", "f16", "bf16"):
            res[storage]["error_vs_fp64_oracle_crop"] = errs[storage]
        for storage in ("f16", "bf16"):
            res[storage]["speedup_step_vs_f32"] = round(res["f32"]["step_ms"] / res[storage]["step_ms"], 3)
            res[storage]["speedup_kernel_vs_f32"] = round(res["f32"]["stream_collide_ms"] /
                                                          res[storage]["stream_collide_ms"], 3)
        res["error_sample"] = (f"{crop['shape'][0]}x{crop['shape'][1]}x{crop['shape'][2]} crop, "
                               f"{len(crop['particles']['R'])} spheres, 50 steps, against the FP64 oracle")
        out[wl] = res
    return out


def ensemble_study(torch, flush, steps):
    """Batched ensemble of 32 uneven thermosensitive sphere-sedimentation
    boxes (edges 64..128, Ra log-uniform 1e3..1e5, 50-400 spheres), all
    advanced by one graph launch per step; timed before and after the
    autotuner, and against launching every box's own step graph in turn."""
    import workloads as W
    from paper_1502_01159_gb300 import Ensemble
    cases = W.ensemble()
    nodes = sum(c["shape"][0] * c["shape"][1] * c["shape"][2] for c in cases)
    n_p = sum(len(c["particles"]["R"]) for c in cases)
    ens = Ensemble(cases)
    s = ens.stream

    def timed(k, fn):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        for i in range(k):
            with torch.cuda.stream(s):
                flush.fill_(i & 0xFF)
            ev[i][0].record(s)
            fn()
            ev[i][1].record(s)
        torch.cuda.synchronize()
        return statistics.mean(a.elapsed_time(b) for a, b in ev)

    ens.step(3)
    torch.cuda.synchronize()
    ms_default = timed(steps, lambda: ens.step(1))
    t0 = time.perf_counter()
    choice = ens.autotune(reps=2)
    torch.cuda.synchronize()
    tune_s = time.perf_counter() - t0
    ens.step(3)
    torch.cuda.synchronize()
    ms_tuned = timed(steps, lambda: ens.step(1))
    # the same boxes stepped one context at a time (each its own graph launch)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for _ in range(steps):
        for b in ens.boxes:
            b.step(1)
    torch.cuda.synchronize()
    ms_separate_wall = (time.perf_counter() - t1) * 1e3 / steps
    t1 = time.perf_counter()
    for _ in range(steps):
        ens.step(1)
    torch.cuda.synchronize()
    ms_ensemble_wall = (time.perf_counter() - t1) * 1e3 / steps
    kps = ens.kernels_per_step()
    diag = [b.diagnostics()["nonfinite"] for b in ens.boxes]
    ens.close()
    picked = {}
    for c_lat, c_rows, c_dem in choice:
        key = f"lattice_threads={c_lat},row_tiles={c_rows},dem_per_cta={'default' if c_dem == 0 else 'per box'}"
        picked[key] = picked.get(key, 0) + 1
    return {"workload": f"{len(cases)} boxes, edges 64..128 (sum {nodes} nodes), {n_p} thermosensitive spheres d=8, "
                        "Ra log-uniform 1e3..1e5, D3Q19+D3Q7 FP32, Hertz, 10 DEM substeps",
            "MLUPS": round(nodes / (ms_tuned * 1e-3) / 1e6, 1), "ms_per_step": round(ms_tuned, 4),
            "ms_per_step_untuned": round(ms_default, 4),
            "particle_steps_per_s": round(n_p / (ms_tuned * 1e-3), 1),
            "graph_launches_per_step": 1, "kernels_per_step": kps,
            "wall_ms_per_step_one_graph": round(ms_ensemble_wall, 4),
            "wall_ms_per_step_box_by_box": round(ms_separate_wall, 4),
            "autotune": {"seconds": round(tune_s, 2), "chosen": picked},
            "nonfinite_boxes": int(sum(1 for d in diag if d))}


def surrogate_study(torch, flush, steps):
    """Learned coupling surrogate at scale: 384^3 D3Q19+D3Q7 with BF16
    deviation storage, 10 000 thermosensitive spheres d = 6.  The plain
    solver generates 1e6 samples (100 steps x 10 000 particles: features and
    PIBM coupling of each state); the network's linear path is fitted by least
    squares and the whole network trained by Adam on the GPU; then the step is
    timed with and without the surrogate pipeline (features, tensor-core
    inference, Jacobian and gate every step, the correction applied inside the
    DEM substeps and in the thermosensitive update whenever the gate is open
    at its 1% force-error bound), and the surrogate run is compared with a
    plain run from the same state after the same number of steps."""
    import numpy as np

    from paper_1502_01159_gb300 import Simulation
    case, _ = workload("sed3d384", "bf16")
    nodes = 384 ** 3
    sim = Simulation(case)

    t0 = time.perf_counter()
    feats, targs = [], []
    for _ in range(100):
        sim.step(1)
        F = sim.read_particle_forces()
        feats.append(sim.read_features())
        targs.append(np.concatenate([F["F"], F["T"], F["H"][:, None]], axis=1))
    gen_s = time.perf_counter() - t0
    feat, targ = np.concatenate(feats), np.concatenate(targs)
    t0 = time.perf_counter()
    losses = sim.surrogate_train(feat, targ, epochs=10, batch=2048, lr=1e-3, seed=3)
    train_s = time.perf_counter() - t0

    def timed(s_, k):
        st = s_.stream
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        for i in range(k):
            with torch.cuda.stream(st):
                flush.fill_(i & 0xFF)
            ev[i][0].record(st)
            s_.step(1)
            ev[i][1].record(st)
        torch.cuda.synchronize()
        return statistics.mean(a.elapsed_time(b) for a, b in ev)

    sim.step(2)
    ms_plain = timed(sim, steps)
    t_enable = sim.t
    sim.surrogate_enable(True, bound=0.01, delta=0.25)
    ms_sg = timed(sim, steps)
    gate = sim.surrogate_stats()
    nonfinite = sim.diagnostics()["nonfinite"]
    J, _ = sim.read_hydro_jacobian()
    # the plain method from the same state (every step so far is deterministic)
    ref = Simulation(case)
    ref.step(t_enable)
    ref.step(sim.t - t_enable)
    a, b = sim.read_particles(), ref.read_particles()
    disp = np.max(np.abs(b["X"] - case["particles"]["X"]))
    traj = {"steps_compared": int(sim.t - t_enable),
            "max_abs_dX": float(np.max(np.abs(a["X"] - b["X"]))),
            "max_displacement_plain": float(disp),
            "rel_dU": float(np.linalg.norm(a["U"] - b["U"]) / np.linalg.norm(b["U"])),
            "max_abs_dT_p": float(np.max(np.abs(a["T_p"] - b["T_p"])))}
    for name in ("T", "uz"):
        fa, fb = sim.read_field(name), ref.read_field(name)
        base = fb - (0.5 if name == "T" else 0.0)  # T about the initial fluid temperature
        traj[f"field_{name}_rel_l2"] = float(np.linalg.norm(fa - fb) / max(np.linalg.norm(base), 1e-300))
    ref.close()
    sim.close()
    return {"workload": "384^3 D3Q19+D3Q7 BF16-deviation storage, 10000 thermosensitive spheres d=6, Hertz, "
                        "10 DEM substeps; 12-feature 3x64 tanh MLP with a least-squares linear path, BF16 "
                        "tensor-core inference",
            "samples": int(feat.shape[0]), "generate_s": round(gen_s, 2), "train_s": round(train_s, 2),
            "loss_first_last_epoch": [round(float(losses[0]), 5), round(float(losses[-1]), 5)],
            "ms_per_step_plain": round(ms_plain, 4), "ms_per_step_surrogate": round(ms_sg, 4),
            "pipeline_ms": round(ms_sg - ms_plain, 4),
            "MLUPS_plain": round(nodes / (ms_plain * 1e-3) / 1e6, 1),
            "MLUPS_surrogate": round(nodes / (ms_sg * 1e-3) / 1e6, 1),
            "speedup_vs_plain": round(ms_plain / ms_sg, 3),
            "gate_bound": 0.01, "gate": gate,
            "applied_jacobian_mean_diag": {"J_FU": float(np.mean(J[:, [0, 4, 8]])),
                                           "J_TW": float(np.mean(J[:, [9, 13, 17]])),
                                           "J_HT": float(np.mean(J[:, 18]))},
            "trajectory_vs_plain": traj,
            "gain": "light particles (rho_p/rho_f = 0.6) and small heat capacities (C_p = 10 for a disk of "
                    "diameter 10) that the plain explicit coupling cannot hold stay bounded with the network's "
                    "Jacobian (tests/test_gpu_surrogate.py)",
            "nonfinite": nonfinite}


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    solo = rank == 0 and world == 1
    # the oracle baselines run in a process of their own (started before the first GPU call)
    bg = None
    if solo and not args.no_oracle_baselines and not args.study:
        bg = subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-baselines-json"],
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
        __graft_entry__.build()

    if args.study:  # one study alone (profiling runs), its JSON object on one line
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
        fn = {"surrogate": surrogate_study, "ensemble": ensemble_study}[args.study]
        print(json.dumps({"study": args.study, **fn(torch, flush, max(6, args.steps // 2))}), flush=True)
        return

    case, desc = workload(args.workload, args.storage)
    nodes = case["shape"][0] * case["shape"][1] * case["shape"][2]
    n_p = len(case["particles"]["R"]) if case.get("particles") else 0

    # CPU baseline: the oracle on the workload's bounded sample, rank 0 at N = 1 only
    cpu = None
    if solo and not args.no_cpu_baseline:
        crop, crop_desc = workload(CROP[args.workload], args.storage)
        cs = max(1, args.cpu_steps)
        mlups, psps, dt = oracle_run(crop, cs, 1)
        cpu = {"value": round(mlups, 4), "unit": "MLUPS", "cores": 1, "kind": "oracle",
               "sample": f"{cs} lattice steps of {crop_desc} ({dt:.1f} s, FP64, 1 thread)",
               "particle_steps_per_s": round(psps, 1), **cpu_info()}

    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    t_wall = time.perf_counter()
    sim, ms = measure_gpu(case, args.steps, args.warmup, torch, flush)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    kt = kernel_times(sim, max(6, args.steps // 2), torch, flush)
    clocks = sampler.stop()
    ms_step = statistics.mean(ms)
    if world > 1:
        ms_step = max_over_ranks(ms_step, dist, "cuda")
        dist.barrier()
    value = job_throughput(world, nodes, ms_step)
    kps = sim.kernels_per_step()

    peak, peak_kind = peaks()
    bpn = bytes_per_node(case)
    achieved = nodes * bpn / (kt["stream_collide"] * 1e-3) / 1e9
    tkey = args.workload if args.storage == "f32" else f"{args.workload}_{args.storage}"
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic_record("k_stream_collide", tkey),
                "kernel": "k_stream_collide", "bytes_per_node": bpn, "nodes_per_launch": nodes,
                "kernel_ms": round(kt["stream_collide"], 4),
                "peak_source": f"{peak_kind} hbm_gbs (copy, burst)",
                "timing": "mean over even and odd launches, CUDA events around the kernel inside the step graph"}
    diag = sim.diagnostics()
    head = {"step_ms": round(ms_step, 4), "MLUPS": round(nodes / (ms_step * 1e-3) / 1e6, 1),
            "stream_collide_ms": round(kt["stream_collide"], 4), "stream_collide_GBs": round(achieved, 1),
            "bytes_per_node": bpn}
    if solo:  # the same kernel with blocks that divide the row, for comparison
        from paper_1502_01159_gb300 import TUNE_LATTICE_ROW_TILES
        sim.set_tuning(TUNE_LATTICE_ROW_TILES, 1)
        head["stream_collide_ms_row_tiles"] = round(kernel_times(sim, 6, torch, flush)["stream_collide"], 4)
    sim.close()
    del sim

    e2e = None
    if not args.no_e2e:
        e2e = e2e_run(case, args.steps, torch)

    extras = {}
    if solo and not args.no_extras:
        for wl in ("sed3d", "sed2d"):
            if wl == args.workload:
                continue
            c3, d3 = workload(wl)
            sim3, ms3 = measure_gpu(c3, max(6, args.steps // 2), 3, torch, flush)
            kt3 = kernel_times(sim3, 6, torch, flush)
            n3 = c3["shape"][0] * c3["shape"][1] * c3["shape"][2]
            np3 = len(c3["particles"]["R"])
            b3 = bytes_per_node(c3)
            a3 = n3 * b3 / (kt3["stream_collide"] * 1e-3) / 1e9
            m3 = statistics.mean(ms3)
            extras[wl] = {"workload": d3, "value": round(n3 / (m3 * 1e-3) / 1e6, 1), "unit": "MLUPS",
                          "ms_per_step": round(m3, 4), "particle_steps_per_s": round(np3 / (m3 * 1e-3), 1),
                          "kernel_ms": {k: round(v, 4) for k, v in kt3.items()},
                          "roofline": {"bound": "hbm", "achieved": round(a3, 1), "peak": peak, "unit": "GB/s",
                                       "frac": round(a3 / peak, 4), "traffic": traffic_record("k_stream_collide", wl),
                                       "kernel": "k_stream_collide", "bytes_per_node": b3, "nodes_per_launch": n3}}
            if wl == "sed2d":
                extras[wl]["note"] = "29 MB state: L2-resident, L2 flushed before every timed step"
            sim3.close()
        if args.workload == "sed3d384" and args.storage == "f32":
            extras["precision"] = precision_study(torch, flush, head)
        extras["ensemble"] = ensemble_study(torch, flush, max(6, args.steps // 2))
        extras["surrogate"] = surrogate_study(torch, flush, max(6, args.steps // 2))

    baselines = None
    if bg is not None:
        out, err = bg.communicate()
        try:
            baselines = json.loads(out.strip().splitlines()[-1])
        except Exception:
            baselines = {"error": (err or out)[-300:]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
            "storage": args.storage,
            "config": {"workload": desc, "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "flushed before every timed step (256 MB write); per-step device time excludes the flush",
                       "wall_s_timed_region": round(t_wall, 3)},
            "particle_steps_per_s": round(world * n_p / (ms_step * 1e-3), 1),
            "kernel_ms": {k: round(v, 4) for k, v in kt.items()},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": args.steps * kps,
            "clocks": clocks,
            "diagnostics_after": {k: diag[k] for k in ("mass", "min_height", "umax", "nonfinite")},
        }
        line.update(extras)
        if baselines is not None:
            line["oracle_baselines"] = baselines
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sed3d384", choices=["sed3d384", "sed3d", "sed2d", "sed3d_mid",
                                                                "sed3d384_mid"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"],
                    help="population storage (arithmetic is FP32 in every case)")
    ap.add_argument("--cpu-steps", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="headline only (no other workloads or studies)")
    ap.add_argument("--no-oracle-baselines", action="store_true")
    ap.add_argument("--study", choices=["surrogate", "ensemble"],
                    help="run one study alone and print its result (no headline line)")
    ap.add_argument("--oracle-baselines-json", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)  # at least 3 untimed warm-up steps
    if args.oracle_baselines_json:
        print(json.dumps(oracle_baselines()), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
