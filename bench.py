"""Throughput of the LBM-PSM hot path on GB300.

One step = one pass of the whole hot path over the 512x512x1024 settling box
(268M cells, 94,692 spheres r in [3, 6] at solid fraction 0.15, density ratio
2.5, gravity, TRT tau = 0.55, 8^3 sub-division sampling, Noble-Torczynski
weighting, FP64 PDFs, pull streaming): particle mapping, fused stream + PSM
collide, fixed-order force/torque reduction, 10 DEM sub-cycles.  Inputs are
synthetic and seeded (random sequential addition of the spheres).

Prints one JSON line (rank 0): MLUPS of the device-resident loop (``value``,
the median of 5 timed runs of K steps), the same through the C ABI with host
buffers (``e2e``: the particle state goes host -> device and the forces and
particle state device -> host every step), the roofline of the dominant
kernel, the FP64 oracle on the host cores (``cpu_baseline``, one thread and
all threads, on a slab of the same box), and the metric's forms measured
against FP64 on the same GPU (``forms``).

``--impl reference`` times the FP64 oracle (the plain CPU implementation) on
all host cores on that slab and prints the same line with
``"impl": "reference"``.
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
sys.path.insert(0, ROOT)

METRIC = "LBM-PSM MLUPS and % of HBM roofline; FP32+MLP-eps vs FP64 at drag err<=0.5%"
WORKLOADS = {
    "settle128": ("settle128: 128^3 periodic box, 400 spheres r=6 (random sequential addition, "
                  "gap>=1, seed 20230321), density ratio 2.5, gravity 2e-5 in -z, D3Q19 TRT "
                  "(Lambda=3/16) tau=0.55, 4^3 sub-division sampling, Noble-Torczynski B, "
                  "spring-dashpot DEM k_n=1e3 e=0.9 x10 sub-cycles"),
    "settle512": ("settle512: 512x512x1024 periodic box (268M cells), 94,692 spheres r in [3,6] "
                  "(random sequential addition, solid fraction 0.15, seed 20230321), density "
                  "ratio 2.5, gravity 2e-5 in -z, D3Q19 TRT (Lambda=3/16) tau=0.55, 8^3 "
                  "sub-division sampling, Noble-Torczynski B, spring-dashpot DEM k_n=1e3 e=0.9 "
                  "x10 sub-cycles"),
    "settle256": ("settle256: 256^3 periodic box (16.8M cells), 5,903 spheres r in [3,6] "
                  "(random sequential addition, solid fraction 0.15, seed 20230321), density "
                  "ratio 2.5, gravity 2e-5 in -z, D3Q19 TRT (Lambda=3/16) tau=0.55, 8^3 "
                  "sub-division sampling, Noble-Torczynski B, spring-dashpot DEM x10 sub-cycles"),
    "channel": ("channel: 256x256x512, walls at the x faces, 12,817 fixed spheres r=5 (random "
                "sequential addition, solid fraction 0.20, seed 20230321), D3Q19 TRT "
                "(Lambda=3/16) tau=0.55, body force 1e-5 along z, 4^3 sub-division sampling, "
                "Noble-Torczynski B"),
    "bed_dilute": ("bed_dilute: stand-in for the paper's dilute fluidized bed, 500x200x800 cells, "
                   "no-slip walls on the four side faces, velocity inflow at the bottom (8.33e-4, "
                   "particle Reynolds number 1) and pressure outflow (density 1) at the top, 627 "
                   "spheres r=10 (random sequential addition), density ratio 1.1, gravity "
                   "2.75e-5, D3Q19 SRT tau=0.55, linear approximation (Eqs. 25-27), B = eps, DEM "
                   "x10 sub-cycles"),
    "bed_dense": ("bed_dense: stand-in for the paper's dense fluidized bed, as bed_dilute with "
                  "8,073 spheres r=10 in hexagonal close-packed layers from the bottom (solid "
                  "fraction 0.42 over the box)"),
}
HBM_FALLBACK_GBS = 6800.0
# FP64 arithmetic peak of the GPU: 2 FP64 fused multiply-adds per clock per SM
FP64_FMA_PER_CLK_SM = 2
# algorithmic FP64 flops of the collision (adds and multiplies, a fused
# multiply-add counts 2): per cell (moments, equilibrium, TRT relaxation with
# forcing, (1 - B) weighting) and per occupied slot (solid operator and force)
FLOP_PER_CELL = 219
FLOP_PER_SLOT = 139


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region.

    The sampler runs every 25 ms from before the region; `start` returns once
    the first sample is in (at most 3 s), and `stop` keeps the samples whose
    timestamps fall inside the region marked by `begin`/`end` (all samples if
    none does, with "in_region": false)."""

    QUERY = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "25"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        deadline = time.time() + 3.0
        while time.time() < deadline and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

    def begin(self):
        self.t0 = time.time()

    def end(self):
        self.t1 = time.time()

    @staticmethod
    def _stamp(text):
        try:
            day, frac = (text.split(".") + ["0"])[:2]
            return time.mktime(time.strptime(day, "%Y/%m/%d %H:%M:%S")) + float("0." + frac)
        except Exception:
            return None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        inside = rows
        if self.t0 is not None and self.t1 is not None:
            inside = [r for r in rows
                      if (ts := self._stamp(r[0])) is not None and self.t0 <= ts <= self.t1]
        in_region = bool(inside)
        rows = inside or rows
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i]
                          and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows), "in_region": in_region}


def source_hash(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def fp64_peak_tflops(sm_max_mhz, sm_count):
    return sm_count * FP64_FMA_PER_CLK_SM * 2 * sm_max_mhz * 1e6 / 1e12


def profiled_traffic(kernel_src, name, cells):
    """DRAM bytes per launch from the committed ncu summary, if the kernel
    source is unchanged since the capture; else None.  A summary taken on a
    smaller box of the same recipe gives bytes per cell
    (``dram_bytes_per_cell``), scaled here to `cells`."""
    path = os.path.join(ROOT, "profiles", f"{name}.md")
    if not os.path.exists(path):
        return None
    want = source_hash(kernel_src)
    traffic, per_cell, h = None, None, None
    for line in open(path):
        if line.startswith("source_sha256_16:"):
            h = line.split(":", 1)[1].strip()
        if line.startswith("dram_bytes_per_launch:"):
            traffic = float(line.split(":", 1)[1].strip())
        if line.startswith("dram_bytes_per_cell:"):
            per_cell = float(line.split(":", 1)[1].strip())
    if h != want:
        return None
    if per_cell:
        return per_cell * cells
    return traffic or None


def max_over_ranks(value, dist, device):
    """The largest of a per-rank value over all ranks (the whole job's time is
    that of its slowest replica); the value itself with one rank."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(cells_per_rank, steps, world, ms):
    """Whole-job throughput: every rank updates its own cells (replicas,
    weak scaling) in the job's time ms."""
    return cells_per_rank * steps * world / (ms * 1e-3) / 1e6


def make_engine(w, capi, precision="fp64", streaming="pull", eps_mode=None):
    e = capi.Engine(w.nx, w.ny, w.nz, w.tau, relax=w.relax, walls=w.walls, fbody=w.fbody,
                    weighting=w.weighting, eps_mode=eps_mode or w.eps_mode, eps_n=w.eps_n,
                    gravity=w.gravity, kn=w.kn, restitution=w.restitution,
                    subcycles=w.subcycles, dem=w.dem, precision=precision,
                    streaming=streaming, bc_velocity=w.bc_velocity, bc_density=w.bc_density)
    p = w.particles
    e.set_particles(p["x"], p["r"], density=p["density"], fixed=p["fixed"])
    return e


def timed_steps(e, torch, K):
    s = torch.cuda.current_stream()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(s)
    e.step(K)
    b.record(s)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def host_cpu():
    """CPU model name and the number of host threads."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return model, os.cpu_count() or 1


def cpu_sample_workload(name, w):
    """The bounded sample the oracle is timed on: for the large settling
    boxes, a 48-cell slab of the same box (whole x-y planes, the spheres
    inside it; see inputs.slab), else the workload itself."""
    from paper_2303_11811_gb300 import inputs
    if name in ("settle512", "settle256"):
        return inputs.slab(w, w.nz // 2 - 24, 48), f"a 48-cell z-slab of {name}"
    return w, name


def oracle_rate(w, seconds, max_steps, threads, warmup=0):
    """MLUPS of the FP64 oracle on `threads` host threads: `warmup` untimed
    steps, then steps until `seconds` (at least one, at most `max_steps`)."""
    from oracle import Oracle
    o = Oracle(w.nx, w.ny, w.nz, w.tau, relax=w.relax, walls=w.walls, fbody=w.fbody,
               weighting=w.weighting, eps_mode=w.eps_mode, eps_n=w.eps_n, gravity=w.gravity,
               kn=w.kn, restitution=w.restitution, subcycles=w.subcycles, dem=w.dem,
               bc_velocity=w.bc_velocity, bc_density=w.bc_density)
    o.set_threads(threads)
    p = w.particles
    o.set_particles(p["x"], p["r"], density=p["density"], fixed=p["fixed"])
    if warmup:
        o.step(warmup)
    n = 0
    t0 = time.perf_counter()
    while n < max_steps:
        o.step(1)
        n += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    return w.cells * n / dt / 1e6, n, dt


def run_reference(args, w, world, rank):
    """The reference arm: the FP64 oracle on all host cores, rank 0 only."""
    if rank != 0:
        return
    budget = float(os.environ.get("PSM_REFERENCE_SECONDS", "150"))
    ws, sample = cpu_sample_workload(args.workload, w)
    model, cores = host_cpu()
    value, n, dt = oracle_rate(ws, budget, args.steps, cores, warmup=min(args.warmup, 1))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": n, "warmup": args.warmup,
        "ms_per_step": dt / n * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": describe(args), "l2": "n/a (host)"},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "cpu_model": model,
                         "kind": "oracle",
                         "sample": f"{n} full steps (of {args.steps} requested, capped at "
                                   f"{budget:.0f} s) of {sample}: {ws.nx}x{ws.ny}x{ws.nz} cells, "
                                   f"{ws.particles['r'].size} spheres, on {cores} threads"},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(args, w, seconds):
    """The oracle on the bounded sample, on one thread and on all threads."""
    ws, sample = cpu_sample_workload(args.workload, w)
    model, cores = host_cpu()
    v1, n1, d1 = oracle_rate(ws, seconds, 1000, 1)
    va, na, da = oracle_rate(ws, seconds, 1000, cores)
    desc = f"{sample}: {ws.nx}x{ws.ny}x{ws.nz} cells, {ws.particles['r'].size} spheres"
    return {"value": va, "unit": "MLUPS", "cores": cores, "cpu_model": model, "kind": "oracle",
            "sample": f"{na} full steps of {desc} on {cores} threads ({da:.1f} s)",
            "single_thread": {"value": v1, "steps": n1, "seconds": d1}}


FORMS = (
    # name, PDF precision, streaming, eps mode, sampling n
    ("fp64_8cubed", "fp64", "pull", "supersample", 8),
    ("df64_8cubed", "df64", "pull", "supersample", 8),
    ("fp32_8cubed", "fp32", "pull", "supersample", 8),
    ("fp32_mlp", "fp32", "pull", "mlp", 8),
    ("fp32_mlp_aa", "fp32", "aa", "mlp", 8),
    ("fp32_4cubed", "fp32", "pull", "supersample", 4),
    ("fp32_linear", "fp32", "pull", "linear", 8),
)
CHANNEL_STEPS = 5000


def train_surrogate(capi, seed=20230321):
    """The surrogate, trained on the device by the engine's own kernels on
    2^21 samples labelled by 8^3 sub-division sampling."""
    from paper_2303_11811_gb300 import inputs
    t0 = time.perf_counter()
    trainer = capi.Engine(32, 8, 8, 0.6)
    trainer.set_mlp(capi.pack_mlp(inputs.mlp_init(1)))
    loss = trainer.train_surrogate(1 << 21, seed, epochs=10, batch=1024, lr=3e-3)
    params = trainer.get_mlp()
    trainer.close()
    return params, {"samples": 1 << 21, "epochs": 10, "batch": 1024, "final_mse": loss,
                    "seconds": time.perf_counter() - t0}


def collide_roofline(prec, cells, ncov, nslot, coll_ms, hbm, sm_count):
    if prec != "fp64":
        b = (152 * cells + 16 * ncov) if prec == "fp32" else (304 * cells + 24 * ncov)
        gbs = b / (coll_ms * 1e-3) / 1e9
        return {"collide_hbm_gbs": gbs, "collide_hbm_frac": gbs / hbm}
    tf = (FLOP_PER_CELL * cells + FLOP_PER_SLOT * nslot) / (coll_ms * 1e-3) / 1e12
    return {"collide_fp64_tflops": tf,
            "collide_fp64_frac": tf / fp64_peak_tflops(2070.0, sm_count),
            "collide_hbm_frac": (304 * cells + 24 * ncov) / (coll_ms * 1e-3) / 1e9 / hbm}


def forms_comparison(capi, torch, params, sm_count, steps=CHANNEL_STEPS):
    """The metric's second half on the channel workload (256x256x512, walls at
    the x faces, 12,817 fixed spheres r=5, TRT tau=0.55, body force 1e-5 along
    z), over the 5,000 steps the workload is defined for: FP64 PDFs with 8^3
    sub-division sampling (the reference) against FP32 deviation storage with
    the trained surrogate (8^3 fallback), and, for the surrogate's gain, FP32
    with 8^3 sampling, 4^3 sampling and the linear approximation of Eqs.
    25-27; beside them the double-float form (FP64 accuracy on the FP32
    pipes) with 8^3 sampling.  Every form runs the same steps from rest on
    the same GPU; drag error = ||F - F_ref|| / ||F_ref|| over all particles
    after the last step, velocity error likewise over the field.  Per form:
    MLUPS over the steps after the first (the first maps the fixed spheres
    once), that one-off mapping time and the collision kernel's roofline
    fraction."""
    from paper_2303_11811_gb300 import inputs
    w = inputs.channel(eps_mode="supersample", eps_n=8)
    out = {"workload": "channel 256x256x512, walls at the x faces, %d fixed spheres r=5 "
           "(solid fraction 0.20), TRT tau=0.55, body force 1e-5 along z"
           % w.particles["r"].size, "steps": steps}
    hbm, _ = peaks()
    res = {}
    for name, prec, stream, mode, n in FORMS:
        e = capi.Engine(w.nx, w.ny, w.nz, w.tau, relax=w.relax, walls=w.walls, fbody=w.fbody,
                        weighting=w.weighting, eps_mode=mode, eps_n=n, precision=prec,
                        streaming=stream)
        p = w.particles
        e.set_particles(p["x"], p["r"], density=p["density"], fixed=p["fixed"])
        if mode == "mlp":
            e.set_mlp(params)
        e.set_timing(True)
        e.step(1)  # first step maps the fixed spheres
        map_ms = e.timings()[0]
        e.set_timing(False)
        ms = timed_steps(e, torch, steps - 11)
        e.set_timing(True)
        e.step(10)  # per-class kernel times of the last 10 steps
        t = e.timings()
        e.set_timing(False)
        coll_ms = t[1] / t[4]
        p0, _, p1, _ = e.slots()
        ncov = int((p0 >= 0).sum())
        nslot = ncov + int((p1 >= 0).sum())
        F, _ = e.force_torque()
        _, u = e.macroscopic()
        r = {"mlups": w.cells * (steps - 11) / (ms * 1e-3) / 1e6, "mapping_ms_once": map_ms,
             "collide_ms": coll_ms}
        r.update(collide_roofline(prec, w.cells, ncov, nslot, coll_ms, hbm, sm_count))
        res[name] = (r, F, u)
        e.close()
        torch.cuda.empty_cache()
    _, Fr, ur = res["fp64_8cubed"]
    for name, _, _, _, _ in FORMS:
        r, F, u = res[name]
        if name != "fp64_8cubed":
            r["speedup_vs_fp64"] = r["mlups"] / res["fp64_8cubed"][0]["mlups"]
            r["drag_rel_err"] = float(np.linalg.norm(F - Fr) / np.linalg.norm(Fr))
            r["velocity_rel_err"] = float(np.linalg.norm(u - ur) / np.linalg.norm(ur))
        out[name] = r
    return out


SETTLE_FORMS = (
    # name, PDF precision, streaming, eps mode, sampling n
    ("df64_8cubed", "df64", "pull", "supersample", 8),
    ("fp32_8cubed_aa", "fp32", "aa", "supersample", 8),
    ("fp32_mlp_aa", "fp32", "aa", "mlp", 8),
    ("fp32_4cubed_aa", "fp32", "aa", "supersample", 4),
    ("fp32_linear_aa", "fp32", "aa", "linear", 8),
)


def settling_summary(w, e, mass):
    _, u, _ = e.particles()
    F, _ = e.force_torque()
    return {"mean_settling_velocity": float(np.sum(mass * u[:, 2]) / np.sum(mass)),
            "mean_drag_z": float(np.mean(F[:, 2]))}


def forms_settling(capi, torch, params, ref, steps, sm_count):
    """The moving-particle form of the metric on the 512x512x1024 periodic box
    (268M cells, 94,692 spheres r in [3, 6] at solid fraction 0.15, density
    ratio 2.5, gravity, DEM).  `ref` is the plain FP64 method (8^3 sampling,
    pull) of the main line after `steps` steps from rest; beside it the
    double-float form, and FP32 AA storage with 8^3 sampling, with the trained
    surrogate, with 4^3 sampling and with the linear approximation.  The
    spheres move, so the mapping runs every step and counts per step.  The
    flow is chaotic: the forms are compared on the mean settling velocity and
    the mean drag over all spheres after the same number of steps from rest.
    MLUPS of each form over its last K = min(steps - 5, 100) steps."""
    from paper_2303_11811_gb300 import inputs
    w = inputs.settle512()
    w.eps_n = 8
    n = w.particles["r"].size
    out = {"workload": "settle512: 512x512x1024 periodic, %d spheres r in [3,6] (solid "
           "fraction 0.15), density ratio 2.5, gravity 2e-5 in -z, TRT tau=0.55, DEM" % n,
           "steps": steps, "fp64_8cubed": ref}
    hbm, _ = peaks()
    mass = w.particles["density"] * 4.0 / 3.0 * math.pi * w.particles["r"] ** 3
    k = min(steps - 5, 100)
    for name, prec, stream, mode, en in SETTLE_FORMS:
        w.eps_n = en
        e = make_engine(w, capi, precision=prec, streaming=stream, eps_mode=mode)
        if mode == "mlp":
            e.set_mlp(params)
        e.step(steps - k - 3)
        ms = timed_steps(e, torch, k)
        e.set_timing(True)
        e.step(3)
        t = e.timings()
        e.set_timing(False)
        p0, _, p1, _ = e.slots()
        ncov = int((p0 >= 0).sum())
        nslot = ncov + int((p1 >= 0).sum())
        r = {"mlups": w.cells * k / (ms * 1e-3) / 1e6, "ms_per_step": ms / k,
             "mapping_ms_per_step": t[0] / t[4], "collide_ms": t[1] / t[4],
             "force_ms": t[2] / t[4], "dem_ms": t[3] / t[4]}
        r.update(collide_roofline(prec, w.cells, ncov, nslot, r["collide_ms"], hbm, sm_count))
        r.update(settling_summary(w, e, mass))
        r["speedup_vs_fp64"] = r["mlups"] / ref["mlups"]
        r["settling_velocity_rel_diff"] = abs(r["mean_settling_velocity"] /
                                              ref["mean_settling_velocity"] - 1.0)
        r["mean_drag_rel_diff"] = abs(r["mean_drag_z"] / ref["mean_drag_z"] - 1.0)
        out[name] = r
        e.close()
        torch.cuda.empty_cache()
    return out


def describe(args):
    prec = {"fp64": "FP64 PDFs", "fp32": "FP32 deviation PDFs",
            "df64": "double-float deviation PDFs (FP32 pairs, 8 B)"}[args.precision]
    d = f"{WORKLOADS[args.workload]}, {prec}, {args.streaming} streaming"
    if args.eps != "supersample" or args.eps_n:
        eps = {"supersample": f"{args.eps_n or 4}^3 sub-division sampling",
               "linear": "linear approximation (Eqs. 25-27)",
               "mlp": "trained surrogate with 8^3 fallback"}[args.eps]
        d += f", eps by {eps}"
    return d


def make_workload(name):
    from paper_2303_11811_gb300 import inputs
    if name == "settle256":
        w = inputs.settle512(nx=256, ny=256, nz=256)
    elif name.startswith("bed_"):
        w = inputs.bed(name[4:])
    else:
        w = {"settle128": inputs.settle128, "channel": inputs.channel,
             "settle512": inputs.settle512}[name]()
    if name in ("settle512", "settle256"):
        w.eps_n = 8
    return w


RUNS = 5  # timed runs of K steps; the line reports the median


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="settle512")
    ap.add_argument("--precision", choices=["fp64", "fp32", "df64"], default="fp64")
    ap.add_argument("--streaming", choices=["pull", "aa"], default="pull")
    ap.add_argument("--eps", choices=["supersample", "linear", "mlp"], default="supersample",
                    help="solid-fraction mode of the main line (default: the workload's)")
    ap.add_argument("--eps-n", type=int, default=0,
                    help="sub-division sampling points per axis (default: the workload's)")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--settle-steps", type=int, default=200,
                    help="steps from rest at which the settling forms are compared")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    default_run = ((args.workload, args.precision, args.streaming, args.eps, args.eps_n) ==
                   ("settle512", "fp64", "pull", "supersample", 0))

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    w = make_workload(args.workload)
    w.eps_mode = args.eps
    if args.eps_n:
        w.eps_n = args.eps_n
    elif args.eps == "mlp":
        w.eps_n = 8

    if args.impl == "reference":
        if rank != 0:
            return
        import oracle
        oracle.build()
        run_reference(args, w, world, rank)
        return

    import torch
    torch.cuda.set_device(local)
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2303_11811_gb300 import build, capi
    if rank == 0 or world == 1:
        build.build()
    if dist:
        dist.barrier()

    params = None
    if args.eps == "mlp" or (default_run and not args.no_forms and rank == 0):
        params, training = train_surrogate(capi)
    e = make_engine(w, capi, precision=args.precision, streaming=args.streaming)
    if args.eps == "mlp":
        e.set_mlp(params)
    e.step(args.warmup)
    steps_done = args.warmup
    torch.cuda.synchronize()

    # RUNS timed runs of K steps each; the clock samples of the whole span
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    clocks.begin()
    runs = []
    launches = 0
    for _ in range(RUNS):
        if dist:
            dist.barrier()
        runs.append(max_over_ranks(timed_steps(e, torch, args.steps), dist, "cuda"))
        launches = e.last_launch_count()
    clocks.end()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    steps_done += RUNS * args.steps
    ms = statistics.median(runs)
    cells = w.cells
    value = job_mlups(cells, args.steps, world, ms)

    # dominant kernel: per-class CUDA-event timings over a second pass of the
    # same loop (steps launched without graphs, events on the engine's stream)
    kr = min(args.steps, 100)
    e.set_timing(True)
    e.step(kr)
    t = e.timings()
    e.set_timing(False)
    steps_done += kr
    lbm_ms = t[1] / t[4]
    p0, _, p1, _ = e.slots()
    ncov = int((p0 >= 0).sum())
    nslot = ncov + int((p1 >= 0).sum())
    fp64 = args.precision == "fp64"
    esz = 4 if args.precision == "fp32" else 8
    bytes_lbm = cells * 19 * 2 * esz
    bytes_psm = bytes_lbm + ncov * (24 if esz == 8 else 16)
    hbm, peak_kind = peaks()
    hbm_achieved = bytes_psm / (lbm_ms * 1e-3) / 1e9
    # the collision kernel of the form: FP64 on compacted warps, FP32 AA
    # staged, FP32 pull and double-float one cell per thread
    if fp64:
        kbase, kname = "lbm_fp64_kernel", f"lbm_fp64_kernel<{args.streaming}>"
    else:
        kbase = "lbm_bulk_kernel" if args.streaming == "aa" and args.precision == "fp32" \
            else "lbm_kernel"
        kname = kbase + f"<{ {'fp32': 'float', 'df64': 'df'}[args.precision] },{args.streaming}>"
    traffic = profiled_traffic(os.path.join(ROOT, "paper_2303_11811_gb300", "csrc",
                                            "lbm_kernels.cu"),
                               f"{kbase}_{args.precision}{args.streaming}_{args.workload}", cells)
    hbm_part = {"achieved": hbm_achieved, "peak": hbm, "unit": "GB/s",
                "frac": hbm_achieved / hbm, "peak_source": peak_kind,
                "bytes_per_launch": bytes_psm, "lbm_only_bytes_per_launch": bytes_lbm}
    common = {"kernel": kname, "traffic": traffic, "covered_cells": ncov, "slots": nslot,
              "avg_launch_ms": lbm_ms,
              "class_ms_per_step": {"mapping": t[0] / t[4], "stream_collide": lbm_ms,
                                    "force_reduce": t[2] / t[4], "dem": t[3] / t[4]}}
    if fp64:
        # FP64 runs at 1/64 of the FP32 rate on this GPU: the FP64 pipe binds
        sm_max = (clk or {}).get("sm_max_mhz") or 2070.0
        peak = fp64_peak_tflops(sm_max, sm_count)
        flops = FLOP_PER_CELL * cells + FLOP_PER_SLOT * nslot
        achieved = flops / (lbm_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak,
                    "peak_source": f"derived: {sm_count} SMs x {FP64_FMA_PER_CLK_SM} FP64 "
                                   f"FMA/clk x 2 flop x {sm_max:.0f} MHz",
                    "flops_per_launch": flops, "hbm": hbm_part, **common}
    else:
        roofline = {"bound": "hbm", "achieved": hbm_achieved, "peak": hbm, "unit": "GB/s",
                    "frac": hbm_achieved / hbm, "peak_source": peak_kind,
                    "bytes_per_launch": bytes_psm, "lbm_only_bytes_per_launch": bytes_lbm,
                    **common}

    # end to end through the C ABI with host buffers in pinned memory
    n = w.particles["r"].size
    xs, us, oms = e.particles()
    hx = torch.from_numpy(xs.copy()).pin_memory()
    hu = torch.from_numpy(us.copy()).pin_memory()
    ho = torch.from_numpy(oms.copy()).pin_memory()
    hF = torch.zeros((n, 3), dtype=torch.float64).pin_memory()
    hT = torch.zeros((n, 3), dtype=torch.float64).pin_memory()
    ke = max(10, min(args.steps, 100))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(ke):
        e.update_particles(hx.data_ptr(), hu.data_ptr(), ho.data_ptr())
        e.step(1)
        e.force_torque_into(hF.data_ptr(), hT.data_ptr())
        e.particles_into(hx.data_ptr(), hu.data_ptr(), ho.data_ptr())
    torch.cuda.synchronize()
    te = time.perf_counter() - t0
    te = max_over_ranks(te, dist, "cuda")
    steps_done += ke
    e2e = {"value": job_mlups(cells, ke, world, te * 1e3), "unit": "MLUPS",
           "h2d_bytes_per_step": 3 * 3 * n * 8, "d2h_bytes_per_step": (6 + 9) * n * 8,
           "steps": ke}

    # the paper's coupling (Sec. 3.2): the same steps with the DEM on the host
    # cores, hydrodynamic forces copied to the host and the particle state
    # back every step (psm_step_host_dem), beside the engine's device DEM.
    # Its arithmetic equals the device DEM's, so the trajectory is unchanged.
    host_dem = None
    if w.dem and not bool(np.all(w.particles["fixed"])):
        kh = max(5, min(args.steps, 50))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        host_ms = e.step_host_dem(kh, threads=0)
        th = time.perf_counter() - t0
        th = max_over_ranks(th, dist, "cuda")
        steps_done += kh
        host_dem = {"mlups": job_mlups(cells, kh, world, th * 1e3), "ms_per_step": th * 1e3 / kh,
                    "host_phase_ms_per_step": host_ms / kh,
                    "device_dem_ms_per_step": t[3] / t[4],
                    "threads": min(os.cpu_count() or 1, max(1, n // 256)),
                    "steps": kh}

    forms = None
    if default_run and not args.no_forms and rank == 0:
        # the main line is the settling forms' FP64 reference: bring it to the
        # comparison step, then free its 82 GB before the other forms run
        settle_steps = max(args.settle_steps, steps_done)
        e.step(settle_steps - steps_done)
        mass = w.particles["density"] * 4.0 / 3.0 * math.pi * w.particles["r"] ** 3
        ref = {"mlups": value, "ms_per_step": ms / args.steps,
               "mapping_ms_per_step": t[0] / t[4], "collide_ms": lbm_ms,
               "force_ms": t[2] / t[4], "dem_ms": t[3] / t[4]}
        ref.update(collide_roofline("fp64", cells, ncov, nslot, lbm_ms, hbm, sm_count))
        ref.update(settling_summary(w, e, mass))
    e.close()
    torch.cuda.empty_cache()
    if default_run and not args.no_forms and rank == 0:
        forms = {"surrogate_training": training,
                 "settling": forms_settling(capi, torch, params, ref, settle_steps, sm_count),
                 "channel": forms_comparison(capi, torch, params, sm_count)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and w.eps_mode != "mlp":
        import oracle
        oracle.build()
        cpu = cpu_baseline(args, w, args.cpu_seconds)

    if rank == 0:
        ws = cells * 19 * esz * (1 if args.streaming == "aa" else 2) / 1e6
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "df64": "f32x2 (double-float)"}[args.precision],
            "data": "synthetic",
            "config": {"workload": describe(args), "cells": cells,
                       "l2": f"working set {ws:.0f} MB of PDFs > 126 MB L2, no flush",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "timing": f"median of {RUNS} runs of {args.steps} steps"},
            "runs_ms": runs, "clocks": clk, "e2e": e2e, "gpu_launches": launches,
            "roofline": roofline, "cpu_baseline": cpu, "host_dem": host_dem, "forms": forms,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
