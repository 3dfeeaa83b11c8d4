#!/usr/bin/env python3
"""Throughput of the FullSWOF_2D time step on the 4096 x 4096 valley flood.

One "step" is one full Heun time step (Algorithm 1: wave-speed/dt kernel,
stage 1, stage 2 with the Heun average and sources) over every interior cell
of the grid, dry cells included; the metric is cell-updates per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Our arm times the CUDA path (libswof through its C ABI) with CUDA events on
the stream the kernels run on; the state of the valley flood evolves over
the warm-up and timed steps.  The headline is the FP32 bulk path; the FP64
path (bit-identical to the oracle) is timed on the same workload and
reported under "variants", beside the fully wet valley in FP32 and FP64
(with an ALU roofline: the operation census's arithmetic per cell-update
over the lanes' operation rate), dry-tile skipping (all cells still
counted; its final state must equal the full step's), the first-order step, D8 flow directions on a 16384^2 DEM, the 256-member
ensemble and the learned surrogate.  --impl reference times the CPU oracle
(the plain FP64 C implementation, all host cores) on the same workload.
With N > 1 (torchrun) every rank runs its own replica of the grid: the path
is one grid per GPU, so N GPUs process N grids ("replicas only").
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import signal
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gcell-updates/s at 4096^2, % HBM roofline; FP32/batch/surrogate vs FP64 plain"
UNIT = "Gcell-updates/s"
FALLBACK_HBM_GBS = 6800.0

# Algorithmic bytes per cell and launch (minimum DRAM traffic of each kernel:
# every input read once, every output written once).
BYTES = {
    "fp32": {"lambda": 12, "stage1": 12 + 8 + 12, "stage2": 12 + 8 + 12 + 12},
    "fp64": {"lambda": 24, "stage1": 24 + 8 + 24, "stage2": 24 + 8 + 24 + 24},
}
# Algorithmic bytes of a whole step with the wave speeds fused away: U^n and
# the bed read and U* written in stage 1, U*, the bed, U^n read and U^{n+1}
# written in stage 2.  FP64 reads z (17 words, 136 B); the FP32 layout reads
# the two per-face differences dz_x, dz_y instead of z (19 words, 76 B) --
# the sum of the per-kernel figures above.
STEP_BYTES = {"fp32": 76, "fp64": 136}
# The rainfall-runoff step adds Green-Ampt: K_s read, V_inf read and written
# (the FP32 layout still reads the two bed differences).
RAIN_STEP_BYTES = {"fp32": 76 + 12, "fp64": 136 + 24}
NOMINAL_HBM_GBS = 8000.0
# wall-time cap of the reference arm's timed region (the plain CPU oracle)
REFERENCE_BUDGET_S = 150.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", type=int, default=4096, help="valley grid side (cells)")
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"],
                    help="precision of the headline measurement (fp64: no variants)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tile", type=int, default=-1, help="fixed tile shape (skips the autotuner)")
    ap.add_argument("--tile2", type=int, default=-1, help="fixed stage-2 tile shape (with --tile)")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-rainfall", action="store_true", help="skip the 2048^2 rainfall-runoff workload")
    ap.add_argument("--no-dambreak", action="store_true", help="skip the 200^2 dam break")
    ap.add_argument("--ens-accuracy-every", type=int, default=8,
                    help="per-instance FP32 error of every k-th ensemble member over the full steps (0: skip)")
    ap.add_argument("--no-skip", action="store_true", help="skip the dry-tile-skipping variant")
    ap.add_argument("--no-order1", action="store_true", help="skip the first-order variant")
    ap.add_argument("--no-d8", action="store_true", help="skip the D8 flow-direction variant")
    ap.add_argument("--d8-side", type=int, default=16384)
    ap.add_argument("--no-wet", action="store_true")
    ap.add_argument("--ens-members", type=int, default=256)
    ap.add_argument("--ens-steps", type=int, default=1000)
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--unet-only", type=int, default=0, metavar="B",
                    help="only time the surrogate network's forward at batch B (randomly initialised, 256^2)")
    ap.add_argument("--sur-train-traj", type=int, default=27, help="training trajectories (750 pairs each)")
    ap.add_argument("--sur-steps", type=int, default=2000, help="training steps")
    ap.add_argument("--sur-batch", type=int, default=16)
    ap.add_argument("--sur-lr", type=float, default=2e-3)
    ap.add_argument("--sur-calls", type=int, default=50)
    ap.add_argument("--sur-members", type=int, default=512)
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def _profile_summary(kernel: str, precision: str, tile):
    """The committed ncu summary of this stage kernel (`kernel` = stage1 or
    stage2) at this tile shape [ntx, rows, form], as a dict, if it was taken
    on the current kernel source; else None."""
    if not tile or len(tile) < 3:
        return None
    ntx, h, form = tile[0], tile[1], tile[2]
    csrc = os.path.join(ROOT, "paper_1307_4839_gb300", "csrc")
    src = b"".join(open(os.path.join(csrc, f), "rb").read() for f in ("swof_kernels.cuh", "swof_sweep.cuh"))
    sha = hashlib.sha256(src).hexdigest()[:16]
    f = os.path.join(ROOT, "profiles", f"k_sweep_{kernel}_{precision}_valley4096_{ntx}x{h}_{form}.txt")
    if not os.path.exists(f):
        return None
    vals = {}
    for line in open(f):
        if ":" in line:
            k, v = line.split(":", 1)
            vals.setdefault(k.strip(), v.strip())
    name = vals.get("kernel", "")
    stage = kernel[-1]
    want = ("k_sweep_reg<" if form == "reg" else "k_sweep<") + \
        ("float" if precision == "fp32" else "double") + f", {stage}, {ntx}, {h}, 0>"
    if vals.get("kernel_source_sha256_16") != sha or want not in name:
        return None
    return vals


def recorded_metric(kernel: str, precision: str, tile, name: str):
    """A figure from the committed ncu summary of this kernel (current source,
    tile shape and form only), else None."""
    vals = _profile_summary(kernel, precision, tile)
    try:
        return float(vals[name]) if vals else None
    except (KeyError, ValueError):
        return None


def census_per_update(case: str) -> dict | None:
    """Operations per cell-update of one step of the scheme, by kind, from
    the committed operation census of the 4096^2 valley (the oracle's
    arithmetic with each value computed once), or None."""
    f = os.path.join(ROOT, "profiles", "op_census_valley4096.txt")
    try:
        for line in open(f):
            if line.startswith(case + ":"):
                return {k: float(v) for k, v in (t.split("=") for t in line.split(":", 1)[1].split())}
    except Exception:
        return None
    return None


def alu_roofline(precision: str, gcells: float, mhz: float) -> dict | None:
    """ALU roofline of a fully wet step: the census's arithmetic operations
    (add, mul, div, sqrt, cube root; each counted once) per cell-update
    times the measured rate, over the lanes' operation rate at the sampled
    SM clock: FP32 152 SMs x 128 lanes; FP64 the nominal 1.25 TFLOP/s
    (an FMA counted as 2) as 0.625 T lane operations per second at
    2070 MHz, scaled to the clock."""
    c = census_per_update("fully_wet")
    if not c or not gcells:
        return None
    peak = 152 * 128 * mhz * 1e6 if precision == "fp32" else 1.25e12 / 2 * (mhz / 2070.0)
    ach = c["flops"] * gcells * 1e9
    return {"bound": "alu", "achieved": ach * 1e-12, "peak": peak * 1e-12, "unit": "T lane-ops/s",
            "frac": ach / peak, "ops_per_cell_update": c["flops"], "all_ops_per_cell_update": c["all"],
            "sm_mhz": mhz, "census": "profiles/op_census_valley4096.txt"}


def bf16_peak() -> float:
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except Exception:
        return 1900.0


def recorded_traffic(kernel: str, precision: str, tile):
    """DRAM bytes per launch from the committed ncu summary of this kernel,
    if it was taken on the current kernel source, tile shape and form (else
    None)."""
    return recorded_metric(kernel, precision, tile, "dram_bytes_per_launch")


def recorded_d8_traffic(n: int):
    """DRAM bytes per launch of the D8 kernel from its committed ncu summary
    (taken on a smaller DEM and scaled by cells, see the summary), if the
    kernel source is unchanged since (else None)."""
    src = open(os.path.join(ROOT, "paper_1307_4839_gb300", "csrc", "swof_d8.cu"), "rb").read()
    sha = hashlib.sha256(src).hexdigest()[:16]
    f = os.path.join(ROOT, "profiles", "k_d8_vec_dem.txt")
    if not os.path.exists(f):
        return None
    vals = {}
    for line in open(f):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256_16") != sha:
        return None
    try:
        return float(vals["dram_bytes_per_cell"]) * n * n
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.send_signal(signal.SIGTERM)
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for k, name in enumerate(names):
                    if f[5 + k].lower().startswith("active"):
                        reasons.add(name)
            os.unlink(self.path)
        except Exception:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(n: int):
    import swof_inputs as si
    return si.valley(n)


def workload_name(w) -> str:
    return (f"valley flood {w.nx}x{w.ny}, dx=dy={w.dx} m, V-valley (side slope 0.15, long. slope 0.003) "
            f"+ fractal noise (1.5 m, H=0.8, seed 1), {w.extra['reservoir']} m level pool behind row "
            f"{w.extra['dam_row']}, Manning n={w.manning_n}, outflow N edge, walls elsewhere")


def time_oracle(w, steps_cap: int, budget_s: float):
    """Oracle on the full grid: steps until the time budget is used."""
    import oracle
    o = oracle.Oracle.from_workload(w)
    t0 = time.perf_counter()
    n = 0
    while n < steps_cap:
        o.step(1)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return n, dt, oracle.threads()


def time_oracle_single_thread(side: int, budget_s: float = 15.0):
    """The oracle restricted to one OpenMP thread (a fresh process, so the
    thread count is fixed before the library starts): full-grid steps of the
    same valley until the budget is used.  Returns (cells per second, steps),
    or None if the child fails."""
    code = ("import sys, time, json; sys.path.insert(0, %r); import oracle, swof_inputs as si; "
            "w = si.valley(%d); o = oracle.Oracle.from_workload(w); t0 = time.perf_counter(); n = 0\n"
            "while True:\n    o.step(1); n += 1\n    if time.perf_counter() - t0 > %f: break\n"
            "print(json.dumps({'n': n, 's': time.perf_counter() - t0, 'threads': oracle.threads()}))"
            % (ROOT, side, budget_s))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        d = json.loads(r.stdout.strip().splitlines()[-1])
        return side * side * d["n"] / d["s"], d["n"], d["threads"]
    except Exception:
        return None


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = workload(args.side)
    cells = w.nx * w.ny
    import oracle as orc
    o = orc.Oracle.from_workload(w)
    # warm-up and timed steps are full-grid oracle steps; the timed region
    # stops early (at a step boundary) once REFERENCE_BUDGET_S is used, so a
    # large --steps still ends within a few minutes: the rate is over the
    # steps actually taken, and the sample says how many
    for _ in range(args.warmup):
        o.step(1)
    t0 = time.perf_counter()
    done = 0
    while done < args.steps:
        o.step(1)
        done += 1
        if time.perf_counter() - t0 > REFERENCE_BUDGET_S:
            break
    el = time.perf_counter() - t0
    value = cells * done / el * 1e-9
    sample = f"{done} of {args.steps} full-grid steps after {args.warmup} warm-up steps"
    if done < args.steps:
        sample += f" (timed region capped at {REFERENCE_BUDGET_S:.0f} s)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / done,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(w), "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": orc.threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measure(sw, torch, w, precision: str, steps: int, warmup: int, ws: int, clocks: Clocks | None,
            autotune: bool = True, tile: int = -1, tile2: int = -1, over: dict | None = None,
            skip: bool = False, tune_tag: str = "", contract: bool = False):
    prec = sw.FP32 if precision == "fp32" else sw.FP64
    # a dedicated (non-null) stream: the kernels and the timing events share it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    s = sw.Solver.from_workload(w, prec, stream=stream.cuda_stream, **(over or {}))
    if contract:
        s.set_fp64_contraction(True)
    s.step(2)                      # a state past t = 0 for the shape choice
    if tile >= 0 or not autotune:
        shape = max(tile, 0)
        shape2 = tile2 if tile2 >= 0 else shape
        s.set_tile_shape(shape, shape2)
        tune = {"shape": [shape, shape2], "stage1": list(sw.tile_shapes()[shape]),
                "stage2": list(sw.tile_shapes()[shape2])}
    else:
        key = None
        if tune_tag:
            key = f"{sw._gpu_name()}|{w.nx}x{w.ny}|{precision}|{tune_tag}"
        tune = s.autotune(reps=3, cache=os.path.join(ROOT, "paper_1307_4839_gb300", "_build", "autotune.json"),
                          key=key)
    if skip:
        s.set_dry_tile_skip(True)
    # warm-up after the choice: the timed steps start from the fused wave
    # speeds of a previous step, as every later step does
    s.step(warmup)
    act0 = s.tile_activity() if skip else None
    torch.cuda.synchronize()
    barrier(ws)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if clocks:
        clocks.start()
    torch.cuda.synchronize()
    e0.record(stream)
    s.step(steps, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    barrier(ws)
    ms = e0.elapsed_time(e1)
    info = s.step(0)
    assert info.status == 0, f"device status {info.status}"
    act1 = s.tile_activity() if skip else None
    # per-kernel device times from a separate block of steps (CUDA events
    # around each launch, on the kernels' stream), outside the timed region
    kt = max(steps, 50)
    s.enable_timing(True)
    s.step(kt, sync=False)
    t = s.timing()
    s.enable_timing(False)
    t = {k: (v / kt if k.endswith("_ms") else v) for k, v in t.items()}
    # repetitions: 10 blocks of steps/10 (>= 10 steps each), best and median ms per step
    per = max(10, steps // 10)
    reps = []
    for _ in range(10):
        e0.record(stream)
        s.step(per, sync=False)
        e1.record(stream)
        torch.cuda.synchronize()
        reps.append(e0.elapsed_time(e1) / per)
    d = s.diagnostics()
    d["tile"] = {k: tune[k] for k in ("stage1", "stage2", "ms_stage1", "ms_stage2") if k in tune}
    forms = sw.tile_shape_forms()
    for k, st in ((0, "stage1"), (1, "stage2")):
        if st in d["tile"]:
            d["tile"][st] = list(d["tile"][st][:2]) + [forms[tune["shape"][k]]]
    d["reps"] = {"blocks": 10, "steps_each": per, "ms_per_step_best": min(reps),
                 "ms_per_step_median": statistics.median(reps)}
    if skip:
        d["live_tile_fraction"] = (act1[0] - act0[0]) / max(act1[1] - act0[1], 1)
    return ms, t, clk, d, s


def measure_d8(sw, torch, n: int, reps: int = 20):
    """D8 flow directions (Sec. 5.2) of an n x n float32 DEM: 4 B read and 1 B
    written per cell; the DEM (n^2 x 4 B) is larger than L2."""
    import swof_inputs as si
    z = torch.from_numpy(si.dem(n, n, seed=7, quantum=0.01)).cuda()
    out = torch.empty((n, n), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for _ in range(3):
            sw.flow_directions(z, out, stream=stream.cuda_stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            sw.flow_directions(z, out, stream=stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    hbm, _ = peaks()
    gbs = 5.0 * n * n / (ms * 1e-3) * 1e-9
    rec = recorded_d8_traffic(n)
    r = {"value": n * n / (ms * 1e-3) * 1e-9, "unit": "Gcells/s", "ms_per_launch": ms, "grid": [n, n],
         "launches": reps, "roofline": {"bound": "hbm", "kernel": "k_d8_vec", "achieved": gbs, "peak": hbm,
                                        "unit": "GB/s", "frac": gbs / hbm, "algorithmic_bytes_per_cell": 5,
                                        "traffic": rec},
         "what": "float32 DEM (tilted fractal, quantised to 0.01 m) -> uint8 D8 codes, one kernel"}
    if rec:
        r["roofline"]["traffic_gbs"] = rec / (ms * 1e-3) * 1e-9
    del z, out
    return r


def measure_ensemble(sw, torch, args, ws):
    """256 seeded valley scenarios of sides in {128, ..., 1024}, FP32, each
    with its own dt, advanced by one persistent launch per call."""
    import swof_inputs as si
    specs = si.ensemble_specs(args.ens_members, seed=4)
    members = [si.ensemble_member(sp) for sp in specs]
    cells = sum(w.nx * w.ny for w in members)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ens = sw.Ensemble(members, precision=sw.FP32, stream=stream.cuda_stream)
    tune = ens.autotune(steps=2, cache=os.path.join(ROOT, "paper_1307_4839_gb300", "_build", "autotune.json"))
    ens.step(3)
    torch.cuda.synchronize()
    barrier(ws)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ens.step(args.ens_steps, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), ws)
    st = ens.step(0)
    assert st == 0, f"ensemble status {st}"
    value = ws * cells * args.ens_steps / (ms * 1e-3) * 1e-9
    sizes = sorted({w.nx for w in members})
    del ens
    # the same members stepped one context at a time (plain solver), FP32 and FP64
    plain = {}
    for name, prec, k in (("fp32", sw.FP32, 20), ("fp64", sw.FP64, 3)):
        solos = [sw.Solver.from_workload(w, prec, stream=stream.cuda_stream) for w in members]
        for s_ in solos:
            s_.step(2, sync=False)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(k):
            for s_ in solos:
                s_.step(1, sync=False)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1)
        plain[name] = cells * k / (t * 1e-3) * 1e-9
        del solos
    return {"value": value, "unit": UNIT, "members": len(members), "cells": cells,
            "steps": args.ens_steps, "ms_total": ms, "launches_per_call": 1,
            "scenario_steps_per_s": ws * len(members) * args.ens_steps / (ms * 1e-3),
            "sides": sizes, "tile_by_side": tune["by_size"], "dtype": "f32",
            "what": "one persistent kernel (queue of step/phase/member/tile items) per call, CUDA graph",
            "plain_fp32_members_one_by_one": plain["fp32"], "plain_fp64_members_one_by_one": plain["fp64"],
            "over_plain_fp32": value / plain["fp32"], "over_plain_fp64": value / plain["fp64"],
            "note": "every member is wet (rain), unlike the mostly dry 4096^2 valley"}


def run_to_end(sw, torch, s, t_end: float, stream, chunk: int = 100, dt_max: float = 1.0):
    """Step a solver until its time reaches t_end (the last step is clamped
    onto it): chunks of `chunk` steps, each timed with CUDA events on the
    kernels' stream, while a chunk cannot reach t_end; then single steps.
    Returns (steps, device ms summed over the steps)."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ms = 0.0
    t = s.diagnostics()["t"]
    while t < t_end:
        k = chunk if t + chunk * dt_max < t_end else 1
        e0.record(stream)
        s.step(k, sync=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        t = s.diagnostics()["t"]
    return s.diagnostics()["steps"], ms


def measure_rainfall(sw, torch, args, hbm: float):
    """The rainfall-runoff workload: 2048^2 hillslope (dx 1 m, slope 0.05,
    furrows, noise), initially dry, 50 mm/h of rain for 600 s, Green-Ampt
    infiltration with the lognormal K_s map, Manning 0.05, outflow at the
    downslope edge, run to t = 1200 s.  FP64 with its own CFL dt (its dt
    sequence is the FP32 run's and the accuracy reference); FP32 on that
    sequence (the same steps; relative L1 at the end time); the oracle on a
    bounded sample of full-grid steps from t = 0 on the host cores."""
    import swof_inputs as si
    w = si.hillslope(2048)
    cells = w.nx * w.ny
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    out = {"workload": "rainfall runoff 2048x2048, dx=1 m, hillslope 0.05 + furrows + noise, 50 mm/h for 600 s, "
                       "Green-Ampt (lognormal K_s, psi 0.1 m, dtheta 0.3), Manning 0.05, outflow downslope, "
                       "t_end 1200 s", "unit": UNIT}
    # shapes: tuned on a wet state (t ~ 100 s), then a fresh run from t = 0
    tunes = {}
    for name, prec in (("fp64", sw.FP64), ("fp32", sw.FP32)):
        s = sw.Solver.from_workload(w, prec, stream=stream.cuda_stream)
        s.step(150)
        tunes[name] = s.autotune(reps=2)["shape"]
        s.close()
    s64 = sw.Solver.from_workload(w, sw.FP64, stream=stream.cuda_stream)
    s64.set_tile_shape(*tunes["fp64"])
    n64, ms64 = run_to_end(sw, torch, s64, w.t_end, stream)
    dts = s64.dt_history(n64)
    a = s64.state() + (s64.infiltrated(),)
    s64.close()
    s32 = sw.Solver.from_workload(w, sw.FP32, stream=stream.cuda_stream)
    s32.set_tile_shape(*tunes["fp32"])
    s32.set_dt_sequence(dts)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    s32.step(n64, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms32 = e0.elapsed_time(e1)
    assert s32.step(0).status == 0
    b = s32.state() + (s32.infiltrated(),)
    s32.close()
    rel = {f: float(np.abs(y - x).sum() / max(np.abs(x).sum(), 1e-300))
           for f, x, y in zip(("h", "hu", "hv", "V_inf"), a, b)}
    rel["hu_vs_discharge"] = float(np.abs(b[1] - a[1]).sum() / max(np.hypot(a[1], a[2]).sum(), 1e-300))
    for name, n, ms in (("fp64", n64, ms64), ("fp32", n64, ms32)):
        v = cells * n / (ms * 1e-3) * 1e-9
        out[name] = {"value": v, "steps": int(n), "ms_total": ms, "ms_per_step": ms / n,
                     "tile": [list(sw.tile_shapes()[k]) + [k] for k in tunes[name]],
                     "step_bytes_per_cell": RAIN_STEP_BYTES[name],
                     "step_frac_of_hbm": RAIN_STEP_BYTES[name] * v * 1e9 * 1e-9 / hbm}
    out["fp32"]["rel_l1_vs_fp64_at_t_end"] = rel
    out["fp32_over_fp64"] = out["fp32"]["value"] / out["fp64"]["value"]
    if not args.no_cpu_baseline:
        import oracle
        o = oracle.Oracle.from_workload(w)
        t0 = time.perf_counter()
        k = 0
        while time.perf_counter() - t0 < 10.0:
            o.step(1)
            k += 1
        el = time.perf_counter() - t0
        out["cpu_oracle"] = {"value": cells * k / el * 1e-9, "cores": oracle.threads(),
                             "sample": f"{k} full-grid FP64 steps from t = 0"}
        out["fp64_over_oracle"] = out["fp64"]["value"] / out["cpu_oracle"]["value"]
    return out


def measure_dam_break(sw, torch):
    """The 200^2 dam break to t = 1 s (flat bed, walls, h = 1 | 0.5 m): FP64
    and FP32, each with its own CFL dt; the whole run is one graph-replayed
    swof_step call.  40,000 cells: launch-bound, so steps/s is the figure."""
    import swof_inputs as si
    w = si.dam_break(200)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    out = {"workload": "dam break 200x200, dx=0.05 m, h 1.0 | 0.5 m, walls, t_end 1 s"}
    for name, prec in (("fp64", sw.FP64), ("fp32", sw.FP32)):
        s = sw.Solver.from_workload(w, prec, stream=stream.cuda_stream)
        s.step(2)
        shape = s.autotune(reps=3)["shape"]
        s.close()
        s = sw.Solver.from_workload(w, prec, stream=stream.cuda_stream)
        s.set_tile_shape(*shape)
        n = 0
        while s.step(1).t < w.t_end:          # the step count of the run (own CFL dt)
            n += 1
        n += 1
        reps = []
        for _ in range(3):
            r = sw.Solver.from_workload(w, prec, stream=stream.cuda_stream)
            r.set_tile_shape(*shape)
            r.use_graph(True)
            r.step(n)                          # capture + a first replay
            r.set_state(w.h, w.qx, w.qy)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            r.step(n, sync=False)
            e1.record(stream)
            torch.cuda.synchronize()
            reps.append(e0.elapsed_time(e1))
            r.close()
        ms = min(reps)
        out[name] = {"steps": n, "ms_run": ms, "steps_per_s": n / (ms * 1e-3), "tile": list(shape),
                     "value": w.nx * w.ny * n / (ms * 1e-3) * 1e-9, "unit": UNIT, "launches_per_step": 3}
        s.close()
    return out


def ensemble_accuracy(sw, every: int, steps: int):
    """Per-instance FP32 error of the ensemble: every `every`-th of the 256
    members, FP64 ensemble (bit for bit the oracle's members) then the FP32
    ensemble on each member's FP64 dt sequence; relative L1 per field after
    `steps` steps."""
    import swof_inputs as si
    specs = si.ensemble_specs(256, seed=4)
    ws = [si.ensemble_member(specs[k]) for k in range(0, len(specs), every)]
    e64 = sw.Ensemble(ws, precision=sw.FP64)
    assert e64.step(steps) == 0
    ref = [(e64.member(k).state(), e64.member(k).dt_history(steps)) for k in range(len(ws))]
    e64.close()
    e32 = sw.Ensemble(ws, precision=sw.FP32)
    for k in range(len(ws)):
        e32.member(k).set_dt_sequence(ref[k][1])
    assert e32.step(steps) == 0
    per = []
    for k in range(len(ws)):
        a, b = ref[k][0], e32.member(k).state()
        r = {f: float(np.abs(y - x).sum() / max(np.abs(x).sum(), 1e-300))
             for f, x, y in zip(("h", "hu", "hv"), a, b)}
        # the cross-valley discharge against the discharge vector (~0 in the pools)
        r["hu_vs_discharge"] = float(np.abs(b[1] - a[1]).sum() / max(np.hypot(a[1], a[2]).sum(), 1e-300))
        r["side"] = ws[k].nx
        per.append(r)
    e32.close()
    summ = {f: {"max": max(r[f] for r in per), "median": statistics.median(r[f] for r in per),
                "members_within_1e-5": sum(r[f] <= 1e-5 for r in per)} for f in ("h", "hu", "hv", "hu_vs_discharge")}
    return {"members": len(ws), "every": every, "steps": steps, "summary": summ,
            "per_member": [{k: (round(v, 9) if isinstance(v, float) else v) for k, v in r.items()} for r in per]}


def measure_fp32_accuracy(sw):
    """Relative L1 of the FP32 path against the FP64 path (which equals the
    CPU oracle bit for bit, tests/test_gpu_parity.py) per workload: the dam
    break to t = 1 s (each with its own CFL dt), the 4096^2 valley and the
    2048^2 rainfall hillslope on the FP64 dt sequence, lake-at-rest drift."""
    import numpy as np
    import swof_inputs as si

    def rel(a, b):
        return float(np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300))

    out = {}
    w = si.dam_break(200)
    st = {}
    for name, prec in (("fp64", sw.FP64), ("fp32", sw.FP32)):
        s = sw.Solver.from_workload(w, prec)
        for _ in range(5000):
            if s.step(1).t >= w.t_end:
                break
        st[name] = s.state()
        s.close()
    out["dam_break_200_t1s"] = {"h": rel(st["fp32"][0], st["fp64"][0]), "hu": rel(st["fp32"][1], st["fp64"][1])}
    # the valley to its end (2000 steps) with the error after 200 steps on the
    # way (the rainfall workload's end time is measured with its throughput)
    for name, w, marks in (("valley_4096", si.valley(4096), (200, 2000)),):
        s64 = sw.Solver.from_workload(w, sw.FP64)
        s32 = sw.Solver.from_workload(w, sw.FP32)
        done = 0
        for n in marks:
            s64.step(n - done)
            dts = s64.dt_history(n)[done:]
            a = s64.state() + (s64.infiltrated(),)
            s32.set_dt_sequence(dts)
            s32.step(n - done)
            b = s32.state() + (s32.infiltrated(),)
            r = {f: rel(y, x) for f, x, y in zip(("h", "hu", "hv", "V_inf"), a, b) if np.abs(x).sum() > 0}
            r["hu_vs_discharge"] = float(np.abs(b[1] - a[1]).sum() / max(np.hypot(a[1], a[2]).sum(), 1e-300))
            r["t_s"] = s64.diagnostics()["t"]
            out[f"{name}_{n}_steps"] = r
            done = n
        s64.close()
        s32.close()
    w = si.lake_at_rest(n=64, level=1.0)
    s = sw.Solver.from_workload(w, sw.FP32)
    s.step(1000)
    h, qx, qy = s.state()
    wet = w.h > 0
    out["lake_at_rest_64_1000_steps"] = {"max_surface_drift_m": float(np.max(np.abs((h + w.z)[wet] - 1.0))),
                                         "max_abs_q": float(max(np.abs(qx).max(), np.abs(qy).max()))}
    s.close()
    out["target"] = "relative L1 <= 1e-5 (FP32 vs FP64)"
    return out


def unet_flops(layout, H: int) -> float:
    """Multiply-adds x 2 of one forward sample over the real (unpadded)
    channels: the algorithmic FLOPs of the network."""
    level = [0, 0, 1, 1, 2, 2, 3, 3, 3, 2, 2, 2, 1, 1, 1, 0, 0, 0]
    fl = 0.0
    for l, d in enumerate(layout):
        taps = 9 if d["kind"] == 0 else 1
        fl += 2.0 * d["ncols"] * taps * d["cin"] * (H >> level[l]) ** 2
    return fl


def measure_surrogate(sw, torch, args, peak_tf):
    """The learned surrogate on coarsened rainfall-runoff hillslopes.

    Fine scenarios: 1024^2 hillslopes (dx 1 m, slope 0.05, furrows, noise,
    lognormal K_s, Green-Ampt, Manning 0.05, outflow downslope) with rain
    U(30, 80) mm/h for 600 s, stepped 1200 s at a fixed dt of 0.1 s (CFL
    checked each step) by the FP32 solver; every 16 steps (1.6 s) the state
    is coarsened 4 x 4 to 256^2.  27 training trajectories give 20,250
    pairs; 4 more are held out.  The base-32 U-Net is trained on the GPU,
    then 512 held-out members (4 trajectories x 128 start times) are rolled
    50 calls (800 fine steps each) with the checks and the fallback.  The
    accuracy judge is the fine solver coarsened (FP32 for all members, FP64
    for the members of one trajectory)."""
    import numpy as np
    from paper_1307_4839_gb300 import surrogate as S
    n, f, dt, span_steps, n_spans = 1024, 4, 0.1, 16, 750
    n_tr, n_te = args.sur_train_traj, 4
    rng = np.random.default_rng(11)
    rain = rng.uniform(30.0, 80.0, n_tr + n_te)
    works = S.hillslope_works(n, seeds=range(n_tr + n_te), rain_mm_h=rain, rain_s=600.05)
    t0 = time.perf_counter()
    ds = S.generate(works, f, dt, span_steps, n_spans)
    gen_s = time.perf_counter() - t0
    pairs = ds.pairs(range(n_tr))
    net = S.make_net(ds, pairs, base=32, max_batch=64, seed=0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    t0 = time.perf_counter()
    losses = S.train(net, ds, pairs, steps=args.sur_steps, batch=args.sur_batch, lr=args.sur_lr, seed=0,
                     stream=stream.cuda_stream)
    train_s = time.perf_counter() - t0
    per = max(1, args.sur_members // n_te)
    span_max = n_spans - args.sur_calls
    starts = [int(round(k * span_max / per)) for k in range(per)]
    members = [(n_tr + i, k) for i in range(n_te) for k in starts][: args.sur_members]
    ro = S.Rollout(ds, net, members)
    start = ro.states[:, :S.OUT_CH].clone()
    # untimed first call on a copy (graph capture of the fallback solvers)
    warm = S.Rollout(ds, net, members[:32])
    warm.run(1, stream=stream.cuda_stream)
    warm.close()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    acc, chk = ro.run(args.sur_calls, stream=stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    judge = ro.judge()
    e_sur = S.rel_l1(ro.states, judge)
    e_per = S.rel_l1(start, judge)
    e_crs = S.rel_l1(S.coarse_baseline(ds, members, args.sur_calls), judge)
    # FP64 judge for the members of the first held-out trajectory
    k_need = max(k for a, k in members if a == n_tr) + args.sur_calls
    ds64 = S.generate([works[n_tr]], f, dt, span_steps, k_need, precision=sw.FP64)
    sel = [b for b, (a, _) in enumerate(members) if a == n_tr]
    idx = torch.tensor([k + args.sur_calls for a, k in members if a == n_tr], device="cuda")
    j64 = ds64.data[0].index_select(0, idx)[:, :S.OUT_CH]
    e_sur64 = S.rel_l1(ro.states[sel], j64)
    e_judge = S.rel_l1(judge[sel], j64)
    ro.close()
    # forward throughput of the network alone (tensor cores)
    B = 64
    x = ro.states[:B].contiguous()
    y = torch.empty((B, S.OUT_CH) + tuple(x.shape[-2:]), device="cuda")
    for _ in range(2):
        net.predict(x, y, stream=stream.cuda_stream)
    e0.record(stream)
    for _ in range(5):
        net.predict(x, y, stream=stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1) / 5
    fl = unet_flops(net.layout(), x.shape[-1])
    # the plain fine solvers on one of these scenarios
    plain = {}
    for name, prec, k in (("fp64", sw.FP64, 48), ("fp32", sw.FP32, 480)):
        s_ = sw.Solver.from_workload(works[n_tr], prec, dt_fixed=dt, t_end=1e30, stream=stream.cuda_stream)
        s_.step(16)
        torch.cuda.synchronize()
        e0.record(stream)
        s_.step(k, sync=False)
        e1.record(stream)
        torch.cuda.synchronize()
        plain[name] = n * n * k / (e0.elapsed_time(e1) * 1e-3) * 1e-9
        s_.close()
    spans = len(members) * args.sur_calls
    eff = spans * span_steps * n * n / (ms * 1e-3) * 1e-9
    ch = ["h", "hu", "hv", "V_inf"]
    out = {"value": eff, "unit": UNIT + " (fine-grid equivalent)",
           "what": "512 members x 50 calls of the BF16 tcgen05 U-Net on 4x-coarsened 1024^2 hillslopes, "
                   "positivity/mass check each call, per-member fallback to the coarse solver",
           "member_spans_per_s": spans / (ms * 1e-3), "ms_total": ms, "members": len(members),
           "calls": args.sur_calls, "fine_steps_per_call": span_steps,
           "accepted_fraction": float(acc.mean()), "worst_check": float(chk.max()),
           "over_plain_fp64": eff / plain["fp64"], "over_plain_fp32": eff / plain["fp32"],
           "plain_fp64_fine": plain["fp64"], "plain_fp32_fine": plain["fp32"],
           "rel_l1_vs_fine_fp32": dict(zip(ch, map(float, e_sur))),
           "rel_l1_vs_fine_fp64_one_traj": dict(zip(ch, map(float, e_sur64))),
           "fp32_judge_vs_fp64": dict(zip(ch, map(float, e_judge))),
           "persistence_rel_l1": dict(zip(ch, map(float, e_per))),
           "coarse_solver_rel_l1": dict(zip(ch, map(float, e_crs))),
           "training": {"pairs": int(len(pairs)), "steps": args.sur_steps, "batch": args.sur_batch,
                        "lr": args.sur_lr, "s": train_s,
                        "loss_first": float(losses[:20].mean()), "loss_last": float(losses[-20:].mean()),
                        "params": net.nparam},
           "data_generation_s": gen_s,
           "unet_forward": {"batch": B, "ms": fwd_ms, "tflops": fl * B / (fwd_ms * 1e-3) * 1e-12,
                            "frac_of_bf16_peak": fl * B / (fwd_ms * 1e-3) * 1e-12 / peak_tf,
                            "gflop_per_sample": fl * 1e-9}}
    net.close()
    del ds, ds64
    torch.cuda.empty_cache()
    return out


def unet_forward_only(sw, torch, B: int, steps: int, warmup: int):
    """The surrogate network's forward alone: base 32, 8 input and 4 output
    channels, 256^2, batch B, random weights and inputs."""
    import numpy as np
    H = 256
    net = sw.UNet(base=32, in_ch=8, out_ch=4, H=H, W=H, max_batch=B, seed=0)
    net.set_norm(np.zeros(8), np.ones(8), np.ones(4))
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    x = torch.randn(B, 8, H, H, device="cuda")
    y = torch.zeros(B, 4, H, H, device="cuda")
    for _ in range(warmup):
        net.predict(x, y, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        net.predict(x, y, stream=stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    fl = unet_flops(net.layout(), H) * B
    print(json.dumps({"what": "surrogate U-Net forward", "batch": B, "ms": ms, "tflops": fl / (ms * 1e-3) * 1e-12,
                      "frac_of_bf16_peak": fl / (ms * 1e-3) * 1e-12 / bf16_peak()}), flush=True)


def summary(value, roofline, variants, accuracy, hbm):
    """The figures of every workload in a few hundred bytes, last in the line
    (a reader that keeps only the line's tail still sees them)."""
    def g(x, *ks, nd=4):
        for k in ks:
            if not isinstance(x, dict) or k not in x:
                return None
            x = x[k]
        return float(f"{x:.{nd}g}") if isinstance(x, (int, float)) else x
    v = variants
    out = {"valley4096_fp32_G": g({"v": value}, "v"), "valley4096_fp32_stage2_hbm_frac": g(roofline, "frac", nd=3),
           "valley4096_fp32_step_hbm_frac": g(roofline, "step_frac_of_hbm", nd=3),
           "valley4096_fp64_G": g(v, "fp64", "value"), "valley4096_fp64_contracted_G": g(v, "fp64_contracted", "value"),
           "valley4096_fp64_step_hbm_frac": g(v, "fp64", "hbm_frac_algorithmic", nd=3),
           "valley4096_fp32_fully_wet_G": g(v, "fp32_fully_wet", "value"),
           "valley4096_fp32_fully_wet_stage2_hbm_frac": g(v, "fp32_fully_wet", "stage2_hbm_frac", nd=3),
           "valley4096_fp64_fully_wet_G": g(v, "fp64_fully_wet", "value"),
           "rainfall2048_fp32_G": g(v, "rainfall", "fp32", "value"), "rainfall2048_fp64_G": g(v, "rainfall", "fp64", "value"),
           "rainfall2048_fp32_step_hbm_frac": g(v, "rainfall", "fp32", "step_frac_of_hbm", nd=3),
           "rainfall2048_oracle_G": g(v, "rainfall", "cpu_oracle", "value"),
           "dam_break200_steps_per_s": {k: g(v, "dam_break", k, "steps_per_s") for k in ("fp64", "fp32")},
           "ensemble256_fp32_G": g(v, "ensemble", "value"),
           "ensemble_fp32_rel_l1_max": {f: g(v, "ensemble", "fp32_accuracy", "summary", f, "max", nd=3)
                                        for f in ("h", "hu", "hv", "hu_vs_discharge")},
           "surrogate_G_fine_equiv": g(v, "surrogate", "value"), "surrogate_accepted": g(v, "surrogate", "accepted_fraction", nd=3),
           "unet_fwd_bf16_frac": g(v, "surrogate", "unet_forward", "frac_of_bf16_peak", nd=3),
           "fp32_rel_l1_end_time": {
               "valley4096_2000": {f: g(accuracy, "valley_4096_2000_steps", f, nd=3) for f in ("h", "hu", "hv")},
               "rainfall2048_1200s": {f: g(v, "rainfall", "fp32", "rel_l1_vs_fp64_at_t_end", f, nd=3)
                                      for f in ("h", "hv", "V_inf", "hu_vs_discharge")}}}
    return out


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    import torch

    import paper_1307_4839_gb300 as sw
    sw.build()
    sw.load()
    torch.cuda.set_device(local)
    if args.unet_only:
        unet_forward_only(sw, torch, args.unet_only, args.steps, args.warmup)
        return
    w = workload(args.side)
    cells = w.nx * w.ny
    hbm, peak_kind = peaks()

    clocks = Clocks(local)
    P = args.precision
    ms, t, clk, diag, solver = measure(sw, torch, w, P, args.steps, args.warmup, ws, clocks,
                                       not args.no_autotune, args.tile, args.tile2)
    ms_max = max_over_ranks(ms, ws)
    ms_step = ms_max / args.steps
    value = ws * cells / (ms_step * 1e-3) * 1e-9

    avg = {"lambda": t["lambda_ms"], "stage1": t["stage1_ms"], "stage2": t["stage2_ms"]}
    dom = max(avg, key=avg.get)
    achieved = BYTES[P][dom] * cells / (avg[dom] * 1e-3) * 1e-9
    tname = "float" if P == "fp32" else "double"
    roofline = {"bound": "hbm", "kernel": f"k_sweep<{tname},{dom[-1]}>" if dom != "lambda" else f"k_lambda<{tname}>",
                "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "peak_kind": f"{peak_kind} copy bandwidth (burst)",
                "traffic": recorded_traffic(dom, P, diag["tile"].get(dom)) if dom != "lambda" else None,
                "algorithmic_bytes_per_cell": BYTES[P][dom],
                "kernel_ms": {kk: round(v, 5) for kk, v in avg.items()},
                "step_frac_of_hbm": STEP_BYTES[P] * cells / (ms_step * 1e-3) * 1e-9 / hbm,
                "step_bytes_per_cell": STEP_BYTES[P],
                "frac_of_nominal_8tbs": achieved / NOMINAL_HBM_GBS,
                "timing": "per-kernel CUDA events around every launch of a separate block of max(K, 50) steps "
                          "right after the timed region (the K timed steps run without them)"}
    # The FP32 stage kernels are bound by instruction issue, not bytes: the
    # issue roofline is one warp instruction per cycle per SM sub-partition
    # (4 per SM, 152 SMs) at the SM clock sampled during the timed region;
    # the instruction count per launch comes from the committed ncu capture
    # of this kernel (current source and tile shape only).
    winst = recorded_metric(dom, P, diag["tile"].get(dom), "warp instructions executed") if dom != "lambda" else None
    mhz = (clk or {}).get("sm_mhz") or 2070.0
    if winst:
        peak_gi = 152 * 4 * mhz * 1e-3                 # G warp instructions / s
        ach_gi = winst / (avg[dom] * 1e-3) * 1e-9
        roofline["issue"] = {"warp_instructions_per_launch": winst, "achieved_ginst_s": ach_gi,
                             "peak_ginst_s": peak_gi, "frac": ach_gi / peak_gi, "sm_mhz": mhz,
                             "issue_active_pct_ncu": recorded_metric(dom, P, diag["tile"].get(dom), "issue active %")}
    if roofline["traffic"]:
        roofline["traffic_gbs"] = roofline["traffic"] / (avg[dom] * 1e-3) * 1e-9
        roofline["traffic_frac"] = roofline["traffic_gbs"] / hbm

    variants = {}
    if not args.no_fp64 and P == "fp32":
        k64 = max(20, args.steps // 4)
        ms64, t64, _, d64, s64 = measure(sw, torch, w, "fp64", k64, args.warmup, ws, None,
                                         not args.no_autotune, args.tile)
        ms64 = max_over_ranks(ms64, ws)
        v64 = ws * cells / (ms64 / k64 * 1e-3) * 1e-9
        avg64 = {"lambda": t64["lambda_ms"], "stage1": t64["stage1_ms"], "stage2": t64["stage2_ms"]}
        variants["fp64"] = {"value": v64, "unit": UNIT, "ms_per_step": ms64 / k64, "steps": k64,
                            "fp32_over_fp64": value / v64,
                            "kernel_ms": {kk: round(v, 4) for kk, v in avg64.items()},
                            "hbm_frac_algorithmic": STEP_BYTES["fp64"] * cells / (ms64 / k64 * 1e-3) * 1e-9 / hbm,
                            "bound": "alu (FP64 pipe)", "tile": d64["tile"],
                            "fp64_pipe_active_pct_ncu": {
                                st: recorded_metric(st, "fp64", d64["tile"].get(st), "FP64 pipe %")
                                for st in ("stage1", "stage2")}}
        del s64
        # the same with multiply-add contraction (within 1e-12 of the oracle
        # under its dt sequence instead of bit for bit)
        msc, tc, _, dc, sc = measure(sw, torch, w, "fp64", k64, args.warmup, ws, None,
                                     not args.no_autotune, args.tile, tune_tag="contracted", contract=True)
        msc = max_over_ranks(msc, ws)
        vc = ws * cells / (msc / k64 * 1e-3) * 1e-9
        variants["fp64_contracted"] = {
            "value": vc, "unit": UNIT, "ms_per_step": msc / k64, "steps": k64,
            "over_fp64_exact": vc / v64,
            "kernel_ms": {kk: round(tc[kk + "_ms"], 4) for kk in ("lambda", "stage1", "stage2")},
            "hbm_frac_algorithmic": STEP_BYTES["fp64"] * cells / (msc / k64 * 1e-3) * 1e-9 / hbm,
            "tile": dc["tile"],
            "parity": "relative L-inf <= 1e-12 against the oracle under its dt sequence (not bit for bit)"}
        del sc

    if P == "fp32" and not args.no_wet:
        # the same grid fully wet (0.5 m of water added everywhere): no dry-face shortcuts
        import copy
        wet = copy.copy(w)
        wet.h = w.h + 0.5
        msw, tw, _, dw, sw_ = measure(sw, torch, wet, "fp32", max(20, args.steps // 4), args.warmup, ws, None,
                                      not args.no_autotune, args.tile, tune_tag="fully_wet")
        kw_ = max(20, args.steps // 4)
        msw = max_over_ranks(msw, ws)
        vw = ws * cells / (msw / kw_ * 1e-3) * 1e-9
        avgw = {"lambda": tw["lambda_ms"], "stage1": tw["stage1_ms"], "stage2": tw["stage2_ms"]}
        variants["fp32_fully_wet"] = {
            "value": vw, "unit": UNIT, "ms_per_step": msw / kw_, "steps": kw_,
            "kernel_ms": {kk: round(v, 5) for kk, v in avgw.items()},
            "stage2_hbm_frac": BYTES["fp32"]["stage2"] * cells / (avgw["stage2"] * 1e-3) * 1e-9 / hbm,
            "alu": alu_roofline("fp32", vw, mhz), "tile": dw["tile"],
            "what": "valley DEM with 0.5 m of water added to every cell"}
        del sw_
        if not args.no_fp64:
            # FP64 fully wet: every cell does the whole scheme, so the FP64
            # pipe bounds it; fixed tile shape (the FP64 valley's default)
            kw64 = 10
            ms6, t6, _, _, s6 = measure(sw, torch, wet, "fp64", kw64, 3, ws, None, False, 0)
            ms6 = max_over_ranks(ms6, ws)
            v6 = ws * cells / (ms6 / kw64 * 1e-3) * 1e-9
            variants["fp64_fully_wet"] = {
                "value": v6, "unit": UNIT, "ms_per_step": ms6 / kw64, "steps": kw64,
                "kernel_ms": {kk: round(t6[kk + "_ms"], 4) for kk in ("lambda", "stage1", "stage2")},
                "alu": alu_roofline("fp64", v6, mhz),
                "what": "valley DEM with 0.5 m of water added to every cell"}
            del s6

    if P == "fp32" and not args.no_skip:
        # the same workload with dry-tile skipping (all cells still counted):
        # exact, so its state must equal the full step's after the same steps
        mss, ts, _, ds, ss = measure(sw, torch, w, "fp32", args.steps, args.warmup, ws, None,
                                     not args.no_autotune, args.tile, args.tile2, skip=True)
        mss = max_over_ranks(mss, ws)
        ks = args.steps
        avgs = {"lambda": ts["lambda_ms"], "stage1": ts["stage1_ms"], "stage2": ts["stage2_ms"]}
        same = all(np.array_equal(a, b) for a, b in zip(ss.state(), solver.state()))
        variants["fp32_dry_tile_skip"] = {
            "value": ws * cells / (mss / ks * 1e-3) * 1e-9, "unit": UNIT, "ms_per_step": mss / ks, "steps": ks,
            "over_full_step": (ms_step) / (mss / ks),
            "live_tile_fraction": ds["live_tile_fraction"],
            "tile": {"stage1": list(sw.tile_shapes()[4]), "stage2": list(sw.tile_shapes()[4])},
            "kernel_ms": {kk: round(v, 5) for kk, v in avgs.items()},
            "state_equal_to_full_step": bool(same),
            "what": "same valley and steps; a tile whose 3x3 tile neighbourhood held no water after the last "
                    "step (no rain, no imposed edge) is left alone; all cells counted"}
        del ss

    if P == "fp32" and not args.no_order1:
        k1 = max(20, args.steps // 4)
        ms1, t1, _, d1, s1 = measure(sw, torch, w, "fp32", k1, args.warmup, ws, None, not args.no_autotune,
                                     args.tile, args.tile2, over={"order": sw.ORDER_1, "cfl": 1.0})
        ms1 = max_over_ranks(ms1, ws)
        avg1 = {"dt": t1["lambda_ms"], "stage": t1["stage1_ms"], "commit": t1["stage2_ms"]}
        variants["fp32_first_order"] = {
            "value": ws * cells / (ms1 / k1 * 1e-3) * 1e-9, "unit": UNIT, "ms_per_step": ms1 / k1, "steps": k1,
            "kernel_ms": {kk: round(v, 5) for kk, v in avg1.items()},
            "step_bytes_per_cell": 56,
            "step_frac_of_hbm": 56 * cells / (ms1 / k1 * 1e-3) * 1e-9 / hbm,
            "what": "same valley, first-order variant (Sec. 3.3): no reconstruction, one Euler stage, "
                    "n_CFL = 1; stage (32 B/cell) + step end (24 B/cell)"}
        del s1

    if not args.no_d8 and P == "fp32":
        variants["d8"] = measure_d8(sw, torch, args.d8_side)

    if not args.no_ensemble and P == "fp32":
        variants["ensemble"] = measure_ensemble(sw, torch, args, ws)
        if args.ens_accuracy_every > 0:
            variants["ensemble"]["fp32_accuracy"] = ensemble_accuracy(sw, args.ens_accuracy_every, args.ens_steps)

    if not args.no_rainfall and P == "fp32":
        variants["rainfall"] = measure_rainfall(sw, torch, args, hbm)

    if not args.no_dambreak and P == "fp32":
        variants["dam_break"] = measure_dam_break(sw, torch)

    if not args.no_surrogate and P == "fp32":
        variants["surrogate"] = measure_surrogate(sw, torch, args, bf16_peak())

    accuracy = measure_fp32_accuracy(sw) if (P == "fp32" and not args.no_accuracy) else None


    e2e = None
    if not args.no_e2e:
        S = args.e2e_steps
        s = sw.Solver.from_workload(w, sw.FP32)
        # the caller's state lives in pinned host memory
        pin = [torch.empty((w.ny, w.nx), dtype=torch.float64, pin_memory=True).numpy() for _ in range(6)]
        for dst, src in zip(pin[:3], (w.h, w.qx, w.qy)):
            dst[...] = src
        h, qx, qy = pin[:3]
        s.set_state(h, qx, qy)
        s.step(2)
        s.state(out=pin[3:])
        # three calls, each from the same host state; the median call counts
        calls = []
        for _ in range(3):
            barrier(ws)
            t0 = time.perf_counter()
            s.set_state(h, qx, qy)
            s.step(S, sync=False)
            out = s.state(out=pin[3:])
            calls.append(time.perf_counter() - t0)
        el = max_over_ranks(statistics.median(calls), ws)
        h2d = sum(a.nbytes for a in (h, qx, qy))          # float64 host arrays in
        d2h = sum(a.nbytes for a in pin[3:])              # and out
        e2e = {"value": ws * cells * S / el * 1e-9, "unit": UNIT,
               "h2d_bytes_per_step": h2d / S, "d2h_bytes_per_step": d2h / S,
               "steps_per_call": S, "call_s": [round(x, 5) for x in calls], "timing": "median of 3 calls",
               "what": "swof_set_state(pinned host float64) + swof_step(S) + swof_get_state(pinned host float64)"}
        del s, out

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        n, el, cores = time_oracle(w, 8, 12.0)
        cpu = {"value": cells * n / el * 1e-9, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n} full-grid FP64 steps of the same valley from its initial state"}
        one = time_oracle_single_thread(args.side)
        if one:
            cpu["single_thread"] = {"value": one[0] * 1e-9, "unit": UNIT, "threads": one[2],
                                    "sample": f"{one[1]} full-grid FP64 steps, one OpenMP thread"}

    launches = 3 * args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if P == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": workload_name(w), "grid": [w.nx, w.ny], "precision": "fp32 bulk, fp64 dt/time/budgets" if P == "fp32" else "fp64",
                   "l2": f"inputs larger than L2 (working set {(9 * (w.ny + 4) * (w.nx + 8) * 4) / 1e6:.0f} MB)",
                   "parallelism": "replicas" if ws > 1 else "single GPU",
                   "counted": "all interior cells, dry cells included",
                   "tile": diag["tile"], "repetitions": diag["reps"]},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "variants": variants,
        "fp32_accuracy": accuracy,
        "final_state": {"t": diag["t"], "volume": diag["volume"], "min_h": diag["min_h"]},
    }
    line["summary"] = summary(value, roofline, variants, accuracy, hbm)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
