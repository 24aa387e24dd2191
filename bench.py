#!/usr/bin/env python
"""Throughput of the fused lattice Boltzmann time step with dynamic mode III
crack propagation (arXiv 2206.12412) on GB300.

Workload: the 4096 x 2048 FP32 single run with K-criterion propagation (edge
crack to x = 512 on the midline, top/bottom ramped to +-2e-3 over 5000
steps).  One benchmark step is one full time step of the method: the bulk
stream + collide + integrate update of all 8.4 M sites with the crack-face
rule and the crack step (K_III evaluation, criterion, advance, link cuts),
one fused kernel launch.

Timing: the lattice first runs --prelude steps (load ramp active), then
--warmup untimed steps; each of the --steps timed steps is bracketed by CUDA
events on the lattice's stream, with a 256 MiB buffer written and then read
between steps (outside the events) so that every step starts with a cold,
clean L2.  The step kernel is also timed by the library's own event hooks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference runs the plain FP64 CPU oracle on the same workload (the
reference arm: there is no other implementation of the method).  With N > 1
(torchrun) every rank runs its own independent replica (weak scaling, no data
exchange); the reference arm runs on rank 0 only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GLUPS and HBM GB/s vs GB300 roofline; batched and adjoint vs plain FP32 forward"
UNIT = "GLUPS"
BYTES_PER_SITE = 16            # FP32 moment form: read w, wdot; write w, wdot
WORKLOAD = "kcrit_single_4096x2048_f32"
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "step_kernel_f32_4096x2048.md")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2206_12412_gb300", "csrc", f)
                  for f in ("lbm_kernels.cu", "lbm_rows.cuh", "lbm_internal.cuh", "lbm_crack.cuh")]


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def reduce_max(pg, x: float, device="cpu") -> float:
    """Max of x over the ranks of the process group (x itself without one)."""
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def replica_value(world: int, units_per_rank: int, steps: int, seconds: float) -> float:
    """Whole-job throughput in G units per second: every rank advances its own
    replica (weak scaling), timed by the slowest rank."""
    return world * units_per_rank * steps / seconds / 1e9


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_sha256() -> str:
    """Hash of the files that define the step kernel (concatenated)."""
    h = hashlib.sha256()
    for path in KERNEL_SOURCES:
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def traffic_from_profile():
    """Per-launch DRAM bytes of the step kernel from the committed ncu summary,
    or None if there is none or the kernel source changed since it was taken."""
    try:
        text = open(PROFILE_SUMMARY).read()
        src = kernel_source_sha256()
    except OSError:
        return None
    m = re.search(r"kernel_source_sha256:\s*([0-9a-f]{64})", text)
    b = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m or not b or m.group(1) != src:
        return None
    return float(b.group(1))


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        loaded = [s for s in sm if s > 0.5 * (max(sm) if sm else 1)]
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons, "samples": len(rows)}


def cpu_baseline(problem, target_s=15.0):
    """The FP64 CPU oracle, as it stands, single-threaded on a bounded sample."""
    import oracle
    oracle.build()
    o = oracle.Oracle(problem)
    t = time.perf_counter()
    o.step(1)
    t1 = time.perf_counter() - t
    n = max(2, min(200, int(target_s / max(t1, 1e-6))))
    t = time.perf_counter()
    o.step(n)
    dt = time.perf_counter() - t
    sites = problem["nx"] * problem["ny"]
    o.close()
    return {"value": sites * n / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{problem['nx']}x{problem['ny']} lattice, {n} consecutive steps from the initial state, "
                      f"FP64 distribution form, one thread ({dt:.1f} s)"}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from paper_2206_12412_gb300 import workloads as W
    import oracle
    oracle.build()
    p = W.kcrit_single()
    o = oracle.Oracle(p)
    sites = p["nx"] * p["ny"]
    t = time.perf_counter()
    o.step(1)
    t1 = time.perf_counter() - t
    # a step is the whole lattice if the run fits in ~3 minutes, else a band of rows
    budget = 180.0
    frac = min(1.0, budget / max(t1 * (args.steps + args.warmup), 1e-9))
    if frac < 1.0:
        o.close()
        ny = max(16, int(p["ny"] * frac) // 2 * 2)
        q = dict(p)
        q["ny"] = ny
        q["crack"] = dict(p["crack"], y=float(ny // 2))
        p, o = q, oracle.Oracle(q)
        sites = p["nx"] * ny
    o.step(args.warmup)
    t = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t
    value = sites * args.steps / dt / 1e9
    sample = (f"{p['nx']}x{p['ny']} lattice per step" + ("" if frac >= 1.0 else " (row band of the 4096x2048 workload)")
              + ", FP64 distribution form, one thread")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "nx": 4096, "ny": 2048},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def measure_batched(lbm, W, torch, stream, steps, peak, count=256):
    """Batched form: 256 independent lattices of uneven sizes, one launch per
    step (graph replay), against the same lattices stepped one after another
    with the single-lattice path.  The 840 MB of state exceed L2."""
    problems = W.batch_problems(count, seed=3)
    sites = sum(p["nx"] * p["ny"] for p in problems)

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e-3

    lats = [lbm.Lattice(p, "f32", stream=stream) for p in problems]
    batch = lbm.Batch(lats)
    batch.step(128)
    t_b = timed(lambda: batch.step(steps))
    info = batch.info()
    batch.close()
    for l in lats:
        l.step(128)
    t_s = timed(lambda: [l.step(steps) for l in lats])
    for l in lats:
        l.close()
    return {"instances": len(problems), "sites": sites, "steps": steps, "ctas_per_step": info["ctas"],
            "glups_batched": sites * steps / t_b / 1e9, "glups_sequential": sites * steps / t_s / 1e9,
            "speedup": t_s / t_b, "achieved_gbs": 16 * sites * steps / t_b / 1e9,
            "frac": 16 * sites * steps / t_b / 1e9 / peak,
            "timing": "CUDA events around the whole run, no flush (state larger than L2)"}


def measure_adjoint(lbm, W, torch, stream, n_steps=None):
    """Sensor-misfit gradient on the 1024 x 1024, 8000-step problem (FP32,
    64 sensors): the plain forward run, the recording forward run and the
    transposed sweep, with stored misfits and with sqrt(T) checkpoints.  The
    16 MB state stays in L2 (the steps are timed back to back)."""
    import numpy as np
    a = W.adjoint_problem() if n_steps is None else W.adjoint_problem(n_steps=n_steps)
    p, T, sens = a["problem"], a["n_steps"], a["sensors"]
    ref = lbm.Lattice(W.with_series_load(p, "top", a["u_ref"]), "f32", stream=stream)
    tref = lbm.Tape(ref, sens, T)
    tref.forward(np.zeros((T, len(sens))))
    targets = torch.tensor(tref.misfits(), device="cuda")
    tref.close()
    ref.close()
    lat = lbm.Lattice(p, "f32", stream=stream)

    def timed(fn, reps=2):
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    def plain():
        lat.reset()
        lat.step(T)

    out = {"workload": f"sensor misfit {p['nx']}x{p['ny']} f32, {T} steps, {len(sens)} sensors, prescribed v=0.4",
           "forward_ms": timed(plain)}
    every_sqrt = int(round(np.sqrt(T)))
    for every, key in ((0, "stored"), (every_sqrt, "checkpointed")):
        tape = lbm.Tape(lat, sens, T, checkpoint_every=every)

        def rec():
            lat.reset()
            tape.forward(targets, loss_to_host=False)

        t_rec = timed(rec)
        rec()
        t_bwd = timed(lambda: tape.backward(device=True))
        out[key] = {"checkpoint_every": every, "recording_forward_ms": t_rec, "adjoint_ms": t_bwd,
                    "ratio_forward_plus_adjoint_over_forward": (t_rec + t_bwd) / out["forward_ms"]}
        tape.close()
    sites = p["nx"] * p["ny"]
    out["adjoint_us_per_step"] = out["stored"]["adjoint_ms"] * 1e3 / (T + 1)
    out["forward_us_per_step"] = out["forward_ms"] * 1e3 / T
    out["adjoint_l2_gbs"] = 16 * sites / (out["adjoint_us_per_step"] * 1e-6) / 1e9
    out["timing"] = "CUDA events around whole runs (graph replay), best of 2, no flush (L2-resident state)"
    lat.close()
    return out


def measure_large(lbm, W, torch, stream, peak):
    """The mixed-precision configuration: 16384 x 16384 (268 M sites, 4.3 GB
    of FP32 state, far larger than L2), crack on the midline from 0 to 2048
    growing at v = 0.5 c_s, +-1e-3 ramped over 2000 steps; the step kernel's
    own CUDA-event time for FP32 storage and for 16-bit wdot storage."""
    p = W.base_problem(16384, 16384, bc_mode="macroscopic")
    p = W.with_crack(p, mode="prescribed", y=8192.0, x_tip=2048.0, v_rel=0.5)
    p = W.with_antisymmetric_ramp(p, 1e-3, 2000.0)
    p["hist_cap"] = 4096
    sites = p["nx"] * p["ny"]
    out = {"workload": "16384x16384, prescribed v=0.5 crack from 0 to 2048", "timing": "library CUDA events around "
           "each step kernel, 20 steps after 20 (state far larger than L2)"}
    for storage, bps in (("f32", 16), ("f32_bf16", 12), ("f32_f16", 12)):
        lat = lbm.Lattice(p, storage, stream=stream)
        lat.step(20)
        lat.set_profiling(True)
        lat.step(20)
        lat.sync()
        pr = lat.profile(reset=True)
        k = pr["step_ms"] / max(pr["n_step"], 1) * 1e-3
        out[storage] = {"kernel_us": k * 1e6, "glups": sites / k / 1e9, "bytes_per_site": bps,
                        "achieved_gbs": bps * sites / k / 1e9, "frac": bps * sites / k / 1e9 / peak}
        lat.close()
        torch.cuda.empty_cache()
    return out


def step_time(lbm, p, storage, stream, flush_l2, prelude, steps):
    """Mean time of one lbm_step(1) (library CUDA events around its launches)
    with the L2 flushed before each step."""
    lat = lbm.Lattice(p, storage, stream=stream)
    lat.step(prelude)
    lat.set_profiling(True)
    for _ in range(steps):
        flush_l2()
        lat.step(1)
    lat.sync()
    pr = lat.profile(reset=True)
    lat.close()
    return pr["step_ms"] / max(pr["n_step"], 1) * 1e-3


def crack_share(lbm, W, torch, stream, problem, flush_l2, t_crack, steps=100):
    """The cost of the crack handling, the GPU analogue of the CPU-time share
    the paper reports (Sec. 5.3): the benchmark lattice's step time with its
    K-criterion crack against the same lattice, loads and state size with no
    crack, and the same for the Sec. 5.2 example (whole 5050-step runs)."""
    q = dict(problem, crack={"mode": "none"})
    t_none = step_time(lbm, q, "f32", stream, flush_l2, 2500, steps)
    out = {"kcrit_single": {"step_us_crack": t_crack * 1e6, "step_us_no_crack": t_none * 1e6,
                            "share": 1.0 - t_none / t_crack}}
    times = {}
    for label, p in (("crack", W.kcrit_centre_crack()), ("none", dict(W.kcrit_centre_crack(), crack={"mode": "none"}))):
        lat = lbm.Lattice(p, "f32", stream=stream)
        lat.step(64)
        lat.reset()
        lat.sync()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        lat.step(W.KCRIT_CENTRE_STEPS)
        ev1.record(stream)
        torch.cuda.synchronize()
        times[label] = ev0.elapsed_time(ev1) * 1e-3 / W.KCRIT_CENTRE_STEPS
        lat.close()
    out["centre_crack_sec52"] = {"step_us_crack": times["crack"] * 1e6, "step_us_no_crack": times["none"] * 1e6,
                                 "share": 1.0 - times["none"] / times["crack"]}
    out["paper"] = "CPU-time share of the crack step in the authors' Python code: 2.8 % (steady growth), 0.7 % (Sec. 5.2)"
    return out


def measure_extensions(lbm, W, torch, stream, problem, peak, flush_l2, steps=100):
    """The two extensions beyond the plain method.  D2Q9: the benchmark
    workload on the nine-velocity lattice (bounce-back crack faces, FP32), the
    update and crack launches timed by the library's CUDA events with the L2
    flushed before each step, against 16 algorithmic bytes per site.  The
    K-criterion centre-crack example of Sec. 5.2 (512 x 192, macroscopic rule
    on every boundary, FP32): the whole 5050-step run timed with CUDA events
    (graph replay; the state fits in L2, so it is launch-bound)."""
    sites = problem["nx"] * problem["ny"]
    q = dict(problem, bc_mode="bounceback", lattice="D2Q9")
    lat = lbm.Lattice(q, "f32", stream=stream)
    lat.step(500)
    lat.set_profiling(True)
    for _ in range(steps):
        flush_l2()
        lat.step(1)
    lat.sync()
    pr = lat.profile(reset=True)
    k = pr["step_ms"] / max(pr["n_step"], 1) * 1e-3
    d2q9 = {"workload": "kcrit_single 4096x2048, D2Q9, bounce-back faces, f32", "step_us": k * 1e6,
            "glups": sites / k / 1e9, "bytes_per_site": 16, "achieved_gbs": 16 * sites / k / 1e9,
            "frac": 16 * sites / k / 1e9 / peak, "launches_per_step": 1,
            "timing": "library CUDA events around each step's launch, L2 flushed before each step"}
    lat.close()

    # a straight crack in another direction (Sec. 4.1): the same lattice and
    # loads, a K-criterion edge crack at 20 degrees, link-local faces
    import numpy as np
    ql = W.kcrit_line()
    lat = lbm.Lattice(ql, "f32", stream=stream)
    lat.step(2500)
    x0, y0 = lat.tip_q()
    lat.set_profiling(True)
    for _ in range(steps):
        flush_l2()
        lat.step(1)
    lat.sync()
    pr = lat.profile(reset=True)
    k = pr["step_ms"] / max(pr["n_step"], 1) * 1e-3
    x1, y1 = lat.tip_q()
    line = {"workload": "kcrit_line 4096x2048, crack at 20 degrees, bounce-back faces, f32", "step_us": k * 1e6,
            "glups": sites / k / 1e9, "bytes_per_site": 16, "achieved_gbs": 16 * sites / k / 1e9,
            "frac": 16 * sites / k / 1e9 / peak, "launches_per_step": 1, "kernel": "line_step_kernel<float>",
            "tip_advance_dh": float(np.hypot(x1 - x0, y1 - y0)) / 2**32,
            "timing": "library CUDA events around each step's launch, L2 flushed before each step"}
    lat.close()

    # a centre crack at 20 degrees with the macroscopic rule on its faces
    # (line_step_kernel, then line_faces_kernel's fixpoint solve); a failure
    # is reported in its entry rather than ending the other measurements
    try:
        qm = W.kcrit_line_centre()
        lat = lbm.Lattice(qm, "f32", stream=stream)
        lat.step(2500)
        lat.set_profiling(True)
        for _ in range(steps):
            flush_l2()
            lat.step(1)
        lat.sync()
        pr = lat.profile(reset=True)
        km = pr["step_ms"] / max(pr["n_step"], 1) * 1e-3
        line_macro = {"workload": "kcrit_line_centre 4096x2048, centre crack at 20 degrees, macroscopic faces, f32",
                      "step_us": km * 1e6, "glups": sites / km / 1e9, "launches_per_step": 2,
                      "kernels": "line_step_kernel<float>, line_faces_kernel<float>",
                      "timing": "library CUDA events around each step's launches, L2 flushed before each step"}
        lat.close()
    except lbm.LbmError as e:
        line_macro = {"error": str(e)[:300]}

    p = W.kcrit_centre_crack()
    n = W.KCRIT_CENTRE_STEPS
    lat = lbm.Lattice(p, "f32", stream=stream)
    lat.step(64)          # capture the step graph
    lat.reset()
    lat.sync()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    lat.step(n)
    ev1.record(stream)
    torch.cuda.synchronize()
    secs = ev0.elapsed_time(ev1) * 1e-3
    hist = lat.history(cap=n)
    centre = {"workload": "Sec. 5.2 centre crack 512x192, macroscopic rule on every boundary, f32, 5050 steps",
              "run_ms": secs * 1e3, "us_per_step": secs / n * 1e6, "glups": p["nx"] * p["ny"] * n / secs / 1e9,
              "launches_per_step": 2, "tip_right_final": float(hist["tip_q"][-1]) / 2**32,
              "timing": "CUDA events around the whole run (graph replay, L2-resident state)"}
    lat.close()

    # a sweep of the same example over K_C (0.8 .. 1.2 K_C, 64 runs) as one batch
    runs, steps_b = 64, 1024
    lats = []
    for q in range(runs):
        pq = W.kcrit_centre_crack()
        pq["crack"] = dict(pq["crack"], K_C=pq["crack"]["K_C"] * (0.8 + 0.4 * q / (runs - 1)))
        pq["hist_cap"] = steps_b
        lats.append(lbm.Lattice(pq, "f32", stream=stream))
    b = lbm.Batch(lats)
    b.step(64)
    torch.cuda.synchronize()
    ev0.record(stream)
    b.step(steps_b)
    ev1.record(stream)
    torch.cuda.synchronize()
    secs_b = ev0.elapsed_time(ev1) * 1e-3
    sweep = {"workload": f"{runs} runs of the Sec. 5.2 example (K_C from 0.8 to 1.2 of the paper's), one batch, f32",
             "steps": steps_b, "us_per_step": secs_b / steps_b * 1e6,
             "glups": runs * p["nx"] * p["ny"] * steps_b / secs_b / 1e9,
             "timing": "CUDA events around the batched steps (graph replay)"}
    b.close()
    for l in lats:
        l.close()
    return {"d2q9": d2q9, "line_crack": line, "line_crack_macroscopic": line_macro, "centre_crack_sec52": centre,
            "centre_crack_sweep": sweep}


def measure_virtual_ranks(lbm, W, torch, stream, problem, steps=256):
    """The benchmark lattice split into 1, 2, 4 and 8 row slabs on this GPU
    (one batched step launch plus one halo-row exchange launch per step),
    timed back to back (graph replay, no flush) against the undivided
    lattice's graph replay."""
    sites = problem["nx"] * problem["ny"]
    out = {"timing": "CUDA events around graph replay of the steps, no flush", "steps": steps, "glups": {}}
    for n in (1, 2, 4, 8):
        d = lbm.Decomp(problem, n, "f32", stream=stream)
        d.step(64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        d.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        out["glups"][str(n)] = sites * steps / (e0.elapsed_time(e1) * 1e-3) / 1e9
        d.close()
    return out


def run_ours(args, rank, world, local):
    import numpy as np
    import torch
    from paper_2206_12412_gb300 import lbm
    from paper_2206_12412_gb300 import workloads as W

    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist

    def barrier():
        if pg is not None:
            pg.barrier()

    def allmax(x: float) -> float:
        return reduce_max(pg, x, "cuda")

    problem = W.kcrit_single()
    if args.profile_only and args.lattice == "D2Q9":
        # the D2Q9 form of the workload (bounce-back crack faces), for its profile
        problem = dict(problem, bc_mode="bounceback", lattice="D2Q9")
    if args.profile_only and args.crack == "line":
        # the workload with its crack at 20 degrees (line_step_kernel), for its profile
        problem = W.kcrit_line()
    if args.profile_only and args.crack == "line_macro":
        # a centre crack at 20 degrees with the macroscopic rule on its faces
        # (line_step_kernel, then line_faces_kernel), for its profile
        problem = W.kcrit_line_centre()
    sites = problem["nx"] * problem["ny"]
    stream = torch.cuda.current_stream()
    lat = lbm.Lattice(problem, "f32", stream=stream)
    lat.step(args.prelude)
    lat.sync()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    flush_sum = torch.empty((), dtype=torch.int64, device="cuda")

    def flush_l2():
        # write a buffer twice the size of L2, then read it back: L2 ends up
        # holding clean lines of the flush buffer, none of the lattice state
        flush.fill_(1)
        flush_sum.copy_(flush.view(torch.int64).sum())

    if args.profile_only:
        lat.set_profiling(True)
        for _ in range(args.warmup + args.steps):
            flush_l2()
            lat.step(1)
        lat.sync()
        prof = lat.profile(reset=True)
        if rank == 0:
            print(json.dumps({"profile_only": True, "steps": args.warmup + args.steps, **prof}), flush=True)
        lat.close()
        return 0

    # timed region: one step per pair of events, L2 flushed in between (outside the events)
    for _ in range(args.warmup):
        flush_l2()
        lat.step(1)
    lat.sync()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush_l2()
        starts[k].record(stream)
        lat.step(1)
        ends[k].record(stream)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    step_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    total_s = allmax(step_ms * 1e-3)
    value = replica_value(world, sites, args.steps, total_s)

    # the step kernel alone, timed by the library's events on the same stream
    lat.set_profiling(True)
    for _ in range(args.steps):
        flush_l2()
        lat.step(1)
    lat.sync()
    prof = lat.profile(reset=True)
    lat.set_profiling(False)
    kern_s = prof["step_ms"] / max(prof["n_step"], 1) * 1e-3
    achieved = BYTES_PER_SITE * sites / kern_s / 1e9
    peak, peak_kind = measured_peaks()
    traffic = traffic_from_profile()

    # the same workload with wdot stored in 16 bits (12 bytes per site update)
    mixed = {}
    for storage in ("f32_bf16", "f32_f16"):
        lm = lbm.Lattice(problem, storage, stream=stream)
        lm.step(args.prelude)
        lm.set_profiling(True)
        for _ in range(min(args.steps, 100)):
            flush_l2()
            lm.step(1)
        lm.sync()
        pr = lm.profile(reset=True)
        km = pr["step_ms"] / max(pr["n_step"], 1) * 1e-3
        mixed[storage] = {"glups": sites / km / 1e9, "kernel_ms": km * 1e3, "bytes_per_site": 12,
                          "achieved_gbs": 12 * sites / km / 1e9, "frac": 12 * sites / km / 1e9 / peak}
        lm.close()

    batched = measure_batched(lbm, W, torch, stream, 128, peak) if not args.no_batched else None
    adjoint = measure_adjoint(lbm, W, torch, stream) if not args.no_adjoint else None
    vranks = measure_virtual_ranks(lbm, W, torch, stream, problem) if not args.no_virtual_ranks else None
    large = measure_large(lbm, W, torch, stream, peak) if not args.no_large else None
    ext = measure_extensions(lbm, W, torch, stream, problem, peak, flush_l2) if not args.no_extensions else None
    if ext is not None:
        ext["crack_share"] = crack_share(lbm, W, torch, stream, problem, flush_l2, kern_s)

    # steady back-to-back replay (CUDA graph, no flush): context only
    lat.sync()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    lat.step(256)
    ev1.record(stream)
    torch.cuda.synchronize()
    steady = sites * 256 / (ev0.elapsed_time(ev1) * 1e-3) / 1e9

    # end to end through the public API with host buffers: upload the state from
    # pinned memory, run the steps, read back the fields and the per-step crack record
    w_h = torch.empty((problem["ny"], problem["nx"]), dtype=torch.float32, pin_memory=True)
    wd_h = torch.empty_like(w_h, pin_memory=True)
    w_np, wd_np = w_h.numpy(), wd_h.numpy()
    w0, wd0 = lat.fields()
    w_np[...] = w0
    wd_np[...] = wd0
    e2e_vals = []
    for _ in range(2):
        barrier()
        torch.cuda.synchronize()
        t = time.perf_counter()
        lbm.lbm_set_fields(lat.h, 0, w_np.ctypes.data, False, lat.dtype_code)
        lbm.lbm_set_fields(lat.h, 1, wd_np.ctypes.data, False, lat.dtype_code)
        lat.step(args.steps)
        lbm.lbm_fields(lat.h, 0, w_np.ctypes.data, False, lat.dtype_code)
        lbm.lbm_fields(lat.h, 1, wd_np.ctypes.data, False, lat.dtype_code)
        hist = lat.history(cap=args.steps)
        e2e_vals.append(time.perf_counter() - t)
    e2e_s = allmax(min(e2e_vals))
    plane = sites * 4
    h2d = 2 * plane / args.steps
    d2h = (2 * plane + len(hist["K"]) * (8 + 8 + 8 + 4)) / args.steps

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": problem["nx"], "ny": problem["ny"], "storage": "f32",
                   "crack": "kcrit", "bc_mode": problem["bc_mode"], "prelude_steps": args.prelude,
                   "l2": "flushed between timed steps (256 MiB buffer written then read, outside the events)",
                   "parallelism": f"{world} independent replicas" if world > 1 else "single GPU",
                   "launch": lat.launch()},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": "step_kernel<float>", "kernel_ms": kern_s * 1e3, "bytes_per_site": BYTES_PER_SITE},
        "e2e": {"value": world * sites * args.steps / e2e_s / 1e9, "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps,
        "steady_graph_glups": steady,
        "mixed_precision": mixed,
        "batched": batched,
        "adjoint": adjoint,
        "virtual_ranks": vranks,
        "large_lattice": large,
        "extensions": ext,
        "wall_s": wall,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(problem)
    if rank == 0:
        print(json.dumps(line), flush=True)
    lat.close()
    if pg is not None:
        pg.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prelude", type=int, default=2500)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 256-lattice batched measurement")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the sensor-misfit gradient measurement")
    ap.add_argument("--no-virtual-ranks", action="store_true", help="skip the row-slab decomposition measurement")
    ap.add_argument("--no-large", action="store_true", help="skip the 16384 x 16384 storage comparison")
    ap.add_argument("--no-extensions", action="store_true", help="skip the D2Q9 and Sec. 5.2 example measurements")
    ap.add_argument("--batched-only", action="store_true",
                    help="only the batched measurement, --steps steps of --batched-count lattices (for ncu)")
    ap.add_argument("--batched-count", type=int, default=256, help="lattices in the batched measurement")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="only the sensor-misfit gradient measurement (for ncu)")
    ap.add_argument("--adjoint-steps", type=int, default=None, help="steps of the adjoint workload (default 8000)")
    ap.add_argument("--lattice", default="D2Q5", choices=["D2Q5", "D2Q9"],
                    help="with --profile-only: the velocity set of the profiled workload")
    ap.add_argument("--crack", default="x", choices=["x", "line", "line_macro"],
                    help="with --profile-only: the crack of the profiled workload (along +x, or at 20 degrees; "
                         "line_macro: a centre crack at 20 degrees with the macroscopic rule on its faces)")
    ap.add_argument("--profile-only", action="store_true",
                    help="only prelude, warm-up and timed steps (for ncu); prints kernel times")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.batched_only:
        # the batched form alone (for profiling the batch kernel)
        import torch
        from paper_2206_12412_gb300 import lbm
        from paper_2206_12412_gb300 import workloads as W
        torch.cuda.set_device(local)
        peak, _ = measured_peaks()
        out = measure_batched(lbm, W, torch, torch.cuda.current_stream(), args.steps, peak, count=args.batched_count)
        if rank == 0:
            print(json.dumps({"batched_only": True, **out}), flush=True)
        return 0
    if args.adjoint_only:
        # the sensor-misfit gradient alone (for profiling the adjoint kernel)
        import torch
        from paper_2206_12412_gb300 import lbm
        from paper_2206_12412_gb300 import workloads as W
        torch.cuda.set_device(local)
        out = measure_adjoint(lbm, W, torch, torch.cuda.current_stream(), n_steps=args.adjoint_steps)
        if rank == 0:
            print(json.dumps({"adjoint_only": True, **out}), flush=True)
        return 0
    return run_ours(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
