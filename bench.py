#!/usr/bin/env python
"""Throughput of the fused lattice Boltzmann time step with dynamic mode III
crack propagation (arXiv 2206.12412) on GB300.

Headline workload: the 16384 x 16384 FP32 lattice (268 M sites, 2.1 GB of
state, far larger than the 129 MB L2) with an edge crack on the midline
from 0 to 2048 growing at the prescribed v = 0.5 c_s, top/bottom ramped to
+-1e-3 over 2000 steps, its state stored as the two FP32 planes w_n and
w_{n-1} (leapfrog storage: 12 bytes per site update; the FP32 moment form,
w and wdot, 16 bytes, is measured beside it).  One benchmark step is one
full time step of the method: the bulk stream + collide + integrate update
of every site with the macroscopic crack-face rule and the crack step
(K_III evaluation, criterion, advance, link cuts), one fused kernel launch.

Timing: the lattice first runs --prelude steps, then --warmup untimed
steps; each of the --steps timed steps is bracketed by CUDA events on the
lattice's stream.  The state is 16x the L2, so no flush is needed between
steps.  The step kernel is also timed by the library's own event hooks
(the roofline figure).  The rest of the JSON line: the former 4096 x 2048
K-criterion headline (L2 flushed between steps), the 128 x 128 FP64
configuration as graph replay, the 16-bit storage forms, the extensions
(D2Q9, cracks in other directions, the Sec. 5.2 example), and last the
three patterns (mixed precision, row slabs, adjoint, batches).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference runs the FP64 CPU oracle on a bounded sample of the same
workload on all host cores (the reference arm: there is no other
implementation of the method).  With N > 1 (torchrun) every rank runs its
own independent replica (weak scaling, no data exchange); the reference arm
runs on rank 0 only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
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
HEADLINE_STORAGE = "f32_lf"    # FP32 leapfrog storage: the state as w_n, w_{n-1}
BYTES_PER_SITE = 12            # read w_n and w_{n-1}, write w_{n+1} (FP32)
WORKLOAD = "prescribed_v05_16384x16384_f32"
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "step_kernel_leapfrog_f32_8192x8192.md")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2206_12412_gb300", "csrc", f)
                  for f in ("lbm_kernels.cu", "lbm_rows.cuh", "lbm_internal.cuh", "lbm_crack.cuh")]


def r4(x):
    """A float rounded to 4 significant digits (keeps the JSON line short)."""
    if x is None:
        return None
    return float(f"{float(x):.4g}")


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


def traffic_from_profile(sites: int):
    """DRAM bytes of one step-kernel launch on `sites` sites, scaled from the
    committed ncu summary of the 8192 x 8192 lattice (1 GB of state, so the
    writes cannot stay in L2) by the sites per launch; None if there is no
    summary or the kernel source changed since it was taken."""
    try:
        text = open(PROFILE_SUMMARY).read()
        src = kernel_source_sha256()
    except OSError:
        return None
    m = re.search(r"kernel_source_sha256:\s*([0-9a-f]{64})", text)
    b = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    n = re.search(r"sites_per_launch:\s*([0-9]+)", text)
    if not m or not b or not n or m.group(1) != src:
        return None
    return float(b.group(1)) * sites / float(n.group(1))


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


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


# ------------------------------------------------------------ CPU oracle

def oracle_band(rows: int = 64) -> dict:
    """A band of rows of the headline workload for the CPU oracle: the full
    16384-wide lattice, `rows` rows high, the crack on its midline from 0 to
    2048 at v = 0.5, the same loads."""
    from paper_2206_12412_gb300 import workloads as W
    p = W.large_prescribed()
    return dict(p, ny=rows, crack=dict(p["crack"], y=float(rows // 2)))


def oracle_mlups(problem: dict, threads: int, target_s: float, max_steps: int = 100000):
    """MLUPS of the FP64 oracle, as it stands, on `threads` host threads: one
    step to size the sample, then consecutive steps for about target_s."""
    import oracle
    o = oracle.Oracle(problem, threads=threads)
    t = time.perf_counter()
    o.step(1)
    t1 = time.perf_counter() - t
    n = max(2, min(max_steps, int(target_s / max(t1, 1e-6))))
    t = time.perf_counter()
    o.step(n)
    dt = time.perf_counter() - t
    used = o.threads
    o.close()
    return problem["nx"] * problem["ny"] * n / dt / 1e6, n, dt, used


def cpu_baseline():
    """The FP64 CPU oracle timed on this host: the headline workload's row
    band on all cores (the reported value) and on one thread, and the small
    configurations (128 x 128, and the 512 x 256 downscale of the 4096 x 2048
    K-criterion run) on one thread and all cores.  About 15-25 s in all."""
    import oracle
    from paper_2206_12412_gb300 import workloads as W
    oracle.build()
    ncore = host_cores()
    band = oracle_band()
    m_all, n_all, t_all, used = oracle_mlups(band, ncore, 6.0)
    m_one, n_one, t_one, _ = oracle_mlups(band, 1, 4.0)
    small = {}
    for name, p in (("c1_128x128", W.plain_fp64("macroscopic")), ("c2_downscale_512x256", W.kcrit_single(scale=8))):
        a, _, _, _ = oracle_mlups(p, 1, 1.5)
        b, _, _, _ = oracle_mlups(p, ncore, 1.5)
        small[name] = {"mlups_1": r4(a), f"mlups_{ncore}": r4(b)}
    return {"value": r4(m_all / 1e3), "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"{band['nx']}x{band['ny']} row band of the workload, {n_all} steps on {used} threads "
                      f"({t_all:.1f} s), FP64 distribution form",
            "single_thread": r4(m_one / 1e3), "cpu_model": cpu_model(), "nproc": ncore, "small_mlups": small}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    ncore = host_cores()
    p = oracle_band()
    o = oracle.Oracle(p, threads=ncore)
    sites = p["nx"] * p["ny"]
    o.step(args.warmup)
    t = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t
    used = o.threads
    o.close()
    value = sites * args.steps / dt / 1e9
    sample = (f"{p['nx']}x{p['ny']} row band of the 16384x16384 workload per step, FP64 distribution form, "
              f"{used} threads ({cpu_model()})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "nx": 16384, "ny": 16384},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- GPU parts

def events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def timed(torch, stream, fn):
    """Seconds of fn's GPU work, CUDA events on `stream`."""
    e0, e1 = events(torch)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) * 1e-3


def kernel_seconds(lat):
    """Mean step-kernel time from the library's profiling events."""
    lat.sync()
    pr = lat.profile(reset=True)
    return pr["step_ms"] / max(pr["n_step"], 1) * 1e-3


def profile_batched(lbm, W, torch, stream, steps, shape, count=256):
    """Only the batched steps of the 256-lattice workload at a given launch
    shape (for ncu captures of the batch kernel)."""
    problems = W.batch_problems(count, seed=3)
    lats = [lbm.Lattice(p, "f32", stream=stream) for p in problems]
    batch = lbm.Batch(lats)
    batch.set_shape(*shape[:2])
    if len(shape) > 2:
        batch.set_lookahead(shape[2])
    secs = timed(torch, stream, lambda: batch.step(steps))
    sites = sum(p["nx"] * p["ny"] for p in problems)
    batch.close()
    for l in lats:
        l.close()
    return {"shape": list(shape), "steps": steps, "glups": r4(sites * steps / secs / 1e9)}


def measure_batched(lbm, W, torch, stream, steps, peak, count=256, full_steps=None):
    """Batched form: 256 independent lattices of uneven sizes, one launch per
    step (graph replay), against the same lattices stepped one after another
    with the single-lattice path.  The 840 MB of state exceed L2.  With
    full_steps, the tuned batch then runs the configuration's whole length
    (20 000 steps) as one timed run."""
    problems = W.batch_problems(count, seed=3)
    sites = sum(p["nx"] * p["ny"] for p in problems)
    lats = [lbm.Lattice(p, "f32", stream=stream) for p in problems]
    batch = lbm.Batch(lats)
    batch.step(128)
    t_d = timed(torch, stream, lambda: batch.step(steps))      # the default shape: 128 threads, 16-row bands
    batch.tune(trial_steps=8)
    batch.step(64)
    t_b = timed(torch, stream, lambda: batch.step(steps))
    info = batch.info()
    # the tuned shape with the other row lookahead of the march
    la = info["lookahead"]
    batch.set_lookahead(3 - la)
    batch.step(16)
    t_o = timed(torch, stream, lambda: batch.step(steps))
    batch.set_lookahead(la)
    lookahead_ab = {str(la): r4(sites * steps / t_b / 1e9), str(3 - la): r4(sites * steps / t_o / 1e9)}
    full = None
    if full_steps:
        for l in lats:
            l.reset()
        t_f = timed(torch, stream, lambda: batch.step(full_steps))
        full = {"steps": full_steps, "s": r4(t_f), "glups": r4(sites * full_steps / t_f / 1e9)}
    # the same shape as one persistent cooperative launch (grid barrier between steps)
    batch.set_persistent(True)
    batch.step(8)
    t_p = timed(torch, stream, lambda: batch.step(steps))
    batch.close()
    for l in lats:
        l.step(128)
    t_s = timed(torch, stream, lambda: [l.step(steps) for l in lats])
    for l in lats:
        l.close()
    # the same batch in leapfrog storage (12 bytes per site update)
    lf = [lbm.Lattice(p, "f32_lf", stream=stream) for p in problems]
    blf = lbm.Batch(lf)
    blf.tune(trial_steps=8)
    blf.step(64)
    t_lf = timed(torch, stream, lambda: blf.step(steps))
    lf_shape = blf.info()
    blf.close()
    for l in lf:
        l.close()
    return {"n": len(problems), "sites": sites, "steps": steps, "ctas": info["ctas"],
            "shape": [info["threads"], info["band_rows"], info["lookahead"]],
            "glups_default_shape": r4(sites * steps / t_d / 1e9), "glups_by_lookahead": lookahead_ab,
            "glups_persistent": r4(sites * steps / t_p / 1e9),
            "glups_sequential": r4(sites * steps / t_s / 1e9), "speedup": r4(t_s / t_b),
            "glups": r4(sites * steps / t_b / 1e9), "frac": r4(16 * sites * steps / t_b / 1e9 / peak),
            "full_run": full,
            "leapfrog": {"glups": r4(sites * steps / t_lf / 1e9), "frac": r4(12 * sites * steps / t_lf / 1e9 / peak),
                         "shape": [lf_shape["threads"], lf_shape["band_rows"], lf_shape["lookahead"]]}}


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

    def best(fn, reps=2):
        return min(timed(torch, stream, fn) for _ in range(reps)) * 1e3

    def plain():
        lat.reset()
        lat.step(T)

    fwd = best(plain)
    out = {"T": T, "fwd_ms": r4(fwd), "fwd_us_step": r4(fwd * 1e3 / T)}
    every_sqrt = int(round(np.sqrt(T)))
    for every, key in ((0, "stored"), (every_sqrt, "ckpt")):
        tape = lbm.Tape(lat, sens, T, checkpoint_every=every)

        def rec():
            lat.reset()
            tape.forward(targets, loss_to_host=False)

        t_rec = best(rec)
        rec()
        t_bwd = best(lambda: tape.backward(device=True))
        out[key] = {"rec_ms": r4(t_rec), "adj_ms": r4(t_bwd), "ratio": r4((t_rec + t_bwd) / fwd)}
        tape.close()
    lat.close()
    return out


def measure_storage_large(lbm, W, torch, stream, peak, n=16384):
    """The other storage forms on the headline lattice (the FP32 moment form,
    FP32 w with 16-bit wdot): the step kernel's own CUDA-event time, 20 steps
    after 20."""
    p = W.large_prescribed(n)
    sites = p["nx"] * p["ny"]
    out = {}
    for storage, bps in (("f32", 16), ("f32_bf16", 12), ("f32_f16", 12)):
        lat = lbm.Lattice(p, storage, stream=stream)
        lat.step(20)
        lat.set_profiling(True)
        lat.step(20)
        k = kernel_seconds(lat)
        out[storage] = {"us": r4(k * 1e6), "glups": r4(sites / k / 1e9), "frac": r4(bps * sites / k / 1e9 / peak)}
        lat.close()
        torch.cuda.empty_cache()
    return out


def step_time(lbm, p, storage, stream, flush_l2, prelude, steps, lattice=None):
    """Mean step-kernel time of lbm_step(1) (library CUDA events) with the
    L2 flushed before each step."""
    lat = lbm.Lattice(p, storage, stream=stream)
    lat.step(prelude)
    lat.set_profiling(True)
    for _ in range(steps):
        flush_l2()
        lat.step(1)
    k = kernel_seconds(lat)
    lat.close()
    return k


def measure_kcrit4096(lbm, W, torch, stream, peak, flush_l2, steps):
    """The 4096 x 2048 K-criterion run (8.4 M sites, 134 MB of state, about
    the size of L2): the step kernel's CUDA-event time with the L2 flushed
    (written then read back, outside the events) before every step."""
    p = W.kcrit_single()
    k = step_time(lbm, p, "f32", stream, flush_l2, 2500, steps)
    sites = p["nx"] * p["ny"]
    return {"us": r4(k * 1e6), "glups": r4(sites / k / 1e9), "frac": r4(16 * sites / k / 1e9 / peak)}, k


def measure_c1(lbm, W, torch, stream):
    """The 128 x 128 FP64 configuration (stationary crack, 2000 steps) as
    graph replay: 16 K sites, launch- and latency-bound, so microseconds per
    step rather than a roofline fraction."""
    p = W.plain_fp64("macroscopic")
    lat = lbm.Lattice(p, "f64", stream=stream)
    lat.step(W.PLAIN_FP64_STEPS)     # captures the step graphs
    lat.reset()
    secs = timed(torch, stream, lambda: lat.step(W.PLAIN_FP64_STEPS))
    lat.close()
    return {"us_step": r4(secs / W.PLAIN_FP64_STEPS * 1e6), "steps": W.PLAIN_FP64_STEPS}


def crack_share(lbm, W, torch, stream, flush_l2, t_crack):
    """The cost of the crack handling, the GPU analogue of the CPU-time share
    the paper reports (Sec. 5.3): the step time with the crack against the
    same lattice, loads and state size with no crack -- on the 4096 x 2048
    K-criterion run and on the whole 5050-step Sec. 5.2 example."""
    p = W.kcrit_single()
    t_none = step_time(lbm, dict(p, crack={"mode": "none"}), "f32", stream, flush_l2, 2500, 100)
    times = {}
    for label, q in (("crack", W.kcrit_centre_crack()), ("none", dict(W.kcrit_centre_crack(), crack={"mode": "none"}))):
        lat = lbm.Lattice(q, "f32", stream=stream)
        lat.step(64)
        lat.reset()
        times[label] = timed(torch, stream, lambda: lat.step(W.KCRIT_CENTRE_STEPS)) / W.KCRIT_CENTRE_STEPS
        lat.close()
    return {"kcrit_4096": r4(1.0 - t_none / t_crack),
            "sec52": r4(1.0 - times["none"] / times["crack"]),
            "sec52_us": [r4(times["crack"] * 1e6), r4(times["none"] * 1e6)],
            "paper_cpu_share": [0.028, 0.007]}


def line_sweep(lbm, W, torch, stream, count=32, steps_l=256):
    """A batch of lattices of 512 x 256, each with an edge crack in another
    direction (0 to 87 degrees, prescribed v = 0.5, link-local faces), against
    the same lattices stepped one after another."""
    import numpy as np
    lines = []
    for q in range(count):
        th = np.radians(2.8 * q)
        pq = W.with_line_crack(W.with_antisymmetric_ramp(W.base_problem(512, 256, bc_mode="bounceback"), 1e-3, 200.0),
                               mode="prescribed",
                               start=(0.0, 128.37), tip=(40.0 * np.cos(th) + 0.013, 128.37 + 40.0 * np.sin(th)),
                               v_rel=0.5, r0=2.0)
        pq["hist_cap"] = 2 * steps_l
        lines.append(lbm.Lattice(pq, "f32", stream=stream))
    for l in lines:
        l.step(8)
    t_seq = timed(torch, stream, lambda: [l.step(steps_l) for l in lines])
    b = lbm.Batch(lines)
    b.step(8)
    t_b = timed(torch, stream, lambda: b.step(steps_l))
    b.close()
    for l in lines:
        l.close()
    return {"us_step": r4(t_b / steps_l * 1e6), "glups": r4(count * 512 * 256 * steps_l / t_b / 1e9),
            "speedup": r4(t_seq / t_b)}


def measure_extensions(lbm, W, torch, stream, peak, flush_l2, steps=100):
    """The extensions beyond the plain method, on the 4096 x 2048 lattice with
    the L2 flushed before each step (library CUDA events): D2Q9 with
    bounce-back crack faces; an edge crack at 20 degrees with link-local
    faces; a centre crack at 20 degrees with the macroscopic rule on its
    faces (two launches per step).  Then the Sec. 5.2 example (512 x 192,
    macroscopic rule on every boundary, 5050 steps, graph replay) and a sweep
    of 64 such runs over K_C as one batch."""
    import numpy as np
    base = W.kcrit_single()
    sites = base["nx"] * base["ny"]
    out = {}
    k = step_time(lbm, dict(base, bc_mode="bounceback", lattice="D2Q9"), "f32", stream, flush_l2, 500, steps)
    out["d2q9"] = {"us": r4(k * 1e6), "glups": r4(sites / k / 1e9), "frac": r4(16 * sites / k / 1e9 / peak)}
    k = step_time(lbm, W.kcrit_line(), "f32", stream, flush_l2, 2500, steps)
    out["line"] = {"us": r4(k * 1e6), "glups": r4(sites / k / 1e9), "frac": r4(16 * sites / k / 1e9 / peak)}
    try:
        km = step_time(lbm, W.kcrit_line_centre(), "f32", stream, flush_l2, 2500, steps)
        out["line_macro"] = {"us": r4(km * 1e6), "glups": r4(sites / km / 1e9)}
    except lbm.LbmError as e:
        out["line_macro"] = {"error": str(e)[:200]}

    p = W.kcrit_centre_crack()
    n = W.KCRIT_CENTRE_STEPS
    lat = lbm.Lattice(p, "f32", stream=stream)
    lat.step(64)          # capture the step graph
    lat.reset()
    secs = timed(torch, stream, lambda: lat.step(n))
    hist = lat.history(cap=n)
    out["sec52"] = {"us_step": r4(secs / n * 1e6), "glups": r4(p["nx"] * p["ny"] * n / secs / 1e9),
                    "tip_final": r4(float(hist["tip_q"][-1]) / 2**32)}
    lat.close()

    # 64 runs of the example over K_C as one batch, on D2Q5 and on D2Q9 (the
    # D2Q9 run alone first, for the speedup)
    runs, steps_b = 64, 1024
    for lattice, key in (("D2Q5", "sec52_sweep64"), ("D2Q9", "sec52_sweep64_d2q9")):
        if lattice == "D2Q9":
            lat = lbm.Lattice(dict(p, lattice="D2Q9"), "f32", stream=stream)
            lat.step(64)
            lat.reset()
            secs = timed(torch, stream, lambda: lat.step(steps_b))
            out["sec52_d2q9_us_step"] = r4(secs / steps_b * 1e6)
            lat.close()
        lats = []
        for q in range(runs):
            pq = dict(W.kcrit_centre_crack(), lattice=lattice)
            pq["crack"] = dict(pq["crack"], K_C=pq["crack"]["K_C"] * (0.8 + 0.4 * q / (runs - 1)))
            pq["hist_cap"] = steps_b
            lats.append(lbm.Lattice(pq, "f32", stream=stream))
        b = lbm.Batch(lats)
        b.step(64)
        secs_b = timed(torch, stream, lambda: b.step(steps_b))
        out[key] = {"us_step": r4(secs_b / steps_b * 1e6),
                    "glups": r4(runs * p["nx"] * p["ny"] * steps_b / secs_b / 1e9)}
        b.close()
        for l in lats:
            l.close()

    # 32 lattices of 512 x 256 with an edge crack in another direction each
    # (0 to 87 degrees, prescribed v = 0.5, link-local faces) as one batch,
    # against the same lattices one after another
    try:
        out["line_sweep32"] = line_sweep(lbm, W, torch, stream)
    except lbm.LbmError as e:
        out["line_sweep32"] = {"error": str(e)[:200]}
    return out


def measure_virtual_ranks(lbm, W, torch, stream, problem, steps=256):
    """The 4096 x 2048 lattice split into 1, 2, 4 and 8 row slabs on this GPU
    (one batched step launch plus one halo-row exchange launch per step),
    timed back to back (graph replay, no flush)."""
    sites = problem["nx"] * problem["ny"]
    out = {}
    for n in (1, 2, 4, 8):
        d = lbm.Decomp(problem, n, "f32", stream=stream)
        d.step(64)
        out[str(n)] = r4(sites * steps / timed(torch, stream, lambda: d.step(steps)) / 1e9)
        d.close()
    return out


def measure_mixed_4096(lbm, W, torch, stream, peak, flush_l2, steps):
    """The 12-byte storage forms on the 4096 x 2048 K-criterion run (L2 flushed)."""
    p = W.kcrit_single()
    sites = p["nx"] * p["ny"]
    out = {}
    for storage in ("f32_lf", "f32_bf16", "f32_f16"):
        k = step_time(lbm, p, storage, stream, flush_l2, 2500, min(steps, 100))
        out[storage] = {"glups": r4(sites / k / 1e9), "frac": r4(12 * sites / k / 1e9 / peak)}
    return out


def profile_problem(args, W):
    """The workload of --profile-only (for ncu captures)."""
    if args.workload == "large":
        return W.large_prescribed(args.size)
    if args.workload == "kcrit":
        return W.kcrit_single()
    if args.workload == "d2q9":
        return dict(W.kcrit_single(), bc_mode="bounceback", lattice="D2Q9")
    if args.workload == "line":
        return W.kcrit_line()
    if args.workload == "line_macro":
        return W.kcrit_line_centre()
    if args.workload == "sec52":
        return W.kcrit_centre_crack()
    if args.workload == "adjoint_fwd":
        return W.adjoint_problem()["problem"]
    raise ValueError(args.workload)


def run_profile(args, W, lbm, torch, rank):
    """Prelude, warm-up and timed steps of one workload, nothing else (for
    ncu); prints the library's kernel times.  Large lattices are not flushed
    (their state exceeds L2), the others are."""
    p = profile_problem(args, W)
    stream = torch.cuda.current_stream()
    lat = lbm.Lattice(p, args.storage, stream=stream)
    if args.bulk:
        lat.set_bulk(True)
    lat.step(args.prelude)
    lat.sync()
    big = p["nx"] * p["ny"] * 16 > (1 << 30)
    flush = None if big else torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    lat.set_profiling(True)
    for _ in range(args.warmup + args.steps):
        if flush is not None:
            flush.fill_(1)
        lat.step(1)
    lat.sync()
    prof = lat.profile(reset=True)
    if rank == 0:
        print(json.dumps({"profile_only": True, "workload": args.workload, "nx": p["nx"], "ny": p["ny"],
                          "steps": args.warmup + args.steps, **prof}), flush=True)
    lat.close()
    return 0


def run_ours(args, rank, world, local):
    import numpy as np
    import torch
    from paper_2206_12412_gb300 import lbm
    from paper_2206_12412_gb300 import workloads as W

    torch.cuda.set_device(local)
    if args.profile_only:
        return run_profile(args, W, lbm, torch, rank)
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

    peak, peak_kind = measured_peaks()
    problem = W.large_prescribed()
    sites = problem["nx"] * problem["ny"]
    stream = torch.cuda.current_stream()
    lat = lbm.Lattice(problem, HEADLINE_STORAGE, stream=stream)
    lat.step(args.prelude)
    for _ in range(args.warmup):
        lat.step(1)
    lat.sync()

    # timed region: one step per pair of events; the 2.1 GB state is 16x the
    # L2, so each step streams its inputs from HBM without a flush
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
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
        lat.step(1)
    kern_s = kernel_seconds(lat)
    # the same kernel with its interior CTAs staging rows by bulk copies (A/B)
    lat.set_bulk(True)
    for _ in range(args.steps):
        lat.step(1)
    kern_bulk_s = kernel_seconds(lat)
    lat.set_bulk(False)
    lat.set_profiling(False)
    achieved = BYTES_PER_SITE * sites / kern_s / 1e9
    traffic = traffic_from_profile(sites)

    # end to end through the public API with host buffers: upload the state
    # from pinned memory, run the steps, read back the fields and the
    # per-step crack record
    w_h = torch.empty((problem["ny"], problem["nx"]), dtype=torch.float32, pin_memory=True)
    wd_h = torch.empty_like(w_h, pin_memory=True)
    w_np, wd_np = w_h.numpy(), wd_h.numpy()
    lbm.lbm_fields(lat.h, 0, w_np.ctypes.data, False, lat.dtype_code)
    lbm.lbm_fields(lat.h, 1, wd_np.ctypes.data, False, lat.dtype_code)
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
    launch = lat.launch()
    lat.close()
    del w_h, wd_h
    torch.cuda.empty_cache()

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    flush_sum = torch.empty((), dtype=torch.int64, device="cuda")

    def flush_l2():
        # write a buffer twice the size of L2, then read it back: L2 ends up
        # holding clean lines of the flush buffer, none of the lattice state
        flush.fill_(1)
        flush_sum.copy_(flush.view(torch.int64).sum())

    extra = {}
    if not args.no_extensions:
        extra["kcrit_4096x2048"], t_kcrit = measure_kcrit4096(lbm, W, torch, stream, peak, flush_l2, 100)
        extra["c1_128x128_f64"] = measure_c1(lbm, W, torch, stream)
        extra["extensions"] = measure_extensions(lbm, W, torch, stream, peak, flush_l2)
        extra["crack_share"] = crack_share(lbm, W, torch, stream, flush_l2, t_kcrit)
    patterns = {}
    if not args.no_mixed:
        patterns["mixed_precision"] = {"16384": measure_storage_large(lbm, W, torch, stream, peak),
                                       "4096": measure_mixed_4096(lbm, W, torch, stream, peak, flush_l2, args.steps)}
    if not args.no_virtual_ranks:
        patterns["virtual_ranks"] = measure_virtual_ranks(lbm, W, torch, stream, W.kcrit_single())
    if not args.no_adjoint:
        patterns["adjoint"] = measure_adjoint(lbm, W, torch, stream)
    if not args.no_batched:
        patterns["batched"] = measure_batched(lbm, W, torch, stream, 128, peak, full_steps=W.BATCH_STEPS)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": problem["nx"], "ny": problem["ny"], "storage": "f32_leapfrog",
                   "crack": "prescribed v=0.5", "bc_mode": problem["bc_mode"], "prelude_steps": args.prelude,
                   "l2": "inputs larger than L2 (2.1 GB state), no flush",
                   "parallelism": f"{world} independent replicas" if world > 1 else "single GPU",
                   "launch": launch},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": "step_kernel<float, Lf>", "kernel_ms": kern_s * 1e3, "bytes_per_site": BYTES_PER_SITE},
        "e2e": {"value": world * sites * args.steps / e2e_s / 1e9, "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps,
        "bulk_march": {"us": r4(kern_bulk_s * 1e6), "frac": r4(BYTES_PER_SITE * sites / kern_bulk_s / 1e9 / peak),
                       "register_us": r4(kern_s * 1e6)},
        "clocks": clk,
        "wall_s": r4(wall),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    line.update(extra)
    line.update(patterns)
    if rank == 0:
        print(json.dumps(line, separators=(",", ":")), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prelude", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 256-lattice batched measurement")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the sensor-misfit gradient measurement")
    ap.add_argument("--no-virtual-ranks", action="store_true", help="skip the row-slab decomposition measurement")
    ap.add_argument("--no-mixed", action="store_true", help="skip the 16-bit storage measurements")
    ap.add_argument("--no-extensions", action="store_true",
                    help="skip the 4096x2048, 128x128, D2Q9, line-crack and Sec. 5.2 measurements")
    ap.add_argument("--batched-only", action="store_true",
                    help="only the batched measurement, --steps steps of --batched-count lattices (for ncu)")
    ap.add_argument("--batched-count", type=int, default=256, help="lattices in the batched measurement")
    ap.add_argument("--batched-shape", default=None,
                    help="with --batched-only: THREADS,ROWS[,LOOKAHEAD] -- only the batched steps at that launch shape")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="only the sensor-misfit gradient measurement (for ncu)")
    ap.add_argument("--adjoint-steps", type=int, default=None, help="steps of the adjoint workload (default 8000)")
    ap.add_argument("--profile-only", action="store_true",
                    help="only prelude, warm-up and timed steps of --workload (for ncu); prints kernel times")
    ap.add_argument("--workload", default="large", choices=["large", "kcrit", "d2q9", "line", "line_macro", "sec52", "adjoint_fwd"],
                    help="with --profile-only: large = the headline lattice at --size (16384: the headline "
                         "itself), kcrit = 4096x2048 K-criterion, d2q9 / line / line_macro = its D2Q9 and "
                         "20-degree forms, sec52 = the Sec. 5.2 example, adjoint_fwd = the 1024 x 1024 prescribed-growth "
                         "forward of the adjoint configuration")
    ap.add_argument("--size", type=int, default=16384, help="with --workload large: the lattice's side")
    ap.add_argument("--storage", default="f32", choices=["f32", "f32_lf", "f32_bf16", "f32_f16", "f64"],
                    help="with --profile-only: the storage form")
    ap.add_argument("--bulk", action="store_true", help="with --profile-only: the bulk-copy march (lbm_set_bulk)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.batched_only or args.adjoint_only:
        import torch
        from paper_2206_12412_gb300 import lbm
        from paper_2206_12412_gb300 import workloads as W
        torch.cuda.set_device(local)
        if args.batched_only and args.batched_shape:
            shape = tuple(int(x) for x in args.batched_shape.split(","))
            out = {"batched_only": True, **profile_batched(lbm, W, torch, torch.cuda.current_stream(), args.steps,
                                                           shape, count=args.batched_count)}
        elif args.batched_only:
            peak, _ = measured_peaks()
            out = {"batched_only": True, **measure_batched(lbm, W, torch, torch.cuda.current_stream(), args.steps,
                                                           peak, count=args.batched_count)}
        else:
            out = {"adjoint_only": True, **measure_adjoint(lbm, W, torch, torch.cuda.current_stream(),
                                                           n_steps=args.adjoint_steps)}
        if rank == 0:
            print(json.dumps(out), flush=True)
        return 0
    return run_ours(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
