"""Benchmark of the PPPM k-space path on GB300.

One step = one full pass of the k-space path (particle_map + sort, make_rho,
forward FFT, influence-function multiply with energy/virial, inverse FFTs,
fieldforce) over the water-like workload: 10,667 rigid 3-site molecules
(32,001 charges) in a 68 A periodic cube, mesh 64^3, order 5, ik
differentiation, FP32 spreading/FFT/interpolation with compensated mesh
accumulation.  Inputs are resident in HBM; the L2 is flushed (256 MiB write)
before every timed step and each step is timed with CUDA events on the plan's
stream.  The step runs as one captured CUDA graph.

Also reported on the same line: Mparticles/s, the force error of this FP32C
form against the FP64 form (same GPU, same inputs), the dominant kernel's
roofline fraction, the end-to-end rate through the host-buffer C-ABI call,
the FP64 oracle timed on the host cores, and the same metric for ad / FP64.
More is measured on rank 0 (key "extra", skipped with --no-extra): the
2,048,001-charge water-like system (256^3, P=7, ad, FP32C; the HBM-sized
case: per-stage times and the make_rho / fieldforce roofline fractions), the
batch of 256 independent systems (one call, one graph; against the FP64 batch
and against 256 single-system plans), the real-space erfc sum of the bench
workload (r_C = 10 A), the other half of the Ewald split, the mesh chosen for
a target accuracy with step times by mesh edge, and the differentiable energy
of the 99,999-charge system (96^3): force step and energy with gradients.

--impl reference times the FP64 CPU oracle on the same workload instead.
Multi-GPU: the path does not shard (one system); N ranks run N independent
replicas and report the summed throughput.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_FLUSH_BYTES = 256 << 20
PROFILE_EVERY = 10  # timed steps per step that carries the dominant kernel's events
WORKLOAD = "c2"


def workload():
    from paper_1702_04250_gb300.workloads import config

    return config(WORKLOAD)


def metric_name():
    return "PPPM k-space steps/sec at 1e-4 rel force error vs FP64 form (water-like 32,001 charges, 64^3, P=5, ik, FP32C)"


def config_dict(w, extra=None):
    d = {"workload": "c2 water-like: 10,667 rigid 3-site molecules (32,001 charges), 68 A cube, mesh 64^3, "
                     "order 5, ik, g_ewald for 1e-4 at r_C = 10 A",
         "n_charges": int(w.n), "mesh": list(w.mesh), "order": int(w.order), "diff": "ik", "precision": "fp32c",
         "l2": "flushed (256 MiB write) before every timed step", "graph": True}
    if extra:
        d.update(extra)
    return d


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([s.strip() for s in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for k, nm in enumerate(names):
                if len(s) > 5 + k and s[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def known_traffic(stage, workload_name, source):
    """DRAM bytes per launch from profiles/dram_traffic.txt for this stage as
    implemented in `source`, or None when no capture of it exists or the
    kernel's sources changed since (the line stores their hash)."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    for ln in lines:
        if ln.startswith("#") or not ln.strip():
            continue
        st, wl, src, sha, nbytes = ln.split()
        if st == stage and wl == workload_name and src == source:
            m = hashlib.sha1()
            for f in (src, "paper_1702_04250_gb300/csrc/pppm_common.cuh"):
                m.update(open(os.path.join(ROOT, f), "rb").read())
            return int(nbytes) if m.hexdigest()[:16] == sha else None
    return None


def aggregate_ms(t_ms, world):
    """Max over ranks of a per-rank time (ms); a no-op for one rank."""
    import torch

    if world <= 1 or not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return float(t_ms)
    dev = "cuda" if torch.distributed.get_backend() == "nccl" else "cpu"
    tt = torch.tensor([float(t_ms)], dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
    return float(tt.item())


def throughput(units_per_rank, t_ms, steps, world):
    """Whole-job units/s: every rank processed units_per_rank per step; the
    slowest rank's time bounds the job."""
    return world * units_per_rank * steps / (t_ms * 1e-3)


# shared-memory int32 atomic adds per SM per clock on GB300, conflict-free
# warps (microbenchmark of ATOMS.ADD without return)
SHARED_ATOMIC_OPS_PER_CLK_SM = 25.9
N_SM = 152


def onchip_make_rho(n, P, ms, sm_mhz):
    """make_rho against its on-chip bound: FP32C adds two int32 words per
    stencil point in shared memory (2 N P^3 atomics per launch)."""
    ops = 2.0 * n * P ** 3
    mhz = sm_mhz or 2070.0
    peak = SHARED_ATOMIC_OPS_PER_CLK_SM * N_SM * mhz * 1e6 / 1e9
    ach = ops / (ms * 1e-3) / 1e9
    return {"resource": "shared-memory int32 atomics", "ops_per_launch": int(ops),
            "achieved_gops": round(ach, 1), "peak_gops": round(peak, 1), "frac": round(ach / peak, 4),
            "peak_source": f"microbenchmark, {SHARED_ATOMIC_OPS_PER_CLK_SM} ops/clk/SM x {N_SM} SMs at {mhz:.0f} MHz"}


def mesh_stage_gbs(mesh, stage_ms, ik=False):
    """Achieved GB/s of the FP32 mesh stages at their minimum traffic: one read
    and one write of each array a stage touches (a lower bound for cuFFT's
    multi-pass transforms).  Forward: real mesh in, half spectrum out; green:
    rho_hat and G in, one (ad) or three (ik) spectra out; inverse: the
    spectra in, the potential or the interleaved field out."""
    m = int(mesh[0]) * int(mesh[1]) * int(mesh[2])
    mh = int(mesh[0]) * int(mesh[1]) * (int(mesh[2]) // 2 + 1)
    nspec = 3 if ik else 1
    nbytes = {"fft_fwd": 4 * m + 8 * mh,
              "green": 8 * mh + 4 * mh + 8 * nspec * mh,
              "fft_inv": 8 * nspec * mh + (16 if ik else 4) * m}
    return {k: {"bytes": b, "gbs": round(b / (stage_ms[k] * 1e-3) / 1e9, 1)}
            for k, b in nbytes.items() if stage_ms.get(k)}


def make_plan(w, g, mode, prec, graph=True):
    from paper_1702_04250_gb300 import pppm

    return pppm.PPPM(w.box, w.n, w.order, w.mesh, g, mode=mode, precision=prec, qqrd2e=w.qqrd2e, graph=graph)


def time_steps(torch, plan, x, q, f, ev, steps, warmup, flush, profile=False, sync_ranks=True, every=1):
    """Returns (total device ms over the timed steps, per-stage ms averages).
    profile: stages to time with events (True = all); every: time them in
    every k-th step only (the plan keeps a captured graph for each event
    set, so the other steps run the graph without event nodes).
    sync_ranks: barrier with the other ranks around the timed region."""
    s = plan.stream
    stage_sum = {k: 0.0 for k in plan.STAGES}
    n_prof = 0
    for i in range(warmup):
        plan.set_profiling(profile if (profile and i % every == 0) else False)
        flush.zero_()
        plan.compute(x, q, f, ev)
    torch.cuda.synchronize()
    if sync_ranks and torch.distributed.is_available() and torch.distributed.is_initialized():
        torch.distributed.barrier()
    torch.cuda.synchronize()
    total = 0.0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for i in range(steps):
        prof_now = bool(profile) and i % every == 0
        plan.set_profiling(profile if prof_now else False)
        with torch.cuda.stream(s):
            flush.zero_()
        e0.record(s)
        plan.compute(x, q, f, ev)
        e1.record(s)
        e1.synchronize()
        total += e0.elapsed_time(e1)
        if prof_now:
            n_prof += 1
            for k, v in plan.stage_times().items():
                if v >= 0:
                    stage_sum[k] += v
    torch.cuda.synchronize()
    if sync_ranks and torch.distributed.is_available() and torch.distributed.is_initialized():
        torch.distributed.barrier()
    plan.set_profiling(False)
    return total, {k: v / max(n_prof, 1) for k, v in stage_sum.items()}


def gpu_arm(args, rank, world):
    import torch

    from paper_1702_04250_gb300 import build, pppm

    build.build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    w = workload()
    q2 = float(np.sum(w.q ** 2))
    g = pppm.estimate_g(w.rel_acc, w.r_cut, w.n, q2, w.box)
    x32 = torch.tensor(w.x, dtype=torch.float32, device="cuda")
    q32 = torch.tensor(w.q, dtype=torch.float32, device="cuda")
    x64 = torch.tensor(w.x, dtype=torch.float64, device="cuda")
    q64 = torch.tensor(w.q, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    plan = make_plan(w, g, "ik", "fp32c")
    f = torch.empty((w.n, 3), dtype=torch.float32, device="cuda")
    ev = torch.zeros(8, dtype=torch.float64, device="cuda")
    variant = plan.autotune(x32, q32)  # what a user of the plan does once
    plan.compute(x32, q32, f, ev)
    plan.sync()

    # accuracy of this form against the FP64 form on the same GPU and inputs
    p64 = make_plan(w, g, "ik", "fp64", graph=False)
    f64, ev64 = p64.compute(x32.double(), q32.double())
    p64.sync()
    f64n = f64.cpu().numpy()
    rel_err = math.sqrt(float(np.sum((f.double().cpu().numpy() - f64n) ** 2) / np.sum(f64n ** 2)))
    e_err = abs(ev[0].item() - ev64[0].item()) / abs(ev64[0].item())

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    # which of our kernels dominates (all stage events on, short untimed pass)
    _, disc = time_steps(torch, plan, x32, q32, f, ev, 20, 3, flush, profile=True)
    own_fft = bool(variant & 8)  # the hand-written Poisson solve (else cuFFT + k_green)
    own = {k: disc[k] for k in ("sort", "make_rho", "green", "fieldforce") + (("fft_fwd", "fft_inv") if own_fft else ())}
    dom = max(own, key=own.get)

    # the timed region: K steps; every 10th carries events around the dominant kernel
    t_ms, stages = time_steps(torch, plan, x32, q32, f, ev, args.steps, args.warmup, flush, profile=[dom],
                              every=PROFILE_EVERY)
    clocks_rep = clocks.stop()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t_ms = aggregate_ms(t_ms, world)
    ms_per_step = t_ms / args.steps
    steps_per_s = throughput(1, t_ms, args.steps, world)

    # the same steps without any stage event (graph of kernels only)
    t_plain, _ = time_steps(torch, plan, x32, q32, f, ev, max(20, args.steps // 2), 3, flush, profile=False)
    ms_plain = t_plain / max(20, args.steps // 2)

    # roofline of the dominant hand-written kernel
    stage_ms = dict(disc)        # all stages, discovery pass (events inflate each)
    stage_ms[dom] = stages[dom]  # the dominant kernel, timed region (every 10th step)
    N, M = w.n, int(np.prod(w.mesh))
    MH = (M // w.mesh[2]) * (w.mesh[2] // 2 + 1)  # half spectrum
    alg_bytes = {
        "sort": (12 + 4) * N * 2 + (16 + 4 + 4 + 4 + 4) * N,   # x,q read twice; record, anchor, perm, rank writes
        "make_rho": (16 + 4) * N + 4 * M,                        # sorted records + anchors in, mesh out once
        "green": 8 * MH * (1 + 3) + 4 * MH,                      # rho_hat in, three spectra out, G in
        "fft_fwd": 4 * M + 8 * MH,                               # mesh in, rho_hat out
        "fft_inv": 8 * MH * 3 + 12 * M,                          # three spectra in, three field components out
        "fieldforce": 16 * M + (16 + 4 + 4 + 12) * N,            # float4 field once, records, anchors, perm, forces
    }[dom]
    source = {"sort": "k_sort.cu", "make_rho": "k_rho.cu", "fieldforce": "k_force.cu", "fft_fwd": "k_fft.cu",
              "fft_inv": "k_fft.cu", "green": "k_fft.cu" if own_fft else "k_green.cu"}[dom]
    # the committed c2 captures are of variant 9 (one-brick make_rho, tile-staged fieldforce)
    traffic_ok = not ((dom == "fieldforce" and not variant & 1) or (dom == "make_rho" and variant & 4))
    peak, peak_kind = measured_peak()
    achieved = alg_bytes / (stage_ms[dom] * 1e-3) / 1e9
    roof = {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": known_traffic(dom, WORKLOAD, "paper_1702_04250_gb300/csrc/" + source) if traffic_ok else None,
            "peak_source": peak_kind,
            "alg_bytes_per_launch": int(alg_bytes), "avg_launch_ms": round(stage_ms[dom], 5),
            "launches_timed": f"every {PROFILE_EVERY}th timed step carries events around this kernel",
            "stage_ms": {k: round(v, 5) for k, v in stage_ms.items()}}

    # end to end through the host-buffer C-ABI call (pinned host memory)
    xh = torch.tensor(w.x, dtype=torch.float32).pin_memory()
    qh = torch.tensor(w.q, dtype=torch.float32).pin_memory()
    fh = torch.empty((w.n, 3), dtype=torch.float32).pin_memory()
    evh = torch.empty(8, dtype=torch.float64).pin_memory()
    for _ in range(3):
        plan.compute_host_into(w.n, xh.data_ptr(), qh.data_ptr(), fh.data_ptr(), evh.data_ptr())
    ne = max(20, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(ne):
        plan.compute_host_into(w.n, xh.data_ptr(), qh.data_ptr(), fh.data_ptr(), evh.data_ptr())
    e2e_s = (time.perf_counter() - t0) / ne

    # the other forms of the same metric, shorter runs
    variants = {}
    for mode, prec, xx, qq in (("ad", "fp32c", x32, q32), ("ik", "fp64", x64, q64), ("ad", "fp64", x64, q64)):
        pv = make_plan(w, g, mode, prec)
        fv = torch.empty((w.n, 3), dtype=xx.dtype, device="cuda")
        tv, _ = time_steps(torch, pv, xx, qq, fv, ev, max(20, args.steps // 4), 3, flush)
        variants[f"{mode}_{prec}"] = {"steps_per_s": round(1000.0 / (tv / max(20, args.steps // 4)), 1)}
        pv.close()

    # particle_map, scatter, make_rho, energy_final, fieldforce, and either green (the 3-D
    # transforms in cuFFT, not ours) or the three hand-written Poisson-solve kernels
    launches_per_step = 8 if own_fft else 6
    line = {
        "metric": metric_name(), "value": round(steps_per_s, 2), "unit": "steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32c", "data": "synthetic",
        "config": config_dict(w, {"parallelism": "replicas" if world > 1 else "single",
                                  "fieldforce_variant": "tile-staged" if variant & 1 else "per-particle L1",
                                  "poisson_solve": "hand-written FFT" if own_fft else "cuFFT"}),
        "mparticles_per_s": round(world * N / (ms_per_step * 1e-3) / 1e6, 2),
        "rel_force_err_vs_fp64": rel_err, "rel_energy_err_vs_fp64": e_err,
        "ms_per_step_without_kernel_events": round(ms_plain, 5),
        "steps_per_s_without_kernel_events": round(world * 1000.0 / ms_plain, 2),
        "roofline": roof,
        "onchip": onchip_make_rho(N, w.order, stage_ms["make_rho"], clocks_rep.get("sm_mhz")),
        "e2e": {"value": round(world / e2e_s, 2), "unit": "steps/s", "h2d_bytes_per_step": int(16 * N),
                "d2h_bytes_per_step": int(12 * N + 56)},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks_rep,
        "variants": variants,
    }
    return line


# ---------------------------------------------------------------------------
# extra workloads (rank 0)
# ---------------------------------------------------------------------------
def large_leg(torch, flush, steps=30):
    """2,048,001 water-like charges, 256^3, P=7, ad, FP32C, one graph per step."""
    from paper_1702_04250_gb300 import pppm
    from paper_1702_04250_gb300.workloads import config

    w = config("c3")
    g = pppm.estimate_g(w.rel_acc, w.r_cut, w.n, float(np.sum(w.q ** 2)), w.box)
    x = torch.tensor(w.x, dtype=torch.float32, device="cuda")
    q = torch.tensor(w.q, dtype=torch.float32, device="cuda")
    plan = pppm.PPPM(w.box, w.n, w.order, w.mesh, g, mode="ad", precision="fp32c", qqrd2e=w.qqrd2e, graph=True)
    variant = plan.autotune(x, q)
    f = torch.empty((w.n, 3), dtype=torch.float32, device="cuda")
    ev = torch.zeros(8, dtype=torch.float64, device="cuda")
    t_plain, _ = time_steps(torch, plan, x, q, f, ev, steps, 3, flush, profile=False, sync_ranks=False)
    _, stage = time_steps(torch, plan, x, q, f, ev, steps, 3, flush, profile=True, sync_ranks=False)
    ms = t_plain / steps
    # error of this form against the FP64 form on a 1 % subsample (every 100th charge)
    p64 = pppm.PPPM(w.box, w.n, w.order, w.mesh, g, mode="ad", precision="fp64", qqrd2e=w.qqrd2e)
    f64, ev64 = p64.compute(x.double(), q.double())
    p64.sync()
    sub = slice(0, w.n, 100)
    a = f[sub].double().cpu().numpy()
    b = f64[sub].cpu().numpy()
    err = math.sqrt(float(np.sum((a - b) ** 2) / np.sum(b ** 2)))
    e_err = abs(ev[0].item() - ev64[0].item()) / abs(ev64[0].item())
    p64.close()
    N, M = w.n, int(np.prod(w.mesh))
    peak, kind = measured_peak()
    alg = {"make_rho": 20 * N + 4 * M, "fieldforce": 4 * M + 36 * N}
    roof = {}
    for k, nbytes in alg.items():
        achieved = nbytes / (stage[k] * 1e-3) / 1e9
        src = "paper_1702_04250_gb300/csrc/" + ("k_rho.cu" if k == "make_rho" else "k_force.cu")
        # the committed capture is of the per-particle fieldforce (the ad default)
        tr = known_traffic(k, "c3", src) if (k == "make_rho" or not variant & 1) else None
        roof[k] = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                   "frac": round(achieved / peak, 4), "traffic": tr, "alg_bytes_per_launch": int(nbytes),
                   "avg_launch_ms": round(stage[k], 4), "peak_source": kind}
    plan.close()
    return {"workload": "water-like 682,667 molecules (2,048,001 charges), 272 A cube, mesh 256^3, order 7, ad, FP32C",
            "steps_per_s": round(1000.0 / ms, 2), "ms_per_step": round(ms, 4),
            "mparticles_per_s": round(N / (ms * 1e-3) / 1e6, 1),
            "rel_force_err_vs_fp64_1pct_subsample": err, "rel_energy_err_vs_fp64": e_err,
            "fieldforce_variant": "tile-staged" if variant & 1 else "per-particle L1",
            "stage_ms": {k: round(v, 4) for k, v in stage.items()},
            "roofline": roof,
            "onchip_make_rho": onchip_make_rho(N, w.order, stage["make_rho"], None),
            "mesh_stage_gbs": mesh_stage_gbs(w.mesh, stage),
            "timing": f"{steps} graph steps, L2 flushed before each; stage times from a second pass with stage events"}


def real_leg(torch, flush, steps=30):
    """Real-space part of the Ewald split on the water-like 32,001 charges,
    r_C = 10 A, FP32, against the FP64 form."""
    from paper_1702_04250_gb300 import pppm
    from paper_1702_04250_gb300.workloads import config

    w = config("c2")
    g = pppm.estimate_g(w.rel_acc, w.r_cut, w.n, float(np.sum(w.q ** 2)), w.box)
    out = {}
    for prec in ("fp32", "fp64"):
        dt = torch.float64 if prec == "fp64" else torch.float32
        rs = pppm.RealSpace(w.box, w.n, w.r_cut, g, precision=prec, qqrd2e=w.qqrd2e)
        x = torch.tensor(w.x, dtype=dt, device="cuda")
        q = torch.tensor(w.q, dtype=dt, device="cuda")
        f = torch.empty((w.n, 3), dtype=dt, device="cuda")
        for _ in range(3):
            rs.compute(x, q, f)
        rs.sync()
        s = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for _ in range(steps):
            flush.zero_()
            e0.record(s)
            rs.compute(x, q, f)
            e1.record(s)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        rs.sync()
        out[prec] = (tot / steps, f.double().cpu().numpy(), rs.info()["cells"])
        rs.close()
    ms, f32, cells = out["fp32"]
    f64 = out["fp64"][1]
    err = math.sqrt(float(np.sum((f32 - f64) ** 2) / np.sum(f64 ** 2)))
    V = float(np.prod(w.box))
    pairs = w.n * (w.n / V) * 4.0 / 3.0 * math.pi * w.r_cut ** 3  # ordered pairs within r_C
    return {"workload": "water-like 32,001 charges, 68 A cube, r_C = 10 A, erfc real-space sum, FP32",
            "cells": list(cells), "ms_per_call": round(ms, 4), "calls_per_s": round(1000.0 / ms, 1),
            "pairs_within_cutoff_per_s": float(f"{pairs / (ms * 1e-3):.4g}"),
            "fp64_ms_per_call": round(out["fp64"][0], 4), "rel_force_err_fp32_vs_fp64": err,
            "timing": f"{steps} calls, L2 flushed before each"}


def autograd_leg(torch, flush, steps=30):
    """The differentiable energy on 99,999 water-like charges (100 A cube,
    96^3, P=5, ik): the force step and the energy with its hand-written
    gradients (dE/dx, dE/dq: one pppm_energy_grad call, what the autograd
    Function runs), FP32C and FP64, one graph per force step."""
    from paper_1702_04250_gb300 import pppm
    from paper_1702_04250_gb300.workloads import config

    w = config("c5")
    g = pppm.estimate_g(w.rel_acc, w.r_cut, w.n, float(np.sum(w.q ** 2)), w.box)
    out = {}
    for prec in ("fp32c", "fp64"):
        dt = torch.float64 if prec == "fp64" else torch.float32
        x = torch.tensor(w.x, dtype=dt, device="cuda")
        q = torch.tensor(w.q, dtype=dt, device="cuda")
        plan = pppm.PPPM(w.box, w.n, w.order, w.mesh, g, mode="ik", precision=prec, qqrd2e=w.qqrd2e, graph=True)
        variant = plan.autotune(x, q)
        f = torch.empty((w.n, 3), dtype=dt, device="cuda")
        ev = torch.zeros(8, dtype=torch.float64, device="cuda")
        t_force, _ = time_steps(torch, plan, x, q, f, ev, steps, 3, flush, sync_ranks=False)
        s = plan.stream
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        for _ in range(3):
            plan.energy_grad(x, q)
        plan.sync()
        tot = 0.0
        for _ in range(steps):
            with torch.cuda.stream(s):
                flush.zero_()
            e0.record(s)
            plan.energy_grad(x, q)
            e1.record(s)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        plan.sync()
        out[prec] = {"force_step_us": round(t_force / steps * 1e3, 1),
                     "energy_and_gradients_us": round(tot / steps * 1e3, 1),
                     "poisson_solve": "hand-written FFT" if variant & 8 else "cuFFT"}
        plan.close()
    return {"workload": "water-like 33,333 molecules (99,999 charges), 100 A cube, mesh 96^3, order 5, ik",
            **out, "timing": f"{steps} calls each, L2 flushed before each"}


def mesh_leg(torch, flush, steps=40):
    """Mesh choice for a target accuracy on the water-like 32,001 charges
    (r_C = 10 A, 1e-4; the error estimate runs as one FP64 kernel per mesh
    tried), why FFT-friendly sizes matter (the same FP32C ik step on mesh
    edges 64 (a power of two), 67 and 71 (primes), 70 (2 5 7) and 72
    (2^3 3^2), with g held fixed), and which order meets the target fastest
    (orders 3-7, each with its chosen mesh)."""
    from paper_1702_04250_gb300 import pppm
    from paper_1702_04250_gb300.workloads import config

    w = config("c2")
    q2 = float(np.sum(w.q ** 2))
    choice = {}
    for name, kind in (("primes_le_7", pppm.FFT_SMOOTH), ("powers_of_two", pppm.FFT_POW2)):
        t0 = time.perf_counter()
        mesh, g, err = pppm.choose_mesh(w.box, w.n, q2, w.order, w.r_cut, w.rel_acc, kind)
        choice[name] = {"mesh": list(mesh), "g_ewald": round(g, 6), "est_rms_force_err": float(f"{err:.4g}"),
                        "choose_ms": round((time.perf_counter() - t0) * 1e3, 1)}
    g = pppm.estimate_g(w.rel_acc, w.r_cut, w.n, q2, w.box)
    x = torch.tensor(w.x, dtype=torch.float32, device="cuda")
    q = torch.tensor(w.q, dtype=torch.float32, device="cuda")
    f = torch.empty((w.n, 3), dtype=torch.float32, device="cuda")
    ev = torch.zeros(8, dtype=torch.float64, device="cuda")
    sizes = {}
    for m in (64, 67, 70, 71, 72):
        plan = pppm.PPPM(w.box, w.n, w.order, (m, m, m), g, mode="ik", precision="fp32c", qqrd2e=w.qqrd2e,
                         graph=True)
        plan.autotune(x, q)
        tot, _ = time_steps(torch, plan, x, q, f, ev, steps, 3, flush, sync_ranks=False)
        sizes[str(m)] = {"us_per_step": round(tot / steps * 1e3, 1),
                         "est_rms_force_err": float(f"{pppm.kspace_error(w.box, (m,) * 3, w.order, g, w.n, q2):.4g}")}
        plan.close()
    # the order that meets the target fastest (a larger stencil allows a coarser mesh)
    orders = []
    for order in (3, 4, 5, 6, 7):
        for name, kind in (("primes_le_7", pppm.FFT_SMOOTH), ("powers_of_two", pppm.FFT_POW2)):
            mesh, go, err = pppm.choose_mesh(w.box, w.n, q2, order, w.r_cut, w.rel_acc, kind)
            plan = pppm.PPPM(w.box, w.n, order, mesh, go, mode="ik", precision="fp32c", qqrd2e=w.qqrd2e,
                             graph=True)
            plan.autotune(x, q)
            tot, _ = time_steps(torch, plan, x, q, f, ev, steps, 3, flush, sync_ranks=False)
            orders.append({"order": order, "sizes": name, "mesh": list(mesh), "est_rms_force_err": float(f"{err:.4g}"),
                           "us_per_step": round(tot / steps * 1e3, 1)})
            plan.close()
    return {"workload": "water-like 32,001 charges, 68 A cube, P=5, ik, r_C = 10 A, target 1e-4",
            "choice": choice, "step_by_mesh_edge_fp32c": sizes, "order_sweep_fp32c": orders,
            "timing": f"{steps} graph steps per mesh, L2 flushed before each"}


def batch_leg(torch, flush, steps=20):
    """256 independent systems in one call and one graph, FP32C ik, against
    the FP64 batch and against one single-system plan per system."""
    from paper_1702_04250_gb300 import pppm
    from paper_1702_04250_gb300.workloads import batch_systems

    ws = batch_systems()
    systems = []
    for w in ws:
        g = pppm.estimate_g(w.rel_acc, w.r_cut, w.n, float(np.sum(w.q ** 2)), w.box)
        systems.append(dict(box=w.box, n=w.n, order=w.order, mesh=w.mesh, g_ewald=g, x=w.x, q=w.q))
    C = ws[0].qqrd2e
    xs = np.concatenate([s["x"] for s in systems])
    qs = np.concatenate([s["q"] for s in systems])
    ntot = len(qs)

    def time_batch(prec):
        dt = torch.float64 if prec == "fp64" else torch.float32
        b = pppm.PPPMBatch(systems, mode="ik", precision=prec, qqrd2e=C, graph=True)
        x = torch.tensor(xs, dtype=dt, device="cuda")
        q = torch.tensor(qs, dtype=dt, device="cuda")
        b.autotune(x, q)
        f = torch.empty((ntot, 3), dtype=dt, device="cuda")
        for _ in range(3):
            b.compute(x, q, f)
        b.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for _ in range(steps):
            with torch.cuda.stream(b.stream):
                flush.zero_()
            e0.record(b.stream)
            b.compute(x, q, f)
            e1.record(b.stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        b.sync()
        out = f.double().cpu().numpy()
        info = b.info()
        b.close()
        return tot / steps, out, info

    ms32, f32, info = time_batch("fp32c")
    ms64, f64, _ = time_batch("fp64")
    err = math.sqrt(float(np.sum((f32 - f64) ** 2) / np.sum(f64 ** 2)))

    # the same 256 systems as 256 single-system plans, one graph each, back to back
    plans, xt, qt, ft = [], [], [], []
    stream = torch.cuda.Stream()
    for sd in systems:
        p = pppm.PPPM(sd["box"], sd["n"], sd["order"], sd["mesh"], sd["g_ewald"], "ik", "fp32c", C,
                      stream=stream, graph=True)
        plans.append(p)
        xt.append(torch.tensor(sd["x"], dtype=torch.float32, device="cuda"))
        qt.append(torch.tensor(sd["q"], dtype=torch.float32, device="cuda"))
        ft.append(torch.empty((sd["n"], 3), dtype=torch.float32, device="cuda"))
    for _ in range(2):
        for p, x, q, f in zip(plans, xt, qt, ft):
            p.compute(x, q, f)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    tot = 0.0
    for _ in range(max(3, steps // 4)):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0.record(stream)
        for p, x, q, f in zip(plans, xt, qt, ft):
            p.compute(x, q, f)
        e1.record(stream)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    ms_single = tot / max(3, steps // 4)
    for p in plans:
        p.close()
    return {"workload": f"{len(systems)} independent neutral +-1 systems, N 500-20,000 (total {ntot:,}), "
                        f"meshes 16^3-64^3 ({info['mesh_classes']} mesh classes), orders 3/5/7, ik",
            "fp32c": {"calls_per_s": round(1000.0 / ms32, 2), "ms_per_call": round(ms32, 4),
                      "systems_per_s": round(len(systems) * 1000.0 / ms32, 1),
                      "mparticles_per_s": round(ntot / (ms32 * 1e-3) / 1e6, 1)},
            "fp64": {"calls_per_s": round(1000.0 / ms64, 2), "ms_per_call": round(ms64, 4)},
            "fp32c_over_fp64": round(ms64 / ms32, 3),
            "rel_force_err_fp32c_vs_fp64": err,
            "single_plans_fp32c": {"ms_for_all_systems": round(ms_single, 4),
                                   "batch_speedup": round(ms_single / ms32, 2)},
            "timing": f"{steps} graph calls, L2 flushed before each"}


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ---------------------------------------------------------------------------
def oracle_rate(w, budget_s=12.0, max_steps=50):
    from oracle import OraclePPPM, estimate_g_ewald

    g = estimate_g_ewald(w.rel_acc, w.r_cut, w.n, float(np.sum(w.q ** 2)), w.box)
    o = OraclePPPM(w.box, w.mesh, w.order, g, "ik", w.qqrd2e)
    x = w.x.astype(np.float32).astype(np.float64)
    q = w.q.astype(np.float32).astype(np.float64)
    o.compute(x, q)
    n = 0
    t0 = time.perf_counter()
    while n < max_steps and time.perf_counter() - t0 < budget_s:
        o.compute(x, q)
        n += 1
    dt = time.perf_counter() - t0
    return n / dt, n, dt


def cpu_cores_used():
    # numpy's FFT and bincount run on one thread
    return 1


def cpu_baseline_obj(rate, sample):
    """The oracle's timing: the threads it used and the host's core count."""
    return {"value": round(rate, 4), "unit": "steps/s", "cores": cpu_cores_used(),
            "host_cores": os.cpu_count(), "kind": "oracle", "sample": sample}


def reference_arm(args, rank, world):
    if rank != 0:
        return None
    w = workload()
    steps = max(1, args.steps)
    budget = 60.0
    rate, n, dt = oracle_rate(w, budget_s=budget, max_steps=steps)
    return {"impl": "reference", "metric": metric_name(), "value": round(rate, 4), "unit": "steps/s",
            "n_gpus": world, "steps": n, "warmup": 1, "ms_per_step": round(1000.0 / rate, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(w, {"precision": "fp64 (oracle)"}),
            "cpu_baseline": cpu_baseline_obj(rate, f"{n} full oracle steps of the workload ({dt:.1f} s)"),
            "e2e": {"value": round(rate, 4), "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the 2M-charge and batched workloads")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        torch.distributed.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        line = reference_arm(args, rank, world)
        if line is not None:
            print(json.dumps(line))
        return
    line = gpu_arm(args, rank, world)
    if rank == 0 and not args.no_extra:
        import torch

        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        line["extra"] = {"large": large_leg(torch, flush), "batch": batch_leg(torch, flush),
                         "real_space": real_leg(torch, flush), "mesh_choice": mesh_leg(torch, flush),
                         "autograd_c5": autograd_leg(torch, flush)}
    if rank == 0:
        if not args.no_cpu_baseline:
            rate, n, dt = oracle_rate(workload())
            line["cpu_baseline"] = cpu_baseline_obj(rate, f"{n} full FP64 oracle steps of the same workload ({dt:.1f} s)")
        print(json.dumps(line))
    if world > 1:
        import torch

        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
