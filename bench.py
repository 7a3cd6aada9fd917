#!/usr/bin/env python3
"""Benchmark of the GB300 FDLB step: node-velocity updates/s (radial cells x momenta x SSP-RK3
steps per second) on the cylindrical Fourier-flow workload (1024 stretched cells, 16 x 8 x 8 =
1024 momenta, FP32 populations with FP64 moment sums).

One timed step = one SSP-RK3 step of the whole instance: one launch of the persistent step
kernel (per stage and tile the closure and the fused stage, grid barriers between stages) where
it applies, else 3 closure + 3 fused-stage launches replayed from a one-step CUDA graph; L2 is
flushed (256 MB write) before every timed step because the 4 MB population arrays would
otherwise stay L2-resident.  Device time from CUDA
events on the solver's stream; max over ranks (one independent replica per GPU: weak scaling).

Also reported: the dominant kernel against its roofline (it is bound by FP32 arithmetic issue:
algorithmic flops per launch / its event-timed duration against the FP32 CUDA-core peak;
the HBM view of the same launch for context), the end-to-end rate through the C ABI with host
buffers, the FP64 CPU oracle timed on the host cores (`cpu_baseline`), SM clocks sampled during
the run.

--impl reference times the FP64 CPU oracle on the same workload (the comparison arm).
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# the CPU legs time the oracle on one host thread: numpy's BLAS pools are held to one thread
# before numpy loads them (the library's host set-up keeps its OpenMP threads: the Fischer-Methfessel
# bands of a 512-instance batch take minutes on one core)
for _var in ("OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ[_var] = "1"

import numpy as np  # noqa: E402

from paper_2403_15051_gb300 import workloads as wl  # noqa: E402

METRIC = "node-velocity updates/s"
UNIT = "updates/s"
L2_FLUSH_BYTES = 256 << 20
REF_BUDGET_S = 120.0
KERNEL_SOURCES = ["paper_2403_15051_gb300/csrc/" + f for f in (
    "step_kernel.cuh", "stream_kernel.cuh", "closure_item.cuh", "device_common.cuh", "kernels_decl.h", "kernels.cuh")]


def accept_kn(kn, eta0):
    """C >= 3 for the confinement ratio the library derives from (Kn, eta0) (its host-only
    parameter conversion; C does not depend on the gap width)."""
    from paper_2403_15051_gb300 import fdlb

    C, _, _ = fdlb.physical_parameters(kn, eta0, 1.0)
    return C >= 3.0


def workload(name):
    if name == "fourier_cyl_1024":
        return [wl.fourier_cyl_1024()]
    if name == "couette_cyl_64":
        return [wl.couette_cyl_64()]
    if name == "fourier_sph_2048":
        return [wl.fourier_sph_2048(accept_kn)]
    if name == "batch_512":
        return wl.batch_instances(lambda kn, e, r: accept_kn(kn, e))
    if name == "batch_64":  # the first 64 instances of the same sweep (profiling captures)
        return wl.batch_instances(lambda kn, e, r: accept_kn(kn, e), n=64)
    if name == "couette_cyl_reduced_q20":  # the paper's HHLB(7,20) x HLB(7,8), p_z integrated out
        return [wl.couette_cyl_reduced()]
    raise SystemExit(f"unknown workload {name}")


FP32_LANES = 152 * 128  # SMs x FP32 lanes per SM
SM_MAX_MHZ = 2070.0
HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e nominal bandwidth


def alg_flops_per_update(geometry, nR, n2, n3):
    """Arithmetic of one population update in one fused stage (adds and multiplies, an FMA
    counted as two, a division as one): WENO5 face value of f/w 76 (five scalings, smoothness
    indicators 36, weights 11, candidate values 15, combination 9), advection flux difference 5,
    curvature force 2 nR + 2 n2 (+ 2 n3 on the sphere) plus 5 (8), Shakhov + J1 collision 52,
    RK combination 5, the 13 raw moment sums 30."""
    force = 2 * nR + 2 * n2 + (2 * n3 + 8 if geometry == wl.SPH else 5)
    return 76 + 5 + force + 52 + 5 + 30


def n_third(d):
    """Entries of the third momentum index: Q_3 nodes, or the pair (phi, chi) with p_z integrated out."""
    return 2 if d["geometry"] == wl.CYL_Z else d["Q_3"]


def units_per_step(ds):
    return sum(d["n_cells"] * 2 * d["Q_R"] * d["Q_2"] * n_third(d) for d in ds)


def oracle_problem(d):
    from oracle import solver as osolver

    reduced = d["geometry"] == wl.CYL_Z
    return osolver.make_problem(wl.CYL if reduced else d["geometry"], d["R_in"], d["R_out"], d["n_cells"], d["Q_R"],
                                d["Q_2"], d["Q_3"], eta0=d["eta0"], Kn=d.get("Kn"), sigma=d.get("sigma"),
                                beta=d.get("beta", 0.0) or 0.0, chi_model=d.get("chi_model", 0),
                                T_wall=tuple(d["T_wall"]), u_wall=tuple(d["u_wall"]), dt=d.get("dt"), reduced=reduced)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def hbm_view(alg_bytes, avg_ms, peak, peak_kind):
    """The HBM view of one launch: algorithmic bytes over its event-timed duration, against the
    measured copy bandwidth (`peak`) and, for context, the nominal HBM3e bandwidth."""
    achieved = alg_bytes / (avg_ms * 1e-3) / 1e9
    return {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "alg_bytes_per_launch": alg_bytes, "peak_source": peak_kind,
            "nominal_peak": HBM_NOMINAL_GBS, "frac_of_nominal": achieved / HBM_NOMINAL_GBS}


def kernel_source_hash():
    """Hash of the timed kernels' code: the sources with comments removed and whitespace collapsed
    (a change of prose leaves the recorded counters valid, any change of code does not)."""
    import re

    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(workload_name, kernel):
    """DRAM bytes per launch of `kernel` on the workload from the committed ncu summary, if it
    was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except Exception:
        return None
    ent = rec.get(workload_name + ":" + kernel)
    if not ent or ent.get("source_hash") != kernel_source_hash():
        return None
    return float(ent["dram_bytes_per_launch"])


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200", "-i",
                 str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
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
        except Exception:
            self.proc.kill()
        return self.summarise(self.lines)

    @staticmethod
    def summarise(lines):
        """Median and maximum SM clock and the throttle reasons seen active, from the CSV lines."""
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                clock, clock_max = float(parts[1]), float(parts[2])
            except ValueError:
                continue
            sm.append(clock)
            mx.append(clock_max)
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        if dist.is_initialized():
            pass
        elif torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:  # the bookkeeping of the replicas on host cores (tests)
            dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_step, steps, world, ms_max):
    """Whole-job throughput of `world` independent replicas: every rank advanced its own copy of
    the workload by `steps` steps; the job took the slowest rank's time."""
    return units_per_step * steps * world / (ms_max * 1e-3)


def cpu_baseline(ds, budget_s=15.0):
    """The FP64 oracle as it stands, on the host cores: whole SSP-RK3 steps of the workload
    (the first instance for a batch) until about `budget_s` seconds of work."""
    from oracle import solver as osolver

    d = ds[0]
    P = oracle_problem(d)
    f = osolver.uniform_state(P)
    steps, t0 = 0, time.perf_counter()
    while True:
        f = osolver.rk3_step(f, P)
        steps += 1
        el = time.perf_counter() - t0
        if el > budget_s or steps >= 200:
            break
    units = units_per_step([d])
    return {"value": units * steps / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} SSP-RK3 steps of one {d['n_cells']}-cell x {units // d['n_cells']}-momentum instance "
                      f"({el:.1f} s, numpy FP64, one thread)"}


def bench_config(args, ds, world, flush_needed, persistent=False):
    d = ds[0]
    units = units_per_step(ds)
    return {"workload": args.workload, "instances": len(ds), "n_cells": sum(x["n_cells"] for x in ds),
            "n_momenta": 2 * d["Q_R"] * d["Q_2"] * n_third(d), "precision": d["precision"],
            "updates_per_step": units,
            "l2": "flushed by a 256 MB write before every timed step" if flush_needed else "inputs larger than L2",
            "launch": ("one persistent step-kernel launch per timed step" if persistent
                       else "one-step CUDA graph per timed step"),
            "parallelism": f"{world} independent replicas"}


def needs_flush(ds):
    tsize = 4 if ds[0]["precision"] == "fp32" else 8
    return 3 * units_per_step(ds) * tsize < 2 * (129 << 20)


def run_reference(args):
    world, rank, _ = dist_setup() if int(os.environ.get("WORLD_SIZE", "1")) > 1 else (1, 0, 0)
    if rank != 0:
        return 0
    from oracle import solver as osolver

    ds = workload(args.workload)
    d = ds[0]
    P = oracle_problem(d)
    f = osolver.uniform_state(P)
    n_warm = min(args.warmup, 3)  # the oracle has nothing to warm up beyond its first steps
    for _ in range(n_warm):
        f = osolver.rk3_step(f, P)
    # each timed step is the whole instance; the timed sample stops after REF_BUDGET_S seconds so
    # that long runs end within a few minutes (the rate, steps and warm-up reported are those done)
    t0 = time.perf_counter()
    done = 0
    while done < args.steps:
        f = osolver.rk3_step(f, P)
        done += 1
        if time.perf_counter() - t0 > REF_BUDGET_S:
            break
    el = time.perf_counter() - t0
    units = units_per_step([d])
    val = units * done / el
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": done,
            "warmup": n_warm, "ms_per_step": 1e3 * el / done, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": bench_config(args, ds, args.gpus, needs_flush(ds)),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{done} of {args.steps} requested SSP-RK3 steps of the full instance "
                                       f"({el:.1f} s; the sample stops after {REF_BUDGET_S:.0f} s), numpy FP64, "
                                       "one thread"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch

    from paper_2403_15051_gb300 import build as fbuild
    from paper_2403_15051_gb300 import fdlb

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    fbuild.build()
    ds = workload(args.workload)
    t_create = time.perf_counter()
    S = fdlb.Solver(ds)
    t_create = time.perf_counter() - t_create
    if args.tiling:
        # a pinned tiling instead of the tuner's choice (profiling: a profiler's serialisation of the
        # launches would steer the tuner's timings)
        parts = args.tiling.split(",")
        cells, threads, form = parts[:3]
        S.set_autotune(0)
        S.set_tiling(int(cells), 0, int(threads))
        S.closure_form(1 if form == "batch" else 0)
        if len(parts) > 3:
            S.stage_min_blocks(int(parts[3]))
    persistent = S.set_persistent_step(None)  # the library's default scheduling
    S.set_graph_steps(1)
    stream = torch.cuda.ExternalStream(S.stream_handle())
    units = units_per_step(ds)
    tsize = 4 if ds[0]["precision"] == "fp32" else 8
    state_bytes = units * tsize
    flush_needed = needs_flush(ds)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda") if flush_needed else None

    def l2_flush(k):
        if flush_needed:
            with torch.cuda.stream(stream):
                flush.fill_(float(k % 7))

    if args.profile:
        # lean run for launch lists under a profiler: warm-up and K steps, nothing else; the K steps
        # inside the NVTX range "fdlb_timed" (a profiler can capture from them alone, past the
        # tuner's candidate launches)
        for k in range(args.warmup):
            l2_flush(k)
            S.step(1)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("fdlb_timed")
        for k in range(args.warmup, args.warmup + args.steps):
            l2_flush(k)
            S.step(1)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile_run": args.workload, "steps": args.steps, "warmup": args.warmup}))
        S.close()
        return 0

    # warm-up (also brings the clocks up before the sampler window)
    for k in range(args.warmup):
        l2_flush(k)
        S.step(1)
    torch.cuda.synchronize()
    tiling = S.tiling()  # after the first step: the autotuned tiling of a batch
    # the FP32 FMA rate the chip sustains now: the denominator of the arithmetic roofline
    probe_sampler = ClockSampler(torch.cuda.current_device())
    probe_sampler.start()
    time.sleep(0.3)
    fma_tflops, fma_ms = fdlb.fp32_fma_peak(S.stream_handle(), repeats=20)
    probe_clocks = probe_sampler.stop()
    t_end = time.perf_counter() + 0.6
    k = 0
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    while time.perf_counter() < t_end:
        l2_flush(k)
        S.step(1)
        k += 1
        if k % 50 == 0:
            torch.cuda.synchronize()
    torch.cuda.synchronize()
    barrier(world)

    # ---- timed region: exactly K steps
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches = 0
    for k in range(args.steps):
        l2_flush(k)
        evs[k][0].record(stream)
        S.step(1)
        evs[k][1].record(stream)
        launches += S.launch_count()
    torch.cuda.synchronize()
    barrier(world)
    ms = sum(a.elapsed_time(b) for a, b in evs)
    ms_max = max_over_ranks(ms, world)
    value = job_rate(units, args.steps, world, ms_max)

    # ---- kernel timing over K more steps (events around every launch): the persistent step
    # kernel where it is in use, else the closure and fused-stage kernels
    S.set_kernel_timing(True)
    S.kernel_times()
    S.step_kernel_times()
    for k in range(args.steps):
        l2_flush(k)
        S.step(1)
    stream_ms, n_stream, closure_ms, n_closure = S.kernel_times()
    step_ms, n_step_launch, n_step_steps = S.step_kernel_times()
    S.set_kernel_timing(False)
    clocks = sampler.stop()

    hot_value = None
    if flush_needed:
        # hot-L2 rate (steps back to back, no flush) for context
        torch.cuda.synchronize()
        S.set_graph_steps(20)
        S.step(20)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        S.step(200)
        e1.record(stream)
        torch.cuda.synchronize()
        hot_value = units * 200 / (e0.elapsed_time(e1) * 1e-3)
        S.set_graph_steps(1)

    # ---- end to end through the C ABI with host buffers: every step, H2D of the whole state from
    # pinned memory (one copy, the raw sums recomputed), one step, D2H of every cell's moments into
    # pinned memory.  (1) one handle, the three in sequence; (2) the headline: the batch as G
    # handles on G streams, the copies of one overlapping the steps of the others (the copy engines
    # run beside the SMs)
    e2e_steps = max(3, min(args.steps, 100))

    def e2e_run(handles, steps):
        hs = [torch.empty(H.state_bytes(), dtype=torch.uint8, pin_memory=True) for H in handles]
        hm = [torch.empty((sum(H.shape(q)[0] for q in range(H.n_instances)), fdlb.NMOM), dtype=torch.float64,
                          pin_memory=True).numpy() for H in handles]
        for H, h in zip(handles, hs):
            H.get_state_raw(h.data_ptr(), -1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d2h = 0
        # round robin: as soon as a handle's moments of step k are read, its copy and step k + 1
        # are issued, so they run while the other handles finish step k
        for H, h in zip(handles, hs):
            H.set_state_raw(h.data_ptr(), -1)
            H.step(1)
        for k in range(steps):
            for H, h, m in zip(handles, hs, hm):
                d2h += H.moments_all(out=m).nbytes
                if k + 1 < steps:
                    H.set_state_raw(h.data_ptr(), -1)
                    H.step(1)
        el = max_over_ranks(time.perf_counter() - t0, world)
        return {"value": units * steps * world / el, "unit": UNIT,
                "h2d_bytes_per_step": sum(H.state_bytes() for H in handles), "d2h_bytes_per_step": d2h // steps}

    e2e_seq = e2e_run([S], e2e_steps)
    G = args.e2e_handles if len(ds) >= 2 * args.e2e_handles else 1
    if G > 1:
        order = sorted(range(len(ds)), key=lambda q: -ds[q]["n_cells"])
        streams = [torch.cuda.Stream() for _ in range(G)]
        handles = [fdlb.Solver([ds[q] for q in order[g::G]], stream=streams[g].cuda_stream) for g in range(G)]
        for H in handles:  # tuning and the one-step graph before the timed region
            H.set_graph_steps(1)
            H.step(2)
        torch.cuda.synchronize()
        e2e = e2e_run(handles, e2e_steps)
        e2e["pipeline"] = ("%d handles on %d streams (instances dealt by size), per step each copies its state in, "
                           "steps once and reads its moments out, a handle's next step issued as soon as its "
                           "moments are read; one handle in sequence: %.4g" % (G, G, e2e_seq["value"]))
        for H in handles:
            H.close()
    else:
        e2e = e2e_seq

    # ---- roofline of the dominant kernel: the persistent step kernel (one launch per timed step:
    # three stages, each with its closure) or else the fused-stage kernel (one stage per launch).
    # Two views of the same event-timed launch: arithmetic (algorithmic flops against the measured
    # FP32 FMA rate) and HBM (8/3 population passes per stage against the measured copy
    # bandwidth); the bound is the view with the larger fraction.
    hbm_peak, peak_kind = measured_peaks()
    d0 = ds[0]
    nR, n2, n3 = 2 * d0["Q_R"], d0["Q_2"], n_third(d0)
    fpu = alg_flops_per_update(d0["geometry"], nR, n2, n3)
    if persistent and n_step_launch:
        kernel = "step_kernel"
        stages_per_launch = 3.0 * n_step_steps / n_step_launch
        avg_ms = step_ms / n_step_launch
    else:
        kernel = "stream_kernel"
        stages_per_launch = 1.0
        avg_ms = stream_ms / max(n_stream, 1)
    alg_flops = fpu * units * stages_per_launch
    alu_achieved = alg_flops / (avg_ms * 1e-3) / 1e12
    alg_bytes = 8.0 / 3.0 * state_bytes * stages_per_launch
    hv = hbm_view(alg_bytes, avg_ms, hbm_peak, peak_kind)
    alu = {"achieved": alu_achieved, "peak": fma_tflops, "unit": "TFLOP/s", "frac": alu_achieved / fma_tflops,
           "peak_source": "measured: FP32 FMA probe kernel (fdlb_fp32_fma_peak), best of 20 launches of "
                          "%.2f ms at a median SM clock of %s MHz" % (fma_ms, (probe_clocks or {}).get("sm_mhz")),
           "alg_flops_per_update": fpu, "alg_flops_per_launch": alg_flops}
    bound = "alu" if alu["frac"] >= hv["frac"] else "hbm"
    top = alu if bound == "alu" else hv
    traffic = recorded_traffic(args.workload, kernel)
    roofline = {"bound": bound, "achieved": top["achieved"], "peak": top["peak"], "unit": top["unit"],
                "frac": top["frac"], "traffic": traffic, "kernel": kernel, "stages_per_launch": stages_per_launch,
                "avg_launch_ms": avg_ms, "alu_view": alu, "hbm_view": hv}
    if not persistent:
        cl_avg = closure_ms / max(n_closure, 1)
        roofline["closure_avg_launch_ms"] = cl_avg
        roofline["kernel_time_share"] = {"stream_kernel": stream_ms / (stream_ms + closure_ms),
                                         "closure_kernel": closure_ms / (stream_ms + closure_ms)}

    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(ds)
    tts = None
    if rank == 0 and world == 1 and not args.no_tts:
        S.close()
        # the compact form of the warm-start comparison (bench.py --time-to-steady runs the stated
        # counts): 256 training steady states, 32 held-out instances, the plain FP64 arm on 8
        tts = time_to_steady(256, 32, 8, epochs=200, ref_tol=1e-10, ref_steps=150_000)
    if rank == 0:
        cfg = bench_config(args, ds, world, flush_needed, persistent)
        cfg["tiling"] = tiling
        cfg["create_seconds"] = t_create
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if tsize == 4 else "f64", "data": "synthetic",
                "config": cfg, "roofline": roofline, "cpu_baseline": base, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks, "fma_probe_clocks": probe_clocks}
        if hot_value is not None:
            line["hot_l2_value"] = hot_value
        if tts is not None:
            line["time_to_steady"] = tts
        print(json.dumps(line))
    S.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def time_to_steady(n_train, n_eval, n_plain, cells=64, q=4, tol=1e-8, min_kn=0.01, max_steps=150_000, epochs=300,
                   ref_tol=1e-11, ref_steps=300_000, check_every=200, stall_checks=50):
    """Time to steady state (moment residual <= tol) on held-out sweep instances (the batched-sweep
    parameter distribution at a reduced grid: `cells` cells, Q = q on every axis):
    (A) the plain form - FP64, one instance at a time, uniform start - on a fixed seeded subset of
        n_plain held-out instances;
    (B) the batched form - all n_eval held-out instances in one FP32 handle, warm-started by the
        network trained (with the library's kernels) on the steady states of n_train other sweep
        instances, run to the tolerance and then polished in FP64 by the library
        (fdlb_run_to_steady_mixed) to reach the FP64 level of accuracy;
    plus, for what they show, (C) the batched FP32 form alone and (D) the batched FP32 form from the
    uniform start (the network's gain).  Accuracy: the largest moment error of each arm's steady
    state against an FP64 reference run to ref_tol, on the n_plain subset.  Instances whose FP64
    residual never reaches tol (a small self-sustained oscillation) are left out and counted.  Every
    run but the references uses the library's stall rule (an instance whose residual has not halved
    its lowest value for stall_checks checks stops stepping, unconverged), so that an instance that
    settles on such an oscillation does not hold a batch to max_steps; training data are the
    instances with finite profiles."""
    import torch

    from paper_2403_15051_gb300 import fdlb
    from paper_2403_15051_gb300 import warmstart as wsm

    def instances(n, seed):
        ds = wl.batch_instances(lambda kn, e, r: accept_kn(kn, e) and kn >= min_kn, n=n, seed=seed, n_lo=cells,
                                n_hi=cells)
        for d in ds:
            d.update(Q_R=q, Q_2=q, Q_3=q)
        return ds

    P = 256
    ce = check_every
    t0 = time.perf_counter()
    train_ds = instances(n_train, 1)
    raw, tg, st_train, res_train, rc_data = wsm.steady_states(train_ds, n_points=P, tol=tol, max_steps=max_steps,
                                                              stall_checks=stall_checks)
    finite = np.isfinite(res_train) & np.all(np.isfinite(tg), axis=(1, 2))
    raw, tg = raw[finite], tg[finite]
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    net, losses = wsm.train(raw, tg, epochs=epochs, batch=32, lr=2e-3)
    t_train = time.perf_counter() - t0
    eval_all = instances(n_eval, 2)

    def moment_err(ma, mb, n0):
        return {"n/n0": float(np.max(np.abs(ma["n"] - mb["n"]))) / n0,
                "u2": float(np.max(np.abs(ma["u2"] - mb["u2"]))),
                "T": float(np.max(np.abs(ma["T"] - mb["T"]))),
                "qR/n0": float(np.max(np.abs(ma["q1"] - mb["q1"]))) / n0}

    def worst(errs):
        out = {k: 0.0 for k in ("n/n0", "u2", "T", "qR/n0")}
        for e in errs:
            out = {k: max(out[k], e[k]) for k in out}
        return out

    # (R) which held-out instances have a steady state: FP64, batched, to tol (instances that never
    # get there even in FP64 settle on a small self-sustained oscillation; they are left out and
    # counted); then FP64 references to ref_tol of the fixed subset the plain arm runs (the first
    # n_plain kept, in seeded order), on which every arm's accuracy is measured
    t0 = time.perf_counter()
    R = fdlb.Solver([dict(d, precision="fp64") for d in eval_all])
    R.set_stall_checks(stall_checks)
    _, _, res_tol = R.run_to_steady(tol=tol, max_steps=max_steps, check_every=ce)
    R.close()
    keep = [k for k in range(len(eval_all)) if float(res_tol[k]) <= tol]
    plain_idx = keep[:n_plain]
    R = fdlb.Solver([dict(eval_all[k], precision="fp64") for k in plain_idx])
    _, _, res_ref = R.run_to_steady(tol=ref_tol, max_steps=ref_steps, check_every=ce)
    ref_m = {k: R.moments(j) for j, k in enumerate(plain_idx)}
    n0s = {k: R.info(j)["n0"] for j, k in enumerate(plain_idx)}
    R.close()
    t_ref = time.perf_counter() - t0
    eval_ds = [eval_all[k] for k in keep]
    # (A) plain FP64, one instance after another, uniform start
    plain_steps, plain_err = [], []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in plain_idx:
        S = fdlb.Solver(dict(eval_all[k], precision="fp64"))
        S.set_stall_checks(stall_checks)
        _, st, res = S.run_to_steady(tol=tol, max_steps=max_steps, check_every=ce)
        plain_steps.append(int(st[0]))
        plain_err.append(moment_err(S.moments(), ref_m[k], n0s[k]))
        S.close()
    t_plain = time.perf_counter() - t0

    def batched(warm, polish):
        t0 = time.perf_counter()
        B = fdlb.Solver([dict(d, precision="fp32") for d in eval_ds])
        B.set_stall_checks(stall_checks)
        if warm:
            for j, d in enumerate(eval_ds):
                net.warm_start(B, j, wsm.raw_parameters(d))
        if polish:
            rc, s32, s64, res = B.run_to_steady_mixed(tol=tol, max_steps=max_steps, check_every=ce)
        else:
            rc, s32, res = B.run_to_steady(tol=tol, max_steps=max_steps, check_every=ce)
            s64 = np.zeros_like(s32)
        t = time.perf_counter() - t0
        errs = [moment_err(B.moments(j), ref_m[k], n0s[k]) for j, k in enumerate(keep) if k in plain_idx]
        B.close()
        return {"seconds": t, "seconds_per_instance": t / len(eval_ds), "instances": len(eval_ds),
                "steps_fp32": [int(x) for x in s32], "steps_fp64": [int(x) for x in s64],
                "converged": int(sum(float(r) <= tol for r in res)),
                "moment_error_vs_reference_on_plain_subset": worst(errs)}

    arm_b = batched(True, True)
    arm_c = batched(True, False)
    arm_d = batched(False, False)
    per_plain = t_plain / max(len(plain_idx), 1)
    return {"metric": "time to steady state (moment residual <= %g)" % tol, "unit": "s", "higher_is_better": False,
            "grid": {"cells": cells, "momenta": 2 * q ** 3}, "residual_check_every": ce, "max_steps": max_steps,
            "stall_checks": stall_checks,
            "held_out": len(eval_all), "excluded_nonconvergent_fp64": len(eval_all) - len(keep),
            "reference": {"precision": "fp64", "tol": ref_tol, "max_steps": ref_steps, "seconds": t_ref,
                          "instances": len(plain_idx), "residuals": [float(r) for r in res_ref]},
            "plain_fp64_sequential": {"instances": len(plain_idx), "seconds": t_plain, "seconds_per_instance": per_plain,
                                      "steps": plain_steps, "moment_error_vs_reference": worst(plain_err)},
            "batched_fp32_warm_start_fp64_polish": arm_b,
            "batched_fp32_warm_start": arm_c,
            "batched_fp32_uniform_start": arm_d,
            "speedup_per_instance_same_accuracy": per_plain / arm_b["seconds_per_instance"],
            "training": {"instances": int(len(raw)), "generated": len(train_ds), "data_seconds": t_data, "train_seconds": t_train,
                         "epochs": epochs, "first_loss": losses[0], "final_loss": losses[-1], "data_status": rc_data,
                         "data_steps_max": int(np.max(st_train))}}


def run_time_to_steady(args):
    """The learned-warm-start configuration at its stated counts (4096 training steady states, 256
    held-out instances; the plain FP64 arm on a fixed subset of 16) on the reduced grid."""
    import torch

    from paper_2403_15051_gb300 import build as fbuild

    fbuild.build()
    torch.cuda.set_device(0)
    out = time_to_steady(args.tts_train, args.tts_eval, args.tts_plain, cells=args.tts_cells, q=args.tts_q,
                         tol=args.tts_tol, min_kn=args.tts_min_kn, max_steps=args.tts_max_steps,
                         epochs=args.tts_epochs, ref_tol=args.tts_ref_tol, ref_steps=args.tts_ref_steps)
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="batch_512",
                    choices=["fourier_cyl_1024", "couette_cyl_64", "fourier_sph_2048", "batch_512", "batch_64",
                             "couette_cyl_reduced_q20"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tts", action="store_true", help="leave out the compact time-to-steady comparison")
    ap.add_argument("--e2e-handles", type=int, default=4,
                    help="handles (one stream each) the end-to-end pipeline deals a batch's instances over")
    ap.add_argument("--profile", action="store_true", help="warm-up + K steps only (for ncu launch lists)")
    ap.add_argument("--tiling", default="",
                    help="CELLS,THREADS,chain|batch[,MIN_BLOCKS]: a pinned tiling (and stage register bound), tuner off")
    ap.add_argument("--time-to-steady", action="store_true",
                    help="time-to-steady comparison: plain FP64 sequential vs batched warm-started FP32")
    ap.add_argument("--tts-train", type=int, default=4096)
    ap.add_argument("--tts-eval", type=int, default=256)
    ap.add_argument("--tts-plain", type=int, default=16)
    ap.add_argument("--tts-cells", type=int, default=64)
    ap.add_argument("--tts-q", type=int, default=4)
    ap.add_argument("--tts-tol", type=float, default=1e-8)
    ap.add_argument("--tts-min-kn", type=float, default=0.01)
    ap.add_argument("--tts-max-steps", type=int, default=150_000)
    ap.add_argument("--tts-epochs", type=int, default=300)
    ap.add_argument("--tts-ref-tol", type=float, default=1e-11)
    ap.add_argument("--tts-ref-steps", type=int, default=300_000)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.time_to_steady:
        return run_time_to_steady(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
