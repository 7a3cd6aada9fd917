"""Host logic of bench.py.  The replica bookkeeping on two ranks of the gloo backend (host
cores): the timing is the maximum over the ranks, the whole-job rate counts every rank's work,
and the comparison arm runs on rank 0 alone while the other ranks exit without work.  Also the
JSON line's helpers: the HBM view, the clock summary, the flop and unit counts."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank)
    ms = bench.max_over_ranks(10.0 + rank, w)
    rate = bench.job_rate(1000, 5, w, ms)
    bench.barrier(w)
    buf = io.StringIO()
    args = bench.argparse.Namespace(workload="couette_cyl_64", steps=2, warmup=3, gpus=world, no_cpu_baseline=True)
    with redirect_stdout(buf):
        rc = bench.run_reference(args)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
        json.dump({"ms": ms, "rate": rate, "rc": rc, "stdout": buf.getvalue()}, fh)
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    r0 = json.load(open(tmp_path / "rank0.json"))
    r1 = json.load(open(tmp_path / "rank1.json"))
    assert r0["ms"] == r1["ms"] == 11.0  # the slowest rank
    assert r0["rate"] == pytest.approx(1000 * 5 * 2 / 11.0e-3)
    assert r0["rc"] == r1["rc"] == 0
    assert r1["stdout"] == ""  # the comparison arm runs on rank 0 only
    line = json.loads(r0["stdout"].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    # the rest of the one-line contract of the comparison arm
    assert line["metric"] == "node-velocity updates/s" and line["unit"] == "updates/s"
    assert line["higher_is_better"] is True and line["vs_baseline"] is None and line["dtype"] == "f64"
    assert line["steps"] == 2 and line["warmup"] == 3 and line["ms_per_step"] > 0
    assert line["config"]["workload"] == "couette_cyl_64"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_hbm_view_against_measured_and_nominal_bandwidth():
    """The HBM view of a launch: algorithmic bytes over its duration, as a fraction of the measured
    copy bandwidth and of the nominal HBM3e bandwidth."""
    sys.path.insert(0, ROOT)
    import bench

    v = bench.hbm_view(6.0e6, 0.01, 6000.0, "measured")  # 6 MB in 10 us = 600 GB/s
    assert v["achieved"] == pytest.approx(600.0) and v["unit"] == "GB/s"
    assert v["frac"] == pytest.approx(0.1) and v["peak_source"] == "measured"
    assert v["frac_of_nominal"] == pytest.approx(600.0 / bench.HBM_NOMINAL_GBS)


def test_clock_samples_summary():
    """The clock record of the JSON line: median SM clock, maximum clock and every throttle reason
    seen active in the nvidia-smi CSV samples; malformed lines are skipped."""
    sys.path.insert(0, ROOT)
    import bench

    lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 2040, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 1980, 2070, 1390.2, 0x8, Active, Not Active, Not Active, Active",
             "garbage", "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 1000, [N/A], 1.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    out = bench.ClockSampler.summarise(lines)
    assert out == {"sm_mhz": 2040.0, "sm_max_mhz": 2070.0, "reasons": ["hw_slowdown", "sw_power_cap"], "samples": 3}
    assert bench.ClockSampler.summarise([])["samples"] == 0


def test_algorithmic_flops_and_units_of_the_benchmark_workloads():
    """The roofline's per-update flop counts (221 on the 16 x 8 x 8 cylinder, 272 on the
    24 x 12 x 12 sphere) and the updates per step of the two single-instance workloads."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2403_15051_gb300 import workloads as wl

    assert bench.alg_flops_per_update(wl.CYL, 16, 8, 8) == 221
    assert bench.alg_flops_per_update(wl.SPH, 24, 12, 12) == 272
    assert bench.units_per_step([wl.fourier_cyl_1024()]) == 1024 * 1024
    assert bench.units_per_step(bench.workload("fourier_sph_2048")) == 2048 * 3456


def test_recorded_traffic_follows_the_kernel_code_not_its_comments(tmp_path, monkeypatch):
    """The roofline's traffic comes from the committed ncu record only while the timed kernels' code
    is the code it was taken on: the source hash ignores comments and spacing and changes with any
    change of code."""
    sys.path.insert(0, ROOT)
    import bench

    src = tmp_path / "k.cuh"
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "KERNEL_SOURCES", ["k.cuh"])
    src.write_text("// the stage\n__global__ void k(float* a) { a[0] = 1.f; }  /* one store */\n")
    h0 = bench.kernel_source_hash()
    rec = {"batch_512:stream_kernel": {"source_hash": h0, "dram_bytes_per_launch": 6.0e9}}
    (tmp_path / "profiles" / "roofline_traffic.json").write_text(json.dumps(rec))
    assert bench.recorded_traffic("batch_512", "stream_kernel") == 6.0e9
    assert bench.recorded_traffic("batch_64", "stream_kernel") is None
    src.write_text("// the fused stage\n__global__ void k(float* a)\n{\n    a[0] = 1.f;  // a store\n}\n")
    assert bench.kernel_source_hash() == h0
    assert bench.recorded_traffic("batch_512", "stream_kernel") == 6.0e9
    src.write_text("__global__ void k(float* a) { a[0] = 2.f; }\n")
    assert bench.kernel_source_hash() != h0
    assert bench.recorded_traffic("batch_512", "stream_kernel") is None
