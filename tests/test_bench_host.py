"""Host-side paths of bench.py without a GPU: the multi-rank helpers over gloo (world size 2,
127.0.0.1) that give the barrier and the max-over-ranks timing, and the reference arm (the
FP64 oracle timed on the host cores), whose JSON line the driver reads."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    w, r, loc = bench.dist_init()
    assert (w, r, loc) == (world, rank, rank)
    assert dist.get_backend() == "gloo"
    bench.barrier(w)
    # every rank reports its own time; the line uses the slowest
    m = bench.max_over_ranks(w, 1.5 + rank)
    with open(f"{out_path}.{rank}", "w") as f:
        f.write(repr(m))
    dist.destroy_process_group()


def test_max_over_ranks_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    out = str(tmp_path / "max")
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    for r in range(2):
        assert float(open(f"{out}.{r}").read()) == 2.5


def test_reference_arm_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    res = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "snapshot", "--steps", "2",
                          "--warmup", "3"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    line = json.loads(res.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 3
    assert line["value"] > 0 and line["unit"] == "pair-evals/s" and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"].startswith("snapshot")


def test_reference_arm_other_ranks_print_nothing(capsys):
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    args = argparse.Namespace(workload="snapshot", steps=1, warmup=3)
    bench.run_reference(args, world=2, rank=1)
    assert capsys.readouterr().out == ""


def test_clock_sampler_keeps_the_timed_region():
    """The clock summary takes the samples inside the timed region (time-stamped nvidia-smi
    lines), falls back to those within 0.25 s of a region shorter than the sampling period, and
    reports the throttle reasons of the samples it kept."""
    import time as _time

    sys.path.insert(0, ROOT)
    import bench

    clk = bench.ClockSampler(0)

    def line(t, mhz, thermal="Not Active"):
        stamp = _time.strftime("%Y/%m/%d %H:%M:%S", _time.localtime(int(t))) + ".%03d" % int(round((t % 1) * 1000))
        return f"{stamp}, 0, {mhz}, 2070, 900.0, 0x0, Not Active, {thermal}, Not Active, Not Active"

    base = float(int(_time.time())) + 0.5
    clk.lines = [line(base - 1.0, 345, "Active"), line(base + 0.10, 2070), line(base + 0.15, 2055),
                 line(base + 0.20, 2070), line(base + 2.0, 600)]
    clk.mark(base + 0.09, base + 0.21)
    s = clk.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["reasons"] == [] and s["window"] == "timed region"
    clk.mark(base + 0.30, base + 0.31)  # shorter than the period: the neighbours within 0.25 s
    s = clk.summary()
    assert s["samples"] == 3 and s["window"].startswith("within")
    clk.window = None
    s = clk.summary()
    assert s["samples"] == 5 and "hw_thermal_slowdown" in s["reasons"] and s["window"] == "whole measurement"
