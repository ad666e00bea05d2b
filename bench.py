#!/usr/bin/env python3
"""Benchmark of the RBE k-space hot path on GB300: one JSON line on rank 0.

A step is one RBE k-space evaluation of the whole workload through the C ABI:
sample P frequencies, reduce rho(k) over all N particles, gather the N forces, and
reduce the energy and the 3x3 virial (``rbe_kspace_forces_virial``).  The metric is
N*P pair evaluations per second (one evaluation = both passes over a (particle,
frequency) pair).  Inputs sit in HBM before the timed region; the L2 is flushed
(a 256 MB write) between timed steps, outside the per-step CUDA events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload slab|uniform1e6|...]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

Under torchrun each rank runs its own replica of the workload (independent systems,
no collective on the data path); rank 0 prints the max-over-ranks timing.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2110_14362_gb300 import inputs  # noqa: E402

METRIC = "RBE k-space N*P pair evaluations/s (FP32-phase at 1e-5; FP64 alongside)"
UNIT = "pair-evals/s"
SEED = 12345

# MUFU sine/cosine operations per pair in each pass of the two-pass schedule: the rho pass
# takes sin and cos of every phase; the force pass one sine of the phase shifted by arg rho.
MUFU_OPS_PER_PAIR = {"k_rho": 2.0, "k_force": 1.0}

# DRAM bytes per launch of the dominant kernel measured by ncu on this workload
# (dram__bytes_read.sum + dram__bytes_write.sum), or None when not captured for the
# current kernel version.  Source: profiles/ summaries.
NCU_TRAFFIC = {("k_rho", "uniform-N4000000-P2000"): 128415488 + 3578368}

# launches of the library's own kernels per evaluation at a fixed box: the sampler, the rho
# pass, the rho reduction and the force pass
GPU_LAUNCHES_PER_STEP = 4


def workload(name: str):
    if name == "slab":
        return inputs.slab()
    if name == "snapshot":
        return inputs.small_snapshot()
    if name.startswith("uniform"):
        # uniform<N>[-P<P>], e.g. uniform1e6-P500
        spec = name[len("uniform"):]
        P = 100
        if "-P" in spec:
            spec, p = spec.split("-P")
            P = int(p)
        return inputs.uniform_density(int(float(spec)), P=P)
    if name == "water":
        return inputs.water()
    raise SystemExit(f"unknown workload {name}")


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x: float) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms while running, each sample
    time-stamped, so that the summary can keep the samples of the timed region only."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.window = None  # (t0, t1) in time.time() seconds: the timed region

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        return self

    def mark(self, t0: float, t1: float):
        """The timed region, as time.time() values."""
        self.window = (t0, t1)

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    @staticmethod
    def _epoch(stamp: str):
        # nvidia-smi writes local time as "YYYY/MM/DD HH:MM:SS.mmm"
        try:
            base, _, frac = stamp.partition(".")
            return time.mktime(time.strptime(base, "%Y/%m/%d %H:%M:%S")) + (float("0." + frac) if frac else 0.0)
        except ValueError:
            return None

    def summary(self):
        rows = []
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 10:
                continue
            try:
                rows.append((self._epoch(parts[0]), float(parts[2]), float(parts[3]), parts[6:10]))
            except ValueError:
                continue
        label = "whole measurement"
        if self.window is not None:
            # the samples inside the timed region (the sampler's clock and time.time() agree to
            # well under the 50 ms period); a region shorter than the period falls back to the
            # samples within 0.25 s of it
            t0, t1 = self.window
            for pad, name in ((0.05, "timed region"), (0.25, "within 0.25 s of the timed region")):
                inside = [r for r in rows if r[0] is not None and t0 - pad <= r[0] <= t1 + pad]
                if inside:
                    rows, label = inside, name
                    break
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for name, flag in zip(names, r[3]):
                if flag.lower() in ("active", "1"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median([r[1] for r in rows]), "sm_max_mhz": max(r[2] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows), "window": label}


ACCUM_NAMES = {0: "fp64 per pair", 1: "compensated fp32 (Kahan) per tile, float-float across tiles",
               2: "plain fp32 per tile, float-float across tiles"}


def measure_kspace(rbe, s, args, world, rank, local, precision, accum, with_fp64=True, with_e2e=True):
    """One k-space workload through rbe_kspace_forces_virial: device-timed pair evaluations/s
    (CUDA events per step on the launching stream, L2 flushed between steps outside the events),
    per-kernel times, the roofline of the dominant kernel, the end-to-end rate through the
    host-buffer call, the FP64 path on the same workload and the errors of the FP32-phase path
    against it on one shared batch."""
    import torch
    dev = torch.device("cuda", local)
    pos = torch.as_tensor(s.pos).to(dev).contiguous()
    q = torch.as_tensor(s.q).to(dev).contiguous()
    F = torch.empty((s.N, 3), dtype=torch.float64, device=dev)
    W = torch.empty(9, dtype=torch.float64, device=dev)
    E = torch.empty(2, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    seed = SEED + rank
    pairs = float(s.N) * s.P

    def timed_loop(ctx, steps, warmup, first_step):
        ctx.set_stream(stream.cuda_stream)
        for w in range(warmup):
            ctx.forces_virial(pos, q, first_step + w, F, W, E)
        ctx.sync()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0 = time.time()
        for k in range(steps):
            flush.fill_(float(k))
            evs[k][0].record(stream)
            ctx.forces_virial(pos, q, first_step + warmup + k, F, W, E)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        wall = time.perf_counter() - t0
        window = (e0, time.time())
        ctx.sync()
        return [a.elapsed_time(b) for a, b in evs], wall, window

    ctx = rbe.Context(s.box, s.alpha, s.P, seed, precision, accum)
    with ClockSampler(local) as clk:
        time.sleep(0.3)  # the sampler's first samples before the warm-up
        ms, wall, window = timed_loop(ctx, args.steps, args.warmup, 0)
        clk.mark(*window)
    clocks = clk.summary()
    dev_s_max = max_over_ranks(world, sum(ms) / 1e3)
    value = world * args.steps * pairs / dev_s_max

    # per-kernel durations (live, CUDA events recorded by the library on its stream)
    ctx.set_kernel_timing(True)
    kt = []
    for k in range(max(3, min(args.steps, 10))):
        flush.fill_(float(k))
        ctx.forces_virial(pos, q, 10_000 + k, F, W, E)
        kt.append(ctx.kernel_times())
    ctx.set_kernel_timing(False)
    kmean = np.mean(np.array(kt), axis=0)
    names = ["k_sample", "k_rho", "k_reduce", "k_force"]
    dom = int(np.argmax(kmean))
    out = {"value": value, "unit": UNIT, "ms_per_step": dev_s_max * 1e3 / args.steps, "wall_s_timed_region": wall,
           "clocks": clocks, "phases_per_s": 2.0 * value,
           "kernel_ms": {n: float(v) for n, v in zip(names, kmean)}}

    if precision == rbe.RBE_FP32_PHASE:
        peak = rbe.rbe_measure_pipe(0, 4096)
        dom_ms = float(kmean[dom])
        achieved = MUFU_OPS_PER_PAIR[names[dom]] * pairs / (dom_ms * 1e-3)
        out["roofline"] = {
            "bound": "alu", "pipe": "MUFU (sin/cos)", "kernel": names[dom], "achieved": achieved / 1e9,
            "peak": peak / 1e9, "unit": "Gop/s", "frac": achieved / peak,
            "peak_source": "of measured: MUFU sin.approx rate on this GPU (rbe_measure_pipe; 16/clk/SM x 152 SMs "
                           "x 2.07 GHz nominal)",
            "traffic": NCU_TRAFFIC.get((names[dom], s.name))}
        # the whole evaluation against the same peak, at the schedule's 3 MUFU operations per pair
        out["evaluation_mufu_frac"] = 3.0 * value / world / peak
        # and against the algorithmic minimum of one sine and one cosine per pair
        out["evaluation_mufu_frac_algorithmic_min"] = 2.0 * value / world / peak

    if with_fp64 and precision == rbe.RBE_FP32_PHASE:
        ctx64 = rbe.Context(s.box, s.alpha, s.P, seed, rbe.RBE_FP64)
        n64 = 2 if pairs > 1e9 else max(2, min(args.steps, 5))
        ms64, _, _ = timed_loop(ctx64, n64, 1 if pairs > 1e9 else 2, 50_000)
        other = {"precision": "fp64", "value": pairs / (sum(ms64) / len(ms64) / 1e3), "unit": UNIT,
                 "ms_per_step": sum(ms64) / len(ms64), "steps": n64}
        # accuracy of the timed FP32-phase path against the FP64 path on the same frequencies
        # (the same seed and step draw the same batch in both contexts)
        ctx64.forces_virial(pos, q, 60_000, F, W, E)
        ctx64.sync()
        F0, W0, E0 = F.cpu().numpy(), W.cpu().numpy().reshape(3, 3), E.cpu().numpy()
        ctx.forces_virial(pos, q, 60_000, F, W, E)
        ctx.sync()
        F1, W1, E1 = F.cpu().numpy(), W.cpu().numpy().reshape(3, 3), E.cpu().numpy()
        dW = np.abs(np.diag(W1) - np.diag(W0))
        other["fp32_phase_vs_fp64"] = {
            "force_rel_rms": float(np.sqrt(np.mean((F1 - F0) ** 2) / np.mean(F0 ** 2))),
            "virial_rel": float(np.linalg.norm(W1 - W0) / np.linalg.norm(W0)),
            "pressure_diag_rel": [float(x) for x in dW / np.abs(np.diag(W0))],
            "pressure_diag_err_over_max_diag": float(np.max(dW) / np.max(np.abs(np.diag(W0)))),
            "energy_rel": float(abs(E1[0] - E0[0]) / abs(E0[0])),
            "bar": "force relative RMS <= 1e-5"}
        out["fp32_phase_over_fp64"] = value / world / other["value"]
        out["fp64_same_workload"] = other
        ctx64.close()

    if with_e2e:
        # end to end through the public host-buffer call: pinned host inputs in, forces out
        pos_h = torch.empty((s.N, 3), dtype=torch.float64, pin_memory=True)
        q_h = torch.empty((s.N,), dtype=torch.float64, pin_memory=True)
        F_h = torch.empty((s.N, 3), dtype=torch.float64, pin_memory=True)
        pos_h.copy_(torch.as_tensor(s.pos))
        q_h.copy_(torch.as_tensor(s.q))
        pn, qn, Fn = pos_h.numpy(), q_h.numpy(), F_h.numpy()
        for w in range(2):
            rbe.rbe_kspace_forces_virial_host(ctx.h, pn, qn, 20_000 + w, Fn)
        barrier(world)
        t0 = time.perf_counter()
        for k in range(args.steps):
            rbe.rbe_kspace_forces_virial_host(ctx.h, pn, qn, 30_000 + k, Fn)
        e2e_s = max_over_ranks(world, time.perf_counter() - t0)
        out["e2e"] = {"value": world * args.steps * pairs / e2e_s, "unit": UNIT,
                      "h2d_bytes_per_step": int(pn.nbytes + qn.nbytes),
                      "d2h_bytes_per_step": int(Fn.nbytes + 11 * 8)}
    ctx.close()
    del pos, q, F, flush
    return out


def run_ours(args, world, rank, local):
    import torch
    import paper_2110_14362_gb300 as rbe

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    s = workload(args.workload)
    precision = rbe.RBE_FP32_PHASE if args.precision == "fp32" else rbe.RBE_FP64
    accum = {"comp32": rbe.RBE_RHO_COMP32, "fp32": rbe.RBE_RHO_FP32, "fp64": rbe.RBE_RHO_FP64}[args.rho_accum]
    head = measure_kspace(rbe, s, args, world, rank, local, precision, accum, with_fp64=not args.skip_fp64)

    extra = {}
    if not args.skip_slab and args.workload != "slab":
        # the semi-isotropic slab (300k charges, P = 200): Pxx, Pyy, Pzz of both paths
        extra["slab"] = dict(workload="slab-N300000-P200", rho_accum=ACCUM_NAMES[accum],
                             **measure_kspace(rbe, workload("slab"), args, world, rank, local, precision, accum))
    serving = None if args.skip_serving else run_serving(args, world, rank)
    npt1 = None if args.skip_serving else run_npt_single(rbe, [1000, 10000, 100000], 20)
    batched = None if args.skip_serving else run_batched(rbe)
    water = None if args.skip_serving else run_water_both(rbe)
    sweep = None if args.skip_sweep else run_sweep(rbe)

    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        cpu = cpu_baseline(s, budget_s=args.cpu_seconds)
        cpu_all = cpu_baseline_all_cores(s, budget_s=args.cpu_seconds / 3)

    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32-phase (int32 fixed-point phase, fp32 sincos) / f64 sums" if precision == rbe.RBE_FP32_PHASE
                 else "f64",
        "data": "synthetic (seeded NumPy; shapes of the paper's workloads)",
        "config": {"workload": s.name, "N": s.N, "P": s.P, "alpha": s.alpha, "box": [float(b) for b in s.box],
                   "precision": args.precision,
                   "rho_accum": ACCUM_NAMES[accum] if precision == rbe.RBE_FP32_PHASE else "fp64",
                   "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"replicas x{world} (independent systems, no collective)"},
        "phases_per_s": head["phases_per_s"],
        "kernel_ms": head["kernel_ms"],
        "wall_s_timed_region": head["wall_s_timed_region"],
        "gpu_launches": GPU_LAUNCHES_PER_STEP * args.steps,
        "e2e": head["e2e"],
        "roofline": head.get("roofline"),
        "evaluation_mufu_frac": head.get("evaluation_mufu_frac"),
        "evaluation_mufu_frac_algorithmic_min": head.get("evaluation_mufu_frac_algorithmic_min"),
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_all,
        "clocks": head["clocks"],
    }
    if "fp64_same_workload" in head:
        line["fp64_same_workload"] = head["fp64_same_workload"]
        line["fp32_phase_over_fp64"] = head["fp32_phase_over_fp64"]
    line.update(extra)
    if serving:
        line["serving"] = serving
    if batched:
        line["batched_kspace"] = batched
    if water:
        line["water_npt"] = water
    if sweep:
        line["sweep"] = sweep
    if npt1:
        line["npt_one_replica"] = {"system": "jittered-lattice +-1 charges at 0.1/A^3, P=100, rc=7, Langevin NPT",
                                   "launch": "direct, one stream", "by_N": npt1}
    if rank == 0:
        print(json.dumps(line), flush=True)


# Serving workload: Langevin NPT replicas with RBE k-space, erfc real space and LJ 12-6
# (300 K, 1 bar, dt = 1 fs, gamma = 10/ps, gamma_V = 2/ps, tau_P = 0.5 ps, beta_T = 4.5e-5/bar),
# charges screened by the relative permittivity of water (primitive electrolyte model),
# starting from jittered-lattice positions.
SERVE_ALPHA, SERVE_P, SERVE_RC, SERVE_EPS_R, SERVE_SKIN = 0.2, 100, 7.0, 78.5, 1.0
KB = 0.00831446261815324
BAR = 6.02214076e-5


def serve_params(rbe, box, barostat=1):
    """NPT parameters of the serving system; barostat 2 / 3 are the anisotropic and
    semi-isotropic rectangular cells with the same relaxation time and compressibility."""
    V0 = float(np.prod(box))
    prm = rbe.NptParams(dt=0.001, kT=KB * 300.0, P_ext=1.0 * BAR, gamma=10.0, gamma_V=2.0,
                        M_V=rbe.piston_mass(0.5, 4.5e-5 / BAR, V0), rc=SERVE_RC, qqr2e=1389.35457644382 / SERVE_EPS_R,
                        lj_sigma=2.0, lj_eps=0.5, max_disp=0.05, kspace=1, real=1, noise=1, barostat=barostat,
                        skin=SERVE_SKIN)
    if barostat >= 2:
        prm.M_cell = (type(prm.M_cell))(*rbe.piston_masses_rect(barostat, 0.5, 4.5e-5 / BAR, box))
    return prm


def serve(rbe, reqs, states, precision, max_slots, chunk, nsteps, use_graphs=True, open_loop=False,
          budget=32 << 30, deadline_s=600.0, batched=0):
    """Drive the C++ serving loop: submit every request at t = 0 (closed loop) or at its
    Poisson arrival time (open loop), poll until all are done.  batched: 0 replicas on their own
    chunks, 2 lockstep groups with the persistent batched k-space (tiles autotuned once).
    Returns the metrics."""
    srv = rbe.Server(SERVE_ALPHA, SERVE_P, precision, max_slots=max_slots, chunk_steps=chunk,
                     mem_budget=budget, use_graphs=use_graphs, batched=batched)
    try:
        t0 = time.perf_counter()
        nxt = 0
        order = sorted(range(len(reqs)), key=lambda i: reqs[i].arrival_s)
        done = 0
        while done < len(reqs):
            now = time.perf_counter() - t0
            while nxt < len(order) and (not open_loop or reqs[order[nxt]].arrival_s <= now):
                i = order[nxt]
                pos, mom, q, m, box = states[i]
                srv.submit(pos, mom, q, m, box, serve_params(rbe, box), 1000 + reqs[i].rid, nsteps)
                nxt += 1
            nq, na, done = srv.progress(wait=not open_loop or nxt == len(order))
            if open_loop and na == 0 and nq == 0 and nxt < len(order):
                time.sleep(max(0.0, reqs[order[nxt]].arrival_s - (time.perf_counter() - t0)))
            if time.perf_counter() - t0 > deadline_s:
                raise RuntimeError("serving loop exceeded its deadline")
        wall = time.perf_counter() - t0
        lat, steps, span = srv.stats()
    finally:
        srv.close()
    return {"requests": len(reqs), "replica_steps": int(steps), "wall_s": wall,
            "replica_steps_per_s": steps / wall,
            "pair_evals_per_s": sum(r.N for r in reqs) * SERVE_P * nsteps / wall,
            "chunk_latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3), "p99": float(np.percentile(lat, 99) * 1e3),
                                 "max": float(lat.max() * 1e3), "chunks": int(lat.size)}}


FLEX_TILT = (0.10, -0.08, 0.12)  # xy, xz, yz tilts of the flexible-cell workload, in units of the edge


def flex_replica(rbe, N, device):
    """The serving system in a sheared cell h = L (I + T) (tilts FLEX_TILT), the fully flexible
    cell with the rectangular barostat's masses on the diagonal and their geometric means off it,
    the serving system's neighbour-list skin; the cell starts at rest.  Returns the FlexReplica."""
    pos, mom, q, m, box = inputs.npt_replica(N, 3)
    L = float(box[0])
    h = np.diag(box).astype(np.float64)
    h[0, 1], h[0, 2], h[1, 2] = FLEX_TILT[0] * L, FLEX_TILT[1] * L, FLEX_TILT[2] * L
    Md = np.asarray(rbe.piston_masses_rect(2, 0.5, 4.5e-5 / BAR, box))
    prm = rbe.FlexParams(dt=0.001, kT=KB * 300.0, P_ext=1.0 * BAR, gamma=10.0, gamma_h=2.0, M=np.sqrt(np.outer(Md, Md)),
                         rc=SERVE_RC, qqr2e=1389.35457644382 / SERVE_EPS_R, lj_sigma=2.0, lj_eps=0.5, max_disp=0.05,
                         chi=2.0, kspace=1, real=1, noise=1, skin=SERVE_SKIN)
    return rbe.FlexReplica((pos / L) @ h.T, mom, q, m, h, prm, device)


def npt_single(rbe, N, precision, steps, warmup=3, barostat=1, sampler=0, ptilde=0, reuse=1):
    """ms per NPT step of one replica of N particles (the serving system), launched directly
    on one stream, timed with CUDA events after `warmup` steps.  barostat 4: the fully flexible
    cell (flex_replica)."""
    import torch
    pos, mom, q, m, box = inputs.npt_replica(N, 3)
    stream = torch.cuda.current_stream()
    with rbe.Context(box, SERVE_ALPHA, SERVE_P, 1003, precision, stream=stream.cuda_stream) as ctx:
        ctx.set_sampler(sampler)
        ctx.set_pressure_batch(ptilde)
        ctx.set_sample_reuse(reuse)
        dev = torch.device("cuda", torch.cuda.current_device())
        rep = flex_replica(rbe, N, dev) if barostat == 4 else rbe.NptReplica(pos, mom, q, m, box,
                                                                          serve_params(rbe, box, barostat), dev)
        rep.init(ctx, batch=0)
        rep.step(ctx, warmup)
        ctx.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rep.step(ctx, steps)
        e1.record(stream)
        ctx.sync()
        return e0.elapsed_time(e1) / steps


def run_npt_single(rbe, sizes, steps):
    out = {}
    for N in sizes:
        f32 = npt_single(rbe, N, rbe.RBE_FP32_PHASE, steps)
        f64 = npt_single(rbe, N, rbe.RBE_FP64, max(2, steps // 4))
        out[str(N)] = {"fp32_ms_per_step": f32, "fp64_ms_per_step": f64, "fp32_over_fp64": f64 / f32,
                       # the rectangular cells (per-axis virial and pistons), FP32-phase path
                       "fp32_aniso_ms_per_step": npt_single(rbe, N, rbe.RBE_FP32_PHASE, steps, barostat=2),
                       "fp32_semi_ms_per_step": npt_single(rbe, N, rbe.RBE_FP32_PHASE, steps, barostat=3),
                       # the fully flexible (sheared) cell: general-cell k-space and triclinic real space
                       "fp32_flex_ms_per_step": npt_single(rbe, N, rbe.RBE_FP32_PHASE, steps, barostat=4)}
    return out


WATER_MASS = (15.9994, 1.008, 1.008)


def run_water(rbe, steps=1000, warmup=20, alpha=None, barostat=1, dense_steps=10):
    """The plain-method rigid-water NPT run: 3000 molecules (O -0.8476, H +0.4238, O-H 1 A,
    H-O-H 109.47 deg, LJ O-O 3.166 A / 0.650 kJ/mol) at random orientations on a jittered lattice
    at 1 g/cm^3 (`inputs.water`), alpha = 0.25, rc = 10 A, P = 100, FP64, Langevin isotropic NPT at
    300 K and 1 bar, dt = 1 fs, a 0.05 A cap on the centres' peculiar displacement per step (the
    random orientations overlap at the start).  ms per step by CUDA events over `steps` steps after
    `warmup`; density, molecular pressure, temperature (6 degrees of freedom per molecule) and the
    largest bond error at the end; `dense_steps` steps after the first three timed on their own
    (the system still at 1 g/cm^3), with the density and temperature after them.  alpha (default: the configuration's 0.25) and barostat (0: fixed
    box) can be changed to study the run."""
    import torch
    s = inputs.water(3000)
    box = np.asarray(s.box, dtype=np.float64)
    n = len(s.q) // 3
    m = np.tile(WATER_MASS, n)
    rng = np.random.default_rng(7)
    mom = rng.standard_normal((3 * n, 3)) * np.sqrt(KB * 300.0 * 100.0 * m)[:, None]
    V0 = float(np.prod(box))
    prm = rbe.NptParams(dt=0.001, kT=KB * 300.0, P_ext=1.0 * BAR, gamma=10.0, gamma_V=2.0,
                        M_V=rbe.piston_mass(0.5, 4.5e-5 / BAR, V0), rc=10.0, qqr2e=1389.35457644382,
                        lj_sigma=3.166, lj_eps=0.650, max_disp=0.05, kspace=1, real=1, noise=1, barostat=barostat)
    stream = torch.cuda.current_stream()
    dev = torch.device("cuda", torch.cuda.current_device())
    a = s.alpha if alpha is None else alpha
    def density(L):
        return n * 18.01528 / (0.602214076 * float(np.prod(L)))

    def temperature(p):
        return float(np.sum(p ** 2 / m[:, None]) / 100.0 / (6 * n * KB))

    def timed(rep, ctx, k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rep.step(ctx, k)
        e1.record(stream)
        ctx.sync()
        return e0.elapsed_time(e1) / k

    with rbe.Context(box, a, s.P, 2024, rbe.RBE_FP64, stream=stream.cuda_stream) as ctx:
        rep = rbe.WaterReplica(np.asarray(s.pos), mom, np.asarray(s.q), m, box, prm, dev)
        rep.init(ctx, batch=0)
        rep.step(ctx, 3)
        ctx.sync()
        # the first steps, still at the starting density of 1 g/cm^3
        ms_dense = timed(rep, ctx, dense_steps)
        _, p_d, _, L_d, _ = rep.state()
        rep.step(ctx, max(0, warmup - 3 - dense_steps))
        ctx.sync()
        ms = timed(rep, ctx, steps)
        r, p, F, L, cell = rep.state()
    mol = r.reshape(-1, 3, 3)
    bond = float(np.abs(np.linalg.norm(mol[:, 1:] - mol[:, :1], axis=2) - 1.0).max())
    return {"molecules": n, "sites": 3 * n, "alpha": a, "P": s.P, "rc": 10.0, "precision": "fp64",
            "barostat": barostat, "steps": steps, "warmup": warmup, "ms_per_step": ms, "steps_per_s": 1e3 / ms,
            "T_K": temperature(p), "density_g_cm3": density(L), "P_ins_bar": float(cell[6]) / BAR,
            "site_pair_evals_per_s": 3 * n * s.P / (ms * 1e-3),
            "first_steps": {"steps": dense_steps, "ms_per_step": ms_dense, "density_g_cm3_after": density(L_d),
                            "T_K_after": temperature(p_d)},
            "max_bond_error_A": bond}


def run_water_both(rbe, steps=1000, warmup=20):
    """The water configuration's run at its alpha = 0.25 (the RBE force noise of P = 100 heats
    it and the cell expands: final T and density are reported beside the ms per step, and the
    first steps at 1 g/cm^3 are timed on their own) and the same run at alpha = 0.08, which
    holds ~300 K and ~1 g/cm^3 over the run."""
    return {"configuration_alpha_0.25": run_water(rbe, steps=steps, warmup=warmup),
            "alpha_0.08": run_water(rbe, steps=steps, warmup=warmup, alpha=0.08)}


def run_general(rbe, steps=20, warmup=3):
    """The general-cell (triclinic) k-space path on the slab workload with the box sheared
    (tilts 10, -8 and 12 A), FP32-phase and FP64, against the rectangular path on the unsheared
    slab: N P pair evaluations per second, CUDA events per evaluation, L2 flushed between them."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    s = inputs.slab()
    box = np.asarray(s.box, dtype=np.float64)
    h = np.array([[box[0], 10.0, -8.0], [0.0, box[1], 12.0], [0.0, 0.0, box[2]]])
    frac = np.asarray(s.pos) / box  # the slab's scaled coordinates, placed in the sheared cell
    pos_g = torch.as_tensor(frac @ h.T).to(dev)
    pos_r = torch.as_tensor(np.asarray(s.pos)).to(dev)
    q = torch.as_tensor(np.asarray(s.q)).to(dev)
    N = q.shape[0]
    F = torch.empty((N, 3), dtype=torch.float64, device=dev)
    W = torch.empty(9, dtype=torch.float64, device=dev)
    E = torch.empty(2, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    out = {"N": int(N), "P": int(s.P), "tilts_A": [10.0, -8.0, 12.0]}
    for name, prec in (("fp32_phase", rbe.RBE_FP32_PHASE), ("fp64", rbe.RBE_FP64)):
        n = steps if prec == rbe.RBE_FP32_PHASE else max(2, steps // 4)
        with rbe.Context(box, s.alpha, s.P, 12345, prec, stream=stream.cuda_stream) as ctx:
            for label, fn in (("general", lambda k: ctx.forces_virial_general(pos_g, q, h, k, F, W, E)),
                              ("rectangular", lambda k: ctx.forces_virial(pos_r, q, k, F, W, E))):
                for k in range(warmup):
                    fn(k)
                ms = []
                for k in range(n):
                    flush.fill_(float(k))
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    fn(warmup + k)
                    e1.record(stream)
                    ctx.sync()
                    ms.append(e0.elapsed_time(e1))
                t = float(np.median(ms))
                out[f"{name}_{label}_ms"] = t
                out[f"{name}_{label}_pair_evals_per_s"] = N * s.P / (t * 1e-3)
    return out


def run_batched(rbe, n_items=64, P=100, iters=20, tiles=None):
    """Batched k-space (one evaluation of n_items uneven systems in one persistent launch,
    autotuned tiles; also timed as one launch per pass) against a loop of single-system
    evaluations of the same systems on one stream:
    the first n_items request sizes of the serving stream, +-1 charges at 0.1 per A^3."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    reqs = inputs.request_stream(n_items, 20.0, seed=0)
    items, ctxs = [], []
    stream = torch.cuda.current_stream()
    for r in reqs:
        pos, _, q, _, box = inputs.npt_replica(r.N, r.seed)
        it = dict(pos=torch.as_tensor(pos).to(dev), q=torch.as_tensor(q).to(dev),
                  F=torch.empty((r.N, 3), dtype=torch.float64, device=dev),
                  W=torch.empty(9, dtype=torch.float64, device=dev), E=torch.empty(2, dtype=torch.float64, device=dev),
                  box=box, seed=1000 + r.rid, step=0)
        items.append(it)
        ctxs.append(rbe.Context(box, SERVE_ALPHA, P, 1000 + r.rid, rbe.RBE_FP32_PHASE, stream=stream.cuda_stream))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    max_box = max(float(np.max(it["box"])) for it in items) * 1.01
    out = {"items": n_items, "N_total": int(sum(r.N for r in reqs)), "P": P,
           "N_range": [int(min(r.N for r in reqs)), int(max(r.N for r in reqs))]}
    with rbe.Batch(SERVE_ALPHA, P, n_items, max_box, stream=stream.cuda_stream) as b:
        arr = b.items(items)
        if tiles:  # pinned shapes (rho lanes, frequencies per lane, rho chunk, force block)
            b.set_tiles(tiles[0], tiles[2], tiles[3])
            b.set_rho_f(tiles[1])
            out["autotune_ms"] = None
        else:
            out["autotune_ms"] = b.autotune(arr, reps=3)
        out["tiles"] = {"rho_k": b.tiles()[0], "rho_f": b.rho_f(), "rho_chunk": b.tiles()[1],
                        "force_block": b.tiles()[2]}

        def timed(fn):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            ms = []
            for k in range(iters):
                flush.fill_(float(k))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                ms.append((e0, e1))
            torch.cuda.synchronize()
            return float(np.mean([a.elapsed_time(c) for a, c in ms]))

        def loop():
            for c, it in zip(ctxs, items):
                c.forces_virial(it["pos"], it["q"], 0, it["F"], it["W"], it["E"])

        out["batched_ms"] = timed(lambda: b.evaluate(arr))
        b.sync()
        # the same tile bodies and work lists, one launch per pass instead of the persistent launch
        b.set_persistent(False)
        out["batched_one_launch_per_pass_ms"] = timed(lambda: b.evaluate(arr))
        b.sync()
        b.set_persistent(True)
        out["loop_ms"] = timed(loop)
        for c in ctxs:
            c.sync()
            c.close()
    pairs = out["N_total"] * P
    out["pair_evals_per_s_batched"] = pairs / (out["batched_ms"] * 1e-3)
    out["pair_evals_per_s_loop"] = pairs / (out["loop_ms"] * 1e-3)
    out["batched_over_loop"] = out["loop_ms"] / out["batched_ms"]
    out["launches"] = {"batched": 1, "batched_one_launch_per_pass": 5, "loop": 4 * n_items}
    # against the measured MUFU rate at 3 MUFU operations per pair (a sine and a cosine in the
    # rho pass, one sine in the force pass), like the single-system evaluation
    peak = rbe.rbe_measure_pipe(0, 4096)
    out["mufu_frac"] = {"persistent": 3.0 * pairs / (out["batched_ms"] * 1e-3) / peak,
                        "one_launch_per_pass": 3.0 * pairs / (out["batched_one_launch_per_pass_ms"] * 1e-3) / peak,
                        "peak": peak}
    # and against instruction issue, which binds both pair passes at P = 100: the warp instructions
    # of one evaluation of these 64 systems (ncu, profiles/batched_kspace_64systems_P100.md: the
    # rho, reduction and force passes one launch each, 132.7 M; the persistent kernel 139.1 M)
    # over 152 SMs x 4 schedulers x 2.07 GHz
    if n_items == 64 and P == 100:
        import torch
        issue = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count * 4 * 2.07e9
        out["issue_frac"] = {"persistent": 139.1e6 / (out["batched_ms"] * 1e-3) / issue,
                             "one_launch_per_pass": 132.7e6 / (out["batched_one_launch_per_pass_ms"] * 1e-3) / issue,
                             "peak_warp_instructions_per_s": issue}
    return out


def run_sweep(rbe, steps=3):
    """Large-N precision and roofline sweep: N in {1e5, 1e6, 4e6} uniform +-1 charges at 0.1 per
    A^3, P in {100, 500, 2000}; the FP32-phase path with each rho accumulation (FP32 within a
    tile, compensated FP32, FP64) and the FP64 path; pair evaluations/s (CUDA events, L2
    flushed between steps), the MUFU fraction of the FP32-phase passes, and the errors of each
    FP32-phase variant against the FP64 path on the same frequencies (forces: relative RMS;
    virial: relative Frobenius; Pxx/Pyy/Pzz: largest relative error; E_k: relative)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    peak = rbe.rbe_measure_pipe(0, 4096)
    out = []
    for N in (100_000, 1_000_000, 4_000_000):
        s = inputs.uniform_density(N)
        pos = torch.as_tensor(s.pos).to(dev)
        q = torch.as_tensor(s.q).to(dev)
        F = torch.empty((N, 3), dtype=torch.float64, device=dev)
        W = torch.empty(9, dtype=torch.float64, device=dev)
        E = torch.empty(2, dtype=torch.float64, device=dev)
        for P in (100, 500, 2000):
            row = {"N": N, "P": P}
            ref = None
            variants = [("fp64", rbe.RBE_FP64, rbe.RBE_RHO_FP32), ("fp32_rho_fp32", rbe.RBE_FP32_PHASE, rbe.RBE_RHO_FP32),
                        ("fp32_rho_comp32", rbe.RBE_FP32_PHASE, rbe.RBE_RHO_COMP32),
                        ("fp32_rho_fp64", rbe.RBE_FP32_PHASE, rbe.RBE_RHO_FP64)]
            for name, prec, acc in variants:
                with rbe.Context(s.box, s.alpha, P, SEED, prec, acc, stream=stream.cuda_stream) as ctx:
                    n = 1 if (prec == rbe.RBE_FP64 and N * P > 1e9) else steps
                    ctx.forces_virial(pos, q, 7, F, W, E)  # warm-up
                    ms = []
                    for k in range(n):
                        flush.fill_(float(k))
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        ctx.forces_virial(pos, q, 7, F, W, E)  # the same frequencies every time
                        e1.record(stream)
                        ms.append((e0, e1))
                    torch.cuda.synchronize()
                    ctx.sync()
                    t = float(np.mean([a.elapsed_time(b) for a, b in ms])) * 1e-3
                    r = {"pair_evals_per_s": N * P / t, "ms": t * 1e3}
                    if prec != rbe.RBE_FP64:
                        r["mufu_frac_of_measured"] = 3.0 * N * P / t / peak
                    if ref is None:
                        ref = (F.cpu().numpy(), W.cpu().numpy().reshape(3, 3), E.cpu().numpy())
                    else:
                        F1, W1, E1 = F.cpu().numpy(), W.cpu().numpy().reshape(3, 3), E.cpu().numpy()
                        F0, W0, E0 = ref
                        r["force_rel_rms"] = float(np.sqrt(np.mean((F1 - F0) ** 2) / np.mean(F0 ** 2)))
                        r["virial_rel"] = float(np.linalg.norm(W1 - W0) / np.linalg.norm(W0))
                        dW = np.abs(np.diag(W1) - np.diag(W0))
                        r["pressure_diag_rel_max"] = float(np.max(dW / np.abs(np.diag(W0))))
                        r["pressure_diag_err_over_max_diag"] = float(np.max(dW) / np.max(np.abs(np.diag(W0))))
                        r["energy_rel"] = float(abs(E1[0] - E0[0]) / abs(E0[0]))
                    row[name] = r
            # float32 (x, y, z, q) input, compensated accumulation: the error of the input's rounding
            # (the FP64 path on the rounded positions against the FP64 path on the FP64 ones) apart
            # from the error of the evaluation (against the FP64 path on the rounded positions)
            xyzq = torch.cat([pos, q[:, None]], dim=1).to(torch.float32).contiguous()
            pos_r = xyzq[:, :3].to(torch.float64).contiguous()
            q_r = xyzq[:, 3].to(torch.float64).contiguous()
            with rbe.Context(s.box, s.alpha, P, SEED, rbe.RBE_FP64, stream=stream.cuda_stream) as ctx:
                ctx.forces_virial(pos_r, q_r, 7, F, W, E)
                ctx.sync()
                Fr, Wr, Er = F.cpu().numpy(), W.cpu().numpy().reshape(3, 3), E.cpu().numpy()
            with rbe.Context(s.box, s.alpha, P, SEED, rbe.RBE_FP32_PHASE, rbe.RBE_RHO_COMP32,
                             stream=stream.cuda_stream) as ctx:
                ctx.forces_virial_xyzq(xyzq, 7, F, W, E)
                ms = []
                for k in range(steps):
                    flush.fill_(float(k))
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    ctx.forces_virial_xyzq(xyzq, 7, F, W, E)
                    e1.record(stream)
                    ms.append((e0, e1))
                torch.cuda.synchronize()
                ctx.sync()
                t = float(np.mean([a.elapsed_time(b) for a, b in ms])) * 1e-3
                F1, W1, E1 = F.cpu().numpy(), W.cpu().numpy().reshape(3, 3), E.cpu().numpy()
            F0, W0, E0 = ref

            def errs(Fa, Wa, Ea, Fb, Wb, Eb):
                return {"force_rel_rms": float(np.sqrt(np.mean((Fa - Fb) ** 2) / np.mean(Fb ** 2))),
                        "virial_rel": float(np.linalg.norm(Wa - Wb) / np.linalg.norm(Wb)),
                        "pressure_diag_rel_max": float(np.max(np.abs(np.diag(Wa) - np.diag(Wb)) / np.abs(np.diag(Wb)))),
                        "energy_rel": float(abs(Ea[0] - Eb[0]) / abs(Eb[0]))}
            row["fp32_xyzq_comp32"] = {"pair_evals_per_s": N * P / t, "ms": t * 1e3,
                                       "mufu_frac_of_measured": 3.0 * N * P / t / peak,
                                       "input_rounding_error": errs(Fr, Wr, Er, F0, W0, E0),
                                       "compute_error": errs(F1, W1, E1, Fr, Wr, Er)}
            del xyzq, pos_r, q_r
            out.append(row)
        del pos, q, F
    return {"system": "uniform +-1 charges at 0.1 per A^3, alpha = 0.2", "steps": steps,
            "mufu_peak_measured": peak, "points": out}


# Warp instructions of one NPT step per particle (FP32-phase, P = 100, neighbour list, at the
# serving stream's mean size N = 2e4; all kernels of 24 evaluations summed and divided by
# 24 N: ncu smsp__inst_executed.sum of every launch, 80 % of them the real-space list evaluation).
NPT_WARP_INSTR_PER_PARTICLE_STEP = 644.7e6 / (24 * 20000)


def served_roofline(rbe, closed):
    """The served form against its binding resources: the NPT step is bound by instruction issue
    (the real-space list evaluation, about 80 % of its instructions), so the served particle-steps
    per second times the warp instructions of a particle-step (measured) is set against the GPU's
    issue rate (one warp instruction per clock per scheduler, four per SM); the k-space part
    against the measured MUFU rate at 3 MUFU operations per pair."""
    import torch
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sm_hz = 2.07e9  # the maximum SM clock, which the clock samples of the timed regions show under load
    issue_peak = props.multi_processor_count * 4 * sm_hz
    particle_steps = closed["pair_evals_per_s"] / SERVE_P
    achieved = particle_steps * NPT_WARP_INSTR_PER_PARTICLE_STEP
    mufu = rbe.rbe_measure_pipe(0, 4096)
    return {"bound": "issue", "unit": "warp-instructions/s", "achieved": achieved, "peak": issue_peak,
            "frac": achieved / issue_peak, "particle_steps_per_s": particle_steps,
            "warp_instructions_per_particle_step": NPT_WARP_INSTR_PER_PARTICLE_STEP,
            "kspace_mufu_frac": 3.0 * closed["pair_evals_per_s"] / mufu,
            "source": "profiles/npt_replica_N20000_fp32_instruction_counts.md (ncu, N = 2e4)"}


def run_serving(args, world, rank):
    """Requests of Poisson arrivals at 20/s, N log-uniform in [1e3, 1e5] at 0.1 per A^3,
    P = 100, 100 NPT steps each, chunks of 10 steps: closed-loop capacity and open-loop
    latency of the FP32-phase server, against FP64 one request at a time on a sample."""
    import paper_2110_14362_gb300 as rbe
    reqs = inputs.request_stream(args.serve_requests, 20.0, seed=0)
    states = [inputs.npt_replica(r.N, r.seed) for r in reqs]
    steps, chunk = args.serve_steps, 10
    # warm-up: a few requests through a server (module load, pools, first graph)
    serve(rbe, reqs[:4], states[:4], rbe.RBE_FP32_PHASE, args.serve_slots, chunk, chunk)
    closed = serve(rbe, reqs, states, rbe.RBE_FP32_PHASE, args.serve_slots, chunk, steps)
    wall = max_over_ranks(world, closed["wall_s"])
    closed["replica_steps_per_s_all_ranks"] = world * closed["replica_steps"] / wall
    out = {"workload": f"{len(reqs)} NPT replica requests, Poisson 20/s, N log-uniform [1e3, 1e5] at 0.1/A^3, "
                       f"P={SERVE_P}, {steps} steps, chunk {chunk} steps, FP32-phase",
           "slots": args.serve_slots, "closed_loop": closed, "roofline": served_roofline(rbe, closed)}
    if not args.skip_open_loop:
        out["open_loop_20_per_s"] = serve(rbe, reqs, states, rbe.RBE_FP32_PHASE, args.serve_slots, chunk, steps,
                                          open_loop=True)
    # lockstep groups: every step's k-space of the resident replicas in one persistent batched
    # launch, a stable group replayed as one captured graph
    serve(rbe, reqs[:4], states[:4], rbe.RBE_FP32_PHASE, args.serve_slots, chunk, chunk, batched=2)
    lock = serve(rbe, reqs, states, rbe.RBE_FP32_PHASE, args.serve_slots, chunk, steps, batched=2)
    lock["replica_steps_per_s_all_ranks"] = world * lock["replica_steps"] / max_over_ranks(world, lock["wall_s"])
    out["lockstep_batched_closed_loop"] = lock
    if not args.skip_open_loop:
        out["lockstep_batched_open_loop_20_per_s"] = serve(rbe, reqs, states, rbe.RBE_FP32_PHASE, args.serve_slots,
                                                           chunk, steps, open_loop=True, batched=2)
    k = min(args.serve_fp64_sample, len(reqs))
    if k > 0:
        fp64 = serve(rbe, reqs[:k], states[:k], rbe.RBE_FP64, 1, chunk, steps, use_graphs=False)
        same = serve(rbe, reqs[:k], states[:k], rbe.RBE_FP32_PHASE, args.serve_slots, chunk, steps)
        out["fp64_one_at_a_time"] = dict(fp64, sample=f"first {k} requests")
        out["fp32_served_same_sample"] = dict(same, sample=f"first {k} requests")
        out["served_fp32_over_fp64_one_at_a_time"] = same["replica_steps_per_s"] / fp64["replica_steps_per_s"]
    return out


def cpu_baseline(s, budget_s: float = 15.0):
    """The FP64 oracle, as it stands, on a bounded sample: the same P frequencies against
    the first n particles, n sized so the run takes about budget_s seconds."""
    import oracle
    m, S = oracle.sample_k(s.box, s.alpha, s.P, SEED, 0)
    n = min(s.N, 256)
    t0 = time.perf_counter()
    oracle.rbe_kspace(s.pos[:n], s.q[:n], s.box, s.alpha, m, S / s.P)
    dt = time.perf_counter() - t0
    n2 = int(min(s.N, max(n, n * budget_s / max(dt, 1e-6) * 0.8)))
    t0 = time.perf_counter()
    oracle.rbe_kspace(s.pos[:n2], s.q[:n2], s.box, s.alpha, m, S / s.P)
    dt = time.perf_counter() - t0
    return {"value": n2 * s.P / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {n2} of {s.N} particles x all P={s.P} frequencies (rho pass + force pass, FP64, "
                      f"single thread), {dt:.1f} s"}


def cpu_baseline_all_cores(s, budget_s: float = 5.0):
    """The same oracle loops built with OpenMP (frequencies of the rho pass and particles of
    the force pass shared among every host core, the results the same bits), on a bounded
    sample sized like cpu_baseline's; None where gcc has no OpenMP runtime."""
    import subprocess
    import oracle
    try:
        oracle.build_omp()
    except (subprocess.CalledProcessError, OSError):
        return None
    cores = int(os.environ.get("OMP_NUM_THREADS", 0)) or len(os.sched_getaffinity(0))
    m, S = oracle.sample_k(s.box, s.alpha, s.P, SEED, 0)
    n = min(s.N, 1024)
    t0 = time.perf_counter()
    oracle.rbe_kspace(s.pos[:n], s.q[:n], s.box, s.alpha, m, S / s.P, all_cores=True)
    dt = time.perf_counter() - t0
    n2 = int(min(s.N, max(n, n * budget_s / max(dt, 1e-6) * 0.8)))
    t0 = time.perf_counter()
    oracle.rbe_kspace(s.pos[:n2], s.q[:n2], s.box, s.alpha, m, S / s.P, all_cores=True)
    dt = time.perf_counter() - t0
    return {"value": n2 * s.P / dt, "unit": UNIT, "cores": cores, "kind": "oracle (OpenMP build)",
            "sample": f"first {n2} of {s.N} particles x all P={s.P} frequencies (rho pass + force pass, FP64, "
                      f"{cores} threads), {dt:.1f} s"}


def run_reference(args, world, rank):
    if rank != 0:
        return
    s = workload(args.workload)
    import oracle
    m, S = oracle.sample_k(s.box, s.alpha, s.P, SEED, 0)
    # each step: the oracle on a bounded sample sized so that the whole run takes minutes
    n = min(s.N, 256)
    t0 = time.perf_counter()
    oracle.rbe_kspace(s.pos[:n], s.q[:n], s.box, s.alpha, m, S / s.P)
    dt = time.perf_counter() - t0
    per_step = max(1.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    n = int(min(s.N, max(n, n * per_step / max(dt, 1e-6))))
    for w in range(args.warmup):
        oracle.rbe_kspace(s.pos[:n], s.q[:n], s.box, s.alpha, m, S / s.P)
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle.rbe_kspace(s.pos[:n], s.q[:n], s.box, s.alpha, m, S / s.P)
    dt = time.perf_counter() - t0
    value = args.steps * n * s.P / dt
    sample = f"first {n} of {s.N} particles x all P={s.P} frequencies per step (FP64 oracle, single thread)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded NumPy)",
        "config": {"workload": s.name, "N": s.N, "P": s.P, "precision": "fp64 (oracle)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="uniform4e6-P2000")
    ap.add_argument("--rho-accum", choices=["comp32", "fp32", "fp64"], default="comp32",
                    help="rho accumulation of the FP32-phase path (default: compensated FP32)")
    ap.add_argument("--skip-slab", action="store_true", help="leave out the slab workload's line")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--skip-serving", action="store_true")
    ap.add_argument("--skip-open-loop", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=256)
    ap.add_argument("--serve-steps", type=int, default=100)
    ap.add_argument("--serve-slots", type=int, default=64)
    ap.add_argument("--serve-fp64-sample", type=int, default=16)
    ap.add_argument("--profile-npt", type=int, default=0, help="time only NPT steps of one replica of this N")
    ap.add_argument("--barostat", type=int, default=1, choices=(0, 1, 2, 3, 4),
                    help="with --profile-npt: 0 fixed box, 1 isotropic, 2 anisotropic, 3 semi-isotropic, "
                         "4 fully flexible (sheared) cell")
    ap.add_argument("--sampler", choices=["exact", "offline", "mh"], default="exact",
                    help="with --profile-npt: the frequency sampler (Sec. 4.3 variants)")
    ap.add_argument("--ptilde", type=int, default=0, help="with --profile-npt: a separate pressure batch")
    ap.add_argument("--reuse", type=int, default=1, help="with --profile-npt: samples drawn every M steps")
    ap.add_argument("--profile-batched", action="store_true", help="time only the batched k-space evaluation")
    ap.add_argument("--batched-tiles", default=None,
                    help="with --profile-batched: pin the tiles 'lanes,freqs_per_lane,chunk,force_block' (no autotune)")
    ap.add_argument("--profile-serving", action="store_true", help="run only the serving measurements")
    ap.add_argument("--profile-water", action="store_true",
                    help="run only the rigid-water NPT run (3000 molecules, FP64, --steps steps)")
    ap.add_argument("--water-alpha", type=float, default=None, help="with --profile-water: another alpha")
    ap.add_argument("--water-barostat", type=int, default=1, choices=(0, 1),
                    help="with --profile-water: 0 keeps the box fixed")
    ap.add_argument("--profile-general", action="store_true",
                    help="time only the general-cell (triclinic) k-space path on the sheared slab")
    ap.add_argument("--skip-sweep", action="store_true", help="leave out the large-N precision and roofline sweep")
    ap.add_argument("--profile-sweep", action="store_true", help="run only the large-N sweep")
    ap.add_argument("--profile-kspace", action="store_true",
                    help="run only --warmup + --steps evaluations of --workload (back to back, no L2 flush)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_init()
    if args.profile_npt:
        # profiling aid: only the NPT steps of one replica of this many particles
        import torch
        import paper_2110_14362_gb300 as rbe
        torch.cuda.set_device(local)
        prec = rbe.RBE_FP32_PHASE if args.precision == "fp32" else rbe.RBE_FP64
        smp = {"exact": rbe.RBE_SAMPLER_EXACT, "offline": rbe.RBE_SAMPLER_OFFLINE, "mh": rbe.RBE_SAMPLER_MH}
        ms = npt_single(rbe, args.profile_npt, prec, args.steps, args.warmup, barostat=args.barostat,
                        sampler=smp[args.sampler], ptilde=args.ptilde, reuse=args.reuse)
        print(json.dumps({"metric": "NPT steps of one replica", "value": 1e3 / ms, "unit": "replica-steps/s",
                          "ms_per_step": ms, "N": args.profile_npt, "precision": args.precision,
                          "barostat": args.barostat, "sampler": args.sampler, "ptilde": args.ptilde,
                          "reuse": args.reuse}), flush=True)
        return
    if args.profile_kspace:
        # profiling aid: only evaluations of the workload (the command of the ncu summaries)
        import torch
        import paper_2110_14362_gb300 as rbe
        torch.cuda.set_device(local)
        s = workload(args.workload)
        prec = rbe.RBE_FP32_PHASE if args.precision == "fp32" else rbe.RBE_FP64
        acc = {"comp32": rbe.RBE_RHO_COMP32, "fp32": rbe.RBE_RHO_FP32, "fp64": rbe.RBE_RHO_FP64}[args.rho_accum]
        dev = torch.device("cuda", local)
        pos = torch.as_tensor(s.pos).to(dev)
        q = torch.as_tensor(s.q).to(dev)
        F = torch.empty((s.N, 3), dtype=torch.float64, device=dev)
        W = torch.empty(9, dtype=torch.float64, device=dev)
        E = torch.empty(2, dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream()
        with rbe.Context(s.box, s.alpha, s.P, SEED, prec, acc, stream=stream.cuda_stream) as ctx:
            for k in range(args.warmup):
                ctx.forces_virial(pos, q, k, F, W, E)
            ctx.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(args.steps):
                ctx.forces_virial(pos, q, args.warmup + k, F, W, E)
            e1.record(stream)
            ctx.sync()
        ms = e0.elapsed_time(e1) / args.steps
        print(json.dumps({"metric": "k-space evaluations", "workload": s.name, "precision": args.precision,
                          "rho_accum": args.rho_accum, "ms_per_step": ms,
                          "pair_evals_per_s": s.N * s.P / (ms * 1e-3)}), flush=True)
        return
    if args.profile_sweep:
        import torch
        import paper_2110_14362_gb300 as rbe
        torch.cuda.set_device(local)
        print(json.dumps({"metric": "large-N sweep", "sweep": run_sweep(rbe, steps=args.steps)}), flush=True)
        return
    if args.profile_water:
        import torch
        import paper_2110_14362_gb300 as rbe
        torch.cuda.set_device(local)
        print(json.dumps({"metric": "rigid-water NPT run",
                          "water_npt": run_water(rbe, steps=args.steps, warmup=args.warmup, alpha=args.water_alpha,
                                                 barostat=args.water_barostat)}), flush=True)
        return
    if args.profile_general:
        import torch
        import paper_2110_14362_gb300 as rbe
        torch.cuda.set_device(local)
        print(json.dumps({"metric": "general-cell k-space", "general": run_general(rbe, steps=args.steps)}),
              flush=True)
        return
    if args.profile_serving:
        import torch
        torch.cuda.set_device(local)
        print(json.dumps({"metric": "serving", "serving": run_serving(args, world, rank)}), flush=True)
        return
    if args.profile_batched:
        # profiling aid: only the batched-versus-loop k-space measurement
        import torch
        import paper_2110_14362_gb300 as rbe
        torch.cuda.set_device(local)
        tiles = [int(x) for x in args.batched_tiles.split(",")] if args.batched_tiles else None
        print(json.dumps({"metric": "batched k-space", "batched_kspace": run_batched(rbe, iters=args.steps, tiles=tiles)}),
              flush=True)
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
