#!/usr/bin/env python3
"""Benchmark of the GB300 percolation-inspection hot path.

Workload (one "step"): the p-sweep of the Markov inspection -- modified-FCC
fibre lattice W = 8, L = 64 (A = 217 columns, N = 13,888 sites), p = 0.100 ..
0.200 in steps of 0.005 (21 values), 10^4 configurations per p from the
Philox4x32-10 stream with seed 2, one inspection launch per p.  Metric:
site-updates per second (every step m of the forward recursion that computes
mu_m sweeps the causal window of min(m+1, L) layers of A sites).

Default arm: libpercol on the GPU.  ``--impl reference``: the CPU oracle
(explicit FP64 transition matrix, Sec. II.B) on the host cores, each step a
bounded sample of the same workload.

Multi-GPU (torchrun, one rank per GPU): weak scaling -- rank r inspects
configurations [r * 10^4, (r + 1) * 10^4) at every p; no data-path collective.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

W, L, SEED, N_CFG = 8, 64, 2, 10_000
PS = [round(0.100 + 0.005 * k, 3) for k in range(21)]
A_COLS = 3 * W * (W + 1) + 1
# Shared-memory traffic model of one site update in the resident solver
# (gather form): 14 neighbour nu reads + 1/deg read + nu write, FP32.
SMEM_BYTES_PER_SU = 14 * 4 + 4 + 4
METRIC = "site-updates/s"
UNIT = "SU/s"
L2_FLUSH_BYTES = 256 << 20


def site_updates(A, L_, verdict, first_hit, m_stop) -> int:
    v = np.asarray(verdict).astype(np.int64)
    fh = np.asarray(first_hit).astype(np.int64)
    ms = np.asarray(m_stop).astype(np.int64)
    M = np.maximum(np.where(v != 0, fh - 1, ms), 0)
    k = np.minimum(M, L_ - 1)
    return int((k * (k + 3) // 2 + np.maximum(M - k, 0) * L_).sum()) * A


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.t = None

    def __enter__(self):
        cmd = ["nvidia-smi", f"--id={self.index}",
               "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
               "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
               "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "100"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.t:
                self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0])); mx = float(f[1])
            except ValueError:
                continue
            for nm, val in zip(names, f[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def cpu_sample(per_p: int, threads: int, cfg0: int = 0):
    """Time the oracle (Markov mode, as it stands) on per_p configurations at
    each p of the sweep; returns (site_updates, seconds)."""
    import oracle
    oracle.build()
    su, t = 0, 0.0
    for p in PS:
        t0 = time.perf_counter()
        r = oracle.inspect(W, L, p=p, seed=SEED, cfg0=cfg0, n=per_p, mode="markov",
                           threads=threads)
        t += time.perf_counter() - t0
        su += site_updates(A_COLS, L, r["verdict"], r["first_hit"], r["m_stop"])
    return su, t


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    threads = os.cpu_count() or 1
    per_p = args.ref_per_p
    for _ in range(args.warmup):
        cpu_sample(max(per_p // 10, 1), threads)
    su_tot, t_tot = 0, 0.0
    for k in range(args.steps):
        su, t = cpu_sample(per_p, threads, cfg0=k * per_p)
        su_tot += su; t_tot += t
    value = su_tot / t_tot
    sample = f"{per_p} configurations per p x 21 p per step (of 10^4 per p)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "p-sweep W=8 L=64 p=0.100..0.200/0.005 seed=2",
                   "W": W, "L": L, "n_p": len(PS), "configs_per_p": N_CFG, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--ref-per-p", type=int, default=200)
    ap.add_argument("--cpu-per-p", type=int, default=2000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_1401_2130_gb300 as pc

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pc.build()
    pc.load()
    cfg0 = rank * N_CFG
    stream = torch.cuda.current_stream()
    outs = [pc._alloc_outputs(N_CFG, True, pc.ALL_OUTPUTS) for _ in PS]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def one_step(evs=None):
        for i, p in enumerate(PS):
            if evs is not None:
                evs[i][0].record(stream)
            pc.pc_inspect(W, L, p, SEED, cfg0, N_CFG, device=True, out=outs[i], stream=stream)
            if evs is not None:
                evs[i][1].record(stream)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    # per-configuration work of one step (identical every step: same inputs)
    su_step = 0
    for i, p in enumerate(PS):
        o = {k: v.cpu().numpy() for k, v in outs[i].items()}
        su_step += site_updates(A_COLS, L, o["verdict"], o["first_hit"], o["m_stop"])
    n_perc = [int(outs[i]["n_percolating"].item()) for i in range(len(PS))]

    step_ms, launch_ms = [], []
    with Clocks(local) as clk:
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1.0)  # evict L2 between timed steps (outside the events)
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in PS]
            one_step(evs)
            torch.cuda.synchronize()
            ms = [a.elapsed_time(b) for a, b in evs]
            launch_ms.extend(ms)
            step_ms.append(sum(ms))
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        wall = time.perf_counter() - t_wall
    t_step = float(np.mean(step_ms)) / 1e3
    if dist is not None:
        tt = torch.tensor([t_step], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_step = float(tt.item())
    value = su_step * world / t_step

    # end to end through the public call with host outputs (D2H inside)
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for p in PS:
            pc.pc_inspect(W, L, p, SEED, cfg0, N_CFG, device=False)
    e2e_t = (time.perf_counter() - t0) / e2e_steps
    if dist is not None:
        tt = torch.tensor([e2e_t], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_t = float(tt.item())
    d2h = len(PS) * (N_CFG * (1 + 4 + 4 + 4) + 8)

    peaks = measured_peaks()
    clocks = clk.summary()
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    sm_max = peaks.get("sm_max_mhz") or clocks.get("sm_max_mhz") or 2070.0
    smem_peak = nsm * 128 * sm_max * 1e6 / 1e9  # GB/s: 32 banks x 4 B per clock per SM
    achieved = SMEM_BYTES_PER_SU * su_step / (sum(launch_ms) / len(step_ms) / 1e3) / 1e9

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "p-sweep W=8 L=64 p=0.100..0.200/0.005 seed=2",
                   "W": W, "L": L, "n_p": len(PS), "configs_per_p": N_CFG,
                   "configs_per_step": N_CFG * len(PS) * world,
                   "site_updates_per_step_per_gpu": su_step,
                   "percolating_per_p": n_perc, "solver": "resident",
                   "l2": "flushed between steps (256 MiB write, outside the timed events)",
                   "parallelism": f"configs sharded over {world} GPU(s)"},
        "configs_per_s": N_CFG * len(PS) * world / t_step,
        "roofline": {"bound": "smem", "achieved": achieved, "peak": smem_peak, "unit": "GB/s",
                     "frac": achieved / smem_peak, "traffic": None,
                     "model": f"{SMEM_BYTES_PER_SU} B of shared-memory traffic per site update; "
                              f"peak = {nsm} SMs x 128 B/clk x {sm_max:.0f} MHz (derived)"},
        "clocks": clocks,
        "e2e": {"value": su_step * world / e2e_t, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": len(PS) * args.steps,
        "wall_s_timed": wall,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        su, t = cpu_sample(args.cpu_per_p, threads)
        line["cpu_baseline"] = {"value": su / t, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"{args.cpu_per_p} configurations per p x 21 p, "
                                          f"Markov mode (FP64 CSR), {t:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
