#!/usr/bin/env python3
"""Benchmark of the GB300 percolation-inspection hot path.

Default workload (``--workload large``): the HBM-bound single-lattice case --
modified-FCC fibre lattice W = 64, L = 4096 (A = 12,481 columns, N = 51.1 M
sites), p in {0.14, 0.1533, 0.17}, 64 configurations per p from the
Philox4x32-10 stream with seed 4, solved by the streamed solver (FP32 vector,
exact reached-set bits, bulk-copy-staged plane segments).  One "step" is one
block of 8 configurations at each of the three p (three inspection calls);
the steps cycle through the 8 blocks of the 64 configurations.  Metric:
site-updates per second (every step m of the forward recursion sweeps the
causal window of min(m+1, L) layers of A sites), roofline against the
measured HBM copy bandwidth at 8.375 B per site-update.

Other workloads: ``--workload psweep`` (W = 8, L = 64, p = 0.100 .. 0.200, 10^4
configurations per p, seed 2, the shared-memory resident solver), ``batch``,
``serving``, ``fss``.

Default arm: libpercol on the GPU.  ``--impl reference``: the CPU oracle
(explicit FP64 transition matrix, Sec. II.B) on the host cores, each step a
bounded sample of the same workload.

Multi-GPU (torchrun, one rank per GPU): weak scaling -- rank r inspects its own
configuration range at every p; no data-path collective.
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

# p-sweep workload (resident solver)
W, L, SEED, N_CFG = 8, 64, 2, 10_000
PS = [round(0.100 + 0.005 * k, 3) for k in range(21)]
A_COLS = 3 * W * (W + 1) + 1
# large single-lattice workload (streamed solver, HBM bound)
LW, LL, LSEED = 64, 4096, 4
LPS = (0.14, 0.1533, 0.17)
LA = 3 * LW * (LW + 1) + 1
# Shared-memory traffic of one site update in the resident solver's gather
# form (14 neighbour nu reads + 1/deg read + nu write, FP32): a secondary
# figure of the p-sweep line.
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


def shard_range(rank: int, n_per_rank: int) -> tuple[int, int]:
    """Weak scaling: rank r owns configurations [r * n, (r + 1) * n) at every p.
    Ranks share no data; the only cross-rank step is the timing maximum."""
    return rank * n_per_rank, n_per_rank


def aggregate(site_updates_per_rank: list[int], seconds_per_rank: list[float]) -> float:
    """Whole-job throughput: all ranks' site updates over the slowest rank's time."""
    return float(sum(site_updates_per_rank)) / max(seconds_per_rank)


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


def cpu_sample(per_p: int, threads: int, cfg0: int = 0, results: list | None = None):
    """Time the oracle (Markov mode, as it stands) on per_p configurations at
    each p of the sweep; returns (site_updates, seconds).  ``results``, if
    given, receives the oracle's outputs per p."""
    import oracle
    oracle.build()
    su, t = 0, 0.0
    for p in PS:
        t0 = time.perf_counter()
        r = oracle.inspect(W, L, p=p, seed=SEED, cfg0=cfg0, n=per_p, mode="markov",
                           threads=threads)
        t += time.perf_counter() - t0
        su += site_updates(A_COLS, L, r["verdict"], r["first_hit"], r["m_stop"])
        if results is not None:
            results.append(r)
    return su, t


def sample_parity(pc, refs, per_p: int, **kw) -> dict:
    """The CUDA path's outputs on the oracle's sample (configurations
    0..per_p-1 at each p, host outputs, outside every timed region):
    verdicts, first_hit and m_stop must be equal, mass within 1e-5."""
    bad, err, n_gpu, n_ref = 0, 0.0, 0, 0
    for p, r in zip(PS, refs):
        g = pc.pc_inspect(W, L, p, SEED, 0, per_p, **kw)
        same = ((g["verdict"].astype(np.int32) == r["verdict"]) & (g["first_hit"] == r["first_hit"])
                & (g["m_stop"] == r["m_stop"]))
        bad += int((~same).sum())
        err = max(err, float(np.abs(g["mass"].astype(np.float64) - r["mass"]).max()))
        n_gpu += int(g["n_percolating"]); n_ref += int(r["verdict"].sum())
    return {"configs": per_p * len(PS), "mismatched_configs": bad, "mass_max_abs_err": err,
            "mass_tolerance": 1e-5, "percolating": [n_gpu, n_ref],
            "ok": bad == 0 and err <= 1e-5 and n_gpu == n_ref}


def run_reference(args):
    """The oracle as it stands on the host cores (rank 0 only; other ranks
    exit 0 without work), on the workload the GPU arm runs."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    if args.workload == "psweep":
        return run_reference_psweep(args, world)
    if args.workload != "large":
        print(json.dumps({"impl": "reference", "unavailable":
                          f"no oracle timing for --workload {args.workload}; it has none on the default line"}))
        return 0
    return run_reference_large(args, world)


def markov_sample_large(p: float, cfg0: int, n: int, threads: int):
    """The oracle's Markov mode on n configurations of the large lattice at p
    (one configuration per thread); returns (outputs, site_updates, seconds)."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    r = oracle.inspect(LW, LL, p=p, seed=LSEED, cfg0=cfg0, n=n, mode="markov", threads=threads)
    dt = time.perf_counter() - t0
    return r, site_updates(LA, LL, r["verdict"], r["first_hit"], r["m_stop"]), dt


def run_reference_large(args, world):
    """Each timed step: the oracle's Markov mode (explicit FP64 CSR over the
    whole lattice, every step) on ``--ref-configs`` configurations at
    p = 0.14, one per core.  At 51 M sites a p = 0.1533 configuration takes
    ~45 s in this mode and a p = 0.17 one (about 12,000 steps) on the order
    of half an hour, so the bounded sample is the low-p one."""
    import oracle
    threads = os.cpu_count() or 1
    n_ref = args.ref_configs or threads
    p0 = LPS[0]
    oracle.build()
    for w in range(args.warmup):  # warm-up: one BFS inspection (page cache, allocator)
        oracle.inspect(LW, LL, p=p0, seed=LSEED, cfg0=1_000_000 + w, n=1, mode="bfs", threads=1)
    su_tot, t_tot = 0, 0.0
    for k in range(args.steps):
        _, su, dt = markov_sample_large(p0, k * n_ref, n_ref, threads)
        su_tot += su; t_tot += dt
    value = su_tot / t_tot
    sample = (f"Markov mode on {n_ref} configurations per step at p = {p0} (configurations "
              f"0..{args.steps * n_ref - 1}), one per core")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "large W=64 L=4096 p=0.14/0.1533/0.17 x 64 configs seed=4",
                   "W": LW, "L": LL, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_reference_psweep(args, world):
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


# HBM traffic model of one site update of the streamed solver, from the
# method's data: nu read 4 B + nu write 4 B + occupancy 1/8 B + reached-set
# bit read and write 1/4 B (the per-unit figure of the measurement plan).
HBM_BYTES_PER_SU = 8.375
# DRAM bytes (read + write) measured with ncu on the current kernels, to be
# re-measured whenever they change: the resident kernel per p-sweep launch
# (tables and outputs only), and the streamed sweep per site-update
# (controlled capture of the large lattice with 4 active slots, ticks
# 600..631 -- one period of the word-row preparation -- i.e. steps 599..630:
# 4 x 12,481 columns x (600 + ... + 631) layers)
RESIDENT_DRAM_BYTES_PER_LAUNCH = 81152.0  # p = 0.2, 2,000 configurations
SWEEP_DRAM_BYTES_PER_SU = (5688.3e6 + 2947.8e6) / (4 * 12481 * 32 * (600 + 631) / 2)
# bits-only variant: occupancy 1/8 B + reached-set bit read and write 1/4 B
BITS_BYTES_PER_SU = 0.375
# The verdict-only solver with temporal blocking keeps a slab on chip for 32
# steps: measured DRAM bytes per site-update of its pass kernel (controlled
# capture: 4 slots at p = 0.17, pass of steps 1889..1920, 24.80 MB for
# 4 x 12,481 x (1890 + ... + 1921) site-updates), and its shared-memory bytes
# per site-update (each 32-tube word step loads the column's next word, its
# occupancy word and its 12 contacts' words, and stores one word: 60 B / 32)
BLOCKED_DRAM_BYTES_PER_SU = 24.80e6 / (4 * 12481 * 32 * (1890 + 1921) / 2)
BLOCKED_SMEM_BYTES_PER_SU = 60 / 32


def batching_specs(n=10_000):
    return [(Wb, Wb * r, 0.1533, 3, 0, n) for Wb in (4, 8, 16, 32) for r in (1, 2, 4, 8, 16, 32, 64)]


def blocked_launches(verdict, first_hit, m_stop) -> int:
    """Kernels of one verdict-only solve by the blocked solver whose
    configurations all hold a slot at once: the init kernel, then a pass and a
    control kernel per tick inside the graph's WHILE node; one tick draws the
    first rows, then one tick per 32 steps of the longest configuration."""
    v = np.asarray(verdict) != 0
    last = np.where(v, np.asarray(first_hit) - 1, np.asarray(m_stop))  # terminating step (0: none)
    passes = np.where(last >= 1, (last - 1) // 32 + 1, 0)
    ticks = 1 + int(passes.max(initial=0))
    return 1 + 2 * ticks


def solve_ticks(verdict, first_hit, m_stop) -> int:
    """Ticks of one streamed solve whose configurations all hold a slot at
    once: the draw and preparation ticks, then one tick per step of the
    longest configuration."""
    steps = np.where(np.asarray(verdict) != 0, np.asarray(first_hit) - 1, np.asarray(m_stop))
    return int(steps.max(initial=0)) + 3


def run_large(args, pc, torch, rank, world, local, dist):
    """W = 64, L = 4096 (51.1 M sites), p in {0.14, 0.1533, 0.17}, 64
    configurations each, seed 4: the streamed solver, HBM bound.  One step =
    one block of configurations at each p; steps cycle through the blocks."""
    ps = list(LPS) if args.large_p is None else [float(v) for v in args.large_p.split(",")]
    n = args.large_configs
    block = max(1, min(args.large_block, n))
    # verdict-only solves run 32 steps per visit of a slab held by one
    # thread-block cluster (PC_BITS_STEPWISE=1 keeps the step-synchronous path)
    shape = pc.pc_bits_blocked_shape(LW) if args.bits_only else None
    blocked = shape is not None and not os.environ.get("PC_BITS_STEPWISE")
    nb = max(1, n // block)
    base = rank * n  # weak scaling: rank r owns configurations [r n, (r + 1) n) at every p
    stream = torch.cuda.current_stream()
    outs = {p: pc._alloc_outputs(nb * block, True, pc.ALL_OUTPUTS) for p in ps}
    nperc = torch.zeros((nb, len(ps)), dtype=torch.int64, device="cuda")

    def block_out(i, p, b):
        o, sl = outs[p], slice(b * block, (b + 1) * block)
        return {"verdict": o["verdict"][sl], "first_hit": o["first_hit"][sl], "mass": o["mass"][sl],
                "m_stop": o["m_stop"][sl], "n_percolating": nperc[b, i:i + 1]}

    def step(b):
        for i, p in enumerate(ps):
            pc.pc_inspect(LW, LL, p, LSEED, base + b * block, block, device=True, out=block_out(i, p, b),
                          stream=stream, bits_only=args.bits_only)

    # warm-up: one configuration per p, outside the timed configuration range
    wo = pc._alloc_outputs(1, True, pc.ALL_OUTPUTS)
    for w in range(args.warmup):
        for p in ps:
            pc.pc_inspect(LW, LL, p, LSEED, base + nb * block + w, 1, device=True, out=wo, stream=stream,
                          bits_only=args.bits_only)
    torch.cuda.synchronize()
    times, blocks = [], []
    with Clocks(local) as clk:
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        for k in range(args.steps):
            b = k % nb
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(b)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            blocks.append(b)
        if dist is not None:
            dist.barrier()
        wall = time.perf_counter() - t_wall
    host = {p: {k: v.cpu().numpy() for k, v in outs[p].items()} for p in ps}

    def block_su(b):
        sl = slice(b * block, (b + 1) * block)
        return sum(site_updates(LA, LL, host[p]["verdict"][sl], host[p]["first_hit"][sl],
                                host[p]["m_stop"][sl]) for p in ps)

    def block_ticks(b):
        sl = slice(b * block, (b + 1) * block)
        return sum(solve_ticks(host[p]["verdict"][sl], host[p]["first_hit"][sl], host[p]["m_stop"][sl])
                   for p in ps)

    def block_launches(b):
        sl = slice(b * block, (b + 1) * block)
        if blocked:
            return sum(blocked_launches(host[p]["verdict"][sl], host[p]["first_hit"][sl], host[p]["m_stop"][sl])
                       for p in ps)
        # query upload and init, then a sweep and a control kernel per tick
        return block_ticks(b) * 2 + 2 * len(ps)

    su_rank = sum(block_su(b) for b in blocks)
    t_rank = float(sum(times))
    su_all, t_max = su_rank, t_rank
    if dist is not None:
        tt = torch.tensor([t_rank], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
        st_ = torch.tensor([float(su_rank)], dtype=torch.float64, device="cuda")
        dist.all_reduce(st_, op=dist.ReduceOp.SUM)
        su_all = int(st_.item())
    value = su_all / t_max

    # end to end through the public call with host outputs (D2H inside);
    # --e2e-steps 0 skips it (profiling runs only)
    e2e_steps = min(args.steps, args.e2e_steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    su_e2e = 0
    for k in range(e2e_steps):
        b = k % nb
        for p in ps:
            r = pc.pc_inspect(LW, LL, p, LSEED, base + b * block, block, bits_only=args.bits_only)
            su_e2e += site_updates(LA, LL, r["verdict"], r["first_hit"], r["m_stop"])
    e2e_t = time.perf_counter() - t0
    if dist is not None:
        tt = torch.tensor([e2e_t], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_t = float(tt.item())
        st_ = torch.tensor([float(su_e2e)], dtype=torch.float64, device="cuda")
        dist.all_reduce(st_, op=dist.ReduceOp.SUM)
        su_e2e = int(st_.item())

    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs") or 6800.0
    bps = BITS_BYTES_PER_SU if args.bits_only else HBM_BYTES_PER_SU
    # per step of this rank (the unit the events time): algorithmic bytes / time
    achieved = bps * su_rank / t_rank / 1e9
    traffic = None
    if blocked:
        traffic = BLOCKED_DRAM_BYTES_PER_SU * su_rank / len(times)
    elif not args.bits_only and SWEEP_DRAM_BYTES_PER_SU is not None:
        traffic = SWEEP_DRAM_BYTES_PER_SU * su_rank / len(times)
    perc = {str(p): int(host[p]["verdict"][:len(set(blocks)) * block].sum()) for p in ps}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / len(times) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"large W=64 L=4096 p={'/'.join(str(p) for p in ps)} x {n} configs seed=4"
                               + (" (bits only)" if args.bits_only else ""),
                   "W": LW, "L": LL, "configs_per_p": n, "configs_per_step": block * len(ps) * world,
                   "step": f"configurations [{block}b, {block}b + {block}) at each p, b = step mod {nb}",
                   "site_updates_per_step": su_all / len(times), "percolating_per_p": perc,
                   "solver": (f"verdict-only, temporally blocked: 32 steps per slab of "
                              f"{shape['slab_rows'] - 2} word rows, clusters of {shape['cluster_size']} CTAs "
                              f"({shape['clusters']} resident)" if blocked else "streamed"),
                   "parallelism": f"configs sharded over {world} GPU(s)",
                   "l2": "inputs larger than L2 (each configuration's state is ~0.5 GB), no flush"},
        "configs_per_s": block * len(ps) * world * len(times) / t_max,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic,
                     "traffic_note": ("ncu DRAM bytes (read + write) per site-update of "
                                      + ("blocked_pass_kernel (controlled capture, 4 slots)" if blocked else
                                         "sweep_kernel (controlled capture, all slots active)")
                                      + " x the step's site-updates"),
                     "model": f"{bps} B/site-update x site-updates of a step / CUDA-event time of the "
                              "step (every kernel of the solve), peak = measured copy bandwidth "
                              "(MEASURED_PEAKS.json hbm_gbs)"},
        "clocks": clk.summary(),
        "e2e": {"value": su_e2e / e2e_t if e2e_steps else None, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": len(ps) * (block * (1 + 4 + 4 + 4) + 8)},
        "gpu_launches": sum(block_launches(b) for b in blocks),
        "step_ms": [round(t * 1e3, 3) for t in times],
        "wall_s_timed": wall,
    }
    if blocked:
        # the step-synchronous model's bytes do not reach DRAM here: the slab
        # stays in shared memory for 32 steps, so shared memory bounds it
        smem_peak = 152 * 128 * (line["clocks"].get("sm_mhz") or 2070.0) * 1e6 / 1e9
        ach = BLOCKED_SMEM_BYTES_PER_SU * su_rank / t_rank / 1e9
        line["roofline_onchip"] = {
            "bound": "smem", "achieved": ach, "peak": smem_peak, "unit": "GB/s", "frac": ach / smem_peak,
            "model": f"{BLOCKED_SMEM_BYTES_PER_SU} B of shared-memory traffic per site-update (12 contact "
                     "words, the next own word and the occupancy word loaded, one word stored per 32-tube "
                     "word step); peak = 152 SMs x 128 B/clock x the median SM clock (derived, not "
                     f"measured); {shape['clusters']} clusters of {shape['cluster_size']} CTAs occupy "
                     f"{shape['clusters'] * shape['cluster_size']} SMs"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"], line["parity"] = large_cpu_leg(args, host, ps, block, sorted(set(blocks)))
    return line


def large_cpu_leg(args, host, ps, block, seen):
    """The oracle on the host cores: Markov mode timed on a bounded sample
    (cpu_baseline), plus BFS on the first block at every p; both compared with
    the CUDA path's outputs of the same configurations (parity)."""
    import oracle
    threads = os.cpu_count() or 1
    avail = len(seen) * block if seen == list(range(len(seen))) else block
    n_m = max(1, min(args.cpu_configs or threads, avail))
    p0 = ps[0]
    ref, su_m, tm = markov_sample_large(p0, 0, n_m, threads)
    t0 = time.perf_counter()
    bfs = {p: oracle.inspect(LW, LL, p=p, seed=LSEED, cfg0=0, n=block, mode="bfs", threads=threads)
           for p in ps}
    tb = time.perf_counter() - t0
    su_b = sum(site_updates(LA, LL, r["verdict"], r["first_hit"], r["m_stop"]) for r in bfs.values())
    cpu = {"value": su_m / tm, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"Markov mode (explicit FP64 CSR over the whole lattice every step) on configurations "
                     f"0..{n_m - 1} at p = {p0}, {tm:.1f} s; the p = 0.1533 and 0.17 configurations take "
                     f"~45 s and ~30 min each in this mode",
           "bfs_route": {"configs_per_s": len(ps) * block / tb, "seconds": tb,
                         "sample": f"configurations 0..{block - 1} at every p",
                         "note": "breadth-first search: verdict, first_hit and m_stop only, no mass; "
                                 f"the Markov site-updates of these configurations would be {su_b:.3e}"}}
    bad, n_cmp, n_gpu, n_ref = 0, 0, 0, 0
    for p in ps:
        g, r = host[p], bfs[p]
        same = ((g["verdict"][:block].astype(np.int32) == r["verdict"]) & (g["first_hit"][:block] == r["first_hit"])
                & (g["m_stop"][:block] == r["m_stop"]))
        bad += int((~same).sum()); n_cmp += block
        n_gpu += int(g["verdict"][:block].sum()); n_ref += int(r["verdict"].sum())
    g = host[p0]
    same = ((g["verdict"][:n_m].astype(np.int32) == ref["verdict"]) & (g["first_hit"][:n_m] == ref["first_hit"])
            & (g["m_stop"][:n_m] == ref["m_stop"]))
    bad_m = int((~same).sum())
    err = float(np.abs(g["mass"][:n_m].astype(np.float64) - ref["mass"]).max(initial=0.0))
    parity = {"configs": n_cmp + n_m, "routes": f"BFS: {n_cmp} configurations (block 0 at every p); "
                                                f"Markov: {n_m} at p = {p0}",
              "mismatched_configs": bad + bad_m, "mass_max_abs_err": err, "mass_tolerance": 1e-5,
              "percolating_bfs_sample": [n_gpu, n_ref],
              "ok": bad + bad_m == 0 and err <= 1e-5 and n_gpu == n_ref}
    return cpu, parity


def run_batch(args, pc, torch):
    """28 (W, L) queries of the finite-size-scaling set, 10^4 configurations
    each at p = 0.1533, seed 3: one batched submission (cached CUDA graph)
    against 28 plain one-lattice-per-launch calls."""
    specs = batching_specs(args.batch_configs)
    stream = torch.cuda.current_stream()
    queries, outs = pc.batch_queries(specs, device=True)
    plain_outs = [pc._alloc_outputs(sp[5], True, pc.ALL_OUTPUTS) for sp in specs]

    def batched():
        pc.pc_batch_run(specs, device=True, async_=True, stream=stream, outs=outs, queries=queries)

    def plain():
        for sp, o in zip(specs, plain_outs):
            W_, L_, p_, seed_, b_, n_ = sp
            pc.pc_inspect(W_, L_, p_, seed_, b_, n_, device=True, out=o, stream=stream)

    def timed(fn, steps):
        ts = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream); fn(); e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        return float(np.mean(ts))

    for _ in range(args.warmup):
        batched(); plain()
    torch.cuda.synchronize()
    with Clocks(0) as clk:
        tb = timed(batched, args.steps)
        tp = timed(plain, args.steps)
    # where the plain time goes: each per-size launch timed alone, with its
    # site-update rate and solver
    per_query_ms, per_query_su_s = {}, {}
    for sp, o in zip(specs, plain_outs):
        W_, L_, p_, seed_, b_, n_ = sp
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pc.pc_inspect(W_, L_, p_, seed_, b_, n_, device=True, out=o, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        h = {k: v.cpu().numpy() for k, v in o.items()}
        su_q = site_updates(3 * W_ * (W_ + 1) + 1, L_, h["verdict"], h["first_hit"], h["m_stop"])
        per_query_ms[f"{W_},{L_}"] = round(ms, 3)
        per_query_su_s[f"{W_},{L_}"] = float(f"{su_q / (ms / 1e3):.4g}")
    # a naive GPU path for contrast: one configuration per launch, on a
    # sample of each size's configurations (extrapolated per configuration)
    n_one = 8
    t_one = 0.0
    one = pc._alloc_outputs(1, True, pc.ALL_OUTPUTS)
    for sp in specs:
        W_, L_, p_, seed_, b_, n_ = sp
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for c in range(n_one):
            pc.pc_inspect(W_, L_, p_, seed_, b_ + c, 1, device=True, out=one, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        t_one += e0.elapsed_time(e1) / 1e3 / n_one * n_
    su, n_tot, same = 0, 0, True
    for sp, o, po in zip(specs, outs, plain_outs):
        W_, L_ = sp[0], sp[1]
        h = {k: v.cpu().numpy() for k, v in o.items()}
        hp = {k: v.cpu().numpy() for k, v in po.items()}
        same &= all(np.array_equal(h[k], hp[k]) for k in ("verdict", "first_hit", "m_stop"))
        su += site_updates(3 * W_ * (W_ + 1) + 1, L_, h["verdict"], h["first_hit"], h["m_stop"])
        n_tot += sp[5]
    return {
        "metric": "configs/s (batched)", "value": n_tot / tb, "unit": "configs/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tb * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "batching W in {4,8,16,32} x L/W in {1..64}, p=0.1533, seed=3",
                   "queries": len(specs), "configs_per_query": args.batch_configs,
                   "l2": "no flush (per-launch working sets differ; see plain)"},
        "plain_configs_per_s": n_tot / tp, "batched_over_plain": tp / tb,
        "plain_ms_per_query": per_query_ms, "plain_site_updates_per_s": per_query_su_s,
        "one_config_per_launch": {"configs_per_s": n_tot / t_one, "batched_over": t_one / tb,
                                  "sample": f"first {n_one} configurations of each size, extrapolated"},
        "site_updates_per_s_batched": su / tb, "results_identical": bool(same),
        "clocks": clk.summary(),
    }


def serving_specs(n_queries: int, seed: int = 5):
    """The serving query stream (seed 5): W ~ U{4..64}, L = round(W e^U(0, ln 64)),
    p ~ U[0.12, 0.19], n_configs = round(e^U(ln 100, ln 10^4)); the first
    n_queries queries, and the Poisson arrival gaps (unit rate) of the stream."""
    rng = np.random.default_rng(seed)
    specs, gaps = [], []
    for i in range(n_queries):
        W_ = int(rng.integers(4, 65))
        L_ = int(round(W_ * np.exp(rng.uniform(0.0, np.log(64.0)))))
        p_ = float(rng.uniform(0.12, 0.19))
        n_ = int(round(np.exp(rng.uniform(np.log(100.0), np.log(1e4)))))
        specs.append((W_, max(L_, 1), p_, seed, 0, n_))
    arr = np.random.default_rng(seed + 1000)
    gaps = arr.exponential(1.0, size=n_queries)
    return specs, gaps


def run_serving(args, pc, torch):
    specs, gaps = serving_specs(args.serve_queries)
    n_tot = sum(sp[5] for sp in specs)
    # plain: one query after another through pc_inspect
    for sp in specs[:2]:
        pc.pc_inspect(*sp)
    torch.cuda.synchronize()
    svc, plain = [], []
    for sp in specs:
        t0 = time.perf_counter()
        plain.append(pc.pc_inspect(*sp))
        svc.append(time.perf_counter() - t0)
    t_plain = float(sum(svc))
    # at most 1,024 slots a query in a 128 GB arena: a cap of 4,096 (200 GB)
    # helps a short prefix (40 queries: 4,264 against 3,086 configurations/s
    # at saturation) but lets one large query hold the arena and stop
    # admission behind it on a longer one (100 queries: 512 against 590,
    # open-loop p99 193 against 93 s)
    opts = dict(hbm_budget_bytes=args.serve_budget_gb << 30, max_slots=4096,
                max_slots_per_query=args.serve_slots_per_query, ticks_per_poll=8, max_W=64)

    def serve(arrivals):
        srv = pc.Server(**opts)
        try:
            t0 = time.perf_counter()
            tickets = []
            for sp, ta in zip(specs, arrivals):
                while time.perf_counter() - t0 < ta:
                    time.sleep(min(0.001, ta - (time.perf_counter() - t0)))
                tickets.append(srv.submit(sp))
            res = {}
            while len(res) < len(tickets):
                for t in tickets:
                    if t not in res:
                        r = srv.poll(t, timeout_s=0.002)
                        if r is not None:
                            res[t] = r
            st = srv.stats()
        finally:
            srv.close()
        return [res[t] for t in tickets], st

    with Clocks(0) as clk:
        sat, st_sat = serve([0.0] * len(specs))
        lam = 0.7 * len(specs) / t_plain  # queries per second at 70% of plain capacity
        arrivals = np.cumsum(gaps) / lam
        arrivals -= arrivals[0]
        _, st_open = serve(list(arrivals))
    same = all(np.array_equal(a["verdict"], b["verdict"]) and np.array_equal(a["first_hit"], b["first_hit"])
               and np.array_equal(a["m_stop"], b["m_stop"]) for a, b in zip(sat, plain))
    # a plain FIFO server on the same arrivals with the measured service times
    t_free, lat = 0.0, []
    for ta, sv in zip(arrivals, svc):
        start = max(ta, t_free)
        t_free = start + sv
        lat.append((t_free - ta) * 1e3)
    lat = np.sort(np.array(lat))
    pq = lambda a, f: float(a[min(len(a) - 1, int(round(f * (len(a) - 1))))])
    return {
        "metric": "configs/s (served)", "value": st_sat["configs_per_s"], "unit": "configs/s",
        "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": n_tot / st_sat["configs_per_s"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"serving stream seed=5, first {len(specs)} queries "
                               f"({n_tot} configurations)", "server": opts,
                   "arrival_rate_qps": lam, "l2": "n/a (mixed working sets)"},
        "plain_configs_per_s": n_tot / t_plain, "served_over_plain": t_plain * st_sat["configs_per_s"] / n_tot,
        "open_loop": {"p50_ms": st_open["p50_ms"], "p99_ms": st_open["p99_ms"],
                      "mean_ms": st_open["mean_ms"], "configs_per_s": st_open["configs_per_s"]},
        "plain_fifo_same_arrivals": {"p50_ms": pq(lat, 0.5), "p99_ms": pq(lat, 0.99)},
        "saturation_latency": {"p50_ms": st_sat["p50_ms"], "p99_ms": st_sat["p99_ms"]},
        "results_identical": bool(same), "clocks": clk.summary(),
    }


def run_fss(args, pc, torch):
    """Finite-size scaling (Sec. III, Eqs. (5)-(9)): Pi(p) of 35 sizes,
    W in {4, 6, 8, 12, 16, 24, 32} x W/L in {2, 1, 1/2, 1/4, 1/8}, seed 6
    (256 configurations per p on a coarse grid, 1024 per p at 13 values
    around each transition, verdicts only), fitted for p_c_inf and alpha."""
    from paper_1401_2130_gb300 import fss
    sizes = [(Wf, int(Wf / r)) for Wf in (4, 6, 8, 12, 16, 24, 32) for r in (2.0, 1.0, 0.5, 0.25, 0.125)
             if int(Wf / r) >= 2]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    curves = fss.scan(sizes, seed=6)
    t = time.perf_counter() - t0
    n_cfg = len(sizes) * (len(fss.COARSE_P) * 256 + 13 * 1024)
    fits = {}
    for wmin in (4, 8, 12):
        sub_ = {k: v for k, v in curves.items() if k[0] >= wmin}
        f, law = fss.extrapolate(sub_)
        fits[f"W>={wmin}"] = {"p_c_inf": f.p_inf, "p_c_inf_err": f.p_inf_err, "chi2": f.chi2, "dof": f.dof,
                              "C0_C1_alpha": None if law is None else law[0]}
    best = fits["W>=12"]
    return {
        "metric": "p_c_inf", "value": best["p_c_inf"], "unit": "probability", "n_gpus": 1, "steps": 1,
        "warmup": 0, "ms_per_step": t * 1e3, "higher_is_better": None, "scaling": "weak",
        "vs_baseline": None, "dtype": "bits", "data": "synthetic",
        "config": {"workload": "finite-size scaling, W in {4..32} x W/L in {2..1/8}, seed 6",
                   "sizes": len(sizes), "configurations": n_cfg},
        "configs_per_s": n_cfg / t,
        "paper": {"p_c_inf": 0.1533, "p_c_inf_err": 0.0013, "alpha": -1.23, "C0": -0.83, "C1": 0.31},
        "fits": fits,
        "p_c": {f"{k[0]},{k[1]}": [v[0].p_c, v[0].p_c_err] for k, v in sorted(curves.items())},
    }


def run_psweep(args, pc, torch, rank, world, local, dist):
    """W = 8, L = 64 p-sweep through the shared-memory resident solver (one
    launch per p, 10^4 configurations each)."""
    n_cfg = args.configs_per_p
    cfg0, _ = shard_range(rank, n_cfg)
    stream = torch.cuda.current_stream()
    outs = [pc._alloc_outputs(n_cfg, True, pc.ALL_OUTPUTS) for _ in PS]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def one_step(evs=None):
        for i, p in enumerate(PS):
            if evs is not None:
                evs[i][0].record(stream)
            pc.pc_inspect(W, L, p, SEED, cfg0, n_cfg, device=True, out=outs[i], stream=stream,
                          verdict_first=args.verdict_first)
            if evs is not None:
                evs[i][1].record(stream)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    # per-configuration work of one step (identical every step: same inputs);
    # with --verdict-first the FP32 recursion runs on percolating ones only
    su_step, su_fp = 0, 0
    for i, p in enumerate(PS):
        o = {k: v.cpu().numpy() for k, v in outs[i].items()}
        su_step += site_updates(A_COLS, L, o["verdict"], o["first_hit"], o["m_stop"])
        pm = o["verdict"] != 0
        su_fp += site_updates(A_COLS, L, o["verdict"][pm], o["first_hit"][pm], o["m_stop"][pm])
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
    # the units all ranks processed (each rank inspects its own configurations)
    su_all = su_step
    if dist is not None:
        st_ = torch.tensor([su_step], dtype=torch.float64, device="cuda")
        dist.all_reduce(st_, op=dist.ReduceOp.SUM)
        su_all = int(st_.item())
    value = su_all / t_step

    # end to end through the public call with host outputs (D2H inside)
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for p in PS:
            pc.pc_inspect(W, L, p, SEED, cfg0, n_cfg, device=False, verdict_first=args.verdict_first)
    e2e_t = (time.perf_counter() - t0) / e2e_steps
    if dist is not None:
        tt = torch.tensor([e2e_t], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_t = float(tt.item())
    d2h = len(PS) * (n_cfg * (1 + 4 + 4 + 4) + 8)

    peaks = measured_peaks()
    clocks = clk.summary()
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    sm_max = peaks.get("sm_max_mhz") or clocks.get("sm_max_mhz") or 2070.0
    smem_peak = nsm * 128 * sm_max * 1e6 / 1e9  # GB/s: 32 banks x 4 B per clock per SM
    t_launch = sum(launch_ms) / len(step_ms) / 1e3  # resident launches of one step
    achieved = HBM_BYTES_PER_SU * su_step / t_launch / 1e9
    gather = SMEM_BYTES_PER_SU * su_step / t_launch / 1e9

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": ("p-sweep W=8 L=64 p=0.100..0.200/0.005 seed=2" if len(PS) > 1 else
                                f"p-sweep subset W=8 L=64 p={PS[0]} seed=2"),
                   "W": W, "L": L, "n_p": len(PS), "configs_per_p": n_cfg,
                   "configs_per_step": n_cfg * len(PS) * world,
                   "site_updates_per_step": su_all,
                   "percolating_per_p": n_perc, "solver": "resident",
                   "l2": "flushed between steps (256 MiB write, outside the timed events)",
                   "parallelism": f"configs sharded over {world} GPU(s)"},
        "configs_per_s": n_cfg * len(PS) * world / t_step,
        "roofline": {"bound": "smem", "achieved": achieved, "peak": smem_peak, "unit": "GB/s",
                     "frac": achieved / smem_peak, "traffic": RESIDENT_DRAM_BYTES_PER_LAUNCH,
                     "traffic_note": "HBM bytes per resident_kernel launch (ncu): the state lives in "
                                     "shared memory, HBM carries tables and outputs only",
                     "model": f"{HBM_BYTES_PER_SU} B per site update (nu read and write, occupancy, "
                              f"reached-set bits) / CUDA-event time of the step's launches; peak = "
                              f"{nsm} SMs x 128 B/clk x {sm_max:.0f} MHz (derived shared-memory rate)",
                     # the same throughput under the gather form of Eq. (3):
                     # 14 neighbour reads, 1/deg and the write, 4 B each
                     "gather_model": {"bytes_per_su": SMEM_BYTES_PER_SU, "achieved": gather,
                                      "frac": gather / smem_peak}},
        "clocks": clocks,
        "e2e": {"value": su_all / e2e_t, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": len(PS) * args.steps,
        "per_p_ms": [float(np.mean(launch_ms[i::len(PS)])) for i in range(len(PS))],
        "wall_s_timed": wall,
    }
    if args.verdict_first:
        # the reached set runs over every configuration's causal window, the
        # FP32 recursion over the percolating ones' only: report configurations
        # per second, and the site-updates each part performed
        t_launch = sum(launch_ms) / len(step_ms) / 1e3
        line["metric"], line["unit"] = "configs/s", "configs/s"
        line["value"] = n_cfg * len(PS) * world / t_step
        line["config"]["mode"] = "verdict first (PC_VERDICT_FIRST)"
        line["site_updates_per_s"] = {"fp32_performed": su_fp / t_launch, "reached_set": su_step / t_launch,
                                      "single_pass_equivalent": su_step / t_launch}
        bytes_ = HBM_BYTES_PER_SU * su_fp + BITS_BYTES_PER_SU * su_step
        line["roofline"]["achieved"] = bytes_ / t_launch / 1e9
        line["roofline"]["frac"] = line["roofline"]["achieved"] / line["roofline"]["peak"]
        line["roofline"]["model"] = (f"{HBM_BYTES_PER_SU} B per FP32 site-update performed + "
                                     f"{BITS_BYTES_PER_SU} B per reached-set site-update / CUDA-event time; "
                                     + line["roofline"]["model"].split("; ", 1)[1])
        line["roofline"].pop("gather_model", None)
        line["e2e"]["value"] = n_cfg * len(PS) * world / e2e_t
        line["e2e"]["unit"] = "configs/s"
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        refs = []
        su, t = cpu_sample(args.cpu_per_p, threads, results=refs)
        line["cpu_baseline"] = {"value": su / t, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"{args.cpu_per_p} configurations per p x {len(PS)} p, "
                                          f"Markov mode (FP64 CSR), {t:.1f} s"}
        if args.verdict_first:
            line["cpu_baseline"]["value"] = args.cpu_per_p * len(PS) / t
            line["cpu_baseline"]["unit"] = "configs/s"
        # verdict and Pi parity on the same sample (first configurations of
        # the timed workload)
        try:
            line["parity"] = sample_parity(pc, refs, args.cpu_per_p,
                                           **({"verdict_first": True} if args.verdict_first else {}))
        except Exception as e:  # reported in the line, never silently dropped
            line["parity"] = {"ok": False, "error": repr(e)}
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="large", choices=["large", "psweep", "batch", "serving", "fss"])
    ap.add_argument("--ref-per-p", type=int, default=1000, help="psweep reference arm: configurations per p")
    ap.add_argument("--ref-configs", type=int, default=0,
                    help="large reference arm: Markov configurations per step (0 = one per core)")
    ap.add_argument("--cpu-per-p", type=int, default=N_CFG)
    ap.add_argument("--cpu-configs", type=int, default=0,
                    help="large line's cpu_baseline: Markov configurations (0 = one per core)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--configs-per-p", type=int, default=N_CFG,
                    help="smaller cases for profiling only; the benchmark workload is 10^4")
    ap.add_argument("--serve-queries", type=int, default=100)
    ap.add_argument("--serve-budget-gb", type=int, default=128)
    ap.add_argument("--serve-slots-per-query", type=int, default=1024)
    ap.add_argument("--large-configs", type=int, default=64)
    ap.add_argument("--large-block", type=int, default=8,
                    help="configurations per p in one step of the large workload")
    ap.add_argument("--e2e-steps", type=int, default=2,
                    help="large workload: steps timed end to end with host outputs (0 = none, profiling only)")
    ap.add_argument("--batch-configs", type=int, default=10_000)
    ap.add_argument("--verdict-first", action="store_true",
                    help="psweep: PC_VERDICT_FIRST (FP32 recursion on percolating configurations only)")
    ap.add_argument("--bits-only", action="store_true",
                    help="verdicts only (PC_BITS_ONLY): the reached-set propagation without the FP32 recursion")
    ap.add_argument("--large-p", default=None,
                    help="comma list of p for the large workload (a profiling subset)")
    ap.add_argument("--only-p", type=float, default=None,
                    help="p-sweep at this one p (a profiling subset, not the benchmark workload)")
    args = ap.parse_args()
    global PS
    if args.only_p is not None:
        PS = [args.only_p]
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("batch", "serving", "fss"):
        import torch
        import paper_1401_2130_gb300 as pc
        torch.cuda.set_device(0)
        pc.build()
        pc.load()
        fn = {"batch": run_batch, "serving": run_serving, "fss": run_fss}[args.workload]
        print(json.dumps(fn(args, pc, torch)), flush=True)
        return 0

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
    fn = run_large if args.workload == "large" else run_psweep
    line = fn(args, pc, torch, rank, world, local, dist)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
