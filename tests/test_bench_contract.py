"""bench.py's reference arm runs the CPU oracle only, so its JSON line can be
checked without a GPU: the contract's keys, the oracle baseline block, and the
multi-rank rule (only rank 0 prints; other ranks exit 0 without work)."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, *args):
    env = dict(os.environ, **(extra_env or {}))
    args = args or ("--workload", "psweep", "--ref-per-p", "5")
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--steps", "1", "--warmup", "0", *args],
                          capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)


def _check_line(r):
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e",
              "cpu_baseline", "impl"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == "site-updates/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    return d


def test_reference_arm_large_workload_line():
    """The default workload's reference arm: the oracle's Markov mode on the
    W = 64, L = 4096 lattice, one configuration per step here."""
    d = _check_line(_run(None, "--ref-configs", "1"))
    assert "W=64 L=4096" in d["config"]["workload"]


def test_reference_arm_prints_one_contract_line():
    r = _run()
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e",
              "cpu_baseline", "impl"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == "site-updates/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_reference_arm_other_ranks_exit_quietly():
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not r.stdout.strip()


def test_sample_parity_block_flags_any_difference():
    # the psweep line's "parity" block: the CUDA outputs on the oracle's own
    # sample; a planted difference in one configuration must be reported
    import importlib
    import numpy as np
    sys.path.insert(0, ROOT)
    bench = importlib.import_module("bench")
    refs = []
    bench.cpu_sample(4, 2, results=refs)
    by_p = dict(zip(bench.PS, refs))

    class Fake:
        plant = None

        def pc_inspect(self, W, L, p, seed, b, n):
            r = by_p[p]
            out = {"verdict": r["verdict"].astype(np.uint8), "first_hit": r["first_hit"].copy(),
                   "m_stop": r["m_stop"].copy(), "mass": r["mass"].astype(np.float32),
                   "n_percolating": int(r["verdict"].sum())}
            if self.plant == p:
                out["m_stop"][0] += 1
            return out

    f = Fake()
    ok = bench.sample_parity(f, refs, 4)
    assert ok["ok"] and ok["mismatched_configs"] == 0 and ok["configs"] == 4 * len(bench.PS)
    f.plant = bench.PS[7]
    bad = bench.sample_parity(f, refs, 4)
    assert not bad["ok"] and bad["mismatched_configs"] == 1


def test_launch_accounting_follows_the_solvers_tick_rules():
    """gpu_launches of the large lines is counted from the outputs: the
    streamed solver runs a draw tick, a preparation tick and one tick per
    step of the longest configuration; the blocked verdict-only solver a draw
    tick and one pass per 32 steps (its pass planner is simulated on the CPU
    in test_host_parts), each tick one pass and one control kernel after one
    init kernel."""
    sys.path.insert(0, ROOT)
    import bench
    import numpy as np
    # three configurations: percolating at first_hit 100 (last step 99),
    # stopping at m_stop 33, and none metallic at t = 0 (m_stop 0)
    v = np.array([1, 0, 0]); fh = np.array([100, -1, -1]); ms = np.array([100, 33, 0])
    assert bench.solve_ticks(v, fh, ms) == 99 + 3
    # passes: step 99 lies in pass (99 - 1) // 32 + 1 = 4, step 33 in pass 2
    assert bench.blocked_launches(v, fh, ms) == 1 + 2 * (1 + 4)
    # a step exactly at a pass boundary: step 32 is the last of pass 1, 33 the first of pass 2
    assert bench.blocked_launches(np.array([0]), np.array([-1]), np.array([32])) == 1 + 2 * 2
    assert bench.blocked_launches(np.array([0]), np.array([-1]), np.array([33])) == 1 + 2 * 3
    assert bench.blocked_launches(np.array([0]), np.array([-1]), np.array([0])) == 1 + 2 * 1
