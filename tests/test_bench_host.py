"""Host-side parts of bench.py on the CPU: the oracle pool that times the
oracle on several host processes, and the reference arm's JSON line."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import estimator as E  # noqa: E402
from oracle import reference as R  # noqa: E402
from paper_2308_01037_gb300 import inputs as I  # noqa: E402


def test_oracle_pool_counts_the_oracles_steps():
    """Two spawn-started workers over the CSR in shared memory run the
    unchanged oracle; the steps they report for a node sample are the steps
    the oracle reports in this process for the same nodes."""
    g = I.barabasi_albert(300, 3, 1)
    w = dict(bench.WORKLOADS["ba1000_tc"], walks_per_node=50)
    lam = R.lambda_max(g)
    pool = bench.OraclePool(g, w, procs=2)
    try:
        nodes = np.array([0, 5, 299], np.int64)
        got = pool.pool.map(bench._oracle_worker_task, [(nodes, lam), (nodes, lam)])
        res = pool.run(lam, 0.2)
    finally:
        pool.close()
    ref = E.action(g, bench.exp_coeffs(w["K"]), gamma=1.0 / lam, walks_per_node=50, seed=1, nodes=nodes,
                   precision=1)["steps"]
    assert got == [ref, ref]
    assert res["cores"] == 2 and res["value"] > 0 and "2 processes" in res["sample"]


@pytest.mark.timeout(300)
def test_reference_arm_prints_one_json_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "ba1000_tc",
           "--steps", "2", "--warmup", "0", "--ref-seconds", "3"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=280, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["cores"] >= 1 and d["e2e"]["h2d_bytes_per_step"] == 0


def test_clock_summary_parses_nvidia_smi_samples():
    """The clocks object of the bench line: median SM clock under load, the
    maximum clock, and every throttle reason seen active in any sample."""
    c = bench.ClockSampler(0)
    c.lines = [
        "0, 1980, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 1100.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2010, 2070, 1000.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = c.summary()
    assert s == {"sm_mhz": 2010.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c.lines = ["0, 1500, 2070, 1.0, 0x8, Active, Not Active, Active, Not Active"]
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    c.lines = []
    assert c.summary()["samples"] == 0


def test_reference_arm_other_ranks_exit_without_work():
    """Under torchrun only rank 0 times the oracle and prints; another rank exits 0 silently."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "ba1000_tc",
           "--steps", "1", "--warmup", "0", "--ref-seconds", "1"]
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=120, cwd=ROOT, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    assert not [ln for ln in out.stdout.splitlines() if ln.startswith("{")]


def test_bench_runs_the_oracle_only_in_its_baseline_and_reference_legs():
    """Every import of oracle/ in bench.py sits in the CPU-baseline functions or
    the reference arm; the accuracy figures use bench's own float64 series,
    which equal the oracle's on a small graph."""
    import ast

    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    allowed = {"cpu_baseline", "cpu_baseline_all_cores", "_oracle_worker_init", "_oracle_worker_task", "run_reference"}
    found = []
    for fn in ast.walk(tree):
        if isinstance(fn, ast.FunctionDef):
            for node in ast.walk(fn):
                if isinstance(node, (ast.Import, ast.ImportFrom)):
                    mod = node.module if isinstance(node, ast.ImportFrom) else node.names[0].name
                    if mod and mod.split(".")[0] == "oracle":
                        found.append(fn.name)
    top = [n for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))
           and ((n.module if isinstance(n, ast.ImportFrom) else n.names[0].name) or "").split(".")[0] == "oracle"]
    assert not top and found and set(found) <= allowed, found
    g = I.rmat(9, 8, seed=2)
    c = bench.exp_coeffs(20)
    lam = R.lambda_max(g)
    np.testing.assert_allclose(bench.F64Ref.series_action(g, c, 1.0 / lam), R.series_action(g, c, 1.0 / lam),
                               rtol=1e-14)
    nodes = np.array([0, 3, 100])
    np.testing.assert_allclose(bench.F64Ref.series_diag(g, c, nodes, 1.0 / lam),
                               R.series_diag(g, c, nodes, 1.0 / lam), rtol=1e-14)
