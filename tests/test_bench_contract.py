"""bench.py's main measurement flow on the CPU, with the device calls replaced
by stand-ins: the JSON line it prints carries every key of the benchmark
contract (metric, value, unit, steps, timing, roofline, clocks, e2e, launches)
and its derived numbers follow from the timed work.  The stand-in solver
returns the float64 series as the estimate and fixed walk statistics; no
library or GPU code runs here (the GPU path is covered by the -m gpu tests)."""
import io
import json
import os
import sys
import time
import types
from contextlib import redirect_stdout

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import reference as R  # noqa: E402

STEPS_PER_SOLVE = 1_000_000
WALKS_PER_SOLVE = 100_000
KERNEL_MS = 2.0


class _Event:
    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream=None):
        self.t = time.perf_counter()

    def elapsed_time(self, other):
        return (other.t - self.t) * 1000.0


class _Graph:
    def __init__(self, n):
        self.n = n
        self.closed = False

    def close(self):
        self.closed = True


LAUNCHES_PER_SOLVE = 17
GATHER = 4.0e10


def _fake_library(g):
    M = types.SimpleNamespace(MCF_F32W_F64ACC=1)
    M.load = lambda: None
    M.launches = 0
    M.mcf_kernel_launches = lambda: M.launches
    M.mcf_gather_probe = lambda nbytes, reads, stream=None: GATHER
    M.mcf_create_graph = lambda n, rp, ci, *a, **k: _Graph(n)
    M.mcf_spectral_radius = lambda h, tol=1e-10, max_iter=1000: R.lambda_max(g)

    def solve(h, coeffs, out=None, stats=False, scale=1.0, **kw):
        M.launches += LAUNCHES_PER_SOLVE
        y = R.series_action(g, coeffs, scale)
        out.copy_(torch.from_numpy(y))
        st = {"walks": WALKS_PER_SOLVE, "walk_steps": STEPS_PER_SOLVE, "kernel_ms": KERNEL_MS, "flags": 0,
              "max_rel_se": 0.0}
        return (out, st) if stats else out

    M.mcf_total_communicability = solve
    M.mcf_subgraph_centrality = solve
    return M


def test_main_prints_one_contract_line(monkeypatch):
    w = bench.WORKLOADS["ba1000_tc"]
    g = bench.make_graph(w)
    fake = _fake_library(g)
    import paper_2308_01037_gb300 as pkg

    monkeypatch.setitem(sys.modules, "paper_2308_01037_gb300.mcf", fake)
    monkeypatch.setattr(pkg, "mcf", fake, raising=False)
    monkeypatch.setattr(torch.cuda, "set_device", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a, **k: types.SimpleNamespace(cuda_stream=0))
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.Tensor, "cuda", lambda self, *a, **k: self)
    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self, *a, **k: self)
    real_empty = torch.empty

    def empty(*a, device=None, **k):
        return real_empty(*a, **k)

    monkeypatch.setattr(torch, "empty", empty)
    monkeypatch.setitem(bench.NCU_DRAM_BYTES_PER_STEP, "ba1000_tc", 32.0)
    for key in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(key, raising=False)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "ba1000_tc", "--steps", "3", "--warmup", "3",
                                      "--e2e-steps", "2", "--no-cpu-baseline", "--no-batch"])
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.main()
    lines = [ln for ln in buf.getvalue().splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "clocks", "e2e", "gpu_launches",
                "cpu_baseline"):
        assert key in d, key
    assert d["metric"] == d["unit"] == "walk-steps/s" and d["n_gpus"] == 1 and d["steps"] == 3
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["data"] == "synthetic"
    assert d["config"]["workload"] == w["label"]
    # value = all walk steps of the timed solves / the timed region
    assert d["value"] == pytest.approx(STEPS_PER_SOLVE / (d["ms_per_step"] / 1000.0), rel=1e-9)
    assert d["gpu_launches"] == 3 * LAUNCHES_PER_SOLVE      # counted over the timed solves only
    assert d["roofline"]["gather_ceiling"] == GATHER
    assert d["roofline"]["frac_of_gather_ceiling"] == pytest.approx(STEPS_PER_SOLVE / (KERNEL_MS / 1000.0) / GATHER)
    rf = d["roofline"]
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and rf["kernel"] == "walk_tc_kernel"
    achieved = 16 * STEPS_PER_SOLVE / (KERNEL_MS / 1000.0) / 1e9
    assert rf["achieved"] == pytest.approx(achieved) and rf["frac"] == pytest.approx(achieved / rf["peak"])
    assert rf["traffic"] == pytest.approx(32.0 * STEPS_PER_SOLVE)
    assert rf["useful_bytes_fraction"] == pytest.approx(0.5)
    assert rf["dram_gbs"] == pytest.approx(2 * achieved) and rf["dram_frac"] == pytest.approx(2 * rf["frac"])
    e2e = d["e2e"]
    assert e2e["unit"] == "walk-steps/s" and e2e["value"] > 0
    assert e2e["h2d_bytes_per_step"] == (g.n + 1) * 8 + g.nnz * 4   # row_ptr int64 + col_idx int32
    assert e2e["d2h_bytes_per_step"] == g.n * 8
    assert d["rel_err_vs_fp64"] == pytest.approx(0.0, abs=1e-15)
    assert d["clocks"]["samples"] >= 0 and "reasons" in d["clocks"]
    assert np.isfinite(d["solves_per_s"])
