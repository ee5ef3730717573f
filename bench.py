"""Benchmark: total communicability exp(A')1 on an R-MAT graph of scale 22
(4,194,304 nodes, edge factor 16, (a,b,c) = (0.57,0.19,0.19), symmetrised,
unweighted), A' = A / lambda_max, exp truncated at K = 30, W_c = 1e-6,
N_s = 1e8 walks, float32 walk weights with float64 accumulators.

One step = one full RandFunmAction solve on the device-resident graph
(r = A'v, walk allocation, the walk kernel, the A'q epilogue).  The metric is
walk-steps/s (transitions l_k -> l_{k+1} of all walks per second); solves/s
and the relative l_inf error against the float64 truncated series are
reported beside it.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--workload NAME]

Under torchrun (N > 1) every rank solves its own requests (different request
ids) on its own GPU: independent problems, no collective on the data path,
weak scaling; the JSON line reports the whole job.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (generator kwargs, query, walk parameters)
    "rmat22_tc": dict(gen=("rmat", dict(scale=22, edge_factor=16, seed=1)), query="tc",
                      n_walks=100_000_000, walks_per_node=0, w_cutoff=1e-6, K=30,
                      label="total communicability exp(A/lambda_max)1, R-MAT scale 22 ef16 (0.57,0.19,0.19), "
                            "1e8 walks, K=30, W_c=1e-6"),
    "rmat21_tc": dict(gen=("rmat", dict(scale=21, edge_factor=16, seed=1)), query="tc",
                      n_walks=25_000_000, walks_per_node=0, w_cutoff=1e-6, K=30,
                      label="total communicability exp(A/lambda_max)1, R-MAT scale 21 ef16 (0.57,0.19,0.19), "
                            "2.5e7 walks, K=30, W_c=1e-6 (profiling case)"),
    "ba1000_tc": dict(gen=("barabasi_albert", dict(n=1000, m=3, seed=0)), query="tc",
                      n_walks=0, walks_per_node=100_000, w_cutoff=0.0, K=30,
                      label="total communicability exp(A/lambda_max)1, BA n=1000 m=3, 1e5 walks per node, K=30"),
    "ba1000_sc": dict(gen=("barabasi_albert", dict(n=1000, m=3, seed=0)), query="sc",
                      n_walks=0, walks_per_node=100_000, w_cutoff=0.0, K=30,
                      label="subgraph centrality diag exp(A/lambda_max), BA n=1000 m=3, 1e5 walks per node, K=30"),
    "cm2m_sc_w100": dict(gen=("config_powerlaw", dict(n=2_000_000, exponent=2.5, mean_degree=20.0, seed=2)),
                         query="sc", n_walks=0, walks_per_node=100, w_cutoff=1e-6, K=30,
                         label="subgraph centrality diag exp(A/lambda_max), configuration model n=2e6 k^-2.5 mean 20, "
                               "100 walks per node (timing case), K=30, W_c=1e-6"),
    "cm2m_sc": dict(gen=("config_powerlaw", dict(n=2_000_000, exponent=2.5, mean_degree=20.0, seed=2)), query="sc",
                    n_walks=0, walks_per_node=2000, w_cutoff=1e-6, K=30,
                    label="subgraph centrality diag exp(A/lambda_max), configuration model n=2e6 k^-2.5 mean 20, "
                          "2000 walks per node, K=30, W_c=1e-6"),
}

ALGO_BYTES_PER_STEP = 16  # row offset pair 8 B + column index 4 B + r_l 4 B per transition


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def make_graph(w):
    from paper_2308_01037_gb300 import inputs as I

    name, kw = w["gen"]
    t = time.time()
    g = getattr(I, name)(**kw)
    log(f"[bench] graph {g.name}: n={g.n} nnz={g.nnz} max_deg={int(g.degree.max())} ({time.time() - t:.1f}s)")
    return g


def exp_coeffs(K):
    import math

    return np.array([1.0 / math.factorial(k) for k in range(K + 1)])


class ClockSampler:
    """nvidia-smi clock/throttle samples every 100 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not mhz:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(mhz)}


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def cpu_baseline(g, lam, w, seconds=15.0):
    """The oracle (single-threaded C) on a bounded sample of the same workload:
    RandFunmAction entries for a random node sample (walks from their neighbours)."""
    from oracle import estimator as E

    c = exp_coeffs(w["K"])
    rng = np.random.default_rng(123)
    n_nodes = 64
    total_steps, total_t, sample = 0, 0.0, []
    while total_t < seconds and n_nodes <= 1 << 16:
        nodes = rng.choice(g.n, size=n_nodes, replace=False)
        t = time.perf_counter()
        out = (E.action if w["query"] == "tc" else E.diag)(
            g, c, gamma=1.0 / lam, n_walks=w["n_walks"], walks_per_node=w["walks_per_node"],
            w_cutoff=w["w_cutoff"], seed=1, nodes=nodes, **({"precision": 1}))
        dt = time.perf_counter() - t
        total_steps += out["steps"]
        total_t += dt
        sample.append(n_nodes)
        n_nodes *= 2
    return {"value": total_steps / total_t, "unit": "walk-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"entries of {sum(sample)} random nodes (walks from their neighbours, same allocation and "
                      f"seed as the full run), {total_steps} walk-steps in {total_t:.1f} s"}


def run_reference(args, w):
    """--impl reference: the oracle as it stands, timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import reference as R

    g = make_graph(w)
    lam = R.lambda_max(g)
    per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_baseline(g, lam, w, seconds=per_step / 4)
    vals = []
    t0 = time.perf_counter()
    last = None
    for _ in range(args.steps):
        last = cpu_baseline(g, lam, w, seconds=per_step)
        vals.append(last["value"])
    el = time.perf_counter() - t0
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": "walk-steps/s", "value": v, "unit": "walk-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * el / max(1, args.steps), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 walk weights, f64 accumulation", "data": "synthetic",
            "config": {"workload": w["label"]},
            "cpu_baseline": {"value": v, "unit": "walk-steps/s", "cores": 1, "kind": "oracle",
                             "sample": last["sample"] if last else ""},
            "e2e": {"value": v, "unit": "walk-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mcf", choices=["mcf", "reference"])
    ap.add_argument("--workload", default="rmat22_tc", choices=sorted(WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    from paper_2308_01037_gb300 import mcf as M

    M.load()
    g = make_graph(w)
    h = M.mcf_create_graph(g.n, torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col_idx).cuda())
    lam = M.mcf_spectral_radius(h, tol=1e-10, max_iter=10000)
    gam = 1.0 / lam
    c = exp_coeffs(w["K"])
    stream = torch.cuda.current_stream()
    out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    base = dict(scale=gam, n_walks=w["n_walks"], walks_per_node=w["walks_per_node"], w_cutoff=w["w_cutoff"],
                seed=1, precision=M.MCF_F32W_F64ACC, stream=stream.cuda_stream)
    solve = M.mcf_total_communicability if w["query"] == "tc" else M.mcf_subgraph_centrality
    log(f"[bench] lambda_max={lam:.6f}; warm-up {args.warmup}")
    for i in range(args.warmup):
        solve(h, c, out=out, request_id=1000 + i, **base)
    torch.cuda.synchronize()

    # ---- timed region: K full solves, inputs resident in HBM (CSR 4 B/nnz >> L2)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps_total, walks_total, kern_ms = 0, 0, []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for i in range(args.steps):
            _, st = solve(h, c, out=out, request_id=rank * 1_000_000 + i, stats=True, **base)
            steps_total += st["walk_steps"]
            walks_total += st["walks"]
            kern_ms.append(st["kernel_ms"])
        ev1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    tmax = ms
    steps_all = steps_total
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tmax = float(t.item())
        s = torch.tensor([float(steps_total)], device="cuda", dtype=torch.float64)
        dist.all_reduce(s)
        steps_all = float(s.item())
    value = steps_all / (tmax / 1000.0)
    solves_per_s = world * args.steps / (tmax / 1000.0)
    kernel_ms = float(np.mean(kern_ms))
    peak, peak_kind = measured_peak()
    achieved = ALGO_BYTES_PER_STEP * (steps_total / args.steps) / (kernel_ms / 1000.0) / 1e9

    # ---- accuracy of one solve against the float64 truncated series
    rel_err = None
    if not args.no_accuracy and rank == 0:
        from oracle import reference as R

        y = out.cpu().numpy()
        t = time.time()
        if w["query"] == "tc":
            ref = R.series_action(g, c, gam)
            rel_err = float(np.abs(y - ref).max() / np.abs(ref).max())
        else:
            nodes = np.random.default_rng(0).choice(g.n, size=min(g.n, 2000), replace=False)
            ref = R.series_diag(g, c, nodes, gam)
            rel_err = float(np.abs(y[nodes] - ref).max() / np.abs(ref).max())
        log(f"[bench] rel l_inf error vs float64 series: {rel_err:.3e} ({time.time() - t:.1f}s)")

    # ---- end to end through the C ABI from pinned host memory
    e2e = None
    if args.e2e_steps > 0:
        rp_h = torch.from_numpy(g.row_ptr).pin_memory()
        ci_h = torch.from_numpy(g.col_idx).pin_memory()
        y_h = torch.empty(g.n, dtype=torch.float64).pin_memory()
        hb = rp_h.numel() * 8 + ci_h.numel() * 4
        torch.cuda.synchronize()
        steps_e2e = 0
        t0 = time.perf_counter()
        for i in range(args.e2e_steps):
            he = M.mcf_create_graph(g.n, rp_h, ci_h)
            _, st = solve(he, c, out=y_h, request_id=5_000_000 + i, stats=True, **base)
            steps_e2e += st["walk_steps"]
            he.close()
        el = time.perf_counter() - t0
        e2e = {"value": steps_e2e / el, "unit": "walk-steps/s", "h2d_bytes_per_step": int(hb),
               "d2h_bytes_per_step": int(g.n * 8),
               "note": "per step: mcf_create_graph from pinned host CSR (copy + validation), the solve, "
                       "result read back to pinned host memory, mcf_destroy_graph"}
        if dist:
            t = torch.tensor([e2e["value"]], device="cuda", dtype=torch.float64)
            dist.all_reduce(t)
            e2e["value"] = float(t.item())

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(g, lam, w)
    if rank == 0:
        line = {
            "metric": "walk-steps/s", "value": value, "unit": "walk-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tmax / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 walk weights, f64 accumulation", "data": "synthetic",
            "config": {"workload": w["label"], "n": g.n, "nnz": g.nnz, "lambda_max": lam,
                       "walks_per_solve": walks_total // args.steps, "l2": "inputs larger than L2 (CSR > 129 MB)",
                       "parallelism": f"{world} independent solves per step" if world > 1 else "1 GPU"},
            "solves_per_s": solves_per_s, "rel_err_vs_fp64": rel_err,
            "walk_steps_per_solve": steps_total / args.steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                         "kernel": "walk_action_kernel", "kernel_ms": kernel_ms,
                         "algorithmic_bytes_per_step": ALGO_BYTES_PER_STEP},
            "clocks": clk.summary(), "e2e": e2e, "gpu_launches": args.steps * 16,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    h.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
