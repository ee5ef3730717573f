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
import collections
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

# Algorithmic bytes per walk step of the dominant kernel: total communicability
# reads a row offset pair 8 B + column index 4 B + r_l 4 B per transition;
# subgraph centrality reads 12 B (no r_l) and reduces into the L2-resident row Q_k.
ALGO_BYTES_PER_STEP = {"tc": 16, "sc": 12}
KERNEL = {"tc": "walk_tc_kernel", "sc": "walk_diag_od_kernel"}
# DRAM bytes (read + write) per walk step of walk_tc_kernel from one ncu
# capture of the R-MAT scale 21 profiling case with the current kernel
# (7.794e9 B over 264,240,439 steps of one launch); a launch of the larger
# case is scaled by its steps.
NCU_DRAM_BYTES_PER_STEP = {"rmat22_tc": 29.495, "rmat21_tc": 29.495}


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


class F64Ref:
    """The float64 truncated series the accuracy figures compare against:
    plain scipy sparse products written here, so that this script runs the
    oracle only in its CPU-baseline and reference legs."""

    @staticmethod
    def _matrix(g, gamma):
        import scipy.sparse as sp

        return sp.csr_matrix((np.full(g.nnz, float(gamma)), g.col_idx, g.row_ptr), shape=(g.n, g.n))

    @staticmethod
    def series_action(g, coeffs, gamma):
        """sum_k zeta_k (gamma A)^k 1 by K sparse products."""
        A = F64Ref._matrix(g, gamma)
        t = np.ones(g.n)
        y = coeffs[0] * t
        for z in coeffs[1:]:
            t = A @ t
            y = y + z * t
        return y

    @staticmethod
    def series_diag(g, coeffs, nodes, gamma, block=64):
        """(sum_k zeta_k (gamma A)^k)_ii for i in nodes, blocks of unit vectors."""
        A = F64Ref._matrix(g, gamma)
        nodes = np.asarray(nodes, dtype=np.int64)
        out = np.zeros(len(nodes))
        for b0 in range(0, len(nodes), block):
            idx = nodes[b0:b0 + block]
            cols = np.arange(len(idx))
            T = np.zeros((g.n, len(idx)))
            T[idx, cols] = 1.0
            D = coeffs[0] * T
            for z in coeffs[1:]:
                T = A @ T
                D = D + z * T
            out[b0:b0 + block] = D[idx, cols]
        return out

    @staticmethod
    def katz_coeffs(K):
        return np.ones(K + 1)

    @staticmethod
    def katz_terms_for_tail(rho, tol):
        """Smallest K >= 2 with rho^(K+1) / (1 - rho) <= tol."""
        import math

        return max(2, int(math.ceil(math.log(tol * (1.0 - rho)) / math.log(rho) - 1.0)))


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


# ---------------------------------------------------------------- the oracle on every host core
# Worker processes are started with spawn (never forked from a process that
# has used the GPU) and map the parent's CSR from shared memory; each task is
# the unchanged oracle on one node sample.
_ORC = {}


def _oracle_worker_init(shm_names, n, nnz, w):
    from multiprocessing import shared_memory

    from paper_2308_01037_gb300 import inputs as I

    rp_shm = shared_memory.SharedMemory(name=shm_names[0])
    ci_shm = shared_memory.SharedMemory(name=shm_names[1])
    rp = np.ndarray((n + 1,), dtype=np.int64, buffer=rp_shm.buf)
    ci = np.ndarray((max(nnz, 1),), dtype=np.int32, buffer=ci_shm.buf)[:nnz]
    _ORC.update(g=I.Graph(n, rp, ci, "shared"), w=w, shm=(rp_shm, ci_shm))


def _oracle_worker_task(args):
    from oracle import estimator as E

    nodes, lam = args
    g, w = _ORC["g"], _ORC["w"]
    out = (E.action if w["query"] == "tc" else E.diag)(
        g, exp_coeffs(w["K"]), gamma=1.0 / lam, n_walks=w["n_walks"], walks_per_node=w["walks_per_node"],
        w_cutoff=w["w_cutoff"], seed=1, nodes=nodes, precision=1)
    return int(out["steps"])


class OraclePool:
    """The oracle run by one spawn-started process per host core."""

    def __init__(self, g, w, procs=None):
        import multiprocessing as mp
        from multiprocessing import shared_memory

        self.procs = procs or max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
                                   else os.cpu_count() or 1)
        self.n = g.n
        self.shm = [shared_memory.SharedMemory(create=True, size=max(8, g.row_ptr.nbytes)),
                    shared_memory.SharedMemory(create=True, size=max(8, g.col_idx.nbytes))]
        np.ndarray(g.row_ptr.shape, dtype=np.int64, buffer=self.shm[0].buf)[:] = g.row_ptr
        np.ndarray(g.col_idx.shape, dtype=np.int32, buffer=self.shm[1].buf)[:] = g.col_idx
        ctx = mp.get_context("spawn")
        self.pool = ctx.Pool(self.procs, initializer=_oracle_worker_init,
                             initargs=([m.name for m in self.shm], g.n, int(g.col_idx.size), w))

    def run(self, lam, seconds, seed=123):
        rng = np.random.default_rng(seed)
        n_nodes, total_steps, total_t, entries = 8, 0, 0.0, 0
        while total_t < seconds and n_nodes <= 1 << 14:
            tasks = [(rng.choice(self.n, size=min(n_nodes, self.n), replace=False), lam) for _ in range(self.procs)]
            t = time.perf_counter()
            total_steps += sum(self.pool.map(_oracle_worker_task, tasks))
            total_t += time.perf_counter() - t
            entries += sum(len(x[0]) for x in tasks)
            n_nodes *= 2
        return {"value": total_steps / total_t, "unit": "walk-steps/s", "cores": self.procs, "kind": "oracle",
                "sample": f"entries of {entries} random nodes on {self.procs} processes (walks from their neighbours, "
                          f"same allocation and seed as the full run), {total_steps} walk-steps in {total_t:.1f} s"}

    def close(self):
        self.pool.close()
        self.pool.join()
        for m in self.shm:
            m.close()
            m.unlink()


def cpu_baseline_all_cores(g, lam, w, seconds=15.0):
    """cpu_baseline on every host core, with the single-core rate beside it."""
    one = cpu_baseline(g, lam, w, seconds=seconds / 3)
    pool = OraclePool(g, w)
    try:
        pool.run(lam, 0.5)            # start-up of the workers
        res = pool.run(lam, seconds)
    finally:
        pool.close()
    res["single_core_value"] = one["value"]
    res["single_core_sample"] = one["sample"]
    return res


def aggregate(ms, steps, device="cpu"):
    """Whole-job numbers over the ranks of the default process group: the
    slowest rank's time (ms) and the walk-steps of all ranks."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    s = torch.tensor([float(steps)], dtype=torch.float64, device=device)
    dist.all_reduce(s)
    return float(t.item()), float(s.item())


# ---------------------------------------------------------------- accuracy-targeted walk budgets
# Every batched and served query runs with a walk budget calibrated once per
# (graph, kind) from the library's error estimate (an accuracy-targeted solve
# held to two replicas of a pilot budget), aiming at half the 1e-3 bar with a
# margin on the walk count: the estimate is the spread of the error, not a
# bound.  The errors of the results are then measured against the float64
# series.
CAL_TARGET = 5e-4
CAP_WINDOW = 128   # requests a closed-loop serving client keeps outstanding
CAL_MARGIN = 1.5
KINDS = ("tc", "sc", "katz")


def calibrate(M, solve, pilot, n, cap_factor):
    """Walk budget for an estimated relative l_inf error of CAL_TARGET: two
    replicas of the pilot budget (an accuracy-targeted solve capped at two
    replicas) estimate the error e2 of their mean; the error falls like N^-1/2
    (Theorem 1), so the budget is 2 x pilot x (e2 / CAL_TARGET)^2 x CAL_MARGIN,
    at least the pilot and at most cap_factor per node.  Returns (budget,
    met: whether that budget stays within the cap, e2)."""
    key = "walks_per_node" if pilot.get("walks_per_node", 0) > 0 else "n_walks"
    per_replica = int(pilot[key]) * (1 if key == "n_walks" else n)
    _, st = solve(dict(pilot, target_rel_err=CAL_TARGET, max_walks=2 * per_replica + n))
    e2 = float(st["est_rel_err"])
    want = 2.0 * pilot[key] * (e2 / CAL_TARGET) ** 2 * CAL_MARGIN
    cap = cap_factor * (n if key == "n_walks" else 1)
    budget = int(min(max(want, pilot[key]), cap))
    return {key: budget}, want <= cap, e2


def query_solver(M, h, kind, coeffs=None, gamma=None, katz_gamma=None, nodes=None):
    """A one-argument single-query solve (kwargs -> (result, stats)) for calibration."""
    if kind == "tc":
        return lambda kw: M.mcf_total_communicability(h, coeffs, scale=gamma, stats=True, **kw)
    if kind == "katz":
        return lambda kw: M.mcf_katz(h, katz_gamma, 0, stats=True, **kw)
    return lambda kw: M.mcf_subgraph_centrality(h, coeffs, nodes=nodes, scale=gamma, stats=True, **kw)


def batch_queries(M, R, I, n_graphs, log_n_max, seed=3):
    """The mixed multi-graph workload: n = round(10^U[3, log_n_max]); half
    Barabasi-Albert (m in 2..8), half Erdos-Renyi (mean degree U[8, 32]);
    queries cycle total communicability exp(A/lambda)1, subgraph centrality
    diag exp(A/lambda) and Katz with gamma = 0.85 / lambda_max, float32 walk
    weights, each with a walk budget calibrated to 1e-3 (CAL_TARGET)."""
    rng = np.random.default_rng(seed)
    graphs, qs, cal = [], [], []
    c = exp_coeffs(30)
    t_gen = t_cal = 0.0
    for j in range(n_graphs):
        t0 = time.perf_counter()
        n = int(round(10 ** rng.uniform(3, log_n_max)))
        if j % 2 == 0:
            g = I.barabasi_albert(n, int(rng.integers(2, 9)), seed + j)
        else:
            g = I.erdos_renyi(n, float(rng.uniform(8, 32)), seed + j)
        h = M.mcf_create_graph(g.n, g.row_ptr, g.col_idx)
        lam = M.mcf_spectral_radius(h, tol=1e-10, max_iter=10000)
        graphs.append((g, h, lam))
        t1 = time.perf_counter()
        t_gen += t1 - t0
        base = dict(graph=h, seed=seed * 1000 + j, request_id=j, precision=M.MCF_F32W_F64ACC)
        kind = KINDS[j % 3]
        common = dict(seed=base["seed"], request_id=j, precision=M.MCF_F32W_F64ACC)
        if kind == "tc":
            pilot = dict(common, n_walks=16 * g.n, w_cutoff=1e-6)
            budget, met, est = calibrate(M, query_solver(M, h, "tc", c, 1.0 / lam), pilot, g.n, 8192)
            qs.append(dict(base, kind=M.MCF_QUERY_TOTAL_COMMUNICABILITY, coeffs=c, scale=1.0 / lam, w_cutoff=1e-6,
                           **budget))
        elif kind == "sc":
            pilot = dict(common, walks_per_node=4, w_cutoff=1e-6)
            budget, met, est = calibrate(M, query_solver(M, h, "sc", c, 1.0 / lam), pilot, g.n, 8192)
            qs.append(dict(base, kind=M.MCF_QUERY_SUBGRAPH_CENTRALITY, coeffs=c, scale=1.0 / lam, w_cutoff=1e-6,
                           **budget))
        else:
            kg = 0.85 / lam
            pilot = dict(common, walks_per_node=4)
            budget, met, est = calibrate(M, query_solver(M, h, "katz", katz_gamma=kg), pilot, g.n, 256)
            qs.append(dict(base, kind=M.MCF_QUERY_KATZ, katz_gamma=kg, katz_terms=0, **budget))
        per_node = list(budget.values())[0] / (g.n if "n_walks" in budget else 1)
        cal.append({"kind": kind, "n": g.n, "budget_met": met, "est_rel_err_pilot": est, "walks_per_node": per_node})
        t_cal += time.perf_counter() - t1
    log(f"[bench] batch graphs generated and uploaded in {t_gen:.1f}s, budgets calibrated in {t_cal:.1f}s")
    return graphs, qs, cal


def solve_single(M, q):
    keys = ("scale", "n_walks", "walks_per_node", "w_cutoff", "seed", "request_id", "precision")
    kw = {k: q[k] for k in keys if k in q}
    if q["kind"] == M.MCF_QUERY_TOTAL_COMMUNICABILITY:
        return M.mcf_total_communicability(q["graph"], q["coeffs"], out=q.get("out"), **kw)
    if q["kind"] == M.MCF_QUERY_KATZ:
        return M.mcf_katz(q["graph"], q["katz_gamma"], q["katz_terms"], out=q.get("out"), **kw)
    return M.mcf_subgraph_centrality(q["graph"], q["coeffs"], nodes=q.get("nodes"), out=q.get("out"), **kw)


def _kind_of(M, q):
    return {M.MCF_QUERY_TOTAL_COMMUNICABILITY: "tc", M.MCF_QUERY_KATZ: "katz",
            M.MCF_QUERY_SUBGRAPH_CENTRALITY: "sc"}[q["kind"]]


def run_batched(M, R, I, n_graphs, log_n_max, reps=1):
    """Solves/s of the batch (plain and CUDA-graph replay) against the same
    queries solved one at a time, for the whole mix and for each kind alone;
    budgets calibrated to 1e-3; the worst relative error per kind against the
    float64 series on the graphs up to 1e5 nodes (subgraph centrality on 32
    sampled nodes of each); Katz at gamma = 0.85 /
    lambda_max with the second-moment radius rho(diag(s')|A'|) per graph and
    the queries whose calibration stopped at the walk cap."""
    import torch

    t = time.time()
    graphs, qs, cal = batch_queries(M, R, I, n_graphs, log_n_max)
    log(f"[bench] batch workload: {len(qs)} graphs, sum n = {sum(g.n for g, _, _ in graphs)}, calibrated "
        f"({time.time() - t:.1f}s)")
    for q, (g, _, _) in zip(qs, graphs):
        q["out"] = torch.empty(g.n, dtype=torch.float64, device="cuda")
    res = {"queries": len(qs), "sum_n": int(sum(g.n for g, _, _ in graphs))}

    def time_single(sel):
        for q in sel[:2]:
            solve_single(M, q)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            for q in sel:
                solve_single(M, q)
        torch.cuda.synchronize()
        return len(sel) / ((time.perf_counter() - t0) / reps)

    def time_batch(sel, flags):
        b = M.mcf_batch_create(sel, flags=flags)
        M.mcf_batch_run(b)
        t0 = time.perf_counter()
        for _ in range(reps):
            _, st = M.mcf_batch_run(b, stats=True)
        el = (time.perf_counter() - t0) / reps
        b.close()
        return len(sel) / el, st["walk_steps"] / el

    per_kind = {}
    for kind in ("all",) + KINDS:
        t0 = time.perf_counter()
        sel = qs if kind == "all" else [q for q in qs if _kind_of(M, q) == kind]
        one = time_single(sel)
        cg, steps = time_batch(sel, M.MCF_BATCH_CUDA_GRAPH | M.MCF_BATCH_AUTOTUNE)
        per_kind[kind] = {"queries": len(sel), "one_at_a_time_solves_per_s": one,
                          "batched_cuda_graph_solves_per_s": cg, "speedup": cg / one}
        if kind == "all":
            bat, _ = time_batch(sel, M.MCF_BATCH_AUTOTUNE)
            per_kind[kind]["batched_solves_per_s"] = bat
            res["batched_cuda_graph_walk_steps_per_s"] = steps
        log(f"[bench] batch timing ({kind}): {time.perf_counter() - t0:.1f}s")
    res["solves_per_s"] = per_kind
    res["speedup_vs_one_at_a_time"] = per_kind["all"]["speedup"]
    # accuracy of the batch results (last run) on the graphs up to 1e5 nodes, per kind
    errs = {k: [] for k in KINDS}
    miss = {k: [] for k in KINDS}
    rho2 = []
    for q, (g, h, lam), cl in zip(qs, graphs, cal):
        kind = _kind_of(M, q)
        if kind == "katz":
            rho2.append(M.mcf_second_moment_radius(h, q["katz_gamma"], tol=1e-4, max_iter=500))
        if g.n > 100_000:
            continue
        y = q["out"].cpu().numpy()
        if kind == "tc":
            ref = R.series_action(g, exp_coeffs(30), 1.0 / lam)
        elif kind == "katz":
            K = R.katz_terms_for_tail(q["katz_gamma"] * lam, 1e-4)
            ref = R.series_action(g, R.katz_coeffs(K), q["katz_gamma"])
        else:
            # sampled entries; the norm of the whole result (the relative l_inf error's
            # denominator) from the estimate itself, whose largest entry is among the samples
            top = int(np.argmax(np.abs(y)))
            nodes = np.unique(np.append(np.arange(0, g.n, max(1, g.n // 32)), top))
            ref = R.series_diag(g, exp_coeffs(30), nodes, 1.0 / lam)
            e = float(np.abs(y[nodes] - ref).max() / max(np.abs(ref).max(), np.abs(y).max()))
            (errs if cl["budget_met"] else miss)[kind].append(e)
            continue
        e = float(np.abs(y - ref).max() / np.abs(ref).max())
        (errs if cl["budget_met"] else miss)[kind].append(e)
    res["max_rel_err_vs_fp64"] = {k: (max(v) if v else None) for k, v in errs.items()}
    res["budget_misses_rel_err_vs_fp64"] = {k: (max(v) if v else None) for k, v in miss.items()}
    res["calibration"] = {
        "target_rel_err": CAL_TARGET,
        "budget_met": {k: sum(1 for c_ in cal if c_["kind"] == k and c_["budget_met"]) for k in KINDS},
        "budget_missed": {k: sum(1 for c_ in cal if c_["kind"] == k and not c_["budget_met"]) for k in KINDS},
        "margin": CAL_MARGIN,
        "median_walks_per_node": {k: float(np.median([c_["walks_per_node"] for c_ in cal if c_["kind"] == k] or [0]))
                                  for k in KINDS}}
    res["katz_gamma"] = "0.85 / lambda_max"
    res["katz_second_moment_radius"] = {"min": float(min(rho2)), "median": float(np.median(rho2)),
                                        "max": float(max(rho2)), "above_1": int(sum(r > 1 for r in rho2))} if rho2 else None
    for _, h, _ in graphs:
        h.close()
    return res


def run_serving(M, R, I, scales, n_requests, rate=200.0, seed=5, workers=6):
    """Poisson arrivals (rate req/s) over a resident R-MAT pool; query mix 50%
    total communicability, 30% Katz (gamma = 0.85 / max_i sum_k |a_ik|, the
    paper's setting), 20% subgraph centrality on 10^4 sampled nodes; walk
    budgets calibrated per graph and kind to 1e-3; p50/p99 latency from the
    server's counters, device overlap of batches, errors on sampled graphs;
    the capacity of the server (all requests queued at once) against the
    same requests solved one at a time."""
    t = time.time()
    pool = []
    c = exp_coeffs(30)
    rng = np.random.default_rng(seed)
    for sc in scales:
        g = I.rmat(sc, 16, seed=sc)
        h = M.mcf_create_graph(g.n, g.row_ptr, g.col_idx)
        lam = M.mcf_spectral_radius(h, tol=1e-10, max_iter=10000)
        kg = 0.85 / M.mcf_gershgorin(h)
        nodes = rng.choice(g.n, size=min(10_000, g.n), replace=False).astype(np.int64)
        common = dict(seed=seed, request_id=0, precision=M.MCF_F32W_F64ACC)
        budgets = {
            "tc": calibrate(M, query_solver(M, h, "tc", c, 1.0 / lam), dict(common, n_walks=g.n, w_cutoff=1e-6),
                            g.n, 1024)[0],
            "katz": calibrate(M, query_solver(M, h, "katz", katz_gamma=kg), dict(common, walks_per_node=1), g.n,
                              1024)[0],
            "sc": calibrate(M, query_solver(M, h, "sc", c, 1.0 / lam, nodes=nodes),
                            dict(common, walks_per_node=1, w_cutoff=1e-6), g.n, 1024)[0]}
        pool.append((g, h, lam, kg, nodes, budgets))
        log(f"[bench] serving pool: R-MAT scale {sc} ready, budgets {budgets} ({time.time() - t:.1f}s)")
    qs, arrivals, tnow = [], [], 0.0
    for i in range(n_requests):
        tnow += rng.exponential(1.0 / rate)
        arrivals.append(tnow)
        g, h, lam, kg, nodes, budgets = pool[int(rng.integers(len(pool)))]
        u = rng.random()
        base = dict(graph=h, seed=seed * 100000 + i, request_id=i, precision=M.MCF_F32W_F64ACC)
        if u < 0.5:
            qs.append(dict(base, kind=M.MCF_QUERY_TOTAL_COMMUNICABILITY, coeffs=c, scale=1.0 / lam, w_cutoff=1e-6,
                           **budgets["tc"]))
        elif u < 0.8:
            qs.append(dict(base, kind=M.MCF_QUERY_KATZ, katz_gamma=kg, katz_terms=0, **budgets["katz"]))
        else:
            qs.append(dict(base, kind=M.MCF_QUERY_SUBGRAPH_CENTRALITY, coeffs=c, scale=1.0 / lam, w_cutoff=1e-6,
                           nodes=nodes, **budgets["sc"]))
    srv = M.mcf_server_create(hbm_budget_bytes=64 << 30, max_inflight=workers, max_batch=16, batch_window_ms=0.5)
    for q in qs[:8]:     # warm-up of the server path
        M.mcf_server_wait(srv, M.mcf_server_submit(srv, dict(q)))
    srv.close()
    graph_of = {id(p[1]): p for p in pool}
    keep = {}   # (kind, n) -> output of the first such request, for the accuracy check

    def take(srv, i, tk):
        # a client takes each result when it completes and lets its buffer go
        # (page-locked host blocks return to torch's cache), so host memory
        # holds only the requests in flight
        y, _ = M.mcf_server_wait(srv, tk)
        M.mcf_server_release(srv, tk)
        g = graph_of[id(qs[i]["graph"])][0]
        key = (_kind_of(M, qs[i]), g.n)
        if key not in keep and g.n <= (1 << (20 if key[0] == "sc" else 22)):
            keep[key] = np.array(y, copy=True)

    srv = M.mcf_server_create(hbm_budget_bytes=64 << 30, max_inflight=workers, max_batch=16, batch_window_ms=0.5)
    t0 = time.perf_counter()
    pending = collections.deque()
    for i, (q, ta) in enumerate(zip(qs, arrivals)):
        while pending and M.mcf_server_poll(srv, pending[0][1])[0]:
            take(srv, *pending.popleft())
        d = ta - (time.perf_counter() - t0)
        if d > 0:
            time.sleep(d)
        pending.append((i, M.mcf_server_submit(srv, q)))
    while pending:
        take(srv, *pending.popleft())
    wall = time.perf_counter() - t0
    st = M.mcf_server_get_stats(srv)
    srv.close()
    # capacity, closed loop: the same requests through the server from a
    # client that keeps CAP_WINDOW of them outstanding (more than the
    # server's workers x batch size), against the plain loop that solves them
    # one at a time (each result read back to the host before the next
    # request, as a client of the single-query calls does)
    srv = M.mcf_server_create(hbm_budget_bytes=64 << 30, max_inflight=workers, max_batch=16, batch_window_ms=0.5)
    t1 = time.perf_counter()
    pending = collections.deque()
    for q in qs:
        if len(pending) >= CAP_WINDOW:
            tk = pending.popleft()
            M.mcf_server_wait(srv, tk)
            M.mcf_server_release(srv, tk)
        pending.append(M.mcf_server_submit(srv, q))
    while pending:
        tk = pending.popleft()
        M.mcf_server_wait(srv, tk)
        M.mcf_server_release(srv, tk)
    wall_served = time.perf_counter() - t1
    srv.close()
    for q in qs[:8]:
        solve_single(M, q)
    t1 = time.perf_counter()
    for q in qs:
        solve_single(M, q)
    wall_single = time.perf_counter() - t1
    capacity = {"served_solves_per_s": n_requests / wall_served,
                "one_at_a_time_solves_per_s": n_requests / wall_single,
                "speedup": wall_single / wall_served, "outstanding_requests": CAP_WINDOW}
    log(f"[bench] serving capacity: served {capacity['served_solves_per_s']:.1f}/s, one at a time "
        f"{capacity['one_at_a_time_solves_per_s']:.1f}/s")
    # accuracy of the first request per kind and graph: TC and Katz on graphs
    # up to 2^22 nodes (whole vectors), SC on graphs up to 2^20 nodes (64 of
    # the sampled nodes)
    errs = {"tc": [], "katz": [], "sc": []}
    for (kind, n), y in sorted(keep.items()):
        g, h, lam, kg, nodes, _ = next(p for p in pool if p[0].n == n)
        if kind == "tc":
            ref = R.series_action(g, c, 1.0 / lam)
        elif kind == "katz":
            K = R.katz_terms_for_tail(kg * lam, 1e-4)
            ref = R.series_action(g, R.katz_coeffs(K), kg)
        else:
            ref, y = R.series_diag(g, c, nodes[:64], 1.0 / lam), y[:64]
        errs[kind].append((g.n, float(np.abs(y - ref).max() / np.abs(ref).max())))
    for p_ in pool:
        p_[1].close()
    return {"requests": n_requests, "rate_req_per_s": rate, "scales": [scales[0], scales[-1]], "workers": workers,
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"], "mean_ms": st["mean_ms"],
            "solves_per_s": st["completed"] / wall, "batches": st["batches"], "rejected": st["rejected"],
            "walk_steps_per_s": st["walk_steps"] / wall, "device_overlap_ms": st["device_overlap_ms"],
            "max_concurrent_batches": st["max_concurrent_batches"], "wall_s": wall, "capacity": capacity,
            "worker_plan_s": st["plan_s"], "worker_run_s": st["run_s"],
            "max_rel_err_vs_fp64": {k: (max(e for _, e in v) if v else None) for k, v in errs.items()},
            "checked_graph_sizes": {k: sorted(n for n, _ in v) for k, v in errs.items()},
            "walk_budgets": "calibrated per graph and kind for an estimated relative l_inf error of "
                            f"{CAL_TARGET} (two replicas of a pilot budget, scaled by the N^-1/2 law, margin "
                            f"{CAL_MARGIN})",
            "katz_gamma": "0.85 / max_i sum_k |a_ik| (Gershgorin, Section 4.5)"}


def run_config1(M, I, reps=3):
    """The plain method at the small size: Barabasi-Albert n = 1000, m = 3
    (seed 0), A / lambda_max, exp truncated at K = 30, 1e5 walks per node,
    float64 throughout; total communicability and subgraph centrality, time
    per solve (CUDA events) and the relative l_inf error against dense
    expm(A / lambda_max) (scipy, float64)."""
    import torch
    from scipy.linalg import expm

    g = I.barabasi_albert(1000, 3, 0)
    h = M.mcf_create_graph(g.n, g.row_ptr, g.col_idx)
    lam = M.mcf_spectral_radius(h, tol=1e-12, max_iter=100000)
    c = exp_coeffs(30)
    A = np.zeros((g.n, g.n))
    for i in range(g.n):
        A[i, g.col_idx[g.row_ptr[i]:g.row_ptr[i + 1]]] = 1.0
    E = expm(A / lam)
    ref = {"tc": E.sum(axis=1), "sc": np.diag(E).copy()}
    kw = dict(scale=1.0 / lam, walks_per_node=100_000, w_cutoff=0.0, seed=0, precision=M.MCF_F64)
    out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    res = {"workload": "BA n=1000 m=3 seed 0, exp(A/lambda_max) truncated at K=30, 1e5 walks per node, float64",
           "lambda_max": lam}
    for kind, fn in (("tc", M.mcf_total_communicability), ("sc", M.mcf_subgraph_centrality)):
        fn(h, c, out=out, request_id=1, **kw)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        steps = 0
        for i in range(reps):
            _, st = fn(h, c, out=out, request_id=2 + i, stats=True, **kw)
            steps += st["walk_steps"]
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        y = out.cpu().numpy()
        res[kind] = {"ms_per_solve": ms, "walk_steps_per_s": steps / reps / (ms / 1000.0),
                     "rel_err_vs_dense_expm": float(np.abs(y - ref[kind]).max() / np.abs(ref[kind]).max())}
    h.close()
    return res


def run_sc_config3(M, R, I, steps=2):
    """Subgraph centrality diag exp(A/lambda_max) of every node of the erased
    configuration model n = 2e6 (k^-2.5, mean degree 20), 2000 walks per node,
    W_c = 1e-6, float32 weights with float64 accumulation: time per solve,
    walk-steps/s, the walk kernel's roofline at 12 algorithmic bytes per step,
    the difference between float32 and float64 walk arithmetic on the same
    walks (100 walks per node), and the error against the float64 series on
    sampled nodes."""
    import torch

    peak, peak_kind = measured_peak()
    g = I.config_powerlaw(2_000_000, 2.5, 20.0, 2)
    h = M.mcf_create_graph(g.n, torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col_idx).cuda())
    lam = M.mcf_spectral_radius(h, tol=1e-10, max_iter=10000)
    gam = 1.0 / lam
    c = exp_coeffs(30)
    d = torch.empty(g.n, dtype=torch.float64, device="cuda")
    kw = dict(scale=gam, walks_per_node=2000, w_cutoff=1e-6, seed=2, precision=M.MCF_F32W_F64ACC)
    M.mcf_subgraph_centrality(h, c, out=d, request_id=100, **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    kms, steps_ = [], 0
    for i in range(steps):
        _, st = M.mcf_subgraph_centrality(h, c, out=d, request_id=101 + i, stats=True, **kw)
        kms.append(st["kernel_ms"])
        steps_ += st["walk_steps"]
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    kernel_ms = float(np.mean(kms))
    per = steps_ / steps
    achieved = 12 * per / (kernel_ms / 1000.0) / 1e9
    y = d.cpu().numpy()
    nodes = np.unique(np.append(np.random.default_rng(0).choice(g.n, size=7, replace=False), int(np.argmax(y))))
    ref = R.series_diag(g, c, nodes, gam)
    # float32 against float64 walk arithmetic on the same walks (100 walks per node)
    kw100 = dict(kw, walks_per_node=100)
    d32 = M.mcf_subgraph_centrality(h, c, out=torch.empty_like(d), request_id=7, **kw100).cpu().numpy()
    d64 = M.mcf_subgraph_centrality(h, c, out=torch.empty_like(d), request_id=7,
                                    **dict(kw100, precision=M.MCF_F64)).cpu().numpy()
    h.close()
    return {"workload": "subgraph centrality diag exp(A/lambda_max), erased configuration model n=2e6 k^-2.5 "
                        "mean 20, 2000 walks per node, K=30, W_c=1e-6",
            "n": g.n, "nnz": g.nnz, "ms_per_solve": ms, "solves_per_s": 1000.0 / ms,
            "walk_steps_per_solve": per, "walk_steps_per_s": per / (ms / 1000.0),
            "roofline": {"bound": "hbm", "kernel": "walk_diag_od_kernel", "kernel_ms": kernel_ms,
                         "algorithmic_bytes_per_step": 12, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind},
            "rel_err_vs_fp64_sampled": float(np.abs(y[nodes] - ref).max() / max(np.abs(ref).max(), np.abs(y).max())),
            "sampled_nodes": len(nodes),
            "float32_vs_float64_walks_max_rel_diff": float(np.max(np.abs(d32 - d64) / np.abs(d64))),
            "precision": "float32 walk weights with compensated float32 sums per walk, float64 accumulation; "
                         "compared with float64 throughout on the same walks"}


def run_subset(M, h, g, c, base, full_out, reps=5):
    """Single-entry and subset total communicability on the resident graph
    (Section 4.3, Table 3): only the columns adjacent to the requested nodes
    are walked, with the full run's walk ids, so each entry equals the full
    solve's entry; time per call and walks taken against the full solve."""
    import torch

    full_y, full_st = M.mcf_total_communicability(h, c, out=full_out, request_id=77, stats=True, **base)
    full_y = full_y.cpu().numpy()
    res = {}
    rng = np.random.default_rng(11)
    for name, nodes in (("max_degree_node", np.array([int(np.argmax(g.degree))], np.int64)),
                        ("1000_random_nodes", rng.choice(g.n, size=1000, replace=False).astype(np.int64))):
        nd = torch.from_numpy(nodes).cuda()
        M.mcf_action_nodes(h, nd, c, request_id=77, **base)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            y, st = M.mcf_action_nodes(h, nd, c, request_id=77, stats=True, **base)
        torch.cuda.synchronize()
        ms = 1e3 * (time.perf_counter() - t0) / reps
        y = y.cpu().numpy()
        res[name] = {"ms_per_call": ms, "walks": st["walks"], "walk_steps": st["walk_steps"],
                     "max_rel_diff_vs_full_solve": float(np.max(np.abs(y - full_y[nodes]) / np.abs(full_y[nodes])))}
    res["full_solve_walks"] = full_st["walks"]
    return res


def run_funm_full(M, R, I, n=16384, m=8, wpn=100, reps=3):
    """Dense RandFunm (Algorithm 2) at the largest supported n: time of one
    solve (walks + the A'QA' epilogue), and the error of F 1 and of diag F on
    sampled nodes against the float64 series."""
    import torch

    g = I.barabasi_albert(n, m, 31)
    h = M.mcf_create_graph(g.n, g.row_ptr, g.col_idx)
    gam = 1.0 / M.mcf_spectral_radius(h)
    c = exp_coeffs(30)
    out = torch.empty(g.n * g.n, dtype=torch.float64, device="cuda")
    kw = dict(scale=gam, walks_per_node=wpn, w_cutoff=1e-6, seed=2, precision=M.MCF_F32W_F64ACC)
    M.mcf_funm_full(h, c, out=out, **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    walk_ms = []
    for i in range(reps):
        _, st = M.mcf_funm_full(h, c, out=out, stats=True, request_id=i, **kw)
        walk_ms.append(st["kernel_ms"])
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    F = out.view(g.n, g.n)
    ones = torch.ones(g.n, dtype=torch.float64, device="cuda")
    y = (F @ ones).cpu().numpy()
    ref = R.series_action(g, c, gam)
    nodes = np.arange(0, g.n, g.n // 128)
    dref = R.series_diag(g, c, nodes, gam)
    d = torch.diagonal(F).cpu().numpy()[nodes]
    res = {"graph": f"BA n={n} m={m}", "nnz": g.nnz, "walks_per_node": wpn, "ms_per_solve": ms,
           "walk_kernel_ms": float(np.mean(walk_ms)), "walk_steps": st["walk_steps"],
           "epilogue_min_hbm_bytes": int(g.nnz * g.n * 8 + g.n * g.n * 8),
           "rel_err_F1_vs_fp64": float(np.abs(y - ref).max() / np.abs(ref).max()),
           "rel_err_diag_vs_fp64": float(np.abs(d - dref).max() / np.abs(dref).max())}
    del F, out
    h.close()
    return res


def run_mc_classic(M, R, I, n=1000, m=3, wpn=10_000):
    """The classical method (Algorithm 1) against row sampling (Algorithm 3)
    at the same number of walks per node, float64 both: error of f(A')1
    against the float64 series and walk-steps/s."""
    import torch

    g = I.barabasi_albert(n, m, 0)
    h = M.mcf_create_graph(g.n, g.row_ptr, g.col_idx)
    gam = 1.0 / M.mcf_spectral_radius(h)
    c = exp_coeffs(30)
    ref = R.series_action(g, c, gam)
    res = {"graph": f"BA n={n} m={m}", "walks_per_node": wpn}
    for name, fn in (("classic", lambda i: M.mcf_mc_classic(h, c, wpn, scale=gam, seed=3, request_id=i, stats=True)),
                     ("row_sampling", lambda i: M.mcf_total_communicability(
                         h, c, scale=gam, walks_per_node=wpn, seed=3, request_id=i, precision=M.MCF_F64,
                         stats=True))):
        fn(100)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        errs, steps = [], 0
        for i in range(3):
            y, st = fn(i)
            steps += st["walk_steps"]
            errs.append(float(np.abs(y - ref).max() / np.abs(ref).max()))
        el = time.perf_counter() - t0
        res[name] = {"rel_err_vs_fp64": float(np.mean(errs)), "walk_steps_per_s": steps / el,
                     "solves_per_s": 3 / el}
    res["error_ratio_classic_over_row_sampling"] = res["classic"]["rel_err_vs_fp64"] / res["row_sampling"]["rel_err_vs_fp64"]
    h.close()
    return res


def run_reference(args, w):
    """--impl reference: the oracle as it stands, timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import reference as R

    g = make_graph(w)
    lam = R.lambda_max(g)
    per_step = max(min(2.0, args.ref_seconds), args.ref_seconds / max(1, args.steps + args.warmup))
    pool = OraclePool(g, w)
    try:
        for i in range(args.warmup):
            pool.run(lam, per_step / 4, seed=1000 + i)
        vals = []
        t0 = time.perf_counter()
        last = None
        for i in range(args.steps):
            last = pool.run(lam, per_step, seed=2000 + i)
            vals.append(last["value"])
        el = time.perf_counter() - t0
    finally:
        pool.close()
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": "walk-steps/s", "value": v, "unit": "walk-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * el / max(1, args.steps), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 walk weights, f64 accumulation", "data": "synthetic",
            "config": {"workload": w["label"]},
            "cpu_baseline": {"value": v, "unit": "walk-steps/s", "cores": pool.procs, "kind": "oracle",
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
    ap.add_argument("--no-batch", action="store_true", help="skip the batched, serving, dense RandFunm and classical-method measurements")
    ap.add_argument("--batch-graphs", type=int, default=256)
    ap.add_argument("--batch-log-n-max", type=float, default=6.0)
    ap.add_argument("--serve-scales", default="16-26")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--section", default="main",
                    choices=["main", "funm_full", "mc_classic", "batched", "serving", "sc_config3", "config1"],
                    help="run only that measurement (1 GPU) and print its JSON")
    ap.add_argument("--funm-n", type=int, default=16384, help="nodes of the dense RandFunm measurement")
    ap.add_argument("--ref-seconds", type=float, default=60.0,
                    help="--impl reference: oracle time budget of the whole run, split over the steps")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)
    if args.section != "main":
        R = F64Ref
        from paper_2308_01037_gb300 import inputs as I
        from paper_2308_01037_gb300 import mcf as M

        M.load()
        if args.section == "funm_full":
            res = run_funm_full(M, R, I, n=args.funm_n)
        elif args.section == "mc_classic":
            res = run_mc_classic(M, R, I)
        elif args.section == "batched":
            res = run_batched(M, R, I, args.batch_graphs, args.batch_log_n_max)
        elif args.section == "sc_config3":
            res = run_sc_config3(M, R, I)
        elif args.section == "config1":
            res = run_config1(M, I)
        else:
            lo, hi = (int(x) for x in args.serve_scales.split("-"))
            res = run_serving(M, R, I, list(range(lo, hi + 1)), args.serve_requests)
        print(json.dumps({"section": args.section, **res}), flush=True)
        return

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
    launches0 = M.mcf_kernel_launches()   # the library's own kernel-execution counter (synchronises)
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
    launches = M.mcf_kernel_launches() - launches0
    ms = ev0.elapsed_time(ev1)
    tmax = ms
    steps_all = steps_total
    if dist:
        tmax, steps_all = aggregate(ms, steps_total, device="cuda")
    value = steps_all / (tmax / 1000.0)
    solves_per_s = world * args.steps / (tmax / 1000.0)
    log(f"[bench] timed: {tmax / args.steps:.2f} ms per step, {value:.3e} walk-steps/s")
    kernel_ms = float(np.mean(kern_ms))
    peak, peak_kind = measured_peak()
    steps_per_launch = steps_total / args.steps
    achieved = ALGO_BYTES_PER_STEP[w["query"]] * steps_per_launch / (kernel_ms / 1000.0) / 1e9
    traffic = None
    if args.workload in NCU_DRAM_BYTES_PER_STEP:
        traffic = NCU_DRAM_BYTES_PER_STEP[args.workload] * steps_per_launch
    # the random-read ceiling of this GPU, measured here: independent random
    # 8-byte reads over an array the size of the per-entry walk records
    gather = None
    if w["query"] == "tc":
        gather = M.mcf_gather_probe(max(g.nnz, 1) * 8, 1 << 28, stream.cuda_stream)
    kernel_steps_per_s = steps_per_launch / (kernel_ms / 1000.0)

    # ---- accuracy of one solve against the float64 truncated series
    rel_err = None
    if not args.no_accuracy and rank == 0:
        R = F64Ref

        y = out.cpu().numpy()
        t = time.time()
        if w["query"] == "tc":
            ref = R.series_action(g, c, gam)
            rel_err = float(np.abs(y - ref).max() / np.abs(ref).max())
        else:
            # float64 series on the host costs K sparse products per sampled node:
            # keep it near 1e10 multiply-adds (at least 16 nodes, at most 2000)
            m = int(min(g.n, 2000, max(16, 1e10 // (w["K"] * max(g.nnz, 1)))))
            nodes = np.random.default_rng(0).choice(g.n, size=m, replace=False)
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

    subset = None
    max_rel_se = None
    if rank == 0 and world == 1 and w["query"] == "tc" and not args.no_batch:
        subset = run_subset(M, h, g, c, base, out)
        # the library's own standard-error estimate of one solve (Section 3.5)
        _, st_se = solve(h, c, out=out, request_id=88, stats=True, error_estimate=True, **base)
        max_rel_se = st_se["max_rel_se"]
    batched = serving = funm_full = mc_classic = sc3 = config1 = None
    if rank == 0 and world == 1 and not args.no_batch:
        R = F64Ref
        from paper_2308_01037_gb300 import inputs as I

        h.close()    # the sections below bring their own graphs
        t = time.time()
        config1 = run_config1(M, I)
        log(f"[bench] section config1: {time.time() - t:.1f}s")
        t = time.time()
        sc3 = run_sc_config3(M, R, I)
        log(f"[bench] section sc_config3: {time.time() - t:.1f}s")
        t = time.time()
        batched = run_batched(M, R, I, args.batch_graphs, args.batch_log_n_max)
        log(f"[bench] section batched: {time.time() - t:.1f}s")
        t = time.time()
        lo, hi = (int(x) for x in args.serve_scales.split("-"))
        serving = run_serving(M, R, I, list(range(lo, hi + 1)), args.serve_requests)
        log(f"[bench] section serving: {time.time() - t:.1f}s")
        t = time.time()
        funm_full = run_funm_full(M, R, I)
        mc_classic = run_mc_classic(M, R, I)
        log(f"[bench] sections funm_full, mc_classic: {time.time() - t:.1f}s")
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_all_cores(g, lam, w)
    if rank == 0:
        line = {
            "metric": "walk-steps/s", "value": value, "unit": "walk-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tmax / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 walk weights, f64 accumulation", "data": "synthetic",
            "config": {"workload": w["label"], "n": g.n, "nnz": g.nnz, "lambda_max": lam,
                       "walks_per_solve": walks_total // args.steps, "l2": "inputs larger than L2 (CSR > 129 MB)",
                       "parallelism": f"{world} independent solves per step" if world > 1 else "1 GPU"},
            "solves_per_s": solves_per_s, "rel_err_vs_fp64": rel_err, "max_rel_se_estimate": max_rel_se,
            "walk_steps_per_solve": steps_total / args.steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": KERNEL[w["query"]], "kernel_ms": kernel_ms,
                         "algorithmic_bytes_per_step": ALGO_BYTES_PER_STEP[w["query"]],
                         "useful_bytes_fraction": None if traffic is None else
                         ALGO_BYTES_PER_STEP[w["query"]] * steps_per_launch / traffic,
                         # DRAM bytes actually moved per second (traffic / live launch time) and their share
                         # of the measured copy peak
                         "dram_gbs": None if traffic is None else traffic / (kernel_ms / 1000.0) / 1e9,
                         "dram_frac": None if traffic is None else traffic / (kernel_ms / 1000.0) / 1e9 / peak,
                         "traffic_note": None if traffic is None else
                         "DRAM bytes per launch: ncu dram__bytes_read.sum + dram__bytes_write.sum per walk step on "
                         "the R-MAT scale 21 case (one 32-B sector per random step) x the walk steps of a launch",
                         # one walk step is one random read of an 8-byte record: the rate of independent random
                         # 8-byte reads this GPU serves over an array of the records' size, measured in this run
                         "gather_ceiling": gather, "gather_ceiling_unit": "random 8-byte reads/s",
                         "kernel_walk_steps_per_s": kernel_steps_per_s,
                         "frac_of_gather_ceiling": None if not gather else kernel_steps_per_s / gather},
            "clocks": clk.summary(), "e2e": e2e, "gpu_launches": launches,
            "cpu_baseline": cpu,
            "subset": subset, "config1": config1, "subgraph_centrality_config3": sc3, "batched": batched,
            "serving": serving,
            "funm_full": funm_full,
            "mc_classic": mc_classic,
        }
        print(json.dumps(line), flush=True)
    h.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
