"""The multi-rank reduction of bench.py (slowest rank's time, all ranks'
work) on two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    tmax, steps = bench.aggregate(ms=10.0 + 5.0 * rank, steps=1000 * (rank + 1))
    q.put((rank, tmax, steps))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tmax, steps in got:
        assert tmax == 15.0 and steps == 3000.0


def _bench_rank(rank, world, port, q):
    """One rank of bench.main() with the device calls stood in (see
    test_bench_contract.py): gloo instead of NCCL, CPU tensors for "cuda"."""
    import io
    import sys
    import types
    from contextlib import redirect_stdout

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    import bench
    import paper_2308_01037_gb300 as pkg
    import test_bench_contract as C

    g = bench.make_graph(bench.WORKLOADS["ba1000_tc"])
    fake = C._fake_library(g)
    sys.modules["paper_2308_01037_gb300.mcf"] = fake
    pkg.mcf = fake
    torch.cuda.set_device = lambda *a, **k: None
    torch.cuda.synchronize = lambda *a, **k: None
    torch.cuda.current_stream = lambda *a, **k: types.SimpleNamespace(cuda_stream=0)
    torch.cuda.Event = C._Event
    torch.Tensor.cuda = lambda self, *a, **k: self
    torch.Tensor.pin_memory = lambda self, *a, **k: self
    real_empty, real_tensor = torch.empty, torch.tensor
    torch.empty = lambda *a, device=None, **k: real_empty(*a, **k)
    torch.tensor = lambda *a, device=None, **k: real_tensor(*a, **k)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.argv = ["bench.py", "--workload", "ba1000_tc", "--steps", "2", "--warmup", "3", "--e2e-steps", "1",
                "--no-cpu-baseline", "--no-batch", "--no-accuracy", "--gpus", str(world)]
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.main()
    q.put((rank, [ln for ln in buf.getvalue().splitlines() if ln.startswith("{")]))


def test_two_rank_bench_line():
    """Two ranks: rank 0 alone prints, value = walk steps of both ranks / the
    slowest rank's timed region, n_gpus = 2, e2e summed over the ranks."""
    import json

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_bench_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[1] == [] and len(got[0]) == 1
    d = json.loads(got[0][0])
    assert d["n_gpus"] == 2 and d["scaling"] == "weak"
    assert d["config"]["parallelism"] == "2 independent solves per step"
    # both ranks' steps over the slowest rank's time
    assert d["value"] == pytest.approx(2 * 2 * 1_000_000 / (d["ms_per_step"] * 2 / 1000.0), rel=1e-9)
    assert d["e2e"]["value"] > 0
