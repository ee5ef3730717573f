"""Batched solves (mcf_batch_*): many queries on many graphs in one pass.

Every query of a batch keeps its own walk ids and Philox streams, so its
result must equal the single call's result for the same parameters (parity
tolerance 1e-12 relative) -- alone and in the mix, with and without CUDA-graph
capture and autotuning -- and the single calls in turn equal the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import estimator as E
from oracle import reference as R
from paper_2308_01037_gb300 import inputs as I
from paper_2308_01037_gb300 import mcf as M

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-12, 1e-13


def close(a, b):
    a = np.asarray(a.cpu() if hasattr(a, "cpu") else a)
    b = np.asarray(b.cpu() if hasattr(b, "cpu") else b)
    assert a.shape == b.shape
    err = np.abs(a - b)
    assert np.all(err <= RTOL * np.abs(b) + ATOL), f"max rel {np.max(err / np.maximum(np.abs(b), 1e-300)):.3e}"


@pytest.fixture(scope="module")
def graphs():
    gs = {
        "ba500": I.barabasi_albert(500, 3, 1),
        "er3000": I.erdos_renyi(3000, 12, 2),
        "rmat11": I.rmat(11, 16, seed=3),
        "ba20k": I.barabasi_albert(20000, 4, 4),      # hashed row Q_k in the diag kernel
    }
    out = {}
    for k, g in gs.items():
        h = M.mcf_create_graph(g.n, g.row_ptr, g.col_idx)
        out[k] = (g, h, 1.0 / R.lambda_max(g))
    w = I.barabasi_albert(400, 3, 5)
    vals = I.symmetric_weights(w, seed=1, signed=True)
    hw = M.mcf_create_graph(w.n, w.row_ptr, w.col_idx, vals)
    out["weighted"] = (w, hw, 1.0 / np.abs(np.linalg.eigvalsh(R.csr_matrix(w, vals).toarray())).max())
    return out


def make_queries(graphs):
    c30 = R.exp_coeffs(30)
    qs = []
    for j, (name, (g, h, gam)) in enumerate(graphs.items()):
        if name == "weighted":
            continue
        qs.append(dict(graph=h, kind=M.MCF_QUERY_TOTAL_COMMUNICABILITY, coeffs=c30, scale=gam, n_walks=40 * g.n,
                       w_cutoff=1e-6, seed=10 + j, request_id=j, precision=M.MCF_F32W_F64ACC))
        qs.append(dict(graph=h, kind=M.MCF_QUERY_KATZ, katz_gamma=0.85 * gam, katz_terms=0, walks_per_node=8,
                       seed=20 + j, request_id=100 + j, precision=M.MCF_F32W_F64ACC))
        qs.append(dict(graph=h, kind=M.MCF_QUERY_SUBGRAPH_CENTRALITY, coeffs=c30, scale=gam,
                       walks_per_node=30 if g.n > 5000 else 200, seed=30 + j, request_id=200 + j,
                       precision=M.MCF_F32W_F64ACC))
    g, h, gam = graphs["rmat11"]
    qs.append(dict(graph=h, kind=M.MCF_QUERY_SUBGRAPH_CENTRALITY, coeffs=c30, scale=gam, walks_per_node=100,
                   nodes=np.array([5, 17, 1000, 5, int(np.argmax(g.degree))], np.int64), seed=7, request_id=300,
                   precision=M.MCF_F32W_F64ACC))
    # queries served by the single-query path inside the batch
    v = np.random.default_rng(3).standard_normal(g.n)
    qs.append(dict(graph=h, kind=M.MCF_QUERY_ACTION, coeffs=c30, v=v, scale=gam, n_walks=50000, seed=8,
                   request_id=400, precision=M.MCF_F32W_F64ACC))
    qs.append(dict(graph=h, kind=M.MCF_QUERY_TOTAL_COMMUNICABILITY, coeffs=c30, scale=gam, n_walks=50000, seed=9,
                   request_id=500, precision=M.MCF_F64))
    # a query large enough to run through the single-query kernel inside the batch
    qs.append(dict(graph=h, kind=M.MCF_QUERY_TOTAL_COMMUNICABILITY, coeffs=c30, scale=gam, n_walks=1 << 25, seed=12,
                   request_id=700, precision=M.MCF_F32W_F64ACC))
    gw, hw, gamw = graphs["weighted"]
    qs.append(dict(graph=hw, kind=M.MCF_QUERY_SUBGRAPH_CENTRALITY, coeffs=R.exp_coeffs(20), scale=gamw,
                   walks_per_node=40, seed=11, request_id=600, precision=M.MCF_F32W_F64ACC))
    return qs


def single(q):
    keys = ("scale", "n_walks", "walks_per_node", "w_cutoff", "seed", "request_id", "precision")
    kw = {k: q[k] for k in keys if k in q}
    if q["kind"] == M.MCF_QUERY_TOTAL_COMMUNICABILITY:
        return M.mcf_total_communicability(q["graph"], q["coeffs"], **kw)
    if q["kind"] == M.MCF_QUERY_KATZ:
        return M.mcf_katz(q["graph"], q["katz_gamma"], q["katz_terms"], **kw)
    if q["kind"] == M.MCF_QUERY_SUBGRAPH_CENTRALITY:
        return M.mcf_subgraph_centrality(q["graph"], q["coeffs"], nodes=q.get("nodes"), **kw)
    return M.mcf_action(q["graph"], q["v"], q["coeffs"], **kw)


@pytest.mark.parametrize("flags", [0, M.MCF_BATCH_CUDA_GRAPH, M.MCF_BATCH_CUDA_GRAPH | M.MCF_BATCH_AUTOTUNE])
def test_batch_equals_single_calls(graphs, flags):
    qs = make_queries(graphs)
    b = M.mcf_batch_create(qs, flags=flags)
    outs, st = M.mcf_batch_run(b, stats=True)
    assert st["walks"] > 0 and st["walk_steps"] > 0
    for q, out in zip(qs, outs):
        close(out, single(q))
    # a second run reproduces the first
    first = [np.array(o, copy=True) for o in outs]
    outs2 = M.mcf_batch_run(b)
    for a, o in zip(first, outs2):
        close(o, a)
    b.close()


def test_batch_device_outputs_and_oracle(graphs):
    g, h, gam = graphs["ba500"]
    c = R.exp_coeffs(30)
    out_tc = torch.empty(g.n, dtype=torch.float64, device="cuda")
    out_sc = torch.empty(g.n, dtype=torch.float64, device="cuda")
    qs = [dict(graph=h, kind=M.MCF_QUERY_TOTAL_COMMUNICABILITY, coeffs=c, scale=gam, walks_per_node=64, seed=3,
               request_id=1, precision=M.MCF_F32W_F64ACC, out=out_tc),
          dict(graph=h, kind=M.MCF_QUERY_SUBGRAPH_CENTRALITY, coeffs=c, scale=gam, walks_per_node=64, seed=3,
               request_id=1, precision=M.MCF_F32W_F64ACC, out=out_sc)]
    b = M.mcf_batch_create(qs, flags=M.MCF_BATCH_CUDA_GRAPH)
    M.mcf_batch_run(b)
    close(out_tc, E.action(g, c, gamma=gam, walks_per_node=64, seed=3, request_id=1, precision=1)["y"])
    close(out_sc, E.diag(g, c, gamma=gam, walks_per_node=64, seed=3, request_id=1, precision=1)["d"])
    b.close()


def test_batch_rejects_bad_queries(graphs):
    g, h, gam = graphs["ba500"]
    with pytest.raises(M.McfError):
        M.mcf_batch_create([dict(graph=h, kind=7, coeffs=[1.0, 1.0, 0.5], n_walks=10)])
    with pytest.raises(M.McfError):
        M.mcf_batch_create([dict(graph=h, kind=M.MCF_QUERY_KATZ, katz_gamma=2.0 * gam, walks_per_node=2)])
