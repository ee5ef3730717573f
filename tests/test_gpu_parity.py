"""Parity of the CUDA path (through the C ABI) with the oracle.

Same seed -> same walks: the GPU estimate must equal the oracle's estimator
up to float64 summation order, |gpu - oracle| <= 1e-12 |oracle| per entry
(plus 1e-13 absolute for entries near zero).  Both precisions are covered:
in MCF_F32W_F64ACC every float32 product is rounded identically on both
sides, so the same bound holds.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import estimator as E
from oracle import reference as R
from paper_2308_01037_gb300 import inputs as I
from paper_2308_01037_gb300 import mcf as M

pytestmark = pytest.mark.gpu

RTOL = 1e-12
ATOL = 1e-13


def assert_parity(gpu, ref, rtol=RTOL, atol=ATOL):
    gpu = np.asarray(gpu.cpu() if hasattr(gpu, "cpu") else gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert gpu.shape == ref.shape
    err = np.abs(gpu - ref)
    bound = rtol * np.abs(ref) + atol
    bad = np.nonzero(err > bound)[0]
    assert bad.size == 0, f"{bad.size} entries off; worst rel {np.max(err / np.maximum(np.abs(ref), 1e-300)):.3e} at {bad[:5]}"


def upload(g, values=None, device=False):
    if device:
        return M.mcf_create_graph(g.n, torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col_idx).cuda(),
                                  None if values is None else torch.from_numpy(values).cuda())
    return M.mcf_create_graph(g.n, g.row_ptr, g.col_idx, values)


@pytest.fixture(scope="module")
def ba1000():
    g = I.barabasi_albert(1000, 3, 0)
    lam = R.lambda_max(g)
    return g, upload(g), 1.0 / lam


@pytest.fixture(scope="module")
def rmat12():
    g = I.rmat(12, 16, seed=5)          # 4096 nodes, ragged degrees, isolated nodes
    lam = R.lambda_max(g)
    return g, upload(g), 1.0 / lam


# ------------------------------------------------------------------ total communicability / action
@pytest.mark.parametrize("precision", [M.MCF_F64, M.MCF_F32W_F64ACC])
def test_total_communicability_walks_per_node(ba1000, precision):
    g, h, gam = ba1000
    c = R.exp_coeffs(30)
    kw = dict(scale=gam, walks_per_node=200, seed=11, request_id=3, precision=precision)
    y, st = M.mcf_total_communicability(h, c, stats=True, **kw)
    ref = E.action(g, c, gamma=gam, walks_per_node=200, seed=11, request_id=3, precision=precision)
    assert_parity(y, ref["y"])
    assert st["walks"] == ref["walks"] and st["walk_steps"] == ref["steps"]


@pytest.mark.parametrize("precision", [M.MCF_F64, M.MCF_F32W_F64ACC])
def test_total_communicability_allocation_and_cutoff(rmat12, precision):
    g, h, gam = rmat12
    c = R.exp_coeffs(30)
    kw = dict(scale=gam, n_walks=300000, w_cutoff=1e-6, seed=2, precision=precision)
    y, st = M.mcf_total_communicability(h, c, stats=True, **kw)
    ref = E.action(g, c, gamma=gam, n_walks=300000, w_cutoff=1e-6, seed=2, precision=precision)
    assert_parity(y, ref["y"])
    assert st["walks"] == ref["walks"] and st["walk_steps"] == ref["steps"]


def test_action_general_vector_device_buffers(rmat12):
    g, h, gam = rmat12
    c = R.exp_coeffs(20, beta=0.5)
    v = np.random.default_rng(4).standard_normal(g.n)
    vd = torch.from_numpy(v).cuda()
    y = M.mcf_action(h, vd, c, scale=gam, n_walks=100000, seed=9, precision=M.MCF_F32W_F64ACC)
    assert y.is_cuda
    ref = E.action(g, c, v=v, gamma=gam, n_walks=100000, seed=9, precision=1)
    assert_parity(y, ref["y"])


def test_default_host_outputs_are_page_locked(rmat12):
    """Without an ``out``, host results come back in page-locked memory (the
    library's device-to-host copy is then a plain DMA), as numpy arrays equal
    to the device-output result of the same walks."""
    g, h, gam = rmat12
    c = R.exp_coeffs(20)
    kw = dict(scale=gam, n_walks=50000, seed=3, precision=M.MCF_F32W_F64ACC)
    y = M.mcf_total_communicability(h, c, **kw)
    assert isinstance(y, np.ndarray) and torch.from_numpy(y).is_pinned()
    yd = M.mcf_total_communicability(h, c, out=torch.empty(g.n, dtype=torch.float64, device="cuda"), **kw)
    assert_parity(y, yd.cpu().numpy())
    b = M.mcf_batch_create([dict(graph=h, kind=M.MCF_QUERY_TOTAL_COMMUNICABILITY, coeffs=c, **kw)])
    (yb,) = M.mcf_batch_run(b)
    b.close()
    assert torch.from_numpy(yb).is_pinned()
    assert_parity(yb, yd.cpu().numpy())


def test_katz_explicit_terms(ba1000):
    g, h, gam = ba1000
    gk = 0.85 * gam
    K = 40
    y = M.mcf_katz(h, gk, K, walks_per_node=100, seed=5, precision=M.MCF_F64)
    ref = E.action(g, R.katz_coeffs(K), gamma=gk, walks_per_node=100, seed=5, precision=0)
    assert_parity(y, ref["y"])


def test_katz_terms_from_tail_bound(ba1000):
    g, h, gam = ba1000
    lam = M.mcf_spectral_radius(h)
    gk = 0.85 / lam
    K = R.katz_terms_for_tail(gk * lam, 1e-4)
    y = M.mcf_katz(h, gk, 0, walks_per_node=50, seed=6, precision=M.MCF_F32W_F64ACC)
    ref = E.action(g, R.katz_coeffs(K), gamma=gk, walks_per_node=50, seed=6, precision=1)
    assert_parity(y, ref["y"])


@pytest.mark.parametrize("precision", [M.MCF_F64, M.MCF_F32W_F64ACC])
def test_weighted_signed_matrix(precision):
    g = I.barabasi_albert(700, 4, 12)
    w = I.symmetric_weights(g, seed=1, signed=True)
    A = R.csr_matrix(g, w)
    gam = 1.0 / np.abs(np.linalg.eigvalsh(A.toarray())).max()
    h = upload(g, w)
    c = R.exp_coeffs(25)
    v = np.random.default_rng(2).uniform(0.5, 1.5, g.n)
    y = M.mcf_action(h, v, c, scale=gam, walks_per_node=64, seed=8, precision=precision)
    ref = E.action(g, c, v=v, gamma=gam, walks_per_node=64, seed=8, precision=precision, values=w)
    assert_parity(y, ref["y"])
    d = M.mcf_subgraph_centrality(h, c, scale=gam, walks_per_node=64, seed=8, precision=precision)
    refd = E.diag(g, c, gamma=gam, walks_per_node=64, seed=8, precision=precision, values=w)
    assert_parity(d, refd["d"])


@pytest.mark.parametrize("precision", [M.MCF_F64, M.MCF_F32W_F64ACC])
def test_action_node_subset_equals_full_run(rmat12, precision):
    """Single-entry / subset total communicability (Section 4.3): the entries equal the
    full run's (same walk ids) and the oracle's subset computation."""
    g, h, gam = rmat12
    c = R.exp_coeffs(30)
    hub = int(np.argmax(g.degree))
    nodes = np.array([hub, 3, 3, g.n - 1, 100, 2047], dtype=np.int64)
    kw = dict(scale=gam, n_walks=200000, w_cutoff=1e-6, seed=6, precision=precision)
    sub, st = M.mcf_action_nodes(h, nodes, c, stats=True, **kw)
    full = M.mcf_total_communicability(h, c, **kw)
    assert_parity(sub, full[nodes])
    ref = E.action(g, c, gamma=gam, n_walks=200000, w_cutoff=1e-6, seed=6, precision=precision, nodes=nodes)
    assert_parity(sub, ref["y"])
    assert st["walks"] == ref["walks"] and st["walk_steps"] == ref["steps"]
    v = np.random.default_rng(5).standard_normal(g.n)
    dsub = M.mcf_action_nodes(h, torch.from_numpy(nodes).cuda(), c, v=torch.from_numpy(v).cuda(), **kw)
    assert_parity(dsub.cpu().numpy(), M.mcf_action(h, v, c, **kw)[nodes])


# ------------------------------------------------------------------ subgraph centrality
@pytest.mark.parametrize("precision", [M.MCF_F64, M.MCF_F32W_F64ACC])
def test_subgraph_centrality_dense_row(ba1000, precision):
    g, h, gam = ba1000
    c = R.exp_coeffs(30)
    d, st = M.mcf_subgraph_centrality(h, c, scale=gam, walks_per_node=300, seed=21, precision=precision, stats=True)
    ref = E.diag(g, c, gamma=gam, walks_per_node=300, seed=21, precision=precision)
    assert_parity(d, ref["d"])
    assert st["walks"] == ref["walks"] and st["walk_steps"] == ref["steps"]


@pytest.mark.parametrize("precision", [M.MCF_F64, M.MCF_F32W_F64ACC])
def test_subgraph_centrality_hashed_row_with_flushes(precision):
    # n > 16384 selects the hashed row Q_k (at most 2^12 slots); 3000 walks of up
    # to 28 steps from a hub overflow it, exercising the flush-and-replay path
    g = I.rmat(15, 16, seed=7)
    gam = 1.0 / R.lambda_max(g)
    h = upload(g)
    c = R.exp_coeffs(30)
    hub = int(np.argmax(g.degree))
    nodes = np.array([hub, 0, 1, 77, g.n - 1, hub], dtype=np.int64)
    d = M.mcf_subgraph_centrality(h, c, nodes=nodes, scale=gam, walks_per_node=3000, seed=4, precision=precision)
    ref = E.diag(g, c, gamma=gam, walks_per_node=3000, seed=4, precision=precision, nodes=nodes)
    assert_parity(d, ref["d"])


@pytest.mark.timeout(600)
def test_subgraph_centrality_subset_hashed_rows_neighbour_records():
    """A node subset on a graph with >= 2^20 entries and n > 16384: rows Q_k
    keyed by row offset in a shared-memory table, 8-byte walk records and the
    per-column lists of requested rows together.  Nodes: the top hub, three of its neighbours, a low-degree node,
    an isolated node if any, and a duplicate; only the columns adjacent to them
    are walked, and the dot phase of a hub column touches only the listed rows."""
    g = I.rmat(16, 16, seed=9)
    assert g.nnz >= 1 << 20 and g.n > 16384
    gam = 1.0 / R.lambda_max(g)
    h = upload(g)
    c = R.exp_coeffs(30)
    hub = int(np.argmax(g.degree))
    nbrs = g.col_idx[g.row_ptr[hub]:g.row_ptr[hub + 1]]
    low = int(np.nonzero(g.degree == 1)[0][0]) if np.any(g.degree == 1) else 3
    iso = np.nonzero(g.degree == 0)[0]
    nodes = [hub, int(nbrs[0]), int(nbrs[len(nbrs) // 2]), int(nbrs[-1]), low, hub]
    if iso.size:
        nodes.append(int(iso[0]))
    nodes = np.array(nodes, dtype=np.int64)
    kw = dict(scale=gam, walks_per_node=16, w_cutoff=1e-6, seed=12, precision=M.MCF_F32W_F64ACC)
    d, st = M.mcf_subgraph_centrality(h, c, nodes=nodes, stats=True, **kw)
    ref = E.diag(g, c, gamma=gam, walks_per_node=16, w_cutoff=1e-6, seed=12, precision=1, nodes=nodes)
    assert_parity(d, ref["d"])
    assert st["walks"] == ref["walks"] and st["walk_steps"] == ref["steps"]
    # the same entries from device-resident indices
    d2 = M.mcf_subgraph_centrality(h, c, nodes=torch.from_numpy(nodes).cuda(), **kw)
    assert_parity(d2.cpu().numpy(), ref["d"])


@pytest.mark.timeout(600)
def test_subgraph_centrality_hub_rows_longer_than_the_table():
    """A hub joined to all of 20,000 nodes of a random graph (n > 16384: rows
    keyed by row offset): a row far longer than a start's table takes the
    path that looks the table's keys up in the row.  Full solve and a node
    subset holding the hub (twice), against the oracle."""
    rng = np.random.default_rng(21)
    n = 20001
    a, b = rng.integers(1, n, size=60000), rng.integers(1, n, size=60000)
    e = np.concatenate([np.stack([np.zeros(n - 1, dtype=np.int64), np.arange(1, n)], 1),
                        np.stack([a[a != b], b[a != b]], 1)])
    e = np.unique(np.sort(e, axis=1), axis=0)
    g = I.from_edges(n, e, "star+er")
    assert g.degree[0] == n - 1
    gam = 1.0 / R.lambda_max(g)
    h = upload(g)
    c = R.exp_coeffs(30)
    kw = dict(scale=gam, walks_per_node=4, w_cutoff=1e-6, seed=13, precision=M.MCF_F32W_F64ACC)
    ref = E.diag(g, c, gamma=gam, walks_per_node=4, w_cutoff=1e-6, seed=13, precision=1)
    assert_parity(M.mcf_subgraph_centrality(h, c, **kw), ref["d"])
    nodes = np.array([0, 1, 2, 500, 0], dtype=np.int64)
    refs = E.diag(g, c, gamma=gam, walks_per_node=4, w_cutoff=1e-6, seed=13, precision=1, nodes=nodes)
    assert_parity(M.mcf_subgraph_centrality(h, c, nodes=nodes, **kw), refs["d"])


def test_subgraph_centrality_subset_weighted_signed():
    """The per-column lists carry the entries a_ik of a weighted, signed A."""
    g = I.barabasi_albert(400, 3, 5)
    vals = I.symmetric_weights(g, seed=6, signed=True)
    h = upload(g, vals)
    gam = 0.05
    c = R.exp_coeffs(12)
    nodes = np.array([0, 7, 399, 7, 123], dtype=np.int64)
    for precision in (M.MCF_F64, M.MCF_F32W_F64ACC):
        d = M.mcf_subgraph_centrality(h, c, nodes=nodes, scale=gam, walks_per_node=200, seed=8, precision=precision)
        ref = E.diag(g, c, gamma=gam, walks_per_node=200, seed=8, precision=precision, nodes=nodes, values=vals)
        assert_parity(d, ref["d"])


def test_subgraph_centrality_subset_equals_full(ba1000):
    g, h, gam = ba1000
    c = R.exp_coeffs(30)
    kw = dict(scale=gam, walks_per_node=100, seed=3, precision=M.MCF_F64)
    full = M.mcf_subgraph_centrality(h, c, **kw)
    nodes = torch.tensor([5, 0, 999, 5, 17], dtype=torch.int64, device="cuda")
    sub = M.mcf_subgraph_centrality(h, c, nodes=nodes, **kw)
    assert sub.is_cuda
    assert_parity(sub.cpu().numpy(), full[nodes.cpu().numpy()])


# ------------------------------------------------------------------ accuracy vs the FP64 reference
def test_small_config_accuracy_vs_dense_expm(ba1000):
    """BA n=1000, m=3, A/lambda_max, exp truncated at K=30, 1e5 walks per node:
    relative l_inf error of TC and SC against dense eigh/expm below 1e-3."""
    g, h, gam = ba1000
    c = R.exp_coeffs(30)
    F = R.dense_funm(gam * g.dense(), c)
    y = M.mcf_total_communicability(h, c, scale=gam, walks_per_node=100000, seed=1, precision=M.MCF_F64)
    tc = F.sum(1)
    assert np.abs(y - tc).max() / np.abs(tc).max() < 1e-3
    d = M.mcf_subgraph_centrality(h, c, scale=gam, walks_per_node=100000, seed=1, precision=M.MCF_F64)
    sc = np.diag(F)
    assert np.abs(d - sc).max() / np.abs(sc).max() < 1e-3


# ------------------------------------------------------------------ graph preprocessing
def test_spectral_radius_and_gershgorin(rmat12):
    g, h, gam = rmat12
    lam = M.mcf_spectral_radius(h, tol=1e-12, max_iter=20000)
    assert lam == pytest.approx(1.0 / gam, rel=1e-9)
    assert M.mcf_gershgorin(h) == g.degree.max()
    info = M.mcf_graph_info(h)
    assert info == {"n": g.n, "nnz": g.nnz, "max_degree": int(g.degree.max()), "n_loops": 0}


def test_device_pointer_graph_upload(ba1000):
    g, _, gam = ba1000
    hd = upload(g, device=True)
    c = R.exp_coeffs(10)
    y = M.mcf_total_communicability(hd, c, scale=gam, walks_per_node=20, seed=1, precision=M.MCF_F64)
    ref = E.action(g, c, gamma=gam, walks_per_node=20, seed=1, precision=0)
    assert_parity(y, ref["y"])


@pytest.mark.parametrize("case", ["unsorted", "duplicate", "asymmetric", "range", "nan"])
def test_invalid_graphs_rejected(case):
    g = I.path(5)
    rp, ci = g.row_ptr.copy(), g.col_idx.copy()
    val = None
    if case == "unsorted":
        ci[1], ci[2] = ci[2], ci[1]
    elif case == "duplicate":
        ci[2] = ci[1]
    elif case == "asymmetric":
        ci[0] = 2
    elif case == "range":
        ci[-1] = 99
    elif case == "nan":
        val = np.ones(g.nnz, np.float32)
        val[3] = np.nan
    with pytest.raises(M.McfError) as ei:
        M.mcf_create_graph(g.n, rp, ci, val)
    assert ei.value.status == 2


# ------------------------------------------------------------------ edge cases
def test_degenerate_inputs():
    c = R.exp_coeffs(12)
    # isolated nodes only
    e = I.add_isolated(I.from_edges(1, np.zeros((0, 2))), 5)
    h = upload(e)
    assert np.all(M.mcf_total_communicability(h, c, n_walks=100) == 1.0)
    assert np.all(M.mcf_subgraph_centrality(h, c, n_walks=100) == 1.0)
    # empty graph
    z = I.Graph(0, np.zeros(1, np.int64), np.zeros(0, np.int32))
    hz = upload(z)
    assert M.mcf_total_communicability(hz, c, n_walks=10).shape == (0,)
    # series of degree <= 1: no walks at all
    g = I.path(6)
    hp = upload(g)
    y = M.mcf_total_communicability(hp, [2.0, 0.5], scale=0.5, n_walks=10)
    assert np.allclose(y, 2.0 + 0.5 * 0.5 * g.degree)
    d = M.mcf_subgraph_centrality(hp, [2.0], n_walks=10)
    assert np.all(d == 2.0)
    # empty node list
    assert M.mcf_subgraph_centrality(hp, c, nodes=np.zeros(0, np.int64), n_walks=10).shape == (0,)
    # out-of-range node
    with pytest.raises(M.McfError):
        M.mcf_subgraph_centrality(hp, c, nodes=np.array([6]), n_walks=10)
    # graph with isolated nodes appended: exact values on them
    gi = I.add_isolated(I.barabasi_albert(200, 2, 1), 7)
    hi = upload(gi)
    y = M.mcf_total_communicability(hi, c, scale=0.1, walks_per_node=10, seed=2, precision=M.MCF_F64)
    ref = E.action(gi, c, gamma=0.1, walks_per_node=10, seed=2)
    assert_parity(y, ref["y"])
    assert np.all(y[200:] == 1.0)


def test_repeat_calls_identical_and_request_ids_differ(ba1000):
    g, h, gam = ba1000
    c = R.exp_coeffs(30)
    kw = dict(scale=gam, walks_per_node=50, seed=7, precision=M.MCF_F32W_F64ACC)
    a = M.mcf_total_communicability(h, c, request_id=1, **kw)
    b = M.mcf_total_communicability(h, c, request_id=1, **kw)
    assert_parity(a, b, rtol=1e-13, atol=0)
    other = M.mcf_total_communicability(h, c, request_id=2, **kw)
    assert np.abs(other - a).max() > 1e-9


def test_mittag_leffler_coefficients(ba1000):
    """Other functions come through the coefficient list: E_{0.8,1.2}(A') v."""
    g, h, gam = ba1000
    c = R.mittag_leffler_coeffs(30, 0.8, 1.2)
    v = np.random.default_rng(5).uniform(0.5, 1.5, g.n)
    y = M.mcf_action(h, v, c, scale=gam, walks_per_node=64, seed=9, precision=M.MCF_F32W_F64ACC)
    assert_parity(y, E.action(g, c, v=v, gamma=gam, walks_per_node=64, seed=9, precision=1)["y"])
    ref = R.series_action(g, c, gam, v=v)
    assert np.abs(y - ref).max() / np.abs(ref).max() < 0.02
