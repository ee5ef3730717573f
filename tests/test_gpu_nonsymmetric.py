"""Parity of the CUDA path with the oracle on a general (non-symmetric) A
(graphs created with MCF_GRAPH_NONSYMMETRIC), and on the symmetrised digraph
B = [0 A; A^T 0] of the paper's Section 4.

Same seed -> same walks; entries agree to 1e-12 relative (an absolute floor
of 1e-12 of the largest entry where signed weights let sums cancel)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import estimator as E
from oracle import reference as R
from paper_2308_01037_gb300 import inputs as I
from paper_2308_01037_gb300 import mcf as M

pytestmark = pytest.mark.gpu

RTOL = 1e-12


def close(gpu, ref, atol=1e-13):
    gpu = np.asarray(gpu.cpu() if hasattr(gpu, "cpu") else gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert gpu.shape == ref.shape
    err = np.abs(gpu - ref)
    bad = np.argwhere(err > RTOL * np.abs(ref) + atol)
    assert bad.size == 0, f"{len(bad)} entries off, e.g. {bad[:3].tolist()}: max err {err.max():.3e}"


def signed(g, seed):
    rng = np.random.default_rng(seed)
    return (rng.uniform(0.25, 2.0, g.nnz) * rng.choice([-1.0, 1.0], g.nnz)).astype(np.float32)


@pytest.fixture(scope="module")
def dw():
    """Directed, signed weights, with sources and sinks."""
    g = I.directed_erdos_renyi(400, 5.0, 7)
    w = signed(g, 1)
    A = R.csr_matrix(g, w).toarray()
    gam = 0.9 / np.abs(np.linalg.eigvals(A)).max()
    return g, w, M.mcf_create_graph(g.n, g.row_ptr, g.col_idx, w, symmetric=False), gam


@pytest.fixture(scope="module")
def db():
    """Directed, binary, ragged in/out degrees (the neighbour-record walk path)."""
    g = I.directed_erdos_renyi(3000, 8.0, 8)
    gam = 0.9 / np.abs(np.linalg.eigvals(g.dense())).max()
    return g, M.mcf_create_graph(g.n, g.row_ptr, g.col_idx, symmetric=False), gam


@pytest.mark.parametrize("precision", [M.MCF_F64, M.MCF_F32W_F64ACC])
def test_action_and_diag_weighted_nonsymmetric(dw, precision):
    g, w, h, gam = dw
    c = R.exp_coeffs(25)
    v = np.random.default_rng(2).uniform(0.5, 1.5, g.n)
    y = M.mcf_action(h, v, c, scale=gam, walks_per_node=64, seed=3, precision=precision)
    ref = E.action(g, c, v=v, gamma=gam, walks_per_node=64, seed=3, precision=precision, values=w)["y"]
    close(y, ref, atol=1e-12 * np.abs(ref).max())
    y2 = M.mcf_action(h, v, c, scale=gam, n_walks=50 * g.n, seed=4, precision=precision)   # column-norm allocation
    ref2 = E.action(g, c, v=v, gamma=gam, n_walks=50 * g.n, seed=4, precision=precision, values=w)["y"]
    close(y2, ref2, atol=1e-12 * np.abs(ref2).max())
    d = M.mcf_subgraph_centrality(h, c, scale=gam, walks_per_node=64, seed=5, precision=precision)
    refd = E.diag(g, c, gamma=gam, walks_per_node=64, seed=5, precision=precision, values=w)["d"]
    close(d, refd, atol=1e-12 * np.abs(refd).max())


@pytest.mark.parametrize("precision", [M.MCF_F64, M.MCF_F32W_F64ACC])
def test_binary_nonsymmetric_tc_subset_and_diag(db, precision):
    g, h, gam = db
    c = R.exp_coeffs(30)
    y = M.mcf_total_communicability(h, c, scale=gam, n_walks=20 * g.n, w_cutoff=1e-6, seed=6, precision=precision)
    ref = E.action(g, c, gamma=gam, n_walks=20 * g.n, w_cutoff=1e-6, seed=6, precision=precision)["y"]
    close(y, ref)
    nodes = np.array([0, 17, 2999, 17, 1500], np.int64)
    ys = M.mcf_action_nodes(h, nodes, c, scale=gam, n_walks=20 * g.n, w_cutoff=1e-6, seed=6, precision=precision)
    close(ys, ref[nodes])
    d = M.mcf_subgraph_centrality(h, c, scale=gam, walks_per_node=40, seed=7, precision=precision)
    refd = E.diag(g, c, gamma=gam, walks_per_node=40, seed=7, precision=precision)["d"]
    close(d, refd)
    ds = M.mcf_subgraph_centrality(h, c, nodes=nodes, scale=gam, walks_per_node=40, seed=7, precision=precision)
    close(ds, refd[nodes])


def test_full_and_classic_nonsymmetric(dw):
    g, w, h, gam = dw
    c = R.exp_coeffs(20)
    F = M.mcf_funm_full(h, c, scale=gam, walks_per_node=30, seed=8, precision=M.MCF_F32W_F64ACC)
    ref = E.funm_full(g, c, gamma=gam, walks_per_node=30, seed=8, precision=1, values=w)
    close(F, ref, atol=1e-12 * np.abs(ref).max())
    v = np.random.default_rng(9).standard_normal(g.n)
    nodes = np.arange(0, g.n, 7, dtype=np.int64)
    y = M.mcf_mc_classic(h, c, 50, v=v, nodes=nodes, scale=gam, seed=9)
    refc = E.mc_classic_action(g, c, nodes, 50, v=v, gamma=gam, seed=9, values=w)
    close(y, refc, atol=1e-12 * np.abs(refc).max())


def test_directed_cycle_exact_on_gpu():
    n = 7
    g = I.directed_cycle(n)
    h = M.mcf_create_graph(g.n, g.row_ptr, g.col_idx, symmetric=False)
    c = np.random.default_rng(1).uniform(0.1, 1.0, 20)
    y = M.mcf_total_communicability(h, c, walks_per_node=1, seed=1, precision=M.MCF_F64)
    assert np.allclose(y, c.sum(), rtol=1e-14)
    d = M.mcf_subgraph_centrality(h, c, walks_per_node=1, seed=1, precision=M.MCF_F64)
    assert np.allclose(d, c[::n].sum(), rtol=1e-14)
    # float32 walk weights round the coefficients: equal to the oracle, near the closed form
    d32 = M.mcf_subgraph_centrality(h, c, walks_per_node=1, seed=1, precision=M.MCF_F32W_F64ACC)
    close(d32, E.diag(g, c, walks_per_node=1, seed=1, precision=1)["d"])
    assert np.allclose(d32, c[::n].sum(), rtol=1e-6)
    F = M.mcf_funm_full(h, c, walks_per_node=1, seed=1, precision=M.MCF_F64)
    assert np.allclose(F, R.dense_powers_series(g.dense(), c), rtol=1e-14, atol=1e-15)


def test_symmetric_graph_through_the_general_path_is_identical():
    """A symmetric A created as general reads the same values in the same order
    from its column-major copy: the allocation and every walk are identical,
    results equal up to the order of the float64 atomic sums."""
    g = I.barabasi_albert(600, 3, 4)
    w = I.symmetric_weights(g, seed=2, signed=True)
    gam = 1.0 / np.abs(np.linalg.eigvalsh(R.csr_matrix(g, w).toarray())).max()
    c = R.exp_coeffs(25)
    for vals in (None, w):
        hs = M.mcf_create_graph(g.n, g.row_ptr, g.col_idx, vals)
        hg = M.mcf_create_graph(g.n, g.row_ptr, g.col_idx, vals, symmetric=False)
        kw = dict(scale=gam, n_walks=30 * g.n, seed=2, precision=M.MCF_F32W_F64ACC)
        ys, st_s = M.mcf_total_communicability(hs, c, stats=True, **kw)
        yg, st_g = M.mcf_total_communicability(hg, c, stats=True, **kw)
        assert st_s["walks"] == st_g["walks"] and st_s["walk_steps"] == st_g["walk_steps"]
        close(yg, ys, atol=0.0)
        close(M.mcf_subgraph_centrality(hg, c, **kw), M.mcf_subgraph_centrality(hs, c, **kw), atol=0.0)


def test_batch_with_a_nonsymmetric_graph(db):
    g, h, gam = db
    c = R.exp_coeffs(30)
    qs = [dict(graph=h, kind=M.MCF_QUERY_TOTAL_COMMUNICABILITY, coeffs=c, scale=gam, n_walks=10 * g.n, seed=1,
               request_id=1, precision=M.MCF_F32W_F64ACC),
          dict(graph=h, kind=M.MCF_QUERY_SUBGRAPH_CENTRALITY, coeffs=c, scale=gam, walks_per_node=20, seed=2,
               request_id=2, precision=M.MCF_F32W_F64ACC),
          dict(graph=h, kind=M.MCF_QUERY_KATZ, katz_gamma=0.5 * gam, katz_terms=12, walks_per_node=8, seed=3,
               request_id=3, precision=M.MCF_F32W_F64ACC)]
    b = M.mcf_batch_create(qs, flags=M.MCF_BATCH_CUDA_GRAPH)
    outs = M.mcf_batch_run(b)
    b.close()
    close(outs[0], M.mcf_total_communicability(h, c, scale=gam, n_walks=10 * g.n, seed=1, request_id=1))
    close(outs[1], M.mcf_subgraph_centrality(h, c, scale=gam, walks_per_node=20, seed=2, request_id=2))
    close(outs[2], M.mcf_katz(h, 0.5 * gam, 12, walks_per_node=8, seed=3, request_id=3))
    close(outs[0], E.action(g, c, gamma=gam, n_walks=10 * g.n, seed=1, request_id=1, precision=1)["y"])


def test_nonsymmetric_limits(db):
    g, h, gam = db
    with pytest.raises(M.McfError):
        M.mcf_spectral_radius(h)
    with pytest.raises(M.McfError):
        M.mcf_katz(h, 0.5 * gam, 0, walks_per_node=4)
    assert M.mcf_gershgorin(h) == g.degree.max()
    # the symmetry check still rejects a directed graph created as symmetric
    with pytest.raises(M.McfError):
        M.mcf_create_graph(g.n, g.row_ptr, g.col_idx)


def test_bipartite_symmetrization_matches_oracle():
    d = I.directed_erdos_renyi(1500, 6.0, 9)
    b = I.bipartite_symmetrization(d)
    h = M.mcf_create_graph(b.n, b.row_ptr, b.col_idx)
    gam = 1.0 / M.mcf_spectral_radius(h)
    c = R.exp_coeffs(30)
    y = M.mcf_total_communicability(h, c, scale=gam, n_walks=20 * b.n, seed=3)
    close(y, E.action(b, c, gamma=gam, n_walks=20 * b.n, seed=3, precision=1)["y"])
    dd = M.mcf_subgraph_centrality(h, c, scale=gam, walks_per_node=30, seed=4)
    close(dd, E.diag(b, c, gamma=gam, walks_per_node=30, seed=4, precision=1)["d"])
