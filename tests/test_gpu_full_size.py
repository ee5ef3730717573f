"""Parity at the full sizes of the benchmark configurations, in the launch
configuration bench.py times: the GPU solves the whole problem; the oracle
computes sampled entries one by one (walks from their neighbours only, with
the full run's allocation and walk ids), and the sampled entries must agree
to 1e-12 relative.

* R-MAT scale 22 (4,194,304 nodes), total communicability, N_s = 1e8,
  K = 30, W_c = 1e-6, float32 walk weights (the default bench line);
* configuration model n = 2e6, k^-2.5, mean degree 20, subgraph centrality
  with 2000 walks per node, W_c = 1e-6, float32 walk weights;
* Barabasi-Albert n = 1000, m = 3, 1e5 walks per node, W_c = 0, float64:
  total communicability and subgraph centrality.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import estimator as E
from oracle import reference as R
from paper_2308_01037_gb300 import inputs as I
from paper_2308_01037_gb300 import mcf as M

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-12, 1e-13


def close(gpu, ref):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    err = np.abs(gpu - ref)
    bad = np.nonzero(err > RTOL * np.abs(ref) + ATOL)[0]
    assert bad.size == 0, f"{bad.size} sampled entries off; worst rel {np.max(err / np.abs(ref)):.3e}"


def device_graph(g):
    return M.mcf_create_graph(g.n, torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col_idx).cuda())


def test_rmat22_total_communicability_sampled_entries():
    g = I.rmat(22, 16, seed=1)
    h = device_graph(g)
    gam = 1.0 / M.mcf_spectral_radius(h, tol=1e-10, max_iter=10000)
    c = R.exp_coeffs(30)
    kw = dict(n_walks=100_000_000, w_cutoff=1e-6, seed=1, request_id=7)
    y = torch.empty(g.n, dtype=torch.float64, device="cuda")
    _, st = M.mcf_total_communicability(h, c, out=y, scale=gam, precision=M.MCF_F32W_F64ACC, stats=True, **kw)
    assert st["walks"] == 99_938_035
    # 24 random nodes and one of degree about 1000 (the hub's entry alone needs
    # 2.8e7 walks from its 162,307 neighbours: minutes for the oracle)
    rng = np.random.default_rng(22)
    mid = int(np.argmin(np.abs(g.degree - 1000)))
    nodes = np.concatenate([rng.choice(g.n, size=24, replace=False), [mid]]).astype(np.int64)
    ref = E.action(g, c, gamma=gam, precision=1, nodes=nodes, **kw)["y"]
    close(y.cpu().numpy()[nodes], ref)


def test_config_model_subgraph_centrality_sampled_entries():
    g = I.config_powerlaw(2_000_000, 2.5, 20.0, 2)
    h = device_graph(g)
    gam = 1.0 / M.mcf_spectral_radius(h, tol=1e-10, max_iter=10000)
    c = R.exp_coeffs(30)
    kw = dict(walks_per_node=2000, w_cutoff=1e-6, seed=3, request_id=3)
    d = torch.empty(g.n, dtype=torch.float64, device="cuda")
    M.mcf_subgraph_centrality(h, c, out=d, scale=gam, precision=M.MCF_F32W_F64ACC, **kw)
    rng = np.random.default_rng(3)
    nodes = rng.choice(g.n, size=8, replace=False).astype(np.int64)
    ref = E.diag(g, c, gamma=gam, precision=1, nodes=nodes, **kw)["d"]
    close(d.cpu().numpy()[nodes], ref)


def test_ba1000_float64_sampled_entries():
    g = I.barabasi_albert(1000, 3, 0)
    h = device_graph(g)
    gam = 1.0 / M.mcf_spectral_radius(h, tol=1e-10, max_iter=10000)
    c = R.exp_coeffs(30)
    kw = dict(walks_per_node=100_000, w_cutoff=0.0, seed=1, request_id=1)
    y = M.mcf_total_communicability(h, c, scale=gam, precision=M.MCF_F64, **kw)
    d = M.mcf_subgraph_centrality(h, c, scale=gam, precision=M.MCF_F64, **kw)
    nodes = np.array([17, 999], np.int64)
    close(y[nodes], E.action(g, c, gamma=gam, precision=0, nodes=nodes, **kw)["y"])
    close(d[nodes], E.diag(g, c, gamma=gam, precision=0, nodes=nodes, **kw)["d"])
    # and the whole vector against the float64 reference (the config's check)
    F = R.dense_funm(R.csr_matrix(g, gamma=gam).toarray(), c)
    assert np.max(np.abs(y - F.sum(1))) / np.max(np.abs(F.sum(1))) < 1e-3
    assert np.max(np.abs(d - np.diag(F))) / np.max(np.abs(np.diag(F))) < 1e-3
