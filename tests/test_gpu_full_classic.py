"""Parity of the dense RandFunm estimate (Algorithm 2) and of the classical
Monte Carlo method (Algorithm 1) on the GPU with the oracle.

Same seed -> same walks; the GPU sums in another order, so entries agree to
1e-12 relative (plus an absolute floor: 1e-13 for the non-negative binary
cases, 1e-12 of the largest entry where signed weights or a signed v let
sums cancel).
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


def assert_close(gpu, ref, atol=1e-13):
    gpu = np.asarray(gpu.cpu() if hasattr(gpu, "cpu") else gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert gpu.shape == ref.shape
    err = np.abs(gpu - ref)
    bad = np.argwhere(err > RTOL * np.abs(ref) + atol)
    assert bad.size == 0, f"{len(bad)} entries off, e.g. {bad[:3].tolist()}: max err {err.max():.3e}"


@pytest.fixture(scope="module")
def ba300():
    g = I.barabasi_albert(300, 3, 21)
    return g, M.mcf_create_graph(g.n, g.row_ptr, g.col_idx), 1.0 / R.lambda_max(g)


@pytest.fixture(scope="module")
def weighted():
    g = I.add_isolated(I.barabasi_albert(250, 3, 22), 3)
    w = I.symmetric_weights(g, seed=4, signed=True)
    gam = 1.0 / np.abs(np.linalg.eigvalsh(R.csr_matrix(g, w).toarray())).max()
    return g, w, M.mcf_create_graph(g.n, g.row_ptr, g.col_idx, w), gam


# ------------------------------------------------------------------ RandFunm, dense F
@pytest.mark.parametrize("precision", [M.MCF_F64, M.MCF_F32W_F64ACC])
@pytest.mark.parametrize("wc", [0.0, 1e-6])
def test_funm_full_matches_oracle(ba300, precision, wc):
    g, h, gam = ba300
    c = R.exp_coeffs(30)
    F, st = M.mcf_funm_full(h, c, scale=gam, walks_per_node=40, w_cutoff=wc, seed=5, request_id=2,
                            precision=precision, stats=True)
    ref = E.funm_full(g, c, gamma=gam, walks_per_node=40, w_cutoff=wc, seed=5, request_id=2, precision=precision)
    assert_close(F, ref)
    assert st["walks"] == 40 * g.n and st["walk_steps"] > 0


def test_funm_full_weighted_signed_with_isolated_nodes(weighted):
    g, w, h, gam = weighted
    c = R.exp_coeffs(20)
    F = M.mcf_funm_full(h, c, scale=gam, n_walks=30 * g.n, seed=9, precision=M.MCF_F32W_F64ACC)
    ref = E.funm_full(g, c, gamma=gam, n_walks=30 * g.n, seed=9, precision=1, values=w)
    assert_close(F, ref, atol=1e-12 * np.abs(ref).max())


def test_funm_full_diagonal_equals_subgraph_centrality(ba300):
    g, h, gam = ba300
    c = R.exp_coeffs(30)
    F = M.mcf_funm_full(h, c, scale=gam, walks_per_node=64, seed=3, precision=M.MCF_F32W_F64ACC)
    d = M.mcf_subgraph_centrality(h, c, scale=gam, walks_per_node=64, seed=3, precision=M.MCF_F32W_F64ACC)
    assert_close(np.diag(F), d)
    # the estimate is symmetric in expectation only; its error is the method's
    ex = R.dense_funm(R.csr_matrix(g, gamma=gam).toarray(), c)
    assert np.max(np.abs(F - ex)) / np.max(np.abs(ex)) < 0.05


def test_funm_full_short_series_and_device_output(ba300):
    g, h, gam = ba300
    for K in (0, 1):                     # no walks: F = zeta_0 I (+ zeta_1 A')
        c = R.exp_coeffs(K)
        out = torch.empty(g.n * g.n, dtype=torch.float64, device="cuda")
        F = M.mcf_funm_full(h, c, scale=gam, walks_per_node=4, out=out)
        A = R.csr_matrix(g).toarray()
        assert_close(F, c[0] * np.eye(g.n) + (c[1] * gam * A if K >= 1 else 0.0))


def test_funm_full_rejects_large_graphs():
    g = I.path(M.MCF_FULL_MAX_NODES + 1)
    h = M.mcf_create_graph(g.n, g.row_ptr, g.col_idx)
    with pytest.raises(M.McfError):
        M.mcf_funm_full(h, R.exp_coeffs(5), scale=0.5, walks_per_node=1)


# ------------------------------------------------------------------ classical Monte Carlo
@pytest.mark.parametrize("wc", [0.0, 1e-6])
def test_mc_classic_matches_oracle(ba300, wc):
    g, h, gam = ba300
    c = R.exp_coeffs(30)
    nodes = np.array([0, 7, 299, 150, 7, int(np.argmax(g.degree))], np.int64)
    y, st = M.mcf_mc_classic(h, c, 300, nodes=nodes, scale=gam, w_cutoff=wc, seed=4, request_id=1, stats=True)
    ref = E.mc_classic_action(g, c, nodes, 300, gamma=gam, w_cutoff=wc, seed=4, request_id=1)
    assert_close(y, ref)
    assert st["walks"] == 300 * len(nodes)


def test_mc_classic_all_rows_signed_v_weighted(weighted):
    g, w, h, gam = weighted
    c = R.exp_coeffs(20)
    v = np.random.default_rng(1).standard_normal(g.n)
    vd = torch.from_numpy(v).cuda()
    y = M.mcf_mc_classic(h, c, 37, v=vd, scale=gam, seed=2)          # ragged: 37 walks per row
    ref = E.mc_classic_action(g, c, np.arange(g.n), 37, v=v, gamma=gam, seed=2, values=w)
    assert_close(y, ref, atol=1e-12 * np.abs(ref).max())


def test_mc_classic_is_unbiased_and_noisier_than_row_sampling(ba300):
    """Both estimate f(A')1; at an equal number of walks the row-sampling
    estimator (Algorithm 3) has the smaller error (the paper's Section 4 claim)."""
    g, h, gam = ba300
    c = R.exp_coeffs(30)
    ex = R.series_action(g, c, gam)
    yc = M.mcf_mc_classic(h, c, 2000, scale=gam, seed=11)
    yr = M.mcf_total_communicability(h, c, scale=gam, walks_per_node=2000, seed=11, precision=M.MCF_F64)
    ec = np.max(np.abs(yc - ex) / ex)
    er = np.max(np.abs(yr - ex) / ex)
    assert ec < 0.05 and er < ec


def test_mc_classic_rejects_bad_arguments(ba300):
    g, h, gam = ba300
    with pytest.raises(M.McfError):
        M.mcf_mc_classic(h, R.exp_coeffs(5), 10, scale=gam, precision=M.MCF_F32W_F64ACC)
    with pytest.raises(M.McfError):
        M.mcf_mc_classic(h, R.exp_coeffs(5), 0, scale=gam)
    with pytest.raises(M.McfError):
        M.mcf_mc_classic(h, R.exp_coeffs(5), 10, nodes=np.array([g.n], np.int64), scale=gam)
