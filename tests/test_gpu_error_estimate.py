"""The standard-error estimate of RandFunmAction solves (params.error_estimate,
mcf_stats.max_rel_se) against the oracle's, which follows the estimator's
variance (Section 3.5) with the same walks: sample variance of each column's
walk sums, Var(y_j) = sum_i a'_ji^2 s_i^2 / N_i.  The two agree to rounding
(1e-8 relative: the sum-of-squares formula cancels a few digits)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import estimator as E
from oracle import reference as R
from paper_2308_01037_gb300 import inputs as I
from paper_2308_01037_gb300 import mcf as M

pytestmark = pytest.mark.gpu


def oracle_max_rel_se(g, c, nodes=None, **kw):
    y = E.action(g, c, nodes=nodes, **kw)["y"]
    se = E.action_se(g, c, nodes=nodes, **kw)
    ok = y != 0
    return float(np.max(se[ok] / np.abs(y[ok]))), y, se


@pytest.fixture(scope="module")
def ba():
    g = I.barabasi_albert(1500, 3, 7)
    return g, M.mcf_create_graph(g.n, g.row_ptr, g.col_idx), 1.0 / R.lambda_max(g)


@pytest.mark.parametrize("precision", [M.MCF_F64, M.MCF_F32W_F64ACC])
def test_total_communicability_standard_error(ba, precision):
    g, h, gam = ba
    c = R.exp_coeffs(30)
    kw = dict(gamma=gam, n_walks=40 * g.n, w_cutoff=1e-6, seed=3, request_id=2, precision=precision)
    ref, _, _ = oracle_max_rel_se(g, c, **kw)
    y, st = M.mcf_total_communicability(h, c, scale=gam, n_walks=40 * g.n, w_cutoff=1e-6, seed=3, request_id=2,
                                        precision=precision, stats=True, error_estimate=True)
    assert st["max_rel_se"] > 0
    assert st["max_rel_se"] == pytest.approx(ref, rel=1e-8)
    _, st0 = M.mcf_total_communicability(h, c, scale=gam, n_walks=40 * g.n, seed=3, precision=precision, stats=True)
    assert st0["max_rel_se"] == 0.0


@pytest.mark.parametrize("precision", [M.MCF_F64, M.MCF_F32W_F64ACC])
def test_weighted_action_and_subset_standard_error(precision):
    g = I.barabasi_albert(600, 3, 8)
    w = I.symmetric_weights(g, seed=2, signed=False)
    gam = 1.0 / np.abs(np.linalg.eigvalsh(R.csr_matrix(g, w).toarray())).max()
    h = M.mcf_create_graph(g.n, g.row_ptr, g.col_idx, w)
    c = R.exp_coeffs(25)
    v = np.random.default_rng(4).uniform(0.5, 1.5, g.n)
    kw = dict(gamma=gam, walks_per_node=50, seed=5, precision=precision, values=w)
    ref, _, _ = oracle_max_rel_se(g, c, v=v, **kw)
    _, st = M.mcf_action(h, v, c, scale=gam, walks_per_node=50, seed=5, precision=precision, stats=True,
                         error_estimate=True)
    assert st["max_rel_se"] == pytest.approx(ref, rel=1e-8)
    nodes = np.array([5, 0, 599, 5, 300], np.int64)
    ref_s, _, _ = oracle_max_rel_se(g, c, v=v, nodes=nodes, **kw)
    _, st_s = M.mcf_action_nodes(h, nodes, c, v=v, scale=gam, walks_per_node=50, seed=5, precision=precision,
                                 stats=True, error_estimate=True)
    assert st_s["max_rel_se"] == pytest.approx(ref_s, rel=1e-8)


def test_standard_error_predicts_the_error(ba):
    """The estimate is a real standard error: the error against the float64
    series stays within a few of them, and shrinks like 1/sqrt(N_s)."""
    g, h, gam = ba
    c = R.exp_coeffs(30)
    ex = R.series_action(g, c, gam)
    ratios = []
    for nw in (10 * g.n, 160 * g.n):
        y, st = M.mcf_total_communicability(h, c, scale=gam, n_walks=nw, seed=9, precision=M.MCF_F64, stats=True,
                                            error_estimate=True)
        err = float(np.max(np.abs(y - ex) / np.abs(ex)))
        assert err < 6 * st["max_rel_se"]
        ratios.append(st["max_rel_se"])
    assert 3.0 < ratios[0] / ratios[1] < 5.3      # sqrt(16) = 4


def test_katz_standard_error(ba):
    g, h, gam = ba
    y, st = M.mcf_katz(h, 0.5 * gam, 20, walks_per_node=16, seed=2, stats=True, error_estimate=True)
    ref, _, _ = oracle_max_rel_se(g, R.katz_coeffs(20), gamma=0.5 * gam, walks_per_node=16, seed=2, precision=1)
    assert st["max_rel_se"] == pytest.approx(ref, rel=1e-8)
