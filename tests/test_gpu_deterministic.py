"""The deterministic mode of RandFunmAction solves (params.deterministic = 1):
each walk's value goes to a float64 slot of its own and a start's walks are
summed in walk order, so repeated runs give bit-identical results (float64
atomics add in arrival order and differ in the last bits from run to run),
equal to the oracle's same-seed estimate within the parity tolerance; solves
the mode does not cover say so."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import estimator as E
from oracle import reference as R
from paper_2308_01037_gb300 import inputs as I
from paper_2308_01037_gb300 import mcf as M

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-12, 1e-13


def close(got, ref):
    got = np.asarray(got)
    assert np.all(np.abs(got - ref) <= RTOL * np.abs(ref) + ATOL)


@pytest.mark.parametrize("precision", [M.MCF_F64, M.MCF_F32W_F64ACC])
def test_repeated_runs_are_bit_identical_and_match_the_oracle(precision):
    g = I.rmat(12, 16, seed=31)
    h = M.mcf_create_graph(g.n, g.row_ptr, g.col_idx)
    gam = 1.0 / M.mcf_spectral_radius(h)
    c = R.exp_coeffs(30)
    kw = dict(scale=gam, n_walks=40 * g.n, w_cutoff=1e-6, seed=8, request_id=2, precision=precision)
    a = M.mcf_total_communicability(h, c, deterministic=True, **kw)
    b = M.mcf_total_communicability(h, c, deterministic=True, **kw)
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
    close(a, E.action(g, c, gamma=gam, n_walks=40 * g.n, w_cutoff=1e-6, seed=8, request_id=2,
                      precision=precision)["y"])
    # general v (weighted path for float64), and a node subset
    v = np.random.default_rng(3).standard_normal(g.n)
    y1 = M.mcf_action(h, v, c, deterministic=True, **kw)
    y2 = M.mcf_action(h, v, c, deterministic=True, **kw)
    assert np.array_equal(y1.view(np.uint64), y2.view(np.uint64))
    close(y1, E.action(g, c, v=v, gamma=gam, n_walks=40 * g.n, w_cutoff=1e-6, seed=8, request_id=2,
                       precision=precision)["y"])
    nodes = np.array([5, 100, 4000], np.int64)
    ys = M.mcf_action_nodes(h, nodes, c, deterministic=True, **kw)
    close(ys, a[nodes])
    h.close()


def test_katz_and_uncovered_solves():
    g = I.barabasi_albert(1500, 4, 2)
    h = M.mcf_create_graph(g.n, g.row_ptr, g.col_idx)
    kg = 0.85 / M.mcf_gershgorin(h)
    kw = dict(walks_per_node=16, seed=4, precision=M.MCF_F32W_F64ACC, deterministic=True)
    a = M.mcf_katz(h, kg, 12, **kw)
    b = M.mcf_katz(h, kg, 12, **kw)
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
    close(a, E.action(g, R.katz_coeffs(12), gamma=kg, walks_per_node=16, seed=4, precision=1)["y"])
    with pytest.raises(M.McfError) as ei:
        M.mcf_subgraph_centrality(h, R.exp_coeffs(10), scale=0.1, **kw)
    assert ei.value.status == 10     # MCF_ERR_UNSUPPORTED
    h.close()
