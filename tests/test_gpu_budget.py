"""Accuracy-targeted solves and the second-moment growth factor, on the GPU.

* mcf_second_moment_radius against the oracle's dense / ARPACK value of
  rho(diag(s')|A'|) (the growth of the walk weights' second moments, which
  decides whether the estimator's variance stays bounded, Theorem 1);
* a solve with params.target_rel_err runs replicas of the plain solve with
  seeds seed + r * 0x9E3779B97F4A7C15: its mean equals the mean of the
  oracle's same-seed replicas (parity, 1e-12), and replica 0 is the plain
  solve;
* budgeted total communicability, subgraph centrality and Katz on
  Barabasi-Albert, Erdos-Renyi and R-MAT graphs land within 1e-3 of the
  float64 series (relative l_inf), or the call says it could not
  (MCF_ERR_ACCURACY_BUDGET) -- Katz with gamma = 0.85 / lambda_max on a graph
  whose second-moment radius exceeds 1 is such a case.
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
GOLDEN = 0x9E3779B97F4A7C15


def rel_linf(y, ref):
    return float(np.max(np.abs(np.asarray(y) - ref)) / np.max(np.abs(ref)))


def upload(g):
    return M.mcf_create_graph(g.n, g.row_ptr, g.col_idx)


@pytest.mark.parametrize("name", ["ba", "rmat"])
def test_second_moment_radius_matches_oracle(name):
    g = I.barabasi_albert(1500, 4, 3) if name == "ba" else I.rmat(13, 16, seed=4)
    h = upload(g)
    lam = M.mcf_spectral_radius(h)
    for gam in (0.85 / lam, 0.85 / M.mcf_gershgorin(h)):
        rho = M.mcf_second_moment_radius(h, gam, tol=1e-12, max_iter=20000)
        assert rho == pytest.approx(R.second_moment_radius(g, gam), rel=1e-6)
    h.close()


def test_budgeted_mean_equals_the_oracle_replicas():
    g = I.barabasi_albert(800, 3, 7)
    h = upload(g)
    gam = 1.0 / M.mcf_spectral_radius(h)
    c = R.exp_coeffs(30)
    base = dict(scale=gam, walks_per_node=8, w_cutoff=1e-6, seed=5, request_id=3, precision=M.MCF_F32W_F64ACC)
    # a loose target: the first two replicas meet it
    y, st = M.mcf_total_communicability(h, c, target_rel_err=0.5, stats=True, **base)
    assert st["replicas"] == 2 and st["budget_met"]
    reps = [E.action(g, c, gamma=gam, walks_per_node=8, w_cutoff=1e-6, seed=(5 + r * GOLDEN) % (1 << 64),
                     request_id=3, precision=1)["y"] for r in range(2)]
    ref = np.mean(reps, axis=0)
    assert np.all(np.abs(y - ref) <= RTOL * np.abs(ref) + ATOL)
    # replica 0 is the plain solve
    plain = M.mcf_total_communicability(h, c, **base)
    assert np.all(np.abs(plain - reps[0]) <= RTOL * np.abs(reps[0]) + ATOL)
    # a tighter target on subgraph centrality: more replicas, same identity
    nodes = np.array([0, 5, 799, 5], np.int64)
    d, st = M.mcf_subgraph_centrality(h, c, nodes=nodes, target_rel_err=1e-4, stats=True,
                                      **dict(base, walks_per_node=16))
    R_ = st["replicas"]
    assert 2 < R_ <= 4096 and R_ % 2 == 0
    reps = [E.diag(g, c, gamma=gam, walks_per_node=16, w_cutoff=1e-6, seed=(5 + r * GOLDEN) % (1 << 64),
                   request_id=3, precision=1, nodes=nodes)["d"] for r in range(R_)]
    ref = np.mean(reps, axis=0)
    assert np.all(np.abs(d - ref) <= RTOL * np.abs(ref) + ATOL)
    h.close()


@pytest.mark.timeout(900)
@pytest.mark.parametrize("name", ["ba", "er", "rmat"])
def test_budgeted_solves_meet_1e3_against_the_float64_series(name):
    g = {"ba": lambda: I.barabasi_albert(3000, 4, 11), "er": lambda: I.erdos_renyi(3000, 12.0, 12),
         "rmat": lambda: I.rmat(12, 16, seed=13)}[name]()
    h = upload(g)
    lam = M.mcf_spectral_radius(h)
    gam = 1.0 / lam
    c = R.exp_coeffs(30)
    kw = dict(scale=gam, walks_per_node=32, w_cutoff=1e-6, seed=9, precision=M.MCF_F32W_F64ACC,
              target_rel_err=2.5e-4, stats=True)
    y, st = M.mcf_total_communicability(h, c, **kw)
    assert st["budget_met"] and st["est_rel_err"] <= 2.5e-4
    assert rel_linf(y, R.series_action(g, c, gam)) < 1e-3
    nodes = np.random.default_rng(1).choice(g.n, 200, replace=False).astype(np.int64)
    d, st = M.mcf_subgraph_centrality(h, c, nodes=nodes, **kw)
    assert st["budget_met"]
    assert rel_linf(d, R.series_diag(g, c, nodes, gam)) < 1e-3
    # Katz at the Gershgorin gamma (Section 4.5): Theorem 1's condition holds
    kg = 0.85 / M.mcf_gershgorin(h)
    K = R.katz_terms_for_tail(kg * lam, 1e-4)
    y, st = M.mcf_katz(h, kg, 0, **dict(kw, scale=0.0))
    assert st["budget_met"]
    assert rel_linf(y, R.series_action(g, R.katz_coeffs(K), kg)) < 1e-3
    h.close()


def test_katz_at_085_over_lambda_meets_the_target_or_says_so():
    """gamma = 0.85 / lambda_max on a Barabasi-Albert graph: the second-moment
    radius is above 1, so the variance grows with K; within a walk cap the
    solve either meets 1e-3 or returns MCF_ERR_ACCURACY_BUDGET with its mean."""
    g = I.barabasi_albert(2000, 3, 21)
    h = upload(g)
    lam = M.mcf_spectral_radius(h)
    gam = 0.85 / lam
    rho2 = M.mcf_second_moment_radius(h, gam)
    assert rho2 > 1.0
    K = R.katz_terms_for_tail(0.85, 1e-4)
    ref = R.series_action(g, R.katz_coeffs(K), gam)
    y, st = M.mcf_katz(h, gam, 0, walks_per_node=4, seed=3, precision=M.MCF_F32W_F64ACC, target_rel_err=5e-4,
                       max_walks=40 * g.n * 4, stats=True)
    if st["budget_met"]:
        assert rel_linf(y, ref) < 1e-3
    else:
        assert st["est_rel_err"] > 5e-4 and st["walks"] <= 40 * g.n * 4
    with pytest.raises(M.McfError) as ei:     # without stats the binding raises
        M.mcf_katz(h, gam, 0, walks_per_node=4, seed=3, precision=M.MCF_F32W_F64ACC, target_rel_err=1e-9,
                   max_walks=8 * g.n)
    assert ei.value.status == 8
    h.close()
