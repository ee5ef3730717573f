"""Pins of the C estimator (oracle part 1) against what the paper and the
mathematics fix: Lemma 2's exact expectation (by enumerating every walk),
exactness of degree <= 2 polynomials, zero variance on regular graphs,
closed forms, the trace invariant, the N_s^-1/2 error decay (Theorem 1),
the walk allocation of Definition 1, the cutoff of Eq. weight_cutoff and the
equality of RandFunmDiag with the diagonal of RandFunm (Algorithm 2)."""
import math

import numpy as np
import pytest

from oracle import estimator as E
from oracle import reference as R
from paper_2308_01037_gb300 import inputs as I

Z_MAX = 5.0   # |mean - exact| / sigma bound over a handful of entries


@pytest.fixture(scope="module")
def ba12():
    return I.barabasi_albert(12, 2, 3)


def _zscore(est, mean, var):
    sd = np.sqrt(var)
    ok = sd > 0
    z = np.zeros_like(est)
    z[ok] = (est[ok] - mean[ok]) / sd[ok]
    assert np.all(np.abs(est[~ok] - mean[~ok]) <= 1e-12 * np.maximum(1, np.abs(mean[~ok])))
    return np.abs(z).max()


# ------------------------------------------------------------ allocation (Definition 1)
def test_allocation_rule_star_by_hand():
    """Star S_5, gamma = 0.5: ||C_0|| = 0.5*2 = 1, ||C_leaf|| = 0.5, p_0 = 1/3, p_leaf = 1/6.
    N_s = 100 -> N_0 = llround(33.33) = 33, N_leaf = llround(16.67) = 17."""
    g = I.star(5)
    ra, cn, nw, off = E.allocation(g, gamma=0.5, n_walks=100)
    assert ra.tolist() == [2.0, 0.5, 0.5, 0.5, 0.5]
    assert cn.tolist() == [1.0, 0.5, 0.5, 0.5, 0.5]
    assert nw.tolist() == [33, 17, 17, 17, 17]
    assert off.tolist() == [0, 33, 50, 67, 84, 101]


def test_allocation_rounding_floor_and_isolated():
    """A node with N_s p_i < 0.5 still gets one walk; an empty column gets none."""
    g = I.add_isolated(I.star(5), 2)
    _, _, nw, off = E.allocation(g, gamma=1.0, n_walks=3)
    # p_0 = 2/6, p_leaf = 1/6: 3*2/6 = 1.0 -> 1, 3/6 = 0.5 -> llround 1 (half away from zero)
    assert nw.tolist() == [1, 1, 1, 1, 1, 0, 0]
    # N_s = 2: 2/6 = 0.33 rounds to 0, and the floor of one walk lifts every leaf to 1
    _, _, nw, off = E.allocation(g, gamma=1.0, n_walks=2)
    assert nw.tolist() == [1, 1, 1, 1, 1, 0, 0] and off[-1] == 5
    _, _, nw, _ = E.allocation(g, gamma=1.0, n_walks=0, walks_per_node=4)
    assert nw.tolist() == [4, 4, 4, 4, 4, 0, 0]


def test_allocation_weighted_norms():
    g = I.path(3)
    w = np.array([2.0, 2.0, -3.0, -3.0], np.float32)   # a01 = 2, a12 = -3
    ra, cn, _, _ = E.allocation(g, gamma=0.5, walks_per_node=1, values=w)
    assert ra.tolist() == [1.0, 2.5, 1.5]
    assert cn.tolist() == pytest.approx([1.0, 0.5 * math.sqrt(13.0), 1.5], rel=1e-15)


def test_alias_table_reproduces_row_distribution():
    a = np.array([0.5, -2.0, 1.0, 0.25, 3.0, 1.25], np.float32)
    prob, alias = E.alias_row(a)
    d = len(a)
    implied = np.zeros(d)
    for b in range(d):
        implied[b] += prob[b] / d
        implied[alias[b]] += (1 - prob[b]) / d
    assert np.allclose(implied, np.abs(a) / np.abs(a).sum(), rtol=1e-6, atol=1e-7)


# ------------------------------------------------------------ exactness
def test_degree_two_polynomial_is_exact(ba12):
    """With zeta_k = 0 for k > 2 only the k = 0 term of Eq. random_walk_realization
    survives: W^(0) r_{l0} is deterministic, so one walk per node is exact."""
    g = ba12
    gam = 0.3
    c = np.array([0.7, -1.3, 0.45])
    A = gam * g.dense()
    v = np.random.default_rng(0).standard_normal(g.n)
    y = E.action(g, c, v=v, gamma=gam, walks_per_node=1, seed=9)["y"]
    exact = c[0] * v + c[1] * A @ v + c[2] * A @ A @ v
    assert np.allclose(y, exact, rtol=1e-13, atol=1e-13)
    d = E.diag(g, c, gamma=gam, walks_per_node=1, seed=9)["d"]
    assert np.allclose(d, c[0] + c[2] * np.diag(A @ A), rtol=1e-13, atol=1e-13)


def test_degree_two_polynomial_with_loops_is_exact():
    """A symmetric signed A with loops: a'_ii enters d_i through zeta_1 (the
    zeta_1 A' term of Eq. rand_funm_formula_diag) and F = zeta_0 I + zeta_1 A'
    + zeta_2 A'^2 for Algorithm 2; with zeta_k = 0 for k > 2 one walk per
    node is exact for all three estimators."""
    n = 8
    und = np.array([(0, 1), (1, 2), (2, 3), (3, 0), (1, 5), (4, 5), (5, 6), (6, 7), (2, 6)])
    loops = np.array([1, 4, 6])
    src = np.concatenate([und[:, 0], und[:, 1], loops])
    dst = np.concatenate([und[:, 1], und[:, 0], loops])
    g = I.directed_from_edges(n, src, dst)
    A0 = g.dense()
    assert np.array_equal(A0, A0.T) and np.count_nonzero(np.diag(A0)) == 3
    # symmetric signed values: the value of (i, j) is that of (min, max)
    rows = np.repeat(np.arange(n), np.diff(g.row_ptr))
    cols = g.col_idx.astype(np.int64)
    rng = np.random.default_rng(11)
    table = rng.uniform(0.5, 1.5, (n, n)) * rng.choice([-1.0, 1.0], (n, n))
    w = table[np.minimum(rows, cols), np.maximum(rows, cols)].astype(np.float32)
    gam = 0.4
    A = gam * R.csr_matrix(g, w).toarray()
    c = np.array([0.6, -1.1, 0.35])
    exact_F = c[0] * np.eye(n) + c[1] * A + c[2] * A @ A
    v = rng.standard_normal(n)
    y = E.action(g, c, v=v, gamma=gam, walks_per_node=1, seed=2, values=w)["y"]
    assert np.allclose(y, exact_F @ v, rtol=1e-13, atol=1e-13)
    d = E.diag(g, c, gamma=gam, walks_per_node=1, seed=2, values=w)["d"]
    assert np.allclose(d, np.diag(exact_F), rtol=1e-13, atol=1e-13)
    F = E.funm_full(g, c, gamma=gam, walks_per_node=1, seed=2, values=w)
    assert np.allclose(F, exact_F, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("G", [lambda: I.complete(7), lambda: I.cycle(9)])
def test_regular_graph_total_communicability_has_zero_variance(G):
    """On a d-regular graph W^(k) = (gamma d)^k and r = gamma d for every walk."""
    g = G()
    d = int(g.degree[0])
    gam = 0.9 / d
    c = R.exp_coeffs(12)
    y = E.action(g, c, gamma=gam, walks_per_node=3, seed=4)["y"]
    assert np.allclose(y, sum(ck * (gam * d) ** k for k, ck in enumerate(c)), rtol=1e-14, atol=0)
    K = 40
    yk = E.action(g, R.katz_coeffs(K), gamma=gam, walks_per_node=2, seed=4)["y"]
    assert np.allclose(yk, sum((gam * d) ** k for k in range(K + 1)), rtol=1e-14, atol=0)


# ------------------------------------------------------------ Lemma 2 by enumeration
@pytest.mark.parametrize("K", [2, 3, 5, 7])
def test_enumeration_reproduces_truncated_series(ba12, K):
    """Lemma 2: E[Z] = U, term by term, so the enumerated mean equals sum_k zeta_k A'^k."""
    g = ba12
    gam = 1 / R.lambda_max(g)
    c = np.random.default_rng(K).uniform(0.1, 1.0, K + 1)
    v = np.random.default_rng(K + 1).standard_normal(g.n)
    F = R.dense_powers_series(gam * g.dense(), c)
    ex = R.enumerate_action(g, c, gamma=gam, v=v)
    assert np.allclose(ex["mean_y"], F @ v, rtol=1e-13, atol=1e-13)
    ed = R.enumerate_diag(g, c, gamma=gam)
    assert np.allclose(ed["mean_d"], np.diag(F), rtol=1e-13, atol=1e-13)


def test_enumeration_signed_weights_reproduces_series():
    g = I.barabasi_albert(9, 2, 1)
    w = I.symmetric_weights(g, seed=3, signed=True)
    A = R.csr_matrix(g, w).toarray()
    gam = 1 / np.abs(np.linalg.eigvalsh(A)).max()
    c = R.exp_coeffs(6)
    F = R.dense_powers_series(gam * A, c)
    ex = R.enumerate_action(g, c, gamma=gam, values=w)
    assert np.allclose(ex["mean_y"], F.sum(1), rtol=1e-13, atol=1e-13)
    ed = R.enumerate_diag(g, c, gamma=gam, values=w)
    assert np.allclose(ed["mean_d"], np.diag(F), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("precision", [0, 1])
def test_action_is_unbiased_within_sigma(ba12, precision):
    g = ba12
    gam = 1 / R.lambda_max(g)
    c = R.exp_coeffs(7)
    v = np.random.default_rng(2).uniform(0.5, 1.5, g.n)
    ex = R.enumerate_action(g, c, gamma=gam, v=v)
    wpn = 20000
    nw = np.full(g.n, wpn)
    var = R.action_variance(ex, nw)
    y = E.action(g, c, v=v, gamma=gam, walks_per_node=wpn, seed=11, precision=precision)["y"]
    assert _zscore(y, ex["mean_y"], var + (1e-6 * ex["mean_y"]) ** 2 * precision) < Z_MAX


def test_action_with_allocation_is_unbiased(ba12):
    g = ba12
    gam = 1 / R.lambda_max(g)
    c = R.exp_coeffs(7)
    ex = R.enumerate_action(g, c, gamma=gam)
    _, _, nw, _ = E.allocation(g, gamma=gam, n_walks=150000)
    y = E.action(g, c, gamma=gam, n_walks=150000, seed=12)["y"]
    assert _zscore(y, ex["mean_y"], R.action_variance(ex, nw)) < Z_MAX


def test_diag_is_unbiased_within_sigma(ba12):
    g = ba12
    gam = 1 / R.lambda_max(g)
    c = R.exp_coeffs(7)
    wpn = 20000
    ed = R.enumerate_diag(g, c, gamma=gam, nw=np.full(g.n, wpn))
    d = E.diag(g, c, gamma=gam, walks_per_node=wpn, seed=13)["d"]
    assert _zscore(d, ed["mean_d"], ed["var_d"]) < Z_MAX


def test_signed_weighted_estimators_unbiased():
    g = I.barabasi_albert(9, 2, 1)
    w = I.symmetric_weights(g, seed=3, signed=True)
    A = R.csr_matrix(g, w).toarray()
    gam = 1 / np.abs(np.linalg.eigvalsh(A)).max()
    c = R.exp_coeffs(6)
    wpn = 30000
    ex = R.enumerate_action(g, c, gamma=gam, values=w)
    y = E.action(g, c, gamma=gam, walks_per_node=wpn, seed=14, values=w)["y"]
    assert _zscore(y, ex["mean_y"], R.action_variance(ex, np.full(g.n, wpn))) < Z_MAX
    ed = R.enumerate_diag(g, c, gamma=gam, values=w, nw=np.full(g.n, wpn))
    d = E.diag(g, c, gamma=gam, walks_per_node=wpn, seed=14, values=w)["d"]
    assert _zscore(d, ed["mean_d"], ed["var_d"]) < Z_MAX


def test_weight_cutoff_bias_matches_enumeration(ba12):
    """Eq. weight_cutoff: a walk stops once |W^(m)| <= W_c W^(0).  The enumeration
    with the same cutoff gives the (biased) expectation; the estimator must hit it,
    and it must differ from the unbiased one by many sigma (so the test has power)."""
    g = ba12
    gam = 1 / R.lambda_max(g)
    c = R.exp_coeffs(7)
    wc = 0.7
    wpn = 20000
    ex_c = R.enumerate_action(g, c, gamma=gam, w_cutoff=wc)
    ex_0 = R.enumerate_action(g, c, gamma=gam)
    var = R.action_variance(ex_c, np.full(g.n, wpn))
    y = E.action(g, c, gamma=gam, walks_per_node=wpn, w_cutoff=wc, seed=15)["y"]
    assert _zscore(y, ex_c["mean_y"], var) < Z_MAX
    assert np.abs(ex_c["mean_y"] - ex_0["mean_y"]).max() > 50 * np.sqrt(var.max())


# ------------------------------------------------------------ closed forms and invariants
def test_complete_graph_diag_within_sigma():
    n = 6
    g = I.complete(n)
    gam = 1 / (n - 1)
    c = R.exp_coeffs(8)
    f = lambda x: sum(ck * x ** k for k, ck in enumerate(c))
    exact = (f(gam * (n - 1)) + (n - 1) * f(-gam)) / n
    wpn = 20000
    ed = R.enumerate_diag(g, c, gamma=gam, nw=np.full(n, wpn))
    assert np.allclose(ed["mean_d"], exact, rtol=1e-13)
    d = E.diag(g, c, gamma=gam, walks_per_node=wpn, seed=3)["d"]
    assert _zscore(d, ed["mean_d"], ed["var_d"]) < Z_MAX


def test_trace_invariant_estrada_index():
    """sum_i d_i estimates trace f(A') = sum_j f(lambda_j) (the Estrada index)."""
    g = I.barabasi_albert(10, 2, 7)
    gam = 1 / R.lambda_max(g)
    c = R.exp_coeffs(7)
    lam = np.linalg.eigvalsh(gam * g.dense())
    trace = np.polynomial.polynomial.polyval(lam, c).sum()
    wpn = 20000
    ed = R.enumerate_diag(g, c, gamma=gam, nw=np.full(g.n, wpn))
    assert ed["mean_d"].sum() == pytest.approx(trace, rel=1e-13)
    d = E.diag(g, c, gamma=gam, walks_per_node=wpn, seed=21)["d"]
    # the d_i share walks, so bound the sum's error by the sum of the standard deviations
    assert abs(d.sum() - trace) < Z_MAX * np.sqrt(ed["var_d"]).sum()


def test_error_decays_like_inverse_sqrt_walks():
    """Theorem 1 / Section 4.1: relative l_inf error ~ N_s^-1/2 (slope -0.5)."""
    g = I.barabasi_albert(40, 2, 8)
    gam = 1 / R.lambda_max(g)
    c = R.exp_coeffs(20)
    exact = R.dense_funm(gam * g.dense(), c).sum(1)
    ns = [40, 400, 4000, 40000]
    errs = []
    for N in ns:
        e = [np.abs(E.action(g, c, gamma=gam, walks_per_node=N, seed=s)["y"] - exact).max() for s in range(6)]
        errs.append(np.mean(e) / np.abs(exact).max())
    slope = np.polyfit(np.log(ns), np.log(errs), 1)[0]
    assert -0.6 < slope < -0.4, (slope, errs)


# ------------------------------------------------------------ structural equalities
def test_diag_equals_diagonal_of_randfunm_same_walks(ba12):
    """RandFunmDiag computes the diagonal of Algorithm 2's F = zeta_0 I + zeta_1 A' + A'QA'
    from the same walks (Section 4.2: same core algorithm)."""
    g = ba12
    gam = 1 / R.lambda_max(g)
    c = R.exp_coeffs(9)
    F = E.funm_full(g, c, gamma=gam, walks_per_node=50, seed=5)
    d = E.diag(g, c, gamma=gam, walks_per_node=50, seed=5)["d"]
    assert np.allclose(d, np.diag(F), rtol=1e-12, atol=1e-14)
    y = E.action(g, c, gamma=gam, walks_per_node=50, seed=5)["y"]
    assert np.allclose(y, F.sum(1), rtol=1e-12, atol=1e-14)


def test_subset_equals_full_run_entries():
    g = I.barabasi_albert(300, 3, 9)
    gam = 1 / R.lambda_max(g)
    c = R.exp_coeffs(15)
    nodes = np.array([0, 5, 17, 123, 299, 5])
    full = E.action(g, c, gamma=gam, n_walks=20000, seed=6)["y"]
    sub = E.action(g, c, gamma=gam, n_walks=20000, seed=6, nodes=nodes)["y"]
    assert np.array_equal(sub, full[nodes])
    fd = E.diag(g, c, gamma=gam, walks_per_node=20, seed=6)["d"]
    sd = E.diag(g, c, gamma=gam, walks_per_node=20, seed=6, nodes=nodes)["d"]
    assert np.array_equal(sd, fd[nodes])


def test_float32_weights_track_float64(ba12):
    g = ba12
    gam = 1 / R.lambda_max(g)
    c = R.exp_coeffs(12)
    y0 = E.action(g, c, gamma=gam, walks_per_node=500, seed=7, precision=0)["y"]
    y1 = E.action(g, c, gamma=gam, walks_per_node=500, seed=7, precision=1)["y"]
    assert np.abs(y1 - y0).max() < 1e-6 * np.abs(y0).max()
    assert not np.array_equal(y0, y1)


def test_isolated_nodes_and_empty_graph():
    g = I.add_isolated(I.path(4), 3)
    c = R.exp_coeffs(6)
    y = E.action(g, c, gamma=0.5, walks_per_node=5, seed=1)["y"]
    assert np.all(y[4:] == 1.0)
    d = E.diag(g, c, gamma=0.5, walks_per_node=5, seed=1)["d"]
    assert np.all(d[4:] == 1.0)
    e = I.add_isolated(I.from_edges(1, np.zeros((0, 2))), 4)
    assert np.all(E.action(e, c, gamma=1.0, n_walks=100)["y"] == 1.0)


def test_classical_mc_is_unbiased_within_sigma():
    """Algorithm 1 with W_c = 0 is unbiased for the truncated series
    sum_k zeta_k (A'^k v)_i: the mean of 40 independent runs (seeds) lies within
    a few standard errors (estimated from the runs) of the exact value on a
    graph with unequal degrees and a general v."""
    g = I.barabasi_albert(30, 2, 9)
    gam = 1.0 / R.lambda_max(g)
    c = R.exp_coeffs(8)
    v = np.random.default_rng(2).standard_normal(g.n)
    exact = R.dense_powers_series(gam * g.dense(), c) @ v
    runs = 40
    ys = np.array([E.mc_classic_action(g, c, np.arange(g.n), 500, v=v, gamma=gam, seed=s) for s in range(runs)])
    z = (ys.mean(0) - exact) / (ys.std(0, ddof=1) / np.sqrt(runs))
    assert np.abs(z).max() < 4.5


def test_randfunm_action_beats_classical_mc_single_entry():
    """Section 4.3 / Table 3: for the highest-degree node, sampling whole rows gives a
    smaller error than Algorithm 1 with the same number of walks (Table 3 uses a small
    gamma; here gamma = 0.5 / lambda_max, mean absolute error over 24 seeds)."""
    g = I.barabasi_albert(200, 3, 10)
    gam = 0.5 / R.lambda_max(g)
    c = R.exp_coeffs(20)
    exact = R.dense_funm(gam * g.dense(), c).sum(1)
    i = int(np.argmax(g.degree))
    nbrs = g.col_idx[g.row_ptr[i]:g.row_ptr[i + 1]]
    per = 4000 // len(nbrs)
    err_rf, err_mc = [], []
    for s in range(24):
        # RandFunmAction spends its walks on the neighbours of i (N_s split evenly)
        y = E.action(g, c, gamma=gam, walks_per_node=per, seed=s, nodes=[i])["y"][0]
        err_rf.append(abs(y - exact[i]))
        ymc = E.mc_classic_action(g, c, [i], walks_per_row=per * len(nbrs), gamma=gam, seed=s)[0]
        err_mc.append(abs(ymc - exact[i]))
    assert np.mean(err_rf) < 0.5 * np.mean(err_mc)


# ------------------------------------------------------------ standard error (Section 3.5)
@pytest.mark.parametrize("precision", [0, 1])
def test_standard_error_matches_enumerated_variance(ba12, precision):
    """Var(y_j) = sum_i a'_ji^2 Var(X_i) / N_i for independent walks; the
    sample-variance estimate from 2e4 walks per node must match the exact
    variance from the enumeration to a few percent (its own sampling error
    is about sqrt(2 / N) = 1 %)."""
    g = ba12
    gam = 1 / R.lambda_max(g)
    c = R.exp_coeffs(7)
    v = np.random.default_rng(5).uniform(0.5, 1.5, g.n)
    wpn = 20000
    ex = R.enumerate_action(g, c, gamma=gam, v=v)
    var = R.action_variance(ex, np.full(g.n, wpn))
    se = E.action_se(g, c, v=v, gamma=gam, walks_per_node=wpn, seed=3, precision=precision)
    assert np.max(np.abs(se ** 2 / var - 1)) < 0.04
    sub = E.action_se(g, c, v=v, gamma=gam, walks_per_node=wpn, seed=3, precision=precision, nodes=[3, 0, 3])
    assert np.array_equal(sub, se[[3, 0, 3]])


def test_standard_error_vanishes_without_variance():
    """On K_n every walk of total communicability has the same sum: the
    estimate is exact and its standard error is zero up to the rounding of
    the sum-of-squares formula."""
    g = I.complete(7)
    c = R.exp_coeffs(10)
    y = E.action(g, c, gamma=0.2, walks_per_node=50, seed=1)["y"]
    se = E.action_se(g, c, gamma=0.2, walks_per_node=50, seed=1)
    assert np.all(se <= 1e-7 * y)


def test_enumerated_variances_match_repeated_runs():
    """The enumerated variances that every sigma-bound above divides by, checked
    against the spread of the C estimator itself: 3000 independent runs
    (seeds) with the N_s allocation of Definition 1, so N_i differs between
    nodes (Var(y_j) = sum_i a'_ji^2 Var(X_i) / N_i, and for the diagonal
    sum_k a'_ik^2 Var(Y_k,i) / N_k).  The sample variance of a near-Gaussian
    mean over 3000 runs is within a few percent of the true one."""
    g = I.barabasi_albert(10, 2, 5)
    w = I.symmetric_weights(g, seed=4, signed=True, low=0.1, high=5.0)
    gam = 0.8 / np.abs(np.linalg.eigvalsh(R.csr_matrix(g, w).toarray())).max()
    c = R.exp_coeffs(6)
    ns = 150 * g.n
    _, _, nw, _ = E.allocation(g, gamma=gam, n_walks=ns, values=w)
    assert nw.max() > 2 * nw.min()
    ex = R.enumerate_action(g, c, gamma=gam, values=w)
    var_y = R.action_variance(ex, nw)
    ed = R.enumerate_diag(g, c, gamma=gam, values=w, nw=nw)
    runs = 3000
    ys = np.array([E.action(g, c, gamma=gam, n_walks=ns, seed=s, values=w)["y"] for s in range(runs)])
    ds = np.array([E.diag(g, c, gamma=gam, n_walks=ns, seed=s, values=w)["d"] for s in range(runs)])
    assert np.all(var_y > 0) and np.all(ed["var_d"] > 0)
    assert np.all(np.abs(ys.var(0, ddof=1) / var_y - 1.0) < 0.12)
    assert np.all(np.abs(ds.var(0, ddof=1) / ed["var_d"] - 1.0) < 0.12)
    assert _zscore(ys.mean(0), ex["mean_y"], var_y / runs) < Z_MAX
    assert _zscore(ds.mean(0), ed["mean_d"], ed["var_d"] / runs) < Z_MAX


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
def test_enumerated_second_moments_closed_form(k):
    """With one non-zero coefficient zeta_(k+2) = 1 a walk's sum is X = W^(k) r_(l_k)
    (the graph has no sinks), so E[X] = (A'^k r)_i and, because every step
    multiplies E[W^2 g] by t_lj (a'_lj / t_lj)^2 = rowabs_l |a'_lj|,
    E[X^2] = (M^k (r o r))_i with M = diag(rowabs) |A'| (Eq. weights, Definition 1).
    For the diagonal, Y_(k,i) = W^(k) a'_(l_k, i): E[Y] = (A'^(k+1))_(ki) and
    E[Y^2] = (M^k (A' o A'))_(ki)."""
    g = I.barabasi_albert(12, 2, 3)
    w = I.symmetric_weights(g, seed=5, signed=True)
    A = R.csr_matrix(g, w).toarray()
    gam = 0.7 / np.abs(np.linalg.eigvalsh(A)).max()
    Ap = gam * A
    M = np.abs(Ap).sum(1)[:, None] * np.abs(Ap)
    Mk = np.linalg.matrix_power(M, k)
    v = np.random.default_rng(1).standard_normal(g.n)
    r = Ap @ v
    c = np.zeros(k + 3)
    c[k + 2] = 1.0
    ex = R.enumerate_action(g, c, gamma=gam, v=v, values=w)
    m1 = np.linalg.matrix_power(Ap, k) @ r
    m2 = Mk @ (r * r)
    assert np.allclose(ex["Eq"], m1, rtol=1e-12, atol=1e-15)
    assert np.allclose(ex["var_walk"], m2 - m1 ** 2, rtol=1e-10, atol=1e-14 * m2.max())
    ed = R.enumerate_diag(g, c, gamma=gam, values=w, nw=np.ones(g.n, np.int64))
    EY = np.linalg.matrix_power(Ap, k + 1)
    EY2 = Mk @ (Ap * Ap)
    assert np.allclose(ed["mean_d"], (Ap * EY).sum(0), rtol=1e-12, atol=1e-15)   # zeta_0 = zeta_1 = 0
    var_d = ((Ap * Ap) * (EY2 - EY ** 2)).sum(0)
    assert np.allclose(ed["var_d"], var_d, rtol=1e-10, atol=1e-14 * max(EY2.max(), 1e-300))


def test_enumeration_with_loops_reproduces_series():
    """Lemma 2 on a signed symmetric A with loops: a walk may stay on its node,
    and the diagonal adds zeta_1 a'_ii."""
    n = 7
    und = np.array([(0, 1), (1, 2), (2, 3), (3, 4), (4, 0), (1, 5), (5, 6), (2, 6)])
    loops = np.array([0, 2, 5])
    g = I.directed_from_edges(n, np.concatenate([und[:, 0], und[:, 1], loops]),
                              np.concatenate([und[:, 1], und[:, 0], loops]))
    rows = np.repeat(np.arange(n), np.diff(g.row_ptr))
    cols = g.col_idx.astype(np.int64)
    rng = np.random.default_rng(6)
    table = rng.uniform(0.5, 1.5, (n, n)) * rng.choice([-1.0, 1.0], (n, n))
    w = table[np.minimum(rows, cols), np.maximum(rows, cols)].astype(np.float32)
    A = R.csr_matrix(g, w).toarray()
    assert np.array_equal(A, A.T) and np.count_nonzero(np.diag(A)) == 3
    gam = 0.9 / np.abs(np.linalg.eigvalsh(A)).max()
    c = np.random.default_rng(7).uniform(0.1, 1.0, 6)
    F = R.dense_powers_series(gam * A, c)
    v = rng.standard_normal(n)
    assert np.allclose(R.enumerate_action(g, c, gamma=gam, v=v, values=w)["mean_y"], F @ v, rtol=1e-13, atol=1e-13)
    assert np.allclose(R.enumerate_diag(g, c, gamma=gam, values=w)["mean_d"], np.diag(F), rtol=1e-13, atol=1e-13)


# ------------------------------------------------------------ SelectNextState frequencies
@pytest.mark.parametrize("weighted", [False, True])
def test_sampler_frequencies_chi_square(weighted):
    """Pearson's chi-square of the picked positions of one row over 2e5 walk
    steps against t_lj = |a_lj| / sum_k |a_lk| (Definition 1): the statistic
    stays below the 0.999 quantile for its degrees of freedom (fixed seeds,
    so the outcome is deterministic)."""
    from scipy import stats

    g = I.star(41)                          # row 0 has 40 entries
    w = None
    p = np.full(40, 1 / 40)
    if weighted:
        w = I.symmetric_weights(g, seed=6, signed=True, low=0.1, high=3.0)
        a = np.abs(w[g.row_ptr[0]:g.row_ptr[1]]).astype(np.float64)
        p = a / a.sum()
    n = 200_000
    for seed in (1, 2):
        counts = E.sample_counts(g, 0, n, seed=seed, values=w)
        assert counts.sum() == n
        chi2 = float(np.sum((counts - n * p) ** 2 / (n * p)))
        assert chi2 < stats.chi2.ppf(0.999, df=39), chi2
    # a plausible mistake: sampling uniformly on the weighted row fails the test
    if weighted:
        counts = E.sample_counts(g, 0, n, seed=1)
        assert float(np.sum((counts - n * p) ** 2 / (n * p))) > stats.chi2.ppf(0.999, df=39)
