"""Pins of the oracle on a general (non-symmetric) A, on other coefficient
families, and of the bipartite symmetrisation of directed graphs.

Definition 1 draws the start column from the column norms ||C_i|| and walks
along rows; Eq. rand_funm_formula_diag pairs column k (the rows i with
a_ik != 0) with column i; Algorithm 2 multiplies A'Q by A' from the right.
For a symmetric A rows and columns coincide, so these pins are the ones that
catch a row/column (transposed operand) mistake."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import estimator as E
from oracle import reference as R
from paper_2308_01037_gb300 import inputs as I

Z_MAX = 5.0


def _zscore(est, mean, var):
    sd = np.sqrt(var)
    ok = sd > 0
    assert np.all(np.abs(est[~ok] - mean[~ok]) <= 1e-12 * np.maximum(1, np.abs(mean[~ok])))
    return np.abs((est[ok] - mean[ok]) / sd[ok]).max() if ok.any() else 0.0


@pytest.fixture(scope="module")
def dg():
    """A small directed graph with sources, sinks and unequal in/out degrees."""
    g = I.directed_erdos_renyi(9, 2.2, 5)
    assert not np.array_equal(g.dense(), g.dense().T)
    return g


def _signed(g, seed):
    rng = np.random.default_rng(seed)
    return (rng.uniform(0.25, 2.0, g.nnz) * rng.choice([-1.0, 1.0], g.nnz)).astype(np.float32)


def _gamma(A):
    return 0.9 / max(np.abs(np.linalg.eigvals(A)).max(), 1e-12)


# ------------------------------------------------------------ allocation from columns
def test_allocation_uses_column_norms():
    """Arcs 0->1, 0->2, 1->2: out-degrees (2, 1, 0), in-degrees (0, 1, 2).
    rowabs = gamma * out-degree, ||C_i|| = gamma * sqrt(in-degree)."""
    g = I.directed_from_edges(3, [0, 0, 1], [1, 2, 2])
    ra, cn, nw, _ = E.allocation(g, gamma=0.5, walks_per_node=3)
    assert ra.tolist() == [1.0, 0.5, 0.0]
    assert cn.tolist() == pytest.approx([0.0, 0.5, 0.5 * math.sqrt(2.0)], rel=1e-15)
    assert nw.tolist() == [0, 3, 3]          # column 0 is empty: no walks start there
    w = np.array([2.0, -1.0, 3.0], np.float32)   # a01 = 2, a02 = -1, a12 = 3
    ra, cn, _, _ = E.allocation(g, gamma=1.0, walks_per_node=1, values=w)
    assert ra.tolist() == [3.0, 3.0, 0.0]
    assert cn.tolist() == pytest.approx([0.0, 2.0, math.sqrt(10.0)], rel=1e-15)


# ------------------------------------------------------------ Lemma 2 on a general A
@pytest.mark.parametrize("weighted", [False, True])
def test_enumeration_reproduces_series_nonsymmetric(dg, weighted):
    w = _signed(dg, 1) if weighted else None
    A = R.csr_matrix(dg, w).toarray()
    gam = _gamma(A)
    c = R.exp_coeffs(6)
    v = np.random.default_rng(3).standard_normal(dg.n)
    F = R.dense_powers_series(gam * A, c)
    ex = R.enumerate_action(dg, c, gamma=gam, v=v, values=w)
    assert np.allclose(ex["mean_y"], F @ v, rtol=1e-13, atol=1e-13)
    ed = R.enumerate_diag(dg, c, gamma=gam, values=w)
    assert np.allclose(ed["mean_d"], np.diag(F), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("precision", [0, 1])
def test_estimators_unbiased_nonsymmetric(dg, precision):
    w = _signed(dg, 2)
    A = R.csr_matrix(dg, w).toarray()
    gam = _gamma(A)
    c = R.exp_coeffs(6)
    v = np.random.default_rng(4).uniform(0.5, 1.5, dg.n)
    wpn = 30000
    nw = np.where(np.abs(A).sum(0) > 0, wpn, 0)
    ex = R.enumerate_action(dg, c, gamma=gam, v=v, values=w)
    y = E.action(dg, c, v=v, gamma=gam, walks_per_node=wpn, seed=21, precision=precision, values=w)["y"]
    var = R.action_variance(ex, nw) + (1e-6 * ex["mean_y"]) ** 2 * precision
    assert _zscore(y, ex["mean_y"], var) < Z_MAX
    ed = R.enumerate_diag(dg, c, gamma=gam, values=w, nw=nw)
    d = E.diag(dg, c, gamma=gam, walks_per_node=wpn, seed=22, precision=precision, values=w)["d"]
    assert _zscore(d, ed["mean_d"], ed["var_d"] + (1e-6 * ed["mean_d"]) ** 2 * precision) < Z_MAX


def test_full_estimate_nonsymmetric_matches_diag_and_is_unbiased(dg):
    A = R.csr_matrix(dg).toarray()
    gam = _gamma(A)
    c = R.exp_coeffs(6)
    F = E.funm_full(dg, c, gamma=gam, walks_per_node=20000, seed=23)
    d = E.diag(dg, c, gamma=gam, walks_per_node=20000, seed=23)["d"]
    assert np.allclose(np.diag(F), d, rtol=1e-12, atol=1e-14)
    ex = R.dense_powers_series(gam * A, c)
    assert np.abs(F - ex).max() < 0.02 * np.abs(ex).max()
    # a transposed right factor (A'Q A'^T) would be far off for this A
    assert np.abs(F - ex.T).max() > 5 * np.abs(F - ex).max()


# ------------------------------------------------------------ the directed cycle: exact
@pytest.mark.parametrize("n", [3, 5])
def test_directed_cycle_is_exact(n):
    """A = P (i -> i+1): every row has one entry, every weight ratio is 1, so
    one walk per node is exact.  f(P) = sum_k zeta_k P^k; its row sums are
    sum_k zeta_k and its diagonal collects the zeta_k with n | k."""
    g = I.directed_cycle(n)
    c = np.random.default_rng(n).uniform(0.1, 1.0, 12)
    P = g.dense()
    F_ex = R.dense_powers_series(P, c)
    y = E.action(g, c, walks_per_node=1, seed=1)["y"]
    assert np.allclose(y, c.sum(), rtol=1e-14)
    d = E.diag(g, c, walks_per_node=1, seed=1)["d"]
    assert np.allclose(d, sum(c[k] for k in range(0, len(c), n)), rtol=1e-14)
    F = E.funm_full(g, c, walks_per_node=1, seed=1)
    assert np.allclose(F, F_ex, rtol=1e-14, atol=1e-15)
    yc = E.mc_classic_action(g, c, np.arange(n), 1, seed=1)
    assert np.allclose(yc, c.sum(), rtol=1e-14)
    # a general v: (P^k v)_i = v_{(i + k) mod n}, so y_i = sum_k zeta_k v_{(i+k) mod n}
    v = np.random.default_rng(n + 1).standard_normal(n)
    y_ex = np.array([sum(c[k] * v[(i + k) % n] for k in range(len(c))) for i in range(n)])
    assert np.allclose(F_ex @ v, y_ex, rtol=1e-14)
    assert np.allclose(E.action(g, c, v=v, walks_per_node=1, seed=1)["y"], y_ex, rtol=1e-13, atol=1e-14)
    assert np.allclose(E.mc_classic_action(g, c, np.arange(n), 1, v=v, seed=1), y_ex, rtol=1e-13, atol=1e-14)


def test_signed_weighted_directed_cycle_is_exact():
    """Arc i -> i+1 carries a signed weight s_i: a row has one entry, so its
    row sum |s_i| and sign fix the weight ratio of Eq. weights and every walk
    is deterministic, (A'^k v)_i = gamma^k s_i s_(i+1) ... s_(i+k-1) v_(i+k).
    One walk per node is exact for all four estimators; a dropped sign fails."""
    n = 5
    g = I.directed_cycle(n)
    s = np.array([0.8, -1.25, 1.5, -0.6, 1.1], np.float32)   # row i's single value
    gam = 0.7
    A = gam * R.csr_matrix(g, s).toarray()
    c = np.random.default_rng(2).uniform(0.1, 1.0, 11)
    F_ex = R.dense_powers_series(A, c)
    v = np.random.default_rng(3).standard_normal(n)
    kw = dict(gamma=gam, walks_per_node=1, seed=4, values=s)
    assert np.allclose(E.action(g, c, v=v, **kw)["y"], F_ex @ v, rtol=1e-13, atol=1e-14)
    assert np.allclose(E.diag(g, c, **kw)["d"], np.diag(F_ex), rtol=1e-13, atol=1e-14)
    assert np.allclose(E.funm_full(g, c, **kw), F_ex, rtol=1e-13, atol=1e-14)
    yc = E.mc_classic_action(g, c, np.arange(n), 1, v=v, gamma=gam, seed=4, values=s)
    assert np.allclose(yc, F_ex @ v, rtol=1e-13, atol=1e-14)


def test_nilpotent_dag_is_polynomial():
    """A strictly upper triangular A (arcs i -> j, i < j) has A^n = 0: the series
    ends after n terms whatever the coefficients, and walks end at the sink."""
    n = 6
    src, dst = np.triu_indices(n, 1)
    g = I.directed_from_edges(n, src, dst)
    A = g.dense()
    gam = 0.5
    c = R.exp_coeffs(12)
    F = R.dense_powers_series(gam * A, c)
    assert np.allclose(F, sla.expm(gam * A), rtol=1e-14, atol=1e-15)
    ex = R.enumerate_action(g, c, gamma=gam)
    assert np.allclose(ex["mean_y"], F.sum(1), rtol=1e-13)
    y = E.action(g, c, gamma=gam, walks_per_node=20000, seed=5)["y"]
    assert _zscore(y, ex["mean_y"], R.action_variance(ex, np.full(n, 20000))) < Z_MAX


# ------------------------------------------------------------ other coefficient families
def test_mittag_leffler_coefficients_closed_forms():
    x = 0.7
    ev = lambda c: sum(ck * x ** k for k, ck in enumerate(c))   # noqa: E731
    assert np.allclose(R.mittag_leffler_coeffs(20, 1.0, 1.0), R.exp_coeffs(20), rtol=1e-14)
    assert ev(R.mittag_leffler_coeffs(30, 1.0, 2.0)) == pytest.approx((math.exp(x) - 1) / x, rel=1e-14)
    assert ev(R.mittag_leffler_coeffs(30, 2.0, 1.0)) == pytest.approx(math.cosh(math.sqrt(x)), rel=1e-14)
    assert ev(R.mittag_leffler_coeffs(60, 0.5, 1.0)) == pytest.approx(
        math.exp(x * x) * math.erfc(-x), rel=1e-12)


def test_mittag_leffler_estimator_unbiased():
    g = I.barabasi_albert(12, 2, 3)
    gam = 1 / R.lambda_max(g)
    c = R.mittag_leffler_coeffs(7, 0.8, 1.2)
    F = R.dense_powers_series(gam * g.dense(), c)
    ex = R.enumerate_action(g, c, gamma=gam)
    assert np.allclose(ex["mean_y"], F.sum(1), rtol=1e-13)
    y = E.action(g, c, gamma=gam, walks_per_node=20000, seed=31)["y"]
    assert _zscore(y, ex["mean_y"], R.action_variance(ex, np.full(g.n, 20000))) < Z_MAX


# ------------------------------------------------------------ digraph symmetrisation
def test_bipartite_symmetrization_block_exponential(dg):
    """B = [0 A; A^T 0] (Eq. digraph_sym); with A = U S V^T,
    exp(B) = [U cosh(S) U^T, U sinh(S) V^T; V sinh(S) U^T, V cosh(S) V^T]."""
    b = I.bipartite_symmetrization(dg)
    B = b.dense()
    A = dg.dense()
    n = dg.n
    assert np.array_equal(B[:n, n:], A) and np.array_equal(B[n:, :n], A.T) and not B[:n, :n].any()
    U, S, Vt = np.linalg.svd(A)
    V = Vt.T
    blk = np.block([[U @ np.diag(np.cosh(S)) @ U.T, U @ np.diag(np.sinh(S)) @ Vt],
                    [V @ np.diag(np.sinh(S)) @ U.T, V @ np.diag(np.cosh(S)) @ Vt]])
    assert np.allclose(sla.expm(B), blk, rtol=1e-12, atol=1e-12)
    bw, w = I.bipartite_symmetrization(dg, values=_signed(dg, 3))
    Bw = R.csr_matrix(bw, w).toarray()
    Aw = R.csr_matrix(dg, _signed(dg, 3)).toarray()
    assert np.array_equal(Bw[:n, n:], Aw) and np.array_equal(Bw, Bw.T)
