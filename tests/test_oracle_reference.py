"""Pins of the float64 reference (oracle part 2) against closed forms and
library routines: spectra of K_n, P_n and the star, scipy's expm and solve,
and the equality of the spectral, explicit-power and sparse-series forms."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import reference as R
from paper_2308_01037_gb300 import inputs as I


def test_lambda_max_closed_forms():
    assert R.lambda_max(I.complete(7)) == pytest.approx(6.0, rel=1e-13)
    assert R.lambda_max(I.path(9)) == pytest.approx(2 * math.cos(math.pi / 10), rel=1e-13)
    assert R.lambda_max(I.star(10)) == pytest.approx(3.0, rel=1e-13)
    assert R.lambda_max(I.cycle(8)) == pytest.approx(2.0, rel=1e-13)


def test_lambda_max_arpack_matches_dense():
    g = I.barabasi_albert(2500, 3, 4)
    dense = float(np.linalg.eigvalsh(g.dense())[-1])
    assert R.lambda_max(g) == pytest.approx(dense, rel=1e-11)


def test_gershgorin_is_max_degree():
    g = I.barabasi_albert(300, 3, 0)
    assert R.gershgorin(g) == g.degree.max()


def test_gershgorin_signed_weights_by_hand():
    """P_3 with a01 = 2, a12 = -3: absolute row sums 2, 5, 3 (a signed sum would give -1 for row 1)."""
    g = I.path(3)
    w = np.array([2.0, 2.0, -3.0, -3.0], np.float32)
    assert R.gershgorin(g, w) == 5.0
    assert R.gershgorin(g, -w) == 5.0


@pytest.mark.parametrize("n", [3, 6, 11])
def test_complete_graph_closed_form(n):
    """K_n = J - I has eigenvalues n-1 (eigenvector 1) and -1 (multiplicity n-1)."""
    gam = 0.7 / (n - 1)
    c = R.exp_coeffs(30)
    f = lambda x: sum(ck * x ** k for k, ck in enumerate(c))
    F = R.dense_funm(gam * I.complete(n).dense(), c)
    assert np.allclose(F.sum(1), f(gam * (n - 1)), rtol=1e-13, atol=0)
    assert np.allclose(np.diag(F), (f(gam * (n - 1)) + (n - 1) * f(-gam)) / n, rtol=1e-13, atol=0)


def test_path_graph_closed_form():
    """P_n: lambda_j = 2 cos(pi j/(n+1)), v_j(i) = sqrt(2/(n+1)) sin(pi i j/(n+1))."""
    n = 9
    c = R.exp_coeffs(30, beta=0.4)
    F = R.dense_funm(I.path(n).dense(), c)
    j = np.arange(1, n + 1)
    lam = 2 * np.cos(np.pi * j / (n + 1))
    f = np.polynomial.polynomial.polyval(lam, c)
    for i in range(1, n + 1):
        v = np.sqrt(2 / (n + 1)) * np.sin(np.pi * i * j / (n + 1))
        assert F[i - 1, i - 1] == pytest.approx(np.sum(f * v * v), rel=1e-13)


def test_star_closed_form():
    """Star S_n: eigenvalues +-sqrt(n-1) and 0; the centre's diagonal entry is (f(s)+f(-s))/2."""
    n = 8
    c = R.exp_coeffs(30, beta=0.3)
    F = R.dense_funm(I.star(n).dense(), c)
    s = math.sqrt(n - 1)
    f = lambda x: sum(ck * x ** k for k, ck in enumerate(c))
    assert F[0, 0] == pytest.approx((f(s) + f(-s)) / 2, rel=1e-13)


def test_truncated_exp_matches_scipy_expm():
    g = I.barabasi_albert(200, 3, 1)
    A = g.dense() / R.lambda_max(g)
    F = R.dense_funm(A, R.exp_coeffs(30))
    assert np.abs(F - sla.expm(A)).max() < 1e-13 * np.abs(F).max()


def test_spectral_and_explicit_powers_agree():
    g = I.barabasi_albert(60, 2, 5)
    A = g.dense() / R.lambda_max(g)
    c = np.random.default_rng(0).uniform(0, 1, 9)
    assert np.abs(R.dense_funm(A, c) - R.dense_powers_series(A, c)).max() < 1e-13


def test_series_action_and_diag_match_dense():
    g = I.barabasi_albert(300, 3, 2)
    gam = 1 / R.lambda_max(g)
    c = R.exp_coeffs(30)
    F = R.dense_funm(gam * g.dense(), c)
    v = np.random.default_rng(1).standard_normal(g.n)
    assert np.allclose(R.series_action(g, c, gam, v), F @ v, rtol=0, atol=1e-12 * np.abs(F @ v).max())
    nodes = np.arange(0, g.n, 7)
    assert np.allclose(R.series_diag(g, c, nodes, gam), np.diag(F)[nodes], rtol=1e-12, atol=0)


def test_katz_series_matches_solve():
    g = I.barabasi_albert(300, 3, 3)
    gam = 0.85 / R.lambda_max(g)
    K = R.katz_terms_for_tail(0.85, 1e-14)
    y = R.series_action(g, R.katz_coeffs(K), gam)
    x = np.linalg.solve(np.eye(g.n) - gam * g.dense(), np.ones(g.n))
    assert np.abs(y - x).max() < 1e-12 * np.abs(x).max()
    assert 0.85 ** (K + 1) / 0.15 <= 1e-14 < 0.85 ** K / 0.15


def test_weighted_series_matches_dense():
    g = I.barabasi_albert(80, 3, 6)
    w = I.symmetric_weights(g, seed=2, signed=True)
    A = R.csr_matrix(g, w).toarray()
    assert np.allclose(A, A.T)
    gam = 1 / np.abs(np.linalg.eigvalsh(A)).max()
    c = R.exp_coeffs(30)
    F = R.dense_funm(gam * A, c)
    assert np.allclose(R.series_action(g, c, gam, values=w), F.sum(1), rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- second-moment growth rho(diag(s') |A'|)
def test_second_moment_radius_closed_forms():
    """rho(diag(s')|A'|) in closed form: K_n (s' = gamma (n-1) everywhere, so
    M = gamma^2 (n-1) A: rho = gamma^2 (n-1)^2); the star S_n (S = D^1/2 A D^1/2
    = sqrt(n-1) A: rho = gamma^2 (n-1)); the complete bipartite K_{p,q}
    (S = sqrt(pq) A, rho(A) = sqrt(pq): rho = gamma^2 p q); K_n with every weight
    w (rho = gamma^2 w^2 (n-1)^2), and with random signs (|A'| enters)."""
    gam = 0.37
    for n in (3, 6, 11):
        assert R.second_moment_radius(I.complete(n), gam) == pytest.approx(gam ** 2 * (n - 1) ** 2, rel=1e-12)
        assert R.second_moment_radius(I.star(n), gam) == pytest.approx(gam ** 2 * (n - 1), rel=1e-12)
    p, q = 3, 5
    kpq = I.from_edges(p + q, [(i, p + j) for i in range(p) for j in range(q)])
    assert R.second_moment_radius(kpq, gam) == pytest.approx(gam ** 2 * p * q, rel=1e-12)
    g = I.complete(7)
    w = np.full(g.nnz, 1.5, np.float32)
    assert R.second_moment_radius(g, gam, values=w) == pytest.approx(gam ** 2 * 1.5 ** 2 * 36, rel=1e-6)
    signs = np.where(np.random.default_rng(1).random(g.nnz) < 0.5, -1.5, 1.5).astype(np.float32)
    assert R.second_moment_radius(g, gam, values=signs) == pytest.approx(gam ** 2 * 1.5 ** 2 * 36, rel=1e-6)


def test_second_moment_radius_is_the_growth_of_the_enumerated_second_moment():
    """With the single coefficient zeta_K = 1 the exact second moment of a
    walk's contribution (Lemma 2 enumerated term by term) grows by rho per
    step for large K, on an irregular graph (BA n = 9)."""
    g = I.barabasi_albert(9, 2, 4)
    gam = 0.3
    rho = R.second_moment_radius(g, gam)
    m2 = []
    for K in (8, 9):
        c = np.zeros(K + 1)
        c[K] = 1.0
        ex = R.enumerate_action(g, c, gamma=gam)
        m2.append(np.sum(ex["var_walk"] + ex["Eq"] ** 2))
    assert rho > 1.0    # this graph's hubs make the second moment grow
    assert m2[1] / m2[0] == pytest.approx(rho, rel=0.01)
