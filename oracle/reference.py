"""FP64 reference values (ORACLE -- test infrastructure only).

What the estimators of the paper converge to, computed without sampling:

* ``dense_funm``: f(A') = V diag(sum_k zeta_k lambda^k) V^T from a dense
  symmetric eigendecomposition (Eq. power_series evaluated on the spectrum),
  for tiny and small graphs.
* ``series_action`` / ``series_diag``: the truncated series
  sum_{k<=K} zeta_k A'^k v (and its diagonal on chosen nodes) by repeated
  float64 sparse products, for large graphs.
* ``second_moment_radius``: the spectral radius of M = diag(sum_j |a'_ij|) |A'|,
  the matrix whose powers carry the second moments of the walk weights
  (Definition 1 and Eq. weights: E[(W^(k))^2 ...] = (M^k ...)), from a dense
  eigendecomposition (or ARPACK) of the similar symmetric D^1/2 |A'| D^1/2.
* ``enumerate_action`` / ``enumerate_diag``: the exact expectation and
  variance of one walk's contribution, by enumerating every walk with its
  probability p_{l0} t_{l0 l1} ... (Definition 1) and weight (Eq. weights),
  i.e. Lemma 2 evaluated term by term, including the cutoff of
  Eq. weight_cutoff.  Plain Python loops: tiny graphs only.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# ---------------------------------------------------------------- coefficients
def exp_coeffs(K: int, beta: float = 1.0) -> np.ndarray:
    """zeta_k = beta^k / k!, k = 0..K (the exponential, Section 2.2)."""
    return np.array([beta ** k / math.factorial(k) for k in range(K + 1)], dtype=np.float64)


def katz_coeffs(K: int) -> np.ndarray:
    """zeta_k = 1, k = 0..K: the Neumann series of (I - A')^{-1} (Section 4.5)."""
    return np.ones(K + 1, dtype=np.float64)


def mittag_leffler_coeffs(K: int, alpha: float, beta: float = 1.0) -> np.ndarray:
    """zeta_k = 1 / Gamma(alpha k + beta), k = 0..K: the Mittag-Leffler function
    E_{alpha,beta} (Section 1 names it among the functions the power series covers)."""
    return np.array([math.exp(-math.lgamma(alpha * k + beta)) if alpha * k + beta > 0 else 0.0
                     for k in range(K + 1)], dtype=np.float64)


def katz_terms_for_tail(rho: float, tol: float) -> int:
    """Smallest K with rho^(K+1) / (1 - rho) <= tol (geometric tail of the Neumann series)."""
    if not (0.0 < rho < 1.0):
        raise ValueError("the Neumann series needs 0 < rho < 1")
    return max(2, int(math.ceil(math.log(tol * (1.0 - rho)) / math.log(rho) - 1.0)))


# ---------------------------------------------------------------- matrices
def csr_matrix(g, values=None, gamma: float = 1.0) -> sp.csr_matrix:
    data = np.ones(g.nnz) if values is None else np.asarray(values, dtype=np.float64)
    return sp.csr_matrix((gamma * data, g.col_idx, g.row_ptr), shape=(g.n, g.n))


def lambda_max(g, values=None) -> float:
    """Largest eigenvalue of the symmetric adjacency matrix (dense for n <= 2000, else ARPACK)."""
    if g.n <= 2000:
        return float(np.linalg.eigvalsh(csr_matrix(g, values).toarray())[-1])
    A = csr_matrix(g, values).astype(np.float64)
    w = spla.eigsh(A, k=1, which="LA", tol=1e-13, return_eigenvectors=False, ncv=32, maxiter=100000)
    return float(w[0])


def gershgorin(g, values=None) -> float:
    """max_i sum_k |a_ik| (Gershgorin bound on the spectral radius, Section 4.5)."""
    A = csr_matrix(g, values)
    return float(np.abs(A).sum(axis=1).max()) if g.n else 0.0


# ---------------------------------------------------------------- dense (small graphs)
def second_moment_radius(g, gamma: float = 1.0, values=None) -> float:
    """rho(diag(s') |A'|), s'_i = sum_j |a'_ij|, A' = gamma A: one step of a walk
    multiplies its weight by s'_l (Eq. weights) and moves to j with
    probability |a'_lj| / s'_l (Definition 1), so the expected squared weight
    after k steps is (M^k 1)_l-weighted with M = diag(s') |A'|, and rho(M) is
    its growth factor.  M = D^1/2 (D^1/2 |A'| D^1/2) D^-1/2 with D = diag(s')
    for a symmetric A, so its spectrum is that of the symmetric middle factor."""
    A = abs(csr_matrix(g, values, gamma))
    s = np.asarray(A.sum(axis=1)).ravel()
    r = np.sqrt(s)
    S = sp.diags(r) @ A @ sp.diags(r)
    if g.n <= 2000:
        return float(np.abs(np.linalg.eigvalsh(S.toarray())).max())
    vals = spla.eigsh(S.tocsc(), k=1, which="LM", return_eigenvectors=False, tol=1e-12)
    return float(np.abs(vals).max())


def dense_funm(A: np.ndarray, coeffs) -> np.ndarray:
    """sum_k zeta_k A^k for symmetric A through its eigendecomposition."""
    lam, V = np.linalg.eigh(A)
    f = np.polynomial.polynomial.polyval(lam, np.asarray(coeffs, dtype=np.float64))
    return (V * f) @ V.T


def dense_powers_series(A: np.ndarray, coeffs) -> np.ndarray:
    """sum_k zeta_k A^k by explicit matrix powers (independent of the eigensolver)."""
    n = A.shape[0]
    F = np.zeros((n, n))
    P = np.eye(n)
    for k, z in enumerate(coeffs):
        if k:
            P = P @ A
        F += z * P
    return F


# ---------------------------------------------------------------- series (large graphs)
def series_action(g, coeffs, gamma: float = 1.0, v=None, values=None) -> np.ndarray:
    """sum_{k=0}^K zeta_k (gamma A)^k v by K float64 sparse products."""
    A = csr_matrix(g, values, gamma)
    t = np.ones(g.n) if v is None else np.asarray(v, dtype=np.float64).copy()
    y = coeffs[0] * t
    for k in range(1, len(coeffs)):
        t = A @ t
        y = y + coeffs[k] * t
    return y


def series_diag(g, coeffs, nodes, gamma: float = 1.0, values=None, block: int = 64) -> np.ndarray:
    """(sum_k zeta_k (gamma A)^k)_ii for i in ``nodes``, blocks of unit vectors."""
    A = csr_matrix(g, values, gamma)
    nodes = np.asarray(nodes, dtype=np.int64)
    out = np.zeros(len(nodes))
    for b0 in range(0, len(nodes), block):
        idx = nodes[b0:b0 + block]
        E = np.zeros((g.n, len(idx)))
        E[idx, np.arange(len(idx))] = 1.0
        T = E
        D = coeffs[0] * E
        for k in range(1, len(coeffs)):
            T = A @ T
            D = D + coeffs[k] * T
        out[b0:b0 + block] = D[idx, np.arange(len(idx))]
    return out


# ---------------------------------------------------------------- exact moments by enumeration
def _chain(g, values, gamma):
    """Definition 1 for a small graph: neighbour lists, a'_ij, t_ij, p_i."""
    n = g.n
    nbr, aval, tval = [], [], []
    rowabs = np.zeros(n)
    colnorm = np.zeros(n)
    colsq = np.zeros(n)
    for i in range(n):
        cols = g.col_idx[g.row_ptr[i]:g.row_ptr[i + 1]].tolist()
        a = ([1.0] * len(cols)) if values is None else [float(x) for x in values[g.row_ptr[i]:g.row_ptr[i + 1]]]
        a = [gamma * x for x in a]
        s = sum(abs(x) for x in a)
        nbr.append(cols)
        aval.append(a)
        tval.append([abs(x) / s for x in a] if s > 0 else [])
        rowabs[i] = s
        for j, x in zip(cols, a):
            colsq[j] += x * x            # column j collects a'_ij over the rows i
    colnorm = np.sqrt(colsq)
    return nbr, aval, tval, rowabs, colnorm


def _walk_moments(nbr, aval, tval, start, coeffs, w_cutoff, contrib):
    """E[X], E[X^2] of one walk from ``start`` where X = sum_k zeta_{k+2} W^(k) contrib(l_k).

    ``contrib(l)`` returns a vector; moments are returned per component.
    Every walk of at most K-2 transitions is enumerated with probability
    prod t and weight prod a/t (Eq. weights), stopped by the cutoff."""
    K = len(coeffs) - 1
    e1 = None
    e2 = None
    stack = [(start, 0, 1.0, 1.0, 0.0)]   # (state, step k, W, probability, partial X)
    while stack:
        l, k, W, P, X = stack.pop()
        if not (abs(W) > w_cutoff):
            leaf = True
        else:
            X = X + coeffs[k + 2] * W * contrib(l)
            leaf = (k + 2 >= K) or len(nbr[l]) == 0
        if leaf:
            x = np.asarray(X, dtype=np.float64)
            e1 = P * x if e1 is None else e1 + P * x
            e2 = P * x * x if e2 is None else e2 + P * x * x
            continue
        for j, a, t in zip(nbr[l], aval[l], tval[l]):
            stack.append((j, k + 1, W * (a / t), P * t, X))
    return e1, e2


def enumerate_action(g, coeffs, gamma: float = 1.0, v=None, w_cutoff: float = 0.0, values=None):
    """Exact E[y] and per-walk moments of RandFunmAction (Algorithm 3).

    Returns dict(mean_y, var_walk, r) where mean_y = zeta_0 v + zeta_1 r + A' E[q]
    and var_walk[i] = Var[X_i] of a single walk from i; with N_i walks the
    variance of y_j is sum_i a'_ji^2 var_walk[i] / N_i."""
    coeffs = np.asarray(coeffs, dtype=np.float64)
    K = len(coeffs) - 1
    n = g.n
    v = np.ones(n) if v is None else np.asarray(v, dtype=np.float64)
    nbr, aval, tval, rowabs, colnorm = _chain(g, values, gamma)
    r = np.array([sum(a * v[j] for j, a in zip(nbr[i], aval[i])) for i in range(n)])
    Eq = np.zeros(n)
    Vq = np.zeros(n)
    if K >= 2:
        for i in range(n):
            if colnorm[i] == 0:
                continue
            e1, e2 = _walk_moments(nbr, aval, tval, i, coeffs, w_cutoff, lambda l: r[l])
            Eq[i] = e1
            Vq[i] = max(e2 - e1 * e1, 0.0)
    y = coeffs[0] * v + (coeffs[1] * r if K >= 1 else 0.0)
    y = y + np.array([sum(a * Eq[j] for j, a in zip(nbr[i], aval[i])) for i in range(n)])
    return {"mean_y": y, "var_walk": Vq, "Eq": Eq, "r": r, "rowabs": rowabs, "colnorm": colnorm,
            "nbr": nbr, "aval": aval}


def action_variance(ex, nw) -> np.ndarray:
    """Variance of y_j = ... + sum_i a'_ji q_i with q_i the mean of N_i independent walks."""
    n = len(ex["mean_y"])
    var = np.zeros(n)
    for j in range(n):
        for i, a in zip(ex["nbr"][j], ex["aval"][j]):
            if nw[i] > 0:
                var[j] += a * a * ex["var_walk"][i] / nw[i]
    return var


def enumerate_diag(g, coeffs, gamma: float = 1.0, w_cutoff: float = 0.0, values=None, nw=None):
    """Exact E[d] and Var[d] of RandFunmDiag (Eq. rand_funm_formula_diag).

    For a walk from k, Y_{k,i} = sum_j a'_ji X_kj with X_kj = sum over visits
    of j of zeta_{m+2} W^(m); d_i = zeta_0 + zeta_1 a'_ii + sum_k a'_ik mean(Y_{k,i}).
    ``nw`` (walks per start) is needed for the variance."""
    coeffs = np.asarray(coeffs, dtype=np.float64)
    K = len(coeffs) - 1
    n = g.n
    nbr, aval, tval, rowabs, colnorm = _chain(g, values, gamma)
    # Arow[l] = row l of A' (a'_li for every i): what a visit of l adds to Y_{k, .}
    Arow = np.zeros((n, n))
    for i in range(n):
        for j, a in zip(nbr[i], aval[i]):
            Arow[i, j] += a
    mean = np.array([coeffs[0] + (coeffs[1] * Arow[i, i] if K >= 1 else 0.0) for i in range(n)])
    var = np.zeros(n)
    if K >= 2:
        for k in range(n):
            if colnorm[k] == 0:
                continue
            # contribution vector of visiting l: Y_{k,i} += zeta W a'_li for every i
            e1, e2 = _walk_moments(nbr, aval, tval, k, coeffs, w_cutoff, lambda l: Arow[l])
            for i in np.nonzero(Arow[:, k])[0]:        # the rows i of column k: a'_ik != 0
                a = Arow[i, k]
                mean[i] += a * e1[i]
                if nw is not None and nw[k] > 0:
                    var[i] += a * a * max(e2[i] - e1[i] ** 2, 0.0) / nw[k]
    return {"mean_d": mean, "var_d": var}
