"""The seeded synthetic inputs that stand in for the paper's graphs (Section 4:
kronecker, smallworld and the real networks; the benchmark configurations'
R-MAT, Barabasi-Albert, Erdos-Renyi and configuration-model graphs): every
generator returns a valid symmetric, loop-free, duplicate-free CSR with the
structure its recipe states, reproducibly from its seed and independently of
the number of host threads."""
import os
import subprocess
import sys

import numpy as np

from paper_2308_01037_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def assert_valid_undirected(g):
    rp, ci = g.row_ptr, g.col_idx
    assert rp.dtype == np.int64 and ci.dtype == np.int32
    assert rp[0] == 0 and rp[-1] == len(ci) and np.all(np.diff(rp) >= 0)
    assert np.all((ci >= 0) & (ci < g.n))
    rows = np.repeat(np.arange(g.n, dtype=np.int64), g.degree)
    same_row = rows[1:] == rows[:-1]
    assert np.all(ci[1:][same_row] > ci[:-1][same_row]), "rows sorted, no duplicates"
    assert not np.any(rows == ci), "no loops"
    fwd = np.sort(rows * g.n + ci)
    bwd = np.sort(ci.astype(np.int64) * g.n + rows)
    assert np.array_equal(fwd, bwd), "symmetric"


def test_rmat_structure_and_permutation():
    """Graph500 R-MAT: 2^s nodes, at most 2 * 16 * 2^s entries after
    symmetrisation and de-duplication, a heavy-tailed degree sequence; without
    the random permutation ids correlate with degree (node 0 is the corner the
    quadrant probabilities favour), with it they do not."""
    g = I.rmat(12, 16, seed=1)
    assert_valid_undirected(g)
    assert g.n == 4096 and 0.5 * 2 * 16 * 4096 < g.nnz <= 2 * 16 * 4096
    d = g.degree
    assert d.max() > 20 * d.mean()
    raw = I.rmat(12, 16, seed=1, permute=False)
    assert_valid_undirected(raw)
    assert int(np.argmax(raw.degree)) == 0
    ids = np.arange(g.n)
    assert np.corrcoef(ids, np.argsort(np.argsort(raw.degree)))[0, 1] < -0.3
    assert abs(np.corrcoef(ids, np.argsort(np.argsort(d)))[0, 1]) < 0.1
    # the permutation relabels nodes: same degree multiset
    assert np.array_equal(np.sort(d), np.sort(raw.degree))


def test_generators_are_reproducible_and_seeded():
    for make in (lambda s: I.rmat(10, 16, seed=s), lambda s: I.barabasi_albert(500, 3, s),
                 lambda s: I.erdos_renyi(800, 10.0, s), lambda s: I.config_powerlaw(2000, 2.5, 20.0, s),
                 lambda s: I.smallworld(600, 10, 0.2, s)):
        a, b, c = make(3), make(3), make(4)
        assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col_idx, b.col_idx)
        assert not (np.array_equal(a.row_ptr, c.row_ptr) and np.array_equal(a.col_idx, c.col_idx))


def test_output_does_not_depend_on_host_threads():
    code = ("import hashlib, sys; sys.path.insert(0, %r)\n"
            "from paper_2308_01037_gb300 import inputs as I\n"
            "h = hashlib.sha256()\n"
            "for g in (I.rmat(13, 16, seed=5), I.smallworld(5000, 10, 0.3, 2), I.config_powerlaw(20000, 2.5, 20.0, 1)):\n"
            "    h.update(g.row_ptr.tobytes()); h.update(g.col_idx.tobytes())\n"
            "print(h.hexdigest())\n") % ROOT
    out = []
    for threads in ("1", "4"):
        env = dict(os.environ, OMP_NUM_THREADS=threads)
        out.append(subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                                  check=True, timeout=300).stdout.strip())
    assert out[0] == out[1] and len(out[0]) == 64


def test_barabasi_albert_edge_count_and_seed_clique():
    """Start from K_{m+1}; each later node adds m distinct edges: exactly
    m(m+1)/2 + (n - m - 1) m edges, minimum degree m."""
    n, m = 2000, 3
    g = I.barabasi_albert(n, m, 0)
    assert_valid_undirected(g)
    assert g.nnz == 2 * (m * (m + 1) // 2 + (n - m - 1) * m)
    assert g.degree.min() >= m
    A = g.dense()
    assert np.all(A[: m + 1, : m + 1] + np.eye(m + 1) == 1.0)
    assert g.degree.max() > 10 * m   # preferential attachment grows hubs


def test_erdos_renyi_mean_and_poisson_spread():
    g = I.erdos_renyi(20000, 12.0, 0)
    assert_valid_undirected(g)
    d = g.degree
    assert abs(d.mean() / 12.0 - 1.0) < 0.02
    assert 0.9 < d.var() / d.mean() < 1.1   # binomial(n - 1, p): variance close to the mean


def test_configuration_model_power_law():
    """k^-2.5 on [k_min, sqrt(20 n)] with k_min fitted to mean 20: after erasing
    loops and multi-edges the mean stays within 5-10 % above 20, and the
    degree CCDF falls by 2^-1.5 per doubling of k."""
    n = 200_000
    g = I.config_powerlaw(n, 2.5, 20.0, 2)
    assert_valid_undirected(g)
    d = g.degree
    assert 20.0 <= d.mean() <= 22.0
    assert d.max() <= int(np.sqrt(20.0 * n))
    kmin = int(d.min())
    ccdf = [(d >= kmin * 2 ** t).mean() for t in range(1, 5)]
    ratios = np.array(ccdf[1:]) / np.array(ccdf[:-1])
    assert np.all(np.abs(ratios / 2 ** -1.5 - 1.0) < 0.12), ratios


def test_watts_strogatz_ring_and_rewiring():
    n, k = 1000, 10
    ring = I.smallworld(n, k, 0.0, 0)
    assert_valid_undirected(ring)
    assert np.all(ring.degree == k)
    off = (ring.col_idx.astype(np.int64) - np.repeat(np.arange(n), k)) % n
    assert set(np.unique(off)) == {1, 2, 3, 4, 5, n - 5, n - 4, n - 3, n - 2, n - 1}
    g = I.smallworld(10000, k, 0.1, 0)
    assert_valid_undirected(g)
    assert 0.99 * 10000 * k <= g.nnz <= 10000 * k
    assert g.degree.min() < k < g.degree.max()


def test_closed_form_graphs():
    for g, deg in ((I.complete(6), [5] * 6), (I.path(4), [1, 2, 2, 1]), (I.cycle(5), [2] * 5),
                   (I.star(5), [4, 1, 1, 1, 1])):
        assert_valid_undirected(g)
        assert g.degree.tolist() == deg
    g = I.add_isolated(I.path(3), 2)
    assert g.n == 5 and g.degree.tolist() == [1, 2, 1, 0, 0]


def test_symmetric_weights():
    g = I.barabasi_albert(300, 3, 1)
    for signed in (False, True):
        w = I.symmetric_weights(g, seed=2, signed=signed, low=0.25, high=2.0)
        assert w.dtype == np.float32 and len(w) == g.nnz
        A = np.zeros((g.n, g.n))
        A[np.repeat(np.arange(g.n), g.degree), g.col_idx] = w
        assert np.array_equal(A, A.T)
        assert np.all((np.abs(w) >= 0.25) & (np.abs(w) < 2.0))
        assert (w < 0).any() == signed


def test_directed_generators_and_bipartite_symmetrization():
    g = I.directed_erdos_renyi(50, 4.0, 1)
    rows = np.repeat(np.arange(g.n), g.degree)
    assert not np.any(rows == g.col_idx)
    gl = I.directed_erdos_renyi(50, 4.0, 1, loops=True)
    assert np.any(np.repeat(np.arange(gl.n), gl.degree) == gl.col_idx)
    A = g.dense()
    assert not np.array_equal(A, A.T)
    c = I.directed_cycle(4).dense()
    assert np.array_equal(c, np.roll(np.eye(4), 1, axis=1))
    w = np.random.default_rng(0).uniform(-1.0, 1.0, g.nnz).astype(np.float32)
    b, bw = I.bipartite_symmetrization(g, w)
    assert_valid_undirected(b)
    W = np.zeros((g.n, g.n))
    W[rows, g.col_idx] = w
    B = np.zeros((2 * g.n, 2 * g.n))
    B[np.repeat(np.arange(b.n), b.degree), b.col_idx] = bw
    expect = np.block([[np.zeros_like(W), W], [W.T, np.zeros_like(W)]])
    assert np.array_equal(B, expect)
