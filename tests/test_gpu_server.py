"""The request server (mcf_server_*): continuous batching over resident graphs.

Requests submitted concurrently are grouped into batches that run on several
streams at once; each request keeps its own walk ids, so its result must equal
the oracle's same-seed estimate and the single call's (parity tolerance 1e-12
relative) whatever it was batched with, and batches' device work must overlap
in time.  Admission by device footprint (checked against what a batch really
allocates), releasing tickets and the latency counters are checked too.
"""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import estimator as E
from oracle import reference as R
from paper_2308_01037_gb300 import inputs as I
from paper_2308_01037_gb300 import mcf as M

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-12, 1e-13


@pytest.fixture(scope="module")
def pool():
    gs = [I.rmat(10, 16, seed=11), I.rmat(12, 16, seed=12), I.barabasi_albert(3000, 4, 13)]
    out = []
    for g in gs:
        h = M.mcf_create_graph(g.n, g.row_ptr, g.col_idx)
        out.append((g, h, 1.0 / R.lambda_max(g)))
    return out


def request(pool, i, rng):
    g, h, gam = pool[i % len(pool)]
    kind = [M.MCF_QUERY_TOTAL_COMMUNICABILITY, M.MCF_QUERY_KATZ, M.MCF_QUERY_SUBGRAPH_CENTRALITY,
            M.MCF_QUERY_ACTION][i % 4]
    base = dict(graph=h, kind=kind, seed=1000 + i, request_id=i, precision=M.MCF_F32W_F64ACC)
    c = R.exp_coeffs(30)
    if kind == M.MCF_QUERY_TOTAL_COMMUNICABILITY:
        base.update(coeffs=c, scale=gam, n_walks=20 * g.n, w_cutoff=1e-6)
    elif kind == M.MCF_QUERY_KATZ:
        base.update(katz_gamma=0.85 * gam, katz_terms=0, walks_per_node=4)
    elif kind == M.MCF_QUERY_SUBGRAPH_CENTRALITY:
        base.update(coeffs=c, scale=gam, walks_per_node=40,
                    nodes=rng.choice(g.n, size=min(64, g.n), replace=False).astype(np.int64))
    else:
        base.update(coeffs=c, scale=gam, n_walks=10 * g.n, v=rng.standard_normal(g.n))
    return base


def single(q):
    keys = ("scale", "n_walks", "walks_per_node", "w_cutoff", "seed", "request_id", "precision")
    kw = {k: q[k] for k in keys if k in q}
    if q["kind"] == M.MCF_QUERY_TOTAL_COMMUNICABILITY:
        return M.mcf_total_communicability(q["graph"], q["coeffs"], **kw)
    if q["kind"] == M.MCF_QUERY_KATZ:
        return M.mcf_katz(q["graph"], q["katz_gamma"], q["katz_terms"], **kw)
    if q["kind"] == M.MCF_QUERY_SUBGRAPH_CENTRALITY:
        return M.mcf_subgraph_centrality(q["graph"], q["coeffs"], nodes=q["nodes"], **kw)
    return M.mcf_action(q["graph"], q["v"], q["coeffs"], **kw)


def oracle_of(q, pool):
    """The oracle's same-seed estimate of a served request (float32 walk weights)."""
    g = next(gg for gg, hh, _ in pool if hh is q["graph"])
    kw = dict(seed=q["seed"], request_id=q["request_id"], precision=1)
    if q["kind"] == M.MCF_QUERY_TOTAL_COMMUNICABILITY:
        return E.action(g, q["coeffs"], gamma=q["scale"], n_walks=q["n_walks"], w_cutoff=q["w_cutoff"], **kw)["y"]
    if q["kind"] == M.MCF_QUERY_KATZ:
        # K from the tail bound with the library's lambda_max (the value mcf_katz uses)
        K = R.katz_terms_for_tail(q["katz_gamma"] * M.mcf_spectral_radius(q["graph"]), 1e-4)
        return E.action(g, R.katz_coeffs(K), gamma=q["katz_gamma"], walks_per_node=q["walks_per_node"], **kw)["y"]
    if q["kind"] == M.MCF_QUERY_SUBGRAPH_CENTRALITY:
        return E.diag(g, q["coeffs"], gamma=q["scale"], walks_per_node=q["walks_per_node"], nodes=q["nodes"], **kw)["d"]
    return E.action(g, q["coeffs"], v=q["v"], gamma=q["scale"], n_walks=q["n_walks"], **kw)["y"]


def test_results_in_the_mix_equal_results_alone(pool):
    rng = np.random.default_rng(0)
    qs = [request(pool, i, rng) for i in range(48)]
    srv = M.mcf_server_create(hbm_budget_bytes=8 << 30, max_inflight=3, max_batch=8, batch_window_ms=1.0)
    tickets = [None] * len(qs)

    def client(lo, hi):
        for i in range(lo, hi):
            tickets[i] = M.mcf_server_submit(srv, qs[i])

    th = [threading.Thread(target=client, args=(k * 12, (k + 1) * 12)) for k in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    outs = [M.mcf_server_wait(srv, t, timeout_s=120.0) for t in tickets]
    st = M.mcf_server_get_stats(srv)
    srv.close()
    assert st["completed"] == len(qs) and st["rejected"] == 0
    assert st["batches"] >= 2 and 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    for q, (out, lat) in zip(qs, outs):
        out = np.asarray(out)
        for ref in (oracle_of(q, pool), single(q)):
            assert np.all(np.abs(out - ref) <= RTOL * np.abs(ref) + ATOL), q["kind"]
        assert lat > 0


def test_batches_overlap_on_the_device(pool):
    """Two long requests (tens of milliseconds of walks each) handed to two
    workers at once: the second batch's first kernel runs before the first
    batch's last kernel has finished (the device windows from the GPU's global
    timer overlap), and sampled entries of both results equal the oracle's."""
    g, h, gam = pool[1]
    c = R.exp_coeffs(30)
    qs = [dict(graph=h, kind=M.MCF_QUERY_TOTAL_COMMUNICABILITY, coeffs=c, scale=gam, n_walks=20000 * g.n,
               w_cutoff=1e-6, seed=77 + i, request_id=900 + i, precision=M.MCF_F32W_F64ACC) for i in range(2)]
    srv = M.mcf_server_create(hbm_budget_bytes=8 << 30, max_inflight=2, max_batch=1)
    tickets = [M.mcf_server_submit(srv, q) for q in qs]
    outs = [M.mcf_server_wait(srv, t, timeout_s=120.0)[0] for t in tickets]
    st = M.mcf_server_get_stats(srv)
    srv.close()
    assert st["batches"] == 2
    assert st["max_concurrent_batches"] == 2 and st["device_overlap_ms"] > 0.0, st
    nodes = np.nonzero((g.degree >= 1) & (g.degree <= 3))[0][:4].astype(np.int64)   # cheap for the oracle
    for q, out in zip(qs, outs):
        ref = E.action(g, c, gamma=gam, n_walks=q["n_walks"], w_cutoff=1e-6, seed=q["seed"],
                       request_id=q["request_id"], precision=1, nodes=nodes)["y"]
        got = np.asarray(out)[nodes]
        assert np.all(np.abs(got - ref) <= RTOL * np.abs(ref) + ATOL)


def test_footprint_covers_what_a_batch_allocates(pool):
    """The admission estimate of a request is at least the device memory
    mcf_batch_create allocates for a batch of that request alone (and not
    more than twice that plus 64 MiB for the fused kinds)."""
    rng = np.random.default_rng(3)
    for i in range(8):
        q = request(pool, i, rng)
        q["out"] = torch.empty(len(q["nodes"]) if "nodes" in q else q["graph"].n, dtype=torch.float64,
                               device="cuda")
        est = M.mcf_query_footprint(q)
        b = M.mcf_batch_create([q])
        got = M.mcf_batch_device_bytes(b)
        b.close()
        assert est >= got, (i, est, got)
        if q["kind"] != M.MCF_QUERY_ACTION:
            assert est <= 2 * got + (64 << 20), (i, est, got)


def test_released_tickets_are_forgotten(pool):
    g, h, gam = pool[0]
    srv = M.mcf_server_create(hbm_budget_bytes=1 << 30, max_inflight=1, max_batch=2)
    t = M.mcf_server_submit(srv, dict(graph=h, kind=M.MCF_QUERY_TOTAL_COMMUNICABILITY, coeffs=R.exp_coeffs(10),
                                      scale=gam, n_walks=1000, seed=1))
    M.mcf_server_wait(srv, t, timeout_s=60.0)
    M.mcf_server_release(srv, t)
    with pytest.raises(M.McfError):
        M.mcf_server_poll(srv, t)
    with pytest.raises(M.McfError):
        M.mcf_server_release(srv, t)
    srv.close()


def test_admission_by_memory_budget(pool):
    g, h, gam = pool[1]
    q = dict(graph=h, kind=M.MCF_QUERY_TOTAL_COMMUNICABILITY, coeffs=R.exp_coeffs(10), scale=gam, n_walks=1000)
    srv = M.mcf_server_create(hbm_budget_bytes=M.mcf_query_footprint(q) - 1, max_inflight=1, max_batch=4)
    t = M.mcf_server_submit(srv, q)
    done, res = M.mcf_server_poll(srv, t)
    assert done and res == 5   # MCF_ERR_ADMISSION
    with pytest.raises(M.McfError):
        M.mcf_server_wait(srv, t)
    assert M.mcf_server_get_stats(srv)["rejected"] == 1
    srv.close()


def test_requests_queue_until_memory_frees(pool):
    """A budget that fits one request at a time still serves them all, one batch each."""
    g, h, gam = pool[0]
    c = R.exp_coeffs(20)
    qs = [dict(graph=h, kind=M.MCF_QUERY_TOTAL_COMMUNICABILITY, coeffs=c, scale=gam, n_walks=10 * g.n, seed=i,
               request_id=i) for i in range(6)]
    # the server's device-footprint estimate of one such request; 1.5 of it admits one at a time
    one = M.mcf_query_footprint(qs[0])
    srv = M.mcf_server_create(hbm_budget_bytes=int(1.5 * one), max_inflight=2, max_batch=8)
    tickets = [M.mcf_server_submit(srv, q) for q in qs]
    outs = [M.mcf_server_wait(srv, t, timeout_s=60.0)[0] for t in tickets]
    st = M.mcf_server_get_stats(srv)
    srv.close()
    assert st["batches"] == len(qs)
    for q, out in zip(qs, outs):
        ref = single(q)
        assert np.all(np.abs(out - ref) <= RTOL * np.abs(ref) + ATOL)


def test_cancel_a_queued_request(pool):
    """With one worker busy on a long request, a queued request can be
    cancelled (it completes with MCF_ERR_CANCELLED, output untouched) while
    the next one is still served; a running request cannot be cancelled."""
    g, h, gam = pool[1]
    c = R.exp_coeffs(30)
    long_q = dict(graph=h, kind=M.MCF_QUERY_TOTAL_COMMUNICABILITY, coeffs=c, scale=gam, n_walks=100000 * g.n,
                  w_cutoff=1e-6, seed=1, request_id=1)
    small = [dict(graph=h, kind=M.MCF_QUERY_TOTAL_COMMUNICABILITY, coeffs=c, scale=gam, n_walks=10 * g.n,
                  seed=10 + i, request_id=10 + i, out=np.full(g.n, -7.0)) for i in range(2)]
    srv = M.mcf_server_create(hbm_budget_bytes=8 << 30, max_inflight=1, max_batch=1)
    t_long = M.mcf_server_submit(srv, long_q)
    t_b = M.mcf_server_submit(srv, small[0])
    t_c = M.mcf_server_submit(srv, small[1])
    M.mcf_server_cancel(srv, t_c)
    done, status = M.mcf_server_poll(srv, t_c)
    assert done and status == 7                     # MCF_ERR_CANCELLED
    with pytest.raises(M.McfError):
        M.mcf_server_cancel(srv, t_c)               # not queued any more
    out_b, _ = M.mcf_server_wait(srv, t_b, timeout_s=120.0)
    M.mcf_server_wait(srv, t_long, timeout_s=120.0)
    st = M.mcf_server_get_stats(srv)
    srv.close()
    assert st["cancelled"] == 1 and st["completed"] == 3
    assert np.all(small[1]["out"] == -7.0)          # the cancelled request wrote nothing
    ref = single(small[0])
    assert np.all(np.abs(out_b - ref) <= RTOL * np.abs(ref) + ATOL)
