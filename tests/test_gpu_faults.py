"""Error paths under an injected allocation failure (host-side injection,
mcf_inject_allocation_failure): for every allocation point of a solve and of
a batch plan the call returns MCF_ERR_OOM and releases what it took, and the
next call -- with the injection spent -- computes the same result as before.
No GPU fault is involved: the failing allocation is refused on the host."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import reference as R
from paper_2308_01037_gb300 import inputs as I
from paper_2308_01037_gb300 import mcf as M

pytestmark = pytest.mark.gpu


def test_injected_allocation_failures_return_oom_and_leave_the_library_usable():
    g = I.rmat(11, 16, seed=3)
    h = M.mcf_create_graph(g.n, g.row_ptr, g.col_idx)
    gam = 1.0 / M.mcf_spectral_radius(h)
    c = R.exp_coeffs(30)
    kw = dict(scale=gam, walks_per_node=8, w_cutoff=1e-6, seed=4, precision=M.MCF_F32W_F64ACC)
    nodes = np.array([3, 40, 400], np.int64)
    calls = {
        "tc": lambda: M.mcf_total_communicability(h, c, **kw),
        "sc_subset": lambda: M.mcf_subgraph_centrality(h, c, nodes=nodes, **kw),
        "budgeted": lambda: M.mcf_total_communicability(h, c, target_rel_err=1e-3, **kw),
        "batch": lambda: M.mcf_batch_run(M.mcf_batch_create(
            [dict(graph=h, kind=M.MCF_QUERY_SUBGRAPH_CENTRALITY, coeffs=c, nodes=nodes, **kw),
             dict(graph=h, kind=M.MCF_QUERY_TOTAL_COMMUNICABILITY, coeffs=c, **kw)]))[0],
    }
    try:
        for name, call in calls.items():
            clean = call()
            clean = clean.copy() if isinstance(clean, np.ndarray) else clean
            failures = 0
            for after in range(0, 40):
                M.mcf_inject_allocation_failure(after)
                try:
                    call()
                except M.McfError as e:
                    assert e.status == 3, (name, after, e)      # MCF_ERR_OOM
                    failures += 1
                M.mcf_inject_allocation_failure(-1)
                again = call()
                if isinstance(clean, np.ndarray):
                    assert np.array_equal(again, clean) or np.allclose(again, clean, rtol=1e-12, atol=1e-13), name
            assert failures > 0, name
    finally:
        M.mcf_inject_allocation_failure(-1)
        h.close()
