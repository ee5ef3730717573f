"""The allocation-free total-communicability entry point.

Some callers cannot let a library call cudaMalloc: code that runs inside a
framework owning every device allocation, or a process whose allocator is
exhausted.  For them
mcf_total_communicability_noalloc keeps all its scratch in one fixed device
array inside libmcf.  These tests call it through the C ABI and check that it
returns what the allocating entry point (mcf_total_communicability) returns
for the same inputs and seed, within the parity tolerance of the other GPU
tests, over consecutive calls that reuse the array; that sizes beyond its
limits are refused with a clear error before any device work; and that a
malformed CSR is refused by its device-side check before any walk runs,
leaving the output untouched (every malformed case below keeps every index
the check reads inside the arrays it is given).  The file is named so that pytest
collects it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import reference as R
from paper_2308_01037_gb300 import inputs as I
from paper_2308_01037_gb300 import mcf as M

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-12, 1e-13
MAX_NODES = 1 << 17


def _call_noalloc(lib, g_rp, g_ci, n, params, y):
    return lib.mcf_total_communicability_noalloc(n, int(g_ci.numel()), g_rp.data_ptr(), g_ci.data_ptr(),
                                                 ctypes.byref(params), y.data_ptr())


def _case(name):
    if name == "ba":
        g = I.barabasi_albert(1000, 3, 0)
        kw = dict(walks_per_node=200, w_cutoff=0.0, seed=3, request_id=1, precision=M.MCF_F64)
    else:
        g = I.rmat(12, 16, seed=5)
        kw = dict(n_walks=200000, w_cutoff=1e-6, seed=4, request_id=2, precision=M.MCF_F32W_F64ACC)
    gam = 1.0 / R.lambda_max(g)
    return g, gam, kw


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls():
    lib = M.load()
    c = R.exp_coeffs(30)
    for name in ("ba", "rmat", "ba"):          # three calls in a row share the scratch array
        g, gam, kw = _case(name)
        rp = torch.from_numpy(g.row_ptr).cuda()
        ci = torch.from_numpy(g.col_idx).cuda()
        y = torch.full((g.n,), float("nan"), dtype=torch.float64, device="cuda")
        p, keep = M._params(c, scale=gam, stream=torch.cuda.current_stream().cuda_stream, **kw)
        status = _call_noalloc(lib, rp, ci, g.n, p, y)
        assert status == 0, M.mcf_last_error()
        torch.cuda.synchronize()
        h = M.mcf_create_graph(g.n, rp, ci)
        ref = M.mcf_total_communicability(h, c, scale=gam, **kw)
        h.close()
        got = y.cpu().numpy()
        assert np.all(np.abs(got - ref) <= RTOL * np.abs(ref) + ATOL), (name, np.abs(got - ref).max())


def test_noalloc_refuses_sizes_beyond_its_limits():
    lib = M.load()
    c = R.exp_coeffs(30)
    g = I.path(8)
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    y = torch.zeros(MAX_NODES + 1, dtype=torch.float64, device="cuda")
    p, keep = M._params(c, scale=0.5, n_walks=100)
    assert _call_noalloc(lib, rp, ci, MAX_NODES + 1, p, y) == 1
    assert str(MAX_NODES) in M.mcf_last_error()
    p, keep = M._params(c, scale=0.5, walks_per_node=1 << 30)
    assert _call_noalloc(lib, rp, ci, g.n, p, y) == 1
    assert "walk" in M.mcf_last_error()
    # N_s + n would overflow a signed 64-bit sum: refused on the host
    p, keep = M._params(c, scale=0.5, n_walks=(1 << 63) - 2)
    assert _call_noalloc(lib, rp, ci, g.n, p, y) == 1
    assert "walk" in M.mcf_last_error()
    p, keep = M._params(c, scale=0.5, walks_per_node=(1 << 62))
    assert _call_noalloc(lib, rp, ci, g.n, p, y) == 1
    host_y = np.zeros(g.n)
    p, keep = M._params(c, scale=0.5, n_walks=100)
    assert lib.mcf_total_communicability_noalloc(g.n, g.nnz, rp.data_ptr(), ci.data_ptr(), ctypes.byref(p),
                                                 host_y.ctypes.data) == 1
    assert "device" in M.mcf_last_error()


def _malformed(kind):
    """A binary CSR of P_8 broken in one way; nnz is always the true length of col."""
    g = I.path(8)
    rp, ci = g.row_ptr.copy(), g.col_idx.copy()
    if kind == "row_ptr_end":        # row_ptr[n] != nnz
        rp[-1] = rp[-1] - 1
    elif kind == "column_out_of_range":
        ci[-1] = g.n
    elif kind == "unsorted_row":     # row 3 holds (2, 4): swap them
        b = rp[3]
        ci[b], ci[b + 1] = ci[b + 1], ci[b]
    elif kind == "duplicate_column":  # row 3 holds (2, 4): make it (2, 2)
        b = rp[3]
        ci[b + 1] = ci[b]
    return g.n, rp, ci


@pytest.mark.parametrize("kind", ["row_ptr_end", "column_out_of_range", "unsorted_row", "duplicate_column"])
def test_noalloc_refuses_a_malformed_csr(kind):
    lib = M.load()
    n, rp_h, ci_h = _malformed(kind)
    rp = torch.from_numpy(rp_h).cuda()
    ci = torch.from_numpy(ci_h).cuda()
    y = torch.full((n,), 7.0, dtype=torch.float64, device="cuda")
    p, keep = M._params(R.exp_coeffs(30), scale=0.5, n_walks=1000,
                        stream=torch.cuda.current_stream().cuda_stream)
    assert _call_noalloc(lib, rp, ci, n, p, y) == 2      # MCF_ERR_INVALID_GRAPH
    assert "CSR" in M.mcf_last_error()
    torch.cuda.synchronize()
    assert torch.all(y == 7.0)
