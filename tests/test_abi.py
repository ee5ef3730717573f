"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every entry point include/mcf.h declares; argument errors are
reported without touching the device."""
import ctypes
import os
import re

import pytest

from paper_2308_01037_gb300 import build as B
from paper_2308_01037_gb300 import mcf as M

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "mcf.h")


def declared_entry_points():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mcf_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return M.load()


def test_header_declares_the_survey_boundary():
    names = declared_entry_points()
    for required in ("mcf_create_graph", "mcf_destroy_graph", "mcf_spectral_radius", "mcf_action",
                     "mcf_total_communicability", "mcf_subgraph_centrality", "mcf_katz", "mcf_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_entry_points():
        assert hasattr(lib, name), name
    assert set(declared_entry_points()) == set(M.SIGNATURES), "binding and header disagree"


def test_version_and_empty_error(lib):
    assert "sm_103a" in M.mcf_version()
    assert isinstance(M.mcf_last_error(), str)


def test_null_arguments_rejected_without_device(lib):
    p, keep = M._params([1.0, 1.0, 0.5], n_walks=10)
    y = (ctypes.c_double * 4)()
    assert lib.mcf_total_communicability(None, ctypes.byref(p), y, None) == 1
    assert "graph" in M.mcf_last_error()
    assert lib.mcf_create_graph(3, None, None, None, 0, None) == 1
    assert lib.mcf_katz(None, 0.1, 0, ctypes.byref(p), y, None) == 1
    assert lib.mcf_destroy_graph(None) == 0
    out = ctypes.c_double()
    assert lib.mcf_gershgorin(None, ctypes.byref(out)) == 1


def test_params_struct_layout_matches_c():
    # offsets of the C struct on LP64: pointer 0, int32 8, double 16, int64 24, int64 32,
    # double 40, uint64 48, uint32 56, int32 60, int32 64, pointer 72
    offs = {f[0]: getattr(M.mcf_params, f[0]).offset for f in M.mcf_params._fields_}
    assert offs == {"coeffs": 0, "n_coeffs": 8, "scale": 16, "n_walks": 24, "walks_per_node": 32, "w_cutoff": 40,
                    "seed": 48, "request_id": 56, "precision": 60, "deterministic": 64, "stream": 72}
    assert ctypes.sizeof(M.mcf_params) == 80
    assert ctypes.sizeof(M.mcf_stats) == 32
