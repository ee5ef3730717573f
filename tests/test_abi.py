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


def test_header_declares_the_core_entry_points():
    names = declared_entry_points()
    for required in ("mcf_create_graph", "mcf_destroy_graph", "mcf_spectral_radius", "mcf_action",
                     "mcf_total_communicability", "mcf_subgraph_centrality", "mcf_katz", "mcf_last_error"):
        assert required in names


def declared_arg_counts():
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for name, args in re.findall(r"\b(mcf_[a-z_0-9]+)\s*\(([^)]*)\)\s*;", text):
        args = args.strip()
        out[name] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_binding_signatures_have_the_header_argument_counts():
    counts = declared_arg_counts()
    assert set(counts) == set(M.SIGNATURES)
    for name, (args, _) in M.SIGNATURES.items():
        assert len(args) == counts[name], name


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


def test_struct_layouts_match_the_header(tmp_path):
    """Every ctypes struct of the binding has the field offsets and size the
    C compiler gives the header's struct (a small C program prints them)."""
    import subprocess

    structs = {"mcf_params": M.mcf_params, "mcf_stats": M.mcf_stats, "mcf_query": M.mcf_query,
               "mcf_server_config": M.mcf_server_config, "mcf_server_stats": M.mcf_server_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mcf.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f in cls._fields_:
            lines.append(f'printf("{name} {f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.check_call(["gcc", "-std=c11", "-I", inc, str(src), "-o", str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        name, field, val = line.split()
        got[(name, field)] = int(val)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for f in cls._fields_:
            assert got[(name, f[0])] == getattr(cls, f[0]).offset, (name, f[0])



def test_no_device_means_an_error_not_a_fallback(lib):
    """On a host without a usable CUDA device the first device call of the
    product path returns MCF_ERR_CUDA and the binding raises: nothing is
    computed on the CPU instead."""
    import numpy as np
    import torch

    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    rp = np.array([0, 1, 2], np.int64)
    ci = np.array([1, 0], np.int32)
    with pytest.raises(M.McfError) as ei:
        M.mcf_create_graph(2, rp, ci)
    assert ei.value.status == 4 and "CUDA" in str(ei.value)


def test_outputs_must_be_float64_contiguous():
    """The library writes results in place: an output of another dtype or a
    strided view is refused (a converted copy would silently take the results)."""
    import types

    import numpy as np
    import torch

    g = types.SimpleNamespace(n=4, handle=None)
    for bad in (np.zeros(4, np.float32), np.zeros(8)[::2], torch.zeros(4, dtype=torch.float32),
                torch.zeros(8, dtype=torch.float64)[::2]):
        with pytest.raises(TypeError):
            M.mcf_total_communicability(g, [1.0, 1.0, 0.5], out=bad, n_walks=10)
    ro = np.zeros(4)
    ro.flags.writeable = False
    with pytest.raises(TypeError):
        M.mcf_subgraph_centrality(g, [1.0, 1.0, 0.5], out=ro, n_walks=10)
