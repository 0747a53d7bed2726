"""C-ABI contract checks that need no GPU: the library builds, loads, exports
every function declared in include/tpg.h, and rejects malformed input on the
host before any device work."""
import ctypes

import numpy as np
import pytest

from paper_2210_16998_gb300 import cfggen as G
from paper_2210_16998_gb300 import tpg


@pytest.fixture(scope="module")
def lib():
    return tpg.load_library(build=True, install_torch_allocator=False)


def test_exports_every_declared_function(lib):
    names = tpg.declared_functions()
    assert {"tpg_load_cfg", "tpg_prime_paths", "tpg_test_paths", "tpg_free"} <= set(names)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_has_same_names():
    for n in tpg.declared_functions():
        assert hasattr(tpg, n), n


def test_strerror_and_version(lib):
    for code in range(0, -8, -1):
        assert tpg.tpg_strerror(code)
    assert "sm_103a" in tpg.tpg_version()


def _load(n, rp, col, entry, exit):
    lib = tpg.load_library(install_torch_allocator=False)
    h = ctypes.c_void_p()
    rp = np.ascontiguousarray(rp, dtype=np.int32)
    col = np.ascontiguousarray(col if len(col) else [0], dtype=np.int32)
    rc = lib.tpg_load_cfg(n, rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                          col.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), entry, exit, ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("case", [
    "n0", "rp0", "rp_decreasing", "col_range", "col_negative", "duplicate_arc", "unsorted",
    "entry_range", "exit_range", "entry_eq_exit", "indeg_entry", "outdeg_exit",
])
def test_load_rejects_malformed(lib, case):
    rp, col = G.csr_from_arcs(4, [(0, 1), (1, 2), (2, 3)])
    rp, col = rp.copy(), col.copy()
    n, entry, exit = 4, 0, 3
    if case == "n0":
        n = 0
    elif case == "rp0":
        rp[0] = 1
    elif case == "rp_decreasing":
        rp[2] = 0
    elif case == "col_range":
        col[1] = 7
    elif case == "col_negative":
        col[1] = -1
    elif case == "duplicate_arc":
        rp, col = np.array([0, 1, 3, 4, 4], np.int32), np.array([1, 2, 2, 3], np.int32)
    elif case == "unsorted":
        rp, col = np.array([0, 1, 3, 4, 4], np.int32), np.array([1, 3, 2, 3], np.int32)
    elif case == "entry_range":
        entry = 9
    elif case == "exit_range":
        exit = -2
    elif case == "entry_eq_exit":
        exit = 0
    elif case == "indeg_entry":
        rp, col = G.csr_from_arcs(4, [(0, 1), (1, 0), (1, 2), (2, 3)])
    elif case == "outdeg_exit":
        rp, col = G.csr_from_arcs(4, [(0, 1), (1, 2), (2, 3), (3, 1)])
    rc, h = _load(n, rp, col, entry, exit)
    assert rc == tpg.TPG_EINVAL
    assert not h.value


def test_load_rejects_too_big(lib):
    n = tpg.TPG_MAX_N + 1
    rp, col = G.csr_from_arcs(n, [(i, i + 1) for i in range(n - 1)])
    rc, h = _load(n, rp, col, 0, n - 1)
    assert rc == tpg.TPG_ETOOBIG and not h.value


def test_null_handles(lib):
    out = ctypes.POINTER(tpg._Paths)()
    assert lib.tpg_prime_paths(None, ctypes.byref(out)) == tpg.TPG_EHANDLE
    assert lib.tpg_test_paths(None, ctypes.byref(out)) == tpg.TPG_EHANDLE
    assert lib.tpg_set_result_location(None, 0) == tpg.TPG_EHANDLE
    assert lib.tpg_get_stats(None, ctypes.byref(tpg._Stats())) == tpg.TPG_EHANDLE
    assert lib.tpg_set_tile_shape(None, 512, 1) == tpg.TPG_EHANDLE
    assert lib.tpg_set_work_split(None, 2) == tpg.TPG_EHANDLE
    assert lib.tpg_set_wait_limit(None, 1000) == tpg.TPG_EHANDLE
    assert lib.tpg_set_level_trace(None, 1) == tpg.TPG_EHANDLE
    n = ctypes.c_int32(0)
    assert lib.tpg_get_level_trace(None, (ctypes.c_int64 * 4)(), 1, ctypes.byref(n)) == tpg.TPG_EHANDLE
    lib.tpg_free(None)  # no-op


def test_batch_load_rejects_bad_graph(lib):
    cfgs = [G.diamond_chain(2), G.diamond_chain(3)]
    ns, rp, col, ent, ext = G.concat_batch(cfgs)
    ext = ext.copy()
    ext[1] = ent[1]
    lib_ = tpg.load_library(install_torch_allocator=False)
    h = ctypes.c_void_p()

    def p(a):
        return np.ascontiguousarray(a, np.int32).ctypes.data_as(ctypes.POINTER(ctypes.c_int32))

    arrs = [np.ascontiguousarray(a, np.int32) for a in (ns, rp, col, ent, ext)]
    rc = lib_.tpg_load_cfg_batch(2, *[a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) for a in arrs],
                                 ctypes.byref(h))
    assert rc == tpg.TPG_EINVAL and not h.value


def test_struct_layouts_match_header(tmp_path):
    """The binding's ctypes structures have the header's field offsets and
    sizes (compiled with the system C compiler against include/tpg.h)."""
    import subprocess

    structs = {"tpg_paths": tpg._Paths, "tpg_stats": tpg._Stats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "tpg.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    from paper_2210_16998_gb300 import build as B

    subprocess.check_call(["gcc", "-I", B.INCLUDE, "-o", str(exe), str(src)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    got = {}
    for line in out:
        if line:
            s, f, v = line.split()
            got[(s, f)] = int(v)
    for cname, cls in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
    # the first six fields of tpg_paths keep the order of the boundary's
    # definition: magic, num_graphs, num_paths, graph_path_ptr, offsets, vertices
    order = sorted(("magic", "num_graphs", "num_paths", "graph_path_ptr", "offsets", "vertices",
                    "num_vertices", "location", "reserved"), key=lambda f: got[("tpg_paths", f)])
    assert order[:6] == ["magic", "num_graphs", "num_paths", "graph_path_ptr", "offsets", "vertices"]
