"""CPU oracle for prime paths and test paths.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package;
the CUDA library never does, and the oracle never imports the library.

``tpg_oracle.c`` is a plain single-threaded enumeration written from the
paper's definitions (Sec. 2 simple path, Def. 1 prime path, Problem 1 output)
and is compiled here with the system C compiler.  Its root-parallel driver
(``run_parallel``) runs the same enumeration root by root on every host core
for the all-core CPU baseline.  ``literal.py`` is a second,
quadratic oracle for tiny graphs that applies the definitions word for word.
``orc_test_paths_greedy`` (``run(..., greedy=True)``) is the longest-first
touring of Sec. 7.3: a smaller TP set.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tpg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK, ORC_EINVAL, ORC_EUNREACH, ORC_ELIMIT, ORC_ENOMEM = 0, -1, -2, -3, -4


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with code {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc -O2, portable flags) and return the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                           "-o", tmp, _SRC])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.orc_prime_paths.restype = P
        lib.orc_prime_paths.argtypes = [ctypes.c_int, i32p, i32p, ctypes.c_int, ctypes.c_int64]
        lib.orc_run_parallel.restype = P
        lib.orc_run_parallel.argtypes = [ctypes.c_int, i32p, i32p, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.orc_test_paths.restype = ctypes.c_int
        lib.orc_test_paths.argtypes = [P, i32p, i32p, ctypes.c_int, ctypes.c_int]
        lib.orc_test_paths_greedy.restype = ctypes.c_int
        lib.orc_test_paths_greedy.argtypes = [P, i32p, i32p, ctypes.c_int, ctypes.c_int]
        lib.orc_bfs_tables.restype = ctypes.c_int
        lib.orc_bfs_tables.argtypes = [ctypes.c_int, i32p, i32p, i32p, i32p]
        for name in ("orc_n_simple", "orc_pp_count", "orc_pp_total",
                     "orc_tp_count", "orc_tp_total", "orc_gtp_count", "orc_gtp_total"):
            getattr(lib, name).restype = ctypes.c_int64
            getattr(lib, name).argtypes = [P]
        for name in ("orc_pp_offsets", "orc_tp_offsets", "orc_gtp_offsets", "orc_len_counts",
                     "orc_pp_len_counts", "orc_root_paths", "orc_root_pp_ints", "orc_root_pps"):
            getattr(lib, name).restype = ctypes.POINTER(ctypes.c_int64)
            getattr(lib, name).argtypes = [P]
        for name in ("orc_pp_vertices", "orc_tp_vertices", "orc_gtp_vertices"):
            getattr(lib, name).restype = ctypes.POINTER(ctypes.c_int32)
            getattr(lib, name).argtypes = [P]
        lib.orc_error.restype = ctypes.c_int
        lib.orc_error.argtypes = [P]
        lib.orc_free.restype = None
        lib.orc_free.argtypes = [P]
        _lib = lib
        return lib


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _copy(ptr, count, dtype):
    if count == 0:
        return np.zeros(0, dtype=dtype)
    return np.ctypeslib.as_array(ptr, shape=(count,)).astype(dtype, copy=True)


@dataclass
class OracleResult:
    n: int
    n_simple: int
    len_counts: np.ndarray      # simple paths by vertex count, index 0..n+1
    pp_len_counts: np.ndarray   # PPs by vertex count
    root_paths: np.ndarray      # simple paths per first vertex
    root_pp_ints: np.ndarray    # PP vertices per first vertex
    root_pps: np.ndarray        # PPs per first vertex
    pp_offsets: np.ndarray | None = None
    pp_vertices: np.ndarray | None = None
    tp_offsets: np.ndarray | None = None
    tp_vertices: np.ndarray | None = None
    gtp_offsets: np.ndarray | None = None   # longest-first touring
    gtp_vertices: np.ndarray | None = None

    @property
    def num_pp(self) -> int:
        return int(self.pp_len_counts.sum())

    def pp_list(self):
        o, v = self.pp_offsets, self.pp_vertices
        return [tuple(int(x) for x in v[o[i]:o[i + 1]]) for i in range(len(o) - 1)]

    def tp_list(self):
        o, v = self.tp_offsets, self.tp_vertices
        return [tuple(int(x) for x in v[o[i]:o[i + 1]]) for i in range(len(o) - 1)]

    def gtp_list(self):
        o, v = self.gtp_offsets, self.gtp_vertices
        return [tuple(int(x) for x in v[o[i]:o[i + 1]]) for i in range(len(o) - 1)]


def run(n, row_ptr, col, entry=None, exit=None, want_paths=True, limit=0,
        test_paths=False, greedy=False) -> OracleResult:
    """Run the oracle on one graph (int32 CSR, ascending adjacency).  With
    `greedy`, also the longest-first touring TP set (gtp_*)."""
    lib = _load()
    rp, rpp = _i32(row_ptr)
    cl, clp = _i32(col if len(col) else np.zeros(1, np.int32))
    paths = want_paths or test_paths or greedy
    h = lib.orc_prime_paths(int(n), rpp, clp, 1 if paths else 0, int(limit))
    if not h:
        raise OracleError(ORC_ENOMEM, "prime_paths")
    try:
        res = _result(lib, h, n, paths)
        if test_paths:
            rc = lib.orc_test_paths(h, rpp, clp, int(entry), int(exit))
            if rc:
                raise OracleError(rc, "test_paths")
            _take_tps(lib, h, res)
        if greedy:
            rc = lib.orc_test_paths_greedy(h, rpp, clp, int(entry), int(exit))
            if rc:
                raise OracleError(rc, "test_paths_greedy")
            cnt = int(lib.orc_gtp_count(h))
            res.gtp_offsets = _copy(lib.orc_gtp_offsets(h), cnt + 1, np.int64)
            res.gtp_vertices = _copy(lib.orc_gtp_vertices(h), int(lib.orc_gtp_total(h)), np.int32)
        return res
    finally:
        lib.orc_free(h)


def run_parallel(n, row_ptr, col, entry=None, exit=None, want_paths=True, test_paths=False,
                 threads=None) -> OracleResult:
    """The same result as run(), computed by the root-parallel driver on
    `threads` host threads (default: every core)."""
    lib = _load()
    threads = int(threads or os.cpu_count() or 1)
    rp, rpp = _i32(row_ptr)
    cl, clp = _i32(col if len(col) else np.zeros(1, np.int32))
    h = lib.orc_run_parallel(int(n), rpp, clp, int(entry if entry is not None else -1),
                             int(exit if exit is not None else -1), 1 if want_paths else 0,
                             1 if test_paths else 0, threads)
    if not h:
        raise OracleError(ORC_ENOMEM, "run_parallel")
    try:
        res = _result(lib, h, n, want_paths or test_paths)
        if test_paths:
            _take_tps(lib, h, res)
        return res
    finally:
        lib.orc_free(h)


def run_cfg_parallel(cfg, test_paths=True, want_paths=True, threads=None) -> OracleResult:
    return run_parallel(cfg.n, cfg.row_ptr, cfg.col, cfg.entry, cfg.exit, want_paths=want_paths,
                        test_paths=test_paths, threads=threads)


def _take_tps(lib, h, res):
    cnt = int(lib.orc_tp_count(h))
    res.tp_offsets = _copy(lib.orc_tp_offsets(h), cnt + 1, np.int64)
    res.tp_vertices = _copy(lib.orc_tp_vertices(h), int(lib.orc_tp_total(h)), np.int32)


def _result(lib, h, n, with_paths):
    err = lib.orc_error(h)
    if err:
        raise OracleError(err, "prime_paths")
    res = OracleResult(
        n=int(n),
        n_simple=int(lib.orc_n_simple(h)),
        len_counts=_copy(lib.orc_len_counts(h), n + 3, np.int64),
        pp_len_counts=_copy(lib.orc_pp_len_counts(h), n + 3, np.int64),
        root_paths=_copy(lib.orc_root_paths(h), n, np.int64),
        root_pp_ints=_copy(lib.orc_root_pp_ints(h), n, np.int64),
        root_pps=_copy(lib.orc_root_pps(h), n, np.int64),
    )
    if with_paths:
        cnt = int(lib.orc_pp_count(h))
        res.pp_offsets = _copy(lib.orc_pp_offsets(h), cnt + 1, np.int64)
        res.pp_vertices = _copy(lib.orc_pp_vertices(h), int(lib.orc_pp_total(h)), np.int32)
    return res


def run_cfg(cfg, test_paths=True, want_paths=True, limit=0, greedy=False) -> OracleResult:
    return run(cfg.n, cfg.row_ptr, cfg.col, cfg.entry, cfg.exit,
               want_paths=want_paths, limit=limit, test_paths=test_paths, greedy=greedy)


def bfs_tables(n, row_ptr, col):
    """All-pairs BFS distance and lowest-id predecessor tables (int32 n x n)."""
    lib = _load()
    rp, rpp = _i32(row_ptr)
    cl, clp = _i32(col if len(col) else np.zeros(1, np.int32))
    dist = np.empty(n * n, np.int32)
    pred = np.empty(n * n, np.int32)
    rc = lib.orc_bfs_tables(int(n), rpp, clp,
                            dist.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                            pred.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if rc:
        raise OracleError(rc, "bfs_tables")
    return dist.reshape(n, n), pred.reshape(n, n)
