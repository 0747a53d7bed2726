"""Python binding of libtpg (ctypes; argument marshalling only).

Every function of ``include/tpg.h`` has a Python function of the same name.
All path computation happens in the CUDA kernels of ``libtpg.so``; this
module only converts arrays to pointers and results to numpy arrays (host
results) or zero-copy torch tensors (device results).  PyTorch supplies the
device memory (its caching allocator is installed as the library allocator)
and the CUDA stream (the current torch stream at load time).

There is no CPU fallback: if the library is not built, or no GPU is present,
the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

from . import build as _build

TPG_OK = 0
TPG_EINVAL = -1
TPG_EUNREACH = -2
TPG_ETOOBIG = -3
TPG_ENOMEM = -4
TPG_ECUDA = -5
TPG_ETIMEOUT = -6
TPG_EHANDLE = -7
TPG_RESULT_HOST = 0
TPG_RESULT_DEVICE = 1
TPG_MAX_N = 4096

HEADER = os.path.join(_build.INCLUDE, "tpg.h")


class TPGError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib_strerror(code)
        super().__init__(f"{where}: {msg} ({code})")
        self.code = code


class _Paths(ctypes.Structure):
    _fields_ = [
        ("magic", ctypes.c_uint32),
        ("num_graphs", ctypes.c_int32),
        ("num_paths", ctypes.c_int64),
        ("graph_path_ptr", ctypes.c_void_p),
        ("offsets", ctypes.c_void_p),
        ("vertices", ctypes.c_void_p),
        ("num_vertices", ctypes.c_int64),
        ("location", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class _Stats(ctypes.Structure):
    _fields_ = [
        ("simple_paths", ctypes.c_int64),
        ("prime_paths", ctypes.c_int64),
        ("pp_vertices", ctypes.c_int64),
        ("levels", ctypes.c_int32),
        ("pp_levels", ctypes.c_int32),
        ("peak_level_nodes", ctypes.c_int64),
        ("arena_bytes_used", ctypes.c_int64),
        ("arena_bytes_alloc", ctypes.c_int64),
        ("frontier_bytes_alloc", ctypes.c_int64),
        ("attempts", ctypes.c_int32),
        ("bitset_words", ctypes.c_int32),
        ("test_paths", ctypes.c_int64),
        ("tp_vertices", ctypes.c_int64),
        ("t_enumerate_ms", ctypes.c_float),
        ("t_order_ms", ctypes.c_float),
        ("t_test_paths_ms", ctypes.c_float),
        ("enumerate_grid", ctypes.c_int32),
        ("tile_block", ctypes.c_int32),
        ("tile_items", ctypes.c_int32),
        ("t_graph_ms", ctypes.c_float),
        ("graph_launches", ctypes.c_int32),
        ("graph_fallbacks", ctypes.c_int32),
        ("graph_flags", ctypes.c_int32),
        ("graph_enum_error", ctypes.c_int32),
        ("t_result_copy_ms", ctypes.c_float),
        ("result_copy_bytes", ctypes.c_int64),
        ("t_touring_ms", ctypes.c_float),
        ("touring_sweeps", ctypes.c_int32),
        ("touring_test_paths", ctypes.c_int64),
        ("touring_edges", ctypes.c_int64),
        ("t_pervertex_ms", ctypes.c_float),
        ("pervertex_paths", ctypes.c_int64),
        ("pervertex_bytes", ctypes.c_int64),
        ("t_scc_ms", ctypes.c_float),
        ("scc_pps", ctypes.c_int64),
        ("scc_internal_pps", ctypes.c_int64),
        ("t_compositional_ms", ctypes.c_float),
        ("comp_entry_exit_paths", ctypes.c_int64),
        ("comp_exit_paths", ctypes.c_int64),
        ("comp_entry_paths", ctypes.c_int64),
        ("comp_crossing_pps", ctypes.c_int64),
    ]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

_lock = threading.Lock()
_lib = None
_callbacks = None


def declared_functions():
    """Names of the functions declared in include/tpg.h."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tpg_[a-z_0-9]+)\s*\(", text)) - {"tpg_alloc_fn", "tpg_release_fn"})


def library_path(build: bool = False) -> str:
    if build:
        return _build.build()
    return _build.LIB


def load_library(path: str | None = None, build: bool = False, install_torch_allocator: bool = True):
    """Load libtpg.so (building it first if asked) and declare the signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or library_path(build)
        if not os.path.exists(path):
            raise RuntimeError(f"libtpg.so is not built ({path}); call __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        i32p = ctypes.POINTER(ctypes.c_int32)
        P = ctypes.c_void_p
        lib.tpg_load_cfg.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(P)]
        lib.tpg_load_cfg_device.argtypes = [ctypes.c_int32, ctypes.c_int32, P, P, ctypes.c_int32, ctypes.c_int32,
                                            P, ctypes.POINTER(P)]
        lib.tpg_load_cfg_batch.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, i32p, ctypes.POINTER(P)]
        lib.tpg_prime_paths.argtypes = [P, ctypes.POINTER(ctypes.POINTER(_Paths))]
        lib.tpg_test_paths.argtypes = [P, ctypes.POINTER(ctypes.POINTER(_Paths))]
        lib.tpg_test_paths_greedy.argtypes = [P, ctypes.POINTER(ctypes.POINTER(_Paths))]
        lib.tpg_prime_paths_pervertex.argtypes = [P, ctypes.POINTER(ctypes.POINTER(_Paths))]
        lib.tpg_scc_internal_pps.argtypes = [P, ctypes.POINTER(ctypes.POINTER(_Paths))]
        lib.tpg_scc_ids.argtypes = [P, ctypes.POINTER(ctypes.c_int32)]
        lib.tpg_prime_paths_compositional.argtypes = [P, ctypes.POINTER(ctypes.POINTER(_Paths))]
        lib.tpg_free.argtypes = [P]
        lib.tpg_free.restype = None
        lib.tpg_set_stream.argtypes = [P, P]
        lib.tpg_set_result_location.argtypes = [P, ctypes.c_int32]
        lib.tpg_set_tile_shape.argtypes = [P, ctypes.c_int32, ctypes.c_int32]
        lib.tpg_set_work_split.argtypes = [P, ctypes.c_int32]
        lib.tpg_set_capacity.argtypes = [P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]
        lib.tpg_set_wait_limit.argtypes = [P, ctypes.c_int64]
        lib.tpg_set_level_trace.argtypes = [P, ctypes.c_int32]
        lib.tpg_get_level_trace.argtypes = [P, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32,
                                            ctypes.POINTER(ctypes.c_int32)]
        lib.tpg_set_output_capacity.argtypes = [P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]
        lib.tpg_graph_capture.argtypes = [P]
        lib.tpg_root_counts.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
        lib.tpg_root_counts.restype = ctypes.c_int
        fp = ctypes.POINTER(ctypes.c_float)
        i64p = ctypes.POINTER(ctypes.c_int64)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.tpg_sizer_num_params.restype = ctypes.c_int
        lib.tpg_sizer_create.argtypes = [ctypes.c_uint64, ctypes.POINTER(P)]
        lib.tpg_sizer_add_batch.argtypes = [P, P, i64p]
        lib.tpg_sizer_train.argtypes = [P, ctypes.c_int32, ctypes.c_float, fp]
        lib.tpg_sizer_predict.argtypes = [P, P, fp, dp]
        lib.tpg_sizer_presize.argtypes = [P, P, ctypes.c_double, i64p]
        lib.tpg_sizer_features.argtypes = [P, fp]
        lib.tpg_sizer_get_params.argtypes = [P, fp]
        lib.tpg_sizer_set_params.argtypes = [P, fp]
        lib.tpg_sizer_loss_grad.argtypes = [P, ctypes.c_int32, dp, fp]
        lib.tpg_sizer_batch_targets.argtypes = [P, ctypes.c_int32, fp]
        lib.tpg_sizer_save.argtypes = [P, ctypes.c_char_p]
        lib.tpg_sizer_load.argtypes = [P, ctypes.c_char_p]
        for name in ("tpg_sizer_create", "tpg_sizer_add_batch", "tpg_sizer_train", "tpg_sizer_predict",
                     "tpg_sizer_presize", "tpg_sizer_features", "tpg_sizer_get_params", "tpg_sizer_set_params",
                     "tpg_sizer_loss_grad", "tpg_sizer_batch_targets", "tpg_sizer_save", "tpg_sizer_load"):
            getattr(lib, name).restype = ctypes.c_int
        lib.tpg_graph_launch.argtypes = [P, ctypes.POINTER(ctypes.POINTER(_Paths)),
                                         ctypes.POINTER(ctypes.POINTER(_Paths))]
        lib.tpg_set_allocator.argtypes = [_ALLOC_FN, _RELEASE_FN, P]
        lib.tpg_get_stats.argtypes = [P, ctypes.POINTER(_Stats)]
        lib.tpg_strerror.argtypes = [ctypes.c_int]
        lib.tpg_strerror.restype = ctypes.c_char_p
        lib.tpg_version.restype = ctypes.c_char_p
        lib.tpg_kernel_launches.restype = ctypes.c_int64
        lib.tpg_prime_paths_noalloc.argtypes = [ctypes.c_int32, ctypes.c_int32, P, P, P, ctypes.c_int64, P,
                                                ctypes.c_int64, P, ctypes.POINTER(ctypes.c_int64),
                                                ctypes.POINTER(ctypes.c_int64)]
        lib.tpg_prime_paths_noalloc.restype = ctypes.c_int
        for name in ("tpg_load_cfg", "tpg_load_cfg_device", "tpg_load_cfg_batch", "tpg_prime_paths",
                     "tpg_test_paths", "tpg_test_paths_greedy", "tpg_prime_paths_pervertex", "tpg_scc_ids",
                     "tpg_scc_internal_pps", "tpg_prime_paths_compositional", "tpg_set_stream",
                     "tpg_set_result_location",
                     "tpg_set_allocator",
                     "tpg_get_stats", "tpg_set_tile_shape", "tpg_set_work_split", "tpg_set_capacity",
                     "tpg_set_output_capacity",
                     "tpg_graph_capture", "tpg_graph_launch"):
            getattr(lib, name).restype = ctypes.c_int
        lib.tpg_release_cached_memory.argtypes = []
        lib.tpg_release_cached_memory.restype = ctypes.c_int
        _lib = lib
    if install_torch_allocator:
        _install_torch_allocator()
    return _lib


def _install_torch_allocator():
    """Route the library's device allocations through torch's caching allocator."""
    global _callbacks
    import torch

    if not torch.cuda.is_available():
        return

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:  # out of memory -> the library returns TPG_ENOMEM
            return None

    def _release(ptr, stream, ctx):
        if ptr:
            torch.cuda.caching_allocator_delete(int(ptr))

    cb = (_ALLOC_FN(_alloc), _RELEASE_FN(_release))
    rc = _lib.tpg_set_allocator(cb[0], cb[1], None)
    if rc != TPG_OK:
        raise TPGError(rc, "tpg_set_allocator")
    _callbacks = cb


def _lib_strerror(code: int) -> str:
    if _lib is None:
        return f"error {code}"
    return _lib.tpg_strerror(code).decode()


def tpg_strerror(code: int) -> str:
    return load_library().tpg_strerror(int(code)).decode()


def tpg_version() -> str:
    return load_library().tpg_version().decode()


def _check(rc: int, where: str):
    if rc != TPG_OK:
        raise TPGError(rc, where)


def _i32(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int32))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


class Cfg:
    """A loaded graph (or batch of graphs): owns a tpg_cfg*."""

    def __init__(self, handle: int, num_graphs: int):
        self.handle = ctypes.c_void_p(handle)
        self.num_graphs = num_graphs

    def close(self):
        if self.handle:
            load_library().tpg_free(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class _CudaArray:
    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (ptr, False), "version": 3,
                                         "strides": None}


class Paths:
    """A path list returned by the library (owns a tpg_paths*)."""

    def __init__(self, ptr):
        self._ptr = ptr
        p = ptr.contents
        self.num_graphs = int(p.num_graphs)
        self.num_paths = int(p.num_paths)
        self.num_vertices = int(p.num_vertices)
        self.location = int(p.location)
        self._raw = (p.graph_path_ptr, p.offsets, p.vertices)
        self._arrays = None  # built on first access (views of the library's buffers)

    def _views(self):
        if self._arrays is None:
            if self._ptr is None:
                raise ValueError("path list already freed")
            gp_ptr, off_ptr, v_ptr = self._raw
            nv = self.num_vertices
            if self.location == TPG_RESULT_HOST:
                gp = np.ctypeslib.as_array(ctypes.cast(gp_ptr, ctypes.POINTER(ctypes.c_int64)),
                                           shape=(self.num_graphs + 1,))
                off = np.ctypeslib.as_array(ctypes.cast(off_ptr, ctypes.POINTER(ctypes.c_int64)),
                                            shape=(self.num_paths + 1,))
                vert = (np.ctypeslib.as_array(ctypes.cast(v_ptr, ctypes.POINTER(ctypes.c_int32)), shape=(nv,))
                        if nv else np.zeros(0, np.int32))
            else:
                import torch

                gp = torch.as_tensor(_CudaArray(gp_ptr, (self.num_graphs + 1,), "<i8"), device="cuda")
                off = torch.as_tensor(_CudaArray(off_ptr, (self.num_paths + 1,), "<i8"), device="cuda")
                vert = (torch.as_tensor(_CudaArray(v_ptr, (nv,), "<i4"), device="cuda")
                        if nv else torch.zeros(0, dtype=torch.int32, device="cuda"))
            self._arrays = (gp, off, vert)
        return self._arrays

    @property
    def graph_path_ptr(self):
        """[num_graphs + 1] int64: paths of graph g are [ptr[g], ptr[g+1])."""
        return self._views()[0]

    @property
    def offsets(self):
        """[num_paths + 1] int64."""
        return self._views()[1]

    @property
    def vertices(self):
        """[num_vertices] int32, graph-local vertex ids."""
        return self._views()[2]

    def host_arrays(self):
        """(graph_path_ptr, offsets, vertices) as numpy copies."""
        if self.location == TPG_RESULT_HOST:
            return self.graph_path_ptr.copy(), self.offsets.copy(), self.vertices.copy()
        return (self.graph_path_ptr.cpu().numpy(), self.offsets.cpu().numpy(), self.vertices.cpu().numpy())

    def to_lists(self, graph: int | None = None):
        gp, off, v = self.host_arrays()
        lo, hi = (0, self.num_paths) if graph is None else (int(gp[graph]), int(gp[graph + 1]))
        return [tuple(int(x) for x in v[off[i]:off[i + 1]]) for i in range(lo, hi)]

    def free(self):
        if self._ptr is not None:
            # drop views first: they alias library memory
            self._arrays = None
            load_library().tpg_free(ctypes.cast(self._ptr, ctypes.c_void_p))
            self._ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()


def _current_stream():
    import torch

    if torch.cuda.is_available():
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(0)


def tpg_load_cfg(n, row_ptr, col, entry, exit, location=TPG_RESULT_HOST) -> Cfg:
    lib = load_library()
    rp, rpp = _i32(row_ptr)
    cl, clp = _i32(col if len(col) else np.zeros(1, np.int32))
    h = ctypes.c_void_p()
    _check(lib.tpg_load_cfg(int(n), rpp, clp, int(entry), int(exit), ctypes.byref(h)), "tpg_load_cfg")
    cfg = Cfg(h.value, 1)
    tpg_set_stream(cfg, _current_stream())
    tpg_set_result_location(cfg, location)
    return cfg


def tpg_load_cfg_device(n, m, row_ptr_dev, col_dev, entry, exit, stream=None, location=TPG_RESULT_DEVICE) -> Cfg:
    """row_ptr_dev / col_dev: int32 CUDA tensors (or raw device addresses)."""
    lib = load_library()

    def addr(t):
        return ctypes.c_void_p(t if isinstance(t, int) else t.data_ptr())

    s = _current_stream() if stream is None else ctypes.c_void_p(stream)
    h = ctypes.c_void_p()
    _check(lib.tpg_load_cfg_device(int(n), int(m), addr(row_ptr_dev), addr(col_dev), int(entry), int(exit), s,
                                   ctypes.byref(h)), "tpg_load_cfg_device")
    cfg = Cfg(h.value, 1)
    tpg_set_result_location(cfg, location)
    return cfg


def tpg_load_cfg_batch(n_per_graph, row_ptr_cat, col_cat, entries, exits, location=TPG_RESULT_HOST) -> Cfg:
    lib = load_library()
    ns, nsp = _i32(n_per_graph)
    rp, rpp = _i32(row_ptr_cat)
    cl, clp = _i32(col_cat if len(col_cat) else np.zeros(1, np.int32))
    en, enp = _i32(entries)
    ex, exp = _i32(exits)
    h = ctypes.c_void_p()
    _check(lib.tpg_load_cfg_batch(len(ns), nsp, rpp, clp, enp, exp, ctypes.byref(h)), "tpg_load_cfg_batch")
    cfg = Cfg(h.value, len(ns))
    tpg_set_stream(cfg, _current_stream())
    tpg_set_result_location(cfg, location)
    return cfg


def tpg_prime_paths(cfg: Cfg) -> Paths:
    out = ctypes.POINTER(_Paths)()
    _check(load_library().tpg_prime_paths(cfg.handle, ctypes.byref(out)), "tpg_prime_paths")
    return Paths(out)


def tpg_test_paths(cfg: Cfg) -> Paths:
    out = ctypes.POINTER(_Paths)()
    _check(load_library().tpg_test_paths(cfg.handle, ctypes.byref(out)), "tpg_test_paths")
    return Paths(out)


def tpg_test_paths_greedy(cfg: Cfg) -> Paths:
    """The longest-first touring TP set (a subset of tpg_test_paths's list)."""
    out = ctypes.POINTER(_Paths)()
    _check(load_library().tpg_test_paths_greedy(cfg.handle, ctypes.byref(out)), "tpg_test_paths_greedy")
    return Paths(out)


def tpg_prime_paths_pervertex(cfg: Cfg) -> Paths:
    """The paper-style per-vertex-list baseline: the PPs grouped by end vertex
    (num_graphs = n)."""
    out = ctypes.POINTER(_Paths)()
    _check(load_library().tpg_prime_paths_pervertex(cfg.handle, ctypes.byref(out)), "tpg_prime_paths_pervertex")
    return Paths(out)


def tpg_scc_ids(cfg: Cfg, n: int) -> np.ndarray:
    """SCC of each of the graph's n vertices, named by its smallest member."""
    out = np.empty(int(n), np.int32)
    _check(load_library().tpg_scc_ids(cfg.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), "tpg_scc_ids")
    return out


def tpg_scc_internal_pps(cfg: Cfg) -> Paths:
    """The SccInternalPPs of every SCC (Def. 9), canonical order."""
    out = ctypes.POINTER(_Paths)()
    _check(load_library().tpg_scc_internal_pps(cfg.handle, ctypes.byref(out)), "tpg_scc_internal_pps")
    return Paths(out)


def tpg_prime_paths_compositional(cfg: Cfg) -> Paths:
    """The PPs by the SCC-compositional route (same list as tpg_prime_paths)."""
    out = ctypes.POINTER(_Paths)()
    _check(load_library().tpg_prime_paths_compositional(cfg.handle, ctypes.byref(out)),
           "tpg_prime_paths_compositional")
    return Paths(out)


def tpg_free(obj):
    if isinstance(obj, (Cfg, Sizer)):
        obj.close()
    elif isinstance(obj, Paths):
        obj.free()


def tpg_set_stream(cfg: Cfg, stream):
    s = stream if isinstance(stream, ctypes.c_void_p) else ctypes.c_void_p(stream)
    _check(load_library().tpg_set_stream(cfg.handle, s), "tpg_set_stream")


def tpg_set_result_location(cfg: Cfg, location: int):
    _check(load_library().tpg_set_result_location(cfg.handle, int(location)), "tpg_set_result_location")


def tpg_release_cached_memory():
    """Hand the device blocks the library keeps for reuse back to their allocator."""
    _check(load_library().tpg_release_cached_memory(), "tpg_release_cached_memory")


def tpg_set_tile_shape(cfg: Cfg, block: int, items: int):
    _check(load_library().tpg_set_tile_shape(cfg.handle, int(block), int(items)), "tpg_set_tile_shape")


def tpg_set_work_split(cfg: Cfg, split: int):
    _check(load_library().tpg_set_work_split(cfg.handle, int(split)), "tpg_set_work_split")


def set_tile(cfg: Cfg, tile):
    """Apply a tuned tile: (block, items) or (block, items, split)."""
    tpg_set_tile_shape(cfg, int(tile[0]), int(tile[1]))
    tpg_set_work_split(cfg, int(tile[2]) if len(tile) > 2 else 1)


def tpg_set_wait_limit(cfg: Cfg, ns: int):
    """Limit of each grid-barrier wait of the handle's frontier launches (ns < 0: default)."""
    _check(load_library().tpg_set_wait_limit(cfg.handle, int(ns)), "tpg_set_wait_limit")


def tpg_set_level_trace(cfg: Cfg, on: bool = True):
    """Record a per-level trace of the frontier launch on later tpg_prime_paths calls."""
    _check(load_library().tpg_set_level_trace(cfg.handle, 1 if on else 0), "tpg_set_level_trace")


def tpg_get_level_trace(cfg: Cfg, max_levels: int = 4200):
    """The last call's trace: int64 [levels, 4] = (start ns, last warp end ns,
    summed warp busy ns, warps with work) per level, level 1 in row 1."""
    out = np.zeros((max_levels, 4), dtype=np.int64)
    used = ctypes.c_int32(0)
    _check(load_library().tpg_get_level_trace(cfg.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                              int(max_levels), ctypes.byref(used)), "tpg_get_level_trace")
    return out[:used.value]


def tpg_set_capacity(cfg: Cfg, nodes: int, level_nodes: int, prime_paths: int):
    _check(load_library().tpg_set_capacity(cfg.handle, int(nodes), int(level_nodes), int(prime_paths)),
           "tpg_set_capacity")


def tpg_set_output_capacity(cfg: Cfg, prime_paths: int, pp_vertices: int, tp_vertices_raw: int, tp_vertices: int):
    _check(load_library().tpg_set_output_capacity(cfg.handle, int(prime_paths), int(pp_vertices),
                                                  int(tp_vertices_raw), int(tp_vertices)), "tpg_set_output_capacity")


def tpg_root_counts(cfg: Cfg, num_vertices: int):
    """Per first vertex: (simple paths, prime paths, prime-path vertices), int64 [N, 3]."""
    out = np.zeros((num_vertices, 3), dtype=np.int64)
    _check(load_library().tpg_root_counts(cfg.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))),
           "tpg_root_counts")
    return out


def tpg_graph_capture(cfg: Cfg):
    _check(load_library().tpg_graph_capture(cfg.handle), "tpg_graph_capture")


def tpg_graph_launch(cfg: Cfg):
    """Replay the captured hot path; returns (prime paths, test paths)."""
    pp = ctypes.POINTER(_Paths)()
    tp = ctypes.POINTER(_Paths)()
    _check(load_library().tpg_graph_launch(cfg.handle, ctypes.byref(pp), ctypes.byref(tp)), "tpg_graph_launch")
    return Paths(pp), Paths(tp)


def tpg_set_allocator(alloc=None, release=None):
    """Install Python callables alloc(nbytes, stream) -> ptr / release(ptr, stream), or None for the default."""
    global _callbacks
    lib = load_library(install_torch_allocator=False)
    if alloc is None:
        _check(lib.tpg_set_allocator(_ALLOC_FN(), _RELEASE_FN(), None), "tpg_set_allocator")
        _callbacks = None
        return
    cb = (_ALLOC_FN(lambda n, s, c: alloc(n, s)), _RELEASE_FN(lambda p, s, c: release(p, s)))
    _check(lib.tpg_set_allocator(cb[0], cb[1], None), "tpg_set_allocator")
    _callbacks = cb


def tpg_get_stats(cfg: Cfg, as_dict: bool = True):
    """Statistics of the handle's last calls: a dict, or with as_dict=False
    the raw structure (cheaper; stats_dict() converts it later)."""
    st = _Stats()
    _check(load_library().tpg_get_stats(cfg.handle, ctypes.byref(st)), "tpg_get_stats")
    return stats_dict(st) if as_dict else st


def stats_dict(st) -> dict:
    return {name: (float(getattr(st, name)) if name.startswith("t_") else int(getattr(st, name)))
            for name, _ in _Stats._fields_}


def tpg_prime_paths_noalloc(n, m, row_ptr_dev, col_dev, offsets_dev, vertices_dev, stream=None):
    """Prime paths of one small graph into caller-owned device buffers, with no
    allocation inside the library (for callers that cannot allocate at call
    time: a memory budget fixed in advance, or a host framework that owns
    every allocation).  row_ptr_dev / col_dev / offsets_dev / vertices_dev
    are contiguous CUDA tensors on the current device of dtype int32 [n+1],
    int32 [>= m], int64 [cap_paths+1] and int32 [cap_vertices].  Returns
    (rc, num_paths, num_vertices); rc is TPG_OK or a TPG_E* code (TPG_ETOOBIG
    also when the output buffers are too small, with the sizes needed).
    Arguments of the wrong dtype, device, layout or size give TPG_EINVAL
    without calling the library."""
    import torch

    want = ((row_ptr_dev, torch.int32), (col_dev, torch.int32), (offsets_dev, torch.int64),
            (vertices_dev, torch.int32))
    for t, dt in want:
        if not isinstance(t, torch.Tensor) or t.dtype != dt or not t.is_cuda or not t.is_contiguous():
            return TPG_EINVAL, 0, 0
    dev = torch.cuda.current_device()
    if any(t.device.index != dev for t, _ in want):
        return TPG_EINVAL, 0, 0
    if int(n) < 1 or int(m) < 0 or row_ptr_dev.numel() != int(n) + 1 or col_dev.numel() < int(m) \
            or offsets_dev.numel() < 1:
        return TPG_EINVAL, 0, 0
    lib = load_library()
    npaths, nverts = ctypes.c_int64(0), ctypes.c_int64(0)
    s = _current_stream() if stream is None else ctypes.c_void_p(stream)
    rc = lib.tpg_prime_paths_noalloc(int(n), int(m), ctypes.c_void_p(row_ptr_dev.data_ptr()),
                                     ctypes.c_void_p(col_dev.data_ptr()), ctypes.c_void_p(offsets_dev.data_ptr()),
                                     int(offsets_dev.numel()) - 1, ctypes.c_void_p(vertices_dev.data_ptr()),
                                     int(vertices_dev.numel()), s, ctypes.byref(npaths), ctypes.byref(nverts))
    return int(rc), int(npaths.value), int(nverts.value)


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class Sizer:
    """The learned sizer (owns a tpg_sizer*)."""

    def __init__(self, handle: int):
        self.handle = ctypes.c_void_p(handle)

    def close(self):
        if self.handle:
            load_library().tpg_free(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def tpg_sizer_num_params() -> int:
    return int(load_library().tpg_sizer_num_params())


def tpg_sizer_create(seed: int = 0) -> Sizer:
    h = ctypes.c_void_p()
    _check(load_library().tpg_sizer_create(int(seed), ctypes.byref(h)), "tpg_sizer_create")
    return Sizer(h.value)


def tpg_sizer_add_batch(z: Sizer, cfg: Cfg):
    """Keep (graph, features, exact labels) of a handle; returns its volumes
    (simple paths, peak level, PPs, PP vertices, TP vertices raw, TP vertices)."""
    vol = np.zeros(6, np.int64)
    _check(load_library().tpg_sizer_add_batch(z.handle, cfg.handle, vol.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))),
           "tpg_sizer_add_batch")
    return vol


def tpg_sizer_train(z: Sizer, epochs: int, lr: float):
    losses = np.zeros(max(epochs, 1), np.float32)
    _check(load_library().tpg_sizer_train(z.handle, int(epochs), float(lr), _fptr(losses)), "tpg_sizer_train")
    return losses[:epochs]


def tpg_sizer_predict(z: Sizer, cfg: Cfg, num_vertices: int):
    pred = np.zeros((num_vertices, 3), np.float32)
    tot = np.zeros(3, np.float64)
    _check(load_library().tpg_sizer_predict(z.handle, cfg.handle, _fptr(pred),
                                           tot.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "tpg_sizer_predict")
    return pred, tot


def tpg_sizer_presize(z: Sizer, cfg: Cfg, margin: float):
    caps = np.zeros(7, np.int64)
    _check(load_library().tpg_sizer_presize(z.handle, cfg.handle, float(margin),
                                           caps.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))), "tpg_sizer_presize")
    return caps


def tpg_sizer_features(cfg: Cfg, num_vertices: int):
    x = np.zeros((num_vertices, 8), np.float32)
    _check(load_library().tpg_sizer_features(cfg.handle, _fptr(x)), "tpg_sizer_features")
    return x


def tpg_sizer_get_params(z: Sizer):
    p = np.zeros(tpg_sizer_num_params(), np.float32)
    _check(load_library().tpg_sizer_get_params(z.handle, _fptr(p)), "tpg_sizer_get_params")
    return p


def tpg_sizer_set_params(z: Sizer, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    assert p.size == tpg_sizer_num_params()
    _check(load_library().tpg_sizer_set_params(z.handle, _fptr(p)), "tpg_sizer_set_params")


def tpg_sizer_loss_grad(z: Sizer, batch: int):
    g = np.zeros(tpg_sizer_num_params(), np.float32)
    loss = ctypes.c_double(0.0)
    _check(load_library().tpg_sizer_loss_grad(z.handle, int(batch), ctypes.byref(loss), _fptr(g)),
           "tpg_sizer_loss_grad")
    return float(loss.value), g


def tpg_sizer_batch_targets(z: Sizer, batch: int, num_vertices: int):
    t = np.zeros((num_vertices, 3), np.float32)
    _check(load_library().tpg_sizer_batch_targets(z.handle, int(batch), _fptr(t)), "tpg_sizer_batch_targets")
    return t


def tpg_sizer_save(z: Sizer, path: str):
    _check(load_library().tpg_sizer_save(z.handle, path.encode()), "tpg_sizer_save")


def tpg_sizer_load(z: Sizer, path: str):
    _check(load_library().tpg_sizer_load(z.handle, path.encode()), "tpg_sizer_load")


def tpg_kernel_launches() -> int:
    return int(load_library().tpg_kernel_launches())
