"""Python binding of libgp (include/gp.h): argument marshalling only.

Every function has the name of the C entry point it calls.  All evaluation
and crossover work runs in libgp's CUDA kernels; if libgp.so is missing or
fails to load, every call raises.  Streams may be given as None (legacy
default stream), a raw cudaStream_t integer, or any object with a
`cuda_stream` attribute (e.g. torch.cuda.Stream).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

GP_OK, GP_EINVAL, GP_ENOMEM, GP_EMALFORMED, GP_ECUDA, GP_ETIMEOUT, GP_ELIMIT = range(7)
KERNEL_KINDS = ["eval", "eval_upper", "plan", "scan", "validate", "extent", "copy", "unused"]

EXPORTED = [
    "gp_create_population", "gp_crossover", "gp_evaluate", "gp_evaluate_ex", "gp_fitness",
    "gp_tree_size", "gp_tree_read", "gp_population_get_info", "gp_destroy_population",
    "gp_status_string", "gp_eval_stats_get", "gp_kernel_launch_count", "gp_profile_enable",
    "gp_profile_read", "gp_evaluate_noalloc", "gp_select",
    "gp_generation_create", "gp_generation_step", "gp_generation_rewind", "gp_generation_fitness",
    "gp_generation_records", "gp_generation_trees", "gp_generation_tree_read", "gp_generation_get_info",
    "gp_generation_destroy",
    "gp_generation_recover",
    "gp_server_create", "gp_server_open_run", "gp_server_open_run_from", "gp_server_submit", "gp_server_wait", "gp_server_run_fitness",
    "gp_server_run_trees", "gp_server_close_run", "gp_server_get_stats", "gp_server_destroy",
]
NOALLOC_MAX_TREES = 16384
NOALLOC_MAX_TREE_NODES = 4096


class gp_problem(C.Structure):
    _fields_ = [("n_cases", C.c_uint32), ("x", C.POINTER(C.c_float)), ("y", C.POINTER(C.c_float)),
                ("n_consts", C.c_uint32), ("consts", C.POINTER(C.c_float)),
                ("protected_div_value", C.c_float), ("max_tree_nodes", C.c_uint64),
                ("hbm_budget_bytes", C.c_uint64)]


class gp_xo(C.Structure):
    _fields_ = [("mum", C.c_uint32), ("dad", C.c_uint32), ("mum_point", C.c_uint64),
                ("dad_point", C.c_uint64)]


class gp_eval_options(C.Structure):
    _fields_ = [("chunk_nodes", C.c_uint32), ("warps_per_cta", C.c_uint32),
                ("window_entries", C.c_uint32), ("upper_window_entries", C.c_uint32)]


class gp_population_info(C.Structure):
    _fields_ = [("n_trees", C.c_uint32), ("n_cases", C.c_uint32), ("total_nodes", C.c_uint64),
                ("d_nodes", C.c_void_p), ("d_tree_start", C.c_void_p), ("d_tree_size", C.c_void_p),
                ("d_fitness", C.c_void_p), ("d_case_values", C.c_void_p), ("d_hits", C.c_void_p)]


class gp_eval_stats(C.Structure):
    _fields_ = [("levels", C.c_uint32), ("redone", C.c_uint32), ("items", C.c_uint64),
                ("upper_codes", C.c_uint64), ("value_entries", C.c_uint64), ("upper_ops", C.c_uint64)]


class gp_generation_params(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("tournament_size", C.c_uint32), ("chunk_nodes", C.c_uint32),
                ("arena_bytes", C.c_uint64), ("workspace_codes", C.c_uint64),
                ("workspace_values", C.c_uint64), ("use_graph", C.c_uint32), ("max_levels", C.c_uint32),
                ("warps_per_cta", C.c_uint32), ("window_entries", C.c_uint32),
                ("upper_window_entries", C.c_uint32), ("pad", C.c_uint32)]


class gp_generation_info(C.Structure):
    _fields_ = [("generation", C.c_uint64), ("n_trees", C.c_uint32), ("chunk_nodes", C.c_uint32),
                ("total_nodes", C.c_uint64), ("levels", C.c_uint32), ("graph", C.c_uint32),
                ("kernels_per_generation", C.c_uint32), ("error_generation", C.c_uint32),
                ("arena_bytes", C.c_uint64), ("workspace_codes", C.c_uint64),
                ("workspace_values", C.c_uint64), ("autotune_chunk", C.c_uint32 * 8),
                ("autotune_ms", C.c_float * 8), ("warps_per_cta", C.c_uint32), ("window_entries", C.c_uint32),
                ("upper_warps", C.c_uint32), ("upper_window_entries", C.c_uint32),
                ("rope_warps", C.c_uint32), ("rope_window_entries", C.c_uint32),
                ("autotune_shape", C.c_uint32 * 8), ("autotune_shape_ms", C.c_float * 8)]


class gp_server_params(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_uint64), ("max_runs", C.c_uint32), ("max_batch_runs", C.c_uint32),
                ("max_batch_trees", C.c_uint32), ("chunk_nodes", C.c_uint32), ("max_batch_nodes", C.c_uint64),
                ("workspace_codes", C.c_uint64), ("workspace_values", C.c_uint64), ("use_graph", C.c_uint32),
                ("pad", C.c_uint32)]


class gp_server_result(C.Structure):
    _fields_ = [("run_id", C.c_uint64), ("request_id", C.c_uint64), ("generation", C.c_uint64),
                ("best_fitness", C.c_float), ("best_tree", C.c_uint32), ("best_hits", C.c_uint32),
                ("status", C.c_int), ("total_nodes", C.c_uint64), ("latency_ms", C.c_double),
                ("queue_ms", C.c_double)]


class gp_server_stats(C.Structure):
    _fields_ = [("batches", C.c_uint64), ("run_generations", C.c_uint64), ("requests_done", C.c_uint64),
                ("child_nodes", C.c_uint64), ("device_ms", C.c_double), ("mean_runs_per_batch", C.c_double),
                ("latency_p50_ms", C.c_double), ("latency_p99_ms", C.c_double), ("heap_bytes", C.c_uint64),
                ("heap_free", C.c_uint64), ("runs_admitted", C.c_uint32), ("runs_waiting", C.c_uint32),
                ("most_level_codes", C.c_uint64), ("most_level_values", C.c_uint64), ("retries", C.c_uint64),
                ("regrown", C.c_uint64)]


class gp_kernel_profile(C.Structure):
    _fields_ = [("launches", C.c_uint64 * 8), ("total_ms", C.c_double * 8)]


class GpError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {gp_status_string(status)}")


_lock = threading.Lock()
_lib = None


def lib():
    """The loaded libgp.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"libgp.so not found at {path}: run __graft_entry__.build()")
            L = C.CDLL(path)
            P, vp = C.POINTER, C.c_void_p
            L.gp_create_population.argtypes = [P(gp_problem), C.c_uint32, P(C.c_uint8), P(C.c_uint64), vp, P(vp)]
            L.gp_crossover.argtypes = [vp, P(gp_xo), C.c_uint32, vp, P(vp)]
            L.gp_evaluate.argtypes = [vp, vp]
            L.gp_evaluate_ex.argtypes = [vp, P(gp_eval_options), vp]
            L.gp_fitness.argtypes = [vp, P(C.c_float), P(C.c_float), P(C.c_uint32)]
            L.gp_tree_size.argtypes = [vp, C.c_uint32, P(C.c_uint64)]
            L.gp_tree_read.argtypes = [vp, C.c_uint32, P(C.c_uint8), C.c_uint64]
            L.gp_population_get_info.argtypes = [vp, P(gp_population_info)]
            L.gp_destroy_population.argtypes = [vp]
            L.gp_destroy_population.restype = None
            L.gp_status_string.argtypes = [C.c_int]
            L.gp_status_string.restype = C.c_char_p
            L.gp_eval_stats_get.argtypes = [vp, P(gp_eval_stats)]
            L.gp_kernel_launch_count.argtypes = []
            L.gp_kernel_launch_count.restype = C.c_uint64
            L.gp_profile_enable.argtypes = [C.c_int]
            L.gp_profile_read.argtypes = [P(gp_kernel_profile), C.c_int]
            L.gp_evaluate_noalloc.argtypes = [P(gp_problem), C.c_uint32, vp, P(C.c_uint64), vp, vp, vp, vp]
            L.gp_select.argtypes = [vp, vp, C.c_uint32, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                    vp, vp]
            L.gp_generation_create.argtypes = [P(gp_problem), P(gp_generation_params), C.c_uint32,
                                               P(C.c_uint8), P(C.c_uint64), vp, P(vp)]
            L.gp_generation_step.argtypes = [vp, C.c_uint32, vp]
            L.gp_generation_rewind.argtypes = [vp, vp]
            L.gp_generation_recover.argtypes = [vp, vp]
            L.gp_generation_fitness.argtypes = [vp, P(C.c_float), P(C.c_float), P(C.c_uint32)]
            L.gp_generation_records.argtypes = [vp, P(gp_xo)]
            L.gp_generation_trees.argtypes = [vp, P(C.c_uint64), P(C.c_uint8), C.c_uint64]
            L.gp_generation_tree_read.argtypes = [vp, C.c_uint32, P(C.c_uint8), C.c_uint64, P(C.c_uint64)]
            L.gp_generation_get_info.argtypes = [vp, P(gp_generation_info)]
            L.gp_generation_destroy.argtypes = [vp]
            L.gp_generation_destroy.restype = None
            L.gp_server_create.argtypes = [P(gp_problem), P(gp_server_params), P(vp)]
            L.gp_server_open_run.argtypes = [vp, P(gp_generation_params), C.c_uint32, P(C.c_uint8),
                                             P(C.c_uint64), P(C.c_uint64)]
            L.gp_server_open_run_from.argtypes = [vp, P(gp_generation_params), vp, C.c_uint32, P(C.c_uint32),
                                                  P(C.c_uint64)]
            L.gp_server_submit.argtypes = [vp, C.c_uint64, C.c_uint32, P(C.c_uint64)]
            L.gp_server_wait.argtypes = [vp, C.c_uint64, C.c_double, P(gp_server_result)]
            L.gp_server_run_fitness.argtypes = [vp, C.c_uint64, P(C.c_float), P(C.c_float), P(C.c_uint32)]
            L.gp_server_run_trees.argtypes = [vp, C.c_uint64, P(C.c_uint64), P(C.c_uint8), C.c_uint64]
            L.gp_server_close_run.argtypes = [vp, C.c_uint64]
            L.gp_server_get_stats.argtypes = [vp, P(gp_server_stats)]
            L.gp_server_destroy.argtypes = [vp]
            L.gp_server_destroy.restype = None
            _lib = L
    return _lib


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return C.c_void_p(s)
    return C.c_void_p(int(s.cuda_stream))


def _check(st, where):
    if st != GP_OK:
        raise GpError(st, where)


def _ptr(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def gp_status_string(st: int) -> str:
    return lib().gp_status_string(int(st)).decode()


class Problem:
    """Fitness cases, constants and limits (kept alive while in use)."""

    def __init__(self, x, y, consts, protected_div_value=1.0, max_tree_nodes=0, hbm_budget_bytes=0):
        self.x = np.ascontiguousarray(x, dtype=np.float32)
        self.y = np.ascontiguousarray(y, dtype=np.float32)
        self.consts = np.ascontiguousarray(consts, dtype=np.float32)
        if self.x.shape != self.y.shape:
            raise ValueError("x and y must have the same length")
        c = self.consts if self.consts.size else np.zeros(1, np.float32)
        self._c = c
        self.struct = gp_problem(self.x.shape[0], _ptr(self.x, C.c_float), _ptr(self.y, C.c_float),
                                 self.consts.shape[0], _ptr(c, C.c_float), float(protected_div_value),
                                 int(max_tree_nodes), int(hbm_budget_bytes))

    @property
    def n_cases(self):
        return self.x.shape[0]


class Population:
    """Owns one gp_population handle."""

    def __init__(self, handle, n_trees, n_cases):
        self.handle = handle
        self.n_trees = n_trees
        self.n_cases = n_cases

    def __del__(self):
        try:
            gp_destroy_population(self)
        except Exception:
            pass

    @property
    def _h(self):
        if self.handle is None:
            raise RuntimeError("population destroyed")
        return self.handle


def gp_create_population(problem: Problem, nodes, offsets, stream=None) -> Population:
    """nodes: a host array, or the device address (int) of packed trees on
    this device; offsets: host array of n_trees + 1 entries."""
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    n = offsets.shape[0] - 1
    if n < 0:
        raise ValueError("offsets needs n_trees + 1 entries")
    if isinstance(nodes, int):
        nb = C.cast(C.c_void_p(nodes), C.POINTER(C.c_uint8))
    else:
        nodes = np.ascontiguousarray(nodes, dtype=np.uint8)
        nb = _ptr(nodes if nodes.size else np.zeros(1, np.uint8), C.c_uint8)
    out = C.c_void_p()
    st = lib().gp_create_population(C.byref(problem.struct), n, nb,
                                    _ptr(offsets, C.c_uint64), _stream(stream), C.byref(out))
    _check(st, "gp_create_population")
    return Population(out, n, problem.n_cases)


# gp_xo records as a numpy structured type with the C struct's field offsets
_XO_DTYPE = np.dtype({"names": ["mum", "dad", "mum_point", "dad_point"],
                      "formats": [np.uint32, np.uint32, np.uint64, np.uint64],
                      "offsets": [gp_xo.mum.offset, gp_xo.dad.offset, gp_xo.mum_point.offset,
                                  gp_xo.dad_point.offset],
                      "itemsize": C.sizeof(gp_xo)})


def make_xo(mum, dad, mum_point, dad_point):
    """A ctypes array of gp_xo from four equal-length integer sequences
    (values wrap to the fields' widths, as ctypes assignment does)."""
    def column(v, dt):
        a = np.asarray(v)
        if a.dtype.kind in "iu":
            return a.reshape(-1).astype(dt, casting="unsafe")
        mask = (1 << (8 * dt.itemsize)) - 1              # other values: wrap one by one
        return np.array([int(x) & mask for x in np.asarray(v, dtype=object).reshape(-1)], dtype=dt)

    cols = [column(v, _XO_DTYPE[name]) for v, name in zip((mum, dad, mum_point, dad_point), _XO_DTYPE.names)]
    n = len(cols[0])
    if any(len(v) != n for v in cols):
        raise ValueError("mum, dad, mum_point and dad_point need the same length")
    rec = np.zeros(n, _XO_DTYPE)
    for name, v in zip(_XO_DTYPE.names, cols):
        rec[name] = v
    ops = (gp_xo * n)()
    if n:
        C.memmove(ops, rec.ctypes.data, rec.nbytes)
    return ops


def gp_crossover(parents: Population, ops, stream=None) -> Population:
    """ops: a ctypes array of gp_xo, or a tuple (mum, dad, mum_point, dad_point)."""
    if isinstance(ops, tuple):
        ops = make_xo(*ops)
    out = C.c_void_p()
    st = lib().gp_crossover(parents._h, ops, len(ops), _stream(stream), C.byref(out))
    _check(st, "gp_crossover")
    return Population(out, len(ops), parents.n_cases)


def gp_evaluate(pop: Population, stream=None, chunk_nodes=0, warps_per_cta=0, window_entries=0,
                upper_window_entries=0):
    if chunk_nodes or warps_per_cta or window_entries or upper_window_entries:
        o = gp_eval_options(int(chunk_nodes), int(warps_per_cta), int(window_entries),
                            int(upper_window_entries))
        st = lib().gp_evaluate_ex(pop._h, C.byref(o), _stream(stream))
    else:
        st = lib().gp_evaluate(pop._h, _stream(stream))
    _check(st, "gp_evaluate")


def gp_fitness(pop: Population, case_values=False, hits=False):
    fit = np.empty(max(pop.n_trees, 1), np.float32)
    vals = np.empty((max(pop.n_trees, 1), pop.n_cases), np.float32) if case_values else None
    h = np.empty(max(pop.n_trees, 1), np.uint32) if hits else None
    st = lib().gp_fitness(pop._h, _ptr(fit, C.c_float),
                          _ptr(vals, C.c_float) if vals is not None else None,
                          _ptr(h, C.c_uint32) if h is not None else None)
    _check(st, "gp_fitness")
    n = pop.n_trees
    return fit[:n], (vals[:n] if vals is not None else None), (h[:n] if h is not None else None)


def gp_tree_size(pop: Population, tree: int) -> int:
    n = C.c_uint64()
    _check(lib().gp_tree_size(pop._h, int(tree), C.byref(n)), "gp_tree_size")
    return int(n.value)


def gp_tree_read(pop: Population, tree: int) -> np.ndarray:
    n = gp_tree_size(pop, tree)
    buf = np.empty(max(n, 1), np.uint8)
    _check(lib().gp_tree_read(pop._h, int(tree), _ptr(buf, C.c_uint8), n), "gp_tree_read")
    return buf[:n]


def gp_population_get_info(pop: Population) -> gp_population_info:
    info = gp_population_info()
    _check(lib().gp_population_get_info(pop._h, C.byref(info)), "gp_population_get_info")
    return info


def gp_destroy_population(pop: Population):
    if pop.handle is not None:
        lib().gp_destroy_population(pop.handle)
        pop.handle = None


def gp_eval_stats_get(pop: Population) -> dict:
    s = gp_eval_stats()
    _check(lib().gp_eval_stats_get(pop._h, C.byref(s)), "gp_eval_stats_get")
    return {"levels": s.levels, "redone": s.redone, "items": s.items, "upper_codes": s.upper_codes,
            "value_entries": s.value_entries, "upper_ops": s.upper_ops}


def gp_kernel_launch_count() -> int:
    return int(lib().gp_kernel_launch_count())


def gp_profile_enable(on: bool):
    _check(lib().gp_profile_enable(1 if on else 0), "gp_profile_enable")


def gp_profile_read(reset: bool = False) -> dict:
    p = gp_kernel_profile()
    _check(lib().gp_profile_read(C.byref(p), 1 if reset else 0), "gp_profile_read")
    return {k: {"launches": int(p.launches[i]), "ms": float(p.total_ms[i])}
            for i, k in enumerate(KERNEL_KINDS) if k != "unused"}


def gp_evaluate_noalloc(problem: Problem, offsets, d_nodes: int, d_fitness: int, d_case_values: int,
                        d_hits: int, stream=None):
    """Evaluate trees already on the device (packed as `offsets` describes)
    into caller-provided device outputs, without any allocation in libgp.
    Device arguments are raw addresses (e.g. torch tensor data_ptr())."""
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    n = offsets.shape[0] - 1
    st = lib().gp_evaluate_noalloc(C.byref(problem.struct), n, C.c_void_p(int(d_nodes)),
                                   _ptr(offsets, C.c_uint64), C.c_void_p(int(d_fitness)),
                                   C.c_void_p(int(d_case_values)), C.c_void_p(int(d_hits)),
                                   _stream(stream))
    _check(st, "gp_evaluate_noalloc")


def gp_select(d_fitness: int, d_sizes: int, n_pop: int, seed, generation: int, child_lo: int, n_children: int,
              d_out: int, tournament_size=7, stream=None):
    """Selection records of children [child_lo, child_lo + n_children) from a
    whole population's fitness and sizes (device addresses, e.g. torch
    tensors' data_ptr()); writes n_children gp_xo records at d_out."""
    _check(lib().gp_select(C.c_void_p(int(d_fitness)), C.c_void_p(int(d_sizes)), int(n_pop),
                           int(seed) & ((1 << 64) - 1), int(generation), int(child_lo), int(n_children),
                           int(tournament_size), C.c_void_p(int(d_out)), _stream(stream)), "gp_select")


XO_RECORD_BYTES = C.sizeof(gp_xo)


class Generation:
    """Owns one gp_generation handle (a device-resident evolving population)."""

    def __init__(self, handle, n_trees, n_cases):
        self._h = handle
        self.n_trees = n_trees
        self.n_cases = n_cases

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h and _lib is not None:
            _lib.gp_generation_destroy(h)


def gp_generation_create(problem: Problem, nodes, offsets, seed, tournament_size=7, chunk_nodes=0,
                         arena_bytes=0, workspace_codes=0, workspace_values=0, use_graph=True,
                         max_levels=0, stream=None, warps_per_cta=0, window_entries=0,
                         upper_window_entries=0) -> Generation:
    nodes = np.ascontiguousarray(nodes, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    n = offsets.shape[0] - 1
    prm = gp_generation_params(int(seed) & ((1 << 64) - 1), int(tournament_size), int(chunk_nodes),
                               int(arena_bytes), int(workspace_codes), int(workspace_values),
                               1 if use_graph else 0, int(max_levels), int(warps_per_cta), int(window_entries),
                               int(upper_window_entries), 0)
    h = C.c_void_p()
    st = lib().gp_generation_create(C.byref(problem.struct), C.byref(prm), n, _ptr(nodes, C.c_uint8),
                                    _ptr(offsets, C.c_uint64), _stream(stream), C.byref(h))
    _check(st, "gp_generation_create")
    return Generation(h, n, problem.n_cases)


def gp_generation_step(g: Generation, n=1, stream=None):
    _check(lib().gp_generation_step(g._h, int(n), _stream(stream)), "gp_generation_step")


def gp_generation_rewind(g: Generation, stream=None):
    _check(lib().gp_generation_rewind(g._h, _stream(stream)), "gp_generation_rewind")


def gp_generation_recover(g: Generation, stream=None):
    _check(lib().gp_generation_recover(g._h, _stream(stream)), "gp_generation_recover")


def gp_generation_fitness(g: Generation, case_values=False, hits=False):
    fit = np.empty(g.n_trees, np.float32)
    vals = np.empty((g.n_trees, g.n_cases), np.float32) if case_values else None
    h = np.empty(g.n_trees, np.uint32) if hits else None
    st = lib().gp_generation_fitness(g._h, _ptr(fit, C.c_float),
                                     _ptr(vals, C.c_float) if vals is not None else None,
                                     _ptr(h, C.c_uint32) if h is not None else None)
    _check(st, "gp_generation_fitness")
    return fit, vals, h


def gp_generation_records(g: Generation):
    recs = (gp_xo * g.n_trees)()
    _check(lib().gp_generation_records(g._h, recs), "gp_generation_records")
    return split_xo(recs)


def split_xo(recs):
    """(mum, dad, mum_point, dad_point) arrays of a ctypes array of gp_xo."""
    rec = np.frombuffer(bytes(recs), dtype=_XO_DTYPE, count=len(recs))
    return tuple(rec[name].copy() for name in _XO_DTYPE.names)


def gp_generation_trees(g: Generation):
    offs = np.empty(g.n_trees + 1, np.uint64)
    _check(lib().gp_generation_trees(g._h, _ptr(offs, C.c_uint64), None, 0), "gp_generation_trees")
    nodes = np.empty(max(int(offs[-1]), 1), np.uint8)
    _check(lib().gp_generation_trees(g._h, _ptr(offs, C.c_uint64), _ptr(nodes, C.c_uint8), nodes.shape[0]),
           "gp_generation_trees")
    return nodes[:int(offs[-1])], offs


def gp_generation_tree_read(g: Generation, tree: int) -> np.ndarray:
    """Bytes of one tree of the current population."""
    n = C.c_uint64()
    _check(lib().gp_generation_tree_read(g._h, int(tree), None, 0, C.byref(n)), "gp_generation_tree_read")
    out = np.empty(max(int(n.value), 1), np.uint8)
    _check(lib().gp_generation_tree_read(g._h, int(tree), _ptr(out, C.c_uint8), out.shape[0], C.byref(n)),
           "gp_generation_tree_read")
    return out[:int(n.value)]


def gp_generation_get_info(g: Generation) -> dict:
    i = gp_generation_info()
    _check(lib().gp_generation_get_info(g._h, C.byref(i)), "gp_generation_get_info")
    d = {k: getattr(i, k) for k, _ in gp_generation_info._fields_}
    d["autotune_chunk"] = list(i.autotune_chunk)
    d["autotune_ms"] = list(i.autotune_ms)
    # (warps, window entries, "level0" | "upper"); (0, 0, "") for an unused slot
    d["autotune_shape"] = [(v >> 16, v & 0x7FFF, ("upper" if v & 0x8000 else "level0") if v else "")
                           for v in i.autotune_shape]
    d["autotune_shape_ms"] = list(i.autotune_shape_ms)
    return d


def gp_generation_destroy(g: Generation):
    h, g._h = g._h, None
    if h:
        lib().gp_generation_destroy(h)


class Server:
    """Owns one gp_server handle (a serving loop over many runs)."""

    def __init__(self, handle, n_cases):
        self._h = handle
        self.n_cases = n_cases
        self.problem = None          # kept alive with the server
        self.run_trees = {}          # run id -> number of trees
        self.sources = {}            # run id -> the population its initial trees come from

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h and _lib is not None:
            _lib.gp_server_destroy(h)


def gp_server_create(problem: Problem, hbm_budget_bytes, max_runs=64, max_batch_trees=1 << 20,
                     max_batch_runs=0, chunk_nodes=0, max_batch_nodes=0, workspace_codes=0,
                     workspace_values=0, use_graph=True) -> Server:
    prm = gp_server_params(int(hbm_budget_bytes), int(max_runs), int(max_batch_runs), int(max_batch_trees),
                           int(chunk_nodes), int(max_batch_nodes), int(workspace_codes), int(workspace_values),
                           1 if use_graph else 0, 0)
    h = C.c_void_p()
    _check(lib().gp_server_create(C.byref(problem.struct), C.byref(prm), C.byref(h)), "gp_server_create")
    s = Server(h, problem.n_cases)
    s.problem = problem
    return s


def gp_server_open_run(srv: Server, nodes, offsets, seed, tournament_size=7, arena_bytes=0) -> int:
    nodes = np.ascontiguousarray(nodes, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    n = offsets.shape[0] - 1
    prm = gp_generation_params(int(seed) & ((1 << 64) - 1), int(tournament_size), 0, int(arena_bytes), 0, 0, 0, 0,
                               0, 0, 0, 0)
    rid = C.c_uint64()
    _check(lib().gp_server_open_run(srv._h, C.byref(prm), n, _ptr(nodes, C.c_uint8), _ptr(offsets, C.c_uint64),
                                    C.byref(rid)), "gp_server_open_run")
    srv.run_trees[rid.value] = n
    return rid.value


def gp_server_open_run_from(srv: Server, pop: Population, trees, seed, tournament_size=7, arena_bytes=0) -> int:
    """A run whose initial trees are `trees` (indices into `pop`, which must
    stay alive until the run is admitted or closed)."""
    trees = np.ascontiguousarray(trees, dtype=np.uint32)
    prm = gp_generation_params(int(seed) & ((1 << 64) - 1), int(tournament_size), 0, int(arena_bytes), 0, 0, 0, 0,
                               0, 0, 0, 0)
    rid = C.c_uint64()
    _check(lib().gp_server_open_run_from(srv._h, C.byref(prm), pop._h, trees.shape[0], _ptr(trees, C.c_uint32),
                                         C.byref(rid)), "gp_server_open_run_from")
    srv.run_trees[rid.value] = int(trees.shape[0])
    srv.sources[rid.value] = pop              # kept alive with the run
    return rid.value


def gp_server_submit(srv: Server, run_id, n_generations=1) -> int:
    q = C.c_uint64()
    _check(lib().gp_server_submit(srv._h, int(run_id), int(n_generations), C.byref(q)), "gp_server_submit")
    return q.value


def gp_server_wait(srv: Server, request_id, timeout_ms=-1.0) -> dict:
    r = gp_server_result()
    _check(lib().gp_server_wait(srv._h, int(request_id), float(timeout_ms), C.byref(r)), "gp_server_wait")
    return {k: getattr(r, k) for k, _ in gp_server_result._fields_}


def gp_server_run_fitness(srv: Server, run_id, case_values=False, hits=False):
    n = srv.run_trees[run_id]
    fit = np.empty(n, np.float32)
    vals = np.empty((n, srv.n_cases), np.float32) if case_values else None
    h = np.empty(n, np.uint32) if hits else None
    _check(lib().gp_server_run_fitness(srv._h, int(run_id), _ptr(fit, C.c_float),
                                       _ptr(vals, C.c_float) if vals is not None else None,
                                       _ptr(h, C.c_uint32) if h is not None else None), "gp_server_run_fitness")
    return fit, vals, h


def gp_server_run_trees(srv: Server, run_id):
    n = srv.run_trees[run_id]
    offs = np.empty(n + 1, np.uint64)
    _check(lib().gp_server_run_trees(srv._h, int(run_id), _ptr(offs, C.c_uint64), None, 0), "gp_server_run_trees")
    nodes = np.empty(max(int(offs[-1]), 1), np.uint8)
    _check(lib().gp_server_run_trees(srv._h, int(run_id), _ptr(offs, C.c_uint64), _ptr(nodes, C.c_uint8),
                                     nodes.shape[0]), "gp_server_run_trees")
    return nodes[:int(offs[-1])], offs


def gp_server_close_run(srv: Server, run_id):
    _check(lib().gp_server_close_run(srv._h, int(run_id)), "gp_server_close_run")
    srv.run_trees.pop(run_id, None)
    srv.sources.pop(run_id, None)


def gp_server_get_stats(srv: Server) -> dict:
    st = gp_server_stats()
    _check(lib().gp_server_get_stats(srv._h, C.byref(st)), "gp_server_get_stats")
    return {k: getattr(st, k) for k, _ in gp_server_stats._fields_}


def gp_server_destroy(srv: Server):
    h, srv._h = srv._h, None
    if h:
        lib().gp_server_destroy(h)


def read_all_trees(pop: Population):
    """(nodes, offsets) of every tree, packed."""
    trees = [gp_tree_read(pop, t) for t in range(pop.n_trees)]
    sizes = np.array([t.shape[0] for t in trees], dtype=np.uint64)
    offs = np.zeros(len(trees) + 1, np.uint64)
    np.cumsum(sizes, out=offs[1:])
    return (np.concatenate(trees) if trees else np.zeros(0, np.uint8)), offs
