"""Python access to the CPU oracle (oracle/gp_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline leg and reference arm (--impl reference), never by
the product package.  It shares no
code with the CUDA library; both sides only share the seeded input
generators of paper_1902_09215_gb300.synth.

The oracle follows the paper's traditional recursive EVAL (Sec. 2.2), the
protected division and MAE fitness of Table gp.details, hits of Sec. 3.2 and
the subtree crossover of Sec. 3.1.  Pins that tie it to the paper and to
mathematics (not to itself) live in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_M64 = (1 << 64) - 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-pthread"]

OK, EINVAL, ENOMEM, EMALFORMED = 0, 1, 2, 3
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            u8p, f32p, f64p = C.POINTER(C.c_uint8), C.POINTER(C.c_float), C.POINTER(C.c_double)
            u64p, u32p = C.POINTER(C.c_uint64), C.POINTER(C.c_uint32)
            L.oracle_eval_tree_f32.argtypes = [u8p, C.c_uint64, f32p, C.c_uint32, f32p, C.c_uint32, C.c_float, f32p]
            L.oracle_eval_tree_f64.argtypes = [u8p, C.c_uint64, f32p, C.c_uint32, f32p, C.c_uint32, C.c_float, f64p]
            L.oracle_mae_f32.argtypes = [f32p, f32p, C.c_uint32, u32p]
            L.oracle_mae_f32.restype = C.c_float
            L.oracle_mae_f64.argtypes = [f64p, f64p, C.c_uint32]
            L.oracle_mae_f64.restype = C.c_double
            L.oracle_tree_depth.argtypes = [u8p, C.c_uint64]
            L.oracle_tree_depth.restype = C.c_uint64
            L.oracle_check_tree.argtypes = [u8p, C.c_uint64, C.c_uint32]
            L.oracle_subtree_end.argtypes = [u8p, C.c_uint64, C.c_uint64, u64p]
            L.oracle_crossover.argtypes = [u8p, C.c_uint64, u8p, C.c_uint64, C.c_uint64, C.c_uint64,
                                           u8p, C.c_uint64, u64p]
            L.oracle_eval_population.argtypes = [u8p, u64p, C.c_uint32, f32p, f32p, C.c_uint32, f32p,
                                                 C.c_uint32, C.c_float, f32p, f32p, u32p, f64p, f64p,
                                                 C.c_int]
            L.oracle_sm64_at.argtypes = [C.c_uint64, C.c_uint64]
            L.oracle_sm64_at.restype = C.c_uint64
            L.oracle_bounded.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
            L.oracle_bounded.restype = C.c_uint64
            L.oracle_tournament.argtypes = [f32p, C.c_uint32, C.c_uint64, C.c_uint64, C.c_uint64,
                                            C.c_uint32, C.c_uint32]
            L.oracle_tournament.restype = C.c_uint32
            L.oracle_generation.argtypes = [f32p, u64p, C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint64,
                                            C.c_uint32, u32p, u32p, u64p, u64p]
            _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


class OracleError(RuntimeError):
    pass


def eval_tree(tree, x, consts, div0: float = 1.0, dtype=np.float32) -> np.ndarray:
    """Per-case outputs of one prefix tree (FP32 or FP64 recursion)."""
    t, x, c = _u8(tree), _f32(x), _f32(consts)
    if dtype == np.float64:
        out = np.empty(x.shape[0], dtype=np.float64)
        st = lib().oracle_eval_tree_f64(_p(t, C.c_uint8), t.shape[0], _p(x, C.c_float), x.shape[0],
                                        _p(c, C.c_float), c.shape[0], div0, _p(out, C.c_double))
    else:
        out = np.empty(x.shape[0], dtype=np.float32)
        st = lib().oracle_eval_tree_f32(_p(t, C.c_uint8), t.shape[0], _p(x, C.c_float), x.shape[0],
                                        _p(c, C.c_float), c.shape[0], div0, _p(out, C.c_float))
    if st:
        raise OracleError(f"oracle eval failed: status {st}")
    return out


def mae_f32(out, y):
    o, yy = _f32(out), _f32(y)
    h = C.c_uint32(0)
    f = lib().oracle_mae_f32(_p(o, C.c_float), _p(yy, C.c_float), o.shape[0], C.byref(h))
    return np.float32(f), int(h.value)


def mae_f64(out, y):
    o = np.ascontiguousarray(out, dtype=np.float64)
    yy = np.ascontiguousarray(y, dtype=np.float64)
    return float(lib().oracle_mae_f64(_p(o, C.c_double), _p(yy, C.c_double), o.shape[0]))


def tree_depth(tree) -> int:
    t = _u8(tree)
    return int(lib().oracle_tree_depth(_p(t, C.c_uint8), t.shape[0]))


def check_tree(tree, n_consts: int = 127) -> bool:
    t = _u8(tree)
    return bool(lib().oracle_check_tree(_p(t, C.c_uint8), t.shape[0], n_consts))


def subtree_end(tree, i: int) -> int:
    t = _u8(tree)
    e = C.c_uint64(0)
    st = lib().oracle_subtree_end(_p(t, C.c_uint8), t.shape[0], int(i), C.byref(e))
    if st:
        raise OracleError(f"subtree_end failed: status {st}")
    return int(e.value)


def crossover(mum, dad, i: int, j: int) -> np.ndarray:
    m, d = _u8(mum), _u8(dad)
    n = C.c_uint64(0)
    st = lib().oracle_crossover(_p(m, C.c_uint8), m.shape[0], _p(d, C.c_uint8), d.shape[0],
                                int(i), int(j), None, 0, C.byref(n))
    if st:
        raise OracleError(f"crossover failed: status {st}")
    child = np.empty(n.value, dtype=np.uint8)
    st = lib().oracle_crossover(_p(m, C.c_uint8), m.shape[0], _p(d, C.c_uint8), d.shape[0],
                                int(i), int(j), _p(child, C.c_uint8), child.shape[0], C.byref(n))
    if st:
        raise OracleError(f"crossover failed: status {st}")
    return child


def crossover_population(nodes, offsets, mum, dad, mum_point, dad_point):
    """Children of a list of crossover records, packed as (nodes, offsets)."""
    nodes, offsets = _u8(nodes), np.asarray(offsets, dtype=np.uint64)
    kids = []
    for a, b, i, j in zip(mum, dad, mum_point, dad_point):
        M = nodes[int(offsets[a]):int(offsets[a + 1])]
        D = nodes[int(offsets[b]):int(offsets[b + 1])]
        kids.append(crossover(M, D, int(i), int(j)))
    sizes = np.array([k.shape[0] for k in kids], dtype=np.uint64)
    offs = np.zeros(len(kids) + 1, dtype=np.uint64)
    np.cumsum(sizes, out=offs[1:])
    return (np.concatenate(kids) if kids else np.zeros(0, np.uint8)), offs


def eval_population(nodes, offsets, x, y, consts, div0: float = 1.0, n_threads: int = 1,
                    want_f64: bool = False):
    """Evaluate every tree: returns dict with out, fitness, hits (FP32) and,
    if want_f64, out64 and fitness64 (FP64 recursion, FP64 MAE)."""
    nodes = _u8(nodes)
    offs = np.ascontiguousarray(offsets, dtype=np.uint64)
    x, y, c = _f32(x), _f32(y), _f32(consts)
    P = offs.shape[0] - 1
    nc = x.shape[0]
    out = np.empty((P, nc), dtype=np.float32)
    fit = np.empty(P, dtype=np.float32)
    hits = np.empty(P, dtype=np.uint32)
    out64 = np.empty((P, nc), dtype=np.float64) if want_f64 else None
    fit64 = np.empty(P, dtype=np.float64) if want_f64 else None
    nullf64 = C.POINTER(C.c_double)()
    st = lib().oracle_eval_population(
        _p(nodes, C.c_uint8), _p(offs, C.c_uint64), P, _p(x, C.c_float), _p(y, C.c_float), nc,
        _p(c, C.c_float), c.shape[0], div0, _p(out, C.c_float), _p(fit, C.c_float),
        _p(hits, C.c_uint32), _p(out64, C.c_double) if want_f64 else nullf64,
        _p(fit64, C.c_double) if want_f64 else nullf64, int(n_threads))
    if st:
        raise OracleError(f"oracle population eval failed: status {st}")
    r = {"out": out, "fitness": fit, "hits": hits}
    if want_f64:
        r["out64"], r["fitness64"] = out64, fit64
    return r


# ---------------------------------------------------------------------------
# Generation: counter-based draws, tournament selection, crossover records
# ---------------------------------------------------------------------------

def draw_counter(g: int, c: int, purpose: int, k: int = 0, attempt: int = 0) -> int:
    """Counter of one draw (generation, child, purpose, index, attempt)."""
    return (g << 40) | (c << 12) | (purpose << 9) | (k << 4) | attempt


def sm64_at(seed: int, i: int) -> int:
    """Output i of SplitMix64 seeded with `seed`."""
    return int(lib().oracle_sm64_at(seed & _M64, i & _M64))


def bounded(seed: int, base: int, n: int) -> int:
    """Unbiased draw in [0, n) from the counters base, base+1, ... ."""
    return int(lib().oracle_bounded(seed & _M64, base & _M64, n))


def tournament(fitness, seed: int, g: int, c: int, purpose: int, size: int) -> int:
    f = _f32(fitness)
    return int(lib().oracle_tournament(_p(f, C.c_float), f.shape[0], seed & _M64, g, c, purpose, size))


def generation_records(fitness, sizes, n_children: int, seed: int, g: int, tsize: int = 7):
    """(mum, dad, mum_point, dad_point) of every child of generation g."""
    f = _f32(fitness)
    sz = np.ascontiguousarray(sizes, dtype=np.uint64)
    mum = np.empty(n_children, np.uint32)
    dad = np.empty(n_children, np.uint32)
    mp = np.empty(n_children, np.uint64)
    dp = np.empty(n_children, np.uint64)
    st = lib().oracle_generation(_p(f, C.c_float), _p(sz, C.c_uint64), f.shape[0], n_children,
                                 seed & _M64, g, tsize, _p(mum, C.c_uint32), _p(dad, C.c_uint32),
                                 _p(mp, C.c_uint64), _p(dp, C.c_uint64))
    if st:
        raise OracleError(f"generation records failed: status {st}")
    return mum, dad, mp, dp
