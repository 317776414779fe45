"""Seeded synthetic inputs for the Sextic GP workloads.

This module only draws inputs: constant tables, fitness-case tables, random
prefix trees, crossover points.  It holds none of the evaluation arithmetic
and is the one module that both the CUDA path's tests and the CPU oracle's
tests import.  Every generator is seeded and deterministic.

Encoding (one byte per node, prefix / root-first order, Sec. 2.1-2.2):
    0 '+'   1 '-'   2 '*'   3 protected '/'   (arity 2)
    4 'x'   5..131 constant table entry code-5 (arity 0)
"""
from __future__ import annotations

import math

import numpy as np

OP_ADD, OP_SUB, OP_MUL, OP_DIV, LEAF_X, CONST0 = 0, 1, 2, 3, 4, 5
N_CASES = 48          # Sec. 3 / Table gp.details: 48 fitness cases
N_CONSTS = 127        # constant codes 5..131
_M64 = (1 << 64) - 1


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n outputs of SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) from `seed`."""
    out = np.empty(n, dtype=np.uint64)
    s = seed & _M64
    for i in range(n):
        s = (s + 0x9E3779B97F4A7C15) & _M64
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        out[i] = z ^ (z >> 31)
    return out


def constants(seed: int = 2, n: int = N_CONSTS) -> np.ndarray:
    """n float32 constants uniform on [-1, 1): c = 2u - 1, u = (r >> 40) / 2^24.

    Stand-in for the paper's 250 ephemeral random constants (Sec. 2.1,
    Table gp.details), which are not printed.  Every value is exact in FP32.
    """
    r = splitmix64(seed, n)
    u = (r >> np.uint64(40)).astype(np.float64) * (2.0 ** -24)
    return (2.0 * u - 1.0).astype(np.float32)


def paper_grid_constants(seed: int = 7, n: int = 250) -> np.ndarray:
    """Optional paper-style constants: k/1000 on the 2001-point grid [-1, 1],
    excluding 0 and the end points (Sec. 2.1), rounded to FP32."""
    rng = np.random.default_rng(seed)
    grid = np.array([k for k in range(-999, 1000) if k != 0], dtype=np.int64)
    ks = rng.choice(grid, size=n, replace=False)
    return (ks.astype(np.float64) / 1000.0).astype(np.float32)


def cases(n: int = N_CASES) -> np.ndarray:
    """n fitness-case inputs evenly spaced on [-1, 1]: x_i = fl32(-1 + 2i/(n-1)).

    Stand-in for the paper's 48 random inputs in [-0.97789, 0.979541]
    (Table gp.details), whose values are not printed.
    """
    i = np.arange(n, dtype=np.float64)
    return (-1.0 + 2.0 * i / max(n - 1, 1)).astype(np.float32)


def sextic_targets_f32(x: np.ndarray) -> np.ndarray:
    """Problem data: y = x*x*(x-1)*(x-1)*(x+1)*(x+1) (Table gp.details),
    evaluated left to right with every operation rounded to FP32."""
    x = np.asarray(x, dtype=np.float32)
    one = np.float32(1.0)
    y = np.empty_like(x)
    for i, xi in enumerate(x):
        a = np.float32(xi * xi)
        a = np.float32(a * np.float32(xi - one))
        a = np.float32(a * np.float32(xi - one))
        a = np.float32(a * np.float32(xi + one))
        a = np.float32(a * np.float32(xi + one))
        y[i] = a
    return y


def sextic_targets_f64(x: np.ndarray) -> np.ndarray:
    """The same target polynomial evaluated in double from the FP32 inputs."""
    xd = np.asarray(x, dtype=np.float32).astype(np.float64)
    return xd * xd * (xd - 1.0) * (xd - 1.0) * (xd + 1.0) * (xd + 1.0)


def problem(n_cases: int = N_CASES, n_consts: int = N_CONSTS, const_seed: int = 2):
    """(x, y, consts) for the Sextic problem, all float32."""
    x = cases(n_cases)
    return x, sextic_targets_f32(x), constants(const_seed, n_consts)


# ---------------------------------------------------------------------------
# Random prefix trees
# ---------------------------------------------------------------------------

def random_shape(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random full binary tree with n nodes (n odd) as a boolean
    'is internal' mask in prefix order.

    Cycle lemma: shuffle (n-1)/2 internal (+1) and (n+1)/2 leaf (-1) steps,
    then rotate to start at the first index where the partial sum is
    minimal; exactly one rotation is a valid prefix tree.
    """
    if n < 1 or n % 2 == 0:
        raise ValueError("tree size must be odd and >= 1")
    n_int = (n - 1) // 2
    step = np.full(n, -1, dtype=np.int8)
    step[:n_int] = 1
    rng.shuffle(step)
    ps = np.cumsum(step, dtype=np.int64 if n > (1 << 30) else np.int32)
    j = int(np.argmin(ps)) + 1          # first index of the minimum, 1-based
    if j == n:
        j = 0
    internal = np.concatenate([step[j:], step[:j]]) > 0
    return internal


def label_tree(rng: np.random.Generator, internal: np.ndarray, p_x: float = 0.5,
               n_consts: int = N_CONSTS, ops: tuple = (0, 1, 2, 3)) -> np.ndarray:
    """Fill a shape with codes: internal nodes uniform over `ops`; leaves are
    x with probability p_x, else a uniform constant code."""
    n = internal.shape[0]
    codes = np.empty(n, dtype=np.uint8)
    n_int = int(internal.sum())
    opsarr = np.asarray(ops, dtype=np.uint8)
    codes[internal] = opsarr[rng.integers(0, len(opsarr), size=n_int)]
    n_leaf = n - n_int
    is_x = rng.random(n_leaf) < p_x
    leaf = (CONST0 + rng.integers(0, n_consts, size=n_leaf)).astype(np.uint8)
    leaf[is_x] = LEAF_X
    codes[~internal] = leaf
    return codes


def random_tree(rng: np.random.Generator, n: int, p_x: float = 0.5,
                n_consts: int = N_CONSTS, ops: tuple = (0, 1, 2, 3)) -> np.ndarray:
    return label_tree(rng, random_shape(rng, n), p_x, n_consts, ops)


def left_spine_tree(rng: np.random.Generator, depth: int, hang_size: int,
                    n_consts: int = N_CONSTS) -> np.ndarray:
    """A deliberately stringy tree: a chain of `depth` operators, each one's
    first child continuing the chain and each second child a random subtree
    of `hang_size` nodes.  Prefix: op_1 .. op_D base S_D .. S_1.  Its depth
    is >= depth and a right-to-left stack evaluation holds ~depth values."""
    ops = rng.integers(0, 4, size=depth).astype(np.uint8)
    base = random_tree(rng, hang_size, n_consts=n_consts)
    hangs = [random_tree(rng, hang_size, n_consts=n_consts) for _ in range(depth)]
    return np.concatenate([ops, base] + hangs[::-1])


def pack(trees) -> tuple[np.ndarray, np.ndarray]:
    """Concatenate trees into (nodes uint8[N], offsets uint64[P+1])."""
    sizes = np.array([t.shape[0] for t in trees], dtype=np.uint64)
    offsets = np.zeros(len(trees) + 1, dtype=np.uint64)
    np.cumsum(sizes, out=offsets[1:])
    nodes = np.concatenate(trees).astype(np.uint8) if trees else np.zeros(0, np.uint8)
    return nodes, offsets


def odd(n: int) -> int:
    return n if n % 2 == 1 else n + 1


def loguniform_sizes(rng: np.random.Generator, count: int, lo: int, hi: int) -> np.ndarray:
    """Odd sizes round(exp(U[ln lo, ln hi])), kept within [lo, hi]."""
    u = rng.uniform(math.log(lo), math.log(hi), size=count)
    s = np.rint(np.exp(u)).astype(np.int64)
    s = np.where(s % 2 == 0, s + 1, s)
    s = np.where(s > hi, s - 2, s)
    return np.clip(s, lo, hi)


def population_small(seed: int = 1, count: int = 50, max_nodes: int = 63):
    """50 trees of 1..63 nodes, odd sizes uniform (smallest workload)."""
    rng = np.random.default_rng(seed)
    sizes = 1 + 2 * rng.integers(0, (max_nodes + 1) // 2, size=count)
    return pack([random_tree(rng, int(n)) for n in sizes])


def population_loguniform(seed: int = 3, count: int = 4000, lo: int = 31, hi: int = 32767,
                          p_x: float = 0.5):
    """`count` random trees with odd sizes log-uniform on [lo, hi]."""
    rng = np.random.default_rng(seed)
    sizes = loguniform_sizes(rng, count, lo, hi)
    return pack([random_tree(rng, int(n), p_x=p_x) for n in sizes])


def crossover_points(seed: int, sizes: np.ndarray, n_ops: int, n_parents: int | None = None):
    """Uniformly chosen (mum, dad, mum_point, dad_point) records (Sec. 3.1):
    parents uniform over the population, points uniform over all nodes."""
    rng = np.random.default_rng(seed)
    sizes = np.asarray(sizes, dtype=np.int64)
    p = sizes.shape[0] if n_parents is None else n_parents
    mum = rng.integers(0, p, size=n_ops)
    dad = rng.integers(0, p, size=n_ops)
    mp = (rng.random(n_ops) * sizes[mum]).astype(np.int64)
    dp = (rng.random(n_ops) * sizes[dad]).astype(np.int64)
    mp = np.minimum(mp, sizes[mum] - 1)
    dp = np.minimum(dp, sizes[dad] - 1)
    return (mum.astype(np.uint32), dad.astype(np.uint32),
            mp.astype(np.uint64), dp.astype(np.uint64))
