"""Seeded synthetic inputs for the Sextic GP workloads.

This module only draws inputs: constant tables, fitness-case tables, random
prefix trees, crossover points.  It holds none of the evaluation arithmetic
and is the one module that both the CUDA path's tests and the CPU oracle's
tests import.  Every generator is seeded and deterministic.

Encoding (one byte per node, prefix / root-first order, Sec. 2.1-2.2):
    0 '+'   1 '-'   2 '*'   3 protected '/'   (arity 2)
    4 'x'   5..5+n_consts-1 constant table entry code-5 (arity 0); 127
            constants by default, up to 250 (the paper's grid, codes 5..254)
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


def paper_grid_population(seed: int = 12, count: int = 300, lo: int = 1, hi: int = 20001):
    """Random trees over the paper's 250 grid constants (codes up to 254),
    odd sizes log-uniform on [lo, hi]."""
    rng = np.random.default_rng(seed)
    sizes = loguniform_sizes(rng, count, lo, hi)
    return pack([random_tree(rng, int(n), n_consts=250) for n in sizes])


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


def ramped_half_and_half(seed: int = 1, count: int = 4000, min_depth: int = 2, max_depth: int = 6,
                         n_consts: int = N_CONSTS, p_function: float = 2.0 / 3.0, p_x: float = 0.5):
    """Koza's ramped half-and-half initial population (Table gp.details:
    4000 trees, depth between 2 and 6): depths cycle over min_depth ..
    max_depth, and at each depth the trees alternate between the full method
    (every leaf at that depth) and the grow method (below that depth a node
    is an operator with probability p_function, else a leaf).  The root is
    always an operator.  Leaves are x with probability p_x, else a uniform
    constant; operators are uniform.  Depth counts edges from the root."""
    rng = np.random.default_rng(seed)
    depths = list(range(min_depth, max_depth + 1))
    trees = []
    for i in range(count):
        d = depths[i % len(depths)]
        full = (i // len(depths)) % 2 == 0
        codes = []
        stack = [0]                                 # depths of the nodes still to write
        while stack:
            depth = stack.pop()
            leaf = depth == d or (not full and depth > 0 and rng.random() >= p_function)
            if leaf:
                codes.append(LEAF_X if rng.random() < p_x else CONST0 + int(rng.integers(0, n_consts)))
            else:
                codes.append(int(rng.integers(0, 4)))
                stack.extend((depth + 1, depth + 1))
        trees.append(np.array(codes, dtype=np.uint8))
    return pack(trees)


def deepest_leaf(tree: np.ndarray) -> tuple[int, int]:
    """(position, depth) of the first deepest leaf of a prefix tree (root
    depth 0).  A stack of open child slots, each tagged with its depth."""
    slots = [0]
    best_pos, best_d = 0, -1
    for i, c in enumerate(tree.tolist()):
        d = slots.pop()
        if c < LEAF_X:
            slots.append(d + 1)
            slots.append(d + 1)
        elif d > best_d:
            best_pos, best_d = i, d
    return best_pos, best_d


class _Piece:
    """One grafted tree inside a bloated tree: its codes and, per replaced
    leaf position, the piece grafted there."""
    __slots__ = ("codes", "leaves", "kids")

    def __init__(self, codes, leaves=None):
        self.codes = codes
        self.leaves = leaves
        self.kids = {}

    def leaf_positions(self):
        if self.leaves is None:
            self.leaves = np.flatnonzero(self.codes >= LEAF_X)
        return self.leaves


def _write_pieces(root: _Piece, out: np.ndarray, at: int) -> int:
    """Write the prefix array of a tree of pieces into out[at:], iteratively
    (chains of grafts nest deeply); returns the end position."""
    stack = [[root, sorted(root.kids), 0, 0]]
    while stack:
        fr = stack[-1]
        piece, kids, k, frm = fr
        if k < len(kids):
            p = kids[k]
            n = p - frm
            out[at:at + n] = piece.codes[frm:p]
            at += n
            fr[2], fr[3] = k + 1, p + 1
            child = piece.kids[p]
            stack.append([child, sorted(child.kids), 0, 0])
        else:
            n = piece.codes.shape[0] - frm
            out[at:at + n] = piece.codes[frm:]
            at += n
            stack.pop()
    return at


def _graft_tree(rng, target, pool, donor_hi, chain=None, chain_depth=0, pool_leaves=None):
    """The pieces of a tree of exactly `target` nodes grown by repeated
    subtree crossover (Sec. 3.1) whose dad point is the root of a whole
    donor tree and whose mum point is a leaf of the tree grown so far.
    Optionally a chain of grafts at the deepest leaf first, until the depth
    reaches `chain_depth`; then grafts at leaves chosen uniformly over the
    whole tree, the last one a fresh random tree sized to land on `target`.
    Returns (root piece, depth reached by the chain)."""
    pieces, free = [], []
    size = 0

    def add(piece):
        pieces.append(piece)
        free.append(piece.leaf_positions().shape[0])

    reached = 0
    if chain is not None:
        trees, deep = chain                         # deep[k] = (position, depth)
        k = int(rng.integers(0, len(trees)))
        root = cur = _Piece(trees[k])
        add(root)
        size = trees[k].shape[0]
        base = 0                                    # depth of cur's root
        while base + deep[k][1] < chain_depth:
            j = int(rng.integers(0, len(trees)))
            if size + trees[j].shape[0] - 1 > target:
                break
            nxt = _Piece(trees[j])
            cur.kids[int(deep[k][0])] = nxt
            free[-1] -= 1
            add(nxt)
            base += deep[k][1]
            cur, k, size = nxt, j, size + trees[j].shape[0] - 1
        reached = base + deep[k][1]
    else:
        need = target
        first = random_tree(rng, int(need)) if need <= donor_hi else pool[int(rng.integers(0, len(pool)))]
        root = _Piece(first)
        add(root)
        size = first.shape[0]
    while size < target:
        need = target - size + 1                    # odd: both sizes are odd
        dl = None
        if need <= donor_hi:
            d = random_tree(rng, int(need))
        else:
            k = int(rng.integers(0, len(pool)))
            d = pool[k]
            dl = pool_leaves[k] if pool_leaves is not None else None
        cum = np.cumsum(free)
        r = int(rng.integers(0, int(cum[-1])))
        j = int(np.searchsorted(cum, r, side="right"))
        host = pieces[j]
        leaves = host.leaf_positions()
        while True:
            pos = int(leaves[int(rng.integers(0, leaves.shape[0]))])
            if pos not in host.kids:
                break
        piece = _Piece(d, dl)
        host.kids[pos] = piece
        free[j] -= 1
        add(piece)
        size += d.shape[0] - 1
    return root, reached


def graft_population(seed: int = 4, count: int = 48, lo: int = 10**6, hi: int = 4 * 10**8,
                     donor_lo: int = 10**5, donor_hi: int = 10**6, n_donors: int = 32,
                     chain_depth: int = 10**5, chain_lo: int = 2 * 10**4, chain_hi: int = 10**5,
                     n_chain: int = 8):
    """Bloated trees: odd sizes log-uniform on [lo, hi], each grown by chains
    of subtree crossover from a pool of `n_donors` random trees (sizes
    log-uniform on [donor_lo, donor_hi]).  The largest tree first follows a
    chain of grafts at the deepest leaf (donors from a second pool, sizes
    [chain_lo, chain_hi]) until its depth reaches `chain_depth`, which makes
    it deep and stringy (no chain when chain_depth <= 0).  Returns (nodes,
    offsets, info) with info =
    {"sizes", "deep_tree", "chain_depth"}; the nodes array is written in
    place, so memory is one copy of the population."""
    rng = np.random.default_rng(seed)
    sizes = loguniform_sizes(rng, count, lo, hi)
    pool = [random_tree(rng, int(n)) for n in loguniform_sizes(rng, n_donors, donor_lo, donor_hi)]
    chain = None
    if chain_depth > 0:
        chain_trees = [random_tree(rng, int(n)) for n in loguniform_sizes(rng, n_chain, chain_lo, chain_hi)]
        chain = (chain_trees, [deepest_leaf(t) for t in chain_trees])
    pool_leaves = [np.flatnonzero(d >= LEAF_X) for d in pool]
    deep = int(np.argmax(sizes))
    offsets = np.zeros(count + 1, dtype=np.uint64)
    np.cumsum(sizes.astype(np.uint64), out=offsets[1:])
    nodes = np.empty(int(offsets[-1]), dtype=np.uint8)
    reached = 0
    for t in range(count):
        root, r = _graft_tree(rng, int(sizes[t]), pool, donor_hi,
                              chain if (t == deep and chain is not None) else None, chain_depth,
                              pool_leaves)
        end = _write_pieces(root, nodes, int(offsets[t]))
        assert end == int(offsets[t + 1])
        if t == deep:
            reached = r
    return nodes, offsets, {"sizes": sizes, "deep_tree": deep, "chain_depth": reached}


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
