"""How the evaluator cuts trees into chunks, restated in plain numpy for the
tests: the arity walk, the operators a chunk sends to the upper tree, and
the low-point chunk ends of trees planned on the device."""
import numpy as np


def arity_walk(tree):
    """P[j]: open argument slots after reading the first j codes in prefix
    order (P[0] = 1; an operator adds one, a leaf takes one, Sec. 2.1)."""
    return np.concatenate([[1], 1 + np.cumsum(np.where(tree < 4, 1, -1))])


def spine_operators(tree, C, ends=None):
    """Operators a chunk cannot evaluate, summed over the chunks of one tree
    (chunks of C codes, or ending at `ends`): reading right to left from a
    chunk's right end, the stack of the whole tree at position j holds P[j]
    values; an operator at j lacks an argument inside the chunk exactly
    when P[j] is no higher than every P[k] for j < k <= the chunk's end,
    i.e. when the walk reaches its running minimum there."""
    n = tree.shape[0]
    if n <= C:
        return 0
    op = tree < 4
    P = arity_walk(tree)
    if ends is None:
        ends = list(range(C, n, C))
    total = 0
    for b, e in zip([0] + list(ends), list(ends) + [n]):
        run_min = np.minimum.accumulate(P[b + 1:e + 1][::-1])[::-1]   # min of P[j+1 .. e]
        total += int(np.sum(op[b:e] & (P[b:e] <= run_min)))
    return total


def low_point_ends(tree, C, max_chunks=32, window=512):
    """Chunk ends of a tree planned on the device: each next end is the
    multiple of 16 among the last `window` positions before the longest
    chunk (C codes) where the arity walk is lowest (the rightmost of
    equals), among the ends that leave the rest within the chunks still
    allowed (ceil(n / C) + 1 in all, at most max_chunks); none such: the
    longest chunk's end.  The tree starts 16-aligned."""
    n = tree.shape[0]
    P = arity_walk(tree)
    m = -(-n // C)
    cap = min(m + 1, max(m, max_chunks))
    a, j, ends = 0, 1, []
    while n - a > C:
        lo = max(a + 1, a + C - window if C > window else 0, n - (cap - j) * C)
        lo = (lo + 15) // 16 * 16
        hi = (a + C) // 16 * 16
        e = a + C
        if lo <= hi:
            cand = np.arange(lo, hi + 1, 16)
            v = P[cand]
            e = int(cand[len(v) - 1 - int(np.argmin(v[::-1]))])
        ends.append(e)
        a, j = e, j + 1
    return ends
