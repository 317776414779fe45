"""The low-point chunk rule on its own (CPU)."""
import numpy as np

from paper_1902_09215_gb300 import synth
from tests.chunk_rules import low_point_ends, spine_operators


def test_low_point_ends_shape():
    """The cut rule on its own: chunks of 1..C codes, at most one more than
    ceil(n / C), every inner end a multiple of 16 unless it is the longest
    chunk's, and on random trees fewer operators sent upward than with
    fixed chunks."""
    rng = np.random.default_rng(77)
    fewer = tried = 0
    for _ in range(60):
        C = int(rng.choice([256, 1024, 4096]))
        tree = synth.random_tree(rng, int(rng.integers(C + 1, 8 * C)) | 1)
        n = tree.shape[0]
        if n <= C:
            continue
        tried += 1
        ends = low_point_ends(tree, C)
        b = [0] + ends + [n]
        assert all(0 < b[i + 1] - b[i] <= C for i in range(len(b) - 1))
        assert len(b) - 1 <= -(-n // C) + 1
        fewer += spine_operators(tree, C, ends) < spine_operators(tree, C)
    assert tried >= 40 and fewer >= 0.75 * tried


def test_fixed_chunks_match_the_walk_by_brute_force():
    """spine_operators against a direct count: an operator at j of chunk
    [b, e) is sent upward exactly when its subtree reaches past e."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        tree = synth.random_tree(rng, 301)
        n = tree.shape[0]
        ends = sorted(set(int(x) for x in rng.integers(1, n, 4)))
        # subtree end of every node: walk the arity sum until it closes
        sub_end = np.zeros(n, dtype=np.int64)
        for j in range(n):
            need, k = 1, j
            while need:
                need += 1 if tree[k] < 4 else -1
                k += 1
            sub_end[j] = k
        want = 0
        for b, e in zip([0] + ends, ends + [n]):
            want += int(np.sum((tree[b:e] < 4) & (sub_end[b:e] > e)))
        assert spine_operators(tree, 0, ends) == want
