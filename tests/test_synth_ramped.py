"""Ramped half-and-half initial populations (Table gp.details: depths 2..6):
valid prefix trees; full trees are complete binary trees of their depth;
grow trees stay within it; depths and methods are spread evenly; seeded."""
import numpy as np

from paper_1902_09215_gb300 import synth


def trees_of(nodes, offs):
    return [nodes[int(offs[i]):int(offs[i + 1])] for i in range(offs.shape[0] - 1)]


def test_ramped_half_and_half_shapes(oracle):
    nodes, offs = synth.ramped_half_and_half(seed=1, count=400)
    ts = trees_of(nodes, offs)
    depths = list(range(2, 7))
    for i, t in enumerate(ts):
        assert oracle.check_tree(t)
        d = depths[i % 5]
        full = (i // 5) % 2 == 0
        depth = oracle.tree_depth(t) - 1            # the oracle counts nodes on the path
        assert t[0] < 4                              # an operator at the root
        if full:
            assert t.shape[0] == 2 ** (d + 1) - 1 and depth == d
        else:
            assert 1 <= depth <= d
    grow = [t for i, t in enumerate(ts) if (i // 5) % 2 == 1]
    full = [t for i, t in enumerate(ts) if (i // 5) % 2 == 0]
    assert np.mean([t.shape[0] for t in grow]) < np.mean([t.shape[0] for t in full])


def test_ramped_leaf_and_operator_mix():
    nodes, _ = synth.ramped_half_and_half(seed=2, count=4000)
    ops = nodes[nodes < 4]
    leaves = nodes[nodes >= 4]
    assert abs(np.mean(leaves == synth.LEAF_X) - 0.5) < 0.02
    counts = np.bincount(ops, minlength=4) / ops.size
    assert np.all(np.abs(counts - 0.25) < 0.02)


def test_ramped_deterministic():
    a = synth.ramped_half_and_half(seed=3, count=100)
    b = synth.ramped_half_and_half(seed=3, count=100)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
