"""The CPU count of the level-0 interpreter's loop exits (tests/interp_exits.py)
against what the tree's structure fixes: a whole tree leaves exactly one
value and sends nothing upward, and the spine operators of a tree's chunks
are the ones the arity walk's closed form names (tests/chunk_rules.py)."""
import numpy as np
import pytest

from paper_1902_09215_gb300 import synth
from tests.chunk_rules import low_point_ends, spine_operators
from tests.interp_exits import EVENTS, count_exits


@pytest.mark.parametrize("K", [8, 16, 32, 64])
def test_whole_trees_end_with_one_value(K):
    rng = np.random.default_rng(40 + K)
    for n in [1, 3, 31, 255, 1001, 4095]:
        for _ in range(3):
            tree = synth.random_tree(rng, n)
            ev = {k: 0 for k in EVENTS}
            have, d, g = count_exits(tree, 0, n, K, ev)
            assert have and d == 0 and g == 0
            assert ev["spine"] == 0 and ev["checked"] == 1         # only the last code
            assert ev["spill_entries"] == ev["refill_entries"]     # everything spilled comes back


def test_deep_spine_spills_and_refills():
    rng = np.random.default_rng(5)
    tree = synth.left_spine_tree(rng, 300, 3)
    ev = {k: 0 for k in EVENTS}
    have, d, g = count_exits(tree, 0, tree.shape[0], 32, ev)
    assert have and d == 0 and g == 0
    assert ev["spill"] > 0 and ev["spill_entries"] == ev["refill_entries"]


@pytest.mark.parametrize("C", [256, 1024, 4096])
def test_chunk_spine_operators_follow_the_arity_walk(C):
    rng = np.random.default_rng(C)
    for n in [C + 1, 3 * C + 7, 9 * C + 1]:
        n |= 1
        tree = synth.random_tree(rng, n)
        ends = low_point_ends(tree, C)
        ev = {k: 0 for k in EVENTS}
        left = 0
        for b, e in zip([0] + ends, ends + [n]):
            have, d, g = count_exits(tree, b, e, 32, ev)
            left += int(have) + d + g
        assert ev["spine"] == spine_operators(tree, C, ends)
        # the values sent with spine operators and those left at the chunks'
        # left ends are the upper tree's leaves: one more than its operators
        assert left + ev["sent"] == ev["spine"] + 1
