"""The bloated-tree generator (chains of subtree crossover): every tree is a
valid prefix tree of exactly its drawn size, the chained tree is as deep as
asked, and the output depends only on the seed."""
import numpy as np

from paper_1902_09215_gb300 import synth

TINY = dict(seed=4, count=6, lo=10**3, hi=10**5, donor_lo=10**2, donor_hi=10**3, n_donors=8,
            chain_depth=500, chain_lo=100, chain_hi=300, n_chain=4)


def test_graft_population_valid_exact_sizes(oracle):
    nodes, offs, info = synth.graft_population(**TINY)
    sizes = np.diff(offs.astype(np.int64))
    assert np.array_equal(sizes, info["sizes"])
    assert sizes.min() >= TINY["lo"] and sizes.max() <= TINY["hi"] and np.all(sizes % 2 == 1)
    for t in range(TINY["count"]):
        assert oracle.check_tree(nodes[int(offs[t]):int(offs[t + 1])])


def test_graft_population_chain_depth(oracle):
    nodes, offs, info = synth.graft_population(**TINY)
    d = info["deep_tree"]
    assert d == int(np.argmax(info["sizes"]))
    assert info["chain_depth"] >= TINY["chain_depth"]
    assert oracle.tree_depth(nodes[int(offs[d]):int(offs[d + 1])]) - 1 >= info["chain_depth"]


def test_graft_population_deterministic():
    a = synth.graft_population(**TINY)
    b = synth.graft_population(**TINY)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    c = synth.graft_population(**dict(TINY, seed=5))
    assert not np.array_equal(a[0][:1000], c[0][:1000])


def test_deepest_leaf_matches_depth(oracle):
    """deepest_leaf counts edges from the root; the oracle's depth counts
    nodes on the longest root-to-leaf path."""
    rng = np.random.default_rng(12)
    for n in (1, 3, 5, 31, 1001):
        t = synth.random_tree(rng, n)
        pos, d = synth.deepest_leaf(t)
        assert t[pos] >= synth.LEAF_X
        assert d == oracle.tree_depth(t) - 1
