"""The sampled reconstruction of a generation (only the sampled children's
tournament entrants scored) equals the oracle's whole generation on the
same children: records, child bytes, per-case outputs, fitness and hits.
CPU only; it is what lets the GPU check a generation too large for the
oracle's whole-generation path."""
import numpy as np
import pytest

from paper_1902_09215_gb300 import synth
from tests.sampled_generation import expected_children


def whole_generation(oracle, nodes, offs, tables, seed, g, tsize=7):
    x, y, c = tables
    fit = oracle.eval_population(nodes, offs, x, y, c)["fitness"]
    sizes = np.diff(np.asarray(offs, dtype=np.int64)).astype(np.uint64)
    recs = oracle.generation_records(fit, sizes, sizes.shape[0], seed=seed, g=g, tsize=tsize)
    kids, koffs = oracle.crossover_population(nodes, offs, *recs)
    return recs, kids, koffs, oracle.eval_population(kids, koffs, x, y, c)


@pytest.mark.parametrize("g", [0, 3])
def test_sampled_children_equal_the_whole_generation(oracle, g):
    tables = synth.problem()
    nodes, offs = synth.population_loguniform(seed=31, count=300, lo=31, hi=20001)
    seed = 1234
    recs, kids, koffs, ref = whole_generation(oracle, nodes, offs, tables, seed, g)
    sample = [0, 1, 150, 299] + list(np.random.default_rng(g).choice(300, 6, replace=False))
    got = expected_children(oracle, nodes, offs, tables, seed, g, sample)
    for a, b in zip(got["records"], recs):
        assert np.array_equal(a.astype(np.uint64), b[sample].astype(np.uint64))
    for k, ch in enumerate(sample):
        mine = got["nodes"][int(got["offsets"][k]):int(got["offsets"][k + 1])]
        whole = kids[int(koffs[ch]):int(koffs[ch + 1])]
        assert np.array_equal(mine, whole), ch
    f = ref["fitness"][sample]
    assert np.array_equal(got["fitness"].view(np.uint32), f.view(np.uint32))
    assert np.array_equal(got["out"].view(np.uint32), ref["out"][sample].view(np.uint32))
    assert np.array_equal(got["hits"], ref["hits"][sample])


def test_entrants_are_scored_and_only_they(oracle):
    tables = synth.problem()
    nodes, offs = synth.population_loguniform(seed=32, count=500, lo=31, hi=2001)
    got = expected_children(oracle, nodes, offs, tables, 77, 0, [7])
    assert 1 <= got["parents"].shape[0] <= 14        # two tournaments of seven
    x, y, c = tables
    full = oracle.eval_population(nodes, offs, x, y, c)["fitness"]
    assert np.array_equal(got["parent_fitness"].view(np.uint32), full[got["parents"]].view(np.uint32))
    mum, dad = int(got["records"][0][0]), int(got["records"][1][0])
    assert mum in set(got["parents"].tolist()) and dad in set(got["parents"].tolist())
