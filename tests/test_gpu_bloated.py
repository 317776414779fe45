"""GPU parity on bloated trees built by chains of subtree crossover: 48
trees with sizes log-uniform 1e6..4e8 nodes at full size, the largest one
first grafted at its deepest leaf until its depth passes 1e5 (so its
operand stack spills).  Exercises the planned multi-level evaluation of
trees far larger than a chunk and 64-bit node positions (the population
holds more than 2^32 nodes).  Bit-exact against the FP32 oracle, every
tree, every case."""
import os

import numpy as np
import pytest

from paper_1902_09215_gb300 import synth
from tests.gpu_util import first_mismatch, gpu, same_f32  # noqa: F401

pytestmark = pytest.mark.gpu

SCALED = dict(seed=4, count=48, lo=10**4, hi=4 * 10**6, donor_lo=10**3, donor_hi=10**4, n_donors=16,
              chain_depth=10**4, chain_lo=2000, chain_hi=5000, n_chain=8)


def check_population(gp, oracle, nodes, offs, **opt):
    import torch
    x, y, c = synth.problem()
    ref = oracle.eval_population(nodes, offs, x, y, c, n_threads=os.cpu_count() or 1)
    s = torch.cuda.current_stream()
    prob = gp.Problem(x, y, c)
    pop = gp.gp_create_population(prob, nodes, offs, s)
    gp.gp_evaluate(pop, s, **opt)
    fit, vals, hits = gp.gp_fitness(pop, case_values=True, hits=True)
    stats = gp.gp_eval_stats_get(pop)
    gp.gp_destroy_population(pop)
    assert same_f32(vals, ref["out"]), first_mismatch(vals, ref["out"])
    assert same_f32(fit, ref["fitness"]), first_mismatch(fit, ref["fitness"])
    assert np.array_equal(hits, ref["hits"])
    return stats


def test_bloated_population_scaled(gpu, oracle):
    """1/100 of the full sizes: trees 1e4..4e6 nodes, chained depth 1e4."""
    nodes, offs, info = synth.graft_population(**SCALED)
    stats = check_population(gpu, oracle, nodes, offs)
    assert stats["levels"] >= 2


def test_bloated_population_scaled_small_chunks(gpu, oracle):
    """Same trees with 1024-node chunks: more levels of upper trees."""
    nodes, offs, info = synth.graft_population(**SCALED)
    stats = check_population(gpu, oracle, nodes, offs, chunk_nodes=1024)
    assert stats["levels"] >= 3


@pytest.mark.slow
def test_bloated_population_full_size(gpu, oracle):
    """48 trees, 1e6..4e8 nodes (about 4.5e9 in all), depth above 1e5."""
    nodes, offs, info = synth.graft_population()
    assert int(offs[-1]) > (1 << 32)
    assert info["chain_depth"] >= 10**5
    check_population(gpu, oracle, nodes, offs)
