"""GPU parity of one device generation at the batched workloads' sizes, on
sampled children: 4000 parents of 1e2..1e6 nodes (reduced) or 1e2..1e8
nodes (full, 2.9e10 nodes), size-7 tournaments, 4000 crossovers, the
children evaluated on the device.  For the sampled children the records,
the child bytes, the per-case outputs, fitness and hits are compared with
the oracle's (tests/sampled_generation.py: only the sampled children's
tournament entrants are scored), and the device's fitness of those entrants
with the oracle's.  The full size builds 29 GB of parents on the host and
takes about two minutes; the reduced size a few seconds."""
import os

import numpy as np
import pytest

from paper_1902_09215_gb300 import synth
from tests.gpu_util import first_mismatch, gpu, same_f32  # noqa: F401
from tests.sampled_generation import expected_children

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

THREADS = os.cpu_count() or 1

SIZES = {
    "reduced": dict(seed=5, count=4000, lo=100, hi=10**6, donor_lo=10**4, donor_hi=10**5, n_donors=32,
                    chain_depth=0),
    "full": dict(seed=5, count=4000, lo=100, hi=10**8, donor_lo=10**5, donor_hi=10**6, n_donors=32,
                 chain_depth=0),
}


@pytest.mark.parametrize("size", ["reduced", "full"])
def test_batched_generation_sampled_children(gpu, oracle, size):
    tables = synth.problem()
    x, y, c = tables
    nodes, offs = synth.graft_population(**SIZES[size])[:2]
    sizes = np.diff(offs.astype(np.int64))
    used = int(np.sum((sizes + 15) // 16 * 16)) + 64
    seed = 21
    G = gpu.gp_generation_create(gpu.Problem(x, y, c), nodes, offs, seed=seed,
                                 arena_bytes=int(used * 1.3) + (64 << 20), use_graph=True)
    parent_fit, _, _ = gpu.gp_generation_fitness(G)
    gpu.gp_generation_step(G)
    rng = np.random.default_rng(7)
    sample = sorted({0, 3999} | set(rng.choice(4000, 8, replace=False).tolist()))
    want = expected_children(oracle, nodes, offs, tables, seed, 0, sample, n_threads=THREADS)
    # the device scored the sampled tournaments' entrants as the oracle did
    assert same_f32(parent_fit[want["parents"]], want["parent_fitness"])
    recs = gpu.gp_generation_records(G)
    for got, exp, name in zip(recs, want["records"], ("mum", "dad", "mum_point", "dad_point")):
        assert np.array_equal(got[sample].astype(np.uint64), exp.astype(np.uint64)), name
    for k, ch in enumerate(sample):
        exp = want["nodes"][int(want["offsets"][k]):int(want["offsets"][k + 1])]
        assert np.array_equal(gpu.gp_generation_tree_read(G, ch), exp), ch
    fit, vals, hits = gpu.gp_generation_fitness(G, case_values=True, hits=True)
    assert same_f32(vals[sample], want["out"]), first_mismatch(vals[sample], want["out"])
    assert same_f32(fit[sample], want["fitness"]), first_mismatch(fit[sample], want["fitness"])
    assert np.array_equal(hits[sample], want["hits"])
    gpu.gp_generation_destroy(G)
