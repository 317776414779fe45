"""The sharded population on CPU: two and three gloo ranks, each holding a
node-balanced range of the trees, make two generations (fitness and sizes
all-gathered, children selected per rank from the counter-based draws,
parents fetched from their owners by all-to-all, children made and
evaluated per rank), and the population they end with equals, tree for
tree and bit for bit, the one a single process makes with the oracle.
The ranks' work is done by the oracle here (a backend with the interface
of `shard.LibgpBackend`); the GPU tests cover libgp's selection, crossover
and evaluation against the same oracle."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SEED, GENERATIONS = 404, 2


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleBackend:
    """A rank's trees on the host, its work done by the oracle."""

    def __init__(self, oracle, tables, nodes, offs):
        self.o, self.tables = oracle, tables
        self._set(nodes, offs)

    def _set(self, nodes, offs):
        self.nodes, self.offs = nodes, np.asarray(offs, np.uint64)
        self.sizes = np.diff(self.offs.astype(np.int64)).astype(np.uint64)
        self.fit = self.o.eval_population(nodes, self.offs, *self.tables)["fitness"]

    def fitness(self):
        return self.fit

    def select(self, fit_all, size_all, seed, g, lo, n, tsize):
        recs = self.o.generation_records(fit_all, size_all, lo + n, seed=seed, g=g, tsize=tsize)
        return tuple(np.asarray(r)[lo:lo + n] for r in recs)

    def read_trees(self, idx):
        parts = [self.nodes[int(self.offs[t]):int(self.offs[t + 1])] for t in idx]
        sizes = np.array([p.shape[0] for p in parts], dtype=np.uint64)
        return (np.concatenate(parts) if parts else np.zeros(0, np.uint8)), sizes

    def replace(self, pool_nodes, pool_offs, mum, dad, mp, dp):
        self._set(*self.o.crossover_population(pool_nodes, pool_offs, mum, dad, mp, dp))


def population():
    from paper_1902_09215_gb300 import synth
    return synth.population_loguniform(seed=41, count=150, lo=31, hi=3001)


def rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as O
    from paper_1902_09215_gb300 import shard, synth
    O.build()
    nodes, offs = population()
    ranges = shard.balanced_ranges(np.diff(offs.astype(np.int64)), world)
    lo, hi = ranges[rank]
    sub = synth.pack([nodes[int(offs[t]):int(offs[t + 1])] for t in range(lo, hi)])
    sp = shard.ShardedPopulation(OracleBackend(O, synth.problem(), *sub), ranges, rank, world, SEED)
    for _ in range(GENERATIONS):
        sp.step()
    mine = (rank, sp.b.nodes.tobytes(), sp.b.offs.tolist(), np.asarray(sp.b.fit, np.float32).tobytes())
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    if rank == 0:
        out.put(gathered)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_generations_equal_one_process(world, oracle):
    from paper_1902_09215_gb300 import synth
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    gathered = out.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # one process: the oracle's whole generations
    x, y, c = synth.problem()
    nodes, offs = population()
    fit = oracle.eval_population(nodes, offs, x, y, c)["fitness"]
    for g in range(GENERATIONS):
        sizes = np.diff(offs.astype(np.int64)).astype(np.uint64)
        recs = oracle.generation_records(fit, sizes, sizes.shape[0], seed=SEED, g=g)
        nodes, offs = oracle.crossover_population(nodes, offs, *recs)
        fit = oracle.eval_population(nodes, offs, x, y, c)["fitness"]
    got_nodes, got_sizes, got_fit = [], [], []
    for rank, nb, of, fb in sorted(gathered):
        of = np.asarray(of, np.uint64)
        got_nodes.append(np.frombuffer(nb, np.uint8))
        got_sizes.append(np.diff(of.astype(np.int64)))
        got_fit.append(np.frombuffer(fb, np.float32))
    assert np.array_equal(np.concatenate(got_nodes), nodes)
    assert np.array_equal(np.concatenate(got_sizes), np.diff(offs.astype(np.int64)))
    want = np.asarray(fit, np.float32)
    got = np.concatenate(got_fit)
    assert np.all((got.view(np.uint32) == want.view(np.uint32)) | (np.isnan(got) & np.isnan(want)))


def test_balanced_ranges_and_owners():
    from paper_1902_09215_gb300 import shard
    sizes = np.array([10, 10, 10, 10, 1000, 10, 10, 10])
    r = shard.balanced_ranges(sizes, 2)
    assert r[0][0] == 0 and r[-1][1] == 8 and r[0][1] == r[1][0]
    assert r == [(0, 4), (4, 8)]                  # the big tree starts the second half
    assert shard.balanced_ranges(np.ones(10), 5) == [(0, 2), (2, 4), (4, 6), (6, 8), (8, 10)]
    assert shard.balanced_ranges(np.ones(2), 3)[-1][1] == 2       # more ranks than trees
    assert list(shard.owner_of([(0, 4), (4, 8)], [0, 3, 4, 7])) == [0, 0, 1, 1]
