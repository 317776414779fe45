"""The sharded population's GPU backend (shard.LibgpBackend: gp_select,
reading trees, gp_crossover on the fetched parents, gp_evaluate) driven by
the sharding loop on one rank: its generations equal the ones a
gp_generation makes on the device from the same trees and seed (bytes and
fitness), which the generation tests pin to the oracle."""
import socket

import numpy as np
import pytest

from paper_1902_09215_gb300 import synth
from tests.gpu_util import gpu, same_f32  # noqa: F401

pytestmark = pytest.mark.gpu


def test_one_rank_sharded_generations_equal_device_generations(gpu):
    import torch.distributed as dist
    from paper_1902_09215_gb300 import shard
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        x, y, c = synth.problem()
        prob = gpu.Problem(x, y, c)
        nodes, offs = synth.population_loguniform(seed=43, count=300, lo=31, hi=20001)
        seed = 515
        sp = shard.ShardedPopulation(shard.LibgpBackend(gpu, prob, nodes, offs, chunk_nodes=4096),
                                     shard.balanced_ranges(np.diff(offs.astype(np.int64)), 1), 0, 1, seed)
        G = gpu.gp_generation_create(prob, nodes, offs, seed=seed, chunk_nodes=4096)
        for g in range(3):
            sp.step()
            gpu.gp_generation_step(G)
            gn, go = gpu.gp_generation_trees(G)
            sn, so = gpu.read_all_trees(sp.b.pop)
            assert np.array_equal(so, go) and np.array_equal(sn, gn), g
            assert same_f32(sp.b.fitness(), gpu.gp_generation_fitness(G)[0]), g
        gpu.gp_generation_destroy(G)
    finally:
        dist.destroy_process_group()
