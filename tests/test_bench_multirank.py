"""The multi-GPU path of bench.py on CPU: two gloo ranks agree on the
slowest rank's time, the job's throughput counts every rank's units over
that time, and every rank works on its own population (weak scaling,
independent replicas: no data-path collective)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import importlib.util
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    mine = 10.0 + 7.5 * rank                       # rank 1 is the slower one
    m = bench.max_over_ranks(mine, world, "cpu")
    v = bench.weak_scaling_value(1e9, world, m)
    _, _, _, nodes, offs, _ = bench.make_workload(rank)
    out.put((rank, m, v, int(offs[-1]), int(nodes[:4096].astype(np.int64).sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, v0, n0, h0), (r1, m1, v1, n1, h1) = res
    assert m0 == m1 == pytest.approx(17.5)          # both see the slowest rank
    assert v0 == v1 == pytest.approx(2 * 1e9 / 0.0175)
    assert (n0, h0) != (n1, h1)                     # independent populations per rank
