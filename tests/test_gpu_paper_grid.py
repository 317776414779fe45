"""The paper's constant table (Sec. 2.1, Table gp.details: 250 constants on
the 0.001 grid) on the GPU: leaf codes up to 254, which also travel through
upper-tree levels as leaves (value entries start at code 256).  Bit-exact
against the oracle for whole trees, chunked trees at several chunk sizes,
the allocation-free path and one device-made generation."""
import os

import numpy as np
import pytest

from paper_1902_09215_gb300 import synth
from tests.gpu_util import first_mismatch, gpu, same_f32  # noqa: F401

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1


def grid_problem(gp):
    x, y, _ = synth.problem()
    c = synth.paper_grid_constants()
    return x, y, c, gp.Problem(x, y, c)


def check(vals, fit, hits, ref):
    assert same_f32(vals, ref["out"]), first_mismatch(vals, ref["out"])
    assert same_f32(fit, ref["fitness"]), first_mismatch(fit, ref["fitness"])
    assert np.array_equal(hits, ref["hits"])


@pytest.mark.parametrize("chunk", [0, 64, 256, 1024])
def test_grid_constants_through_levels(gpu, oracle, chunk):
    x, y, c, prob = grid_problem(gpu)
    nodes, offs = synth.paper_grid_population()
    assert nodes.max() > 131                       # codes beyond the default table
    ref = oracle.eval_population(nodes, offs, x, y, c, n_threads=THREADS)
    pop = gpu.gp_create_population(prob, nodes, offs)
    gpu.gp_evaluate(pop, chunk_nodes=chunk)
    fit, vals, hits = gpu.gp_fitness(pop, case_values=True, hits=True)
    check(vals, fit, hits, ref)
    if chunk == 64:
        assert gpu.gp_eval_stats_get(pop)["levels"] >= 3


def test_grid_constants_code_255_rejected(gpu):
    _, _, _, prob = grid_problem(gpu)
    nodes, offs = synth.pack([np.array([0, 4, 255], np.uint8)])
    with pytest.raises(gpu.GpError) as e:
        gpu.gp_create_population(prob, nodes, offs)
    assert e.value.status == gpu.GP_EMALFORMED


def test_grid_constants_noalloc_and_generation(gpu, oracle):
    import torch
    x, y, c, prob = grid_problem(gpu)
    nodes, offs = synth.paper_grid_population(seed=13, count=200, hi=4095)
    ref = oracle.eval_population(nodes, offs, x, y, c, n_threads=THREADS)
    total = int(offs[-1])
    d_nodes = torch.zeros((total + 15) // 16 * 16 + 16, dtype=torch.uint8, device="cuda")
    d_nodes[:total] = torch.from_numpy(nodes).to("cuda")
    n = offs.shape[0] - 1
    d_fit = torch.empty(n, dtype=torch.float32, device="cuda")
    d_vals = torch.empty((n, 48), dtype=torch.float32, device="cuda")
    d_hits = torch.empty(n, dtype=torch.int32, device="cuda")
    gpu.gp_evaluate_noalloc(prob, offs, d_nodes.data_ptr(), d_fit.data_ptr(), d_vals.data_ptr(), d_hits.data_ptr())
    torch.cuda.synchronize()
    check(d_vals.cpu().numpy(), d_fit.cpu().numpy(), d_hits.cpu().numpy().astype(np.uint32), ref)
    # one generation on the device
    G = gpu.gp_generation_create(prob, nodes, offs, seed=4, chunk_nodes=256)
    gpu.gp_generation_step(G)
    sizes = np.diff(offs.astype(np.int64)).astype(np.uint64)
    recs = oracle.generation_records(ref["fitness"], sizes, n, seed=4, g=0)
    kn, ko = oracle.crossover_population(nodes, offs, *recs)
    gn, go = gpu.gp_generation_trees(G)
    assert np.array_equal(gn, kn) and np.array_equal(go, ko)
    fit, vals, hits = gpu.gp_generation_fitness(G, case_values=True, hits=True)
    check(vals, fit, hits, oracle.eval_population(kn, ko, x, y, c, n_threads=THREADS))
