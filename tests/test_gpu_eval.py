"""GPU parity: libgp's evaluator (through the C ABI) against the CPU oracle,
bit-exact per case, per fitness and per hit count."""
import numpy as np
import pytest

from paper_1902_09215_gb300 import synth
from tests.chunk_rules import low_point_ends, spine_operators
from tests.gpu_util import first_mismatch, gpu, same_f32  # noqa: F401

pytestmark = pytest.mark.gpu


def run_gpu(gp, nodes, offs, x, y, c, div0=1.0, **opt):
    import torch
    s = torch.cuda.current_stream()
    prob = gp.Problem(x, y, c, protected_div_value=div0)
    pop = gp.gp_create_population(prob, nodes, offs, s)
    gp.gp_evaluate(pop, s, **opt)
    fit, vals, hits = gp.gp_fitness(pop, case_values=True, hits=True)
    stats = gp.gp_eval_stats_get(pop)
    gp.gp_destroy_population(pop)
    return fit, vals, hits, stats


def check(gp, oracle, nodes, offs, x, y, c, div0=1.0, **opt):
    fit, vals, hits, stats = run_gpu(gp, nodes, offs, x, y, c, div0, **opt)
    ref = oracle.eval_population(nodes, offs, x, y, c, div0=div0, n_threads=8)
    assert same_f32(vals, ref["out"]), first_mismatch(vals, ref["out"])
    assert same_f32(fit, ref["fitness"]), first_mismatch(fit, ref["fitness"])
    assert np.array_equal(hits, ref["hits"])
    return stats


def test_smallest_workload_50_trees(gpu, oracle):
    x, y, c = synth.problem()
    nodes, offs = synth.population_small(seed=1)
    st = check(gpu, oracle, nodes, offs, x, y, c)
    assert st["levels"] == 1


def test_population_4000_loguniform_full(gpu, oracle):
    x, y, c = synth.problem()
    nodes, offs = synth.population_loguniform(seed=3)
    st = check(gpu, oracle, nodes, offs, x, y, c)
    assert st["levels"] == 2          # trees above one chunk go through an upper level


@pytest.mark.parametrize("chunk", [64, 256, 1024, 4096, 32768])
def test_chunking_levels_bit_exact(gpu, oracle, chunk):
    """Small chunks force several upper-tree levels; results must not change."""
    x, y, c = synth.problem()
    rng = np.random.default_rng(42)
    sizes = synth.loguniform_sizes(rng, 60, 31, 60001)
    trees = [synth.random_tree(rng, int(n)) for n in sizes]
    nodes, offs = synth.pack(trees)
    st = check(gpu, oracle, nodes, offs, x, y, c, chunk_nodes=chunk)
    if chunk <= 256:
        assert st["levels"] >= 3


@pytest.mark.parametrize("warps,window", [(32, 32), (16, 64), (8, 48), (24, 16), (4, 256), (1, 64)])
def test_launch_shapes(gpu, oracle, warps, window):
    x, y, c = synth.problem()
    nodes, offs = synth.population_loguniform(seed=13, count=300, lo=31, hi=20001)
    check(gpu, oracle, nodes, offs, x, y, c, chunk_nodes=2048, warps_per_cta=warps,
          window_entries=window)


@pytest.mark.parametrize("chunk", [128, 4096])
def test_deep_stacks_spill(gpu, oracle, chunk):
    """Left spines keep thousands of values on the operand stack (spill to
    global memory), alone and cut into chunks."""
    x, y, c = synth.problem()
    rng = np.random.default_rng(7)
    trees = [synth.left_spine_tree(rng, d, h) for d, h in [(300, 3), (2000, 1), (1500, 5), (40, 31)]]
    trees.append(synth.random_tree(rng, 4095))
    nodes, offs = synth.pack(trees)
    check(gpu, oracle, nodes, offs, x, y, c, chunk_nodes=chunk)


def test_chunk_boundary_sizes(gpu, oracle):
    x, y, c = synth.problem()
    rng = np.random.default_rng(99)
    sizes = [1, 3, 15, 17, 31, 33, 1023, 1025, 4095, 4097, 8191, 8193, 12289]
    nodes, offs = synth.pack([synth.random_tree(rng, n) for n in sizes])
    for chunk in (16 * 64, 4096):
        check(gpu, oracle, nodes, offs, x, y, c, chunk_nodes=chunk)


def test_special_values_and_protected_division(gpu, oracle):
    """Zeros of both signs, subnormals, NaN and infinities in the constant
    table; division-heavy trees produce protected results, overflow, NaN."""
    x, y, _ = synth.problem()
    table = np.array([0.0, -0.0, 1e-45, -3e-39, np.nan, np.inf, -np.inf, 1e30, -1e-30, 0.5, 3.0],
                     np.float32)
    rng = np.random.default_rng(5)
    trees = []
    for n in [3, 5, 7, 15, 63, 255, 1023, 5001]:
        for ops in [(3,), (1, 3), (2, 3), (0, 1, 2, 3)]:
            trees.append(synth.random_tree(rng, n, p_x=0.2, n_consts=len(table), ops=ops))
    nodes, offs = synth.pack(trees)
    for div0 in (1.0, -0.0, 0.25):
        check(gpu, oracle, nodes, offs, x, y, table, div0=div0, chunk_nodes=1024)


@pytest.mark.parametrize("n_cases", [1, 2, 7, 16, 17, 33, 47, 48, 63, 64])
def test_case_counts(gpu, oracle, n_cases):
    x = synth.cases(n_cases)
    y = synth.sextic_targets_f32(x)
    c = synth.constants(2)
    nodes, offs = synth.population_loguniform(seed=17, count=80, lo=1, hi=9001)
    check(gpu, oracle, nodes, offs, x, y, c, chunk_nodes=1024)


def test_sextic_tree_zero_fitness(gpu, oracle):
    x, y, c = synth.problem()
    one = [3, 4, 4]
    t = [2, 2, 2, 2, 2, 4, 4] + [1, 4] + one + [1, 4] + one + [0, 4] + one + [0, 4] + one
    nodes, offs = synth.pack([np.array(t, np.uint8)] * 3)
    fit, vals, hits, _ = run_gpu(gpu, nodes, offs, x, y, c)
    assert np.all(fit.view(np.uint32) == 0) and np.all(hits == 48)
    assert same_f32(vals[0], y)


def test_empty_population(gpu):
    x, y, c = synth.problem()
    prob = gpu.Problem(x, y, c)
    pop = gpu.gp_create_population(prob, np.zeros(0, np.uint8), np.zeros(1, np.uint64))
    gpu.gp_evaluate(pop)
    fit, _, _ = gpu.gp_fitness(pop)
    assert fit.shape == (0,)


@pytest.mark.parametrize("bad", ["truncated", "extra", "code", "leaf_first"])
def test_malformed_upload_rejected(gpu, bad):
    x, y, c = synth.problem()
    rng = np.random.default_rng(1)
    good = synth.random_tree(rng, 41)
    t = {"truncated": good[:-1], "extra": np.concatenate([good, [4]]),
         "code": np.concatenate([good[:-1], [200]]), "leaf_first": np.array([4, 0, 4, 4], np.uint8)}[bad]
    nodes, offs = synth.pack([synth.random_tree(rng, 9), t, synth.random_tree(rng, 5)])
    with pytest.raises(gpu.GpError) as e:
        gpu.gp_create_population(gpu.Problem(x, y, c), nodes, offs)
    assert e.value.status == gpu.GP_EMALFORMED


def test_invalid_arguments(gpu):
    x, y, c = synth.problem()
    with pytest.raises(gpu.GpError) as e:
        gpu.gp_create_population(gpu.Problem(x, y, c), np.array([4], np.uint8),
                                 np.array([0, 1, 1], np.uint64))
    assert e.value.status == gpu.GP_EINVAL
    pop = gpu.gp_create_population(gpu.Problem(x, y, c), np.array([4], np.uint8), np.array([0, 1], np.uint64))
    with pytest.raises(gpu.GpError):
        gpu.gp_fitness(pop)           # not evaluated yet
    with pytest.raises(gpu.GpError):
        gpu.gp_evaluate(pop, chunk_nodes=100)   # not a multiple of 16


def test_budget_admission(gpu):
    x, y, c = synth.problem()
    nodes, offs = synth.population_small()
    with pytest.raises(gpu.GpError) as e:
        gpu.gp_create_population(gpu.Problem(x, y, c, hbm_budget_bytes=1000), nodes, offs)
    assert e.value.status == gpu.GP_ENOMEM


def test_repeat_evaluation_is_deterministic(gpu):
    x, y, c = synth.problem()
    nodes, offs = synth.population_loguniform(seed=5, count=500, hi=20001)
    prob = gpu.Problem(x, y, c)
    pop = gpu.gp_create_population(prob, nodes, offs)
    outs = []
    for chunk in (0, 512, 0):
        gpu.gp_evaluate(pop, chunk_nodes=chunk)
        outs.append(gpu.gp_fitness(pop, case_values=True))
    for f, v, _ in outs[1:]:
        assert same_f32(f, outs[0][0]) and same_f32(v, outs[0][1])


@pytest.mark.parametrize("C", [1024, 4096, 8192])
def test_operators_sent_upward_follow_the_arity_walk(gpu, oracle, C):
    """The count of operators evaluated above level 0 (gp_eval_stats) equals
    the spine operators of every chunk, for an uploaded population (levels
    planned on the host) and for crossover children (planned on the device),
    and the results stay exact."""
    import torch
    s = torch.cuda.current_stream()
    x, y, c = synth.problem()
    prob = gpu.Problem(x, y, c)
    nodes, offs = synth.population_loguniform(seed=23, count=60, lo=31, hi=60001)
    trees = [nodes[int(offs[i]):int(offs[i + 1])] for i in range(60)]
    st = check(gpu, oracle, nodes, offs, x, y, c, chunk_nodes=C)
    assert st["upper_ops"] == sum(spine_operators(t, C) for t in trees) > 0
    pop = gpu.gp_create_population(prob, nodes, offs, s)
    sizes = np.diff(offs.astype(np.int64))
    mum, dad, mp, dp = synth.crossover_points(31, sizes, 60)
    kids = gpu.gp_crossover(pop, (mum, dad, mp, dp), s)
    gpu.gp_evaluate(kids, s, chunk_nodes=C)
    fit, _, _ = gpu.gp_fitness(kids)
    kn, ko = oracle.crossover_population(nodes, offs, mum, dad, mp, dp)
    assert same_f32(fit, oracle.eval_population(kn, ko, x, y, c, n_threads=8)["fitness"])
    kt = [kn[int(ko[i]):int(ko[i + 1])] for i in range(60)]
    # children whose size bounds stay within 32 chunks are planned on the
    # device, where chunks end at low points of the arity walk
    bound = sizes[mum] + sizes[dad] - dp.astype(np.int64) - 1
    if bound.max() <= 32 * C:
        want = sum(spine_operators(t, C, low_point_ends(t, C)) for t in kt)
    else:
        want = sum(spine_operators(t, C) for t in kt)
    assert gpu.gp_eval_stats_get(kids)["upper_ops"] == want


def test_slot_overflow_is_evaluated_again_in_gp_fitness(gpu, oracle):
    """Left-spine trees whose chunks leave more complete subtrees on the
    stack than a fused chunk's slot holds (a slot keeps max(128, C/8) value
    entries): gp_evaluate queues them, gp_fitness evaluates them again
    through planned levels (redone > 0), and every result equals the
    oracle's; for uploaded trees and for crossover children sized on the
    device (mum point 0 and dad point 0 copy the dad whole)."""
    import torch
    s = torch.cuda.current_stream()
    x, y, c = synth.problem()
    prob = gpu.Problem(x, y, c)
    rng = np.random.default_rng(17)
    trees = [synth.left_spine_tree(rng, 3000, 3) for _ in range(3)] + \
        [synth.random_tree(rng, int(n)) for n in (31, 4095, 9001, 20001)]
    nodes, offs = synth.pack(trees)
    ref = oracle.eval_population(nodes, offs, x, y, c, n_threads=8)
    st = check(gpu, oracle, nodes, offs, x, y, c, chunk_nodes=4096)
    assert st["redone"] >= 3
    pop = gpu.gp_create_population(prob, nodes, offs, s)
    n = len(trees)
    idx = np.arange(n, dtype=np.uint32)
    zero = np.zeros(n, np.uint64)
    kids = gpu.gp_crossover(pop, (idx, idx, zero, zero), s)
    gpu.gp_evaluate(kids, s, chunk_nodes=4096)
    fit, vals, hits = gpu.gp_fitness(kids, case_values=True, hits=True)
    assert gpu.gp_eval_stats_get(kids)["redone"] >= 3
    assert same_f32(vals, ref["out"]), first_mismatch(vals, ref["out"])
    assert same_f32(fit, ref["fitness"])
    assert np.array_equal(hits, ref["hits"])
