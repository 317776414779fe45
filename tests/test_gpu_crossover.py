"""GPU parity for subtree crossover (Sec. 3.1): children byte-identical to
the oracle's three-segment copy."""
import numpy as np
import pytest

from paper_1902_09215_gb300 import synth
from tests.gpu_util import gpu, same_f32  # noqa: F401

pytestmark = pytest.mark.gpu


def make_pop(gp, nodes, offs, **kw):
    x, y, c = synth.problem()
    return gp.gp_create_population(gp.Problem(x, y, c, **kw), nodes, offs)


def test_crossover_population_4000(gpu, oracle):
    nodes, offs = synth.population_loguniform(seed=3)
    pop = make_pop(gpu, nodes, offs)
    sizes = np.diff(offs.astype(np.int64))
    ops = synth.crossover_points(11, sizes, 4000)
    kids = gpu.gp_crossover(pop, ops)
    kn, ko = gpu.read_all_trees(kids)
    rn, ro = oracle.crossover_population(nodes, offs, *ops)
    assert np.array_equal(ko, ro)
    assert np.array_equal(kn, rn)


def test_crossover_edge_points(gpu, oracle):
    rng = np.random.default_rng(3)
    trees = [synth.random_tree(rng, n) for n in (1, 3, 31, 1001, 20001)]
    nodes, offs = synth.pack(trees)
    pop = make_pop(gpu, nodes, offs)
    sizes = np.diff(offs.astype(np.int64))
    recs = []
    for a in range(len(trees)):
        for b in range(len(trees)):
            for i in {0, int(sizes[a]) - 1, int(sizes[a]) // 2}:
                for j in {0, int(sizes[b]) - 1, int(sizes[b]) // 3}:
                    recs.append((a, b, i, j))
    ops = tuple(np.array(v) for v in zip(*recs))
    kids = gpu.gp_crossover(pop, ops)
    kn, ko = gpu.read_all_trees(kids)
    rn, ro = oracle.crossover_population(nodes, offs, *ops)
    assert np.array_equal(kn, rn) and np.array_equal(ko, ro)


def test_children_evaluate_like_oracle(gpu, oracle):
    x, y, c = synth.problem()
    nodes, offs = synth.population_loguniform(seed=8, count=600, hi=20001)
    pop = make_pop(gpu, nodes, offs)
    ops = synth.crossover_points(2, np.diff(offs.astype(np.int64)), 600)
    kids = gpu.gp_crossover(pop, ops)
    gpu.gp_evaluate(kids)
    fit, vals, hits = gpu.gp_fitness(kids, case_values=True, hits=True)
    rn, ro = oracle.crossover_population(nodes, offs, *ops)
    ref = oracle.eval_population(rn, ro, x, y, c, n_threads=8)
    assert same_f32(vals, ref["out"]) and same_f32(fit, ref["fitness"])
    assert np.array_equal(hits, ref["hits"])


def test_node_limit(gpu):
    rng = np.random.default_rng(4)
    nodes, offs = synth.pack([synth.random_tree(rng, 101), synth.random_tree(rng, 101)])
    pop = make_pop(gpu, nodes, offs, max_tree_nodes=150)
    # replacing a leaf of tree 0 by the whole of tree 1 gives 201 nodes
    leaf = int(np.nonzero(nodes[:101] >= 4)[0][0])
    with pytest.raises(gpu.GpError) as e:
        gpu.gp_crossover(pop, (np.array([0]), np.array([1]), np.array([leaf]), np.array([0])))
    assert e.value.status == gpu.GP_ELIMIT
    ok = gpu.gp_crossover(pop, (np.array([0]), np.array([1]), np.array([0]), np.array([0])))
    assert gpu.gp_tree_size(ok, 0) == 101


def test_bad_points_rejected(gpu):
    nodes, offs = synth.population_small()
    pop = make_pop(gpu, nodes, offs)
    with pytest.raises(gpu.GpError) as e:
        gpu.gp_crossover(pop, (np.array([0]), np.array([1]), np.array([10 ** 6]), np.array([0])))
    assert e.value.status == gpu.GP_EINVAL
    with pytest.raises(gpu.GpError):
        gpu.gp_crossover(pop, (np.array([0]), np.array([999]), np.array([0]), np.array([0])))


def test_children_chain_sized_on_the_device(gpu, oracle):
    """Children whose bounds allow it are laid out on the device without a
    synchronisation; their sizes reach the host only when a call needs
    them (parents of the next crossover, tree reads, info).  Three
    generations, each evaluated with items built on the device, against the
    oracle's chain."""
    x, y, c = synth.problem()
    nodes, offs = synth.population_loguniform(seed=12, count=700, hi=40001)
    pop = make_pop(gpu, nodes, offs)
    rn, ro = nodes, offs
    for g in range(3):
        ops = synth.crossover_points(30 + g, np.diff(ro.astype(np.int64)), 700)
        kids = gpu.gp_crossover(pop, ops)
        gpu.gp_evaluate(kids)
        fit, vals, hits = gpu.gp_fitness(kids, case_values=True, hits=True)
        rn, ro = oracle.crossover_population(rn, ro, *ops)
        ref = oracle.eval_population(rn, ro, x, y, c, n_threads=8)
        assert same_f32(vals, ref["out"]) and same_f32(fit, ref["fitness"]), g
        assert np.array_equal(hits, ref["hits"])
        st = gpu.gp_eval_stats_get(kids)
        assert st["levels"] == 2 and st["items"] > 700          # chunks of the multi-chunk trees + ropes
        info = gpu.gp_population_get_info(kids)
        assert info.total_nodes == int(ro[-1])
        t = int(np.argmax(np.diff(ro.astype(np.int64))))
        assert gpu.gp_tree_size(kids, t) == int(ro[t + 1] - ro[t])
        pop = kids


@pytest.mark.parametrize("chunk", [256, 1024])
def test_children_device_planning_and_host_fallback(gpu, oracle, chunk):
    """The same children evaluated with chunk sizes for which every bound is
    within 32 chunks (items built on the device) or not (sizes read back,
    planned upper levels): identical results either way."""
    x, y, c = synth.problem()
    nodes, offs = synth.population_loguniform(seed=13, count=300, hi=9001)
    pop = make_pop(gpu, nodes, offs)
    ops = synth.crossover_points(5, np.diff(offs.astype(np.int64)), 300)
    rn, ro = oracle.crossover_population(nodes, offs, *ops)
    ref = oracle.eval_population(rn, ro, x, y, c, n_threads=8)
    kids = gpu.gp_crossover(pop, ops)
    gpu.gp_evaluate(kids, chunk_nodes=chunk)
    fit, vals, _ = gpu.gp_fitness(kids, case_values=True)
    assert same_f32(vals, ref["out"]) and same_f32(fit, ref["fitness"])
    kn, ko = gpu.read_all_trees(kids)
    assert np.array_equal(kn, rn) and np.array_equal(ko, ro)


def test_crossover_on_another_stream_then_parents_freed(gpu, oracle):
    """Parents made on one stream, crossed on a second (after the first
    finished) and destroyed at once: the parents' memory is freed on the
    stream that read them, so the children are intact; they are evaluated
    on that stream and match the oracle."""
    import torch
    x, y, c = synth.problem()
    nodes, offs = synth.population_loguniform(seed=14, count=500, hi=60001)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    pop = gpu.gp_create_population(gpu.Problem(x, y, c), nodes, offs, sa)
    sa.synchronize()
    ops = synth.crossover_points(6, np.diff(offs.astype(np.int64)), 500)
    kids = gpu.gp_crossover(pop, ops, sb)
    gpu.gp_destroy_population(pop)
    # new allocations on the first stream while the copies may still run
    other = gpu.gp_create_population(gpu.Problem(x, y, c), nodes, offs, sa)
    gpu.gp_evaluate(kids, sb)
    fit, vals, _ = gpu.gp_fitness(kids, case_values=True)
    rn, ro = oracle.crossover_population(nodes, offs, *ops)
    ref = oracle.eval_population(rn, ro, x, y, c, n_threads=8)
    assert same_f32(vals, ref["out"]) and same_f32(fit, ref["fitness"])
    kn, ko = gpu.read_all_trees(kids)
    assert np.array_equal(kn, rn) and np.array_equal(ko, ro)
    gpu.gp_destroy_population(other)


def test_long_subtree_walks(gpu, oracle):
    """Subtree ends found by the two-phase walk (a 512-byte warp step, then
    a CTA per still-open walk at 16 KB per step): points at and near the
    roots of trees of 1e5..3e5 nodes and of a left spine of depth 2e4 (its
    subtrees end near the tree's end, so the CTA steps run into the tree's
    last bytes), every child equal to the oracle's."""
    rng = np.random.default_rng(31)
    trees = [synth.random_tree(rng, 300001), synth.random_tree(rng, 100001),
             synth.left_spine_tree(rng, 20000, 3), synth.random_tree(rng, 16385)]
    nodes, offs = synth.pack(trees)
    pop = make_pop(gpu, nodes, offs)
    sizes = np.diff(offs.astype(np.int64))
    recs = []
    for a in range(len(trees)):
        pts = sorted({0, 1, 2, 3, 17, int(sizes[a]) // 7, int(sizes[a]) - 2, int(sizes[a]) - 1})
        for i in pts:
            recs.append((a, (a + 1) % len(trees), i, pts[len(pts) // 2]))
            recs.append((a, a, int(sizes[a]) - 1, i))
    ops = tuple(np.array(v) for v in zip(*recs))
    kids = gpu.gp_crossover(pop, ops)
    kn, ko = gpu.read_all_trees(kids)
    rn, ro = oracle.crossover_population(nodes, offs, *ops)
    assert np.array_equal(kn, rn) and np.array_equal(ko, ro)
