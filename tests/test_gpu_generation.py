"""GPU parity for generations made on the device: tournament selection and
crossover points (identical records), children (identical bytes) and their
evaluation (bit-exact per case, fitness and hits) against the oracle,
generation after generation; graph replay against plain launches and other
chunk sizes; rewind; node limit and capacity errors at the generation the
oracle predicts."""
import os

import numpy as np
import pytest

from paper_1902_09215_gb300 import synth
from tests.gpu_util import first_mismatch, gpu, same_f32  # noqa: F401

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1


def oracle_step(oracle, nodes, offs, fit, seed, g, prob_tables, tsize=7):
    """Generation g -> g+1 on the CPU: records, children, their evaluation."""
    x, y, c = prob_tables
    sizes = np.diff(offs.astype(np.int64)).astype(np.uint64)
    recs = oracle.generation_records(fit, sizes, sizes.shape[0], seed=seed, g=g, tsize=tsize)
    kids, koffs = oracle.crossover_population(nodes, offs, *recs)
    ref = oracle.eval_population(kids, koffs, x, y, c, n_threads=THREADS)
    return recs, kids, koffs, ref


def assert_same_eval(gp, G, ref):
    fit, vals, hits = gp.gp_generation_fitness(G, case_values=True, hits=True)
    assert same_f32(vals, ref["out"]), first_mismatch(vals, ref["out"])
    assert same_f32(fit, ref["fitness"]), first_mismatch(fit, ref["fitness"])
    assert np.array_equal(hits, ref["hits"])


def test_generations_match_oracle(gpu, oracle):
    x, y, c = synth.problem()
    prob = gpu.Problem(x, y, c)
    nodes, offs = synth.population_loguniform(seed=3, count=300, lo=31, hi=32767)
    seed = 21
    G = gpu.gp_generation_create(prob, nodes, offs, seed=seed, use_graph=True)
    info = gpu.gp_generation_get_info(G)
    assert info["graph"] == 1 and info["kernels_per_generation"] > 0
    assert info["chunk_nodes"] in [k for k in info["autotune_chunk"] if k]
    ref = oracle.eval_population(nodes, offs, x, y, c, n_threads=THREADS)
    assert_same_eval(gpu, G, ref)
    for g in range(3):
        recs, kids, koffs, ref_next = oracle_step(oracle, nodes, offs, ref["fitness"], seed, g, (x, y, c))
        gpu.gp_generation_step(G)
        got = gpu.gp_generation_records(G)
        for a, b, name in zip(got, recs, ("mum", "dad", "mum_point", "dad_point")):
            assert np.array_equal(a.astype(np.uint64), b.astype(np.uint64)), (g, name)
        gn, go = gpu.gp_generation_trees(G)
        assert np.array_equal(go, koffs) and np.array_equal(gn, kids), g
        assert_same_eval(gpu, G, ref_next)
        assert gpu.gp_generation_get_info(G)["generation"] == g + 1
        nodes, offs, ref = kids, koffs, ref_next


def test_graph_and_plain_launches_agree(gpu, oracle):
    x, y, c = synth.problem()
    prob = gpu.Problem(x, y, c)
    nodes, offs = synth.population_loguniform(seed=5, count=200, lo=31, hi=20001)
    runs = []
    for use_graph, chunk in ((False, 1024), (True, 4096), (True, 2048)):
        G = gpu.gp_generation_create(prob, nodes, offs, seed=7, chunk_nodes=chunk, use_graph=use_graph)
        gpu.gp_generation_step(G, 3)
        tn, to = gpu.gp_generation_trees(G)
        fit, vals, hits = gpu.gp_generation_fitness(G, case_values=True, hits=True)
        runs.append((tn, to, fit, vals, hits))
        gpu.gp_generation_destroy(G)
    for r in runs[1:]:
        assert np.array_equal(r[0], runs[0][0]) and np.array_equal(r[1], runs[0][1])
        assert same_f32(r[2], runs[0][2]) and same_f32(r[3], runs[0][3])
        assert np.array_equal(r[4], runs[0][4])


def test_many_levels_large_trees(gpu, oracle):
    """Trees up to 3e5 nodes with 1024-node chunks: three or more levels."""
    x, y, c = synth.problem()
    prob = gpu.Problem(x, y, c)
    nodes, offs = synth.population_loguniform(seed=8, count=40, lo=31, hi=300001)
    seed = 99
    G = gpu.gp_generation_create(prob, nodes, offs, seed=seed, chunk_nodes=1024, use_graph=True)
    assert gpu.gp_generation_get_info(G)["levels"] >= 3
    ref = oracle.eval_population(nodes, offs, x, y, c, n_threads=THREADS)
    assert_same_eval(gpu, G, ref)
    for g in range(2):
        recs, kids, koffs, ref_next = oracle_step(oracle, nodes, offs, ref["fitness"], seed, g, (x, y, c))
        gpu.gp_generation_step(G)
        gn, go = gpu.gp_generation_trees(G)
        assert np.array_equal(go, koffs) and np.array_equal(gn, kids), g
        assert_same_eval(gpu, G, ref_next)
        nodes, offs, ref = kids, koffs, ref_next


def test_creation_grows_dedicated_spill_of_upper_levels(gpu, oracle):
    """Comb-shaped trees (every operator's first argument an x leaf, its
    second the rest of the tree) cut into 1024-node chunks have upper trees
    that do not shrink, so the first upper level makes them final items with
    dedicated spill areas far above the creation's first guess: its sizing
    pass must grow the pool, build that level again from the same chunk
    counts, and go on to every later level."""
    rng = np.random.default_rng(21)
    trees = []
    for k in (60000, 90000, 150000):
        t = np.full(2 * k + 1, 4, np.uint8)
        t[0:2 * k:2] = rng.integers(0, 4, k).astype(np.uint8)
        trees.append(t)
    trees += [synth.random_tree(rng, n) for n in (101, 2001, 30001)]
    nodes, offs = synth.pack(trees)
    x, y, c = synth.problem()
    prob = gpu.Problem(x, y, c)
    G = gpu.gp_generation_create(prob, nodes, offs, seed=3, chunk_nodes=1024, use_graph=True)
    ref = oracle.eval_population(nodes, offs, x, y, c, n_threads=THREADS)
    assert_same_eval(gpu, G, ref)
    gpu.gp_generation_destroy(G)


def test_fused_slots_overflow_falls_back(gpu, oracle):
    """Left combs (all operators first, then all leaves) of 10..20 chunks of
    1024 nodes: their leaf-only chunks leave 1024 values each, far above a
    slot's first 128 value entries, and their ropes would hold 10^4 values:
    the creation doubles the entries per slot up to the chunk size and then
    plans such trees instead; generations stay exact."""
    rng = np.random.default_rng(31)
    trees = []
    for k in (5000, 8000, 10000):
        trees.append(np.concatenate([rng.integers(0, 4, k).astype(np.uint8), np.full(k + 1, 4, np.uint8)]))
    trees += [synth.random_tree(rng, n) for n in (101, 2001, 15001, 25001)]
    nodes, offs = synth.pack(trees)
    x, y, c = synth.problem()
    prob = gpu.Problem(x, y, c)
    seed = 8
    G = gpu.gp_generation_create(prob, nodes, offs, seed=seed, chunk_nodes=1024, use_graph=True)
    ref = oracle.eval_population(nodes, offs, x, y, c, n_threads=THREADS)
    assert_same_eval(gpu, G, ref)
    for g in range(2):
        recs, kids, koffs, ref_next = oracle_step(oracle, nodes, offs, ref["fitness"], seed, g, (x, y, c))
        gpu.gp_generation_step(G)
        gn, go = gpu.gp_generation_trees(G)
        assert np.array_equal(go, koffs) and np.array_equal(gn, kids), g
        assert_same_eval(gpu, G, ref_next)
        nodes, offs, ref = kids, koffs, ref_next
    gpu.gp_generation_destroy(G)


def test_level_budget_follows_growth(gpu, oracle):
    """Generation 0 fits one chunk per tree (one level), so the level budget
    starts at three; children of a few hundred nodes with 256-node chunks
    reach the last level, which makes every open upper tree a final item
    (still exact) and widens the budget for the next generations."""
    x, y, c = synth.problem()
    prob = gpu.Problem(x, y, c)
    nodes, offs = synth.population_loguniform(seed=17, count=120, lo=101, hi=255)
    seed = 5
    G = gpu.gp_generation_create(prob, nodes, offs, seed=seed, chunk_nodes=256, use_graph=True)
    k0 = gpu.gp_generation_get_info(G)["kernels_per_generation"]
    ref = oracle.eval_population(nodes, offs, x, y, c, n_threads=THREADS)
    widened = False
    for g in range(8):
        recs, kids, koffs, ref_next = oracle_step(oracle, nodes, offs, ref["fitness"], seed, g, (x, y, c))
        gpu.gp_generation_step(G)
        gn, go = gpu.gp_generation_trees(G)
        assert np.array_equal(go, koffs) and np.array_equal(gn, kids), g
        assert_same_eval(gpu, G, ref_next)
        widened = widened or gpu.gp_generation_get_info(G)["kernels_per_generation"] > k0
        nodes, offs, ref = kids, koffs, ref_next
    if int(np.diff(offs.astype(np.int64)).max()) > 256 * 27:
        assert widened


def test_rewind_repeats_the_step(gpu):
    x, y, c = synth.problem()
    prob = gpu.Problem(x, y, c)
    nodes, offs = synth.population_loguniform(seed=9, count=120, lo=31, hi=8191)
    G = gpu.gp_generation_create(prob, nodes, offs, seed=3, chunk_nodes=2048)
    gpu.gp_generation_step(G, 2)
    t2 = gpu.gp_generation_trees(G)
    f2 = gpu.gp_generation_fitness(G)[0]
    gpu.gp_generation_rewind(G)
    assert gpu.gp_generation_get_info(G)["generation"] == 1
    gpu.gp_generation_step(G)
    t2b = gpu.gp_generation_trees(G)
    assert np.array_equal(t2[0], t2b[0]) and np.array_equal(t2[1], t2b[1])
    assert same_f32(gpu.gp_generation_fitness(G)[0], f2)


def sizes_of(offs):
    return np.diff(offs.astype(np.int64))


def test_node_limit_stops_at_the_right_generation(gpu, oracle):
    """The oracle's run without a limit gives the largest child of every
    generation; with the limit set to the largest size seen before the first
    generation that sets a new record, exactly that generation's step fails
    and the population stays at the generation before it."""
    x, y, c = synth.problem()
    nodes, offs = synth.population_small(seed=1, count=100, max_nodes=63)   # small trees grow
    seed = 5
    n0, o0 = nodes, offs
    ref = oracle.eval_population(n0, o0, x, y, c, n_threads=THREADS)
    record = int(sizes_of(offs).max())
    fail_at, limit = None, None
    for g in range(10):
        recs, kids, koffs, ref_next = oracle_step(oracle, n0, o0, ref["fitness"], seed, g, (x, y, c))
        m = int(sizes_of(koffs).max())
        if g >= 1 and m > record:
            fail_at, limit = g, record
            break
        record = max(record, m)
        n0, o0, ref = kids, koffs, ref_next
    if fail_at is None:
        pytest.skip("no generation set a new size record within 10 generations")
    prob = gpu.Problem(x, y, c, max_tree_nodes=limit)
    G = gpu.gp_generation_create(prob, nodes, offs, seed=seed, chunk_nodes=1024)
    gpu.gp_generation_step(G, fail_at + 3)          # the steps after the failing one do nothing
    with pytest.raises(gpu.GpError) as e:
        gpu.gp_generation_fitness(G)
    assert e.value.status == gpu.GP_ELIMIT
    info = gpu.gp_generation_get_info(G)
    assert info["generation"] == fail_at and info["error_generation"] == fail_at


def test_population_buffer_too_small(gpu, oracle):
    x, y, c = synth.problem()
    prob = gpu.Problem(x, y, c)
    for seed in range(1, 40):
        nodes, offs = synth.population_loguniform(seed=11, count=60, lo=31, hi=4095)
        used = int(np.sum((sizes_of(offs) + 15) // 16 * 16)) + 64
        ref = oracle.eval_population(nodes, offs, x, y, c, n_threads=THREADS)
        recs, kids, koffs, _ = oracle_step(oracle, nodes, offs, ref["fitness"], seed, 0, (x, y, c))
        need = int(np.sum((sizes_of(koffs) + 15) // 16 * 16)) + 64
        if need > used:
            break
    else:
        pytest.skip("no seed with a larger generation")
    G = gpu.gp_generation_create(prob, nodes, offs, seed=seed, chunk_nodes=1024, arena_bytes=need - 1)
    gpu.gp_generation_step(G)
    with pytest.raises(gpu.GpError) as e:
        gpu.gp_generation_fitness(G)
    assert e.value.status == gpu.GP_ENOMEM
    assert gpu.gp_generation_get_info(G)["generation"] == 0
    # recovery: larger buffers, the same generation made again
    gpu.gp_generation_recover(G)
    gpu.gp_generation_step(G)
    gn, go = gpu.gp_generation_trees(G)
    assert np.array_equal(gn, kids) and np.array_equal(go, koffs)
    assert gpu.gp_generation_get_info(G)["arena_bytes"] == 2 * (need - 1)
    with pytest.raises(gpu.GpError):
        gpu.gp_generation_recover(G)                 # nothing to recover from
    # the exact size is enough
    G2 = gpu.gp_generation_create(prob, nodes, offs, seed=seed, chunk_nodes=1024, arena_bytes=need)
    gpu.gp_generation_step(G2)
    gn, go = gpu.gp_generation_trees(G2)
    assert np.array_equal(gn, kids) and np.array_equal(go, koffs)


def test_generation_rejects_bad_parameters(gpu):
    x, y, c = synth.problem()
    prob = gpu.Problem(x, y, c)
    nodes, offs = synth.population_small()
    for kw in (dict(tournament_size=0), dict(tournament_size=33), dict(chunk_nodes=100),
               dict(chunk_nodes=1000), dict(max_levels=1)):
        with pytest.raises(gpu.GpError) as e:
            gpu.gp_generation_create(prob, nodes, offs, seed=1, **kw)
        assert e.value.status == gpu.GP_EINVAL
    bad = nodes.copy()
    bad[0] = 200                                     # undefined code
    with pytest.raises(gpu.GpError) as e:
        gpu.gp_generation_create(prob, bad, offs, seed=1)
    assert e.value.status == gpu.GP_EMALFORMED
    G = gpu.gp_generation_create(prob, nodes, offs, seed=1, chunk_nodes=256)
    with pytest.raises(gpu.GpError):
        gpu.gp_generation_rewind(G)                  # nothing to undo
    with pytest.raises(gpu.GpError) as e:
        gpu.gp_generation_records(G)                 # no step has made generation 0
    assert e.value.status == gpu.GP_EINVAL


def test_paper_run_start_ramped_half_and_half(gpu, oracle):
    """Table gp.details' run: 4000 ramped half-and-half trees (depths 2..6),
    size-7 tournaments, 100% subtree crossover; five generations, every one
    identical to the oracle's (records, children, fitness)."""
    x, y, c = synth.problem()
    prob = gpu.Problem(x, y, c)
    nodes, offs = synth.ramped_half_and_half(seed=1, count=4000)
    seed = 2019
    G = gpu.gp_generation_create(prob, nodes, offs, seed=seed, use_graph=True)
    ref = oracle.eval_population(nodes, offs, x, y, c, n_threads=THREADS)
    assert_same_eval(gpu, G, ref)
    for g in range(5):
        recs, kids, koffs, ref_next = oracle_step(oracle, nodes, offs, ref["fitness"], seed, g, (x, y, c))
        gpu.gp_generation_step(G)
        got = gpu.gp_generation_records(G)
        assert all(np.array_equal(a.astype(np.uint64), b.astype(np.uint64)) for a, b in zip(got, recs)), g
        gn, go = gpu.gp_generation_trees(G)
        assert np.array_equal(go, koffs) and np.array_equal(gn, kids), g
        assert_same_eval(gpu, G, ref_next)
        nodes, offs, ref = kids, koffs, ref_next


@pytest.mark.parametrize("trees", [[31], [1, 1], [1, 3, 1]])
def test_degenerate_populations(gpu, oracle, trees):
    """A one-tree population (every tournament picks it; it crosses with
    itself) and populations of single leaves (every child is a leaf of a
    parent): three generations identical to the oracle's."""
    x, y, c = synth.problem()
    prob = gpu.Problem(x, y, c)
    rng = np.random.default_rng(len(trees))
    nodes, offs = synth.pack([synth.random_tree(rng, n) for n in trees])
    seed = 77
    G = gpu.gp_generation_create(prob, nodes, offs, seed=seed)
    ref = oracle.eval_population(nodes, offs, x, y, c, n_threads=1)
    assert_same_eval(gpu, G, ref)
    for g in range(3):
        recs, kids, koffs, ref_next = oracle_step(oracle, nodes, offs, ref["fitness"], seed, g, (x, y, c))
        gpu.gp_generation_step(G)
        got = gpu.gp_generation_records(G)
        assert all(np.array_equal(a.astype(np.uint64), b.astype(np.uint64)) for a, b in zip(got, recs)), g
        gn, go = gpu.gp_generation_trees(G)
        assert np.array_equal(go, koffs) and np.array_equal(gn, kids), g
        assert_same_eval(gpu, G, ref_next)
        nodes, offs, ref = kids, koffs, ref_next
    gpu.gp_generation_destroy(G)


def test_launch_shapes_are_exact_and_reported(gpu, oracle):
    """Every launch shape the creation may choose (level 0's warps per SM x
    window entries, the upper levels' window) gives the oracle's
    generations exactly; get_info reports the shape in use and the
    autotuner's candidates and times."""
    x, y, c = synth.problem()
    prob = gpu.Problem(x, y, c)
    nodes, offs = synth.population_loguniform(seed=19, count=250, lo=31, hi=70001)
    seed = 33
    ref = oracle.eval_population(nodes, offs, x, y, c, n_threads=THREADS)
    want = []
    n, o, r = nodes, offs, ref
    for g in range(2):
        _, n, o, r = oracle_step(oracle, n, o, r["fitness"], seed, g, (x, y, c))
        want.append((n, o, r))
    shapes = [(32, 32, 128), (28, 36, 96), (16, 64, 192), (0, 0, 0)]     # the last one autotuned
    for W, K, Ku in shapes:
        G = gpu.gp_generation_create(prob, nodes, offs, seed=seed, chunk_nodes=4096, warps_per_cta=W,
                                     window_entries=K, upper_window_entries=Ku)
        info = gpu.gp_generation_get_info(G)
        if W:
            assert (info["warps_per_cta"], info["window_entries"], info["upper_window_entries"]) == (W, K, Ku)
        else:
            tried = [s for s in info["autotune_shape"] if s[0]]
            level0 = [(w, k) for w, k, lv in tried if lv == "level0"]
            upper = [(w, k) for w, k, lv in tried if lv == "upper"]
            assert len(level0) >= 1 and len(upper) == 3, tried
            assert (info["warps_per_cta"], info["window_entries"]) in level0
            assert (info["upper_warps"], info["upper_window_entries"]) in upper
            assert info["upper_window_entries"] in (96, 128, 192)
            assert all(t > 0 for t in info["autotune_shape_ms"][:len(tried)])
        for g in range(2):
            gpu.gp_generation_step(G)
            gn, go = gpu.gp_generation_trees(G)
            assert np.array_equal(go, want[g][1]) and np.array_equal(gn, want[g][0]), (W, K, Ku, g)
            assert_same_eval(gpu, G, want[g][2])
        gpu.gp_generation_destroy(G)
    with pytest.raises(gpu.GpError) as e:                 # does not fit shared memory
        gpu.gp_generation_create(prob, nodes, offs, seed=seed, warps_per_cta=32, window_entries=64)
    assert e.value.status == gpu.GP_EINVAL


def test_select_range_matches_the_oracle_draws(gpu, oracle):
    """gp_select, for any range of children, gives the records the oracle's
    generation draws (size-7 tournaments with NaN worst, uniform points)."""
    import torch
    x, y, c = synth.problem()
    nodes, offs = synth.population_loguniform(seed=29, count=500, lo=31, hi=4001)
    fit = np.asarray(oracle.eval_population(nodes, offs, x, y, c, n_threads=THREADS)["fitness"], np.float32)
    fit[::37] = np.nan                                    # unfit trees rank worst
    sizes = np.diff(offs.astype(np.int64)).astype(np.uint64)
    seed, g = 77, 3
    want = oracle.generation_records(fit, sizes, 500, seed=seed, g=g)
    d_fit = torch.from_numpy(fit).cuda()
    d_sz = torch.from_numpy(sizes.view(np.int64)).cuda()
    for lo, n in ((0, 500), (123, 77), (499, 1)):
        out = torch.zeros(n * gpu.XO_RECORD_BYTES, dtype=torch.uint8, device="cuda")
        gpu.gp_select(d_fit.data_ptr(), d_sz.data_ptr(), 500, seed, g, lo, n, out.data_ptr())
        torch.cuda.synchronize()
        got = np.frombuffer(out.cpu().numpy().tobytes(), dtype=gpu._XO_DTYPE)
        for name, w in zip(("mum", "dad", "mum_point", "dad_point"), want):
            assert np.array_equal(got[name].astype(np.uint64), np.asarray(w)[lo:lo + n].astype(np.uint64)), (lo, name)


def test_population_from_device_bytes(gpu, oracle):
    """gp_create_population takes packed trees already in device memory (e.g.
    received from another process) and validates them as host ones."""
    import torch
    x, y, c = synth.problem()
    prob = gpu.Problem(x, y, c)
    nodes, offs = synth.population_loguniform(seed=31, count=200, lo=31, hi=9001)
    d = torch.zeros(nodes.shape[0] + 64, dtype=torch.uint8, device="cuda")
    d[:nodes.shape[0]] = torch.from_numpy(nodes).cuda()
    torch.cuda.synchronize()
    pop = gpu.gp_create_population(prob, d.data_ptr(), offs)
    gpu.gp_evaluate(pop)
    fit, _, _ = gpu.gp_fitness(pop)
    assert same_f32(fit, oracle.eval_population(nodes, offs, x, y, c, n_threads=THREADS)["fitness"])
    kn, ko = gpu.read_all_trees(pop)
    assert np.array_equal(kn, nodes) and np.array_equal(ko, offs)
    bad = d.clone()
    bad[0] = 200                                          # an undefined code
    torch.cuda.synchronize()
    with pytest.raises(gpu.GpError) as e:
        gpu.gp_create_population(prob, bad.data_ptr(), offs)
    assert e.value.status == gpu.GP_EMALFORMED
