"""GPU tests of the serving loop: runs served together in shared batches
end exactly where the same runs end when each is advanced alone (bytes of
every tree, bits of every fitness value), one of them also against the
oracle; admission under an HBM budget; retries after a workspace overflow;
a failing run does not affect the others."""
import os
import threading

import numpy as np
import pytest

from paper_1902_09215_gb300 import synth
from tests.gpu_util import first_mismatch, gpu, same_f32  # noqa: F401

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1


def make_runs(k, lo=11, hi=20001):
    """k populations of uneven sizes (48..300 trees, log-uniform trees)."""
    rng = np.random.default_rng(77)
    runs = []
    for i in range(k):
        n = int(rng.integers(48, 301))
        nodes, offs = synth.population_loguniform(seed=100 + i, count=n, lo=lo, hi=hi)
        runs.append((nodes, offs, 1000 + 17 * i))
    return runs


def alone(gp, prob, nodes, offs, seed, gens):
    G = gp.gp_generation_create(prob, nodes, offs, seed=seed, chunk_nodes=8192)
    gp.gp_generation_step(G, gens)
    tn, to = gp.gp_generation_trees(G)
    fit, vals, hits = gp.gp_generation_fitness(G, case_values=True, hits=True)
    gp.gp_generation_destroy(G)
    return tn, to, fit, vals, hits


def serve_all(gp, srv, runs, gens_per_run, chunks=1):
    """Open every run and submit its generations in `chunks` requests from
    one thread per run; returns run ids and the request results."""
    ids = [gp.gp_server_open_run(srv, n, o, seed=s) for n, o, s in runs]
    results = {}

    def client(rid, gens):
        out = []
        per = [gens // chunks + (1 if j < gens % chunks else 0) for j in range(chunks)]
        for g in per:
            if g:
                try:
                    q = gp.gp_server_submit(srv, rid, g)
                except gp.GpError as e:             # the run has failed
                    out.append({"status": e.status})
                    break
                out.append(gp.gp_server_wait(srv, q))
        results[rid] = out

    th = [threading.Thread(target=client, args=(rid, g)) for rid, g in zip(ids, gens_per_run)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    return ids, results


def test_runs_in_a_shared_batch_equal_runs_alone(gpu, oracle):
    x, y, c = synth.problem()
    prob = gpu.Problem(x, y, c)
    runs = make_runs(6)
    gens = [3, 1, 4, 2, 3, 2]
    srv = gpu.gp_server_create(prob, hbm_budget_bytes=4 << 30, max_runs=16, max_batch_trees=1 << 16,
                               chunk_nodes=8192)
    ids, results = serve_all(gpu, srv, runs, gens, chunks=2)
    for rid, (n, o, s), g in zip(ids, runs, gens):
        assert all(r["status"] == gpu.GP_OK for r in results[rid]), results[rid]
        assert results[rid][-1]["generation"] == g
        tn, to = gpu.gp_server_run_trees(srv, rid)
        fit, vals, hits = gpu.gp_server_run_fitness(srv, rid, case_values=True, hits=True)
        an, ao, afit, avals, ahits = alone(gpu, prob, n, o, s, g)
        assert np.array_equal(to, ao) and np.array_equal(tn, an), rid
        assert same_f32(vals, avals) and same_f32(fit, afit) and np.array_equal(hits, ahits)
        best = int(np.argmin(np.where(np.isnan(fit), np.inf, fit)))
        assert results[rid][-1]["best_tree"] == best
    # one run against the oracle: its final trees evaluated on the CPU
    rid = ids[2]
    tn, to = gpu.gp_server_run_trees(srv, rid)
    fit, vals, hits = gpu.gp_server_run_fitness(srv, rid, case_values=True, hits=True)
    ref = oracle.eval_population(tn, to, x, y, c, n_threads=THREADS)
    assert same_f32(vals, ref["out"]), first_mismatch(vals, ref["out"])
    assert same_f32(fit, ref["fitness"]) and np.array_equal(hits, ref["hits"])
    st = gpu.gp_server_get_stats(srv)
    assert st["run_generations"] == sum(gens)
    assert st["requests_done"] == sum(min(2, g) for g in gens)
    assert st["batches"] < sum(gens)                 # runs shared batches
    assert st["child_nodes"] > 0 and st["latency_p99_ms"] >= st["latency_p50_ms"] > 0
    for rid in ids:
        gpu.gp_server_close_run(srv, rid)
    gpu.gp_server_destroy(srv)


def test_admission_by_hbm_budget(gpu):
    """A budget that holds two runs at a time: the others wait, are admitted
    as runs close, and still end as they would alone."""
    x, y, c = synth.problem()
    prob = gpu.Problem(x, y, c)
    runs = make_runs(5, hi=4001)
    arena = 1 << 22                                   # 4 MiB per buffer, 8 MiB per run
    budget = 2 * 2 * arena + (1 << 20)                # room for two runs
    srv = gpu.gp_server_create(prob, hbm_budget_bytes=budget, max_runs=8, max_batch_trees=1 << 14,
                               chunk_nodes=4096)
    ids = [gpu.gp_server_open_run(srv, n, o, seed=s, arena_bytes=arena) for n, o, s in runs]
    reqs = [gpu.gp_server_submit(srv, rid, 2) for rid in ids]
    # the first two complete; the rest cannot be admitted until runs close
    r0 = gpu.gp_server_wait(srv, reqs[0])
    r1 = gpu.gp_server_wait(srv, reqs[1])
    assert r0["status"] == r1["status"] == gpu.GP_OK
    with pytest.raises(gpu.GpError) as e:
        gpu.gp_server_wait(srv, reqs[2], timeout_ms=300)
    assert e.value.status == gpu.GP_ETIMEOUT
    st = gpu.gp_server_get_stats(srv)
    assert st["runs_admitted"] == 2 and st["runs_waiting"] == 3
    finals = {}
    done = {0: r0, 1: r1}                             # a request's result is collected once
    for k, rid in enumerate(ids):
        r = done[k] if k in done else gpu.gp_server_wait(srv, reqs[k])
        assert r["status"] == gpu.GP_OK and r["generation"] == 2
        finals[rid] = gpu.gp_server_run_trees(srv, rid)
        gpu.gp_server_close_run(srv, rid)             # frees room for the next
    assert gpu.gp_server_get_stats(srv)["runs_admitted"] == 5
    with pytest.raises(gpu.GpError):
        gpu.gp_server_wait(srv, reqs[0])              # already collected
    for rid, (n, o, s) in zip(ids, runs):
        an, ao, *_ = alone(gpu, prob, n, o, s, 2)
        assert np.array_equal(finals[rid][0], an) and np.array_equal(finals[rid][1], ao)
    gpu.gp_server_destroy(srv)


def test_workspace_overflow_retries_in_smaller_batches(gpu):
    """A value workspace that holds any one run's level but not several
    runs' together: the batches that overflow are retried smaller, and every
    run still ends as it does alone."""
    x, y, c = synth.problem()
    prob = gpu.Problem(x, y, c)
    runs = make_runs(4, lo=1001, hi=20001)
    # first pass: one run per batch, a large workspace; the most any single
    # run's level needed
    srv = gpu.gp_server_create(prob, hbm_budget_bytes=2 << 30, max_runs=8, max_batch_trees=1 << 14,
                               max_batch_runs=1, chunk_nodes=1024)
    serve_all(gpu, srv, runs, [2, 2, 2, 2])
    one = gpu.gp_server_get_stats(srv)["most_level_values"]
    gpu.gp_server_destroy(srv)
    assert one > 0
    srv = gpu.gp_server_create(prob, hbm_budget_bytes=2 << 30, max_runs=8, max_batch_trees=1 << 14,
                               chunk_nodes=1024, workspace_values=one + 16)
    ids, results = serve_all(gpu, srv, runs, [2, 2, 2, 2])
    st = gpu.gp_server_get_stats(srv)
    assert st["retries"] > 0                          # some shared batch overflowed
    for rid, (n, o, s) in zip(ids, runs):
        assert results[rid][-1]["status"] == gpu.GP_OK
        tn, to = gpu.gp_server_run_trees(srv, rid)
        an, ao, *_ = alone(gpu, prob, n, o, s, 2)
        assert np.array_equal(tn, an) and np.array_equal(to, ao)
    gpu.gp_server_destroy(srv)


def oracle_max_sizes(oracle, nodes, offs, seed, gens):
    """Largest child of each of `gens` generations of a run (oracle)."""
    x, y, c = synth.problem()
    out = []
    ref = oracle.eval_population(nodes, offs, x, y, c, n_threads=THREADS)
    for g in range(gens):
        sizes = np.diff(offs.astype(np.int64)).astype(np.uint64)
        recs = oracle.generation_records(ref["fitness"], sizes, sizes.shape[0], seed=seed, g=g)
        nodes, offs = oracle.crossover_population(nodes, offs, *recs)
        out.append(int(np.diff(offs.astype(np.int64)).max()))
        ref = oracle.eval_population(nodes, offs, x, y, c, n_threads=THREADS)
    return out


def test_a_run_that_outgrows_its_buffers_is_moved(gpu, oracle):
    """A run whose buffers are one byte too small for its first generation
    (sized by the oracle) is moved to larger ones and the generation made
    again: it ends exactly as the same run alone, and so do the others."""
    x, y, c = synth.problem()
    nodes, offs = synth.population_small(seed=1, count=100, max_nodes=63)
    sizes = np.diff(offs.astype(np.int64))
    used = int(np.sum((sizes + 15) // 16 * 16)) + 64
    ref = oracle.eval_population(nodes, offs, x, y, c, n_threads=THREADS)
    for seed in range(5, 60):
        recs = oracle.generation_records(ref["fitness"], sizes.astype(np.uint64), 100, seed=seed, g=0)
        kids, koffs = oracle.crossover_population(nodes, offs, *recs)
        need = int(np.sum((np.diff(koffs.astype(np.int64)) + 15) // 16 * 16)) + 64
        if need > used:
            break
    else:
        pytest.skip("no seed whose first generation outgrows the population")
    prob = gpu.Problem(x, y, c)
    srv = gpu.gp_server_create(prob, hbm_budget_bytes=1 << 30, max_runs=8, max_batch_trees=1 << 14)
    tight = gpu.gp_server_open_run(srv, nodes, offs, seed=seed, arena_bytes=need - 1)
    others = make_runs(2)
    ids, results = serve_all(gpu, srv, others, [3, 3])
    rt = gpu.gp_server_wait(srv, gpu.gp_server_submit(srv, tight, 3))
    assert rt["status"] == gpu.GP_OK and rt["generation"] == 3
    assert gpu.gp_server_get_stats(srv)["regrown"] >= 1
    tn, to = gpu.gp_server_run_trees(srv, tight)
    an, ao, *_ = alone(gpu, prob, nodes, offs, seed, 3)
    assert np.array_equal(tn, an) and np.array_equal(to, ao)
    for rid, (n, o, s) in zip(ids, others):
        assert results[rid][-1]["status"] == gpu.GP_OK
        tn, to = gpu.gp_server_run_trees(srv, rid)
        an, ao, *_ = alone(gpu, prob, n, o, s, 3)
        assert np.array_equal(tn, an) and np.array_equal(to, ao)
    gpu.gp_server_destroy(srv)


def test_a_failing_run_leaves_the_others_alone(gpu, oracle):
    """Node limit 1000: a run of 901..999-node trees exceeds it in its first
    generation and its request fails with GP_ELIMIT; runs of small trees
    (which the oracle shows stay below the limit) end exactly as alone."""
    x, y, c = synth.problem()
    limit = 1000
    big = synth.population_loguniform(seed=21, count=64, lo=901, hi=999)
    small = make_runs(2, hi=81)
    if oracle_max_sizes(oracle, big[0], big[1], 5, 1)[0] <= limit:
        pytest.skip("the large run stays below the limit")
    if any(max(oracle_max_sizes(oracle, n, o, s, 3)) > limit for n, o, s in small):
        pytest.skip("a small run grows past the limit")
    prob = gpu.Problem(x, y, c, max_tree_nodes=limit)
    srv = gpu.gp_server_create(prob, hbm_budget_bytes=1 << 30, max_runs=8, max_batch_trees=1 << 14)
    bad = gpu.gp_server_open_run(srv, big[0], big[1], seed=5)
    ids, results = serve_all(gpu, srv, small, [3, 3])
    rb = gpu.gp_server_wait(srv, gpu.gp_server_submit(srv, bad, 2))
    assert rb["status"] == gpu.GP_ELIMIT
    for rid, (n, o, s) in zip(ids, small):
        assert results[rid][-1]["status"] == gpu.GP_OK
        tn, to = gpu.gp_server_run_trees(srv, rid)
        an, ao, *_ = alone(gpu, prob, n, o, s, 3)
        assert np.array_equal(tn, an) and np.array_equal(to, ao)
    with pytest.raises(gpu.GpError) as e:
        gpu.gp_server_submit(srv, bad, 1)
    assert e.value.status == gpu.GP_ELIMIT
    gpu.gp_server_destroy(srv)


def test_closing_a_waiting_run_fails_its_requests(gpu):
    x, y, c = synth.problem()
    prob = gpu.Problem(x, y, c)
    runs = make_runs(2, hi=4001)
    arena = 1 << 22
    srv = gpu.gp_server_create(prob, hbm_budget_bytes=2 * arena + (1 << 20), max_runs=4,
                               max_batch_trees=1 << 14, chunk_nodes=4096)
    a = gpu.gp_server_open_run(srv, runs[0][0], runs[0][1], seed=1, arena_bytes=arena)
    b = gpu.gp_server_open_run(srv, runs[1][0], runs[1][1], seed=2, arena_bytes=arena)   # waits for room
    qa = gpu.gp_server_submit(srv, a, 1)
    qb = gpu.gp_server_submit(srv, b, 1)
    assert gpu.gp_server_wait(srv, qa)["status"] == gpu.GP_OK
    gpu.gp_server_close_run(srv, b)                   # never admitted
    assert gpu.gp_server_wait(srv, qb)["status"] == gpu.GP_EINVAL
    gpu.gp_server_close_run(srv, a)
    gpu.gp_server_destroy(srv)


def test_two_waiters_on_one_request(gpu):
    """Two threads wait on the same request: one collects its result, the
    other is told the request is unknown (GP_EINVAL); neither hangs."""
    x, y, c = synth.problem()
    prob = gpu.Problem(x, y, c)
    nodes, offs, seed = make_runs(1, hi=4001)[0]
    srv = gpu.gp_server_create(prob, hbm_budget_bytes=1 << 30, max_runs=2, chunk_nodes=4096)
    rid = gpu.gp_server_open_run(srv, nodes, offs, seed=seed)
    q = gpu.gp_server_submit(srv, rid, 3)
    outcome = []

    def waiter():
        try:
            outcome.append(gpu.gp_server_wait(srv, q, timeout_ms=60000)["status"])
        except gpu.GpError as e:
            outcome.append(e.status)

    th = [threading.Thread(target=waiter) for _ in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=120)
    assert not any(t.is_alive() for t in th)
    assert sorted(outcome) == sorted([gpu.GP_OK, gpu.GP_EINVAL])
    gpu.gp_server_close_run(srv, rid)
    gpu.gp_server_destroy(srv)


def test_runs_opened_from_a_device_population_equal_runs_from_host_trees(gpu):
    """A run whose initial trees are picked (with repeats) from a device
    population ends, after two served generations, exactly where the same
    trees opened from host memory end: every tree's bytes and fitness."""
    import torch
    s = torch.cuda.current_stream()
    x, y, c = synth.problem()
    prob = gpu.Problem(x, y, c)
    pool_nodes, pool_offs = synth.population_loguniform(seed=61, count=300, lo=11, hi=20001)
    pool = gpu.gp_create_population(prob, pool_nodes, pool_offs, s)
    rng = np.random.default_rng(5)
    picks = [rng.integers(0, 300, size=int(rng.integers(48, 200))).astype(np.uint32) for _ in range(3)]
    srv = gpu.gp_server_create(prob, hbm_budget_bytes=1 << 30, max_runs=8, chunk_nodes=4096)
    dev_ids = [gpu.gp_server_open_run_from(srv, pool, p, seed=700 + k) for k, p in enumerate(picks)]
    host_ids = []
    for k, p in enumerate(picks):
        nodes, offs = synth.pack([pool_nodes[int(pool_offs[t]):int(pool_offs[t + 1])] for t in p])
        host_ids.append(gpu.gp_server_open_run(srv, nodes, offs, seed=700 + k))
    reqs = [gpu.gp_server_submit(srv, rid, 2) for rid in dev_ids + host_ids]
    for q in reqs:
        assert gpu.gp_server_wait(srv, q)["status"] == gpu.GP_OK
    for a, b in zip(dev_ids, host_ids):
        ta, tb = gpu.gp_server_run_trees(srv, a), gpu.gp_server_run_trees(srv, b)
        assert np.array_equal(ta[0], tb[0]) and np.array_equal(ta[1], tb[1])
        fa, _, _ = gpu.gp_server_run_fitness(srv, a)
        fb, _, _ = gpu.gp_server_run_fitness(srv, b)
        assert same_f32(fa, fb)
    with pytest.raises(gpu.GpError) as e:                 # an index past the population
        gpu.gp_server_open_run_from(srv, pool, np.array([0, 300], np.uint32), seed=1)
    assert e.value.status == gpu.GP_EINVAL
    for rid in dev_ids + host_ids:
        gpu.gp_server_close_run(srv, rid)
    gpu.gp_server_destroy(srv)
