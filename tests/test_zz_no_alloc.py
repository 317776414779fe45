"""gp_evaluate_noalloc: the evaluation entry point for callers that cannot
allocate device memory while they evaluate (their GPU memory belongs to their
own allocator, or they cannot afford the synchronisation of cudaMalloc).  Its
scratch is a fixed static device array inside libgp; it must give exactly the
results of the allocating entry points, also when called again (the array
keeps the previous call's contents)."""
import numpy as np
import pytest

from paper_1902_09215_gb300 import synth
from tests.gpu_util import first_mismatch, gpu, same_f32  # noqa: F401

pytestmark = pytest.mark.gpu


def population(seed, count, hi):
    rng = np.random.default_rng(seed)
    sizes = synth.loguniform_sizes(rng, count, 1, hi)
    trees = [synth.random_tree(rng, int(n)) for n in sizes]
    one = [3, 4, 4]
    trees.append(np.array([2, 2, 2, 2, 2, 4, 4, 1, 4] + one + [1, 4] + one + [0, 4] + one + [0, 4] + one,
                          np.uint8))          # the exact Sextic tree
    return synth.pack(trees)


def reference(gp, prob, nodes, offs):
    pop = gp.gp_create_population(prob, nodes, offs)
    gp.gp_evaluate(pop)
    out = gp.gp_fitness(pop, case_values=True, hits=True)
    gp.gp_destroy_population(pop)
    return out


def device_buffers(nodes, offs, n_cases):
    import torch
    total = int(offs[-1])
    d_nodes = torch.zeros((total + 15) // 16 * 16 + 16, dtype=torch.uint8, device="cuda")
    d_nodes[:total] = torch.from_numpy(nodes).to("cuda")
    n = offs.shape[0] - 1
    d_fit = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
    d_vals = torch.full((n, n_cases), float("nan"), dtype=torch.float32, device="cuda")
    d_hits = torch.full((n,), 12345, dtype=torch.int32, device="cuda")
    return d_nodes, d_fit, d_vals, d_hits


def test_noalloc_matches_allocating_path_on_two_calls(gpu):
    import torch
    x, y, c = synth.problem()
    prob = gpu.Problem(x, y, c)
    stream = torch.cuda.current_stream()
    for seed, count in ((41, 700), (42, 300)):       # two calls in a row, different inputs
        nodes, offs = population(seed, count, 4095)
        fit, vals, hits = reference(gpu, prob, nodes, offs)
        d_nodes, d_fit, d_vals, d_hits = device_buffers(nodes, offs, 48)
        gpu.gp_evaluate_noalloc(prob, offs, d_nodes.data_ptr(), d_fit.data_ptr(), d_vals.data_ptr(),
                                d_hits.data_ptr(), stream)
        torch.cuda.synchronize()
        assert same_f32(d_vals.cpu().numpy(), vals), first_mismatch(d_vals.cpu().numpy(), vals)
        assert same_f32(d_fit.cpu().numpy(), fit), first_mismatch(d_fit.cpu().numpy(), fit)
        assert np.array_equal(d_hits.cpu().numpy().astype(np.uint32), hits)
        assert d_fit[-1].item() == 0.0                # the exact Sextic tree


def test_noalloc_limits(gpu):
    import torch
    x, y, c = synth.problem()
    prob = gpu.Problem(x, y, c)
    rng = np.random.default_rng(3)
    nodes, offs = synth.pack([synth.random_tree(rng, 4097)])
    d_nodes, d_fit, d_vals, d_hits = device_buffers(nodes, offs, 48)
    with pytest.raises(gpu.GpError) as e:                           # tree too large
        gpu.gp_evaluate_noalloc(prob, offs, d_nodes.data_ptr(), d_fit.data_ptr(), d_vals.data_ptr(),
                                d_hits.data_ptr())
    assert e.value.status == gpu.GP_ELIMIT
    many = np.arange(gpu.NOALLOC_MAX_TREES + 2, dtype=np.uint64)    # too many trees
    with pytest.raises(gpu.GpError) as e:
        gpu.gp_evaluate_noalloc(prob, many, d_nodes.data_ptr(), d_fit.data_ptr(), d_vals.data_ptr(),
                                d_hits.data_ptr())
    assert e.value.status == gpu.GP_ELIMIT
    small, soffs = synth.pack([synth.random_tree(rng, 31)])
    d2 = torch.zeros(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(gpu.GpError) as e:                           # misaligned nodes
        gpu.gp_evaluate_noalloc(prob, soffs, d2.data_ptr() + 1, d_fit.data_ptr(), d_vals.data_ptr(),
                                d_hits.data_ptr())
    assert e.value.status == gpu.GP_EINVAL


def test_noalloc_errors_then_recovers(gpu):
    """A stack deeper than the window and malformed trees are reported; the
    next call, on the same static scratch, is exact again."""
    import torch
    x, y, c = synth.problem()
    prob = gpu.Problem(x, y, c)
    rng = np.random.default_rng(8)
    ok = [synth.random_tree(rng, 63) for _ in range(5)]
    deep = synth.left_spine_tree(rng, 600, 1)                       # ~600 values on the stack
    cases = [
        (ok + [deep], gpu.GP_ELIMIT),
        (ok + [np.array([0, 4], np.uint8)], gpu.GP_EMALFORMED),     # operand missing
        (ok + [np.array([4, 4], np.uint8)], gpu.GP_EMALFORMED),     # two trees in one
        (ok + [np.array([0, 4, 200], np.uint8)], gpu.GP_EMALFORMED),  # undefined code
    ]
    for trees, want in cases:
        nodes, offs = synth.pack(trees)
        bufs = device_buffers(nodes, offs, 48)
        with pytest.raises(gpu.GpError) as e:
            gpu.gp_evaluate_noalloc(prob, offs, *(b.data_ptr() for b in bufs))
        assert e.value.status == want
    nodes, offs = synth.pack(ok)
    fit, vals, hits = reference(gpu, prob, nodes, offs)
    d_nodes, d_fit, d_vals, d_hits = device_buffers(nodes, offs, 48)
    gpu.gp_evaluate_noalloc(prob, offs, d_nodes.data_ptr(), d_fit.data_ptr(), d_vals.data_ptr(),
                            d_hits.data_ptr())
    torch.cuda.synchronize()
    assert same_f32(d_vals.cpu().numpy(), vals)
    assert same_f32(d_fit.cpu().numpy(), fit)
    assert np.array_equal(d_hits.cpu().numpy().astype(np.uint32), hits)


def test_noalloc_beside_another_thread_evaluating(gpu):
    """gp_evaluate_noalloc on one host thread while a second thread evaluates
    through gp_evaluate with a launch that needs less shared memory: the
    evaluator's shared-memory limit is only ever raised, so neither thread's
    launches fail and both stay exact."""
    import threading

    import torch
    x, y, c = synth.problem()
    prob = gpu.Problem(x, y, c)
    nodes, offs = population(43, 200, 4095)
    fit, vals, hits = reference(gpu, prob, nodes, offs)
    errors = []

    def other():
        try:
            torch.cuda.set_device(0)
            s = torch.cuda.Stream()
            pop = gpu.gp_create_population(prob, nodes, offs, s)
            for _ in range(40):
                gpu.gp_evaluate(pop, s, warps_per_cta=4, window_entries=16)
                f, _, _ = gpu.gp_fitness(pop)
                if not same_f32(f, fit):
                    errors.append("fitness of the allocating path")
            gpu.gp_destroy_population(pop)
        except Exception as e:                        # reported below
            errors.append(repr(e))

    th = threading.Thread(target=other)
    th.start()
    s = torch.cuda.Stream()
    d_nodes, d_fit, d_vals, d_hits = device_buffers(nodes, offs, 48)
    try:
        for _ in range(40):
            gpu.gp_evaluate_noalloc(prob, offs, d_nodes.data_ptr(), d_fit.data_ptr(), d_vals.data_ptr(),
                                    d_hits.data_ptr(), s)
            s.synchronize()
            assert same_f32(d_fit.cpu().numpy(), fit)
    finally:
        th.join(timeout=300)
    assert not th.is_alive() and not errors, errors
    assert same_f32(d_vals.cpu().numpy(), vals)
    assert np.array_equal(d_hits.cpu().numpy().astype(np.uint32), hits)
