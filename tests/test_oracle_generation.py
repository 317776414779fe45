"""Pins for the oracle's generation step: the counter-based draws, the
unbiased bounded draw, tournament selection and the crossover records.
Each check rests on something outside the oracle: a published test vector,
an exact special case, or a closed-form distribution (chi-square)."""
import math

import numpy as np
import pytest

from paper_1902_09215_gb300 import synth

# SplitMix64 seeded with 1234567: its first five outputs as published with
# the generator's reference implementation.
SPLITMIX64_1234567 = [6457827717110365317, 3203168211198807973, 9817491932198370423,
                      4593380528125082431, 16408922859458223821]


def chi2_ok(counts, probs, alpha_sigma=6.0):
    """Pearson chi-square within mean + alpha_sigma * sd (df = bins - 1)."""
    counts = np.asarray(counts, dtype=np.float64)
    exp = counts.sum() * np.asarray(probs, dtype=np.float64)
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    df = len(counts) - 1
    return chi2 < df + alpha_sigma * math.sqrt(2 * df), chi2


def test_sm64_published_vector(oracle):
    assert [oracle.sm64_at(1234567, i) for i in range(5)] == SPLITMIX64_1234567


def test_sm64_counter_is_the_sequence(oracle):
    """Output i of the counter form is the i-th output of the sequential
    generator (synth's sequential SplitMix64)."""
    seq = [int(v) for v in synth.splitmix64(987654321, 50)]
    assert [oracle.sm64_at(987654321, i) for i in range(50)] == seq


def test_bounded_power_of_two_is_top_bits(oracle):
    """n = 2^k: 2^64 mod n = 0, nothing is rejected, and the high word of
    r * 2^k is the top k bits of r."""
    for k in (1, 3, 10, 31, 63):
        for base in (0, 16, 12345 << 4):
            assert oracle.bounded(77, base, 1 << k) == oracle.sm64_at(77, base) >> (64 - k)


def test_bounded_one_and_range(oracle):
    assert all(oracle.bounded(5, b << 4, 1) == 0 for b in range(100))
    for n in (2, 3, 7, 1000, (1 << 40) + 7, (1 << 64) - 1):
        assert all(0 <= oracle.bounded(9, b << 4, n) < n for b in range(200))


def test_bounded_uniform_small_n(oracle):
    for n in (7, 48):
        counts = np.bincount([oracle.bounded(3, b << 4, n) for b in range(20000)], minlength=n)
        ok, chi2 = chi2_ok(counts, np.full(n, 1.0 / n))
        assert ok, (n, chi2)


def test_bounded_rejection_removes_bias(oracle):
    """n = 3 * 2^62: without rejection the high word floor(3r/4) takes values
    divisible by 3 twice as often (probability 1/2 instead of 1/3)."""
    n = 3 << 62
    v = np.array([oracle.bounded(11, b << 4, n) % 3 == 0 for b in range(30000)])
    frac = v.mean()
    assert abs(frac - 1 / 3) < 0.015, frac


def test_tournament_trivial_cases(oracle):
    assert all(oracle.tournament(np.array([0.5], np.float32), 1, 0, c, 0, 7) == 0 for c in range(50))
    # equal fitness everywhere: the winner is the first entrant drawn
    f = np.full(100, 0.25, np.float32)
    for c in range(200):
        assert oracle.tournament(f, 4, 2, c, 1, 7) == oracle.bounded(4, oracle.draw_counter(2, c, 1, 0), 100)


def test_tournament_size_one_is_uniform(oracle):
    f = np.random.default_rng(0).random(10).astype(np.float32)
    counts = np.bincount([oracle.tournament(f, 8, 0, c, 0, 1) for c in range(20000)], minlength=10)
    ok, chi2 = chi2_ok(counts, np.full(10, 0.1))
    assert ok, chi2


def test_tournament_winner_rank_distribution(oracle):
    """Distinct fitness, T entrants with replacement from P: the winner has
    rank r (0 = best) with probability ((P-r)/P)^T - ((P-r-1)/P)^T."""
    P, T = 20, 7
    rng = np.random.default_rng(1)
    f = rng.permutation(P).astype(np.float32) * 0.125
    rank = np.argsort(np.argsort(f))
    wins = [rank[oracle.tournament(f, 21, 3, c, 0, T)] for c in range(40000)]
    counts = np.bincount(wins, minlength=P)
    probs = np.array([((P - r) / P) ** T - ((P - r - 1) / P) ** T for r in range(P)])
    keep = probs * len(wins) >= 5                       # pool sparse tail bins
    c2 = np.append(counts[keep], counts[~keep].sum())
    p2 = np.append(probs[keep], probs[~keep].sum())
    ok, chi2 = chi2_ok(c2, p2)
    assert ok, chi2


def test_tournament_nan_is_worst(oracle):
    """P = 2 with one NaN: the NaN wins only if it is the only entrant
    drawn, probability 2^-T."""
    T = 3
    f = np.array([np.nan, 5.0], np.float32)
    wins0 = sum(oracle.tournament(f, 6, 0, c, 0, T) == 0 for c in range(16000))
    assert abs(wins0 / 16000 - 2.0 ** -T) < 0.01, wins0
    g = np.array([np.inf, np.nan], np.float32)         # +Inf ties NaN: first entrant
    for c in range(100):
        assert oracle.tournament(g, 6, 0, c, 0, T) == oracle.bounded(6, oracle.draw_counter(0, c, 0, 0), 2)


def test_generation_records_points_uniform_and_in_range(oracle):
    P, M = 50, 4000
    rng = np.random.default_rng(2)
    sizes = np.full(P, 11, np.uint64)
    fit = rng.random(P).astype(np.float32)
    mum, dad, mp, dp = oracle.generation_records(fit, sizes, M, seed=13, g=0)
    assert mum.max() < P and dad.max() < P and mp.max() < 11 and dp.max() < 11
    for pts in (mp, dp):
        ok, chi2 = chi2_ok(np.bincount(pts.astype(np.int64), minlength=11), np.full(11, 1 / 11))
        assert ok, chi2
    # tournament selection favours fitter parents: the best tree is chosen
    # far more often than the worst
    best, worst = int(np.argmin(fit)), int(np.argmax(fit))
    assert np.sum(mum == best) > 20 * max(1, np.sum(mum == worst))


def test_generation_records_parents_and_points_independent(oracle):
    """Both parents come from tournaments of their own (Table gp.details):
    mum == dad happens with probability sum_r p_r^2, p_r the rank-r winning
    probability of a size-T tournament.  Each point is uniform over the nodes
    of its own parent (Sec. 3.1), whatever the other parent's size."""
    P, T, M = 40, 7, 20000
    rng = np.random.default_rng(4)
    fit = rng.permutation(P).astype(np.float32) * 0.5
    sizes = (1 + 2 * rng.permutation(P)).astype(np.uint64)          # 1, 3, .., 79
    mum, dad, mp, dp = oracle.generation_records(fit, sizes, M, seed=17, g=3, tsize=T)
    pr = np.array([((P - r) / P) ** T - ((P - r - 1) / P) ** T for r in range(P)])
    q = float((pr ** 2).sum())
    same = float(np.mean(mum == dad))
    assert abs(same - q) < 6 * math.sqrt(q * (1 - q) / M), (same, q)
    assert np.all(mp < sizes[mum]) and np.all(dp < sizes[dad])
    best = int(np.argmin(fit))
    for who, pts in ((mum, mp), (dad, dp)):
        sel = pts[who == best].astype(np.int64)
        s = int(sizes[best])
        if s > 1:
            ok, chi2 = chi2_ok(np.bincount(sel, minlength=s), np.full(s, 1.0 / s))
            assert ok, chi2


def test_generation_records_deterministic_and_distinct(oracle):
    P = 30
    rng = np.random.default_rng(3)
    sizes = (1 + 2 * rng.integers(0, 20, P)).astype(np.uint64)
    fit = rng.random(P).astype(np.float32)
    a = oracle.generation_records(fit, sizes, 100, seed=5, g=7)
    b = oracle.generation_records(fit, sizes, 100, seed=5, g=7)
    c = oracle.generation_records(fit, sizes, 100, seed=5, g=8)
    d = oracle.generation_records(fit, sizes, 100, seed=6, g=7)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert not np.array_equal(a[2], c[2]) and not np.array_equal(a[2], d[2])
    # the child index only selects counters: child c of a longer list is the same
    e = oracle.generation_records(fit, sizes, 150, seed=5, g=7)
    assert all(np.array_equal(x, y[:100]) for x, y in zip(a, e))


def test_generation_rejects_bad_arguments(oracle):
    f = np.zeros(4, np.float32)
    s = np.ones(4, np.uint64)
    with pytest.raises(oracle.OracleError):
        oracle.generation_records(f, s, 10, seed=1, g=0, tsize=33)
    with pytest.raises(oracle.OracleError):
        oracle.generation_records(f, s, 10, seed=1, g=1 << 24)


def test_child_size_bound(oracle):
    """The arena a crossover sizes without reading the children back rests on
    child size <= n_mum + n_dad - dad_point - 1 (the child keeps at most
    mum's nodes other than the one at the crossover point, and gains at most
    dad's nodes from dad_point on).  Checked on the oracle's children for
    random points, and exact when mum's subtree is a leaf and dad's subtree
    runs to the end of dad."""
    rng = np.random.default_rng(77)
    trees = [synth.random_tree(rng, int(n)) for n in rng.choice(np.arange(1, 400, 2), 60)]
    nodes, offs = synth.pack(trees)
    sizes = np.diff(offs.astype(np.int64))
    mum, dad, mp, dp = synth.crossover_points(9, sizes, 500)
    kn, ko = oracle.crossover_population(nodes, offs, mum, dad, mp, dp)
    child = np.diff(ko.astype(np.int64))
    bound = sizes[mum] + sizes[dad] - dp.astype(np.int64) - 1
    assert np.all(child <= bound)
    # equality: mum's point a leaf, dad's point the root (its subtree is all of dad)
    m_leaf = [(t, int(np.nonzero(tr >= 4)[0][0])) for t, tr in enumerate(trees)]
    mum2 = np.array([t for t, _ in m_leaf], np.uint32)
    mp2 = np.array([i for _, i in m_leaf], np.uint64)
    dad2 = np.roll(mum2, 1)
    dp2 = np.zeros_like(mp2)
    kn2, ko2 = oracle.crossover_population(nodes, offs, mum2, dad2, mp2, dp2)
    child2 = np.diff(ko2.astype(np.int64))
    assert np.array_equal(child2, sizes[mum2] + sizes[dad2] - 1)
