"""Pins for the CPU oracle: what the paper and mathematics fix, checked
against the oracle without using the oracle to produce the expectation."""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_1902_09215_gb300 import synth
from tests import exact

ADD, SUB, MUL, DIV, X = 0, 1, 2, 3, 4


def bits(a):
    return np.asarray(a, dtype=np.float32).view(np.uint32)


def same_f32(a, b):
    """Bit equality, except any NaN equals any NaN."""
    a = np.asarray(a, dtype=np.float32)
    b = np.asarray(b, dtype=np.float32)
    nan = np.isnan(a) & np.isnan(b)
    return bool(np.all(nan | (a.view(np.uint32) == b.view(np.uint32))))


@pytest.fixture(scope="module")
def prob():
    return synth.problem()


def C(k):
    """Byte code of constant table entry k."""
    return 5 + k


# ---------------------------------------------------------------- closed forms

def test_leaf_x_and_constant(oracle, prob):
    x, y, c = prob
    assert same_f32(oracle.eval_tree([X], x, c), x)
    for k in (0, 17, 126):
        assert same_f32(oracle.eval_tree([C(k)], x, c), np.full(48, c[k], np.float32))


def test_closed_forms_tiny_trees(oracle, prob):
    x, y, c = prob
    assert not np.any(x == 0)
    # (/ x x) = 1 exactly for x != 0
    assert same_f32(oracle.eval_tree([DIV, X, X], x, c), np.ones(48, np.float32))
    # (- x x) = +0 (round to nearest: exact cancellation gives +0)
    assert np.all(bits(oracle.eval_tree([SUB, X, X], x, c)) == 0)
    # (/ x (- x x)) is protected: 1.0
    assert same_f32(oracle.eval_tree([DIV, X, SUB, X, X], x, c), np.ones(48, np.float32))
    # (+ x x) = 2x exactly; (* x x) = x^2 correctly rounded (product of two
    # 24-bit significands is exact in double, so one rounding to binary32)
    assert same_f32(oracle.eval_tree([ADD, X, X], x, c), 2 * x)
    sq = (x.astype(np.float64) * x.astype(np.float64)).astype(np.float32)
    assert same_f32(oracle.eval_tree([MUL, X, X], x, c), sq)


def test_operand_order(oracle, prob):
    """First child is the left operand: (- a b) = a - b, (/ a b) = a / b."""
    x, y, c = prob
    a, b = 3, 40
    out_sub = oracle.eval_tree([SUB, C(a), C(b)], x, c)
    out_div = oracle.eval_tree([DIV, C(a), C(b)], x, c)
    ea = Fraction(float(c[a]))
    eb = Fraction(float(c[b]))
    want_sub = exact.to_float(exact.round_to(exact.V(ea - eb), "f32"))
    want_div = exact.to_float(exact.round_to(exact.V(ea / eb), "f32"))
    assert np.all(out_sub == np.float32(want_sub))
    assert np.all(out_div == np.float32(want_div))
    assert want_sub != exact.to_float(exact.round_to(exact.V(eb - ea), "f32"))


def test_mae_of_x_closed_form(oracle, prob):
    x, y, c = prob
    out = oracle.eval_tree([X], x, c)
    f32, hits = oracle.mae_f32(out, y)
    exact_mae = sum(abs(Fraction(float(a)) - Fraction(float(b))) for a, b in zip(x, y)) / 48
    # 48 subtractions + 48 additions + 1 division, each within half an ulp:
    # relative error well under 200 * 2^-24
    assert abs(Fraction(float(f32)) - exact_mae) <= exact_mae * Fraction(200, 2 ** 24)
    y64 = synth.sextic_targets_f64(x)
    f64 = oracle.mae_f64(oracle.eval_tree([X], x, c, dtype=np.float64), y64)
    exact64 = sum(abs(Fraction(float(a)) - Fraction(float(b))) for a, b in zip(x, y64)) / 48
    assert abs(Fraction(f64) - exact64) <= exact64 * Fraction(200, 2 ** 53)
    assert abs(f64 - 0.51064) < 1e-4


# ---------------------------------------------------------------- exact Sextic

def sextic_tree():
    one = [DIV, X, X]                         # (/ x x) = 1
    xm1 = [SUB, X] + one
    xp1 = [ADD, X] + one
    # (* (* (* (* (* x x) (x-1)) (x-1)) (x+1)) (x+1))
    return [MUL, MUL, MUL, MUL, MUL, X, X] + xm1 + xm1 + xp1 + xp1


def test_exact_sextic_tree_zero_error(oracle, prob):
    x, y, c = prob
    t = sextic_tree()
    assert oracle.check_tree(t)
    out = oracle.eval_tree(t, x, c)
    assert same_f32(out, y)
    f, hits = oracle.mae_f32(out, y)
    assert bits(f) == 0 and hits == 48
    y64 = synth.sextic_targets_f64(x)
    out64 = oracle.eval_tree(t, x, c, dtype=np.float64)
    assert np.array_equal(out64, y64)
    assert oracle.mae_f64(out64, y64) == 0.0
    # the FP32 and FP64 target tables differ by at most a few FP32 ulps
    ulp = np.spacing(np.abs(y).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(y.astype(np.float64) - y64) <= 4 * np.maximum(ulp, 2.0 ** -149))


# ---------------------------------------------------------------- protected division

def test_protected_division_special_values(oracle, prob):
    x, _, _ = prob
    tiny = np.float32(1e-45)          # smallest subnormal
    table = np.array([1.5, 0.0, -0.0, tiny, np.nan, np.inf, -np.inf, 0.0], np.float32)
    def div(a, b):
        return oracle.eval_tree([DIV, C(a), C(b)], x, table)[0]
    assert div(0, 1) == 1.0 and div(0, 2) == 1.0          # +0, -0 divisors
    assert div(1, 2) == 1.0                               # 0 / -0 -> 1
    assert div(5, 1) == 1.0                               # inf / 0 -> 1
    assert math.isinf(div(0, 3)) and div(0, 3) > 0        # 1.5 / subnormal overflows
    assert math.isnan(div(0, 4))                          # NaN divisor is not zero
    assert bits(div(0, 5)) == 0                           # 1.5 / +inf = +0
    assert bits(div(0, 6)) == 0x80000000                  # 1.5 / -inf = -0
    # protected value follows the problem definition (1.0 by default)
    assert oracle.eval_tree([DIV, C(0), C(1)], x, table, div0=0.25)[0] == np.float32(0.25)


# ---------------------------------------------------------------- MAE fold order, hits

def test_mae_is_a_sequential_fold_from_zero(oracle):
    # e_0 = 1, e_1..47 = 2^-24: adding half an ulp of 1.0 rounds back to 1.0
    # (ties to even), so a left-to-right fold gives exactly 1.0 / 48, while
    # the exact sum (or any tree-shaped sum of the small terms first) is larger.
    out = np.zeros(48, np.float32)
    out[0] = 1.0
    out[1:] = np.float32(2.0 ** -24)
    y = np.zeros(48, np.float32)
    f, _ = oracle.mae_f32(out, y)
    assert f == np.float32(1.0) / np.float32(48.0)
    rev = out[::-1].copy()
    f2, _ = oracle.mae_f32(rev, y)
    assert f2 > f          # small terms first accumulate before meeting 1.0


def test_hits_threshold_is_strict(oracle):
    y = np.zeros(48, np.float32)
    out = np.full(48, 1.0, np.float32)
    out[0] = np.float32(0.01)                       # exactly 0.01f: not a hit
    out[1] = np.nextafter(np.float32(0.01), np.float32(0))
    out[2] = np.float32(-0.005)
    _, hits = oracle.mae_f32(out, y)
    assert hits == 2


# ---------------------------------------------------------------- structure

def arity_walk_ok(t):
    s = np.cumsum(np.where(np.asarray(t) < 4, 1, -1))
    return s[-1] == -1 and np.all(s[:-1] >= 0)


def test_prefix_invariant_generated_and_malformed(oracle):
    rng = np.random.default_rng(11)
    for n in [1, 3, 5, 31, 63, 1001, 4095]:
        t = synth.random_tree(rng, n)
        assert arity_walk_ok(t)
        assert oracle.check_tree(t)
    t = synth.random_tree(rng, 31)
    assert not oracle.check_tree(t[:-1])                          # truncated
    assert not oracle.check_tree(np.concatenate([t, [4]]))        # trailing node
    # a complete tree followed by an operator and one leaf: the node count
    # balances again, but the walk reached -1 before the last node
    more = np.concatenate([t, [ADD, X]]).astype(np.uint8)
    assert not arity_walk_ok(more) and not oracle.check_tree(more)
    bad = t.copy(); bad[-1] = 5 + 127
    assert not oracle.check_tree(bad)                             # code beyond table
    assert not oracle.check_tree(np.zeros(0, np.uint8))


def py_end(t, i):
    """Subtree end by recursive descent (independent of the oracle's walk)."""
    def rec(k):
        return k + 1 if t[k] >= 4 else rec(rec(k + 1))
    return rec(i)


def test_subtree_end_consistency(oracle):
    rng = np.random.default_rng(5)
    t = synth.random_tree(rng, 301)
    for i in range(len(t)):
        e = oracle.subtree_end(t, i)
        assert e == py_end(t, i)
        if t[i] < 4:
            e1 = oracle.subtree_end(t, i + 1)
            assert oracle.subtree_end(t, e1) == e          # children tile the node
        else:
            assert e == i + 1


def test_tree_depth(oracle):
    assert oracle.tree_depth([X]) == 1
    assert oracle.tree_depth([ADD, X, X]) == 2
    assert oracle.tree_depth([ADD, ADD, X, X, X]) == 3
    assert oracle.tree_depth([ADD, X, ADD, X, ADD, X, X]) == 4
    rng = np.random.default_rng(9)
    t = synth.left_spine_tree(rng, 200, 3)
    assert oracle.tree_depth(t) >= 201


def test_generator_depth_near_flajolet_limit(oracle):
    """Random binary trees have depth about 2 sqrt(pi * ceil(n/2)) (Sec. 2.2,
    Flajolet & Sedgewick); the cycle-lemma generator must be near it."""
    rng = np.random.default_rng(21)
    n = 4001
    d = np.mean([oracle.tree_depth(synth.random_tree(rng, n)) for _ in range(40)])
    lim = 2 * math.sqrt(math.pi * math.ceil(n / 2))
    assert 0.7 * lim < d < 1.1 * lim


# ---------------------------------------------------------------- crossover (Sec. 3.1)

def test_crossover_hand_examples(oracle):
    mum = np.array([ADD, X, MUL, 5, 6], np.uint8)
    dad = np.array([SUB, DIV, 7, 8, 9], np.uint8)
    # leaf for leaf: exactly one byte changes
    ch = oracle.crossover(mum, dad, 1, 4)
    assert list(ch) == [ADD, 9, MUL, 5, 6]
    # root of mum replaced: child is dad's subtree
    assert list(oracle.crossover(mum, dad, 0, 1)) == [DIV, 7, 8]
    assert list(oracle.crossover(mum, dad, 0, 0)) == list(dad)
    # subtree for subtree
    assert list(oracle.crossover(mum, dad, 2, 1)) == [ADD, X, DIV, 7, 8]


def test_crossover_brute_force(oracle):
    rng = np.random.default_rng(8)
    for _ in range(300):
        M = synth.random_tree(rng, int(rng.integers(0, 40)) * 2 + 1)
        D = synth.random_tree(rng, int(rng.integers(0, 40)) * 2 + 1)
        i = int(rng.integers(0, len(M)))
        j = int(rng.integers(0, len(D)))
        want = np.concatenate([M[:i], D[j:py_end(D, j)], M[py_end(M, i):]])
        got = oracle.crossover(M, D, i, j)
        assert np.array_equal(got, want)
        assert arity_walk_ok(got)
        assert len(got) == len(M) - (py_end(M, i) - i) + (py_end(D, j) - j)


# ---------------------------------------------------------------- brute force

@pytest.mark.parametrize("n", [1, 3, 5, 7, 9, 11, 13, 15])
def test_brute_force_all_shapes_exact_rounding(oracle, prob, n):
    """Every tree shape with n <= 15 nodes, random labels: each FP32 (FP64)
    oracle output equals exact rational evaluation with one round-to-nearest-
    even binary32 (binary64) rounding per node."""
    x, y, c = prob
    rng = np.random.default_rng(100 + n)
    shapes = exact.all_shapes(n)
    case_idx = [0, 7, 23, 24, 40, 47]
    for s in shapes:
        t = synth.label_tree(rng, np.array(s, dtype=bool))
        o32 = oracle.eval_tree(t, x, c)
        o64 = oracle.eval_tree(t, x, c, dtype=np.float64)
        for i in case_idx:
            w32 = exact.eval_exact_rounded(t, float(x[i]), c, "f32")
            w64 = exact.eval_exact_rounded(t, float(x[i]), c, "f64")
            assert same_f32(o32[i], w32), (t, i, o32[i], w32)
            assert (math.isnan(o64[i]) and math.isnan(w64)) or \
                np.float64(o64[i]).view(np.uint64) == np.float64(w64).view(np.uint64), (t, i)


def test_brute_force_division_heavy(oracle, prob):
    """Division-only and subtraction-heavy trees (zeros, protected division,
    signed zeros) against the exact evaluator."""
    x, y, c = prob
    rng = np.random.default_rng(77)
    table = np.array([0.5, -0.5, 0.0, -0.0, 0.25, 3.0, -2.0], np.float32)
    for n in (5, 7, 9, 11):
        for s in exact.all_shapes(n):
            t = synth.label_tree(rng, np.array(s, dtype=bool), p_x=0.3, n_consts=7,
                                 ops=(1, 3, 3, 2))
            o = oracle.eval_tree(t, x, table)
            for i in (0, 13, 47):
                w = exact.eval_exact_rounded(t, float(x[i]), table, "f32")
                assert same_f32(o[i], w), (t, i, o[i], w)


def test_fp32_error_bound_vs_exact(oracle, prob):
    """FP32 recursion stays within a derived bound of the exact value on
    random 31-node trees without division (|rel err| <= n_ops * 2^-24 times
    the condition number, checked loosely via the sum of |terms|)."""
    x, y, c = prob
    rng = np.random.default_rng(3)
    for _ in range(30):
        t = synth.random_tree(rng, 31, ops=(0, 2))      # + and * only
        o = oracle.eval_tree(t, x, c)
        absmax = [abs(v) for v in (exact.eval_exact_unrounded(
            [ADD if b == SUB else b for b in t], abs(float(x[i])),
            np.abs(c)) for i in (0, 30)) ]
        for k, i in enumerate((0, 30)):
            ex = exact.eval_exact_unrounded(t, float(x[i]), c)
            bound = absmax[k] * Fraction(15 * 2, 2 ** 24)
            assert abs(Fraction(float(o[i])) - ex) <= bound


def test_population_matches_single_tree_and_threads(oracle):
    x, y, c = synth.problem()
    nodes, offs = synth.population_small()
    r1 = oracle.eval_population(nodes, offs, x, y, c, n_threads=1, want_f64=True)
    r4 = oracle.eval_population(nodes, offs, x, y, c, n_threads=4, want_f64=True)
    assert same_f32(r1["out"], r4["out"]) and same_f32(r1["fitness"], r4["fitness"])
    assert np.array_equal(r1["hits"], r4["hits"])
    for t in (0, 7, 49):
        tree = nodes[int(offs[t]):int(offs[t + 1])]
        o = oracle.eval_tree(tree, x, c)
        assert same_f32(r1["out"][t], o)
        f, h = oracle.mae_f32(o, y)
        assert same_f32(r1["fitness"][t], f) and r1["hits"][t] == h


def test_paper_grid_code_range(oracle):
    """With the paper's 250 constants, codes 5..254 are leaves and 255 is not
    a code (Sec. 2.1: one byte per node)."""
    assert oracle.check_tree(np.array([0, 254, 4], np.uint8), n_consts=250)
    assert not oracle.check_tree(np.array([0, 255, 4], np.uint8), n_consts=250)
    assert not oracle.check_tree(np.array([0, 132, 4], np.uint8), n_consts=127)
    x, _, _ = synth.problem()
    c = synth.paper_grid_constants()
    out = oracle.eval_tree(np.array([254], np.uint8), x, c)
    assert np.all(out == c[249])
