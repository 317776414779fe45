"""Planted mistakes in the CPU oracle, for tests/test_oracle_mutants.py.

Each mutant is one plausible slip in oracle/gp_oracle.c (a swapped operand,
a dropped absolute value, an off-by-one index, a wrong comparison, a wrong
random-stream counter), written as an exact text substitution.  A mutant is
compiled on the CPU into a library of its own and the oracle's pins (the
tests in test_oracle_pins.py and test_oracle_generation.py, which rest on
the paper, closed forms, exact rational arithmetic, published vectors and
distributions, never on the oracle itself) are run against it in a child
process.  Every mutant must make at least one pin fail: that is the evidence
that the pins would catch such a mistake in the oracle.

Mutants that cannot change any result are not listed (for instance an FP32
product computed in double and rounded once, which is the same number), nor
mistakes that would make the oracle read or write outside its buffers.

    python -m tests.oracle_mutants LIB [--all]

runs the pins against the oracle library LIB and prints one JSON line: the
first pin that fails (or, with --all, every failing pin).
"""
from __future__ import annotations

import json
import sys
import traceback

# (name, text in gp_oracle.c, replacement, occurrence of the text: 0 = first)
MUTANTS = [
    # ---- recursive EVAL, binary32 (Sec. 2.2, Table gp.details)
    ("eval32: '-' operands swapped",
     "out[i] = a[i] - b[i];", "out[i] = b[i] - a[i];", 0),
    ("eval32: '/' operands swapped",
     "(b[i] != 0.0f) ? a[i] / b[i]", "(b[i] != 0.0f) ? b[i] / a[i]", 0),
    ("eval32: '/' through a reciprocal",
     "(b[i] != 0.0f) ? a[i] / b[i]", "(b[i] != 0.0f) ? a[i] * (1.0f / b[i])", 0),
    ("eval32: protection tests the dividend",
     "(b[i] != 0.0f) ?", "(a[i] != 0.0f) ?", 0),
    ("eval32: protected value fixed at 1",
     ": s->div0; break;", ": 1.0f; break;", 0),
    ("eval32: second argument evaluated first",
     "eval32(s, a);            /* first argument  */\n    eval32(s, b);",
     "eval32(s, b);            /* first argument  */\n    eval32(s, a);", 0),
    ("eval32: x leaf reads the cases in reverse",
     "out[i] = s->x[i];", "out[i] = s->x[s->ncases - 1 - i];", 0),
    ("eval32: first constant code taken for an operator",
     "if (op >= CONST0) {", "if (op > CONST0) {", 0),
    ("codes: ADD and SUB exchanged",
     "ADD = 0, SUB = 1,", "ADD = 1, SUB = 0,", 0),
    ("codes: MUL and DIV exchanged",
     "MUL = 2, DIV = 3,", "MUL = 3, DIV = 2,", 0),
    # ---- recursive EVAL, binary64
    ("eval64: '-' operands swapped",
     "out[i] = a[i] - b[i];", "out[i] = b[i] - a[i];", 1),
    ("eval64: '/' operands swapped",
     "(b[i] != 0.0) ? a[i] / b[i]", "(b[i] != 0.0) ? b[i] / a[i]", 0),
    ("eval64: protection tests the dividend",
     "(b[i] != 0.0) ?", "(a[i] != 0.0) ?", 0),
    ("eval64: protected value 0",
     ": s->div0; break;", ": 0.0; break;", 1),
    ("eval64: second argument evaluated first",
     "eval64(s, a);\n    eval64(s, b);", "eval64(s, b);\n    eval64(s, a);", 0),
    ("eval64: '*' rounded to binary32",
     "out[i] = a[i] * b[i]; break;", "out[i] = (float)(a[i] * b[i]); break;", 1),
    ("eval64: '+' rounded to binary32",
     "out[i] = a[i] + b[i]; break;", "out[i] = (float)(a[i] + b[i]); break;", 1),
    # ---- fitness (Table gp.details, Sec. 3.2)
    ("mae_f32: absolute value dropped",
     "float e = fabsf(out[i] - y[i]);", "float e = (out[i] - y[i]);", 0),
    ("mae_f32: hit threshold inclusive",
     "if (e < 0.01f) h++;", "if (e <= 0.01f) h++;", 0),
    ("mae_f32: mean over n - 1 cases",
     "return s / (float)n_cases;", "return s / (float)(n_cases - 1);", 0),
    ("mae_f32: first case skipped",
     "for (i = 0; i < n_cases; i++) {", "for (i = 1; i < n_cases; i++) {", 0),
    ("mae_f32: cases folded last to first",
     "float e = fabsf(out[i] - y[i]);",
     "float e = fabsf(out[n_cases - 1 - i] - y[n_cases - 1 - i]);", 0),
    ("mae_f32: sum kept in binary64",
     "float s = 0.0f;", "double s = 0.0;", 0),
    ("mae_f64: absolute value dropped",
     "s = s + fabs(out[i] - y[i]);", "s = s + (out[i] - y[i]);", 0),
    ("mae_f64: mean over n - 1 cases",
     "return s / (double)n_cases;", "return s / (double)(n_cases - 1);", 0),
    # ---- tree structure (Sec. 2.1, 3.1)
    ("check_tree: nodes after a complete tree not refused",
     "if (need <= 0) return 0;\n", "", 0),
    ("check_tree: last code of the table refused one too late",
     "if (t[k] >= CONST0 + n_consts) return 0;", "if (t[k] > CONST0 + n_consts) return 0;", 0),
    ("check_tree: DIV counted as a leaf",
     "need += (t[k] < XVAR) ? 1 : -1;", "need += (t[k] < DIV) ? 1 : -1;", 0),
    ("subtree_end: x counted as an operator",
     "need += (t[k] < XVAR) ? 1 : -1;", "need += (t[k] <= XVAR) ? 1 : -1;", 1),
    ("subtree_end: end one node short",
     "*end = k;", "*end = k - 1;", 0),
    ("tree_depth: the root at depth 0",
     "if (top + 1 > best) best = top + 1;", "if (top > best) best = top;", 0),
    ("crossover: mum's tail taken from the point instead of the subtree end",
     "memcpy(child + i + (ed - j), mum + em, n_m - em);",
     "memcpy(child + i + (ed - j), mum + i + 1, n_m - em);", 0),
    ("crossover: dad's subtree copied from one node early",
     "memcpy(child + i, dad + j, ed - j);", "memcpy(child + i, dad + (j ? j - 1 : 0), ed - j);", 0),
    # ---- draws, tournaments and crossover records (Table gp.details, Sec. 3.1)
    ("SplitMix64: output i uses i Weyl steps",
     "z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;", "z = seed + i * 0x9E3779B97F4A7C15ull;", 0),
    ("SplitMix64: first mixing shift 31",
     "z = (z ^ (z >> 30)) *", "z = (z ^ (z >> 31)) *", 0),
    ("SplitMix64: Weyl increment off by two",
     "0x9E3779B97F4A7C15ull", "0x9E3779B97F4A7C17ull", 0),
    ("bounded: no rejection",
     "const uint64_t t = (0 - n) % n;", "const uint64_t t = 0;", 0),
    ("bounded: low word modulo n",
     "return (uint64_t)(m >> 64);", "return (uint64_t)m % n;", 0),
    ("bounded: every attempt on the same counter",
     "oracle_sm64_at(seed, base + (uint64_t)a)", "oracle_sm64_at(seed, base)", 0),
    ("tournament: ties go to the last entrant drawn",
     "if (k == 0 || f < best_f) {", "if (k == 0 || f <= best_f) {", 0),
    ("tournament: the largest fitness wins",
     "if (k == 0 || f < best_f) {", "if (k == 0 || f > best_f) {", 0),
    ("tournament: NaN not ranked worst",
     "isnan(fitness[e]) ? INFINITY : fitness[e]", "fitness[e]", 0),
    ("tournament: every entrant from one counter",
     "draw_counter(g, c, purpose, k, 0)", "draw_counter(g, c, purpose, 0, 0)", 0),
    ("generation: dad from mum's tournament stream",
     "dad[c] = oracle_tournament(fitness, n_pop, seed, g, c, 1, tsize);",
     "dad[c] = oracle_tournament(fitness, n_pop, seed, g, c, 0, tsize);", 0),
    ("generation: dad's point bounded by mum's size",
     "draw_counter(g, c, 3, 0, 0), sizes[dad[c]]", "draw_counter(g, c, 3, 0, 0), sizes[mum[c]]", 0),
]


def mutate(src: str, find: str, repl: str, occurrence: int) -> str:
    """src with the given occurrence of `find` replaced; raises if absent."""
    at = -1
    for _ in range(occurrence + 1):
        at = src.find(find, at + 1)
        if at < 0:
            raise ValueError(f"mutant text not found: {find!r} (occurrence {occurrence})")
    return src[:at] + repl + src[at + len(find):]


def pins():
    """(name, callable) for every oracle pin, cheapest first."""
    from paper_1902_09215_gb300 import synth
    from tests import test_oracle_generation as G
    from tests import test_oracle_pins as P
    prob = synth.problem()
    out = []

    def add(mod, name, *extra):
        fn = getattr(mod, name)
        params = list(fn.__code__.co_varnames[:fn.__code__.co_argcount])
        out.append((name + (f"[{extra[0]}]" if extra else ""),
                    lambda O, fn=fn, params=params, extra=extra:
                    fn(*[O if p == "oracle" else prob if p == "prob" else extra[0] for p in params])))

    for name in ["test_leaf_x_and_constant", "test_closed_forms_tiny_trees", "test_operand_order",
                 "test_mae_of_x_closed_form", "test_exact_sextic_tree_zero_error",
                 "test_protected_division_special_values", "test_mae_is_a_sequential_fold_from_zero",
                 "test_hits_threshold_is_strict", "test_prefix_invariant_generated_and_malformed",
                 "test_subtree_end_consistency", "test_tree_depth", "test_crossover_hand_examples",
                 "test_paper_grid_code_range"]:
        add(P, name)
    for name in ["test_sm64_published_vector", "test_sm64_counter_is_the_sequence",
                 "test_bounded_power_of_two_is_top_bits", "test_bounded_one_and_range",
                 "test_tournament_trivial_cases", "test_generation_rejects_bad_arguments",
                 "test_generation_records_deterministic_and_distinct",
                 "test_generation_records_points_uniform_and_in_range",
                 "test_generation_records_parents_and_points_independent",
                 "test_bounded_uniform_small_n", "test_bounded_rejection_removes_bias",
                 "test_tournament_size_one_is_uniform", "test_tournament_nan_is_worst",
                 "test_tournament_winner_rank_distribution", "test_child_size_bound"]:
        add(G, name)
    for name in ["test_crossover_brute_force", "test_brute_force_division_heavy",
                 "test_fp32_error_bound_vs_exact", "test_population_matches_single_tree_and_threads",
                 "test_generator_depth_near_flajolet_limit"]:
        add(P, name)
    for n in (1, 3, 5, 7, 9, 11, 13, 15):
        add(P, "test_brute_force_all_shapes_exact_rounding", n)
    return out


def run(lib_path: str, run_all: bool = False) -> dict:
    import pytest

    from oracle import oracle as O
    O.build = lambda force=False: lib_path     # load this library, never rebuild
    O._lib = None
    failed = []
    for name, call in pins():
        try:
            call(O)
        except (Exception, pytest.fail.Exception) as e:   # an assertion, an oracle error, pytest.raises
            failed.append({"pin": name, "error": type(e).__name__,
                           "where": traceback.format_exc(limit=-1).strip().splitlines()[-1][:200]})
            if not run_all:
                break
    return {"lib": lib_path, "failed": failed}


if __name__ == "__main__":
    print(json.dumps(run(sys.argv[1], "--all" in sys.argv[2:])))
