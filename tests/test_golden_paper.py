"""Sanity checks against numbers the paper prints (tests/golden/paper_printed.json).

The paper's own fitness cases and constants are not printed, so none of these
can pin bits; they check that the oracle's semantics are consistent with
what the paper reports (parity against the paper's data stays unpinned)."""
import json
import os

import numpy as np

from paper_1902_09215_gb300 import synth

G = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_printed.json")))


def test_three_node_constants_reachable_from_paper_grid(oracle):
    """Each printed three-node constant is (op a b) for grid constants a, b in
    [-0.995, 0.997] (step 0.001, no 0) under FP32 with protected division,
    printed to 6 significant digits."""
    ks = np.array([k for k in range(-995, 998) if k != 0])
    grid = (ks / 1000.0).astype(np.float32)
    A, B = np.meshgrid(grid, grid, indexing="ij")
    with np.errstate(all="ignore"):
        cand = {0: A + B, 1: A - B, 2: A * B, 3: np.where(B != 0, A / B, np.float32(1))}
    x = synth.cases()
    for v in G["three_node_constant_trees"]["values"]:
        found = None
        for op, vals in cand.items():
            # candidates within a few units of the 6th significant digit
            hit = np.argwhere(np.abs(vals.astype(np.float64) - v) <= 5e-6 * abs(v))
            for i, j in hit:
                if "%.6g" % float(vals[i, j]) == "%.6g" % v:
                    found = (op, grid[i], grid[j])
                    break
            if found:
                break
        assert found is not None, v
        op, a, b = found
        out = oracle.eval_tree([op, 5, 6], x, np.array([a, b], np.float32))
        assert "%.6g" % float(out[0]) == "%.6g" % v


def test_constant_tree_fitness_magnitude(oracle):
    """The paper's constant tree 0.0769947 scores MAE 0.0462157 with 4 hits on
    its 48 random cases; on the evenly spaced stand-in cases the MAE must be
    of the same size (within 5 percent) and hits a handful."""
    x, y, _ = synth.problem()
    c = np.array([G["constant_tree"]["value"]], np.float32)
    out = oracle.eval_tree([5], x, c)
    f, hits = oracle.mae_f32(out, y)
    paper = -G["constant_tree"]["fitness"]
    assert abs(float(f) - paper) / paper < 0.05
    assert 0 < hits <= 8


def test_stand_in_tables_match_paper_ranges():
    x = synth.cases()
    assert x.shape[0] == G["fitness_cases"]["n"]
    assert x.min() >= -1.0 and x.max() <= 1.0
    c = synth.paper_grid_constants()
    assert c.shape[0] == G["constants"]["n"]
    assert np.all(c != 0) and c.min() >= -0.999 and c.max() <= 0.999
