"""FP32 evaluation error against FP64, per workload, from the oracle alone.

TEST INFRASTRUCTURE ONLY (calls oracle/ and the seeded generators).  The
CUDA path's FP32 results equal the FP32 oracle's bit for bit (GPU parity
tests), so these numbers are the GPU's FP32 error too.

For every tree: fitness in FP32 (FP32 cases, FP32 targets, FP32 fold, Sec.
2.2 / Table gp.details) and in FP64 (the same tables widened, FP64 targets,
FP64 fold).  Reported: the relative fitness error |f32 - f64| / |f64|
(median, 99th percentile, maximum over the trees whose FP64 fitness is
finite), the share of trees above 1e-3 relative, and the largest per-case
relative error among trees below that threshold.  Large errors come from
protected division whose divisor is 0 in FP32 but not in FP64 (or the
reverse) and from cancellation; they are counted, not hidden.

    python oracle/fp32_vs_fp64.py [--full]       (--full adds the 4.5e9-node workload)
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import oracle  # noqa: E402
from paper_1902_09215_gb300 import synth  # noqa: E402


def report(name, nodes, offs):
    x, y, c = synth.problem()
    r = oracle.eval_population(nodes, offs, x, y, c, n_threads=os.cpu_count() or 1, want_f64=True)
    f32 = r["fitness"].astype(np.float64)
    f64 = r["fitness64"]
    ok = np.isfinite(f64) & np.isfinite(f32) & (np.abs(f64) > 0)
    rel = np.abs(f32[ok] - f64[ok]) / np.abs(f64[ok])
    big = rel > 1e-3
    out32 = r["out"].astype(np.float64)[ok][~big]
    out64 = r["out64"][ok][~big]
    m = np.isfinite(out64) & np.isfinite(out32) & (np.abs(out64) > 1e-30)
    case_rel = np.abs(out32[m] - out64[m]) / np.abs(out64[m])
    return {
        "workload": name, "trees": int(offs.shape[0] - 1), "nodes": int(offs[-1]),
        "fitness_rel_err_median": float(np.median(rel)) if rel.size else None,
        "fitness_rel_err_p99": float(np.quantile(rel, 0.99)) if rel.size else None,
        "fitness_rel_err_max": float(rel.max()) if rel.size else None,
        "share_above_1e-3": float(big.mean()) if rel.size else None,
        "trees_not_compared": int((~ok).sum()),
        "case_rel_err_max_below_threshold": float(case_rel.max()) if case_rel.size else None,
    }


def main():
    oracle.build()
    rows = [
        report("50 trees, 1..63 nodes (seed 1)", *synth.population_small()),
        report("4000 trees, log-uniform 31..32767 (seed 3)", *synth.population_loguniform(seed=3)),
        report("48 bloated trees, 1e4..4e6 nodes (seed 4, 1/100 scale)",
               *synth.graft_population(seed=4, count=48, lo=10**4, hi=4 * 10**6, donor_lo=10**3,
                                       donor_hi=10**4, n_donors=16, chain_depth=10**4, chain_lo=2000,
                                       chain_hi=5000, n_chain=8)[:2]),
    ]
    if "--full" in sys.argv:
        rows.append(report("48 bloated trees, 1e6..4e8 nodes (seed 4)", *synth.graft_population()[:2]))
    for r in rows:
        print(json.dumps(r))


if __name__ == "__main__":
    main()
