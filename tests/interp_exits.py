"""A CPU count of where the level-0 byte-code interpreter leaves its PTX
group loop, for the evaluator's design notes and tests/test_interp_exits.py.

The model follows eval_item's byte-code path in gp_eval.cu: an item's codes
are read right to left with the top of stack in a register and `d` values
in a window of K entries (`g` more spilled below it).  The PTX loop runs
while the stack has a value; it stops before a word (four codes, the word's
highest position first) that lacks room for four pushes, and at an operator
that finds the window empty.  The C++ side then spills (down to K/2 window
entries), refills (up to K/2), or takes checked steps: the item's first
codes up to its first leaf, and an operator whose arguments lie beyond the
chunk (a spine operator, sent to the upper tree) with the codes after it up
to the next leaf.  `sent` counts the values that spine operators send
upward with themselves.

    python -m tests.interp_exits [K] [C]

prints the counts per 1000 codes for the 4000 children of the benchmark's
generation step (seed-3 population, seed-11 crossover records), chunks of C
codes ending at low points of the arity walk.
"""
from __future__ import annotations

import sys

EVENTS = ("codes", "enters", "checked", "spine", "sent", "spill", "spill_entries", "refill", "refill_entries")


def count_exits(tree, b: int, e: int, K: int = 32, ev: dict | None = None):
    """Counts for the item tree[b:e) added to `ev`; returns (have, d, g),
    the stack left at the item's left end."""
    ev = {k: 0 for k in EVENTS} if ev is None else ev
    ev["codes"] += e - b
    d = g = 0
    have = False
    in_loop = False
    i = e - 1
    while i >= b:
        c = int(tree[i])
        if not have:                       # checked step on the C++ side
            ev["checked"] += 1
            in_loop = False
            if c >= 4:
                have = True
            else:
                ev["spine"] += 1
            i -= 1
            continue
        if not in_loop:
            if d > K - 4:
                h = d - K // 2
                ev["spill"] += 1; ev["spill_entries"] += h; g += h; d -= h
            ev["enters"] += 1
            in_loop = True
        if (i & 15) % 4 == 3 and d > K - 4:          # word without room: spill
            h = d - K // 2
            ev["spill"] += 1; ev["spill_entries"] += h; g += h; d -= h
            in_loop = False
            continue
        if c >= 4:
            d += 1
        elif d > 0:
            d -= 1
        else:                              # operator with the window empty
            in_loop = False
            if g > 0:
                h = min(g, K // 2)
                ev["refill"] += 1; ev["refill_entries"] += h; g -= h; d += h
                continue
            ev["spine"] += 1
            ev["sent"] += 1                # its first argument, the top of stack, goes upward
            ev["checked"] += 1
            have = False
        i -= 1
    return have, d, g


def bench_children_counts(K: int = 32, C: int = 4096) -> dict:
    from oracle import oracle as O
    from paper_1902_09215_gb300 import synth
    from tests.chunk_rules import low_point_ends
    nodes, offs = synth.population_loguniform(seed=3)
    sizes = (offs[1:] - offs[:-1]).astype("int64")
    mum, dad, mp, dp = synth.crossover_points(11, sizes, 4000)
    kn, ko = O.crossover_population(nodes, offs, mum, dad, mp, dp)
    ko = ko.astype("int64")
    ev = {k: 0 for k in EVENTS}
    for t in range(ko.shape[0] - 1):
        tree = kn[ko[t]:ko[t + 1]]
        n = tree.shape[0]
        ends = low_point_ends(tree, C) if n > C else []
        for b, e in zip([0] + ends, ends + [n]):
            count_exits(tree, b, e, K, ev)
    return ev


if __name__ == "__main__":
    K = int(sys.argv[1]) if len(sys.argv) > 1 else 32
    C = int(sys.argv[2]) if len(sys.argv) > 2 else 4096
    ev = bench_children_counts(K, C)
    n = ev["codes"]
    for k in EVENTS[1:]:
        print(f"{k:>15}: {ev[k]:9d}  {1000.0 * ev[k] / n:7.2f} per 1000 codes")
