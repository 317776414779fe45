"""Expected results for a sample of the children of one generation, from the
oracle alone, for populations too large to run the oracle's whole
generation on.

A child's two tournaments draw their entrants from the counter-based stream
(generation, child, purpose, entrant index), which does not depend on
fitness (Table gp.details: size-7 tournaments; Sec. 3.1: points chosen in a
fixed order).  So only the entrants of the sampled children need the
oracle's fitness; the oracle's own tournament then picks each parent, the
oracle's bounded draw picks each point, the oracle's three-segment copy
makes the child and the oracle's EVAL scores it.  Nothing here comes from
the CUDA path."""
import numpy as np


def gather(nodes, offs, trees):
    """The listed trees packed as (nodes, offsets)."""
    offs = np.asarray(offs, dtype=np.uint64)
    parts = [nodes[int(offs[t]):int(offs[t + 1])] for t in trees]
    sizes = np.array([p.shape[0] for p in parts], dtype=np.uint64)
    o = np.zeros(len(parts) + 1, dtype=np.uint64)
    np.cumsum(sizes, out=o[1:])
    return (np.concatenate(parts) if parts else np.zeros(0, np.uint8)), o


def expected_children(oracle, nodes, offs, tables, seed, g, children, tsize=7, n_threads=1):
    """Records, bytes and evaluation of `children` of generation g (made
    from the population (nodes, offs), whose own index is g)."""
    x, y, c = tables
    offs = np.asarray(offs, dtype=np.uint64)
    sizes = np.diff(offs.astype(np.int64))
    n_pop = int(sizes.shape[0])
    entrants = set()
    for ch in children:
        for purpose in (0, 1):
            for k in range(tsize):
                entrants.add(oracle.bounded(seed, oracle.draw_counter(g, int(ch), purpose, k), n_pop))
    need = sorted(entrants)
    sub_nodes, sub_offs = gather(nodes, offs, need)
    need_fit = oracle.eval_population(sub_nodes, sub_offs, x, y, c, n_threads=n_threads)["fitness"]
    # trees that are never drawn are never read by the tournament
    fit = np.full(n_pop, np.inf, dtype=np.float32)
    fit[need] = need_fit
    recs = []
    for ch in children:
        mum = oracle.tournament(fit, seed, g, int(ch), 0, tsize)
        dad = oracle.tournament(fit, seed, g, int(ch), 1, tsize)
        mp = oracle.bounded(seed, oracle.draw_counter(g, int(ch), 2), int(sizes[mum]))
        dp = oracle.bounded(seed, oracle.draw_counter(g, int(ch), 3), int(sizes[dad]))
        recs.append((mum, dad, mp, dp))
    mum = np.array([r[0] for r in recs], dtype=np.uint32)
    dad = np.array([r[1] for r in recs], dtype=np.uint32)
    mp = np.array([r[2] for r in recs], dtype=np.uint64)
    dp = np.array([r[3] for r in recs], dtype=np.uint64)
    kids, koffs = oracle.crossover_population(nodes, offs, mum, dad, mp, dp)
    ev = oracle.eval_population(kids, koffs, x, y, c, n_threads=n_threads)
    return {"parents": np.array(need, dtype=np.int64), "parent_fitness": need_fit,
            "records": (mum, dad, mp, dp), "nodes": kids, "offsets": koffs,
            "fitness": ev["fitness"], "out": ev["out"], "hits": ev["hits"]}
