"""One GP population sharded over the processes of a torch.distributed group.

The paper's trees are independent (Sec. 2.3): evaluating or crossing one
tree never touches another, and only tournament selection (Table
gp.details) reads the whole population's fitness.  So every rank holds a
contiguous range of the population's trees, the ranges split by node count
so that every rank has about the same evaluation work, and one generation
is:

1. all ranks gather every tree's fitness and size (P floats and P sizes);
2. each rank draws the records of its own children (`gp_select`: the
   counter-based draws, so the records equal the ones a single process
   draws for the same seed and generation);
3. each rank fetches the parents its children need from the ranks that
   hold them: an all-to-all of tree indices, then of sizes and bytes;
4. each rank makes its children from those parents (`gp_crossover` on a
   population of them) and evaluates them (`gp_evaluate`).

Child c of a generation is made by the rank that holds index c, so the
index ranges stay fixed across generations and the node balance of later
generations follows the draws.  Steps 1 and 3 are the only collectives.

A `Backend` does the work of a rank (its trees, selection, reading trees,
making and evaluating children); `LibgpBackend` does it on the rank's GPU
through libgp.  The collectives run on the process group's device: CUDA
tensors for NCCL, CPU tensors for gloo.
"""
from __future__ import annotations

import numpy as np


def balanced_ranges(sizes, world: int) -> list[tuple[int, int]]:
    """Contiguous index ranges [lo, hi), one per rank, each starting at the
    tree boundary where the running node count comes closest to rank /
    world of the total (at least one tree per rank while trees last)."""
    sizes = np.asarray(sizes, dtype=np.int64)
    n = sizes.shape[0]
    cum = np.concatenate([[0], np.cumsum(sizes)])
    total = int(cum[-1])
    cuts = [0]
    for r in range(1, world):
        target = total * r / world
        c = int(np.searchsorted(cum, target, side="left"))
        if 0 < c <= n and target - cum[c - 1] < cum[c] - target:
            c -= 1
        c = max(c, cuts[-1] + 1 if cuts[-1] < n else n)
        cuts.append(min(c, n))
    cuts.append(n)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def owner_of(ranges, idx):
    """Rank holding each global tree index."""
    los = np.array([lo for lo, _ in ranges], dtype=np.int64)
    return np.searchsorted(los, np.asarray(idx, dtype=np.int64), side="right") - 1


class LibgpBackend:
    """A rank's trees as a libgp population on its GPU."""

    def __init__(self, gp, problem, nodes, offsets, chunk_nodes=0, stream=None):
        self.gp, self.problem, self.chunk, self.stream = gp, problem, chunk_nodes, stream
        self.pop = gp.gp_create_population(problem, nodes, offsets, stream)
        gp.gp_evaluate(self.pop, stream, chunk_nodes=chunk_nodes)
        self.sizes = np.diff(np.asarray(offsets, dtype=np.uint64).astype(np.int64)).astype(np.uint64)

    def fitness(self) -> np.ndarray:
        return self.gp.gp_fitness(self.pop)[0]

    def select(self, fit_all, size_all, seed, g, lo, n, tsize):
        import torch
        gp = self.gp
        d_fit = torch.from_numpy(np.ascontiguousarray(fit_all, np.float32)).cuda()
        d_sz = torch.from_numpy(np.ascontiguousarray(size_all, np.uint64).view(np.int64)).cuda()
        out = torch.zeros(max(n, 1) * gp.XO_RECORD_BYTES, dtype=torch.uint8, device="cuda")
        if n:
            gp.gp_select(d_fit.data_ptr(), d_sz.data_ptr(), fit_all.shape[0], seed, g, lo, n, out.data_ptr(),
                         tsize, self.stream)
        rec = np.frombuffer(out[:n * gp.XO_RECORD_BYTES].cpu().numpy().tobytes(), dtype=gp._XO_DTYPE)
        return tuple(rec[k].copy() for k in ("mum", "dad", "mum_point", "dad_point"))

    def read_trees(self, local_idx):
        parts = [self.gp.gp_tree_read(self.pop, int(t)) for t in local_idx]
        sizes = np.array([p.shape[0] for p in parts], dtype=np.uint64)
        return (np.concatenate(parts) if parts else np.zeros(0, np.uint8)), sizes

    def replace(self, pool_nodes, pool_offsets, mum, dad, mum_point, dad_point):
        gp = self.gp
        parents = gp.gp_create_population(self.problem, pool_nodes, pool_offsets, self.stream)
        kids = gp.gp_crossover(parents, (mum, dad, mum_point, dad_point), self.stream)
        gp.gp_evaluate(kids, self.stream, chunk_nodes=self.chunk)
        self.pop = kids
        self.sizes = np.array([gp.gp_tree_size(kids, t) for t in range(kids.n_trees)], dtype=np.uint64)


class ShardedPopulation:
    """This rank's part of a population of `n_total` trees; `backend` holds
    the trees of range `ranges[rank]` (already evaluated)."""

    def __init__(self, backend, ranges, rank: int, world: int, seed: int, tsize: int = 7, device="cpu",
                 group=None):
        self.b, self.ranges, self.rank, self.world = backend, ranges, rank, world
        self.lo, self.hi = ranges[rank]
        self.n_total = ranges[-1][1]
        self.seed, self.tsize, self.device, self.group = seed, tsize, device, group
        self.generation = 0

    # ---- collectives ------------------------------------------------------

    def _gather(self, local: np.ndarray, dtype) -> np.ndarray:
        """Every rank's local array (lengths from the ranges), concatenated."""
        import torch
        import torch.distributed as dist
        width = max(hi - lo for lo, hi in self.ranges)
        buf = np.zeros(width, dtype=dtype)
        buf[:local.shape[0]] = local
        t = torch.from_numpy(buf.view(np.int64) if dtype == np.uint64 else buf).to(self.device)
        outs = [torch.empty_like(t) for _ in range(self.world)]
        dist.all_gather(outs, t, group=self.group)
        parts = []
        for r, o in enumerate(outs):
            lo, hi = self.ranges[r]
            a = o.cpu().numpy()
            parts.append((a.view(np.uint64) if dtype == np.uint64 else a)[:hi - lo])
        return np.concatenate(parts)

    def _all_to_all(self, send: np.ndarray, send_counts) -> tuple[np.ndarray, list[int]]:
        """Variable all-to-all of a flat array: send_counts[r] elements go to
        rank r; returns what arrived (in rank order) and the counts."""
        import torch
        import torch.distributed as dist
        sc = torch.tensor(list(send_counts), dtype=torch.int64, device=self.device)
        rc = torch.empty_like(sc)
        dist.all_to_all_single(rc, sc, group=self.group)
        recv_counts = [int(v) for v in rc.cpu()]
        src = torch.from_numpy(np.ascontiguousarray(send)).to(self.device)
        dst = torch.empty(sum(recv_counts), dtype=src.dtype, device=self.device)
        dist.all_to_all_single(dst, src, output_split_sizes=recv_counts, input_split_sizes=list(send_counts),
                               group=self.group)
        return dst.cpu().numpy(), recv_counts

    # ---- one generation -----------------------------------------------------

    def step(self) -> None:
        g = self.generation
        fit_all = self._gather(np.asarray(self.b.fitness(), np.float32), np.float32)
        size_all = self._gather(np.asarray(self.b.sizes, np.uint64), np.uint64)
        n_kids = self.hi - self.lo
        mum, dad, mp, dp = self.b.select(fit_all, size_all, self.seed, g, self.lo, n_kids, self.tsize)
        need = np.unique(np.concatenate([mum, dad]).astype(np.int64))
        owners = owner_of(self.ranges, need)
        # requests: the global indices wanted from each rank, in rank order
        req_counts = [int(np.sum(owners == r)) for r in range(self.world)]
        wanted, got_counts = self._all_to_all(need, req_counts)
        # answer: the requested trees' sizes and bytes, per requester in rank order
        sizes_out, bytes_out, size_counts, byte_counts = [], [], [], []
        pos = 0
        for r in range(self.world):
            idx = wanted[pos:pos + got_counts[r]] - self.lo
            pos += got_counts[r]
            nb, sz = self.b.read_trees(idx)
            sizes_out.append(sz)
            bytes_out.append(nb)
            size_counts.append(sz.shape[0])
            byte_counts.append(nb.shape[0])
        pool_sizes, _ = self._all_to_all(np.concatenate(sizes_out).view(np.int64), size_counts)
        pool_bytes, _ = self._all_to_all(np.concatenate(bytes_out), byte_counts)
        pool_sizes = pool_sizes.view(np.uint64)
        pool_offs = np.zeros(pool_sizes.shape[0] + 1, dtype=np.uint64)
        np.cumsum(pool_sizes, out=pool_offs[1:])
        # `need` is sorted and owners hold increasing ranges, so the pool is in
        # `need` order: a parent's pool index is its rank in `need`
        pm = np.searchsorted(need, mum.astype(np.int64)).astype(np.uint32)
        pd = np.searchsorted(need, dad.astype(np.int64)).astype(np.uint32)
        self.b.replace(pool_bytes.astype(np.uint8), pool_offs, pm, pd, mp, dp)
        self.generation = g + 1
