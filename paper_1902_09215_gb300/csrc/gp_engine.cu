// The generation engine: tournament selection (Table gp.details: size 7,
// both parents), subtree crossover with uniform points (Sec. 3.1) and the
// evaluation of the children (Sec. 2.2), for a batch of independent runs
// whose populations live in one device heap.  Every count of a batch is in
// device memory, so a batch is a fixed launch sequence (captured once as a
// CUDA graph); a run's failure (node limit, its buffer too small) stops that
// run only, a workspace overflow fails the batch and no run advances.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "gp_engine.cuh"

using namespace gpk;

namespace gpe {
namespace {

constexpr uint32_t kScanT = 1024;        // threads of the single-CTA scan kernels
constexpr uint32_t kBuckets = 40;        // final items ordered by floor(log2(size)), largest first
constexpr uint64_t kHeapLead = 256;      // heap bytes [0, 256): code 4 ('x'), a one-node tree
                                         // that idle extent queries point at

__device__ __forceinline__ void run_err(RunDev *R, uint32_t bits)
{
    if (atomicOr(&R->err, bits) == 0) R->err_gen = R->gen;
}

// ---- counter-based draws --------------------------------------------------

// Output i of SplitMix64 seeded with `seed` (Steele, Lea & Flood 2014): the
// (i+1)-th state of its Weyl sequence through the generator's mixer.
__device__ __forceinline__ uint64_t sm64_at(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t draw_counter(uint32_t g, uint32_t c, uint32_t purpose, uint32_t k)
{
    return ((uint64_t)g << 40) | ((uint64_t)c << 12) | ((uint64_t)purpose << 9) | ((uint64_t)k << 4);
}

// Uniform in [0, n): Lemire's multiply-shift, rejecting low words below
// 2^64 mod n; attempts use counters base .. base+15, the last one is kept.
__device__ uint64_t bounded(uint64_t seed, uint64_t base, uint64_t n)
{
    const uint64_t t = (0ull - n) % n;
    uint64_t hi = 0;
    for (uint32_t a = 0; a < 16; ++a) {
        const uint64_t r = sm64_at(seed, base + a);
        hi = __umul64hi(r, n);
        if (r * n >= t) break;
    }
    return hi;
}

// Lowest fitness wins; NaN ranks worst; ties go to the entrant drawn first.
__device__ uint32_t tournament(const float *__restrict__ fit, uint32_t n_pop, uint64_t seed, uint32_t g,
                               uint32_t c, uint32_t purpose, uint32_t size)
{
    uint32_t best = 0;
    float best_f = 0.0f;
    for (uint32_t k = 0; k < size; ++k) {
        const uint32_t e = (uint32_t)bounded(seed, draw_counter(g, c, purpose, k), n_pop);
        float f = fit[e];
        if (isnan(f)) f = __int_as_float(0x7f800000);
        if (k == 0 || f < best_f) {
            best = e;
            best_f = f;
        }
    }
    return best;
}

// Batch slot of global tree g: the last slot whose first tree is <= g.
__device__ __forceinline__ uint32_t slot_of(const uint32_t *__restrict__ tree_base, uint32_t n_runs, uint32_t g)
{
    uint32_t lo = 0, hi = n_runs;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (tree_base[mid] <= g) lo = mid;
        else hi = mid;
    }
    return lo;
}

// ---- selection, child layout, copy bookkeeping ---------------------------

__global__ void select_kernel(BatchCtl *ctl, RunDev *runs, const uint32_t *__restrict__ slot_run,
                              const uint32_t *__restrict__ tree_base, gp_xo *__restrict__ recs,
                              ExtentQuery *__restrict__ q)
{
    const BatchHead h = ctl->head;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (h.mode != kModeGenerate) {
        if (tid == 0) ctl->n_queries = 0;
        return;
    }
    if (tid == 0) ctl->n_queries = 2 * h.n_trees;
    for (uint32_t g = tid; g < h.n_trees; g += gridDim.x * blockDim.x) {
        const uint32_t slot = slot_of(tree_base, h.n_runs, g);
        RunDev *R = runs + slot_run[slot];
        const uint32_t c = g - tree_base[slot];
        if (R->err == 0 && R->gen >= (1u << 24) && c == 0) run_err(R, kGErrGen);
        if (R->err != 0 || R->gen >= (1u << 24)) {
            recs[g] = gp_xo{0, 0, 0, 0};
            q[2 * g] = q[2 * g + 1] = ExtentQuery{0, 1, 0};     // the one-node tree at heap offset 0
            continue;
        }
        const RunBuf &P = R->buf[R->cur];
        gp_xo r;
        r.mum = tournament(P.fit, R->n, R->seed, R->gen, c, 0, R->tsize);
        r.dad = tournament(P.fit, R->n, R->seed, R->gen, c, 1, R->tsize);
        r.mum_point = bounded(R->seed, draw_counter(R->gen, c, 2, 0), P.size[r.mum]);
        r.dad_point = bounded(R->seed, draw_counter(R->gen, c, 3, 0), P.size[r.dad]);
        recs[g] = r;
        q[2 * g] = ExtentQuery{P.start[r.mum], P.size[r.mum], r.mum_point};
        q[2 * g + 1] = ExtentQuery{P.start[r.dad], P.size[r.dad], r.dad_point};
    }
}

// Records of children [lo, lo + n) of generation g, from the whole
// population's fitness and sizes (gp_select).
__global__ void select_range_kernel(const float *__restrict__ fit, const uint64_t *__restrict__ size,
                                    uint32_t n_pop, uint64_t seed, uint32_t g, uint32_t lo, uint32_t n,
                                    uint32_t tsize, gp_xo *__restrict__ out)
{
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const uint32_t c = lo + k;
        gp_xo r;
        r.mum = tournament(fit, n_pop, seed, g, c, 0, tsize);
        r.dad = tournament(fit, n_pop, seed, g, c, 1, tsize);
        r.mum_point = bounded(seed, draw_counter(g, c, 2, 0), size[r.mum]);
        r.dad_point = bounded(seed, draw_counter(g, c, 3, 0), size[r.dad]);
        out[k] = r;
    }
}

// Block-wide inclusive scan of two 64-bit values per thread (kScanT
// threads): warp scans by shuffles, a scan of the 32 warp totals by warp 0,
// then each thread's warp offset; the results land in sa[t], sb[t] (the
// block totals in sa[kScanT-1], sb[kScanT-1]) once it returns.
__device__ void block_scan2(uint64_t *sa, uint64_t *sb, uint64_t a, uint64_t b)
{
    __shared__ uint64_t wa[kScanT / 32], wb[kScanT / 32];
    const uint32_t t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (uint32_t off = 1; off < 32; off <<= 1) {
        const uint64_t oa = __shfl_up_sync(0xffffffffu, a, off);
        const uint64_t ob = __shfl_up_sync(0xffffffffu, b, off);
        if (lane >= off) {
            a += oa;
            b += ob;
        }
    }
    if (lane == 31) {
        wa[warp] = a;
        wb[warp] = b;
    }
    __syncthreads();
    if (warp == 0) {
        uint64_t xa = wa[lane], xb = wb[lane];
        for (uint32_t off = 1; off < 32; off <<= 1) {
            const uint64_t oa = __shfl_up_sync(0xffffffffu, xa, off);
            const uint64_t ob = __shfl_up_sync(0xffffffffu, xb, off);
            if (lane >= off) {
                xa += oa;
                xb += ob;
            }
        }
        wa[lane] = xa;                       // inclusive warp totals
        wb[lane] = xb;
    }
    __syncthreads();
    if (warp > 0) {
        a += wa[warp - 1];
        b += wb[warp - 1];
    }
    sa[t] = a;
    sb[t] = b;
    __syncthreads();
}

// Children of a batch in three steps.  children_size_kernel (a thread per
// child): the child's size i + (e_d - j) + (n_m - e_m) from the extent
// queries and ends, into bsize; runs stopped by an error and evaluate-mode
// batches take their current trees instead.  children_scan_kernel (one CTA
// per run): 16-byte aligned offsets and copy tiles by a block scan over the
// run's children (coalesced, no gathers), node limit and buffer capacity;
// a run that does not fit gets its error and no children.  children_place_
// kernel (a thread per child): copy records and the new buffer's starts and
// sizes.
__global__ void children_size_kernel(const BatchCtl *ctl, RunDev *runs, const uint32_t *__restrict__ slot_run,
                                     const uint32_t *__restrict__ tree_base, const ExtentQuery *__restrict__ q,
                                     const uint64_t *__restrict__ ends, uint64_t *__restrict__ bstart,
                                     uint64_t *__restrict__ bsize)
{
    pdl_wait();
    const BatchHead h = ctl->head;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < h.n_trees; g += gridDim.x * blockDim.x) {
        const uint32_t slot = slot_of(tree_base, h.n_runs, g);
        const RunDev *R = runs + slot_run[slot];
        const uint32_t c = g - tree_base[slot];
        const bool stopped = R->err != 0 || (h.mode == kModeGenerate && ctl->eval_err[1] != 0);
        if (stopped || h.mode == kModeEvaluate) {
            const RunBuf &B = R->buf[R->cur];
            bstart[g] = stopped ? 0 : B.start[c];
            bsize[g] = stopped ? 0 : B.size[c];
            continue;
        }
        const ExtentQuery qm = q[2 * g], qd = q[2 * g + 1];
        bsize[g] = qm.point + (ends[2 * g + 1] - qd.point) + (qm.tree_size - ends[2 * g]);
    }
}

__global__ void __launch_bounds__(kScanT) children_scan_kernel(
    BatchCtl *ctl, RunDev *runs, const uint32_t *__restrict__ slot_run, const uint32_t *__restrict__ tree_base,
    uint32_t *__restrict__ tile_local, uint32_t *__restrict__ run_tiles, uint64_t *__restrict__ bstart,
    uint64_t *__restrict__ bsize, uint32_t tile)
{
    pdl_wait();
    __shared__ uint64_t sa[kScanT], sb[kScanT];
    __shared__ uint32_t s_bad;
    __shared__ unsigned long long s_nodes;
    const BatchHead h = ctl->head;
    const uint32_t slot = blockIdx.x, t = threadIdx.x;
    if (slot >= h.n_runs) return;
    RunDev *R = runs + slot_run[slot];
    const uint32_t base = tree_base[slot], n = R->n;
    const bool stopped = R->err != 0 || (h.mode == kModeGenerate && ctl->eval_err[1] != 0);
    if (stopped || h.mode == kModeEvaluate) {
        if (t == 0) run_tiles[slot] = 0;
        return;
    }
    if (t == 0) {
        s_bad = 0;
        s_nodes = 0;
    }
    __syncthreads();
    const RunBuf Cb = R->buf[R->cur ^ 1];
    const uint64_t max_nodes = R->max_nodes;
    // rounds of kScanT children (coalesced), a block scan per round and a
    // running carry; this run's children offsets go to bstart for now
    uint64_t carry_a = 0, carry_b = 0, nodes = 0;
    uint32_t bad = 0;
    for (uint32_t r0 = 0; r0 < n; r0 += kScanT) {
        const uint32_t c = r0 + t;
        uint64_t m = 0;
        if (c < n) {
            m = bsize[base + c];
            if (max_nodes && m > max_nodes) bad |= kGErrLimit;
            nodes += m;
        }
        const uint64_t a = (m + 15) & ~15ull, b = (m + tile - 1) / tile;
        block_scan2(sa, sb, a, b);
        if (c < n) {
            bstart[base + c] = carry_a + sa[t] - a;
            tile_local[base + c] = (uint32_t)(carry_b + sb[t] - b);
        }
        carry_a += sa[kScanT - 1];
        carry_b += sb[kScanT - 1];
        __syncthreads();                      // sa / sb are rewritten by the next round
    }
    if (bad) atomicOr(&s_bad, bad);
    // the run's node total: a warp sum, then one shared atomic per warp (a
    // 64-bit shared atomic from every thread of the CTA serialises)
    unsigned long long wsum = nodes;
    for (int o = 16; o > 0; o >>= 1) wsum += __shfl_down_sync(0xffffffffu, wsum, o);
    if ((t & 31) == 0) atomicAdd(&s_nodes, wsum);
    __syncthreads();
    uint32_t err = s_bad;
    if (carry_a + 64 > Cb.cap || carry_b >= 0x7fffffffull) err |= kGErrArena;
    if (err) {
        for (uint32_t c = t; c < n; c += kScanT) bsize[base + c] = 0;
        if (t == 0) {
            run_tiles[slot] = 0;
            run_err(R, err);
        }
        return;
    }
    if (t == 0) {
        run_tiles[slot] = (uint32_t)carry_b;
        R->next_nodes = s_nodes;
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->child_nodes), s_nodes);
    }
}

__global__ void children_place_kernel(const BatchCtl *ctl, RunDev *runs, const uint32_t *__restrict__ slot_run,
                                      const uint32_t *__restrict__ tree_base, const ExtentQuery *__restrict__ q,
                                      const uint64_t *__restrict__ ends, XoChild *__restrict__ kids,
                                      uint64_t *__restrict__ bstart, const uint64_t *__restrict__ bsize)
{
    pdl_wait();
    const BatchHead h = ctl->head;
    if (h.mode != kModeGenerate || ctl->eval_err[1] != 0) return;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < h.n_trees; g += gridDim.x * blockDim.x) {
        const uint32_t slot = slot_of(tree_base, h.n_runs, g);
        RunDev *R = runs + slot_run[slot];
        if (R->err != 0) continue;           // stopped before, or its children did not fit
        const uint32_t c = g - tree_base[slot];
        const RunBuf &Cb = R->buf[R->cur ^ 1];
        const ExtentQuery qm = q[2 * g], qd = q[2 * g + 1];
        const uint64_t em = ends[2 * g], ed = ends[2 * g + 1];
        const uint64_t dst = Cb.lo + bstart[g], m = bsize[g];
        XoChild k;
        k.dst = dst;
        k.n = m;
        k.head_src = qm.tree_start;
        k.i = qm.point;
        k.mid_src = qd.tree_start + qd.point;
        k.ld = ed - qd.point;
        k.tail_src = qm.tree_start + em;         // tail byte p comes from mum[em + p - i - ld]
        k.pad = 0;
        kids[g] = k;
        Cb.start[c] = dst;
        Cb.size[c] = m;
        bstart[g] = dst;
    }
}

// Run tile counts -> exclusive offsets (entry n_runs = all tiles).
__global__ void run_tiles_scan_kernel(BatchCtl *ctl, uint32_t *run_tiles)
{
    pdl_wait();
    if (threadIdx.x != 0) return;
    const uint32_t n = ctl->head.n_runs;
    uint64_t s = 0;
    for (uint32_t i = 0; i < n; ++i) {
        const uint32_t v = run_tiles[i];
        run_tiles[i] = (uint32_t)s;
        s += v;
    }
    run_tiles[n] = (uint32_t)umin64(s, 0x7fffffffull);
    ctl->n_tiles = ctl->head.mode == kModeGenerate ? run_tiles[n] : 0;
}

// ---- evaluation levels ----------------------------------------------------

// A level launched inside the captured level loop: its number is the
// control block's count of loop levels started, plus one.
constexpr uint32_t kDynLevel = 0xffffffffu;

struct LevelArgs {
    uint32_t level;               // or kDynLevel
    uint32_t C;                   // chunk (codes)
    uint32_t cap_items;
    uint32_t last;                // the last level: every open tree becomes a final item
                                  // (kDynLevel: the number of levels the loop may run)
    uint64_t spill_base;          // first dedicated spill entry (after the per-warp areas)
    uint64_t cap_dedicated;       // dedicated spill entries available
    uint64_t cap_slots;           // fused chunk slots (0: no fused chunks)
};

__device__ __forceinline__ uint32_t size_bucket(uint64_t len)
{
    const uint32_t b = 63u - (uint32_t)__clzll(len | 1ull);
    return min(b, kBuckets - 1);
}

// Level 0, before its items, a warp per tree: the tree's level-0 range and
// state (t_lo, t_hi, t_prev, t_state), and every tree of 2..kFuseMaxChunks
// chunks is cut where its arity walk is low (cut_low; one chunk more than
// ceil(size / C) at most, never more than kFuseMaxChunks).  t_nch[i]: the
// tree's chunk count (0 for the other trees); t_cut[i * (kFuseMaxChunks - 1)
// + j]: the end of its chunk j, relative to the tree's start.
__global__ void cut_fused_kernel(const BatchCtl *ctl, uint32_t C, const uint8_t *__restrict__ heap,
                                 const uint64_t *__restrict__ bstart, const uint64_t *__restrict__ bsize,
                                 uint32_t *__restrict__ t_nch, uint32_t *__restrict__ t_cut,
                                 uint64_t *__restrict__ t_lo, uint64_t *__restrict__ t_hi,
                                 uint64_t *__restrict__ t_prev, uint32_t *__restrict__ t_state)
{
    pdl_wait();
    if (ctl->err != 0) return;
    const uint32_t n = ctl->head.n_trees;
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = warp; i < n; i += warps) {
        const uint64_t z = bsize[i];
        uint32_t k = 0;
        if (z > C && z <= (uint64_t)kFuseMaxChunks * C) {
            const uint64_t b = bstart[i];
            const uint32_t m = (uint32_t)((z + C - 1) / C);
            uint32_t *cut = t_cut + (uint64_t)i * (kFuseMaxChunks - 1);
            k = cut_low(heap, b, z, C, min(m + 1, kFuseMaxChunks), lane, [&](uint32_t j, uint64_t e) {
                if (lane == 0) cut[j - 1] = (uint32_t)(e - b);
            });
        }
        if (lane == 0) {
            t_nch[i] = k;
            const uint64_t b = bstart[i];
            t_lo[i] = b;
            t_hi[i] = b + z;
            t_prev[i] = ~0ull;
            t_state[i] = z != 0;
        }
    }
}

// One CTA.  Level 0: every tree of the batch (size 0: none); a tree of at
// most C nodes is one final item; a tree of 2..kFuseMaxChunks chunks (when
// the workspace has fused slots) becomes fused chunks, each writing its
// fragment into its own slot (the tree's slots consecutive), and its rope
// (a final item over those slots) goes to level 1; a larger tree is cut into
// planned chunks of C.  Level k > 0: every tree that had planned chunks at
// level k-1 now has an upper tree of codes [frag_off[first chunk],
// frag_off[one past its last chunk]); it becomes a final item when it fits
// one chunk, did not at least halve, or this is the last level (a final
// above C gets a dedicated spill area); otherwise it is cut again.  A fused
// tree's chunks are the ones cut_fused_kernel chose (t_nch, t_cut).
// Items: planned chunks first in tree order (their fragments must be
// contiguous per tree), then fused chunks, then finals (ropes included)
// from the largest size bucket down.  This CTA only takes the decisions and
// the offsets (tree-order scans); the items themselves are written by
// fill_items_kernel from three compact lists: fz_tree (the tree of every
// fused chunk), fin_tree (the tree of every final item, bit 31 for a rope)
// and rope_tree (level 0's ropes, largest first), so that one SM does not
// carry every item's bytes.
// Tree states: 0 done or empty, 1 open (planned), 2 rope pending (t_lo: its
// first slot, t_hi: its chunk count).  At level 0, cut_fused_kernel has set
// every tree's range and state; a final with a dedicated spill area keeps
// its spill offset in t_prev.
__global__ void __launch_bounds__(kScanT) items_kernel(
    BatchCtl *ctl, LevelArgs A, const uint64_t *__restrict__ bstart, const uint64_t *__restrict__ bsize,
    const uint64_t *__restrict__ frag_off, uint64_t *__restrict__ t_lo, uint64_t *__restrict__ t_hi,
    uint64_t *__restrict__ t_prev, uint32_t *__restrict__ t_first, uint32_t *__restrict__ t_state,
    const uint32_t *__restrict__ t_nch, uint32_t *__restrict__ fz_tree, uint32_t *__restrict__ fin_tree,
    uint32_t *__restrict__ rope_tree, bool list_ropes)
{
    pdl_wait();
    __shared__ uint64_t sa[kScanT], sb[kScanT];
    __shared__ uint32_t s_cnt[kBuckets], s_fill[kBuckets];
    __shared__ uint32_t s_rcnt[kBuckets], s_rfill[kBuckets], s_rbase[kBuckets];
    __shared__ uint64_t s_base[kBuckets];
    __shared__ uint32_t s_err;
    const uint32_t t = threadIdx.x;
    const uint32_t n = ctl->head.n_trees, C = A.C;
    const bool dyn = A.level == kDynLevel;
    const uint32_t level = dyn ? 1u + ctl->loop_level : A.level;
    const bool last = dyn ? level + 1 >= A.last : A.last != 0;
    __syncthreads();                          // every thread has read the loop count
    if (dyn && t == 0) ctl->loop_level = level;
    // nothing to do: an earlier error, or no tree was cut at the level before
    if (ctl->err != 0 || (level > 0 && ctl->n_chunks == 0 && ctl->n_ropes == 0)) {
        __syncthreads();                      // every thread has read n_chunks / n_ropes
        if (t == 0) ctl->n_items = ctl->n_chunks = ctl->n_ropes = 0;
        return;
    }
    if (t < kBuckets) {
        s_cnt[t] = 0;
        s_fill[t] = 0;
        s_rcnt[t] = 0;
        s_rfill[t] = 0;
    }
    const uint64_t fuse_hi = (level == 0 && A.cap_slots) ? (uint64_t)kFuseMaxChunks * C : 0;
    // Trees go through in rounds of kScanT, one tree per thread (coalesced
    // loads and stores); every prefix over trees is a block scan per round
    // plus a running carry, so all offsets stay in tree order.
    const uint32_t rounds = (n + kScanT - 1) / kScanT;

    // phase 1: this level's range of every open tree (all reads of the old
    // t_first happen before the barrier; phase 3 rewrites it)
    if (level > 0) {
        for (uint32_t i = t; i < n; i += kScanT) {
            if (t_state[i] == 1) {
                t_lo[i] = frag_off[t_first[i]];
                t_hi[i] = frag_off[t_first[i + 1]];
            }
        }
    }
    __syncthreads();
    // level 0: trees of 2..kFuseMaxChunks chunks take fused slots in tree
    // order while slots remain (the ones after are planned: a batch that
    // outgrew the slots still runs); state 3 marks them until phase 3
    if (fuse_hi) {
        uint64_t run_c = 0;                   // slots asked for by the trees of earlier rounds
        for (uint32_t r = 0; r < rounds; ++r) {
            const uint32_t i = r * kScanT + t;
            uint64_t m = 0;
            if (i < n && t_state[i] == 1) {
                const uint64_t len = t_hi[i] - t_lo[i];
                if (len > C && len <= fuse_hi) m = t_nch[i];
            }
            block_scan2(sa, sb, m, 0);
            if (m && run_c + sa[t] <= A.cap_slots) t_state[i] = 3;   // sa[t]: up to and including tree i
            run_c += sa[kScanT - 1];
            __syncthreads();                  // the arrays are scanned again
        }
        if (t == 0) ctl->need_slots = max(ctl->need_slots, run_c);
    }
    // phase 2 (counts) and phase 3 (items) see each tree the same way: its
    // planned chunks, dedicated spill entries and fused chunks, with the
    // finals and ropes counted per size bucket in phase 2
    auto shares = [&](uint32_t i, uint64_t &nch, uint64_t &ded, uint64_t &nfz) {
        nch = ded = nfz = 0;
        if (i >= n) return;
        const uint32_t st = t_state[i];
        if (st == 0 || st == 2) return;
        const uint64_t len = t_hi[i] - t_lo[i];
        if (st == 3) nfz = t_nch[i];
        else if (last || len <= C || 2 * len > t_prev[i]) ded = len > C ? len : 0;
        else nch = (len + C - 1) / C;
    };
    uint64_t tot_ch = 0, tot_ded = 0, tot_fz = 0;
    for (uint32_t r = 0; r < rounds; ++r) {
        const uint32_t i = r * kScanT + t;
        uint64_t nch, ded, nfz;
        shares(i, nch, ded, nfz);
        if (i < n && t_state[i] != 0) {
            const uint32_t st = t_state[i];
            if (st == 2) atomicAdd(&s_cnt[size_bucket(t_hi[i] * C)], 1u);      // a rope: final
            else if (st == 3) atomicAdd(&s_rcnt[size_bucket(t_hi[i] - t_lo[i])], 1u);
            else if (nch == 0) atomicAdd(&s_cnt[size_bucket(t_hi[i] - t_lo[i])], 1u);
        }
        // chunk and fused counts are below 2^32 in all (item counts), so one
        // 64-bit word carries both
        block_scan2(sa, sb, (nch << 32) | nfz, ded);
        tot_ch += sa[kScanT - 1] >> 32;
        tot_fz += sa[kScanT - 1] & 0xffffffffull;
        tot_ded += sb[kScanT - 1];
        __syncthreads();                      // the arrays are scanned again
    }
    if (t == 0) {
        uint64_t pos = tot_ch + tot_fz;       // finals after the chunks, largest bucket first
        for (int b = (int)kBuckets - 1; b >= 0; --b) {
            s_base[b] = pos;
            pos += s_cnt[b];
        }
        uint32_t rpos = 0;                    // level 0's ropes, largest trees first
        for (int b = (int)kBuckets - 1; b >= 0; --b) {
            s_rbase[b] = rpos;
            rpos += s_rcnt[b];
        }
        uint32_t err = 0;
        ctl->need_dedicated = max(ctl->need_dedicated, tot_ded);
        ctl->need_items = max(ctl->need_items, pos);
        if (pos > A.cap_items) err |= kGErrItems;
        if (tot_ded > A.cap_dedicated) err |= kGErrSpill;
        if (err) {
            atomicOr(&ctl->err, err);
            ctl->n_items = ctl->n_chunks = ctl->n_ropes = 0;
        } else {
            ctl->n_items = (uint32_t)pos;
            ctl->n_chunks = (uint32_t)tot_ch;
            ctl->n_ropes = (uint32_t)tot_fz;
            if (pos) ctl->levels = level + 1;
            if (level == 0 && list_ropes) {
                ctl->n_rope_items = rpos;
                if (rpos) ctl->levels = 2;    // the ropes are level 1
            }
        }
        s_err = err;
    }
    __syncthreads();
    if (s_err) return;
    // phase 3: chunk offsets per tree, fused chunks, final items (any order
    // within a bucket), states
    uint64_t c_ch = 0, c_ded = 0, c_fz = 0;   // carries from earlier rounds
    for (uint32_t r = 0; r < rounds; ++r) {
        const uint32_t i = r * kScanT + t;
        uint64_t nch, ded, nfz;
        shares(i, nch, ded, nfz);
        block_scan2(sa, sb, (nch << 32) | nfz, ded);
        const uint64_t ex = sa[t] - ((nch << 32) | nfz);
        const uint64_t ex_ch = c_ch + (ex >> 32), ex_fz = c_fz + (ex & 0xffffffffull);
        const uint64_t ex_ded = c_ded + sb[t] - ded;
        c_ch += sa[kScanT - 1] >> 32;
        c_fz += sa[kScanT - 1] & 0xffffffffull;
        c_ded += sb[kScanT - 1];
        if (i < n) {
            t_first[i] = (uint32_t)ex_ch;
            const uint32_t st = t_state[i];
            const uint64_t fin0 = tot_ch + tot_fz;      // first final item
            if (st == 2) {
                const uint32_t b = size_bucket(t_hi[i] * C);
                fin_tree[s_base[b] - fin0 + atomicAdd(&s_fill[b], 1u)] = i | 0x80000000u;
                t_state[i] = 0;
            } else if (st == 3) {
                const uint64_t len = t_hi[i] - t_lo[i];
                const uint32_t m = t_nch[i];
                for (uint32_t j = 0; j < m; ++j) fz_tree[ex_fz + j] = i;
                if (list_ropes) {
                    const uint32_t b = size_bucket(len);
                    rope_tree[s_rbase[b] + atomicAdd(&s_rfill[b], 1u)] = i;
                }
                t_state[i] = 2;
                t_lo[i] = ex_fz;
                t_hi[i] = m;
            } else if (st != 0 && nch == 0) {
                const uint64_t len = t_hi[i] - t_lo[i];
                const uint32_t b = size_bucket(len);
                if (len > C) t_prev[i] = ex_ded;
                fin_tree[s_base[b] - fin0 + atomicAdd(&s_fill[b], 1u)] = i;
                t_state[i] = 0;
            } else if (st != 0) {
                t_prev[i] = t_hi[i] - t_lo[i];
            }
        }
        __syncthreads();                      // the arrays are scanned again
    }
    if (t == 0) t_first[n] = (uint32_t)tot_ch;
}

// A level's items: [0, n_chunks) planned chunks (item i belongs to the last
// tree whose first chunk is <= i), then the fused chunks of fz_tree (level
// 0), then the finals of fin_tree; and level 0's ropes for a rope-only
// level from rope_tree.  A grid-stride thread per item.
__global__ void fill_items_kernel(const BatchCtl *ctl, LevelArgs A, const uint32_t *__restrict__ t_first,
                                  const uint64_t *__restrict__ t_lo, const uint64_t *__restrict__ t_hi,
                                  const uint64_t *__restrict__ t_prev, const uint64_t *__restrict__ bstart,
                                  const uint64_t *__restrict__ bsize, const uint32_t *__restrict__ t_cut,
                                  const uint32_t *__restrict__ fz_tree, const uint32_t *__restrict__ fin_tree,
                                  const uint32_t *__restrict__ rope_tree, EvalItem *__restrict__ items,
                                  EvalItem *__restrict__ rope_items)
{
    pdl_wait();
    if (ctl->err != 0) return;
    const uint32_t C = A.C;
    const uint32_t n_ch = ctl->n_chunks, n_fz = ctl->n_ropes, n_items = ctl->n_items, n_trees = ctl->head.n_trees;
    const uint32_t n_rope = rope_items ? ctl->n_rope_items : 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n_items; k += stride) {
        EvalItem it{};
        it.spill_off = kNoSpill;
        if (k < n_ch) {
            uint32_t lo = 0, hi = n_trees;
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (t_first[mid] <= k) lo = mid;
                else hi = mid;
            }
            it.begin = t_lo[lo] + (uint64_t)(k - t_first[lo]) * C;
            it.end = umin64(t_hi[lo], it.begin + C);
            it.tree = lo;
        } else if (k < n_ch + n_fz) {
            const uint32_t f = k - n_ch, i = fz_tree[f];
            const uint32_t first = (uint32_t)t_lo[i], m = (uint32_t)t_hi[i], j = f - first;
            const uint32_t *cut = t_cut + (uint64_t)i * (kFuseMaxChunks - 1);
            const uint64_t b = bstart[i];
            it.begin = b + (j ? cut[j - 1] : 0u);
            it.end = j + 1 < m ? b + cut[j] : b + bsize[i];
            it.tree = i;
            it.flags = gpk::kItemFused;
            it.frag_off = f;
            it.pt_base = first;
            it.frag_len = m;
        } else {
            const uint32_t e = fin_tree[k - n_ch - n_fz], i = e & 0x7fffffffu;
            it.tree = i;
            if (e >> 31) {                          // a rope: its slots
                it.flags = kItemFinal | gpk::kItemRope;
                it.pt_base = t_lo[i];
                it.frag_len = (uint32_t)t_hi[i];
            } else {
                it.flags = kItemFinal;
                it.begin = t_lo[i];
                it.end = t_hi[i];
                const uint64_t len = it.end - it.begin;
                if (len > C) {
                    it.spill_off = A.spill_base + t_prev[i];
                    it.spill_cap = len;
                }
            }
        }
        items[k] = it;
    }
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n_rope; k += stride) {
        const uint32_t i = rope_tree[k];
        EvalItem r{};
        r.tree = i;
        r.flags = kItemFinal | gpk::kItemRope;
        r.pt_base = t_lo[i];
        r.frag_len = (uint32_t)t_hi[i];
        r.spill_off = kNoSpill;
        rope_items[k] = r;
    }
}

// After a level's plan scan: the level's upper-tree codes and value entries
// must fit the workspace; the code array is zero-padded past its end (the
// evaluator reads whole 16-code groups).
// In a captured batch it also zeroes the level's work counter (a loop level
// reuses one per parity) and sets the level loop's conditions: `more` (bit
// 0 of cond) to whether the next level has trees, `zero` to 0 (bit 1) or
// to whether this level cut planned chunks (bit 2).
__global__ void check_kernel(BatchCtl *ctl, uint64_t cap_codes, uint64_t cap_values, uint32_t *__restrict__ u_out,
                             uint32_t idx, uint32_t *counter, uint32_t cond, cudaGraphConditionalHandle more,
                             cudaGraphConditionalHandle zero)
{
    pdl_wait();
    __shared__ uint32_t s_ok;
    const uint64_t codes = ctl->totals[0], vals = ctl->totals[1];
    if (threadIdx.x == 0) {
        s_ok = 0;
        if (counter) *counter = 0;
        if (ctl->err == 0) {
            // recorded whether or not they fit: a recovery sizes from them
            ctl->need_codes[idx] = max(ctl->need_codes[idx], codes);
            ctl->need_values[idx] = max(ctl->need_values[idx], vals);
            if (codes + 48 > cap_codes || vals > cap_values || vals + kPtCode0 >= 0xffffffffull) {
                atomicOr(&ctl->err, kGErrWork);
                ctl->n_items = 0;
            } else {
                s_ok = 1;
            }
        } else {
            ctl->n_items = 0;
        }
        // the next level has work when this one cut trees (or left ropes)
        const uint32_t next = ctl->err == 0 && (ctl->n_chunks != 0 || ctl->n_ropes != 0);
        if (cond & 1u) cudaGraphSetConditional(more, next);
        if (cond & 2u) cudaGraphSetConditional(zero, 0u);
        if (cond & 4u) cudaGraphSetConditional(zero, ctl->n_chunks != 0);
    }
    __syncthreads();
    if (!s_ok) return;
    const uint64_t end = ((codes + 15) & ~15ull) + 32;
    for (uint64_t i = codes + threadIdx.x; i < end; i += blockDim.x) u_out[i] = 0;
}

// Batch errors so far, as one word.
__device__ __forceinline__ uint32_t batch_errors(const BatchCtl *ctl)
{
    return ctl->err | (ctl->eval_err[0] ? kGErrEval : 0u) | (ctl->eval_err[1] ? kGErrExtent : 0u) |
           (ctl->n_chunks ? kGErrLevels : 0u);
}

// Evaluation results from the batch's tables into each run's buffer (the
// children's in Generate mode, the current one in Evaluate mode).
__global__ void scatter_kernel(const BatchCtl *ctl, RunDev *runs, const uint32_t *__restrict__ slot_run,
                               const uint32_t *__restrict__ tree_base, const float *__restrict__ bfit,
                               const float *__restrict__ bvals, const uint32_t *__restrict__ bhits,
                               uint32_t n_cases)
{
    const BatchHead h = ctl->head;
    if (batch_errors(ctl)) return;
    const uint64_t n_el = (uint64_t)h.n_trees * n_cases;    // one per-case value per thread
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < n_el;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t g = (uint32_t)(e / n_cases), k = (uint32_t)(e - (uint64_t)g * n_cases);
        const uint32_t slot = slot_of(tree_base, h.n_runs, g);
        const RunDev *R = runs + slot_run[slot];
        if (R->err) continue;
        const RunBuf &B = R->buf[h.mode == kModeGenerate ? (R->cur ^ 1) : R->cur];
        const uint32_t c = g - tree_base[slot];
        B.vals[(uint64_t)c * n_cases + k] = bvals[e];
        if (k == 0) {
            B.fit[c] = bfit[g];
            B.hits[c] = bhits[g];
        }
    }
}

// End of a batch: a batch error stops every run in it (no run advances);
// otherwise each run still going advances one generation (Generate mode).
__global__ void finish_kernel(const BatchCtl *ctl, RunDev *runs, const uint32_t *__restrict__ slot_run,
                              const uint32_t *__restrict__ fz_redo)
{
    const BatchHead h = ctl->head;
    // a rope that found one of its slots overflowed left its tree without
    // results: the batch made nothing (the caller enlarges the slots)
    const uint32_t berr = batch_errors(ctl) | ((fz_redo && fz_redo[0]) ? kGErrSlots : 0u);
    for (uint32_t s = threadIdx.x; s < h.n_runs; s += blockDim.x) {
        RunDev *R = runs + slot_run[s];
        if (R->err) continue;
        if (berr) {
            run_err(R, berr);
            continue;
        }
        R->levels = ctl->levels;
        if (h.mode == kModeGenerate) {
            R->gen += 1;
            R->cur ^= 1u;
            const uint64_t parents = R->nodes;     // kept for a rewind
            R->nodes = R->next_nodes;
            R->next_nodes = parents;
        }
    }
}

__global__ void rebase_kernel(uint64_t *__restrict__ start, uint32_t n, uint64_t delta)
{
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
        start[t] += delta;                                  // modulo 2^64: moves down as well
}

__global__ void rewind_kernel(RunDev *R)
{
    if (R->err == 0 && R->gen > 0) {
        R->gen -= 1;
        R->cur ^= 1u;
        const uint64_t children = R->nodes;
        R->nodes = R->next_nodes;
        R->next_nodes = children;
    }
}

#define GK(call)                                  \
    do {                                          \
        cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess) return gfail(e_);  \
    } while (0)

gp_status gfail(cudaError_t e)
{
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? GP_ENOMEM : GP_ECUDA;
}

gp_status galloc(std::vector<void *> &v, void **p, size_t bytes)
{
    *p = nullptr;
    GK(cudaMalloc(p, bytes ? bytes : 16));
    v.push_back(*p);
    return GP_OK;
}

void gfree(std::vector<void *> &v)
{
    for (void *p : v) cudaFree(p);
    v.clear();
}

int lanes_of(uint32_t n_cases)
{
    return n_cases <= 16 ? 8 : n_cases <= 32 ? 16 : n_cases <= 48 ? 24 : 32;
}

}  // namespace

cudaError_t launch_select_range(const float *fit, const uint64_t *size, uint32_t n_pop, uint64_t seed, uint32_t g,
                                uint32_t lo, uint32_t n, uint32_t tsize, gp_xo *out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const uint32_t blocks = std::min<uint32_t>((n + 127) / 128, 4096);
    select_range_kernel<<<blocks, 128, 0, s>>>(fit, size, n_pop, seed, g, lo, n, tsize, out);
    return cudaGetLastError();
}


// ---- Engine -----------------------------------------------------------------

Engine::~Engine()
{
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(device);
    cudaDeviceSynchronize();
    for (auto &e : exec)
        if (e) cudaGraphExecDestroy(e);
    for (auto &r : runs_host) gfree(r.allocs);
    gfree(work_allocs_);
    gfree(allocs_);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (cudaStream_t b : cap_body)
        if (b) cudaStreamDestroy(b);
    cudaSetDevice(cur);
}

gp_status Engine::init(const gp_problem *problem, uint64_t heap_bytes_, uint32_t max_runs_, uint32_t max_trees_,
                       uint32_t levels_max_)
{
    cudaGetDevice(&device);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    n_cases = problem->n_cases;
    n_consts = problem->n_consts;
    lanes = lanes_of(n_cases);
    div0 = problem->protected_div_value;
    max_runs = max_runs_;
    max_trees = max_trees_;
    levels_max = levels_max_;
    heap_bytes = heap_bytes_;
    GK(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
    for (cudaStream_t &b : cap_body) GK(cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking));
    // The engine's buffers come from cudaMalloc: memory that the stream-ordered
    // pool kept after earlier populations were freed is handed back first.
    {
        cudaMemPool_t pool;
        if (cudaDeviceSynchronize() == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess)
            cudaMemPoolTrimTo(pool, 0);
        const char *vb = std::getenv("GP_VERBOSE");
        size_t fr = 0, tot = 0;
        if (vb && vb[0] == '1' && cudaMemGetInfo(&fr, &tot) == cudaSuccess)
            std::fprintf(stderr, "engine init: %.1f of %.1f GB free; heap %.1f GB\n", fr / 1e9, tot / 1e9,
                         heap_bytes / 1e9);
    }
    // launch shape as in gp_evaluate
    int maxsm = 0;
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    rows = (int)std::max<uint32_t>(1 + n_consts, 1);
    while (W > 1 && eval_smem_bytes(lanes, (int)W, (int)K, false, rows) > (size_t)maxsm) --W;
    Wu = std::min<uint32_t>(W, 16);
    while (Wu > 1 && eval_smem_bytes(lanes, (int)Wu, (int)Ku, true, rows) > (size_t)maxsm) --Wu;
    smem = eval_smem_bytes(lanes, (int)W, (int)K, false, rows);
    smem_u = eval_smem_bytes(lanes, (int)Wu, (int)Ku, true, rows);
    if (smem > (size_t)maxsm || smem_u > (size_t)maxsm) return GP_EINVAL;
    Kr = std::max<uint32_t>(K, 192);
    Wr = std::min<uint32_t>(W, 16);
    while (Wr > 1 && eval_smem_bytes(lanes, (int)Wr, (int)Kr, true, rows) > (size_t)maxsm) --Wr;
    smem_r = eval_smem_bytes(lanes, (int)Wr, (int)Kr, true, rows);
    if (smem_r > (size_t)maxsm) {
        Kr = Ku;
        Wr = Wu;
        smem_r = smem_u;
    }
    GK(eval_prepare_at_least(lanes, false, smem));
    GK(eval_prepare_at_least(lanes, true, std::max(smem_u, smem_r)));

    auto &v = allocs_;
    gp_status st;
    if ((st = galloc(v, (void **)&heap, kHeapLead + heap_bytes + 64))) return st;
    GK(cudaMemset(heap, 4, kHeapLead));                     // the idle queries' one-node tree
    free_.assign(1, {kHeapLead, heap_bytes});
    if ((st = galloc(v, (void **)&runs_dev, sizeof(RunDev) * max_runs))) return st;
    GK(cudaMemset(runs_dev, 0, sizeof(RunDev) * max_runs));
    runs_host.assign(max_runs, RunHost{});
    if ((st = galloc(v, (void **)&ctl, sizeof(BatchCtl)))) return st;
    GK(cudaMemset(ctl, 0, sizeof(BatchCtl)));
    const uint64_t T = max_trees;
    if ((st = galloc(v, (void **)&slot_run_, sizeof(uint32_t) * max_runs))) return st;
    if ((st = galloc(v, (void **)&tree_base_, sizeof(uint32_t) * (max_runs + 1)))) return st;
    if ((st = galloc(v, (void **)&run_tiles_, sizeof(uint32_t) * (max_runs + 1)))) return st;
    if ((st = galloc(v, (void **)&recs_, sizeof(gp_xo) * T))) return st;
    if ((st = galloc(v, (void **)&q_, sizeof(ExtentQuery) * 2 * T))) return st;
    if ((st = galloc(v, (void **)&xlong_, sizeof(ExtentLong) * 2 * T))) return st;
    if ((st = galloc(v, (void **)&ends_, sizeof(uint64_t) * 2 * T))) return st;
    if ((st = galloc(v, (void **)&kids_, sizeof(XoChild) * T))) return st;
    if ((st = galloc(v, (void **)&tile_local_, sizeof(uint32_t) * T))) return st;
    if ((st = galloc(v, (void **)&bstart_, sizeof(uint64_t) * T))) return st;
    if ((st = galloc(v, (void **)&bsize_, sizeof(uint64_t) * T))) return st;
    if ((st = galloc(v, (void **)&bfit_, sizeof(float) * T))) return st;
    if ((st = galloc(v, (void **)&bvals_, sizeof(float) * T * n_cases))) return st;
    if ((st = galloc(v, (void **)&bhits_, sizeof(uint32_t) * T))) return st;
    if ((st = galloc(v, (void **)&t_lo_, sizeof(uint64_t) * T))) return st;
    if ((st = galloc(v, (void **)&t_hi_, sizeof(uint64_t) * T))) return st;
    if ((st = galloc(v, (void **)&t_prev_, sizeof(uint64_t) * T))) return st;
    if ((st = galloc(v, (void **)&t_first_, sizeof(uint32_t) * (T + 1)))) return st;
    if ((st = galloc(v, (void **)&t_state_, sizeof(uint32_t) * T))) return st;
    if ((st = galloc(v, (void **)&t_nch_, sizeof(uint32_t) * T))) return st;
    if ((st = galloc(v, (void **)&t_cut_, sizeof(uint32_t) * T * (kFuseMaxChunks - 1)))) return st;
    if ((st = galloc(v, (void **)&fz_tree_, sizeof(uint32_t) * T * kFuseMaxChunks))) return st;
    if ((st = galloc(v, (void **)&fin_tree_, sizeof(uint32_t) * T))) return st;
    if ((st = galloc(v, (void **)&rope_tree_, sizeof(uint32_t) * T))) return st;
    if ((st = galloc(v, (void **)&rope_items_, sizeof(EvalItem) * T))) return st;
    if ((st = galloc(v, (void **)&x_, sizeof(float) * 2 * lanes))) return st;
    if ((st = galloc(v, (void **)&y_, sizeof(float) * 2 * lanes))) return st;
    if ((st = galloc(v, (void **)&c_, sizeof(float) * (n_consts + 1)))) return st;
    std::vector<float> hx(2 * lanes, 0.f), hy(2 * lanes, 0.f);
    std::memcpy(hx.data(), problem->x, sizeof(float) * n_cases);
    std::memcpy(hy.data(), problem->y, sizeof(float) * n_cases);
    GK(cudaMemcpy(x_, hx.data(), sizeof(float) * hx.size(), cudaMemcpyHostToDevice));
    GK(cudaMemcpy(y_, hy.data(), sizeof(float) * hy.size(), cudaMemcpyHostToDevice));
    if (n_consts) GK(cudaMemcpy(c_, problem->consts, sizeof(float) * n_consts, cudaMemcpyHostToDevice));
    return GP_OK;
}

uint64_t Engine::heap_alloc(uint64_t bytes)
{
    bytes = (bytes + 255) & ~255ull;
    for (size_t i = 0; i < free_.size(); ++i) {
        if (free_[i].second >= bytes) {
            const uint64_t off = free_[i].first;
            free_[i].first += bytes;
            free_[i].second -= bytes;
            if (free_[i].second == 0) free_.erase(free_.begin() + (long)i);
            return off;
        }
    }
    return ~0ull;
}

void Engine::heap_release(uint64_t off, uint64_t bytes)
{
    bytes = (bytes + 255) & ~255ull;
    auto it = std::lower_bound(free_.begin(), free_.end(), std::make_pair(off, (uint64_t)0));
    it = free_.insert(it, {off, bytes});
    // merge with the next and the previous block
    auto nx = it + 1;
    if (nx != free_.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        free_.erase(nx);
    }
    if (it != free_.begin()) {
        auto pv = it - 1;
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            free_.erase(it);
        }
    }
}

uint64_t Engine::heap_free() const
{
    uint64_t s = 0;
    for (auto &f : free_) s += f.second;
    return s;
}

uint64_t Engine::heap_largest_free() const
{
    uint64_t m = 0;
    for (auto &f : free_) m = std::max(m, f.second);
    return m;
}

gp_status Engine::open_run(uint32_t n, uint64_t arena_cap, uint64_t seed, uint32_t tsize, uint64_t max_nodes,
                           uint32_t *run)
{
    uint32_t r = 0;
    while (r < max_runs && runs_host[r].used) ++r;
    if (r == max_runs || n == 0 || n > max_trees) return r == max_runs ? GP_ENOMEM : GP_EINVAL;
    // (allocations are rounded up to 256 bytes; the capacity checked is the
    // one asked for)
    const uint64_t lo0 = heap_alloc(arena_cap);
    if (lo0 == ~0ull) return GP_ENOMEM;
    const uint64_t lo1 = heap_alloc(arena_cap);
    if (lo1 == ~0ull) {
        heap_release(lo0, arena_cap);
        return GP_ENOMEM;
    }
    RunHost &H = runs_host[r];
    H = RunHost{};
    H.used = true;
    H.n = n;
    H.arena_cap = arena_cap;
    H.lo[0] = lo0;
    H.lo[1] = lo1;
    RunDev D{};
    D.seed = seed;
    D.max_nodes = max_nodes;
    D.n = n;
    D.tsize = tsize;
    gp_status st = GP_OK;
    for (int b = 0; b < 2 && !st; ++b) {
        RunBuf &B = D.buf[b];
        B.lo = H.lo[b];
        B.cap = arena_cap;
        if ((st = galloc(H.allocs, (void **)&B.start, sizeof(uint64_t) * n))) break;
        if ((st = galloc(H.allocs, (void **)&B.size, sizeof(uint64_t) * n))) break;
        if ((st = galloc(H.allocs, (void **)&B.fit, sizeof(float) * n))) break;
        if ((st = galloc(H.allocs, (void **)&B.vals, sizeof(float) * (uint64_t)n * n_cases))) break;
        if ((st = galloc(H.allocs, (void **)&B.hits, sizeof(uint32_t) * n))) break;
    }
    if (!st && cudaMemcpy(runs_dev + r, &D, sizeof(D), cudaMemcpyHostToDevice) != cudaSuccess) st = GP_ECUDA;
    if (st) {
        close_run(r);
        return st;
    }
    *run = r;
    return GP_OK;
}

void Engine::close_run(uint32_t r)
{
    if (r >= max_runs || !runs_host[r].used) return;
    cudaDeviceSynchronize();
    RunHost &H = runs_host[r];
    heap_release(H.lo[0], H.arena_cap);
    heap_release(H.lo[1], H.arena_cap);
    gfree(H.allocs);
    H = RunHost{};
    RunDev D{};
    cudaMemcpy(runs_dev + r, &D, sizeof(D), cudaMemcpyHostToDevice);
}

gp_status Engine::grow_run(uint32_t r, uint64_t arena_cap, cudaStream_t s)
{
    if (r >= max_runs || !runs_host[r].used) return GP_EINVAL;
    RunHost &H = runs_host[r];
    if (arena_cap <= H.arena_cap) return GP_EINVAL;
    const uint64_t lo0 = heap_alloc(arena_cap);
    if (lo0 == ~0ull) return GP_ENOMEM;
    const uint64_t lo1 = heap_alloc(arena_cap);
    if (lo1 == ~0ull) {
        heap_release(lo0, arena_cap);
        return GP_ENOMEM;
    }
    const uint64_t lo[2] = {lo0, lo1};
    RunDev D{};
    gp_status st = read_run(r, &D, s);
    if (st) return st;
    const uint32_t c = D.cur;
    GK(cudaMemcpyAsync(heap + lo[c], heap + H.lo[c], H.arena_cap, cudaMemcpyDeviceToDevice, s));
    rebase_kernel<<<std::max<uint32_t>(1, std::min<uint32_t>((H.n + 255) / 256, sms * 4)), 256, 0, s>>>(
        D.buf[c].start, H.n, lo[c] - H.lo[c]);
    GK(cudaGetLastError());
    for (int b = 0; b < 2; ++b) {
        D.buf[b].lo = lo[b];
        D.buf[b].cap = arena_cap;
    }
    GK(cudaMemcpyAsync(runs_dev + r, &D, sizeof(D), cudaMemcpyHostToDevice, s));
    GK(cudaStreamSynchronize(s));
    heap_release(H.lo[0], H.arena_cap);
    heap_release(H.lo[1], H.arena_cap);
    H.lo[0] = lo0;
    H.lo[1] = lo1;
    H.arena_cap = arena_cap;
    return GP_OK;
}

gp_status Engine::grow_heap(uint64_t new_bytes)
{
    if (new_bytes <= heap_bytes) return GP_EINVAL;
    GK(cudaDeviceSynchronize());
    uint8_t *nh = nullptr;
    GK(cudaMalloc((void **)&nh, kHeapLead + new_bytes + 64));
    cudaError_t e = cudaMemcpy(nh, heap, kHeapLead + heap_bytes + 64, cudaMemcpyDeviceToDevice);
    if (e != cudaSuccess) {
        cudaFree(nh);
        return gfail(e);
    }
    for (auto &p : allocs_)
        if (p == heap) p = nh;
    cudaFree(heap);
    heap = nh;
    heap_release(kHeapLead + heap_bytes, new_bytes - heap_bytes);
    heap_bytes = new_bytes;
    forget_head();
    for (auto &x : exec)
        if (x) {
            cudaGraphExecDestroy(x);
            x = nullptr;
        }
    return GP_OK;
}

gp_status Engine::load_run(uint32_t r, const uint8_t *nodes, const uint64_t *offsets, cudaStream_t s)
{
    if (r >= max_runs || !runs_host[r].used) return GP_EINVAL;
    RunHost &H = runs_host[r];
    const uint32_t n = H.n;
    std::vector<uint64_t> hstart(n), hsize(n);
    uint64_t pos = 0;
    for (uint32_t t = 0; t < n; ++t) {
        if (offsets[t + 1] <= offsets[t]) return GP_EINVAL;
        hsize[t] = offsets[t + 1] - offsets[t];
        hstart[t] = H.lo[0] + pos;
        pos = (pos + hsize[t] + 15) & ~15ull;
    }
    if (pos + 64 > H.arena_cap) return GP_ENOMEM;
    // upload and validate through the population API, then take its layout
    // (the same 16-byte aligned starts)
    gp_problem pr{};
    std::vector<float> dummy(n_cases, 0.f), cz(n_consts + 1, 0.f);
    pr.n_cases = n_cases;
    pr.x = dummy.data();
    pr.y = dummy.data();
    pr.n_consts = n_consts;
    pr.consts = cz.data();
    pr.protected_div_value = div0;
    gp_population *tmp = nullptr;
    gp_status st = gp_create_population(&pr, n, nodes, offsets, s, &tmp);
    if (st) return st;
    gp_population_info pi{};
    gp_population_get_info(tmp, &pi);
    RunDev D{};
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(heap + H.lo[0], pi.d_nodes, pos, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(&D, runs_dev + r, sizeof(D), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(D.buf[0].start, hstart.data(), sizeof(uint64_t) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(D.buf[0].size, hsize.data(), sizeof(uint64_t) * n, cudaMemcpyHostToDevice);
    D.gen = 0;
    D.cur = 0;
    D.err = 0;
    D.err_gen = 0;
    D.nodes = offsets[n];
    if (e == cudaSuccess) e = cudaMemcpy(runs_dev + r, &D, sizeof(D), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    gp_destroy_population(tmp);
    // the upload's buffers went back to the stream-ordered pool, which keeps
    // freed memory: hand it back so the engine's own allocations can use it
    cudaMemPool_t pool;
    if (cudaDeviceSynchronize() == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess)
        cudaMemPoolTrimTo(pool, 0);
    return e == cudaSuccess ? GP_OK : gfail(e);
}

gp_status Engine::load_run_from(uint32_t r, const gp_population *src, const uint32_t *trees, cudaStream_t s)
{
    if (r >= max_runs || !runs_host[r].used || !src || !trees) return GP_EINVAL;
    RunHost &H = runs_host[r];
    const uint32_t n = H.n;
    std::vector<uint64_t> hstart(n), hsize(n);
    gp_status st = gpk::gather_trees(src, trees, n, heap, H.lo[0], H.arena_cap, hstart.data(), hsize.data(), s);
    if (st) return st;
    uint64_t total = 0;
    for (uint64_t z : hsize) total += z;
    RunDev D{};
    cudaError_t e = cudaMemcpyAsync(&D, runs_dev + r, sizeof(D), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(D.buf[0].start, hstart.data(), sizeof(uint64_t) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(D.buf[0].size, hsize.data(), sizeof(uint64_t) * n, cudaMemcpyHostToDevice, s);
    D.gen = 0;
    D.cur = 0;
    D.err = 0;
    D.err_gen = 0;
    D.nodes = total;
    if (e == cudaSuccess) e = cudaMemcpyAsync(runs_dev + r, &D, sizeof(D), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);    // the host arrays are read by then
    return e == cudaSuccess ? GP_OK : gfail(e);
}

gp_status Engine::set_shape(uint32_t W_, uint32_t K_, uint32_t Wu_, uint32_t Ku_, uint32_t Wr_, uint32_t Kr_)
{
    int maxsm = 0;
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    auto ok = [&](uint32_t w, uint32_t k, bool wide) {
        return w >= 1 && w <= 32 && k >= 16 && k % 2 == 0 && k <= 1024 && (!wide || w <= 16) &&
               eval_smem_bytes(lanes, (int)w, (int)k, wide, rows) <= (size_t)maxsm;
    };
    if (!ok(W_, K_, false) || !ok(Wu_, Ku_, true) || !ok(Wr_, Kr_, true)) return GP_EINVAL;
    W = W_;
    K = K_;
    Wu = Wu_;
    Ku = Ku_;
    Wr = Wr_;
    Kr = Kr_;
    smem = eval_smem_bytes(lanes, (int)W, (int)K, false, rows);
    smem_u = eval_smem_bytes(lanes, (int)Wu, (int)Ku, true, rows);
    smem_r = eval_smem_bytes(lanes, (int)Wr, (int)Kr, true, rows);
    GK(eval_prepare_at_least(lanes, false, smem));
    GK(eval_prepare_at_least(lanes, true, std::max(smem_u, smem_r)));
    for (auto &e : exec)                 // the graphs captured the old shapes
        if (e) {
            cudaGraphExecDestroy(e);
            e = nullptr;
        }
    return GP_OK;
}

gp_status Engine::set_slots(uint64_t cap_slots, uint32_t fz_cap_pt)
{
    cudaDeviceSynchronize();
    for (void *p : {(void *)w.fz_codes, (void *)w.fz_pt, (void *)w.fz_len, (void *)w.fz_over, (void *)w.fz_redo})
        if (p) {
            cudaFree(p);
            work_allocs_.erase(std::remove(work_allocs_.begin(), work_allocs_.end(), p), work_allocs_.end());
        }
    w.fz_codes = w.fz_len = w.fz_over = w.fz_redo = nullptr;
    w.fz_pt = nullptr;
    w.cap_slots = cap_slots;
    w.fz_cap_pt = fz_cap_pt ? fz_cap_pt : std::max<uint32_t>(128, w.C / 8);
    for (auto &e : exec)                 // the graphs captured the old slots
        if (e) {
            cudaGraphExecDestroy(e);
            e = nullptr;
        }
    if (!cap_slots) return GP_OK;
    auto &v = work_allocs_;
    gp_status st;
    if ((st = galloc(v, (void **)&w.fz_codes, sizeof(uint32_t) * (cap_slots * w.C + 32)))) return st;
    if ((st = galloc(v, (void **)&w.fz_pt, sizeof(float2) * (cap_slots * w.fz_cap_pt * lanes + 1)))) return st;
    if ((st = galloc(v, (void **)&w.fz_len, sizeof(uint32_t) * cap_slots))) return st;
    if ((st = galloc(v, (void **)&w.fz_over, sizeof(uint32_t) * max_trees))) return st;
    if ((st = galloc(v, (void **)&w.fz_redo, sizeof(uint32_t) * (1 + (uint64_t)max_trees)))) return st;
    if (cudaMemset(w.fz_over, 0, sizeof(uint32_t) * max_trees) != cudaSuccess ||
        cudaMemset(w.fz_redo, 0, sizeof(uint32_t)) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
        return GP_ECUDA;                 // done before any stream uses the slots
    return GP_OK;
}

gp_status Engine::set_workspace(uint32_t C, const uint64_t cap_codes[2], const uint64_t cap_values[2],
                                uint64_t cap_dedicated, uint64_t cap_items, uint64_t cap_slots, uint32_t fz_cap_pt)
{
    cudaDeviceSynchronize();
    gfree(work_allocs_);
    w = Work{};
    w.C = C;
    for (int k = 0; k < 2; ++k) {
        w.cap_codes[k] = cap_codes[k];
        w.cap_values[k] = cap_values[k];
    }
    w.cap_items = cap_items;
    w.cap_dedicated = cap_dedicated;
    if (w.cap_items > 0xffffffffull) return GP_ENOMEM;
    const uint64_t warps = (uint64_t)sms * std::max(W, std::max(Wu, Wr));
    w.spill_per_warp = C;
    w.spill_base = warps * C;
    auto &v = work_allocs_;
    gp_status st;
    if ((st = galloc(v, (void **)&w.items, sizeof(EvalItem) * w.cap_items))) return st;
    if ((st = galloc(v, (void **)&w.plan, sizeof(PlanOut) * w.cap_items))) return st;
    if ((st = galloc(v, (void **)&w.frag_off, sizeof(uint64_t) * (w.cap_items + 1)))) return st;
    for (int k = 0; k < 2; ++k) {
        if ((st = galloc(v, (void **)&w.codes[k], sizeof(uint32_t) * (cap_codes[k] + 64)))) return st;
        if ((st = galloc(v, (void **)&w.vals[k], sizeof(float2) * (cap_values[k] * lanes + 1)))) return st;
    }
    if ((st = galloc(v, (void **)&w.spill, sizeof(float2) * lanes * (w.spill_base + w.cap_dedicated)))) return st;
    if ((st = set_slots(cap_slots, fz_cap_pt))) return st;
    const char *vb = std::getenv("GP_VERBOSE");
    size_t fr = 0, tot = 0;
    if (vb && vb[0] == '1' && cudaMemGetInfo(&fr, &tot) == cudaSuccess)
        std::fprintf(stderr, "engine workspace: codes %.1f GB, values %.1f GB, spill %.1f GB; %.1f GB free\n",
                     4.0 * (cap_codes[0] + cap_codes[1]) / 1e9, 8.0 * lanes * (cap_values[0] + cap_values[1]) / 1e9,
                     8.0 * lanes * (w.spill_base + w.cap_dedicated) / 1e9, fr / 1e9);
    // the graphs captured the old workspace
    for (auto &e : exec)
        if (e) {
            cudaGraphExecDestroy(e);
            e = nullptr;
        }
    return GP_OK;
}

gp_status Engine::write_head(uint32_t mode, const std::vector<uint32_t> &runs, cudaStream_t s)
{
    if (runs.empty() || runs.size() > max_runs) return GP_EINVAL;
    std::vector<uint32_t> base(runs.size() + 1);
    uint64_t tot = 0;
    for (size_t i = 0; i < runs.size(); ++i) {
        if (runs[i] >= max_runs || !runs_host[runs[i]].used) return GP_EINVAL;
        base[i] = (uint32_t)tot;
        tot += runs_host[runs[i]].n;
    }
    if (tot > max_trees) return GP_EINVAL;
    if (mode == last_mode_ && runs == last_runs_) return GP_OK;     // already on the device
    base[runs.size()] = (uint32_t)tot;
    BatchHead h{mode, (uint32_t)runs.size(), (uint32_t)tot, 0};
    // pageable sources: each copy has consumed its source when the call returns
    GK(cudaMemcpyAsync(&ctl->head, &h, sizeof(h), cudaMemcpyHostToDevice, s));
    GK(cudaMemcpyAsync(slot_run_, runs.data(), sizeof(uint32_t) * runs.size(), cudaMemcpyHostToDevice, s));
    GK(cudaMemcpyAsync(tree_base_, base.data(), sizeof(uint32_t) * base.size(), cudaMemcpyHostToDevice, s));
    last_mode_ = mode;
    last_runs_ = runs;
    return GP_OK;
}

// Graph conditions and work counter of a level inside the captured level
// loop (all zero for a level launched directly).
struct Engine::LevelCond {
    uint32_t flags = 0;                  // check_kernel: bit 0 sets `more`, bit 1 zeroes `zero`
    cudaGraphConditionalHandle more = 0, zero = 0;
    uint32_t *counter = nullptr;         // the level's work counter, zeroed by check_kernel
};

// One evaluation level: items, chunk fill, plan, plan scan, workspace
// check, evaluator.  `dyn`: a level of the captured loop (its number comes
// from the control block; its buffers alternate by the parity of `level`).
gp_status Engine::enqueue_level(uint32_t level, bool dyn, cudaStream_t s, bool sizing, uint32_t &prev_chunks,
                                const LevelCond &cond, uint32_t *nl_out, bool *stop)
{
    uint32_t nl = 0;
    const bool wide = dyn || level > 0;
    const int k = level & 1;
    const bool pdl = !dyn;               // inside a conditional body: plain launches
    LevelArgs A{dyn ? kDynLevel : level, w.C, (uint32_t)std::min<uint64_t>(w.cap_items, 0xffffffffu),
                dyn ? levels_cap_graph : (level + 1 == levels_max ? 1u : 0u), w.spill_base, w.cap_dedicated,
                w.cap_slots};
    // the level's decisions: at level 0 the cut kernel first (it also sets
    // every tree's level-0 range and state, so a build started again in the
    // sizing pass starts from scratch), then the single-CTA item builder
    auto build = [&](bool use_pdl) -> cudaError_t {
        cudaError_t e = cudaSuccess;
        if (level == 0 && !dyn) {
            if (use_pdl)
                e = launch_pdl(cut_fused_kernel, dim3(sms * 8), dim3(256), 0, s, ctl, w.C, heap, bstart_, bsize_,
                               t_nch_, t_cut_, t_lo_, t_hi_, t_prev_, t_state_);
            else
                cut_fused_kernel<<<sms * 8, 256, 0, s>>>(ctl, w.C, heap, bstart_, bsize_, t_nch_, t_cut_, t_lo_, t_hi_,
                                                         t_prev_, t_state_);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        if (use_pdl)
            return launch_pdl(items_kernel, dim3(1), dim3(kScanT), 0, s, ctl, A, bstart_, bsize_, w.frag_off, t_lo_,
                              t_hi_, t_prev_, t_first_, t_state_, t_nch_, fz_tree_, fin_tree_, rope_tree_,
                              rope_items_ != nullptr);
        items_kernel<<<1, kScanT, 0, s>>>(ctl, A, bstart_, bsize_, w.frag_off, t_lo_, t_hi_, t_prev_, t_first_,
                                          t_state_, t_nch_, fz_tree_, fin_tree_, rope_tree_, rope_items_ != nullptr);
        return cudaGetLastError();
    };
    GK(build(pdl));
    if (level == 0 && !dyn) ++nl;
    if (sizing) {
        // a dedicated spill pool too small for this level's oversized
        // finals: grow it, clear the error and build the level again
        // (the kernel changes nothing else when it raises that error)
        BatchCtl c{};
        GK(cudaMemcpyAsync(&c, ctl, sizeof(c), cudaMemcpyDeviceToHost, s));
        GK(cudaStreamSynchronize(s));
        if (level == 0 && c.err == 0 && w.cap_slots && c.need_slots > w.cap_slots) {
            // more fused-chunk candidates than slots (some went planned):
            // more slots, the level again
            gp_status st = set_slots(std::max<uint64_t>(2 * c.need_slots, w.cap_slots), w.fz_cap_pt);
            if (st) return st;
            A.cap_slots = w.cap_slots;
            GK(cudaMemsetAsync(&ctl->err, 0, sizeof(uint32_t), s));
            GK(cudaMemsetAsync(w.fz_over, 0, sizeof(uint32_t) * max_trees, s));
            GK(cudaMemsetAsync(w.fz_redo, 0, sizeof(uint32_t), s));
            GK(build(false));
            GK(cudaMemcpyAsync(&c, ctl, sizeof(c), cudaMemcpyDeviceToHost, s));
            GK(cudaStreamSynchronize(s));
        }
        if (c.err == kGErrSpill) {
            const uint64_t nd = std::max<uint64_t>(2 * c.need_dedicated, w.cap_dedicated);
            void *p = nullptr;
            GK(cudaMalloc(&p, sizeof(float2) * lanes * (w.spill_base + nd)));
            work_allocs_.push_back(p);
            w.spill = (float2 *)p;
            w.cap_dedicated = nd;
            A.cap_dedicated = nd;
            // the failed build zeroed the chunk count the level starts
            // from: put back the previous level's before building again
            GK(cudaMemsetAsync(&ctl->err, 0, sizeof(uint32_t), s));
            GK(cudaMemcpyAsync(&ctl->n_chunks, &prev_chunks, sizeof(uint32_t), cudaMemcpyHostToDevice, s));
            GK(build(false));
            GK(cudaMemcpyAsync(&c, ctl, sizeof(c), cudaMemcpyDeviceToHost, s));
            GK(cudaStreamSynchronize(s));
        }
        prev_chunks = c.n_chunks;
    }
    EvalItem *ropes_out = (level == 0 && !dyn) ? rope_items_ : nullptr;
    if (pdl) {
        GK(launch_pdl(fill_items_kernel, dim3(sms * 4), dim3(256), 0, s, ctl, A, t_first_, t_lo_, t_hi_, t_prev_,
                      bstart_, bsize_, t_cut_, fz_tree_, fin_tree_, rope_tree_, w.items, ropes_out));
    } else {
        fill_items_kernel<<<sms * 4, 256, 0, s>>>(ctl, A, t_first_, t_lo_, t_hi_, t_prev_, bstart_, bsize_, t_cut_,
                                                  fz_tree_, fin_tree_, rope_tree_, w.items, ropes_out);
        GK(cudaGetLastError());
    }
    const void *codes = wide ? (const void *)w.codes[k ^ 1] : (const void *)heap;
    GK(launch_plan_dev(wide, codes, w.items, (uint32_t)w.cap_items, &ctl->n_chunks, w.plan, sms, s, pdl));
    GK(launch_plan_scan_dev(w.items, w.plan, &ctl->n_chunks, w.frag_off, ctl->totals, s, pdl));
    nl += 4;
    if (sizing) {
        uint64_t tot[2];
        uint32_t err = 0, n_items = 0;
        GK(cudaMemcpyAsync(tot, ctl->totals, sizeof(tot), cudaMemcpyDeviceToHost, s));
        GK(cudaMemcpyAsync(&err, &ctl->err, sizeof(err), cudaMemcpyDeviceToHost, s));
        GK(cudaMemcpyAsync(&n_items, &ctl->n_items, sizeof(n_items), cudaMemcpyDeviceToHost, s));
        GK(cudaStreamSynchronize(s));
        if (err || n_items == 0) {
            *stop = true;
            return GP_OK;
        }
        if (tot[0] + 48 > w.cap_codes[k] || tot[1] > w.cap_values[k]) {
            // grow this level's output buffers; they hold nothing still
            // needed (the outputs of level - 2)
            const uint64_t nc = std::max<uint64_t>(w.cap_codes[k], tot[0] + tot[0] / 8 + 1024);
            const uint64_t nv = std::max<uint64_t>(w.cap_values[k], tot[1] + tot[1] / 8 + 1024);
            void *pc = nullptr, *pv = nullptr;
            const char *vb = std::getenv("GP_VERBOSE");
            if (vb && vb[0] == '1')
                std::fprintf(stderr, "engine sizing: level %u needs %llu codes, %llu value entries (%.1f GB)\n",
                             level, (unsigned long long)tot[0], (unsigned long long)tot[1],
                             (double)nv * lanes * 8 / 1e9);
            GK(cudaMalloc(&pc, sizeof(uint32_t) * (nc + 64)));
            work_allocs_.push_back(pc);
            GK(cudaMalloc(&pv, sizeof(float2) * (nv * lanes + 1)));
            work_allocs_.push_back(pv);
            w.codes[k] = (uint32_t *)pc;
            w.vals[k] = (float2 *)pv;
            w.cap_codes[k] = nc;
            w.cap_values[k] = nv;
        }
    }
    if (pdl && !sizing) {
        GK(launch_pdl(check_kernel, dim3(1), dim3(64), 0, s, ctl, w.cap_codes[k], w.cap_values[k], w.codes[k],
                      (uint32_t)k, cond.counter, cond.flags, cond.more, cond.zero));
    } else {
        check_kernel<<<1, 64, 0, s>>>(ctl, w.cap_codes[k], w.cap_values[k], w.codes[k], (uint32_t)k, cond.counter,
                                      cond.flags, cond.more, cond.zero);
        GK(cudaGetLastError());
    }
    EvalParams p{};
    p.codes = codes;
    p.items = w.items;
    p.n_items = (uint32_t)std::min<uint64_t>(w.cap_items, 0xffffffffu);
    p.n_items_dev = &ctl->n_items;
    p.counter = cond.counter ? cond.counter : &ctl->counter[level];
    p.x = x_;
    p.y = y_;
    p.consts = c_;
    p.n_cases = n_cases;
    p.n_consts = n_consts;
    p.leaf_rows = (uint32_t)rows;
    p.div0 = div0;
    p.window = wide ? Ku : K;
    p.pt_in = wide ? w.vals[k ^ 1] : nullptr;
    p.pt_out = w.vals[k];
    p.u_out = w.codes[k];
    p.values = bvals_;
    p.fitness = bfit_;
    p.hits = bhits_;
    p.spill = w.spill;
    p.spill_per_warp = w.spill_per_warp;
    p.err = &ctl->eval_err[0];
    if (w.cap_slots) {
        p.fz_codes = w.fz_codes;
        p.fz_pt = w.fz_pt;
        p.fz_len = w.fz_len;
        p.fz_over = w.fz_over;
        p.fz_redo = w.fz_redo;
        p.fz_cap_codes = w.C;
        p.fz_cap_pt = w.fz_cap_pt;
    }
    GK(launch_eval(lanes, wide, p, sms, (int)(wide ? Wu : W), wide ? smem_u : smem, s, pdl));
    nl += 2;
    *nl_out += nl;
    return GP_OK;
}

gp_status Engine::enqueue_eval(cudaStream_t s, bool sizing, uint32_t *launches)
{
    uint32_t nl = 0;
    uint32_t prev_chunks = 0;            // sizing: chunks the previous level cut
    bool stop = false;
    if (!capturing_ || sizing) {
        // a fixed sequence of levels_max levels (empty ones return at once)
        for (uint32_t level = 0; level < levels_max && !stop; ++level) {
            gp_status st = enqueue_level(level, false, s, sizing, prev_chunks, LevelCond{}, &nl, &stop);
            if (st) return st;
        }
        if (launches) *launches += nl;
        return GP_OK;
    }
    // Captured: level 0, then an IF/ELSE node.  When level 0 cut planned
    // chunks, a WHILE node runs the upper levels (its body one odd level and
    // an IF node holding the next even level); each level's check kernel
    // says whether the next level has trees, so a replay runs exactly the
    // levels the generation needs (at most levels_cap_graph, the last of
    // which finishes every open tree).  Otherwise the only upper level is
    // the ropes level 0 listed, evaluated by one launch shaped for ropes.
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr, gb = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    GK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphConditionalHandle h_up = 0, h_loop = 0, h_even = 0;
    GK(cudaGraphConditionalHandleCreate(&h_up, g, 0, cudaGraphCondAssignDefault));
    GK(cudaGraphConditionalHandleCreate(&h_loop, g, 0, cudaGraphCondAssignDefault));
    GK(cudaGraphConditionalHandleCreate(&h_even, g, 0, cudaGraphCondAssignDefault));
    LevelCond c0;
    c0.flags = 1 | 4;                    // the loop's first pass; planned chunks choose the loop
    c0.more = h_loop;
    c0.zero = h_up;
    gp_status st = enqueue_level(0, false, s, false, prev_chunks, c0, &nl, &stop);
    if (st) return st;
    GK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphNodeParams up{};
    up.type = cudaGraphNodeTypeConditional;
    up.conditional.handle = h_up;
    up.conditional.type = cudaGraphCondTypeIf;
    up.conditional.size = 2;
    cudaGraphNode_t un;
    GK(cudaGraphAddNode(&un, g, deps, nullptr, nd, &up));
    GK(cudaStreamUpdateCaptureDependencies(s, &un, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaGraphNodeParams wp{};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = h_loop;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wn;
    GK(cudaGraphAddNode(&wn, up.conditional.phGraph_out[0], nullptr, nullptr, 0, &wp));
    GK(cudaStreamBeginCaptureToGraph(cap_body[0], wp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                     cudaStreamCaptureModeThreadLocal));
    uint32_t nl_odd = 0, nl_even = 0;
    auto body = [&]() -> gp_status {
        LevelCond c1;
        c1.flags = 1 | 2;                // the even level's IF; the loop stops unless it continues it
        c1.more = h_even;
        c1.zero = h_loop;
        c1.counter = &ctl->counter[62];
        gp_status e = enqueue_level(1, true, cap_body[0], false, prev_chunks, c1, &nl_odd, &stop);
        if (e) return e;
        cudaGraph_t gi = nullptr;
        GK(cudaStreamGetCaptureInfo(cap_body[0], &cs, nullptr, &gi, &deps, nullptr, &nd));
        cudaGraphNodeParams ip{};
        ip.type = cudaGraphNodeTypeConditional;
        ip.conditional.handle = h_even;
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        cudaGraphNode_t in;
        GK(cudaGraphAddNode(&in, gi, deps, nullptr, nd, &ip));
        GK(cudaStreamUpdateCaptureDependencies(cap_body[0], &in, nullptr, 1, cudaStreamSetCaptureDependencies));
        GK(cudaStreamBeginCaptureToGraph(cap_body[1], ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal));
        LevelCond c2;
        c2.flags = 1;                    // the loop goes on when the next odd level has trees
        c2.more = h_loop;
        c2.counter = &ctl->counter[63];
        e = enqueue_level(2, true, cap_body[1], false, prev_chunks, c2, &nl_even, &stop);
        cudaError_t ce = cudaStreamEndCapture(cap_body[1], &gb);
        if (e) return e;
        GK(ce);
        return GP_OK;
    };
    st = body();
    cudaError_t ce = cudaStreamEndCapture(cap_body[0], &gb);
    if (st) return st;
    GK(ce);
    // the ropes-only branch
    GK(cudaStreamBeginCaptureToGraph(cap_body[0], up.conditional.phGraph_out[1], nullptr, nullptr, 0,
                                     cudaStreamCaptureModeThreadLocal));
    EvalParams p{};
    p.codes = heap;
    p.items = rope_items_;
    p.n_items = max_trees;
    p.n_items_dev = &ctl->n_rope_items;
    p.counter = &ctl->counter[61];
    p.x = x_;
    p.y = y_;
    p.consts = c_;
    p.n_cases = n_cases;
    p.n_consts = n_consts;
    p.leaf_rows = (uint32_t)rows;
    p.div0 = div0;
    p.window = Kr;
    p.values = bvals_;
    p.fitness = bfit_;
    p.hits = bhits_;
    p.spill = w.spill;
    p.spill_per_warp = w.spill_per_warp;
    p.err = &ctl->eval_err[0];
    if (w.cap_slots) {
        p.fz_codes = w.fz_codes;
        p.fz_pt = w.fz_pt;
        p.fz_len = w.fz_len;
        p.fz_over = w.fz_over;
        p.fz_redo = w.fz_redo;
        p.fz_cap_codes = w.C;
        p.fz_cap_pt = w.fz_cap_pt;
    }
    cudaError_t le = launch_eval(lanes, true, p, sms, (int)Wr, smem_r, cap_body[0]);
    ce = cudaStreamEndCapture(cap_body[0], &gb);
    GK(le);
    GK(ce);
    kernels_per_level = nl_odd;
    if (launches) *launches += nl + nl_odd + nl_even + 1;
    return GP_OK;
}

gp_status Engine::enqueue_body(uint32_t mode, cudaStream_t s, bool sizing, uint32_t *launches)
{
    (void)mode;
    uint32_t nl = 0;
    GK(cudaMemsetAsync(ctl->counter, 0, sizeof(ctl->counter), s));
    // err, n_queries, n_tiles, n_items, n_chunks, levels, eval_err[4], n_ropes, loop_level,
    // n_rope_items
    GK(cudaMemsetAsync(&ctl->err, 0, sizeof(uint32_t) * 13, s));
    if (w.cap_slots) {                   // fused slots: overflow flags and the redo list
        GK(cudaMemsetAsync(w.fz_over, 0, sizeof(uint32_t) * max_trees, s));
        GK(cudaMemsetAsync(w.fz_redo, 0, sizeof(uint32_t), s));
    }
    GK(cudaMemsetAsync(&ctl->child_nodes, 0, sizeof(uint64_t), s));
    const uint32_t blocks = std::max<uint32_t>(1, std::min<uint32_t>((max_trees + 127) / 128, sms * 8));
    select_kernel<<<blocks, 128, 0, s>>>(ctl, runs_dev, slot_run_, tree_base_, recs_, q_);
    GK(cudaGetLastError());
    // (eval_err[3], zeroed above, counts the walks left to the long-walk launch)
    GK(launch_extent_dev(heap, q_, 2 * max_trees, &ctl->n_queries, ends_, &ctl->eval_err[1], xlong_,
                         &ctl->eval_err[3], sms, s));
    // from here to level 0's evaluator every kernel is a programmatic
    // dependent launch (its launch overlaps the tail of the one before)
    GK(launch_pdl(children_size_kernel, dim3(blocks), dim3(128), 0, s, ctl, runs_dev, slot_run_, tree_base_, q_, ends_,
                  bstart_, bsize_));
    GK(launch_pdl(children_scan_kernel, dim3(max_runs), dim3(kScanT), 0, s, ctl, runs_dev, slot_run_, tree_base_,
                  tile_local_, run_tiles_, bstart_, bsize_, xo_tile));
    GK(launch_pdl(children_place_kernel, dim3(blocks), dim3(128), 0, s, ctl, runs_dev, slot_run_, tree_base_, q_, ends_,
                  kids_, bstart_, bsize_));
    GK(launch_pdl(run_tiles_scan_kernel, dim3(1), dim3(32), 0, s, ctl, run_tiles_));
    GK(launch_xo_copy_runs(heap, kids_, tile_local_, tree_base_, run_tiles_, &ctl->head.n_runs, &ctl->n_tiles,
                           xo_tile, xo_warp, sms, s));
    nl += 8;
    gp_status st = enqueue_eval(s, sizing, &nl);
    if (st) return st;
    const uint32_t sblocks =
        (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(((uint64_t)max_trees * n_cases + 255) / 256, sms * 8));
    scatter_kernel<<<sblocks, 256, 0, s>>>(ctl, runs_dev, slot_run_, tree_base_, bfit_, bvals_, bhits_, n_cases);
    GK(cudaGetLastError());
    finish_kernel<<<1, 256, 0, s>>>(ctl, runs_dev, slot_run_, w.cap_slots ? w.fz_redo : nullptr);
    GK(cudaGetLastError());
    nl += 2;
    if (launches) *launches = nl;
    return GP_OK;
}

gp_status Engine::enqueue(uint32_t mode, const std::vector<uint32_t> &runs, cudaStream_t s, bool sizing,
                          uint32_t *launches)
{
    gp_status st = write_head(mode, runs, s);
    if (st) return st;
    return enqueue_body(mode, s, sizing, launches);
}

// Kernel nodes at the top level of a graph (conditional bodies not included).
static uint32_t count_kernels(cudaGraph_t graph)
{
    size_t nn = 0;
    if (cudaGraphGetNodes(graph, nullptr, &nn) != cudaSuccess || nn == 0) return 0;
    std::vector<cudaGraphNode_t> nodes(nn);
    if (cudaGraphGetNodes(graph, nodes.data(), &nn) != cudaSuccess) return 0;
    uint32_t kernels = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++kernels;
    }
    return kernels;
}

gp_status Engine::capture(uint32_t mode)
{
    if (mode > 1) return GP_EINVAL;
    if (exec[mode]) {
        cudaGraphExecDestroy(exec[mode]);
        exec[mode] = nullptr;
    }
    cudaGraph_t graph = nullptr;
    GK(cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal));
    capturing_ = true;
    gp_status st = enqueue_body(mode, cap_stream, false, nullptr);
    capturing_ = false;
    cudaError_t e = cudaStreamEndCapture(cap_stream, &graph);
    if (st) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    GK(e);
    e = cudaGraphInstantiate(&exec[mode], graph, 0);
    const uint32_t top = count_kernels(graph);
    cudaGraphDestroy(graph);
    GK(e);
    // the branches hold one odd and one even level, or one rope launch
    kernels_fixed[mode] = top;
    kernels_per_batch[mode] = top + 2 * kernels_per_level + 1;
    return GP_OK;
}

gp_status Engine::launch_graph(uint32_t mode, const std::vector<uint32_t> &runs, cudaStream_t s)
{
    if (mode > 1 || !exec[mode]) return GP_EINVAL;
    gp_status st = write_head(mode, runs, s);
    if (st) return st;
    GK(cudaGraphLaunch(exec[mode], s));
    return GP_OK;
}

gp_status Engine::read_run(uint32_t r, RunDev *out, cudaStream_t s)
{
    if (r >= max_runs) return GP_EINVAL;
    GK(cudaMemcpyAsync(out, runs_dev + r, sizeof(RunDev), cudaMemcpyDeviceToHost, s));
    GK(cudaStreamSynchronize(s));
    return GP_OK;
}

gp_status Engine::read_ctl(BatchCtl *out, cudaStream_t s)
{
    GK(cudaMemcpyAsync(out, ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, s));
    GK(cudaStreamSynchronize(s));
    return GP_OK;
}

gp_status Engine::rewind(uint32_t r, cudaStream_t s)
{
    if (r >= max_runs) return GP_EINVAL;
    rewind_kernel<<<1, 1, 0, s>>>(runs_dev + r);
    GK(cudaGetLastError());
    return GP_OK;
}

gp_status Engine::copy_records(gp_xo *out, uint32_t first, uint32_t n)
{
    if ((uint64_t)first + n > max_trees) return GP_EINVAL;
    GK(cudaDeviceSynchronize());
    GK(cudaMemcpy(out, recs_ + first, sizeof(gp_xo) * n, cudaMemcpyDeviceToHost));
    return GP_OK;
}

gp_status Engine::copy_trees(const RunBuf &B, uint32_t n, uint64_t *offsets, uint8_t *nodes, uint64_t cap)
{
    std::vector<uint64_t> hs(n), hz(n);
    GK(cudaDeviceSynchronize());
    GK(cudaMemcpy(hs.data(), B.start, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost));
    GK(cudaMemcpy(hz.data(), B.size, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost));
    offsets[0] = 0;
    for (uint32_t t = 0; t < n; ++t) offsets[t + 1] = offsets[t] + hz[t];
    if (!nodes) return GP_OK;
    if (cap < offsets[n]) return GP_EINVAL;
    // the trees of a buffer are packed in order with 16-byte aligned starts:
    // one copy of the whole span, then close the gaps on the host
    const uint64_t span = n ? hs[n - 1] + hz[n - 1] - hs[0] : 0;
    std::vector<uint8_t> tmp(span);
    if (span) GK(cudaMemcpy(tmp.data(), heap + hs[0], span, cudaMemcpyDeviceToHost));
    for (uint32_t t = 0; t < n; ++t) std::memcpy(nodes + offsets[t], tmp.data() + (hs[t] - hs[0]), hz[t]);
    return GP_OK;
}

// One tree of a buffer: its size, and its bytes when `nodes` is given.
gp_status Engine::copy_tree(const RunBuf &B, uint32_t t, uint8_t *nodes, uint64_t cap, uint64_t *n_nodes)
{
    uint64_t start = 0, size = 0;
    GK(cudaDeviceSynchronize());
    GK(cudaMemcpy(&start, B.start + t, sizeof(uint64_t), cudaMemcpyDeviceToHost));
    GK(cudaMemcpy(&size, B.size + t, sizeof(uint64_t), cudaMemcpyDeviceToHost));
    if (nodes) {
        if (cap < size) return GP_EINVAL;
        if (size) GK(cudaMemcpy(nodes, heap + start, size, cudaMemcpyDeviceToHost));
    }
    *n_nodes = size;
    return GP_OK;
}

gp_status Engine::clear_error(uint32_t r, cudaStream_t s)
{
    if (r >= max_runs) return GP_EINVAL;
    GK(cudaMemsetAsync(&runs_dev[r].err, 0, sizeof(uint32_t), s));
    return GP_OK;
}

}  // namespace gpe
