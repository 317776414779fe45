// Generations on the device (Table gp.details: panmictic, non-elitist,
// generational, tournament size 7 for both parents; Sec. 3.1: two-parent
// subtree crossover with both points uniform over all nodes, chosen in a
// fixed sequential order).
//
// One generation is a fixed sequence of launches whose counts all live in a
// device control block: tournament selection and crossover points, subtree
// extents, child layout (a single-CTA scan), the segment copy, then the
// evaluation of the children through planned upper-tree levels (per level:
// item building, plan, scan, capacity check, evaluation).  Nothing returns
// to the host, so the sequence is captured once per buffer direction as a
// CUDA graph and replayed.  A failed step (node limit, a capacity) sets a
// sticky error bit; every later kernel sees it and does nothing, so the
// parents' buffer is left as it was.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "gp.h"
#include "gp_internal.cuh"

using namespace gpk;

namespace {

constexpr uint32_t kTile = 16384;        // copy tile (bytes)
constexpr uint32_t kScanT = 256;         // threads of the single-CTA scan kernels
constexpr uint32_t kBuckets = 40;        // final items ordered by floor(log2(size)), largest first

// Sticky error bits of a generation step.
constexpr uint32_t kGErrLimit = 1u;      // a child above the node limit (the run stops)
constexpr uint32_t kGErrArena = 2u;      // children larger than the population buffer
constexpr uint32_t kGErrWork = 4u;       // a level's codes / value entries above the workspace
constexpr uint32_t kGErrLevels = 8u;     // trees unfinished after the last level
constexpr uint32_t kGErrItems = 16u;     // more items than the item buffer holds
constexpr uint32_t kGErrEval = 32u;      // the evaluator reported an error (eval_err[0])
constexpr uint32_t kGErrExtent = 64u;    // a subtree extent ran off its tree
constexpr uint32_t kGErrSpill = 128u;    // oversized finals above the dedicated spill pool
constexpr uint32_t kGErrGen = 256u;      // generation counter past 2^24

struct Ctl {
    uint32_t gen;            // generation index of the current population
    uint32_t err;            // sticky kGErr* bits
    uint32_t err_gen;        // generation whose step raised the first error
    uint32_t n_queries;      // extent queries of this step
    uint32_t n_tiles;        // copy tiles of this step
    uint32_t n_items;        // evaluator items of the current level
    uint32_t n_chunks;       // fragment (planned) items of the current level
    uint32_t levels;         // levels used by the last evaluation
    uint32_t eval_err[4];    // [0] evaluator error word, [1] extent error word
    uint64_t totals[4];      // plan scan totals of the current level: codes, entries, max stack
    uint64_t child_bytes;    // arena bytes of the children
    uint64_t need_codes[2];  // largest level code count seen, per output buffer (sizing)
    uint64_t need_values[2]; // largest level value-entry count seen, per output buffer
    uint64_t need_dedicated; // largest dedicated spill (entries) a level asked for
    uint32_t counter[64];    // evaluator work counters, one per level
};

__device__ __forceinline__ void raise_err(Ctl *ctl, uint32_t bits)
{
    if (atomicOr(&ctl->err, bits) == 0) ctl->err_gen = ctl->gen;
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

__device__ uint32_t tournament(const float *__restrict__ fit, uint32_t n_pop, uint64_t seed, uint32_t g,
                               uint32_t c, uint32_t purpose, uint32_t size)
{
    uint32_t best = 0;
    float best_f = 0.0f;
    for (uint32_t k = 0; k < size; ++k) {
        const uint32_t e = (uint32_t)bounded(seed, draw_counter(g, c, purpose, k), n_pop);
        float f = fit[e];
        if (isnan(f)) f = __int_as_float(0x7f800000);     // NaN ranks with the worst
        if (k == 0 || f < best_f) {
            best = e;
            best_f = f;
        }
    }
    return best;
}

// ---- selection and child layout -----------------------------------------

__global__ void select_kernel(Ctl *ctl, const float *__restrict__ fit, const uint64_t *__restrict__ start,
                              const uint64_t *__restrict__ size, uint32_t n, uint64_t seed, uint32_t tsize,
                              gp_xo *__restrict__ recs, ExtentQuery *__restrict__ q)
{
    const uint32_t g = ctl->gen;
    const bool stop = ctl->err != 0 || g >= (1u << 24);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->n_queries = stop ? 0 : 2 * n;
        if (!ctl->err && g >= (1u << 24)) raise_err(ctl, kGErrGen);
    }
    if (stop) return;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        gp_xo r;
        r.mum = tournament(fit, n, seed, g, c, 0, tsize);
        r.dad = tournament(fit, n, seed, g, c, 1, tsize);
        r.mum_point = bounded(seed, draw_counter(g, c, 2, 0), size[r.mum]);
        r.dad_point = bounded(seed, draw_counter(g, c, 3, 0), size[r.dad]);
        recs[c] = r;
        q[2 * c] = ExtentQuery{start[r.mum], size[r.mum], r.mum_point};
        q[2 * c + 1] = ExtentQuery{start[r.dad], size[r.dad], r.dad_point};
    }
}

// Block-wide inclusive scan of two 64-bit values per thread (kScanT threads).
__device__ void block_scan2(uint64_t *sa, uint64_t *sb, uint64_t a, uint64_t b)
{
    const uint32_t t = threadIdx.x;
    sa[t] = a;
    sb[t] = b;
    __syncthreads();
    for (uint32_t off = 1; off < kScanT; off <<= 1) {
        uint64_t va = 0, vb = 0;
        if (t >= off) {
            va = sa[t - off];
            vb = sb[t - off];
        }
        __syncthreads();
        if (t >= off) {
            sa[t] += va;
            sb[t] += vb;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ uint64_t child_size(const gp_xo &r, const uint64_t *ends, uint32_t c,
                                               const uint64_t *psize)
{
    return r.mum_point + (ends[2 * c + 1] - r.dad_point) + (psize[r.mum] - ends[2 * c]);
}

// One CTA: child sizes (child = mum[0,i) ++ dad[j,e_d) ++ mum[e_m,n_m)),
// node limit, 16-byte aligned starts, copy tiles per child.
__global__ void __launch_bounds__(kScanT) children_kernel(
    Ctl *ctl, const gp_xo *__restrict__ recs, const uint64_t *__restrict__ ends,
    const uint64_t *__restrict__ pstart, const uint64_t *__restrict__ psize, uint32_t n,
    uint64_t max_nodes, uint64_t arena_cap, XoChild *__restrict__ kids, uint64_t *__restrict__ cstart,
    uint64_t *__restrict__ csize, uint32_t *__restrict__ tile_base)
{
    __shared__ uint64_t sa[kScanT], sb[kScanT];
    __shared__ uint32_t s_bad;
    const uint32_t t = threadIdx.x;
    if (t == 0) s_bad = 0;
    __syncthreads();
    if (ctl->err != 0 || ctl->n_queries == 0) {
        if (t == 0) ctl->n_tiles = 0;
        return;
    }
    const uint32_t per = (n + kScanT - 1) / kScanT;
    const uint32_t lo = min(t * per, n), hi = min(lo + per, n);
    uint64_t a = 0, b = 0;
    uint32_t bad = 0;
    for (uint32_t c = lo; c < hi; ++c) {
        const uint64_t m = child_size(recs[c], ends, c, psize);
        if (max_nodes && m > max_nodes) bad |= kGErrLimit;
        a += (m + 15) & ~15ull;
        b += (m + kTile - 1) / kTile;
    }
    if (bad) atomicOr(&s_bad, bad);
    block_scan2(sa, sb, a, b);
    const uint64_t tot_a = sa[kScanT - 1], tot_b = sb[kScanT - 1];
    uint32_t err = s_bad | (ctl->eval_err[1] ? kGErrExtent : 0u);
    if (tot_a + 64 > arena_cap || tot_b >= 0xffffffffull) err |= kGErrArena;
    if (err) {
        if (t == 0) {
            ctl->n_tiles = 0;
            raise_err(ctl, err);
        }
        return;
    }
    uint64_t ra = sa[t] - a, rb = sb[t] - b;
    for (uint32_t c = lo; c < hi; ++c) {
        const gp_xo r = recs[c];
        const uint64_t m = child_size(r, ends, c, psize);
        const uint64_t em = ends[2 * c], ed = ends[2 * c + 1];
        XoChild k;
        k.dst = ra;
        k.n = m;
        k.head_src = pstart[r.mum];
        k.i = r.mum_point;
        k.mid_src = pstart[r.dad] + r.dad_point;
        k.ld = ed - r.dad_point;
        k.tail_src = pstart[r.mum] + em;     // tail byte p comes from mum[em + p - i - ld]
        k.pad = 0;
        kids[c] = k;
        cstart[c] = ra;
        csize[c] = m;
        tile_base[c] = (uint32_t)rb;
        ra += (m + 15) & ~15ull;
        rb += (m + kTile - 1) / kTile;
    }
    if (t == kScanT - 1) {
        tile_base[n] = (uint32_t)tot_b;
        ctl->n_tiles = (uint32_t)tot_b;
        ctl->child_bytes = tot_a;
    }
}

// ---- evaluation levels ----------------------------------------------------

struct LevelArgs {
    uint32_t level;
    uint32_t n_trees;
    uint32_t C;                   // chunk (codes)
    uint32_t cap_items;
    uint64_t spill_base;          // first dedicated spill entry (after the per-warp areas)
    uint64_t cap_dedicated;       // dedicated spill entries available
};

__device__ __forceinline__ uint32_t size_bucket(uint64_t len)
{
    const uint32_t b = 63u - (uint32_t)__clzll(len | 1ull);
    return min(b, kBuckets - 1);
}

// One CTA.  Level 0: every tree of the population (start/size); a tree of at
// most C nodes is one final item, a larger one is cut into chunks of C.
// Level k > 0: every tree that had chunks at level k-1 now has an upper
// tree of codes [frag_off[first chunk], frag_off[one past its last chunk]);
// it becomes a final item when it fits one chunk or did not at least halve
// (a final above C gets a dedicated spill area), otherwise it is cut again.
// Chunk items come first in tree order (their fragments must be contiguous
// per tree), then finals from the largest size bucket down.
__global__ void __launch_bounds__(kScanT) items_kernel(
    Ctl *ctl, LevelArgs A, const uint64_t *__restrict__ start, const uint64_t *__restrict__ size,
    const uint64_t *__restrict__ frag_off, uint64_t *__restrict__ t_lo, uint64_t *__restrict__ t_hi,
    uint64_t *__restrict__ t_prev, uint32_t *__restrict__ t_first, uint32_t *__restrict__ t_state,
    EvalItem *__restrict__ items)
{
    __shared__ uint32_t s_cnt[kBuckets][kScanT];
    __shared__ uint64_t sa[kScanT], sb[kScanT];
    __shared__ uint64_t s_base[kBuckets];
    __shared__ uint32_t s_err;
    const uint32_t t = threadIdx.x;
    const uint32_t n = A.n_trees, C = A.C;
    if (ctl->err != 0) {
        if (t == 0) ctl->n_items = ctl->n_chunks = 0;
        return;
    }
    for (uint32_t b = 0; b < kBuckets; ++b) s_cnt[b][t] = 0;
    const uint32_t per = (n + kScanT - 1) / kScanT;
    const uint32_t lo = min(t * per, n), hi = min(lo + per, n);

    // phase 1: this level's range of every open tree (all reads of the old
    // t_first happen before the barrier; phase 3 rewrites it)
    for (uint32_t i = lo; i < hi; ++i) {
        if (A.level == 0) {
            t_lo[i] = start[i];
            t_hi[i] = start[i] + size[i];
            t_prev[i] = ~0ull;
            t_state[i] = 1;
        } else if (t_state[i]) {
            t_lo[i] = frag_off[t_first[i]];
            t_hi[i] = frag_off[t_first[i + 1]];
        }
    }
    __syncthreads();
    // phase 2: chunks, dedicated spill and finals per size bucket
    uint64_t nch = 0, ded = 0;
    for (uint32_t i = lo; i < hi; ++i) {
        if (!t_state[i]) continue;
        const uint64_t len = t_hi[i] - t_lo[i];
        if (len <= C || 2 * len > t_prev[i]) {
            ++s_cnt[size_bucket(len)][t];
            if (len > C) ded += len;
        } else {
            nch += (len + C - 1) / C;
        }
    }
    block_scan2(sa, sb, nch, ded);
    uint64_t ex_ch = sa[t] - nch, ex_ded = sb[t] - ded;
    const uint64_t tot_ch = sa[kScanT - 1], tot_ded = sb[kScanT - 1];
    if (t < kBuckets) {                       // per bucket: exclusive prefix over threads
        uint32_t run = 0;
        for (uint32_t j = 0; j < kScanT; ++j) {
            const uint32_t v = s_cnt[t][j];
            s_cnt[t][j] = run;
            run += v;
        }
        s_base[t] = run;                      // bucket total for now
    }
    __syncthreads();
    if (t == 0) {
        uint64_t pos = tot_ch;
        for (int b = (int)kBuckets - 1; b >= 0; --b) {
            const uint64_t cnt = s_base[b];
            s_base[b] = pos;
            pos += cnt;
        }
        uint32_t err = 0;
        ctl->need_dedicated = max(ctl->need_dedicated, tot_ded);
        if (pos > A.cap_items) err |= kGErrItems;
        if (tot_ded > A.cap_dedicated) err |= kGErrSpill;
        if (err) {
            raise_err(ctl, err);
            ctl->n_items = ctl->n_chunks = 0;
        } else {
            ctl->n_items = (uint32_t)pos;
            ctl->n_chunks = (uint32_t)tot_ch;
            if (pos) ctl->levels = A.level + 1;
        }
        s_err = err;
    }
    __syncthreads();
    if (s_err) return;
    // phase 3: chunk offsets per tree, final items, states
    for (uint32_t i = lo; i < hi; ++i) {
        t_first[i] = (uint32_t)ex_ch;
        if (!t_state[i]) continue;
        const uint64_t len = t_hi[i] - t_lo[i];
        if (len <= C || 2 * len > t_prev[i]) {
            const uint32_t b = size_bucket(len);
            EvalItem it{};
            it.begin = t_lo[i];
            it.end = t_hi[i];
            it.tree = i;
            it.flags = kItemFinal;
            it.spill_off = kNoSpill;
            if (len > C) {
                it.spill_off = A.spill_base + ex_ded;
                it.spill_cap = len;
                ex_ded += len;
            }
            items[s_base[b] + s_cnt[b][t]++] = it;
            t_state[i] = 0;
        } else {
            t_prev[i] = len;
            ex_ch += (len + C - 1) / C;
        }
    }
    if (t == kScanT - 1) t_first[n] = (uint32_t)tot_ch;
}

// Chunk items: item i belongs to the last tree whose first chunk is <= i.
__global__ void fill_chunks_kernel(const Ctl *ctl, uint32_t n_trees, uint32_t C,
                                   const uint32_t *__restrict__ t_first, const uint64_t *__restrict__ t_lo,
                                   const uint64_t *__restrict__ t_hi, EvalItem *__restrict__ items)
{
    const uint32_t n = ctl->n_chunks;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = n_trees;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (t_first[mid] <= i) lo = mid;
            else hi = mid;
        }
        EvalItem it{};
        it.begin = t_lo[lo] + (uint64_t)(i - t_first[lo]) * C;
        it.end = umin64(t_hi[lo], it.begin + C);
        it.tree = lo;
        it.flags = 0;
        it.spill_off = kNoSpill;
        items[i] = it;
    }
}

// After a level's plan scan: the level's upper-tree codes and value entries
// must fit the workspace; the code array is zero-padded past its end (the
// evaluator reads whole 16-code groups).
__global__ void check_kernel(Ctl *ctl, uint64_t cap_codes, uint64_t cap_values, uint32_t *__restrict__ u_out,
                             uint32_t idx)
{
    __shared__ uint32_t s_ok;
    const uint64_t codes = ctl->totals[0], vals = ctl->totals[1];
    if (threadIdx.x == 0) {
        s_ok = 0;
        if (ctl->err == 0) {
            if (codes + 48 > cap_codes || vals > cap_values || vals + kPtCode0 >= 0xffffffffull) {
                raise_err(ctl, kGErrWork);
                ctl->n_items = 0;
            } else {
                s_ok = 1;
                ctl->need_codes[idx] = max(ctl->need_codes[idx], codes);
                ctl->need_values[idx] = max(ctl->need_values[idx], vals);
            }
        } else {
            ctl->n_items = 0;
        }
    }
    __syncthreads();
    if (!s_ok) return;
    const uint64_t end = ((codes + 15) & ~15ull) + 32;
    for (uint64_t i = codes + threadIdx.x; i < end; i += blockDim.x) u_out[i] = 0;
}

// End of a generation: evaluator errors become a step error; without one
// the generation counter advances (when this sequence made a generation).
__global__ void finish_kernel(Ctl *ctl, uint32_t advance)
{
    if (ctl->err == 0) {
        if (ctl->eval_err[0]) raise_err(ctl, kGErrEval);
        else if (ctl->n_chunks) raise_err(ctl, kGErrLevels);
    }
    if (ctl->err == 0 && advance) ctl->gen += 1;
}

__global__ void rewind_kernel(Ctl *ctl)
{
    if (ctl->err == 0 && ctl->gen > 0) ctl->gen -= 1;
}

// ---- host side --------------------------------------------------------------

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

int lanes_of(uint32_t n_cases)
{
    return n_cases <= 16 ? 8 : n_cases <= 32 ? 16 : n_cases <= 48 ? 24 : 32;
}

struct GenBuf {
    uint8_t *arena = nullptr;
    uint64_t *start = nullptr, *size = nullptr;
    float *fit = nullptr, *vals = nullptr;
    uint32_t *hits = nullptr;
};

struct Work {                        // per-chunk-size evaluator workspace
    uint32_t C = 0;
    // Level k writes buffer k & 1: level 0 (the largest) alone fills buffer
    // 0's need in practice, so the two are sized separately.
    uint64_t cap_codes[2] = {0, 0}, cap_values[2] = {0, 0};
    uint64_t cap_items = 0, cap_dedicated = 0;
    EvalItem *items = nullptr;
    PlanOut *plan = nullptr;
    uint64_t *frag_off = nullptr;
    uint32_t *codes[2] = {nullptr, nullptr};
    float2 *vals[2] = {nullptr, nullptr};
    float2 *spill = nullptr;
    uint64_t spill_per_warp = 0, spill_base = 0;
};

}  // namespace

struct gp_generation {
    int device = 0, sms = 0, lanes = 0;
    uint32_t n_cases = 0, n_consts = 0, n = 0, tsize = 7, levels_max = 8;
    float div0 = 1.0f;
    uint64_t seed = 0, max_nodes = 0, cap_arena = 0;
    uint32_t W = 32, K = 32, Wu = 16, Ku = 96;
    size_t smem = 0, smem_u = 0;
    bool use_graph = false;
    std::vector<void *> allocs;        // everything but the workspace
    std::vector<void *> work_allocs;   // the workspace
    GenBuf buf[2];
    Ctl *ctl = nullptr;
    gp_xo *recs = nullptr;
    ExtentQuery *q = nullptr;
    uint64_t *ends = nullptr;
    XoChild *kids = nullptr;
    uint32_t *tile_base = nullptr;
    uint64_t *t_lo = nullptr, *t_hi = nullptr, *t_prev = nullptr;
    uint32_t *t_first = nullptr, *t_state = nullptr;
    float *x = nullptr, *y = nullptr, *c = nullptr;
    Work w;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    uint32_t kernels_per_gen = 0;
    uint32_t cur = 0;                  // buffer of the current population (host view)
    uint64_t issued = 0;               // generations issued since creation
    cudaStream_t last = nullptr;       // stream of the last enqueue (may be the legacy
                                       // default stream, whose handle is null)
    gp_generation_info info{};
};

namespace {

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

// Workspace for chunk size C with the given capacities.
gp_status alloc_work(gp_generation *G, uint32_t C, const uint64_t cap_codes[2], const uint64_t cap_values[2],
                     uint64_t cap_dedicated)
{
    cudaDeviceSynchronize();
    gfree(G->work_allocs);
    Work &w = G->w;
    w = Work{};
    w.C = C;
    for (int k = 0; k < 2; ++k) {
        w.cap_codes[k] = cap_codes[k];
        w.cap_values[k] = cap_values[k];
    }
    w.cap_items = G->cap_arena / C + 2ull * G->n + 1024;
    w.cap_dedicated = cap_dedicated;
    if (w.cap_items > 0xffffffffull) return GP_ENOMEM;
    const uint64_t warps = (uint64_t)G->sms * std::max(G->W, G->Wu);
    w.spill_per_warp = C;
    w.spill_base = warps * C;
    auto &v = G->work_allocs;
    gp_status st;
    if ((st = galloc(v, (void **)&w.items, sizeof(EvalItem) * w.cap_items))) return st;
    if ((st = galloc(v, (void **)&w.plan, sizeof(PlanOut) * w.cap_items))) return st;
    if ((st = galloc(v, (void **)&w.frag_off, sizeof(uint64_t) * (w.cap_items + 1)))) return st;
    for (int k = 0; k < 2; ++k) {
        if ((st = galloc(v, (void **)&w.codes[k], sizeof(uint32_t) * (cap_codes[k] + 64)))) return st;
        if ((st = galloc(v, (void **)&w.vals[k], sizeof(float2) * (cap_values[k] * G->lanes + 1)))) return st;
    }
    if ((st = galloc(v, (void **)&w.spill, sizeof(float2) * G->lanes * (w.spill_base + w.cap_dedicated)))) return st;
    return GP_OK;
}

// Enqueue the evaluation of the population in buffer `b` (level by level).
// With `sizing`, the host reads each level's totals and grows the workspace
// when they do not fit (used before any capture).
gp_status enqueue_eval(gp_generation *G, int b, bool sizing, cudaStream_t s, uint32_t *launches)
{
    Work &w = G->w;
    const GenBuf &B = G->buf[b];
    uint32_t nl = 0;
    for (uint32_t level = 0; level < G->levels_max; ++level) {
        const bool wide = level > 0;
        LevelArgs A{level, G->n, w.C, (uint32_t)std::min<uint64_t>(w.cap_items, 0xffffffffu), w.spill_base,
                    w.cap_dedicated};
        items_kernel<<<1, kScanT, 0, s>>>(G->ctl, A, B.start, B.size, w.frag_off, G->t_lo, G->t_hi,
                                          G->t_prev, G->t_first, G->t_state, w.items);
        GK(cudaGetLastError());
        if (sizing) {
            // a dedicated spill pool too small for this level's oversized
            // finals: grow it, clear the error and build the level again
            // (the kernel changes nothing else when it raises this error)
            Ctl c{};
            GK(cudaMemcpyAsync(&c, G->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
            GK(cudaStreamSynchronize(s));
            if (c.err == kGErrSpill) {
                const uint64_t nd = std::max<uint64_t>(2 * c.need_dedicated, w.cap_dedicated);
                void *p = nullptr;
                GK(cudaMalloc(&p, sizeof(float2) * G->lanes * (w.spill_base + nd)));
                G->work_allocs.push_back(p);
                w.spill = (float2 *)p;
                w.cap_dedicated = nd;
                A.cap_dedicated = nd;
                GK(cudaMemsetAsync(&G->ctl->err, 0, sizeof(uint32_t), s));
                items_kernel<<<1, kScanT, 0, s>>>(G->ctl, A, B.start, B.size, w.frag_off, G->t_lo, G->t_hi,
                                                  G->t_prev, G->t_first, G->t_state, w.items);
                GK(cudaGetLastError());
            }
        }
        fill_chunks_kernel<<<G->sms * 4, 256, 0, s>>>(G->ctl, G->n, w.C, G->t_first, G->t_lo, G->t_hi,
                                                      w.items);
        GK(cudaGetLastError());
        const void *codes = wide ? (const void *)w.codes[(level - 1) & 1] : (const void *)B.arena;
        GK(launch_plan_dev(wide, codes, w.items, (uint32_t)w.cap_items, &G->ctl->n_chunks, w.plan, G->sms, s));
        GK(launch_plan_scan_dev(w.items, w.plan, &G->ctl->n_chunks, w.frag_off, G->ctl->totals, s));
        nl += 4;
        if (sizing) {
            uint64_t tot[2];
            uint32_t err = 0, n_items = 0;
            GK(cudaMemcpyAsync(tot, G->ctl->totals, sizeof(tot), cudaMemcpyDeviceToHost, s));
            GK(cudaMemcpyAsync(&err, &G->ctl->err, sizeof(err), cudaMemcpyDeviceToHost, s));
            GK(cudaMemcpyAsync(&n_items, &G->ctl->n_items, sizeof(n_items), cudaMemcpyDeviceToHost, s));
            GK(cudaStreamSynchronize(s));
            if (err) break;
            if (n_items == 0) break;
            const int k = level & 1;
            if (tot[0] + 48 > w.cap_codes[k] || tot[1] > w.cap_values[k]) {
                // grow this level's output buffers; they hold nothing still
                // needed (the outputs of level - 2)
                const uint64_t nc = std::max<uint64_t>(w.cap_codes[k], tot[0] + tot[0] / 8 + 1024);
                const uint64_t nv = std::max<uint64_t>(w.cap_values[k], tot[1] + tot[1] / 8 + 1024);
                void *pc = nullptr, *pv = nullptr;
                GK(cudaMalloc(&pc, sizeof(uint32_t) * (nc + 64)));
                G->work_allocs.push_back(pc);
                GK(cudaMalloc(&pv, sizeof(float2) * (nv * G->lanes + 1)));
                G->work_allocs.push_back(pv);
                w.codes[k] = (uint32_t *)pc;
                w.vals[k] = (float2 *)pv;
                w.cap_codes[k] = nc;
                w.cap_values[k] = nv;
            }
        }
        check_kernel<<<1, 64, 0, s>>>(G->ctl, w.cap_codes[level & 1], w.cap_values[level & 1],
                                      w.codes[level & 1], level & 1);
        GK(cudaGetLastError());
        EvalParams p{};
        p.codes = codes;
        p.items = w.items;
        p.n_items = (uint32_t)std::min<uint64_t>(w.cap_items, 0xffffffffu);
        p.n_items_dev = &G->ctl->n_items;
        p.counter = &G->ctl->counter[level];
        p.x = G->x;
        p.y = G->y;
        p.consts = G->c;
        p.n_cases = G->n_cases;
        p.n_consts = G->n_consts;
        p.div0 = G->div0;
        p.window = wide ? G->Ku : G->K;
        p.pt_in = wide ? w.vals[(level - 1) & 1] : nullptr;
        p.pt_out = w.vals[level & 1];
        p.u_out = w.codes[level & 1];
        p.values = B.vals;
        p.fitness = B.fit;
        p.hits = B.hits;
        p.spill = w.spill;
        p.spill_per_warp = w.spill_per_warp;
        p.err = &G->ctl->eval_err[0];
        GK(launch_eval(G->lanes, wide, p, G->sms, (int)(wide ? G->Wu : G->W), wide ? G->smem_u : G->smem, s));
        nl += 2;
    }
    if (launches) *launches += nl;
    return GP_OK;
}

// Enqueue one generation: parents in buffer `p`, children into buffer 1-p.
gp_status enqueue_step(gp_generation *G, int p, cudaStream_t s, uint32_t *launches)
{
    const GenBuf &P = G->buf[p], &Cb = G->buf[p ^ 1];
    GK(cudaMemsetAsync(G->ctl->counter, 0, sizeof(G->ctl->counter), s));
    GK(cudaMemsetAsync(G->ctl->eval_err, 0, sizeof(G->ctl->eval_err), s));
    const uint32_t blocks = std::max<uint32_t>(1, std::min<uint32_t>((G->n + 127) / 128, G->sms * 8));
    select_kernel<<<blocks, 128, 0, s>>>(G->ctl, P.fit, P.start, P.size, G->n, G->seed, G->tsize, G->recs, G->q);
    GK(cudaGetLastError());
    GK(launch_extent_dev(P.arena, G->q, 2 * G->n, &G->ctl->n_queries, G->ends, &G->ctl->eval_err[1], G->sms, s));
    children_kernel<<<1, kScanT, 0, s>>>(G->ctl, G->recs, G->ends, P.start, P.size, G->n, G->max_nodes,
                                         G->cap_arena, G->kids, Cb.start, Cb.size, G->tile_base);
    GK(cudaGetLastError());
    GK(launch_xo_copy_dev(P.arena, Cb.arena, G->kids, G->tile_base, G->n, &G->ctl->n_tiles, kTile, G->sms, s));
    uint32_t nl = 4;
    gp_status st = enqueue_eval(G, p ^ 1, false, s, &nl);
    if (st) return st;
    finish_kernel<<<1, 1, 0, s>>>(G->ctl, 1u);
    GK(cudaGetLastError());
    nl += 1;
    if (launches) *launches = nl;
    return GP_OK;
}

gp_status eval_initial(gp_generation *G, bool sizing, cudaStream_t s)
{
    GK(cudaMemsetAsync(G->ctl->counter, 0, sizeof(G->ctl->counter), s));
    GK(cudaMemsetAsync(G->ctl->eval_err, 0, sizeof(G->ctl->eval_err), s));
    gp_status st = enqueue_eval(G, 0, sizing, s, nullptr);
    if (st) return st;
    finish_kernel<<<1, 1, 0, s>>>(G->ctl, 0u);
    GK(cudaGetLastError());
    return GP_OK;
}

gp_status read_ctl(gp_generation *G, Ctl *out, cudaStream_t s)
{
    GK(cudaMemcpyAsync(out, G->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    GK(cudaStreamSynchronize(s));
    return GP_OK;
}

gp_status map_err(const Ctl &c)
{
    if (!c.err) return GP_OK;
    if (c.err & (kGErrLimit | kGErrGen)) return GP_ELIMIT;
    if (c.err & (kGErrArena | kGErrWork | kGErrItems | kGErrSpill | kGErrLevels)) return GP_ENOMEM;
    if (c.err & kGErrExtent) return GP_EMALFORMED;
    if (c.err & kGErrEval) return (c.eval_err[0] & kErrMalformed) ? GP_EMALFORMED : GP_ECUDA;
    return GP_ECUDA;
}

// Bring the host's view (current buffer, generation) in line with the device
// after a synchronisation.
gp_status sync_state(gp_generation *G, Ctl *c)
{
    gp_status st = read_ctl(G, c, G->last);
    if (st) return st;
    G->cur = c->gen & 1u;
    G->issued = c->gen;
    G->info.generation = c->gen;
    G->info.levels = c->levels;
    G->info.error_generation = c->err ? c->err_gen : 0;
    return GP_OK;
}

float time_initial_eval(gp_generation *G, cudaStream_t s)
{
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
    gp_status st = eval_initial(G, false, s);
    cudaEventRecord(b, s);
    float ms = -1.0f;
    if (!st && cudaEventSynchronize(b) == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return st ? -1.0f : ms;
}

gp_status capture_graphs(gp_generation *G)
{
    for (int p = 0; p < 2; ++p) {
        cudaGraph_t graph = nullptr;
        GK(cudaStreamBeginCapture(G->cap_stream, cudaStreamCaptureModeThreadLocal));
        uint32_t nl = 0;
        gp_status st = enqueue_step(G, p, G->cap_stream, &nl);
        cudaError_t e = cudaStreamEndCapture(G->cap_stream, &graph);
        if (st) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        GK(e);
        e = cudaGraphInstantiate(&G->exec[p], graph, 0);
        size_t nn = 0;
        cudaGraphGetNodes(graph, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        uint32_t kernels = 0;
        if (nn && cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess) {
            for (auto nd : nodes) {
                cudaGraphNodeType ty;
                if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++kernels;
            }
        }
        cudaGraphDestroy(graph);
        GK(e);
        G->kernels_per_gen = kernels;
    }
    return GP_OK;
}

void destroy_gen(gp_generation *G)
{
    if (!G) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(G->device);
    cudaDeviceSynchronize();
    for (auto &e : G->exec)
        if (e) cudaGraphExecDestroy(e);
    gfree(G->work_allocs);
    gfree(G->allocs);
    if (G->cap_stream) cudaStreamDestroy(G->cap_stream);
    cudaSetDevice(cur);
    delete G;
}

// Work enqueued on s runs after everything enqueued on the previous stream.
void order_after_last(gp_generation *G, cudaStream_t s)
{
    if (G->last == s) return;
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(e, G->last);
        cudaStreamWaitEvent(s, e, 0);
        cudaEventDestroy(e);
    }
}

}  // namespace

extern "C" {

gp_status gp_generation_create(const gp_problem *problem, const gp_generation_params *params,
                               uint32_t n_trees, const uint8_t *nodes, const uint64_t *offsets,
                               void *cuda_stream, gp_generation **out)
{
    if (!problem || !params || !out || n_trees == 0 || n_trees > (1u << 28)) return GP_EINVAL;
    if (params->tournament_size < 1 || params->tournament_size > 32) return GP_EINVAL;
    if (params->chunk_nodes && (params->chunk_nodes % 16 || params->chunk_nodes < 256 ||
                                params->chunk_nodes > 65536))
        return GP_EINVAL;
    if (params->max_levels && (params->max_levels < 2 || params->max_levels > 16)) return GP_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    // upload and validate through the population API, then take its layout
    gp_population *init = nullptr;
    gp_status st = gp_create_population(problem, n_trees, nodes, offsets, cuda_stream, &init);
    if (st) return st;
    gp_population_info pi{};
    gp_population_get_info(init, &pi);

    gp_generation *G = new (std::nothrow) gp_generation();
    if (!G) {
        gp_destroy_population(init);
        return GP_ENOMEM;
    }
    auto fail = [&](gp_status e) {
        gp_destroy_population(init);
        destroy_gen(G);
        return e;
    };
    cudaGetDevice(&G->device);
    cudaDeviceGetAttribute(&G->sms, cudaDevAttrMultiProcessorCount, G->device);
    G->n = n_trees;
    G->n_cases = problem->n_cases;
    G->n_consts = problem->n_consts;
    G->lanes = lanes_of(problem->n_cases);
    G->div0 = problem->protected_div_value;
    G->max_nodes = problem->max_tree_nodes;
    G->seed = params->seed;
    G->tsize = params->tournament_size;
    G->levels_max = params->max_levels ? params->max_levels : 8;
    G->use_graph = params->use_graph != 0;
    if (cudaStreamCreateWithFlags(&G->cap_stream, cudaStreamNonBlocking) != cudaSuccess) return fail(GP_ECUDA);

    // launch shape as in gp_evaluate
    int maxsm = 0;
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, G->device);
    while (G->W > 1 && eval_smem_bytes(G->lanes, (int)G->W, (int)G->K, false) > (size_t)maxsm) --G->W;
    G->Wu = std::min<uint32_t>(G->W, 16);
    while (G->Wu > 1 && eval_smem_bytes(G->lanes, (int)G->Wu, (int)G->Ku, true) > (size_t)maxsm) --G->Wu;
    G->smem = eval_smem_bytes(G->lanes, (int)G->W, (int)G->K, false);
    G->smem_u = eval_smem_bytes(G->lanes, (int)G->Wu, (int)G->Ku, true);
    if (G->smem > (size_t)maxsm || G->smem_u > (size_t)maxsm) return fail(GP_EINVAL);
    if (eval_prepare_at_least(G->lanes, false, G->smem) != cudaSuccess ||
        eval_prepare_at_least(G->lanes, true, G->smem_u) != cudaSuccess)
        return fail(GP_ECUDA);

    // population buffers
    std::vector<uint64_t> hstart(n_trees), hsize(n_trees);
    uint64_t pos = 0;
    for (uint32_t t = 0; t < n_trees; ++t) {
        hsize[t] = offsets[t + 1] - offsets[t];
        hstart[t] = pos;
        pos = (pos + hsize[t] + 15) & ~15ull;
    }
    const uint64_t used = pos + 64;
    G->cap_arena = params->arena_bytes ? params->arena_bytes : 2 * used + 16ull * n_trees + (1u << 20);
    if (G->cap_arena < used) return fail(GP_ENOMEM);
    auto &v = G->allocs;
    for (int b = 0; b < 2; ++b) {
        GenBuf &B = G->buf[b];
        if ((st = galloc(v, (void **)&B.arena, G->cap_arena))) return fail(st);
        if ((st = galloc(v, (void **)&B.start, sizeof(uint64_t) * (n_trees + 1)))) return fail(st);
        if ((st = galloc(v, (void **)&B.size, sizeof(uint64_t) * (n_trees + 1)))) return fail(st);
        if ((st = galloc(v, (void **)&B.fit, sizeof(float) * n_trees))) return fail(st);
        if ((st = galloc(v, (void **)&B.vals, sizeof(float) * (uint64_t)n_trees * G->n_cases))) return fail(st);
        if ((st = galloc(v, (void **)&B.hits, sizeof(uint32_t) * n_trees))) return fail(st);
    }
    if ((st = galloc(v, (void **)&G->ctl, sizeof(Ctl)))) return fail(st);
    if ((st = galloc(v, (void **)&G->recs, sizeof(gp_xo) * n_trees))) return fail(st);
    if ((st = galloc(v, (void **)&G->q, sizeof(ExtentQuery) * 2 * n_trees))) return fail(st);
    if ((st = galloc(v, (void **)&G->ends, sizeof(uint64_t) * 2 * n_trees))) return fail(st);
    if ((st = galloc(v, (void **)&G->kids, sizeof(XoChild) * n_trees))) return fail(st);
    if ((st = galloc(v, (void **)&G->tile_base, sizeof(uint32_t) * (n_trees + 1)))) return fail(st);
    if ((st = galloc(v, (void **)&G->t_lo, sizeof(uint64_t) * n_trees))) return fail(st);
    if ((st = galloc(v, (void **)&G->t_hi, sizeof(uint64_t) * n_trees))) return fail(st);
    if ((st = galloc(v, (void **)&G->t_prev, sizeof(uint64_t) * n_trees))) return fail(st);
    if ((st = galloc(v, (void **)&G->t_first, sizeof(uint32_t) * (n_trees + 1)))) return fail(st);
    if ((st = galloc(v, (void **)&G->t_state, sizeof(uint32_t) * n_trees))) return fail(st);
    if ((st = galloc(v, (void **)&G->x, sizeof(float) * 2 * G->lanes))) return fail(st);
    if ((st = galloc(v, (void **)&G->y, sizeof(float) * 2 * G->lanes))) return fail(st);
    if ((st = galloc(v, (void **)&G->c, sizeof(float) * (G->n_consts + 1)))) return fail(st);
    {
        std::vector<float> hx(2 * G->lanes, 0.f), hy(2 * G->lanes, 0.f);
        std::memcpy(hx.data(), problem->x, sizeof(float) * G->n_cases);
        std::memcpy(hy.data(), problem->y, sizeof(float) * G->n_cases);
        if (cudaMemcpy(G->x, hx.data(), sizeof(float) * hx.size(), cudaMemcpyHostToDevice) ||
            cudaMemcpy(G->y, hy.data(), sizeof(float) * hy.size(), cudaMemcpyHostToDevice) ||
            (G->n_consts && cudaMemcpy(G->c, problem->consts, sizeof(float) * G->n_consts,
                                       cudaMemcpyHostToDevice)))
            return fail(GP_ECUDA);
    }
    // the initial population: same 16-byte aligned layout as the upload
    if (cudaStreamSynchronize(s) != cudaSuccess ||
        cudaMemcpy(G->buf[0].arena, pi.d_nodes, pos + 64, cudaMemcpyDeviceToDevice) != cudaSuccess ||
        cudaMemcpy(G->buf[0].start, hstart.data(), sizeof(uint64_t) * n_trees, cudaMemcpyHostToDevice) ||
        cudaMemcpy(G->buf[0].size, hsize.data(), sizeof(uint64_t) * n_trees, cudaMemcpyHostToDevice) ||
        cudaMemset(G->ctl, 0, sizeof(Ctl)) != cudaSuccess)
        return fail(GP_ECUDA);
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(GP_ECUDA);
    gp_destroy_population(init);
    init = nullptr;
    auto fail2 = [&](gp_status e) {
        destroy_gen(G);
        return e;
    };

    // chunk size: the given one, or the fastest candidate on generation 0
    const uint32_t cands[4] = {1024, 2048, 4096, 8192};
    std::vector<uint32_t> tries;
    if (params->chunk_nodes) tries.push_back(params->chunk_nodes);
    else tries.assign(cands, cands + 4);
    uint32_t best_C = 0;
    float best_ms = 0.f;
    uint64_t best_codes[2] = {0, 0}, best_vals[2] = {0, 0}, best_ded = 0;
    cudaStream_t cs = G->cap_stream;
    for (size_t k = 0; k < tries.size(); ++k) {
        const uint32_t C = tries[k];
        const uint64_t c0[2] = {1u << 20, 1u << 20}, v0[2] = {1u << 18, 1u << 18};
        if ((st = alloc_work(G, C, c0, v0, 1u << 16))) return fail2(st);
        Ctl c{};
        if (cudaMemsetAsync(G->ctl, 0, sizeof(Ctl), cs) != cudaSuccess) return fail2(GP_ECUDA);
        if ((st = eval_initial(G, true, cs))) return fail2(st);      // sizing pass
        if ((st = read_ctl(G, &c, cs))) return fail2(st);
        if (c.err) return fail2(map_err(c));
        const uint64_t need_d = c.need_dedicated;
        float ms = -1.f;
        for (int rep = 0; rep < 2; ++rep) {                          // timed, device only
            cudaMemsetAsync(G->ctl, 0, sizeof(Ctl), cs);
            ms = time_initial_eval(G, cs);
        }
        if (ms < 0.f) return fail2(GP_ECUDA);
        if ((st = read_ctl(G, &c, cs))) return fail2(st);
        if (c.err) return fail2(map_err(c));
        if (k < 8) {
            G->info.autotune_chunk[k] = C;
            G->info.autotune_ms[k] = ms;
        }
        if (!best_C || ms < best_ms) {
            best_C = C;
            best_ms = ms;
            for (int k = 0; k < 2; ++k) {
                best_codes[k] = c.need_codes[k];
                best_vals[k] = c.need_values[k];
            }
            best_ded = need_d;
        }
    }
    // capacities: the measured need of generation 0 with a margin for the
    // growth of later generations
    uint64_t cap_codes[2], cap_vals[2];
    for (int k = 0; k < 2; ++k) {
        cap_codes[k] = params->workspace_codes ? params->workspace_codes
                                               : std::max<uint64_t>(best_codes[k] * 3 / 2 + 1024, 1u << 20);
        cap_vals[k] = params->workspace_values ? params->workspace_values
                                               : std::max<uint64_t>(best_vals[k] * 3 / 2 + 1024, 1u << 18);
    }
    const uint64_t cap_ded = std::max<uint64_t>(2 * best_ded, 1u << 20);
    if ((st = alloc_work(G, best_C, cap_codes, cap_vals, cap_ded))) return fail2(st);
    {
        Ctl c{};
        if (cudaMemsetAsync(G->ctl, 0, sizeof(Ctl), cs) != cudaSuccess) return fail2(GP_ECUDA);
        if ((st = eval_initial(G, false, cs))) return fail2(st);
        if ((st = read_ctl(G, &c, cs))) return fail2(st);
        if (c.err) return fail2(map_err(c));
        G->info.levels = c.levels;
    }
    if (G->use_graph && (st = capture_graphs(G))) return fail2(st);
    G->info.n_trees = n_trees;
    G->info.chunk_nodes = best_C;
    G->info.graph = G->use_graph ? 1u : 0u;
    G->info.kernels_per_generation = G->kernels_per_gen;
    G->info.arena_bytes = G->cap_arena;
    G->info.workspace_codes = G->w.cap_codes[0] + G->w.cap_codes[1];
    G->info.workspace_values = G->w.cap_values[0] + G->w.cap_values[1];
    G->last = cs;
    *out = G;
    return GP_OK;
}

gp_status gp_generation_step(gp_generation *G, uint32_t n, void *cuda_stream)
{
    if (!G) return GP_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != G->device) cudaSetDevice(G->device);
    order_after_last(G, s);
    gp_status st = GP_OK;
    for (uint32_t k = 0; k < n && !st; ++k) {
        uint32_t nl = 0;
        if (G->use_graph) {
            if (cudaGraphLaunch(G->exec[G->cur], s) != cudaSuccess) st = gfail(cudaGetLastError());
            nl = G->kernels_per_gen;
        } else {
            st = enqueue_step(G, (int)G->cur, s, &nl);
            G->kernels_per_gen = nl;
        }
        note_launches(nl);
        G->cur ^= 1u;
        ++G->issued;
    }
    G->last = s;
    if (dev != G->device) cudaSetDevice(dev);
    return st;
}

gp_status gp_generation_rewind(gp_generation *G, void *cuda_stream)
{
    if (!G || G->issued == 0) return GP_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    order_after_last(G, s);
    rewind_kernel<<<1, 1, 0, s>>>(G->ctl);
    GK(cudaGetLastError());
    G->cur ^= 1u;
    --G->issued;
    G->last = s;
    return GP_OK;
}

gp_status gp_generation_fitness(gp_generation *G, float *fitness, float *case_values, uint32_t *hits)
{
    if (!G) return GP_EINVAL;
    Ctl c{};
    gp_status st = sync_state(G, &c);
    if (st) return st;
    if ((st = map_err(c))) return st;
    const GenBuf &B = G->buf[G->cur];
    if (fitness) GK(cudaMemcpy(fitness, B.fit, sizeof(float) * G->n, cudaMemcpyDeviceToHost));
    if (case_values)
        GK(cudaMemcpy(case_values, B.vals, sizeof(float) * (uint64_t)G->n * G->n_cases, cudaMemcpyDeviceToHost));
    if (hits) GK(cudaMemcpy(hits, B.hits, sizeof(uint32_t) * G->n, cudaMemcpyDeviceToHost));
    return GP_OK;
}

gp_status gp_generation_records(gp_generation *G, gp_xo *records)
{
    if (!G || !records) return GP_EINVAL;
    Ctl c{};
    gp_status st = sync_state(G, &c);
    if (st) return st;
    if ((st = map_err(c))) return st;
    GK(cudaMemcpy(records, G->recs, sizeof(gp_xo) * G->n, cudaMemcpyDeviceToHost));
    return GP_OK;
}

gp_status gp_generation_trees(gp_generation *G, uint64_t *offsets, uint8_t *nodes, uint64_t cap)
{
    if (!G || !offsets) return GP_EINVAL;
    Ctl c{};
    gp_status st = sync_state(G, &c);
    if (st) return st;
    if ((st = map_err(c))) return st;
    const GenBuf &B = G->buf[G->cur];
    std::vector<uint64_t> hs(G->n), hz(G->n);
    GK(cudaMemcpy(hs.data(), B.start, sizeof(uint64_t) * G->n, cudaMemcpyDeviceToHost));
    GK(cudaMemcpy(hz.data(), B.size, sizeof(uint64_t) * G->n, cudaMemcpyDeviceToHost));
    offsets[0] = 0;
    for (uint32_t t = 0; t < G->n; ++t) offsets[t + 1] = offsets[t] + hz[t];
    if (!nodes) return GP_OK;
    if (cap < offsets[G->n]) return GP_EINVAL;
    for (uint32_t t = 0; t < G->n; ++t)
        GK(cudaMemcpy(nodes + offsets[t], B.arena + hs[t], hz[t], cudaMemcpyDeviceToHost));
    return GP_OK;
}

gp_status gp_generation_get_info(gp_generation *G, gp_generation_info *info)
{
    if (!G || !info) return GP_EINVAL;
    Ctl c{};
    gp_status st = sync_state(G, &c);
    if (st) return st;
    G->info.total_nodes = 0;
    if (!c.err) {
        std::vector<uint64_t> hz(G->n);
        GK(cudaMemcpy(hz.data(), G->buf[G->cur].size, sizeof(uint64_t) * G->n, cudaMemcpyDeviceToHost));
        for (uint64_t z : hz) G->info.total_nodes += z;
    }
    G->info.kernels_per_generation = G->kernels_per_gen;
    *info = G->info;
    return GP_OK;
}

void gp_generation_destroy(gp_generation *G) { destroy_gen(G); }

}  // extern "C"
