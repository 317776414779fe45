// Internal types shared by libgp's host code and its CUDA kernels.
#pragma once
#include <cstdint>
#include <utility>
#include <cuda_runtime.h>

namespace gpk {

constexpr uint32_t kMaxCases = 64;
constexpr uint32_t kMaxConsts = 250;    // constant codes 5 .. 254 (the paper's grid has 250)
constexpr uint32_t kLeafRows = 128;     // default leaf table: 'x' and 127 constants (codes 4 .. 131)
constexpr uint32_t kPtCode0 = 256;      // upper-tree code >= 256: value-buffer entry code-256
constexpr uint32_t kItemFinal = 1u;     // item covers a whole (upper) tree: produce fitness
constexpr uint32_t kItemFused = 2u;     // chunk of a medium tree, finished by its last chunk
constexpr uint32_t kItemRope = 4u;      // final item over a medium tree's chunk fragments
constexpr uint64_t kNoSpill = ~0ull;

// Device error word bits.
constexpr uint32_t kErrMalformed = 1u;  // final item ended with != 1 value or underflowed
constexpr uint32_t kErrSpill = 2u;      // operand stack outgrew its spill area
constexpr uint32_t kErrPlan = 4u;       // fragment emitted a different shape than planned
constexpr uint32_t kErrExtent = 8u;     // subtree extent walked off the end of a tree

__host__ __device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }

// Programmatic dependent launch: a kernel started by launch_pdl may begin
// while the kernel before it in the stream is still finishing, so its
// launch overlaps that kernel's tail; it calls pdl_wait() before it reads or
// writes any memory (the wait returns once the kernel before it has
// completed and its writes are visible; without the launch attribute it
// returns at once).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A &&...args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at{};
    at.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

constexpr uint32_t kLowWindow = 512;       // codes searched before a chunk's longest end (16 per lane)

// Ends of the chunks of one tree (codes [s, s + n), n > C), chosen by the
// calling warp (all 32 lanes).  P(e) = 1 + (operators - leaves among the
// first e - s codes) is the number of subtrees that start at or after e and
// are arguments of operators before it (Sec. 2.1's prefix order, arity 2 or
// 0).  A chunk that ends where P is low has fewer operators whose arguments
// reach past its end, so it sends fewer operators and values up to its
// tree's rope.  Each next end is the 16-aligned position among the last
// kLowWindow codes before the longest chunk allowed (C codes) where P is
// lowest, the rightmost of equals, among the ends that leave the rest of
// the tree within the chunks still allowed (mcap in all); without such a
// position it is the longest chunk's end.  `arena` is 16-byte aligned.
// f(j, e) receives end j (1-based, absolute); returns the number of chunks.
template <typename F>
__device__ __forceinline__ uint32_t cut_low(const uint8_t *__restrict__ arena, uint64_t s, uint64_t n, uint32_t C,
                                            uint32_t mcap, int lane, F f)
{
    uint64_t a = s;
    uint32_t j = 1;
    while (s + n - a > C) {
        const uint64_t left = (uint64_t)(mcap - j) * C;          // codes the later chunks can hold
        uint64_t lo = a + 1;
        if (C > kLowWindow) lo = umax64(lo, a + C - kLowWindow);
        if (n > left) lo = umax64(lo, s + n - left);
        lo = (lo + 15) & ~15ull;
        const uint64_t hi = (a + C) & ~15ull;
        uint64_t e = a + C;
        if (lo <= hi) {
            const uint32_t groups = (uint32_t)((hi - lo) >> 4);  // at most kLowWindow / 16 = 32
            int d = 0;
            if ((uint32_t)lane < groups) {
                const uint4 w = __ldg(reinterpret_cast<const uint4 *>(arena + lo) + lane);
                const uint32_t op_bits = __popc(__vcmpltu4(w.x, 0x04040404u)) + __popc(__vcmpltu4(w.y, 0x04040404u)) +
                                         __popc(__vcmpltu4(w.z, 0x04040404u)) + __popc(__vcmpltu4(w.w, 0x04040404u));
                d = 2 * (int)(op_bits >> 3) - 16;                 // P(lo + 16 (lane + 1)) - P(lo + 16 lane)
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, d, o);
                if (lane >= o) d += v;
            }
            // lowest P first, then the largest candidate index k (e = lo + 16 k)
            uint32_t key = (uint32_t)lane < groups ? ((uint32_t)(d + 1024) << 8) | (255u - (uint32_t)(lane + 1))
                                                   : 0xffffffffu;
            if (lane == 0) key = min(key, (1024u << 8) | 255u);  // k = 0: P(lo) - P(lo) = 0
            key = __reduce_min_sync(0xffffffffu, key);
            e = lo + 16ull * (255u - (key & 255u));
        }
        f(j, e);
        a = e;
        ++j;
    }
    return j;
}

// One unit of evaluator work: a contiguous range of a level's code array.
// A final item covers a whole tree (level 0) or a whole upper tree and
// yields the tree's outputs; a fragment item covers one chunk of a larger
// tree and writes that chunk's part of the next level's upper tree.
// A fused item is a chunk of a medium tree: it writes its fragment into its
// own slot (frag_off = slot, pt_base = the tree's first slot, frag_len = the
// tree's chunk count) and the chunk that completes the tree evaluates the
// tree's upper tree from all its slots.
struct alignas(16) EvalItem {
    uint64_t begin, end;     // code positions [begin, end)
    uint64_t frag_off;       // fragment: upper-tree position of its first code
    uint64_t pt_base;        // fragment: first value-buffer entry it writes
    uint64_t spill_off;      // dedicated spill area (in stack entries) or kNoSpill
    uint64_t spill_cap;      // capacity of the dedicated spill area (entries)
    uint32_t frag_len;       // fragment: number of upper-tree codes it writes
    uint32_t pt_cnt;         // fragment: number of value-buffer entries it writes
    uint32_t tree;
    uint32_t flags;
};
static_assert(sizeof(EvalItem) == 64, "EvalItem layout");

struct PlanOut {
    uint32_t frag_len;       // codes the chunk contributes to the upper tree
    uint32_t pt_cnt;         // value-buffer entries it creates
    uint32_t max_kn;         // deepest operand stack while evaluating it
    uint32_t pad;
};

struct ValOut {              // validation summary of one chunk (right-to-left)
    int64_t need;            // minimum incoming stack size with no underflow
    int64_t delta;           // net change of the stack size
    uint32_t bad_code;
    uint32_t pad;
};

struct EvalParams {
    const void *codes;             // uint8_t (level 0) or uint32_t (upper levels)
    const EvalItem *items;
    uint32_t n_items;
    const uint32_t *n_items_dev;   // if set: the item count, read on the device at launch
    uint32_t *counter;             // work counter, zero at launch
    const float *x;                // [2*lanes], padded with zeros
    const float *y;                // [2*lanes], padded with zeros
    const float *consts;           // [n_consts]
    uint32_t n_cases;
    uint32_t n_consts;
    float div0;
    uint32_t window;               // shared-memory stack entries per warp
    const float2 *pt_in;           // value buffer read by upper-tree codes >= kPtCode0
    float2 *pt_out;                // value buffer written by fragments
    uint32_t *u_out;               // next level's upper-tree codes
    float *values;                 // [n_trees * n_cases]
    float *fitness;                // [n_trees]
    uint32_t *hits;                // [n_trees]
    float2 *spill;                 // spill memory, [entries][lanes] float2
    uint64_t spill_per_warp;       // entries per resident warp
    uint32_t *err;
    // medium trees (fused items)
    uint32_t *fz_codes;            // [slots][fz_cap_codes] fragment codes, right-aligned
    float2 *fz_pt;                 // [slots][fz_cap_pt][lanes] value entries
    uint32_t *fz_len;              // [slots] fragment length
    uint32_t *fz_done;             // [n_trees] finished chunks
    uint32_t *fz_over;             // [n_trees] a chunk ran out of value slots
    uint32_t *fz_redo;             // [1 + n_trees]: count, then trees to re-evaluate
    uint32_t fz_cap_codes;
    uint32_t fz_cap_pt;
    uint32_t leaf_rows;            // leaf table rows ('x' + constants); 0 = kLeafRows
    uint32_t *stat_up;             // nullable: [0] codes, [1] operators, [2] value entries
                                   // that fragments of this launch emitted upward
};

struct XoChild {                   // child = M[0,i) ++ D[j,e_d) ++ M[e_m,n_m)
    uint64_t dst;                  // destination start (16-byte aligned)
    uint64_t n;                    // child size
    uint64_t head_src;             // source of bytes [0, i)
    uint64_t i;
    uint64_t mid_src;              // source of bytes [i, i+ld)
    uint64_t ld;
    uint64_t tail_src;             // source of bytes [i+ld, n)
    uint64_t pad;
};

struct XoTile {
    uint32_t child;
    uint32_t pad;
    uint64_t begin;                // child byte offset of the tile
};

struct ExtentQuery {
    uint64_t tree_start, tree_size, point;
};
// A subtree walk still open after its first step: where the next step
// starts (16-aligned) and the subtrees still to be read there.
struct ExtentLong {
    uint64_t base;
    int64_t need;
    uint32_t w, pad;
};

// Adds n to the library's count of kernel launches (gp_kernel_launch_count).
void note_launches(uint64_t n);

// Launchers (defined in the .cu files; return the launch's error).
size_t eval_smem_bytes(int lanes, int warps, int window, bool wide, int leaf_rows = (int)kLeafRows);
cudaError_t eval_prepare_at_least(int lanes, bool wide, size_t smem);
// pdl: launched with programmatic stream serialization (launch_pdl).
cudaError_t launch_eval(int lanes, bool wide, const EvalParams &p, int ctas, int warps,
                        size_t smem, cudaStream_t s, bool pdl = false);
cudaError_t launch_plan(bool wide, const void *codes, const EvalItem *items, uint32_t n,
                        PlanOut *out, cudaStream_t s);
cudaError_t launch_plan_scan(EvalItem *items, const PlanOut *plan, uint32_t n,
                             uint64_t *frag_off /*[n+1]*/, uint64_t *totals /*[3]*/,
                             cudaStream_t s);
// Device-count forms: at most n_max items, the count read from *n_dev on the
// device (for launch sequences that never return to the host).
cudaError_t launch_plan_dev(bool wide, const void *codes, const EvalItem *items, uint32_t n_max,
                            const uint32_t *n_dev, PlanOut *out, int sms, cudaStream_t s, bool pdl = false);
cudaError_t launch_plan_scan_dev(EvalItem *items, const PlanOut *plan, const uint32_t *n_dev,
                                 uint64_t *frag_off, uint64_t *totals, cudaStream_t s, bool pdl = false);
// Level-0 items of trees whose sizes are on the device, all at most
// max_chunks chunks of C codes: counts[0] items (fused chunks, then
// finals), counts[1] ropes (next launch), counts[2] slots.  A multi-chunk
// tree of m = ceil(n / C) chunks is cut where its arity walk is low and may
// take m + 1 chunks (never more than max_chunks), so items and slots need
// room for one more chunk per multi-chunk tree.  Four launches: the first
// zeroes zero[0 .. n_zero) (which must hold `cls`, plan_level0_scratch_
// words() words, and whatever else the caller needs zeroed), err[0..3],
// err[12] and stat[4..6]; the planned counts also go to stat[0..2].
// `meta`: one word per tree; `cuts`: the multi-chunk trees' chunk counts
// summed (the slot bound).
uint32_t plan_level0_scratch_words();
cudaError_t launch_plan_level0(const uint8_t *arena, const uint64_t *start, const uint64_t *size, uint32_t n,
                               uint32_t C, uint32_t max_chunks, EvalItem *items, EvalItem *ropes, uint32_t *counts,
                               uint32_t *cls, uint32_t *meta, uint32_t *cuts, uint32_t *zero, uint32_t n_zero,
                               uint32_t *err, uint32_t *stat, int sms, cudaStream_t s);
// Children laid out on the device from their extents: copy records, starts,
// sizes, per-child first copy tile ([n+1]) and the tile count (three
// launches; part_len / part_tiles: scratch of xo_layout_parts(n) entries).
uint32_t xo_layout_parts(uint32_t n);
cudaError_t launch_xo_layout(const ExtentQuery *q, const uint64_t *ends, uint32_t n, uint32_t tile_bytes,
                             uint64_t arena_cap, XoChild *kids, uint64_t *cstart, uint64_t *csize,
                             uint32_t *tile_base, uint32_t *tile_child, uint32_t *n_tiles, uint64_t *part_len,
                             uint32_t *part_tiles, uint32_t *err, cudaStream_t s);
// Copy of children laid out by launch_xo_layout (tile -> child map); a CTA
// per tile, or a warp per tile when warp_tiles, over up to max_tiles tiles
// (at least the tile count the layout finds).
cudaError_t launch_xo_copy_map(const uint8_t *src, uint8_t *dst, const XoChild *children, const uint32_t *tile_base,
                               const uint32_t *tile_child, const uint32_t *n_tiles_dev, uint32_t max_tiles,
                               uint32_t tile_bytes, bool warp_tiles, cudaStream_t s);
cudaError_t launch_validate(const uint8_t *codes, const EvalItem *chunks, uint32_t n_chunks,
                            uint32_t n_consts, ValOut *out, cudaStream_t s);
cudaError_t launch_validate_trees(const ValOut *chunk_out, const uint32_t *tree_first_chunk,
                                  uint32_t n_trees, uint32_t *bad_count, cudaStream_t s);
// Subtree ends of n queries (two launches: a warp step per query, then a
// CTA per query still open; `list`: n entries of scratch, *n_long: a zeroed
// counter).
cudaError_t launch_extent(const uint8_t *arena, const ExtentQuery *q, uint32_t n, uint64_t *end, uint32_t *err,
                          ExtentLong *list, uint32_t *n_long, int sms, cudaStream_t s);
cudaError_t launch_extent_dev(const uint8_t *arena, const ExtentQuery *q, uint32_t n_max, const uint32_t *n_dev,
                              uint64_t *end, uint32_t *err, ExtentLong *list, uint32_t *n_long, int sms,
                              cudaStream_t s);
// Copy of children whose tiles are numbered on the device: child c owns
// tiles [tile_base[c], tile_base[c+1]); *n_tiles_dev tiles in all.
// Children of a batch of runs, all in one heap (src = dst = heap).
cudaError_t launch_xo_copy_runs(uint8_t *heap, const XoChild *kids, const uint32_t *tile_local,
                                const uint32_t *tree_base, const uint32_t *run_tile_base,
                                const uint32_t *n_runs_dev, const uint32_t *n_tiles_dev, uint32_t tile_bytes,
                                bool warp_tiles, int sms, cudaStream_t s);
cudaError_t launch_xo_copy_dev(const uint8_t *src, uint8_t *dst, const XoChild *children,
                               const uint32_t *tile_base, uint32_t n_children,
                               const uint32_t *n_tiles_dev, uint32_t tile_bytes, int sms,
                               cudaStream_t s);
cudaError_t launch_xo_copy(const uint8_t *src, uint8_t *dst, const XoChild *children,
                           const XoTile *tiles, uint32_t n_tiles, uint32_t tile_bytes,
                           cudaStream_t s);

}  // namespace gpk
