// Internal: the generation engine shared by gp_generation (one run) and
// gp_server (many runs batched together).
//
// Every population lives in a device heap owned by the engine; positions of
// trees are heap offsets, so the trees of several runs can be crossed and
// evaluated by the same launches.  Each run has a device run-table entry
// (its two population buffers, its draws' seed, its generation, a sticky
// error) and a batch lists the runs it advances.  One batch is one fixed
// launch sequence whose counts live in device memory (BatchCtl), captured
// once as a CUDA graph.
#pragma once
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "gp.h"
#include "gp_internal.cuh"

namespace gpk {
// Trees of a device population copied into device memory at 16-byte aligned
// offsets from dst + dst_lo (gp_api.cu).
gp_status gather_trees(const gp_population *src, const uint32_t *trees, uint32_t n, uint8_t *dst, uint64_t dst_lo,
                       uint64_t cap, uint64_t *start, uint64_t *size, cudaStream_t s);
}  // namespace gpk

namespace gpe {

using gpk::EvalItem;
using gpk::ExtentQuery;
using gpk::ExtentLong;
using gpk::PlanOut;
using gpk::XoChild;

// Sticky error bits (per run, or for a whole batch).
constexpr uint32_t kGErrLimit = 1u;      // a child above the node limit (the run stops)
constexpr uint32_t kGErrArena = 2u;      // children larger than the run's population buffer
constexpr uint32_t kGErrWork = 4u;       // a level's codes / value entries above the workspace
constexpr uint32_t kGErrLevels = 8u;     // trees unfinished after the last level
constexpr uint32_t kGErrItems = 16u;     // more items than the item buffer holds
constexpr uint32_t kGErrEval = 32u;      // the evaluator reported an error
constexpr uint32_t kGErrExtent = 64u;    // a subtree extent ran off its tree
constexpr uint32_t kGErrSpill = 128u;    // oversized finals above the dedicated spill pool
constexpr uint32_t kGErrGen = 256u;      // generation counter past 2^24
constexpr uint32_t kGErrSlots = 512u;    // a fused chunk's slot ran out of value entries
constexpr uint32_t kGErrBatch =
    kGErrWork | kGErrLevels | kGErrItems | kGErrSpill | kGErrEval | kGErrExtent | kGErrSlots;
// Trees of 2..kFuseMaxChunks chunks: fused chunks and a rope.  A rope walks
// its tree's fragments one after the other and restarts its copy pipeline
// at each, so the longest ropes (bloated populations) are kept short; larger
// trees go through planned levels.
constexpr uint32_t kFuseMaxChunks = 8;

constexpr uint32_t kModeGenerate = 0u;   // make one generation of every run in the batch
constexpr uint32_t kModeEvaluate = 1u;   // evaluate every run's current population

struct RunBuf {
    uint64_t lo, cap;                    // arena: heap bytes [lo, lo + cap)
    uint64_t *start, *size;              // [n] heap offsets and sizes of the trees
    float *fit, *vals;                   // [n], [n * n_cases]
    uint32_t *hits;                      // [n]
};

struct RunDev {                          // device run table entry
    RunBuf buf[2];
    uint64_t seed, max_nodes;
    uint32_t n, tsize;
    uint32_t gen, cur;                   // generation and buffer of the current population
    uint32_t err, err_gen;               // sticky error bits, generation whose step raised them
    uint32_t levels, pad;
    uint64_t nodes;                      // nodes of the current population
    uint64_t next_nodes;                 // nodes of the children being made
};

struct BatchHead {                       // written by the host before each batch
    uint32_t mode, n_runs, n_trees, pad;
};

struct BatchCtl {
    BatchHead head;
    uint32_t err;                        // batch-level error bits of this batch
    uint32_t n_queries, n_tiles, n_items, n_chunks, levels;
    uint32_t eval_err[4];                // [0] evaluator error word, [1] extent error word,
                                         // [3] subtree walks left to the long-walk launch
    uint32_t n_ropes;                    // fused chunks cut at level 0 (their ropes are level 1's)
    uint32_t loop_level;                 // upper levels the captured level loop has started
    uint32_t n_rope_items;               // ropes level 0 listed (a rope-only level 1)
    uint64_t totals[4];                  // plan scan totals of the current level
    uint64_t need_codes[2], need_values[2], need_dedicated, need_items, need_slots;   // sizing records
    uint64_t child_nodes;                // nodes of all children made by this batch
    uint32_t counter[64];                // evaluator work counters, one per level
};

struct RunHost {                         // host copy of a run's layout
    bool used = false;
    uint32_t n = 0;
    uint64_t arena_cap = 0;
    uint64_t lo[2] = {0, 0};
    std::vector<void *> allocs;
};

// Evaluator workspace for one chunk size.
struct Work {
    uint32_t C = 0;
    uint64_t cap_codes[2] = {0, 0}, cap_values[2] = {0, 0};
    uint64_t cap_items = 0, cap_dedicated = 0;
    EvalItem *items = nullptr;
    PlanOut *plan = nullptr;
    uint64_t *frag_off = nullptr;
    uint32_t *codes[2] = {nullptr, nullptr};
    float2 *vals[2] = {nullptr, nullptr};
    float2 *spill = nullptr;
    uint64_t spill_per_warp = 0, spill_base = 0;
    // fused chunks (trees of 2..kFuseMaxChunks chunks at level 0): one slot per chunk
    // for its fragment (C codes, fz_cap_pt value entries); cap_slots 0 = off
    uint64_t cap_slots = 0;
    uint32_t fz_cap_pt = 0;
    uint32_t *fz_codes = nullptr, *fz_len = nullptr, *fz_over = nullptr, *fz_redo = nullptr;
    float2 *fz_pt = nullptr;
};

// Records (size-`tsize` tournaments of both parents, uniform points) of
// children [lo, lo + n) of generation g from the whole population's
// fitness and sizes, as a generation step draws them (gp_select).
cudaError_t launch_select_range(const float *fit, const uint64_t *size, uint32_t n_pop, uint64_t seed, uint32_t g,
                                uint32_t lo, uint32_t n, uint32_t tsize, gp_xo *out, cudaStream_t s);

class Engine {
  public:
    ~Engine();
    // heap_bytes: population arenas; max_trees: trees of all runs in one
    // batch; max_runs: runs in the run table (and per batch).
    gp_status init(const gp_problem *problem, uint64_t heap_bytes, uint32_t max_runs, uint32_t max_trees,
                   uint32_t levels_max);
    // A run with two arenas of arena_cap bytes each; GP_ENOMEM if the heap
    // cannot hold them now.
    gp_status open_run(uint32_t n, uint64_t arena_cap, uint64_t seed, uint32_t tsize, uint64_t max_nodes,
                       uint32_t *run);
    void close_run(uint32_t run);
    // Move a run to two larger population buffers (its current population
    // copied, tree offsets rebased); GP_ENOMEM if the heap cannot hold them.
    gp_status grow_run(uint32_t run, uint64_t arena_cap, cudaStream_t s);
    // Replace the heap by a larger one holding the same bytes at the same
    // offsets (graphs must be captured again afterwards).
    gp_status grow_heap(uint64_t heap_bytes);
    // Upload, validate and lay out a run's initial population (generation 0,
    // not evaluated).
    gp_status load_run(uint32_t run, const uint8_t *nodes, const uint64_t *offsets, cudaStream_t s);
    // The same from trees of a device population (validated when it was made).
    gp_status load_run_from(uint32_t run, const gp_population *src, const uint32_t *trees, cudaStream_t s);
    // cap_slots: fused chunk slots (0: every multi-chunk tree is planned);
    // fz_cap_pt: value entries per slot (0: max(128, C / 8)).
    gp_status set_workspace(uint32_t C, const uint64_t cap_codes[2], const uint64_t cap_values[2],
                            uint64_t cap_dedicated, uint64_t cap_items, uint64_t cap_slots = 0,
                            uint32_t fz_cap_pt = 0);
    // Replace the fused slots by cap_slots slots of fz_cap_pt entries each.
    gp_status set_slots(uint64_t cap_slots, uint32_t fz_cap_pt);
    // Evaluator launch shapes: warps per SM and window entries of level 0
    // (W, K), of the upper levels (Wu, Ku) and of a rope-only launch (Wr,
    // Kr); GP_EINVAL if a shape does not fit shared memory.  Call
    // set_workspace afterwards (the per-warp spill areas follow W) and
    // capture again.
    gp_status set_shape(uint32_t W, uint32_t K, uint32_t Wu, uint32_t Ku, uint32_t Wr, uint32_t Kr);
    // Enqueue one batch; `sizing` reads each level's totals back and grows
    // the workspace (never inside a capture).
    gp_status enqueue(uint32_t mode, const std::vector<uint32_t> &runs, cudaStream_t s, bool sizing,
                      uint32_t *launches);
    // Capture the launch sequence of a batch (without its head copy) as a
    // graph; replay with launch_graph after writing the head.
    gp_status capture(uint32_t mode);
    gp_status launch_graph(uint32_t mode, const std::vector<uint32_t> &runs, cudaStream_t s);
    gp_status read_run(uint32_t run, RunDev *out, cudaStream_t s);
    gp_status read_ctl(BatchCtl *out, cudaStream_t s);
    gp_status rewind(uint32_t run, cudaStream_t s);
    gp_status clear_error(uint32_t run, cudaStream_t s);
    // Synchronous copies: crossover records of batch trees [first, first+n);
    // a run buffer's trees packed (offsets [n+1], nodes if not null).
    gp_status copy_records(gp_xo *out, uint32_t first, uint32_t n);
    gp_status copy_trees(const RunBuf &B, uint32_t n, uint64_t *offsets, uint8_t *nodes, uint64_t cap);
    gp_status copy_tree(const RunBuf &B, uint32_t t, uint8_t *nodes, uint64_t cap, uint64_t *n_nodes);
    // The device head was overwritten (e.g. the control block was cleared).
    void forget_head() { last_mode_ = ~0u; last_runs_.clear(); }
    uint64_t heap_free() const;
    uint64_t heap_largest_free() const;

    // configuration (read-only after init)
    int device = 0, sms = 0, lanes = 0;
    uint32_t n_cases = 0, n_consts = 0, max_runs = 0, max_trees = 0, levels_max = 8;
    float div0 = 1.0f;
    uint32_t W = 32, K = 32, Wu = 16, Ku = 128;
    // a launch of ropes only: few long serial walks, so deeper windows
    uint32_t Wr = 4, Kr = 192;
    int rows = 128;                      // leaf table rows: 'x' + the constants
    size_t smem = 0, smem_u = 0, smem_r = 0;
    uint64_t heap_bytes = 0;
    uint8_t *heap = nullptr;
    RunDev *runs_dev = nullptr;
    std::vector<RunHost> runs_host;
    Work w;
    uint32_t kernels_per_batch[2] = {0, 0};
    // kernels of a captured batch outside the level loop, and per loop level
    // children's copy: CTAs on 16 KB tiles, or warps on 2 KB tiles for
    // populations of small trees (set before the first capture)
    uint32_t xo_tile = 16384;
    bool xo_warp = false;
    uint32_t kernels_fixed[2] = {0, 0}, kernels_per_level = 0;
    // levels the captured loop may run (its last makes every open tree final)
    uint32_t levels_cap_graph = 16;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    cudaStream_t cap_stream = nullptr, cap_body[2] = {nullptr, nullptr};
    EvalItem *rope_items_ = nullptr;     // [max_trees] level 0's rope list, largest first
    // kernels a replay of the captured batch `mode` runs when it used `levels` levels
    uint32_t graph_kernels(uint32_t mode, uint32_t levels) const {
        return kernels_fixed[mode & 1] + kernels_per_level * (levels > 1 ? levels - 1 : 0);
    }
    BatchCtl *ctl = nullptr;

  private:
    gp_status write_head(uint32_t mode, const std::vector<uint32_t> &runs, cudaStream_t s);
    gp_status enqueue_body(uint32_t mode, cudaStream_t s, bool sizing, uint32_t *launches);
    gp_status enqueue_eval(cudaStream_t s, bool sizing, uint32_t *launches);
    struct LevelCond;                    // graph conditions a level's check kernel sets
    gp_status enqueue_level(uint32_t level, bool dyn, cudaStream_t s, bool sizing, uint32_t &prev_chunks,
                            const LevelCond &cond, uint32_t *nl, bool *stop);
    bool capturing_ = false;             // enqueue_body is recording the batch graph
    uint64_t heap_alloc(uint64_t bytes);
    void heap_release(uint64_t off, uint64_t bytes);

    std::vector<void *> allocs_, work_allocs_;
    std::vector<std::pair<uint64_t, uint64_t>> free_;   // heap free list: (offset, bytes), sorted
    // batch tables
    uint32_t *slot_run_ = nullptr, *tree_base_ = nullptr, *run_tiles_ = nullptr;
    gp_xo *recs_ = nullptr;
    ExtentQuery *q_ = nullptr;
    uint64_t *ends_ = nullptr;
    XoChild *kids_ = nullptr;
    uint32_t *tile_local_ = nullptr;
    uint64_t *bstart_ = nullptr, *bsize_ = nullptr;
    float *bfit_ = nullptr, *bvals_ = nullptr;
    uint32_t *bhits_ = nullptr;
    uint64_t *t_lo_ = nullptr, *t_hi_ = nullptr, *t_prev_ = nullptr;
    uint32_t *t_first_ = nullptr, *t_state_ = nullptr, *t_nch_ = nullptr, *t_cut_ = nullptr;
    ExtentLong *xlong_ = nullptr;
    uint32_t *fz_tree_ = nullptr, *fin_tree_ = nullptr, *rope_tree_ = nullptr;   // item builder's lists
    float *x_ = nullptr, *y_ = nullptr, *c_ = nullptr;
    // the last head written (a batch whose head is unchanged skips the copies)
    uint32_t last_mode_ = ~0u;
    std::vector<uint32_t> last_runs_;
};

}  // namespace gpe
