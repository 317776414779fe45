/*
 * libgp: GB300 (sm_103a) fitness evaluation and subtree crossover of linear
 * prefix GP trees, after Langdon & Banzhaf, "Faster Genetic Programming
 * GPquick via multicore and Advanced Vector Extensions" (2019).
 *
 * Conventions for every call:
 *   - Plain C ABI: no exceptions cross it; every call returns gp_status and
 *     leaves its out-parameters untouched unless it returns GP_OK.
 *   - Host pointers are owned by the caller and only read (or written, for
 *     outputs) during the call; libgp copies what it keeps.
 *   - libgp owns all device memory of a population.  Device buffers are
 *     allocated with the stream-ordered allocator on the call's stream.
 *   - `cuda_stream` is a cudaStream_t passed as void* (NULL = the legacy
 *     default stream).  Work is enqueued on it asynchronously unless the call
 *     says it synchronises.  Calls that touch the same population must be
 *     ordered by the caller (e.g. all on one stream).
 *   - Tree encoding (Sec. 2.1-2.2: one byte per node, root first, prefix
 *     order): 0 '+', 1 '-', 2 '*', 3 protected '/', 4 'x',
 *     5..5+n_consts-1 constant table entry (code - 5).  Codes 0..3 have two
 *     arguments, the first argument immediately follows the operator.
 *   - Not thread-safe per population; distinct populations may be used from
 *     distinct host threads.
 */
#ifndef GP_H
#define GP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gp_status {
    GP_OK = 0,
    GP_EINVAL = 1,      /* bad argument (null pointer, index or size out of range) */
    GP_ENOMEM = 2,      /* device or host allocation failed, or HBM budget exceeded */
    GP_EMALFORMED = 3,  /* a tree is not one valid prefix tree over the code table */
    GP_ECUDA = 4,       /* a CUDA runtime call or kernel failed */
    GP_ETIMEOUT = 5,    /* a bounded device-side wait ran out */
    GP_ELIMIT = 6       /* a tree would exceed the problem's node limit */
} gp_status;

/* Problem definition (Table gp.details): fitness cases, constants, protected
 * division value and limits.  Copied by gp_create_population. */
typedef struct gp_problem {
    uint32_t n_cases;            /* 1..64 fitness cases (the paper uses 48)            */
    const float *x;              /* host [n_cases] inputs                              */
    const float *y;              /* host [n_cases] targets                             */
    uint32_t n_consts;           /* 0..250 constants, codes 5..5+n_consts-1 (the paper's
                                    grid has 250)                                        */
    const float *consts;         /* host [n_consts]                                    */
    float protected_div_value;   /* result of a/b when b == 0 (the paper: 1.0f)       */
    uint64_t max_tree_nodes;     /* node limit for crossover children, 0 = none        */
    uint64_t hbm_budget_bytes;   /* device bytes a population may hold, 0 = no limit   */
} gp_problem;

/* One subtree crossover (Sec. 3.1): the child is tree `mum` with the subtree
 * rooted at node `mum_point` replaced by the subtree of tree `dad` rooted at
 * node `dad_point`.  Points are node indices in prefix order. */
typedef struct gp_xo {
    uint32_t mum, dad;
    uint64_t mum_point, dad_point;
} gp_xo;

/* Optional evaluation tuning.  Zero fields mean "choose automatically". */
typedef struct gp_eval_options {
    uint32_t chunk_nodes;     /* nodes per independent evaluation chunk (multiple of 16) */
    uint32_t warps_per_cta;   /* warps of the persistent evaluator per SM (1..32)        */
    uint32_t window_entries;  /* shared-memory stack entries per warp (even, >= 16)      */
    uint32_t upper_window_entries; /* the same for upper-tree levels                    */
} gp_eval_options;

/* Device-side view of a population, for zero-copy use by the caller. */
typedef struct gp_population_info {
    uint32_t n_trees;
    uint32_t n_cases;
    uint64_t total_nodes;
    const uint8_t *d_nodes;      /* device arena; tree t starts at d_tree_start[t]    */
    const uint64_t *d_tree_start;
    const uint64_t *d_tree_size;
    const float *d_fitness;      /* [n_trees], valid after gp_evaluate                 */
    const float *d_case_values;  /* [n_trees * n_cases] per-case outputs               */
    const uint32_t *d_hits;      /* [n_trees] cases with |error| < 0.01                */
} gp_population_info;

typedef struct gp_population gp_population;

/* Upload `n_trees` trees (packed: tree t is nodes[offsets[t] .. offsets[t+1]),
 * offsets has n_trees+1 entries, offsets[0] = 0) and validate them on the
 * device (Sec. 2.1 encoding: every tree is exactly one prefix tree and uses
 * only codes < 5 + n_consts).  `nodes` may be host memory or device memory
 * of this device (e.g. trees received from another process); `offsets` is
 * host memory.  Synchronises with `cuda_stream` once to read the validation
 * result.  n_trees may be 0.
 * Errors: GP_EINVAL (null/inconsistent arguments), GP_EMALFORMED (a tree
 * fails validation), GP_ENOMEM (allocation or budget), GP_ECUDA. */
gp_status gp_create_population(const gp_problem *problem, uint32_t n_trees,
                               const uint8_t *nodes, const uint64_t *offsets,
                               void *cuda_stream, gp_population **out);

/* Create one child per record (Sec. 3.1; the choice of points is the
 * caller's, made sequentially as in Sec. 2.3, and the copies run on the
 * device).  Children form a new population with the parents' problem; its
 * fitness is not evaluated.  Every child has at most
 * n_mum + n_dad - dad_point - 1 nodes; when no such bound exceeds
 * problem->max_tree_nodes and their total fits the arena limit (four times
 * the parents' arena or 256 MiB, at most 16 GiB, and the HBM budget), the
 * call does not synchronise: the children are sized and laid out on the
 * device in an arena of that total, and a call that needs their sizes on
 * the host (gp_tree_size, gp_tree_read, gp_population_get_info, a crossover
 * with them as parents) waits for the stream and reads them then.
 * Otherwise it synchronises once to size the children exactly.
 * Errors: GP_EINVAL (index or point out of range), GP_ELIMIT (a child exceeds
 * problem->max_tree_nodes; only a synchronising call can see it),
 * GP_ENOMEM, GP_ECUDA. */
gp_status gp_crossover(const gp_population *parents, const gp_xo *ops, uint32_t n_ops,
                       void *cuda_stream, gp_population **children_out);

/* Evaluate every tree on every fitness case (Sec. 2.2 single-pass
 * evaluation, Table gp.details protected division) and reduce each tree to
 * its mean absolute error with a sequential fold in case order (Sec. 2.2,
 * Sec. 3.2) and its hit count.  Asynchronous on `cuda_stream`, except that
 * trees of more than 32 chunks (chunk_nodes, default 4096) have their upper
 * trees sized on the device and read back, one short synchronisation per
 * upper-tree level.  Children whose sizes are still on the device only and
 * whose bounds stay within 32 chunks get their work items built on the
 * device (no synchronisation); otherwise their sizes are read first.
 * Results are read with gp_fitness.
 * Errors: GP_EINVAL, GP_ENOMEM, GP_ECUDA. */
gp_status gp_evaluate(gp_population *pop, void *cuda_stream);
gp_status gp_evaluate_ex(gp_population *pop, const gp_eval_options *opt, void *cuda_stream);

/* Wait for the last gp_evaluate of `pop` and copy results to the host.
 * gp_evaluate splits medium trees into chunks whose upper-tree fragments
 * use fixed-size slots; a tree whose fragments did not fit (very wide
 * shapes) is queued on the device and evaluated again here, through planned
 * upper-tree levels, before results are copied.  Device-side results
 * (gp_population_get_info) are complete once gp_fitness has returned.
 * fitness: [n_trees] MAE (required); case_values: [n_trees * n_cases] per-case
 * outputs or NULL; hits: [n_trees] or NULL.
 * Errors: GP_EINVAL (not evaluated yet), GP_EMALFORMED / GP_ECUDA (a device
 * error recorded during evaluation). */
gp_status gp_fitness(const gp_population *pop, float *fitness, float *case_values,
                     uint32_t *hits);

/* Node count of tree `tree` (may wait for the stream of a crossover that
 * made the population without a synchronisation).  Errors: GP_EINVAL,
 * GP_EMALFORMED (that crossover met a subtree running off its parent). */
gp_status gp_tree_size(const gp_population *pop, uint32_t tree, uint64_t *n);

/* Copy tree `tree`'s bytes to host `dst` (cap >= its size).  Synchronous.
 * Errors: GP_EINVAL (cap too small / bad index), GP_ECUDA. */
gp_status gp_tree_read(const gp_population *pop, uint32_t tree, uint8_t *dst, uint64_t cap);

/* Device pointers and sizes of a population (valid until it is destroyed). */
gp_status gp_population_get_info(const gp_population *pop, gp_population_info *info);

/* Free a population's device memory, stream-ordered on the stream of the
 * last call that enqueued work on it (its creation, an evaluation, or a
 * crossover that read it as parents).  NULL is ignored. */
void gp_destroy_population(gp_population *pop);

/* Static, human-readable name of a status. */
const char *gp_status_string(gp_status st);

/* Tournament selection of both parents and uniform crossover points
 * (Table gp.details: tournaments of `tournament_size`, lowest MAE wins, NaN
 * worst, ties to the entrant drawn first; Sec. 3.1: points uniform over each
 * parent's nodes) for children [child_lo, child_lo + n_children) of
 * generation `generation` of a run seeded `seed`, from the fitness and node
 * counts of the whole population of n_pop trees: the same counter-based
 * draws a gp_generation step makes, so a population sharded over processes
 * selects each process's children from gathered fitness and sizes and gets
 * the records a single process would.  d_fitness [n_pop], d_sizes [n_pop]
 * and d_out [n_children] (global parent indices and points) are device
 * memory; asynchronous on cuda_stream.  Errors: GP_EINVAL (null pointers,
 * tournament size outside 1..32, generation >= 2^24, children past 2^28),
 * GP_ECUDA. */
gp_status gp_select(const float *d_fitness, const uint64_t *d_sizes, uint32_t n_pop, uint64_t seed,
                    uint32_t generation, uint32_t child_lo, uint32_t n_children, uint32_t tournament_size,
                    gp_xo *d_out, void *cuda_stream);

/* ---- Introspection and measurement (not part of the paper's method). ---- */

/* Shape of the last gp_evaluate of a population: evaluation levels (1 when
 * no tree was split into chunks), work items over all levels, upper-tree
 * codes and value-buffer entries created by all levels, the operators
 * evaluated above level 0, and trees that gp_fitness evaluated again
 * through planned levels because their chunk fragments did not fit the
 * fixed per-chunk slots (known once gp_fitness has returned).  Synchronises
 * with the evaluation's stream. */
typedef struct gp_eval_stats {
    uint32_t levels;
    uint32_t redone;           /* trees re-evaluated through planned levels */
    uint64_t items;
    uint64_t upper_codes;
    uint64_t value_entries;
    uint64_t upper_ops;        /* operators evaluated above level 0 (the rest
                                * of the (n-1)/2 per tree ran in level 0)     */
} gp_eval_stats;
gp_status gp_eval_stats_get(const gp_population *pop, gp_eval_stats *out);

/* Number of CUDA kernels libgp has launched in this process (all devices). */
uint64_t gp_kernel_launch_count(void);

/* Kernel kinds for gp_profile_read. */
enum {
    GP_KERNEL_EVAL = 0,        /* level-0 evaluator over tree bytes           */
    GP_KERNEL_EVAL_UPPER = 1,  /* evaluator over upper-tree codes             */
    GP_KERNEL_PLAN = 2,        /* chunk planning                              */
    GP_KERNEL_SCAN = 3,        /* plan prefix scan                            */
    GP_KERNEL_VALIDATE = 4,    /* upload validation                           */
    GP_KERNEL_EXTENT = 5,      /* crossover subtree extents                   */
    GP_KERNEL_COPY = 6,        /* crossover / upload segment copy             */
    GP_KERNEL_KINDS = 8
};
typedef struct gp_kernel_profile {
    uint64_t launches[GP_KERNEL_KINDS];
    double total_ms[GP_KERNEL_KINDS];
} gp_kernel_profile;

/* When enabled, every kernel launch is bracketed by CUDA events recorded on
 * the stream it is launched on.  gp_profile_read waits for the recorded
 * events, accumulates their elapsed times per kind and returns the running
 * totals (reset != 0 clears them afterwards). */
gp_status gp_profile_enable(int on);
gp_status gp_profile_read(gp_kernel_profile *out, int reset);

/* ---- Generations on the device (Table gp.details: panmictic, non-elitist,
 * generational; every child made by one two-parent subtree crossover whose
 * parents both win tournaments on fitness; Sec. 3.1: crossover points
 * uniform over all nodes, chosen in a fixed sequential order).
 *
 * A gp_generation holds the current population on the device in one of two
 * buffers and makes each next generation into the other: tournament
 * selection, crossover points, subtree extents, child layout, the copy and
 * the evaluation of the children all run on the device, with every count
 * kept in device memory, so one generation is one fixed launch sequence.
 * It is captured once as a CUDA graph (one graph per buffer direction) and
 * replayed.  Draws are a counter-based stream: draw number
 *     (generation << 40) | (child << 12) | (purpose << 9) | (index << 4) | attempt
 * of SplitMix64 (Steele, Lea & Flood 2014) seeded with `seed`, with purpose
 * 0 / 1 = the mum's / dad's tournament (index = entrant), 2 / 3 = the mum /
 * dad point; a draw in [0, n) is the high word of r*n for the first attempt
 * whose low word is >= 2^64 mod n (Lemire 2019; the 16th attempt is taken if
 * all are rejected).  The lowest fitness wins a tournament, NaN ranks
 * worst, ties go to the entrant drawn first.  Generation g's children use
 * counters with generation = g (the initial population is generation 0). */

typedef struct gp_generation gp_generation;

typedef struct gp_generation_params {
    uint64_t seed;               /* seed of the draws                                   */
    uint32_t tournament_size;    /* 1..32 (7 in the paper)                               */
    uint32_t chunk_nodes;        /* evaluator chunk (multiple of 16, 256..65536);
                                    0 = autotuned on the initial population: of
                                    1024..8192 (up to 1e8 nodes) or 4096..16384, the
                                    largest within 3% of the fastest; 4096 when every
                                    initial tree fits 1024 nodes                        */
    uint64_t arena_bytes;        /* capacity of each population buffer; 0 = twice the
                                    initial population plus slack                        */
    uint64_t workspace_codes;    /* upper-tree codes per level; 0 = twice what the
                                    initial population needs, at least 2^20             */
    uint64_t workspace_values;   /* value-buffer entries per level; 0 = as above        */
    uint32_t use_graph;          /* nonzero: replay one CUDA graph per generation        */
    uint32_t max_levels;         /* evaluation levels per generation (2..16); 0 = eight
                                    for the captured level loop, those of generation 0
                                    plus two (3..8) for plain launches, widened by two
                                    when a generation uses them all                     */
    uint32_t warps_per_cta;      /* level-0 evaluator warps per SM (1..32) and       */
    uint32_t window_entries;     /* shared-memory stack entries per warp (even, >= 16);
                                    both 0 = autotuned on the initial population      */
    uint32_t upper_window_entries; /* upper-level window (its warps: as many as fit,
                                    at most 16); 0 = autotuned                         */
    uint32_t pad;
} gp_generation_params;

typedef struct gp_generation_info {
    uint64_t generation;         /* index of the current population                     */
    uint32_t n_trees;
    uint32_t chunk_nodes;        /* chunk size in use (chosen by the autotuner if 0)     */
    uint64_t total_nodes;        /* nodes of the current population                     */
    uint32_t levels;             /* evaluation levels the last generation used          */
    uint32_t graph;              /* 1 if generations replay a captured CUDA graph       */
    uint32_t kernels_per_generation;
    uint32_t error_generation;   /* generation whose step failed (valid after an error)  */
    uint64_t arena_bytes, workspace_codes, workspace_values;
    uint32_t autotune_chunk[8];  /* candidate chunk sizes tried (0 = unused slot)       */
    float autotune_ms[8];        /* their evaluation time on the initial population     */
    uint32_t warps_per_cta, window_entries;             /* level 0's launch shape in use  */
    uint32_t upper_warps, upper_window_entries;         /* upper levels'                  */
    uint32_t rope_warps, rope_window_entries;           /* a rope-only level's            */
    uint32_t autotune_shape[8];  /* shapes tried, (warps << 16) | window entries: level 0's
                                    first, then the upper levels' with 0x8000 added to
                                    the window entries (0 = unused slot)                */
    float autotune_shape_ms[8];  /* their evaluation time on the initial population     */
} gp_generation_info;

/* Upload, validate and evaluate the initial population (generation 0) of
 * `n_trees` trees packed as for gp_create_population, and prepare the
 * generation step.  Synchronises `cuda_stream`.  The problem's
 * max_tree_nodes is the paper's node limit: a child larger than it stops the
 * run (the step that made it reports GP_ELIMIT).
 * Errors: GP_EINVAL (arguments, n_trees > 2^28), GP_EMALFORMED, GP_ENOMEM,
 * GP_ECUDA. */
gp_status gp_generation_create(const gp_problem *problem, const gp_generation_params *params,
                               uint32_t n_trees, const uint8_t *nodes, const uint64_t *offsets,
                               void *cuda_stream, gp_generation **out);

/* Make `n` generations, asynchronously on `cuda_stream` (no host
 * synchronisation).  A generation that fails (node limit, a buffer or
 * workspace too small) sets a device error that turns the remaining
 * launches into no-ops, so the population stays at the last complete
 * generation; the next synchronising call reports it. */
gp_status gp_generation_step(gp_generation *g, uint32_t n, void *cuda_stream);

/* Undo the last generation step (its parents become current again; their
 * buffer is untouched by the step).  Only one step can be undone. */
gp_status gp_generation_rewind(gp_generation *g, void *cuda_stream);

/* After a synchronising call reported GP_ENOMEM (the children outgrew the
 * population buffers, a level outgrew the evaluator workspace, or a fused
 * chunk's slot ran out of value entries): enlarge what ran out (the entries
 * per slot double up to the chunk size, after which trees of 2..8 chunks go
 * through planned levels too), clear the error and capture the generation
 * again.  The next step makes the
 * failed generation again (its draws are the same).  Synchronises.
 * GP_EINVAL if the run has no such error; GP_ENOMEM if the device cannot
 * hold the larger buffers. */
gp_status gp_generation_recover(gp_generation *g, void *cuda_stream);

/* Synchronise and copy the current population's results (any pointer may be
 * null).  Returns the error of a failed step: GP_ELIMIT (node limit),
 * GP_ENOMEM (population buffer, workspace or item capacity), GP_EMALFORMED,
 * GP_ECUDA. */
gp_status gp_generation_fitness(gp_generation *g, float *fitness, float *case_values, uint32_t *hits);

/* Synchronise and copy the crossover records that made the current
 * population: records[n_trees], child t = record t (mum and dad index the
 * previous population).  GP_EINVAL while the current population is
 * generation 0 (before the first step, or after rewinding it); a failed
 * step's error otherwise, as gp_generation_fitness. */
gp_status gp_generation_records(gp_generation *g, gp_xo *records);

/* Synchronise and copy the current population: offsets [n_trees + 1] and,
 * if nodes is not null, the packed trees (cap bytes at least the total,
 * else GP_EINVAL).  A failed step's error as gp_generation_fitness. */
gp_status gp_generation_trees(gp_generation *g, uint64_t *offsets, uint8_t *nodes, uint64_t cap);

/* Synchronise and copy one tree of the current population: its node count
 * to *n_nodes and, if nodes is not null, its bytes (cap at least the count,
 * else GP_EINVAL).  GP_EINVAL for tree >= n_trees; a failed step's error as
 * gp_generation_fitness. */
gp_status gp_generation_tree_read(gp_generation *g, uint32_t tree, uint8_t *nodes, uint64_t cap,
                                  uint64_t *n_nodes);

/* Synchronise and describe the run (also after a failed step, whose
 * generation is then error_generation; total_nodes is 0 in that case). */
gp_status gp_generation_get_info(gp_generation *g, gp_generation_info *info);
/* Free the run's device memory and graphs (waits for its work).  NULL is
 * ignored. */
void gp_generation_destroy(gp_generation *g);

/* ---- Serving: many independent runs on one GPU (continuous batching).
 *
 * A gp_server holds many runs (each a population like a gp_generation, all
 * on the same problem) in one device heap of hbm_budget_bytes.  A run is
 * admitted when the heap can hold its two population buffers (in the order
 * runs were opened); until then it waits, its trees kept on the host.
 * Clients submit generation requests ("advance run r by k generations") from
 * any thread; a scheduler thread advances, in each iteration, every run with
 * a pending request that fits the batch limits by one generation, all of
 * them in one launch sequence (one CUDA graph), so requests that arrive
 * while a batch runs join the next one.  Results do not depend on which runs
 * share a batch (each run's draws and trees are its own).  A workspace
 * overflow in a batch of several runs makes the scheduler retry them in
 * smaller batches.  A run whose children outgrow its buffers is moved to
 * buffers twice as large when the heap has room (until then it waits) and
 * the generation is made again; a run's other failures (node limit)
 * fail its pending requests with that status. */

typedef struct gp_server gp_server;

typedef struct gp_server_params {
    uint64_t hbm_budget_bytes;   /* device heap for the runs' population buffers       */
    uint32_t max_runs;           /* runs held (admitted) at once, 1..4096                */
    uint32_t max_batch_runs;     /* runs advanced by one batch (0 = max_runs)            */
    uint32_t max_batch_trees;    /* trees of all runs in one batch                       */
    uint32_t chunk_nodes;        /* evaluator chunk (0 = 8192)                           */
    uint64_t max_batch_nodes;    /* nodes of all runs in one batch (workspace sizing)    */
    uint64_t workspace_codes;    /* 0 = 8% of max_batch_nodes                            */
    uint64_t workspace_values;   /* 0 = 3% of max_batch_nodes                            */
    uint32_t use_graph;          /* nonzero: replay one captured CUDA graph per batch    */
    uint32_t pad;
} gp_server_params;

typedef struct gp_server_result {
    uint64_t run_id, request_id;
    uint64_t generation;         /* the run's generation when the request completed     */
    float best_fitness;          /* lowest MAE of the population (NaN ranks worst)       */
    uint32_t best_tree, best_hits;
    gp_status status;
    uint64_t total_nodes;        /* nodes of the population                              */
    double latency_ms;           /* submit -> completion                                 */
    double queue_ms;             /* submit -> first batch that served it                 */
} gp_server_result;

typedef struct gp_server_stats {
    uint64_t batches, run_generations, requests_done, child_nodes;
    double device_ms;            /* GPU time of all batches (CUDA events)               */
    double mean_runs_per_batch;
    double latency_p50_ms, latency_p99_ms;
    uint64_t heap_bytes, heap_free;
    uint32_t runs_admitted, runs_waiting;
    uint64_t most_level_codes;   /* largest upper-tree code count of one level of a batch */
    uint64_t most_level_values;  /* largest value-entry count of one level of a batch    */
    uint64_t retries;            /* runs sent back after a workspace overflow            */
    uint64_t regrown;            /* runs moved to larger buffers after outgrowing theirs */
} gp_server_stats;

/* Errors: GP_EINVAL, GP_ENOMEM (budget or workspace), GP_ECUDA. */
gp_status gp_server_create(const gp_problem *problem, const gp_server_params *params, gp_server **out);
/* Open a run (copies the trees); admitted when its buffers fit the heap.
 * params: seed, tournament_size, arena_bytes (0 = twice the trees + slack);
 * the other fields are ignored.  GP_ENOMEM if the run can never fit. */
gp_status gp_server_open_run(gp_server *s, const gp_generation_params *params, uint32_t n_trees,
                             const uint8_t *nodes, const uint64_t *offsets, uint64_t *run_id);
/* Open a run whose initial population is trees[0..n_trees) of the device
 * population `src` (indices may repeat), for initial populations too large
 * to stage on the host: nothing is copied now; at admission the trees are
 * copied on the device from `src`, which must stay alive, and not be
 * destroyed, until the run is admitted (gp_server_get_stats: runs_admitted)
 * or closed.  `src` was validated when it was made, so the trees are not
 * checked again.  Same params and errors as gp_server_open_run; GP_EINVAL
 * for an index past src's trees or a different number of fitness cases. */
gp_status gp_server_open_run_from(gp_server *s, const gp_generation_params *params, const gp_population *src,
                                  uint32_t n_trees, const uint32_t *trees, uint64_t *run_id);
/* Ask for `n_generations` (>= 1) more generations of a run; returns at
 * once with the request's id.  GP_EINVAL for an unknown run or zero
 * generations; the run's failure status if it has failed. */
gp_status gp_server_submit(gp_server *s, uint64_t run_id, uint32_t n_generations, uint64_t *request_id);
/* Wait for a request (timeout_ms < 0: no limit).  GP_ETIMEOUT if it has not
 * completed; otherwise GP_OK with the result (result->status is the
 * request's own outcome), and the request is forgotten: a second wait on it
 * returns GP_EINVAL, and so does a wait that was already waiting on it when
 * another thread collected it. */
gp_status gp_server_wait(gp_server *s, uint64_t request_id, double timeout_ms, gp_server_result *result);
/* After the run's requests completed: its current population's results / trees. */
gp_status gp_server_run_fitness(gp_server *s, uint64_t run_id, float *fitness, float *case_values, uint32_t *hits);
gp_status gp_server_run_trees(gp_server *s, uint64_t run_id, uint64_t *offsets, uint8_t *nodes, uint64_t cap);
/* Waits for the run's requests, then frees its buffers (waiting runs may
 * then be admitted).  A run not admitted yet is closed at once and its
 * requests complete with GP_EINVAL. */
gp_status gp_server_close_run(gp_server *s, uint64_t run_id);
/* Counters since the server was created (latency percentiles over every
 * completed request); does not wait for the scheduler's current batch. */
gp_status gp_server_get_stats(gp_server *s, gp_server_stats *stats);
/* Stops the scheduler and frees everything; no other call on the server may
 * be in progress or follow (clients must have stopped waiting). */
void gp_server_destroy(gp_server *s);

/* ---- Evaluation without allocation.  The paper has no counterpart: this
 * serves callers that cannot allocate device memory while they evaluate,
 * e.g. a loop whose GPU memory is owned by its own allocator, or one that
 * cannot afford the implicit synchronisation of cudaMalloc / cudaFree. ---- */

#define GP_NOALLOC_MAX_TREES 16384u        /* trees per call                      */
#define GP_NOALLOC_MAX_TREE_NODES 4096u    /* nodes per tree                      */

/* Evaluate `n_trees` trees like gp_evaluate + gp_fitness, without allocating
 * anything: no device or host allocation, no stream-ordered pool.  All
 * scratch (work items, per-tree validation results, a work counter, error
 * words, the fitness cases and constants) lives in one static device array
 * inside libgp of about 1.4 MiB (4 KiB + GP_NOALLOC_MAX_TREES x (64 + 24) B),
 * which every GPU that loads libgp holds until the process exits.  The call
 * sets every word of it that it reads, so nothing needs to start at zero.
 *   d_nodes:  device, the trees packed as for gp_create_population
 *             (offsets[], host, n_trees + 1 entries, offsets[0] = 0); 16-byte
 *             aligned and readable up to the next multiple of 16 bytes past
 *             its end, inside one allocation.  Trees are validated (codes
 *             and stack balance) before anything is evaluated.
 *   d_fitness [n_trees], d_case_values [n_trees * n_cases], d_hits [n_trees]:
 *             device outputs, as gp_fitness returns them.
 * Operand stacks get a 256-entry shared-memory window and no spill area.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  The call
 * synchronises `cuda_stream` twice, to read the validation count and the
 * error word.  Every call shares the
 * array and overwrites it: calls that overlap on the GPU (other host
 * threads, other streams) race.
 * Errors: GP_ELIMIT (n_trees > GP_NOALLOC_MAX_TREES, a tree larger than
 * GP_NOALLOC_MAX_TREE_NODES, or an operand stack deeper than its window),
 * GP_EINVAL (null, misaligned or too short buffers, bad offsets or problem),
 * GP_EMALFORMED (a tree is not one prefix tree), GP_ECUDA. */
gp_status gp_evaluate_noalloc(const gp_problem *problem, uint32_t n_trees, const uint8_t *d_nodes,
                              const uint64_t *offsets, float *d_fitness, float *d_case_values,
                              uint32_t *d_hits, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* GP_H */
