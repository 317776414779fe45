// gp_generation: one run on the generation engine (Table gp.details:
// panmictic, non-elitist, generational, size-7 tournaments for both
// parents; Sec. 3.1: subtree crossover with uniform points chosen in a fixed
// order).  The run's population stays on the device; each generation is one
// engine batch, replayed from a captured CUDA graph.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "gp_engine.cuh"

using namespace gpe;

struct gp_generation {
    Engine eng;
    uint32_t run = 0, n = 0;
    bool use_graph = false;
    bool auto_levels = false;         // level budget follows the levels generations use
    uint32_t levels_cap = 8;
    cudaStream_t last = nullptr;      // stream of the last enqueue (the legacy stream is null)
    gp_generation_info info{};
};

namespace {

gp_status map_err(uint32_t err, uint32_t eval_err)
{
    if (!err) return GP_OK;
    if (err & (kGErrLimit | kGErrGen)) return GP_ELIMIT;
    if (err & (kGErrArena | kGErrWork | kGErrItems | kGErrSpill | kGErrLevels | kGErrSlots)) return GP_ENOMEM;
    if (err & kGErrExtent) return GP_EMALFORMED;
    if (err & kGErrEval) return (eval_err & gpk::kErrMalformed) ? GP_EMALFORMED : GP_ECUDA;
    return GP_ECUDA;
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

// Level budget of a run whose trees grow: a generation that used every
// level (its last level made all open upper trees final items, however
// large) widens the budget by two for the next generations, up to the cap.
gp_status widen_levels(gp_generation *G, uint32_t used)
{
    Engine &E = G->eng;
    // (a captured generation runs its upper levels in a loop on the device,
    // up to the cap, so only the plain launch sequence has a budget)
    if (G->use_graph || !G->auto_levels || used < E.levels_max || E.levels_max >= G->levels_cap) return GP_OK;
    E.levels_max = std::min<uint32_t>(G->levels_cap, E.levels_max + 2);
    return GP_OK;
}

// Synchronise and read the run's state; the run's error (if any) as a status.
gp_status sync_run(gp_generation *G, RunDev *R)
{
    gp_status st = G->eng.read_run(G->run, R, G->last);
    if (st) return st;
    BatchCtl c{};
    if ((st = G->eng.read_ctl(&c, G->last))) return st;
    G->info.generation = R->gen;
    G->info.levels = R->levels;
    G->info.error_generation = R->err ? R->err_gen : 0;
    if (!R->err && (st = widen_levels(G, R->levels))) return st;
    return map_err(R->err, c.eval_err[0]);
}

float time_eval(gp_generation *G, cudaStream_t s)
{
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
    gp_status st = G->eng.enqueue(kModeEvaluate, {G->run}, s, false, nullptr);
    cudaEventRecord(b, s);
    float ms = -1.0f;
    if (!st && cudaEventSynchronize(b) == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return st ? -1.0f : ms;
}

}  // namespace

extern "C" {

gp_status gp_generation_create(const gp_problem *problem, const gp_generation_params *params,
                               uint32_t n_trees, const uint8_t *nodes, const uint64_t *offsets,
                               void *cuda_stream, gp_generation **out)
{
    if (!problem || !params || !out || !nodes || !offsets || n_trees == 0 || n_trees > (1u << 28))
        return GP_EINVAL;
    if (problem->n_cases == 0 || problem->n_cases > gpk::kMaxCases || problem->n_consts > gpk::kMaxConsts) return GP_EINVAL;
    if (params->tournament_size < 1 || params->tournament_size > 32) return GP_EINVAL;
    if (params->chunk_nodes && (params->chunk_nodes % 16 || params->chunk_nodes < 256 ||
                                params->chunk_nodes > 65536))
        return GP_EINVAL;
    if (params->max_levels && (params->max_levels < 2 || params->max_levels > 16)) return GP_EINVAL;
    if (offsets[0] != 0) return GP_EINVAL;
    uint64_t used = 0;
    for (uint32_t t = 0; t < n_trees; ++t) {
        if (offsets[t + 1] <= offsets[t]) return GP_EINVAL;
        used = (used + (offsets[t + 1] - offsets[t]) + 15) & ~15ull;
    }
    const uint64_t cap_arena = params->arena_bytes ? params->arena_bytes : 2 * used + 16ull * n_trees + (1u << 20);
    if (cap_arena < used + 64) return GP_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    gp_generation *G = new (std::nothrow) gp_generation();
    if (!G) return GP_ENOMEM;
    // GP_VERBOSE=1 in the environment: say which step of the creation failed
    const char *verbose = std::getenv("GP_VERBOSE");
    const char *step = "init";
    auto fail = [&](gp_status e) {
        if (verbose && verbose[0] == '1') {
            size_t fr = 0, tot = 0;
            cudaMemGetInfo(&fr, &tot);
            std::fprintf(stderr, "gp_generation_create: %s failed (status %d); device memory free %.1f GB of %.1f GB\n",
                         step, (int)e, fr / 1e9, tot / 1e9);
        }
        delete G;
        return e;
    };
    G->n = n_trees;
    G->use_graph = params->use_graph != 0;
    Engine &E = G->eng;
    gp_status st = E.init(problem, 2 * ((cap_arena + 255) & ~255ull), 1, n_trees,
                          params->max_levels ? params->max_levels : 8);
    if (st) return fail(st);
    if (n_trees && offsets[n_trees] < 8192ull * n_trees) {   // small trees: warps copy 2 KB tiles
        E.xo_tile = 2048;
        E.xo_warp = true;
    }
    step = "open_run";
    if ((st = E.open_run(n_trees, cap_arena, params->seed, params->tournament_size, problem->max_tree_nodes,
                         &G->run)))
        return fail(st);
    step = "load_run";
    if ((st = E.load_run(G->run, nodes, offsets, s))) return fail(st);

    // chunk size: the given one, or the fastest candidate on generation 0,
    // a larger chunk preferred within 3% of the fastest (larger populations
    // favour larger chunks: fewer fragment boundaries, fewer value entries;
    // the per-warp spill area grows with the chunk).  A population whose
    // trees all fit the smallest candidate says nothing about chunks (every
    // candidate evaluates whole trees), and runs grow: 4096 then.
    const uint32_t small_c[4] = {1024, 2048, 4096, 8192}, large_c[3] = {4096, 8192, 16384};
    uint64_t maxn = 0;
    for (uint32_t t = 0; t < n_trees; ++t) maxn = std::max<uint64_t>(maxn, offsets[t + 1] - offsets[t]);
    std::vector<uint32_t> tries;
    if (params->chunk_nodes) tries.push_back(params->chunk_nodes);
    else if (maxn <= small_c[0]) tries.push_back(4096);
    else if (used <= 100000000ull) tries.assign(small_c, small_c + 4);
    else tries.assign(large_c, large_c + 3);
    cudaStream_t cs = E.cap_stream;
    uint32_t best_C = 0;
    float min_ms = 0.f;
    uint64_t best_codes[2] = {0, 0}, best_vals[2] = {0, 0}, best_ded = 0, best_slots = 0;
    uint32_t best_pt = 0;
    for (size_t k = 0; k < tries.size(); ++k) {
        const uint32_t C = tries[k];
        const uint64_t c0[2] = {1u << 20, 1u << 20}, v0[2] = {1u << 18, 1u << 18};
        // fused chunk slots: grown by the sizing pass; a slot whose value
        // entries overflowed doubles the entries per slot (up to C, after
        // which multi-chunk trees are planned instead)
        uint64_t slots = 1024;
        uint32_t pt = std::max<uint32_t>(128, C / 8);
        BatchCtl c{};
        RunDev R{};
        for (;;) {
            step = "autotune workspace";
            if ((st = E.set_workspace(C, c0, v0, 1u << 16, cap_arena / C + 2ull * n_trees + 1024, slots, pt)))
                return fail(st);
            step = "autotune sizing pass";
            // on the sizing stream: a legacy-stream memset is not ordered
            // with the non-blocking stream and could land after the pass
            // has recorded its needs
            if (cudaMemsetAsync(E.ctl, 0, sizeof(BatchCtl), cs) != cudaSuccess) return fail(GP_ECUDA);
            E.forget_head();
            if ((st = E.enqueue(kModeEvaluate, {G->run}, cs, true, nullptr))) return fail(st);   // sizing pass
            if ((st = E.read_ctl(&c, cs)) || (st = E.read_run(G->run, &R, cs))) return fail(st);
            if (R.err != kGErrSlots || !slots) break;      // a slot's value entries overflowed:
            slots = std::max<uint64_t>(slots, c.need_slots + c.need_slots / 2 + 64);
            if (pt < C) pt *= 2;                           // more entries, or no fused chunks
            else slots = 0;
            if ((st = E.clear_error(G->run, cs))) return fail(st);
        }
        if (R.err) {
            if (verbose && verbose[0] == '1')
                std::fprintf(stderr, "gp_generation_create: chunk %u: run error bits 0x%x, batch error 0x%x, "
                             "level needs codes %llu/%llu values %llu/%llu\n", C, R.err, c.err,
                             (unsigned long long)c.need_codes[0], (unsigned long long)c.need_codes[1],
                             (unsigned long long)c.need_values[0], (unsigned long long)c.need_values[1]);
            return fail(map_err(R.err, c.eval_err[0]));
        }
        step = "autotune timing";
        float ms = -1.f;
        for (int rep = 0; rep < 2; ++rep) ms = time_eval(G, cs);             // timed, device only
        if ((st = E.read_run(G->run, &R, cs))) return fail(st);
        if (ms < 0.f || R.err) {
            if (verbose && verbose[0] == '1' && R.err == 0) {
                std::fprintf(stderr, "gp_generation_create: chunk %u: timing launch failed\n", C);
            } else if (verbose && verbose[0] == '1') {
                BatchCtl c2{};
                E.read_ctl(&c2, cs);
                std::fprintf(stderr, "gp_generation_create: chunk %u timed: run error bits 0x%x, batch error 0x%x, "
                             "eval error 0x%x, caps codes %llu/%llu values %llu/%llu items %llu ded %llu, "
                             "needs codes %llu/%llu values %llu/%llu items %llu ded %llu\n", C, R.err, c2.err,
                             c2.eval_err[0], (unsigned long long)E.w.cap_codes[0], (unsigned long long)E.w.cap_codes[1],
                             (unsigned long long)E.w.cap_values[0], (unsigned long long)E.w.cap_values[1],
                             (unsigned long long)E.w.cap_items, (unsigned long long)E.w.cap_dedicated,
                             (unsigned long long)c2.need_codes[0], (unsigned long long)c2.need_codes[1],
                             (unsigned long long)c2.need_values[0], (unsigned long long)c2.need_values[1],
                             (unsigned long long)c2.need_items, (unsigned long long)c2.need_dedicated);
            }
            return fail(R.err ? map_err(R.err, 0) : GP_ECUDA);
        }
        if (k < 8) {
            G->info.autotune_chunk[k] = C;
            G->info.autotune_ms[k] = ms;
        }
        if (verbose && verbose[0] == '1')
            std::fprintf(stderr, "gp_generation_create: chunk %u: %.3f ms, fused slots %llu needed (%llu x %u held)\n",
                         C, ms, (unsigned long long)c.need_slots, (unsigned long long)E.w.cap_slots, E.w.fz_cap_pt);
        min_ms = best_C ? std::min(min_ms, ms) : ms;
        if (!best_C || ms <= 1.03f * min_ms) {          // candidates come in increasing chunk size
            best_C = C;
            for (int i = 0; i < 2; ++i) {
                best_codes[i] = c.need_codes[i];
                best_vals[i] = c.need_values[i];
            }
            best_ded = c.need_dedicated;
            best_slots = slots ? std::max<uint64_t>(c.need_slots + c.need_slots / 2 + 64, 256) : 0;
            best_pt = pt;
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
    const uint64_t cap_items = cap_arena / best_C + 2ull * n_trees + 1024;

    // launch shapes: the given ones, or the fastest of a few on generation 0
    // with the chosen chunk: level 0's warps per SM x window entries (deeper
    // windows spill less, more warps hide more latency; the sum is bounded
    // by shared memory), then, when some tree has upper levels, the upper
    // levels' window (with as many warps as fit, at most 16)
    int maxsm = 0;
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, E.device);
    auto upper_warps = [&](uint32_t Ku) {
        uint32_t w = 16;
        while (w > 1 && gpk::eval_smem_bytes(E.lanes, (int)w, (int)Ku, true, E.rows) > (size_t)maxsm) --w;
        return w;
    };
    uint32_t shape_k = 0;
    auto time_shape = [&](uint32_t W, uint32_t K, uint32_t Ku, bool upper, float *ms) -> gp_status {
        gp_status e = E.set_shape(W, K, upper_warps(Ku), Ku, E.Wr, E.Kr);
        if (e) return e;
        if ((e = E.set_workspace(best_C, cap_codes, cap_vals, cap_ded, cap_items, best_slots, best_pt))) return e;
        float t = -1.f;
        for (int rep = 0; rep < 2; ++rep) t = time_eval(G, cs);
        RunDev R{};
        if ((e = E.read_run(G->run, &R, cs))) return e;
        if (t < 0.f || R.err) return R.err ? map_err(R.err, 0) : GP_ECUDA;
        if (shape_k < 8) {
            G->info.autotune_shape[shape_k] = upper ? (upper_warps(Ku) << 16) | 0x8000u | Ku : (W << 16) | K;
            G->info.autotune_shape_ms[shape_k] = t;
            ++shape_k;
        }
        *ms = t;
        return GP_OK;
    };
    // (the engine's starting shape already fits this problem's leaf table)
    uint32_t bW = params->warps_per_cta ? params->warps_per_cta : E.W;
    uint32_t bK = params->window_entries ? params->window_entries : E.K;
    uint32_t bKu = params->upper_window_entries ? params->upper_window_entries : 128;
    if (!params->warps_per_cta && !params->window_entries) {
        step = "autotune level-0 shape";
        const uint32_t cand[3][2] = {{32, 32}, {28, 36}, {16, 64}};
        float best = -1.f;
        uint32_t done[3] = {0, 0, 0};
        for (int i = 0; i < 3; ++i) {
            uint32_t W = cand[i][0];
            const uint32_t K = cand[i][1];
            // fewer warps when a large leaf table leaves less shared memory
            while (W > 1 && gpk::eval_smem_bytes(E.lanes, (int)W, (int)K, false, E.rows) > (size_t)maxsm) --W;
            if (gpk::eval_smem_bytes(E.lanes, (int)W, (int)K, false, E.rows) > (size_t)maxsm) continue;
            if (done[0] == ((W << 16) | K) || done[1] == ((W << 16) | K)) continue;
            done[i] = (W << 16) | K;
            float ms = 0.f;
            if ((st = time_shape(W, K, bKu, false, &ms))) return fail(st);
            if (best < 0.f || ms < best) {
                best = ms;
                bW = W;
                bK = K;
            }
        }
    }
    if (!params->upper_window_entries && maxn > best_C) {
        step = "autotune upper shape";
        const uint32_t cand[3] = {128, 96, 192};
        float best = -1.f;
        for (uint32_t Ku : cand) {
            float ms = 0.f;
            if ((st = time_shape(bW, bK, Ku, true, &ms))) return fail(st);
            if (best < 0.f || ms < best) {
                best = ms;
                bKu = Ku;
            }
        }
    }
    step = "launch shape";
    if ((st = E.set_shape(bW, bK, upper_warps(bKu), bKu, E.Wr, E.Kr))) return fail(st);
    step = "final workspace";
    if ((st = E.set_workspace(best_C, cap_codes, cap_vals, cap_ded, cap_items, best_slots, best_pt))) return fail(st);
    step = "generation 0 evaluation";
    if ((st = E.enqueue(kModeEvaluate, {G->run}, cs, false, nullptr))) return fail(st);
    {
        RunDev R{};
        if ((st = E.read_run(G->run, &R, cs))) return fail(st);
        if (R.err && verbose && verbose[0] == '1') {
            BatchCtl c2{};
            E.read_ctl(&c2, cs);
            std::fprintf(stderr, "gp_generation_create: generation 0: run error bits 0x%x, batch error 0x%x, "
                         "eval error 0x%x, slots %llu (need %llu) x %u entries, items %llu (need %llu)\n", R.err,
                         c2.err, c2.eval_err[0], (unsigned long long)E.w.cap_slots,
                         (unsigned long long)c2.need_slots, E.w.fz_cap_pt, (unsigned long long)E.w.cap_items,
                         (unsigned long long)c2.need_items);
        }
        if (R.err) return fail(map_err(R.err, 0));
        G->info.levels = R.levels;
    }
    // Level budget: generation 0's levels and two more (the last level of a
    // generation finishes every open tree, so any budget is correct; a
    // generation that uses them all widens it).  A given max_levels is fixed.
    G->auto_levels = params->max_levels == 0;
    if (G->auto_levels) E.levels_max = std::min<uint32_t>(G->levels_cap, std::max<uint32_t>(3, G->info.levels + 2));
    step = "graph capture";
    E.levels_cap_graph = params->max_levels ? params->max_levels : G->levels_cap;
    if (G->use_graph && (st = E.capture(kModeGenerate))) return fail(st);
    G->info.n_trees = n_trees;
    G->info.chunk_nodes = best_C;
    G->info.graph = G->use_graph ? 1u : 0u;
    G->info.kernels_per_generation = G->use_graph ? E.kernels_per_batch[kModeGenerate] : 0;
    G->info.warps_per_cta = E.W;
    G->info.window_entries = E.K;
    G->info.upper_warps = E.Wu;
    G->info.upper_window_entries = E.Ku;
    G->info.rope_warps = E.Wr;
    G->info.rope_window_entries = E.Kr;
    G->info.arena_bytes = cap_arena;
    G->info.workspace_codes = E.w.cap_codes[0] + E.w.cap_codes[1];
    G->info.workspace_values = E.w.cap_values[0] + E.w.cap_values[1];
    G->last = cs;
    *out = G;
    return GP_OK;
}

gp_status gp_generation_step(gp_generation *G, uint32_t n, void *cuda_stream)
{
    if (!G) return GP_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    order_after_last(G, s);
    gp_status st = GP_OK;
    for (uint32_t k = 0; k < n && !st; ++k) {
        uint32_t nl = 0;
        if (G->use_graph) {
            st = G->eng.launch_graph(kModeGenerate, {G->run}, s);
            nl = G->eng.graph_kernels(kModeGenerate, std::max<uint32_t>(G->info.levels, 1));
        } else {
            st = G->eng.enqueue(kModeGenerate, {G->run}, s, false, &nl);
            G->info.kernels_per_generation = nl;
        }
        gpk::note_launches(nl);
    }
    G->last = s;
    return st;
}

gp_status gp_generation_rewind(gp_generation *G, void *cuda_stream)
{
    if (!G) return GP_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    RunDev R{};
    gp_status st = G->eng.read_run(G->run, &R, G->last);    // synchronises the previous stream
    if (st) return st;
    if (R.gen == 0 || R.err) return GP_EINVAL;
    order_after_last(G, s);
    st = G->eng.rewind(G->run, s);
    G->last = s;
    return st;
}

gp_status gp_generation_recover(gp_generation *G, void *cuda_stream)
{
    if (!G) return GP_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    Engine &E = G->eng;
    RunDev R{};
    gp_status st = E.read_run(G->run, &R, G->last);
    if (st) return st;
    const uint32_t room = kGErrArena | kGErrWork | kGErrItems | kGErrSpill | kGErrSlots;
    if (!R.err || (R.err & ~room)) return GP_EINVAL;
    if (R.err & kGErrArena) {
        const uint64_t cap = 2 * G->info.arena_bytes;
        const uint64_t need = 2 * ((cap + 255) & ~255ull);
        if (E.heap_largest_free() < need && (st = E.grow_heap(E.heap_bytes + need))) return st;
        if ((st = E.grow_run(G->run, cap, s))) return st;
        G->info.arena_bytes = cap;
    }
    if (R.err & kGErrSlots) {
        // a slot's value entries overflowed: twice the entries per slot (and
        // room for every candidate), or (at C entries already) no fused
        // chunks at all
        BatchCtl c{};
        if ((st = E.read_ctl(&c, s))) return st;
        const uint64_t slots = std::max<uint64_t>(E.w.cap_slots, c.need_slots + c.need_slots / 2);
        if (E.w.fz_cap_pt < E.w.C) st = E.set_slots(slots, 2 * E.w.fz_cap_pt);
        else st = E.set_slots(0, 0);
        if (st) return st;
    }
    if (R.err & (kGErrWork | kGErrItems | kGErrSpill)) {
        BatchCtl c{};
        if ((st = E.read_ctl(&c, s))) return st;
        // Only what ran out grows: to 1.5x the largest need recorded (the
        // failing level records its need before it stops), at least double.
        auto grown = [](uint64_t cap, uint64_t need, uint64_t slack) {
            return need + slack > cap ? std::max<uint64_t>(2 * cap, need + need / 2 + slack) : cap;
        };
        uint64_t codes[2], vals[2];
        for (int k = 0; k < 2; ++k) {
            codes[k] = grown(E.w.cap_codes[k], c.need_codes[k], 48);
            vals[k] = grown(E.w.cap_values[k], c.need_values[k], 0);
        }
        const uint64_t ded = grown(E.w.cap_dedicated, c.need_dedicated, 0);
        const uint64_t items = grown(E.w.cap_items, c.need_items, 0);
        bool same = ded == E.w.cap_dedicated && items == E.w.cap_items;
        for (int k = 0; k < 2; ++k) same = same && codes[k] == E.w.cap_codes[k] && vals[k] == E.w.cap_values[k];
        if (same) return GP_EINVAL;              // nothing recorded as short: not a sizing failure
        if ((st = E.set_workspace(E.w.C, codes, vals, ded, items, E.w.cap_slots, E.w.fz_cap_pt))) return st;
        G->info.workspace_codes = E.w.cap_codes[0] + E.w.cap_codes[1];
        G->info.workspace_values = E.w.cap_values[0] + E.w.cap_values[1];
    }
    if ((st = E.clear_error(G->run, s))) return st;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GP_ECUDA;
    if (G->use_graph && !E.exec[kModeGenerate] && (st = E.capture(kModeGenerate))) return st;
    G->last = s;
    return GP_OK;
}

gp_status gp_generation_fitness(gp_generation *G, float *fitness, float *case_values, uint32_t *hits)
{
    if (!G) return GP_EINVAL;
    RunDev R{};
    gp_status st = sync_run(G, &R);
    if (st) return st;
    const RunBuf &B = R.buf[R.cur];
    if (fitness && cudaMemcpy(fitness, B.fit, sizeof(float) * G->n, cudaMemcpyDeviceToHost)) return GP_ECUDA;
    if (case_values && cudaMemcpy(case_values, B.vals, sizeof(float) * (uint64_t)G->n * G->eng.n_cases,
                                  cudaMemcpyDeviceToHost))
        return GP_ECUDA;
    if (hits && cudaMemcpy(hits, B.hits, sizeof(uint32_t) * G->n, cudaMemcpyDeviceToHost)) return GP_ECUDA;
    return GP_OK;
}

gp_status gp_generation_records(gp_generation *G, gp_xo *records)
{
    if (!G || !records) return GP_EINVAL;
    RunDev R{};
    gp_status st = sync_run(G, &R);
    if (st) return st;
    if (R.gen == 0) return GP_EINVAL;      // no step has made the current population
    return G->eng.copy_records(records, 0, G->n);
}

gp_status gp_generation_trees(gp_generation *G, uint64_t *offsets, uint8_t *nodes, uint64_t cap)
{
    if (!G || !offsets) return GP_EINVAL;
    RunDev R{};
    gp_status st = sync_run(G, &R);
    if (st) return st;
    return G->eng.copy_trees(R.buf[R.cur], G->n, offsets, nodes, cap);
}

gp_status gp_generation_tree_read(gp_generation *G, uint32_t tree, uint8_t *nodes, uint64_t cap,
                                  uint64_t *n_nodes)
{
    if (!G || !n_nodes || tree >= G->n) return GP_EINVAL;
    RunDev R{};
    gp_status st = sync_run(G, &R);
    if (st) return st;
    return G->eng.copy_tree(R.buf[R.cur], tree, nodes, cap, n_nodes);
}

gp_status gp_generation_get_info(gp_generation *G, gp_generation_info *info)
{
    if (!G || !info) return GP_EINVAL;
    RunDev R{};
    sync_run(G, &R);                   // the info describes a failed run as well
    G->info.total_nodes = 0;
    if (!R.err) {
        std::vector<uint64_t> hz(G->n);
        if (cudaMemcpy(hz.data(), R.buf[R.cur].size, sizeof(uint64_t) * G->n, cudaMemcpyDeviceToHost))
            return GP_ECUDA;
        for (uint64_t z : hz) G->info.total_nodes += z;
    }
    *info = G->info;
    return GP_OK;
}

void gp_generation_destroy(gp_generation *G) { delete G; }

gp_status gp_select(const float *d_fitness, const uint64_t *d_sizes, uint32_t n_pop, uint64_t seed,
                    uint32_t generation, uint32_t child_lo, uint32_t n_children, uint32_t tournament_size,
                    gp_xo *d_out, void *cuda_stream)
{
    if (n_children == 0) return GP_OK;
    if (!d_fitness || !d_sizes || !d_out || n_pop == 0 || tournament_size < 1 || tournament_size > 32)
        return GP_EINVAL;
    if ((uint64_t)child_lo + n_children > (1ull << 28) || generation >= (1u << 24)) return GP_EINVAL;
    const cudaError_t e = gpe::launch_select_range(d_fitness, d_sizes, n_pop, seed, generation, child_lo, n_children,
                                                   tournament_size, d_out, static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return GP_ECUDA;
    gpk::note_launches(1);
    return GP_OK;
}

}  // extern "C"
