// gp_server: a serving loop for many independent GP runs on one GPU.
//
// Runs live in the engine's device heap (admitted in the order they were
// opened, while their two population buffers fit the HBM budget).  Clients
// submit "advance run r by k generations" requests from any thread.  A
// scheduler thread repeatedly forms a batch of the runs that have pending
// requests (oldest request first, within the batch limits), advances each by
// one generation in a single engine batch, and completes the requests whose
// generations are done; requests arriving meanwhile join the next batch
// (continuous batching at generation granularity).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "gp_engine.cuh"

using namespace gpe;

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Req {
    uint64_t id = 0, run = 0;
    uint32_t remaining = 0;
    Clock::time_point t_submit, t_first;
    bool started = false, done = false;
    gp_server_result res{};
};

enum RunState { kWaiting, kReady, kFailed };

struct Run {
    uint64_t id = 0;
    RunState state = kWaiting;
    uint32_t slot = 0;                 // engine run index once admitted
    uint32_t n = 0, tsize = 7;
    uint64_t nodes = 0, arena = 0, seed = 0;
    std::vector<uint8_t> h_nodes;      // the initial trees, until admitted
    std::vector<uint64_t> h_offs;
    const gp_population *src = nullptr; // or trees of a device population, until admitted
    std::vector<uint32_t> src_trees;
    std::deque<uint64_t> pending;      // request ids, oldest first
    bool in_batch = false;
    bool needs_room = false;           // outgrew its buffers; waits for a larger pair
    gp_status fail_status = GP_OK;
};

gp_status map_err(uint32_t err)
{
    if (!err) return GP_OK;
    if (err & (kGErrLimit | kGErrGen)) return GP_ELIMIT;
    if (err & (kGErrArena | kGErrWork | kGErrItems | kGErrSpill | kGErrLevels)) return GP_ENOMEM;
    if (err & kGErrExtent) return GP_EMALFORMED;
    return GP_ECUDA;
}

}  // namespace

struct gp_server {
    Engine eng;
    gp_server_params prm{};
    uint64_t max_nodes = 0;                  // the problem's node limit
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    uint64_t next_run = 1, next_req = 1;
    std::map<uint64_t, Run> runs;            // by id: opening order
    std::map<uint64_t, Req> reqs;
    std::vector<double> lat;                 // latencies of completed requests (ms)
    gp_server_stats st{};
    uint64_t runs_in_batches = 0;
    uint32_t limit_runs = 0;                 // batch size cap (halved after a workspace overflow)
    cudaStream_t stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<RunDev> table;
};

namespace {

void fail_run(gp_server *S, Run &R, gp_status status)
{
    R.state = kFailed;
    R.fail_status = status;
    for (uint64_t q : R.pending) {
        Req &rq = S->reqs[q];
        rq.done = true;
        rq.res.status = status;
        rq.res.latency_ms = ms_between(rq.t_submit, Clock::now());
    }
    R.pending.clear();
}

// Admit waiting runs in opening order while the heap holds them (under the lock).
void admit(gp_server *S)
{
    for (auto &kv : S->runs) {
        Run &R = kv.second;
        if (R.state != kWaiting) continue;
        uint32_t slot = 0;
        gp_status st = S->eng.open_run(R.n, R.arena, R.seed, R.tsize, S->max_nodes, &slot);
        if (st == GP_ENOMEM) break;                          // first come, first served
        if (!st)
            st = R.src ? S->eng.load_run_from(slot, R.src, R.src_trees.data(), S->stream)
                       : S->eng.load_run(slot, R.h_nodes.data(), R.h_offs.data(), S->stream);
        if (!st) st = S->eng.enqueue(kModeEvaluate, {slot}, S->stream, false, nullptr);
        RunDev D{};
        if (!st) st = S->eng.read_run(slot, &D, S->stream);
        if (!st && D.err) st = map_err(D.err);
        if (st) {
            S->eng.close_run(slot);
            fail_run(S, R, st);
            continue;
        }
        R.slot = slot;
        R.state = kReady;
        R.nodes = D.nodes;
        std::vector<uint8_t>().swap(R.h_nodes);
        std::vector<uint64_t>().swap(R.h_offs);
        std::vector<uint32_t>().swap(R.src_trees);
        R.src = nullptr;
        ++S->st.runs_admitted;
    }
}

// Runs whose children outgrew their buffers get buffers twice as large when
// the heap has room (the failed generation is then made again); until then
// they wait.
void regrow(gp_server *S)
{
    for (auto &kv : S->runs) {
        Run &R = kv.second;
        if (R.state != kReady || !R.needs_room) continue;
        if (S->eng.grow_run(R.slot, 2 * R.arena, S->stream) != GP_OK) continue;
        S->eng.clear_error(R.slot, S->stream);
        cudaStreamSynchronize(S->stream);
        R.arena *= 2;
        R.needs_room = false;
        ++S->st.regrown;
    }
}

// Best tree of a run's current population (lowest MAE, NaN worst, first on ties).
gp_status best_of(gp_server *S, const Run &R, const RunDev &D, gp_server_result *res)
{
    std::vector<float> fit(R.n);
    std::vector<uint32_t> hits(R.n);
    const RunBuf &B = D.buf[D.cur];
    if (cudaMemcpy(fit.data(), B.fit, sizeof(float) * R.n, cudaMemcpyDeviceToHost) ||
        cudaMemcpy(hits.data(), B.hits, sizeof(uint32_t) * R.n, cudaMemcpyDeviceToHost))
        return GP_ECUDA;
    uint32_t best = 0;
    for (uint32_t t = 1; t < R.n; ++t) {
        const float a = std::isnan(fit[t]) ? INFINITY : fit[t];
        const float b = std::isnan(fit[best]) ? INFINITY : fit[best];
        if (a < b) best = t;
    }
    res->best_tree = best;
    res->best_fitness = fit[best];
    res->best_hits = hits[best];
    return GP_OK;
}

void worker_main(gp_server *S)
{
    cudaSetDevice(S->eng.device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        regrow(S);
        admit(S);
        // the batch: runs with pending requests, oldest request first
        std::vector<Run *> cand;
        for (auto &kv : S->runs) {
            Run &R = kv.second;
            if (R.state == kReady && !R.needs_room && !R.pending.empty()) cand.push_back(&R);
        }
        std::sort(cand.begin(), cand.end(),
                  [](const Run *a, const Run *b) { return a->pending.front() < b->pending.front(); });
        std::vector<Run *> batch;
        std::vector<uint32_t> slots;
        uint64_t trees = 0, nodes = 0;
        for (Run *R : cand) {
            if (batch.size() >= S->limit_runs) break;
            if (trees + R->n > S->prm.max_batch_trees) continue;
            if (!batch.empty() && nodes + R->nodes > S->prm.max_batch_nodes) continue;
            batch.push_back(R);
            slots.push_back(R->slot);
            trees += R->n;
            nodes += R->nodes;
        }
        if (batch.empty()) {
            S->cv_work.wait_for(lk, std::chrono::milliseconds(20));
            continue;
        }
        const Clock::time_point t0 = Clock::now();
        for (Run *R : batch) {
            R->in_batch = true;
            Req &q = S->reqs[R->pending.front()];
            if (!q.started) {
                q.started = true;
                q.t_first = t0;
            }
        }
        gp_status st = GP_OK;
        cudaEventRecord(S->ev0, S->stream);
        uint32_t nl = 0;
        if (S->prm.use_graph) st = S->eng.launch_graph(kModeGenerate, slots, S->stream);
        else st = S->eng.enqueue(kModeGenerate, slots, S->stream, false, &nl);
        cudaEventRecord(S->ev1, S->stream);
        lk.unlock();
        const cudaError_t e = cudaEventSynchronize(S->ev1);
        lk.lock();
        BatchCtl c{};
        if (!st && e != cudaSuccess) st = GP_ECUDA;
        if (!st) st = S->eng.read_ctl(&c, S->stream);
        gpk::note_launches(S->prm.use_graph ? S->eng.graph_kernels(kModeGenerate, std::max<uint32_t>(c.levels, 1)) : nl);
        if (!st && cudaMemcpy(S->table.data(), S->eng.runs_dev, sizeof(RunDev) * S->table.size(),
                              cudaMemcpyDeviceToHost) != cudaSuccess)
            st = GP_ECUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, S->ev0, S->ev1);
        ++S->st.batches;
        S->st.device_ms += ms;
        S->runs_in_batches += batch.size();
        bool overflow = false, slots_short = false;
        for (Run *R : batch) {
            R->in_batch = false;
            if (st) {
                fail_run(S, *R, st);
                continue;
            }
            const RunDev &D = S->table[R->slot];
            const uint32_t batch_bits = kGErrWork | kGErrItems | kGErrSpill | kGErrLevels;
            if (D.err == kGErrSlots) {
                // a fused chunk's slot ran out of value entries: the batch
                // goes again once the slots are larger (or off)
                S->eng.clear_error(R->slot, S->stream);
                slots_short = true;
                ++S->st.retries;
                continue;
            }
            if (D.err) {
                if (D.err == kGErrArena && 2 * R->arena + 512 <= S->prm.hbm_budget_bytes / 2) {
                    // outgrew its buffers: larger ones when there is room
                    R->needs_room = true;
                    continue;
                }
                if ((D.err & batch_bits) && !(D.err & ~batch_bits) && batch.size() > 1) {
                    // the batch did not fit the workspace: this run goes again
                    // in a smaller batch
                    S->eng.clear_error(R->slot, S->stream);
                    overflow = true;
                    ++S->st.retries;
                } else {
                    fail_run(S, *R, map_err(D.err));
                }
                continue;
            }
            R->nodes = D.nodes;
            ++S->st.run_generations;
            Req &q = S->reqs[R->pending.front()];
            if (--q.remaining == 0) {
                q.done = true;
                q.res.generation = D.gen;
                q.res.total_nodes = D.nodes;
                q.res.status = best_of(S, *R, D, &q.res);
                const Clock::time_point t1 = Clock::now();
                q.res.latency_ms = ms_between(q.t_submit, t1);
                q.res.queue_ms = ms_between(q.t_submit, q.t_first);
                S->lat.push_back(q.res.latency_ms);
                ++S->st.requests_done;
                R->pending.pop_front();
            }
        }
        if (!st) {
            S->st.child_nodes += c.child_nodes;
            S->st.most_level_codes = std::max<uint64_t>(c.need_codes[0], c.need_codes[1]);
            S->st.most_level_values = std::max<uint64_t>(c.need_values[0], c.need_values[1]);
        }
        if (slots_short) {
            // twice the value entries per slot, up to the chunk size; then
            // every multi-chunk tree is planned
            cudaStreamSynchronize(S->stream);
            Engine &E = S->eng;
            gp_status g = E.w.fz_cap_pt < E.w.C ? E.set_slots(E.w.cap_slots, 2 * E.w.fz_cap_pt) : E.set_slots(0, 0);
            if (!g && S->prm.use_graph) g = E.capture(kModeGenerate);
            if (g) {
                for (Run *R : batch) fail_run(S, *R, g);
            }
        }
        if (overflow) {
            cudaStreamSynchronize(S->stream);
            S->limit_runs = std::max<uint32_t>(1, (uint32_t)batch.size() / 2);
        } else if (S->limit_runs < S->prm.max_batch_runs) {
            S->limit_runs = std::min<uint32_t>(S->prm.max_batch_runs, S->limit_runs * 2);
        }
        S->cv_done.notify_all();
    }
}

// Wait (under the lock) until run id has no pending request and is not in
// a batch; false if it does not exist.
bool wait_idle(gp_server *S, std::unique_lock<std::mutex> &lk, uint64_t id)
{
    S->cv_done.wait(lk, [&] {
        auto it = S->runs.find(id);
        return it == S->runs.end() || (it->second.pending.empty() && !it->second.in_batch);
    });
    return S->runs.count(id) != 0;
}

}  // namespace

extern "C" {

gp_status gp_server_create(const gp_problem *problem, const gp_server_params *params, gp_server **out)
{
    if (!problem || !params || !out) return GP_EINVAL;
    if (problem->n_cases == 0 || problem->n_cases > gpk::kMaxCases || problem->n_consts > gpk::kMaxConsts) return GP_EINVAL;
    gp_server_params p = *params;
    if (p.max_runs == 0 || p.max_runs > 4096 || p.max_batch_trees == 0 || p.hbm_budget_bytes < (1u << 20))
        return GP_EINVAL;
    if (p.max_batch_runs == 0 || p.max_batch_runs > p.max_runs) p.max_batch_runs = p.max_runs;
    if (!p.chunk_nodes) p.chunk_nodes = 8192;
    if (p.chunk_nodes % 16 || p.chunk_nodes < 256 || p.chunk_nodes > 65536) return GP_EINVAL;
    if (!p.max_batch_nodes) p.max_batch_nodes = std::max<uint64_t>(p.hbm_budget_bytes / 4, 1u << 20);
    gp_server *S = new (std::nothrow) gp_server();
    if (!S) return GP_ENOMEM;
    S->prm = p;
    S->max_nodes = problem->max_tree_nodes;
    S->limit_runs = p.max_batch_runs;
    gp_status st = S->eng.init(problem, p.hbm_budget_bytes, p.max_runs, p.max_batch_trees, 8);
    const uint64_t N = p.max_batch_nodes;
    uint64_t codes[2], vals[2];
    codes[0] = p.workspace_codes ? p.workspace_codes : std::max<uint64_t>(N / 12, 1u << 20);
    vals[0] = p.workspace_values ? p.workspace_values : std::max<uint64_t>(N / 33, 1u << 18);
    codes[1] = std::max<uint64_t>(codes[0] / 8, 1u << 20);
    vals[1] = std::max<uint64_t>(vals[0] / 8, 1u << 18);
    // fused chunk slots for trees of 2..8 chunks (taken in tree order while
    // they last, the rest planned): one per chunk of about an eighth of a
    // full batch, at most 8192
    const uint64_t fz_slots = std::max<uint64_t>(256, std::min<uint64_t>(N / p.chunk_nodes / 8, 8192));
    // dedicated spill for upper-tree finals above one chunk: a sixteenth of
    // the code workspace (entries of 8 B per lane each)
    if (!st) st = S->eng.set_workspace(p.chunk_nodes, codes, vals, std::max<uint64_t>(codes[0] / 16, 1u << 20),
                                       N / p.chunk_nodes + p.max_batch_trees + 1024, fz_slots);
    if (!st && p.use_graph) st = S->eng.capture(kModeGenerate);
    if (!st && (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreate(&S->ev0) != cudaSuccess || cudaEventCreate(&S->ev1) != cudaSuccess))
        st = GP_ECUDA;
    if (st) {
        delete S;
        return st;
    }
    S->table.resize(p.max_runs);
    S->st.heap_bytes = p.hbm_budget_bytes;
    S->worker = std::thread(worker_main, S);
    *out = S;
    return GP_OK;
}

gp_status gp_server_open_run(gp_server *S, const gp_generation_params *params, uint32_t n_trees,
                             const uint8_t *nodes, const uint64_t *offsets, uint64_t *run_id)
{
    if (!S || !params || !nodes || !offsets || !run_id || n_trees == 0) return GP_EINVAL;
    if (params->tournament_size < 1 || params->tournament_size > 32) return GP_EINVAL;
    if (n_trees > S->prm.max_batch_trees || offsets[0] != 0) return GP_EINVAL;
    uint64_t used = 0;
    for (uint32_t t = 0; t < n_trees; ++t) {
        if (offsets[t + 1] <= offsets[t]) return GP_EINVAL;
        used = (used + (offsets[t + 1] - offsets[t]) + 15) & ~15ull;
    }
    Run R;
    R.n = n_trees;
    R.tsize = params->tournament_size;
    R.seed = params->seed;
    R.arena = params->arena_bytes ? params->arena_bytes : 2 * used + 16ull * n_trees + (1u << 20);
    if (R.arena < used + 64) return GP_ENOMEM;
    if (2 * ((R.arena + 255) & ~255ull) > S->prm.hbm_budget_bytes) return GP_ENOMEM;   // can never fit
    R.h_nodes.assign(nodes, nodes + offsets[n_trees]);
    R.h_offs.assign(offsets, offsets + n_trees + 1);
    R.nodes = offsets[n_trees];
    {
        std::lock_guard<std::mutex> lk(S->mu);
        R.id = S->next_run++;
        *run_id = R.id;
        S->runs.emplace(R.id, std::move(R));
    }
    S->cv_work.notify_all();
    return GP_OK;
}

gp_status gp_server_open_run_from(gp_server *S, const gp_generation_params *params, const gp_population *src,
                                  uint32_t n_trees, const uint32_t *trees, uint64_t *run_id)
{
    if (!S || !params || !src || !trees || !run_id || n_trees == 0) return GP_EINVAL;
    if (params->tournament_size < 1 || params->tournament_size > 32) return GP_EINVAL;
    if (n_trees > S->prm.max_batch_trees) return GP_EINVAL;
    gp_population_info pi{};
    if (gp_population_get_info(src, &pi) != GP_OK) return GP_EINVAL;
    if (pi.n_cases != S->eng.n_cases) return GP_EINVAL;
    uint64_t used = 0, nodes = 0;
    for (uint32_t k = 0; k < n_trees; ++k) {
        uint64_t z = 0;
        if (trees[k] >= pi.n_trees || gp_tree_size(src, trees[k], &z) != GP_OK) return GP_EINVAL;
        used = (used + z + 15) & ~15ull;
        nodes += z;
    }
    Run R;
    R.n = n_trees;
    R.tsize = params->tournament_size;
    R.seed = params->seed;
    R.arena = params->arena_bytes ? params->arena_bytes : 2 * used + 16ull * n_trees + (1u << 20);
    if (R.arena < used + 64) return GP_ENOMEM;
    if (2 * ((R.arena + 255) & ~255ull) > S->prm.hbm_budget_bytes) return GP_ENOMEM;   // can never fit
    R.src = src;
    R.src_trees.assign(trees, trees + n_trees);
    R.nodes = nodes;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        R.id = S->next_run++;
        *run_id = R.id;
        S->runs.emplace(R.id, std::move(R));
    }
    S->cv_work.notify_all();
    return GP_OK;
}

gp_status gp_server_submit(gp_server *S, uint64_t run_id, uint32_t n_generations, uint64_t *request_id)
{
    if (!S || !request_id || n_generations == 0) return GP_EINVAL;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->runs.find(run_id);
        if (it == S->runs.end()) return GP_EINVAL;
        if (it->second.state == kFailed) return it->second.fail_status;
        Req q;
        q.id = S->next_req++;
        q.run = run_id;
        q.remaining = n_generations;
        q.t_submit = Clock::now();
        q.res.run_id = run_id;
        q.res.request_id = q.id;
        q.res.status = GP_OK;
        it->second.pending.push_back(q.id);
        *request_id = q.id;
        S->reqs.emplace(q.id, q);
    }
    S->cv_work.notify_all();
    return GP_OK;
}

gp_status gp_server_wait(gp_server *S, uint64_t request_id, double timeout_ms, gp_server_result *result)
{
    if (!S) return GP_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(request_id);
    if (it == S->reqs.end()) return GP_EINVAL;
    // A request another waiter collected meanwhile counts as done here (and
    // is reported as unknown below): looking it up never re-creates it.
    auto done = [&] {
        auto f = S->reqs.find(request_id);
        return f == S->reqs.end() || f->second.done;
    };
    if (timeout_ms < 0) S->cv_done.wait(lk, done);
    else if (!S->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), done))
        return GP_ETIMEOUT;
    it = S->reqs.find(request_id);
    if (it == S->reqs.end()) return GP_EINVAL;
    if (result) *result = it->second.res;
    S->reqs.erase(it);                              // a completed request is collected once
    return GP_OK;
}

gp_status gp_server_run_fitness(gp_server *S, uint64_t run_id, float *fitness, float *case_values, uint32_t *hits)
{
    if (!S) return GP_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    if (!wait_idle(S, lk, run_id)) return GP_EINVAL;
    const Run &R = S->runs[run_id];
    if (R.state == kFailed) return R.fail_status;
    if (R.state != kReady) return GP_EINVAL;
    RunDev D{};
    gp_status st = S->eng.read_run(R.slot, &D, S->stream);
    if (st) return st;
    const RunBuf &B = D.buf[D.cur];
    if (fitness && cudaMemcpy(fitness, B.fit, sizeof(float) * R.n, cudaMemcpyDeviceToHost)) return GP_ECUDA;
    if (case_values && cudaMemcpy(case_values, B.vals, sizeof(float) * (uint64_t)R.n * S->eng.n_cases,
                                  cudaMemcpyDeviceToHost))
        return GP_ECUDA;
    if (hits && cudaMemcpy(hits, B.hits, sizeof(uint32_t) * R.n, cudaMemcpyDeviceToHost)) return GP_ECUDA;
    return GP_OK;
}

gp_status gp_server_run_trees(gp_server *S, uint64_t run_id, uint64_t *offsets, uint8_t *nodes, uint64_t cap)
{
    if (!S || !offsets) return GP_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    if (!wait_idle(S, lk, run_id)) return GP_EINVAL;
    const Run &R = S->runs[run_id];
    if (R.state == kFailed) return R.fail_status;
    if (R.state != kReady) return GP_EINVAL;
    RunDev D{};
    gp_status st = S->eng.read_run(R.slot, &D, S->stream);
    if (st) return st;
    return S->eng.copy_trees(D.buf[D.cur], R.n, offsets, nodes, cap);
}

gp_status gp_server_close_run(gp_server *S, uint64_t run_id)
{
    if (!S) return GP_EINVAL;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        auto it = S->runs.find(run_id);
        if (it == S->runs.end()) return GP_EINVAL;
        if (it->second.state == kWaiting) {          // never admitted: its requests cannot run
            fail_run(S, it->second, GP_EINVAL);
            S->runs.erase(it);
            S->cv_done.notify_all();
            return GP_OK;
        }
        if (!wait_idle(S, lk, run_id)) return GP_EINVAL;
        Run &R = S->runs[run_id];
        if (R.state == kReady) S->eng.close_run(R.slot);
        S->runs.erase(run_id);
    }
    S->cv_work.notify_all();
    return GP_OK;
}

gp_status gp_server_get_stats(gp_server *S, gp_server_stats *out)
{
    if (!S || !out) return GP_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    gp_server_stats s = S->st;
    s.mean_runs_per_batch = s.batches ? (double)S->runs_in_batches / (double)s.batches : 0.0;
    std::vector<double> l = S->lat;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        // nearest rank: the ceil(q n)-th smallest request latency
        auto rank = [&](double q) {
            const size_t k = (size_t)std::ceil(q * (double)l.size());
            return l[std::min(l.size() - 1, k ? k - 1 : 0)];
        };
        s.latency_p50_ms = rank(0.50);
        s.latency_p99_ms = rank(0.99);
    }
    s.heap_free = S->eng.heap_free();
    s.runs_waiting = 0;
    for (auto &kv : S->runs)
        if (kv.second.state == kWaiting) ++s.runs_waiting;
    *out = s;
    return GP_OK;
}

void gp_server_destroy(gp_server *S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    cudaDeviceSynchronize();
    if (S->ev0) cudaEventDestroy(S->ev0);
    if (S->ev1) cudaEventDestroy(S->ev1);
    if (S->stream) cudaStreamDestroy(S->stream);
    delete S;
}

}  // extern "C"
