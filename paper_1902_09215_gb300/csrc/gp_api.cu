// libgp host side: the C ABI of include/gp.h, population memory, the chunk /
// upper-tree level planner and kernel launches.
#include <algorithm>
#include <atomic>
#include <deque>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "gp.h"
#include "gp_internal.cuh"

using namespace gpk;

namespace {

// ---------------------------------------------------------------- profiling

std::atomic<uint64_t> g_launches{0};

struct ProfRec {
    int kind;
    cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof_pending;
double g_prof_ms[GP_KERNEL_KINDS] = {};
uint64_t g_prof_n[GP_KERNEL_KINDS] = {};

struct ProfScope {
    int kind;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(int k, cudaStream_t st) : kind(k), s(st) {
        g_launches.fetch_add(1, std::memory_order_relaxed);
        std::lock_guard<std::mutex> lk(g_prof_mu);
        if (g_prof_on && cudaEventCreate(&a) == cudaSuccess) {
            if (cudaEventCreate(&b) == cudaSuccess) {
                cudaEventRecord(a, s);
                return;
            }
            cudaEventDestroy(a);
        }
        a = b = nullptr;
    }
    ~ProfScope() {
        if (a) {
            cudaEventRecord(b, s);
            std::lock_guard<std::mutex> lk(g_prof_mu);
            g_prof_pending.push_back({kind, a, b});
        }
    }
};

// ---------------------------------------------------------------- helpers

#define CK(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return fail_cuda(e_); \
    } while (0)

gp_status fail_cuda(cudaError_t e)
{
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return GP_ENOMEM;
    }
    return GP_ECUDA;
}

std::once_flag g_pool_once[64];

void configure_pool(int dev)
{
    if (dev < 0 || dev >= 64) return;
    std::call_once(g_pool_once[dev], [dev]() {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    });
}

inline uint64_t round_up(uint64_t v, uint64_t a) { return (v + a - 1) / a * a; }

int lanes_for(uint32_t n_cases)
{
    if (n_cases <= 16) return 8;
    if (n_cases <= 32) return 16;
    if (n_cases <= 48) return 24;
    return 32;
}

// Pinned host staging for the small per-call tables (work items, crossover
// records, extent queries), so their copies are truly asynchronous.  A ring
// of pinned bytes; each region is fenced by an event recorded after the copy
// that reads it, and a region is reused only after its event completed.
class PinnedRing {
  public:
    static PinnedRing &get() {
        static PinnedRing r;
        return r;
    }
    // Copy `bytes` from host `src` to device `dst` on stream s via the ring
    // (falls back to a direct copy for large or unavailable staging).
    cudaError_t h2d(void *dst, const void *src, size_t bytes, cudaStream_t s) {
        if (bytes == 0) return cudaSuccess;
        std::lock_guard<std::mutex> lk(mu_);
        if (!base_ && !init()) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
        if (bytes > kCap / 4) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
        size_t off = (head_ + 255) & ~size_t(255);
        if (off + bytes > kCap) off = 0;
        // drop regions whose copies finished; wait for live ones that overlap
        while (!live_.empty() && cudaEventQuery(live_.front().ev) == cudaSuccess) {
            free_ev_.push_back(live_.front().ev);
            live_.pop_front();
        }
        for (auto r = live_.begin(); r != live_.end();) {
            if (r->off < off + bytes && off < r->off + r->len) {
                cudaEventSynchronize(r->ev);
                free_ev_.push_back(r->ev);
                r = live_.erase(r);
            } else {
                ++r;
            }
        }
        std::memcpy(base_ + off, src, bytes);
        cudaError_t e = cudaMemcpyAsync(dst, base_ + off, bytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return e;
        cudaEvent_t ev;
        if (!free_ev_.empty()) {
            ev = free_ev_.back();
            free_ev_.pop_back();
        } else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            return cudaStreamSynchronize(s);
        }
        cudaEventRecord(ev, s);
        live_.push_back(Region{off, bytes, ev});
        head_ = off + bytes;
        return cudaSuccess;
    }

  private:
    static constexpr size_t kCap = (size_t)64 << 20;
    struct Region {
        size_t off, len;
        cudaEvent_t ev;
    };
    bool init() {
        void *p = nullptr;
        if (cudaHostAlloc(&p, kCap, cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        base_ = static_cast<char *>(p);
        return true;
    }
    std::mutex mu_;
    char *base_ = nullptr;
    size_t head_ = 0;
    std::deque<Region> live_;
    std::vector<cudaEvent_t> free_ev_;
};

cudaError_t h2d(void *dst, const void *src, size_t bytes, cudaStream_t s)
{
    return PinnedRing::get().h2d(dst, src, bytes, s);
}

// Device allocations freed together (stream-ordered).
struct DevBufs {
    std::vector<void *> ptrs;
    cudaError_t alloc(void **p, size_t bytes, cudaStream_t s) {
        *p = nullptr;
        if (bytes == 0) bytes = 16;
        cudaError_t e = cudaMallocAsync(p, bytes, s);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    void release(cudaStream_t s) {
        for (void *p : ptrs) cudaFreeAsync(p, s);
        ptrs.clear();
    }
};

int sm_count(int dev)
{
    static std::mutex mu;
    static int cache[64] = {};
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 64 && cache[dev]) return cache[dev];
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (dev >= 0 && dev < 64) cache[dev] = v;
    return v;
}

}  // namespace

// ---------------------------------------------------------------- population

struct EvalCfg {
    uint32_t C = 0, W = 0, K = 0, Wu = 0, Ku = 0;  // chunk, warps and windows (level 0 / upper)
    uint32_t Wr = 0, Kr = 0;                       // a launch of ropes only
    int rows = (int)kLeafRows;                     // leaf table rows: 'x' + the constants
    int lanes = 0, sms = 0;
    size_t smem = 0, smem_u = 0, smem_r = 0;
};

struct gp_population {
    int device = 0;
    cudaStream_t stream = nullptr;          // stream of the last call
    // problem
    uint32_t n_cases = 0, lanes = 0, n_consts = 0;
    float div0 = 1.0f;
    uint64_t max_tree_nodes = 0, hbm_budget = 0;
    std::vector<float> hx, hy, hc;          // x, y padded to 2*lanes; constants
    // trees
    uint32_t n_trees = 0;
    uint64_t total_nodes = 0, arena_bytes = 0;
    std::vector<uint64_t> h_start, h_size;
    // Children made without a host synchronisation have their layout on the
    // device only (d_start, d_size) until a call needs it on the host; until
    // then h_bound holds an upper bound of every tree's size.
    bool host_layout = true;
    std::vector<uint64_t> h_bound;
    bool up_read = true;                     // stats.upper_ops read back since the last evaluation
    uint32_t *d_stat = nullptr;              // [0..2] device-planned evaluation: items, ropes,
                                             // slots; [3] error of a device-side layout
    bool stat_pending = false;
    // device
    DevBufs mem;
    uint8_t *d_arena = nullptr;
    uint64_t *d_start = nullptr, *d_size = nullptr;
    float *d_x = nullptr, *d_y = nullptr, *d_c = nullptr;
    float *d_fitness = nullptr, *d_values = nullptr;
    uint32_t *d_hits = nullptr, *d_err = nullptr;
    uint32_t *d_redo = nullptr;              // [1 + n_trees] trees to evaluate again
    cudaEvent_t ev = nullptr;
    bool evaluated = false;
    bool redo_pending = false;
    EvalCfg cfg{};
    gp_eval_stats stats{};
};

namespace {

uint64_t population_bytes(uint64_t arena, uint32_t n_trees, uint32_t n_cases)
{
    return arena + (uint64_t)n_trees * (16 + 8 + 4ull * n_cases) + 4096;
}

// Allocate a population's device memory for the given layout (trees not
// copied yet) and upload the problem tables.  Two allocations: the tree
// arena, and one block carved into every per-tree array and the tables
// (fewer API calls per population: children are made every generation).
gp_status alloc_population(gp_population *P, cudaStream_t s)
{
    P->stream = s;
    CK(P->mem.alloc((void **)&P->d_arena, P->arena_bytes, s));
    const uint64_t n1 = (uint64_t)P->n_trees + 1;
    uint64_t off = 0;
    auto take = [&](uint64_t bytes) {
        const uint64_t o = off;
        off = round_up(off + bytes, 256);
        return o;
    };
    const uint64_t o_pos = take(2 * sizeof(uint64_t) * n1);        // starts, then sizes
    const uint64_t o_err = take(sizeof(uint32_t) * (16 + n1));      // error words, counts, redo list
    const uint64_t o_tab = take(sizeof(float) * (4 * P->lanes + P->n_consts + 1));   // x, y, constants
    const uint64_t o_fit = take(sizeof(float) * n1);
    const uint64_t o_hits = take(sizeof(uint32_t) * n1);
    const uint64_t o_vals = take(sizeof(float) * ((uint64_t)P->n_trees * P->n_cases + 1));
    uint8_t *blk = nullptr;
    CK(P->mem.alloc((void **)&blk, off, s));
    P->d_start = reinterpret_cast<uint64_t *>(blk + o_pos);
    P->d_size = P->d_start + n1;
    P->d_err = reinterpret_cast<uint32_t *>(blk + o_err);
    P->d_stat = P->d_err + 4;                // [0..2] planned counts, [3] layout error,
                                             // [4..6] codes, operators, values sent upward
    P->d_redo = P->d_err + 12;
    P->d_x = reinterpret_cast<float *>(blk + o_tab);
    P->d_y = P->d_x + 2 * P->lanes;
    P->d_c = P->d_y + 2 * P->lanes;
    P->d_fitness = reinterpret_cast<float *>(blk + o_fit);
    P->d_hits = reinterpret_cast<uint32_t *>(blk + o_hits);
    P->d_values = reinterpret_cast<float *>(blk + o_vals);
    CK(cudaMemsetAsync(P->d_err, 0, sizeof(uint32_t) * 13, s));   // error words, counts, redo count
    std::vector<float> tab(4 * P->lanes + P->n_consts);
    std::copy(P->hx.begin(), P->hx.begin() + 2 * P->lanes, tab.begin());
    std::copy(P->hy.begin(), P->hy.begin() + 2 * P->lanes, tab.begin() + 2 * P->lanes);
    std::copy(P->hc.begin(), P->hc.begin() + P->n_consts, tab.begin() + 4 * P->lanes);
    CK(h2d(P->d_x, tab.data(), sizeof(float) * tab.size(), s));
    if (P->n_trees && P->host_layout) {
        std::vector<uint64_t> pos(2 * n1, 0);
        std::copy(P->h_start.begin(), P->h_start.end(), pos.begin());
        std::copy(P->h_size.begin(), P->h_size.end(), pos.begin() + n1);
        CK(h2d(P->d_start, pos.data(), sizeof(uint64_t) * pos.size(), s));
    }
    CK(cudaEventCreateWithFlags(&P->ev, cudaEventDisableTiming));
    return GP_OK;
}

// Brings a device-only layout (children made without a synchronisation) to
// the host: waits for the population's stream, reads starts and sizes.
gp_status ensure_host_layout(gp_population *P)
{
    if (P->host_layout) return GP_OK;
    const uint64_t n1 = (uint64_t)P->n_trees + 1;
    std::vector<uint64_t> pos(2 * n1);
    CK(cudaStreamSynchronize(P->stream));
    CK(cudaMemcpy(pos.data(), P->d_start, sizeof(uint64_t) * 2 * n1, cudaMemcpyDeviceToHost));
    uint32_t lerr = 0;
    CK(cudaMemcpy(&lerr, P->d_stat + 3, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (lerr) return GP_EMALFORMED;
    P->h_start.assign(pos.begin(), pos.begin() + P->n_trees);
    P->h_size.assign(pos.begin() + n1, pos.begin() + n1 + P->n_trees);
    P->total_nodes = 0;
    for (uint64_t z : P->h_size) P->total_nodes += z;
    P->host_layout = true;
    P->h_bound.clear();
    return GP_OK;
}

// 16-byte aligned starts for the given sizes.
void layout_trees(gp_population *P)
{
    uint64_t pos = 0;
    P->h_start.resize(P->n_trees);
    P->total_nodes = 0;
    for (uint32_t t = 0; t < P->n_trees; ++t) {
        P->h_start[t] = pos;
        pos = round_up(pos + P->h_size[t], 16);
        P->total_nodes += P->h_size[t];
    }
    P->arena_bytes = pos + 64;                // padding for 16-code groups and word loads
}

void destroy(gp_population *P)
{
    if (!P) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(P->device);
    P->mem.release(P->stream);
    if (P->ev) cudaEventDestroy(P->ev);
    cudaSetDevice(cur);
    delete P;
}

struct Stream {
    cudaStream_t s;
    explicit Stream(void *p) : s(static_cast<cudaStream_t>(p)) {}
};

// Copy contiguous source ranges to aligned destinations with the segment
// copy kernel (used for upload re-layout and crossover children).
gp_status run_copy(const uint8_t *src, uint8_t *dst, const std::vector<XoChild> &kids,
                   cudaStream_t s, DevBufs &tmp)
{
    const uint32_t tile = 16384;
    std::vector<XoTile> tiles;
    for (uint32_t c = 0; c < kids.size(); ++c)
        for (uint64_t b = 0; b < kids[c].n; b += tile) tiles.push_back(XoTile{c, 0, b});
    if (tiles.empty()) return GP_OK;
    if (tiles.size() > 0x7fffffffu) return GP_EINVAL;
    uint8_t *blk;
    const uint64_t o_tiles = round_up(sizeof(XoChild) * kids.size(), 256);
    CK(tmp.alloc((void **)&blk, o_tiles + sizeof(XoTile) * tiles.size(), s));
    XoChild *d_kids = reinterpret_cast<XoChild *>(blk);
    XoTile *d_tiles = reinterpret_cast<XoTile *>(blk + o_tiles);
    CK(h2d(d_kids, kids.data(), sizeof(XoChild) * kids.size(), s));
    CK(h2d(d_tiles, tiles.data(), sizeof(XoTile) * tiles.size(), s));
    ProfScope ps(GP_KERNEL_COPY, s);
    CK(launch_xo_copy(src, dst, d_kids, d_tiles, (uint32_t)tiles.size(), tile, s));
    return GP_OK;
}

// Device validation of every tree (see gp_create_population).
gp_status validate_population(gp_population *P, cudaStream_t s, DevBufs &tmp, bool *ok)
{
    const uint64_t VC = 1 << 16;
    std::vector<EvalItem> chunks;
    std::vector<uint32_t> first(P->n_trees + 1);
    for (uint32_t t = 0; t < P->n_trees; ++t) {
        first[t] = (uint32_t)chunks.size();
        for (uint64_t b = 0; b < P->h_size[t]; b += VC) {
            EvalItem it{};
            it.begin = P->h_start[t] + b;
            it.end = P->h_start[t] + std::min(P->h_size[t], b + VC);
            it.tree = t;
            chunks.push_back(it);
        }
    }
    first[P->n_trees] = (uint32_t)chunks.size();
    EvalItem *d_chunks;
    ValOut *d_out;
    uint32_t *d_first, *d_bad;
    CK(tmp.alloc((void **)&d_chunks, sizeof(EvalItem) * chunks.size(), s));
    CK(tmp.alloc((void **)&d_out, sizeof(ValOut) * chunks.size(), s));
    CK(tmp.alloc((void **)&d_first, sizeof(uint32_t) * first.size(), s));
    CK(tmp.alloc((void **)&d_bad, sizeof(uint32_t), s));
    CK(h2d(d_chunks, chunks.data(), sizeof(EvalItem) * chunks.size(), s));
    CK(h2d(d_first, first.data(), sizeof(uint32_t) * first.size(), s));
    CK(cudaMemsetAsync(d_bad, 0, sizeof(uint32_t), s));
    {
        ProfScope ps(GP_KERNEL_VALIDATE, s);
        CK(launch_validate(P->d_arena, d_chunks, (uint32_t)chunks.size(), P->n_consts, d_out, s));
    }
    {
        ProfScope ps(GP_KERNEL_VALIDATE, s);
        CK(launch_validate_trees(d_out, d_first, P->n_trees, d_bad, s));
    }
    uint32_t bad = 0;
    CK(cudaMemcpyAsync(&bad, d_bad, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *ok = (bad == 0);
    return GP_OK;
}

gp_status copy_problem(gp_population *P, const gp_problem *pr)
{
    if (!pr || pr->n_cases == 0 || pr->n_cases > kMaxCases || !pr->x || !pr->y) return GP_EINVAL;
    if (pr->n_consts > kMaxConsts || (pr->n_consts && !pr->consts)) return GP_EINVAL;
    P->n_cases = pr->n_cases;
    P->lanes = lanes_for(pr->n_cases);
    P->n_consts = pr->n_consts;
    P->div0 = pr->protected_div_value;
    P->max_tree_nodes = pr->max_tree_nodes;
    P->hbm_budget = pr->hbm_budget_bytes;
    P->hx.assign(2 * P->lanes, 0.0f);
    P->hy.assign(2 * P->lanes, 0.0f);
    std::memcpy(P->hx.data(), pr->x, sizeof(float) * pr->n_cases);
    std::memcpy(P->hy.data(), pr->y, sizeof(float) * pr->n_cases);
    P->hc.assign(pr->consts ? pr->consts : nullptr, pr->consts ? pr->consts + pr->n_consts : nullptr);
    return GP_OK;
}

void copy_problem_from(gp_population *dst, const gp_population *src)
{
    dst->n_cases = src->n_cases;
    dst->lanes = src->lanes;
    dst->n_consts = src->n_consts;
    dst->div0 = src->div0;
    dst->max_tree_nodes = src->max_tree_nodes;
    dst->hbm_budget = src->hbm_budget;
    dst->hx = src->hx;
    dst->hy = src->hy;
    dst->hc = src->hc;
}

struct DeviceGuard {
    int prev = 0;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = 0;
        cudaGetDevice(&cur);
        if (cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

namespace gpk {

// Copies trees `trees[0..n)` of population `src` to dst + dst_lo onward, each
// at a 16-byte aligned offset (enqueued on s; synchronises only to bring a
// device-only layout to the host).  Writes each tree's offset from dst and
// size; GP_ENOMEM when they need more than `cap` bytes from dst_lo.
gp_status gather_trees(const gp_population *srcc, const uint32_t *trees, uint32_t n, uint8_t *dst, uint64_t dst_lo,
                       uint64_t cap, uint64_t *start, uint64_t *size, cudaStream_t s)
{
    gp_population *src = const_cast<gp_population *>(srcc);
    if (!src || (n && !trees)) return GP_EINVAL;
    gp_status st = ensure_host_layout(src);
    if (st) return st;
    std::vector<XoChild> kids(n);
    uint64_t pos = 0;
    for (uint32_t k = 0; k < n; ++k) {
        const uint32_t t = trees[k];
        if (t >= src->n_trees) return GP_EINVAL;
        XoChild c{};
        c.dst = dst_lo + pos;
        c.n = src->h_size[t];
        c.head_src = src->h_start[t];
        c.i = c.n;                            // the whole tree is the head segment
        kids[k] = c;
        start[k] = c.dst;
        size[k] = c.n;
        pos = round_up(pos + c.n, 16);
    }
    if (pos + 64 > cap) return GP_ENOMEM;
    if (src->stream && src->stream != s) {    // the source's last writer first
        cudaEvent_t e;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        cudaEventRecord(e, src->stream);
        cudaStreamWaitEvent(s, e, 0);
        cudaEventDestroy(e);
    }
    DevBufs tmp;
    st = run_copy(src->d_arena, dst, kids, s, tmp);
    tmp.release(s);
    return st;
}

}  // namespace gpk

// ================================================================= ABI

extern "C" {

const char *gp_status_string(gp_status st)
{
    switch (st) {
    case GP_OK: return "GP_OK";
    case GP_EINVAL: return "GP_EINVAL: invalid argument";
    case GP_ENOMEM: return "GP_ENOMEM: out of memory or over the HBM budget";
    case GP_EMALFORMED: return "GP_EMALFORMED: malformed tree";
    case GP_ECUDA: return "GP_ECUDA: CUDA error";
    case GP_ETIMEOUT: return "GP_ETIMEOUT: device wait timed out";
    case GP_ELIMIT: return "GP_ELIMIT: tree exceeds the node limit";
    }
    return "unknown gp_status";
}

gp_status gp_create_population(const gp_problem *problem, uint32_t n_trees, const uint8_t *nodes,
                               const uint64_t *offsets, void *cuda_stream, gp_population **out)
{
    if (!out || !problem) return GP_EINVAL;
    if (n_trees > 0 && (!nodes || !offsets)) return GP_EINVAL;
    if (n_trees > 0 && offsets[0] != 0) return GP_EINVAL;
    for (uint32_t t = 0; t < n_trees; ++t)
        if (offsets[t + 1] <= offsets[t]) return GP_EINVAL;
    cudaStream_t s = Stream(cuda_stream).s;
    gp_population *P = new (std::nothrow) gp_population();
    if (!P) return GP_ENOMEM;
    gp_status st = copy_problem(P, problem);
    if (st) { delete P; return st; }
    cudaGetDevice(&P->device);
    configure_pool(P->device);
    P->n_trees = n_trees;
    P->h_size.resize(n_trees);
    for (uint32_t t = 0; t < n_trees; ++t) P->h_size[t] = offsets[t + 1] - offsets[t];
    layout_trees(P);
    if (P->hbm_budget && population_bytes(P->arena_bytes, n_trees, P->n_cases) > P->hbm_budget) {
        delete P;
        return GP_ENOMEM;
    }
    st = alloc_population(P, s);
    if (st) { destroy(P); return st; }
    if (n_trees > 0) {
        DevBufs tmp;
        uint8_t *d_stage = nullptr;
        const uint64_t packed = offsets[n_trees];
        std::vector<XoChild> kids(n_trees);
        auto run = [&]() -> gp_status {
            CK(tmp.alloc((void **)&d_stage, packed + 64, s));
            CK(cudaMemcpyAsync(d_stage, nodes, packed, cudaMemcpyDefault, s));   // host or device bytes
            for (uint32_t t = 0; t < n_trees; ++t) {
                XoChild &k = kids[t];
                k = XoChild{};
                k.dst = P->h_start[t];
                k.n = P->h_size[t];
                k.head_src = offsets[t];
                k.i = k.n;
            }
            gp_status r = run_copy(d_stage, P->d_arena, kids, s, tmp);
            if (r) return r;
            bool ok = false;
            r = validate_population(P, s, tmp, &ok);
            if (r) return r;
            return ok ? GP_OK : GP_EMALFORMED;
        };
        st = run();
        tmp.release(s);
        if (st) { destroy(P); return st; }
    }
    *out = P;
    return GP_OK;
}

gp_status gp_tree_size(const gp_population *Pc, uint32_t tree, uint64_t *n)
{
    gp_population *P = const_cast<gp_population *>(Pc);
    if (!P || !n || tree >= P->n_trees) return GP_EINVAL;
    DeviceGuard dg(P->device);
    gp_status st = ensure_host_layout(P);
    if (st) return st;
    *n = P->h_size[tree];
    return GP_OK;
}

gp_status gp_tree_read(const gp_population *Pc, uint32_t tree, uint8_t *dst, uint64_t cap)
{
    gp_population *P = const_cast<gp_population *>(Pc);
    if (!P || !dst || tree >= P->n_trees) return GP_EINVAL;
    DeviceGuard dg(P->device);
    gp_status st = ensure_host_layout(P);
    if (st) return st;
    if (cap < P->h_size[tree]) return GP_EINVAL;
    CK(cudaStreamSynchronize(P->stream));
    CK(cudaMemcpy(dst, P->d_arena + P->h_start[tree], P->h_size[tree], cudaMemcpyDeviceToHost));
    return GP_OK;
}

gp_status gp_population_get_info(const gp_population *Pc, gp_population_info *info)
{
    gp_population *P = const_cast<gp_population *>(Pc);
    if (!P || !info) return GP_EINVAL;
    DeviceGuard dg(P->device);
    gp_status st = ensure_host_layout(P);
    if (st) return st;
    info->n_trees = P->n_trees;
    info->n_cases = P->n_cases;
    info->total_nodes = P->total_nodes;
    info->d_nodes = P->d_arena;
    info->d_tree_start = P->d_start;
    info->d_tree_size = P->d_size;
    info->d_fitness = P->d_fitness;
    info->d_case_values = P->d_values;
    info->d_hits = P->d_hits;
    return GP_OK;
}

void gp_destroy_population(gp_population *P) { destroy(P); }

// ---------------------------------------------------------------- evaluate

gp_status gp_evaluate(gp_population *P, void *cuda_stream) { return gp_evaluate_ex(P, nullptr, cuda_stream); }

}  // extern "C"

namespace {

// Medium trees (more than one chunk, at most kFuseMaxChunks) are evaluated
// without a planning pass: every chunk right-aligns its upper-tree fragment
// in a slot of C codes and keeps up to kFusePt value entries per slot; one
// "rope" item per tree then walks the slots in a second launch.
constexpr uint32_t kFuseMaxChunks = 32;

uint32_t fuse_pt_cap(uint32_t C) { return std::max<uint32_t>(128, C / 8); }

gp_status eval_config(const gp_population *P, const gp_eval_options *opt, EvalCfg *cfg)
{
    EvalCfg c{};
    c.C = opt && opt->chunk_nodes ? opt->chunk_nodes : 4096;
    c.W = opt && opt->warps_per_cta ? opt->warps_per_cta : 32;
    c.K = opt && opt->window_entries ? opt->window_entries : 32;
    // Upper trees hold many pending values (the residual subtrees of every
    // chunk), so their window is deeper.
    c.Ku = opt && opt->upper_window_entries ? opt->upper_window_entries : std::max<uint32_t>(c.K, 128);
    if (c.C % 16 || c.C < 64 || c.C > (1u << 24) || c.W < 1 || c.W > 32 || c.K < 16 || c.K % 2 ||
        c.K > 1024 || c.Ku < 16 || c.Ku % 2 || c.Ku > 1024)
        return GP_EINVAL;
    c.lanes = (int)P->lanes;
    c.rows = (int)std::max<uint32_t>(1 + P->n_consts, 1);
    c.sms = sm_count(P->device);
    int maxsm = 0;
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device);
    if (!(opt && opt->warps_per_cta))        // as many warps as shared memory holds
        while (c.W > 1 && eval_smem_bytes(c.lanes, (int)c.W, (int)c.K, false, c.rows) > (size_t)maxsm) --c.W;
    // Upper levels (32-bit codes) run at most 16 warps per SM, with staging.
    c.Wu = std::min<uint32_t>(c.W, 16);
    while (c.Wu > 1 && eval_smem_bytes(c.lanes, (int)c.Wu, (int)c.Ku, true, c.rows) > (size_t)maxsm) --c.Wu;
    c.smem = eval_smem_bytes(c.lanes, (int)c.W, (int)c.K, false, c.rows);
    c.smem_u = eval_smem_bytes(c.lanes, (int)c.Wu, (int)c.Ku, true, c.rows);
    // A launch of ropes only: few long serial walks, latency-bound; a deeper
    // window (fewer spills) beats more warps there (0.173 against 0.188 ms
    // for the bench population's ropes at 192 and 128 entries).
    c.Kr = opt && opt->upper_window_entries ? c.Ku : std::max<uint32_t>(c.K, 192);
    c.Wr = std::min<uint32_t>(c.W, 16);
    while (c.Wr > 1 && eval_smem_bytes(c.lanes, (int)c.Wr, (int)c.Kr, true, c.rows) > (size_t)maxsm) --c.Wr;
    c.smem_r = eval_smem_bytes(c.lanes, (int)c.Wr, (int)c.Kr, true, c.rows);
    if (c.smem_r > (size_t)maxsm) {
        c.Kr = c.Ku;
        c.Wr = c.Wu;
        c.smem_r = c.smem_u;
    }
    if (c.smem > (size_t)maxsm || c.smem_u > (size_t)maxsm) return GP_EINVAL;
    *cfg = c;
    return GP_OK;
}

// Evaluate the given trees (all enqueued on s).  Small trees are one final
// item; medium trees are fused chunks plus a rope item (when allowed);
// large trees go through planned upper-tree levels, which synchronise once
// per level to size the next one.
gp_status eval_trees(gp_population *P, const std::vector<uint32_t> &trees, const EvalCfg &cfg,
                     bool allow_fused, cudaStream_t s)
{
    const uint32_t C = cfg.C;
    const int lanes = cfg.lanes, sms = cfg.sms;
    CK(eval_prepare_at_least(lanes, false, cfg.smem));
    CK(eval_prepare_at_least(lanes, true, cfg.smem_u));
    DevBufs ws;
    auto body = [&]() -> gp_status {
        // Small and medium trees, largest first (ties in the given order):
        // sorted as 64-bit keys (size complement, position), sizes of both
        // fit 32 bits.
        std::vector<uint32_t> small, medium, big;
        std::vector<uint64_t> ks, km;
        ks.reserve(trees.size());
        uint64_t n_chunks = 0;
        for (uint32_t i = 0; i < (uint32_t)trees.size(); ++i) {
            const uint64_t n = P->h_size[trees[i]];
            const uint64_t key = ((0xFFFFFFFFull - n) << 32) | i;
            if (n <= C) {
                ks.push_back(key);
            } else if (allow_fused && n <= (uint64_t)kFuseMaxChunks * C) {
                km.push_back(key);
                n_chunks += (n + C - 1) / C;
            } else {
                big.push_back(trees[i]);
                n_chunks += (n + C - 1) / C;
            }
        }
        std::sort(ks.begin(), ks.end());
        std::sort(km.begin(), km.end());
        small.resize(ks.size());
        medium.resize(km.size());
        for (size_t k = 0; k < ks.size(); ++k) small[k] = trees[(uint32_t)ks[k]];
        for (size_t k = 0; k < km.size(); ++k) medium[k] = trees[(uint32_t)km[k]];

        // ---- level 0: planned chunks of large trees, fused chunks of medium
        // trees (largest first), whole small trees (largest first)
        std::vector<EvalItem> items;
        items.reserve(n_chunks + small.size());
        std::vector<uint32_t> first_chunk;          // per large tree: first fragment item
        for (uint32_t t : big) {
            first_chunk.push_back((uint32_t)items.size());
            for (uint64_t b = 0; b < P->h_size[t]; b += C) {
                EvalItem it{};
                it.begin = P->h_start[t] + b;
                it.end = P->h_start[t] + std::min<uint64_t>(P->h_size[t], b + C);
                it.tree = t;
                it.spill_off = kNoSpill;
                items.push_back(it);
            }
        }
        first_chunk.push_back((uint32_t)items.size());
        const uint32_t n_frag0 = (uint32_t)items.size();
        std::vector<EvalItem> ropes;
        ropes.reserve(medium.size());
        uint64_t slots = 0;
        for (uint32_t t : medium) {
            const uint32_t m = (uint32_t)((P->h_size[t] + C - 1) / C);
            for (uint32_t j = 0; j < m; ++j) {
                EvalItem it{};
                it.begin = P->h_start[t] + (uint64_t)j * C;
                it.end = P->h_start[t] + std::min<uint64_t>(P->h_size[t], (uint64_t)(j + 1) * C);
                it.tree = t;
                it.flags = kItemFused;
                it.frag_off = slots + j;
                it.pt_base = slots;
                it.frag_len = m;
                it.spill_off = kNoSpill;
                items.push_back(it);
            }
            EvalItem r{};
            r.tree = t;
            r.flags = kItemFinal | kItemRope;
            r.pt_base = slots;
            r.frag_len = m;
            r.spill_off = kNoSpill;
            ropes.push_back(r);
            slots += m;
        }
        for (uint32_t t : small) {
            EvalItem it{};
            it.begin = P->h_start[t];
            it.end = P->h_start[t] + P->h_size[t];
            it.tree = t;
            it.flags = kItemFinal;
            it.spill_off = kNoSpill;
            items.push_back(it);
        }

        const uint64_t warps_total = (uint64_t)sms * cfg.W;   // >= warps of any level
        const uint64_t spill_per_warp = C;                    // a chunk never holds more
        // One block for the level counters and the fused slots: counters and
        // overflow flags (zeroed together), slot lengths, codes, values.
        const uint32_t pt_cap = fuse_pt_cap(C);
        uint32_t *d_counter, *fz_codes = nullptr, *fz_len = nullptr, *fz_over = nullptr;
        float2 *fz_pt = nullptr;
        {
            const uint64_t o_over = 256, o_len = round_up(o_over + 4ull * (slots ? P->n_trees : 0), 256);
            const uint64_t o_codes = round_up(o_len + 4ull * slots, 256);
            const uint64_t o_pt = round_up(o_codes + (slots ? 4ull * (slots * C + 32) : 0), 256);
            const uint64_t end = o_pt + (slots ? 8ull * (slots * pt_cap * lanes + 1) : 0);
            uint8_t *blk;
            CK(ws.alloc((void **)&blk, end, s));
            CK(cudaMemsetAsync(blk, 0, o_len, s));
            d_counter = reinterpret_cast<uint32_t *>(blk);
            if (slots) {
                fz_over = reinterpret_cast<uint32_t *>(blk + o_over);
                fz_len = reinterpret_cast<uint32_t *>(blk + o_len);
                fz_codes = reinterpret_cast<uint32_t *>(blk + o_codes);
                fz_pt = reinterpret_cast<float2 *>(blk + o_pt);
                P->redo_pending = true;
            }
        }

        // level state
        const void *codes = P->d_arena;
        bool wide = false;
        const float2 *pt_in = nullptr;
        std::vector<uint64_t> prev_len(big.size());
        for (size_t k = 0; k < big.size(); ++k) prev_len[k] = P->h_size[big[k]];
        std::vector<EvalItem> cur_items = std::move(items);
        uint32_t n_frag = n_frag0;
        std::vector<uint32_t> cur_big = big;
        std::vector<uint32_t> cur_first = first_chunk;
        uint32_t level = 0;

        for (;;) {
            if (level >= 63) return GP_EINVAL;
            if (cur_items.empty()) break;
            EvalItem *d_items;
            CK(ws.alloc((void **)&d_items, sizeof(EvalItem) * cur_items.size(), s));
            CK(h2d(d_items, cur_items.data(), sizeof(EvalItem) * cur_items.size(), s));
            uint32_t *u_next = nullptr;
            float2 *pt_next = nullptr;
            std::vector<uint64_t> frag_off;
            if (n_frag) {
                PlanOut *d_plan;
                uint64_t *d_fo, *d_tot;
                CK(ws.alloc((void **)&d_plan, sizeof(PlanOut) * n_frag, s));
                CK(ws.alloc((void **)&d_fo, sizeof(uint64_t) * (n_frag + 1), s));
                CK(ws.alloc((void **)&d_tot, sizeof(uint64_t) * 4, s));
                {
                    ProfScope ps(GP_KERNEL_PLAN, s);
                    CK(launch_plan(wide, codes, d_items, n_frag, d_plan, s));
                }
                {
                    ProfScope ps(GP_KERNEL_SCAN, s);
                    CK(launch_plan_scan(d_items, d_plan, n_frag, d_fo, d_tot, s));
                }
                frag_off.resize(n_frag + 1);
                uint64_t tot[4] = {};
                CK(cudaMemcpyAsync(frag_off.data(), d_fo, sizeof(uint64_t) * (n_frag + 1),
                                   cudaMemcpyDeviceToHost, s));
                CK(cudaMemcpyAsync(tot, d_tot, sizeof(uint64_t) * 3, cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                if (tot[1] + kPtCode0 >= 0xffffffffull) return GP_ENOMEM;
                if (tot[2] > spill_per_warp) return GP_EINVAL;   // cannot happen: chunks <= C
                CK(ws.alloc((void **)&u_next, sizeof(uint32_t) * (round_up(tot[0], 16) + 32), s));
                CK(cudaMemsetAsync(u_next + tot[0], 0,
                                   sizeof(uint32_t) * (round_up(tot[0], 16) + 32 - tot[0]), s));
                CK(ws.alloc((void **)&pt_next, sizeof(float2) * (tot[1] * lanes + 1), s));
                P->stats.upper_codes += tot[0];
                P->stats.value_entries += tot[1];
            }
            // dedicated spill areas for oversized final items
            uint64_t dedicated = 0;
            for (auto &it : cur_items) {
                if ((it.flags & kItemFinal) && !(it.flags & kItemRope) && it.end - it.begin > spill_per_warp) {
                    it.spill_off = warps_total * spill_per_warp + dedicated;
                    it.spill_cap = it.end - it.begin;
                    dedicated += it.spill_cap;
                }
            }
            if (dedicated) {
                // re-upload the items with their spill areas (fragment fields
                // written by the scan are kept: only finals changed)
                for (uint32_t i = n_frag; i < cur_items.size(); ++i)
                    CK(h2d(d_items + i, &cur_items[i], sizeof(EvalItem), s));
            }
            float2 *d_spill;
            CK(ws.alloc((void **)&d_spill,
                        sizeof(float2) * lanes * (warps_total * spill_per_warp + dedicated), s));

            EvalParams p{};
            p.codes = codes;
            p.items = d_items;
            p.n_items = (uint32_t)cur_items.size();
            p.counter = d_counter + level;
            p.stat_up = level == 0 ? P->d_stat + 4 : nullptr;   // what level 0 sends upward
            p.x = P->d_x;
            p.y = P->d_y;
            p.consts = P->d_c;
            p.n_cases = P->n_cases;
            p.n_consts = P->n_consts;
            p.leaf_rows = (uint32_t)cfg.rows;
            p.div0 = P->div0;
            p.window = wide ? cfg.Ku : cfg.K;
            p.pt_in = pt_in;
            p.pt_out = pt_next;
            p.u_out = u_next;
            p.values = P->d_values;
            p.fitness = P->d_fitness;
            p.hits = P->d_hits;
            p.spill = d_spill;
            p.spill_per_warp = spill_per_warp;
            p.err = P->d_err;
            p.fz_codes = fz_codes;
            p.fz_pt = fz_pt;
            p.fz_len = fz_len;
            p.fz_over = fz_over;
            p.fz_redo = P->d_redo;
            p.fz_cap_codes = C;
            p.fz_cap_pt = pt_cap;
            {
                ProfScope ps(wide ? GP_KERNEL_EVAL_UPPER : GP_KERNEL_EVAL, s);
                CK(launch_eval(lanes, wide, p, sms, (int)(wide ? cfg.Wu : cfg.W), wide ? cfg.smem_u : cfg.smem, s));
            }
            P->stats.levels = level + 1;
            P->stats.items += cur_items.size();

            // ---- next level: one upper tree per large tree, plus the ropes
            std::vector<EvalItem> next;
            std::vector<uint32_t> nb, nf;
            std::vector<uint64_t> nprev;
            std::vector<EvalItem> finals;
            if (n_frag) {
                for (size_t k = 0; k < cur_big.size(); ++k) {
                    const uint32_t t = cur_big[k];
                    const uint64_t ub = frag_off[cur_first[k]], ue = frag_off[cur_first[k + 1]];
                    const uint64_t len = ue - ub;
                    if (len <= C || len * 2 > prev_len[k]) {
                        EvalItem it{};
                        it.begin = ub;
                        it.end = ue;
                        it.tree = t;
                        it.flags = kItemFinal;
                        it.spill_off = kNoSpill;
                        finals.push_back(it);
                    } else {
                        nb.push_back(t);
                        nf.push_back((uint32_t)next.size());
                        nprev.push_back(len);
                        for (uint64_t b = ub; b < ue; b += C) {
                            EvalItem it{};
                            it.begin = b;
                            it.end = std::min<uint64_t>(ue, b + C);
                            it.tree = t;
                            it.spill_off = kNoSpill;
                            next.push_back(it);
                        }
                    }
                }
            }
            nf.push_back((uint32_t)next.size());
            n_frag = (uint32_t)next.size();
            std::stable_sort(finals.begin(), finals.end(), [](const EvalItem &a, const EvalItem &b) {
                return a.end - a.begin > b.end - b.begin;
            });
            // ropes join the first upper level, largest trees first
            next.insert(next.end(), ropes.begin(), ropes.end());
            ropes.clear();
            next.insert(next.end(), finals.begin(), finals.end());
            cur_items = std::move(next);
            cur_big = std::move(nb);
            cur_first = std::move(nf);
            prev_len = std::move(nprev);
            codes = u_next;
            wide = true;
            pt_in = pt_next;
            ++level;
        }
        return GP_OK;
    };
    gp_status st = body();
    ws.release(s);
    return st;
}

// Evaluation of a population whose sizes are on the device only and whose
// bounds keep every tree within kFuseMaxChunks chunks: the level-0 items
// and the ropes are built on the device (plan0), so nothing returns to the
// host between the crossover that made the trees and their evaluation.
// Scratch is sized from the bounds.
gp_status eval_device_planned(gp_population *P, const EvalCfg &cfg, cudaStream_t s)
{
    const uint32_t C = cfg.C;
    const int lanes = cfg.lanes, sms = cfg.sms;
    CK(eval_prepare_at_least(lanes, false, cfg.smem));
    CK(eval_prepare_at_least(lanes, true, std::max(cfg.smem_u, cfg.smem_r)));
    uint64_t max_items = 0, max_slots = 0, max_ropes = 0;
    for (uint64_t b : P->h_bound) {
        const uint64_t m = (b + C - 1) / C;
        max_items += m;
        if (b > C) {
            max_slots += m;
            ++max_ropes;
        }
    }
    // cut at low points of the arity walk, a multi-chunk tree may take one
    // chunk more than ceil(size / C): room for one more item and slot each
    const uint64_t max_cuts = max_slots;
    max_items += max_ropes;
    max_slots += max_ropes;
    if (max_items > 0x7fffffffull || max_cuts >= (1ull << 27)) return GP_ENOMEM;
    const uint32_t pt_cap = fuse_pt_cap(C);
    const uint64_t warps_total = (uint64_t)sms * cfg.W, spill_per_warp = C;
    DevBufs ws;
    auto body = [&]() -> gp_status {
        // counters and counts, overflow flags (zeroed together), slot
        // lengths, slot codes, slot values, items, ropes, spill
        uint64_t off = 0;
        auto take = [&](uint64_t bytes) {
            const uint64_t o = off;
            off = round_up(off + bytes, 256);
            return o;
        };
        const uint64_t o_cls = take(4ull * plan_level0_scratch_words());
        const uint64_t o_cnt = take(256 + 16 + 4ull * P->n_trees);
        const uint64_t o_meta = take(4ull * P->n_trees);
        const uint64_t o_cuts = take(4ull * max_cuts + 4);
        const uint64_t o_len = take(4ull * max_slots);
        const uint64_t o_codes = take(4ull * (max_slots * C + 32));
        const uint64_t o_pt = take(8ull * (max_slots * pt_cap * lanes + 1));
        const uint64_t o_items = take(sizeof(EvalItem) * max_items);
        const uint64_t o_ropes = take(sizeof(EvalItem) * (max_ropes + 1));
        const uint64_t o_spill = take(8ull * lanes * warps_total * spill_per_warp);
        uint8_t *blk;
        CK(ws.alloc((void **)&blk, off, s));
        uint32_t *d_counter = reinterpret_cast<uint32_t *>(blk + o_cnt);
        uint32_t *d_counts = d_counter + 64;
        EvalItem *items = reinterpret_cast<EvalItem *>(blk + o_items);
        EvalItem *ropes = reinterpret_cast<EvalItem *>(blk + o_ropes);
        // one launch zeroes the cursors, counters and flags of `blk` and the
        // population's error, stat and redo words; the planned counts go to
        // d_stat[0..2] from the planner itself
        CK(launch_plan_level0(P->d_arena, P->d_start, P->d_size, P->n_trees, C, kFuseMaxChunks, items, ropes,
                              d_counts, reinterpret_cast<uint32_t *>(blk + o_cls),
                              reinterpret_cast<uint32_t *>(blk + o_meta), reinterpret_cast<uint32_t *>(blk + o_cuts),
                              reinterpret_cast<uint32_t *>(blk), (uint32_t)((o_cnt + 256 + 16 + 4ull * P->n_trees) / 4),
                              P->d_err, P->d_stat, sms, s));
        note_launches(4);
        EvalParams p{};
        p.codes = P->d_arena;
        p.items = items;
        p.n_items = (uint32_t)max_items;
        p.n_items_dev = d_counts;
        p.counter = d_counter;
        p.x = P->d_x;
        p.y = P->d_y;
        p.consts = P->d_c;
        p.n_cases = P->n_cases;
        p.n_consts = P->n_consts;
        p.leaf_rows = (uint32_t)cfg.rows;
        p.div0 = P->div0;
        p.window = cfg.K;
        p.values = P->d_values;
        p.fitness = P->d_fitness;
        p.hits = P->d_hits;
        p.spill = reinterpret_cast<float2 *>(blk + o_spill);
        p.spill_per_warp = spill_per_warp;
        p.err = P->d_err;
        p.stat_up = P->d_stat + 4;
        if (max_slots) {
            p.fz_codes = reinterpret_cast<uint32_t *>(blk + o_codes);
            p.fz_pt = reinterpret_cast<float2 *>(blk + o_pt);
            p.fz_len = reinterpret_cast<uint32_t *>(blk + o_len);
            p.fz_over = d_counts + 4;
            p.fz_redo = P->d_redo;
            p.fz_cap_codes = C;
            p.fz_cap_pt = pt_cap;
        }
        {
            ProfScope ps(GP_KERNEL_EVAL, s);
            CK(launch_eval(lanes, false, p, sms, (int)cfg.W, cfg.smem, s, true));
        }
        if (max_ropes) {
            p.items = ropes;
            p.n_items = (uint32_t)max_ropes;
            p.n_items_dev = d_counts + 1;
            p.counter = d_counter + 1;
            p.window = cfg.Kr;
            ProfScope ps(GP_KERNEL_EVAL_UPPER, s);
            CK(launch_eval(lanes, true, p, sms, (int)cfg.Wr, cfg.smem_r, s, true));
            P->redo_pending = true;
        }
        P->stat_pending = true;
        return GP_OK;
    };
    gp_status st = body();
    ws.release(s);
    return st;
}

}  // namespace

extern "C" {

gp_status gp_evaluate_ex(gp_population *P, const gp_eval_options *opt, void *cuda_stream)
{
    if (!P) return GP_EINVAL;
    DeviceGuard dg(P->device);
    cudaStream_t s = Stream(cuda_stream).s;
    P->stream = s;
    P->stats = gp_eval_stats{};
    P->stat_pending = false;
    P->redo_pending = false;
    if (P->n_trees == 0) {
        CK(cudaEventRecord(P->ev, s));
        P->evaluated = true;
        return GP_OK;
    }
    EvalCfg cfg;
    gp_status st = eval_config(P, opt, &cfg);
    if (st) return st;
    P->cfg = cfg;
    P->up_read = false;
    if (!P->host_layout) {
        uint64_t bmax = 0;
        for (uint64_t b : P->h_bound) bmax = std::max(bmax, b);
        if (bmax <= (uint64_t)kFuseMaxChunks * cfg.C) {
            // (the planner's first launch zeroes the error, stat and redo words)
            st = eval_device_planned(P, cfg, s);
            if (st) return st;
            CK(cudaEventRecord(P->ev, s));
            P->evaluated = true;
            return GP_OK;
        }
        if ((st = ensure_host_layout(P))) return st;
    }
    CK(cudaMemsetAsync(P->d_err, 0, sizeof(uint32_t) * 4, s));
    CK(cudaMemsetAsync(P->d_stat + 4, 0, sizeof(uint32_t) * 3, s));
    CK(cudaMemsetAsync(P->d_redo, 0, sizeof(uint32_t), s));
    std::vector<uint32_t> all(P->n_trees);
    for (uint32_t t = 0; t < P->n_trees; ++t) all[t] = t;
    st = eval_trees(P, all, cfg, true, s);
    if (st) return st;
    CK(cudaEventRecord(P->ev, s));
    P->evaluated = true;
    return GP_OK;
}

gp_status gp_fitness(const gp_population *Pc, float *fitness, float *case_values, uint32_t *hits)
{
    gp_population *P = const_cast<gp_population *>(Pc);
    if (!P || (!fitness && P->n_trees)) return GP_EINVAL;
    if (!P->evaluated) return GP_EINVAL;
    DeviceGuard dg(P->device);
    CK(cudaEventSynchronize(P->ev));
    if (P->redo_pending) {
        // Trees whose chunk fragments did not fit their slots are evaluated
        // again through planned upper-tree levels (rare: very wide shapes).
        P->redo_pending = false;
        uint32_t n = 0;
        CK(cudaMemcpy(&n, P->d_redo, sizeof(uint32_t), cudaMemcpyDeviceToHost));
        if (n) {
            std::vector<uint32_t> redo(n);
            CK(cudaMemcpy(redo.data(), P->d_redo + 1, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost));
            std::sort(redo.begin(), redo.end());
            gp_status st = ensure_host_layout(P);
            if (st) return st;
            st = eval_trees(P, redo, P->cfg, false, P->stream);
            if (st) return st;
            CK(cudaStreamSynchronize(P->stream));
            P->stats.redone = n;
        }
    }
    uint32_t ew[8] = {};
    CK(cudaMemcpy(ew, P->d_err, sizeof(ew), cudaMemcpyDeviceToHost));
    const uint32_t err = ew[0];
    if (ew[7]) return GP_EMALFORMED;             // a child's subtree extent ran off its parent
    if (err & kErrMalformed) return GP_EMALFORMED;
    if (err) return GP_ECUDA;
    if (P->n_trees == 0) return GP_OK;
    CK(cudaMemcpy(fitness, P->d_fitness, sizeof(float) * P->n_trees, cudaMemcpyDeviceToHost));
    if (case_values)
        CK(cudaMemcpy(case_values, P->d_values, sizeof(float) * (uint64_t)P->n_trees * P->n_cases,
                      cudaMemcpyDeviceToHost));
    if (hits) CK(cudaMemcpy(hits, P->d_hits, sizeof(uint32_t) * P->n_trees, cudaMemcpyDeviceToHost));
    return GP_OK;
}

gp_status gp_eval_stats_get(const gp_population *Pc, gp_eval_stats *out)
{
    gp_population *P = const_cast<gp_population *>(Pc);
    if (!P || !out) return GP_EINVAL;
    if (P->stat_pending || !P->up_read) {    // counts kept on the device
        DeviceGuard dg(P->device);
        uint32_t c[7] = {};
        CK(cudaStreamSynchronize(P->stream));
        CK(cudaMemcpy(c, P->d_stat, sizeof(c), cudaMemcpyDeviceToHost));
        if (P->stat_pending) {               // a device-planned evaluation
            P->stats.items = (uint64_t)c[0] + c[1];
            P->stats.levels = c[1] ? 2u : 1u;
            P->stats.upper_codes = c[4];
            P->stats.value_entries = c[6];
            P->stat_pending = false;
        }
        P->stats.upper_ops = c[5];
        P->up_read = true;
    }
    *out = P->stats;
    return GP_OK;
}

// ---------------------------------------------------------------- crossover

gp_status gp_crossover(const gp_population *M, const gp_xo *ops, uint32_t n_ops, void *cuda_stream,
                       gp_population **children_out)
{
    if (!M || !children_out || (n_ops && !ops)) return GP_EINVAL;
    {
        DeviceGuard dg(M->device);
        gp_status st = ensure_host_layout(const_cast<gp_population *>(M));   // parents made without a sync
        if (st) return st;
    }
    for (uint32_t k = 0; k < n_ops; ++k) {
        const gp_xo &o = ops[k];
        if (o.mum >= M->n_trees || o.dad >= M->n_trees) return GP_EINVAL;
        if (o.mum_point >= M->h_size[o.mum] || o.dad_point >= M->h_size[o.dad]) return GP_EINVAL;
    }
    DeviceGuard dg(M->device);
    cudaStream_t s = Stream(cuda_stream).s;
    // the parents are read on `s` from here on: their memory is freed there
    const_cast<gp_population *>(M)->stream = s;
    gp_population *C = new (std::nothrow) gp_population();
    if (!C) return GP_ENOMEM;
    copy_problem_from(C, M);
    C->device = M->device;
    C->n_trees = n_ops;
    DevBufs tmp;
    std::vector<uint64_t> ends(2 * (size_t)n_ops);
    // Without a synchronisation when it is safe: every child is at most
    // n_m + n_d - j - 1 nodes (mum minus at least the node at i, plus dad's
    // nodes from j on), so an arena sized from those bounds holds the
    // children laid out on the device, and no child can exceed the node
    // limit when no bound does.  Otherwise the sizes are read back first.
    std::vector<uint64_t> bound;
    uint64_t bound_arena = 64, bound_max = 0;
    bool async = n_ops > 0;
    if (async) {
        bound.resize(n_ops);
        for (uint32_t k = 0; k < n_ops; ++k) {
            bound[k] = M->h_size[ops[k].mum] + M->h_size[ops[k].dad] - ops[k].dad_point - 1;
            bound_max = std::max(bound_max, bound[k]);
            bound_arena += round_up(bound[k], 16);
        }
        const uint64_t cap = std::min<uint64_t>(std::max<uint64_t>(4 * M->arena_bytes, 256ull << 20), 16ull << 30);
        if ((C->max_tree_nodes && bound_max > C->max_tree_nodes) || bound_arena > cap ||
            (C->hbm_budget && population_bytes(bound_arena, n_ops, C->n_cases) > C->hbm_budget))
            async = false;
    }
    auto run_async = [&]() -> gp_status {
        C->host_layout = false;
        C->h_bound = std::move(bound);
        C->arena_bytes = bound_arena;
        gp_status r = alloc_population(C, s);
        if (r) return r;
        // the queries go up with one zeroed entry after them, whose first
        // word is the long-walk counter of the extent launches
        const uint32_t n_q = 2 * n_ops;
        std::vector<ExtentQuery> q(n_q + 1, ExtentQuery{0, 0, 0});
        for (uint32_t k = 0; k < n_ops; ++k) {
            q[2 * k] = ExtentQuery{M->h_start[ops[k].mum], M->h_size[ops[k].mum], ops[k].mum_point};
            q[2 * k + 1] = ExtentQuery{M->h_start[ops[k].dad], M->h_size[ops[k].dad], ops[k].dad_point};
        }
        // one block: tile count, ends, queries, copy records, first tiles
        const uint64_t o_end = 256, o_q = round_up(o_end + sizeof(uint64_t) * n_q, 256);
        const uint64_t o_kids = round_up(o_q + sizeof(ExtentQuery) * q.size(), 256);
        const uint64_t o_tb = round_up(o_kids + sizeof(XoChild) * n_ops, 256);
        const uint32_t parts = xo_layout_parts(n_ops);
        // copy tiles: a warp per 2 KB tile when the children are small (mean
        // bound under 8 KB; a CTA per tile would idle most of its threads),
        // else a CTA per 16 KB tile
        const bool warp_tiles = (bound_arena - 64) < 8192ull * n_ops;
        const uint32_t tile = warp_tiles ? 2048 : 16384;
        uint64_t max_tiles = 0;                // children are no larger than their bounds
        for (uint64_t b : C->h_bound) max_tiles += (b + tile - 1) / tile;
        if (max_tiles > 0x7fffffffull) return GP_ENOMEM;
        const uint64_t o_pl = round_up(o_tb + sizeof(uint32_t) * (n_ops + 1), 256);
        const uint64_t o_pt = round_up(o_pl + sizeof(uint64_t) * parts, 256);
        const uint64_t o_tc = round_up(o_pt + sizeof(uint32_t) * parts, 256);
        const uint64_t o_long = round_up(o_tc + sizeof(uint32_t) * max_tiles, 256);
        uint8_t *blk;
        CK(tmp.alloc((void **)&blk, o_long + sizeof(ExtentLong) * n_q, s));
        uint32_t *d_ntiles = reinterpret_cast<uint32_t *>(blk);
        uint64_t *d_end = reinterpret_cast<uint64_t *>(blk + o_end);
        ExtentQuery *d_q = reinterpret_cast<ExtentQuery *>(blk + o_q);
        XoChild *d_kids = reinterpret_cast<XoChild *>(blk + o_kids);
        uint32_t *d_tb = reinterpret_cast<uint32_t *>(blk + o_tb);
        uint32_t *d_lerr = C->d_stat + 3;
        uint32_t *d_nlong = reinterpret_cast<uint32_t *>(d_q + n_q);
        CK(h2d(d_q, q.data(), sizeof(ExtentQuery) * q.size(), s));
        {
            ProfScope ps(GP_KERNEL_EXTENT, s);
            CK(launch_extent(M->d_arena, d_q, n_q, d_end, d_lerr,
                             reinterpret_cast<ExtentLong *>(blk + o_long), d_nlong, sm_count(M->device), s));
        }
        note_launches(1);                      // the long-walk launch (the scope counts one)
        uint32_t *d_tc = reinterpret_cast<uint32_t *>(blk + o_tc);
        CK(launch_xo_layout(d_q, d_end, n_ops, tile, C->arena_bytes, d_kids, C->d_start, C->d_size, d_tb, d_tc,
                            d_ntiles, reinterpret_cast<uint64_t *>(blk + o_pl),
                            reinterpret_cast<uint32_t *>(blk + o_pt), d_lerr, s));
        {
            ProfScope ps(GP_KERNEL_COPY, s);
            CK(launch_xo_copy_map(M->d_arena, C->d_arena, d_kids, d_tb, d_tc, d_ntiles, (uint32_t)max_tiles, tile,
                                  warp_tiles, s));
        }
        note_launches(3);                      // the layout kernels (the others are counted by scope)
        return GP_OK;
    };
    auto run = [&]() -> gp_status {
        if (async) return run_async();
        C->h_size.resize(n_ops);
        if (n_ops) {
            std::vector<ExtentQuery> q(2 * (size_t)n_ops);
            for (uint32_t k = 0; k < n_ops; ++k) {
                q[2 * k] = ExtentQuery{M->h_start[ops[k].mum], M->h_size[ops[k].mum], ops[k].mum_point};
                q[2 * k + 1] = ExtentQuery{M->h_start[ops[k].dad], M->h_size[ops[k].dad], ops[k].dad_point};
            }
            // one block: error word, ends, queries
            const uint64_t o_end = 256, o_q = round_up(o_end + sizeof(uint64_t) * q.size(), 256);
            const uint64_t o_long = round_up(o_q + sizeof(ExtentQuery) * q.size(), 256);
            uint8_t *blk;
            CK(tmp.alloc((void **)&blk, o_long + sizeof(ExtentLong) * q.size(), s));
            uint32_t *d_err = reinterpret_cast<uint32_t *>(blk);
            uint32_t *d_nlong = reinterpret_cast<uint32_t *>(blk + 64);
            uint64_t *d_end = reinterpret_cast<uint64_t *>(blk + o_end);
            ExtentQuery *d_q = reinterpret_cast<ExtentQuery *>(blk + o_q);
            CK(cudaMemsetAsync(d_err, 0, 128, s));          // error word and long-walk counter
            CK(h2d(d_q, q.data(), sizeof(ExtentQuery) * q.size(), s));
            {
                ProfScope ps(GP_KERNEL_EXTENT, s);
                CK(launch_extent(M->d_arena, d_q, (uint32_t)q.size(), d_end, d_err,
                                 reinterpret_cast<ExtentLong *>(blk + o_long), d_nlong, sm_count(M->device), s));
            }
            note_launches(1);
            // error word and ends in one read-back
            std::vector<uint64_t> back(32 + q.size());
            CK(cudaMemcpyAsync(back.data(), blk, o_end + sizeof(uint64_t) * q.size(), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            const uint32_t err = static_cast<uint32_t>(back[0]);
            std::copy(back.begin() + 32, back.end(), ends.begin());
            if (err) return GP_EMALFORMED;
        }
        for (uint32_t k = 0; k < n_ops; ++k) {
            const uint64_t i = ops[k].mum_point, j = ops[k].dad_point;
            const uint64_t em = ends[2 * k], ed = ends[2 * k + 1];
            C->h_size[k] = i + (ed - j) + (M->h_size[ops[k].mum] - em);
            if (C->max_tree_nodes && C->h_size[k] > C->max_tree_nodes) return GP_ELIMIT;
        }
        layout_trees(C);
        if (C->hbm_budget && population_bytes(C->arena_bytes, n_ops, C->n_cases) > C->hbm_budget)
            return GP_ENOMEM;
        gp_status r = alloc_population(C, s);
        if (r) return r;
        std::vector<XoChild> kids(n_ops);
        for (uint32_t k = 0; k < n_ops; ++k) {
            const uint64_t i = ops[k].mum_point, j = ops[k].dad_point;
            const uint64_t em = ends[2 * k], ed = ends[2 * k + 1];
            const uint64_t ms = M->h_start[ops[k].mum], ds = M->h_start[ops[k].dad];
            XoChild &c = kids[k];
            c = XoChild{};
            c.dst = C->h_start[k];
            c.n = C->h_size[k];
            c.head_src = ms;
            c.i = i;
            c.mid_src = ds + j;
            c.ld = ed - j;
            c.tail_src = ms + em;                // tail byte p comes from mum[em + p - i - ld]
        }
        return run_copy(M->d_arena, C->d_arena, kids, s, tmp);
    };
    gp_status st = run();
    tmp.release(s);
    if (st) { destroy(C); return st; }
    *children_out = C;
    return GP_OK;
}

// ---------------------------------------------------------------- profiling ABI

uint64_t gp_kernel_launch_count(void) { return g_launches.load(); }

gp_status gp_profile_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on != 0;
    return GP_OK;
}

gp_status gp_profile_read(gp_kernel_profile *out, int reset)
{
    if (!out) return GP_EINVAL;
    std::vector<ProfRec> recs;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        recs.swap(g_prof_pending);
    }
    for (auto &r : recs) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            std::lock_guard<std::mutex> lk(g_prof_mu);
            g_prof_ms[r.kind] += ms;
            g_prof_n[r.kind] += 1;
        }
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (int k = 0; k < GP_KERNEL_KINDS; ++k) {
        out->launches[k] = g_prof_n[k];
        out->total_ms[k] = g_prof_ms[k];
        if (reset) { g_prof_n[k] = 0; g_prof_ms[k] = 0.0; }
    }
    return GP_OK;
}

}  // extern "C"

namespace gpk {
void note_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace gpk
