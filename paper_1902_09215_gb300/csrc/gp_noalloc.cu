// gp_evaluate_noalloc: fitness evaluation that allocates nothing.
//
// Some callers cannot allocate device memory while they evaluate: a host
// loop that owns all GPU memory through its own allocator (and must not see
// memory appear behind its back), a latency-critical loop that cannot
// afford the implicit synchronisation of cudaMalloc / cudaFree, or a caller
// running with the stream-ordered pool disabled.  This entry point keeps all
// of the evaluator's scratch (work items, work counter, error word, fitness
// cases and constants) in one file-scope device array, and gives every warp a
// deep shared-memory operand window instead of a global spill area.  The
// caller passes device inputs and outputs.
#include <cstdint>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "gp.h"
#include "gp_internal.cuh"

using namespace gpk;

namespace {

constexpr size_t kCtlBytes = 4096;   // counter, error words, x, y, constants
constexpr size_t kItemBytes = (size_t)GP_NOALLOC_MAX_TREES * sizeof(EvalItem);
constexpr size_t kScratchBytes = kCtlBytes + kItemBytes + (size_t)GP_NOALLOC_MAX_TREES * sizeof(ValOut);
constexpr uint32_t kWindow = 256;    // operand-stack entries per warp (no spill area)

// Held by every GPU that loads libgp until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct Ctl {                          // layout of the first kCtlBytes
    uint32_t counter;
    uint32_t err[4];                  // [0] evaluator error bits, [1] malformed trees
    uint32_t pad[59];
    float x[kMaxCases];
    float y[kMaxCases];
    float consts[256];
};
static_assert(sizeof(Ctl) <= kCtlBytes, "control block");

std::mutex g_mu;
unsigned char *g_scratch_ptr[64] = {};   // device address of the array, per device

// Device address of the scratch array on the current device (looked up once
// per device with that device current).
gp_status scratch_address(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= 64) return GP_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return GP_ECUDA;
        }
        g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_ptr[dev];
    return GP_OK;
}

// True if [p, p + bytes) lies inside one device allocation (driver query
// through the runtime's entry-point lookup; unknown is treated as false).
bool readable_range(const void *p, size_t bytes)
{
    typedef int (*range_fn)(unsigned long long *, size_t *, unsigned long long);
    static range_fn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<range_fn>(f);
        cudaGetLastError();
    });
    if (!fn) return false;
    unsigned long long base = 0;
    size_t size = 0;
    if (fn(&base, &size, reinterpret_cast<unsigned long long>(p)) != 0) return false;
    return reinterpret_cast<unsigned long long>(p) + bytes <= base + size;
}

// One thread per tree: the tree (one chunk) must need no incoming operand,
// leave exactly one value and hold only defined codes.
__global__ void noalloc_check_kernel(const ValOut *__restrict__ v, uint32_t n, uint32_t *bad)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const ValOut c = v[t];
    if (c.bad_code || c.need > 0 || c.delta != 1) atomicAdd(bad, 1u);
}

int noalloc_lanes(uint32_t n_cases)
{
    return n_cases <= 16 ? 8 : n_cases <= 32 ? 16 : n_cases <= 48 ? 24 : 32;
}

}  // namespace

extern "C" gp_status gp_evaluate_noalloc(const gp_problem *problem, uint32_t n_trees,
                                         const uint8_t *d_nodes, const uint64_t *offsets,
                                         float *d_fitness, float *d_case_values, uint32_t *d_hits,
                                         void *cuda_stream)
{
    if (!problem || problem->n_cases == 0 || problem->n_cases > kMaxCases || !problem->x || !problem->y)
        return GP_EINVAL;
    if (problem->n_consts > kMaxConsts || (problem->n_consts && !problem->consts)) return GP_EINVAL;
    if (n_trees > GP_NOALLOC_MAX_TREES) return GP_ELIMIT;
    if (n_trees == 0) return GP_OK;
    if (!d_nodes || !offsets || !d_fitness || !d_case_values || !d_hits) return GP_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_nodes) % 16 || offsets[0] != 0) return GP_EINVAL;
    for (uint32_t t = 0; t < n_trees; ++t) {
        if (offsets[t + 1] <= offsets[t]) return GP_EINVAL;
        if (offsets[t + 1] - offsets[t] > GP_NOALLOC_MAX_TREE_NODES) return GP_ELIMIT;
    }
    // The evaluator reads whole 16-byte groups of codes.
    if (!readable_range(d_nodes, (offsets[n_trees] + 15) & ~15ull)) return GP_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GP_ECUDA;
    unsigned char *scratch = nullptr;
    gp_status st = scratch_address(dev, &scratch);
    if (st) return st;
    Ctl *ctl = reinterpret_cast<Ctl *>(scratch);
    EvalItem *items = reinterpret_cast<EvalItem *>(scratch + kCtlBytes);
    ValOut *checks = reinterpret_cast<ValOut *>(scratch + kCtlBytes + kItemBytes);

    // Problem tables and work items: built in fixed host buffers, copied in.
    const int lanes = noalloc_lanes(problem->n_cases);
    float tables[2 * kMaxCases + 256] = {};
    std::memcpy(tables, problem->x, sizeof(float) * problem->n_cases);
    std::memcpy(tables + kMaxCases, problem->y, sizeof(float) * problem->n_cases);
    if (problem->n_consts) std::memcpy(tables + 2 * kMaxCases, problem->consts, sizeof(float) * problem->n_consts);
    if (cudaMemcpyAsync(ctl->x, tables, sizeof(tables), cudaMemcpyHostToDevice, s) != cudaSuccess) return GP_ECUDA;
    if (cudaMemsetAsync(ctl, 0, offsetof(Ctl, pad), s) != cudaSuccess) return GP_ECUDA;   // counter, err
    EvalItem batch[256];
    for (uint32_t t0 = 0; t0 < n_trees; t0 += 256) {
        const uint32_t nb = (n_trees - t0) < 256 ? (n_trees - t0) : 256;
        for (uint32_t k = 0; k < nb; ++k) {
            EvalItem it{};
            it.begin = offsets[t0 + k];
            it.end = offsets[t0 + k + 1];
            it.tree = t0 + k;
            it.flags = kItemFinal;
            it.spill_off = kNoSpill;
            batch[k] = it;
        }
        // pageable source: the copy is complete when the call returns
        if (cudaMemcpyAsync(items + t0, batch, sizeof(EvalItem) * nb, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return GP_ECUDA;
    }

    // Validate first, as gp_create_population does: the evaluator indexes its
    // leaf table by code and assumes every tree is one complete prefix tree.
    if (launch_validate(d_nodes, items, n_trees, problem->n_consts, checks, s) != cudaSuccess) return GP_ECUDA;
    noalloc_check_kernel<<<(n_trees + 255) / 256, 256, 0, s>>>(checks, n_trees, &ctl->err[1]);
    if (cudaGetLastError() != cudaSuccess) return GP_ECUDA;
    uint32_t bad = 0;
    if (cudaMemcpyAsync(&bad, &ctl->err[1], sizeof(bad), cudaMemcpyDeviceToHost, s) != cudaSuccess) return GP_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GP_ECUDA;
    if (bad) return GP_EMALFORMED;

    // Launch shape: as many warps per SM as shared memory holds with the deep
    // window; the kernel attribute is only ever raised.
    int sms = 0, maxsm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int warps = 16;
    const int rows = (int)(1 + problem->n_consts);
    while (warps > 1 && eval_smem_bytes(lanes, warps, (int)kWindow, false, rows) > (size_t)maxsm) --warps;
    const size_t smem = eval_smem_bytes(lanes, warps, (int)kWindow, false, rows);
    if (smem > (size_t)maxsm) return GP_ECUDA;
    if (eval_prepare_at_least(lanes, false, smem) != cudaSuccess) return GP_ECUDA;

    EvalParams p{};
    p.codes = d_nodes;
    p.items = items;
    p.n_items = n_trees;
    p.counter = &ctl->counter;
    p.x = ctl->x;
    p.y = ctl->y;
    p.consts = ctl->consts;
    p.n_cases = problem->n_cases;
    p.n_consts = problem->n_consts;
    p.leaf_rows = (uint32_t)rows;
    p.div0 = problem->protected_div_value;
    p.window = kWindow;
    p.values = d_case_values;
    p.fitness = d_fitness;
    p.hits = d_hits;
    p.spill = nullptr;                 // no spill area: a deeper stack is an error
    p.spill_per_warp = 0;
    p.err = ctl->err;
    if (launch_eval(lanes, false, p, sms, warps, smem, s) != cudaSuccess) return GP_ECUDA;

    uint32_t err = 0;
    if (cudaMemcpyAsync(&err, ctl->err, sizeof(err), cudaMemcpyDeviceToHost, s) != cudaSuccess) return GP_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GP_ECUDA;
    if (err & kErrSpill) return GP_ELIMIT;
    if (err & kErrMalformed) return GP_EMALFORMED;
    if (err) return GP_ECUDA;
    return GP_OK;
}
