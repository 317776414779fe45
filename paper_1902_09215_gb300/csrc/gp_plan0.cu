// Level-0 work items built on the device for trees whose sizes never came
// back to the host (children of a crossover that did not synchronise).
#include <cstdint>
#include <cuda_runtime.h>

#include "gp_internal.cuh"

namespace gpk {

// Level-0 items of a population whose tree sizes are on the device only and
// at most max_chunks chunks of C codes, in three grid-wide steps: (1) every
// multi-chunk tree is cut into chunks (`cut_low`) and adds its chunk count
// and one rope to its size class (floor of log2), every other tree one final
// item; (2) one thread turns the class counts into cursors, larger classes
// first: the chunks of every multi-chunk tree (fused items, the tree's slots
// consecutive), then every single-chunk tree as a final item, and the ropes
// for the next launch; (3) every tree takes its places from the cursors.
// counts: [0] level-0 items, [1] ropes, [2] slots (one per chunk).  `cls`
// (3 x 64 cursors, the slot cursor and the cut cursor) starts zeroed.
// Items of one class are in no particular order (the results do not depend
// on the order).
constexpr int kCls = 64;

__device__ __forceinline__ int size_class(uint64_t z) { return 63 - __clzll((long long)(z | 1)); }

// One warp per tree.  A multi-chunk tree's ends go to cuts[base .. base +
// chunks - 2] (relative to the tree's start), base from the cut cursor;
// meta[t] = base << 5 | (chunks - 1).
__global__ void plan0_count_kernel(const uint8_t *__restrict__ arena, const uint64_t *__restrict__ start,
                                   const uint64_t *__restrict__ size, uint32_t n, uint32_t C, uint32_t mcap_max,
                                   uint32_t *cls, uint32_t *meta, uint32_t *cuts)
{
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t t = warp; t < n; t += warps) {
        const uint64_t z = size[t];
        const int c = size_class(z);
        if (z <= C) {
            if (lane == 0) atomicAdd(&cls[kCls + c], 1u);
            continue;
        }
        const uint64_t b = start[t];
        const uint32_t m = (uint32_t)((z + C - 1) / C);
        const uint32_t mcap = min(m + 1, max(m, mcap_max));
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(&cls[3 * kCls + 1], mcap - 1);
        base = __shfl_sync(0xffffffffu, base, 0);
        const uint32_t k = cut_low(arena, b, z, C, mcap, lane, [&](uint32_t j, uint64_t e) {
            if (lane == 0) cuts[base + j - 1] = (uint32_t)(e - b);
        });
        if (lane == 0) {
            meta[t] = (base << 5) | (k - 1);
            atomicAdd(&cls[c], k);
            atomicAdd(&cls[2 * kCls + c], 1u);
        }
    }
}

// Zeroes the planner's scratch words and the population's evaluation
// words: err[0..3] (error words), stat[4..6] (what level 0 sends upward),
// err[12] (the redo count); stat[3] (the crossover layout's error) stays.
__global__ void plan0_zero_kernel(uint32_t *__restrict__ zero, uint32_t n_zero, uint32_t *err, uint32_t *stat)
{
    pdl_wait();
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_zero; i += gridDim.x * blockDim.x) zero[i] = 0;
    if (blockIdx.x == 0 && threadIdx.x < 4) err[threadIdx.x] = 0;
    if (blockIdx.x == 0 && threadIdx.x >= 4 && threadIdx.x < 7) stat[threadIdx.x] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 7) err[12] = 0;
}

// counts[0..2] (and stat[0..2] when given) from the class counts.
__global__ void plan0_bases_kernel(uint32_t *cls, uint32_t *counts, uint32_t *stat)
{
    pdl_wait();
    __shared__ uint32_t v[3 * kCls];
    for (int i = threadIdx.x; i < 3 * kCls; i += blockDim.x) v[i] = cls[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t pos = 0, r = 0;
        for (int c = kCls - 1; c >= 0; --c) {
            const uint32_t x = v[c];
            v[c] = pos;
            pos += x;
        }
        counts[2] = pos;                 // one slot per chunk
        for (int c = kCls - 1; c >= 0; --c) {
            const uint32_t x = v[kCls + c];
            v[kCls + c] = pos;
            pos += x;
        }
        for (int c = kCls - 1; c >= 0; --c) {
            const uint32_t x = v[2 * kCls + c];
            v[2 * kCls + c] = r;
            r += x;
        }
        counts[0] = pos;
        counts[1] = r;
        if (stat) {
            stat[0] = pos;
            stat[1] = r;
            stat[2] = counts[2];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * kCls; i += blockDim.x) cls[i] = v[i];
}

__global__ void plan0_place_kernel(const uint64_t *__restrict__ start, const uint64_t *__restrict__ size, uint32_t n,
                                   uint32_t C, const uint32_t *__restrict__ meta, const uint32_t *__restrict__ cuts,
                                   EvalItem *__restrict__ items, EvalItem *__restrict__ ropes, uint32_t *cls)
{
    pdl_wait();
    uint32_t *slots = cls + 3 * kCls;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const uint64_t z = size[t], b = start[t];
        const int c = size_class(z);
        if (z > C) {
            const uint32_t mt = meta[t], m = (mt & 31u) + 1, base = mt >> 5;
            const uint32_t p = atomicAdd(&cls[c], m);
            const uint32_t slot = atomicAdd(slots, m);
            uint64_t lo = b;
            for (uint32_t j = 0; j < m; ++j) {
                const uint64_t hi = j + 1 < m ? b + cuts[base + j] : b + z;
                EvalItem it{};
                it.begin = lo;
                it.end = hi;
                it.tree = t;
                it.flags = kItemFused;
                it.frag_off = slot + j;
                it.pt_base = slot;
                it.frag_len = m;
                it.spill_off = kNoSpill;
                items[p + j] = it;
                lo = hi;
            }
            EvalItem r{};
            r.tree = t;
            r.flags = kItemFinal | kItemRope;
            r.pt_base = slot;
            r.frag_len = m;
            r.spill_off = kNoSpill;
            ropes[atomicAdd(&cls[2 * kCls + c], 1u)] = r;
        } else {
            EvalItem it{};
            it.begin = b;
            it.end = b + z;
            it.tree = t;
            it.flags = kItemFinal;
            it.spill_off = kNoSpill;
            items[atomicAdd(&cls[kCls + c], 1u)] = it;
        }
    }
}

uint32_t plan_level0_scratch_words() { return 3 * kCls + 2; }

cudaError_t launch_plan_level0(const uint8_t *arena, const uint64_t *start, const uint64_t *size, uint32_t n,
                               uint32_t C, uint32_t max_chunks, EvalItem *items, EvalItem *ropes, uint32_t *counts,
                               uint32_t *cls, uint32_t *meta, uint32_t *cuts, uint32_t *zero, uint32_t n_zero,
                               uint32_t *err, uint32_t *stat, int sms, cudaStream_t s)
{
    if (max_chunks == 0 || max_chunks > 32) return cudaErrorInvalidValue;   // meta holds chunks - 1 in 5 bits
    if (n == 0) return cudaSuccess;
    const uint32_t blocks = (uint32_t)umin64((n + 255) / 256, (uint64_t)sms * 4);
    const uint32_t warp_blocks = (uint32_t)umin64((n + 7) / 8, (uint64_t)sms * 16);   // a warp per tree
    cudaError_t e = launch_pdl(plan0_zero_kernel, dim3((uint32_t)umin64((n_zero + 255) / 256 + 1, (uint64_t)sms * 4)),
                               dim3(256), 0, s, zero, n_zero, err, stat);
    if (e != cudaSuccess) return e;
    e = launch_pdl(plan0_count_kernel, dim3(warp_blocks), dim3(256), 0, s, arena, start, size, n, C, max_chunks, cls,
                   meta, cuts);
    if (e != cudaSuccess) return e;
    e = launch_pdl(plan0_bases_kernel, dim3(1), dim3(3 * kCls), 0, s, cls, counts, stat);
    if (e != cudaSuccess) return e;
    return launch_pdl(plan0_place_kernel, dim3(blocks), dim3(256), 0, s, start, size, n, C, meta, cuts, items, ropes,
                      cls);
}

}  // namespace gpk
