// Level-0 work items built on the device for trees whose sizes never came
// back to the host (children of a crossover that did not synchronise).
#include <cstdint>
#include <cuda_runtime.h>

#include "gp_internal.cuh"

namespace gpk {

// Level-0 items of a population whose tree sizes are on the device only and
// at most max_chunks chunks of C codes, in three grid-wide steps: (1) every
// tree adds its chunk count (multi-chunk trees, also one rope) or one final
// to its size class (floor of log2); (2) one thread turns the class counts
// into cursors, larger classes first: the chunks of every multi-chunk tree
// (fused items, the tree's slots consecutive), then every single-chunk tree
// as a final item, and the ropes for the next launch; (3) every tree takes
// its places from the cursors.  counts: [0] level-0 items, [1] ropes,
// [2] slots (one per chunk).  `cls` (3 x 64 cursors and the slot cursor)
// starts zeroed.
// Items of one class are in no particular order (the results do not depend
// on the order).
constexpr int kCls = 64;

__device__ __forceinline__ int size_class(uint64_t z) { return 63 - __clzll((long long)(z | 1)); }

__global__ void plan0_count_kernel(const uint64_t *__restrict__ size, uint32_t n, uint32_t C, uint32_t *cls)
{
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const uint64_t z = size[t];
        const int c = size_class(z);
        if (z > C) {
            atomicAdd(&cls[c], (uint32_t)((z + C - 1) / C));
            atomicAdd(&cls[2 * kCls + c], 1u);
        } else {
            atomicAdd(&cls[kCls + c], 1u);
        }
    }
}

__global__ void plan0_bases_kernel(uint32_t *cls, uint32_t *counts)
{
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
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * kCls; i += blockDim.x) cls[i] = v[i];
}

__global__ void plan0_place_kernel(const uint64_t *__restrict__ start, const uint64_t *__restrict__ size, uint32_t n,
                                   uint32_t C, EvalItem *__restrict__ items, EvalItem *__restrict__ ropes, uint32_t *cls)
{
    uint32_t *slots = cls + 3 * kCls;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const uint64_t z = size[t], b = start[t];
        const int c = size_class(z);
        if (z > C) {
            const uint32_t m = (uint32_t)((z + C - 1) / C);
            const uint32_t p = atomicAdd(&cls[c], m);
            const uint32_t slot = atomicAdd(slots, m);
            for (uint32_t j = 0; j < m; ++j) {
                EvalItem it{};
                it.begin = b + (uint64_t)j * C;
                it.end = b + umin64(z, (uint64_t)(j + 1) * C);
                it.tree = t;
                it.flags = kItemFused;
                it.frag_off = slot + j;
                it.pt_base = slot;
                it.frag_len = m;
                it.spill_off = kNoSpill;
                items[p + j] = it;
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

uint32_t plan_level0_scratch_words() { return 3 * kCls + 1; }

cudaError_t launch_plan_level0(const uint64_t *start, const uint64_t *size, uint32_t n, uint32_t C,
                               EvalItem *items, EvalItem *ropes, uint32_t *counts, uint32_t *cls, int sms,
                               cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const uint32_t blocks = (uint32_t)umin64((n + 255) / 256, (uint64_t)sms * 4);
    plan0_count_kernel<<<blocks, 256, 0, s>>>(size, n, C, cls);
    plan0_bases_kernel<<<1, 3 * kCls, 0, s>>>(cls, counts);
    plan0_place_kernel<<<blocks, 256, 0, s>>>(start, size, n, C, items, ropes, cls);
    return cudaGetLastError();
}

}  // namespace gpk
