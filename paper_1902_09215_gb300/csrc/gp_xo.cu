// Subtree crossover on the device (Sec. 3.1, Sec. 2.3): the host chooses the
// points sequentially; the device finds the two subtree extents and copies
// child = mum[0,i) ++ dad[j,e_d) ++ mum[e_m,n_m).
#include <cstdint>
#include <cuda_runtime.h>

#include "gp_internal.cuh"

namespace gpk {

// The end (exclusive) of the subtree rooted at `point`.  Reading left to
// right, `need` counts subtrees still to be read: an operator adds one, a
// leaf removes one; the subtree ends where it reaches zero.  Two phases:
// every query first takes one step of one warp (32 lanes x 16 bytes from a
// 16-byte aligned base: most subtrees are a few nodes); a query still open
// after it goes to a list that the second kernel walks with a whole CTA
// per query (512 threads x 32 bytes: 16 KB per step), since a query's time
// is its number of dependent steps and few subtrees are long.  Bytes before `point` or past the tree do not count; a
// lane loads only if its first byte is inside the tree, and trees are
// followed by at least 64 padding bytes.
constexpr uint32_t kExtLane = 16;
constexpr int kExtT = 512;                  // threads of a long-query CTA
constexpr uint32_t kExtThr = 32;            // bytes per thread and step there

// Arity walk over the four bytes of w (byte 0 first): +1 for an operator
// (code < 4), -1 for a leaf, 0 for a byte whose byte in `cm` is zero.
// *net: the change over the word; returns the lowest running value after
// each of its bytes.  Byte-wise, without carries between bytes: bit 7 of
// ((w & 0x7c) + 0x7f) | w is set exactly when the byte is >= 4; e = 2 for
// an operator, 0 for a leaf, 1 for a byte that does not count; multiplying
// by 0x01010101 puts e_0 + ... + e_k (at most 8) in byte k, and the
// running value after byte k is that sum - (k + 1).
__device__ __forceinline__ int walk_word(uint32_t w, uint32_t cm, int *net)
{
    const uint32_t nz = ((w & 0x7c7c7c7cu) + 0x7f7f7f7fu) | w;
    uint32_t e = (~nz & 0x80808080u) >> 6;
    e = (e & cm) | (0x01010101u & ~cm);
    const uint32_t E = e * 0x01010101u;
    const uint32_t M = E + 0x00010203u;          // byte k: running value after byte k, + 4
    uint32_t m = __vminu4(M, M >> 16);
    m = __vminu4(m, m >> 8);
    *net = (int)(E >> 24) - 4;
    return (int)(m & 0xffu) - 4;
}

// Bytes x.. of a word (x <= 0: all four, x >= 4: none).
__device__ __forceinline__ uint32_t bytes_from(int x)
{
    return __funnelshift_lc(0u, 0xffffffffu, 8u * (uint32_t)max(x, 0));
}

// (net change, lowest running value) over bytes [ia, ib) of the NW words
// of v; the lowest value is no higher than the value before the first
// counted byte (a word with no counted byte reports that value), which
// cannot close a walk that has not closed before.
template <int NW>
__device__ __forceinline__ void walk_bytes(const uint32_t *v, int ia, int ib, int &s, int &mn)
{
    s = 0;
    mn = 1 << 30;
#pragma unroll
    for (int k = 0; k < NW; ++k) {
        const uint32_t cm = bytes_from(ia - 4 * k) & ~bytes_from(ib - 4 * k);
        int net;
        const int wm = walk_word(v[k], cm, &net);
        mn = min(mn, s + wm);
        s += net;
    }
}

// First byte j in [ia, ib) of v's bytes where the running value, starting
// from r, reaches zero (-1 if none).
template <int NB>
__device__ __forceinline__ int first_close(const uint32_t *v, int ia, int ib, int64_t r)
{
    int e = -1;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        if (e < 0 && j >= ia && j < ib) {
            r += ((v[j >> 2] >> (8 * (j & 3))) & 0xFFu) < 4 ? 1 : -1;
            if (r == 0) e = j;
        }
    }
    return e;
}

__device__ __forceinline__ void extent_one(const uint8_t *__restrict__ arena, const ExtentQuery *__restrict__ q,
                                           uint32_t w, int lane, uint64_t *__restrict__ end_out,
                                           uint32_t *err, ExtentLong *__restrict__ list, uint32_t *n_long)
{
    const ExtentQuery Q = q[w];
    const uint64_t tend = Q.tree_start + Q.tree_size;
    const uint64_t p0 = Q.tree_start + Q.point;
    const uint64_t base = p0 & ~15ull;
    if (base >= tend) {
        if (lane == 0) {
            atomicOr(err, kErrExtent);
            end_out[w] = Q.tree_size;
        }
        return;
    }
    const uint64_t lo = base + (uint64_t)kExtLane * lane;
    uint32_t v[kExtLane / 4];
#pragma unroll
    for (int k = 0; k < (int)(kExtLane / 16); ++k) {
        const uint4 x = lo < tend ? __ldg(reinterpret_cast<const uint4 *>(arena + lo) + k) : make_uint4(0, 0, 0, 0);
        v[4 * k] = x.x;
        v[4 * k + 1] = x.y;
        v[4 * k + 2] = x.z;
        v[4 * k + 3] = x.w;
    }
    // bytes [ia, ib) of this lane's kExtLane count
    const int ia = p0 > lo ? (int)umin64(p0 - lo, kExtLane) : 0;
    const int ib = tend > lo ? (int)umin64(tend - lo, kExtLane) : 0;
    int s, mn;
    walk_bytes<kExtLane / 4>(v, ia, ib, s, mn);
    // exclusive prefix of s over lanes
    int incl = s;
    for (int off = 1; off < 32; off <<= 1) {
        const int o = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += o;
    }
    const int excl = incl - s;
    const bool closes = 1 + excl + mn <= 0;
    const unsigned ball = __ballot_sync(0xffffffffu, closes);
    if (ball) {
        if (lane == __ffs(ball) - 1)
            end_out[w] = lo + (uint64_t)first_close<kExtLane>(v, ia, ib, 1 + excl) + 1 - Q.tree_start;
        return;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (lane == 0) list[atomicAdd(n_long, 1u)] = ExtentLong{base + 32ull * kExtLane, 1 + (int64_t)total, w, 0};
}

// A CTA per query of the list: 16 KB per step, a block scan of the
// threads' net changes, the first thread whose bytes close the walk.
__global__ void __launch_bounds__(kExtT) extent_long_kernel(const uint8_t *__restrict__ arena,
                                                          const ExtentQuery *__restrict__ q,
                                                          const ExtentLong *__restrict__ list,
                                                          const uint32_t *n_long, uint64_t *__restrict__ end_out,
                                                          uint32_t *err)
{
    pdl_wait();
    __shared__ int s_wsum[kExtT / 32];
    __shared__ int s_first;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const uint32_t n = *n_long;
    for (uint32_t i = blockIdx.x; i < n; i += gridDim.x) {
        const ExtentLong L = list[i];
        const ExtentQuery Q = q[L.w];
        const uint64_t tend = Q.tree_start + Q.tree_size;
        uint64_t base = L.base;                        // 16-aligned, past the query's point
        int64_t need = L.need;
        for (;;) {
            if (base >= tend) {
                if (tid == 0) {
                    atomicOr(err, kErrExtent);
                    end_out[L.w] = Q.tree_size;
                }
                break;
            }
            if (tid == 0) s_first = kExtT;
            const uint64_t lo = base + (uint64_t)kExtThr * tid;
            uint32_t v[kExtThr / 4];
#pragma unroll
            for (int k = 0; k < (int)(kExtThr / 16); ++k) {
                const uint4 x =
                    lo < tend ? __ldg(reinterpret_cast<const uint4 *>(arena + lo) + k) : make_uint4(0, 0, 0, 0);
                v[4 * k] = x.x;
                v[4 * k + 1] = x.y;
                v[4 * k + 2] = x.z;
                v[4 * k + 3] = x.w;
            }
            const int ib = tend > lo ? (int)umin64(tend - lo, kExtThr) : 0;
            int s, mn;
            walk_bytes<kExtThr / 4>(v, 0, ib, s, mn);
            int incl = s;
            for (int off = 1; off < 32; off <<= 1) {
                const int o = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += o;
            }
            if (lane == 31) s_wsum[wid] = incl;
            __syncthreads();
            int before = 0, total = 0;
#pragma unroll
            for (int k = 0; k < kExtT / 32; ++k) {
                const int x = s_wsum[k];
                before += k < wid ? x : 0;
                total += x;
            }
            const int64_t r0 = need + before + incl - s;   // the running value before this thread's bytes
            if (r0 + mn <= 0) atomicMin(&s_first, tid);
            __syncthreads();
            const int f = s_first;
            if (f < kExtT) {
                if (tid == f) end_out[L.w] = lo + (uint64_t)first_close<kExtThr>(v, 0, ib, r0) + 1 - Q.tree_start;
                break;
            }
            need += total;
            base += (uint64_t)kExtT * kExtThr;
            __syncthreads();                               // s_wsum and s_first are written again
        }
        __syncthreads();
    }
}

// (8 CTAs of 256 per SM: the 8000 queries of 4000 children in one wave)
__global__ void __launch_bounds__(256, 8) extent_kernel(const uint8_t *__restrict__ arena, const ExtentQuery *__restrict__ q,
                              uint32_t n, uint64_t *__restrict__ end_out, uint32_t *err,
                              ExtentLong *__restrict__ list, uint32_t *n_long)
{
    const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= n) return;
    extent_one(arena, q, w, threadIdx.x & 31, end_out, err, list, n_long);
}

// Same, with the query count read on the device and a grid-stride loop.
__global__ void __launch_bounds__(256, 8) extent_dev_kernel(const uint8_t *__restrict__ arena, const ExtentQuery *__restrict__ q,
                                  uint32_t n_max, const uint32_t *n_dev, uint64_t *__restrict__ end_out,
                                  uint32_t *err, ExtentLong *__restrict__ list, uint32_t *n_long)
{
    pdl_wait();
    const uint32_t n = min(n_max, *n_dev);
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n; w += n_warps)
        extent_one(arena, q, w, threadIdx.x & 31, end_out, err, list, n_long);
}

cudaError_t launch_extent(const uint8_t *arena, const ExtentQuery *q, uint32_t n, uint64_t *end, uint32_t *err,
                          ExtentLong *list, uint32_t *n_long, int sms, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const int threads = 256;
    const uint32_t blocks = (uint32_t)(((uint64_t)n * 32 + threads - 1) / threads);
    extent_kernel<<<blocks, threads, 0, s>>>(arena, q, n, end, err, list, n_long);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_pdl(extent_long_kernel, dim3((uint32_t)umin64(n, (uint64_t)sms * 4)), dim3(kExtT), 0, s, arena, q,
                      (const ExtentLong *)list, (const uint32_t *)n_long, end, err);
}

cudaError_t launch_extent_dev(const uint8_t *arena, const ExtentQuery *q, uint32_t n_max, const uint32_t *n_dev,
                              uint64_t *end, uint32_t *err, ExtentLong *list, uint32_t *n_long, int sms,
                              cudaStream_t s)
{
    if (n_max == 0) return cudaSuccess;
    const int threads = 256;
    const uint64_t want = ((uint64_t)n_max * 32 + threads - 1) / threads;
    const uint32_t blocks = (uint32_t)umin64(want, (uint64_t)sms * 16);
    cudaError_t e = launch_pdl(extent_dev_kernel, dim3(blocks), dim3(threads), 0, s, arena, q, n_max, n_dev, end, err,
                               list, n_long);
    if (e != cudaSuccess) return e;
    return launch_pdl(extent_long_kernel, dim3((uint32_t)umin64(n_max, (uint64_t)sms * 4)), dim3(kExtT), 0, s, arena,
                      q, (const ExtentLong *)list, (const uint32_t *)n_long, end, err);
}


// Source byte of child byte p.
__device__ __forceinline__ uint64_t xo_src(const XoChild &c, uint64_t p) {
    if (p < c.i) return c.head_src + p;
    if (p < c.i + c.ld) return c.mid_src + (p - c.i);
    return c.tail_src + (p - c.i - c.ld);
}

// Sixteen source bytes starting at byte address a (any alignment), from five
// aligned words.  Sources are padded by at least 8 bytes on both ends.
__device__ __forceinline__ uint4 load16_unaligned(const uint8_t *src, uint64_t a) {
    const uint32_t *w = reinterpret_cast<const uint32_t *>(src + (a & ~3ull));
    const uint32_t w0 = __ldg(w), w1 = __ldg(w + 1), w2 = __ldg(w + 2), w3 = __ldg(w + 3), w4 = __ldg(w + 4);
    const uint32_t sel = 0x3210u + 0x1111u * (uint32_t)(a & 3);
    return make_uint4(__byte_perm(w0, w1, sel), __byte_perm(w1, w2, sel), __byte_perm(w2, w3, sel),
                      __byte_perm(w3, w4, sel));
}

// One tile of one child, by the threads first, first + stride, ... of a
// CTA or a warp; every thread writes aligned 16-byte words
// (children start 16-byte aligned, tiles are multiples of 16 bytes; the
// bytes from the child's end to the next 16-byte boundary are its padding
// and are written as zeros).  A word inside one of the child's three
// segments is assembled from aligned loads; the few words across a segment
// boundary or the child's end go byte by byte.
__device__ __forceinline__ void copy_tile(const uint8_t *__restrict__ src, uint8_t *__restrict__ dst,
                                          const XoChild &c, uint64_t tbegin, uint32_t tile_bytes,
                                          uint32_t first, uint32_t stride)
{
    const uint64_t tend = umin64(tbegin + tile_bytes, (c.n + 15) & ~15ull);
    uint4 *d16 = reinterpret_cast<uint4 *>(dst + c.dst);
    const uint64_t b1 = c.i, b2 = c.i + c.ld;
#pragma unroll 4
    for (uint64_t p = tbegin + 16ull * first; p < tend; p += 16ull * stride) {
        uint4 v;
        const uint64_t q = p + 15;
        const bool one_seg = (q < c.n) && ((q < b1) || (p >= b1 && q < b2) || (p >= b2));
        if (one_seg) {
            v = load16_unaligned(src, xo_src(c, p));
        } else {
            uint32_t w[4] = {0, 0, 0, 0};
            for (int k = 0; k < 16; ++k)
                if (p + k < c.n) w[k >> 2] |= (uint32_t)src[xo_src(c, p + k)] << (8 * (k & 3));
            v = make_uint4(w[0], w[1], w[2], w[3]);
        }
        d16[p >> 4] = v;
    }
}

__global__ void xo_copy_kernel(const uint8_t *__restrict__ src, uint8_t *__restrict__ dst,
                               const XoChild *__restrict__ children, const XoTile *__restrict__ tiles,
                               uint32_t tile_bytes)
{
    const XoTile T = tiles[blockIdx.x];
    copy_tile(src, dst, children[T.child], T.begin, tile_bytes, threadIdx.x, blockDim.x);
}

// Tiles numbered on the device: a CTA takes tiles t = blockIdx.x, +gridDim.x,
// ... and finds the owning child by binary search over tile_base.
__global__ void xo_copy_dev_kernel(const uint8_t *__restrict__ src, uint8_t *__restrict__ dst,
                                   const XoChild *__restrict__ children,
                                   const uint32_t *__restrict__ tile_base, uint32_t n_children,
                                   const uint32_t *n_tiles_dev, uint32_t tile_bytes)
{
    const uint32_t n_tiles = *n_tiles_dev;
    for (uint32_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        uint32_t lo = 0, hi = n_children;          // last c with tile_base[c] <= t
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (tile_base[mid] <= t) lo = mid;
            else hi = mid;
        }
        copy_tile(src, dst, children[lo], (uint64_t)(t - tile_base[lo]) * tile_bytes, tile_bytes, threadIdx.x,
                  blockDim.x);
    }
}

cudaError_t launch_xo_copy(const uint8_t *src, uint8_t *dst, const XoChild *children,
                           const XoTile *tiles, uint32_t n_tiles, uint32_t tile_bytes,
                           cudaStream_t s)
{
    if (n_tiles == 0) return cudaSuccess;
    xo_copy_kernel<<<n_tiles, 256, 0, s>>>(src, dst, children, tiles, tile_bytes);
    return cudaGetLastError();
}

// Children of a batch of runs in one heap: tile t belongs to the last run
// whose first tile is <= t, then to the last of that run's children whose
// first tile (counted within the run) is <= the tile's index in the run.
// A CTA per tile, or a warp per tile (WARP, small children).
template <bool WARP>
__global__ void xo_copy_runs_kernel(uint8_t *__restrict__ heap, const XoChild *__restrict__ kids,
                                    const uint32_t *__restrict__ tile_local, const uint32_t *__restrict__ tree_base,
                                    const uint32_t *__restrict__ run_tile_base, const uint32_t *n_runs_dev,
                                    const uint32_t *n_tiles_dev, uint32_t tile_bytes)
{
    pdl_wait();
    const uint32_t n_tiles = *n_tiles_dev, n_runs = *n_runs_dev;
    const uint32_t first = WARP ? (threadIdx.x & 31) : threadIdx.x, stride = WARP ? 32 : blockDim.x;
    const uint32_t unit = WARP ? (blockIdx.x * blockDim.x + threadIdx.x) >> 5 : blockIdx.x;
    const uint32_t units = WARP ? (gridDim.x * blockDim.x) >> 5 : gridDim.x;
    for (uint32_t t = unit; t < n_tiles; t += units) {
        uint32_t lo = 0, hi = n_runs;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (run_tile_base[mid] <= t) lo = mid;
            else hi = mid;
        }
        const uint32_t lt = t - run_tile_base[lo];
        uint32_t a = tree_base[lo], b = tree_base[lo + 1];
        while (b - a > 1) {
            const uint32_t mid = (a + b) >> 1;
            if (tile_local[mid] <= lt) a = mid;
            else b = mid;
        }
        copy_tile(heap, heap, kids[a], (uint64_t)(lt - tile_local[a]) * tile_bytes, tile_bytes, first, stride);
    }
}

cudaError_t launch_xo_copy_runs(uint8_t *heap, const XoChild *kids, const uint32_t *tile_local,
                                const uint32_t *tree_base, const uint32_t *run_tile_base,
                                const uint32_t *n_runs_dev, const uint32_t *n_tiles_dev, uint32_t tile_bytes,
                                bool warp_tiles, int sms, cudaStream_t s)
{
    if (warp_tiles)
        return launch_pdl(xo_copy_runs_kernel<true>, dim3(sms * 8), dim3(256), 0, s, heap, kids, tile_local, tree_base,
                          run_tile_base, n_runs_dev, n_tiles_dev, tile_bytes);
    return launch_pdl(xo_copy_runs_kernel<false>, dim3(sms * 8), dim3(256), 0, s, heap, kids, tile_local, tree_base,
                      run_tile_base, n_runs_dev, n_tiles_dev, tile_bytes);
}

// Exclusive scan of a (64-bit, 32-bit) pair over the CTA (a multiple of 32
// threads, at most 1024), with the block totals.
__device__ __forceinline__ void block_scan_pair(uint64_t a, uint32_t b, uint64_t &ea, uint32_t &eb,
                                                uint64_t &ta, uint32_t &tb)
{
    __shared__ uint64_t wa[33];
    __shared__ uint32_t wb[33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint64_t ia = a;
    uint32_t ib = b;
    for (int off = 1; off < 32; off <<= 1) {
        const uint64_t oa = __shfl_up_sync(0xffffffffu, ia, off);
        const uint32_t ob = __shfl_up_sync(0xffffffffu, ib, off);
        if (lane >= off) {
            ia += oa;
            ib += ob;
        }
    }
    if (lane == 31) {
        wa[warp] = ia;
        wb[warp] = ib;
    }
    __syncthreads();
    if (threadIdx.x == 0) {              // at most 32 warp totals: a serial pass
        uint64_t sa = 0;
        uint32_t sb = 0;
        for (int w = 0; w < nw; ++w) {
            const uint64_t x = wa[w];
            const uint32_t y = wb[w];
            wa[w] = sa;
            wb[w] = sb;
            sa += x;
            sb += y;
        }
        wa[32] = sa;
        wb[32] = sb;
    }
    __syncthreads();
    ea = wa[warp] + (ia - a);
    eb = wb[warp] + (ib - b);
    ta = wa[32];
    tb = wb[32];
    __syncthreads();                     // the arrays are reused by the next call
}

// Children laid out on the device in three grid-wide steps: (1) every
// child's size i + (e_d - j) + (n_m - e_m) from its two extents, and per CTA
// the sums of the children's 16-byte aligned lengths and copy tiles; (2) one
// CTA scans those sums; (3) every CTA scans its children again from its
// offset: start, copy record, first copy tile.  A child that would end past
// the arena's capacity (not possible when the capacity was sized from the
// bound n_m + n_d - j - 1) is not copied and sets kErrExtent.
constexpr int kLayoutT = 256;

__device__ __forceinline__ uint64_t child_size(const ExtentQuery *__restrict__ q, const uint64_t *__restrict__ ends,
                                               uint32_t k)
{
    return q[2 * k].point + (ends[2 * k + 1] - q[2 * k + 1].point) + (q[2 * k].tree_size - ends[2 * k]);
}

__global__ void __launch_bounds__(kLayoutT) xo_size_kernel(const ExtentQuery *__restrict__ q,
                                                           const uint64_t *__restrict__ ends, uint32_t n,
                                                           uint32_t tile_bytes, uint64_t *__restrict__ csize,
                                                           uint64_t *__restrict__ part_len, uint32_t *__restrict__ part_tiles)
{
    pdl_wait();
    const uint32_t k = blockIdx.x * kLayoutT + threadIdx.x;
    uint64_t z = 0;
    if (k < n) {
        z = child_size(q, ends, k);
        csize[k] = z;
    }
    uint64_t ea, ta;
    uint32_t eb, tb;
    block_scan_pair((z + 15) & ~15ull, (uint32_t)((z + tile_bytes - 1) / tile_bytes), ea, eb, ta, tb);
    if (threadIdx.x == 0) {
        part_len[blockIdx.x] = ta;
        part_tiles[blockIdx.x] = tb;
    }
}

__global__ void __launch_bounds__(1024) xo_part_scan_kernel(uint64_t *__restrict__ part_len,
                                                            uint32_t *__restrict__ part_tiles, uint32_t n_parts,
                                                            uint32_t *__restrict__ tile_base, uint32_t n,
                                                            uint32_t *n_tiles)
{
    pdl_wait();
    __shared__ uint64_t carry_len;
    __shared__ uint32_t carry_t;
    if (threadIdx.x == 0) {
        carry_len = 0;
        carry_t = 0;
    }
    __syncthreads();
    for (uint32_t base = 0; base < n_parts; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const uint64_t a = i < n_parts ? part_len[i] : 0;
        const uint32_t b = i < n_parts ? part_tiles[i] : 0;
        uint64_t ea, ta;
        uint32_t eb, tb;
        block_scan_pair(a, b, ea, eb, ta, tb);
        if (i < n_parts) {
            part_len[i] = carry_len + ea;
            part_tiles[i] = carry_t + eb;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            carry_len += ta;
            carry_t += tb;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        tile_base[n] = carry_t;
        *n_tiles = carry_t;
    }
}

__global__ void __launch_bounds__(kLayoutT) xo_place_kernel(const ExtentQuery *__restrict__ q,
                                                            const uint64_t *__restrict__ ends, uint32_t n,
                                                            uint32_t tile_bytes, uint64_t arena_cap,
                                                            const uint64_t *__restrict__ part_len,
                                                            const uint32_t *__restrict__ part_tiles,
                                                            XoChild *__restrict__ kids, uint64_t *__restrict__ cstart,
                                                            const uint64_t *__restrict__ csize,
                                                            uint32_t *__restrict__ tile_base,
                                                            uint32_t *__restrict__ tile_child, uint32_t *err)
{
    pdl_wait();
    const uint32_t k = blockIdx.x * kLayoutT + threadIdx.x;
    const uint64_t z = k < n ? csize[k] : 0;
    const uint64_t alen = (z + 15) & ~15ull;
    uint64_t ea, ta;
    uint32_t eb, tb;
    block_scan_pair(alen, (uint32_t)((z + tile_bytes - 1) / tile_bytes), ea, eb, ta, tb);
    if (k >= n) return;
    const uint64_t start = part_len[blockIdx.x] + ea;
    const ExtentQuery qm = q[2 * k], qd = q[2 * k + 1];
    XoChild c{};
    c.dst = start;
    c.n = z;
    c.head_src = qm.tree_start;
    c.i = qm.point;
    c.mid_src = qd.tree_start + qd.point;
    c.ld = ends[2 * k + 1] - qd.point;
    c.tail_src = qm.tree_start + ends[2 * k];
    if (start + alen + 64 > arena_cap) {
        atomicOr(err, kErrExtent);
        c.n = 0;
    }
    kids[k] = c;
    cstart[k] = start;
    const uint32_t tb0 = part_tiles[blockIdx.x] + eb;
    tile_base[k] = tb0;
    const uint32_t nt = (uint32_t)((z + tile_bytes - 1) / tile_bytes);
    for (uint32_t i = 0; i < nt; ++i) tile_child[tb0 + i] = k;     // the copy's tile -> child map
}

uint32_t xo_layout_parts(uint32_t n) { return (n + kLayoutT - 1) / kLayoutT; }

cudaError_t launch_xo_layout(const ExtentQuery *q, const uint64_t *ends, uint32_t n, uint32_t tile_bytes,
                             uint64_t arena_cap, XoChild *kids, uint64_t *cstart, uint64_t *csize,
                             uint32_t *tile_base, uint32_t *tile_child, uint32_t *n_tiles, uint64_t *part_len,
                             uint32_t *part_tiles, uint32_t *err, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const uint32_t parts = xo_layout_parts(n);
    cudaError_t e = launch_pdl(xo_size_kernel, dim3(parts), dim3(kLayoutT), 0, s, q, ends, n, tile_bytes, csize,
                               part_len, part_tiles);
    if (e != cudaSuccess) return e;
    e = launch_pdl(xo_part_scan_kernel, dim3(1), dim3(1024), 0, s, part_len, part_tiles, parts, tile_base, n, n_tiles);
    if (e != cudaSuccess) return e;
    return launch_pdl(xo_place_kernel, dim3(parts), dim3(kLayoutT), 0, s, q, ends, n, tile_bytes, arena_cap, part_len,
                      part_tiles, kids, cstart, csize, tile_base, tile_child, err);
}

// Copy tiles numbered on the device, each tile's child read from the map the
// layout wrote: a CTA takes tiles t = blockIdx.x, +gridDim.x, ...
// A CTA per tile (large children), or a warp per tile (small children:
// a CTA per tile would leave most of its threads idle).
template <bool WARP>
__global__ void xo_copy_map_kernel(const uint8_t *__restrict__ src, uint8_t *__restrict__ dst,
                                   const XoChild *__restrict__ children, const uint32_t *__restrict__ tile_base,
                                   const uint32_t *__restrict__ tile_child, const uint32_t *n_tiles_dev,
                                   uint32_t tile_bytes)
{
    pdl_wait();
    const uint32_t n_tiles = *n_tiles_dev;
    const uint32_t first = WARP ? (threadIdx.x & 31) : threadIdx.x, stride = WARP ? 32 : blockDim.x;
    const uint32_t unit = WARP ? (blockIdx.x * blockDim.x + threadIdx.x) >> 5 : blockIdx.x;
    const uint32_t units = WARP ? (gridDim.x * blockDim.x) >> 5 : gridDim.x;
    for (uint32_t t = unit; t < n_tiles; t += units) {
        const uint32_t k = tile_child[t];
        copy_tile(src, dst, children[k], (uint64_t)(t - tile_base[k]) * tile_bytes, tile_bytes, first, stride);
    }
}

cudaError_t launch_xo_copy_map(const uint8_t *src, uint8_t *dst, const XoChild *children, const uint32_t *tile_base,
                               const uint32_t *tile_child, const uint32_t *n_tiles_dev, uint32_t max_tiles,
                               uint32_t tile_bytes, bool warp_tiles, cudaStream_t s)
{
    if (max_tiles == 0) return cudaSuccess;
    if (warp_tiles)
        return launch_pdl(xo_copy_map_kernel<true>, dim3((uint32_t)umin64((max_tiles + 7) / 8, 2048)), dim3(256), 0,
                          s, src, dst, children, tile_base, tile_child, n_tiles_dev, tile_bytes);
    return launch_pdl(xo_copy_map_kernel<false>, dim3((uint32_t)umin64(max_tiles, 8192)), dim3(256), 0, s, src, dst,
                      children, tile_base, tile_child, n_tiles_dev, tile_bytes);
}

cudaError_t launch_xo_copy_dev(const uint8_t *src, uint8_t *dst, const XoChild *children,
                               const uint32_t *tile_base, uint32_t n_children,
                               const uint32_t *n_tiles_dev, uint32_t tile_bytes, int sms,
                               cudaStream_t s)
{
    if (n_children == 0) return cudaSuccess;
    xo_copy_dev_kernel<<<sms * 8, 256, 0, s>>>(src, dst, children, tile_base, n_children, n_tiles_dev,
                                                tile_bytes);
    return cudaGetLastError();
}

}  // namespace gpk
