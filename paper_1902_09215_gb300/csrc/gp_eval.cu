// Fitness evaluation kernels for linear prefix GP trees (sm_103a).
//
// The paper (Sec. 2.2) evaluates a tree in a single pass over its prefix
// byte buffer, every opcode acting on all 48 fitness cases at once through
// an external stack of 48-float frames; the reduction to fitness is a plain
// loop in case order.  Here:
//   - one warp interprets one item; lane l holds fitness cases 2l and 2l+1 as
//     a float2, so each '+', '-', '*' is one packed f32x2 instruction for
//     all cases, and every opcode decision is warp-uniform;
//   - the tree is read right to left (reversed prefix order is a postfix
//     program): a leaf pushes, an operator pops its second argument and
//     combines it with the top of stack, which holds its first argument.
//     Every node is still one IEEE operation on its children's values, so
//     the per-case results are bit-identical to the recursive EVAL;
//   - the top of stack lives in registers, the next entries in a per-warp
//     shared-memory window, and deeper entries spill to global memory;
//   - a tree longer than one chunk is cut into chunks evaluated
//     independently: each chunk evaluates its complete subtrees and emits an
//     "upper tree" fragment in which those subtrees are value-buffer leaves
//     and the operators whose arguments reach past the chunk stay operators.
//     The upper tree is evaluated by the next launch (recursively if large).
#include <cstdint>
#include <map>
#include <mutex>
#include <utility>

#include <cuda_runtime.h>

#include "gp_internal.cuh"

namespace gpk {

// ---------------------------------------------------------------- arithmetic

__device__ __forceinline__ unsigned long long f2u(float2 a) {
    return *reinterpret_cast<unsigned long long *>(&a);
}
__device__ __forceinline__ float2 u2f(unsigned long long u) {
    return *reinterpret_cast<float2 *>(&u);
}
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(r);
}
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(r);
}
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(r);
}
// Protected division (Table gp.details): a / b, or the problem's value
// (1.0f in the paper) when b == 0.  IEEE round-to-nearest division.
__device__ __forceinline__ float pdiv(float a, float b, float d0) {
    return (b != 0.0f) ? __fdiv_rn(a, b) : d0;
}
__device__ __forceinline__ float2 apply_op(uint32_t c, float2 a, float2 b, float d0) {
    if (c == 0) return f2_add(a, b);
    if (c == 1) return f2_sub(a, b);
    if (c == 2) return f2_mul(a, b);
    return make_float2(pdiv(a.x, b.x, d0), pdiv(a.y, b.y, d0));
}

// ---------------------------------------------------------------- code groups

// 16 consecutive codes, 16-code aligned, loaded with 128-bit loads.  Every
// lane loads the same address, so one request serves the warp.  The group is
// walked as four sub-words of four codes each (sub(q), code(sub, k)), so the
// interpreter body is unrolled only four times: the loop stays small enough
// for the instruction cache despite data-dependent branching.
template <typename Code> struct Group;

template <> struct Group<uint8_t> {
    typedef uint32_t Sub;
    uint4 w;
    __device__ __forceinline__ void load(const uint8_t *p) {
        w = __ldg(reinterpret_cast<const uint4 *>(p));
    }
    __device__ __forceinline__ Sub sub(int q) const {
        return q == 3 ? w.w : q == 2 ? w.z : q == 1 ? w.y : w.x;
    }
    __device__ __forceinline__ static uint32_t code(Sub v, int k) { return (v >> (8 * k)) & 0xFFu; }
    // All lanes hold the same word; an OR-reduction over the warp returns it
    // as a value the compiler knows to be uniform.
    __device__ __forceinline__ static Sub uniform(Sub v, uint32_t mask) { return __reduce_or_sync(mask, v); }
    __device__ __forceinline__ uint32_t first() const { return w.x & 0xFFu; }
};

template <> struct Group<uint32_t> {
    typedef uint4 Sub;
    uint4 w[4];
    __device__ __forceinline__ void load(const uint32_t *p) {
        const uint4 *q = reinterpret_cast<const uint4 *>(p);
        w[0] = __ldg(q); w[1] = __ldg(q + 1); w[2] = __ldg(q + 2); w[3] = __ldg(q + 3);
    }
    __device__ __forceinline__ Sub sub(int q) const {
        return q == 3 ? w[3] : q == 2 ? w[2] : q == 1 ? w[1] : w[0];
    }
    __device__ __forceinline__ static uint32_t code(Sub v, int k) {
        return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
    }
    __device__ __forceinline__ static Sub uniform(Sub v, uint32_t mask) {
        return make_uint4(__reduce_or_sync(mask, v.x), __reduce_or_sync(mask, v.y),
                          __reduce_or_sync(mask, v.z), __reduce_or_sync(mask, v.w));
    }
    __device__ __forceinline__ uint32_t first() const { return w[0].x; }
};

// Upper-tree variant of the group interpreter: one 32-bit code per operand
// (%3 + position), leaves >= 256 (kPtCode0) read the staged value entry of
// their position in the group (%24 + position * S), other leaves the leaf
// table.
static_assert(kPtCode0 == 256, "the PTX of GP_UNODE compares codes with 256");
#define GP_UNODE(CREG, J, IDX)                                                   \
    "setp.gt.u32 pl, " CREG ", 3;\n\t"                                         \
    "@pl bra.uni LF" #IDX ";\n\t"                                              \
    "sub.u32 %1, %1, %23;\n\t"                                                 \
    "ld.shared.b64 v, [%1];\n\t"                                               \
    "setp.lt.u32 p, " CREG ", 2;\n\t"                                          \
    "@p bra.uni LO" #IDX ";\n\t"                                               \
    "setp.eq.u32 p, " CREG ", 2;\n\t"                                          \
    "@p bra.uni MU" #IDX ";\n\t"                                               \
    "mov.u32 ret, " #IDX ";\n\t"                                               \
    "bra.uni DIVR;\n"                                                          \
    "MU" #IDX ":\n\tmul.rn.f32x2 %0, %0, v;\n\tbra.uni E" #IDX ";\n"              \
    "LO" #IDX ":\n\tsetp.eq.u32 p, " CREG ", 0;\n\t@p bra.uni AD" #IDX ";\n\t"   \
    "sub.rn.f32x2 %0, %0, v;\n\tbra.uni E" #IDX ";\n"                          \
    "AD" #IDX ":\n\tadd.rn.f32x2 %0, %0, v;\n\tbra.uni E" #IDX ";\n"              \
    "LF" #IDX ":\n\tst.shared.b64 [%1], %0;\n\tadd.u32 %1, %1, %23;\n\t"          \
    "setp.lt.u32 p, " CREG ", 256;\n\t@p bra.uni TB" #IDX ";\n\t"              \
    "ld.shared.b64 %0, [%24+" #J "*%23];\n\tbra.uni E" #IDX ";\n"                \
    "TB" #IDX ":\n\tmad.lo.u32 a, " CREG ", %23, %19;\n\tld.shared.b64 %0, [a];\n" \
    "E" #IDX ":\n\t"

#define GP_UWORD(Q, C3, C2, C1, C0, J3, J2, J1, J0, I0, I1, I2, I3)              \
    "W" #Q ":\n\tsub.u32 dd, %1, %21;\n\tsetp.gt.u32 p, dd, %22;\n\t"               \
    "@p bra.uni X" #Q ";\n\t"                                                     \
    GP_UNODE(C3, J3, I0) GP_UNODE(C2, J2, I1) GP_UNODE(C1, J1, I2) GP_UNODE(C0, J0, I3)

template <uint32_t S>
__device__ __forceinline__ int group_u32(uint64_t &tos, uint32_t &t, int q, const uint4 *w, uint32_t tb,
                                         float d0, uint32_t lo, uint32_t span, uint32_t stage)
{
    asm volatile(
        "{\n\t.reg .pred p, pl;\n\t.reg .b32 a, ret, dd;\n\t.reg .b64 v;\n\t"
        ".reg .f32 tx, ty, bx, by, qx, qy;\n\t"
        "ENT: .branchtargets W0, W1, W2, W3;\n\t"
        "brx.idx.uni %2, ENT;\n"
        GP_UWORD(3, "%18", "%17", "%16", "%15", 15, 14, 13, 12, 0, 1, 2, 3)
        GP_UWORD(2, "%14", "%13", "%12", "%11", 11, 10, 9, 8, 4, 5, 6, 7)
        GP_UWORD(1, "%10", "%9", "%8", "%7", 7, 6, 5, 4, 8, 9, 10, 11)
        GP_UWORD(0, "%6", "%5", "%4", "%3", 3, 2, 1, 0, 12, 13, 14, 15)
        "mov.s32 %2, -1;\n\tbra.uni DONE;\n"
        "X3:\n\tmov.s32 %2, 3;\n\tbra.uni DONE;\n"
        "X2:\n\tmov.s32 %2, 2;\n\tbra.uni DONE;\n"
        "X1:\n\tmov.s32 %2, 1;\n\tbra.uni DONE;\n"
        "X0:\n\tmov.s32 %2, 0;\n\tbra.uni DONE;\n"
        "DIVR:\n\tmov.b64 {tx, ty}, %0;\n\tmov.b64 {bx, by}, v;\n\t"
        "div.rn.f32 qx, tx, bx;\n\tsetp.neu.f32 p, bx, 0f00000000;\n\tselp.f32 tx, qx, %20, p;\n\t"
        "div.rn.f32 qy, ty, by;\n\tsetp.neu.f32 p, by, 0f00000000;\n\tselp.f32 ty, qy, %20, p;\n\t"
        "mov.b64 %0, {tx, ty};\n\t"
        "RET: .branchtargets E0, E1, E2, E3, E4, E5, E6, E7, E8, E9, E10, E11, E12, E13, E14, E15;\n\t"
        "brx.idx.uni ret, RET;\n"
        "DONE:\n\t}"
        : "+l"(tos), "+r"(t), "+r"(q)
        : "r"(w[0].x), "r"(w[0].y), "r"(w[0].z), "r"(w[0].w), "r"(w[1].x), "r"(w[1].y), "r"(w[1].z),
          "r"(w[1].w), "r"(w[2].x), "r"(w[2].y), "r"(w[2].z), "r"(w[2].w), "r"(w[3].x), "r"(w[3].y),
          "r"(w[3].z), "r"(w[3].w), "r"(tb), "f"(d0), "r"(lo), "r"(span), "n"(S), "r"(stage));
    return q;
}

// ---------------------------------------------------------------- one item

// Dynamic shared memory: the leaf table at offset 0, then one stack window
// per warp, then per-warp scratch for the fitness fold.  Stack and table
// accesses use 32-bit byte offsets into this array.
extern __shared__ __align__(16) unsigned char smem[];

__device__ __forceinline__ float2 &sm2(uint32_t off) {
    return *reinterpret_cast<float2 *>(smem + off);
}

// Stack entries are handled as packed float2 in a 64-bit register and moved
// with volatile shared-memory accesses at absolute 32-bit shared addresses,
// so they stay ordered with respect to the inline-PTX interpreter below.
__device__ __forceinline__ uint64_t pk(float2 v) { return f2u(v); }
__device__ __forceinline__ float2 upk(uint64_t v) { return u2f(v); }
__device__ __forceinline__ void sts64(uint32_t a, uint64_t v) {
    asm volatile("st.shared.b64 [%0], %1;" ::"r"(a), "l"(v));
}
__device__ __forceinline__ uint64_t lds64(uint32_t a) {
    uint64_t v;
    asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"(a));
    return v;
}

// Asynchronous 8-byte global -> shared copies (value-buffer staging).
__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;"); }

// The byte-code group loop below keeps the top of stack `tos` in a register
// and the rest of the operand stack in this lane's column of the shared
// window; `t` is the shared address of the next free entry (entries S bytes
// apart) and `wb` the window's bottom.
//   leaf c >= 4 : push tos; tos = table[c] (shared address tb + c*S)
//   op   c < 4  : tos = tos (op) pop -- tos holds the operator's first
//                 argument, the popped entry its second
//   '/' is protected: a zero divisor gives d0.
// One node at group position K (0..15, read from 15 down), its code in byte
// K&3 of word register W (prmt selector SEL).  Operands: %0 tos, %1 t,
// %5 tb, %7 wb, %9 S.  An operator that finds the window empty (its second
// argument lies to the right of what the window holds: spilled entries, or
// a spine operator of a chunk) leaves with %2 = 16 + K before popping.
#define GP_BN(K, W, SEL)                                                         \
    "N" #K ":\n\tprmt.b32 c, " W ", z, " SEL ";\n\t"                           \
    "setp.gt.u32 pl, c, 3;\n\t@pl bra.uni L" #K ";\n\t"                        \
    "setp.eq.u32 p, %1, %7;\n\t@p bra.uni U" #K ";\n\t"                        \
    "sub.u32 %1, %1, %9;\n\tld.shared.b64 v, [%1];\n\t"                        \
    "setp.lt.u32 p, c, 2;\n\t@p bra.uni LO" #K ";\n\t"                         \
    "setp.eq.u32 p, c, 2;\n\t@p bra.uni MU" #K ";\n\t"                         \
    "mov.u32 ret, " #K ";\n\tbra.uni DIVR;\n"                                  \
    "MU" #K ":\n\tmul.rn.f32x2 %0, %0, v;\n\tbra.uni E" #K ";\n"                 \
    "LO" #K ":\n\tsetp.eq.u32 p, c, 0;\n\t@p bra.uni AD" #K ";\n\t"            \
    "sub.rn.f32x2 %0, %0, v;\n\tbra.uni E" #K ";\n"                            \
    "AD" #K ":\n\tadd.rn.f32x2 %0, %0, v;\n\tbra.uni E" #K ";\n"                 \
    "L" #K ":\n\tmad.lo.u32 a, c, %9, %5;\n\t"                                 \
    "st.shared.b64 [%1], %0;\n\tadd.u32 %1, %1, %9;\n\tld.shared.b64 %0, [a];\n" \
    "E" #K ":\n\t"
// Word Q (positions 4Q+3 .. 4Q): it runs only with room for four pushes
// (t - wb <= %8), else the loop leaves with %2 = 4Q+3.
#define GP_BW(Q, W, K3, K2, K1, K0)                                              \
    "W" #Q ":\n\tsub.u32 dd, %1, %7;\n\tsetp.gt.u32 p, dd, %8;\n\t@p bra.uni X" #Q ";\n\t" \
    GP_BN(K3, W, "0x4443") GP_BN(K2, W, "0x4442") GP_BN(K1, W, "0x4441") GP_BN(K0, W, "0x4440")
#define GP_BU(K) "U" #K ":\n\tmov.s32 %2, 16+" #K ";\n\tbra.uni DONE;\n"

// Interprets 16-code groups of byte codes from the group at address %3
// down to the group at %4 (both 16-byte aligned, %3 >= %4), entering the
// first group at position %2 (a word start enters through its room check).
// Groups are loaded with 16-byte loads, the next one a group ahead; codes
// are warp-uniform, so every branch is .uni.  Leaves with %3 = the current
// group and %2 = -1 (every group done), 4Q+3 (word Q needs room: spill) or
// 16 + K (the operator at position K found the window empty).
template <uint32_t S>
__device__ __forceinline__ int groups_u8(uint64_t &tos, uint32_t &t, const uint8_t *&p, int pos,
                                         const uint8_t *plo, uint32_t tb, float d0, uint32_t wb,
                                         uint32_t room)
{
    uint64_t pa = reinterpret_cast<uint64_t>(p);
    asm volatile(
        "{\n\t.reg .pred p, pl;\n\t.reg .b32 c, a, ret, dd, z, w0, w1, w2, w3, n0, n1, n2, n3;\n\t"
        ".reg .b64 v, pn;\n\t.reg .f32 tx, ty, bx, by, qx, qy;\n\t"
        "mov.b32 z, 0;\n\t"
        "ld.global.nc.v4.u32 {w0, w1, w2, w3}, [%3];\n\t"
        "setp.gt.u64 p, %3, %4;\n\tsub.u64 pn, %3, 16;\n\t"
        "@p ld.global.nc.v4.u32 {n0, n1, n2, n3}, [pn];\n\t"
        "ENT: .branchtargets N0, N1, N2, W0, N4, N5, N6, W1, N8, N9, N10, W2, N12, N13, N14, W3;\n\t"
        "brx.idx.uni %2, ENT;\n"
        GP_BW(3, "w3", 15, 14, 13, 12)
        GP_BW(2, "w2", 11, 10, 9, 8)
        GP_BW(1, "w1", 7, 6, 5, 4)
        GP_BW(0, "w0", 3, 2, 1, 0)
        "setp.le.u64 p, %3, %4;\n\t@p bra.uni FIN;\n\t"
        "sub.u64 %3, %3, 16;\n\t"
        "mov.b32 w0, n0;\n\tmov.b32 w1, n1;\n\tmov.b32 w2, n2;\n\tmov.b32 w3, n3;\n\t"
        "setp.gt.u64 p, %3, %4;\n\tsub.u64 pn, %3, 16;\n\t"
        "@p ld.global.nc.v4.u32 {n0, n1, n2, n3}, [pn];\n\t"
        "bra.uni W3;\n"
        "FIN:\n\tmov.s32 %2, -1;\n\tbra.uni DONE;\n"
        "X3:\n\tmov.s32 %2, 15;\n\tbra.uni DONE;\n"
        "X2:\n\tmov.s32 %2, 11;\n\tbra.uni DONE;\n"
        "X1:\n\tmov.s32 %2, 7;\n\tbra.uni DONE;\n"
        "X0:\n\tmov.s32 %2, 3;\n\tbra.uni DONE;\n"
        GP_BU(0) GP_BU(1) GP_BU(2) GP_BU(3) GP_BU(4) GP_BU(5) GP_BU(6) GP_BU(7)
        GP_BU(8) GP_BU(9) GP_BU(10) GP_BU(11) GP_BU(12) GP_BU(13) GP_BU(14) GP_BU(15)
        "DIVR:\n\tmov.b64 {tx, ty}, %0;\n\tmov.b64 {bx, by}, v;\n\t"
        "div.rn.f32 qx, tx, bx;\n\tsetp.neu.f32 p, bx, 0f00000000;\n\tselp.f32 tx, qx, %6, p;\n\t"
        "div.rn.f32 qy, ty, by;\n\tsetp.neu.f32 p, by, 0f00000000;\n\tselp.f32 ty, qy, %6, p;\n\t"
        "mov.b64 %0, {tx, ty};\n\t"
        "RET: .branchtargets E0, E1, E2, E3, E4, E5, E6, E7, E8, E9, E10, E11, E12, E13, E14, E15;\n\t"
        "brx.idx.uni ret, RET;\n"
        "DONE:\n\t}"
        : "+l"(tos), "+r"(t), "+r"(pos), "+l"(pa)
        : "l"(reinterpret_cast<uint64_t>(plo)), "r"(tb), "f"(d0), "r"(wb), "r"(room),
          "n"(S)
        : "memory");
    p = reinterpret_cast<const uint8_t *>(pa);
    return pos;
}

template <int LANES, typename Code, bool WIDE>
__device__ __forceinline__ void eval_item(const EvalParams &P, const EvalItem *itp, uint32_t win_sa,
                                          uint32_t tbl_sa, uint32_t stage_sa, float *errs,
                                          float2 *__restrict__ spill, uint64_t spill_cap, int lane,
                                          uint32_t mask, float y0, float y1)
{
    constexpr uint32_t S = LANES * sizeof(float2);          // bytes per stack entry / table row
    const Code *codes0 = static_cast<const Code *>(P.codes);
    const int K = (int)P.window;
    const float d0 = P.div0;
    // Item fields other than its range are re-read when needed (cold paths)
    // rather than kept live across the interpreter loop; `itp` points to
    // this warp's shared-memory copy of the item.
#define IT(f) (itp->f)
    const uint32_t flags = IT(flags);
    const bool is_final = (flags & kItemFinal) != 0;
    const bool fused = (flags & kItemFused) != 0;      // chunk of a medium tree
    const bool rope = WIDE && (flags & kItemRope) != 0; // final over a medium tree's slots
    const uint32_t tb = tbl_sa + lane * 8u - 4u * S;        // + code * S = leaf table row
    const uint32_t wb = win_sa + lane * 8u;                 // this lane's column of the window

    uint64_t tos = 0;                     // top of stack (first argument of the next operator)
    bool have = false;                    // tos holds a value of this item
    uint32_t t = wb;                      // next free window entry (shared address)
    uint32_t g = 0;                       // entries spilled below the window
    // Fragment output: planned items write at planned offsets; fused chunks
    // right-align their codes in their own slot and number their value
    // entries from the slot's first entry.  Counters of what was emitted:
    uint32_t n_emit = 0, n_pt = 0, n_op_emit = 0;
    bool pt_full = false;                 // a fused chunk ran out of value slots
    uint32_t prev = 0xFFFFFFFFu;          // code at the position right of the current one
    uint32_t fault = 0;                   // kErr* bits; any fault ends the item
    const uint32_t dmax = (uint32_t)(K - 4) * S;   // room for four pushes below this

    // Upper trees: value-buffer leaves of the current group were copied to
    // staging buffer `buf`, slot = position in the group (jcur).
    uint32_t buf = 0, jcur = 0;
    auto leafval = [&](uint32_t c) -> uint64_t {
        if (WIDE && c >= kPtCode0) return lds64(stage_sa + (buf * 16 + jcur) * S);
        return lds64(tb + c * S);
    };
    if (rope && P.fz_over[IT(tree)]) {
        // A chunk of this tree ran out of value slots: queue the tree for a
        // re-evaluation through planned upper-tree levels.
        if (lane == 0) P.fz_redo[1 + atomicAdd(P.fz_redo, 1u)] = IT(tree);
        return;
    }
    const float2 *pt_src = P.pt_in;       // value entries read by the current range
    uint64_t rb = IT(begin), re = IT(end);  // the current range
    auto stage = [&](const Group<Code> &grp, int64_t gbase, uint32_t into) {
        const uint32_t sbase = stage_sa + into * 16 * S;
        const float2 *src = pt_src + lane;
        if ((uint64_t)gbase >= rb && (uint64_t)gbase + 16 <= re) {   // a whole group of the range
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const typename Group<Code>::Sub v = grp.sub(q);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t c = Group<Code>::code(v, k);
                    if (c >= kPtCode0) cp_async8(sbase + (4 * q + k) * S, src + (uint64_t)(c - kPtCode0) * LANES);
                }
            }
            return;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const typename Group<Code>::Sub v = grp.sub(q);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t c = Group<Code>::code(v, k);
                const uint64_t pos = (uint64_t)gbase + 4 * q + k;
                if (pos >= rb && pos < re && c >= kPtCode0)
                    cp_async8(sbase + (4 * q + k) * S, src + (uint64_t)(c - kPtCode0) * LANES);
            }
        }
    };
    // Fragment output stays inside the slot reserved for it.
    auto emit = [&](uint32_t code) {
        const uint64_t cap = fused ? P.fz_cap_codes : IT(frag_len);
        if (n_emit >= cap) { fault |= kErrPlan; return; }
        const uint64_t end = fused ? (IT(frag_off) + 1) * P.fz_cap_codes : IT(frag_off) + IT(frag_len);
        ++n_emit;
        if (lane == 0) (fused ? P.fz_codes : P.u_out)[end - n_emit] = code;
    };
    auto new_pt = [&](uint64_t v) -> uint32_t {
        const uint32_t cap = fused ? P.fz_cap_pt : IT(pt_cnt);
        if (n_pt >= cap) {
            if (fused) pt_full = true;    // the tree is re-evaluated without chunk slots
            else fault |= kErrPlan;
            return kPtCode0;
        }
        const uint64_t idx = (fused ? IT(frag_off) * P.fz_cap_pt : IT(pt_base)) + n_pt;
        (fused ? P.fz_pt : P.pt_out)[idx * LANES + lane] = upk(v);
        // planned fragments number entries globally, fused chunks per slot
        return (uint32_t)(kPtCode0 + (fused ? n_pt++ : (n_pt++, idx)));
    };
    // Keep room for four pushes in the window, and four pops whenever
    // entries are spilled; the window is refilled / spilled half-way.
    auto rebalance = [&]() {
        const uint32_t d = t - wb;
        if (d > dmax) {
            const int sp = (int)(d / S);
            const int h = sp - K / 2;
            if ((uint64_t)g + h > spill_cap) {
                fault |= kErrSpill;
                return;
            }
            for (int i = 0; i < h; ++i) spill[(g + i) * LANES + lane] = upk(lds64(wb + i * S));
            for (int i = h; i < sp; ++i) sts64(wb + (i - h) * S, lds64(wb + i * S));
            g += h;
            t -= h * S;
        } else if (d < 4 * S && g > 0) {
            const int sp = (int)(d / S);
            const int h = min((int)g, K / 2 - sp);
            for (int i = sp - 1; i >= 0; --i) sts64(wb + (i + h) * S, lds64(wb + i * S));
            for (int i = 0; i < h; ++i) sts64(wb + i * S, pk(spill[(g - h + i) * LANES + lane]));
            g -= h;
            t += h * S;
        }
    };
    // Checked step (nothing spilled, fewer than five values known): detects
    // operators whose arguments lie beyond the item.
    auto step_checked = [&](uint32_t c) {
        if (c >= 4) {
            const uint64_t v = leafval(c);
            if (have) {
                sts64(t, tos);
                t += S;
            }
            tos = v;
            have = true;
        } else if (t != wb) {             // a window entry implies have
            t -= S;
            tos = pk(apply_op(c, upk(tos), upk(lds64(t)), d0));
        } else if (is_final) {
            fault |= kErrMalformed;       // stack underflow: not a valid tree
        } else {
            // Spine operator: its second argument (and maybe its first) lies
            // to the right of this chunk.  Emit it into the upper tree; a
            // first argument that is an x/constant leaf passes through, any
            // other first argument becomes an entry of this level's value
            // buffer (entries of the previous level's buffer are not visible
            // to the next level, so they are copied too).
            if (have) emit((prev >= 4 && prev < kPtCode0) ? prev : new_pt(tos));
            emit(c);
            ++n_op_emit;
            have = false;
        }
        prev = c;
    };

    const uint32_t fast_span = (uint32_t)(K - 8) * S;   // fast iff 4S <= depth <= (K-4)S
    const uint32_t fast_lo = wb + 4 * S;
    // A rope item walks its tree's chunk fragments from the last to the
    // first, each right to left, on one continuous stack.
    const uint32_t nranges = rope ? IT(frag_len) : 1;
    for (uint32_t r = 0; r < nranges && !fault; ++r) {
    const Code *codes = codes0;
    if (rope) {
        const uint64_t slot = IT(pt_base) + (nranges - 1 - r);
        codes = reinterpret_cast<const Code *>(P.fz_codes + slot * P.fz_cap_codes);
        re = P.fz_cap_codes;
        rb = re - P.fz_len[slot];
        pt_src = P.fz_pt + slot * P.fz_cap_pt * LANES;
    }
    const uint64_t b = rb, e = re;
    if (e <= b) continue;
    if constexpr (!WIDE) {
        // Byte codes: the group loop runs whole 16-byte groups, from the
        // item's last group down to its first whole one, and leaves only
        // where the stack needs the C++ side: before a word without room
        // for four pushes (spill), at an operator that finds the window
        // empty (refill, or a spine operator of a chunk), and after the
        // last group.  A stack without a value (the item's start, after a
        // spine operator) takes checked steps up to its first leaf.
        const uint8_t *cb = reinterpret_cast<const uint8_t *>(codes);
        const int64_t glo = (int64_t)(b & ~15ull);
        const int64_t gfast = (b & 15) ? glo + 16 : glo;   // lowest group the loop runs
        int64_t gs = (int64_t)((e - 1) & ~15ull);
        int pos = (int)((int64_t)(e - 1) - gs);
        auto code_at = [&](int64_t i) -> uint32_t { return __ldg(cb + i); };
        const uint32_t room = (uint32_t)(K - 4) * S;
        while (!fault && gs >= gfast) {
            if (!have) {
                step_checked(code_at(gs + pos));
                if (--pos < 0) { pos = 15; gs -= 16; }
                continue;
            }
            if (t - wb > room) {
                rebalance();
                if (fault) break;
            }
            const uint8_t *pg = cb + gs;
            const int r = groups_u8<S>(tos, t, pg, pos, cb + gfast, tb, d0, wb, room);
            gs = (int64_t)(pg - cb);
            if (r < 0) {                      // every group down to gfast done
                gs -= 16;
                pos = 15;
                break;
            }
            if (r < 16) {                     // word at r needs room: spill half the window
                pos = r;
                rebalance();
                continue;
            }
            pos = r - 16;                     // operator at pos with an empty window
            if (g > 0) {                      // its argument was spilled: refill
                rebalance();
                continue;
            }
            prev = (gs + pos + 1 < (int64_t)e) ? code_at(gs + pos + 1) : 0xFFFFFFFFu;
            step_checked(code_at(gs + pos));  // spine operator (or a malformed tree)
            if (--pos < 0) { pos = 15; gs -= 16; }
        }
        // codes of an item that starts inside a group
        for (int64_t i = gs + pos; !fault && i >= (int64_t)b; --i) {
            rebalance();
            if (fault) break;
            step_checked(code_at(i));
        }
    } else {
        // Upper-tree codes: the value entries a group names are copied
        // (cp.async) into a staging buffer one group ahead of the
        // interpreter, the codes themselves are loaded two groups ahead.
        int64_t gs = (int64_t)((e - 1) & ~15ull);
        const int64_t glo = (int64_t)(b & ~15ull);
        Group<Code> cur, nxt;
        cur.load(codes + gs);
        if (gs - 16 >= glo) nxt.load(codes + gs - 16);
        buf = 0;                              // each range starts its own pipeline
        stage(cur, gs, 0);
        cp_async_commit();
        for (; gs >= glo; gs -= 16) {
            Group<Code> nxt2;
            if (gs - 32 >= glo) nxt2.load(codes + gs - 32);
            // Copies for the next group overlap this group's work.
            if (gs - 16 >= glo) stage(nxt, gs - 16, buf ^ 1);
            cp_async_commit();
            cp_async_wait1();
            const bool full = (uint64_t)gs >= b && (uint64_t)gs + 16 <= e;
            if (full) {
                int q = 3;
                for (;;) {
                    q = group_u32<S>(tos, t, q, cur.w, tb, d0, fast_lo, fast_span, stage_sa + buf * 16 * S);
                    if (q < 0) break;
                    rebalance();
                    if (fault) break;
                    if ((t - fast_lo) <= fast_span) continue;     // runnable after all
                    if (q < 3) prev = Group<Code>::code(cur.sub(q + 1), 0);
                    const typename Group<Code>::Sub v = cur.sub(q);
#pragma unroll
                    for (int k = 3; k >= 0; --k) {
                        jcur = 4 * q + k;
                        step_checked(Group<Code>::code(v, k));
                    }
                    if (fault || --q < 0) break;
                }
                prev = cur.first();
            } else {
#pragma unroll 1
                for (int q = 3; q >= 0 && !fault; --q) {
                    const typename Group<Code>::Sub v = Group<Code>::uniform(cur.sub(q), mask);
                    rebalance();
                    if (fault) break;
#pragma unroll
                    for (int k = 3; k >= 0; --k) {
                        const uint64_t pos = (uint64_t)gs + 4 * q + k;
                        jcur = 4 * q + k;
                        if (pos >= b && pos < e) step_checked(Group<Code>::code(v, k));
                    }
                }
            }
            if (fault) break;
            cur = nxt;
            nxt = nxt2;
            buf ^= 1;
        }
        cp_async_wait0();                     // staging is idle before the next item
    }
    }
    if (!rope && IT(end) <= IT(begin) && is_final) {
        fault |= kErrMalformed;
    }
    const int sp = (int)((t - wb) / S);

    if (is_final) {
        const uint32_t tr = IT(tree);
        const uint32_t nc = P.n_cases;
        const bool ok = !fault && have && sp == 0 && g == 0;
        if (rope && fault) {              // e.g. deeper than the spill area: redo as planned
            if (lane == 0) P.fz_redo[1 + atomicAdd(P.fz_redo, 1u)] = tr;
            return;
        }
        if (!ok) {
            if (lane == 0) {
                atomicOr(P.err, fault ? fault : kErrMalformed);
                P.fitness[tr] = __int_as_float(0x7fffffff);
                P.hits[tr] = 0;
            }
            return;
        }
        const float2 o = upk(tos);
        const uint32_t i0 = 2 * lane, i1 = i0 + 1;
        if (i0 < nc) P.values[(uint64_t)tr * nc + i0] = o.x;
        if (i1 < nc) P.values[(uint64_t)tr * nc + i1] = o.y;
        const float e0 = fabsf(o.x - y0), e1 = fabsf(o.y - y1);
        errs[i0] = e0;
        errs[i1] = e1;
        const unsigned h0 = __ballot_sync(mask, i0 < nc && e0 < 0.01f);
        const unsigned h1 = __ballot_sync(mask, i1 < nc && e1 < 0.01f);
        __syncwarp(mask);
        if (lane == 0) {
            // Sec. 2.2 / 3.2: fixed-order reduction, a plain loop over cases.
            float acc = 0.0f;
            for (uint32_t i = 0; i < nc; ++i) acc = acc + errs[i];
            P.fitness[tr] = __fdiv_rn(acc, (float)nc);
            P.hits[tr] = __popc(h0) + __popc(h1);
        }
        __syncwarp(mask);
        return;
    }

    if (fault) {
        if (lane == 0) atomicOr(P.err, fault);
        return;
    }
    // Values left on the stack are the complete subtrees at the chunk's left
    // end; the bottom one is the rightmost, so it is emitted first.
    for (uint64_t i = 0; i < g; ++i) emit(new_pt(pk(spill[i * LANES + lane])));
    for (int i = 0; i < sp; ++i) emit(new_pt(lds64(wb + i * S)));
    if (have) emit(new_pt(tos));
    if (P.stat_up && lane == 0) {
        atomicAdd(P.stat_up, n_emit);
        atomicAdd(P.stat_up + 1, n_op_emit);
        atomicAdd(P.stat_up + 2, n_pt);
    }
    if (fused) {
        if (lane == 0) {
            P.fz_len[IT(frag_off)] = n_emit;
            if (pt_full) P.fz_over[IT(tree)] = 1u;
        }
        if (fault && lane == 0) atomicOr(P.err, kErrPlan);
        return;
    }
    if (fault || n_emit != IT(frag_len) || n_pt != IT(pt_cnt)) {
        if (lane == 0) atomicOr(P.err, kErrPlan);
    }
#undef IT
}

// ---------------------------------------------------------------- kernel

template <int LANES, typename Code, bool WIDE>
__global__ void __launch_bounds__(WIDE ? 512 : 1024, 1) eval_kernel(EvalParams P)
{
    pdl_wait();
    const int nwarps = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr uint32_t S = LANES * sizeof(float2);
    const uint32_t rows = P.leaf_rows ? P.leaf_rows : kLeafRows;
    const uint32_t win0 = rows * S;                         // first window (bytes)
    // Upper-tree kernels: two 16-entry staging buffers per warp after the windows.
    const uint32_t stage0 = win0 + (uint32_t)nwarps * P.window * S;
    // Then one item copy (64 bytes) per warp.
    const uint32_t item0 = stage0 + (WIDE ? (uint32_t)nwarps * 32 * S : 0u);

    // (a launch whose device-side item count is zero does no setup at all)
    if (P.n_items_dev && *P.n_items_dev == 0) return;
    // Leaf table: row 0 is x (per lane, two cases), row r >= 1 constant r-1.
    for (int i = threadIdx.x; i < (int)(rows * LANES); i += blockDim.x) {
        const int row = i / LANES, l = i - row * LANES;
        float2 v;
        if (row == 0) v = make_float2(P.x[2 * l], P.x[2 * l + 1]);
        else if ((uint32_t)(row - 1) < P.n_consts) v = make_float2(P.consts[row - 1], P.consts[row - 1]);
        else v = make_float2(0.f, 0.f);
        sm2(row * S + l * 8) = v;
    }
    __syncthreads();
    if (lane >= LANES) return;

    const uint32_t mask = (LANES == 32) ? 0xffffffffu : ((1u << LANES) - 1u);
    const uint32_t win_off = win0 + (uint32_t)warp * P.window * S;
    // The fitness fold's scratch reuses the window, which is empty by then.
    float *errs = reinterpret_cast<float *>(smem + win_off);
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    const float y0 = P.y[2 * lane], y1 = P.y[2 * lane + 1];
    const uint64_t gw = (uint64_t)blockIdx.x * nwarps + warp;
    float2 *myspill = P.spill + gw * P.spill_per_warp * LANES;
    const uint32_t n_items = P.n_items_dev ? *P.n_items_dev : P.n_items;

    for (;;) {
        uint32_t idx = 0;
        if (lane == 0) idx = atomicAdd(P.counter, 1u);
        idx = __shfl_sync(mask, idx, 0);
        if (idx >= n_items) break;
        EvalItem *itp = reinterpret_cast<EvalItem *>(smem + item0 + warp * sizeof(EvalItem));
        __syncwarp(mask);                 // the previous item's readers are done
        for (int w = lane; w < (int)(sizeof(EvalItem) / 4); w += LANES)   // any lane count
            reinterpret_cast<uint32_t *>(itp)[w] =
                __ldg(reinterpret_cast<const uint32_t *>(P.items + idx) + w);
        __syncwarp(mask);
        float2 *area = myspill;
        uint64_t cap = P.spill_per_warp;
        const uint64_t soff = itp->spill_off;
        if (soff != kNoSpill) {
            area = P.spill + soff * LANES;
            cap = itp->spill_cap;
        }
        eval_item<LANES, Code, WIDE>(P, itp, sbase + win_off, sbase,
                                     sbase + stage0 + (uint32_t)warp * 32 * S + lane * 8u, errs, area,
                                     cap, lane, mask, y0, y1);
    }
}

size_t eval_smem_bytes(int lanes, int warps, int window, bool wide, int leaf_rows)
{
    return (size_t)leaf_rows * lanes * sizeof(float2) +
           (size_t)warps * (window + (wide ? 32 : 0)) * lanes * sizeof(float2) +
           (size_t)warps * sizeof(EvalItem);
}

template <int LANES>
static void *eval_fn(bool wide)
{
    return wide ? (void *)eval_kernel<LANES, uint32_t, true>
                : (void *)eval_kernel<LANES, uint8_t, false>;
}

static void *eval_fn_for(int lanes, bool wide)
{
    switch (lanes) {
    case 8: return eval_fn<8>(wide);
    case 16: return eval_fn<16>(wide);
    case 24: return eval_fn<24>(wide);
    case 32: return eval_fn<32>(wide);
    default: return nullptr;
    }
}

// Raise (never lower) the kernel's dynamic shared-memory limit on the
// current device to `smem`.  Every launcher goes through here, so a limit
// only grows: a launch prepared on one host thread stays valid while another
// thread prepares a smaller one.  One lock covers the check and the set; the
// record of what was raised is kept per device, like the attribute itself.
cudaError_t eval_prepare_at_least(int lanes, bool wide, size_t smem)
{
    void *fn = eval_fn_for(lanes, wide);
    if (!fn) return cudaErrorInvalidValue;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static std::mutex mu;
    static std::map<std::pair<int, int>, size_t> raised;   // (device, kernel) -> limit
    std::lock_guard<std::mutex> lk(mu);
    size_t &cur = raised[std::make_pair(dev, lanes * 2 + (wide ? 1 : 0))];
    if (cur >= smem) return cudaSuccess;
    cudaFuncAttributes a;
    e = cudaFuncGetAttributes(&a, fn);
    if (e != cudaSuccess) return e;
    if ((size_t)a.maxDynamicSharedSizeBytes >= smem) {
        cur = (size_t)a.maxDynamicSharedSizeBytes;
        return cudaSuccess;
    }
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) cur = smem;
    return e;
}

cudaError_t launch_eval(int lanes, bool wide, const EvalParams &p, int ctas, int warps,
                        size_t smem, cudaStream_t s, bool pdl)
{
    void *fn = eval_fn_for(lanes, wide);
    if (!fn) return cudaErrorInvalidValue;
    EvalParams pp = p;
    void *args[] = {&pp};
    if (!pdl) return cudaLaunchKernel(fn, dim3(ctas), dim3(warps * 32), args, smem, s);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(warps * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at{};
    at.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

// ---------------------------------------------------------------- planning

// Stack-size transfer function of a run of codes read right to left:
// k -> max(k + d, c).  A leaf maps k -> k+1; an operator maps k -> k-1 when
// both arguments are on the stack and otherwise (a spine operator) leaves no
// known value, k -> max(k-1, 0).  The family is closed under composition.
struct Xfer {
    int64_t d, c;
};
__device__ __forceinline__ Xfer xfer_after(Xfer first, Xfer then) {
    return Xfer{first.d + then.d, max(first.c + then.d, then.c)};
}
constexpr int64_t kNegInf = -(int64_t(1) << 60);

// Calls f(code) for the codes at positions hi-1 down to lo, reading whole
// aligned 16-byte words (code arrays are 16-byte aligned and readable one
// word past either end of any item).
template <typename Code, typename F>
__device__ __forceinline__ void codes_reverse(const Code *__restrict__ codes, uint64_t lo, uint64_t hi, F &&f)
{
    constexpr uint32_t PER = 16 / sizeof(Code);
    if (hi <= lo) return;
    const uint64_t wlo = lo / PER;
    for (uint64_t w = (hi - 1) / PER + 1; w-- > wlo;) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(codes) + w);
        const uint32_t word[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int j = (int)PER - 1; j >= 0; --j) {
            const uint64_t p = w * PER + (uint64_t)j;
            if (p >= lo && p < hi)
                f(sizeof(Code) == 1 ? (word[j >> 2] >> (8 * (j & 3))) & 0xFFu : word[j & 3]);
        }
    }
}

// One warp per fragment item: counts the codes and value-buffer entries the
// chunk will emit, replaying exactly the evaluator's spine rule.
template <typename Code>
__global__ void plan_kernel(const Code *__restrict__ codes, const EvalItem *__restrict__ items,
                            uint32_t n, const uint32_t *n_dev, PlanOut *__restrict__ out)
{
    pdl_wait();
    const int lane = threadIdx.x & 31;
    if (n_dev) n = min(n, *n_dev);
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n; w += n_warps) {
    const EvalItem it = items[w];
    const uint64_t len = it.end - it.begin;
    const uint64_t seg = (len + 31) / 32;
    const uint64_t lo = umin64(it.begin + lane * seg, it.end);
    const uint64_t hi = umin64(lo + seg, it.end);

    Xfer f{0, kNegInf};
    codes_reverse(codes, lo, hi, [&](uint32_t c) {
        if (c >= 4) f = Xfer{f.d + 1, f.c + 1};
        else f = Xfer{f.d - 1, max(f.c - 1, (int64_t)0)};
    });
    // suffix composition: G_lane = F_lane after F_{lane+1} after ... F_31
    Xfer G = f;
    for (int off = 1; off < 32; off <<= 1) {
        Xfer o;
        o.d = __shfl_down_sync(0xffffffffu, G.d, off);
        o.c = __shfl_down_sync(0xffffffffu, G.c, off);
        if (lane + off < 32) G = xfer_after(o, G);
    }
    Xfer R;
    R.d = __shfl_down_sync(0xffffffffu, G.d, 1);
    R.c = __shfl_down_sync(0xffffffffu, G.c, 1);
    int64_t kn = (lane == 31) ? 0 : max(R.d, R.c);

    uint32_t spine = 0, spine1 = 0, spine1_pt = 0;
    int64_t mx = kn;
    uint32_t prev = (hi < it.end) ? (uint32_t)codes[hi] : 0xFFFFFFFFu;
    codes_reverse(codes, lo, hi, [&](uint32_t c) {
        if (c >= 4) {
            ++kn;
            mx = max(mx, kn);
        } else if (kn >= 2) {
            --kn;
        } else {
            ++spine;
            if (kn == 1) {
                ++spine1;
                if (prev < 4 || prev >= kPtCode0) ++spine1_pt;
            }
            kn = 0;
        }
        prev = c;
    });
    const int64_t kn_final = __shfl_sync(0xffffffffu, kn, 0);
    uint32_t a = spine + spine1, bcount = spine1_pt;
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        bcount += __shfl_down_sync(0xffffffffu, bcount, off);
        mx = max(mx, __shfl_down_sync(0xffffffffu, mx, off));
    }
    if (lane == 0) {
        PlanOut o;
        o.frag_len = a + (uint32_t)kn_final;
        o.pt_cnt = bcount + (uint32_t)kn_final;
        o.max_kn = (uint32_t)mx;
        o.pad = 0;
        out[w] = o;
    }
    }
}

cudaError_t launch_plan(bool wide, const void *codes, const EvalItem *items, uint32_t n,
                        PlanOut *out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const int threads = 256;
    const uint32_t blocks = (uint32_t)(((uint64_t)n * 32 + threads - 1) / threads);
    if (wide) plan_kernel<uint32_t><<<blocks, threads, 0, s>>>((const uint32_t *)codes, items, n, nullptr, out);
    else plan_kernel<uint8_t><<<blocks, threads, 0, s>>>((const uint8_t *)codes, items, n, nullptr, out);
    return cudaGetLastError();
}

cudaError_t launch_plan_dev(bool wide, const void *codes, const EvalItem *items, uint32_t n_max,
                            const uint32_t *n_dev, PlanOut *out, int sms, cudaStream_t s, bool pdl)
{
    if (n_max == 0) return cudaSuccess;
    const int threads = 256;
    const uint64_t want = ((uint64_t)n_max * 32 + threads - 1) / threads;
    const uint32_t blocks = (uint32_t)umin64(want, (uint64_t)sms * 16);
    if (pdl) {
        if (wide)
            return launch_pdl(plan_kernel<uint32_t>, dim3(blocks), dim3(threads), 0, s, (const uint32_t *)codes, items,
                              n_max, n_dev, out);
        return launch_pdl(plan_kernel<uint8_t>, dim3(blocks), dim3(threads), 0, s, (const uint8_t *)codes, items,
                          n_max, n_dev, out);
    }
    if (wide) plan_kernel<uint32_t><<<blocks, threads, 0, s>>>((const uint32_t *)codes, items, n_max, n_dev, out);
    else plan_kernel<uint8_t><<<blocks, threads, 0, s>>>((const uint8_t *)codes, items, n_max, n_dev, out);
    return cudaGetLastError();
}

// Single-CTA exclusive scan of the plan: fragment offsets and value-buffer
// bases, written into the items; totals = {codes, entries, max stack}.
__global__ void plan_scan_kernel(EvalItem *items, const PlanOut *plan, uint32_t n,
                                 const uint32_t *n_dev, uint64_t *frag_off, uint64_t *totals)
{
    pdl_wait();
    if (n_dev) n = *n_dev;
    if (n == 0) {
        if (threadIdx.x == 0) {
            frag_off[0] = 0;
            totals[0] = totals[1] = totals[2] = 0;
        }
        return;
    }
    __shared__ uint64_t sa[1024], sb[1024];
    __shared__ uint32_t smx[1024];
    const uint32_t t = threadIdx.x, T = blockDim.x;
    const uint32_t per = (n + T - 1) / T;
    const uint32_t lo = min(t * per, n), hi = min(lo + per, n);
    uint64_t a = 0, b = 0;
    uint32_t mx = 0;
    for (uint32_t i = lo; i < hi; ++i) {
        a += plan[i].frag_len;
        b += plan[i].pt_cnt;
        mx = max(mx, plan[i].max_kn);
    }
    sa[t] = a; sb[t] = b; smx[t] = mx;
    __syncthreads();
    for (uint32_t off = 1; off < T; off <<= 1) {
        uint64_t va = 0, vb = 0;
        uint32_t vm = 0;
        if (t >= off) { va = sa[t - off]; vb = sb[t - off]; vm = smx[t - off]; }
        __syncthreads();
        if (t >= off) { sa[t] += va; sb[t] += vb; smx[t] = max(smx[t], vm); }
        __syncthreads();
    }
    uint64_t ra = sa[t] - a, rb = sb[t] - b;   // exclusive
    for (uint32_t i = lo; i < hi; ++i) {
        const PlanOut p = plan[i];
        items[i].frag_off = ra;
        items[i].frag_len = p.frag_len;
        items[i].pt_base = rb;
        items[i].pt_cnt = p.pt_cnt;
        frag_off[i] = ra;
        ra += p.frag_len;
        rb += p.pt_cnt;
    }
    if (t == T - 1) {
        frag_off[n] = sa[t];
        totals[0] = sa[t];
        totals[1] = sb[t];
        totals[2] = smx[t];
    }
}

cudaError_t launch_plan_scan(EvalItem *items, const PlanOut *plan, uint32_t n,
                             uint64_t *frag_off, uint64_t *totals, cudaStream_t s)
{
    plan_scan_kernel<<<1, 1024, 0, s>>>(items, plan, n, nullptr, frag_off, totals);
    return cudaGetLastError();
}

cudaError_t launch_plan_scan_dev(EvalItem *items, const PlanOut *plan, const uint32_t *n_dev,
                                 uint64_t *frag_off, uint64_t *totals, cudaStream_t s, bool pdl)
{
    if (pdl) return launch_pdl(plan_scan_kernel, dim3(1), dim3(1024), 0, s, items, plan, 0u, n_dev, frag_off, totals);
    plan_scan_kernel<<<1, 1024, 0, s>>>(items, plan, 0, n_dev, frag_off, totals);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- validation

// Upload check (Sec. 2.1 encoding): read right to left, every operator needs
// two values on the stack and exactly one value remains.  Per chunk: the
// smallest incoming stack that avoids underflow and the net change; chunks
// compose as  need = max(need_R, need_L - delta_R), delta = delta_R + delta_L.
struct Need {
    int64_t need, delta;
};
__device__ __forceinline__ Need need_after(Need first, Need then) {
    return Need{max(first.need, then.need - first.delta), first.delta + then.delta};
}

__global__ void validate_kernel(const uint8_t *__restrict__ codes, const EvalItem *__restrict__ chunks,
                                uint32_t n, uint32_t n_consts, ValOut *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= n) return;
    const EvalItem it = chunks[w];
    const uint64_t len = it.end - it.begin;
    const uint64_t seg = (len + 31) / 32;
    const uint64_t lo = umin64(it.begin + lane * seg, it.end);
    const uint64_t hi = umin64(lo + seg, it.end);
    Need f{kNegInf, 0};
    uint32_t bad = 0;
    for (uint64_t p = hi; p > lo; --p) {
        const uint32_t c = codes[p - 1];
        if (c >= 5 + n_consts) bad = 1;
        if (c >= 4) {
            f.delta += 1;
        } else {
            f.need = max(f.need, 2 - f.delta);
            f.delta -= 1;
        }
    }
    Need G = f;
    for (int off = 1; off < 32; off <<= 1) {
        Need o;
        o.need = __shfl_down_sync(0xffffffffu, G.need, off);
        o.delta = __shfl_down_sync(0xffffffffu, G.delta, off);
        if (lane + off < 32) G = need_after(o, G);
    }
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
        ValOut v;
        v.need = G.need;
        v.delta = G.delta;
        v.bad_code = bad;
        v.pad = 0;
        out[w] = v;
    }
}

cudaError_t launch_validate(const uint8_t *codes, const EvalItem *chunks, uint32_t n_chunks,
                            uint32_t n_consts, ValOut *out, cudaStream_t s)
{
    if (n_chunks == 0) return cudaSuccess;
    const int threads = 256;
    const uint32_t blocks = (uint32_t)(((uint64_t)n_chunks * 32 + threads - 1) / threads);
    validate_kernel<<<blocks, threads, 0, s>>>(codes, chunks, n_chunks, n_consts, out);
    return cudaGetLastError();
}

__global__ void validate_trees_kernel(const ValOut *__restrict__ v, const uint32_t *__restrict__ first,
                                      uint32_t n_trees, uint32_t *bad_count)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_trees) return;
    const uint32_t a = first[t], b = first[t + 1];
    Need acc{kNegInf, 0};
    bool bad = (a == b);
    for (uint32_t k = b; k > a; --k) {
        const ValOut c = v[k - 1];
        bad |= c.bad_code != 0;
        acc = need_after(acc, Need{c.need, c.delta});
    }
    if (bad || acc.need > 0 || acc.delta != 1) atomicAdd(bad_count, 1u);
}

cudaError_t launch_validate_trees(const ValOut *chunk_out, const uint32_t *tree_first_chunk,
                                  uint32_t n_trees, uint32_t *bad_count, cudaStream_t s)
{
    if (n_trees == 0) return cudaSuccess;
    validate_trees_kernel<<<(n_trees + 255) / 256, 256, 0, s>>>(chunk_out, tree_first_chunk,
                                                               n_trees, bad_count);
    return cudaGetLastError();
}

}  // namespace gpk
