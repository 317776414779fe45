"""The evaluator's group interpreters (hand-written inline PTX in
gp_eval.cu: the byte-code group loop, and the upper trees' 32-bit codes
whose value-buffer leaves read staged entries), run on the CPU by a model
of the PTX forms they use, against their plain push/pop meaning (Sec. 2.2
EVAL read right to left; protected division of Table gp.details) on random
groups: operator mixes, entries at every position,
stack depths that make words stop for room and operators that find the
window empty, NaN, signed zeros, subnormals and zero divisors.  No GPU: this checks the interpreter's control flow (labels,
branches, the divide routine's return index, the window checks) bit for
bit; the GPU parity tests check the compiled kernel."""
import os
import shutil

import numpy as np
import pytest

from tests.ptx_group_emu import F, M32, group_asm, parse, run

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_1902_09215_gb300", "csrc", "gp_eval.cu")

pytestmark = pytest.mark.skipif(not (shutil.which("gcc") or shutil.which("cc")), reason="needs a C compiler")

K, S = 32, 192                       # window entries, bytes per entry (24 lanes x float2)
WB, TB = 0x1000, 0x100000 - 4 * S    # window base, leaf table base (row = TB + code * S)
LO, SPAN = WB + 4 * S, (K - 8) * S   # a word runs with >= 4 entries below and room for 4


def push_pop(word_codes, leaf, q, tos, t, d0, shared):
    """word_codes(q): the (code, position) pairs of word q in reading order;
    leaf(code, position, shared): a leaf's value."""
    sh = dict(shared)
    while q >= 0:
        if ((t - LO) & M32) > SPAN:
            return tos, t, q, sh
        for c, j in word_codes(q):
            if c > 3:
                sh[t] = tos
                t += S
                tos = leaf(c, j, sh)
                continue
            t -= S
            v = sh[t]
            with np.errstate(all="ignore"):
                if c == 0:
                    tos = (F(tos[0] + v[0]), F(tos[1] + v[1]))
                elif c == 1:
                    tos = (F(tos[0] - v[0]), F(tos[1] - v[1]))
                elif c == 2:
                    tos = (F(tos[0] * v[0]), F(tos[1] * v[1]))
                else:
                    tos = tuple(F(a / b) if (np.isnan(b) or b != 0) else F(d0) for a, b in zip(tos, v))
        q -= 1
    return tos, t, -1, sh


def same(a, b):
    return all((np.isnan(x) and np.isnan(y)) or F(x).view(np.uint32) == F(y).view(np.uint32)
               for x, y in zip(a, b))


GBASE = 0x40000                      # global address of the lowest group of the byte-code loop
ROOM = (K - 4) * S                   # a word of the byte-code loop runs with room for 4 pushes


def loop_meaning(groups, pos, tos, t, d0, shared):
    """The byte-code group loop's meaning: groups[g] holds the 16 codes of
    the group at GBASE + 16 g (code j at position j); reading starts at
    position `pos` of the highest group and goes right to left, group after
    group.  A word start reached on the way (and the entry itself, if it
    is one) needs room for four pushes, else the loop stops there (exit
    4Q+3); an operator that finds the window empty stops before popping
    (exit 16 + position); after the lowest group the exit is -1."""
    sh = dict(shared)
    g = len(groups) - 1
    j = pos
    while True:
        while j >= 0:
            if j % 4 == 3 and ((t - WB) & M32) > ROOM:
                return j, g, tos, t, sh
            c = groups[g][j]
            if c > 3:
                sh[t] = tos
                t += S
                tos = sh[TB + c * S]
            else:
                if t == WB:
                    return 16 + j, g, tos, t, sh
                t -= S
                v = sh[t]
                with np.errstate(all="ignore"):
                    if c == 0:
                        tos = (F(tos[0] + v[0]), F(tos[1] + v[1]))
                    elif c == 1:
                        tos = (F(tos[0] - v[0]), F(tos[1] - v[1]))
                    elif c == 2:
                        tos = (F(tos[0] * v[0]), F(tos[1] * v[1]))
                    else:
                        tos = tuple(F(a / b) if (np.isnan(b) or b != 0) else F(d0) for a, b in zip(tos, v))
            j -= 1
        if g == 0:
            return -1, 0, tos, t, sh
        g -= 1
        j = 15


def one_loop(parsed, rng):
    """Run the byte-code group loop on 1..3 random groups through the PTX
    model and its plain meaning; returns None when they agree, else a
    description."""
    pool = [F(0.0), F(-0.0), F(1.0), F(np.nan), F(2.5e-40), F(-3.0)]

    def rv():
        return F(rng.choice(pool)) if rng.random() < 0.2 else F(rng.standard_normal())

    shared = {TB + code * S: (rv(), rv()) for code in range(4, 256)}
    for k in range(K + 8):
        shared[WB + k * S] = (rv(), rv())
    t = WB + int(rng.integers(0, K + 1)) * S
    p_op = rng.uniform(0.2, 0.8)
    n = int(rng.integers(1, 4))
    groups = [[int(rng.integers(0, 4)) if rng.random() < p_op else int(rng.integers(4, 132)) for _ in range(16)]
              for _ in range(n)]
    gmem = {GBASE + 16 * g: bytes(groups[g]) for g in range(n)}
    pos, tos, d0 = int(rng.integers(0, 16)), (rv(), rv()), F(1.0)
    if pos % 4 != 3 and t - WB > (K - 3) * S:       # mid-word entries come with room for the word
        t = WB + (K - 3) * S
    regs = {"%0": tos, "%1": t, "%2": pos, "%3": GBASE + 16 * (n - 1), "%4": GBASE, "%5": TB, "%6": d0,
            "%7": WB, "%8": ROOM, "%9": S}
    got_sh = dict(shared)
    r = run(parsed, regs, got_sh, gmem)
    w_x, w_g, w_tos, w_t, w_sh = loop_meaning(groups, pos, tos, t, d0, shared)
    x_out = r["%2"] - (1 << 32) if r["%2"] > 0x7FFFFFFF else r["%2"]
    g_out = (r["%3"] - GBASE) // 16
    if not same(r["%0"], w_tos) or r["%1"] != w_t or x_out != w_x or g_out != w_g:
        return (f"groups {groups} from {pos}: tos {r['%0']} vs {w_tos}, t {r['%1']} vs {w_t}, "
                f"exit {x_out} vs {w_x}, group {g_out} vs {w_g}")
    for addr in range(WB, w_t, S):                   # the live stack
        if not same(got_sh[addr], w_sh[addr]):
            return f"groups {groups}: stack entry {(addr - WB) // S} differs"
    return None


@pytest.fixture(scope="module")
def parsed():
    return parse(group_asm(SRC))


def test_group_loop_matches_push_pop(parsed):
    rng = np.random.default_rng(2019)
    for _ in range(1500):
        bad = one_loop(parsed, rng)
        assert bad is None, bad


# Planted mistakes in the PTX text (function, text, replacement, every
# occurrence or only the first): each must make some random run disagree
# with the plain meaning.  A run that the model cannot finish (a read of a
# shared entry below the window, which on the GPU would read another lane's
# or warp's data) counts as caught too.
PLANTS = [
    ("groups_u8", "sub.rn.f32x2 %0, %0, v;", "sub.rn.f32x2 %0, v, %0;", False),
    ("groups_u8", "mul.rn.f32x2 %0, %0, v;", "add.rn.f32x2 %0, %0, v;", False),
    ("groups_u8", "setp.lt.u32 p, c, 2;", "setp.lt.u32 p, c, 1;", False),
    ("groups_u8", "selp.f32 tx, qx, %6, p;", "selp.f32 tx, %6, qx, p;", False),
    ("groups_u8", "RET: .branchtargets E0, E1,", "RET: .branchtargets E1, E0,", False),
    ("groups_u8", "setp.gt.u32 p, dd, %8;", "setp.lt.u32 p, dd, %8;", False),
    ("groups_u8", "st.shared.b64 [%1], %0;\n\tadd.u32 %1, %1, %9;",
     "add.u32 %1, %1, %9;\n\tst.shared.b64 [%1], %0;", False),
    ("groups_u8", "setp.eq.u32 p, %1, %7;", "setp.eq.u32 p, %1, %5;", True),
    ("groups_u8", "ENT: .branchtargets N0, N1, N2, W0,", "ENT: .branchtargets N0, N1, N2, N3,", False),
    ("group_u32", "sub.rn.f32x2 %0, %0, v;", "sub.rn.f32x2 %0, v, %0;", False),
    ("group_u32", "ld.shared.b64 %0, [%24+15*%23];", "ld.shared.b64 %0, [%24+14*%23];", False),
    ("group_u32", "256;", "128;", True),
    ("group_u32", "selp.f32 ty, qy, %20, p;", "selp.f32 ty, %20, qy, p;", False),
    ("group_u32", "setp.gt.u32 p, dd, %22;", "setp.lt.u32 p, dd, %22;", False),
]


@pytest.mark.parametrize("fn,find,repl,every", PLANTS,
                         ids=[f"{p[0]}:{p[1][:28]}" for p in PLANTS])
def test_model_catches_planted_mistakes(fn, find, repl, every):
    """The comparison has teeth: with one mistake planted in the PTX text,
    some run disagrees."""
    text = group_asm(SRC, fn)
    assert find in text
    planted = text.replace(find, repl) if every else text.replace(find, repl, 1)
    prog = parse(planted)
    trial = one_loop if fn == "groups_u8" else one_upper_group
    rng = np.random.default_rng(7)
    for _ in range(3000):
        try:
            if trial(prog, rng):
                return
        except (KeyError, RuntimeError):
            return
    pytest.fail("planted mistake not caught")


STAGE = 0x200000                     # staged value entries of the group: STAGE + position * S


def one_upper_group(parsed, rng):
    """The upper-tree interpreter (32-bit codes; codes >= 256 are
    value-buffer leaves read from the staged entry of their position in the
    group) on one random group, against the same plain meaning."""
    pool = [F(0.0), F(-0.0), F(1.0), F(np.nan), F(2.5e-40), F(-3.0)]

    def rv():
        return F(rng.choice(pool)) if rng.random() < 0.2 else F(rng.standard_normal())

    shared = {TB + code * S: (rv(), rv()) for code in range(4, 256)}
    for j in range(16):
        shared[STAGE + j * S] = (rv(), rv())
    for k in range(K + 8):
        shared[WB + k * S] = (rv(), rv())
    t = WB + int(rng.integers(0, K + 1)) * S
    p_op = rng.uniform(0.2, 0.8)

    def code():
        if rng.random() < p_op:
            return int(rng.integers(0, 4))
        return int(rng.integers(4, 132)) if rng.random() < 0.5 else 256 + int(rng.integers(0, 1 << 20))

    codes = [code() for _ in range(16)]          # codes[j]: position j of the group
    q, tos, d0 = int(rng.integers(0, 4)), (rv(), rv()), F(1.0)
    regs = {"%0": tos, "%1": t, "%2": q, "%19": TB, "%20": d0, "%21": LO, "%22": SPAN, "%23": S, "%24": STAGE}
    regs.update({f"%{3 + j}": codes[j] for j in range(16)})
    got_sh = dict(shared)
    r = run(parsed, regs, got_sh)
    w_tos, w_t, w_q, w_sh = push_pop(
        lambda qq: [(codes[j], j) for j in (4 * qq + 3, 4 * qq + 2, 4 * qq + 1, 4 * qq)],
        lambda c, j, sh: sh[STAGE + j * S] if c >= 256 else sh[TB + c * S], q, tos, t, d0, shared)
    q_out = r["%2"] - (1 << 32) if r["%2"] > 0x7FFFFFFF else r["%2"]
    if not same(r["%0"], w_tos) or r["%1"] != w_t or q_out != w_q:
        return f"codes {codes} from word {q}: tos {r['%0']} vs {w_tos}, t {r['%1']} vs {w_t}, q {q_out} vs {w_q}"
    for addr in range(WB, w_t, S):
        if not same(got_sh[addr], w_sh[addr]):
            return f"codes {codes}: stack entry {(addr - WB) // S} differs"
    return None


def test_upper_group_interpreter_matches_push_pop():
    parsed = parse(group_asm(SRC, "group_u32"))
    rng = np.random.default_rng(1902)
    for _ in range(1000):
        bad = one_upper_group(parsed, rng)
        assert bad is None, bad
