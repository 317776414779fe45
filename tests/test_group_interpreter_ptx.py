"""The evaluator's group interpreters (hand-written inline PTX in
gp_eval.cu: byte codes, and the upper trees' 32-bit codes whose
value-buffer leaves read staged entries), run on the CPU by a model of the
PTX forms they use, against
its plain push/pop meaning (Sec. 2.2 EVAL read right to left; protected
division of Table gp.details) on random 16-code groups: operator mixes,
stack depths that make words exit early, NaN, signed zeros, subnormals and
zero divisors.  No GPU: this checks the interpreter's control flow (labels,
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


def one_group(parsed, rng):
    """Run one random group through the PTX model and the plain meaning;
    returns None when they agree, else a description."""
    pool = [F(0.0), F(-0.0), F(1.0), F(np.nan), F(2.5e-40), F(-3.0)]

    def rv():
        return F(rng.choice(pool)) if rng.random() < 0.2 else F(rng.standard_normal())

    shared = {TB + code * S: (rv(), rv()) for code in range(4, 256)}
    for k in range(K + 8):
        shared[WB + k * S] = (rv(), rv())
    t = WB + int(rng.integers(0, K + 1)) * S
    p_op = rng.uniform(0.2, 0.8)
    codes = [int(rng.integers(0, 4)) if rng.random() < p_op else int(rng.integers(4, 132)) for _ in range(16)]
    words = [0, 0, 0, 0]
    for wi in range(4):
        for k, bit in enumerate((24, 16, 8, 0)):
            words[3 - wi] |= codes[4 * wi + k] << bit
    q, tos, d0 = int(rng.integers(0, 4)), (rv(), rv()), F(1.0)
    regs = {"%0": tos, "%1": t, "%2": q, "%3": words[0], "%4": words[1], "%5": words[2], "%6": words[3],
            "%7": TB, "%8": d0, "%9": LO, "%10": SPAN, "%11": S}
    got_sh = dict(shared)
    r = run(parsed, regs, got_sh)
    w_tos, w_t, w_q, w_sh = push_pop(
        lambda qq: [((words[qq] >> bit) & 0xFF, None) for bit in (24, 16, 8, 0)],
        lambda c, j, sh: sh[TB + c * S], q, tos, t, d0, shared)
    q_out = r["%2"] - (1 << 32) if r["%2"] > 0x7FFFFFFF else r["%2"]
    if not same(r["%0"], w_tos) or r["%1"] != w_t or q_out != w_q:
        return f"codes {codes} from word {q}: tos {r['%0']} vs {w_tos}, t {r['%1']} vs {w_t}, q {q_out} vs {w_q}"
    for addr in range(WB, w_t, S):                   # the live stack
        if not same(got_sh[addr], w_sh[addr]):
            return f"codes {codes}: stack entry {(addr - WB) // S} differs"
    return None


@pytest.fixture(scope="module")
def parsed():
    return parse(group_asm(SRC))


def test_group_interpreter_matches_push_pop(parsed):
    rng = np.random.default_rng(2019)
    for _ in range(1000):
        bad = one_group(parsed, rng)
        assert bad is None, bad


def test_model_catches_a_planted_operand_swap(parsed):
    """The comparison has teeth: with the operands of one subtraction
    swapped in the PTX text, some group disagrees."""
    text = group_asm(SRC)
    planted = text.replace("sub.rn.f32x2 %0, %0, v;", "sub.rn.f32x2 %0, v, %0;", 1)
    assert planted != text
    rng = np.random.default_rng(7)
    assert any(one_group(parse(planted), rng) for _ in range(300))


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
