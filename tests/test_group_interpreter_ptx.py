"""The evaluator's byte-code group interpreter (hand-written inline PTX in
gp_eval.cu), run on the CPU by a model of the PTX forms it uses, against
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


def push_pop(words, q, tos, t, d0, shared):
    sh = dict(shared)
    while q >= 0:
        if ((t - LO) & M32) > SPAN:
            return tos, t, q, sh
        for bit in (24, 16, 8, 0):
            c = (words[q] >> bit) & 0xFF
            if c > 3:
                sh[t] = tos
                t += S
                tos = sh[TB + c * S]
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
    w_tos, w_t, w_q, w_sh = push_pop(words, q, tos, t, d0, shared)
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
