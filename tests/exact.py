"""Independent exact evaluator used to pin the oracle.

Values are exact rationals (fractions.Fraction) carried with an explicit
sign-of-zero flag; every tree node is the exact result of its operation on
its children's values, then rounded once to the target format with round to
nearest, ties to even, implemented here from the definition of the binary32
and binary64 formats (IEEE 754-2008 Sec. 4.3.1), not with the C library.
Protected division returns 1 for a zero divisor (Table gp.details).

It parses prefix trees recursively in Python and shares nothing with the C
oracle beyond the input tables.
"""
from __future__ import annotations

import math
from fractions import Fraction

INF = float("inf")


class V:
    """An IEEE value: exact rational q, or +-inf / nan, plus a zero sign."""
    __slots__ = ("q", "neg0", "special")

    def __init__(self, q=None, neg0=False, special=None):
        self.q, self.neg0, self.special = q, neg0, special

    @staticmethod
    def of(f: float) -> "V":
        if math.isnan(f):
            return V(special="nan")
        if math.isinf(f):
            return V(special="+inf" if f > 0 else "-inf")
        if f == 0.0:
            return V(Fraction(0), neg0=math.copysign(1.0, f) < 0)
        return V(Fraction(f))

    def is_zero(self):
        return self.special is None and self.q == 0


def _round_binary(a: Fraction, p: int, emin: int, emax: int):
    """Round a > 0 to a binary format with p significand bits; returns a
    Fraction, or None on overflow."""
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    elif Fraction(2) ** (e + 1) <= a:
        e += 1
    q_exp = max(e, emin) - (p - 1)
    quantum = Fraction(2) ** q_exp
    m = a / quantum
    fl = m.numerator // m.denominator
    r = m - fl
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    res = fl * quantum
    if res >= Fraction(2) ** (emax + 1):
        return None
    return res


def round_to(v: V, fmt: str) -> V:
    if v.special is not None or v.q == 0:
        return v
    p, emin, emax = (24, -126, 127) if fmt == "f32" else (53, -1022, 1023)
    r = _round_binary(abs(v.q), p, emin, emax)
    neg = v.q < 0
    if r is None:
        return V(special="-inf" if neg else "+inf")
    if r == 0:
        return V(Fraction(0), neg0=neg)
    return V(-r if neg else r)


def _sign_neg(v: V) -> bool:
    if v.special == "-inf":
        return True
    if v.special == "+inf":
        return False
    return v.q < 0 or (v.q == 0 and v.neg0)


def op_exact(op: int, a: V, b: V, div0: V) -> V:
    """Exact IEEE-semantics result (before rounding) of a op b."""
    if op == 3 and b.is_zero():
        return div0
    if a.special == "nan" or b.special == "nan":
        return V(special="nan")
    if a.special or b.special:
        fa = INF if a.special == "+inf" else -INF if a.special == "-inf" else float(a.q)
        fb = INF if b.special == "+inf" else -INF if b.special == "-inf" else float(b.q)
        if a.special is None and a.q == 0:
            fa = -0.0 if a.neg0 else 0.0
        if b.special is None and b.q == 0:
            fb = -0.0 if b.neg0 else 0.0
        # at least one operand is infinite: IEEE rules give an infinity, a
        # zero or NaN, which Python's float arithmetic reproduces exactly
        with_inf = {0: lambda: fa + fb, 1: lambda: fa - fb, 2: lambda: fa * fb,
                    3: lambda: fa / fb}[op]()
        return V.of(with_inf)
    if op == 0:
        q = a.q + b.q
        if q == 0:
            return V(Fraction(0), neg0=(a.q == 0 and b.q == 0 and a.neg0 and b.neg0))
        return V(q)
    if op == 1:
        q = a.q - b.q
        if q == 0:
            return V(Fraction(0), neg0=(a.q == 0 and b.q == 0 and a.neg0 and not b.neg0))
        return V(q)
    if op == 2:
        q = a.q * b.q
        if q == 0:
            return V(Fraction(0), neg0=_sign_neg(a) != _sign_neg(b))
        return V(q)
    q = a.q / b.q
    if q == 0:
        return V(Fraction(0), neg0=_sign_neg(a) != _sign_neg(b))
    return V(q)


def to_float(v: V) -> float:
    if v.special == "nan":
        return float("nan")
    if v.special:
        return INF if v.special == "+inf" else -INF
    if v.q == 0:
        return -0.0 if v.neg0 else 0.0
    return float(v.q)


def eval_exact_rounded(tree, xval: float, consts, fmt: str = "f32", div0: float = 1.0) -> float:
    """Evaluate a prefix tree for one case, rounding every node to `fmt`."""
    pos = [0]
    d0 = V.of(div0)

    def rec():
        code = int(tree[pos[0]])
        pos[0] += 1
        if code == 4:
            return V.of(float(xval))
        if code >= 5:
            return V.of(float(consts[code - 5]))
        a = rec()
        b = rec()
        return round_to(op_exact(code, a, b, d0), fmt)

    v = rec()
    assert pos[0] == len(tree)
    return to_float(v)


def eval_exact_unrounded(tree, xval: float, consts, div0: float = 1.0):
    """Exact real value of the tree for one case (no rounding); None if a
    division by an exact zero or a non-finite value occurs."""
    pos = [0]

    def rec():
        code = int(tree[pos[0]])
        pos[0] += 1
        if code == 4:
            return Fraction(float(xval))
        if code >= 5:
            return Fraction(float(consts[code - 5]))
        a = rec()
        b = rec()
        if a is None or b is None:
            return None
        if code == 0:
            return a + b
        if code == 1:
            return a - b
        if code == 2:
            return a * b
        return None if b == 0 else a / b

    return rec()


def all_shapes(n: int):
    """Every full binary tree with n nodes (n odd) as a prefix list of
    booleans (True = internal)."""
    if n == 1:
        return [[False]]
    res = []
    for left in range(1, n - 1, 2):
        right = n - 1 - left
        for L in all_shapes(left):
            for R in all_shapes(right):
                res.append([True] + L + R)
    return res
