"""The subtree walk's word step on CPU: the byte-wise formula the extent
kernels use for the net change and lowest running value of the arity walk
over four bytes (an operator, code < 4, adds one; a leaf takes one; a byte
outside the counted range adds nothing), restated in numpy uint32
arithmetic, against a direct walk over every word made of codes that sit
on the formula's edges (0..5, 0x7b..0x85, 0xfb..0xff) and every byte mask."""
import itertools

import numpy as np

U = np.uint32


def word_step(w, cm):
    w, cm = U(w), U(cm)
    nz = ((w & U(0x7C7C7C7C)) + U(0x7F7F7F7F)) | w
    e = (~nz & U(0x80808080)) >> U(6)
    e = (e & cm) | (U(0x01010101) & ~cm)
    E = U((int(e) * 0x01010101) & 0xFFFFFFFF)
    M = U(int(E) + 0x00010203)
    b = [(int(M) >> (8 * k)) & 0xFF for k in range(4)]
    return (int(E) >> 24) - 4, min(b) - 4


def direct(codes, counted):
    r, lo = 0, None
    for c, k in zip(codes, counted):
        if k:
            r += 1 if c < 4 else -1
        lo = r if lo is None else min(lo, r)
    return r, lo


def test_word_step_matches_a_direct_walk():
    edge = [0, 1, 2, 3, 4, 5, 0x7B, 0x7C, 0x7F, 0x80, 0x83, 0x84, 0x85, 0xFB, 0xFC, 0xFF]
    masks = list(itertools.product([0, 1], repeat=4))
    checked = 0
    for codes in itertools.product(edge, repeat=4):
        w = sum(c << (8 * k) for k, c in enumerate(codes))
        for counted in masks:
            cm = sum(0xFF << (8 * k) for k in range(4) if counted[k])
            assert word_step(w, cm) == direct(codes, counted), (codes, counted)
            checked += 1
    assert checked == 16 ** 4 * 16


def test_bytes_from_masks():
    """bytes_from(x): bytes x.. of a word; the counted bytes [a, b) of a
    word are bytes_from(a) & ~bytes_from(b)."""
    def bytes_from(x):
        s = 8 * max(x, 0)
        return (0xFFFFFFFF << s) & 0xFFFFFFFF if s < 32 else 0
    for a in range(-3, 8):
        for b in range(-3, 8):
            cm = bytes_from(a) & ~bytes_from(b) & 0xFFFFFFFF
            want = sum(0xFF << (8 * k) for k in range(4) if a <= k < b)
            assert cm == want
