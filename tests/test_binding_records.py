"""Argument marshalling of the Python binding (no GPU): crossover records
built from arrays are the same bytes as records built one by one through
ctypes, for every integer width and sign the fields can receive."""
import ctypes

import numpy as np
import pytest

from paper_1902_09215_gb300 import gp


def one_by_one(mum, dad, mum_point, dad_point):
    ops = (gp.gp_xo * len(mum))()
    for k, (a, b, i, j) in enumerate(zip(mum, dad, mum_point, dad_point)):
        ops[k] = gp.gp_xo(int(a), int(b), int(i), int(j))
    return ops


@pytest.mark.parametrize("n", [0, 1, 7, 4000])
def test_records_from_arrays(n):
    rng = np.random.default_rng(n)
    mum = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    dad = rng.integers(0, 4000, n)
    mp = rng.integers(0, 2 ** 63, n, dtype=np.int64).astype(np.uint64)
    dp = rng.integers(0, 10 ** 6, n, dtype=np.int32)
    assert bytes(gp.make_xo(mum, dad, mp, dp)) == bytes(one_by_one(mum, dad, mp, dp))


def test_records_wrap_like_ctypes():
    cases = ([-1, 5], [2 ** 32 + 3, 0], [-2, 2 ** 63], [0, 2 ** 64 - 1])
    assert bytes(gp.make_xo(*cases)) == bytes(one_by_one(*cases))
    assert ctypes.sizeof(gp.gp_xo) == 24


def test_records_need_equal_lengths():
    with pytest.raises(ValueError):
        gp.make_xo([0, 1], [0], [0, 0], [0, 0])


@pytest.mark.parametrize("n", [0, 1, 300])
def test_records_split_back_to_arrays(n):
    rng = np.random.default_rng(10 + n)
    cols = (rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32),
            rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32),
            rng.integers(0, 2 ** 63, n, dtype=np.int64).astype(np.uint64) * 2 + 1,
            rng.integers(0, 2 ** 63, n, dtype=np.int64).astype(np.uint64))
    out = gp.split_xo(one_by_one(*cols))
    for got, want, dt in zip(out, cols, (np.uint32, np.uint32, np.uint64, np.uint64)):
        assert got.dtype == dt and np.array_equal(got, want)
