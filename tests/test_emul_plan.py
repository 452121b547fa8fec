"""Host-side launch plan of the digit-split FP64 products (no GPU needed).

Each value is written as 8 digits of 7 bits (|d_1| <= 2^7, |d_i| <= 2^6 for i > 1);
the product keeps the digit pairs (i, j) with i + j <= nd + 1.  A launch sums, per
output, kreal products of each of its pairs in FP32, which is exact as long as every
partial sum stays an integer below 2^24.  The plan must cover every kept pair exactly
once, smallest significance first, with each launch inside that bound, and refuse a
K for which one pair alone could round.
"""
import ctypes

import pytest

from paper_2206_07660_gb300 import LIB_PATH


def _plan(kreal, nd):
    lib = ctypes.CDLL(LIB_PATH)
    lib.gwdbg_emul_plan.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int]
    lib.gwdbg_emul_plan.restype = ctypes.c_int
    buf = (ctypes.c_int * 192)()
    n = lib.gwdbg_emul_plan(kreal, nd, buf, 64)
    return n, [tuple(buf[3 * i:3 * i + 3]) for i in range(max(n, 0))]


def _bound(i, j):
    return 2 ** (7 if i == 1 else 6) * 2 ** (7 if j == 1 else 6)


@pytest.mark.parametrize("kreal", [2, 64, 184, 200, 400, 800, 1024])
@pytest.mark.parametrize("nd", [8, 5, 4, 1])
def test_plan_is_exact_and_complete(kreal, nd):
    n, plan = _plan(kreal, nd)
    assert n == len(plan) and n > 0
    seen = []
    last_g = None
    for g, i0, i1 in plan:
        assert 1 <= i0 <= i1 <= nd and 2 <= g <= nd + 1
        if last_g is not None:
            assert g <= last_g                      # smallest contributions first
        last_g = g
        pairs = [(i, g - i) for i in range(i0, i1 + 1)]
        assert all(1 <= j <= nd for _, j in pairs)
        assert sum(kreal * _bound(i, j) for i, j in pairs) <= 2 ** 24
        seen += pairs
    want = [(i, j) for i in range(1, nd + 1) for j in range(1, nd + 1) if i + j <= nd + 1]
    assert sorted(seen) == sorted(want)            # every kept pair exactly once


def test_plan_refuses_inexact_k():
    assert _plan(1025, 8)[0] == -1
    assert _plan(1024, 9)[0] == -1                 # more digits than stored


def test_plan_merges_pairs_when_k_is_small():
    # K = 2 ntau = 184 (a transform at ntau 92): every significance in one launch
    n, plan = _plan(184, 8)
    assert n == 8
    # K = 2 naux = 800 (the screened residual at naux 400): the (1, 1) pair alone,
    # and no launch split finer than the bound requires
    n, plan = _plan(800, 8)
    assert plan[-1] == (2, 1, 1)
    assert n == 13
