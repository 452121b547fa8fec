"""The k-point batch of the 16-bit chains (a host-side plan, no GPU needed): a
nao-sized step of one (q, k) pair has ceil(naux nao / 128) * ntau output tiles,
and small systems put enough k-points of one q into each launch for ~16 rounds of
the 152 SMs (at most 32 and nk)."""
import ctypes
import math

import pytest

from paper_2206_07660_gb300 import LIB_PATH


def _plan():
    lib = ctypes.CDLL(LIB_PATH)
    fn = lib.gwdbg_chain_pbatch
    fn.argtypes = [ctypes.c_int] * 4
    fn.restype = ctypes.c_int
    return fn


@pytest.mark.parametrize("nao,naux,nk,ntau,want", [
    (52, 400, 64, 100, 1),   # C3: one k per launch
    (26, 200, 27, 92, 1),    # C2
    (8, 32, 8, 32, 8),       # C1: the whole mesh
    (8, 64, 64, 64, 10),     # C4, smallest systems
    (12, 96, 64, 64, 5),
    (16, 128, 64, 64, 3),
    (26, 208, 64, 64, 1),
    (40, 320, 64, 64, 1),
])
def test_batch_sizes(nao, naux, nk, ntau, want):
    fn = _plan()
    tiles = math.ceil(naux * nao / 128) * ntau
    expect = max(1, min(32, nk, math.ceil(16 * 152 / tiles)))
    assert expect == want
    assert fn(nao, naux, nk, ntau) == want
