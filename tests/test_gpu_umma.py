"""The split-TF32 tensor-core GEMM under the P~0 and Sigma~ contractions.

Complex operands are embedded as real [re, im] rows, split into TF32 high and
low planes, and multiplied with tcgen05 (kind::tf32) into FP32 tensor memory.
With three products (hi*hi, hi*lo, lo*hi) the result must match a complex128
matrix product to a few 1e-7 relative; with the high planes alone, to TF32's
~1e-3.  Both kernel variants (a persistent tile loop and one tile per block)
run on shapes with ragged M/N/K edges, several tiles per block and a split K
range.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [
    # M, N, K, conjB, nseg, ksplit
    (128, 16, 16, 1, 1, 1),
    (128, 16, 16, 1, 3, 1),
    (257, 70, 45, 0, 3, 1),
    (300, 200, 100, 1, 3, 1),
    (1000, 400, 676, 1, 3, 1),
    (4000, 900, 80, 1, 3, 1),     # ~250 output tiles: several per persistent block
    (384, 400, 2704, 1, 3, 1),
    (384, 400, 2704, 1, 3, 4),    # split K range, atomically added partials
    (200, 52, 1300, 0, 3, 3),
]


def _lib():
    import torch
    from paper_2206_07660_gb300 import load
    torch.cuda.set_device(0)
    lib = load()
    lib.gwdbg_umma_cgemm_split.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int] * 6 + [ctypes.c_void_p]
    lib.gwdbg_umma_cgemm_split.restype = ctypes.c_int
    lib.gwdbg_umma_set_persistent.argtypes = [ctypes.c_int]
    lib.gwdbg_umma_set_persistent.restype = ctypes.c_int
    return lib


@pytest.mark.parametrize("persistent", [1, 0])
@pytest.mark.parametrize("M,N,K,conjB,nseg,ksplit", SHAPES)
def test_split_tf32_gemm(persistent, M, N, K, conjB, nseg, ksplit):
    import torch
    lib = _lib()
    rng = np.random.default_rng(M * 7919 + N * 31 + K + 1000 * ksplit)
    A = rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))
    if conjB:
        B = rng.standard_normal((N, K)) + 1j * rng.standard_normal((N, K))
        ref = A @ np.conj(B).T
    else:
        B = rng.standard_normal((K, N)) + 1j * rng.standard_normal((K, N))
        ref = A @ B
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = torch.full((M, N), np.nan + 0j, dtype=torch.complex128, device="cuda")
    old = lib.gwdbg_umma_set_persistent(persistent)
    try:
        st = lib.gwdbg_umma_cgemm_split(dA.data_ptr(), dB.data_ptr(), M, N, K, conjB, nseg, ksplit, dC.data_ptr())
    finally:
        lib.gwdbg_umma_set_persistent(old)
    assert st == 0
    C = dC.cpu().numpy()
    assert np.all(np.isfinite(C))
    # entrywise error against the size of the terms summed: sqrt(K) * |a||b|
    scale = np.sqrt(2.0 * K) * 2.0
    err = np.abs(C - ref).max() / scale
    tol = 3e-6 if nseg == 3 else 3e-3
    assert err < tol, err


def test_autotuned_tiles_match_cost_model():
    """The N-tile autotuner changes only the tiling: results agree with the
    cost-model tile, and accumulating outputs are not disturbed by the trial runs."""
    import torch
    lib = _lib()
    lib.gwdbg_umma_set_autotune.argtypes = [ctypes.c_int]
    lib.gwdbg_umma_set_autotune.restype = ctypes.c_int
    lib.gwdbg_umma_tuned.argtypes = [ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 3
    lib.gwdbg_umma_tuned.restype = ctypes.c_int
    M, N, K = 700, 300, 400
    rng = np.random.default_rng(77)
    A = rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))
    B = rng.standard_normal((N, K)) + 1j * rng.standard_normal((N, K))
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    out = {}
    for tune in (0, 1):
        for ks in (1, 3):   # ks > 1: accumulating output (split K range)
            old = lib.gwdbg_umma_set_autotune(tune)
            dC = torch.zeros((M, N), dtype=torch.complex128, device="cuda")
            try:
                st = lib.gwdbg_umma_cgemm_split(dA.data_ptr(), dB.data_ptr(), M, N, K, 1, 3, ks, dC.data_ptr())
            finally:
                lib.gwdbg_umma_set_autotune(old)
            assert st == 0
            out[(tune, ks)] = dC.cpu().numpy()
    ref = A @ np.conj(B).T
    scale = np.sqrt(2.0 * K) * 2.0
    for v in out.values():
        assert np.abs(v - ref).max() / scale < 3e-6
    assert np.abs(out[(1, 1)] - out[(0, 1)]).max() / scale < 1e-6
    assert np.abs(out[(1, 3)] - out[(0, 3)]).max() / scale < 1e-6
    n = lib.gwdbg_umma_tuned(0, None, None, None)
    assert n >= 1
    bn = ctypes.c_int()
    lib.gwdbg_umma_tuned(0, None, None, ctypes.byref(bn))
    assert bn.value in (32, 48, 64, 80, 96, 112, 128, 160, 192, 224, 256)


@pytest.mark.parametrize("bn", [256, 224, 192, 160, 128, 80])
@pytest.mark.parametrize("M,N,K,ksplit", [(300, 200, 100, 1), (257, 130, 700, 3), (700, 260, 45, 1)])
def test_forced_tiles(bn, M, N, K, ksplit):
    """N tiles of the persistent kernel on ragged shapes: ping-pong epilogues (two
    groups of 4 warps, up to 128 columns) and the split epilogue of the 160..256-column
    tiles (8 warps, each half of the columns)."""
    import torch
    lib = _lib()
    lib.gwdbg_umma_force_bn.argtypes = [ctypes.c_int]
    lib.gwdbg_umma_force_bn.restype = ctypes.c_int
    rng = np.random.default_rng(bn + M + N)
    A = rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))
    B = rng.standard_normal((N, K)) + 1j * rng.standard_normal((N, K))
    ref = A @ np.conj(B).T
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.full((M, N), np.nan + 0j, dtype=torch.complex128, device="cuda")
    old = lib.gwdbg_umma_force_bn(bn)
    try:
        st = lib.gwdbg_umma_cgemm_split(dA.data_ptr(), dB.data_ptr(), M, N, K, 1, 3, ksplit, dC.data_ptr())
    finally:
        lib.gwdbg_umma_force_bn(old)
    assert st == 0
    C = dC.cpu().numpy()
    assert np.all(np.isfinite(C))
    assert np.abs(C - ref).max() / (np.sqrt(2.0 * K) * 2.0) < 3e-6
