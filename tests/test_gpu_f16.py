"""fp16 pieces on the kind::f16 tensor cores: each operand row x is stored as
2^e (hi + lo) with hi = rn16(x 2^-e), lo = rn16(x 2^-e - hi) and one power-of-two
exponent e per row (max |x| 2^-e < 2^15); three products (hi*hi, hi*lo, lo*hi) in
FP32 and the epilogue's exact rescaling by 2^(eA + eB) must match a complex128
product to the ~2^-21 relative level of the TF32 pieces, on ragged shapes and on
rows whose scales span 2^-30 .. 2^30.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [(128, 16, 16), (257, 70, 45), (300, 200, 100), (1000, 400, 676), (4000, 900, 80), (384, 400, 2704)]


def _lib():
    import torch
    from paper_2206_07660_gb300 import load
    torch.cuda.set_device(0)
    lib = load()
    lib.gwdbg_umma_cgemm_f16.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int] * 3 + [ctypes.c_void_p]
    lib.gwdbg_umma_cgemm_f16.restype = ctypes.c_int
    return lib


@pytest.mark.parametrize("M,N,K", SHAPES)
@pytest.mark.parametrize("spread", [0, 30])
def test_f16_pieces_gemm(M, N, K, spread):
    import torch
    lib = _lib()
    rng = np.random.default_rng(M * 7919 + N * 31 + K + spread)
    A = rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))
    B = rng.standard_normal((N, K)) + 1j * rng.standard_normal((N, K))
    if spread:
        A *= np.exp2(rng.integers(-spread, spread + 1, (M, 1)))
        B *= np.exp2(rng.integers(-spread, spread + 1, (N, 1)))
    ref = A @ np.conj(B).T
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.full((M, N), np.nan + 0j, dtype=torch.complex128, device="cuda")
    st = lib.gwdbg_umma_cgemm_f16(dA.data_ptr(), dB.data_ptr(), M, N, K, dC.data_ptr())
    assert st == 0
    C = dC.cpu().numpy()
    assert np.all(np.isfinite(C))
    # entrywise error against the size of the terms summed: sqrt(2K) |a_row| |b_row|
    scale = np.sqrt(2.0 * K) * np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=1)[None, :]
    err = (np.abs(C - ref) / scale).max()
    assert err < 3e-6, err
