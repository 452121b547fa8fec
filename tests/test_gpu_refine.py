"""Screened solve as a complex64 inversion refined to FP64 accuracy.

Y0 = (I - P~0)^{-1} in complex64, then Newton steps E = I - Y + P~0 Y (the product
FP64-exact up to ~2^-54 through digit-split tensor-core GEMMs), Y <- Y + Y E.
Pinned against numpy's complex128 inverse: each step squares the relative error
(~1e-7 -> ~1e-13 -> FP64 rounding).  The batched digit-split product itself is
checked against complex128 matmul on ragged shapes with a wide dynamic range
across rows and columns.
"""
import ctypes

import numpy as np
import pytest

from gpu_helpers import gpu, rel, system

pytestmark = pytest.mark.gpu


def _lib():
    import torch
    from paper_2206_07660_gb300 import load
    torch.cuda.set_device(0)
    lib = load()
    lib.gwdbg_emul_cgemm.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int] * 5
    lib.gwdbg_emul_cgemm.restype = ctypes.c_int
    lib.gwdbg_screened_refine.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int]
    lib.gwdbg_screened_refine.restype = ctypes.c_int
    lib.gwdbg_screened_refine_bytes.argtypes = [ctypes.c_int64, ctypes.c_int64]
    lib.gwdbg_screened_refine_bytes.restype = ctypes.c_int64
    return lib


def _cn(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("count,M,N,K", [(3, 130, 70, 45), (2, 200, 200, 200), (1, 5, 7, 3), (2, 64, 96, 512),
                                         (5, 129, 33, 260)])
@pytest.mark.parametrize("nd", [8, 5])
def test_emul_cgemm_batched(count, M, N, K, nd):
    import torch
    lib = _lib()
    rng = np.random.default_rng(M * 1000 + N * 10 + K)
    # rows of A and columns of B scaled over 2^-20 .. 2^20 (per-row / per-column exponents)
    A = _cn(rng, (count, M, K)) * np.exp2(rng.integers(-20, 21, (count, M, 1)))
    B = _cn(rng, (count, K, N)) * np.exp2(rng.integers(-20, 21, (count, 1, N)))
    ref = A @ B
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.full((count, M, N), np.nan + 0j, dtype=torch.complex128, device="cuda")
    st = lib.gwdbg_emul_cgemm(dA.data_ptr(), dB.data_ptr(), dC.data_ptr(), count, M, N, K, nd)
    assert st == 0
    C = dC.cpu().numpy()
    # error bound of the digit expansion: 2K products, each below max|A_row| max|B_col|
    # times 2^-52 (8 digits) or (nd + 1) 2^(13 - 7 (nd + 2)) (leading nd digits)
    bound = 2 * K * np.abs(A).max(axis=2, keepdims=True) * np.abs(B).max(axis=1, keepdims=True)
    per = 2.0 ** -50 if nd == 8 else (nd + 1) * 2.0 ** (13 - 7 * (nd + 2))
    err = np.abs(C - ref)
    assert np.all(err <= per * bound)
    if nd < 8:   # the truncation is visible: not an FP64-exact product
        assert err.max() > 2.0 ** -50 * bound.min()


def _p0(nq, ntau, n, seed):
    # negative-definite Hermitian part, as the polarization has: I - P~0 well conditioned
    rng = np.random.default_rng(seed)
    A = _cn(rng, (nq, ntau, n, n)) / np.sqrt(n)
    return -0.5 * (A @ np.conj(np.swapaxes(A, -1, -2))) + 0.3 * (A - np.conj(np.swapaxes(A, -1, -2)))


@pytest.mark.parametrize("n", [130, 400])
def test_refinement_converges(n):
    import torch
    lib = _lib()
    lib.gw_screened_solve_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                              ctypes.c_void_p]
    lib.gw_screened_solve_noalloc.restype = ctypes.c_int
    P0 = _p0(1, 3, n, 7).reshape(3, n, n)
    exact = np.linalg.inv(np.eye(n) - P0) - np.eye(n)
    errs = []
    for steps in (0, 1, 2):
        X = torch.from_numpy(P0.copy()).cuda()
        st = lib.gwdbg_screened_refine(X.data_ptr(), n, 3, 1 << 30, steps)
        assert st == 0
        errs.append(rel(X.cpu().numpy(), exact))
    # the FP64 Gauss-Jordan solve as the yardstick of FP64 accuracy
    src = torch.from_numpy(P0.copy()).cuda()
    dst = torch.empty_like(src)
    assert lib.gw_screened_solve_noalloc(src.data_ptr(), dst.data_ptr(), n, 3, None) == 0
    err_fp64 = rel(dst.cpu().numpy(), exact)
    assert errs[0] < 1e-5          # complex64 inversion
    assert errs[1] < 1e-11         # one Newton step: ~ errs[0]^2
    assert errs[1] < errs[0] ** 2 * 1e3
    assert errs[2] <= 2 * err_fp64 + 1e-16   # as accurate as the FP64 solve


def test_refinement_batches():
    # a workspace for 2 systems forces balanced batches over 7 systems
    import torch
    lib = _lib()
    n, count = 70, 7
    P0 = _p0(1, count, n, 8).reshape(count, n, n)
    exact = np.linalg.inv(np.eye(n) - P0) - np.eye(n)
    one = torch.from_numpy(P0.copy()).cuda()
    assert lib.gwdbg_screened_refine(one.data_ptr(), n, count, 1 << 30, 2) == 0
    small = torch.from_numpy(P0.copy()).cuda()
    wb = lib.gwdbg_screened_refine_bytes(n, 2)
    assert lib.gwdbg_screened_refine(small.data_ptr(), n, count, wb, 2) == 0
    assert rel(small.cpu().numpy(), exact) < 2e-15
    assert rel(small.cpu().numpy(), one.cpu().numpy()) < 2e-15
    # a workspace below one system is refused, not overrun
    bad = torch.from_numpy(P0.copy()).cuda()
    assert lib.gwdbg_screened_refine(bad.data_ptr(), n, count, lib.gwdbg_screened_refine_bytes(n, 1) - 1, 2) != 0


def test_refined_matches_native_fp64_solve():
    naux, nq, ntau = 100, 2, 8
    sysd = system(2, naux, (nq, 1, 1), ntau, 30.0, 5)
    P0 = _p0(nq, ntau, naux, 9)
    out = {}
    for mode in ("tensor", "native"):
        g = gpu(sysd, fp64_gemm=mode)
        g.set("P0_iw", P0)
        g.screened()
        out[mode] = (g.get("P_iw"), g.get("P_tau"))
    assert rel(out["tensor"][0], out["native"][0]) < 1e-14
    assert rel(out["tensor"][1], out["native"][1]) < 1e-13
