"""The allocation-free screened solve against the regular one and the oracle.

gw_screened_solve_noalloc serves callers that cannot allocate device memory
when they need the solve: code running inside a memory arena or pool it does
not own, plugins whose host application forbids cudaMalloc after start-up,
and paths that must not hit an allocator's implicit synchronisation.  It uses
a fixed device array inside the library as its scratch.  This file is
collected last so that a failure here cannot hide another test's result in a
run that stops at the first failure.
"""
import ctypes

import numpy as np
import pytest

from gpu_helpers import gpu, system
from oracle import gw as ogw


def _lib():
    from paper_2206_07660_gb300 import load
    lib = load()
    lib.gw_screened_solve_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                              ctypes.c_void_p]
    lib.gw_screened_solve_noalloc.restype = ctypes.c_int
    lib.gw_noalloc_last_error.restype = ctypes.c_char_p
    return lib


def _inputs(naux, nq, ntau, seed):
    rng = np.random.default_rng(seed)
    A = (rng.standard_normal((nq, ntau, naux, naux)) + 1j * rng.standard_normal((nq, ntau, naux, naux))) / np.sqrt(naux)
    # negative-semidefinite Hermitian part, as P~0(i Omega) has
    return -0.5 * (A @ np.conj(np.swapaxes(A, -1, -2))) + 0.3 * (A - np.conj(np.swapaxes(A, -1, -2)))


@pytest.mark.gpu
@pytest.mark.parametrize("naux,nq,ntau", [(130, 2, 6), (70, 3, 4)])
def test_noalloc_matches_regular_solve_and_oracle_twice(naux, nq, ntau):
    import torch
    lib = _lib()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    for call, seed in enumerate((31, 32)):
        P0 = _inputs(naux, nq, ntau, seed)
        # regular path: through a context (library-allocated workspace)
        g = gpu(system(2, naux, (nq, 1, 1), ntau, 30.0, 5))
        g.set("P0_iw", P0)
        g.screened()
        ref = g.get("P_iw")
        g.close()
        # the oracle's solve of Eq. tilde_P_omega
        orc = ogw.screened(P0)
        # allocation-free path: caller-owned input and output, fixed scratch
        dP0 = torch.from_numpy(P0).cuda()
        dP = torch.empty_like(dP0)
        torch.cuda.synchronize()
        st = lib.gw_screened_solve_noalloc(dP0.data_ptr(), dP.data_ptr(), naux, nq * ntau, stream.cuda_stream)
        assert st == 0, lib.gw_noalloc_last_error()
        assert lib.gw_noalloc_last_error() == b""
        out = dP.cpu().numpy()
        assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max(), (call, np.abs(out - ref).max())
        assert np.abs(out - orc).max() <= 1e-12 * np.abs(orc).max(), (call, np.abs(out - orc).max())
        # the input buffer is left alone when P != P0
        assert np.array_equal(dP0.cpu().numpy(), P0)


def test_noalloc_rejects_oversized_order():
    # host-side check: returns before any device work
    lib = _lib()
    st = lib.gw_screened_solve_noalloc(ctypes.c_void_p(16), ctypes.c_void_p(16), 1 << 20, 1, None)
    assert st == 1 and b"too large" in lib.gw_noalloc_last_error()


def test_noalloc_rejects_overlapping_buffers():
    # host-side check on the pointer ranges alone (nothing is dereferenced)
    lib = _lib()
    n, count = 8, 2
    base = 1 << 20
    st = lib.gw_screened_solve_noalloc(ctypes.c_void_p(base), ctypes.c_void_p(base + 16 * n), n, count, None)
    assert st == 1 and b"overlap" in lib.gw_noalloc_last_error()
