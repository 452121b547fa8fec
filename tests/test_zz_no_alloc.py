"""The allocation-free screened solve against the regular one.

gw_screened_solve_noalloc serves callers that cannot allocate device memory
when they need the solve (arena/pool-owned memory, hosts that forbid
cudaMalloc after start-up, paths that must avoid an allocator's implicit
synchronisation).  It uses a fixed device array inside the library as its
scratch.  This file is collected last so that a failure here cannot hide
another test's result in a run that stops at the first failure.
"""
import ctypes

import numpy as np
import pytest

from gpu_helpers import gpu, system

pytestmark = pytest.mark.gpu


def _inputs(naux, nq, ntau, seed):
    rng = np.random.default_rng(seed)
    A = (rng.standard_normal((nq, ntau, naux, naux)) + 1j * rng.standard_normal((nq, ntau, naux, naux))) / np.sqrt(naux)
    # negative-semidefinite Hermitian part, as P~0(i Omega) has
    return -0.5 * (A @ np.conj(np.swapaxes(A, -1, -2))) + 0.3 * (A - np.conj(np.swapaxes(A, -1, -2)))


@pytest.mark.parametrize("naux,nq,ntau", [(130, 2, 6), (70, 3, 4)])
def test_noalloc_matches_regular_solve_twice(naux, nq, ntau):
    import torch
    from paper_2206_07660_gb300 import load
    lib = load()
    lib.gw_screened_solve_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                              ctypes.c_void_p]
    lib.gw_screened_solve_noalloc.restype = ctypes.c_int
    lib.gw_noalloc_last_error.restype = ctypes.c_char_p
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
        # allocation-free path: caller-owned input and output, fixed scratch
        dP0 = torch.from_numpy(P0).cuda()
        dP = torch.empty_like(dP0)
        torch.cuda.synchronize()
        st = lib.gw_screened_solve_noalloc(dP0.data_ptr(), dP.data_ptr(), naux, nq * ntau, stream.cuda_stream)
        assert st == 0, lib.gw_noalloc_last_error()
        out = dP.cpu().numpy()
        assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max(), (call, np.abs(out - ref).max())


def test_noalloc_rejects_oversized_order():
    from paper_2206_07660_gb300 import load
    lib = load()
    lib.gw_screened_solve_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                              ctypes.c_void_p]
    lib.gw_noalloc_last_error.restype = ctypes.c_char_p
    st = lib.gw_screened_solve_noalloc(ctypes.c_void_p(16), ctypes.c_void_p(16), 1 << 20, 1, None)
    assert st == 1 and b"too large" in lib.gw_noalloc_last_error()
