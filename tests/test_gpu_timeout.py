"""Bounded waits of the tensor-core GEMM: a wait that runs out is reported, not hung.

Every mbarrier wait of the GEMM kernels has an iteration limit.  A test hook
lowers the limit of the pipeline waits to one try, so that the kernel gives up
at its first stage handshake that is not already complete; it must then let
its TMA loads and MMAs in flight finish, free its TMEM, and report the timeout
through the error flag (100 + the role that gave up).  Nothing faults or hangs:
the same process then runs the GEMM again at the normal limit and gets the
exact result, and a GW context maps the flag to GW_ERR_TIMEOUT and stays usable.
"""
import ctypes

import numpy as np
import pytest

from gpu_helpers import gpu, hermitian_noise, system

pytestmark = pytest.mark.gpu

GW_ERR_TIMEOUT = 6


def _lib():
    import torch
    from paper_2206_07660_gb300 import load
    torch.cuda.set_device(0)
    lib = load()
    lib.gwdbg_umma_cgemm_split.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int] * 6 + [ctypes.c_void_p]
    lib.gwdbg_umma_cgemm_split.restype = ctypes.c_int
    for name in ("gwdbg_umma_set_persistent", "gwdbg_umma_force_bn"):
        getattr(lib, name).argtypes = [ctypes.c_int]
        getattr(lib, name).restype = ctypes.c_int
    lib.gwdbg_umma_set_spin.argtypes = [ctypes.c_uint]
    lib.gwdbg_umma_set_spin.restype = ctypes.c_uint
    return lib


@pytest.mark.parametrize("persistent,bn,must_time_out", [(1, 64, True), (1, 224, False), (0, 64, False)])
def test_gemm_wait_limit(persistent, bn, must_time_out):
    import torch
    lib = _lib()
    M, N, K = 4000, 900, 2704
    rng = np.random.default_rng(5)
    A = rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))
    B = rng.standard_normal((N, K)) + 1j * rng.standard_normal((N, K))
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = torch.zeros((M, N), dtype=torch.complex128, device="cuda")
    old_p = lib.gwdbg_umma_set_persistent(persistent)
    old_bn = lib.gwdbg_umma_force_bn(bn)
    try:
        old_spin = lib.gwdbg_umma_set_spin(1)
        try:
            st = lib.gwdbg_umma_cgemm_split(dA.data_ptr(), dB.data_ptr(), M, N, K, 1, 3, 1, dC.data_ptr())
        finally:
            lib.gwdbg_umma_set_spin(old_spin)
        # ping-pong tiles: the second epilogue group's first wait spans a whole
        # K loop of the first tile (507 stages), far beyond one try
        if must_time_out:
            assert 101 <= st <= 104, st
        else:
            assert st == 0 or 101 <= st <= 104, st
        torch.cuda.synchronize()   # the context is intact
        dC.fill_(float("nan"))
        st2 = lib.gwdbg_umma_cgemm_split(dA.data_ptr(), dB.data_ptr(), M, N, K, 1, 3, 1, dC.data_ptr())
    finally:
        lib.gwdbg_umma_force_bn(old_bn)
        lib.gwdbg_umma_set_persistent(old_p)
    assert st2 == 0
    C = dC.cpu().numpy()
    ref = A @ np.conj(B).T
    assert np.abs(C - ref).max() / (np.sqrt(2.0 * K) * 2.0) < 3e-6


def test_context_reports_timeout_and_recovers():
    import torch
    from paper_2206_07660_gb300 import GWError
    lib = _lib()
    nao, naux, kmesh, ntau = 26, 200, (2, 2, 2), 32
    sysd = system(nao, naux, kmesh, ntau, 40.0, 61)
    G = hermitian_noise((ntau, 8, nao, nao), 0.2, 62)
    old_bn = lib.gwdbg_umma_force_bn(64)
    try:
        ref = gpu(sysd, precision="split_tf32")
        ref.set("G_tau", G)
        ref.polarization()
        # gw_polarization writes P~0(tau) and its transform P~0(i Omega) (Eqs.
        # tilde_P0_tau, P0t_to_P0w); those are the quantities to compare
        P_ref = ref.get("P0_tau")
        Pw_ref = ref.get("P0_iw")
        g = gpu(sysd, precision="split_tf32")
        g.set("G_tau", G)
        old_spin = lib.gwdbg_umma_set_spin(1)
        try:
            with pytest.raises(GWError) as e:
                g.polarization()
        finally:
            lib.gwdbg_umma_set_spin(old_spin)
        assert e.value.status == GW_ERR_TIMEOUT
        torch.cuda.synchronize()
        g.polarization()
        P = g.get("P0_tau")
        Pw = g.get("P0_iw")
    finally:
        lib.gwdbg_umma_force_bn(old_bn)
    assert np.abs(P_ref).max() > 0
    assert np.abs(P - P_ref).max() <= 1e-12 * np.abs(P_ref).max()
    assert np.abs(Pw - Pw_ref).max() <= 1e-12 * np.abs(Pw_ref).max()
