"""Several k-points per launch in the 16-bit chains (split-fp16 / split-bf16).

A small system puts kb k-points of one q into each GEMM of the P~0 and Sigma~
chains (batch entries (k, tau)), with whole groups of the P~0 last step at most.
Batching changes which block computes an output tile, not the order of any sum,
so P~0 must come out bit for bit the same at every batch size (cap 3 on an
8-point mesh makes blocks of 3, 3 and 2).  Sigma~'s last step splits its K range
over blocks by the number of tiles and adds the FP64 partials atomically, so its
batch sizes agree to the FP32 rounding of those partials.  All of them must also
match the oracle to the mixed path's accuracy.
"""
import ctypes

import numpy as np
import pytest

from gpu_helpers import gpu, hermitian_noise, rel, system
from oracle import gw as ogw

pytestmark = pytest.mark.gpu


def _cap(lib, cap):
    lib.gwdbg_set_pbatch_cap.argtypes = [ctypes.c_int]
    lib.gwdbg_set_pbatch_cap.restype = ctypes.c_int
    return lib.gwdbg_set_pbatch_cap(cap)


@pytest.mark.parametrize("precision", ["split_f16", "split_bf16"])
def test_batch_sizes_give_identical_bits(precision):
    from paper_2206_07660_gb300 import load
    lib = load()
    nao, naux, kmesh, ntau = 8, 32, (2, 2, 2), 12
    sysd = system(nao, naux, kmesh, ntau, 30.0, 81)
    km = ogw.KMesh(kmesh)
    G = hermitian_noise((ntau, km.nk, nao, nao), 0.2, 82)
    P = hermitian_noise((km.nk, ntau, naux, naux), 0.05, 83)
    refP = ogw.polarization_tau(sysd["V"], G, km)
    refS = ogw.selfenergy_tau(sysd["V"], G, P, km)
    out = {}
    for cap in (1, 3, 0):
        old = _cap(lib, cap)
        try:
            g = gpu(sysd, precision=precision)
        finally:
            _cap(lib, old)
        g.set("G_tau", G)
        g.polarization()
        p0 = g.get("P0_tau")
        g.set("P_tau", P)
        g.selfenergy()
        out[cap] = (p0, g.get("Sigma_tau"))
        g.close()
        tol = 3e-6 if precision == "split_f16" else 3e-4
        assert rel(out[cap][0], refP) < tol
        assert rel(out[cap][1], refS) < tol
    for cap in (3, 0):
        assert np.array_equal(out[cap][0], out[1][0])
        assert rel(out[cap][1], out[1][1]) < 2e-6
