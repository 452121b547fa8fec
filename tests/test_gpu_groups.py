"""The last P~0 step of several k-points as one tensor-core GEMM.

With split-TF32 contractions the Z operands and embedded V slabs of a group of
k-points sit side by side along K, and one GEMM per group adds their sum into
P~0^q(tau).  Groups of 1, 2 and all k-points (with a ragged last group) must give
the oracle's P~0 to split-TF32 accuracy and agree with each other to FP32-class
rounding.
"""
import ctypes

import numpy as np
import pytest

from gpu_helpers import gpu, hermitian_noise, rel, system
from oracle import gw as ogw

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("small", ["tensor", "simt"])
def test_pgroup_sizes_agree(small):
    from paper_2206_07660_gb300 import load
    lib = load()
    lib.gwdbg_set_pgroup_cap.argtypes = [ctypes.c_int]
    lib.gwdbg_set_pgroup_cap.restype = ctypes.c_int
    nao, naux, kmesh, ntau = 6, 40, (3, 1, 1), 10
    sysd = system(nao, naux, kmesh, ntau, 40.0, 71)
    km = ogw.KMesh(kmesh)
    G = hermitian_noise((ntau, km.nk, nao, nao), 0.2, 72)
    ref = ogw.polarization_tau(sysd["V"], G, km)
    out = {}
    for cap in (1, 2, 0):
        old = lib.gwdbg_set_pgroup_cap(cap)
        try:
            g = gpu(sysd, precision="split_tf32", small_steps=small)
        finally:
            lib.gwdbg_set_pgroup_cap(old)
        g.set("G_tau", G)
        g.polarization()
        out[cap] = g.get("P0_tau")
        assert rel(out[cap], ref) < 2e-5
    assert rel(out[2], out[1]) < 1e-6
    assert rel(out[0], out[1]) < 1e-6
