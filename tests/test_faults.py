"""Failure paths of gw_init injected on the host, without a GPU.

A device allocator that returns NULL (at the first request, or after some
requests succeeded) must make gw_init return GW_ERR_OOM with no context, and
every allocation that did succeed must be given back exactly once.  Nothing
here touches device memory: the allocator hands out fake addresses and the
failure is reported before any copy is issued.
"""
import ctypes

import numpy as np
import pytest

from synth import matsubara_indices

GW_ERR_OOM = 3


@pytest.fixture(scope="module")
def lib():
    from paper_2206_07660_gb300 import build as b
    b.build()
    from paper_2206_07660_gb300 import load
    return load()


def _config(fail_after, log, precision=0):
    from paper_2206_07660_gb300.gw import ALLOC_FN, FREE_FN, GwConfig
    nao, naux, ntau = 4, 6, 8
    fn, bm = matsubara_indices(ntau)
    cfg = GwConfig()
    cfg.nao, cfg.naux, cfg.ntau = nao, naux, ntau
    for i, n in enumerate((2, 1, 1)):
        cfg.kmesh[i] = n
    cfg.beta, cfg.n_elec, cfg.mu_tol, cfg.mu_maxit, cfg.damping = 10.0, float(nao), 1e-9, 50, 0.5
    cfg.contract_prec, cfg.spin_factor = precision, 2
    keep = [np.ascontiguousarray(fn, dtype=np.int32), np.ascontiguousarray(bm, dtype=np.int32)]
    cfg.fermi_n = keep[0].ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    cfg.bose_m = keep[1].ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    state = {"next": 1 << 20}

    def alloc(user, nbytes):
        if len(log["alloc"]) >= fail_after:
            log["refused"] += 1
            return None
        p = state["next"]
        state["next"] += (int(nbytes) + 255) // 256 * 256
        log["alloc"].append(p)
        return p

    def free(user, p):
        log["free"].append(int(p))

    cb = (ALLOC_FN(alloc), FREE_FN(free))
    cfg.dev_alloc, cfg.dev_free = cb
    return cfg, (keep, cb, state)


@pytest.mark.parametrize("fail_after", [0, 1, 7, 25])
@pytest.mark.parametrize("precision", [0, 3])
def test_allocator_failure_returns_oom_and_frees_everything(lib, fail_after, precision):
    log = {"alloc": [], "free": [], "refused": 0}
    cfg, keep = _config(fail_after, log, precision)
    dummy = np.zeros(4096)
    out = ctypes.c_void_p()
    st = lib.gw_init(ctypes.byref(cfg), dummy.ctypes.data, dummy.ctypes.data, dummy.ctypes.data, ctypes.byref(out))
    assert st == GW_ERR_OOM, (st, lib.gw_last_error(None))
    assert not out.value
    assert b"allocation" in lib.gw_last_error(None)
    assert log["refused"] >= 1
    assert sorted(log["free"]) == sorted(log["alloc"])     # every granted block returned once
