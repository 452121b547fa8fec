"""Shared helpers of the GPU parity tests: one synthetic system fed to both
the CUDA library (through its C ABI) and the CPU oracle."""
import numpy as np

from synth import make_system, matsubara_indices


def system(nao, naux, kmesh, ntau, beta, seed, trs=False, n_elec=None):
    sysd = make_system(nao, naux, kmesh, seed, trs=trs)
    fn, bm = matsubara_indices(ntau)
    sysd.update(beta=float(beta), ntau=int(ntau), fermi_n=fn, bose_m=bm,
                n_elec=float(nao if n_elec is None else n_elec))
    return sysd


def gpu(sysd, **kw):
    import torch
    from paper_2206_07660_gb300 import GW
    torch.cuda.set_device(0)
    return GW(sysd["H0"], sysd["S"], sysd["V"], sysd["kmesh"], sysd["ntau"], sysd["beta"],
              sysd["fermi_n"], sysd["bose_m"], n_elec=sysd["n_elec"], **kw)


def oracle_state(sysd, **kw):
    from oracle import gw as ogw
    return ogw.State(sysd, **kw)


def rel(a, b):
    return float(np.abs(a - b).max() / max(1e-300, np.abs(b).max()))


def hermitian_noise(shape, scale, seed):
    """Seeded Hermitian perturbation over the last two axes."""
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * scale
    return 0.5 * (X + np.conj(np.swapaxes(X, -1, -2)))
