"""GPU parity of the adjoint chains (gw_polarization_vjp, gw_selfenergy_vjp)
against the oracle's torch-autograd gradients (themselves pinned by finite
differences in test_oracle_adjoint.py), and the autograd.Function wrappers."""
import numpy as np
import pytest

from gpu_helpers import gpu, hermitian_noise, rel, system
from oracle import adjoint as oad
from oracle import gw as ogw

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nao,naux,kmesh,ntau", [(3, 5, (3, 1, 1), 6), (8, 20, (2, 2, 1), 10), (5, 70, (2, 1, 1), 8)])
@pytest.mark.parametrize("precision", ["fp64", "split_tf32"])
def test_polarization_vjp(nao, naux, kmesh, ntau, precision):
    import torch
    sysd = system(nao, naux, kmesh, ntau, 40.0, 31)
    rng = np.random.default_rng(2)
    km = ogw.KMesh(kmesh)
    G = hermitian_noise((ntau, km.nk, nao, nao), 0.2, 3)
    Pbar = rng.standard_normal((km.nk, ntau, naux, naux)) + 1j * rng.standard_normal((km.nk, ntau, naux, naux))
    ref = oad.polarization_vjp(sysd["V"], G, km, Pbar)
    g = gpu(sysd, precision=precision)
    g.set("G_tau", G)
    got = g.polarization_vjp(torch.from_numpy(Pbar).cuda()).cpu().numpy()
    assert rel(got, ref) < 1e-12


@pytest.mark.parametrize("nao,naux,kmesh,ntau", [(3, 5, (3, 1, 1), 6), (8, 20, (2, 2, 1), 10), (5, 70, (2, 1, 1), 8)])
def test_selfenergy_vjp(nao, naux, kmesh, ntau):
    import torch
    sysd = system(nao, naux, kmesh, ntau, 40.0, 33)
    rng = np.random.default_rng(4)
    km = ogw.KMesh(kmesh)
    G = hermitian_noise((ntau, km.nk, nao, nao), 0.2, 5)
    P = hermitian_noise((km.nk, ntau, naux, naux), 0.2, 6)
    Sbar = rng.standard_normal((ntau, km.nk, nao, nao)) + 1j * rng.standard_normal((ntau, km.nk, nao, nao))
    rG, rP = oad.selfenergy_vjp(sysd["V"], G, P, km, Sbar)
    g = gpu(sysd)
    g.set("G_tau", G)
    g.set("P_tau", P)
    gG, gP = g.selfenergy_vjp(torch.from_numpy(Sbar).cuda())
    assert rel(gG.cpu().numpy(), rG) < 1e-12
    assert rel(gP.cpu().numpy(), rP) < 1e-12


def test_autograd_functions():
    import torch
    from paper_2206_07660_gb300.autograd import Polarization, SelfEnergy
    nao, naux, kmesh, ntau = 4, 9, (2, 1, 1), 8
    sysd = system(nao, naux, kmesh, ntau, 40.0, 35)
    km = ogw.KMesh(kmesh)
    rng = np.random.default_rng(7)
    G = hermitian_noise((ntau, km.nk, nao, nao), 0.2, 8)
    P = hermitian_noise((km.nk, ntau, naux, naux), 0.2, 9)
    W1 = rng.standard_normal((km.nk, ntau, naux, naux)) + 1j * rng.standard_normal((km.nk, ntau, naux, naux))
    W2 = rng.standard_normal((ntau, km.nk, nao, nao)) + 1j * rng.standard_normal((ntau, km.nk, nao, nao))
    g = gpu(sysd, damping=1.0)
    Gt = torch.from_numpy(G).cuda().requires_grad_(True)
    Pt = torch.from_numpy(P).cuda().requires_grad_(True)
    L = (torch.from_numpy(W1).cuda().conj() * Polarization.apply(Gt, g)).real.sum() + \
        (torch.from_numpy(W2).cuda().conj() * SelfEnergy.apply(Gt, Pt, g)).real.sum()
    L.backward()
    gG1 = oad.polarization_vjp(sysd["V"], G, km, W1)
    gG2, gP2 = oad.selfenergy_vjp(sysd["V"], G, P, km, W2)
    assert rel(Gt.grad.cpu().numpy(), gG1 + gG2) < 1e-12
    assert rel(Pt.grad.cpu().numpy(), gP2) < 1e-12


@pytest.mark.parametrize("nao,naux,kmesh,ntau", [(3, 5, (3, 1, 1), 6), (8, 20, (2, 2, 1), 10), (5, 70, (2, 1, 1), 8)])
def test_vjps_complex64(nao, naux, kmesh, ntau):
    # complex64 adjoint chains against the complex128 oracle gradient (the reading of
    # the complex64 gradient check: compare with the complex128 analytic gradient)
    import torch
    sysd = system(nao, naux, kmesh, ntau, 40.0, 37)
    rng = np.random.default_rng(11)
    km = ogw.KMesh(kmesh)
    G = hermitian_noise((ntau, km.nk, nao, nao), 0.2, 12)
    P = hermitian_noise((km.nk, ntau, naux, naux), 0.2, 13)
    Pbar = rng.standard_normal((km.nk, ntau, naux, naux)) + 1j * rng.standard_normal((km.nk, ntau, naux, naux))
    Sbar = rng.standard_normal((ntau, km.nk, nao, nao)) + 1j * rng.standard_normal((ntau, km.nk, nao, nao))
    g = gpu(sysd)
    g.set("G_tau", G)
    g.set("P_tau", P)
    got = g.polarization_vjp(torch.from_numpy(Pbar).cuda(), c64=True).cpu().numpy()
    assert rel(got, oad.polarization_vjp(sysd["V"], G, km, Pbar)) < 2e-6
    gG, gP = g.selfenergy_vjp(torch.from_numpy(Sbar).cuda(), c64=True)
    rG, rP = oad.selfenergy_vjp(sysd["V"], G, P, km, Sbar)
    assert rel(gG.cpu().numpy(), rG) < 2e-6
    assert rel(gP.cpu().numpy(), rP) < 2e-6


def test_vjp_complex64_against_finite_differences():
    # coarse central differences of the GPU's own forward map at step 1e-3 (Eq. tilde_P0_tau):
    # d/de Re<W, P(G + e D)> = Re<Gbar, D> for the cotangent W
    import torch
    nao, naux, kmesh, ntau = 4, 9, (2, 1, 1), 8
    sysd = system(nao, naux, kmesh, ntau, 40.0, 39)
    km = ogw.KMesh(kmesh)
    rng = np.random.default_rng(14)
    G = hermitian_noise((ntau, km.nk, nao, nao), 0.2, 15)
    W = rng.standard_normal((km.nk, ntau, naux, naux)) + 1j * rng.standard_normal((km.nk, ntau, naux, naux))
    g = gpu(sysd)
    g.set("G_tau", G)
    Gbar = g.polarization_vjp(torch.from_numpy(W).cuda(), c64=True).cpu().numpy()
    for seed in (16, 17, 18):
        D = hermitian_noise(G.shape, 1.0, seed)

        def f(eps):
            g.set("G_tau", G + eps * D)
            g.polarization()
            return float(np.real(np.vdot(W, g.get("P0_tau"))))
        h = 1e-3
        fd = (f(h) - f(-h)) / (2 * h)
        an = float(np.real(np.vdot(Gbar, D)))
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (seed, fd, an)
