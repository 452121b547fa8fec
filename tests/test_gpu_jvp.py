"""GPU parity of the tangent chains (gw_polarization_jvp, gw_screened_jvp,
gw_selfenergy_jvp) against central differences of the FP64 oracle.

P~0 is a quadratic form in G and Sigma~ is bilinear in (G, P~), so their
central differences are exact up to rounding: the tangents must match to
~1e-10.  The screened block is a matrix inverse between two linear
transforms; its central difference carries an O(h^2) error, bounded here
by comparing two step sizes.
"""
import numpy as np
import pytest

from gpu_helpers import gpu, hermitian_noise, rel, system
from oracle import gw as ogw

pytestmark = pytest.mark.gpu

CASES = [(3, 5, (3, 1, 1), 6), (6, 20, (2, 2, 1), 10), (4, 40, (2, 1, 1), 8)]


def _noise(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("nao,naux,kmesh,ntau", CASES)
def test_polarization_jvp(nao, naux, kmesh, ntau):
    import torch
    sysd = system(nao, naux, kmesh, ntau, 40.0, 41)
    km = ogw.KMesh(kmesh)
    G = hermitian_noise((ntau, km.nk, nao, nao), 0.2, 1)
    dG = _noise(G.shape, 2)
    h = 1e-3
    ref = (ogw.polarization_tau(sysd["V"], G + h * dG, km) - ogw.polarization_tau(sysd["V"], G - h * dG, km)) / (2 * h)
    g = gpu(sysd)
    g.set("G_tau", G)
    got = g.polarization_jvp(torch.from_numpy(dG).cuda()).cpu().numpy()
    assert rel(got, ref) < 1e-10


@pytest.mark.parametrize("nao,naux,kmesh,ntau", CASES)
def test_selfenergy_jvp(nao, naux, kmesh, ntau):
    import torch
    sysd = system(nao, naux, kmesh, ntau, 40.0, 43)
    km = ogw.KMesh(kmesh)
    G = hermitian_noise((ntau, km.nk, nao, nao), 0.2, 3)
    P = hermitian_noise((km.nk, ntau, naux, naux), 0.2, 4)
    dG, dP = _noise(G.shape, 5), _noise(P.shape, 6)
    h = 1e-3
    V = sysd["V"]
    ref = (ogw.selfenergy_tau(V, G + h * dG, P + h * dP, km) - ogw.selfenergy_tau(V, G - h * dG, P - h * dP, km)) / (2 * h)
    g = gpu(sysd)
    g.set("G_tau", G)
    g.set("P_tau", P)
    got = g.selfenergy_jvp(torch.from_numpy(dG).cuda(), torch.from_numpy(dP).cuda()).cpu().numpy()
    assert rel(got, ref) < 1e-10


@pytest.mark.parametrize("nao,naux,kmesh,ntau", CASES)
def test_screened_jvp(nao, naux, kmesh, ntau):
    import torch
    sysd = system(nao, naux, kmesh, ntau, 40.0, 47)
    st = ogw.State(sysd)
    st.dyson()
    grid = st.grid
    P0 = ogw.polarization_tau(sysd["V"], st.G_tau, st.km)
    dP0 = _noise(P0.shape, 7) * np.abs(P0).max()

    def screened_tau(X):
        return ogw.herm(ogw.to_matsubara(grid.TBb, ogw.screened(ogw.to_matsubara(grid.TFb, X, 1)), 1))

    fd = {}
    for h in (1e-4, 5e-5):
        fd[h] = (screened_tau(P0 + h * dP0) - screened_tau(P0 - h * dP0)) / (2 * h)
    # the O(h^2) error of the smaller step, estimated from the two steps
    err_fd = np.abs(fd[5e-5] - fd[1e-4]).max() / 3.0
    g = gpu(sysd)
    g.set("G_tau", st.G_tau)
    g.polarization()
    g.screened()
    got = g.screened_jvp(torch.from_numpy(dP0).cuda()).cpu().numpy()
    scale = np.abs(fd[5e-5]).max()
    assert np.abs(got - fd[5e-5]).max() <= 4 * err_fd + 1e-10 * scale


@pytest.mark.parametrize("precision", ["fp32", "split_tf32"])
def test_mixed_precision_tangents(precision):
    # the tangents run the forward chains of the context's precision: complex64-level
    # agreement with the oracle's central differences
    import torch
    nao, naux, kmesh, ntau = 6, 20, (2, 2, 1), 10
    sysd = system(nao, naux, kmesh, ntau, 40.0, 53)
    km = ogw.KMesh(kmesh)
    G = hermitian_noise((ntau, km.nk, nao, nao), 0.2, 8)
    P = hermitian_noise((km.nk, ntau, naux, naux), 0.2, 9)
    dG, dP = _noise(G.shape, 10), _noise(P.shape, 11)
    h = 1e-3
    V = sysd["V"]
    refP = (ogw.polarization_tau(V, G + h * dG, km) - ogw.polarization_tau(V, G - h * dG, km)) / (2 * h)
    refS = (ogw.selfenergy_tau(V, G + h * dG, P + h * dP, km) - ogw.selfenergy_tau(V, G - h * dG, P - h * dP, km)) / (2 * h)
    g = gpu(sysd, precision=precision)
    g.set("G_tau", G)
    g.set("P_tau", P)
    gotP = g.polarization_jvp(torch.from_numpy(dG).cuda()).cpu().numpy()
    gotS = g.selfenergy_jvp(torch.from_numpy(dG).cuda(), torch.from_numpy(dP).cuda()).cpu().numpy()
    assert rel(gotP, refP) < 2e-5
    assert rel(gotS, refS) < 2e-5
