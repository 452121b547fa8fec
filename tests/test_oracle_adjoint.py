"""Pin P8 of the oracle's gradients: the torch restatement reproduces the NumPy
oracle's forward maps, and its autograd gradients match central finite
differences of L = Re sum conj(W) f (step 1e-6, complex128)."""
import numpy as np
import pytest

from oracle import adjoint as oad
from oracle import gw as ogw
from synth import make_system

torch = pytest.importorskip("torch")


def _setup(seed=3):
    sysd = make_system(3, 4, (3, 1, 1), seed)
    km = ogw.KMesh((3, 1, 1))
    rng = np.random.default_rng(seed)
    ntau = 6
    G = (rng.standard_normal((ntau, 3, 3, 3)) + 1j * rng.standard_normal((ntau, 3, 3, 3))) * 0.3
    P = (rng.standard_normal((3, ntau, 4, 4)) + 1j * rng.standard_normal((3, ntau, 4, 4))) * 0.3
    return sysd["V"], G, P, km, rng


def test_torch_restatement_matches_numpy_oracle():
    V, G, P, km, _ = _setup()
    assert np.abs(oad.forward_numpy(V, G, km) - ogw.polarization_tau(V, G, km)).max() < 1e-13
    assert np.abs(oad.selfenergy_numpy(V, G, P, km) - ogw.selfenergy_tau(V, G, P, km)).max() < 1e-13


def _fd_check(f, x, W, grad, rng, n=6, h=1e-6):
    """Central differences of L(x) = Re sum conj(W) f(x) at n random entries."""
    flat = x.reshape(-1)
    for _ in range(n):
        i = int(rng.integers(flat.size))
        d = np.zeros_like(flat)
        fd = 0j
        for unit in (1.0, 1j):
            d[:] = 0
            d[i] = h * unit
            Lp = np.real(np.vdot(W, f((flat + d).reshape(x.shape))))
            Lm = np.real(np.vdot(W, f((flat - d).reshape(x.shape))))
            fd += unit * (Lp - Lm) / (2 * h)
        assert abs(fd - grad.reshape(-1)[i]) < 1e-7 * max(1.0, abs(fd)), (i, fd, grad.reshape(-1)[i])


def test_polarization_gradient_finite_differences():
    V, G, P, km, rng = _setup(4)
    Pout = ogw.polarization_tau(V, G, km)
    W = rng.standard_normal(Pout.shape) + 1j * rng.standard_normal(Pout.shape)
    gG = oad.polarization_vjp(V, G, km, W)
    _fd_check(lambda g: ogw.polarization_tau(V, g, km), G, W, gG, rng)


def test_selfenergy_gradient_finite_differences():
    V, G, P, km, rng = _setup(5)
    Sout = ogw.selfenergy_tau(V, G, P, km)
    W = rng.standard_normal(Sout.shape) + 1j * rng.standard_normal(Sout.shape)
    gG, gP = oad.selfenergy_vjp(V, G, P, km, W)
    _fd_check(lambda g: ogw.selfenergy_tau(V, g, P, km), G, W, gG, rng)
    _fd_check(lambda p: ogw.selfenergy_tau(V, G, p, km), P, W, gP, rng)
