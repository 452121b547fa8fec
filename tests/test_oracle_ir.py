"""Pins of the oracle's IR basis (Sec. "Representation on the imaginary axes"):
the project's own singular value expansion of the fermionic and bosonic kernels,
with sparse sampling on tau and Matsubara points.

* the basis is orthonormal on [0, beta] and has the kernel's parity;
* the truncated expansion reproduces the kernel to the cutoff;
* the closed-form Fourier transforms of the basis functions agree with brute-force
  quadrature at small frequencies;
* a single pole, whose tau and Matsubara forms are known in closed form, is carried
  from one axis to the other by the sampling transforms to ~eps times the sampling
  matrices' condition numbers;
* the sizes: L grows slowly with lambda (the paper: 10-200 coefficients), and each
  axis has at least L well-conditioned sampling points.
"""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle.ir import IRBasis, kernel


def _pole_tau(tau, e, beta, stat):
    """-e^{-tau e} / (1 + e^{-beta e}) (fermions) or / (1 - e^{-beta e}) (bosons)."""
    if stat == "F":
        return -np.exp(-tau * e) / (1 + np.exp(-beta * e)) if e >= 0 else -np.exp((beta - tau) * e) / (np.exp(beta * e) + 1)
    return -np.exp(-tau * e) / (-np.expm1(-beta * e)) if e > 0 else np.exp((beta - tau) * e) / (-np.expm1(beta * e))


def _fine_tau_quadrature(b, n=80):
    xs, ws = npleg.leggauss(n)
    br = np.concatenate([-b.breaks[::-1], b.breaks[1:]])   # the basis' segments on [0, 1], mirrored
    seg = list(zip(br[:-1], br[1:]))
    x = np.concatenate([0.5 * (xs + 1) * (hi - lo) + lo for lo, hi in seg])
    w = np.concatenate([0.5 * ws * (hi - lo) for lo, hi in seg])
    return 0.5 * b.beta * (x + 1), 0.5 * b.beta * w


@pytest.mark.parametrize("stat", ["F", "B"])
@pytest.mark.parametrize("lam,beta", [(100.0, 10.0), (1000.0, 100.0)])
def test_orthonormal_and_parity(stat, lam, beta):
    b = IRBasis(lam, beta, stat, eps=1e-8)
    tau, w = _fine_tau_quadrature(b)
    U = b.u(tau)
    assert np.abs((U * w[:, None]).T @ U - np.eye(b.size)).max() < 1e-12
    # each parity sector is its own SVD: u_l(-x) = parity_l u_l(x) exactly, and the
    # parities alternate with l as the kernel's total positivity requires
    x = np.linspace(-0.999, 0.999, 101)
    assert np.array_equal(b._u_x(-x), b._u_x(x) * b.parity[None, :])
    assert np.array_equal(b.parity, (-1) ** np.arange(b.size))


@pytest.mark.parametrize("stat", ["F", "B"])
def test_kernel_reconstruction(stat):
    lam, eps = 300.0, 1e-8
    b = IRBasis(lam, 30.0, stat, eps=eps)
    rng = np.random.default_rng(4)
    x = rng.uniform(-1, 1, 40)
    iy = rng.choice(b.y_nodes.size, 40, replace=False)
    for sgn in (1.0, -1.0):       # v_l(-y) = parity_l v_l(y)
        K = kernel(lam, x, sgn * b.y_nodes[iy], stat)
        v = b.v_nodes[iy] * np.where(sgn < 0, b.parity, 1.0)[None, :]
        approx = (b._u_x(x) * b.s[None, :]) @ v.T
        assert np.abs(K - approx).max() < 10 * eps * b.s[0]


@pytest.mark.parametrize("stat", ["F", "B"])
def test_fourier_transform_closed_form(stat):
    b = IRBasis(200.0, 20.0, stat, eps=1e-8)
    n = np.arange(-6, 7)
    tau, w = _fine_tau_quadrature(b, 120)
    brute = (np.exp(1j * np.outer(b.freq(n), tau)) * w[None, :]) @ b.u(tau)
    assert np.abs(b.uhat(n) - brute).max() < 1e-12 * np.abs(brute).max()


@pytest.mark.parametrize("stat", ["F", "B"])
@pytest.mark.parametrize("lam,beta,eps", [(100.0, 10.0, 1e-8), (1000.0, 100.0, 1e-8), (1000.0, 100.0, 1e-10)])
def test_pole_through_sparse_sampling(stat, lam, beta, eps):
    b = IRBasis(lam, beta, stat, eps=eps)
    tp, npts, TF, TB = b.transforms()
    assert len(tp) >= b.size and len(npts) >= b.size
    ct, cw = np.linalg.cond(b.u(tp)), np.linalg.cond(b.uhat(npts))
    assert ct < 1e3 and cw < 1e3
    wmax = lam / beta
    for e in (-0.9 * wmax, -0.3 * wmax, 0.01 * wmax, 0.5 * wmax, wmax):
        g = _pole_tau(tp, e, beta, stat)
        ex = 1.0 / (1j * b.freq(npts) - e)
        assert np.abs(TF @ g - ex).max() <= 100 * eps * np.abs(ex).max()
        assert np.abs(TB @ ex - g).max() <= 100 * eps * np.abs(g).max()


def test_basis_sizes():
    sizes = [IRBasis(lam, 1.0, "F", eps=1e-8).size for lam in (10.0, 100.0, 1000.0)]
    assert sizes[0] < sizes[1] < sizes[2] <= 60
    assert 10 <= sizes[0]
