"""Pin P1: the oracle's tau <-> Matsubara transforms against exact integrals.

Eq. tau_to_iw applied to a polynomial of degree < ntau has an exact closed
form by repeated integration by parts; it is evaluated here in 80-digit
arithmetic, independently of the oracle's Gauss-Legendre quadrature.
"""
import numpy as np
import pytest

from oracle.grids import Grid, fourier_matrix, lagrange_eval, tau_nodes
from synth import matsubara_indices

mpmath = pytest.importorskip("mpmath")


def _cheb_to_monomial_mp(c):
    """Monomial coefficients (in x) of sum_k c_k T_k(x), exact in mp."""
    n = len(c)
    Tkm1 = [mpmath.mpf(1)]            # T_0
    Tk = [mpmath.mpf(0), mpmath.mpf(1)]  # T_1
    out = [mpmath.mpf(0)] * n
    out[0] += mpmath.mpf(c[0])
    if n > 1:
        for i, t in enumerate(Tk):
            out[i] += mpmath.mpf(c[1]) * t
    for k in range(2, n):
        Tn = [mpmath.mpf(0)] * (k + 1)
        for i, t in enumerate(Tk):
            Tn[i + 1] += 2 * t
        for i, t in enumerate(Tkm1):
            Tn[i] -= t
        for i, t in enumerate(Tn):
            out[i] += mpmath.mpf(c[k]) * t
        Tkm1, Tk = Tk, Tn
    return out


def _exact_fourier(mono, beta, nu):
    """int_0^beta p(tau) e^{i nu tau} dtau with p(x), x = 2 tau/beta - 1 (IBP, exact)."""
    a = mpmath.mpf(nu) * mpmath.mpf(beta) / 2
    deg = len(mono) - 1
    if a == 0:
        s = mpmath.mpf(0)
        for i, c in enumerate(mono):
            s += c * (1 - (-1) ** (i + 1)) / (i + 1)
        return complex(mpmath.mpf(beta) / 2 * s)
    ia = mpmath.mpc(0, a)
    coef = list(mono)
    total = mpmath.mpc(0)
    sign = 1
    for r in range(deg + 1):
        p1 = sum(coef[i] for i in range(len(coef)))
        pm1 = sum(coef[i] * (-1) ** i for i in range(len(coef)))
        total += sign * (p1 * mpmath.expj(a) - pm1 * mpmath.expj(-a)) / ia ** (r + 1)
        coef = [coef[i] * i for i in range(1, len(coef))]
        sign = -sign
        if not coef:
            break
    return complex(mpmath.mpf(beta) / 2 * mpmath.expj(a) * total)


@pytest.mark.parametrize("beta,ntau", [(100.0, 16), (100.0, 32), (1000.0, 24)])
def test_forward_transform_exact_on_polynomials(beta, ntau):
    mpmath.mp.dps = 80
    rng = np.random.default_rng(11)
    fn, bm = matsubara_indices(ntau)
    g = Grid(beta, ntau, fn, bm)
    x = 2 * g.tau / beta - 1
    for trial in range(2):
        c = rng.standard_normal(ntau) * np.exp(-0.1 * np.arange(ntau))
        vals = np.polynomial.chebyshev.chebval(x, c)
        mono = _cheb_to_monomial_mp(c)
        for nu, T in ((g.wf, g.TFf), (g.wb, g.TFb)):
            exact = np.array([_exact_fourier(mono, beta, v) for v in nu])
            got = T @ vals
            scale = np.abs(exact).max()
            assert np.abs(got - exact).max() <= 1e-13 * scale


@pytest.mark.parametrize("ntau", [8, 32, 92, 100])
def test_backward_is_inverse_and_conditioning(ntau):
    fn, bm = matsubara_indices(ntau)
    g = Grid(1000.0, ntau, fn, bm)
    I = np.eye(ntau)
    for TF, TB in ((g.TFf, g.TBf), (g.TFb, g.TBb)):
        c = np.linalg.cond(TF)
        assert c < 5e3
        assert np.abs(TB @ TF - I).max() < 1e-12 * max(1.0, c)
        assert np.abs(TF @ TB - I).max() < 1e-12 * max(1.0, c)


def test_quadrature_converged():
    ntau = 32
    fn, _ = matsubara_indices(ntau)
    nu = (2 * fn + 1) * np.pi / 100.0
    A = fourier_matrix(100.0, ntau, nu)
    B = fourier_matrix(100.0, ntau, nu, npts=2 * (5 * ntau + 200))
    assert np.abs(A - B).max() < 1e-13 * np.abs(B).max()


def test_lagrange_basis_and_endpoints():
    ntau = 20
    j = np.arange(ntau)
    x = -np.cos(np.pi * (2 * j + 1) / (2 * ntau))
    L = lagrange_eval(x, ntau)
    assert np.abs(L - np.eye(ntau)).max() < 1e-13
    # endpoint rows reproduce a polynomial's values at 0 and beta
    rng = np.random.default_rng(3)
    c = rng.standard_normal(ntau)
    fn, bm = matsubara_indices(ntau)
    g = Grid(50.0, ntau, fn, bm)
    vals = np.polynomial.chebyshev.chebval(x, c)
    assert abs(g.lb @ vals - np.polynomial.chebyshev.chebval(1.0, c)) < 1e-12 * np.abs(c).sum()
    assert abs(g.l0 @ vals - np.polynomial.chebyshev.chebval(-1.0, c)) < 1e-12 * np.abs(c).sum()
    assert np.allclose(tau_nodes(50.0, ntau), 25.0 * (1 + x))
    # nodes are symmetric: tau_{n-1-j} = beta - tau_j (used for G(-tau))
    t = tau_nodes(50.0, ntau)
    assert np.abs(t[::-1] - (50.0 - t)).max() < 1e-12


def test_matsubara_index_sets():
    for ntau in (1, 2, 7, 8, 32, 92, 100):
        fn, bm = matsubara_indices(ntau)
        assert len(fn) == ntau and len(bm) == ntau
        assert len(set(fn)) == ntau and len(set(bm)) == ntau
        assert 0 in bm
        if ntau % 2 == 0:
            assert set(fn) == set(-fn - 1)        # symmetric fermionic set


def test_jacobi_anger_matches_quadrature_low_frequencies():
    # two independent evaluations of the same integrals agree where the
    # quadrature is accurate (moderate a)
    from oracle.grids import fourier_matrix_ja, fermionic_a
    ntau = 24
    n = np.arange(-12, 12)
    A = fourier_matrix_ja(30.0, ntau, fermionic_a(n))
    B = fourier_matrix(30.0, ntau, (2 * n + 1) * np.pi / 30.0)
    assert np.abs(A - B).max() < 1e-13 * np.abs(B).max()
