"""Oracle: imaginary-time grid and tau <-> Matsubara transforms (test infrastructure).

This module is part of the slow, obviously-correct CPU oracle. Only the test
suite, the smoke check and the CPU-baseline leg of the benchmark may use it;
the product path never imports it.

What it computes (Sec. "Self-consistent finite-temperature GW", Eqs. tau_to_iw
and iw_to_tau; Sec. "Representation on the imaginary axes"):

* tau nodes: first-kind Chebyshev roots mapped to [0, beta], ascending,
  tau_j = (beta/2) (1 - cos(pi (2j+1) / (2 ntau))).  Endpoints are excluded.
* A function of tau is represented by its values at the nodes, i.e. by the
  degree-(ntau-1) interpolating polynomial  f(tau) = sum_j f(tau_j) L_j(tau).
  The Lagrange basis L_j is written through its Chebyshev series,
  L_j(x) = sum_k C[k, j] T_k(x), C[k, j] = (2 - delta_k0)/ntau * T_k(x_j).
* The forward transform is Eq. tau_to_iw applied to that interpolant:
  TF[n, j] = int_0^beta L_j(tau) exp(i nu_n tau) dtau.  With tau = (beta/2)(1+x)
  and a = nu beta / 2 this is (beta/2) e^{i a} sum_k C[k, j] I_k(a), where the
  Chebyshev moments I_k(a) = int_{-1}^{1} T_k(x) e^{i a x} dx are summed from
  the Jacobi-Anger expansion e^{i a x} = sum_m eps_m i^m J_m(a) T_m(x) and the
  exact integrals int T_k T_m dx (Bessel values from scipy.special.jv).  This
  keeps full double accuracy at large a, where a quadrature's node rounding
  is amplified by a.  a = (2n+1) pi/2 for fermions and m pi for bosons, so the
  matrices depend on beta only through the prefactor beta/2; the sampled
  integers n, m are inputs.  A Gauss-Legendre version is kept for checks.
* The backward transform is the exact inverse on the sampled frequencies,
  TB = TF^{-1}: the unique interpolant whose Fourier integrals reproduce the
  sampled values (the discrete stand-in for the Matsubara sum of
  Eq. iw_to_tau; the paper uses IR sparse sampling for the same purpose).
* Endpoint rows lb_j = L_j(beta^-) and l0_j = L_j(0^+), used for the density
  matrix gamma = -G(beta^-).
"""
import numpy as np


def tau_nodes(beta, ntau):
    """Chebyshev first-kind roots on [0, beta], ascending."""
    j = np.arange(ntau)
    return 0.5 * beta * (1.0 - np.cos(np.pi * (2 * j + 1) / (2 * ntau)))


def lagrange_cheb_coeffs(ntau):
    """C[k, j] with L_j(x) = sum_k C[k, j] T_k(x) on x in [-1, 1].

    Discrete orthogonality of T_0..T_{ntau-1} on the ntau first-kind roots.
    """
    j = np.arange(ntau)
    x = -np.cos(np.pi * (2 * j + 1) / (2 * ntau))       # ascending nodes
    k = np.arange(ntau)[:, None]
    T = np.cos(k * np.arccos(np.clip(x, -1.0, 1.0))[None, :])  # T_k(x_j)
    C = (2.0 / ntau) * T
    C[0, :] = 1.0 / ntau
    return C


def lagrange_eval(x, ntau):
    """L[m, j] = L_j(x_m) for points x_m in [-1, 1] (Chebyshev series)."""
    C = lagrange_cheb_coeffs(ntau)
    x = np.asarray(x, dtype=np.float64)
    k = np.arange(ntau)[None, :]
    T = np.cos(k * np.arccos(np.clip(x, -1.0, 1.0))[:, None])  # [m, k]
    return T @ C


def cheb_moments(a, nmom):
    """I[f, k] = int_{-1}^{1} T_k(x) e^{i a_f x} dx, k < nmom (Jacobi-Anger series)."""
    from scipy.special import jv
    a = np.asarray(a, dtype=np.float64)
    out = np.zeros((len(a), nmom), dtype=np.complex128)
    k = np.arange(nmom)
    for f, af in enumerate(a):
        mmax = int(abs(af) + 20 * abs(af) ** (1.0 / 3.0) + 40) + nmom
        m = np.arange(mmax + 1)
        eps = np.where(m == 0, 1.0, 2.0)
        c = eps * (1j ** (m % 4)) * jv(m, af)            # e^{iax} = sum_m c_m T_m(x)
        kk, mm = k[:, None], m[None, :]
        even = ((kk + mm) % 2 == 0)
        with np.errstate(divide="ignore"):
            W = np.where(even, 1.0 / (1.0 - (kk + mm) ** 2.0) + 1.0 / (1.0 - (kk - mm) ** 2.0), 0.0)
        out[f] = W @ c
    return out


def fourier_matrix_ja(beta, ntau, a):
    """TF[n, j] from the half-angle arguments a_n (exact e^{i a} for a = integer * pi/2)."""
    a = np.asarray(a, dtype=np.float64)
    I = cheb_moments(a, ntau)                               # [n, k]
    C = lagrange_cheb_coeffs(ntau)                          # [k, j]
    return (beta / 2.0) * np.exp(1j * a)[:, None] * (I @ C)


def fermionic_a(n):
    """a = w_n beta / 2 = (2n+1) pi / 2."""
    return (2 * np.asarray(n, dtype=np.float64) + 1) * (np.pi / 2)


def bosonic_a(m):
    """a = Omega_m beta / 2 = m pi."""
    return np.asarray(m, dtype=np.float64) * np.pi


def fourier_matrix(beta, ntau, nu, npts=None):
    """Gauss-Legendre evaluation of TF[n, j] = int_0^beta L_j(tau) exp(i nu_n tau) dtau.

    With tau = (beta/2)(1+x):  TF = (beta/2) e^{i a} int_{-1}^{1} L_j(x) e^{i a x} dx,
    a = nu beta / 2.  Gauss-Legendre with npts points; the default is large
    enough for the oscillation a and the polynomial degree ntau-1.
    """
    nu = np.asarray(nu, dtype=np.float64)
    a = nu * beta / 2.0
    if npts is None:
        npts = int(5 * ntau + np.max(np.abs(a)) + 32)
    x, w = np.polynomial.legendre.leggauss(npts)
    L = lagrange_eval(x, ntau)                               # [m, j]
    E = np.exp(1j * a[:, None] * x[None, :]) * w[None, :]    # [n, m]
    return (beta / 2.0) * np.exp(1j * a)[:, None] * (E @ L)


def fermionic_freqs(beta, n):
    return (2 * np.asarray(n, dtype=np.float64) + 1) * np.pi / beta


def bosonic_freqs(beta, m):
    return 2 * np.asarray(m, dtype=np.float64) * np.pi / beta


class Grid:
    """All discrete transform data for one (beta, ntau, index sets)."""

    def __init__(self, beta, ntau, fermi_n, bose_m):
        self.beta = float(beta)
        self.ntau = int(ntau)
        self.fermi_n = np.asarray(fermi_n, dtype=np.int64)
        self.bose_m = np.asarray(bose_m, dtype=np.int64)
        assert self.fermi_n.shape == (ntau,) and self.bose_m.shape == (ntau,)
        self.tau = tau_nodes(beta, ntau)
        self.wf = fermionic_freqs(beta, self.fermi_n)
        self.wb = bosonic_freqs(beta, self.bose_m)
        self.TFf = fourier_matrix_ja(beta, ntau, fermionic_a(self.fermi_n))
        self.TFb = fourier_matrix_ja(beta, ntau, bosonic_a(self.bose_m))
        self.TBf = np.linalg.inv(self.TFf)
        self.TBb = np.linalg.inv(self.TFb)
        ends = lagrange_eval(np.array([-1.0, 1.0]), ntau)
        self.l0 = ends[0]          # L_j(0+)
        self.lb = ends[1]          # L_j(beta-)
        # weights of the density: gamma = -sum_j lb_j G(tau_j) = -sum_n r_n G(i w_n)
        self.r = self.lb @ self.TBf
