"""Oracle: the dynamical part of the GW Luttinger-Ward functional (test infrastructure).

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
use this module; the product path never imports it.

What it computes (Sec. "Thermodynamics", Eqs. Phi_GW and tilde_Phi_GW):

    Phi~ = 1/(2 Nk) sum_q (1/beta) sum_n tr{ ln[I - P~0^q(i Omega_n)] + P~0^q(i Omega_n) }

Readings where the paper leaves the discrete form open:
* The bosonic Matsubara sum runs over every integer n.  It is evaluated with
  the grid's own representation of bosonic functions, as every other
  Matsubara sum of the method is (the density matrix gamma = -G(beta^-) of
  Eq. HF_J is the fermionic case): for F(i Omega_n) = tr{...} above,
  (1/beta) sum_n F(i Omega_n) = F(tau) at tau = 0 = beta (F decays like
  Omega^-4, so its tau form is continuous and periodic), and F(beta^-) is read
  off the interpolant whose transforms at the sampled frequencies are the
  sampled values: sum_j lb_j sum_m TBb[j, m] F(i Omega_m).
* tr ln(I - A) is the sum of the principal logarithms of the eigenvalues of
  I - A.  For a polarization whose Hermitian part is negative semidefinite
  (Eq. P0_tau's sign) every eigenvalue has real part >= 1, so this is the
  branch that is continuous from A = 0.
* Phi~ is real (P~0(-i Omega) = P~0(i Omega)^H); the real part is returned.
  The imaginary part left by an index set that is not symmetric under
  Omega -> -Omega is returned separately for inspection.
"""
import numpy as np

from .gw import to_matsubara


def matsubara_sum_weights(grid):
    """w_m with (1/beta) sum_n F(i Omega_n) = sum_m w_m F(i Omega_m) on the grid:
    w = lb TBb (the interpolant's value at tau = beta^-)."""
    return grid.lb @ grid.TBb


def trace_log_plus(A):
    """tr ln(I - A) + tr A for one square matrix A (principal log of each eigenvalue of I - A)."""
    lam = np.linalg.eigvals(np.eye(A.shape[0]) - A)
    return np.sum(np.log(lam)) + np.trace(A)


def phi_tilde(grid, P0_tau, return_imag=False):
    """Eq. tilde_Phi_GW from P~0^q(tau) [nq][ntau][naux][naux] on the grid.

    Steps in the paper's order: P~0^q(i Omega_m) (Eq. P0t_to_P0w), the trace of
    ln(I - P~0) + P~0 per (q, m), the Matsubara sum, the mean over q with the
    factor 1/2."""
    nq = P0_tau.shape[0]
    P0_iw = to_matsubara(grid.TFb, P0_tau, 1)
    w = matsubara_sum_weights(grid)
    total = 0j
    for q in range(nq):
        for m in range(len(w)):
            total += w[m] * trace_log_plus(P0_iw[q, m])
    phi = total / (2.0 * nq)
    return (phi.real, phi.imag) if return_imag else phi.real
