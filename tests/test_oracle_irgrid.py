"""The oracle's GW steps on the IR sparse-sampling grid (oracle.ir.IRGrid) against
closed forms and against the independent Chebyshev representation.

* the non-interacting G(tau) from the Dyson equation on the fermionic sampling
  frequencies, brought back to the sampling times, equals the closed form
  -U diag(e^{-tau (e - mu)} / (1 + e^{-beta (e - mu)})) U^H of the generalized
  eigenproblem H0 U = S U diag(e);
* the tau points are symmetric (tau_{n-1-j} = beta - tau_j), which G(-tau) needs;
* one GW step (Sigma_inf and Sigma~(tau)) on 47 IR points agrees with the same step
  on 128 Chebyshev nodes, interpolated to the IR points, to ~1e-11 — the two
  representations share no code.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import gw as ogw
from oracle.grids import lagrange_eval
from oracle.ir import IRGrid
from synth import make_config_system, matsubara_indices


@pytest.fixture(scope="module")
def c1():
    sysd = make_config_system("C1")
    grid = IRGrid(sysd["beta"], lam=6.0 * sysd["beta"], eps=1e-10)
    return sysd, grid


def test_tau_points_symmetric(c1):
    _, grid = c1
    assert np.abs(grid.tau[::-1] - (grid.beta - grid.tau)).max() < 1e-12 * grid.beta


def test_g0_closed_form(c1):
    sysd, grid = c1
    st = ogw.State(sysd, grid=grid)
    st.dyson()
    beta, mu = grid.beta, st.mu
    for k in range(sysd["H0"].shape[0]):
        e, U = scipy.linalg.eigh(sysd["H0"][k], sysd["S"][k])     # U^H S U = I
        x = e - mu
        occ = np.where(x >= 0, np.exp(-np.outer(grid.tau, x)) / (1 + np.exp(-beta * x)),
                       np.exp(np.outer(beta - grid.tau, x)) / (np.exp(beta * x) + 1))
        G = -np.einsum("ia,ta,ja->tij", U, occ, U.conj())
        assert np.abs(G - st.G_tau[:, k]).max() < 1e-10


def test_gw_step_matches_chebyshev(c1):
    sysd, grid = c1
    st = ogw.State(sysd, grid=grid)
    st.dyson()
    Sinf, Stau, _ = st.sigma()
    nt = 128
    fn, bm = matsubara_indices(nt)
    s2 = dict(sysd)
    s2.update(ntau=nt, fermi_n=fn, bose_m=bm)
    ch = ogw.State(s2)
    ch.dyson()
    Sinf_c, Stau_c, _ = ch.sigma()
    assert abs(st.mu - ch.mu) < 1e-10
    assert np.abs(Sinf - Sinf_c).max() < 1e-10
    L = lagrange_eval(2 * grid.tau / grid.beta - 1, nt)
    assert np.abs(np.einsum("mj,jkab->mkab", L, Stau_c) - Stau).max() < 1e-9


def test_scgw_iterations_match_chebyshev():
    # three damped scGW iterations (mu search, Dyson, Sigma, mixing): the IR grid with
    # 58 points (lambda = 20 beta, covering the spectrum shifted by Sigma) and 192
    # Chebyshev nodes give the same iterates
    sysd = make_config_system("C1")
    beta = sysd["beta"]
    grid = IRGrid(beta, lam=20.0 * beta, eps=1e-10)
    st = ogw.State(sysd, grid=grid, damping=0.5)
    nt = 192
    fn, bm = matsubara_indices(nt)
    s2 = dict(sysd)
    s2.update(ntau=nt, fermi_n=fn, bose_m=bm)
    ch = ogw.State(s2, damping=0.5)
    L = lagrange_eval(2 * grid.tau / beta - 1, nt)
    for _ in range(3):
        st.iterate()
        ch.iterate()
        assert abs(st.mu - ch.mu) < 1e-9
        assert abs(st.N - st.n_elec) < 1e-8
        assert np.abs(np.einsum("mj,jkab->mkab", L, ch.G_tau) - st.G_tau).max() < 1e-9
