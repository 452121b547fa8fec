"""Pins P2-P7 of the oracle against closed forms, brute force and invariants.

Each case is chosen so that a plausible slip in the oracle (a dropped spin
factor, a wrong sign, G(tau) and G(-tau) swapped, a transposed V, a missed
k+q / k-q) fails at least one of them; tests/test_oracle_mutations.py plants
such slips and checks that they are caught.
"""
import numpy as np
import pytest

from oracle import closed_forms as cf
from oracle import gw as ogw
from oracle.brute import hf_4idx, selfenergy_tau_4idx
from oracle.grids import Grid
from synth import make_config_system, make_system, matsubara_indices


def small_state(nao=4, naux=12, kmesh=(2, 1, 1), beta=10.0, ntau=64, seed=5, trs=False, n_elec=None):
    sysd = make_system(nao, naux, kmesh, seed, trs=trs)
    fn, bm = matsubara_indices(ntau)
    sysd.update(beta=beta, ntau=ntau, fermi_n=fn, bose_m=bm, n_elec=float(n_elec or nao))
    return ogw.State(sysd)


# ------------------------------------------------------------------ P2
def test_p2_discrete_dyson_matches_closed_form_g0():
    st = small_state()
    st.dyson()
    eps, C = cf.bands(st.H0, st.S)
    mu_exact = cf.mu0(st.grid.beta, eps, st.n_elec)
    G0 = cf.g0_tau(st.grid.beta, st.grid.tau, eps, C, st.mu)
    assert abs(st.mu - mu_exact) < 1e-9
    assert np.abs(G0 - st.G_tau).max() < 1e-10
    assert abs(st.N - st.n_elec) <= 1e-9


# ------------------------------------------------------------------ P3
@pytest.mark.parametrize("trs", [False, True])
def test_p3_noninteracting_p0_at_nodes(trs):
    st = small_state(nao=4, naux=10, kmesh=(3, 1, 1), beta=100.0, ntau=32, trs=trs)
    eps, C = cf.bands(st.H0, st.S)
    mu = cf.mu0(st.grid.beta, eps, st.n_elec)
    G0 = cf.g0_tau(st.grid.beta, st.grid.tau, eps, C, mu)
    P = ogw.polarization_tau(st.V, G0, st.km, symmetrize=False)
    Pc = cf.p0_tau_closed(st.grid.beta, st.grid.tau, eps, C, mu, st.V, st.km)
    assert np.abs(P - Pc).max() < 1e-13 * max(1.0, np.abs(Pc).max())


def test_p3_lindhard_through_bosonic_transform():
    # beta small enough that the node interpolant is converged: the discrete
    # transform then reproduces the Lindhard form to near roundoff.
    st = small_state(nao=3, naux=8, kmesh=(2, 1, 1), beta=5.0, ntau=64)
    eps, C = cf.bands(st.H0, st.S)
    mu = cf.mu0(st.grid.beta, eps, st.n_elec)
    Pc = cf.p0_tau_closed(st.grid.beta, st.grid.tau, eps, C, mu, st.V, st.km)
    Piw = ogw.to_matsubara(st.grid.TFb, Pc, 1)
    Pl = cf.p0_iw_closed(st.grid.beta, st.grid.wb, eps, C, mu, st.V, st.km)
    assert np.abs(Piw - Pl).max() < 1e-10 * np.abs(Pl).max()


# ------------------------------------------------------------------ P4
@pytest.mark.parametrize("trs", [False, True])
def test_p4_density_fitted_equals_four_index_c1(trs):
    sysd = make_config_system("C1", trs=trs)
    st = ogw.State(sysd)
    st.dyson()
    st.sigma(symmetrize_p=False)
    S_df = ogw.selfenergy_tau(st.V, st.G_tau, st.P_tau, st.km, symmetrize=False)
    S_4 = selfenergy_tau_4idx(st.V, st.G_tau, st.grid, st.km)
    assert np.abs(S_df - S_4).max() < 1e-12


@pytest.mark.parametrize("kmesh,nao,naux", [((3, 1, 1), 2, 5), ((2, 2, 1), 3, 4), ((1, 1, 1), 3, 7)])
def test_p4_tiny_variants(kmesh, nao, naux):
    st = small_state(nao=nao, naux=naux, kmesh=kmesh, beta=30.0, ntau=12, seed=17)
    st.dyson()
    # perturb G off its equilibrium value (non-Hermitian part included) so the
    # check does not lean on any symmetry of the equilibrium G
    rng = np.random.default_rng(1)
    G = st.G_tau + 0.05 * (rng.standard_normal(st.G_tau.shape) + 1j * rng.standard_normal(st.G_tau.shape))
    P0 = ogw.polarization_tau(st.V, G, st.km, symmetrize=False)
    P = ogw.to_matsubara(st.grid.TBb, ogw.screened(ogw.to_matsubara(st.grid.TFb, P0, 1)), 1)
    S_df = ogw.selfenergy_tau(st.V, G, P, st.km, symmetrize=False)
    S_4 = selfenergy_tau_4idx(st.V, G, st.grid, st.km)
    assert np.abs(S_df - S_4).max() < 1e-12 * max(1.0, np.abs(S_4).max())


# ------------------------------------------------------------------ P5
def test_p5_hf_matches_four_index():
    st = small_state(nao=4, naux=9, kmesh=(2, 2, 1), beta=20.0, ntau=16)
    st.dyson()
    gamma = ogw.density_matrix(st.grid, st.G_tau)
    J = ogw.hartree(st.V, gamma)
    K = ogw.exchange(st.V, gamma)
    J4, K4 = hf_4idx(st.V, gamma)
    assert np.abs(J - J4).max() < 1e-13 and np.abs(K - K4).max() < 1e-13
    # J, K Hermitian for Hermitian gamma
    assert np.abs(J - np.conj(np.swapaxes(J, 1, 2))).max() < 1e-13


# ------------------------------------------------------------------ P6
@pytest.mark.parametrize("eps,v,beta", [(0.3, 0.7, 10.0), (0.02, 1.1, 50.0)])
def test_p6_single_orbital_model(eps, v, beta):
    ntau = 16
    fn, bm = matsubara_indices(ntau)
    grid = Grid(beta, ntau, fn, bm)
    km = ogw.KMesh((1, 1, 1))
    mu = 0.05
    cl = cf.single_orbital(beta, eps, v, mu, grid.tau)
    G = cl["G"].reshape(ntau, 1, 1, 1).astype(np.complex128)
    V = np.full((1, 1, 1, 1, 1), v, dtype=np.complex128)
    P0 = ogw.polarization_tau(V, G, km)
    assert np.abs(P0 - cl["c"]).max() < 1e-14
    P = ogw.to_matsubara(grid.TBb, ogw.screened(ogw.to_matsubara(grid.TFb, P0, 1)), 1)
    # round trip through the transforms: roundoff grows with cond(TF) and |beta c|
    tol = 50 * np.linalg.cond(grid.TFb) * np.finfo(float).eps * (1 + abs(beta * cl["c"]))
    assert np.abs(P - cl["P_tau"]).max() < tol * abs(cl["P_tau"])
    Sig = ogw.selfenergy_tau(V, G, P, km)
    assert np.abs(Sig[:, 0, 0, 0] - cl["Sigma_tau"]).max() < tol * np.abs(cl["Sigma_tau"]).max()
    gamma = np.array([[[cl["gamma"]]]], dtype=np.complex128)
    assert abs(ogw.hartree(V, gamma)[0, 0, 0] - cl["J"]) < 1e-14
    assert abs(ogw.exchange(V, gamma)[0, 0, 0] - cl["K"]) < 1e-14


# ------------------------------------------------------------------ P7
def test_p7_invariants_after_iteration():
    sysd = make_config_system("C1")
    st = ogw.State(sysd)
    st.dyson()
    st.iterate()
    # electron count at the converged mu
    assert abs(st.N - st.n_elec) <= 1e-9
    # Hermiticity defects of the raw contractions are at roundoff level
    P0_raw = ogw.polarization_tau(st.V, st.G_tau, st.km, symmetrize=False)
    assert np.abs(P0_raw - ogw.herm(P0_raw)).max() < 1e-12 * np.abs(P0_raw).max()
    st.sigma(symmetrize_p=True)
    S_raw = ogw.selfenergy_tau(st.V, st.G_tau, st.P_tau, st.km, symmetrize=False)
    assert np.abs(S_raw - ogw.herm(S_raw)).max() < 1e-12 * np.abs(S_raw).max()
    # P~0(i Omega_0) negative semidefinite
    m0 = list(st.grid.bose_m).index(0)
    for q in range(st.km.nk):
        assert np.linalg.eigvalsh(ogw.herm(st.P0_iw[q, m0])).max() <= 1e-12


def test_p7_g_endpoint_sum_rule_converged_grid():
    # G(0+) + G(beta-) = -S^{-1}; on a converged (small beta W) grid it holds to roundoff
    st = small_state()
    st.dyson()
    g0p = np.einsum("j,jkab->kab", st.grid.l0, st.G_tau)
    gbm = np.einsum("j,jkab->kab", st.grid.lb, st.G_tau)
    assert np.abs(g0p + gbm + np.linalg.inv(st.S)).max() < 1e-10


def test_damping_is_linear_mixing_of_successive_self_energies():
    # O11 (reading C-9): from the second iteration on, the self-energy that enters the
    # Dyson step is (1 - a) Sigma_old + a Sigma_new for both the static part and
    # Sigma~(i w); the first iteration is not mixed.  Rebuilt here by hand from the
    # unmixed self-energies of a copy of the state (State.sigma), not from iterate().
    from oracle import gw as ogw
    from synth import make_system, matsubara_indices
    sysd = make_system(3, 6, (2, 1, 1), 5)
    fn, bm = matsubara_indices(12)
    sysd.update(beta=10.0, ntau=12, fermi_n=fn, bose_m=bm, n_elec=3.0)
    a = 0.3
    st = ogw.State(sysd, damping=a)
    st.iterate()                                  # first iteration: unmixed
    ref = ogw.State(sysd, damping=a)
    ref.dyson()
    Sinf1, _, Siw1 = ref.sigma()
    assert np.array_equal(st.Sigma_inf, Sinf1) and np.array_equal(st.Sigma_iw, Siw1)
    ref.Sigma_inf, ref.Sigma_iw = Sinf1, Siw1
    ref.dyson()
    Sinf2, _, Siw2 = ref.sigma()                  # unmixed second self-energy from G(Sigma_1)
    st.iterate()
    assert np.abs(st.Sigma_inf - ((1 - a) * Sinf1 + a * Sinf2)).max() < 1e-14
    assert np.abs(st.Sigma_iw - ((1 - a) * Siw1 + a * Siw2)).max() < 1e-14
    # the mixing is not the identity on this system
    assert np.abs(Siw2 - Siw1).max() > 1e-6
