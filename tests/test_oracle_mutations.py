"""Plant plausible mistakes in (copies of) the oracle's contractions and check
that the pins of test_oracle_pins.py catch each one.  Mistakes are planted on
the CPU in the oracle only."""
import numpy as np
import pytest

from oracle import closed_forms as cf
from oracle import gw as ogw
from oracle.brute import selfenergy_tau_4idx
from oracle.grids import Grid
from synth import make_system, matsubara_indices


def _pol_variant(V, G_tau, km, s=2.0, kind="ok"):
    ntau, nk = G_tau.shape[0], G_tau.shape[1]
    naux = V.shape[2]
    Gm = ogw.g_minus_tau(G_tau)
    if kind == "no_antiperiodic_sign":
        Gm = G_tau[::-1]
    P = np.zeros((nk, ntau, naux, naux), dtype=np.complex128)
    for q in range(nk):
        for k in range(nk):
            kq = km.add(k, q) if kind != "k_minus_q" else km.sub(k, q)
            Ga, Gb = G_tau[:, kq], Gm[:, k]
            if kind == "swap_orientation":
                Ga, Gb = Gm[:, kq], G_tau[:, k]
            V2 = V[kq, k] if kind != "transpose_v" else np.swapaxes(V[kq, k], 1, 2)
            VG = np.einsum("Qda,tab->tQdb", V[k, kq], Ga)
            Z = np.einsum("tcd,tQdb->tQcb", Gb, VG)
            P[q] += np.einsum("tQcb,Rbc->tQR", Z, V2)
    fac = s / nk if kind != "drop_spin" else 1.0 / nk
    return P * fac


def _checks(pol):
    """Run the P3/P4/P6-type checks with a polarization implementation; True if all pass."""
    ok = True
    # P3 at nodes (non-TRS, 3 k-points)
    sysd = make_system(3, 6, (3, 1, 1), 5)
    fn, bm = matsubara_indices(16)
    sysd.update(beta=20.0, ntau=16, fermi_n=fn, bose_m=bm, n_elec=3.0)
    st = ogw.State(sysd)
    eps, C = cf.bands(st.H0, st.S)
    mu = cf.mu0(st.grid.beta, eps, 3.0)
    G0 = cf.g0_tau(st.grid.beta, st.grid.tau, eps, C, mu)
    Pc = cf.p0_tau_closed(st.grid.beta, st.grid.tau, eps, C, mu, st.V, st.km)
    ok &= np.abs(pol(st.V, G0, st.km) - Pc).max() < 1e-12
    # P4: DF route vs four-index with a generic (perturbed) G
    rng = np.random.default_rng(2)
    G = G0 + 0.05 * (rng.standard_normal(G0.shape) + 1j * rng.standard_normal(G0.shape))
    P0 = pol(st.V, G, st.km)
    P = ogw.to_matsubara(st.grid.TBb, ogw.screened(ogw.to_matsubara(st.grid.TFb, P0, 1)), 1)
    S_df = ogw.selfenergy_tau(st.V, G, P, st.km, symmetrize=False)
    S_4 = selfenergy_tau_4idx(st.V, G, st.grid, st.km)
    ok &= np.abs(S_df - S_4).max() < 1e-11
    # P6 single orbital
    grid = Grid(10.0, 8, *matsubara_indices(8))
    cl = cf.single_orbital(10.0, 0.3, 0.7, 0.05, grid.tau)
    G1 = cl["G"].reshape(8, 1, 1, 1).astype(np.complex128)
    V1 = np.full((1, 1, 1, 1, 1), 0.7, dtype=np.complex128)
    ok &= np.abs(pol(V1, G1, ogw.KMesh((1, 1, 1))) - cl["c"]).max() < 1e-13
    return bool(ok)


def test_unmutated_passes():
    assert _checks(lambda V, G, km: _pol_variant(V, G, km, kind="ok"))


@pytest.mark.parametrize("kind", ["no_antiperiodic_sign", "swap_orientation", "k_minus_q",
                                  "transpose_v", "drop_spin"])
def test_mutation_caught(kind):
    assert not _checks(lambda V, G, km: _pol_variant(V, G, km, kind=kind))
