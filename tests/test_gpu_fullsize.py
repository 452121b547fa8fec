"""Parity at the full C2 size (nao 26, naux 200, 3x3x3 k-mesh, ntau 92, beta 1000),
in absolute units, on outputs the oracle computes on its own in seconds:

* P~0^q(tau) for one q (all k summed, every tau, Q, Q') from the oracle's
  non-interacting G;
* P~(i Omega) for every (q, Omega) from a seeded P~0 with a negative-definite
  Hermitian part (the complex64 inversion refined by two Newton steps);
* Sigma~^k(tau) for one k (all q summed) from the same G and a P~(tau) of the
  workload's own magnitude: the oracle's screened P~^q(tau) of one q, used for
  every q.

Targets: Sigma~ of the mixed path (split tensor-core contractions) within 1e-6 Ha
of the FP64 oracle, of the FP64 path within 1e-10 Ha; P~0 (dimensionless) within
3e-6 (mixed) and 1e-12 (FP64) of its largest entry.  Every input is seeded or
computed by the oracle; nothing comes from the CUDA path.
"""
import numpy as np
import pytest

from gpu_helpers import gpu, hermitian_noise, rel
from oracle import gw as ogw
from synth import make_config_system

pytestmark = pytest.mark.gpu

TOL_HA = {"split_tf32": 1e-6, "split_f16": 1e-6, "fp64": 1e-10}
# P~0 is dimensionless (P~ = V P V, W~ = (1 - P~)^-1 P~): relative to its largest entry
TOL_P_REL = {"split_tf32": 3e-6, "split_f16": 3e-6, "fp64": 1e-12}
Q_SLICE, K_SLICE = 5, 13


@pytest.fixture(scope="module")
def c2():
    sysd = make_config_system("C2")
    st = ogw.State(sysd)
    st.dyson()                      # G0(tau) of the non-interacting system
    q = Q_SLICE
    P0q = ogw.polarization_tau(sysd["V"], st.G_tau, st.km, qs=[q])[q]
    Pw = ogw.screened(ogw.to_matsubara(st.grid.TFb, P0q, 0))
    Pq = ogw.herm(ogw.to_matsubara(st.grid.TBb, Pw, 0))
    P = np.ascontiguousarray(np.broadcast_to(Pq, (st.km.nk,) + Pq.shape))
    return sysd, st, P0q, P


@pytest.mark.parametrize("precision", ["split_tf32", "split_f16", "fp64"])
def test_c2_polarization_one_q(c2, precision):
    sysd, st, ref, _ = c2
    g = gpu(sysd, precision=precision)
    g.set("G_tau", st.G_tau)
    g.polarization()
    got = g.get("P0_tau")[Q_SLICE]
    g.close()
    err = np.abs(got - ref).max()
    assert err < TOL_P_REL[precision] * np.abs(ref).max(), (err, np.abs(ref).max())


def test_c2_screened_all(c2):
    sysd, st, _, _ = c2
    nk, ntau, naux = st.km.nk, sysd["ntau"], sysd["V"].shape[2]
    rng = np.random.default_rng(2206)
    A = (rng.standard_normal((nk, ntau, naux, naux)) + 1j * rng.standard_normal((nk, ntau, naux, naux))) / np.sqrt(naux)
    P0 = -0.5 * (A @ np.conj(np.swapaxes(A, -1, -2))) + 0.3 * (A - np.conj(np.swapaxes(A, -1, -2)))
    ref = ogw.screened(P0)
    g = gpu(sysd, precision="split_tf32")
    g.set("P0_iw", P0)
    g.screened()
    assert rel(g.get("P_iw"), ref) < 1e-12
    g.close()


@pytest.mark.parametrize("precision", ["split_tf32", "split_f16", "fp64"])
def test_c2_selfenergy_one_k(c2, precision):
    sysd, st, _, P = c2
    k = K_SLICE
    ref = ogw.selfenergy_tau(sysd["V"], st.G_tau, P, st.km, ks=[k])[:, k]
    g = gpu(sysd, precision=precision)
    g.set("G_tau", st.G_tau)
    g.set("P_tau", P)
    g.selfenergy()
    got = g.get("Sigma_tau")[:, k]
    g.close()
    err = np.abs(got - ref).max()
    assert np.abs(ref).max() > 1e-4        # a Sigma~ of the workload's own size
    assert err < TOL_HA[precision], (err, np.abs(ref).max())


def test_c2_selfenergy_seeded_p_relative(c2):
    # a seeded Hermitian P~(tau) without the decay over Q of the real one
    sysd, st, _, _ = c2
    k = K_SLICE
    nk, ntau, naux = st.km.nk, sysd["ntau"], sysd["V"].shape[2]
    P = hermitian_noise((nk, ntau, naux, naux), 0.05, 2207)
    ref = ogw.selfenergy_tau(sysd["V"], st.G_tau, P, st.km, ks=[k])[:, k]
    g = gpu(sysd, precision="split_tf32")
    g.set("G_tau", st.G_tau)
    g.set("P_tau", P)
    g.selfenergy()
    got = g.get("Sigma_tau")[:, k]
    assert rel(got, ref) < 5e-6
    g.close()
