"""Parity at the full C2 size (nao 26, naux 200, 3x3x3 k-mesh, ntau 92, beta 1000),
in the configuration the benchmark times (split-TF32 contractions, refined FP64
screened solve), on outputs the oracle computes on its own in seconds:

* P~0^q(tau) for one q (all k summed, every tau, Q, Q') from the oracle's
  non-interacting G: split-TF32 accuracy;
* P~(i Omega) for every (q, Omega) from a seeded P~0 with a negative-definite
  Hermitian part: FP64 accuracy (the complex64 inversion refined by two Newton steps);
* Sigma~^k(tau) for one k (all q summed) from the same G and a seeded P~(tau):
  split-TF32 accuracy.

Every input is seeded or computed by the oracle; nothing comes from the CUDA path.
"""
import numpy as np
import pytest

from gpu_helpers import gpu, hermitian_noise, rel
from oracle import gw as ogw
from synth import make_config_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c2():
    sysd = make_config_system("C2")
    st = ogw.State(sysd)
    st.dyson()                      # G0(tau) of the non-interacting system
    return sysd, st


def test_c2_polarization_one_q(c2):
    sysd, st = c2
    q = 5
    ref = ogw.polarization_tau(sysd["V"], st.G_tau, st.km, qs=[q])[q]
    g = gpu(sysd, precision="split_tf32")
    g.set("G_tau", st.G_tau)
    g.polarization()
    got = g.get("P0_tau")[q]
    assert rel(got, ref) < 2e-5
    g.close()


def test_c2_screened_all(c2):
    sysd, st = c2
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


def test_c2_selfenergy_one_k(c2):
    sysd, st = c2
    k = 13
    nk, ntau, naux = st.km.nk, sysd["ntau"], sysd["V"].shape[2]
    P = hermitian_noise((nk, ntau, naux, naux), 0.05, 2207)
    ref = ogw.selfenergy_tau(sysd["V"], st.G_tau, P, st.km, ks=[k])[:, k]
    g = gpu(sysd, precision="split_tf32")
    g.set("G_tau", st.G_tau)
    g.set("P_tau", P)
    g.selfenergy()
    got = g.get("Sigma_tau")[:, k]
    assert rel(got, ref) < 2e-5
    g.close()
