"""Pins of the oracle's DIIS extrapolation for the self-consistency loop.

* affine combination: the coefficients sum to one, and a fixed point stays put;
* on a linear contraction F(x) = A x + b the DIIS iterates (mix = 1) solve the
  fixed-point problem once the history spans the Krylov space (2n real dimensions
  for n complex unknowns), like GMRES;
* on the small configuration (nao 8, naux 32, 2x2x2 k-mesh, ntau 32, beta 100) the
  damped iteration (mixing 0.5) does not converge — the residual ||F(x) - x|| of the
  GW map stays near 50 — while DIIS over the last 6 steps brings it below 1e-2 in
  20 steps.
"""
import numpy as np

from oracle import gw as ogw
from oracle.diis import DIIS
from synth import make_config_system


def test_affine_and_fixed_point():
    d = DIIS(m=4)
    x = np.arange(5.0) + 1j
    for _ in range(3):
        (y,), rn = d.push([x], [x])
        assert rn == 0.0
        assert np.allclose(y, x)
    rng = np.random.default_rng(3)
    d = DIIS(m=4)
    for _ in range(4):
        x = rng.standard_normal(6)
        d.push([x], [0.5 * x + 1.0])
        assert abs(d.last_c.sum() - 1.0) < 1e-12


def test_linear_fixed_point_like_gmres():
    rng = np.random.default_rng(1)
    n = 8
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A *= 0.9 / np.max(np.abs(np.linalg.eigvals(A)))
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    xstar = np.linalg.solve(np.eye(n) - A, b)
    d = DIIS(m=2 * n + 4, mix=1.0)
    x = np.zeros(n, complex)
    for _ in range(2 * n + 2):
        (x,), _ = d.push([x], [A @ x + b])
    assert np.abs(x - xstar).max() < 1e-9 * np.abs(xstar).max()


def _gw_residuals(mode, steps=20):
    sysd = make_config_system("C1")
    st = ogw.State(sysd, damping=0.5)
    st.dyson()
    d = DIIS(m=6, mix=0.5)
    res = []
    for it in range(steps):
        Sinf, _, Siw = st.sigma()
        if it == 0:
            nxt = (Sinf, Siw)
            if mode == "diis":
                d.push([np.zeros_like(Sinf), np.zeros_like(Siw)], [Sinf, Siw])
        else:
            r = np.concatenate([(Sinf - st.Sigma_inf).ravel(), (Siw - st.Sigma_iw).ravel()])
            res.append(float(np.linalg.norm(r)))
            if mode == "damp":
                nxt = (0.5 * st.Sigma_inf + 0.5 * Sinf, 0.5 * st.Sigma_iw + 0.5 * Siw)
            else:
                nxt, _ = d.push([st.Sigma_inf, st.Sigma_iw], [Sinf, Siw])
        st.Sigma_inf, st.Sigma_iw, st.have_sigma = nxt[0], nxt[1], True
        st.dyson()
        assert abs(st.N - st.n_elec) < 1e-8
    return res


def test_diis_converges_where_damping_stalls():
    damp = _gw_residuals("damp")
    diis = _gw_residuals("diis")
    assert min(damp[-5:]) > 10.0
    assert diis[-1] < 1e-2 and diis[-1] < 1e-3 * diis[0]
