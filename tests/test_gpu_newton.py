"""The tangent of the whole self-consistency map (gw_sc_jvp: Dyson with the mu
constraint, Hartree-Fock, P~0, screened block, Sigma~, transforms) against
central differences of the forward map on the GPU, and Newton-Krylov
self-consistency built on it (gw_iterate_newton)."""
import numpy as np
import pytest

from gpu_helpers import gpu, system

pytestmark = pytest.mark.gpu


def _forward(g, xi, xw):
    """F(x): Sigma <- x, Dyson, P~0, screened, Sigma (damping 1: unmixed)."""
    g.set("Sigma_inf", xi)
    g.set("Sigma_iw", xw)
    g.dyson()
    g.polarization()
    g.screened()
    g.selfenergy()
    return g.get("Sigma_inf"), g.get("Sigma_iw")


def test_sc_jvp_matches_finite_differences():
    import torch
    sysd = system(4, 16, (2, 1, 1), 32, 30.0, 61)
    g = gpu(sysd, precision="fp64", damping=1.0, mu_tol=1e-12)
    g.iterate(2)
    xi, xw = g.get("Sigma_inf"), g.get("Sigma_iw")
    rng = np.random.default_rng(5)
    vi = (rng.standard_normal(xi.shape) + 1j * rng.standard_normal(xi.shape)) * 0.1
    vw = (rng.standard_normal(xw.shape) + 1j * rng.standard_normal(xw.shape)) * 0.1
    h = 1e-4
    fpi, fpw = _forward(g, xi + h * vi, xw + h * vw)
    fmi, fmw = _forward(g, xi - h * vi, xw - h * vw)
    fdi, fdw = (fpi - fmi) / (2 * h), (fpw - fmw) / (2 * h)
    _forward(g, xi, xw)   # state at x for the tangent
    ji, jw = g.sc_jvp(torch.from_numpy(vi).cuda(), torch.from_numpy(vw).cuda())
    ji, jw = ji.cpu().numpy(), jw.cpu().numpy()
    assert np.abs(ji - fdi).max() <= 1e-6 * max(1e-3, np.abs(fdi).max())
    assert np.abs(jw - fdw).max() <= 1e-6 * max(1e-3, np.abs(fdw).max())


@pytest.mark.parametrize("precision", ["fp64", "split_tf32"])
def test_newton_krylov_converges(precision):
    sysd = system(4, 16, (2, 1, 1), 32, 30.0, 61)
    g = gpu(sysd, precision=precision, damping=1.0, mu_tol=1e-12)
    g.iterate(1)
    # from ||F(x) - x|| ~ 8 the steps converge superlinearly (measured: 8.2, 2.5, 0.91,
    # 0.11, 5.2e-3, 1.9e-5, ...); the split-TF32 tangents stop at that precision's floor
    tol = 1e-8 if precision == "fp64" else 1e-4
    res = g.iterate_newton(8, m=12, tol=tol)
    assert res[-1] <= tol, res
    assert all(b < a for a, b in zip(res[:4], res[1:5])), res
    # the fixed point: one more plain (unmixed) evaluation changes Sigma by about the residual
    xi, xw = g.get("Sigma_inf"), g.get("Sigma_iw")
    g.polarization()
    g.screened()
    g.selfenergy()
    d = max(np.abs(g.get("Sigma_inf") - xi).max(), np.abs(g.get("Sigma_iw") - xw).max())
    assert d <= 10 * res[-1] + 1e-12, (d, res)
