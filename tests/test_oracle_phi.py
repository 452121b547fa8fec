"""Pins of the oracle's Phi~ (Eq. tilde_Phi_GW) against closed forms.

A single bosonic pole per auxiliary channel, p(tau) = -a cosh(w0 (tau - beta/2)) / sinh(beta w0 / 2),
has p(i Omega_n) = -2 a w0 / (Omega_n^2 + w0^2), so 1 - p = (Omega_n^2 + w1^2) / (Omega_n^2 + w0^2)
with w1^2 = w0^2 + 2 a w0.  The product formula of sinh and the sum
(1/beta) sum_n 1/(Omega_n^2 + w^2) = coth(beta w / 2) / (2 w) give the exact infinite sums

    (1/beta) sum_n [ln(1 - p) + p] = (2/beta) ln[sinh(beta w1/2) / sinh(beta w0/2)] - a coth(beta w0/2).

A matrix P~0(tau) = U diag(p_Q(tau)) U^H (U unitary) has the same trace, so Phi~ for it is
1/(2 Nk) sum_q sum_Q of the scalar result.  The oracle evaluates the sum with the grid's
sampled frequencies; the check holds to the grid's representation accuracy.
"""
import numpy as np
import pytest

from oracle.grids import Grid
from oracle import thermo
from synth import matsubara_indices


def pole_tau(tau, beta, a, w0):
    return -a * np.cosh(w0 * (tau - beta / 2)) / np.sinh(beta * w0 / 2)


def log_sinh(x):
    return x + np.log1p(-np.exp(-2 * x)) - np.log(2.0)


def pole_sum(beta, a, w0):
    w1 = np.sqrt(w0 ** 2 + 2 * a * w0)
    return (2.0 / beta) * (log_sinh(beta * w1 / 2) - log_sinh(beta * w0 / 2)) - a / np.tanh(beta * w0 / 2)


def rotated_poles(grid, params, seed):
    """P~0^q(tau) = U_q diag(p(tau; a_qQ, w_qQ)) U_q^H for each q."""
    rng = np.random.default_rng(seed)
    out = []
    for a, w0 in params:
        n = len(a)
        U, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
        d = pole_tau(grid.tau[:, None], grid.beta, a[None], w0[None])
        out.append(np.einsum("ab,tb,cb->tac", U, d, U.conj()))
    return np.array(out)


@pytest.mark.parametrize("beta,ntau", [(10.0, 32), (100.0, 100)])
def test_single_pole_closed_form(beta, ntau):
    grid = Grid(beta, ntau, *matsubara_indices(ntau))
    rng = np.random.default_rng(7)
    params = [(rng.uniform(0.05, 0.9, 5), rng.uniform(0.3, 1.5, 5)) for _ in range(3)]
    P0 = rotated_poles(grid, params, 11)
    ref = sum(np.sum(pole_sum(beta, a, w0)) for a, w0 in params) / (2 * len(params))
    phi, im = thermo.phi_tilde(grid, P0, return_imag=True)
    assert abs(phi - ref) <= 1e-11 * abs(ref), (phi, ref)
    assert abs(im) <= 1e-11 * abs(ref)


def test_second_order_limit():
    # a -> 0: ln(1 - p) + p = -p^2/2 + O(a^3), so Phi~ / a^2 tends to the second-order
    # coefficient, a derivative of (1/beta) sum_n 1/(Omega_n^2 + w^2) = coth(beta w/2) / (2 w)
    beta, ntau = 10.0, 32
    grid = Grid(beta, ntau, *matsubara_indices(ntau))
    w0 = np.array([0.7])
    vals = []
    for a in (1e-2, 1e-3):
        P0 = rotated_poles(grid, [(np.array([a]), w0)], 3)
        vals.append(thermo.phi_tilde(grid, P0) / a ** 2)
        ref = pole_sum(beta, a, w0[0]) / 2
        # ln(1 - p) + p cancels to O(a^2): allow the rounding of the O(a) terms it cancels
        assert abs(vals[-1] * a ** 2 - ref) <= 1e-9 * abs(ref) + 1e-14
    x = beta * w0[0] / 2
    # second-order coefficient: -(1/2)(1/2) (1/beta) sum_n 4 w0^2 / (Omega_n^2 + w0^2)^2
    # = -(w0^2/beta) sum_n 1/(Omega_n^2 + w0^2)^2 = (w0/2) d/dw0 [coth(x)/(2 w0)] with x = beta w0 / 2
    c2 = (w0[0] / 2) * (-np.cosh(x) / np.sinh(x) / (2 * w0[0] ** 2) - beta / (4 * w0[0] * np.sinh(x) ** 2))
    assert abs(vals[-1] - c2) <= 2e-3 * abs(c2)
    assert abs(vals[0] - c2) > abs(vals[-1] - c2)


def test_zero_and_trace_terms():
    beta, ntau = 10.0, 32
    grid = Grid(beta, ntau, *matsubara_indices(ntau))
    assert thermo.phi_tilde(grid, np.zeros((2, ntau, 4, 4), dtype=np.complex128)) == 0.0
    # the Matsubara-sum weights reproduce a bosonic function's tau = 0 value: for the pole,
    # (1/beta) sum_n p(i Omega_n) = p(tau = 0) = -a coth(beta w0 / 2)
    a, w0 = 0.4, 0.9
    F = thermo.matsubara_sum_weights(grid) @ (grid.TFb @ pole_tau(grid.tau, beta, a, w0))
    assert abs(F - (-a / np.tanh(beta * w0 / 2))) < 1e-12


def test_symmetric_frequency_set_gives_a_real_sum():
    # with an odd ntau the sampled bosonic set is closed under m -> -m; a Hermitian
    # P~0(tau) without any other symmetry has P~0(-i Omega) = P~0(i Omega)^H, so the
    # terms at +-m are complex conjugates and the sampled Matsubara sum is real
    beta, ntau = 10.0, 33
    fn, bm = matsubara_indices(ntau)
    assert set((-bm).tolist()) == set(bm.tolist())
    grid = Grid(beta, ntau, fn, bm)
    rng = np.random.default_rng(19)
    n = 6
    U, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    a, w0 = rng.uniform(0.1, 0.6, n), rng.uniform(0.4, 1.2, n)
    # two poles per channel with unequal weights at +-w0: complex p(i Omega), Hermitian P~0(tau)
    t = grid.tau[:, None]
    d = -(a * np.exp(-w0 * t) + 0.3 * a * np.exp(-w0 * (beta - t))) / (1 - np.exp(-beta * w0))
    P = np.einsum("ab,tb,cb->tac", U, d, U.conj())[None]
    assert np.abs(P - np.conj(np.swapaxes(P, -1, -2))).max() < 1e-15
    Piw = grid.TFb @ P[0].reshape(ntau, -1)
    assert np.abs(Piw.imag).max() > 1e-3                     # P~0(i Omega) is not real
    phi, im = thermo.phi_tilde(grid, P, return_imag=True)
    assert abs(im) <= 1e-12 * abs(phi)


def _closed_form_case():
    beta, ntau = 10.0, 32
    grid = Grid(beta, ntau, *matsubara_indices(ntau))
    rng = np.random.default_rng(23)
    params = [(rng.uniform(0.05, 0.9, 4), rng.uniform(0.3, 1.5, 4)) for _ in range(2)]
    P0 = rotated_poles(grid, params, 29)
    ref = sum(np.sum(pole_sum(beta, a, w0)) for a, w0 in params) / (2 * len(params))
    return grid, P0, ref


@pytest.mark.parametrize("slip", ["no_trace_term", "weights_x2", "backward_transform"])
def test_planted_slips_fail_the_closed_form(monkeypatch, slip):
    # each plausible mistake, planted in the oracle, moves Phi~ far from the closed form
    grid, P0, ref = _closed_form_case()
    assert abs(thermo.phi_tilde(grid, P0) - ref) <= 1e-11 * abs(ref)
    if slip == "no_trace_term":
        monkeypatch.setattr(thermo, "trace_log_plus",
                            lambda A: np.sum(np.log(np.linalg.eigvals(np.eye(A.shape[0]) - A))))
    elif slip == "weights_x2":
        monkeypatch.setattr(thermo, "matsubara_sum_weights", lambda g: 2.0 * (g.lb @ g.TBb))
    elif slip == "backward_transform":
        class Swapped:
            pass
        sw = Swapped()
        sw.__dict__.update(grid.__dict__)
        sw.TFb = grid.TBb.T.copy()
        grid = sw
    bad = thermo.phi_tilde(grid, P0)
    assert abs(bad - ref) > 1e-4 * abs(ref)
