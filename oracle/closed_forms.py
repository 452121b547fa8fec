"""Oracle: closed forms that pin the discrete method (test infrastructure).

* Non-interacting G0 from the generalized eigenproblem H0 C = S C eps,
  C^H S C = I:  G0^k(tau) = -C diag((1-f) e^{-xi tau}) C^H, xi = eps - mu
  (Eq. G for a quadratic Hamiltonian).
* Non-interacting P~0 at any tau (Eq. tilde_P0_tau with G = G0), in the band
  basis M(Q) = C^{kH} V^{k,k+q}(Q) C^{k+q}:
  P~0^q_QQ'(tau) = -(s/Nk) sum_k sum_{m m'} M_{m'm}(Q) conj(M_{m'm}(Q'))
                     (1-f_m) f_m' e^{-(xi_m - xi_m') tau}
  and its bosonic Fourier integral (Lindhard form, Eq. P0t_to_P0w)
  P~0^q_QQ'(i Omega) = -(s/Nk) sum M M* (f_m' - f_m) / (xi_m - xi_m' - i Omega).
* Single-orbital model (nao = naux = nk = 1): P~0 is the constant
  c = -s v^2 f (1-f), so P~(tau) = c / (1 - beta c) and
  Sigma~(tau) = v^2 c / (1 - beta c) (1-f) e^{-xi tau}.
"""
import numpy as np
import scipy.linalg as sla


def fermi(beta, xi):
    return 0.5 * (1.0 - np.tanh(0.5 * beta * np.asarray(xi)))


def log_fermi(beta, xi):
    """log f(xi) = -log(1 + e^{beta xi})."""
    return -np.logaddexp(0.0, beta * np.asarray(xi))


def bands(H0, S):
    """eps[k, m], C[k] with H0 C = S C eps, C^H S C = I."""
    nk, nao = H0.shape[0], H0.shape[1]
    eps = np.zeros((nk, nao))
    C = np.zeros_like(H0)
    for k in range(nk):
        eps[k], C[k] = sla.eigh(H0[k], S[k])
    return eps, C


def electron_count0(beta, eps, mu, s=2.0):
    return s * fermi(beta, eps - mu).sum() / eps.shape[0]


def mu0(beta, eps, n_elec, s=2.0):
    lo, hi = eps.min() - 5.0, eps.max() + 5.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if electron_count0(beta, eps, mid, s) < n_elec:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def g0_tau(beta, tau, eps, C, mu):
    """G0[t, k] = -C diag((1-f) e^{-xi tau}) C^H, evaluated stably."""
    xi = eps - mu                                          # [k, m]
    # log[(1-f) e^{-xi tau}] = -xi tau + log f(-xi)
    lw = -xi[None, :, :] * tau[:, None, None] + log_fermi(beta, -xi)[None]
    w = np.exp(lw)                                         # [t, k, m]
    return -np.einsum("kim,tkm,kjm->tkij", C, w, C.conj())


def p0_tau_closed(beta, tau, eps, C, mu, V, km, s=2.0):
    """Non-interacting P~0^q(tau) at arbitrary tau points, [nq, ntau, naux, naux]."""
    nk = eps.shape[0]
    naux = V.shape[2]
    xi = eps - mu
    P = np.zeros((nk, len(tau), naux, naux), dtype=np.complex128)
    for q in range(nk):
        for k in range(nk):
            kq = km.add(k, q)
            M = np.einsum("ai,Qab,bm->Qim", C[k].conj(), V[k, kq], C[kq])   # [Q, m', m]
            # (1-f_m) f_m' e^{-(xi_m - xi_m') tau}
            lw = (-(xi[kq][None, None, :] - xi[k][None, :, None]) * tau[:, None, None]
                  + log_fermi(beta, -xi[kq])[None, None, :] + log_fermi(beta, xi[k])[None, :, None])
            w = np.exp(lw)                                                  # [t, m', m]
            P[q] -= np.einsum("Qim,tim,Rim->tQR", M, w, M.conj())
    return P * (s / nk)


def p0_iw_closed(beta, Omega, eps, C, mu, V, km, s=2.0):
    """Lindhard form of the bosonic Fourier integral of P~0, [nq, nw, naux, naux]."""
    nk = eps.shape[0]
    naux = V.shape[2]
    xi = eps - mu
    f = fermi(beta, xi)
    P = np.zeros((nk, len(Omega), naux, naux), dtype=np.complex128)
    for q in range(nk):
        for k in range(nk):
            kq = km.add(k, q)
            M = np.einsum("ai,Qab,bm->Qim", C[k].conj(), V[k, kq], C[kq])
            d = xi[kq][None, :] - xi[k][:, None]                             # xi_m - xi_m' [m', m]
            df = f[k][:, None] - f[kq][None, :]                              # f_m' - f_m
            for iw, Om in enumerate(Omega):
                den = d - 1j * Om
                with np.errstate(divide="ignore", invalid="ignore"):
                    w = df / den
                if Om == 0.0:
                    # degenerate limit: beta f(1-f)
                    small = np.abs(d) < 1e-10
                    w = np.where(small, beta * f[kq][None, :] * (1 - f[kq][None, :]), w)
                P[q, iw] -= np.einsum("Qim,im,Rim->QR", M, w, M.conj())
    return P * (s / nk)


def single_orbital(beta, eps, v, mu, tau, s=2.0):
    """Closed forms of the nao = naux = nk = 1 model at given tau points."""
    xi = eps - mu
    f = float(fermi(beta, xi))
    g = -(1 - f) * np.exp(-xi * np.asarray(tau))
    c = -s * v * v * f * (1 - f)
    Pt = c / (1 - beta * c)
    return dict(f=f, G=g, c=c, P_tau=Pt, Sigma_tau=v * v * Pt * (1 - f) * np.exp(-xi * np.asarray(tau)),
                gamma=f, J=s * v * v * f, K=-v * v * f)
