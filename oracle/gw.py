"""Oracle: one fully self-consistent GW iteration, step by step (test infrastructure).

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
use this module.  Everything is complex128 NumPy; each function names the
equation it evaluates.  Matrix products are grouped so that no four-index
object is formed (the association of a matrix chain is the only freedom
taken); the four-index route of oracle.brute pins that grouping.

Conventions (readings of the paper where it is silent or inconsistent):
* spin-restricted, spin-diagonal G; the spin sum gives a factor s = 2 in P~0,
  in the Hartree term and in the electron count, none in K and Sigma~.
* P~0 takes the orientation of Eq. tilde_P0_tau with a positive prefactor
  on G(tau) G(-tau): P~0 = +(s/Nk) sum V G^{k+q}(tau) V G^k(-tau), where
  G(-tau_j) = -G(beta - tau_j) = -G(tau_{ntau-1-j}) (antiperiodicity).  This is
  the sign that makes P~0(i Omega_0) negative semidefinite, as the four-index
  Eqs. W and P0_tau require.
* Sigma~ follows Eq. tilde_sigma2 literally.
* Hermitian symmetrisation (X + X^H)/2 of P~0(tau), P~(tau), Sigma~(tau) and
  G(tau) is part of the discrete definition (sampled frequency sets are not
  symmetric under Omega -> -Omega).
* Chemical potential: bisection on N(mu) - N_e until |N - N_e| <= mu_tol and
  the bracket is narrower than 1e-13 (paper: threshold 1e-9).
* Damping (linear mixing, factor alpha) of Sigma_inf and Sigma~(i w) from the
  second GW iteration on.
"""
import numpy as np
import scipy.linalg as sla

from .grids import Grid


class KMesh:
    """Gamma-centred n1 x n2 x n3 mesh; k = (i1 n2 + i2) n3 + i3."""

    def __init__(self, kmesh):
        self.dims = tuple(int(x) for x in kmesh)
        n1, n2, n3 = self.dims
        self.nk = n1 * n2 * n3
        self.vec = np.array([(a, b, c) for a in range(n1) for b in range(n2) for c in range(n3)])

    def index(self, v):
        n1, n2, n3 = self.dims
        return (int(v[0]) % n1 * n2 + int(v[1]) % n2) * n3 + int(v[2]) % n3

    def add(self, k, q):
        return self.index(self.vec[k] + self.vec[q])

    def sub(self, k, q):
        return self.index(self.vec[k] - self.vec[q])


def herm(X):
    """(X + X^H)/2 over the last two axes."""
    return 0.5 * (X + np.conj(np.swapaxes(X, -1, -2)))


def g_minus_tau(G_tau):
    """G(-tau_j) = -G(beta - tau_j) = -G(tau_{ntau-1-j}) (fermionic antiperiodicity)."""
    return -G_tau[::-1]


# ---------------------------------------------------------------- A1: gamma, HF

def density_matrix(grid, G_tau):
    """gamma^k = -G^k(beta^-) = -sum_j lb_j G^k(tau_j)."""
    return -np.einsum("j,jkab->kab", grid.lb, G_tau)


def hartree(V, gamma, s=2.0):
    """Eq. HF_J: J^k_ij = (s/Nk) sum_{k',Q,ab} V^{kk}_ij(Q) gamma^{k'}_ab V^{k'k'}_ba(Q)."""
    nk = gamma.shape[0]
    Vd = V[np.arange(nk), np.arange(nk)]                      # [k, Q, i, j] = V^{kk}
    t = np.einsum("kab,kQba->Q", gamma, Vd)
    return (s / nk) * np.einsum("kQij,Q->kij", Vd, t)


def exchange(V, gamma, kps=None, ks=None):
    """Eq. HF_K: K^k_ij = -(1/Nk) sum_{k',Q,ab} V^{kk'}_ia(Q) gamma^{k'}_ab V^{k'k}_bj(Q).

    `kps` restricts the k' sum (timing samples only); `ks` computes only the rows
    of those k (the others stay zero; sampled checks)."""
    nk = gamma.shape[0]
    K = np.zeros_like(gamma)
    naux, nao = V.shape[2], V.shape[3]
    for k in (range(nk) if ks is None else ks):
        for kp in (range(nk) if kps is None else kps):
            A = np.matmul(V[k, kp], gamma[kp])                # [Q, i, b]
            At = A.transpose(1, 0, 2).reshape(nao, naux * nao)  # [i, (Q, b)]
            K[k] -= At @ V[kp, k].reshape(naux * nao, nao)
    return K / nk


# ---------------------------------------------------------------- A2: P~0(tau)

def polarization_tau(V, G_tau, km, s=2.0, symmetrize=True, qs=None, ks=None):
    """Eq. tilde_P0_tau (sign/orientation as in the module docstring).

    P~0^q_{QQ'}(tau) = (s/Nk) sum_k sum_abcd V^{k,k+q}_da(Q) G^{k+q}_ab(tau)
                                          V^{k+q,k}_bc(Q') G^k_cd(-tau)
    Returns [nq, ntau, naux, naux] (only the q in `qs` are filled when given;
    `ks` restricts the k-sum, for timing samples only).
    """
    ntau, nk, nao = G_tau.shape[0], G_tau.shape[1], G_tau.shape[2]
    naux = V.shape[2]
    Gm = g_minus_tau(G_tau)
    P = np.zeros((nk, ntau, naux, naux), dtype=np.complex128)
    for q in (range(nk) if qs is None else qs):
        for k in (range(nk) if ks is None else ks):
            kq = km.add(k, q)
            # VG[t, Q, d, b] = sum_a V^{k,k+q}_da(Q) G^{k+q}_ab(t)
            VG = np.matmul(V[k, kq].reshape(naux * nao, nao)[None], G_tau[:, kq])
            VG = VG.reshape(ntau, naux, nao, nao)
            # Z[t, Q, c, b] = sum_d G^k_cd(-t) VG[t, Q, d, b]
            VGt = VG.transpose(0, 2, 1, 3).reshape(ntau, nao, naux * nao)
            Z = np.matmul(Gm[:, k], VGt).reshape(ntau, nao, naux, nao).transpose(0, 2, 1, 3)
            # P[t, Q, R] += sum_{c,b} Z[t, Q, c, b] V^{k+q,k}_bc(R)
            B = V[kq, k].transpose(2, 1, 0).reshape(nao * nao, naux)
            P[q] += (np.ascontiguousarray(Z).reshape(ntau * naux, nao * nao) @ B).reshape(ntau, naux, naux)
    P *= s / nk
    return herm(P) if symmetrize else P


# ---------------------------------------------------------------- A3/A5: bosonic transforms

def to_matsubara(T, X_tau, axis):
    """Y(i nu_m) = sum_j T[m, j] X(tau_j) along `axis` (Eqs. tau_to_iw, P0t_to_P0w)."""
    return np.moveaxis(np.tensordot(T, X_tau, axes=([1], [axis])), 0, axis)


# ---------------------------------------------------------------- A4: screened solve

def screened(P0_iw):
    """Eq. tilde_P_omega: P~(i Omega) = [I - P~0(i Omega)]^{-1} P~0(i Omega), per (q, m)."""
    naux = P0_iw.shape[-1]
    A = np.eye(naux) - P0_iw
    return np.linalg.solve(A, P0_iw)


# ---------------------------------------------------------------- A6: Sigma~(tau)

def selfenergy_tau(V, G_tau, P_tau, km, symmetrize=True, qs=None, ks=None):
    """Eq. tilde_sigma2:
    Sigma~^k_ij(tau) = -(1/Nk) sum_q sum_ab sum_QQ' G^{k-q}_ab(tau) V^{k,k-q}_ia(Q)
                                                   P~^q_QQ'(tau) V^{k-q,k}_bj(Q')
    P_tau: [nq, ntau, naux, naux].  Returns [ntau, nk, nao, nao] (the sum runs
    over the q in `qs` only when given).
    """
    ntau, nk, nao = G_tau.shape[0], G_tau.shape[1], G_tau.shape[2]
    naux = V.shape[2]
    Sig = np.zeros((ntau, nk, nao, nao), dtype=np.complex128)
    for q in (range(nk) if qs is None else qs):
        PT = np.ascontiguousarray(P_tau[q].transpose(0, 2, 1))           # [t, Q', Q]
        for k in (range(nk) if ks is None else ks):
            kmq = km.sub(k, q)
            # X[t, Q', i, a] = sum_Q P~^q_QQ'(t) V^{k,k-q}_ia(Q)
            X = np.matmul(PT, V[k, kmq].reshape(naux, nao * nao)[None])
            # Y[t, Q', i, b] = sum_a X[t, Q', i, a] G^{k-q}_ab(t)
            Y = np.matmul(X.reshape(ntau, naux * nao, nao), G_tau[:, kmq]).reshape(ntau, naux, nao, nao)
            # Sigma[t, i, j] += sum_{Q', b} Y[t, Q', i, b] V^{k-q,k}_bj(Q')
            Yt = Y.transpose(0, 2, 1, 3).reshape(ntau, nao, naux * nao)
            Sig[:, k] += np.matmul(Yt, V[kmq, k].reshape(naux * nao, nao)[None])
    Sig *= -1.0 / nk
    return herm(Sig) if symmetrize else Sig


# ---------------------------------------------------------------- A7: Dyson and mu

def dyson_inverse(grid, H0, S, Sigma_inf, Sigma_iw, mu):
    """Eq. Dyson: G^k(i w_n) = [(i w_n + mu) S^k - H0^k - Sigma_inf^k - Sigma~^k(i w_n)]^{-1}."""
    z = (1j * grid.wf + mu)[:, None, None, None]
    A = z * S[None] - H0[None] - Sigma_inf[None] - Sigma_iw
    return np.linalg.inv(A)


def electron_count(grid, S, G_iw, s=2.0):
    """N = (s/Nk) sum_k tr[gamma^k S^k], gamma^k = -sum_n r_n G^k(i w_n); real part."""
    nk = S.shape[0]
    tr = np.einsum("nkab,kba->n", G_iw, S)
    return float(np.real(-(s / nk) * np.dot(grid.r, tr)))


def find_mu(grid, H0, S, Sigma_inf, Sigma_iw, n_elec, s=2.0, tol=1e-9, width=1e-13, maxit=200):
    """Bisection for N(mu) = n_elec.  Returns (mu, N(mu), steps)."""
    def N(mu):
        return electron_count(grid, S, dyson_inverse(grid, H0, S, Sigma_inf, Sigma_iw, mu), s)
    H = H0 + Sigma_inf
    ev = np.concatenate([sla.eigh(0.5 * (H[k] + H[k].conj().T), S[k], eigvals_only=True)
                         for k in range(H.shape[0])])
    lo, hi = ev.min() - 1.0, ev.max() + 1.0
    Nlo, Nhi = N(lo), N(hi)
    steps = 0
    while Nlo > n_elec and steps < maxit:
        lo -= 2.0 * (hi - lo); Nlo = N(lo); steps += 1
    while Nhi < n_elec and steps < maxit:
        hi += 2.0 * (hi - lo); Nhi = N(hi); steps += 1
    mu = 0.5 * (lo + hi)
    Nm = N(mu)
    while steps < maxit and not (abs(Nm - n_elec) <= tol and hi - lo <= width):
        if Nm < n_elec:
            lo = mu
        else:
            hi = mu
        mu = 0.5 * (lo + hi)
        Nm = N(mu)
        steps += 1
    return mu, Nm, steps


def green_tau(grid, G_iw):
    """G(tau_j) = sum_n TBf[j, n] G(i w_n), then Hermitian symmetrisation."""
    return herm(to_matsubara(grid.TBf, G_iw, 0))


# ---------------------------------------------------------------- iteration driver

class State:
    """Oracle state of a self-consistent run."""

    def __init__(self, sysd, s=2.0, damping=0.5, mu_tol=1e-9, grid=None):
        self.H0, self.S, self.V = sysd["H0"], sysd["S"], sysd["V"]
        self.km = KMesh(sysd["kmesh"])
        # the Chebyshev grid of the system's (beta, ntau, index sets), or any grid with
        # the same attributes (oracle.ir.IRGrid)
        self.grid = grid if grid is not None else Grid(sysd["beta"], sysd["ntau"], sysd["fermi_n"], sysd["bose_m"])
        self.s, self.alpha, self.mu_tol = s, damping, mu_tol
        self.n_elec = float(sysd["n_elec"])
        nk, nao = self.H0.shape[0], self.H0.shape[1]
        nw = len(self.grid.wf)
        self.Sigma_inf = np.zeros((nk, nao, nao), dtype=np.complex128)
        self.Sigma_iw = np.zeros((nw, nk, nao, nao), dtype=np.complex128)
        self.have_sigma = False
        self.G_tau = None
        self.mu = None

    def dyson(self):
        """O12-O13: mu search, then G(i w) and G(tau)."""
        g = self.grid
        self.mu, self.N, self.mu_steps = find_mu(g, self.H0, self.S, self.Sigma_inf, self.Sigma_iw,
                                                 self.n_elec, self.s, self.mu_tol)
        self.G_iw = dyson_inverse(g, self.H0, self.S, self.Sigma_inf, self.Sigma_iw, self.mu)
        self.G_tau = green_tau(g, self.G_iw)
        return self.mu

    def sigma(self, symmetrize_p=True):
        """O3-O10 from the current G(tau): returns (Sigma_inf, Sigma~(tau), Sigma~(i w))."""
        g, V, km = self.grid, self.V, self.km
        self.gamma = density_matrix(g, self.G_tau)
        Sinf = hartree(V, self.gamma, self.s) + exchange(V, self.gamma)
        self.P0_tau = polarization_tau(V, self.G_tau, km, self.s, symmetrize=symmetrize_p)
        self.P0_iw = to_matsubara(g.TFb, self.P0_tau, 1)
        self.P_iw = screened(self.P0_iw)
        P_tau = to_matsubara(g.TBb, self.P_iw, 1)
        self.P_tau = herm(P_tau) if symmetrize_p else P_tau
        self.Sigma_tau = selfenergy_tau(V, self.G_tau, self.P_tau, km)
        Siw = to_matsubara(g.TFf, self.Sigma_tau, 0)
        return Sinf, self.Sigma_tau, Siw

    def iterate(self):
        """One full GW iteration (O3-O13) from the current G; O2 first if no G yet."""
        if self.G_tau is None:
            self.dyson()
        Sinf, _, Siw = self.sigma()
        if self.have_sigma:
            a = self.alpha
            Sinf = (1 - a) * self.Sigma_inf + a * Sinf
            Siw = (1 - a) * self.Sigma_iw + a * Siw
        self.Sigma_inf, self.Sigma_iw, self.have_sigma = Sinf, Siw, True
        G_old = self.G_tau
        self.dyson()
        return dict(mu=self.mu, N=self.N, dG=float(np.abs(self.G_tau - G_old).max()))
