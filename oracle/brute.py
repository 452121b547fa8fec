"""Oracle: four-index (non-density-fitted) GW self-energy (test infrastructure).

Only for tiny systems (pair space nk*nao^2 up to a few hundred).  Follows the
four-index equations without the auxiliary-basis algebra:

* Eq. U_decompose builds U^{k1k2k3k4}_{ijkl} = sum_Q V^{k1k2}_ij(Q) V^{k3k4}_kl(Q)
  on momentum-conserving quadruples.
* Eq. P0_tau, with the orientation reading used throughout the oracle:
  Pi^{k5k6k7k8}_{abcd}(tau) = s G^{k5}_da(-tau) G^{k6}_bc(tau) delta_{k5k8} delta_{k6k7}.
* Eq. W: W = U + (1/Nk) U Pi W on each bosonic sampled frequency, so
  W~ = W - U = [(I - U Pi / Nk)^{-1} - I] U.
* Eq. tilde_sigma: Sigma~^k_ij(tau) = -(1/Nk) sum_q sum_ab G^{k-q}_ab(tau)
  W~^{k,k-q,k-q,k}_{iabj}(tau).
For each q the relevant blocks live in the pair spaces {(k, k-q)} (rows of U)
and {(k5, k5+q)} (columns of U).
"""
import numpy as np

from .gw import g_minus_tau, to_matsubara


def four_index_U(V, k1, k2, k3, k4):
    """U^{k1k2k3k4}_{ijkl} (Eq. U_decompose)."""
    return np.einsum("Qij,Qkl->ijkl", V[k1, k2], V[k3, k4])


def selfenergy_tau_4idx(V, G_tau, grid, km, s=2.0):
    ntau, nk, nao = G_tau.shape[0], G_tau.shape[1], G_tau.shape[2]
    n2 = nao * nao
    D = nk * n2
    Gm = g_minus_tau(G_tau)
    Sig = np.zeros((ntau, nk, nao, nao), dtype=np.complex128)
    for q in range(nk):
        # U_q[(k, ij), (k5, ab)] = U^{k, k-q, k5, k5+q}_{ij ab}
        U = np.zeros((D, D), dtype=np.complex128)
        for k in range(nk):
            for k5 in range(nk):
                U[k * n2:(k + 1) * n2, k5 * n2:(k5 + 1) * n2] = \
                    four_index_U(V, k, km.sub(k, q), k5, km.add(k5, q)).reshape(n2, n2)
        # Pi_q(tau)[(k5, ab), (k7, cd)] with k7 = k5 + q (rows of W are (k7, k7-q))
        Pi = np.zeros((ntau, D, D), dtype=np.complex128)
        for k5 in range(nk):
            k6 = km.add(k5, q)
            # s G^{k5}_da(-t) G^{k6}_bc(t) at [t, a, b, c, d]
            blk = s * np.einsum("tda,tbc->tabcd", Gm[:, k5], G_tau[:, k6])
            Pi[:, k5 * n2:(k5 + 1) * n2, k6 * n2:(k6 + 1) * n2] = blk.reshape(ntau, n2, n2)
        Pi_iw = to_matsubara(grid.TFb, Pi, 0)
        Wt_iw = np.empty_like(Pi_iw)
        eye = np.eye(D)
        for m in range(ntau):
            W = np.linalg.solve(eye - U @ Pi_iw[m] / nk, U)
            Wt_iw[m] = W - U
        Wt = to_matsubara(grid.TBb, Wt_iw, 0)
        # Sigma~^k_ij(t) -= (1/Nk) sum_ab G^{k-q}_ab(t) W~[(k, i a), (k-q, b j)]
        for k in range(nk):
            kmq = km.sub(k, q)
            blk = Wt[:, k * n2:(k + 1) * n2, kmq * n2:(kmq + 1) * n2].reshape(ntau, nao, nao, nao, nao)
            Sig[:, k] -= np.einsum("tab,tiabj->tij", G_tau[:, kmq], blk) / nk
    return Sig


def hf_4idx(V, gamma, s=2.0):
    """Eqs. HF_J and HF_K through the explicit four-index U."""
    nk, nao = gamma.shape[0], gamma.shape[1]
    J = np.zeros_like(gamma)
    K = np.zeros_like(gamma)
    for k in range(nk):
        for kp in range(nk):
            J[k] += s * np.einsum("ab,ijba->ij", gamma[kp], four_index_U(V, k, k, kp, kp))
            K[k] -= np.einsum("ab,iabj->ij", gamma[kp], four_index_U(V, k, kp, kp, k))
    return J / nk, K / nk
