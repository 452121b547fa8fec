"""Oracle: gradients of the two contractions (test infrastructure).

A plain PyTorch-CPU complex128 restatement of the oracle's P~0[G] (Eq.
tilde_P0_tau, with the orientation and sign reading of oracle.gw) and
Sigma~[G, P~] (Eq. tilde_sigma2), both Hermitian-symmetrised, differentiated
by torch.autograd.  For a real loss L the gradient follows PyTorch's
convention: dL/dRe(x) + i dL/dIm(x).  Only the test suite uses this module.
"""
import numpy as np
import torch


def _herm(X):
    return 0.5 * (X + X.conj().transpose(-1, -2))


def polarization_t(V, G, kplus, s=2.0):
    """P~0[q, t, Q, R] from V [nk, nk, naux, nao, nao] and G [ntau, nk, nao, nao] (torch)."""
    ntau, nk = G.shape[0], G.shape[1]
    Gm = -G.flip(0)                                   # G(-t_j) = -G(t_{ntau-1-j})
    out = []
    for q in range(nk):
        acc = 0
        for k in range(nk):
            kq = kplus[q][k]
            acc = acc + torch.einsum("Qda,tab,Rbc,tcd->tQR", V[k, kq], G[:, kq], V[kq, k], Gm[:, k])
        out.append(acc)
    return _herm(torch.stack(out) * (s / nk))


def selfenergy_t(V, G, P, kminus):
    """Sigma~[t, k, i, j] from V, G and P~ [nq, ntau, naux, naux] (torch)."""
    ntau, nk = G.shape[0], G.shape[1]
    cols = []
    for k in range(nk):
        acc = 0
        for q in range(nk):
            kmq = kminus[q][k]
            acc = acc + torch.einsum("Qia,tab,tQR,Rbj->tij", V[k, kmq], G[:, kmq], P[q], V[kmq, k])
        cols.append(acc)
    return _herm(torch.stack(cols, dim=1) * (-1.0 / nk))


def _tables(km):
    nk = km.nk
    kplus = [[km.add(k, q) for k in range(nk)] for q in range(nk)]
    kminus = [[km.sub(k, q) for k in range(nk)] for q in range(nk)]
    return kplus, kminus


def polarization_vjp(V, G, km, Pbar, s=2.0):
    """Gbar for the upstream cotangent Pbar (NumPy in, NumPy out)."""
    kplus, _ = _tables(km)
    Vt = torch.from_numpy(V)
    Gt = torch.from_numpy(G).clone().requires_grad_(True)
    out = polarization_t(Vt, Gt, kplus, s)
    (g,) = torch.autograd.grad(out, Gt, grad_outputs=torch.from_numpy(Pbar))
    return g.numpy()


def selfenergy_vjp(V, G, P, km, Sbar):
    """(Gbar, Pbar) for the upstream cotangent Sbar (NumPy in, NumPy out)."""
    _, kminus = _tables(km)
    Vt = torch.from_numpy(V)
    Gt = torch.from_numpy(G).clone().requires_grad_(True)
    Pt = torch.from_numpy(P).clone().requires_grad_(True)
    out = selfenergy_t(Vt, Gt, Pt, kminus)
    gG, gP = torch.autograd.grad(out, (Gt, Pt), grad_outputs=torch.from_numpy(Sbar))
    return gG.numpy(), gP.numpy()


def forward_numpy(V, G, km, s=2.0):
    kplus, _ = _tables(km)
    with torch.no_grad():
        return polarization_t(torch.from_numpy(V), torch.from_numpy(G), kplus, s).numpy()


def selfenergy_numpy(V, G, P, km):
    _, kminus = _tables(km)
    with torch.no_grad():
        return selfenergy_t(torch.from_numpy(V), torch.from_numpy(G), torch.from_numpy(P), kminus).numpy()
