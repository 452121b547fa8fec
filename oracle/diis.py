"""Oracle: DIIS extrapolation for the self-consistency loop (test infrastructure).

This module is part of the slow, obviously-correct CPU oracle.  Only the test
suite, the smoke check and the CPU-baseline leg of the benchmark may use it; the
product path never imports it.

Sec. "Self-consistent finite-temperature GW" (the loop) and the paper's remark that
it converges the Dyson equation with a DIIS scheme: the iteration is a fixed-point
problem x = F(x) for x = (Sigma_inf, Sigma~(i w)), with F one GW step (Dyson with the
mu search, then Sigma from the new G).  DIIS keeps the last m inputs x_i and
residuals r_i = F(x_i) - x_i, finds the affine combination with the smallest
residual,
    min || sum_i c_i r_i ||^2   subject to   sum_i c_i = 1,
(inner product Re <a, b> over all entries), and takes the next input
    x_next = sum_i c_i (x_i + mix r_i).
With mix = 1 and a linear F, the iterates span a Krylov space, and the residual is
zero once the history spans it (GMRES-like); on a nonlinear F it extrapolates the
same way.
"""
import numpy as np


class DIIS:
    def __init__(self, m=6, mix=1.0):
        self.m, self.mix = int(m), float(mix)
        self.xs, self.rs = [], []

    @staticmethod
    def _flat(parts):
        return np.concatenate([np.ravel(p) for p in parts])

    def push(self, x_parts, fx_parts):
        """Record one step (x, F(x)) and return the next input as arrays shaped like x."""
        x = self._flat(x_parts)
        r = self._flat(fx_parts) - x
        self.xs.append(x)
        self.rs.append(r)
        if len(self.xs) > self.m:
            self.xs.pop(0)
            self.rs.pop(0)
        n = len(self.rs)
        R = np.array(self.rs)
        B = np.real(R.conj() @ R.T)
        # bordered system for the constraint sum c = 1 (scaled for conditioning)
        scale = np.max(np.abs(np.diag(B))) or 1.0
        A = np.zeros((n + 1, n + 1))
        A[:n, :n] = B / scale
        A[:n, n] = A[n, :n] = 1.0
        rhs = np.zeros(n + 1)
        rhs[n] = 1.0
        c = np.linalg.lstsq(A, rhs, rcond=None)[0][:n]
        self.last_c = c
        nxt = sum(ci * (xi + self.mix * ri) for ci, xi, ri in zip(c, self.xs, self.rs))
        out, pos = [], 0
        for p in x_parts:
            out.append(nxt[pos:pos + p.size].reshape(p.shape))
            pos += p.size
        return out, float(np.linalg.norm(r))
