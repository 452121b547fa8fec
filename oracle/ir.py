"""Oracle: intermediate-representation (IR) basis with sparse sampling (test
infrastructure).

This module is part of the slow, obviously-correct CPU oracle.  Only the test
suite, the smoke check and the CPU-baseline leg of the benchmark may use it; the
product path never imports it.

Sec. "Representation on the imaginary axes": every dynamical quantity is expanded
in the IR basis, the singular functions of the kernel that maps a spectral
function to its imaginary-time function, truncated by a dimensionless cutoff
lambda >= beta * bandwidth, and sampled sparsely on the tau and Matsubara axes.
The paper takes the basis from an external package; here it comes from this
project's own singular value expansion in double precision: a singular function
with singular value s_l is resolved to ~1e-16 s_0 / s_l (its parity shows it), which
still carries a pole between the axes to ~3e-11 at eps = 1e-12, lambda = 1e3; below
that the highest functions show spurious extrema (more tau points than L).

With x = 2 tau / beta - 1, y = omega / omega_max and lambda = beta omega_max,
  fermions:  K(x, y) = exp(-lambda x y / 2) / (2 cosh(lambda y / 2))
                     = exp(-tau omega) / (1 + exp(-beta omega)),
  bosons:    K(x, y) = y exp(-lambda x y / 2) / (2 sinh(lambda y / 2))
                     = (omega / omega_max) exp(-tau omega) / (1 - exp(-beta omega)),
the bosonic one regular at omega = 0 (limit 1 / lambda).  Both satisfy
K(-x, -y) = K(x, y), so u_l(-x) = (-1)^l u_l(x).

Expansion: K(x, y) = sum_l s_l u_l(x) v_l(y), with u_l orthonormal on [-1, 1].
Discretisation: composite Gauss-Legendre quadrature on x, y in [0, 1] (segments
refined geometrically towards x = 1 and y = 0, where the kernel varies on the scale
1/lambda, plus uniform segments of width 1/8), one SVD of sqrt(w_x) K_pm sqrt(w_y)
per parity sector (see IRBasis).  On [0, beta] the basis functions are
U_l(tau) = sqrt(2/beta) u_l(x) (orthonormal in tau).  Inside a segment u_l is its
Legendre series (exact at the nodes); the Fourier integral of a segment is summed
in closed form,  int_{-1}^{1} P_k(t) e^{i z t} dt = 2 i^k j_k(z),  so
Uhat_l(n) = int_0^beta e^{i nu_n tau} U_l(tau) dtau is exact for every n
(nu_n = (2n+1) pi / beta for fermions, 2 n pi / beta for bosons).

Sparse sampling: tau points at the extrema of u_{L-1} (L of them); Matsubara
points where the nonzero part of Uhat_{L-1}(n) changes sign along n >= 0, mirrored
to negative frequencies, plus tail frequencies (twice the largest) until there are
at least L.  From values at the tau points the coefficients are a
linear solve, and any other tau or Matsubara value follows from them.
"""
import numpy as np
from numpy.polynomial import legendre as npleg
from scipy.special import spherical_jn


def _segments(lam, toward):
    """Breakpoints on [0, 1]: geometric towards `toward` (1 or 0) down to ~1/(8 lambda),
    merged with a uniform grid of step 1/8."""
    kmax = int(np.ceil(np.log2(8.0 * max(lam, 1.0)))) + 1
    geo = 2.0 ** -np.arange(1, kmax + 1)
    pts = 1.0 - geo if toward == 1 else geo
    pts = np.concatenate([pts, np.linspace(0.0, 1.0, 9)])
    return np.unique(np.round(pts, 15))


def _gauss(breaks, ngl):
    t, w = npleg.leggauss(ngl)
    a, b = breaks[:-1], breaks[1:]
    c, h = 0.5 * (a + b), 0.5 * (b - a)
    x = (c[:, None] + h[:, None] * t[None, :]).ravel()
    wx = (h[:, None] * w[None, :]).ravel()
    return x, wx, c, h, t, w


def kernel(lam, x, y, stat):
    """K(x, y) of the module docstring, evaluated without overflow."""
    x = np.asarray(x, dtype=float)[:, None]
    y = np.asarray(y, dtype=float)[None, :]
    z = lam * y
    az = np.abs(z)
    expo = np.exp(-0.5 * z * x - 0.5 * az)
    if stat == "F":
        return expo / (1.0 + np.exp(-az))
    with np.errstate(invalid="ignore", divide="ignore"):
        val = np.abs(y) * expo / (-np.expm1(-az))
    return np.where(az == 0.0, 1.0 / lam + 0.0 * x, val)


class IRBasis:
    """IR basis of one statistics ('F' or 'B') for cutoff lam and inverse
    temperature beta, truncated at s_l / s_0 > eps.

    K(-x, -y) = K(x, y) splits the expansion into an even and an odd sector: on
    x, y in [0, 1] the kernels K(x, y) +- K(x, -y) have the singular functions f_l of
    the even (+) and odd (-) u_l, u_l(x) = f_l(|x|) (sign x for odd) / sqrt(2), with
    the same singular values.  Each sector is its own SVD, so the parity is exact and
    nearly equal singular values of the two sectors (bosons at large lambda) do not
    mix their functions."""

    def __init__(self, lam, beta, stat="F", eps=1e-8, ngl=24):
        self.lam, self.beta, self.stat, self.ngl = float(lam), float(beta), stat, ngl
        bx, by = _segments(lam, 1), _segments(lam, 0)
        x, wx, self.cx, self.hx, self.t, self.w = _gauss(bx, ngl)
        y, wy, _, _, _, _ = _gauss(by, ngl)
        self.breaks = bx
        Kp, Km = kernel(lam, x, y, stat), kernel(lam, x, -y, stat)
        sv, funcs, par, vfun = [], [], [], []
        for p, Ks in ((1, Kp + Km), (-1, Kp - Km)):
            A = np.sqrt(wx)[:, None] * Ks * np.sqrt(wy)[None, :]
            U, s, Vt = np.linalg.svd(A, full_matrices=False)
            sv.append(s)
            funcs.append(U / np.sqrt(wx)[:, None])
            vfun.append(Vt.T / np.sqrt(wy)[:, None])
            par.append(np.full(s.size, p))
        s_all = np.concatenate(sv)
        order = np.argsort(-s_all, kind="stable")
        L = int(np.sum(s_all / s_all[0] > eps))
        order = order[:L]
        f_all = np.concatenate(funcs, axis=1)[:, order]
        v_all = np.concatenate(vfun, axis=1)[:, order]
        self.s = s_all[order]
        self.parity = np.concatenate(par)[order]
        self.size = L
        nseg = len(bx) - 1
        vals = f_all.reshape(nseg, ngl, L)
        # Legendre coefficients per segment: a_k = (2k+1)/2 sum_i w_i f(t_i) P_k(t_i)
        P = npleg.legvander(self.t, ngl - 1)
        self.coef = np.einsum("i,ik,sil->skl", self.w, P, vals) * ((2 * np.arange(ngl) + 1) / 2.0)[None, :, None]
        # sign convention: u_l(1) > 0
        sign = np.sign(self._f(np.array([1.0]))[0])
        sign[sign == 0] = 1.0
        self.coef *= sign[None, None, :]
        # v_l on y in [0, 1] (v_l(-y) = parity * v_l(y)), scaled like u_l
        self.v_nodes, self.y_nodes = v_all * sign[None, :] / np.sqrt(2.0), y

    # ---------------------------------------------------------------- evaluation
    def _f(self, x, deriv=0):
        """Sector functions f_l on [0, 1] (or their derivatives)."""
        x = np.atleast_1d(np.asarray(x, dtype=float))
        seg = np.clip(np.searchsorted(self.breaks, x, side="right") - 1, 0, len(self.breaks) - 2)
        out = np.empty((x.size, self.size))
        for s in np.unique(seg):
            m = seg == s
            t = (x[m] - self.cx[s]) / self.hx[s]
            c = self.coef[s]
            if deriv:
                c = npleg.legder(c, deriv) / self.hx[s] ** deriv
            out[m] = npleg.legval(t, c).T
        return out

    def _u_x(self, x, deriv=0):
        """u_l(x) on [-1, 1] (deriv = 0 or 1)."""
        x = np.atleast_1d(np.asarray(x, dtype=float))
        sx = np.where(x < 0, -1.0, 1.0)[:, None]
        f = self._f(np.abs(x), deriv)
        odd = (self.parity < 0)[None, :]
        # u(x) = f(|x|) (sx if odd) / sqrt 2;  u'(x) = f'(|x|) sx (sx if odd) / sqrt 2
        fac = np.where(odd, sx, 1.0) * (sx if deriv == 1 else 1.0)
        return f * fac / np.sqrt(2.0)

    def u(self, tau):
        """U_l(tau) = sqrt(2/beta) u_l(2 tau / beta - 1): [len(tau), L]."""
        tau = np.atleast_1d(np.asarray(tau, dtype=float))
        return np.sqrt(2.0 / self.beta) * self._u_x(2.0 * tau / self.beta - 1.0)

    def freq(self, n):
        n = np.asarray(n)
        odd = 1 if self.stat == "F" else 0
        return (2 * n + odd) * np.pi / self.beta

    def uhat(self, n):
        """Uhat_l(n) = int_0^beta e^{i nu_n tau} U_l(tau) dtau: [len(n), L] complex."""
        n = np.atleast_1d(np.asarray(n))
        wp = 0.5 * self.freq(n) * self.beta                    # omega' = nu beta / 2
        k = np.arange(self.ngl)
        ik = (1j) ** k
        # int_{-1}^{1} u(x) e^{i w x} dx = (1/sqrt 2) sum over segments [a, b] of [0, 1] of
        #   int_a^b f e^{i w x} dx + parity int_a^b f e^{-i w x} dx
        plus = np.zeros((n.size, self.size), dtype=complex)
        minus = np.zeros((n.size, self.size), dtype=complex)
        for s in range(len(self.cx)):
            z = wp * self.hx[s]
            par = np.where((z < 0)[:, None], ((-1.0) ** k)[None, :], 1.0)   # j_k(-z) = (-1)^k j_k(z)
            jk = spherical_jn(k[None, :], np.abs(z)[:, None]) * par
            m_plus = 2.0 * jk * ik[None, :]                   # int P_k(t) e^{+i z t} dt
            m_minus = 2.0 * jk * np.conj(ik)[None, :]          # int P_k(t) e^{-i z t} dt
            plus += (self.hx[s] * np.exp(1j * wp * self.cx[s]))[:, None] * (m_plus @ self.coef[s])
            minus += (self.hx[s] * np.exp(-1j * wp * self.cx[s]))[:, None] * (m_minus @ self.coef[s])
        integral = (plus + self.parity[None, :] * minus) / np.sqrt(2.0)
        return np.sqrt(0.5 * self.beta) * np.exp(1j * wp)[:, None] * integral

    # ---------------------------------------------------------------- sampling
    def tau_points(self):
        """Extrema of u_{L-1} on [-1, 1], as tau (ascending): the interior ones of
        x > 0 mirrored (u_{L-1} has a definite parity), x = 0 when u_{L-1} is even,
        and the ends while fewer than L were found."""
        grid = np.concatenate([np.linspace(a, b, 64, endpoint=False) for a, b in zip(self.breaks[:-1], self.breaks[1:])]
                              + [np.array([1.0])])
        grid = grid[grid > 0]
        d = self._f(grid, deriv=1)[:, -1]
        roots = []
        for i in np.nonzero(np.sign(d[:-1]) * np.sign(d[1:]) < 0)[0]:
            a, b = grid[i], grid[i + 1]
            fa = d[i]
            for _ in range(60):                                 # bisection on f'_{L-1}
                m = 0.5 * (a + b)
                fm = self._f(np.array([m]), deriv=1)[0, -1]
                if np.sign(fm) == np.sign(fa):
                    a, fa = m, fm
                else:
                    b = m
            roots.append(0.5 * (a + b))
        r = np.array(roots)
        x = np.concatenate([-r[::-1], [0.0], r]) if self.parity[-1] > 0 else np.concatenate([-r[::-1], r])
        if x.size < self.size:
            x = np.concatenate([[-1.0], x, [1.0]])
        return 0.5 * self.beta * (x + 1.0)

    def matsubara_points(self, nmax=None):
        """Sign changes of Uhat_{L-1} along n >= 0, mirrored to negative n."""
        if nmax is None:
            nmax = int(4 * self.lam) + 200
        n = np.arange(0, nmax + 1)
        h = self.uhat(n)[:, -1]              # real or imaginary by the parity of L-1
        part = h.real if np.abs(h.real).max() >= np.abs(h.imag).max() else h.imag
        ch = np.nonzero(np.sign(part[:-1]) * np.sign(part[1:]) < 0)[0]
        pos = list(n[ch])
        # fewer points than basis functions: add tail frequencies (twice the largest)
        while True:
            p = np.array(pos)
            pts = np.concatenate([-p[::-1] - 1, p]) if self.stat == "F" else np.unique(np.concatenate([-p[::-1], [0], p]))
            if pts.size >= self.size:
                return pts
            pos.append(2 * pos[-1] + 1)

    # ---------------------------------------------------------------- transforms
    def fit_tau(self, tau_pts, g_tau):
        """Coefficients g_l from values at the tau points (least squares)."""
        return np.linalg.lstsq(self.u(tau_pts), g_tau, rcond=None)[0]

    def fit_matsubara(self, n_pts, g_iw):
        """Coefficients g_l from values at the Matsubara points (least squares)."""
        return np.linalg.lstsq(self.uhat(n_pts), g_iw, rcond=None)[0]

    def transforms(self):
        """Sparse-sampling transforms between the default points: TF (tau values ->
        Matsubara values) and TB (Matsubara values -> tau values)."""
        tp, npts = self.tau_points(), self.matsubara_points()
        Ft, Fw = self.u(tp), self.uhat(npts)
        return tp, npts, Fw @ np.linalg.pinv(Ft), Ft @ np.linalg.pinv(Fw)


class IRGrid:
    """Sparse-sampling grid of one GW calculation on the IR basis, with the
    attributes the oracle's GW steps read from the Chebyshev grid (tau, wf, wb,
    TFf, TBf, TFb, TBb, l0, lb, r).

    One tau grid serves both statistics: the sampling points of the fermionic basis
    (G and Sigma~ live there; P~ is fitted in the bosonic basis at the same points).
    Fermionic and bosonic Matsubara points are each basis' own, so the transforms are
    rectangular: TFf = Uhat_F pinv(U_F(tau)) maps tau values to fermionic Matsubara
    values, TBf = U_F(tau) pinv(Uhat_F) back (least squares), likewise for bosons.
    lb and l0 are the rows U_F(beta^-) pinv(U_F(tau)) and U_F(0^+) pinv(U_F(tau)), so
    gamma = -G(beta^-) = -lb G(tau) as on the Chebyshev grid, and r = lb TBf gives the
    density from the Matsubara values.
    """

    def __init__(self, beta, lam, eps=1e-10):
        self.beta = float(beta)
        self.basis_f = IRBasis(lam, beta, "F", eps)
        self.basis_b = IRBasis(lam, beta, "B", eps)
        bf, bb = self.basis_f, self.basis_b
        self.tau = bf.tau_points()
        self.ntau = self.tau.size
        self.fermi_n = bf.matsubara_points()
        self.bose_m = bb.matsubara_points()
        self.wf = bf.freq(self.fermi_n)
        self.wb = bb.freq(self.bose_m)
        Ft, Fw = bf.u(self.tau), bf.uhat(self.fermi_n)
        Bt, Bw = bb.u(self.tau), bb.uhat(self.bose_m)
        self.TFf, self.TBf = Fw @ np.linalg.pinv(Ft), Ft @ np.linalg.pinv(Fw)
        self.TFb, self.TBb = Bw @ np.linalg.pinv(Bt), Bt @ np.linalg.pinv(Bw)
        ends = bf.u(np.array([0.0, self.beta])) @ np.linalg.pinv(Ft)
        self.l0, self.lb = ends[0], ends[1]
        self.r = self.lb @ self.TBf
