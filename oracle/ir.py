"""Intermediate-representation (IR) grids, built from the singular value expansion of the
logistic kernel (oracle). TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper runs on IR grids with Lambda = beta omega_max = 1e4 (Sec. 3, grid files of its
distribution) or Chebyshev grids. The grid files are not available, so the grid is built here:

  K(x, y) = exp(-Lambda y (x + 1) / 2) / (1 + exp(-Lambda y)),  x = 2 tau / beta - 1, y = omega / omega_max,
  K(x, y) = sum_l s_l U_l(x) V_l(y)   (SVD on composite Gauss-Legendre panels refined towards
                                      x = +-1 and y = 0; U_l normalised on [-1, 1], with the
                                      parity (-1)^l imposed),
  u_l(tau) = sqrt(2 / beta) U_l(x),   u^_l(i nu) = int_0^beta e^{i nu tau} u_l(tau) dtau.

Readings (the paper gives only Lambda): the basis keeps the L functions with s_l / s_0 > eps;
the tau nodes are the L roots of U_L (symmetric, so beta - tau_j = tau_{L-1-j}); the Matsubara
samples are where the non-vanishing part of u^_L(i nu_n) changes sign on n >= 0, taken at the
side of smaller magnitude, mirrored (fermionic n -> -n-1, bosonic n -> -n), and trimmed from
the top, or padded (one point at a time: a gap's log-midpoint or half again beyond the last,
whichever gives the smallest ||F||_F ||F^+||_F) to the count of the library's symmetric sets (ntau, or
ntau + 1 when the parity differs). F = u^(samples) U_tau^{-1} maps node values to Matsubara
values, B is its least-squares left inverse; for bosons F[nw-1-n][L-1-t] = F[n][t] (and the same
for B) is imposed exactly.
"""
from __future__ import annotations

import numpy as np

NGL = 16


def _panels(J):
    """Breakpoints on [-1, 1]: 0 and +-(1 - 2^-j), j = 1..J, and +-1."""
    pos = [1.0 - 2.0 ** (-j) for j in range(1, J + 1)]
    return np.array(sorted(set([-1.0, 0.0, 1.0] + pos + [-p for p in pos])))


def _panels_y(J):
    """Breakpoints on [-1, 1] refined towards y = 0: +-2^-j, j = 0..J, and 0."""
    pos = [2.0 ** (-j) for j in range(0, J + 1)]
    return np.array(sorted(set([0.0] + pos + [-p for p in pos])))


def _gauss(edges):
    t, w = np.polynomial.legendre.leggauss(NGL)
    lo, hi = edges[:-1], edges[1:]
    x = (0.5 * (hi - lo)[:, None] * (t[None, :] + 1.0) + lo[:, None]).ravel()
    wx = (0.5 * (hi - lo)[:, None] * w[None, :]).ravel()
    return x, wx


def logistic(x, y, lam):
    x, y = np.meshgrid(x, y, indexing="ij")
    out = np.empty_like(x)
    p = y >= 0
    out[p] = np.exp(-0.5 * lam * y[p] * (x[p] + 1.0)) / (1.0 + np.exp(-lam * y[p]))
    out[~p] = np.exp(0.5 * lam * y[~p] * (1.0 - x[~p])) / (1.0 + np.exp(lam * y[~p]))
    return out


class Basis:
    """U_l on the x panels (values at the Gauss nodes), s_l, and the size L."""

    def __init__(self, lam, eps):
        J = int(np.ceil(np.log2(max(lam, 2.0)))) + 1
        self.edges = _panels(J)
        x, wx = _gauss(self.edges)
        y, wy = _gauss(_panels_y(J))
        A = np.sqrt(wx)[:, None] * logistic(x, y, lam) * np.sqrt(wy)[None, :]
        u, s, _ = np.linalg.svd(A, full_matrices=False)
        self.s = s
        self.L = int(np.sum(s / s[0] > eps))
        U = u[:, : self.L + 1] / np.sqrt(wx)[:, None]       # U_l at the nodes, l = 0..L
        U *= np.sign(U[-1])[None, :]                         # U_l(1) > 0
        # parity U_l(-x) = (-1)^l U_l(x), exact (the nodes are mirror images); the SVD in double
        # precision meets it only to about 1e-16 s_0 / (s_l - s_l+1) near the cut-off
        U = 0.5 * (U + ((-1.0) ** np.arange(self.L + 1))[None, :] * U[::-1])
        self.x, self.U = x, U
        self.lam = lam
        # Legendre coefficients per panel: U_l(x) = sum_m c[p, m, l] P_m(t) on panel p
        t, w = np.polynomial.legendre.leggauss(NGL)
        P = np.polynomial.legendre.legvander(t, NGL - 1)           # [node][m]
        proj = (P * w[:, None]).T * ((2 * np.arange(NGL) + 1) / 2.0)[:, None]   # [m][node]
        self.c = np.einsum("mn,pnl->pml", proj, U.reshape(len(self.edges) - 1, NGL, -1))

    def eval(self, l, xq):
        """U_l at the points xq (the panel's Legendre series)."""
        xq = np.atleast_1d(xq)
        p = np.clip(np.searchsorted(self.edges, xq, side="right") - 1, 0, len(self.edges) - 2)
        a, b = self.edges[p], self.edges[p + 1]
        t = (2 * xq - a - b) / (b - a)
        return np.array([np.polynomial.legendre.legval(t[i], self.c[p[i], :, l]) for i in range(len(xq))])

    def fourier(self, nu_beta):
        """int_{-1}^{1} e^{i nu beta (x + 1) / 2} U_l(x) dx for l = 0..L, at the values nu * beta:
        per panel sum_m c_m int P_m(t) e^{i kappa t} dt = sum_m c_m 2 i^m j_m(kappa)."""
        from scipy.special import spherical_jn
        nu_beta = np.atleast_1d(np.asarray(nu_beta, float))
        a, b = self.edges[:-1], self.edges[1:]
        kappa = np.outer(nu_beta, (b - a) / 4.0)                    # [n][p]
        phase = np.exp(1j * np.outer(nu_beta, ((a + b) / 2.0 + 1.0) / 2.0))
        m = np.arange(NGL)
        jm = spherical_jn(m[None, None, :], kappa[:, :, None])      # [n][p][m]
        I = 2.0 * (1j ** m)[None, None, :] * jm * ((b - a) / 2.0)[None, :, None] * phase[:, :, None]
        return np.einsum("npm,pml->nl", I, self.c)


def _roots(basis, l):
    """Roots of U_l on (-1, 1): sign changes on a fine scan, refined by bisection."""
    xs = np.concatenate([np.linspace(basis.edges[p], basis.edges[p + 1], 64, endpoint=False)
                         for p in range(len(basis.edges) - 1)] + [np.array([1.0])])
    v = basis.eval(l, xs)
    out = []
    for i in np.nonzero(np.sign(v[:-1]) * np.sign(v[1:]) < 0)[0]:
        a, b, fa = xs[i], xs[i + 1], v[i]
        for _ in range(60):
            m = 0.5 * (a + b)
            fm = basis.eval(l, m)[0]
            if np.sign(fm) == np.sign(fa):
                a, fa = m, fm
            else:
                b = m
        out.append(0.5 * (a + b))
    return np.array(out)


def _conditioning(F):
    """||F||_F ||F^+||_F, the conditioning measure of the padding choice."""
    return float(np.linalg.norm(F) * np.linalg.norm(np.linalg.pinv(F, rcond=1e-14)))


def sample_count(ntau, stat):
    want_odd = stat == 0
    return ntau if (ntau % 2 == 1) == want_odd else ntau + 1


def ir_grid(beta, lam, eps, stat):
    """(tau [L], Matsubara indices m [nw], F [nw][L], B [L][nw]) of the IR grid."""
    basis = Basis(lam, eps)
    L = basis.L
    x = _roots(basis, L)
    x = 0.5 * (x - x[::-1])                                          # exact mirror symmetry
    tau = 0.5 * beta * (x + 1.0)
    nw = sample_count(L, stat)
    # sign changes of the non-vanishing part of u^_L on n >= 0
    nmax = int(np.ceil(4.0 * lam / (2 * np.pi))) + 2 * L
    n = np.arange(nmax)
    nu_beta = (2 * n + 1) * np.pi if stat == 1 else 2 * n * np.pi
    f = basis.fourier(nu_beta)[:, L]
    g = f.imag if np.abs(f.imag).max() > np.abs(f.real).max() else f.real
    sel = []
    for i in range(len(n) - 1):
        if np.sign(g[i]) * np.sign(g[i + 1]) < 0:
            sel.append(int(n[i] if abs(g[i]) < abs(g[i + 1]) else n[i + 1]))
    if stat == 0 and 0 not in sel:
        sel = [0] + sel
    sel = sorted(set(sel))
    # the symmetric set: fermionic n and -n-1, bosonic n and -n (0 once)
    def full(s):
        if stat == 1:
            return sorted(set(s + [-k - 1 for k in s]))
        return sorted(set(s + [-k for k in s]))
    Ut = np.sqrt(2.0 / beta) * np.stack([basis.eval(l, x) for l in range(L)], axis=1)   # [tau][l]
    Uinv = np.linalg.inv(Ut)

    def transform(mm):
        mm = np.array(mm)
        nub = (2 * mm + 1) * np.pi if stat == 1 else 2 * mm * np.pi
        return np.sqrt(beta / 2.0) * basis.fourier(nub)[:, :L] @ Uinv   # u^_l(i nu) U_tau^{-1}

    m = full(sel)
    while len(m) > nw:
        sel = sel[:-1]
        m = full(sel)
    while len(m) < nw:
        # one more sample: the candidate (a gap's log-midpoint, or half again beyond the last) with
        # the smallest ||F||_F ||F^+||_F
        pos = [k for k in sel if k > 0] or [0]
        cands = {int(round(np.sqrt((a + 1.0) * (b + 1.0)) - 1.0)) for a, b in zip(pos[:-1], pos[1:]) if b - a > 1}
        cands.add(int(1.5 * max(pos)) + 1)
        best = min((_conditioning(transform(full(sorted(sel + [c])))), c) for c in cands if c not in sel)
        sel = sorted(sel + [best[1]])
        m = full(sel)
    m = np.array(m)
    F = transform(m)
    if stat == 0:        # F[nw-1-n][L-1-t] = F[n][t] exactly (it holds to rounding amplified by U_tau^-1)
        F = 0.5 * (F + F[::-1, ::-1])
    B = np.linalg.pinv(F, rcond=1e-14)
    if stat == 0:
        B = 0.5 * (B + B[::-1, ::-1])
    return tau, m, F, B
