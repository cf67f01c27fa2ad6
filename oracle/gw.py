"""GW self-energy, step by step, in plain complex128 (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Array layouts (row-major):
  V   [nk][nk][naux][nao][nao]   V[k1][k2][Q][i][j] = V_{k1 i, k2 j}(Q)   (Eq. CoulombDF)
  G   [nk][ntau][nao][nao]       G^k_ij(tau_t)
  P   [nk][ntau|nomega][naux][naux]   indexed by q
  Sig [nk][ntau][nao][nao]

Readings of the paper used here (each one is listed in the design notes):
  * G^k(-tau) in Eq. (tilde_P0_tau) is the stored array at beta - tau, i.e. the
    mirrored node t -> ntau-1-t of the symmetric Chebyshev grid (no antiperiodic
    minus sign). This makes P0(i Omega_0) negative semidefinite (screening).
  * The spin sum of Eq. (tilde_P0_tau) is a factor spin_factor (2 for a
    spin-restricted G); Eq. (sigma_gw) carries one spin and no factor.
  * k + q and k - q are taken modulo the Gamma-centred mesh.
  * W~ is never transformed: P~ is transformed back to tau, then contracted
    (Eqs. sigma_gw, tilde_W_DF2 are linear in P~).
"""
from __future__ import annotations

import numpy as np

from . import grids


def k_shift(nk3, k: int, q: int, sign: int) -> int:
    """Index of k + sign*q modulo the mesh (flat index (n1*N2+n2)*N3+n3)."""
    n1, n2, n3 = nk3
    a = np.array(np.unravel_index(k, (n1, n2, n3)))
    b = np.array(np.unravel_index(q, (n1, n2, n3)))
    c = (a + sign * b) % np.array([n1, n2, n3])
    return int(np.ravel_multi_index(tuple(c), (n1, n2, n3)))


def polarization(V, G, nk3, spin_factor=2.0, q_list=None, t_list=None):
    """Bare auxiliary polarization, Eq. (tilde_P0_tau), Sec. 2.3:

      P0^q_QQ'(tau) = -(s/N_k) sum_k sum_abcd V^{k,k+q}_da(Q) G^k_cd(beta-tau)
                                             G^{k+q}_ab(tau) V^{k+q,k}_bc(Q')

    Returns P0[len(q_list)][len(t_list)][naux][naux].
    """
    nk = V.shape[0]
    naux = V.shape[2]
    ntau = G.shape[1]
    q_list = range(nk) if q_list is None else q_list
    t_list = range(ntau) if t_list is None else t_list
    out = np.zeros((len(q_list), len(t_list), naux, naux), complex)
    for iq, q in enumerate(q_list):
        for it, t in enumerate(t_list):
            acc = np.zeros((naux, naux), complex)
            for k in range(nk):
                kq = k_shift(nk3, k, q, +1)
                g_minus = G[k, ntau - 1 - t]          # G^k(beta - tau)
                acc += np.einsum("Qda,cd,ab,Pbc->QP", V[k, kq], g_minus, G[kq, t], V[kq, k],
                                 optimize=True)
            out[iq, it] = -(spin_factor / nk) * acc
    return out


def to_matsubara(x_tau, F):
    """X(i w_n) = sum_t F_nt X(tau_t) along axis 1 (Eq. P0t_to_P0w on the grid)."""
    return np.einsum("nt,qt...->qn...", F, x_tau)


def to_tau(x_w, B):
    """X(tau_t) = sum_n B_tn X(i w_n) along axis 1 (inverse of to_matsubara)."""
    return np.einsum("tn,qn...->qt...", B, x_w)


def aux_dyson(P0w):
    """Renormalized auxiliary function, Eq. (tilde_P_omega): P = (I - P0)^{-1} P0,
    per (q, Omega_n), by LU with partial pivoting (numpy.linalg.solve)."""
    naux = P0w.shape[-1]
    eye = np.eye(naux)
    out = np.empty_like(P0w)
    for q in range(P0w.shape[0]):
        for n in range(P0w.shape[1]):
            out[q, n] = np.linalg.solve(eye - P0w[q, n], P0w[q, n])
    return out


def screened_interaction(P0t, F, B):
    """P0(tau) -> P0(i Omega) -> P~(i Omega) -> P~(tau); returns (P0w, Pw, Pt)."""
    P0w = to_matsubara(P0t, F)
    Pw = aux_dyson(P0w)
    Pt = to_tau(Pw, B)
    return P0w, Pw, Pt


def self_energy(V, G, Pt, nk3, k_list=None, t_list=None, q_list=None):
    """GW self-energy, Eqs. (sigma_gw) and (tilde_W_DF2), Sec. 2.3:

      Sigma^k_ij(tau) = -(1/N_k) sum_q sum_ab G^{k-q}_ab(tau) W~^{k,k-q,k-q,k}_{iabj}(tau),
      W~_{iabj} = sum_QQ' V^{k,k-q}_ia(Q) P~^q_QQ'(tau) V^{k-q,k}_bj(Q').

    Returns Sig[len(k_list)][len(t_list)][nao][nao]; q_list restricts the sum over q
    (the contribution of a subset of q, as one rank of a q-sharded run computes it).
    """
    nk = V.shape[0]
    nao = V.shape[3]
    ntau = G.shape[1]
    k_list = range(nk) if k_list is None else k_list
    t_list = range(ntau) if t_list is None else t_list
    q_list = range(nk) if q_list is None else q_list
    out = np.zeros((len(k_list), len(t_list), nao, nao), complex)
    for ik, k in enumerate(k_list):
        for it, t in enumerate(t_list):
            acc = np.zeros((nao, nao), complex)
            for q in q_list:
                kmq = k_shift(nk3, k, q, -1)
                acc += np.einsum("Qia,ab,QP,Pbj->ij", V[k, kmq], G[kmq, t], Pt[q, t], V[kmq, k],
                                 optimize=True)
            out[ik, it] = -acc / nk
    return out


def sigma_eval(V, G, nk3, beta, spin_factor=2.0):
    """One GW self-energy evaluation: P0(tau), P~(tau), Sigma(tau)."""
    ntau = G.shape[1]
    _, F, B = grids.transform_matrices(ntau, beta, 0)
    P0t = polarization(V, G, nk3, spin_factor)
    P0w, Pw, Pt = screened_interaction(P0t, F, B)
    Sig = self_energy(V, G, Pt, nk3)
    return {"P0t": P0t, "P0w": P0w, "Pw": Pw, "Pt": Pt, "Sig": Sig}


def dyson_G(H, Sig, mu, beta):
    """Dyson equation, Eq. (dyson), with S = I and Sigma^inf = 0:

      G^k(i w_n) = [(i w_n + mu) I - H^k - Sigma^k(i w_n)]^{-1},

    Sigma(i w_n) = F^f Sigma(tau), G(tau) = B^f G(i w_n) on the fermionic grid.
    """
    nk, ntau, nao, _ = Sig.shape
    m, Ff, Bf = grids.transform_matrices(ntau, beta, 1)
    wn = (2 * m + 1) * np.pi / beta
    Sw = to_matsubara(Sig, Ff)
    Gw = np.empty_like(Sw)
    eye = np.eye(nao)
    for k in range(nk):
        for n in range(len(wn)):
            Gw[k, n] = np.linalg.inv((1j * wn[n] + mu) * eye - H[k] - Sw[k, n])
    return to_tau(Gw, Bf)


def mix(sig_new, sig_old, alpha):
    """Iteration mixing, Sec. 5.3: Sigma_n = alpha Sigma[G_{n-1}] + (1 - alpha) Sigma_{n-1}."""
    return alpha * sig_new + (1.0 - alpha) * sig_old


def scgw(H, V, G0, nk3, beta, mu, spin_factor=2.0, alpha=0.5, tol=1e-6, itermax=10):
    """Self-consistency loop of Sec. 2.4 at fixed mu with Sigma^inf = 0.

    Iteration 1 takes Sigma_1 = Sigma[G0] unmixed; later iterations mix with alpha.
    Stops when max |Sigma_n - Sigma_{n-1}| < tol or after itermax evaluations.
    Returns (Sigma, G, history of max |dSigma|).
    """
    G = G0
    sig_old = None
    hist = []
    for it in range(itermax):
        sig_new = sigma_eval(V, G, nk3, beta, spin_factor)["Sig"]
        sig = sig_new if sig_old is None else mix(sig_new, sig_old, alpha)
        if sig_old is not None:
            d = float(np.max(np.abs(sig - sig_old)))
            hist.append(d)
        sig_old = sig
        G = dyson_G(H, sig, mu, beta)
        if hist and hist[-1] < tol:
            break
    return sig_old, G, hist
