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


def dyson_G(H, Sig, mu, beta, fermionic=None, S=None):
    """Dyson equation, Eq. (dyson), with Sigma^inf = 0 (it enters through H):

      G^k(i w_n) = [(i w_n + mu) S^k - H^k - Sigma^k(i w_n)]^{-1},

    S = I unless the overlap S [nk][nao][nao] is given. Sigma(i w_n) = F^f Sigma(tau),
    G(tau) = B^f G(i w_n) on the fermionic grid: the Chebyshev one, or fermionic = (w_n, F^f, B^f)
    given (another tau grid, e.g. an IR grid).
    """
    nk, ntau, nao, _ = Sig.shape
    if fermionic is None:
        m, Ff, Bf = grids.transform_matrices(ntau, beta, 1)
        wn = (2 * m + 1) * np.pi / beta
    else:
        wn, Ff, Bf = fermionic
    Sw = to_matsubara(Sig, Ff)
    Gw = np.empty_like(Sw)
    eye = np.eye(nao)
    for k in range(nk):
        ov = eye if S is None else S[k]
        for n in range(len(wn)):
            Gw[k, n] = np.linalg.inv((1j * wn[n] + mu) * ov - H[k] - Sw[k, n])
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


# ---- the static part and the rest of the loop (Sec. 2.2 Eq. sigma_inf, Sec. 2.4, Sec. 5.3) ------


def density_matrix(G, beta):
    """gamma^k = G^k(0^-) = -G^k(beta^-) (antiperiodicity), the density matrix of Eq. (sigma_inf).

    The nodes exclude tau = beta, so G(beta^-) is the Chebyshev interpolant of the node values
    evaluated there: with x = 2 tau / beta - 1, x = 1 where every T_l(1) = 1, so
    G(beta^-) = sum_l c_l with c_l = (2 - delta_l0)/n sum_j G(tau_j) T_l(x_j).
    """
    nk, ntau = G.shape[:2]
    x = 2.0 * grids.chebyshev_nodes(ntau, beta) / beta - 1.0
    l = np.arange(ntau)
    T = np.cos(np.outer(l, np.arccos(np.clip(x, -1.0, 1.0))))    # T_l(x_j)
    coef = ((2.0 - (l == 0)) / ntau)[:, None] * T                  # c_l = sum_j coef[l, j] G_j
    g_beta = np.einsum("lj,kjab->kab", coef, G)                    # sum over l of c_l
    return -g_beta


def sigma_inf(V, gamma, nk3, spin_factor=2.0):
    """Static (Hartree-Fock) self-energy, Eq. (sigma_inf), with G(0^-) = gamma:

      Sigma^inf,k_ij = (s/N_k) sum_{k'Q ab} V_{ik,jk}(Q) gamma^{k'}_ab V_{bk',ak'}(Q)
                     - (1/N_k) sum_{k'Q ab} V_{ik,ak'}(Q) gamma^{k'}_ab V_{bk',jk}(Q),

    s the spin sum of the first (Hartree) term; the exchange term keeps one spin.
    """
    nk = V.shape[0]
    rho = sum(np.einsum("ab,Qba->Q", gamma[kp], V[kp, kp]) for kp in range(nk))
    out = np.empty((nk,) + gamma.shape[1:], complex)
    for k in range(nk):
        hartree = np.einsum("Qij,Q->ij", V[k, k], rho)
        exchange = sum(np.einsum("Qia,ab,Qbj->ij", V[k, kp], gamma[kp], V[kp, k], optimize=True)
                       for kp in range(nk))
        out[k] = (spin_factor * hartree - exchange) / nk
    return out


def particle_number(gamma, spin_factor=2.0, S=None):
    """Electrons per cell, (s/N_k) sum_k Re Tr gamma^k S^k (S = I unless given)."""
    nk = gamma.shape[0]
    if S is None:
        return float(np.real(spin_factor * np.einsum("kii->", gamma) / nk))
    return float(np.real(spin_factor * np.einsum("kij,kji->", gamma, S) / nk))


def dyson_G_static(H, sig_inf, Sig, mu, beta, S=None):
    """Eq. (dyson) with the static part: [(i w_n + mu) S^k - H^k - Sigma^inf,k - Sigma~^k(i w_n)]^{-1};
    the static part enters exactly like H, so this is dyson_G with H + Sigma^inf."""
    return dyson_G(H if sig_inf is None else H + sig_inf, Sig, mu, beta, S=S)


def find_mu(H, sig_inf, Sig, beta, n_target, spin_factor=2.0, lo=-5.0, hi=5.0, tol=1e-10, maxit=200, S=None):
    """Chemical potential with (s/N_k) sum_k Tr gamma^k S^k = n_target (Sec. 2.4, step 3), by
    bisection on the particle number of the Dyson solution, which grows with mu. Returns (mu, G)."""
    def number(mu):
        G = dyson_G_static(H, sig_inf, Sig, mu, beta, S)
        return particle_number(density_matrix(G, beta), spin_factor, S), G
    n_lo, _ = number(lo)
    n_hi, _ = number(hi)
    if not (n_lo <= n_target <= n_hi):
        raise ValueError("target particle number outside [N(lo), N(hi)]")
    for _ in range(maxit):
        mid = 0.5 * (lo + hi)
        n_mid, G = number(mid)
        if n_mid < n_target:
            lo = mid
        else:
            hi = mid
        if hi - lo < tol:
            break
    mu = 0.5 * (lo + hi)
    return mu, number(mu)[1]


def diis_coefficients(residuals):
    """Pulay's extrapolation coefficients (Sec. 5.3): c minimising |sum_i c_i r_i|^2 with
    sum_i c_i = 1, from B_ij = Re <r_i, r_j> and one Lagrange multiplier."""
    m = len(residuals)
    Bm = np.empty((m + 1, m + 1))
    for i in range(m):
        for j in range(m):
            Bm[i, j] = np.real(np.vdot(residuals[i], residuals[j]))
    Bm[m, :m] = Bm[:m, m] = -1.0
    Bm[m, m] = 0.0
    rhs = np.zeros(m + 1)
    rhs[m] = -1.0
    return np.linalg.solve(Bm, rhs)[:m]


def diis_extrapolate(outputs, inputs):
    """Next self-energy sum_i c_i Sigma[G_i] from the outputs Sigma[G_i] of the last iterations and
    the self-energies Sigma_i they were computed from (residual r_i = Sigma[G_i] - Sigma_i)."""
    c = diis_coefficients([o - x for o, x in zip(outputs, inputs)])
    return sum(ci * o for ci, o in zip(c, outputs)), c


def commutator_residual(H, sig_inf, Sig, G, beta, S=None):
    """Error vector of the commutator variant of DIIS (Sec. 5.3, after Pulay's SCF commutator
    F D S - S D F): with F^k(i w_n) = H^k + Sigma^inf,k + Sigma~^k(i w_n),
      e^k(i w_n) = S^k G^k(i w_n) F^k(i w_n) - F^k(i w_n) G^k(i w_n) S^k   (= [G, F] for S = I),
    G(i w) = F^f G(tau), Sigma~(i w) = F^f Sigma~(tau). A G that solves the Dyson equation with this
    very (Sigma^inf, Sigma~) and S makes it vanish, so e vanishes at self-consistency."""
    nk, ntau, nao, _ = G.shape
    _, Ff, _ = grids.transform_matrices(ntau, beta, 1)
    Gw = to_matsubara(G, Ff)
    Fw = to_matsubara(Sig, Ff) + (H + (0 if sig_inf is None else sig_inf))[:, None]
    if S is None:
        return Gw @ Fw - Fw @ Gw
    Sk = S[:, None]
    return Sk @ Gw @ Fw - Fw @ Gw @ Sk


def scgw_full(H, V, G0, nk3, beta, mu, spin_factor=2.0, alpha=0.5, tol=1e-6, itermax=10, static=True,
              n_electrons=None, mu_lo=-5.0, mu_hi=5.0, mu_tol=1e-10, diis_size=0, diis_start=2, diis_kind="diis",
              method="gw", S=None, resume=None):
    """The self-consistency loop of Sec. 2.4 with its four steps per iteration n:

      (1) the static part Sigma^inf[G_{n-1}] (Eq. sigma_inf; left out when static is False) and
          the dynamic part Sigma~[G_{n-1}] (Eq. sigma_gw, Eq. sigma2 with method "gf2", zero with
          method "hf") -- together the output F_n;
      (2) acceleration (Sec. 5.3): Sigma_1 = F_1; afterwards iteration mixing
          Sigma_n = alpha F_n + (1 - alpha) Sigma_{n-1}, or, with diis_size > 0, Pulay's
          extrapolation over the newest diis_size pairs (Sigma_{i-1}, F_i) from iteration
          diis_start on (the iterations before it mix and fill the subspace); the residual of
          a pair is F_i - Sigma_{i-1}, or with diis_kind "cdiis" the commutator
          [G_{i-1}(i w), H + F_i(i w)] (commutator_residual);
      (3) with n_electrons given, mu such that the Dyson solution holds n_electrons per cell;
      (4) G_n = Dyson(H + Sigma^inf_n, Sigma~_n, mu).

    The pair (Sigma^inf, Sigma~) is one vector for mixing, DIIS and the stopping test
    max |Sigma_n - Sigma_{n-1}| < tol; S is the overlap of Eq. (dyson) (identity when None).
    resume = (SigInf, Sig): continue a loop whose last Sigma_{n-1} these are (G0 the G built from
    them): the first iteration then mixes with them instead of taking F_1 as it is.
    Returns a dict with Sig (dynamic), SigInf, G, mu, iterations and hist (the max |dSigma| of
    iterations 2, 3, ...)."""
    nk, ntau, nao, _ = G0.shape
    G = G0
    prev = None                         # (SigInf, Sig) of the previous iteration
    if resume is not None:
        prev = np.concatenate([(resume[0] if static else np.zeros((nk, nao, nao), complex)).ravel(),
                               resume[1].ravel()])
    ins, outs = [], []                  # residuals and outputs of the DIIS subspace
    hist = []
    it = 0
    for it in range(1, itermax + 1):
        sinf = sigma_inf(V, density_matrix(G, beta), nk3, spin_factor) if static else np.zeros((nk, nao, nao), complex)
        if method == "gf2":
            from .gf2 import gf2_self_energy
            sdyn = gf2_self_energy(V, G, nk3, spin_factor)
        elif method == "hf":
            sdyn = np.zeros_like(G)                 # Hartree-Fock: the static part alone
        else:
            sdyn = sigma_eval(V, G, nk3, beta, spin_factor)["Sig"]
        out = np.concatenate([sinf.ravel(), sdyn.ravel()])
        if prev is None:
            cur = out
        else:
            if diis_size > 0:
                if diis_kind == "cdiis":
                    ins.append(commutator_residual(H, out[:nk * nao * nao].reshape(nk, nao, nao),
                                                   out[nk * nao * nao:].reshape(G0.shape), G, beta, S).ravel())
                else:
                    ins.append(out - prev)
                outs.append(out)
                ins, outs = ins[-diis_size:], outs[-diis_size:]
            if diis_size > 0 and it >= diis_start:
                c = diis_coefficients(ins)
                cur = sum(ci * o for ci, o in zip(c, outs))
            else:
                cur = mix(out, prev, alpha)
            hist.append(float(np.max(np.abs(cur - prev))))
        prev = cur
        sinf = cur[:nk * nao * nao].reshape(nk, nao, nao)
        sdyn = cur[nk * nao * nao:].reshape(G0.shape)
        if n_electrons is not None:
            mu, G = find_mu(H, sinf, sdyn, beta, n_electrons, spin_factor, lo=mu_lo, hi=mu_hi, tol=mu_tol, S=S)
        else:
            G = dyson_G_static(H, sinf, sdyn, mu, beta, S)
        if hist and hist[-1] < tol:
            break
    return {"Sig": sdyn, "SigInf": sinf, "G": G, "mu": mu, "iterations": it, "hist": hist}
