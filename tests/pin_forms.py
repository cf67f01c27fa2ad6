"""Independent closed forms and brute-force references that pin the oracle.

None of this code is shared with oracle/ or with the CUDA path; each function
derives its result a different way from the same equations of the paper
(arXiv 2406.18479, Sec. 2):

* pole_form_p0_tau      Eq. (tilde_P0_tau) with G = G0 written in the eigenbasis
* pole_pair_p0_iw       Eq. (P0t_to_P0w) of that, integrated analytically
* brute_force_sigma     Eqs. (sigma_gw), (tilde_W_DF2), (tilde_P_omega) with the full
                        4-index integrals U = sum_Q V V of Eq. (CoulombDF), the RPA
                        solved in pair space (push-through identity)
* t_nl_exact            Eq. (P0t_to_P0w) of a Chebyshev polynomial by repeated
                        integration by parts, in 80-digit decimal arithmetic
"""
from __future__ import annotations

import decimal
import fractions

import numpy as np


def mesh_shift(nk3, k, q, sign):
    n1, n2, n3 = nk3
    k3 = (k // (n2 * n3), (k // n3) % n2, k % n3)
    q3 = (q // (n2 * n3), (q // n3) % n2, q % n3)
    c = [(k3[i] + sign * q3[i]) % nk3[i] for i in range(3)]
    return (c[0] * n2 + c[1]) * n3 + c[2]


def fermi(e, beta):
    """f(e) = 1/(1 + e^{beta e}) without overflow."""
    e = np.asarray(e, float)
    out = np.empty_like(e)
    pos = e >= 0
    out[pos] = np.exp(-beta * e[pos]) / (1.0 + np.exp(-beta * e[pos]))
    out[~pos] = 1.0 / (1.0 + np.exp(beta * e[~pos]))
    return out


def _eig(H, mu):
    ev, U = np.linalg.eigh(H)
    return ev - mu, U


def pole_form_p0_tau(H, V, nk3, beta, mu, tau, s):
    """P0^q_QQ'(tau) = -(s/N_k) sum_k sum_nm Vt_nm(Q) Vt'_mn(Q') f^k_n (1 - f^{k+q}_m)
    e^{(e^k_n - e^{k+q}_m) tau}, with Vt = U_k^+ V^{k,k+q} U_{k+q}, Vt' = U_{k+q}^+ V^{k+q,k} U_k.

    Each factor is a product of two bounded numbers:
    f_n e^{e_n tau} = e^{-e_n (beta - tau)} (1 - f_n) and (1 - f_m) e^{-e_m tau}.
    """
    nk = V.shape[0]
    naux = V.shape[2]
    eig = [_eig(H[k], mu) for k in range(nk)]
    out = np.zeros((nk, len(tau), naux, naux), complex)

    def occ_part(e, t):      # f(e) e^{e t}, bounded
        return np.where(e < 0, np.exp(e * t) / (1 + np.exp(beta * np.minimum(e, 0))),
                        np.exp(-e * (beta - t)) / (1 + np.exp(-beta * np.maximum(e, 0))))

    def emp_part(e, t):      # (1 - f(e)) e^{-e t}, bounded
        return np.where(e >= 0, np.exp(-e * t) / (1 + np.exp(-beta * np.maximum(e, 0))),
                        np.exp(e * (beta - t)) / (1 + np.exp(beta * np.minimum(e, 0))))

    for q in range(nk):
        for k in range(nk):
            kq = mesh_shift(nk3, k, q, +1)
            en, Un = eig[k]
            em, Um = eig[kq]
            vt = np.einsum("dn,Qda,am->Qnm", Un.conj(), V[k, kq], Um)
            vtp = np.einsum("bm,Qbc,cn->Qmn", Um.conj(), V[kq, k], Un)
            for it, t in enumerate(tau):
                w = occ_part(en, t)[:, None] * emp_part(em, t)[None, :]     # [n][m]
                out[q, it] += np.einsum("Qnm,nm,Pmn->QP", vt, w, vtp)
    return -(s / nk) * out


def pole_pair_p0_iw(H, V, nk3, beta, mu, omegas, s):
    """P0^q(i W) = (s/N_k) sum_k sum_nm Vt_nm(Q) Vt'_mn(Q') (f_n - f_m)/(i W + e_n - e_m),
    the analytic integral of pole_form_p0_tau over [0, beta]; where W = 0 and e_n = e_m
    the ratio is replaced by its limit -beta f (1 - f)."""
    nk = V.shape[0]
    naux = V.shape[2]
    eig = [_eig(H[k], mu) for k in range(nk)]
    out = np.zeros((nk, len(omegas), naux, naux), complex)
    for q in range(nk):
        for k in range(nk):
            kq = mesh_shift(nk3, k, q, +1)
            en, Un = eig[k]
            em, Um = eig[kq]
            fn, fm = fermi(en, beta), fermi(em, beta)
            vt = np.einsum("dn,Qda,am->Qnm", Un.conj(), V[k, kq], Um)
            vtp = np.einsum("bm,Qbc,cn->Qmn", Um.conj(), V[kq, k], Un)
            de = en[:, None] - em[None, :]
            df = fn[:, None] - fm[None, :]
            for iw, W in enumerate(omegas):
                den = 1j * W + de
                small = np.abs(den) < 1e-12
                w = np.where(small, 0.0, df / np.where(small, 1.0, den))
                if np.any(small):   # limit (f_n - f_m)/(e_n - e_m) -> -beta f (1 - f)
                    w = w + np.where(small, -beta * fn[:, None] * (1 - fn[:, None]), 0.0)
                out[q, iw] += np.einsum("Qnm,nm,Pmn->QP", vt, w, vtp)
    return (s / nk) * out


def brute_force_sigma(V, G, nk3, F, B, s):
    """Sigma^k(tau) from 4-index integrals, without the auxiliary basis.

    For each q, pair index alpha = (k, d, a): the bubble
      chi[(k,d,a),(k,b,c)](tau) = -(s/N_k) G^{k+q}_ab(tau) G^k_cd(beta - tau),
    transformed with F; then W~(i W) = U_XL (I - chi U_RL)^{-1} chi U_RY with
      U_XL[(k,i,a),(k',d',a')] = U^{k,k-q,k',k'+q}_{ia,d'a'},
      U_RL[(k,b,c),(k',d',a')] = U^{k+q,k,k',k'+q}_{bc,d'a'},
      U_RY[(k,b,c),(k'',b',j)] = U^{k+q,k,k''-q,k''}_{bc,b'j},
      U^{k1k2k3k4}_{ijkl} = sum_Q V^{k1k2}_ij(Q) V^{k3k4}_kl(Q)   (no conjugation),
    back with B, and Sigma^k_ij = -(1/N_k) sum_q sum_ab G^{k-q}_ab W~[(k,i,a),(k,b,j)].
    """
    nk, _, naux, nao, _ = V.shape
    ntau = G.shape[1]
    P = nao * nao
    D = nk * P

    def U(k1, k2, k3, k4):
        return np.einsum("Qij,Qkl->ijkl", V[k1, k2], V[k3, k4]).reshape(P, P)

    sig = np.zeros((nk, ntau, nao, nao), complex)
    for q in range(nk):
        plus = [mesh_shift(nk3, k, q, +1) for k in range(nk)]
        minus = [mesh_shift(nk3, k, q, -1) for k in range(nk)]
        chi_t = np.zeros((ntau, D, D), complex)
        for k in range(nk):
            for t in range(ntau):
                blk = np.einsum("ab,cd->dabc", G[plus[k], t], G[k, ntau - 1 - t])
                chi_t[t, k * P:(k + 1) * P, k * P:(k + 1) * P] = -(s / nk) * blk.reshape(P, P)
        u_xl = np.zeros((D, D), complex)
        u_rl = np.zeros((D, D), complex)
        u_ry = np.zeros((D, D), complex)
        for k in range(nk):
            for kp in range(nk):
                u_xl[k * P:(k + 1) * P, kp * P:(kp + 1) * P] = U(k, minus[k], kp, plus[kp])
                u_rl[k * P:(k + 1) * P, kp * P:(kp + 1) * P] = U(plus[k], k, kp, plus[kp])
                u_ry[k * P:(k + 1) * P, kp * P:(kp + 1) * P] = U(plus[k], k, minus[kp], kp)
        chi_w = np.einsum("nt,tij->nij", F, chi_t)
        w_w = np.empty_like(chi_w)
        for n in range(chi_w.shape[0]):
            w_w[n] = u_xl @ np.linalg.solve(np.eye(D) - chi_w[n] @ u_rl, chi_w[n] @ u_ry)
        w_t = np.einsum("tn,nij->tij", B, w_w)
        for k in range(nk):
            for t in range(ntau):
                blk = w_t[t, k * P:(k + 1) * P, k * P:(k + 1) * P].reshape(nao, nao, nao, nao)  # [i,a,b,j]
                sig[k, t] += -np.einsum("ab,iabj->ij", G[minus[k], t], blk) / nk
    return sig


# ---- exact Fourier integrals of Chebyshev polynomials -----------------------------------

def _dec_pi(prec):
    """pi to prec digits (Machin's formula) in decimal arithmetic."""
    decimal.getcontext().prec = prec + 10

    def arctan_inv(x):
        x = decimal.Decimal(x)
        term = 1 / x
        total = term
        x2 = x * x
        n = 1
        sign = -1
        while True:
            term /= x2
            t = term / (2 * n + 1)
            if t == 0 or abs(t) < decimal.Decimal(10) ** (-(prec + 8)):
                break
            total += sign * t
            sign = -sign
            n += 1
        return total
    return 4 * (4 * arctan_inv(5) - arctan_inv(239))


def t_nl_exact(m, l, stat, prec=80):
    """(1/beta) int_0^beta T_l(2 tau/beta - 1) e^{i w_m tau} dtau, w_m = (2m+stat) pi/beta,
    as a Python complex, from the exact finite sum of repeated integration by parts:

      sum_{j=0}^{l} (-1)^j (2/beta)^j [e^{i w beta} T_l^{(j)}(1) - T_l^{(j)}(-1)] / (i w)^{j+1},
      T_l^{(j)}(1) = prod_{r<j} (l^2 - r^2)/(2r+1),  T_l^{(j)}(-1) = (-1)^{l+j} T_l^{(j)}(1),
      e^{i w beta} = (-1)^stat.

    w = 0 (bosonic m = 0): int_{-1}^{1} T_l / 2 = (1 + (-1)^l) / (2 (1 - l^2)), l != 1.
    """
    nu = 2 * m + stat
    if nu == 0:
        if l == 1:
            return 0j
        return complex(fractions.Fraction(1 + (-1) ** l, 2 * (1 - l * l)))
    pi = _dec_pi(prec)
    re = decimal.Decimal(0)
    im = decimal.Decimal(0)
    d1 = fractions.Fraction(1)
    ewb = (-1) ** stat
    for j in range(l + 1):
        if j > 0:
            d1 *= fractions.Fraction(l * l - (j - 1) * (j - 1), 2 * (j - 1) + 1)
        if d1 == 0:
            break
        dm1 = d1 * (-1) ** (l + j)
        # with beta = 1: (-1)^j 2^j [ewb d1 - dm1] / (i nu pi)^{j+1}
        num = fractions.Fraction((-1) ** j * 2 ** j) * (ewb * d1 - dm1)
        if num == 0:
            continue
        val = decimal.Decimal(num.numerator) / decimal.Decimal(num.denominator)
        val /= (decimal.Decimal(nu) * pi) ** (j + 1)
        # 1/i^{j+1}: j+1 mod 4 = 0 -> 1, 1 -> -i, 2 -> -1, 3 -> i
        r = (j + 1) % 4
        if r == 0:
            re += val
        elif r == 1:
            im -= val
        elif r == 2:
            re -= val
        else:
            im += val
    return complex(float(re), float(im))
