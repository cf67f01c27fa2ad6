"""Second-order (GF2) self-energy, Eq. (sigma2), in plain complex128 (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Eq. (sigma2) restated with the readings used throughout this oracle:
  * G^{k3}(-tau) is taken antiperiodic, -G^{k3}(beta - tau), with beta - tau the mirrored
    node T-1-t; the momentum delta delta_{k+k3, k1+k2} is normalised to N_k (k3 is fixed by
    k, k1, k2). Together these give the overall factor +1/N_k^2 below, for which the direct
    term equals the GW self-energy with P~ replaced by P0 -- the second-order term GW and
    GF2 share (pinned in tests/test_oracle_gf2_pins.py);
  * the spin sum over sigma' gives the spin factor s on the direct term only (the exchange
    term carries delta_{sigma sigma'}).

  Sigma^k_ij(tau) = (1/N_k^2) sum_{k1 k2} sum_{QQ' klmnpq}
        [ s V^{k1 k}_qj(Q') V^{k2 k3}_ln(Q') - V^{k2 k}_lj(Q') V^{k1 k3}_qn(Q') ]
        V^{k k1}_ip(Q) V^{k3 k2}_mk(Q) G^{k1}_pq(tau) G^{k2}_kl(tau) G^{k3}_nm(beta - tau),
  k3 = k1 + k2 - k (modulo the mesh).
"""
from __future__ import annotations

import numpy as np

from .gw import k_shift


def gf2_terms(V, G, nk3, spin_factor=2.0, k_list=None, t_list=None):
    """(direct, exchange) parts of Eq. (sigma2), each [len(k_list)][len(t_list)][nao][nao], so
    that Sigma = direct - exchange; direct includes the spin factor."""
    nk, ntau, nao = G.shape[0], G.shape[1], G.shape[2]
    k_list = range(nk) if k_list is None else k_list
    t_list = range(ntau) if t_list is None else t_list
    d = np.zeros((len(k_list), len(t_list), nao, nao), complex)
    x = np.zeros_like(d)
    for ik, k in enumerate(k_list):
        for k1 in range(nk):
            for k2 in range(nk):
                k3 = k_shift(nk3, k_shift(nk3, k1, k2, +1), k, -1)
                for it, t in enumerate(t_list):
                    gm = G[k3, ntau - 1 - t]                      # G^{k3}(beta - tau)
                    # the Q-side factors V^{k k1}(Q) G^{k1} and V^{k3 k2}(Q) G^{k2}
                    vg1 = np.einsum("Qip,pq->Qiq", V[k, k1], G[k1, t])
                    vg2 = np.einsum("Qmk,kl->Qml", V[k3, k2], G[k2, t])
                    # direct: sum_{QR} [V G V](Q, R)_ij * Tr[V^{k3k2}(Q) G^{k2} V^{k2k3}(R) G^{k3}(beta - tau)]
                    m = np.einsum("Qiq,Rqj->QRij", vg1, V[k1, k])
                    bub = np.einsum("Qml,Rlm->QR", vg2, np.einsum("Rln,nm->Rlm", V[k2, k3], gm))
                    d[ik, it] += np.einsum("QRij,QR->ij", m, bub)
                    # exchange: sum_{QR} [V G](Q)_iq [V^{k1k3} G^{k3}(beta - tau)](R)_qm [V G](Q)_ml V^{k2k}_lj(R)
                    e = np.einsum("Qiq,Rqm->QiRm", vg1, np.einsum("Rqn,nm->Rqm", V[k1, k3], gm))
                    x[ik, it] += np.einsum("Ril,Rlj->ij", np.einsum("QiRm,Qml->Ril", e, vg2), V[k2, k])
    return spin_factor * d / nk ** 2, x / nk ** 2


def gf2_self_energy(V, G, nk3, spin_factor=2.0, k_list=None, t_list=None):
    """Eq. (sigma2): the direct minus the exchange term."""
    d, x = gf2_terms(V, G, nk3, spin_factor, k_list, t_list)
    return d - x
