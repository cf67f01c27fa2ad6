"""Pins of the second-order self-energy (Eq. sigma2) in the oracle, each against something other
than the formula it implements: the second-order GW term built from the separately pinned
polarization and GW self-energy, the Pauli cancellation for one spin-orbital, a brute force
through explicit 4-index integrals, and Hermiticity."""
import numpy as np
import pytest

from oracle import gf2 as F
from oracle import gw as O
from paper_2406_18479_gb300 import inputs as I


def case(nk3, nao, naux, ntau, beta, seed, noise=0.02):
    w = I.Workload("gf2", nk3, nao, naux, ntau, ntau, beta, 0.1, 3.0, seed, solid=int(np.prod(nk3)) > 1)
    h, v, g = I.make_inputs(w)
    rng = np.random.default_rng(seed + 1)
    x = noise * (rng.standard_normal(g.shape) + 1j * rng.standard_normal(g.shape))
    return w, v, g + 0.5 * (x + x.conj().swapaxes(-1, -2))


@pytest.mark.parametrize("nk3", [(1, 1, 1), (2, 1, 1), (3, 1, 1), (2, 2, 1)])
def test_direct_term_is_the_second_order_gw_term(nk3):
    """GW expanded to first order in P0 (P~ = P0 + P0^2 + ...): Sigma_GW[P~ -> P0] is the direct
    second-order term, with its sign and normalisation."""
    w, v, g = case(nk3, 3, 4, 4, 4.0, 3)
    d, _ = F.gf2_terms(v, g, nk3, 2.0)
    p0 = O.polarization(v, g, nk3, 2.0)
    ref = O.self_energy(v, g, p0, nk3)
    assert np.abs(d - ref).max() < 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("naux", [1, 3])
def test_one_spin_orbital_has_no_second_order_term(naux):
    """Pauli: for a single spin-orbital (nao = 1, one k, s = 1) direct and exchange cancel."""
    w, v, g = case((1, 1, 1), 1, naux, 6, 5.0, 5)
    d, x = F.gf2_terms(v, g, (1, 1, 1), 1.0)
    assert np.abs(d).max() > 1e-6
    assert np.abs(d - x).max() < 1e-14 * np.abs(d).max()
    s = F.gf2_self_energy(v, g, (1, 1, 1), 2.0)            # two spins: the direct term survives once
    assert np.abs(s - d).max() < 1e-14 * np.abs(d).max()


def brute_force(V, G, nk3, s, t):
    """Eq. (sigma2) at one tau node through U^{k1 k2, k3 k4}_{ij, kl} = sum_Q V^{k1 k2}_ij(Q) V^{k3 k4}_kl(Q)
    and plain loops over every orbital index."""
    nk, ntau, nao = G.shape[0], G.shape[1], G.shape[2]

    def U(a, b, c, d):
        return np.tensordot(V[a, b], V[c, d], axes=([0], [0]))     # [i j k l]
    out = np.zeros((nk, nao, nao), complex)
    for k in range(nk):
        for k1 in range(nk):
            for k2 in range(nk):
                k3 = O.k_shift(nk3, O.k_shift(nk3, k1, k2, +1), k, -1)
                u1 = U(k, k1, k3, k2)             # (ip, mk) through Q
                ud = U(k1, k, k2, k3)             # (qj, ln) through Q'
                ux = U(k2, k, k1, k3)             # (lj, qn) through Q'
                g1, g2, g3 = G[k1, t], G[k2, t], G[k3, ntau - 1 - t]
                for i in range(nao):
                    for j in range(nao):
                        acc = 0j
                        for p in range(nao):
                            for q in range(nao):
                                for kk in range(nao):
                                    for l in range(nao):
                                        for m in range(nao):
                                            for n in range(nao):
                                                acc += (u1[i, p, m, kk] * (s * ud[q, j, l, n] - ux[l, j, q, n])
                                                        * g1[p, q] * g2[kk, l] * g3[n, m])
                        out[k, i, j] += acc / nk ** 2
    return out


@pytest.mark.parametrize("nk3", [(1, 1, 1), (2, 1, 1)])
def test_against_four_index_brute_force(nk3):
    w, v, g = case(nk3, 2, 2, 3, 3.0, 7)
    sig = F.gf2_self_energy(v, g, nk3, 2.0)
    for t in range(3):
        ref = brute_force(v, g, nk3, 2.0, t)
        assert np.abs(sig[:, t] - ref).max() < 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("nk3", [(1, 1, 1), (3, 1, 1)])
def test_hermitian(nk3):
    """Sigma(tau) is Hermitian for Hermitian G(tau) and V(k2,k1)^Q_ji = conj V(k1,k2)^Q_ij."""
    w, v, g = case(nk3, 3, 5, 4, 4.0, 11)
    sig = F.gf2_self_energy(v, g, nk3, 2.0)
    assert np.abs(sig - sig.conj().swapaxes(-1, -2)).max() < 1e-13 * np.abs(sig).max()


def test_gf2_loop_reaches_its_fixed_point():
    """The loop with the second-order self-energy: at convergence Sigma^inf and Sigma~ are those
    of G (Eq. sigma2), G holds n_electrons and solves the Dyson equation with them."""
    w = I.Workload("gf2loop", (2, 1, 1), 3, 6, 12, 12, 5.0, 0.0, 3.0, 21, solid=True)
    h, v, g = I.make_inputs(w)
    v = 0.4 * v
    r = O.scgw_full(h, v, g, w.nk3, w.beta, 0.0, alpha=0.7, tol=1e-10, itermax=60, n_electrons=2.0,
                    mu_tol=1e-13, diis_size=4, method="gf2")
    assert r["hist"][-1] < 1e-10
    gam = O.density_matrix(r["G"], w.beta)
    assert abs(O.particle_number(gam, 2.0) - 2.0) < 1e-9
    assert np.abs(O.sigma_inf(v, gam, w.nk3, 2.0) - r["SigInf"]).max() < 1e-8
    assert np.abs(F.gf2_self_energy(v, r["G"], w.nk3, 2.0) - r["Sig"]).max() < 1e-8
    assert np.abs(O.dyson_G(h + r["SigInf"], r["Sig"], r["mu"], w.beta) - r["G"]).max() < 1e-12
