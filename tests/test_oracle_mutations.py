"""Planted mistakes in the oracle must fail at least one pin.

Each case replaces one oracle function (on the CPU, via monkeypatch) by a
plausible wrong variant and checks that the pin comparisons of
test_oracle_pins.py no longer hold.
"""
import numpy as np
import pytest

from oracle import grids, gw
import pin_forms as PF
from test_oracle_pins import generic_inputs, rel, small_workload


def _pol_variant(mirror=True, sign=+1, s_factor=1.0):
    def pol(V, G, nk3, spin_factor=2.0, q_list=None, t_list=None):
        nk, naux, ntau = V.shape[0], V.shape[2], G.shape[1]
        out = np.zeros((nk, ntau, naux, naux), complex)
        for q in range(nk):
            for t in range(ntau):
                for k in range(nk):
                    kq = gw.k_shift(nk3, k, q, sign)
                    gm = G[k, ntau - 1 - t] if mirror else G[k, t]
                    out[q, t] += np.einsum("Qda,cd,ab,Pbc->QP", V[k, kq], gm, G[kq, t], V[kq, k])
                out[q, t] *= -(spin_factor * s_factor / nk)
        return out
    return pol


def _sig_variant(conj_right=False, transpose_p=False, sign=-1):
    def sig(V, G, Pt, nk3, k_list=None, t_list=None):
        nk, nao, ntau = V.shape[0], V.shape[3], G.shape[1]
        out = np.zeros((nk, ntau, nao, nao), complex)
        for k in range(nk):
            for t in range(ntau):
                for q in range(nk):
                    kmq = gw.k_shift(nk3, k, q, sign)
                    vr = V[kmq, k].conj() if conj_right else V[kmq, k]
                    p = Pt[q, t].T if transpose_p else Pt[q, t]
                    out[k, t] += np.einsum("Qia,ab,QP,Pbj->ij", V[k, kmq], G[kmq, t], p, vr)
                out[k, t] *= -1.0 / nk
        return out
    return sig


def _pins_hold():
    """The pole-form, brute-force and scalar pins, as booleans."""
    ok = []
    nk3 = (3, 1, 1)
    w = small_workload(nk3=nk3, nao=2, naux=3, ntau=10, beta=5.0)
    h, v, g = generic_inputs(w, rng_seed=7)
    tau = PF.np.array(grids.chebyshev_nodes(w.ntau, w.beta))
    ok.append(rel(gw.polarization(v, g, nk3, 2.0), PF.pole_form_p0_tau(h, v, nk3, w.beta, 0.0, tau, 2.0)) < 1e-13)
    r = gw.sigma_eval(v, g, nk3, w.beta, 2.0)
    _, F, B = grids.transform_matrices(w.ntau, w.beta, 0)
    ok.append(rel(r["Sig"], PF.brute_force_sigma(v, g, nk3, F, B, 2.0)) < 1e-12)
    beta, eps, vv = 10.0, 0.3, 0.7
    hh = np.array([[[eps]]], complex)
    v1 = np.full((1, 1, 1, 1, 1), vv, complex)
    g1 = PF.np.array(__import__("paper_2406_18479_gb300.inputs", fromlist=["g0_tau"]).g0_tau(
        hh, 0.0, beta, grids.chebyshev_nodes(20, beta)))
    r1 = gw.sigma_eval(v1, g1, (1, 1, 1), beta, 2.0)
    f = PF.fermi(np.array([eps]), beta)[0]
    c = -2.0 * vv * vv * f * (1 - f)
    ok.append(rel(r1["Sig"], -vv * vv * g1 * c / (1 - beta * c)) < 1e-10)
    return ok


def test_unmutated_pins_hold():
    assert all(_pins_hold())


@pytest.mark.parametrize("name,target,variant", [
    ("G(tau) for G(beta-tau) in P0", "polarization", _pol_variant(mirror=False)),
    ("k-q for k+q in P0", "polarization", _pol_variant(sign=-1)),
    ("spin factor dropped", "polarization", _pol_variant(s_factor=0.5)),
    ("conjugated right V in Sigma", "self_energy", _sig_variant(conj_right=True)),
    ("transposed P~ in Sigma", "self_energy", _sig_variant(transpose_p=True)),
    ("k+q for k-q in Sigma", "self_energy", _sig_variant(sign=+1)),
    ("(I+P0)^-1 P0 in the aux Dyson", "aux_dyson",
     lambda P0w: np.linalg.solve(np.eye(P0w.shape[-1]) + P0w, P0w)),
])
def test_planted_mistake_is_caught(monkeypatch, name, target, variant):
    monkeypatch.setattr(gw, target, variant)
    assert not all(_pins_hold()), name


# ---- the loop pieces: planted mistakes in Sigma^inf and the density matrix --------------------

def _sigma_inf_variant(hartree_spin=True, exchange_pair_swapped=False, exchange_sign=-1.0):
    def sinf(V, gamma, nk3, spin_factor=2.0):
        nk = V.shape[0]
        rho = sum(np.einsum("ab,Qba->Q", gamma[kp], V[kp, kp]) for kp in range(nk))
        out = np.empty((nk,) + gamma.shape[1:], complex)
        for k in range(nk):
            h = np.einsum("Qij,Q->ij", V[k, k], rho) * (spin_factor if hartree_spin else 1.0)
            x = sum(np.einsum("Qia,ab,Qbj->ij", V[k, kp], gamma[kp], V[k, kp] if exchange_pair_swapped else V[kp, k])
                    for kp in range(nk))
            out[k] = (h + exchange_sign * x) / nk
        return out
    return sinf


@pytest.mark.parametrize("variant", [_sigma_inf_variant(hartree_spin=False),
                                     _sigma_inf_variant(exchange_pair_swapped=True),
                                     _sigma_inf_variant(exchange_sign=+1.0)])
def test_planted_sigma_inf_mistake_is_caught(monkeypatch, variant):
    import test_oracle_loop_pins as LP
    monkeypatch.setattr(gw, "sigma_inf", variant)
    with pytest.raises(AssertionError):
        LP.test_sigma_inf_against_four_index((3, 1, 1))


def test_planted_density_sign_is_caught(monkeypatch):
    import test_oracle_loop_pins as LP
    real = gw.density_matrix
    monkeypatch.setattr(gw, "density_matrix", lambda G, beta: -real(G, beta))
    with pytest.raises(AssertionError):
        LP.test_density_matrix_of_g0_is_fermi((1, 1, 1), 2.0, 0.3)


def test_planted_diis_constraint_sign_is_caught(monkeypatch):
    """Lagrange row with the wrong sign: the coefficients sum to -1."""
    import test_oracle_loop_pins as LP

    def wrong(residuals):
        m = len(residuals)
        Bm = np.empty((m + 1, m + 1))
        for i in range(m):
            for j in range(m):
                Bm[i, j] = np.real(np.vdot(residuals[i], residuals[j]))
        Bm[m, :m] = Bm[:m, m] = -1.0
        Bm[m, m] = 0.0
        rhs = np.zeros(m + 1)
        rhs[m] = 1.0
        return np.linalg.solve(Bm, rhs)[:m]
    monkeypatch.setattr(gw, "diis_coefficients", wrong)
    with pytest.raises(AssertionError):
        LP.test_diis_solves_linear_fixed_points_exactly()


def test_planted_commutator_without_static_part_is_caught(monkeypatch):
    import test_oracle_loop_pins as LP
    real = gw.commutator_residual
    monkeypatch.setattr(gw, "commutator_residual", lambda H, sinf, Sig, G, beta: real(H, None, Sig, G, beta))
    with pytest.raises(AssertionError):
        LP.test_commutator_residual_vanishes_for_a_dyson_solution()


# ---- the second-order self-energy (Eq. sigma2) -----------------------------------------------

def _gf2_variant(mirror=True, exchange_spin=False, exchange_pair_swapped=False):
    from oracle import gf2

    def terms(V, G, nk3, spin_factor=2.0, k_list=None, t_list=None):
        nk, ntau, nao = G.shape[0], G.shape[1], G.shape[2]
        k_list = range(nk) if k_list is None else k_list
        t_list = range(ntau) if t_list is None else t_list
        d = np.zeros((len(k_list), len(t_list), nao, nao), complex)
        x = np.zeros_like(d)
        for ik, k in enumerate(k_list):
            for k1 in range(nk):
                for k2 in range(nk):
                    k3 = gw.k_shift(nk3, gw.k_shift(nk3, k1, k2, +1), k, -1)
                    for it, t in enumerate(t_list):
                        gm = G[k3, ntau - 1 - t] if mirror else G[k3, t]
                        d[ik, it] += np.einsum("Qip,pq,Rqj,Rln,nm,Qmk,kl->ij", V[k, k1], G[k1, t], V[k1, k],
                                               V[k2, k3], gm, V[k3, k2], G[k2, t], optimize=True)
                        vx = V[k, k2] if exchange_pair_swapped else V[k2, k]
                        x[ik, it] += np.einsum("Qip,pq,Rqn,nm,Qmk,kl,Rlj->ij", V[k, k1], G[k1, t], V[k1, k3],
                                               gm, V[k3, k2], G[k2, t], vx, optimize=True)
        return spin_factor * d / nk ** 2, (spin_factor if exchange_spin else 1.0) * x / nk ** 2
    return gf2, terms


@pytest.mark.parametrize("kw,pin", [
    (dict(mirror=False), "direct"),
    (dict(exchange_spin=True), "pauli"),
    (dict(exchange_pair_swapped=True), "brute"),
])
def test_planted_gf2_mistake_is_caught(monkeypatch, kw, pin):
    import test_oracle_gf2_pins as GP
    mod, variant = _gf2_variant(**kw)
    monkeypatch.setattr(mod, "gf2_terms", variant)
    with pytest.raises(AssertionError):
        if pin == "direct":
            GP.test_direct_term_is_the_second_order_gw_term((2, 1, 1))
        elif pin == "pauli":
            GP.test_one_spin_orbital_has_no_second_order_term(3)
        else:
            GP.test_against_four_index_brute_force((2, 1, 1))


# ---- k-space interpolation --------------------------------------------------------------------

@pytest.mark.parametrize("mistake", ["forward_sign", "no_boundary_split"])
def test_planted_kinterp_mistake_is_caught(monkeypatch, mistake):
    import itertools
    import test_oracle_kinterp_pins as KP
    from oracle import kinterp

    real_vectors = kinterp.lattice_vectors
    if mistake == "forward_sign":
        def interp(X, nk3, f_new):           # e^{+i k R} in the forward transform
            fk = kinterp.mesh_fractions(nk3)
            out = np.zeros((len(f_new),) + X.shape[1:], complex)
            for R, w in real_vectors(nk3):
                XR = np.tensordot(np.exp(+2j * np.pi * fk @ R), X, axes=(0, 0)) / fk.shape[0]
                out += w * np.exp(2j * np.pi * np.asarray(f_new) @ R)[(slice(None),) + (None,) * (X.ndim - 1)] * XR
            return out
        monkeypatch.setattr(kinterp, "k_interpolate", interp)
        with pytest.raises(AssertionError):
            KP.test_one_sided_hopping_is_reproduced((3, 3, 1))
    else:
        def vectors(nk3):
            axes = [list(range(-(n // 2), (n - 1) // 2 + 1)) for n in nk3]   # boundary taken once, at -N/2
            return [(np.array(c), 1.0) for c in itertools.product(*axes)]
        monkeypatch.setattr(kinterp, "lattice_vectors", vectors)
        with pytest.raises(AssertionError):
            KP.test_nearest_neighbour_hamiltonian((2, 2, 2))
