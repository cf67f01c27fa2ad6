"""Pins of the oracle's loop pieces (Eq. sigma_inf, Sec. 2.4 steps 2-3, Sec. 5.3), each against
something other than the formula it implements: closed forms of the non-interacting system, the
explicit 4-index interaction, a scalar root finder, and the exact behaviour of Pulay's
extrapolation on linear maps."""
import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import gw as O
from paper_2406_18479_gb300 import inputs as I


def fermi(e, beta):
    return 0.5 * (1.0 - np.tanh(0.5 * beta * e))


@pytest.mark.parametrize("nk3,beta,mu", [((1, 1, 1), 2.0, 0.3), ((2, 1, 1), 1.5, -0.2), ((2, 2, 1), 2.5, 0.0)])
def test_density_matrix_of_g0_is_fermi(nk3, beta, mu):
    """G0(0^-) = U diag(f(eps - mu)) U^dagger; the interpolant is exact to 1e-12 at this beta."""
    w = I.Workload("m", nk3, 5, 10, 40, 40, beta, mu, 4.0, 3, solid=int(np.prod(nk3)) > 1)
    h, v, g = I.make_inputs(w)
    gam = O.density_matrix(g, beta)
    for k in range(w.nk):
        e, u = np.linalg.eigh(h[k])
        assert np.abs(gam[k] - (u * fermi(e - mu, beta)) @ u.conj().T).max() < 1e-12


def test_particle_number_of_g0():
    w = I.Workload("m", (2, 1, 1), 6, 12, 40, 40, 2.0, 0.1, 4.0, 5, solid=True)
    h, v, g = I.make_inputs(w)
    n = O.particle_number(O.density_matrix(g, w.beta), 2.0)
    ref = 2.0 / w.nk * sum(fermi(np.linalg.eigvalsh(h[k]) - w.mu, w.beta).sum() for k in range(w.nk))
    assert abs(n - ref) < 1e-11


def brute_sigma_inf(V, gamma, spin):
    """Eq. (sigma_inf) through the explicit 4-index interaction
    U^{k1 k2, k3 k4}_{ij,kl} = sum_Q V^{k1 k2}_ij(Q) V^{k3 k4}_kl(Q) (no conjugation)."""
    nk, _, naux, nao, _ = V.shape
    out = np.zeros((nk, nao, nao), complex)
    for k in range(nk):
        for kp in range(nk):
            UH = np.tensordot(V[k, k], V[kp, kp], axes=([0], [0]))        # [i j b a]
            UX = np.tensordot(V[k, kp], V[kp, k], axes=([0], [0]))        # [i a b j]
            for i in range(nao):
                for j in range(nao):
                    hart = sum(UH[i, j, b, a] * gamma[kp, a, b] for a in range(nao) for b in range(nao))
                    exch = sum(UX[i, a, b, j] * gamma[kp, a, b] for a in range(nao) for b in range(nao))
                    out[k, i, j] += (spin * hart - exch) / nk
    return out


@pytest.mark.parametrize("nk3", [(1, 1, 1), (3, 1, 1)])
def test_sigma_inf_against_four_index(nk3):
    w = I.Workload("m", nk3, 3, 5, 8, 8, 3.0, 0.0, 3.0, 7, solid=int(np.prod(nk3)) > 1)
    h, v, g = I.make_inputs(w)
    gam = O.density_matrix(g, w.beta)
    s = O.sigma_inf(v, gam, nk3, 2.0)
    assert np.abs(s - brute_sigma_inf(v, gam, 2.0)).max() < 1e-12 * max(1.0, np.abs(s).max())
    # Hermitian for a Hermitian density matrix and V(k2,k1)^Q_ji = conj V(k1,k2)^Q_ij
    assert np.abs(s - s.conj().transpose(0, 2, 1)).max() < 1e-12 * np.abs(s).max()


def test_find_mu_matches_scalar_root_of_fermi_count():
    w = I.Workload("m", (2, 1, 1), 6, 12, 40, 40, 2.0, 0.0, 4.0, 9, solid=True)
    h, v, g = I.make_inputs(w)
    eps = [np.linalg.eigvalsh(h[k]) for k in range(w.nk)]
    target = 5.0

    def count(mu):
        return 2.0 / w.nk * sum(fermi(e - mu, w.beta).sum() for e in eps) - target
    mu_ref = brentq(count, -10, 10, xtol=1e-14)
    Sig = np.zeros_like(g)
    mu, G = O.find_mu(h, None, Sig, w.beta, target, 2.0, lo=-5.0, hi=5.0, tol=1e-12)
    assert abs(mu - mu_ref) < 1e-8
    assert abs(O.particle_number(O.density_matrix(G, w.beta), 2.0) - target) < 1e-8


def test_diis_solves_linear_fixed_points_exactly():
    """On x = A x + b (|A| < 1) Pulay's extrapolation over all past iterates reaches the fixed
    point once the real span of the residuals (real coefficients on C^n: dimension 2n) is
    exhausted, after 2n + 1 iterations; with one vector it returns the newest output unchanged;
    the coefficients sum to 1."""
    rng = np.random.default_rng(0)
    n = 7
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A *= 0.4 / np.abs(np.linalg.eigvals(A)).max()
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    xstar = np.linalg.solve(np.eye(n) - A, b)
    xs, fs = [np.zeros(n, complex)], []
    for it in range(2 * n + 1):
        fs.append(A @ xs[-1] + b)
        nxt, c = O.diis_extrapolate(fs, xs)
        assert abs(c.sum() - 1.0) < 1e-12
        if it == 0:
            assert np.array_equal(nxt, fs[0])
        xs.append(nxt)
    assert np.abs(xs[-1] - xstar).max() < 1e-10 * np.abs(xstar).max()


def loop_case():
    w = I.Workload("m", (2, 1, 1), 4, 8, 16, 16, 5.0, 0.0, 4.0, 21, solid=True)
    h, v, g = I.make_inputs(w)
    return w, h, 0.3 * v, g


def test_full_loop_reduces_to_the_fixed_mu_loop():
    """Without the static part, the mu search and DIIS the full loop is the fixed-mu loop."""
    w, h, v, g = loop_case()
    a = O.scgw_full(h, v, g, w.nk3, w.beta, 0.1, alpha=0.6, tol=1e-9, itermax=4, static=False)
    sig, G, hist = O.scgw(h, v, g, w.nk3, w.beta, 0.1, alpha=0.6, tol=1e-9, itermax=4)
    assert np.array_equal(a["Sig"], sig) and np.array_equal(a["G"], G)
    assert a["hist"] == hist


@pytest.mark.parametrize("diis", [0, 4])
def test_full_loop_reaches_its_fixed_point(diis):
    """At convergence every step of Sec. 2.4 holds at once: Sigma^inf and Sigma~ are those of G,
    G holds n_electrons, and G solves the Dyson equation with them."""
    w, h, v, g = loop_case()
    n_e = 3.0
    r = O.scgw_full(h, v, g, w.nk3, w.beta, 0.0, alpha=0.7, tol=1e-10, itermax=60, n_electrons=n_e,
                    mu_tol=1e-13, diis_size=diis, diis_start=3)
    assert r["hist"][-1] < 1e-10
    gam = O.density_matrix(r["G"], w.beta)
    assert abs(O.particle_number(gam, 2.0) - n_e) < 1e-9
    assert np.abs(O.sigma_inf(v, gam, w.nk3, 2.0) - r["SigInf"]).max() < 1e-8
    assert np.abs(O.sigma_eval(v, r["G"], w.nk3, w.beta)["Sig"] - r["Sig"]).max() < 1e-8
    assert np.abs(O.dyson_G(h + r["SigInf"], r["Sig"], r["mu"], w.beta) - r["G"]).max() < 1e-12


def test_full_loop_fixed_point_does_not_depend_on_the_acceleration():
    """Mixing and DIIS reach the same (Sigma, G, mu); DIIS in fewer iterations here."""
    w, h, v, g = loop_case()
    kw = dict(tol=1e-10, itermax=80, n_electrons=3.0, mu_tol=1e-13)
    a = O.scgw_full(h, v, g, w.nk3, w.beta, 0.0, alpha=0.5, **kw)
    b = O.scgw_full(h, v, g, w.nk3, w.beta, 0.0, alpha=0.5, diis_size=5, diis_start=2, **kw)
    assert abs(a["mu"] - b["mu"]) < 1e-8
    for key in ("Sig", "SigInf", "G"):
        assert np.abs(a[key] - b[key]).max() < 1e-8
    assert b["iterations"] < a["iterations"]


def test_commutator_residual_vanishes_for_a_dyson_solution():
    """G = Dyson(H + Sigma^inf, Sigma~) commutes with H + Sigma^inf + Sigma~(i w) on every sample
    (ntau even: the fermionic sample set is square, F^f B^f = I); a G from another self-energy
    does not, and the residual is linear in the static shift's commutator."""
    w = I.Workload("m", (2, 1, 1), 4, 6, 16, 16, 5.0, 0.0, 4.0, 13, solid=True)
    h, v, g = I.make_inputs(w)
    rng = np.random.default_rng(1)
    sig = 0.05 * (rng.standard_normal(g.shape) + 1j * rng.standard_normal(g.shape))
    sig = 0.5 * (sig + sig.conj().swapaxes(-1, -2))
    sinf = O.sigma_inf(v, O.density_matrix(g, w.beta), w.nk3, 2.0)
    G = O.dyson_G(h + sinf, sig, 0.2, w.beta)
    e = O.commutator_residual(h, sinf, sig, G, w.beta)
    assert np.abs(e).max() < 1e-12
    e_other = O.commutator_residual(h, None, sig, G, w.beta)      # drop the static part
    assert np.abs(e_other).max() > 1e-3
    # [G, X + D] - [G, X] = [G, D] for a static D: here D = -Sigma^inf
    _, Ff, _ = O.grids.transform_matrices(w.ntau, w.beta, 1)
    Gw = np.einsum("nt,ktij->knij", Ff, G)
    D = -sinf[:, None]
    assert np.abs((e_other - e) - (Gw @ D - D @ Gw)).max() < 1e-12


def test_cdiis_loop_reaches_the_same_fixed_point():
    w, h, v, g = loop_case()
    kw = dict(tol=1e-10, itermax=80, n_electrons=3.0, mu_tol=1e-13)
    a = O.scgw_full(h, v, g, w.nk3, w.beta, 0.0, alpha=0.5, **kw)
    b = O.scgw_full(h, v, g, w.nk3, w.beta, 0.0, alpha=0.5, diis_size=5, diis_start=2, diis_kind="cdiis", **kw)
    assert b["hist"][-1] < 1e-10
    assert abs(a["mu"] - b["mu"]) < 1e-8
    for key in ("Sig", "SigInf", "G"):
        assert np.abs(a[key] - b[key]).max() < 1e-8
    assert b["iterations"] < a["iterations"]
    e = O.commutator_residual(h, b["SigInf"], b["Sig"], b["G"], w.beta)
    assert np.abs(e).max() < 1e-8


def test_hartree_fock_loop_fixed_point_is_a_fermi_matrix():
    """With Sigma~ = 0 the converged G is non-interacting in H + Sigma^inf: its density matrix is
    U f(eps - mu) U^dagger of that matrix, Sigma^inf is the one of this density, and N = n."""
    w, h, v, g = loop_case()
    r = O.scgw_full(h, v, g, w.nk3, w.beta, 0.0, alpha=0.7, tol=1e-11, itermax=200, n_electrons=3.0,
                    mu_tol=1e-13, diis_size=5, method="hf")
    assert r["hist"][-1] < 1e-11 and not np.any(r["Sig"])
    gam = O.density_matrix(r["G"], w.beta)
    for k in range(w.nk):
        e, u = np.linalg.eigh(h[k] + r["SigInf"][k])
        assert np.abs(gam[k] - (u * fermi(e - r["mu"], w.beta)) @ u.conj().T).max() < 1e-9
    assert np.abs(O.sigma_inf(v, gam, w.nk3, 2.0) - r["SigInf"]).max() < 1e-9
    assert abs(O.particle_number(gam, 2.0) - 3.0) < 1e-9


def overlap_case():
    w = I.Workload("s", (2, 1, 1), 4, 6, 16, 16, 5.0, 0.0, 4.0, 31, solid=True)
    h, v, g = I.make_inputs(w)
    S = I.overlap(w, np.random.default_rng(3))
    rng = np.random.default_rng(4)
    sig = 0.05 * (rng.standard_normal(g.shape) + 1j * rng.standard_normal(g.shape))
    return w, h, v, g, S, 0.5 * (sig + sig.conj().swapaxes(-1, -2))


def test_dyson_with_overlap_is_the_orthogonalised_problem():
    """With S = L L^dagger, (i w + mu) S - H - Sigma = L [(i w + mu) - L^-1 (H + Sigma) L^-dagger] L^dagger,
    so G = L^-dagger G' L^-1 with G' the S = I solution for the transformed H and Sigma; the
    particle number Tr(gamma S) is Tr(gamma') of the orthogonalised problem."""
    w, h, v, g, S, sig = overlap_case()
    G = O.dyson_G(h, sig, 0.2, w.beta, S=S)
    L = np.linalg.cholesky(S)
    Li = np.linalg.inv(L)
    hp = Li @ h @ Li.conj().swapaxes(-1, -2)
    sp = Li[:, None] @ sig @ Li.conj().swapaxes(-1, -2)[:, None]
    Gp = O.dyson_G(hp, sp, 0.2, w.beta)
    back = Li.conj().swapaxes(-1, -2)[:, None] @ Gp @ Li[:, None]
    assert np.abs(G - back).max() < 1e-12 * np.abs(G).max()
    n = O.particle_number(O.density_matrix(G, w.beta), 2.0, S)
    assert abs(n - O.particle_number(O.density_matrix(Gp, w.beta), 2.0)) < 1e-11


def test_commutator_with_overlap_vanishes_for_a_dyson_solution():
    w, h, v, g, S, sig = overlap_case()
    sinf = O.sigma_inf(v, O.density_matrix(g, w.beta), w.nk3, 2.0)
    G = O.dyson_G(h + sinf, sig, -0.1, w.beta, S=S)
    assert np.abs(O.commutator_residual(h, sinf, sig, G, w.beta, S)).max() < 1e-11
    assert np.abs(O.commutator_residual(h, sinf, sig, G, w.beta)).max() > 1e-3      # S = I does not hold


def test_loop_with_overlap_reaches_its_fixed_point():
    w, h, v, g, S, sig = overlap_case()
    r = O.scgw_full(h, 0.3 * v, g, w.nk3, w.beta, 0.0, alpha=0.6, tol=1e-10, itermax=80, n_electrons=3.0,
                    mu_tol=1e-13, diis_size=5, diis_kind="cdiis", S=S)
    assert r["hist"][-1] < 1e-10
    gam = O.density_matrix(r["G"], w.beta)
    assert abs(O.particle_number(gam, 2.0, S) - 3.0) < 1e-9
    assert np.abs(O.dyson_G(h + r["SigInf"], r["Sig"], r["mu"], w.beta, S=S) - r["G"]).max() < 1e-12


def test_resumed_loop_continues_exactly():
    """2n iterations in one go equal n iterations, then n more resumed from the saved (Sigma, G)
    (mixing only: the DIIS history is not part of the saved state)."""
    w, h, v, g = loop_case()
    kw = dict(alpha=0.6, tol=0.0, n_electrons=3.0, mu_tol=1e-13)
    full = O.scgw_full(h, v, g, w.nk3, w.beta, 0.0, itermax=6, **kw)
    half = O.scgw_full(h, v, g, w.nk3, w.beta, 0.0, itermax=3, **kw)
    rest = O.scgw_full(h, v, half["G"], w.nk3, w.beta, half["mu"], itermax=3, resume=(half["SigInf"], half["Sig"]), **kw)
    assert np.array_equal(rest["Sig"], full["Sig"]) and np.array_equal(rest["G"], full["G"])
    assert rest["hist"] == full["hist"][2:]
