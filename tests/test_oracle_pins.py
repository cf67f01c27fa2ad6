"""Pins of the FP64 oracle against closed forms, brute force and invariants.

Each test cites the passage of arXiv 2406.18479 it checks. These tests run
on the CPU only.
"""
import numpy as np
import pytest

from oracle import grids, gw
from paper_2406_18479_gb300 import inputs as I
import pin_forms as PF


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def small_workload(nk3=(1, 1, 1), nao=3, naux=5, ntau=24, beta=10.0, seed=11, solid=None, decay=4.0):
    return I.Workload("t", nk3, nao, naux, ntau, ntau, beta, 0.0, decay, seed,
                      solid=(np.prod(nk3) > 1) if solid is None else solid)


def generic_inputs(w, rng_seed=5, h_scale=1.0):
    """Random H(k) per k (no k-symmetry) and V with only the k1<->k2 symmetry."""
    rng = np.random.default_rng(rng_seed)
    nk, nao = w.nk, w.nao
    h = np.empty((nk, nao, nao), complex)
    for k in range(nk):
        x = rng.standard_normal((nao, nao)) + 1j * rng.standard_normal((nao, nao))
        x = 0.5 * (x + x.conj().T)
        h[k] = h_scale * x / np.linalg.norm(x, 2)
    v = I.coulomb(w, rng)
    tau = I.chebyshev_tau(w.ntau, w.beta)
    g = I.g0_tau(h, w.mu, w.beta, tau)
    return h, v, g


# ---------------------------------------------------------------- grids (Eq. P0t_to_P0w)

@pytest.mark.parametrize("ntau", [8, 17, 32])
@pytest.mark.parametrize("stat", [0, 1])
def test_tnl_quadrature_matches_exact_integration_by_parts(ntau, stat):
    """T_nl of the oracle (Gauss-Legendre) against the exact finite IBP sum in 80 digits."""
    m, f, _ = grids.transform_matrices(ntau, 1.0, stat)
    tau = grids.chebyshev_nodes(ntau, 1.0)
    tl = np.cos(np.outer(np.arccos(2 * tau - 1), np.arange(ntau)))
    t_nl = f @ tl                         # F T_tl = T_nl
    ls = sorted(set([0, 1, 2, ntau // 2, ntau - 1]))
    ms = sorted(set([m[0], m[len(m) // 2], m[len(m) // 2 + 1], m[-1], m[-2]]))
    for mm in ms:
        n = int(np.where(m == mm)[0][0])
        for l in ls:
            ex = PF.t_nl_exact(int(mm), l, stat)
            assert abs(t_nl[n, l] - ex) < 1e-13, (mm, l, t_nl[n, l], ex)


@pytest.mark.parametrize("stat", [0, 1])
def test_sample_sets_symmetric_and_well_conditioned(stat):
    for ntau in [1, 2, 3, 8, 24, 32, 80, 100, 120]:
        m, f, b = grids.transform_matrices(ntau, 7.0, stat)
        assert len(m) == grids.sample_count(ntau, stat)
        assert np.array_equal(np.sort(-m - stat), m)           # symmetric in w
        assert len(np.unique(m)) == len(m)
        sv = np.linalg.svd(f, compute_uv=False)
        assert sv[0] / sv[-1] < 2e3
        assert np.abs(b @ f - np.eye(ntau)).max() < 1e-12


def test_forward_transform_of_exponential():
    """F applied to node values of e^{-e tau} equals (e^{(iw - e) beta} - 1)/(iw - e) (converged grid)."""
    beta, ntau = 10.0, 64
    for stat in [0, 1]:
        m, f, _ = grids.transform_matrices(ntau, beta, stat)
        w = (2 * m + stat) * np.pi / beta
        tau = grids.chebyshev_nodes(ntau, beta)
        for e in [-1.3, 0.0, 0.4, 1.7]:
            got = f @ np.exp(-e * tau)
            if e == 0.0:
                ex = np.where(w == 0, beta, ((-1) ** stat - 1) / (1j * np.where(w == 0, 1, w)))
            else:
                ex = (np.exp(-e * beta) * (-1) ** stat - 1) / (1j * w - e)
            assert np.abs(got - ex).max() < 1e-12 * np.abs(ex).max()


# ---------------------------------------------------------------- P0 (Eq. tilde_P0_tau)

@pytest.mark.parametrize("nk3", [(1, 1, 1), (3, 1, 1), (2, 2, 1)])
def test_p0_tau_pole_form(nk3):
    """Oracle P0(tau) with G = G0 equals the eigenbasis pole form to 1e-13."""
    w = small_workload(nk3=nk3, nao=3, naux=4, ntau=12, beta=7.0)
    h, v, g = generic_inputs(w)
    tau = I.chebyshev_tau(w.ntau, w.beta)
    got = gw.polarization(v, g, nk3, spin_factor=2.0)
    ex = PF.pole_form_p0_tau(h, v, nk3, w.beta, w.mu, tau, 2.0)
    assert rel(got, ex) < 1e-13


def test_p0_iw_pole_pair_sum_on_converged_grid():
    """F P0(tau) equals the analytic pole-pair sum at every sampled frequency (beta = 10, 64 nodes)."""
    nk3 = (2, 1, 1)
    w = small_workload(nk3=nk3, nao=3, naux=4, ntau=64, beta=10.0)
    h, v, g = generic_inputs(w)
    m, F, _ = grids.transform_matrices(w.ntau, w.beta, 0)
    omegas = 2 * m * np.pi / w.beta
    p0w = gw.to_matsubara(gw.polarization(v, g, nk3, 2.0), F)
    ex = PF.pole_pair_p0_iw(h, v, nk3, w.beta, w.mu, omegas, 2.0)
    assert rel(p0w, ex) < 1e-10


def test_p0_invariants():
    """P0^q(tau) Hermitian; P0^q(beta - tau) = P0^{-q}(tau)^T; Herm P0(i W) <= 0 (screening)."""
    nk3 = (3, 1, 1)
    w = small_workload(nk3=nk3, nao=3, naux=5, ntau=16, beta=6.0)
    h, v, g = generic_inputs(w)
    p0 = gw.polarization(v, g, nk3, 2.0)
    assert rel(p0, p0.conj().swapaxes(-1, -2)) < 1e-13
    for q in range(w.nk):
        mq = PF.mesh_shift(nk3, 0, q, -1)
        assert rel(p0[q, ::-1], p0[mq].swapaxes(-1, -2)) < 1e-13
    _, F, _ = grids.transform_matrices(w.ntau, w.beta, 0)
    p0w = gw.to_matsubara(p0, F)
    scale = np.abs(p0w).max()
    for q in range(w.nk):
        for n in range(p0w.shape[1]):
            x = p0w[q, n]
            assert np.linalg.eigvalsh(0.5 * (x + x.conj().T)).max() < 1e-12 * scale


# ------------------------------------------------ full chain: scalar closed form, brute force

def test_scalar_closed_form_whole_chain():
    """nao = naux = 1: P0(tau) = c = -s v^2 f (1-f); P0(i W_n) = beta c delta_n0;
    P~(tau) = c/(1 - beta c); Sigma(tau) = -v^2 G0(tau) c/(1 - beta c)."""
    for beta, eps, vv in [(10.0, 0.3, 0.7), (25.0, -0.05, 1.3), (5.0, 0.0, 2.0)]:
        ntau = 20
        h = np.array([[[eps]]], complex)
        v = np.full((1, 1, 1, 1, 1), vv, complex)
        tau = I.chebyshev_tau(ntau, beta)
        g = I.g0_tau(h, 0.0, beta, tau)
        r = gw.sigma_eval(v, g, (1, 1, 1), beta, spin_factor=2.0)
        f = PF.fermi(np.array([eps]), beta)[0]
        c = -2.0 * vv * vv * f * (1 - f)
        m, _, _ = grids.transform_matrices(ntau, beta, 0)
        assert np.abs(r["P0t"] - c).max() < 1e-14 * abs(c)
        p0w_ex = np.where(m == 0, beta * c, 0.0)
        assert np.abs(r["P0w"][0, :, 0, 0] - p0w_ex).max() < 1e-13 * abs(beta * c)
        pt_ex = c / (1 - beta * c)
        # Quadrature rounding in F (~1e-16 beta per entry) is amplified by the edge rows
        # of B = F^+ (cond ~1e2); the chain then holds to ~1e-11 relative.
        assert np.abs(r["Pt"] - pt_ex).max() < 1e-10 * abs(pt_ex)
        sig_ex = -vv * vv * g * pt_ex
        assert rel(r["Sig"], sig_ex) < 1e-10


@pytest.mark.parametrize("nk3,nao,naux", [((1, 1, 1), 3, 6), ((2, 1, 1), 2, 3), ((3, 1, 1), 2, 3)])
def test_sigma_against_four_index_brute_force(nk3, nao, naux):
    """Aux-basis oracle Sigma equals the pair-space RPA with U = sum_Q V V (no conjugation)."""
    w = small_workload(nk3=nk3, nao=nao, naux=naux, ntau=10, beta=5.0)
    h, v, g = generic_inputs(w, rng_seed=7)
    r = gw.sigma_eval(v, g, nk3, w.beta, spin_factor=2.0)
    _, F, B = grids.transform_matrices(w.ntau, w.beta, 0)
    bf = PF.brute_force_sigma(v, g, nk3, F, B, 2.0)
    assert rel(r["Sig"], bf) < 1e-12


def test_sigma_hermitian_and_v_symmetry():
    w = I.WORKLOADS["molecule_nao8"]
    h, v, g = I.make_inputs(w)
    assert rel(v[0, 0], v[0, 0].conj().swapaxes(-1, -2)) < 1e-15
    r = gw.sigma_eval(v, g, w.nk3, w.beta)
    s = r["Sig"]
    assert rel(s, s.conj().swapaxes(-1, -2)) < 1e-12
    w2 = small_workload(nk3=(3, 1, 1), nao=3, naux=4, ntau=12, beta=8.0)
    h2, v2, g2 = generic_inputs(w2)
    for k1 in range(3):
        for k2 in range(3):
            assert np.array_equal(v2[k2, k1], v2[k1, k2].conj().swapaxes(-1, -2))
    s2 = gw.sigma_eval(v2, g2, w2.nk3, w2.beta)["Sig"]
    assert rel(s2, s2.conj().swapaxes(-1, -2)) < 1e-12


def test_flat_mesh_reduces_to_molecule():
    """H(k) = H, V(k1,k2) = V for all k: every P~^q and Sigma^k equal the Gamma-only result."""
    w1 = small_workload(nao=3, naux=4, ntau=12, beta=6.0)
    h1, v1, g1 = generic_inputs(w1)
    mol = gw.sigma_eval(v1, g1, (1, 1, 1), w1.beta)
    nk3 = (2, 2, 1)
    nk = 4
    v = np.broadcast_to(v1[0, 0], (nk, nk) + v1.shape[2:]).copy()
    g = np.broadcast_to(g1[0], (nk,) + g1.shape[1:]).copy()
    sol = gw.sigma_eval(v, g, nk3, w1.beta)
    for q in range(nk):
        assert rel(sol["Pt"][q], mol["Pt"][0]) < 1e-13
        assert rel(sol["Sig"][q], mol["Sig"][0]) < 1e-13


def test_small_p_series():
    """P~ = eps P0 + eps^2 P0^2 + O(eps^3), the series form of Eq. (tilde_P_omega)."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal((1, 2, 6, 6)) + 1j * rng.standard_normal((1, 2, 6, 6))
    for eps in [1e-2, 1e-3]:
        got = gw.aux_dyson(eps * x)
        series = eps * x + eps * eps * np.einsum("qnij,qnjk->qnik", x, x)
        err = np.abs(got - series).max()
        bound = 4 * eps ** 3 * np.linalg.norm(x[0, 0], 2) ** 3 * 10
        assert err < bound


# ---------------------------------------------------------------- G Dyson (Eq. dyson)

def test_dyson_sigma_zero_returns_g0():
    """Sigma = 0: G(i w) = (i w + mu - H)^{-1}; back in tau it is G0 to the grid's error."""
    beta, ntau = 8.0, 64
    w = small_workload(nk3=(2, 1, 1), nao=3, naux=2, ntau=ntau, beta=beta)
    h, v, g0 = generic_inputs(w, h_scale=1.0)
    for mu in [0.0, 0.2]:
        tau = I.chebyshev_tau(ntau, beta)
        g0 = I.g0_tau(h, mu, beta, tau)
        gd = gw.dyson_G(h, np.zeros_like(g0), mu, beta)
        assert rel(gd, g0) < 1e-10


def test_dyson_matches_frequency_inverse():
    beta, ntau = 8.0, 16
    w = small_workload(nk3=(1, 1, 1), nao=3, naux=2, ntau=ntau, beta=beta)
    h, v, g0 = generic_inputs(w)
    rng = np.random.default_rng(9)
    sig = 0.1 * (rng.standard_normal(g0.shape) + 1j * rng.standard_normal(g0.shape))
    m, Ff, Bf = grids.transform_matrices(ntau, beta, 1)
    wn = (2 * m + 1) * np.pi / beta
    gd = gw.dyson_G(h, sig, 0.1, beta)
    gw_w = np.einsum("nt,ktij->knij", Ff, gd)
    sw = np.einsum("nt,ktij->knij", Ff, sig)
    for n in range(len(wn)):
        lhs = ((1j * wn[n] + 0.1) * np.eye(3) - h[0] - sw[0, n]) @ gw_w[0, n]
        assert np.abs(lhs - np.eye(3)).max() < 1e-10


def test_mixing_and_loop_converge():
    w = small_workload(nao=3, naux=4, ntau=16, beta=5.0, decay=2.0)
    h, v, g0 = generic_inputs(w)
    v = 0.3 * v
    sig, g, hist = gw.scgw(h, v, g0, w.nk3, w.beta, 0.0, itermax=30, tol=1e-9)
    assert hist[-1] < 1e-9
    # fixed point: Sigma[G(Sigma)] = Sigma
    again = gw.sigma_eval(v, g, w.nk3, w.beta)["Sig"]
    assert rel(again, sig) < 1e-6
    a = np.ones(3)
    assert np.allclose(gw.mix(3 * a, a, 0.5), 2 * a)
