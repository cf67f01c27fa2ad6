"""GPU parity: every C-ABI call against the FP64 oracle on the same seeded inputs.

Tolerance (FP64 path): relative max-norm 1e-10 per array,
rel(x) = max|x - x_oracle| / max|x_oracle|.
"""
import numpy as np
import pytest

from oracle import grids, gw as O
from paper_2406_18479_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_18479_gb300 import gw
    gw.lib()
    return gw


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def random_case(nk3, nao, naux, ntau, beta, seed):
    w = I.Workload("case", nk3, nao, naux, ntau, ntau, beta, 0.0, 4.0, seed, solid=int(np.prod(nk3)) > 1)
    return w, I.make_inputs(w)


CASES = [
    # nk3, nao, naux, ntau, beta, tau_chunk
    ((1, 1, 1), 1, 1, 1, 5.0, 0),
    ((1, 1, 1), 3, 7, 9, 10.0, 0),
    ((1, 1, 1), 13, 33, 17, 20.0, 4),
    ((3, 1, 1), 5, 7, 6, 8.0, 1),
    ((2, 2, 1), 3, 40, 9, 12.0, 3),
    ((2, 1, 3), 2, 5, 4, 6.0, 0),
    ((1, 1, 1), 33, 65, 8, 30.0, 0),
]


@pytest.mark.parametrize("nk3,nao,naux,ntau,beta,chunk", CASES)
def test_fp64_chain_small(G, nk3, nao, naux, ntau, beta, chunk):
    w, (h, v, g) = random_case(nk3, nao, naux, ntau, beta, seed=nao * 100 + naux)
    ref = O.sigma_eval(v, g, nk3, beta, spin_factor=2.0)
    ctx = G.gw_create(nk3, nao, naux, ntau, beta, precision="fp64", tau_chunk=chunk)
    s = ctx.shapes()
    V, Gd = dev(v), dev(g)
    G.gw_set_coulomb(ctx, V)
    P0t = torch.empty(s["Pt"], dtype=torch.complex128, device="cuda")
    G.gw_polarization(ctx, Gd, P0t)
    assert rel(host(P0t), ref["P0t"]) < TOL
    P0w = torch.empty(s["Pw"], dtype=torch.complex128, device="cuda")
    G.gw_to_matsubara(ctx, 0, P0t, P0w)
    assert rel(host(P0w), ref["P0w"]) < TOL
    Pw = torch.empty_like(P0w)
    G.gw_aux_dyson(ctx, P0w, Pw)
    assert rel(host(Pw), ref["Pw"]) < TOL
    Pt = torch.empty_like(P0t)
    G.gw_to_tau(ctx, 0, Pw, Pt)
    assert rel(host(Pt), ref["Pt"]) < TOL
    Pt2 = torch.empty_like(P0t)
    G.gw_screened_interaction(ctx, P0t, Pt2)
    assert rel(host(Pt2), ref["Pt"]) < TOL
    Sig = torch.empty(s["Sig"], dtype=torch.complex128, device="cuda")
    G.gw_self_energy(ctx, Gd, Pt, Sig)
    assert rel(host(Sig), ref["Sig"]) < TOL
    Sig2 = torch.zeros_like(Sig)
    G.gw_sigma_eval(ctx, Gd, Sig2)
    assert rel(host(Sig2), ref["Sig"]) < TOL
    G.gw_synchronize(ctx)
    ctx.destroy()


def test_fp64_molecule_nao8(G):
    w = I.WORKLOADS["molecule_nao8"]
    h, v, g = I.make_inputs(w)
    ref = O.sigma_eval(v, g, w.nk3, w.beta, spin_factor=2.0)
    ctx = G.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision="fp64")
    G.gw_set_coulomb(ctx, dev(v))
    Sig = torch.empty(ctx.shapes()["Sig"], dtype=torch.complex128, device="cuda")
    G.gw_sigma_eval(ctx, dev(g), Sig)
    out = host(Sig)
    assert rel(out, ref["Sig"]) < TOL
    assert rel(out, out.conj().swapaxes(-1, -2)) < 1e-12
    ctx.destroy()


@pytest.mark.parametrize("nk3,nao,ntau,beta,mu", [((1, 1, 1), 8, 32, 50.0, 0.0), ((3, 1, 1), 5, 12, 10.0, 0.1),
                                                 ((2, 2, 1), 13, 9, 7.0, -0.2)])
def test_dyson_g_and_mix(G, nk3, nao, ntau, beta, mu):
    w, (h, v, g) = random_case(nk3, nao, 2, ntau, beta, seed=3)
    rng = np.random.default_rng(4)
    sig = 0.05 * (rng.standard_normal(g.shape) + 1j * rng.standard_normal(g.shape))
    sig = 0.5 * (sig + sig.conj().swapaxes(-1, -2))
    ref = O.dyson_G(h, sig, mu, beta)
    ctx = G.gw_create(nk3, nao, 2, ntau, beta, mu=mu, precision="fp64")
    Gd = torch.empty(ctx.shapes()["G"], dtype=torch.complex128, device="cuda")
    G.gw_dyson_G(ctx, dev(h), dev(sig), Gd)
    assert rel(host(Gd), ref) < TOL
    old = dev(g)
    new = dev(sig)
    d = G.gw_mix(ctx, new, old, 0.5)
    mixed = O.mix(sig, g, 0.5)
    assert rel(host(old), mixed) < 1e-15
    assert abs(d - np.max(np.abs(mixed - g))) < 1e-14 * max(1.0, d)
    bad = sig.copy()
    bad[0, 0, 0, 0] = np.nan
    with pytest.raises(G.GWError) as e:
        G.gw_mix(ctx, dev(bad), dev(g), 0.5)
    assert e.value.code == G.GW_ENOTFINITE
    ctx.destroy()


def test_invalid_arguments_rejected(G):
    with pytest.raises(G.GWError) as e:
        G.gw_create((1, 1, 1), 0, 4, 4, 1.0)
    assert e.value.code == G.GW_EINVAL
    ctx = G.gw_create((1, 1, 1), 3, 4, 4, 5.0)
    with pytest.raises(G.GWError):
        G.gw_polarization(ctx, torch.zeros((1, 4, 3, 3), dtype=torch.complex128, device="cuda"),
                          torch.zeros((1, 4, 4, 4), dtype=torch.complex128, device="cuda"))   # no V yet
    with pytest.raises(G.GWError):
        G.gw_set_coulomb(ctx, torch.zeros((1, 1, 4, 3, 2), dtype=torch.complex128, device="cuda"))
    ctx.destroy()


@pytest.mark.parametrize("n", [1, 15, 16, 17, 33, 200, 430, 431, 519, 800, 801])
def test_aux_dyson_inverse_with_pivoting(G, n):
    """gw_aux_dyson = (I - P0)^{-1} - I per (q, n) (Eq. tilde_P_omega) against numpy, with unit
    diagonals in P0 so that I - P0 has a zero diagonal and every step must pivot; sizes around
    the panels of the blocked inversion (16 columns up to n = 430, 8 up to 800) and beyond."""
    ntau = 4
    ctx = G.gw_create((1, 1, 1), 1, n, ntau, 10.0, precision="fp64")
    nw = ctx.nwb
    rng = np.random.default_rng(n)
    p0 = (rng.standard_normal((1, nw, n, n)) + 1j * rng.standard_normal((1, nw, n, n))) / np.sqrt(n)
    if n > 1:                           # (for n = 1 that would make I - P0 singular)
        idx = np.arange(n)
        p0[..., idx, idx] = 1.0
    out = torch.empty((1, nw, n, n), dtype=torch.complex128, device="cuda")
    G.gw_aux_dyson(ctx, dev(p0), out)
    G.gw_synchronize(ctx)
    ref = np.linalg.inv(np.eye(n) - p0) - np.eye(n)
    assert rel(host(out), ref) < 1e-10
    ctx.destroy()


def _library_grids(ntau, beta):
    tau, mb, Fb, Bb = G_grids(ntau, beta, 0)
    _, mf, Ff, Bf = G_grids(ntau, beta, 1)
    return tau, Fb, Bb, Ff, Bf, 2 * np.pi * mb / beta, (2 * mf + 1) * np.pi / beta


def G_grids(ntau, beta, stat):
    from paper_2406_18479_gb300 import gw
    return gw.gw_grid_build(ntau, beta, stat)


def test_set_grids_uses_the_given_transforms(G):
    """gw_set_grids: the library's own grids give bit-identical results; a different left
    inverse B' = B + N (N F = 0, mirror-symmetric; possible since nb = ntau + 1) gives the
    oracle's chain computed with B'; grids without the mirror symmetry are rejected."""
    nk3, nao, naux, ntau, beta = (2, 1, 1), 4, 9, 6, 8.0
    w, (h, v, g) = random_case(nk3, nao, naux, ntau, beta, 5)
    tau, Fb, Bb, Ff, Bf, wb, wf = _library_grids(ntau, beta)
    ctx = G.gw_create(nk3, nao, naux, ntau, beta, precision="fp64")
    G.gw_set_coulomb(ctx, dev(v))
    S0 = torch.empty(ctx.shapes()["Sig"], dtype=torch.complex128, device="cuda")
    G.gw_sigma_eval(ctx, dev(g), S0)
    G.gw_set_grids(ctx, tau, Fb, Bb, Ff, Bf, wf, wb)
    S1 = torch.empty_like(S0)
    G.gw_sigma_eval(ctx, dev(g), S1)
    assert torch.equal(S0, S1)
    # another left inverse of F with the same mirror symmetry
    rng = np.random.default_rng(1)
    Z = rng.standard_normal(Bb.shape) + 1j * rng.standard_normal(Bb.shape)
    N = Z @ (np.eye(Fb.shape[0]) - Fb @ np.linalg.pinv(Fb))
    N = 0.5 * (N + N[::-1, ::-1])
    N *= 0.1 * np.abs(Bb).max() / np.abs(N).max()
    B2 = Bb + N
    assert np.abs(B2 @ Fb - np.eye(ntau)).max() < 1e-12
    G.gw_set_grids(ctx, tau, Fb, B2, Ff, Bf, wf, wb)
    S2 = torch.empty_like(S0)
    G.gw_sigma_eval(ctx, dev(g), S2)
    G.gw_synchronize(ctx)
    p0 = O.polarization(v, g, nk3, 2.0)
    _, _, pt = O.screened_interaction(p0, Fb, B2)
    ref = O.self_energy(v, g, pt, nk3)
    assert rel(host(S2), ref) < TOL
    assert rel(host(S2), host(S0)) > 1e-6            # the second left inverse changed the result
    with pytest.raises(G.GWError) as e:
        G.gw_set_grids(ctx, tau * 0.9, Fb, Bb, Ff, Bf, wf, wb)
    assert e.value.code == G.GW_EINVAL
    Fbad = Fb.copy()
    Fbad[0, 0] += 0.1
    with pytest.raises(G.GWError) as e:
        G.gw_set_grids(ctx, tau, Fbad, Bb, Ff, Bf, wf, wb)
    assert e.value.code == G.GW_EINVAL
    ctx.destroy()
