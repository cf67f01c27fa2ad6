"""GPU parity of the mixed-precision path (tcgen05, 4 bf16 slices per operand with
exact leading-slice accumulation) against the FP64 oracle.

Tolerances: relative max-norm 1e-7 for P0, P~ and Sigma (the scheme's error is
~1e-9 relative; 1e-7 still fails on any indexing or sign mistake), and the
target max |dSigma| <= 1e-6 Ha on the nao=8 molecule.
"""
import numpy as np
import pytest

from oracle import gw as O
from paper_2406_18479_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-7


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


CASES = [
    # nk3, nao, naux, ntau, beta, tau_chunk
    ((1, 1, 1), 8, 32, 4, 10.0, 0),
    ((1, 1, 1), 3, 7, 9, 10.0, 0),
    ((2, 1, 1), 5, 20, 6, 8.0, 2),
    ((3, 1, 1), 13, 33, 5, 12.0, 0),
    ((2, 2, 1), 6, 40, 7, 9.0, 3),
    ((1, 1, 1), 40, 130, 4, 20.0, 0),
]


@pytest.mark.parametrize("nk3,nao,naux,ntau,beta,chunk", CASES)
def test_mixed_chain_small(G, nk3, nao, naux, ntau, beta, chunk):
    w = I.Workload("case", nk3, nao, naux, ntau, ntau, beta, 0.0, 4.0, nao + naux, solid=int(np.prod(nk3)) > 1)
    h, v, g = I.make_inputs(w)
    ref = O.sigma_eval(v, g, nk3, beta, spin_factor=2.0)
    ctx = G.gw_create(nk3, nao, naux, ntau, beta, precision="bf16x3", tau_chunk=chunk)
    s = ctx.shapes()
    V, Gd = dev(v), dev(g)
    G.gw_set_coulomb(ctx, V)
    P0t = torch.empty(s["Pt"], dtype=torch.complex128, device="cuda")
    G.gw_polarization(ctx, Gd, P0t)
    G.gw_synchronize(ctx)
    assert rel(host(P0t), ref["P0t"]) < TOL
    Pt = torch.empty_like(P0t)
    G.gw_screened_interaction(ctx, P0t, Pt)
    Sig = torch.empty(s["Sig"], dtype=torch.complex128, device="cuda")
    G.gw_self_energy(ctx, Gd, Pt, Sig)
    G.gw_synchronize(ctx)
    assert rel(host(Pt), ref["Pt"]) < TOL
    assert rel(host(Sig), ref["Sig"]) < TOL
    Sig2 = torch.zeros_like(Sig)
    G.gw_sigma_eval(ctx, Gd, Sig2)
    G.gw_synchronize(ctx)
    assert rel(host(Sig2), ref["Sig"]) < TOL
    ctx.destroy()


def test_mixed_molecule_nao8_target(G):
    """The molecule of the paper-shaped configs: max |dSigma| <= 1e-6 Ha against the oracle."""
    w = I.WORKLOADS["molecule_nao8"]
    h, v, g = I.make_inputs(w)
    ref = O.sigma_eval(v, g, w.nk3, w.beta, spin_factor=2.0)
    ctx = G.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision="bf16x3")
    G.gw_set_coulomb(ctx, dev(v))
    Sig = torch.empty(ctx.shapes()["Sig"], dtype=torch.complex128, device="cuda")
    G.gw_sigma_eval(ctx, dev(g), Sig)
    G.gw_synchronize(ctx)
    out = host(Sig)
    err = float(np.max(np.abs(out - ref["Sig"])))
    print(f"molecule nao=8: max|dSigma| = {err:.3e} Ha, max|Sigma| = {np.abs(ref['Sig']).max():.3f} Ha")
    assert err <= 1e-6
    ctx.destroy()


@pytest.mark.parametrize("nk3,nao,naux,ntau,beta,chunk", [CASES[2], CASES[4], ((3, 2, 1), 4, 18, 5, 7.0, 2)])
def test_mixed_v_per_q_equals_all_pairs(G, nk3, nao, naux, ntau, beta, chunk):
    """V sliced per q, just before use, gives bit for bit what slices of all pairs give."""
    w = I.Workload("case", nk3, nao, naux, ntau, ntau, beta, 0.0, 4.0, nao + naux, solid=int(np.prod(nk3)) > 1)
    h, v, g = I.make_inputs(w)
    ref = O.sigma_eval(v, g, nk3, beta, spin_factor=2.0)
    out = {}
    for mode in (G.GW_V_ALL_PAIRS, G.GW_V_PER_Q):
        ctx = G.gw_create(nk3, nao, naux, ntau, beta, precision="bf16x3", tau_chunk=chunk, v_slices=mode)
        G.gw_set_coulomb(ctx, dev(v))
        S = torch.empty(ctx.shapes()["Sig"], dtype=torch.complex128, device="cuda")
        G.gw_sigma_eval(ctx, dev(g), S)
        G.gw_synchronize(ctx)
        out[mode] = host(S)
        ctx.destroy()
    assert np.array_equal(out[G.GW_V_ALL_PAIRS], out[G.GW_V_PER_Q])
    assert rel(out[G.GW_V_PER_Q], ref["Sig"]) < TOL
