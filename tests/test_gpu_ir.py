"""GW on an IR grid (gw_ir_grids + gw_set_grids) against the oracle's chain with the same
transforms: the self-energy in FP64 and in the mixed precision, and the Dyson equation."""
import numpy as np
import pytest

from oracle import gw as O
from paper_2406_18479_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def test_gw_and_dyson_on_an_ir_grid(G):
    beta, lam, eps = 20.0, 200.0, 1e-10
    tau, Fb, Bb, Ff, Bf, wf, wb = G.gw_ir_grids(beta, lam, eps)
    T = len(tau)
    nk3, nao, naux = (2, 1, 1), 3, 5
    w = I.Workload("ir", nk3, nao, naux, T, T, beta, 0.0, 4.0, 3, solid=True)
    rng = np.random.default_rng(w.seed)
    h = I.hamiltonian(w, rng)
    v = I.coulomb(w, rng)
    g = I.g0_tau(h, 0.0, beta, tau)
    p0 = O.polarization(v, g, nk3, 2.0)
    _, _, pt = O.screened_interaction(p0, Fb, Bb)
    ref = O.self_energy(v, g, pt, nk3)
    out = {}
    for prec in ("fp64", "bf16x3"):
        ctx = G.gw_create(nk3, nao, naux, T, beta, precision=prec)
        vd = dev(v)
        G.gw_set_coulomb(ctx, vd)
        G.gw_set_grids(ctx, tau, Fb, Bb, Ff, Bf, wf, wb)
        S = torch.empty(ctx.shapes()["Sig"], dtype=torch.complex128, device="cuda")
        G.gw_sigma_eval(ctx, dev(g), S)
        torch.cuda.synchronize()
        out[prec] = S.cpu().numpy()
        if prec == "fp64":
            Gd = torch.empty_like(S)
            G.gw_dyson_G(ctx, dev(h), S, Gd)
            torch.cuda.synchronize()
            gref = O.dyson_G(h, ref, 0.0, beta, fermionic=(wf, Ff, Bf))
            assert rel(Gd.cpu().numpy(), gref) < 1e-10
        ctx.destroy()
    assert rel(out["fp64"], ref) < 1e-10
    assert np.abs(out["bf16x3"] - ref).max() < 1e-6
