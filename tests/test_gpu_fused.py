"""The mixed path with slice-output epilogues (the V.G products and R write the next
contraction's bf16 slice groups themselves) against the FP64 oracle, against the same path
with a separate slicing pass (gw_config.slice_pass = 1), and at the 1e-6 Ha target.

The fused path takes sizes with nao % 4 == 0, nao <= 56 and naux % 40 == 0; the cases cover one
and several k points, naux an odd multiple of 40 (the last 80-wide tile of R half empty, the
Z tiles straddling two orbitals i), several tau batches, V sliced per q, and a packed V.
Tolerance: relative max-norm 1e-7 for P0, P~ and Sigma, as for the unfused mixed path.
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
    # nk3, nao, naux, ntau, beta, tau_chunk, v_slices
    ((1, 1, 1), 8, 40, 6, 10.0, 0, 0),
    ((2, 1, 1), 4, 120, 7, 8.0, 3, 0),
    ((2, 2, 1), 12, 80, 5, 9.0, 2, 0),
    ((3, 1, 1), 16, 40, 6, 12.0, 0, 2),
    ((1, 1, 1), 52, 40, 4, 20.0, 0, 0),
    ((2, 1, 1), 56, 200, 3, 15.0, 0, 2),
]


def run(G, w, v, g, **kw):
    ctx = G.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision="bf16x3", **kw)
    s = ctx.shapes()
    Vd, Gd = dev(I.pack_v(v) if kw.get("v_packed") else v), dev(g)
    G.gw_set_coulomb(ctx, Vd)
    P0t = torch.empty(s["Pt"], dtype=torch.complex128, device="cuda")
    G.gw_polarization(ctx, Gd, P0t)
    Pt = torch.empty_like(P0t)
    G.gw_screened_interaction(ctx, P0t, Pt)
    Sig = torch.empty(s["Sig"], dtype=torch.complex128, device="cuda")
    G.gw_self_energy(ctx, Gd, Pt, Sig)
    Sig2 = torch.zeros_like(Sig)
    G.gw_sigma_eval(ctx, Gd, Sig2)
    G.gw_synchronize(ctx)
    out = {"P0t": host(P0t), "Pt": host(Pt), "Sig": host(Sig), "Sig_eval": host(Sig2)}
    ctx.destroy()
    return out


@pytest.mark.parametrize("nk3,nao,naux,ntau,beta,chunk,vs", CASES)
def test_fused_chain_against_oracle_and_slicing_pass(G, nk3, nao, naux, ntau, beta, chunk, vs):
    w = I.Workload("f", nk3, nao, naux, ntau, ntau, beta, 0.0, 6.0, 7 * nao + naux, solid=int(np.prod(nk3)) > 1)
    h, v, g = I.make_inputs(w)
    ref = O.sigma_eval(v, g, nk3, beta, spin_factor=2.0)
    fused = run(G, w, v, g, tau_chunk=chunk, v_slices=vs)
    for k in ("P0t", "Pt", "Sig"):
        assert rel(fused[k], ref[k]) < TOL, k
    # gw_sigma_eval builds P~ from the canonical (q, n) and the mirror relation: FP64 rounding apart
    assert rel(fused["Sig_eval"], fused["Sig"]) < 1e-8
    sep = run(G, w, v, g, tau_chunk=chunk, v_slices=vs, slice_pass=True)
    assert rel(sep["Sig"], ref["Sig"]) < TOL
    # the two differ only in chunking and rounding order, far below the tolerance
    assert rel(fused["Sig"], sep["Sig"]) < 1e-8


def test_fused_packed_v_equals_full_v(G):
    """A packed V gives the fused path bit for bit what the full V gives, in both V slicing modes."""
    w = I.Workload("fp", (2, 2, 1), 8, 40, 5, 5, 9.0, 0.0, 6.0, 77, solid=True)
    h, v, g = I.make_inputs(w)
    for vs in (G.GW_V_ALL_PAIRS, G.GW_V_PER_Q):
        a = run(G, w, v, g, v_slices=vs)
        b = run(G, w, v, g, v_slices=vs, v_packed=True)
        assert np.array_equal(a["Sig"], b["Sig"])


def test_fused_target_against_fp64(G):
    """max |dSigma| <= 1e-6 Ha against the GPU FP64 path on a solid of the fused shape."""
    w = I.Workload("ft", (2, 2, 1), 52, 200, 12, 12, 50.0, 0.0, 40.0, 5, solid=True)
    h, v, g = I.make_inputs(w)
    out = {}
    for prec in ("fp64", "bf16x3"):
        ctx = G.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision=prec)
        G.gw_set_coulomb(ctx, dev(v))
        S = torch.empty(ctx.shapes()["Sig"], dtype=torch.complex128, device="cuda")
        G.gw_sigma_eval(ctx, dev(g), S)
        G.gw_synchronize(ctx)
        out[prec] = host(S)
        ctx.destroy()
    err = float(np.max(np.abs(out["bf16x3"] - out["fp64"])))
    print(f"fused solid nao=52: max|dSigma| = {err:.3e} Ha, max|Sigma| = {np.abs(out['fp64']).max():.3f} Ha")
    assert err <= 1e-6
