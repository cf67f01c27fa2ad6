"""The self-energy of a range of momentum transfers, gw_sigma_eval_q.

Eq. sigma_gw sums over q, and P0^q (Eq. tilde_P0_tau) and P~^q (Eq. tilde_P_omega) are per
q, so the part of Sigma from a range of q is a complete, checkable unit: it is what a GPU owns
when the path shards over q, and what a sampled accuracy check compares between precisions.

Checked against the oracle's self_energy restricted to the same q (its q_list), with P0 and P~
of the range against the oracle's per-q stages; the full range equals gw_sigma_eval bit for bit;
disjoint ranges add up to the full Sigma; a q whose -q lies outside its range (computed at every
tau node instead of by the mirror relation) still matches. Tolerances: FP64 1e-10 relative
max-norm; mixed 1e-7 relative to the largest |Sigma| of the full evaluation.
"""
import numpy as np
import pytest

from oracle import grids, gw as O
from paper_2406_18479_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b, scale=None):
    s = np.max(np.abs(b)) if scale is None else scale
    return float(np.max(np.abs(a - b)) / max(s, 1e-300))


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_18479_gb300 import gw
    gw.lib()
    return gw


CASES = [
    # nk3, nao, naux, ntau, beta, ranges (a partition of [0, nk))
    ((3, 1, 1), 5, 14, 8, 8.0, [(0, 1), (1, 2), (2, 3)]),      # q = 1 and q = 2 are each other's -q
    ((2, 2, 1), 6, 20, 9, 12.0, [(0, 3), (3, 4)]),
    ((3, 2, 1), 8, 24, 10, 10.0, [(0, 2), (2, 5), (5, 6)]),
]


def setup(G, nk3, nao, naux, ntau, beta, prec):
    w = I.Workload("q", nk3, nao, naux, ntau, ntau, beta, 0.0, 6.0, 40 + nao, solid=True)
    h, v, g = I.make_inputs(w)
    ctx = G.gw_create(nk3, nao, naux, ntau, beta, precision=prec)
    V = torch.from_numpy(v).cuda()
    Gd = torch.from_numpy(g).cuda()
    G.gw_set_coulomb(ctx, V)
    return w, v, g, ctx, V, Gd


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("bf16x3", 1e-7)])
@pytest.mark.parametrize("nk3,nao,naux,ntau,beta,ranges", CASES)
def test_sigma_eval_q_against_oracle(G, prec, tol, nk3, nao, naux, ntau, beta, ranges):
    w, v, g, ctx, V, Gd = setup(G, nk3, nao, naux, ntau, beta, prec)
    nk = w.nk
    full = torch.empty(ctx.shapes()["Sig"], dtype=torch.complex128, device="cuda")
    G.gw_sigma_eval(ctx, Gd, full)
    # oracle stages for every q
    p0 = O.polarization(v, g, nk3, 2.0)
    _, F, B = grids.transform_matrices(ntau, beta, 0)
    _, _, pt = O.screened_interaction(p0, F, B)
    ref_full = O.self_energy(v, g, pt, nk3)
    scale = np.max(np.abs(ref_full))
    total = torch.zeros_like(full)
    for q0, q1 in ranges:
        part = torch.full_like(full, complex(np.nan, np.nan))
        P0q = torch.empty((q1 - q0, ntau, naux, naux), dtype=torch.complex128, device="cuda")
        Ptq = torch.empty_like(P0q)
        G.gw_sigma_eval_q(ctx, Gd, part, q0, q1, P0q, Ptq)
        torch.cuda.synchronize()
        assert rel(P0q.cpu().numpy(), p0[q0:q1]) < tol
        assert rel(Ptq.cpu().numpy(), pt[q0:q1]) < tol
        ref = O.self_energy(v, g, pt, nk3, q_list=list(range(q0, q1)))
        assert rel(part.cpu().numpy(), ref, scale) < tol
        total += part
    # the parts add up to the full evaluation
    assert rel(total.cpu().numpy(), full.cpu().numpy()) < (1e-13 if prec == "fp64" else tol)
    assert rel(full.cpu().numpy(), ref_full) < tol
    # the whole range is gw_sigma_eval itself
    whole = torch.empty_like(full)
    G.gw_sigma_eval_q(ctx, Gd, whole, 0, nk)
    torch.cuda.synchronize()
    assert torch.equal(whole, full)
    ctx.destroy()


def test_sigma_eval_q_empty_and_bad_ranges(G):
    w, v, g, ctx, V, Gd = setup(G, (2, 1, 1), 4, 9, 6, 6.0, "fp64")
    out = torch.full(ctx.shapes()["Sig"], complex(1.0, 1.0), dtype=torch.complex128, device="cuda")
    G.gw_sigma_eval_q(ctx, Gd, out, 1, 1)
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0
    for q0, q1 in [(-1, 1), (0, 3), (2, 1)]:
        with pytest.raises(G.GWError) as e:
            G.gw_sigma_eval_q(ctx, Gd, out, q0, q1)
        assert e.value.code == G.GW_EINVAL
    ctx.destroy()
