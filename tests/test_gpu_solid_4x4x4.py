"""Parity at the size of the 4x4x4 solid (nk=64, nao=52, naux=400, ntau=120, beta=200) in the
mixed precision. V alone is 71 GB, so the bf16 slices of V are made per q (automatic at this
size) and the tau batch is set to 15 nodes (300 P0 tiles per launch).

The oracle recomputes samples from the same inputs: P0 at 2 q x 3 tau; P~ of one q from the
GPU's own P0 of that q (steps a2-a4 at full size); Sigma at 4 k x 8 tau from the GPU's P~
(step a5 at full size). Tolerance 1e-7 relative per sampled array.

Accuracy in Ha: one FP64 evaluation at this size is about an hour of FP64 work, so the mixed
path is compared with the GPU FP64 path on the part of Sigma from one momentum transfer
(Eq. sigma_gw sums over q; gw_sigma_eval_q), q = 0, whose cost is the average per-q cost. The
full Sigma sums 64 such parts; their rounding errors are independent, so the full error is
about sqrt(64) times the part's (the test asserts that this estimate meets 1e-6 Ha, i.e. the
part's error is at most 1.25e-7 Ha); the triangle inequality bounds it by 64 times the part's.
"""
import numpy as np
import pytest

from oracle import grids, gw as O
from paper_2406_18479_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W = I.WORKLOADS["solid_4x4x4_nao52"]
TOL = 1e-7


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def run():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_18479_gb300 import gw
    h, v, g = I.make_inputs(W)
    ctx = gw.gw_create(W.nk3, W.nao, W.naux, W.ntau, W.beta, precision="bf16x3", tau_chunk=15)
    s = ctx.shapes()
    Gd = torch.from_numpy(g).cuda()
    V = torch.from_numpy(v).cuda()
    gw.gw_set_coulomb(ctx, V)
    P0t = torch.empty(s["Pt"], dtype=torch.complex128, device="cuda")
    gw.gw_polarization(ctx, Gd, P0t)
    Pt = torch.empty_like(P0t)
    gw.gw_screened_interaction(ctx, P0t, Pt)
    Sig = torch.empty(s["Sig"], dtype=torch.complex128, device="cuda")
    gw.gw_self_energy(ctx, Gd, Pt, Sig)
    gw.gw_synchronize(ctx)
    # the part of Sigma from q = 0, mixed (this context) and FP64 (after this context is gone)
    Sig_q = torch.empty_like(Sig)
    gw.gw_sigma_eval_q(ctx, Gd, Sig_q, 0, 1)
    gw.gw_synchronize(ctx)
    sig_q_mixed = Sig_q.cpu().numpy()
    rng = np.random.default_rng(3)
    q_s = sorted(rng.choice(W.nk, 2, replace=False).tolist())
    t_s = sorted(rng.choice(W.ntau, 3, replace=False).tolist())
    k_s = sorted(rng.choice(W.nk, 4, replace=False).tolist())
    kt_t = sorted(rng.choice(W.ntau, 8, replace=False).tolist())
    out = {"P0_s": P0t[q_s][:, t_s].cpu().numpy(), "P0_q": P0t[q_s[:1]].cpu().numpy(),
           "Pt_q": Pt[q_s[:1]].cpu().numpy(), "Pt": Pt.cpu().numpy(),
           "Sig_s": Sig[k_s][:, kt_t].cpu().numpy(), "q_s": q_s, "t_s": t_s, "k_s": k_s, "kt_t": kt_t}
    ctx.destroy()
    del P0t, Pt, Sig
    torch.cuda.empty_cache()
    c64 = gw.gw_create(W.nk3, W.nao, W.naux, W.ntau, W.beta, precision="fp64")
    gw.gw_set_coulomb(c64, V)
    gw.gw_sigma_eval_q(c64, Gd, Sig_q, 0, 1)
    gw.gw_synchronize(c64)
    out["sig_q_fp64"] = Sig_q.cpu().numpy()
    out["sig_q_mixed"] = sig_q_mixed
    c64.destroy()
    del V, Gd, Sig_q
    torch.cuda.empty_cache()
    return h, v, g, out


def test_solid_4x4x4_polarization_sampled(run):
    h, v, g, out = run
    ref = O.polarization(v, g, W.nk3, 2.0, q_list=out["q_s"], t_list=out["t_s"])
    assert rel(out["P0_s"], ref) < TOL


def test_solid_4x4x4_screened_interaction_from_gpu_p0(run):
    h, v, g, out = run
    _, F, B = grids.transform_matrices(W.ntau, W.beta, 0)
    _, _, pt = O.screened_interaction(out["P0_q"], F, B)
    assert rel(out["Pt_q"], pt) < 1e-10


def test_solid_4x4x4_self_energy_sampled_from_gpu_pt(run):
    h, v, g, out = run
    ref = O.self_energy(v, g, out["Pt"], W.nk3, k_list=out["k_s"], t_list=out["kt_t"])
    assert rel(out["Sig_s"], ref) < TOL


def test_solid_4x4x4_sigma_part_of_q0_within_the_ha_target(run):
    h, v, g, out = run
    err = float(np.max(np.abs(out["sig_q_mixed"] - out["sig_q_fp64"])))
    print(f"4x4x4 solid, q = 0: max|dSigma_q| = {err:.3e} Ha (max|Sigma_q| = {np.abs(out['sig_q_fp64']).max():.2f} Ha); "
          f"full Sigma: estimate {np.sqrt(W.nk) * err:.2e} Ha, bound {W.nk * err:.2e} Ha")
    assert err * np.sqrt(W.nk) <= 1e-6
