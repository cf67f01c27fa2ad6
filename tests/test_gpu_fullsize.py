"""Parity at the benchmarked size: the Si-like 3x3x3 solid (nk=27, nao=26, naux=200,
ntau=100, beta=100), run through the C ABI exactly as bench.py runs it (automatic tau
batches), in FP64 and in the mixed precision the benchmark times.

The oracle cannot produce whole arrays at this size in test time, so it recomputes
samples one by one from the same inputs: P0 at sampled (q, tau); P~ of one q from
its own P0 of that q; and Sigma at sampled (k, tau) from the GPU's P~ (which checks
step a5 on its own at full size). Tolerances: FP64 1e-10 relative; mixed 1e-7
relative per sampled array, and the target max |dSigma| <= 1e-6 Ha against the FP64
path over the whole array.
"""
import numpy as np
import pytest

from oracle import grids, gw as O
from paper_2406_18479_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W = I.WORKLOADS["solid_3x3x3_nao26"]


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def inputs():
    return I.make_inputs(W)


def run(precision, v, g):
    from paper_2406_18479_gb300 import gw
    ctx = gw.gw_create(W.nk3, W.nao, W.naux, W.ntau, W.beta, precision=precision)
    s = ctx.shapes()
    V = torch.from_numpy(v).cuda()
    Gd = torch.from_numpy(g).cuda()
    gw.gw_set_coulomb(ctx, V)
    P0t = torch.empty(s["Pt"], dtype=torch.complex128, device="cuda")
    gw.gw_polarization(ctx, Gd, P0t)
    Pt = torch.empty_like(P0t)
    gw.gw_screened_interaction(ctx, P0t, Pt)
    Sig = torch.empty(s["Sig"], dtype=torch.complex128, device="cuda")
    gw.gw_self_energy(ctx, Gd, Pt, Sig)
    Sig2 = torch.empty_like(Sig)
    gw.gw_sigma_eval(ctx, Gd, Sig2)
    gw.gw_synchronize(ctx)
    out = {"P0t": P0t.cpu().numpy(), "Pt": Pt.cpu().numpy(), "Sig": Sig.cpu().numpy(), "Sig_eval": Sig2.cpu().numpy()}
    ctx.destroy()
    return out


@pytest.fixture(scope="module")
def gpu(inputs):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    h, v, g = inputs
    return {"fp64": run("fp64", v, g), "bf16x3": run("bf16x3", v, g)}


@pytest.fixture(scope="module")
def samples(inputs):
    """Oracle samples: P0 at 2 q x 5 tau, P~ of one q (all tau)."""
    h, v, g = inputs
    rng = np.random.default_rng(12)
    q_s = sorted(rng.choice(W.nk, 2, replace=False).tolist())
    t_s = sorted(rng.choice(W.ntau, 3, replace=False).tolist()) + [0, W.ntau - 1]
    p0 = O.polarization(v, g, W.nk3, 2.0, q_list=q_s, t_list=t_s)
    q1 = q_s[:1]
    p0_q = O.polarization(v, g, W.nk3, 2.0, q_list=q1)
    _, F, B = grids.transform_matrices(W.ntau, W.beta, 0)
    _, _, pt_q = O.screened_interaction(p0_q, F, B)
    kt = [(int(rng.integers(W.nk)), int(rng.integers(W.ntau))) for _ in range(3)] + [(0, 0)]
    return {"q_s": q_s, "t_s": t_s, "p0": p0, "q1": q1, "pt_q": pt_q, "kt": kt}


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("bf16x3", 1e-7)])
def test_polarization_sampled(gpu, samples, precision, tol):
    out = gpu[precision]
    assert rel(out["P0t"][samples["q_s"]][:, samples["t_s"]], samples["p0"]) < tol


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("bf16x3", 1e-7)])
def test_screened_interaction_one_q(gpu, samples, precision, tol):
    out = gpu[precision]
    assert rel(out["Pt"][samples["q1"]], samples["pt_q"]) < tol


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("bf16x3", 1e-7)])
def test_self_energy_sampled_from_gpu_pt(gpu, inputs, samples, precision, tol):
    h, v, g = inputs
    out = gpu[precision]
    for k, t in samples["kt"]:
        ref = O.self_energy(v, g, out["Pt"], W.nk3, k_list=[k], t_list=[t])[0, 0]
        assert rel(out["Sig"][k, t], ref) < tol, (k, t)


def test_sigma_eval_equals_staged_calls(gpu):
    # gw_sigma_eval solves the aux Dyson equation at canonical (q, n) only and mirrors the rest,
    # the staged gw_screened_interaction solves every (q, n): equal up to FP64 rounding order.
    # In the mixed precision P~ is then cut into slices whose last digit is 2^-32 of the chunk
    # maximum, so a rounding-order difference in P~ can move Sigma by up to that: 5e-10.
    for prec, tol in (("fp64", 1e-11), ("bf16x3", 5e-10)):
        out = gpu[prec]
        assert rel(out["Sig_eval"], out["Sig"]) < tol


def test_mixed_target_against_fp64(gpu):
    s64, smx = gpu["fp64"]["Sig"], gpu["bf16x3"]["Sig"]
    err = float(np.max(np.abs(smx - s64)))
    print(f"3x3x3 solid: max|dSigma| mixed vs FP64 = {err:.3e} Ha, max|Sigma| = {np.abs(s64).max():.1f} Ha")
    assert err <= 1e-6
    assert rel(s64, s64.conj().swapaxes(-1, -2)) < 1e-11
