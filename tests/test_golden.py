"""The stored fixtures of tests/golden/ (written by tests/golden/make_golden.py from the oracle):
the oracle still reproduces them, the library's IR builder lands on the same nodes, and the GPU
self-energy matches the stored values without the oracle at run time."""
import os
import sys

import numpy as np
import pytest

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, HERE)
import make_golden as MG  # noqa: E402


def load(name):
    return np.loadtxt(os.path.join(HERE, name), comments="#")


def stored_sigma(shape):
    a = load("sigma_gw_small.txt")
    return (a[:, 0] + 1j * a[:, 1]).reshape(shape)


def test_oracle_reproduces_the_stored_sigma():
    from oracle import gw as O
    w, (h, v, g) = MG.small_case()
    sig = O.sigma_eval(v, g, w.nk3, w.beta, 2.0)["Sig"]
    assert np.abs(sig - stored_sigma(sig.shape)).max() < 1e-14 * np.abs(sig).max()


def test_ir_nodes_match_the_stored_ones():
    from paper_2406_18479_gb300 import gw
    try:
        gw.lib()
    except RuntimeError as e:
        pytest.skip(str(e))
    tau = gw.gw_ir_grids(10.0, 100.0, 1e-10)[0]
    ref = load("ir_nodes_l100.txt")
    assert len(tau) == len(ref) and np.abs(tau - ref).max() < 1e-5 * 10.0


@pytest.mark.gpu
def test_gpu_sigma_matches_the_stored_values():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_18479_gb300 import gw
    w, (h, v, g) = MG.small_case()
    ctx = gw.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision="fp64")
    vd = torch.from_numpy(v).cuda()
    gw.gw_set_coulomb(ctx, vd)
    S = torch.empty(ctx.shapes()["Sig"], dtype=torch.complex128, device="cuda")
    gw.gw_sigma_eval(ctx, torch.from_numpy(g).cuda(), S)
    gw.gw_synchronize(ctx)
    ref = stored_sigma(tuple(S.shape))
    assert np.abs(S.cpu().numpy() - ref).max() < 1e-10 * np.abs(ref).max()
    ctx.destroy()
