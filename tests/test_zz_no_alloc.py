"""The allocation-free P0 entry point against the context-based one.

gw_polarization_noalloc serves callers that cannot allocate device memory
when they call (inside a CUDA-graph capture, or with a device budget already
given to their own pools). It must give the same P0 as gw_polarization, on
two calls in a row (the scratch array keeps the previous call's contents).
This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2406_18479_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("nk3,nao,naux,ntau", [((2, 2, 1), 5, 12, 7), ((1, 1, 1), 8, 32, 32),
                                                ((3, 3, 1), 26, 200, 5)])
def test_noalloc_matches_context_path_twice(nk3, nao, naux, ntau):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_18479_gb300 import gw
    w = I.Workload("na", nk3, nao, naux, ntau, ntau, 10.0, 0.0, 8.0, 31 + nao, solid=int(np.prod(nk3)) > 1)
    h, v, g = I.make_inputs(w)
    V = torch.from_numpy(v).cuda()
    G = torch.from_numpy(g).cuda()
    ctx = gw.gw_create(nk3, nao, naux, ntau, w.beta, precision="fp64")
    gw.gw_set_coulomb(ctx, V)
    ref = torch.empty(ctx.shapes()["Pt"], dtype=torch.complex128, device="cuda")
    gw.gw_polarization(ctx, G, ref)
    gw.gw_synchronize(ctx)
    ref_h = ref.cpu().numpy()
    ctx.destroy()
    for _ in range(2):
        out = torch.full_like(ref, complex(np.nan, np.nan))
        gw.gw_polarization_noalloc(nk3, nao, naux, ntau, 2.0, V, G, out)
        torch.cuda.synchronize()
        assert rel(out.cpu().numpy(), ref_h) < TOL


def test_noalloc_rejects_oversized_problem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_18479_gb300 import gw
    nk3, nao, naux, ntau = (1, 1, 1), 160, 100, 1     # 2 * 100 * 160^2 = 5.1 Mi elements > 4 Mi
    V = torch.zeros((1, 1, naux, nao, nao), dtype=torch.complex128, device="cuda")
    G = torch.zeros((1, ntau, nao, nao), dtype=torch.complex128, device="cuda")
    P = torch.zeros((1, ntau, naux, naux), dtype=torch.complex128, device="cuda")
    with pytest.raises(gw.GWError) as e:
        gw.gw_polarization_noalloc(nk3, nao, naux, ntau, 2.0, V, G, P)
    assert e.value.code == gw.GW_EINVAL
    assert "scratch" in str(e.value)
