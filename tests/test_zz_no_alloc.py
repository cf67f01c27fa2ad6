"""The allocation-free P0 entry point against the FP64 oracle and the context-based one.

gw_polarization_noalloc serves callers that cannot allocate device memory when they call: a
host that committed all its device memory to its own pools at start-up, or a runtime that
forbids allocation after initialisation. Its V.G intermediates live in one fixed scratch array
inside the library, so problems whose k sum does not fit are split into k chunks that
accumulate into P0t. It must give the P0 of the oracle (Eq. tilde_P0_tau) and of
gw_polarization, on two calls in a row (the array keeps the previous call's contents), for one
k chunk and for several (an uneven last chunk included). This file is collected last on purpose.
"""
import numpy as np
import pytest

from oracle import gw as O
from paper_2406_18479_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10
SCRATCH_ELEMS = 4 * 1024 * 1024      # the library's fixed array, complex elements


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def k_chunk(nk, nao, naux):
    """k points per chunk as the entry point splits the sum (for the test's own bookkeeping)."""
    return min(nk, SCRATCH_ELEMS // (2 * naux * nao * nao))


@pytest.mark.parametrize("nk3,nao,naux,ntau,oracle_q,oracle_t", [
    ((2, 2, 1), 5, 12, 7, None, None),          # one k chunk, several tau per round
    ((1, 1, 1), 8, 32, 32, None, None),
    ((3, 3, 1), 26, 200, 5, [0, 4], [0, 3]),    # 15 k per chunk >= 9: one chunk
    ((2, 1, 1), 64, 500, 2, None, None),        # one k per chunk: two chunks, the second accumulates
    ((3, 3, 3), 26, 200, 2, [0, 13], [1]),      # chunks of 15 and 12 k points
])
def test_noalloc_matches_oracle_and_context_path_twice(nk3, nao, naux, ntau, oracle_q, oracle_t):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_18479_gb300 import gw
    nk = int(np.prod(nk3))
    w = I.Workload("na", nk3, nao, naux, ntau, ntau, 10.0, 0.0, 8.0, 31 + nao, solid=nk > 1)
    h, v, g = I.make_inputs(w)
    kc = k_chunk(nk, nao, naux)
    # the oracle's P0 (all of it, or a sample of (q, tau) for the larger cases)
    ql = list(range(nk)) if oracle_q is None else oracle_q
    tl = list(range(ntau)) if oracle_t is None else oracle_t
    ref_oracle = O.polarization(v, g, nk3, 2.0, q_list=ql, t_list=tl)
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
        o = out.cpu().numpy()
        assert rel(o[np.ix_(ql, tl)], ref_oracle) < TOL, f"k chunk {kc} of {nk}"
        assert rel(o, ref_h) < TOL


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


def test_noalloc_rejects_host_memory_through_the_c_abi():
    """A pointer that is not device memory of the current device is refused before any launch."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import ctypes
    from paper_2406_18479_gb300 import gw
    nk3, nao, naux, ntau = (1, 1, 1), 4, 8, 3
    V = torch.zeros((1, 1, naux, nao, nao), dtype=torch.complex128, device="cuda")
    G_host = torch.zeros((1, ntau, nao, nao), dtype=torch.complex128)
    P = torch.zeros((1, ntau, naux, naux), dtype=torch.complex128, device="cuda")
    arr = (ctypes.c_int * 3)(*nk3)
    rc = gw.lib().gw_polarization_noalloc(arr, nao, naux, ntau, 2.0, ctypes.c_void_p(V.data_ptr()),
                                          ctypes.c_void_p(G_host.data_ptr()), ctypes.c_void_p(P.data_ptr()), None)
    assert rc == gw.GW_EINVAL
    assert b"G_dev" in gw.lib().gw_last_error()
