"""Failure detection on the GPU without faulting it: a device-side bounded wait that runs out
returns GW_EDEVTIMEOUT and leaves the device usable; workspace guard zones stay intact through
every path and a changed guard byte is reported."""
import numpy as np
import pytest

from oracle import gw as O
from paper_2406_18479_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_18479_gb300 import gw
    gw.lib()
    return gw


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def test_bounded_wait_gives_up_and_the_device_stays_usable(G):
    rc, code = G.gw_selftest_bounded_wait(0.2)
    assert rc == G.GW_EDEVTIMEOUT and code == 99
    w = I.Workload("after", (1, 1, 1), 3, 4, 4, 4, 5.0, 0.0, 4.0, 2)
    h, v, g = I.make_inputs(w)
    ctx = G.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision="bf16x3")
    vd = dev(v)
    G.gw_set_coulomb(ctx, vd)
    S = torch.empty(ctx.shapes()["Sig"], dtype=torch.complex128, device="cuda")
    G.gw_sigma_eval(ctx, dev(g), S)
    G.gw_synchronize(ctx)
    ref = O.sigma_eval(v, g, w.nk3, w.beta)["Sig"]
    assert np.abs(S.cpu().numpy() - ref).max() < 1e-6
    ctx.destroy()


@pytest.mark.parametrize("prec,v_slices,packed", [("fp64", 0, False), ("bf16x3", 1, False), ("bf16x3", 2, True)])
def test_guards_hold_through_every_path(G, prec, v_slices, packed):
    w = I.Workload("guards", (2, 1, 1), 5, 7, 6, 6, 6.0, 0.0, 4.0, 3, solid=True)
    h, v, g = I.make_inputs(w)
    ctx = G.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision=prec, v_slices=v_slices, v_packed=packed)
    vd = dev(I.pack_v(v) if packed else v)
    G.gw_set_coulomb(ctx, vd)
    gd = dev(g)
    S = torch.empty(ctx.shapes()["Sig"], dtype=torch.complex128, device="cuda")
    Sinf = torch.empty((w.nk, w.nao, w.nao), dtype=torch.complex128, device="cuda")
    G.gw_sigma_eval(ctx, gd, S)
    G.gw_sigma_inf(ctx, gd, Sinf)
    G.gw_gf2_self_energy(ctx, gd, S)
    rc, _ = G.gw_scgw(ctx, dev(h), gd.clone(), S, Sinf,
                      G.scgw_options(itermax=2, tol=0.0, diis_size=2, diis_kind="cdiis"))
    G.gw_check_guards(ctx)
    G.gw_debug_mark_guard(ctx, 0)
    with pytest.raises(G.GWError):
        G.gw_check_guards(ctx)
    ctx.destroy()
