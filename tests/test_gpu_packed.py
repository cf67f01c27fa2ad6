"""The packed Coulomb factor (pairs k1 <= k2 only, V^{k2 k1}_ij(Q) = conj V^{k1 k2}_ji(Q)) gives
bit for bit what the full V gives, in every path that reads V: the FP64 and mixed-precision
self-energy (all-pair and per-q slices), the static self-energy, GF2, and a serving job."""
import numpy as np
import pytest

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


def case(nk3, nao, naux, ntau, seed):
    w = I.Workload("packed", nk3, nao, naux, ntau, ntau, 8.0, 0.0, 4.0, seed, solid=True)
    h, v, g = I.make_inputs(w)
    # the generator's V has the symmetry exactly (the lower pairs are conjugate transposes)
    for a in range(w.nk):
        for b in range(w.nk):
            assert np.array_equal(v[b, a], v[a, b].conj().transpose(0, 2, 1))
    return w, h, v, g


def pair_of_contexts(G, w, **kw):
    full = G.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, **kw)
    packed = G.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, v_packed=True, **kw)
    return full, packed


@pytest.mark.parametrize("prec,v_slices", [("fp64", 0), ("bf16x3", 1), ("bf16x3", 2)])
@pytest.mark.parametrize("nk3", [(2, 2, 1), (3, 1, 1)])
def test_sigma_eval_and_static_part(G, prec, v_slices, nk3):
    w, h, v, g = case(nk3, 5, 9, 6, 3)
    full, packed = pair_of_contexts(G, w, precision=prec, v_slices=v_slices)
    assert packed.shapes()["V"] == (w.nk * (w.nk + 1) // 2, w.naux, w.nao, w.nao)
    vf, vp = dev(v), dev(I.pack_v(v))
    G.gw_set_coulomb(full, vf)
    G.gw_set_coulomb(packed, vp)
    gd = dev(g)
    s1 = torch.empty(full.shapes()["Sig"], dtype=torch.complex128, device="cuda")
    s2 = torch.empty_like(s1)
    G.gw_sigma_eval(full, gd, s1)
    G.gw_sigma_eval(packed, gd, s2)
    torch.cuda.synchronize()
    assert torch.equal(s1, s2)
    i1 = torch.empty((w.nk, w.nao, w.nao), dtype=torch.complex128, device="cuda")
    i2 = torch.empty_like(i1)
    G.gw_sigma_inf(full, gd, i1)
    G.gw_sigma_inf(packed, gd, i2)
    torch.cuda.synchronize()
    assert torch.equal(i1, i2)
    assert packed.workspace_bytes() > 0
    full.destroy()
    packed.destroy()


@pytest.mark.parametrize("prec", ["fp64", "bf16x4"])
def test_static_part_above_the_fused_exchange_limit(G, prec):
    """nao = 56 is above the fused exchange kernel's limit (52): the exchange takes the GEMM path,
    which with only the packed V resident unpacks V^{kk'} and V^{k'k} per (k, k')."""
    w, h, v, g = case((2, 1, 1), 56, 8, 4, 5)
    full, packed = pair_of_contexts(G, w, precision=prec)
    G.gw_set_coulomb(full, dev(v))
    G.gw_set_coulomb(packed, dev(I.pack_v(v)))
    gd = dev(g)
    i1 = torch.empty((w.nk, w.nao, w.nao), dtype=torch.complex128, device="cuda")
    i2 = torch.empty_like(i1)
    G.gw_sigma_inf(full, gd, i1)
    G.gw_sigma_inf(packed, gd, i2)
    torch.cuda.synchronize()
    assert torch.equal(i1, i2)
    full.destroy()
    packed.destroy()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_gf2(G, prec):
    w, h, v, g = case((2, 1, 1), 4, 6, 4, 5)
    full, packed = pair_of_contexts(G, w, precision=prec)
    vf, vp = dev(v), dev(I.pack_v(v))
    G.gw_set_coulomb(full, vf)
    G.gw_set_coulomb(packed, vp)
    gd = dev(g)
    s1 = torch.empty(full.shapes()["Sig"], dtype=torch.complex128, device="cuda")
    s2 = torch.empty_like(s1)
    G.gw_gf2_self_energy(full, gd, s1)
    G.gw_gf2_self_energy(packed, gd, s2)
    torch.cuda.synchronize()
    assert torch.equal(s1, s2)
    full.destroy()
    packed.destroy()


def test_serving_job_and_bytes(G):
    w, h, v, g = case((2, 2, 1), 4, 8, 6, 7)
    cf = G.make_config(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision="bf16x3", v_slices=2)
    cp = G.make_config(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision="bf16x3", v_slices=2, v_packed=True)
    vbytes = 16 * w.naux * w.nao ** 2
    # the job's V shrinks from nk^2 to nk (nk + 1) / 2 blocks; the per-q scratch adds nk blocks
    # (and the scratch's 256-byte guard zone)
    assert G.gw_job_bytes(cf) - G.gw_job_bytes(cp) == vbytes * (w.nk * w.nk - w.nk * (w.nk + 1) // 2 - w.nk) - 256
    srv = G.gw_server(8 << 30, 2)
    out = []
    for cfg, vv in ((cf, v), (cp, I.pack_v(v))):
        S = np.empty(g.shape, complex)
        jid = srv.submit(cfg, h, np.ascontiguousarray(vv), g, S, None, alpha=0.5, tol=0.0, itermax=2)
        rc, res = srv.poll(jid, -1)
        assert rc == G.GW_OK and res["status"] in (G.GW_OK, G.GW_ENOTCONV)
        out.append(S)
    srv.destroy()
    assert np.array_equal(out[0], out[1])


def test_bad_packed_flag(G):
    with pytest.raises(G.GWError) as e:
        G.gw_create((1, 1, 1), 2, 2, 2, 1.0, v_packed=2)
    assert e.value.code == G.GW_EINVAL
