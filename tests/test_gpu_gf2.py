"""GPU parity of the second-order self-energy (Eq. sigma2) and of the loop that uses it, against
the FP64 oracle on the same seeded inputs. Tolerance: relative max-norm 1e-10 in FP64; the mixed
precision runs the direct term on the tensor cores (its GW tolerance) and the exchange in FP64."""
import numpy as np
import pytest

from oracle import gf2 as F
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


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def case(nk3, nao, naux, ntau, beta, seed):
    w = I.Workload("gf2", nk3, nao, naux, ntau, ntau, beta, 0.1, 3.0, seed, solid=int(np.prod(nk3)) > 1)
    h, v, g = I.make_inputs(w)
    rng = np.random.default_rng(seed + 1)
    x = 0.02 * (rng.standard_normal(g.shape) + 1j * rng.standard_normal(g.shape))
    return w, h, v, g + 0.5 * (x + x.conj().swapaxes(-1, -2))


CASES = [
    # nk3, nao, naux, ntau, beta, tau_chunk
    ((1, 1, 1), 1, 1, 2, 5.0, 0),
    ((1, 1, 1), 3, 4, 5, 4.0, 2),
    ((2, 1, 1), 2, 3, 4, 4.0, 3),
    ((3, 1, 1), 4, 6, 6, 6.0, 0),
    ((2, 2, 1), 3, 5, 4, 5.0, 1),
    ((1, 1, 1), 13, 30, 8, 10.0, 0),
    ((1, 1, 1), 33, 40, 4, 10.0, 3),
]


@pytest.mark.parametrize("nk3,nao,naux,ntau,beta,chunk", CASES)
def test_gf2_fp64(G, nk3, nao, naux, ntau, beta, chunk):
    w, h, v, g = case(nk3, nao, naux, ntau, beta, 3 + nao)
    d, x = F.gf2_terms(v, g, nk3, 2.0)
    ctx = G.gw_create(nk3, nao, naux, ntau, beta, precision="fp64", tau_chunk=chunk)
    vd = dev(v)
    G.gw_set_coulomb(ctx, vd)
    gd = dev(g)
    S = torch.empty(ctx.shapes()["Sig"], dtype=torch.complex128, device="cuda")
    G.gw_gf2_exchange(ctx, gd, S)
    assert rel(host(S), x) < 1e-10
    G.gw_gf2_self_energy(ctx, gd, S)
    assert rel(host(S), d - x) < 1e-10
    ctx.destroy()


def test_gf2_mixed_precision(G):
    w, h, v, g = case((2, 1, 1), 12, 40, 10, 10.0, 9)
    ref = F.gf2_self_energy(v, g, w.nk3, 2.0)
    ctx = G.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision="bf16x3")
    vd = dev(v)
    G.gw_set_coulomb(ctx, vd)
    S = torch.empty(ctx.shapes()["Sig"], dtype=torch.complex128, device="cuda")
    G.gw_gf2_self_energy(ctx, dev(g), S)
    assert np.abs(host(S) - ref).max() < 1e-6          # Ha, the mixed-precision target
    ctx.destroy()


@pytest.mark.parametrize("kind", ["diis", "cdiis"])
def test_gf2_loop_matches_oracle(G, kind):
    w = I.Workload("gf2loop", (2, 1, 1), 3, 6, 12, 12, 5.0, 0.0, 3.0, 21, solid=True)
    h, v, g = I.make_inputs(w)
    v = 0.4 * v
    ref = O.scgw_full(h, v, g, w.nk3, w.beta, 0.0, alpha=0.7, tol=1e-10, itermax=60, n_electrons=2.0,
                      mu_lo=-4.0, mu_hi=4.0, mu_tol=1e-12, diis_size=4, diis_kind=kind, method="gf2")
    ctx = G.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision="fp64")
    vd = dev(v)
    G.gw_set_coulomb(ctx, vd)
    Gd = dev(g)
    S = torch.empty(ctx.shapes()["Sig"], dtype=torch.complex128, device="cuda")
    Sinf = torch.empty((w.nk, w.nao, w.nao), dtype=torch.complex128, device="cuda")
    opt = G.scgw_options(alpha=0.7, tol=1e-10, itermax=60, diis_size=4, n_electrons=2.0, mu_lo=-4.0, mu_hi=4.0,
                         mu_tol=1e-12, diis_kind=kind, method="gf2")
    rc, r = G.gw_scgw(ctx, dev(h), Gd, S, Sinf, opt)
    assert rc == G.GW_OK
    assert abs(r["iterations"] - ref["iterations"]) <= 1
    assert abs(r["mu"] - ref["mu"]) < 1e-9
    for got, want in ((S, ref["Sig"]), (Sinf, ref["SigInf"]), (Gd, ref["G"])):
        assert np.abs(host(got) - want).max() < 1e-9
    ctx.destroy()
