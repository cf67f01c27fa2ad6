"""GPU parity of the k-space interpolation (Sec. 2.5) against the oracle, and the paper's use of
it: interpolate Sigma^inf and Sigma~ to a k path, solve the Dyson equation there."""
import numpy as np
import pytest

from oracle import gw as O
from oracle import kinterp as K
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


@pytest.mark.parametrize("nk3", [(1, 1, 1), (3, 3, 1), (2, 2, 2), (4, 1, 3)])
def test_against_oracle(G, nk3):
    rng = np.random.default_rng(3)
    nk = int(np.prod(nk3))
    X = rng.standard_normal((nk, 5, 3, 3)) + 1j * rng.standard_normal((nk, 5, 3, 3))
    f = np.concatenate([K.mesh_fractions(nk3)[:2], rng.uniform(-1, 1, (9, 3))])
    Xf = torch.empty((len(f), 5, 3, 3), dtype=torch.complex128, device="cuda")
    G.gw_k_interpolate(nk3, dev(X), f, Xf)
    torch.cuda.synchronize()
    got = Xf.cpu().numpy()
    assert rel(got, K.k_interpolate(X, nk3, f)) < 1e-13
    assert np.abs(got[:2] - X[:2]).max() < 1e-13 * np.abs(X).max()      # exact on the mesh


def test_dyson_on_a_k_path(G):
    """Sigma^inf and Sigma~ of a 2x2x1 solid interpolated to 6 path points, H interpolated too
    (nearest-neighbour, hence exact), G on the path by the Dyson equation: against the oracle."""
    nk3, nao, naux, ntau, beta = (2, 2, 1), 3, 6, 8, 6.0
    w = I.Workload("path", nk3, nao, naux, ntau, ntau, beta, 0.0, 4.0, 13, solid=True)
    h, v, g = I.make_inputs(w)
    ctx = G.gw_create(nk3, nao, naux, ntau, beta, precision="fp64")
    vd = dev(v)
    G.gw_set_coulomb(ctx, vd)
    gd = dev(g)
    S = torch.empty(ctx.shapes()["Sig"], dtype=torch.complex128, device="cuda")
    Sinf = torch.empty((w.nk, nao, nao), dtype=torch.complex128, device="cuda")
    G.gw_sigma_eval(ctx, gd, S)
    G.gw_sigma_inf(ctx, gd, Sinf)
    f = np.stack([np.linspace(0, 0.5, 6), np.linspace(0, 0.25, 6), np.zeros(6)], axis=1)
    nkf = len(f)
    Sf = torch.empty((nkf, ntau, nao, nao), dtype=torch.complex128, device="cuda")
    If = torch.empty((nkf, nao, nao), dtype=torch.complex128, device="cuda")
    Hf = torch.empty_like(If)
    G.gw_k_interpolate(nk3, S, f, Sf)
    G.gw_k_interpolate(nk3, Sinf, f, If)
    G.gw_k_interpolate(nk3, dev(h), f, Hf)
    path = G.gw_create((nkf, 1, 1), nao, naux, ntau, beta, precision="fp64")
    Gf = torch.empty((nkf, ntau, nao, nao), dtype=torch.complex128, device="cuda")
    G.gw_dyson_G(path, Hf + If, Sf, Gf)
    torch.cuda.synchronize()
    s_or = O.sigma_eval(v, g, nk3, beta)["Sig"]
    i_or = O.sigma_inf(v, O.density_matrix(g, beta), nk3, 2.0)
    ref = O.dyson_G(K.k_interpolate(h, nk3, f) + K.k_interpolate(i_or, nk3, f), K.k_interpolate(s_or, nk3, f),
                    0.0, beta)
    assert rel(Gf.cpu().numpy(), ref) < 1e-10
    ctx.destroy()
    path.destroy()


def test_bad_arguments(G):
    X = torch.zeros((4, 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(G.GWError):
        G.gw_k_interpolate((2, 2, 1), X, np.zeros((3, 3)), torch.zeros((2, 2), dtype=torch.complex128, device="cuda"))
    with pytest.raises(G.GWError):
        G.gw_k_interpolate((0, 2, 1), torch.zeros((0, 2), dtype=torch.complex128, device="cuda"), np.zeros((1, 3)),
                           torch.zeros((1, 2), dtype=torch.complex128, device="cuda"))
