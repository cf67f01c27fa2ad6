"""GPU parity of the self-consistency pieces beyond the GW self-energy: the density matrix and
static self-energy (Eq. sigma_inf), the particle number and chemical-potential search (Sec. 2.4),
and Pulay's extrapolation (Sec. 5.3), each against the FP64 oracle on the same seeded inputs.

All of these run in FP64 in every precision; tolerance: relative max-norm 1e-10 unless stated."""
import numpy as np
import pytest

from oracle import gw as O
from paper_2406_18479_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


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


def hermitian_noise(shape, scale, seed):
    rng = np.random.default_rng(seed)
    x = scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    return 0.5 * (x + x.conj().swapaxes(-1, -2))


CASES = [
    # nk3, nao, naux, ntau, beta, precision
    ((1, 1, 1), 1, 1, 2, 5.0, "fp64"),
    ((1, 1, 1), 3, 7, 9, 10.0, "fp64"),
    ((3, 1, 1), 5, 7, 6, 8.0, "fp64"),
    ((2, 2, 1), 3, 40, 9, 12.0, "fp64"),
    ((2, 1, 3), 2, 5, 4, 6.0, "fp64"),
    ((1, 1, 1), 33, 65, 8, 30.0, "fp64"),
    ((3, 3, 1), 7, 20, 12, 20.0, "bf16x3"),
    ((2, 1, 1), 53, 3, 2, 5.0, "fp64"),          # above the fused exchange kernel's limit: GEMM path
]


@pytest.mark.parametrize("nk3,nao,naux,ntau,beta,prec", CASES)
def test_density_sigma_inf_particle_number(G, nk3, nao, naux, ntau, beta, prec):
    w = I.Workload("static", nk3, nao, naux, ntau, ntau, beta, 0.1, 4.0, 17 + nao, solid=int(np.prod(nk3)) > 1)
    h, v, g = I.make_inputs(w)
    # a G that is not the non-interacting one: G0 plus a perturbation
    g = g + hermitian_noise(g.shape, 0.01, 3)
    gam_ref = O.density_matrix(g, beta)
    sinf_ref = O.sigma_inf(v, gam_ref, nk3, 2.0)
    ctx = G.gw_create(nk3, nao, naux, ntau, beta, precision=prec)
    G.gw_set_coulomb(ctx, dev(v))
    gd = dev(g)
    gam = torch.empty((w.nk, nao, nao), dtype=torch.complex128, device="cuda")
    G.gw_density(ctx, gd, gam)
    assert rel(host(gam), gam_ref) < 1e-12
    sinf = torch.empty_like(gam)
    G.gw_sigma_inf(ctx, gd, sinf)
    assert rel(host(sinf), sinf_ref) < TOL
    n = G.gw_particle_number(ctx, gd)
    assert abs(n - O.particle_number(gam_ref, 2.0)) < 1e-11 * max(1.0, abs(n))
    ctx.destroy()


def test_sigma_inf_requires_coulomb(G):
    ctx = G.gw_create((1, 1, 1), 2, 3, 4, 5.0)
    g = torch.zeros(ctx.shapes()["G"], dtype=torch.complex128, device="cuda")
    out = torch.empty((1, 2, 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(G.GWError) as e:
        G.gw_sigma_inf(ctx, g, out)
    assert e.value.code == G.GW_EINVAL
    ctx.destroy()


def test_density_on_a_given_tau_grid(G):
    """After gw_set_grids the density is the polynomial through the given nodes at tau = beta
    (checked against scipy's barycentric interpolator); the library's own grid is left first."""
    interp = pytest.importorskip("scipy.interpolate")
    nk3, nao, naux, ntau, beta = (2, 1, 1), 4, 5, 10, 6.0
    w = I.Workload("grid", nk3, nao, naux, ntau, ntau, beta, 0.0, 4.0, 5, solid=True)
    h, v, g = I.make_inputs(w)
    ctx = G.gw_create(nk3, nao, naux, ntau, beta, precision="fp64")
    tau0, mb, Fb, Bb = G.gw_grid_build(ntau, beta, 0)
    _, mf, Ff, Bf = G.gw_grid_build(ntau, beta, 1)
    wb, wf = 2 * mb * np.pi / beta, (2 * mf + 1) * np.pi / beta
    tau = beta * (np.arange(ntau) + 0.5) / ntau          # a symmetric uniform grid
    G.gw_set_grids(ctx, tau, Fb, Bb, Ff, Bf, wf, wb)
    gam = torch.empty((w.nk, nao, nao), dtype=torch.complex128, device="cuda")
    G.gw_density(ctx, dev(g), gam)
    ref = -interp.BarycentricInterpolator(tau, g, axis=1)(beta)
    assert rel(host(gam), ref) < 1e-11
    G.gw_set_grids(ctx, tau0, Fb, Bb, Ff, Bf, wf, wb)
    G.gw_density(ctx, dev(g), gam)
    assert rel(host(gam), O.density_matrix(g, beta)) < 1e-12
    ctx.destroy()


@pytest.mark.parametrize("nk3,nao,ntau,beta,target", [((2, 1, 1), 6, 40, 2.0, 5.0), ((1, 1, 1), 9, 30, 10.0, 8.0),
                                                      ((3, 1, 1), 4, 24, 5.0, 3.3)])
def test_find_mu(G, nk3, nao, ntau, beta, target):
    w = I.Workload("mu", nk3, nao, 3, ntau, ntau, beta, 0.0, 4.0, 9, solid=int(np.prod(nk3)) > 1)
    h, v, g = I.make_inputs(w)
    sig = hermitian_noise(g.shape, 0.02, 11)
    sinf = O.sigma_inf(v, O.density_matrix(g, beta), nk3, 2.0)
    mu_ref, G_ref = O.find_mu(h, sinf, sig, beta, target, 2.0, lo=-6.0, hi=6.0, tol=1e-12)
    ctx = G.gw_create(nk3, nao, 3, ntau, beta, precision="fp64")
    Gd = torch.empty(ctx.shapes()["G"], dtype=torch.complex128, device="cuda")
    mu = G.gw_find_mu(ctx, dev(h + sinf), dev(sig), target, -6.0, 6.0, 1e-12, Gd)
    assert abs(mu - mu_ref) < 1e-9
    assert rel(host(Gd), G_ref) < 1e-8
    assert abs(G.gw_particle_number(ctx, Gd) - target) < 1e-8
    with pytest.raises(G.GWError) as e:
        G.gw_find_mu(ctx, dev(h + sinf), dev(sig), 2.0 * nao + 1.0, -6.0, 6.0, 1e-12, Gd)
    assert e.value.code == G.GW_EINVAL
    ctx.destroy()


@pytest.mark.parametrize("n,max_vec,pushes", [(1, 1, 3), (1000, 4, 3), (4096, 3, 6), (123457, 8, 10)])
def test_diis_against_oracle(G, n, max_vec, pushes):
    """Coefficients and extrapolation over the newest max_vec pairs match the oracle's."""
    rng = np.random.default_rng(n)
    ins, outs = [], []
    d = G.gw_diis(n, max_vec)
    out = torch.empty(n, dtype=torch.complex128, device="cuda")
    for i in range(pushes):
        x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        f = x + (0.5 ** i) * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
        ins.append(x)
        outs.append(f)
        d.push(dev(x), dev(f))
        c = d.extrapolate(out)
        ref, c_ref = O.diis_extrapolate(outs[-max_vec:], ins[-max_vec:])
        assert len(c) == len(c_ref)
        assert np.abs(np.array(c) - c_ref).max() < 1e-9 * max(1.0, np.abs(c_ref).max())
        assert rel(host(out), ref) < 1e-10
    d.destroy()


def test_diis_linear_fixed_point(G):
    """On x = A x + b the extrapolation over all iterates reaches the fixed point after 2n + 1
    iterations (real coefficients on C^n); the same property pins the oracle."""
    rng = np.random.default_rng(0)
    n = 7
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A *= 0.4 / np.abs(np.linalg.eigvals(A)).max()
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    xstar = np.linalg.solve(np.eye(n) - A, b)
    d = G.gw_diis(n, 16)
    x = np.zeros(n, complex)
    out = torch.empty(n, dtype=torch.complex128, device="cuda")
    for it in range(2 * n + 1):
        f = A @ x + b
        d.push(dev(x), dev(f))
        c = d.extrapolate(out)
        assert abs(sum(c) - 1.0) < 1e-12
        x = host(out)
    assert np.abs(x - xstar).max() < 1e-9 * np.abs(xstar).max()
    d.destroy()


def test_diis_rejects_bad_arguments(G):
    with pytest.raises(G.GWError):
        G.gw_diis(0, 3)
    with pytest.raises(G.GWError):
        G.gw_diis(10, 17)
    d = G.gw_diis(10, 2)
    with pytest.raises(G.GWError) as e:
        d.extrapolate(torch.empty(10, dtype=torch.complex128, device="cuda"))
    assert e.value.code == G.GW_EINVAL
    x = torch.ones(10, dtype=torch.complex128, device="cuda")
    d.push(x, x)                                   # zero residual twice: singular subspace
    d.push(x, x)
    with pytest.raises(G.GWError) as e:
        d.extrapolate(torch.empty(10, dtype=torch.complex128, device="cuda"))
    assert e.value.code == G.GW_ENOTFINITE
    d.destroy()


def loop_case():
    w = I.Workload("loop", (2, 1, 1), 4, 8, 16, 16, 5.0, 0.0, 4.0, 21, solid=True)
    h, v, g = I.make_inputs(w)
    return w, h, 0.3 * v, g


LOOPS = [
    # static part, electrons per cell (None: fixed mu), DIIS size, DIIS start, residual
    (False, None, 0, 2, "diis"),
    (True, None, 0, 2, "diis"),
    (True, 3.0, 0, 2, "diis"),
    (True, 3.0, 5, 2, "diis"),
    (True, None, 3, 3, "diis"),
    (True, 3.0, 5, 2, "cdiis"),
    (False, None, 4, 3, "cdiis"),
]


@pytest.mark.parametrize("static,n_e,diis,start,kind", LOOPS)
def test_scgw_loop_matches_oracle(G, static, n_e, diis, start, kind):
    """gw_scgw against the oracle's loop: the same number of iterations (to one, at the stop
    threshold) and the same fixed point."""
    w, h, v, g = loop_case()
    ref = O.scgw_full(h, v, g, w.nk3, w.beta, 0.1, alpha=0.6, tol=1e-10, itermax=60, static=static,
                      n_electrons=n_e, mu_lo=-4.0, mu_hi=4.0, mu_tol=1e-12, diis_size=diis, diis_start=start,
                      diis_kind=kind)
    ctx = G.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, mu=0.1, precision="fp64")
    vd = dev(v)
    G.gw_set_coulomb(ctx, vd)
    Gd = dev(g)
    S = torch.empty(ctx.shapes()["Sig"], dtype=torch.complex128, device="cuda")
    Sinf = torch.empty((w.nk, w.nao, w.nao), dtype=torch.complex128, device="cuda")
    opt = G.scgw_options(alpha=0.6, tol=1e-10, itermax=60, static_part=static, diis_size=diis, diis_start=start,
                         n_electrons=n_e or 0.0, mu_lo=-4.0, mu_hi=4.0, mu_tol=1e-12, diis_kind=kind)
    rc, r = G.gw_scgw(ctx, dev(h), Gd, S, Sinf, opt)
    assert rc == G.GW_OK
    assert abs(r["iterations"] - ref["iterations"]) <= 1
    assert r["max_abs_dsigma"] < 1e-10
    assert abs(r["mu"] - ref["mu"]) < 1e-9
    for got, want in ((S, ref["Sig"]), (Sinf, ref["SigInf"]), (Gd, ref["G"])):
        assert np.abs(host(got) - want).max() < 1e-9
    if n_e:
        assert abs(r["n_electrons"] - n_e) < 1e-9
    ctx.destroy()


def test_scgw_loop_mixed_precision(G):
    """The mixed-precision loop reaches the FP64 fixed point to within its per-evaluation error."""
    w, h, v, g = loop_case()
    ref = O.scgw_full(h, v, g, w.nk3, w.beta, 0.0, alpha=0.6, tol=1e-9, itermax=60, n_electrons=3.0,
                      mu_lo=-4.0, mu_hi=4.0, mu_tol=1e-12, diis_size=5)
    ctx = G.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision="bf16x3")
    vd = dev(v)
    G.gw_set_coulomb(ctx, vd)
    Gd = dev(g)
    S = torch.empty(ctx.shapes()["Sig"], dtype=torch.complex128, device="cuda")
    opt = G.scgw_options(alpha=0.6, tol=1e-9, itermax=30, diis_size=5, n_electrons=3.0, mu_lo=-4.0, mu_hi=4.0,
                         mu_tol=1e-12)
    rc, r = G.gw_scgw(ctx, dev(h), Gd, S, None, opt)
    assert rc in (G.GW_OK, G.GW_ENOTCONV)
    # the fixed point in the mixed precision is the FP64 one to within the 1e-6 Ha target
    assert abs(r["mu"] - ref["mu"]) < 1e-6
    assert np.abs(host(S) - ref["Sig"]).max() < 1e-6
    assert np.abs(host(Gd) - ref["G"]).max() < 1e-6
    ctx.destroy()


def test_scgw_serving_job_with_the_full_loop(G):
    """A serving job with the static part, the mu search and CDIIS returns the oracle's loop."""
    w, h, v, g = loop_case()
    ref = O.scgw_full(h, v, g, w.nk3, w.beta, 0.0, alpha=0.6, tol=1e-10, itermax=60, n_electrons=3.0,
                      mu_lo=-4.0, mu_hi=4.0, mu_tol=1e-12, diis_size=4, diis_start=2, diis_kind="cdiis")
    cfg = G.make_config(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision="fp64")
    srv = G.gw_server(8 << 30, 2)
    S = np.empty(g.shape, complex)
    Gout = np.empty(g.shape, complex)
    jid = srv.submit(cfg, h, v, g, S, Gout, alpha=0.6, tol=1e-10, itermax=60, static_part=True, diis_size=4,
                     diis_start=2, n_electrons=3.0, mu_lo=-4.0, mu_hi=4.0, mu_tol=1e-12, diis_kind="cdiis")
    rc, res = srv.poll(jid, -1)
    assert rc == G.GW_OK and res["status"] == G.GW_OK
    assert abs(res["mu"] - ref["mu"]) < 1e-9
    assert np.abs(S - ref["Sig"]).max() < 1e-9
    assert np.abs(Gout - ref["G"]).max() < 1e-9
    srv.destroy()


def test_scgw_rejects_bad_options(G):
    w, h, v, g = loop_case()
    ctx = G.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision="fp64")
    G.gw_set_coulomb(ctx, dev(v))
    for bad in (dict(alpha=2.0), dict(itermax=0), dict(diis_size=17), dict(diis_size=2, diis_start=1),
                dict(n_electrons=3.0, mu_lo=1.0, mu_hi=0.0), dict(diis_size=2, diis_kind=2), dict(method=3)):
        with pytest.raises(G.GWError) as e:
            G.gw_scgw(ctx, dev(h), dev(g), None, None, G.scgw_options(**bad))
        assert e.value.code == G.GW_EINVAL
    ctx.destroy()


@pytest.mark.parametrize("static", [True, False])
def test_commutator_residual_against_oracle(G, static):
    w, h, v, g = loop_case()
    sig = hermitian_noise(g.shape, 0.05, 2)
    sinf = hermitian_noise((w.nk, w.nao, w.nao), 0.1, 3) if static else None
    ctx = G.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, mu=0.3, precision="fp64")
    e = torch.empty((w.nk, ctx.nwf, w.nao, w.nao), dtype=torch.complex128, device="cuda")
    G.gw_commutator_residual(ctx, dev(h), None if sinf is None else dev(sinf), dev(sig), dev(g), e)
    ref = O.commutator_residual(h, sinf, sig, g, w.beta)
    assert rel(host(e), ref) < 1e-12
    # a Dyson solution commutes with its own self-energy
    Gd = torch.empty(ctx.shapes()["G"], dtype=torch.complex128, device="cuda")
    heff = h if sinf is None else h + sinf
    G.gw_dyson_G(ctx, dev(heff), dev(sig), Gd)
    G.gw_commutator_residual(ctx, dev(h), None if sinf is None else dev(sinf), dev(sig), Gd, e)
    assert np.abs(host(e)).max() < 1e-12 * np.abs(ref).max() * 1e3
    ctx.destroy()


def test_diis_with_explicit_residuals(G):
    """Residuals of another length than the vectors (the commutator variant's case)."""
    rng = np.random.default_rng(7)
    n, nr, m = 500, 333, 4
    d = G.gw_diis(n, m, n_residual=nr)
    outs, res = [], []
    out = torch.empty(n, dtype=torch.complex128, device="cuda")
    for i in range(6):
        f = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        r = (0.5 ** i) * (rng.standard_normal(nr) + 1j * rng.standard_normal(nr))
        outs.append(f)
        res.append(r)
        d.push_residual(dev(f), dev(r))
        c = d.extrapolate(out)
        c_ref = O.diis_coefficients(res[-m:])
        assert np.abs(np.array(c) - c_ref).max() < 1e-9 * max(1.0, np.abs(c_ref).max())
        assert rel(host(out), sum(ci * o for ci, o in zip(c_ref, outs[-m:]))) < 1e-10
    with pytest.raises(G.GWError) as e:
        d.push(dev(outs[0]), dev(outs[1]))            # difference residuals need n_residual = 0
    assert e.value.code == G.GW_EINVAL
    d.destroy()


def test_hartree_fock_loop_matches_oracle(G):
    w, h, v, g = loop_case()
    ref = O.scgw_full(h, v, g, w.nk3, w.beta, 0.0, alpha=0.7, tol=1e-11, itermax=200, n_electrons=3.0,
                      mu_lo=-4.0, mu_hi=4.0, mu_tol=1e-13, diis_size=5, method="hf")
    ctx = G.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision="fp64")
    vd = dev(v)
    G.gw_set_coulomb(ctx, vd)
    Gd = dev(g)
    S = torch.empty(ctx.shapes()["Sig"], dtype=torch.complex128, device="cuda")
    Sinf = torch.empty((w.nk, w.nao, w.nao), dtype=torch.complex128, device="cuda")
    opt = G.scgw_options(alpha=0.7, tol=1e-11, itermax=200, diis_size=5, n_electrons=3.0, mu_lo=-4.0, mu_hi=4.0,
                         mu_tol=1e-13, method="hf")
    rc, r = G.gw_scgw(ctx, dev(h), Gd, S, Sinf, opt)
    assert rc == G.GW_OK
    assert abs(r["iterations"] - ref["iterations"]) <= 1
    assert abs(r["mu"] - ref["mu"]) < 1e-9
    assert not torch.any(S)
    assert np.abs(host(Sinf) - ref["SigInf"]).max() < 1e-9
    assert np.abs(host(Gd) - ref["G"]).max() < 1e-9
    ctx.destroy()


def overlap_case():
    w = I.Workload("s", (2, 1, 1), 4, 6, 16, 16, 5.0, 0.0, 4.0, 31, solid=True)
    h, v, g = I.make_inputs(w)
    S = I.overlap(w, np.random.default_rng(3))
    return w, h, v, g, S, hermitian_noise(g.shape, 0.05, 4)


def test_overlap_dyson_number_mu_commutator(G):
    w, h, v, g, S, sig = overlap_case()
    ctx = G.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, mu=0.2, precision="fp64")
    Sd = dev(S)
    G.gw_set_overlap(ctx, Sd)
    Gd = torch.empty(ctx.shapes()["G"], dtype=torch.complex128, device="cuda")
    G.gw_dyson_G(ctx, dev(h), dev(sig), Gd)
    ref = O.dyson_G(h, sig, 0.2, w.beta, S=S)
    assert rel(host(Gd), ref) < 1e-10
    n = G.gw_particle_number(ctx, Gd)
    assert abs(n - O.particle_number(O.density_matrix(ref, w.beta), 2.0, S)) < 1e-11
    mu = G.gw_find_mu(ctx, dev(h), dev(sig), 3.0, -4.0, 4.0, 1e-12, Gd)
    mu_ref, G_ref = O.find_mu(h, None, sig, w.beta, 3.0, 2.0, lo=-4.0, hi=4.0, tol=1e-12, S=S)
    assert abs(mu - mu_ref) < 1e-9 and rel(host(Gd), G_ref) < 1e-8
    sinf = hermitian_noise((w.nk, w.nao, w.nao), 0.1, 5)
    e = torch.empty((w.nk, ctx.nwf, w.nao, w.nao), dtype=torch.complex128, device="cuda")
    G.gw_commutator_residual(ctx, dev(h), dev(sinf), dev(sig), dev(g), e)
    assert rel(host(e), O.commutator_residual(h, sinf, sig, g, w.beta, S)) < 1e-12
    G.gw_set_overlap(ctx, None)                   # back to S = I
    G.gw_set_mu(ctx, 0.2)
    G.gw_dyson_G(ctx, dev(h), dev(sig), Gd)
    assert rel(host(Gd), O.dyson_G(h, sig, 0.2, w.beta)) < 1e-10
    ctx.destroy()


def test_overlap_loop_and_job(G):
    w, h, v, g, S, _ = overlap_case()
    v = 0.3 * v
    ref = O.scgw_full(h, v, g, w.nk3, w.beta, 0.0, alpha=0.6, tol=1e-10, itermax=80, n_electrons=3.0,
                      mu_lo=-4.0, mu_hi=4.0, mu_tol=1e-12, diis_size=5, diis_kind="cdiis", S=S)
    ctx = G.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision="fp64")
    vd = dev(v)
    G.gw_set_coulomb(ctx, vd)
    Sd = dev(S)
    G.gw_set_overlap(ctx, Sd)
    Gd = dev(g)
    Sig = torch.empty(ctx.shapes()["Sig"], dtype=torch.complex128, device="cuda")
    opt = G.scgw_options(alpha=0.6, tol=1e-10, itermax=80, diis_size=5, n_electrons=3.0, mu_lo=-4.0, mu_hi=4.0,
                         mu_tol=1e-12, diis_kind="cdiis")
    rc, r = G.gw_scgw(ctx, dev(h), Gd, Sig, None, opt)
    assert rc == G.GW_OK and abs(r["iterations"] - ref["iterations"]) <= 1
    assert abs(r["mu"] - ref["mu"]) < 1e-9 and np.abs(host(Gd) - ref["G"]).max() < 1e-9
    ctx.destroy()
    cfg = G.make_config(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision="fp64")
    srv = G.gw_server(8 << 30, 1)
    Gout = np.empty(g.shape, complex)
    jid = srv.submit(cfg, h, v, g, None, Gout, alpha=0.6, tol=1e-10, itermax=80, static_part=True, diis_size=5,
                     n_electrons=3.0, mu_lo=-4.0, mu_hi=4.0, mu_tol=1e-12, diis_kind="cdiis", S=S)
    rc, res = srv.poll(jid, -1)
    srv.destroy()
    assert rc == G.GW_OK and res["status"] == G.GW_OK
    assert np.abs(Gout - ref["G"]).max() < 1e-9


def test_scgw_resume_through_a_checkpoint(G, tmp_path):
    """6 iterations straight = 3, a checkpoint written and read back, 3 more resumed (bit for bit;
    mixing, static part, mu search), and both match the oracle's loop."""
    w, h, v, g = loop_case()
    kw = dict(alpha=0.6, tol=0.0, static_part=True, n_electrons=3.0, mu_lo=-4.0, mu_hi=4.0, mu_tol=1e-12)
    ref = O.scgw_full(h, v, g, w.nk3, w.beta, 0.0, alpha=0.6, tol=0.0, itermax=6, n_electrons=3.0, mu_lo=-4.0,
                      mu_hi=4.0, mu_tol=1e-12)
    ctx = G.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision="fp64")
    vd = dev(v)
    G.gw_set_coulomb(ctx, vd)
    shp = ctx.shapes()
    S1 = torch.empty(shp["Sig"], dtype=torch.complex128, device="cuda")
    I1 = torch.empty((w.nk, w.nao, w.nao), dtype=torch.complex128, device="cuda")
    G1 = dev(g)
    G.gw_scgw(ctx, dev(h), G1, S1, I1, G.scgw_options(itermax=6, **kw))
    G2, S2, I2 = dev(g), torch.empty_like(S1), torch.empty_like(I1)
    rc, r = G.gw_scgw(ctx, dev(h), G2, S2, I2, G.scgw_options(itermax=3, **kw))
    cfg = G.make_config(w.nk3, w.nao, w.naux, w.ntau, w.beta)
    G.gw_checkpoint_write(tmp_path / "ck", cfg, r["mu"], 3, {"G": host(G2), "Sigma": host(S2), "SigInf": host(I2)})
    _, mu, it, a = G.gw_checkpoint_read(tmp_path / "ck", {"G": shp["G"], "Sigma": shp["Sig"],
                                                          "SigInf": (w.nk, w.nao, w.nao)})
    G3, S3, I3 = dev(a["G"]), dev(a["Sigma"]), dev(a["SigInf"])
    G.gw_set_mu(ctx, mu)
    G.gw_scgw(ctx, dev(h), G3, S3, I3, G.scgw_options(itermax=3, resume=True, **kw))
    torch.cuda.synchronize()
    assert it == 3
    assert torch.equal(G3, G1) and torch.equal(S3, S1) and torch.equal(I3, I1)
    assert np.abs(host(G1) - ref["G"]).max() < 1e-9
    ctx.destroy()
