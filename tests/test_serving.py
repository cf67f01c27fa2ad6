"""Request loop (gw_submit / gw_poll): admission, results, and errors.

A job is the self-consistency loop of Sec. 2.4 at fixed mu (Sigma from G, mixing
of Sec. 5.3, Dyson update of Eq. dyson). The CPU tests cover argument checks and
the admission rule that needs no device; the GPU tests compare a job with the
oracle's loop and concurrent jobs with the same jobs run one at a time.
"""
import numpy as np
import pytest

from paper_2406_18479_gb300 import gw
from paper_2406_18479_gb300 import inputs as I


def small_case(nk3=(2, 1, 1), nao=4, naux=10, ntau=6, beta=8.0, seed=3):
    w = I.Workload("serve", nk3, nao, naux, ntau, ntau, beta, 0.0, 4.0, seed, solid=int(np.prod(nk3)) > 1)
    return w, I.make_inputs(w)


def test_job_bytes_counts_and_rejects():
    c = gw.make_config((2, 1, 1), 4, 10, 6, 8.0)
    b = gw.gw_job_bytes(c)
    nk, nao2 = 2, 16
    buffers = 16 * (nk * nk * 10 * nao2 + nk * nao2 + 3 * nk * 6 * nao2)
    assert b > buffers
    bigger = gw.gw_job_bytes(gw.make_config((2, 1, 1), 4, 20, 6, 8.0))
    assert bigger > b
    assert gw.gw_job_bytes(gw.make_config((0, 1, 1), 4, 10, 6, 8.0)) == 0
    assert gw.gw_job_bytes(gw.make_config((1, 1, 1), 4, 10, 6, -1.0)) == 0
    assert gw.gw_job_bytes(gw.make_config((1, 1, 1), 4, 10, 6, 8.0, precision=7)) == 0
    # the mixed path holds its slice planes in addition
    assert gw.gw_job_bytes(gw.make_config((2, 1, 1), 4, 10, 6, 8.0, precision="bf16x3")) > 0


def test_server_arguments():
    with pytest.raises(gw.GWError) as e:
        gw.gw_server(0, 2)
    assert e.value.code == gw.GW_EINVAL
    with pytest.raises(gw.GWError) as e:
        gw.gw_server(1 << 30, 0)
    assert e.value.code == gw.GW_EINVAL
    with pytest.raises(gw.GWError) as e:
        gw.gw_server(1 << 30, 65)
    assert e.value.code == gw.GW_EINVAL


def test_submit_rejects_without_running():
    w, (h, v, g) = small_case()
    cfg = gw.make_config(w.nk3, w.nao, w.naux, w.ntau, w.beta)
    srv = gw.gw_server(gw.gw_job_bytes(cfg) - 1, 2)
    try:
        with pytest.raises(gw.GWError) as e:
            srv.submit(cfg, h, v, g)
        assert e.value.code == gw.GW_ENOMEM
        with pytest.raises(gw.GWError) as e:
            srv.submit(cfg, h, v, g, itermax=0)
        assert e.value.code == gw.GW_EINVAL
        with pytest.raises(gw.GWError) as e:
            srv.submit(cfg, h, v.astype(np.complex64), g)
        assert e.value.code == gw.GW_EINVAL
        with pytest.raises(gw.GWError) as e:
            srv.submit(cfg, h[:, :2], v, g)
        assert e.value.code == gw.GW_EINVAL
        with pytest.raises(gw.GWError) as e:
            srv.poll(12345, 0)
        assert e.value.code == gw.GW_EINVAL
    finally:
        srv.destroy()


# ---- GPU -------------------------------------------------------------------------------------

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gw.lib()
    return True


def run_alone(cfg, h, v, g, **kw):
    srv = gw.gw_server(1 << 36, 1)
    sig, gout = np.zeros_like(g), np.zeros_like(g)
    try:
        jid = srv.submit(cfg, h, v, g, sig, gout, **kw)
        rc, res = srv.poll(jid, -1)
        assert rc == gw.GW_OK
    finally:
        srv.destroy()
    return res, sig, gout


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "bf16x3"])
def test_job_bytes_equal_context_workspace(cuda, precision):
    w, _ = small_case(nk3=(2, 2, 1), nao=5, naux=13, ntau=7)
    cfg = gw.make_config(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision=precision)
    ctx = gw.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision=precision)
    nk, nao2 = 4, 25
    # V, H, an overlap, G, the Sigma output; the loop's Sigma_{n-1} and F_n (static + dynamic),
    # H + Sigma^inf, flags
    nall = nk * nao2 * (1 + w.ntau)
    buffers = 16 * (nk * nk * w.naux * nao2 + 2 * nk * nao2 + 2 * nk * w.ntau * nao2) + 16 * (2 * nall + nk * nao2) + 256
    assert gw.gw_job_bytes(cfg) == ctx.workspace_bytes() + buffers
    assert gw.gw_scgw_bytes(cfg, gw.scgw_options()) == 16 * (2 * nall + nk * nao2) + 256
    five = gw.gw_scgw_bytes(cfg, gw.scgw_options(diis_size=5))
    assert five == 16 * (2 * nall + nk * nao2) + 256 + 16 * 2 * 5 * nall + 8 * 513
    ctx.destroy()


@pytest.mark.gpu
def test_job_matches_oracle_loop(cuda):
    from oracle import gw as O
    w, (h, v, g) = small_case()
    cfg = gw.make_config(w.nk3, w.nao, w.naux, w.ntau, w.beta, mu=w.mu)
    res, sig, gout = run_alone(cfg, h, v, g, alpha=0.6, tol=1e-9, itermax=4)
    ref_sig, ref_g, hist = O.scgw(h, v, g, w.nk3, w.beta, w.mu, alpha=0.6, tol=1e-9, itermax=4)
    assert res["iterations"] == 4 and res["status"] == gw.GW_ENOTCONV
    assert abs(res["max_abs_dsigma"] - hist[-1]) <= 1e-10 * max(1.0, hist[-1])
    scale = np.max(np.abs(ref_sig))
    assert np.max(np.abs(sig - ref_sig)) <= 1e-10 * scale
    assert np.max(np.abs(gout - ref_g)) <= 1e-10 * np.max(np.abs(ref_g))


@pytest.mark.gpu
def test_converged_job_reports_ok(cuda):
    w, (h, v, g) = small_case(nk3=(1, 1, 1), nao=3, naux=8, ntau=5)
    cfg = gw.make_config(w.nk3, w.nao, w.naux, w.ntau, w.beta, mu=w.mu)
    res, _, _ = run_alone(cfg, h, v, g, alpha=1.0, tol=1.0, itermax=10)
    assert res["status"] == gw.GW_OK
    assert res["iterations"] == 2 and res["max_abs_dsigma"] < 1.0
    assert res["t_submit"] <= res["t_start"] <= res["t_end"]


@pytest.mark.gpu
def test_concurrent_jobs_equal_solo_runs(cuda):
    specs = [((2, 1, 1), 4, 10, 6, "fp64"), ((1, 1, 1), 8, 32, 8, "bf16x3"), ((2, 2, 1), 5, 13, 7, "bf16x3"),
             ((1, 1, 1), 6, 20, 5, "fp64"), ((3, 1, 1), 3, 9, 6, "bf16x3"), ((1, 1, 1), 8, 32, 8, "fp64")]
    jobs = []
    for i, (nk3, nao, naux, ntau, prec) in enumerate(specs):
        w, (h, v, g) = small_case(nk3, nao, naux, ntau, 8.0 + i, seed=10 + i)
        jobs.append((gw.make_config(nk3, nao, naux, ntau, w.beta, precision=prec), h, v, g))
    solo = [run_alone(cfg, h, v, g, alpha=0.7, tol=0.0, itermax=3) for cfg, h, v, g in jobs]
    srv = gw.gw_server(1 << 36, 3)
    outs = []
    try:
        ids = []
        for cfg, h, v, g in jobs:
            sig, gout = np.zeros_like(g), np.zeros_like(g)
            outs.append((sig, gout))
            ids.append(srv.submit(cfg, h, v, g, sig, gout, alpha=0.7, tol=0.0, itermax=3))
        results = [srv.poll(j, -1) for j in ids]
    finally:
        srv.destroy()
    for (rc, res), (sres, ssig, sg), (sig, gout) in zip(results, solo, outs):
        assert rc == gw.GW_OK and res["status"] == gw.GW_ENOTCONV and res["iterations"] == 3
        assert np.array_equal(sig, ssig) and np.array_equal(gout, sg)
        assert res["max_abs_dsigma"] == sres["max_abs_dsigma"]


@pytest.mark.gpu
def test_admission_respects_budget(cuda):
    w, (h, v, g) = small_case()
    cfg = gw.make_config(w.nk3, w.nao, w.naux, w.ntau, w.beta)
    b = gw.gw_job_bytes(cfg)
    srv = gw.gw_server(b + b // 2, 4)   # room for one job at a time
    try:
        ids = [srv.submit(cfg, h, v, g, alpha=0.7, tol=0.0, itermax=2) for _ in range(3)]
        res = [srv.poll(j, -1)[1] for j in ids]
    finally:
        srv.destroy()
    spans = sorted((r["t_start"], r["t_end"]) for r in res)
    for (s0, e0), (s1, e1) in zip(spans, spans[1:]):
        assert s1 >= e0
    # arrival order is kept when every job fits the same budget
    assert [r["t_start"] for r in res] == sorted(r["t_start"] for r in res)


@pytest.mark.gpu
def test_poll_without_waiting(cuda):
    w, (h, v, g) = small_case()
    cfg = gw.make_config(w.nk3, w.nao, w.naux, w.ntau, w.beta)
    srv = gw.gw_server(1 << 36, 1)
    try:
        j1 = srv.submit(cfg, h, v, g, tol=0.0, itermax=6)
        j2 = srv.submit(cfg, h, v, g, tol=0.0, itermax=6)
        rc, _ = srv.poll(j2, 0)
        assert rc in (gw.GW_EAGAIN, gw.GW_OK)
        rc, _ = srv.poll(j2, 1)
        assert rc in (gw.GW_ETIMEOUT, gw.GW_OK)
        assert srv.poll(j1, -1)[0] == gw.GW_OK
        assert srv.poll(j2, -1)[0] == gw.GW_OK
    finally:
        srv.destroy()
