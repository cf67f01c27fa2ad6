"""Batched evaluation of independent systems (gw_batch_*): every mode (per-system loop,
concurrent streams, captured graph, grouped inversion eager and captured) gives, per system,
the oracle's self-energy and exactly what a lone gw_sigma_eval gives; graph replays and the
tuner keep that."""
import ctypes

import numpy as np
import pytest

from paper_2406_18479_gb300 import gw
from paper_2406_18479_gb300 import inputs as I


def test_batch_create_rejects_bad_arguments():
    cfg = gw.make_config((1, 1, 1), 4, 16, 8, 10.0)
    h = ctypes.c_void_p()
    arr = (gw.gw_config * 1)(cfg)
    assert gw.lib().gw_batch_create(ctypes.byref(h), arr, 0, 4, 0, None) == gw.GW_EINVAL
    assert gw.lib().gw_batch_create(ctypes.byref(h), arr, 1, 0, 0, None) == gw.GW_EINVAL
    assert gw.lib().gw_batch_create(ctypes.byref(h), arr, 1, 65, 0, None) == gw.GW_EINVAL


torch = pytest.importorskip("torch")

NAOS = [3, 7, 12, 5, 9]


@pytest.fixture(scope="module")
def systems():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import gw as O
    out = []
    for i, nao in enumerate(NAOS):
        w = I.molecule(f"m{i}", nao, ntau=8, beta=20.0, seed=40 + i)
        h, v, g = I.make_inputs(w)
        ref = O.sigma_eval(v, g, w.nk3, w.beta, spin_factor=2.0)["Sig"]
        out.append((w, v, g, ref))
    return out


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def alone(w, v, g, precision):
    ctx = gw.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision=precision)
    gw.gw_set_coulomb(ctx, torch.from_numpy(v).cuda())
    S = torch.empty(ctx.shapes()["Sig"], dtype=torch.complex128, device="cuda")
    gw.gw_sigma_eval(ctx, torch.from_numpy(g).cuda(), S)
    gw.gw_synchronize(ctx)
    out = S.cpu().numpy()
    ctx.destroy()
    return out


def out_buffers(systems, fill=0.0):
    return [torch.full((1, w.ntau, w.nao, w.nao), fill, dtype=torch.complex128, device="cuda")
            for w, *_ in systems]


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("bf16x3", 1e-7)])
def test_batch_modes_match_oracle_and_lone_runs(systems, precision, tol):
    cfgs = [gw.make_config(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision=precision) for w, *_ in systems]
    b = gw.gw_batch(cfgs, max_streams=3)
    b.set_coulomb([torch.from_numpy(v).cuda() for _, v, _, _ in systems])
    G = [torch.from_numpy(g).cuda() for _, _, g, _ in systems]
    results = {}
    S = out_buffers(systems, float("nan"))
    # the second call of each graph mode replays its capture
    for mode in ("serial", "streams", "graph", "graph", "grouped", "grouped_graph", "grouped_graph"):
        for s in S:
            s.fill_(float("nan"))
        b.sigma_eval(G, S, mode)
        b.synchronize()
        results.setdefault(mode, []).append([s.cpu().numpy() for s in S])
    b.destroy()
    lone = [alone(w, v, g, precision) for w, v, g, _ in systems]
    for i, (w, v, g, ref) in enumerate(systems):
        assert rel(lone[i], ref) < tol
        for mode, runs in results.items():
            for r in runs:
                assert np.array_equal(r[i], lone[i]), (mode, i)


@pytest.mark.gpu
def test_graph_recaptures_when_buffers_change(systems):
    cfgs = [gw.make_config(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision="bf16x3") for w, *_ in systems]
    b = gw.gw_batch(cfgs, max_streams=2)
    b.set_coulomb([torch.from_numpy(v).cuda() for _, v, _, _ in systems])
    G = [torch.from_numpy(g).cuda() for _, _, g, _ in systems]
    S1, S2 = out_buffers(systems), out_buffers(systems)
    b.sigma_eval(G, S1, "graph")
    b.sigma_eval(G, S1, "graph")
    b.sigma_eval(G, S2, "graph")          # new output pointers: a new capture
    b.synchronize()
    for s1, s2 in zip(S1, S2):
        assert torch.equal(s1, s2)
    b.destroy()


@pytest.mark.gpu
def test_autotune_keeps_results(systems):
    cfgs = [gw.make_config(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision="bf16x3") for w, *_ in systems]
    b = gw.gw_batch(cfgs, max_streams=3)
    b.set_coulomb([torch.from_numpy(v).cuda() for _, v, _, _ in systems])
    G = [torch.from_numpy(g).cuda() for _, _, g, _ in systems]
    S = out_buffers(systems)
    chosen = b.autotune(G, S)
    assert len(chosen) == len(systems)
    assert all(1 <= c <= w.ntau for c, (w, *_) in zip(chosen, systems))
    tuned = b.tuned()
    assert [t for t, _ in tuned] == chosen
    assert all(wd in (0, 56, 72, 80) for _, wd in tuned)
    b.sigma_eval(G, S, "graph")
    b.synchronize()
    for s, (w, v, g, ref) in zip(S, systems):
        assert rel(s.cpu().numpy(), ref) < 1e-7
    b.destroy()


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "bf16x4"])
def test_grouped_inversion_spans_both_panel_widths(precision):
    """A batch whose aux bases straddle 430 (the widest matrix of the 16-column panel) and one
    above 800 (the widest of the 8-column panel): the grouped modes invert both panel classes in
    their own launches, leave the largest system's inversion to its own evaluation, and still
    give, bit for bit, what lone evaluations give."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ws = [I.molecule("small", 6, ntau=8, beta=20.0, seed=70),
          I.molecule("naux440", 110, ntau=8, beta=20.0, seed=71),
          I.molecule("naux432", 108, ntau=8, beta=20.0, seed=72),
          I.molecule("naux428", 107, ntau=8, beta=20.0, seed=73),
          I.molecule("naux804", 201, ntau=4, beta=20.0, seed=74)]   # above 800: inverted on its own
    data = [I.make_inputs(w)[1:] for w in ws]
    cfgs = [gw.make_config(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision=precision) for w in ws]
    b = gw.gw_batch(cfgs, max_streams=3)
    b.set_coulomb([torch.from_numpy(v).cuda() for v, _ in data])
    G = [torch.from_numpy(g).cuda() for _, g in data]
    lone = [alone(w, v, g, precision) for w, (v, g) in zip(ws, data)]
    for mode in ("grouped", "grouped_graph", "grouped_graph"):
        S = out_buffers([(w,) for w in ws], float("nan"))
        b.sigma_eval(G, S, mode)
        b.synchronize()
        for i, s in enumerate(S):
            assert np.array_equal(s.cpu().numpy(), lone[i]), (mode, ws[i].name)
    b.destroy()


@pytest.mark.gpu
@pytest.mark.parametrize("tile_n", [56, 72, 80])
def test_tile_width_keeps_results(systems, tile_n):
    """Every tile width of the free-width GEMMs gives the oracle's self-energy, and bit for bit
    what the automatic width gives (a tile's width does not change how any one output element
    is summed); the tuner's candidates are exactly these contexts."""
    for w, v, g, ref in systems:
        out = []
        for width in (0, tile_n):
            ctx = gw.gw_create(w.nk3, w.nao, w.naux, w.ntau, w.beta, precision="bf16x4", tile_n=width)
            gw.gw_set_coulomb(ctx, torch.from_numpy(v).cuda())
            S = torch.empty(ctx.shapes()["Sig"], dtype=torch.complex128, device="cuda")
            gw.gw_sigma_eval(ctx, torch.from_numpy(g).cuda(), S)
            gw.gw_synchronize(ctx)
            out.append(S.cpu().numpy())
            ctx.destroy()
        assert rel(out[1], ref) < 1e-7, (w.name, tile_n)
        assert np.array_equal(out[0], out[1]), (w.name, tile_n)
