"""Checkpoint files (host code, no GPU): round trip, selection by name, and rejection of files
that do not match or are cut short."""
import numpy as np
import pytest

from paper_2406_18479_gb300 import gw


@pytest.fixture(scope="module")
def lib():
    try:
        gw.lib()
    except RuntimeError as e:
        pytest.skip(str(e))
    return gw


def arrays():
    rng = np.random.default_rng(0)
    G = rng.standard_normal((2, 6, 3, 3)) + 1j * rng.standard_normal((2, 6, 3, 3))
    S = rng.standard_normal((2, 6, 3, 3)) + 1j * rng.standard_normal((2, 6, 3, 3))
    I = rng.standard_normal((2, 3, 3)) + 1j * rng.standard_normal((2, 3, 3))
    return G, S, I


def test_round_trip(lib, tmp_path):
    G, S, I = arrays()
    cfg = gw.make_config((2, 1, 1), 3, 5, 6, 8.5, spin_factor=2.0, precision="bf16x3")
    p = tmp_path / "loop.ckpt"
    gw.gw_checkpoint_write(p, cfg, -0.125, 7, {"G": G, "Sigma": S, "SigInf": I})
    c2, mu, it, out = gw.gw_checkpoint_read(p, {"SigInf": I.shape, "G": G.shape})   # any subset, any order
    assert mu == -0.125 and it == 7
    assert tuple(c2.nk) == (2, 1, 1) and (c2.nao, c2.naux, c2.ntau) == (3, 5, 6) and c2.beta == 8.5
    assert np.array_equal(out["G"], G) and np.array_equal(out["SigInf"], I)


def test_rejects_mismatch_and_damage(lib, tmp_path):
    G, S, I = arrays()
    cfg = gw.make_config((2, 1, 1), 3, 5, 6, 8.5)
    p = tmp_path / "loop.ckpt"
    gw.gw_checkpoint_write(p, cfg, 0.0, 1, {"G": G, "Sigma": S})
    for shapes in ({"G": (2, 6, 3, 4)}, {"W": (1,)}):
        with pytest.raises(gw.GWError) as e:
            gw.gw_checkpoint_read(p, shapes)
        assert e.value.code == gw.GW_EINVAL
    data = p.read_bytes()
    (tmp_path / "cut.ckpt").write_bytes(data[:-16])
    with pytest.raises(gw.GWError):
        gw.gw_checkpoint_read(tmp_path / "cut.ckpt", {"G": G.shape, "Sigma": S.shape})
    (tmp_path / "junk.ckpt").write_bytes(b"not a checkpoint\n" + data)
    with pytest.raises(gw.GWError):
        gw.gw_checkpoint_read(tmp_path / "junk.ckpt", {"G": G.shape})
    with pytest.raises(gw.GWError):
        gw.gw_checkpoint_write(p, cfg, 0.0, 1, {"bad name": G})
