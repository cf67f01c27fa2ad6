"""Error paths and size queries of the C ABI that run on the host before any device work, so they
are checked without a GPU: bad arguments give GW_EINVAL with a message, and the
device-byte queries of contexts, jobs and loops add up."""
import ctypes

import numpy as np
import pytest

from paper_2406_18479_gb300 import gw


@pytest.fixture(scope="module")
def L():
    try:
        return gw.lib()
    except RuntimeError as e:
        pytest.skip(str(e))


def test_null_and_out_of_range_arguments(L):
    vp = ctypes.c_void_p
    assert L.gw_scgw(None, None, None, None, None, None, None) == gw.GW_EINVAL
    assert L.gw_sigma_inf(None, None, None) == gw.GW_EINVAL
    assert L.gw_find_mu(None, None, None, 1.0, 0.0, 1.0, 1e-9, None, None) == gw.GW_EINVAL
    assert L.gw_commutator_residual(None, None, None, None, None, None) == gw.GW_EINVAL
    assert L.gw_gf2_self_energy(None, None, None) == gw.GW_EINVAL
    assert L.gw_set_overlap(None, None) == gw.GW_EINVAL
    h = vp()
    assert L.gw_diis_create(ctypes.byref(h), 0, 0, 3, None) == gw.GW_EINVAL
    assert L.gw_diis_create(ctypes.byref(h), 10, 0, 17, None) == gw.GW_EINVAL
    assert L.gw_diis_push(None, None, None) == gw.GW_EINVAL
    assert L.gw_k_interpolate((ctypes.c_int * 3)(0, 1, 1), None, 1, 1, None, None, None) == gw.GW_EINVAL
    code = ctypes.c_int()
    assert L.gw_selftest_bounded_wait(100.0, ctypes.byref(code), None) == gw.GW_EINVAL
    assert L.gw_check_guards(None) == gw.GW_EINVAL
    assert L.gw_debug_mark_guard(None, 0) == gw.GW_EINVAL
    assert b"gw_" in L.gw_last_error()


@pytest.mark.parametrize("field,value", [("nao", 0), ("naux", 5000), ("ntau", 0), ("beta", -1.0), ("precision", 7),
                                         ("precision", 2), ("v_slices", 3), ("v_packed", 2), ("slice_pass", 2),
                                         ("tile_n", 64), ("tile_n", -1)])
def test_bad_configurations(L, field, value):
    cfg = gw.make_config((2, 1, 1), 3, 4, 5, 2.0)
    setattr(cfg, field, value)
    h = ctypes.c_void_p()
    assert L.gw_create(ctypes.byref(h), ctypes.byref(cfg), None) == gw.GW_EINVAL
    assert gw.gw_job_bytes(cfg) == 0


def test_precision_names():
    """The four-slice scheme under its name and its former one; no FP16 precision exists."""
    assert gw.PRECISIONS["bf16x4"] == gw.PRECISIONS["bf16x3"] == gw.GW_MIXED_BF16X4 == 1
    assert "fp16s" not in gw.PRECISIONS


def test_loop_bytes(L):
    cfg = gw.make_config((2, 2, 1), 5, 13, 7, 2.0)
    nk, nao2, T = 4, 25, 7
    nall = nk * nao2 * (1 + T)
    base = 16 * (2 * nall + nk * nao2) + 256
    assert gw.gw_scgw_bytes(cfg, gw.scgw_options()) == base
    assert gw.gw_scgw_bytes(cfg, gw.scgw_options(diis_size=3)) == base + 16 * 3 * 2 * nall + 8 * 513
    nres = nk * gw.gw_sample_count(T, 1) * nao2      # the commutator's residuals live on the samples
    assert gw.gw_scgw_bytes(cfg, gw.scgw_options(diis_size=3, diis_kind="cdiis")) == \
        base + 16 * (3 * (nall + nres) + nres) + 8 * 513


def test_packed_v_halves_the_job(L):
    """A job's V drops from nk^2 to nk (nk + 1) / 2 blocks; the per-q staging scratch adds nk blocks
    (and its 256-byte guard)."""
    for nk3 in [(2, 2, 1), (3, 3, 1)]:
        cf = gw.make_config(nk3, 4, 8, 6, 2.0, precision="bf16x3", v_slices=2)
        cp = gw.make_config(nk3, 4, 8, 6, 2.0, precision="bf16x3", v_slices=2, v_packed=True)
        nk = int(np.prod(nk3))
        vb = 16 * 8 * 16
        assert gw.gw_job_bytes(cf) - gw.gw_job_bytes(cp) == vb * (nk * nk - nk * (nk + 1) // 2 - nk) - 256
        f64 = gw.make_config(nk3, 4, 8, 6, 2.0)
        p64 = gw.make_config(nk3, 4, 8, 6, 2.0, v_packed=True)
        # FP64 keeps a full working copy: the job's input shrinks to nk (nk + 1) / 2 blocks and the
        # context gains nk^2 (and a guard), nk (nk + 1) / 2 blocks more in all
        assert gw.gw_job_bytes(p64) - gw.gw_job_bytes(f64) == vb * (nk * (nk + 1) // 2) + 256
