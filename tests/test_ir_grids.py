"""The library's IR grid builder (gw_ir_grids, host code: no GPU needed) against closed forms and
the oracle's construction (oracle/ir.py)."""
import numpy as np
import pytest

from oracle import ir
from paper_2406_18479_gb300 import gw


def g0(e, tau, beta, stat):
    if stat == 1:
        return -np.exp(-e * tau - np.logaddexp(0.0, -beta * e))
    if e > 0:
        return -np.exp(-e * tau) / (-np.expm1(-beta * e))
    return np.exp(e * (beta - tau)) / (-np.expm1(beta * e))


@pytest.fixture(scope="module")
def lib():
    try:
        gw.lib()
    except RuntimeError as e:
        pytest.skip(str(e))
    return gw


@pytest.mark.parametrize("lam,eps,beta", [(100.0, 1e-10, 10.0), (1000.0, 1e-8, 50.0), (1e4, 1e-10, 100.0)])
def test_closed_form_transforms(lib, lam, eps, beta):
    tau, Fb, Bb, Ff, Bf, wf, wb = lib.gw_ir_grids(beta, lam, eps)
    T = len(tau)
    assert Fb.shape == (gw.gw_sample_count(T, 0), T) and Ff.shape == (gw.gw_sample_count(T, 1), T)
    assert np.abs(tau + tau[::-1] - beta).max() < 1e-12 * beta and np.all(np.diff(tau) > 0)
    for stat, F, B, w in ((0, Fb, Bb, wb), (1, Ff, Bf, wf)):
        assert np.abs(B @ F - np.eye(T)).max() < 1e-10
        assert np.abs(w + w[::-1]).max() < 1e-12 * np.abs(w).max()
        for e in (-0.9 * lam / beta, -1.0, 0.37, 2.0, 0.7 * lam / beta):
            ref = 1.0 / (1j * w - e)
            assert np.abs(F @ g0(e, tau, beta, stat) - ref).max() < 20 * eps * np.abs(ref).max()
    # what gw_set_grids requires of the bosonic transforms
    assert np.abs(Fb[::-1, ::-1] - Fb).max() < 1e-10 * np.abs(Fb).max()
    assert np.abs(Bb[::-1, ::-1] - Bb).max() < 1e-10 * np.abs(Bb).max()


@pytest.mark.parametrize("lam,eps,beta", [(100.0, 1e-10, 10.0), (1000.0, 1e-8, 50.0)])
def test_agrees_with_the_oracle(lib, lam, eps, beta):
    """Same basis size, nodes and samples; transforms equal to the SVD's accuracy at the cut-off
    (double-precision singular vectors near s_L carry about 1e-16 s_0 / gap)."""
    tau, Fb, Bb, Ff, Bf, wf, wb = lib.gw_ir_grids(beta, lam, eps)
    for stat, F, w in ((0, Fb, wb), (1, Ff, wf)):
        to, mo, Fo, Bo = ir.ir_grid(beta, lam, eps, stat)
        assert len(to) == len(tau)
        assert np.abs(tau - to).max() < 1e-5 * beta
        nu = ((2 * mo + 1) if stat == 1 else 2 * mo) * np.pi / beta
        assert np.abs(w - nu).max() < 1e-12 * np.abs(nu).max()
        assert np.abs(F - Fo).max() < 1e-4 * np.abs(Fo).max()


def test_bad_arguments(lib):
    for args in ((-1.0, 100.0, 1e-10), (10.0, 0.5, 1e-10), (10.0, 100.0, 1e-20)):
        with pytest.raises(gw.GWError):
            lib.gw_ir_grids(*args)


@pytest.mark.parametrize("lam,eps", [(1.0, 1e-10), (10.0, 1e-6), (1000.0, 1e-12), (300.0, 1e-4)])
def test_sweep_of_lambda_and_eps(lib, lam, eps):
    """Propagators with poles inside [-omega_max, omega_max] transform to within 20 eps."""
    beta = 50.0
    tau, Fb, Bb, Ff, Bf, wf, wb = lib.gw_ir_grids(beta, lam, eps)
    for stat, F, w in ((0, Fb, wb), (1, Ff, wf)):
        for e in (-0.9 * lam / beta, 0.37 * lam / beta, 0.7 * lam / beta):
            ref = 1.0 / (1j * w - e)
            assert np.abs(F @ g0(e, tau, beta, stat) - ref).max() < 20 * eps * np.abs(ref).max()
