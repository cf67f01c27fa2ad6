"""Pins of the IR grid construction (oracle/ir.py), against closed forms: the Matsubara transform
of e^{-e tau} (fermionic and bosonic propagators of one level) must come out to the truncation
accuracy eps for every level inside [-omega_max, omega_max]; the singular functions are
orthonormal with parity (-1)^l; the sampling sets have the library's sizes and mirror symmetry."""
import numpy as np
import pytest

from oracle import ir


def g0(e, tau, beta, stat):
    """-e^{-e tau} / (1 + e^{-beta e}) (fermions) or / (1 - e^{-beta e}) (bosons), whose Matsubara
    transform int_0^beta e^{i nu tau} g dtau is 1 / (i nu - e)."""
    if stat == 1:
        return -np.exp(-e * tau - np.logaddexp(0.0, -beta * e))
    if e > 0:
        return -np.exp(-e * tau) / (-np.expm1(-beta * e))
    return np.exp(e * (beta - tau)) / (-np.expm1(beta * e))


@pytest.mark.parametrize("lam,eps,beta", [(100.0, 1e-10, 10.0), (1000.0, 1e-8, 50.0)])
@pytest.mark.parametrize("stat", [0, 1])
def test_propagators_transform_to_the_closed_form(lam, eps, beta, stat):
    tau, m, F, B = ir.ir_grid(beta, lam, eps, stat)
    nu = ((2 * m + 1) if stat == 1 else 2 * m) * np.pi / beta
    wmax = lam / beta
    for e in (-0.95 * wmax, -0.3 * wmax, -1.0, 0.37, 2.5, 0.8 * wmax):
        ref = 1.0 / (1j * nu - e)
        got = F @ g0(e, tau, beta, stat)
        assert np.abs(got - ref).max() < 20 * eps * np.abs(ref).max()
        # and back: B recovers the node values
        assert np.abs(B @ ref - g0(e, tau, beta, stat)).max() < 1e3 * eps * np.abs(g0(e, tau, beta, stat)).max()


def test_basis_is_orthonormal_with_parity():
    b = ir.Basis(300.0, 1e-10)
    _, wx = ir._gauss(b.edges)
    G = (b.U * wx[:, None]).T @ b.U
    assert np.abs(G - np.eye(b.L + 1)).max() < 1e-9
    x = np.linspace(-0.99, 0.99, 13)
    for l in (0, 1, 5, b.L):
        assert np.abs(b.eval(l, -x) - (-1) ** l * b.eval(l, x)).max() < 1e-10 * np.abs(b.eval(l, x)).max()
    assert np.all(np.diff(b.s) <= 0)
    assert ir.Basis(30.0, 1e-10).L < b.L < ir.Basis(3000.0, 1e-10).L


@pytest.mark.parametrize("stat", [0, 1])
def test_sampling_sets(stat):
    beta = 20.0
    tau, m, F, B = ir.ir_grid(beta, 200.0, 1e-9, stat)
    assert np.all(np.diff(tau) > 0) and tau[0] > 0 and tau[-1] < beta
    assert np.abs(tau + tau[::-1] - beta).max() < 1e-12
    assert len(m) == ir.sample_count(len(tau), stat)
    mirror = (-m - 1) if stat == 1 else -m
    assert sorted(mirror.tolist()) == m.tolist()
    if stat == 0:   # the library's requirement on bosonic transforms: F[nb-1-n][T-1-t] = F[n][t]
        assert np.abs(F[::-1, ::-1] - F).max() < 1e-10 * np.abs(F).max()
