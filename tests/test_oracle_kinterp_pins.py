"""Pins of the k-space interpolation (Sec. 2.5): exact on the mesh; exact for quantities whose
real-space range fits the R set, including a one-sided (complex) hopping that fixes the signs
of both transforms; the nearest-neighbour Hamiltonian of the input generator at arbitrary k."""
import numpy as np
import pytest

from oracle import kinterp as K
from paper_2406_18479_gb300 import inputs as I


@pytest.mark.parametrize("nk3", [(1, 1, 1), (2, 1, 1), (3, 2, 1), (4, 3, 2)])
def test_exact_on_the_mesh(nk3):
    rng = np.random.default_rng(1)
    nk = int(np.prod(nk3))
    X = rng.standard_normal((nk, 3, 2, 2)) + 1j * rng.standard_normal((nk, 3, 2, 2))
    Y = K.k_interpolate(X, nk3, K.mesh_fractions(nk3))
    assert np.abs(Y - X).max() < 1e-13


@pytest.mark.parametrize("nk3", [(3, 1, 1), (3, 3, 1), (5, 4, 3)])
def test_one_sided_hopping_is_reproduced(nk3):
    """X(k) = A + B e^{i k.a1} + C e^{-i k.a2} (complex, not symmetric in R) is exact at any k when
    the mesh holds R = +-1 in those directions without boundary sharing (N >= 3)."""
    rng = np.random.default_rng(2)
    A, B, C = (rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2)) for _ in range(3))

    def X(f):
        f = np.atleast_2d(f)
        e1 = np.exp(2j * np.pi * f[:, 0])[:, None, None]
        e2 = np.exp(-2j * np.pi * f[:, 1])[:, None, None] if nk3[1] >= 3 else 1.0
        return A + B * e1 + (C * e2 if nk3[1] >= 3 else 0)
    fm = K.mesh_fractions(nk3)
    fnew = rng.uniform(-1, 1, (7, 3))
    assert np.abs(K.k_interpolate(X(fm), nk3, fnew) - X(fnew)).max() < 1e-13


@pytest.mark.parametrize("nk3", [(2, 2, 2), (3, 3, 3), (4, 2, 3)])
def test_nearest_neighbour_hamiltonian(nk3):
    """The generator's H(k) = H0 + sum_d 2 cos(k_d) T_d interpolates exactly (for N_d = 2 through
    the shared boundary terms)."""
    w = I.Workload("k", nk3, 4, 4, 2, 2, 1.0, 0.0, 4.0, 3, solid=True)
    rng = np.random.default_rng(w.seed)
    h = I.hamiltonian(w, rng)
    # rebuild H0 and T_d from the mesh values: H(k) is linear in (1, 2 cos k_x, 2 cos k_y, 2 cos k_z)
    fm = K.mesh_fractions(nk3)
    basis = np.concatenate([np.ones((len(fm), 1)), 2 * np.cos(2 * np.pi * fm)], axis=1)
    coef, *_ = np.linalg.lstsq(basis, h.reshape(len(fm), -1), rcond=None)
    fnew = np.random.default_rng(5).uniform(0, 1, (6, 3))
    want = (np.concatenate([np.ones((6, 1)), 2 * np.cos(2 * np.pi * fnew)], axis=1) @ coef).reshape(6, 4, 4)
    assert np.abs(K.k_interpolate(h, nk3, fnew) - want).max() < 1e-12


def test_weights_sum_to_the_mesh_size():
    for nk3 in [(2, 3, 4), (1, 1, 6), (5, 5, 1)]:
        assert abs(sum(w for _, w in K.lattice_vectors(nk3)) - np.prod(nk3)) < 1e-14
