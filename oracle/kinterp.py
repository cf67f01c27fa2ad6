"""k-space interpolation of momentum-dependent quantities (Sec. 2.5, the Wannier-like
interpolation without the maximally localised basis), in plain complex128 (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

  X(R) = (1/N_k) sum_k X(k) e^{-i k R},      X(k') = sum_R w_R X(R) e^{i k' R},

k = 2 pi (n1/N1, n2/N2, n3/N3) on the Gamma-centred mesh, k' anywhere (given in the same
fractional coordinates, k' = 2 pi f). Reading (the paper does not fix the R set): R runs over
the lattice vectors nearest the origin, R_d in [-N_d/2, N_d/2]; for even N_d the two boundary
vectors +-N_d/2 share one term with weight 1/2 each (per direction, weights multiply), so
that interpolation is exact on the mesh and keeps X(-k) = X(k)^dagger symmetric.
"""
from __future__ import annotations

import itertools

import numpy as np


def lattice_vectors(nk3):
    """[(R, w_R)] in the reading above."""
    axes = []
    for n in nk3:
        if n % 2 == 1:
            axes.append([(r, 1.0) for r in range(-(n // 2), n // 2 + 1)])
        else:
            axes.append([(r, 1.0) for r in range(-(n // 2) + 1, n // 2)] + [(-(n // 2), 0.5), (n // 2, 0.5)])
    out = []
    for combo in itertools.product(*axes):
        out.append((np.array([c[0] for c in combo]), float(np.prod([c[1] for c in combo]))))
    return out


def mesh_fractions(nk3):
    """Fractional coordinates f of the mesh points in flat order (n1 N2 + n2) N3 + n3."""
    n1, n2, n3 = nk3
    return np.array([[a / n1, b / n2, c / n3] for a in range(n1) for b in range(n2) for c in range(n3)])


def k_interpolate(X, nk3, f_new):
    """X [nk][...] on the mesh -> [len(f_new)][...] at the fractional coordinates f_new."""
    fk = mesh_fractions(nk3)
    nk = fk.shape[0]
    out = np.zeros((len(f_new),) + X.shape[1:], complex)
    for R, w in lattice_vectors(nk3):
        XR = np.tensordot(np.exp(-2j * np.pi * fk @ R), X, axes=(0, 0)) / nk      # X(R)
        out += w * np.exp(2j * np.pi * np.asarray(f_new) @ R)[(slice(None),) + (None,) * (X.ndim - 1)] * XR
    return out
