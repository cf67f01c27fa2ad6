"""Imaginary-time grid and Fourier-transform matrices (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper transforms P0 from tau to bosonic Matsubara frequencies with the
integral of Eq. (P0t_to_P0w), Sec. 2.3, on sparse grids read from grid files
(Sec. 5, "--grid_file"). Those files are not available, so the grid is built
here from its definition:

* tau nodes: first-kind Chebyshev nodes on [0, beta]; a function on [0, beta]
  is represented by its Chebyshev interpolant through those nodes.
* F (i Omega <- tau): F = T C, with T_nl = int_0^beta T_l(x(tau)) e^{i w_n tau} dtau
  (Eq. P0t_to_P0w applied to each Chebyshev polynomial) and C the map from
  node values to Chebyshev coefficients. T is evaluated by composite
  Gauss-Legendre quadrature fine enough to integrate the oscillation to
  rounding.
* B (tau <- i Omega) = the least-squares left inverse of F (F^{-1} when
  square): values at the sampled frequencies determine the interpolant, so
  B F = I. The sample set is symmetric in w (sample_count()).
* Frequencies: bosonic w_n = 2 n pi / beta (Sec. 2.3), fermionic
  w_n = (2n+1) pi / beta (Eq. dyson). The sample set is the rule written out in
  matsubara_indices(), restated independently here.
"""
from __future__ import annotations

import functools
import numpy as np


def chebyshev_nodes(ntau: int, beta: float) -> np.ndarray:
    """tau_j = (beta/2)(1 - cos(pi (j + 1/2)/ntau)), j = 0..ntau-1 (ascending)."""
    j = np.arange(ntau)
    return 0.5 * beta * (1.0 - np.cos(np.pi * (j + 0.5) / ntau))


def sample_count(ntau: int, stat: int) -> int:
    """Number of sampled frequencies for an ntau-node grid.

    The sample set is symmetric under w -> -w (so that a Hermitian-valued
    function keeps X(-i w) = X(i w)^dagger and its back-transform stays
    Hermitian). A symmetric bosonic set has odd size and a symmetric fermionic
    set even size, so the count is ntau, or ntau + 1 when the parity differs.
    """
    want_odd = stat == 0
    return ntau if (ntau % 2 == 1) == want_odd else ntau + 1


def matsubara_indices(n: int, stat: int) -> np.ndarray:
    """Sorted integer indices m of n sampled Matsubara frequencies, symmetric in w.

    stat = 0 (bosonic, w = 2 m pi / beta, n odd) or 1 (fermionic,
    w = (2m+1) pi / beta, n even).
    n <= 5: the n frequencies of smallest |w|.
    n >= 6: with M = n // 3, a dense core of every frequency with |w| <= w_M
    (bosonic m in [-M, M]; fermionic m in [-M-1, M]); then K = (n - core)/2 tail
    frequencies on each side, placed uniformly in 1/m:
        m_j = round(M (2K+3) / (2K+3-2j)), j = 1..K   (round half up, exact integers),
    mirrored to -m_j - stat on the negative side.
    """
    if (n % 2 == 1) != (stat == 0):
        raise ValueError("bosonic sets have odd size, fermionic sets even size")
    if n <= 5:
        cand = sorted(range(-n - 1, n + 1), key=lambda m: (abs(2 * m + stat), m < 0))
        return np.array(sorted(cand[:n]), dtype=np.int64)
    big_m = n // 3
    core = list(range(-big_m - stat, big_m + 1))
    k = (n - len(core)) // 2
    tail = []
    for j in range(1, k + 1):
        num = big_m * (2 * k + 3)
        den = 2 * k + 3 - 2 * j
        tail.append((2 * num + den) // (2 * den))
    vals = sorted(core + tail + [-t - stat for t in tail])
    assert len(set(vals)) == n
    return np.array(vals, dtype=np.int64)


def matsubara_frequencies(ntau: int, stat: int, beta: float) -> np.ndarray:
    m = matsubara_indices(sample_count(ntau, stat), stat)
    return (2 * m + stat) * np.pi / beta


@functools.lru_cache(maxsize=64)
def _unit_transform(ntau: int, stat: int):
    """F and B for beta = 1 (F scales with beta, B with 1/beta)."""
    m = matsubara_indices(sample_count(ntau, stat), stat)
    w = (2 * m + stat) * np.pi                              # frequencies for beta = 1
    # Chebyshev polynomials T_l(x), x = 2 tau - 1, at the tau nodes: C = (T_tl)^{-1}
    tau = chebyshev_nodes(ntau, 1.0)
    x_nodes = 2.0 * tau - 1.0
    l = np.arange(ntau)
    t_nodes = np.cos(np.outer(np.arccos(np.clip(x_nodes, -1, 1)), l))   # [t][l]
    c = np.linalg.inv(t_nodes)                              # [l][t]
    # T_nl = int_0^1 T_l(2 tau - 1) e^{i w_n tau} dtau, in x = 2 tau - 1 on [-1, 1]:
    # composite 24-point Gauss-Legendre on panels x_p = -cos(pi p / P), which are
    # graded like the Chebyshev polynomials and span a few radians of phase each.
    panels = int(np.ceil((np.max(np.abs(w)) / 2.0 + ntau) / 2.0)) + 8
    edges = -np.cos(np.pi * np.arange(panels + 1) / panels)
    g, gwt = np.polynomial.legendre.leggauss(24)
    lo, hi = edges[:-1], edges[1:]
    xq = (0.5 * (hi - lo)[:, None] * (g[None, :] + 1.0) + lo[:, None]).ravel()
    wq = (0.5 * (hi - lo)[:, None] * gwt[None, :]).ravel()
    tl_q = np.cos(np.outer(np.arccos(np.clip(xq, -1.0, 1.0)), l))   # [q][l]
    phase = np.exp(1j * np.outer(w, 0.5 * (xq + 1.0)))      # [n][q]
    t_nl = 0.5 * (phase * wq) @ tl_q                        # [n][l]
    f = t_nl @ c                                            # [n][t]
    b = np.linalg.pinv(f, rcond=1e-14)                      # [t][n], least-squares left inverse
    return m, f, b


def transform_matrices(ntau: int, beta: float, stat: int):
    """(indices m, F [nw][ntau], B [ntau][nw]) for the given statistics and beta."""
    m, f, b = _unit_transform(ntau, stat)
    return m.copy(), f * beta, b / beta
