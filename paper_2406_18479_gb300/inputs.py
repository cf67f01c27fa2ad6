"""Seeded synthetic inputs for the GW self-energy hot path.

This module serves both the CUDA path and the CPU oracle. It holds no step
of the GW method itself: it only draws the one-body Hamiltonian H(k), the
density-fitted Coulomb factor V, and the non-interacting Green's function
G0(tau) that starts every self-consistent run.

Shapes follow the paper's workloads (Sec. 2, Eqs. (H), (DF); the Si example
of Sec. 6 fixes nao = 26, beta = 100). The paper's own inputs come from
PySCF, basis sets and grid files that are not available here; these seeded
arrays stand in for them.

Layouts (row-major, complex128):
  H  [nk][nao][nao]
  V  [nk][nk][naux][nao][nao]     V[k1][k2][Q][i][j] = V_{k1 i, k2 j}(Q)
  G  [nk][ntau][nao][nao]
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "Workload", "WORKLOADS", "kmesh_points", "chebyshev_tau", "random_unitary",
    "hamiltonian", "coulomb", "g0_tau", "make_inputs", "batched_molecules", "serving_stream",
]


@dataclasses.dataclass(frozen=True)
class Workload:
    """Sizes of one synthetic GW problem."""
    name: str
    nk3: tuple          # Gamma-centred Monkhorst-Pack mesh (N1, N2, N3)
    nao: int            # orbitals
    naux: int           # auxiliary (density-fitting) functions
    ntau: int           # Chebyshev tau nodes
    nomega: int         # bosonic Matsubara samples (= ntau)
    beta: float         # inverse temperature, 1/Ha
    mu: float = 0.0     # chemical potential, Ha
    decay: float = 8.0  # V^Q scale exp(-Q/decay)
    seed: int = 0
    solid: bool = False
    vscale: float = 1.0  # overall amplitude of V (c_Q = vscale exp(-Q/decay))

    @property
    def nk(self) -> int:
        return int(np.prod(self.nk3))


# Molecule (Gamma only), Si-like 3x3x3 solid, 4x4x4 solid.
WORKLOADS = {
    "molecule_nao8": Workload("molecule_nao8", (1, 1, 1), 8, 32, 32, 32, 50.0, decay=8.0, seed=0),
    "solid_3x3x3_nao26": Workload("solid_3x3x3_nao26", (3, 3, 3), 26, 200, 100, 100, 100.0,
                                  decay=40.0, seed=1, solid=True),
    "solid_4x4x4_nao52": Workload("solid_4x4x4_nao52", (4, 4, 4), 52, 400, 120, 120, 200.0,
                                  decay=40.0, seed=2, solid=True),
    # same orbital and auxiliary sizes as the 3x3x3 solid on a 3x3x1 mesh and 25 tau nodes:
    # a case small enough for full hardware-counter captures
    "solid_3x3x1_nao26": Workload("solid_3x3x1_nao26", (3, 3, 1), 26, 200, 25, 25, 100.0,
                                  decay=40.0, seed=6, solid=True),
    # the 4x4x4 solid's orbital and auxiliary sizes on a 2x2x1 mesh and 16 tau nodes: the
    # hardware-counter case of its kernels
    "solid_2x2x1_nao52": Workload("solid_2x2x1_nao52", (2, 2, 1), 52, 400, 16, 16, 200.0,
                                  decay=40.0, seed=8, solid=True),
}


def kmesh_points(nk3) -> np.ndarray:
    """Integer coordinates (n1, n2, n3) of the Gamma-centred mesh, k = 2*pi*n/N.

    Flat index k = (n1*N2 + n2)*N3 + n3.
    """
    n1, n2, n3 = nk3
    g = np.stack(np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij"), -1)
    return g.reshape(-1, 3)


def chebyshev_tau(ntau: int, beta: float) -> np.ndarray:
    """First-kind Chebyshev nodes on [0, beta], ascending, no endpoints."""
    j = np.arange(ntau)
    return 0.5 * beta * (1.0 - np.cos(np.pi * (j + 0.5) / ntau))


def random_unitary(n: int, rng: np.random.Generator) -> np.ndarray:
    z = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    return q * (d / np.abs(d))


def _hermitian_with_spectrum(evals, rng):
    u = random_unitary(len(evals), rng)
    return (u * evals) @ u.conj().T


def hamiltonian(w: Workload, rng: np.random.Generator) -> np.ndarray:
    """H(k), Hermitian.

    Molecule: eigenvalues uniform in [-1.5, 1.5] Ha.
    Solid: onsite block with eigenvalues in [-0.75, 0.75] Ha plus
    nearest-neighbour hopping 2 cos(k_d) T_d with ||T_d||_2 = 0.125 Ha,
    which gives a total bandwidth of about 2-3 Ha.
    """
    nao = w.nao
    if not w.solid:
        h = _hermitian_with_spectrum(rng.uniform(-1.5, 1.5, nao), rng)
        return np.broadcast_to(h, (w.nk, nao, nao)).copy()
    h0 = _hermitian_with_spectrum(rng.uniform(-0.75, 0.75, nao), rng)
    t = []
    for _ in range(3):
        x = (rng.standard_normal((nao, nao)) + 1j * rng.standard_normal((nao, nao)))
        x = 0.5 * (x + x.conj().T)
        t.append(0.125 * x / np.linalg.norm(x, 2))
    pts = kmesh_points(w.nk3)
    h = np.empty((w.nk, nao, nao), complex)
    for k, n in enumerate(pts):
        kv = 2.0 * np.pi * n / np.asarray(w.nk3)
        h[k] = h0 + sum(2.0 * np.cos(kv[d]) * t[d] for d in range(3))
    return h


def coulomb(w: Workload, rng: np.random.Generator, dtype=np.complex128) -> np.ndarray:
    """V[k1][k2][Q][i][j] with V(k2,k1)^Q_ji = conj V(k1,k2)^Q_ij.

    Diagonal pairs are Hermitian in ij: c_Q (X + X^dagger)/2; pairs k1 < k2 are
    c_Q X / sqrt(2); X_ij = (a + ib)/sqrt(2), a, b ~ N(0, 1); c_Q = vscale exp(-Q/decay).
    """
    nk, nao, naux = w.nk, w.nao, w.naux
    c = w.vscale * np.exp(-np.arange(naux) / w.decay)[:, None, None]
    v = np.empty((nk, nk, naux, nao, nao), dtype)
    for k1 in range(nk):
        for k2 in range(k1, nk):
            x = (rng.standard_normal((naux, nao, nao)) + 1j * rng.standard_normal((naux, nao, nao))) / np.sqrt(2.0)
            if k1 == k2:
                v[k1, k1] = c * 0.5 * (x + x.conj().transpose(0, 2, 1))
            else:
                blk = c * x / np.sqrt(2.0)
                v[k1, k2] = blk
                v[k2, k1] = blk.conj().transpose(0, 2, 1)
    return v


def g0_tau(h: np.ndarray, mu: float, beta: float, tau: np.ndarray) -> np.ndarray:
    """Non-interacting G(k, tau) = -U diag(e^{-e tau} / (1 + e^{-beta e})) U^dagger, e = eps - mu.

    For e < 0 the factor is evaluated as e^{e (beta - tau)} / (1 + e^{beta e}) so that
    no exponential overflows.
    """
    nk, nao, _ = h.shape
    out = np.empty((nk, len(tau), nao, nao), complex)
    for k in range(nk):
        eps, u = np.linalg.eigh(h[k])
        e = eps - mu
        a = np.abs(e)
        # e >= 0: e^{-a tau}/(1+e^{-beta a});  e < 0: e^{-a (beta - tau)}/(1+e^{-beta a})
        s = np.where(e >= 0, tau[:, None], beta - tau[:, None])
        g = np.exp(-a * s) / (1.0 + np.exp(-beta * a))    # [ntau][nao]
        out[k] = -np.einsum("in,tn,jn->tij", u, g, u.conj())
    return out


def make_inputs(w: Workload):
    """(H, V, G0) for a workload, from its seed."""
    rng = np.random.default_rng(w.seed)
    h = hamiltonian(w, rng)
    v = coulomb(w, rng)
    tau = chebyshev_tau(w.ntau, w.beta)
    g = g0_tau(h, w.mu, w.beta, tau)
    return h, v, g


def molecule(name: str, nao: int, ntau: int = 80, beta: float = 100.0, seed: int = 0) -> Workload:
    """Gamma-only system with naux = 4 nao and V^Q decaying as exp(-4 Q / naux) (the nao=8 ratio)."""
    naux = 4 * nao
    return Workload(name, (1, 1, 1), nao, naux, ntau, ntau, beta, decay=naux / 4.0, seed=seed)


def batched_molecules(n: int = 48, seed: int = 4):
    """n Gamma-only systems with nao uniform on {10..120}, naux = 4 nao, 80 tau nodes, beta = 100."""
    rng = np.random.default_rng(seed)
    naos = rng.integers(10, 121, n)
    return [molecule(f"mol{i}_nao{int(a)}", int(a), seed=seed * 1000 + i) for i, a in enumerate(naos)]


# Interaction strength of the serving stream: V scaled per job so that nao sum_Q c_Q^2, the size of
# the exchange-like sums, is the same for every job (0.5^2 / (nao sum_Q exp(-2Q/decay)) times the
# unit-variance V). The unit-variance V gives max|Sigma| of 10^2..10^3 Ha, where the fixed-mu
# loop with mixing 0.5 diverges; at this strength max|Sigma| is of order 0.01 Ha and the loop
# reaches max|dSigma| < 1e-6 within 10 evaluations (mixing halves the change per iteration).
SERVING_STRENGTH = 0.5


def serving_vscale(nao: int, naux: int, decay: float) -> float:
    """V amplitude of a serving job: SERVING_STRENGTH / sqrt(nao sum_Q exp(-2 Q / decay))."""
    return SERVING_STRENGTH / float(np.sqrt(nao * np.sum(np.exp(-2.0 * np.arange(naux) / decay))))


def serving_stream(n: int = 200, seed: int = 5):
    """Seeded scGW job stream: [(gap, Workload)], gaps exponential with unit mean (Poisson arrivals;
    the caller divides by the rate). 70% molecules with nao on {10..120}; 30% solids on a 2x2x2 or
    3x3x3 mesh with nao on {16..52}; naux = 4 nao, 80 tau nodes, beta = 100; V at the serving
    strength (serving_vscale).
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        gap = float(rng.exponential(1.0))
        if rng.random() < 0.7:
            w = molecule(f"job{i}_mol_nao", int(rng.integers(10, 121)), seed=seed * 1000 + i)
            w = dataclasses.replace(w, name=f"job{i}_mol_nao{w.nao}")
        else:
            m = (2, 2, 2) if rng.random() < 0.5 else (3, 3, 3)
            nao = int(rng.integers(16, 53))
            w = Workload(f"job{i}_solid{m[0]}_nao{nao}", m, nao, 4 * nao, 80, 80, 100.0, decay=40.0,
                         seed=seed * 1000 + i, solid=True)
        w = dataclasses.replace(w, vscale=serving_vscale(w.nao, w.naux, w.decay))
        out.append((gap, w))
    return out


def pack_v(v: np.ndarray) -> np.ndarray:
    """The pairs k1 <= k2 of V[k1][k2] in row order of the upper triangle (the packed layout)."""
    nk = v.shape[0]
    return np.ascontiguousarray(np.stack([v[a, b] for a in range(nk) for b in range(a, nk)]))


def overlap(w: Workload, rng: np.random.Generator, spread: float = 0.3) -> np.ndarray:
    """S(k), Hermitian positive definite: eigenvalues uniform in [1 - spread, 1 + spread] in a
    random basis per k (a non-orthogonal orbital basis)."""
    return np.stack([_hermitian_with_spectrum(rng.uniform(1.0 - spread, 1.0 + spread, w.nao), rng)
                     for _ in range(w.nk)])
