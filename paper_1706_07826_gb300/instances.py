"""Seeded synthetic Ising instances shaped like the paper's workloads.

This module holds no step of the method: it only draws couplers and biases.
It serves both the CUDA path (benchmark, tests) and the oracle (tests), so it
imports nothing from either.  Every generator returns an :class:`Instance`
with an edge list (each pair once, ``i != j``), integer couplers, integer
biases and an energy scale (real-valued instances are stored as integers
multiplied by ``scale``).

Shapes follow the paper's problem classes: 3D periodic +-J spin glasses
(Sec. III.D), native Chimera graphs (Sec. III.C) and weak-strong cluster
problems on Chimera (Sec. III.B).
"""
import dataclasses

import numpy as np


@dataclasses.dataclass
class Instance:
    name: str
    n: int
    ei: np.ndarray      # int32 [m]
    ej: np.ndarray      # int32 [m]
    J: np.ndarray       # int32 [m]
    h: np.ndarray       # int32 [n]
    scale: int = 1      # real value = integer / scale
    offset: int = 0

    @property
    def m(self):
        return len(self.ei)


def _rng(seed):
    return np.random.default_rng(np.random.PCG64(seed))


def cubic3d(L, seed, name=None):
    """Periodic L x L x L cubic lattice, couplers uniform in {-1,+1}, h = 0.

    Site (x, y, z) has index x + L*(y + L*z); each site couples to its +x, +y
    and +z neighbours with wrap-around, so there are 3*L^3 couplers (L >= 3).
    """
    if L < 3:
        raise ValueError("L must be >= 3 so that the periodic neighbours are distinct")
    g = _rng(seed)
    n = L ** 3
    idx = np.arange(n, dtype=np.int64)
    x, y, z = idx % L, (idx // L) % L, idx // (L * L)
    nb = [((x + 1) % L) + L * (y + L * z),
          x + L * (((y + 1) % L) + L * z),
          x + L * (y + L * ((z + 1) % L))]
    ei = np.concatenate([idx, idx, idx]).astype(np.int32)
    ej = np.concatenate(nb).astype(np.int32)
    J = (g.integers(0, 2, size=len(ei)) * 2 - 1).astype(np.int32)
    h = np.zeros(n, np.int32)
    return Instance(name or "cubic3d_L%d_s%d" % (L, seed), n, ei, ej, J, h)


def chimera_edges(M):
    """Edges of the Chimera graph C_M (M x M unit cells of K_{4,4}).

    Qubit (row r, column c, side u, position k) has index 8*(r*M + c) + 4*u + k.
    Inside a cell every side-0 qubit couples to every side-1 qubit; side-0
    qubits couple to the same position in the cell below, side-1 qubits to
    the same position in the cell to the right.  16 M^2 + 8 M (M - 1) edges.
    """
    ei, ej, kind = [], [], []

    def q(r, c, u, k):
        return 8 * (r * M + c) + 4 * u + k

    for r in range(M):
        for c in range(M):
            for k0 in range(4):
                for k1 in range(4):
                    ei.append(q(r, c, 0, k0)); ej.append(q(r, c, 1, k1)); kind.append(0)
    for r in range(M):
        for c in range(M):
            for k in range(4):
                if r + 1 < M:
                    ei.append(q(r, c, 0, k)); ej.append(q(r + 1, c, 0, k)); kind.append(1)
                if c + 1 < M:
                    ei.append(q(r, c, 1, k)); ej.append(q(r, c + 1, 1, k)); kind.append(1)
    return (np.array(ei, np.int32), np.array(ej, np.int32), np.array(kind, np.int8))


def chimera(M, seed, name=None):
    """Native Chimera C_M, couplers uniform in {-1,+1}, h = 0 (N = 8 M^2)."""
    g = _rng(seed)
    ei, ej, _ = chimera_edges(M)
    J = (g.integers(0, 2, size=len(ei)) * 2 - 1).astype(np.int32)
    return Instance(name or "chimera_C%d_s%d" % (M, seed), 8 * M * M, ei, ej, J, np.zeros(8 * M * M, np.int32))


def weak_strong(M, seed, h_strong=-100, h_weak=44, j_intra=-100, j_inter=100, scale=100, name=None):
    """Weak-strong cluster problem on Chimera C_M, stored x scale.

    Each unit cell is a ferromagnetic cluster (intra-cell couplers
    ``j_intra``); cells with (r + c) even are strong (bias ``h_strong``),
    the others weak (bias ``h_weak``); inter-cell couplers are uniform in
    {-j_inter, +j_inter}.  The defaults are -1, -1, +0.44 and +-1 times 100.
    """
    g = _rng(seed)
    ei, ej, kind = chimera_edges(M)
    J = np.where(kind == 0, j_intra, (g.integers(0, 2, size=len(ei)) * 2 - 1) * j_inter).astype(np.int32)
    n = 8 * M * M
    cell = np.arange(n) // 8
    r, c = cell // M, cell % M
    h = np.where((r + c) % 2 == 0, h_strong, h_weak).astype(np.int32)
    return Instance(name or "weak_strong_C%d_s%d" % (M, seed), n, ei, ej, J, h, scale=scale)


def chimera_u10(M, seed, name=None):
    """Reduced-degeneracy Chimera C_M problem (the U_10 class of Sec. III.C):
    couplers uniform in {-10, ..., 10} without 0, biases uniform in {-10, ..., 10},
    stored with scale 10 (so that |J| <= 1 in problem units)."""
    g = _rng(seed)
    ei, ej, _ = chimera_edges(M)
    J = (g.integers(1, 11, size=len(ei)) * (g.integers(0, 2, size=len(ei)) * 2 - 1)).astype(np.int32)
    h = g.integers(-10, 11, size=8 * M * M).astype(np.int32)
    return Instance(name or "chimera_u10_C%d_s%d" % (M, seed), 8 * M * M, ei, ej, J, h, scale=10)


def weak_strong_pair(h_strong=-100, h_weak=44, j=-100, scale=100):
    """The two-cluster weak-strong toy (Sec. III.B): two Chimera unit cells,
    ferromagnetic inside and between them (the four inter-cell couplers), the
    first cell strong, the second weak, stored x scale."""
    ei, ej, kind = chimera_edges(2)
    keep = (ei < 16) & (ej < 16)
    ei, ej = ei[keep].astype(np.int32), ej[keep].astype(np.int32)
    h = np.array([h_strong] * 8 + [h_weak] * 8, np.int32)
    return Instance("weak_strong_pair", 16, ei, ej, np.full(len(ei), j, np.int32), h, scale=scale)


def random_graph(n, m, seed, jmax=3, hmax=2, name=None):
    """Small random sparse problem: m distinct pairs, J in [-jmax, jmax] \\ {0},
    h uniform in [-hmax, hmax].  Used for brute-force checks (n <= 20)."""
    g = _rng(seed)
    pairs = set()
    allp = [(i, j) for i in range(n) for j in range(i + 1, n)]
    m = min(m, len(allp))
    pick = g.choice(len(allp), size=m, replace=False) if m else []
    for t in pick:
        pairs.add(allp[int(t)])
    pairs = sorted(pairs)
    ei = np.array([p[0] for p in pairs], np.int32)
    ej = np.array([p[1] for p in pairs], np.int32)
    mag = g.integers(1, jmax + 1, size=len(pairs))
    sgn = g.integers(0, 2, size=len(pairs)) * 2 - 1
    J = (mag * sgn).astype(np.int32)
    h = g.integers(-hmax, hmax + 1, size=n).astype(np.int32)
    return Instance(name or "random_n%d_m%d_s%d" % (n, m, seed), n, ei, ej, J, h)


def uneven_batch(count=64, lmin=6, lmax=12, seed=1400):
    """``count`` 3D +-J instances with L uniform in [lmin, lmax]."""
    g = _rng(seed)
    Ls = g.integers(lmin, lmax + 1, size=count)
    return [cubic3d(int(L), seed + 1 + i) for i, L in enumerate(Ls)]


def poisson_stream(count, rate_per_s, lmin=8, lmax=20, seed=1500):
    """Arrival times (Poisson process) and 3D +-J instances, L in [lmin, lmax]."""
    g = _rng(seed)
    gaps = g.exponential(1.0 / rate_per_s, size=count)
    t = np.cumsum(gaps) - gaps[0]
    Ls = g.integers(lmin, lmax + 1, size=count)
    return t, [cubic3d(int(L), seed + 1 + i) for i, L in enumerate(Ls)]
