"""Seeded synthetic cluster generators (atoms only; no method arithmetic).

The paper's workloads are finite FCC aluminium clusters (Sec. 5: m x m x m FCC
unit cells with M = 14, 172, 666, 1688, 3430 atoms; Al2/Al3; a 5x5x5 cluster
at a = 8.0 bohr).  Its Goodwin-Needs-Heine pseudopotential parameters are not
given, so these generators only build geometries; the pseudocharge model
(Gaussian, sigma = 1 bohr, Z = 3) is chosen by the caller.

This module is shared by the CPU oracle's tests and the GPU path: it holds
positions, charges and seeds, nothing that evaluates the method.
"""
from __future__ import annotations

import dataclasses

import numpy as np

__all__ = [
    "Cluster",
    "fcc_cube_sites",
    "cuboctahedron_sites",
    "displaced",
    "cluster_c1",
    "cluster_c2",
    "cluster_c3",
    "batch_c4",
    "serving_requests_c5",
    "tiny_cluster",
]


@dataclasses.dataclass
class Cluster:
    """A cluster of M nuclei: positions R (M x 3, bohr), charges Z (M,)."""

    name: str
    R: np.ndarray
    Z: np.ndarray
    h: float
    fd_order: int
    vacuum: float
    seed: int

    @property
    def M(self) -> int:
        return int(self.R.shape[0])

    @property
    def N(self) -> float:
        """Electron count of the charge-neutral system (Sec. 2: N = sum Z)."""
        return float(np.sum(self.Z))


def fcc_cube_sites(m: int, a: float) -> np.ndarray:
    """Sites of an m x m x m block of FCC unit cells, centred on the origin.

    Lattice points (i, j, k) * a/2 with 0 <= i, j, k <= 2m and i + j + k even;
    this gives 4m^3 + 6m^2 + 3m + 1 atoms (14, 172, 666, 2457 for m = 1, 3, 5, 8).
    """
    idx = np.arange(2 * m + 1)
    i, j, k = np.meshgrid(idx, idx, idx, indexing="ij")
    keep = ((i + j + k) % 2) == 0
    pts = np.stack([i[keep], j[keep], k[keep]], axis=1).astype(np.float64)
    pts = pts * (a / 2.0)
    pts -= m * a / 2.0
    return pts


def cuboctahedron_sites(a: float) -> np.ndarray:
    """13-atom FCC cuboctahedron: the origin and its 12 nearest neighbours."""
    s = a / 2.0
    pts = [(0.0, 0.0, 0.0)]
    for x in (-s, s):
        for y in (-s, s):
            pts.append((x, y, 0.0))
            pts.append((x, 0.0, y))
            pts.append((0.0, x, y))
    return np.array(pts, dtype=np.float64)


def displaced(R: np.ndarray, amp: float, seed: int) -> np.ndarray:
    """R plus per-coordinate displacements uniform in [-amp, amp] (PCG64 stream)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return R + rng.uniform(-amp, amp, size=R.shape)


def _cluster(name, sites, seed, h, fd_order, vacuum, Z=3.0, amp=0.1):
    R = displaced(sites, amp, seed)
    return Cluster(name=name, R=R, Z=np.full(R.shape[0], Z), h=h,
                   fd_order=fd_order, vacuum=vacuum, seed=seed)


def cluster_c1(seed: int = 1) -> Cluster:
    """13-atom cuboctahedron, a = 7.6 bohr, h = 0.8, 12th order, 8 bohr vacuum (32^3 grid)."""
    return _cluster("cubocta13_h0.8_o12", cuboctahedron_sites(7.6), seed, 0.8, 12, 8.0)


def cluster_c2(seed: int = 2) -> Cluster:
    """5x5x5 FCC cube (666 atoms), a = 7.6, h = 0.5, 12th order, 10 bohr vacuum (128^3)."""
    return _cluster("fcc5_666_h0.5_o12", fcc_cube_sites(5, 7.6), seed, 0.5, 12, 10.0)


def cluster_c3(seed: int = 3) -> Cluster:
    """8x8x8 FCC cube (2457 atoms), a = 7.6, h = 0.45, 12th order, 10 bohr vacuum (192^3)."""
    return _cluster("fcc8_2457_h0.45_o12", fcc_cube_sites(8, 7.6), seed, 0.45, 12, 10.0)


def batch_c4(count: int = 64, seed0: int = 0) -> list[Cluster]:
    """count FCC cubes, m uniform in {1..5} (seeded), h = 0.5, 12th order, 8 bohr vacuum."""
    out = []
    for s in range(seed0, seed0 + count):
        rng = np.random.Generator(np.random.PCG64(10_000 + s))
        m = int(rng.integers(1, 6))
        out.append(_cluster(f"fcc{m}_seed{s}", fcc_cube_sites(m, 7.6), s, 0.5, 12, 8.0))
    return out


def serving_requests_c5(rate: float, count: int, seed: int = 5,
                        max_m: int = 8) -> list[tuple[float, Cluster]]:
    """Poisson arrivals at `rate`/s of clusters with m log-uniform in {1..max_m},
    h in {0.45, 0.5, 0.6}, FD order in {8, 12}, 8 bohr vacuum.

    Returns (arrival time in seconds, cluster) pairs in arrival order.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    logs = np.log(np.arange(1, max_m + 1, dtype=np.float64))
    for r in range(count):
        t += rng.exponential(1.0 / rate)
        x = rng.uniform(0.0, np.log(max_m + 1.0))
        m = int(np.searchsorted(logs, x, side="right"))
        m = min(max(m, 1), max_m)
        h = float(rng.choice([0.45, 0.5, 0.6]))
        order = int(rng.choice([8, 12]))
        out.append((t, _cluster(f"req{r}_fcc{m}", fcc_cube_sites(m, 7.6),
                                seed * 100_000 + r, h, order, 8.0)))
    return out


def tiny_cluster(kind: str = "dimer", seed: int = 7, h: float = 0.8,
                 fd_order: int = 6, vacuum: float = 8.0) -> Cluster:
    """Small clusters for fast CPU tests: 'atom', 'dimer' (5.2 bohr), 'trimer'."""
    if kind == "atom":
        sites = np.zeros((1, 3))
    elif kind == "dimer":
        sites = np.array([[-2.6, 0.0, 0.0], [2.6, 0.0, 0.0]])
    elif kind == "trimer":
        r = 5.3 / np.sqrt(3.0)
        ang = np.array([0.0, 2.0 * np.pi / 3.0, 4.0 * np.pi / 3.0])
        sites = np.stack([r * np.cos(ang), r * np.sin(ang), np.zeros(3)], axis=1)
    else:
        raise ValueError(kind)
    return _cluster(f"{kind}_h{h}_o{fd_order}", sites, seed, h, fd_order, vacuum,
                    amp=0.05 if kind != "atom" else 0.0)
