"""Seeded random packings of equal spheres, shaped like the paper's workloads.

The paper (Sec. 6, Appendix E, Algorithm 5) builds its initial configurations
from a jittered cubic lattice whose scale is bisected until the number of
candidate contacts hits a target.  Its saved configurations are not
available, so synthetic packings stand in for them, built the same way:

1. ``M`` sites of an ``m x m x m`` cubic lattice (``m = ceil(M^(1/3))``; all
   of them for the paper's lattice sizes 2^3, 4^3, 6^3), spaced for the
   nominal volume fraction, plus uniform jitter;
2. the lattice is scaled about its centroid by ``gamma`` and an
   overlap-removal sweep pushes apart every pair closer than ``2a + h_ij``,
   where ``h_ij = delta * (floor + (1 - floor) * u**power)`` with
   ``u ~ U(0, 1)`` drawn once per pair.  The high power leaves most
   candidate pairs nearly touching, as in a clustered suspension, so that a
   good share of the contacts is active at the workloads' time steps;
3. ``gamma`` is bisected until the number of pairs with gap below ``delta``
   is within 10% of the requested contact count (else the closest is kept).

Every gap of the result is strictly positive (asserted).  Janus axes are
normalised Gaussian draws (uniform on the sphere).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Instance:
    """One collision-resolution problem: geometry plus solver parameters."""

    name: str
    seed: int
    centers: np.ndarray  # [M, 3] float64
    axes: np.ndarray  # [M, 3] float64, unit Janus axes
    n_theta: int  # Gauss-Legendre polar nodes per sphere
    n_phi: int  # uniform azimuthal nodes per sphere
    radius: float  # hydrodynamic radius: the boundary-integral surfaces
    contact_radius: float  # steric radius: gaps and contacts are measured with it
    viscosity: float
    dt: float
    delta: float
    tol: float
    phi_nominal: float
    n_candidates: int  # pairs with gap below delta

    @property
    def n_bodies(self) -> int:
        return int(self.centers.shape[0])

    @property
    def nodes_per_body(self) -> int:
        return self.n_theta * self.n_phi


# The boundary-integral surfaces have radius 1 (the hydrodynamic radius).  Gaps
# and contacts are measured on concentric steric spheres of radius 1.25, so the
# surfaces of touching particles stay half a radius apart.  That separation is
# what the 98- to 242-node product grids resolve with the smooth quadrature
# (the near-singular evaluation of the paper's own solver is not part of the
# stand-in operator).
CONTACT_RADIUS = 1.25

# Workloads named by what they are.  Sizes follow the paper's lattices
# (2^3, 4^3, 6^3 particles; Sec. 6.2) and its high-fidelity order p = 8
# (9 x 18 product grid).
WORKLOADS = {
    "spheres8_grid7x14": dict(M=8, n_theta=7, n_phi=14, phi=0.30, delta=0.1,
                              n_target=10, dt=0.01, tol=1e-8, seed_base=1000),
    "spheres64_grid9x18": dict(M=64, n_theta=9, n_phi=18, phi=0.40, delta=0.05,
                               n_target=150, dt=0.01, tol=1e-8, seed_base=2000),
    "spheres216_grid11x22": dict(M=216, n_theta=11, n_phi=22, phi=0.45, delta=0.05,
                                 n_target=600, dt=0.005, tol=1e-8, seed_base=3000),
}


def _pairwise(c: np.ndarray):
    diff = c[:, None, :] - c[None, :, :]
    d = np.sqrt(np.einsum("ijk,ijk->ij", diff, diff))
    return diff, d


def _separate(c: np.ndarray, target: np.ndarray, tol: float,
              max_sweeps: int = 20000) -> np.ndarray:
    """Jacobi sweeps that push every pair closer than ``target - tol`` apart."""
    M = c.shape[0]
    for _ in range(8):
        _, d = _pairwise(c)
        np.fill_diagonal(d, np.inf)
        i, j = np.nonzero(np.triu(d < target + 0.5, 1))  # neighbour list
        tij = target[i, j]
        for _ in range(max_sweeps // 8):
            diff = c[i] - c[j]
            dij = np.sqrt(np.einsum("ij,ij->i", diff, diff))
            deficit = tij - dij
            mask = deficit > tol
            if not mask.any():
                break
            push = (np.where(mask, 0.45 * deficit / dij, 0.0))[:, None] * diff
            c = c + np.stack([np.bincount(i, push[:, k], M) - np.bincount(j, push[:, k], M)
                              for k in range(3)], axis=1)
        _, d = _pairwise(c)
        np.fill_diagonal(d, np.inf)
        if not (d < target - tol).any():
            return c
    raise RuntimeError("overlap removal did not converge")


def random_packing(M: int, phi: float, delta: float, n_target: int, seed: int,
                   a: float = 1.25, gap_power: float = 8.0, gap_floor: float = 1e-3,
                   jitter: float = 0.5) -> tuple[np.ndarray, dict]:
    """Packing of ``M`` spheres of (contact) radius ``a``; see the module docstring."""
    rng = np.random.default_rng(seed)
    m = int(math.ceil(M ** (1.0 / 3.0) - 1e-9))
    grid = np.stack(np.meshgrid(*(np.arange(m),) * 3, indexing="ij"), -1).reshape(-1, 3)
    sites = grid[np.sort(rng.choice(m ** 3, size=M, replace=False))].astype(np.float64)
    spacing = (M * (4.0 / 3.0) * math.pi * a ** 3 / phi) ** (1.0 / 3.0) / m
    base = (sites - sites.mean(axis=0)) * spacing
    base += rng.uniform(-jitter / 2, jitter / 2, size=base.shape)
    u = rng.uniform(0.0, 1.0, size=(M, M))
    u = np.triu(u, 1)
    u = u + u.T
    h = delta * (gap_floor + (1.0 - gap_floor) * u ** gap_power)
    target = 2 * a + h
    np.fill_diagonal(target, 0.0)
    eye = np.eye(M, dtype=bool)

    def build(gamma):
        c = _separate(gamma * base, target, tol=0.05 * delta * gap_floor)
        _, d = _pairwise(c)
        d[eye] = np.inf
        return c, int(np.count_nonzero(np.triu(d - 2 * a < delta, 1)))

    lo, hi = 0.85 * 2 * a / spacing, max(1.0, 1.1 * (2 * a + delta) / spacing)
    c_hi, n_hi = build(hi)
    best = (abs(n_hi - n_target), hi, c_hi, n_hi)
    if n_hi < n_target:
        for _ in range(30):
            mid = 0.5 * (lo + hi)
            c, n = build(mid)
            if abs(n - n_target) < best[0]:
                best = (abs(n - n_target), mid, c, n)
            if abs(n - n_target) <= 0.1 * n_target:
                break
            if n < n_target:
                hi = mid
            else:
                lo = mid
    _, gamma, centers, n_cand = best
    _, d = _pairwise(centers)
    d[eye] = np.inf
    min_gap = float(d.min() - 2 * a)
    assert min_gap > 0.0, min_gap
    centers = centers - centers.mean(axis=0)
    info = dict(phi_nominal=float(M * (4.0 / 3.0) * math.pi * a ** 3 / (m * gamma * spacing) ** 3),
                n_candidates=n_cand, min_gap=min_gap)
    return centers, info


def janus_axes(M: int, seed: int) -> np.ndarray:
    """Unit Janus axes, uniform on the sphere (normalised Gaussian draws)."""
    rng = np.random.default_rng(seed + 7919)
    e = rng.standard_normal((M, 3))
    return e / np.linalg.norm(e, axis=1, keepdims=True)


def make_instance(name: str, index: int = 0, **overrides) -> Instance:
    """Instance ``index`` of a named workload; seed = seed_base + index."""
    w = dict(WORKLOADS[name])
    w.update(overrides)
    seed = w["seed_base"] + index
    centers, info = random_packing(w["M"], w["phi"], w["delta"], w["n_target"], seed,
                                   a=CONTACT_RADIUS)
    return Instance(name=name, seed=seed, centers=centers, axes=janus_axes(w["M"], seed),
                    n_theta=w["n_theta"], n_phi=w["n_phi"], radius=1.0,
                    contact_radius=CONTACT_RADIUS, viscosity=1.0,
                    dt=w["dt"], delta=w["delta"], tol=w["tol"],
                    phi_nominal=info["phi_nominal"], n_candidates=info["n_candidates"])


def batched_instances(count: int = 256, seed: int = 4000) -> list[Instance]:
    """Uneven batch: M ~ U{8..128}, grid 7x14 or 9x18, phi ~ U(0.30, 0.45)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        M = int(rng.integers(8, 129))
        fine = bool(rng.integers(0, 2))
        phi = float(rng.uniform(0.30, 0.45))
        s = seed + 1 + i
        n_target = max(1, int(round(2.3 * M)))
        centers, info = random_packing(M, phi, 0.05, n_target, s, a=CONTACT_RADIUS)
        out.append(Instance(name=f"batch{i}", seed=s, centers=centers, axes=janus_axes(M, s),
                            n_theta=9 if fine else 7, n_phi=18 if fine else 14, radius=1.0,
                            contact_radius=CONTACT_RADIUS, viscosity=1.0, dt=0.01, delta=0.05, tol=1e-8,
                            phi_nominal=info["phi_nominal"], n_candidates=info["n_candidates"]))
    return out


def serving_simulations(count: int = 32, seed: int = 5000) -> list[Instance]:
    """Concurrent simulations: M ~ U{16..216}, 9x18 grid, phi ~ U(0.35, 0.45)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        M = int(rng.integers(16, 217))
        phi = float(rng.uniform(0.35, 0.45))
        s = seed + 1 + i
        centers, info = random_packing(M, phi, 0.05, int(round(2.5 * M)), s, a=CONTACT_RADIUS)
        out.append(Instance(name=f"sim{i}", seed=s, centers=centers, axes=janus_axes(M, s),
                            n_theta=9, n_phi=18, radius=1.0, contact_radius=CONTACT_RADIUS,
                            viscosity=1.0, dt=0.01,
                            delta=0.05, tol=1e-8, phi_nominal=info["phi_nominal"],
                            n_candidates=info["n_candidates"]))
    return out
