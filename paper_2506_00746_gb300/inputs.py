"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module only draws numbers and lays them out on the structured lattice; it holds
none of the method's arithmetic (no quadrature, no basis, no geometry map, no operator).
Both sides of every parity check receive exactly these arrays.

Conventions (the discrete problem of Eq. 1 on a structured lattice of the unit box):

* ``n`` elements per direction, ``dim`` in {2, 3}; vertex ``(i, j[, l])`` has the lexicographic
  index ``i + (n+1)*(j + (n+1)*l)`` (x fastest); coordinates are an array ``[(n+1)**dim, dim]``.
* Degrees of freedom of an order-``k`` continuous Lagrange space form the lattice
  ``(k*n+1)**dim``, again x fastest.  Elements are numbered ``ex + n*(ey + n*ez)``.
* Boundary (essential) DOFs are those with a lattice coordinate equal to 0 or ``k*n``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "lattice_vertices", "smooth_field", "uniform_vector", "design_field",
    "boundary_mask", "Workload", "WORKLOADS", "sweep_workload", "batched_instances",
]


def lattice_index(m: int, dim: int) -> np.ndarray:
    """Integer lattice coordinates ``[dim, m**dim]`` of an ``m**dim`` point lattice, x fastest.

    Column ``q`` holds ``(i_x, i_y[, i_z])`` with ``q = i_x + m*(i_y + m*i_z)``.
    """
    return np.indices((m,) * dim).reshape(dim, -1)[::-1].copy()


def lattice_vertices(dim: int, n: int, seed: int = 0, jitter: float = 0.1) -> np.ndarray:
    """Vertices of an ``n**dim`` lattice on [0,1]^dim with seeded interior jitter.

    Each interior vertex component moves by U[-jitter*h, jitter*h]/sqrt(dim), so the Euclidean
    shift is at most ``jitter*h``; boundary vertices stay where they are, so the domain stays
    the unit box.  ``jitter=0`` gives the undistorted lattice.
    """
    if dim not in (2, 3) or n < 1:
        raise ValueError("dim must be 2 or 3 and n >= 1")
    h = 1.0 / n
    idx = lattice_index(n + 1, dim)
    coords = np.ascontiguousarray(idx.T.astype(np.float64) * h)
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        shift = rng.uniform(-jitter * h, jitter * h, size=coords.shape) / math.sqrt(dim)
        interior = np.all((idx > 0) & (idx < n), axis=0)
        coords[interior] += shift[interior]
    return coords


def _lattice_params(dim: int, n: int, order: int) -> list[np.ndarray]:
    """Lattice coordinate of every DOF divided by k*n (in [0,1]), one array per axis, x fastest."""
    idx = lattice_index(order * n + 1, dim)
    return [idx[d] / float(order * n) for d in range(dim)]


def boundary_mask(dim: int, n: int, order: int) -> np.ndarray:
    """uint8 mask of the essential (boundary) DOFs of the lattice, x fastest."""
    m = order * n + 1
    idx = lattice_index(m, dim)
    return np.any((idx == 0) | (idx == m - 1), axis=0).astype(np.uint8)


def smooth_field(dim: int, n: int, order: int, seed: int = 1, amplitude: float = 1.0) -> np.ndarray:
    """Seeded smooth random state on the DOF lattice, exactly zero on the boundary.

    ``u = sum_{m in {1,2,3}^dim} a_m prod_d sin(m_d*pi*t_d)`` with ``a_m ~ N(0,1)/|m|^2`` and
    ``t_d`` the DOF's lattice coordinate divided by ``k*n``.  Evaluated on lattice parameters (not
    physical node positions) so that no geometry is needed to draw it.
    """
    rng = np.random.default_rng(seed)
    ts = _lattice_params(dim, n, order)
    u = np.zeros(ts[0].shape, dtype=np.float64)
    for mvec in np.ndindex(*(3,) * dim):
        m = np.array(mvec) + 1
        a = rng.standard_normal() / float(np.dot(m, m))
        term = np.full_like(u, a * amplitude)
        for d in range(dim):
            term *= np.sin(m[d] * math.pi * ts[d])
        u += term
    u[boundary_mask(dim, n, order).astype(bool)] = 0.0
    return u


def uniform_vector(size: int, seed: int = 2, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Seeded U[lo, hi] vector (the random direction ``v`` of a Jacobian action)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=size)


def design_field(dim: int, n: int, seed: int = 3) -> np.ndarray:
    """Piecewise-constant design field: one U[0,1] value per element (element order ex fastest)."""
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=n ** dim)


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic workload: mesh, discretisation and the law's constants."""
    name: str
    dim: int
    n: int
    order: int
    p: float = 3.0
    eps: float = 0.0
    f_const: float = 1.0
    mesh_seed: int = 0
    state_seed: int = 1
    dir_seed: int = 2

    @property
    def n_dofs(self) -> int:
        return (self.order * self.n + 1) ** self.dim

    @property
    def n_elements(self) -> int:
        return self.n ** self.dim


# The two fixed single-problem workloads, the 48^3 design workload, and a scaled-down 3D problem
# (16^3, order 2) small enough for a Newton solve by the CPU reference.
WORKLOADS = {
    "2d_p3_k2_16x16": Workload("2d_p3_k2_16x16", 2, 16, 2),
    "3d_p3_k3_64": Workload("3d_p3_k3_64", 3, 64, 3),
    "3d_design_k2_48": Workload("3d_design_k2_48", 3, 48, 2),
    "3d_p3_k2_16": Workload("3d_p3_k2_16", 3, 16, 2),
}

# Order sweep at about 8M DOFs: n chosen so that k*n is about 200.
SWEEP_N = {1: 199, 2: 100, 3: 66, 4: 50, 5: 40, 6: 33}


def sweep_workload(order: int) -> Workload:
    return Workload(f"3d_p3_k{order}_{SWEEP_N[order]}", 3, SWEEP_N[order], order)


def batched_instances(count: int = 64, seed: int = 5, n_range=(8, 40), orders=(1, 2, 3, 4),
                      p_range=(2.5, 4.0)) -> list[Workload]:
    """Independent instances of uneven size and order: p ~ U[2.5,4], n ~ U{8..40}, k ~ U{1..4}."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        p = float(rng.uniform(*p_range))
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        k = int(rng.choice(orders))
        out.append(Workload(f"batch{i}_n{n}_k{k}", 3, n, k, p=p, mesh_seed=seed * 1000 + i,
                            state_seed=seed * 1000 + 100 + i))
    return out
