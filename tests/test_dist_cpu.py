"""The subdomain split (paper_2506_00746_gb300.dist) on CPU: two gloo ranks, each holding one
z-slab of a cube problem, with the oracle's element sums over the slab's elements as the local
operator.  Checks that the partition, the single interface exchange per operator application and
the sums over ranks reproduce the single-domain results: the split Jacobian action, residual and
inner products against the oracle's whole-domain ones, and the split Newton-CG solve against the
oracle's residual of the gathered solution."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_2506_00746_gb300 import dist as D
from paper_2506_00746_gb300 import inputs as I


class OracleSlab:
    """Test-only local operations of one slab: the oracle's sums over the slab's elements of the
    cube problem, with the Dirichlet convention on the cube's boundary DOFs inside the slab."""

    def __init__(self, P, part, rank):
        self.P, self.part = P, part
        self.g0, self.g1 = part.dof_range(rank)
        z0, z1 = part.layers(rank)
        self.e0, self.e1 = z0 * part.n ** 2, z1 * part.n ** 2
        self.ess_g = O.essential(P)
        self.ess = self.ess_g[self.g0:self.g1]
        self.ulin = None

    def _glob(self, x):
        g = np.zeros(self.P.n_dofs)
        g[self.g0:self.g1] = x
        return g

    def zeros(self):
        return np.zeros(self.g1 - self.g0)

    def residual(self, u, out):
        r = O.residual_partial(self.P, self._glob(u), self.e0, self.e1)
        out[:] = np.where(self.ess, 0.0, r[self.g0:self.g1])

    def linearize(self, u):
        self.ulin = np.array(u)

    def jv(self, v, out, precision=64):
        vg = self._glob(v)
        vg[self.ess_g] = 0.0
        y = O.jv_partial(self.P, self._glob(self.ulin), vg, self.e0, self.e1)
        out[:] = np.where(self.ess, v, y[self.g0:self.g1])

    def diag(self, out):
        K, _, dofs = O.element_matrices(self.P, self._glob(self.ulin), self.e0, self.e1)
        d = np.zeros(self.P.n_dofs)
        np.add.at(d, dofs.ravel(), np.einsum("eii->ei", K).ravel())
        out[:] = np.where(self.ess, 1.0, d[self.g0:self.g1])

    def dot(self, a, b, begin, end):
        return float(a[begin:end] @ b[begin:end])

    def axpby(self, alpha, x, beta, y):
        y[:] = alpha * x if beta == 0.0 else alpha * x + beta * y

    def mul(self, d, r, z):
        z[:] = d * r

    def recip(self, x, y):
        y[:] = 1.0 / x

    def face_add(self, face, y, buf):
        pl = self.part.plane
        sl = slice(0, pl) if face == D.FACE_ZLO else slice(len(y) - pl, len(y))
        free = ~self.ess[sl]
        y[sl] = np.where(free, y[sl] + buf, y[sl])


def _worker(rank, world, port, n, k, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        V = I.lattice_vertices(3, n, seed=0)
        P = O.Problem(3, n, k, V, p=3.0)
        part = D.SlabPartition(n, k, world)
        be = OracleSlab(P, part, rank)
        solver = D.SlabSolver(part, rank, be, D.TorchComm(rank, world, staging=True))
        g0, g1 = part.dof_range(rank)
        u0 = I.smooth_field(3, n, k, seed=1)
        v = I.uniform_vector(P.n_dofs, seed=2)
        ul, vl = u0[g0:g1].copy(), v[g0:g1].copy()
        be.linearize(ul)
        y = be.zeros()
        solver.jv(vl, y)
        r = be.zeros()
        solver.residual(ul, r)
        (vv,) = solver.sums([(vl, vl)])
        u = ul.copy()
        rep = solver.newton(u, rtol=1e-10, cg_rtol=1e-4)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), y=y, r=r, u=u, vv=vv, rel=rep["rel"],
                 newton=rep["newton_iters"], cg=rep["cg_iters"], exchanges=rep["exchanges"],
                 allreduces=rep["allreduces"], status=rep["status"])
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world,n,k", [(2, 6, 2), (3, 5, 1)])
def test_split_operator_and_newton_match_single_domain(world, n, k, tmp_path):
    import torch.multiprocessing as mp
    mp.start_processes(_worker, args=(world, _free_port(), n, k, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    V = I.lattice_vertices(3, n, seed=0)
    P = O.Problem(3, n, k, V, p=3.0)
    part = D.SlabPartition(n, k, world)
    u0 = I.smooth_field(3, n, k, seed=1)
    v = I.uniform_vector(P.n_dofs, seed=2)
    res = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    y_ref, r_ref = O.jv(P, u0, v), O.residual(P, u0)
    for rank, d in enumerate(res):
        g0, g1 = part.dof_range(rank)
        # every rank's slice, interface planes included, equals the single-domain result
        np.testing.assert_allclose(d["y"], y_ref[g0:g1], rtol=0, atol=1e-13 * np.abs(y_ref).max())
        np.testing.assert_allclose(d["r"], r_ref[g0:g1], rtol=0, atol=1e-13 * np.abs(r_ref).max())
        assert abs(float(d["vv"]) - v @ v) <= 1e-13 * (v @ v)
        assert str(d["status"]) == "converged" and float(d["rel"]) <= 1e-10
    # the split Newton: all ranks agree on the shared planes, and the oracle's residual of the
    # gathered solution confirms the 1e-10 convergence
    u = np.zeros(P.n_dofs)
    for rank, d in enumerate(res):
        g0, g1 = part.dof_range(rank)
        if rank > 0:
            np.testing.assert_array_equal(u[g0:g0 + part.plane], d["u"][:part.plane])
        u[g0:g1] = d["u"]
    assert np.linalg.norm(O.residual(P, u)) <= 1e-10 * np.linalg.norm(r_ref) * 1.01
    # one exchange per operator application, two all-reduces per CG iteration
    cg, newton = int(res[0]["cg"]), int(res[0]["newton"])
    assert all(int(d["cg"]) == cg and int(d["newton"]) == newton for d in res)
    assert int(res[0]["allreduces"]) >= 2 * cg


def test_partition_covers_the_cube():
    for n, k, world in ((6, 2, 2), (7, 3, 3), (5, 1, 5), (8, 2, 1)):
        part = D.SlabPartition(n, k, world)
        layers = [part.layers(r) for r in range(world)]
        assert layers[0][0] == 0 and layers[-1][1] == n
        assert all(layers[r][1] == layers[r + 1][0] for r in range(world - 1))
        assert max(b - a for a, b in layers) - min(b - a for a, b in layers) <= 1
        # consecutive slabs share exactly one DOF plane; owned ranges tile the global vector
        owned = 0
        for r in range(world):
            g0, g1 = part.dof_range(r)
            b, e = part.owned(r)
            owned += e - b
            if r > 0:
                assert part.dof_range(r - 1)[1] - g0 == part.plane
        assert owned == part.n_dofs
        assert part.natural_faces(0) == (0 if world == 1 else 32)
    with pytest.raises(ValueError):
        D.SlabPartition(3, 2, 4)
