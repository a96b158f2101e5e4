"""The subdomain split on the GPU library: two ranks, each a process with its own slab context on
the same GPU, exchanging interface planes and inner products through gloo (host copies; no
kernel of one rank waits on the other's).  The split Jacobian action and residual must equal the
oracle's whole-domain ones, and the split Newton-CG solve (FP64 and mixed precision) must satisfy
the oracle's residual check on the gathered solution."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_2506_00746_gb300 import dist as D
from paper_2506_00746_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _worker(rank, world, port, n, k, out_dir):
    import torch
    import torch.distributed as dist

    from paper_2506_00746_gb300 import Operator
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        V = I.lattice_vertices(3, n, seed=0)
        part = D.SlabPartition(n, k, world)
        v0, v1 = part.vertex_range(rank)
        op = Operator(3, part.elements(rank), k, V[v0:v1], p=3.0, natural_faces=part.natural_faces(rank))
        be = D.LibraryBackend(op)
        solver = D.SlabSolver(part, rank, be, D.TorchComm(rank, world, staging=True))
        g0, g1 = part.dof_range(rank)
        u0 = torch.from_numpy(I.smooth_field(3, n, k, seed=1)[g0:g1].copy()).cuda()
        v = torch.from_numpy(I.uniform_vector((k * n + 1) ** 3, seed=2)[g0:g1].copy()).cuda()
        be.linearize(u0)
        y, y32, r = be.zeros(), be.zeros(), be.zeros()
        solver.jv(v, y, 64)
        solver.jv(v, y32, -32)
        solver.residual(u0, r)
        out = {"y": y.cpu().numpy(), "y32": y32.cpu().numpy(), "r": r.cpu().numpy()}
        for prec in (64, -32):
            u = u0.clone()
            rep = solver.newton(u, rtol=1e-8, precision=prec)
            out[f"u{prec}"] = u.cpu().numpy()
            out[f"rel{prec}"] = rep["rel"]
            out[f"status{prec}"] = rep["status"]
        op.close()
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), **out)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world,n,k", [(2, 8, 3), (3, 7, 2)])
def test_split_library_operator_and_newton(world, n, k, tmp_path):
    import torch.multiprocessing as mp
    mp.start_processes(_worker, args=(world, _free_port(), n, k, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    V = I.lattice_vertices(3, n, seed=0)
    P = O.Problem(3, n, k, V, p=3.0)
    part = D.SlabPartition(n, k, world)
    u0 = I.smooth_field(3, n, k, seed=1)
    v = I.uniform_vector(P.n_dofs, seed=2)
    y_ref, r_ref = O.jv(P, u0, v), O.residual(P, u0)
    y32_ref = O.jv(P, u0, v.astype(np.float32).astype(np.float64))
    res = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    gathered = {key: np.zeros(P.n_dofs) for key in ("y", "y32", "r", "u64", "u-32")}
    for rank, d in enumerate(res):
        g0, g1 = part.dof_range(rank)
        for key in gathered:
            if rank > 0:        # ranks agree bit for bit on the plane they share
                np.testing.assert_array_equal(gathered[key][g0:g0 + part.plane], d[key][:part.plane])
            gathered[key][g0:g1] = d[key]
        assert str(d["status64"]) == "converged" and float(d["rel64"]) <= 1e-8
        assert str(d["status-32"]) == "converged" and float(d["rel-32"]) <= 1e-8
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(gathered["y"], y_ref) <= 1e-12
    assert rel(gathered["r"], r_ref) <= 1e-12
    assert rel(gathered["y32"], y32_ref) <= 1e-5
    r0 = np.linalg.norm(r_ref)
    for key in ("u64", "u-32"):
        assert np.linalg.norm(O.residual(P, gathered[key])) <= 1e-8 * r0 * 1.01, key
