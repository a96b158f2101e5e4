"""One problem split across ranks: the subdomain restriction P of the operator decomposition
A = P^T G^T B^T D B G P (Fig. 1), with P no longer the identity.

Partition.  The lattice of n x n x nz elements is cut along z into one slab of element layers per
rank (balanced to within one layer).  Rank r sets up its slab as a lattice of n x n x (z1 - z0)
elements with its own copy of the slab's vertices; the slab's faces towards its neighbours are
natural (not essential), the others keep the problem's Dirichlet convention.  The slab's DOFs are
the global DOF planes k z0 .. k z1, a contiguous range of the global vector, so a rank's local
vector is a slice of the global one and the two interface planes are its first and last
(k n + 1)^2 entries.

Operator.  Each local application (residual, Jacobian action, Jacobi diagonal) leaves partial sums
on the interface planes; P^T completes them with ONE exchange: every rank sends its two interface
planes to its neighbours and adds what it receives to its own non-essential interface DOFs
(fe_face_add).  Both ranks then hold the same, complete values (a + b = b + a in floating point).

Inner products.  A DOF plane shared by ranks r and r+1 counts once, for rank r: rank r > 0 sums
its local vector without its first plane.  The local sums are added over ranks by an all-reduce;
the Jacobi-preconditioned CG does two per iteration (p.Jp, then r.z and r.r together), the Newton
iteration one per residual norm.

Every local operation runs in the CUDA library (``LibraryBackend``); the algorithms here only
sequence the calls, the exchanges and the reductions.  ``TorchComm`` moves planes and scalars with
torch.distributed: NCCL on device tensors, or gloo through host copies.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

FACE_ZLO, FACE_ZHI = 4, 5

__all__ = ["SlabPartition", "TorchComm", "LibraryBackend", "SlabSolver", "FACE_ZLO", "FACE_ZHI"]


@dataclasses.dataclass(frozen=True)
class SlabPartition:
    """z-slabs of a lattice of n x n x nz elements (nz = n when not given), order k, over `world`
    ranks."""
    n: int
    order: int
    world: int
    nz: int = 0

    def __post_init__(self):
        if self.nz == 0:
            object.__setattr__(self, "nz", self.n)
        if self.world < 1 or self.world > self.nz:
            raise ValueError("need 1 <= world <= nz (at least one element layer per rank)")

    def layers(self, rank: int) -> tuple[int, int]:
        """Element layers [z0, z1) of `rank`: the first nz % world ranks take one layer more."""
        q, rem = divmod(self.nz, self.world)
        z0 = rank * q + min(rank, rem)
        return z0, z0 + q + (1 if rank < rem else 0)

    def elements(self, rank: int) -> tuple[int, int, int]:
        z0, z1 = self.layers(rank)
        return self.n, self.n, z1 - z0

    def natural_faces(self, rank: int) -> int:
        return (1 << FACE_ZLO if rank > 0 else 0) | (1 << FACE_ZHI if rank < self.world - 1 else 0)

    @property
    def plane(self) -> int:
        """DOFs of one z-plane of the lattice."""
        return (self.order * self.n + 1) ** 2

    @property
    def n_dofs(self) -> int:
        return self.plane * (self.order * self.nz + 1)

    def dof_range(self, rank: int) -> tuple[int, int]:
        """The slab's DOFs as the global range [g0, g1): planes k z0 .. k z1."""
        z0, z1 = self.layers(rank)
        return self.order * z0 * self.plane, (self.order * z1 + 1) * self.plane

    def owned(self, rank: int) -> tuple[int, int]:
        """Local index range whose entries this rank counts in inner products."""
        g0, g1 = self.dof_range(rank)
        return (self.plane if rank > 0 else 0), g1 - g0

    def vertex_range(self, rank: int) -> tuple[int, int]:
        """The slab's vertices as rows [v0, v1) of the lattice's vertex array (z-planes z0 .. z1)."""
        z0, z1 = self.layers(rank)
        nv2 = (self.n + 1) ** 2
        return z0 * nv2, (z1 + 1) * nv2


class TorchComm:
    """Neighbour exchange of interface planes and sums over ranks with torch.distributed.

    ``staging``: move tensors through host memory (gloo); otherwise they travel as they are
    (NCCL, device tensors)."""

    def __init__(self, rank: int, world: int, staging: bool):
        self.rank, self.world, self.staging = rank, world, staging

    def exchange(self, lo_send, hi_send):
        """Send lo_send to rank - 1 and hi_send to rank + 1; return what they sent back (None at
        the ends), as tensors on lo_send's device (host arrays come back as host arrays)."""
        import torch
        import torch.distributed as dist
        if self.world == 1:
            return None, None
        if isinstance(lo_send, np.ndarray):
            lo, hi = self.exchange(torch.from_numpy(np.array(lo_send)), torch.from_numpy(np.array(hi_send)))
            return (None if lo is None else lo.numpy()), (None if hi is None else hi.numpy())
        stage = (lambda t: t.detach().cpu()) if self.staging else (lambda t: t.detach().contiguous())
        ops, lo_recv, hi_recv = [], None, None
        if self.rank > 0:
            snd = stage(lo_send)
            lo_recv = torch.empty_like(snd)
            ops += [dist.P2POp(dist.isend, snd, self.rank - 1), dist.P2POp(dist.irecv, lo_recv, self.rank - 1)]
        if self.rank < self.world - 1:
            snd = stage(hi_send)
            hi_recv = torch.empty_like(snd)
            ops += [dist.P2POp(dist.isend, snd, self.rank + 1), dist.P2POp(dist.irecv, hi_recv, self.rank + 1)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        dev = lo_send.device
        return (None if lo_recv is None else lo_recv.to(dev)), (None if hi_recv is None else hi_recv.to(dev))

    def allreduce(self, values):
        """Sums over ranks of a short list of floats."""
        import torch
        import torch.distributed as dist
        if self.world == 1:
            return [float(v) for v in values]
        dev = "cpu" if self.staging else "cuda"
        t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
        dist.all_reduce(t)
        return [float(x) for x in t.cpu().tolist()]


class LibraryBackend:
    """A rank's local operations on its slab context, each one a call into the CUDA library."""

    def __init__(self, op):
        import torch
        from . import abi
        self.op, self.abi = op, abi
        self._s = torch.empty(1, dtype=torch.float64, device=op.device)

    def zeros(self):
        import torch
        return torch.zeros(self.op.n_dofs, dtype=torch.float64, device=self.op.device)

    def residual(self, u, out):
        self.op.residual(u, out=out)

    def linearize(self, u):
        self.op.linearize(u)

    def jv(self, v, out, precision: int = 64):
        self.op.jacobian_action(v, precision=precision, out=out)

    def diag(self, out):
        self.abi.fe_jacobian_diagonal(self.op.ctx, out)

    def dot(self, a, b, begin: int, end: int) -> float:
        self.abi.fe_dot(self.op.ctx, a, b, begin, end, self._s)
        return float(self._s.item())

    def axpby(self, alpha: float, x, beta: float, y):
        self.abi.fe_axpby(self.op.ctx, alpha, x, beta, y)

    def mul(self, d, r, z):
        self.abi.fe_pointwise_mul(self.op.ctx, d, r, z)

    def recip(self, x, y):
        self.abi.fe_reciprocal(self.op.ctx, x, y)

    def face_add(self, face: int, y, buf):
        self.abi.fe_face_add(self.op.ctx, face, y, buf)


class SlabSolver:
    """The split operator and its solvers on one rank: local calls through `backend`, interface
    exchanges and sums over ranks through `comm`."""

    def __init__(self, part: SlabPartition, rank: int, backend, comm):
        self.part, self.rank, self.be, self.comm = part, rank, backend, comm
        self.own = part.owned(rank)
        self.exchanges = 0
        self.allreduces = 0

    # -- P^T across the interfaces ----------------------------------------------------------
    def assemble(self, y):
        """Add the neighbours' partial sums to this rank's interface planes (one exchange)."""
        pl = self.part.plane
        lo, hi = self.comm.exchange(y[:pl], y[-pl:])
        self.exchanges += 1
        if lo is not None:
            self.be.face_add(FACE_ZLO, y, lo)
        if hi is not None:
            self.be.face_add(FACE_ZHI, y, hi)

    def sums(self, pairs):
        """Global inner products of (a, b) pairs: owned local sums, one all-reduce."""
        self.allreduces += 1
        return self.comm.allreduce([self.be.dot(a, b, *self.own) for a, b in pairs])

    # -- operators ----------------------------------------------------------------------------
    def residual(self, u, out):
        self.be.residual(u, out)
        self.assemble(out)

    def jv(self, v, out, precision: int = 64):
        self.be.jv(v, out, precision)
        self.assemble(out)

    def jacobi(self, out):
        """1 / diag(J) of the current linearisation, assembled across the interfaces."""
        self.be.diag(out)
        self.assemble(out)
        self.be.recip(out, out)

    # -- Jacobi-preconditioned CG on the split operator ----------------------------------------
    def cg(self, b, x, dinv, rtol: float, max_iter: int, precision: int = 64, work=None):
        """J x = b from x = 0 until ||r|| <= rtol ||b||; returns (iterations, status) with status
        'converged', 'max_iter' or 'breakdown'.  b, x, dinv: consistent local vectors."""
        r, z, p, q = work if work is not None else [self.be.zeros() for _ in range(4)]
        be = self.be
        be.axpby(0.0, b, 0.0, x)                      # x = 0
        be.axpby(1.0, b, 0.0, r)                      # r = b
        be.mul(dinv, r, z)
        be.axpby(1.0, z, 0.0, p)
        rz, rr = self.sums([(r, z), (r, r)])
        tol2 = rtol * rtol * rr
        if rr == 0.0 or rr <= tol2:
            return 0, "converged"
        for it in range(1, max_iter + 1):
            self.jv(p, q, precision)
            (pq,) = self.sums([(p, q)])
            if not (pq > 0.0) or not math.isfinite(pq):
                return it, "breakdown"
            alpha = rz / pq
            be.axpby(alpha, p, 1.0, x)
            be.axpby(-alpha, q, 1.0, r)
            be.mul(dinv, r, z)
            rz_new, rr = self.sums([(r, z), (r, r)])
            if rr <= tol2:
                return it, "converged"
            be.axpby(1.0, z, rz_new / rz, p)          # p = z + beta p
            rz = rz_new
        return max_iter, "max_iter"

    # -- Newton-CG with backtracking on ||R|| ---------------------------------------------------
    def newton(self, u, rtol: float = 1e-8, cg_rtol: float = 1e-4, max_newton: int = 50, max_cg: int = 20000,
               armijo: float = 1e-4, max_halvings: int = 20, precision: int = 64) -> dict:
        """Solve R(u) = 0 from u (consistent local vector, overwritten): the algorithm of the
        library's newton_solve with the split operator.  Returns a report."""
        be = self.be
        R, d, trial, Rt, dinv, b = [be.zeros() for _ in range(6)]
        work = [be.zeros() for _ in range(4)]
        self.residual(u, R)
        (rr,) = self.sums([(R, R)])
        r0 = math.sqrt(rr)
        hist, cg_total, status = [r0], 0, "converged"
        rn = r0
        for _ in range(max_newton):
            if rn <= rtol * r0 or r0 == 0.0:
                break
            be.linearize(u)
            self.jacobi(dinv)
            be.axpby(-1.0, R, 0.0, b)
            its, st = self.cg(b, d, dinv, cg_rtol, max_cg, precision, work)
            cg_total += its
            if st == "breakdown":
                status = "breakdown"
                break
            alpha, accepted = 1.0, False
            for _h in range(max_halvings + 1):
                be.axpby(1.0, u, 0.0, trial)
                be.axpby(alpha, d, 1.0, trial)
                self.residual(trial, Rt)
                (tt,) = self.sums([(Rt, Rt)])
                nt = math.sqrt(tt)
                if nt <= (1.0 - armijo * alpha) * rn:
                    accepted = True
                    break
                alpha *= 0.5
            if not accepted:
                status = "line_search_failed"
                break
            be.axpby(1.0, trial, 0.0, u)
            R, Rt = Rt, R
            rn = nt
            hist.append(rn)
        else:
            if rn > rtol * r0:
                status = "max_newton"
        return {"status": status, "newton_iters": len(hist) - 1, "cg_iters": cg_total, "r0": r0, "r_final": rn,
                "rel": rn / r0 if r0 > 0 else 0.0, "history": hist, "exchanges": self.exchanges,
                "allreduces": self.allreduces}
