"""GB300-native matrix-free finite element operator decomposition with quadrature-point AD.

The operator A = P^T G^T B^T D B G P of the steady p-Laplacian (Fig. 1, Eq. 1), its exact
Jacobian J(u) = P^T G^T B^T J_D(u_q) B G P with J_D from forward-mode dual numbers (Eq. 2), a
matrix-free Newton-CG solve and the adjoint design gradient all run in the CUDA library
``libfeod.so`` (include/feod.h).  This package is its thin binding: ``abi`` has the C entry
points under their own names, ``Operator`` wraps one context with torch tensors for device memory
and streams, ``ComplianceFn`` exposes the design gradient to torch autograd.
"""
from __future__ import annotations

import numpy as np

from . import abi, inputs
from .abi import FeodError

__all__ = ["Operator", "Batch", "ComplianceFn", "FeodError", "abi", "inputs", "build_library"]


def build_library(force: bool = False, verbose: bool = False) -> str:
    from .build import build
    return build(force=force, verbose=verbose)


class Operator:
    """One problem instance on one GPU (a ``fe_ctx``).

    ``n``: elements per direction, an int (a cube lattice) or a sequence of ``dim`` counts.
    ``vertices``: host array [prod(n_d + 1), dim] (x fastest).  ``rho``: optional per-element design
    field (host array, element order ex fastest), which makes the flux kappa_rho(rho_e) times the
    p-Laplacian flux with kappa_rho = kappa_eps + rho^kappa_q.  ``natural_faces``: mask of the box
    faces whose DOFs are not essential (bits x-, x+, y-, y+, z-, z+), the interfaces of a
    subdomain.
    """

    def __init__(self, dim: int, n, order: int, vertices, p: float = 3.0, eps: float = 0.0,
                 f_kind: int = 0, f_const: float = 1.0, rho=None, kappa_eps: float = 1e-3,
                 kappa_q: float = 3.0, q1d: int = 0, tile: int = 0, tile_kernel: bool = True,
                 natural_faces: int = 0):
        import ctypes

        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Operator needs a CUDA device: the library has no CPU path")
        self._vert = np.ascontiguousarray(vertices, dtype=np.float64)
        self._rho = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
        mesh = abi.make_mesh(dim, n, self._vert.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), natural_faces)
        prob = abi.fe_problem(p, eps, f_kind, f_const,
                              None if self._rho is None else self._rho.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                              kappa_eps, kappa_q)
        opts = abi.fe_setup_opts(tile, 0 if tile_kernel else 1) if (tile or not tile_kernel) else None
        self.ctx = abi.fe_setup(mesh, order, q1d, prob, opts)
        self.dim, self.n, self.order, self.p = dim, n, order, p
        self.n_dofs, self.n_free = abi.fe_num_dofs(self.ctx)
        self.n_elements = abi.fe_num_elements(self.ctx)
        self.device = torch.device("cuda", torch.cuda.current_device())

    # -- helpers ----------------------------------------------------------------------------
    def _vec(self, dtype=None, n=None):
        import torch
        return torch.empty(self.n_dofs if n is None else n, dtype=dtype or torch.float64, device=self.device)

    def _chk(self, t, dtype, n=None, name="vector"):
        import torch
        n = self.n_dofs if n is None else n
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()
                and t.numel() == n):
            raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor of {n} entries")
        return t

    # -- operators --------------------------------------------------------------------------
    def residual(self, u, out=None, stream=None):
        import torch
        self._chk(u, torch.float64, name="u")
        r = out if out is not None else self._vec()
        abi.fe_residual(self.ctx, u, r, stream)
        return r

    def linearize(self, u, stream=None):
        import torch
        abi.fe_linearize(self.ctx, self._chk(u, torch.float64, name="u"), stream)

    def jacobian_action(self, v, u=None, precision: int = 64, out=None, stream=None):
        """J(u) v: cached linearisation when u is None, else stateless (dual seeded by grad v).

        precision 64 (double v/y), 48 (double v/y, double-float arithmetic: FP32 word pairs on
        the FP32 pipes, about 48 significant bits; cached linearisation only), 32 (float v/y, FP32
        arithmetic) or -32 (double v/y, FP32 arithmetic)."""
        import torch
        io = torch.float32 if precision == 32 else torch.float64
        self._chk(v, io, name="v")
        if u is not None:
            self._chk(u, torch.float64, name="u")
        y = out if out is not None else self._vec(io)
        abi.fe_jacobian_action(self.ctx, u, v, y, precision, stream)
        return y

    def jacobian_action_host(self, v_host, y_host, precision: int = 32, stream=None):
        abi.fe_jacobian_action_host(self.ctx, v_host, y_host, precision, stream)
        return y_host

    def jacobian_diagonal(self, stream=None):
        d = self._vec()
        abi.fe_jacobian_diagonal(self.ctx, d, stream)
        return d

    def load_vector(self, stream=None):
        F = self._vec()
        abi.fe_load_vector(self.ctx, F, stream)
        return F

    def node_coords(self, stream=None):
        import torch
        xyz = torch.empty((self.n_dofs, self.dim), dtype=torch.float64, device=self.device)
        abi.fe_node_coords(self.ctx, xyz, stream)
        return xyz

    def set_design(self, rho, stream=None):
        import torch
        abi.fe_set_design(self.ctx, self._chk(rho, torch.float64, self.n_elements, "rho"), stream)

    def adjoint_vjp(self, u, lam, stream=None):
        import torch
        g = self._vec(n=self.n_elements)
        abi.fe_adjoint_vjp(self.ctx, self._chk(u, torch.float64, name="u"),
                           self._chk(lam, torch.float64, name="lambda"), g, stream)
        return g

    def element_matrices(self, u, method: str = "res", e0: int = 0, count: int | None = None, stream=None):
        """Dense element tangents K_e (Eq. 3) of elements [e0, e0 + count): method "hnd" (hand-coded
        tangent), "res" (AD at the quadrature point) or "elm" (AD at the element level)."""
        import torch
        count = self.n_elements - e0 if count is None else count
        nl = (self.order + 1) ** self.dim
        K = torch.empty((count, nl, nl), dtype=torch.float64, device=self.device)
        abi.fe_element_matrices(self.ctx, self._chk(u, torch.float64, name="u"), {"hnd": 0, "res": 1, "elm": 2}[method],
                                e0, count, K, stream)
        return K

    # -- solvers ----------------------------------------------------------------------------
    def newton_solve(self, u, rtol: float = 1e-8, inner_precision: int = 64, cg_rtol: float = 1e-4,
                     max_newton: int = 50, max_cg: int = 20000, line_search: bool = True,
                     cg_batch: int = 16, use_graph: int = 2, forcing: int = 0, eta_max: float = 0.1,
                     raise_on_error: bool = True, stream=None):
        """Solve R(u) = 0 in place from u (Newton-CG, Jacobi-preconditioned, backtracking line search);
        returns a dict report.  inner_precision: 64 (FP64 CG), 48 (double-float J v inside an FP64
        CG), -32 (FP32 J v inside an FP64 CG) or 32 (FP32 J v and FP32 CG vectors with compensated
        inner products); the residual, norms, Newton update and line search are FP64 in every
        mode.  forcing 0: every CG to cg_rtol; 1: Eisenstat-Walker choice 2 forcing terms, at most
        eta_max."""
        import torch
        self._chk(u, torch.float64, name="u")
        o = abi.fe_newton_default_opts()
        o.forcing, o.eta_max = int(forcing), float(eta_max)
        o.rtol, o.inner_precision, o.cg_rtol = rtol, inner_precision, cg_rtol
        o.max_newton, o.max_cg, o.line_search = max_newton, max_cg, int(line_search)
        o.cg_batch, o.use_graph = cg_batch, int(use_graph)      # 0 plain, 1 graph batches, 2 device loop
        rep = abi.newton_solve(self.ctx, u, o, stream)
        out = {"status": abi.STATUS_NAMES.get(rep.status, rep.status), "newton_iters": rep.newton_iters,
               "cg_iters": rep.cg_iters_total, "halvings": rep.line_search_halvings, "r0": rep.r0,
               "r_final": rep.r_final, "rel": rep.r_final / rep.r0 if rep.r0 > 0 else 0.0,
               "time_ms": rep.t_total_ms, "cg_ms": rep.t_cg_ms, "launches": rep.kernel_launches,
               "r_hist": list(rep.r_hist[:min(rep.newton_iters, abi.FE_NEWTON_HIST)]),
               "cg_hist": list(rep.cg_hist[:min(rep.newton_iters, abi.FE_NEWTON_HIST)])}
        if rep.status != abi.FE_OK:
            out["error"] = getattr(rep, "error", "")
            if raise_on_error:
                raise FeodError(rep.status, "newton_solve", out["error"])
        return out

    def cg_solve(self, b, rtol: float = 1e-10, max_iter: int = 50000, precision: int = 64, stream=None):
        """Solve J x = b with the cached linearisation (x from 0); returns (x, iterations).
        precision as newton_solve's inner_precision."""
        import torch
        x = self._vec()
        it = abi.fe_cg_solve(self.ctx, self._chk(b, torch.float64, name="b"), x, rtol, max_iter, precision, stream)
        return x, it

    # -- profiling --------------------------------------------------------------------------
    def prof_enable(self, on: bool = True):
        abi.fe_prof_enable(self.ctx, on)

    def prof_reset(self):
        abi.fe_prof_reset(self.ctx)

    def prof_read(self) -> dict:
        return abi.fe_prof_read(self.ctx)

    def launch_count(self) -> int:
        return abi.fe_launch_count(self.ctx)

    def memory_bytes(self) -> int:
        return abi.fe_memory_bytes(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            abi.fe_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent 3D instances of order 1..4 in one persistent launch (a ``fe_batch``).

    ``instances``: list of dicts with keys ``vertices`` (host [(n+1)^3, 3]), ``n``, ``order`` and
    optionally ``p`` (3.0), ``eps`` (0.0), ``f_kind`` (0), ``f_const`` (1.0).  Batch vectors are
    the instances' vectors concatenated at ``offsets`` (see ``split``/``concat``).  ``tune``:
    autotune tile edges and launch shape (cached in ``tune_cache``); ``policy``: work policy (-1
    tuned; 0 by instance, 1 interleaved, 2 largest first, each in one persistent launch; 3 one
    launch per tile variant); ``tiles``: per order 1..4 a fixed tile edge (0 = tuned).
    """

    def __init__(self, instances, tune: bool = True, tune_cache: str | None = None, retune: bool = False,
                 policy: int = -1, tiles=None):
        import ctypes

        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Batch needs a CUDA device: the library has no CPU path")
        self.count = len(instances)
        self._keep = []
        items = (abi.fe_batch_item * self.count)()
        for i, d in enumerate(instances):
            vert = np.ascontiguousarray(d["vertices"], dtype=np.float64)
            mesh = abi.make_mesh(3, int(d["n"]), vert.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
            prob = abi.fe_problem(float(d.get("p", 3.0)), float(d.get("eps", 0.0)), int(d.get("f_kind", 0)),
                                  float(d.get("f_const", 1.0)), None, 1e-3, 3.0)
            self._keep += [vert, mesh, prob]
            items[i].mesh = ctypes.pointer(mesh)
            items[i].order = int(d["order"])
            items[i].prob = ctypes.pointer(prob)
        opts = abi.fe_batch_opts()
        self._cache = tune_cache.encode() if tune_cache else None
        opts.tune_cache = self._cache
        opts.tune, opts.retune, opts.policy = int(bool(tune)), int(bool(retune)), int(policy)
        for k in range(4):
            opts.tile[k] = int(tiles[k]) if tiles else 0
        self.batch = abi.fe_batch_create(items, self.count, opts)
        info = [abi.fe_batch_info(self.batch, i) for i in range(self.count)]
        self.offsets = [o for o, _, _ in info]
        self.n_dofs = [n for _, n, _ in info]
        self.tiles = [t for _, _, t in info]
        self.orders = [int(d["order"]) for d in instances]
        self.total = abi.fe_batch_shape(self.batch)["total"]
        self.device = torch.device("cuda", torch.cuda.current_device())

    def shape(self) -> dict:
        return abi.fe_batch_shape(self.batch)

    def vector(self, dtype=None):
        import torch
        return torch.zeros(self.total, dtype=dtype or torch.float64, device=self.device)

    def split(self, vec) -> list:
        return [vec[o:o + n] for o, n in zip(self.offsets, self.n_dofs)]

    def concat(self, parts, dtype=None):
        import torch
        v = self.vector(dtype)
        for o, n, x in zip(self.offsets, self.n_dofs, parts):
            v[o:o + n] = torch.as_tensor(x, dtype=v.dtype).to(self.device)
        return v

    def _chk(self, t, dtype, name):
        import torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()
                and t.numel() == self.total):
            raise ValueError(f"{name} must be a contiguous CUDA {dtype} batch vector of {self.total} entries")
        return t

    def linearize(self, u, stream=None):
        import torch
        abi.fe_batch_linearize(self.batch, self._chk(u, torch.float64, "u"), stream)

    def jacobian_action(self, v, out=None, stream=None):
        import torch
        y = out if out is not None else self.vector(torch.float32)
        abi.fe_batch_jacobian_action(self.batch, self._chk(v, torch.float32, "v"), self._chk(y, torch.float32, "y"),
                                     stream)
        return y

    def newton_solve(self, u, rtol: float = 1e-8, cg_rtol: float = 1e-4, max_newton: int = 50,
                     max_cg: int = 20000, cg_batch: int = 16, use_graph: int = 2, line_search: bool = True,
                     raise_on_error: bool = True, stream=None):
        """Newton on every instance in lock step (FP32 CG, FP64 outer); returns (reports, total)."""
        import torch
        self._chk(u, torch.float64, "u")
        o = abi.fe_newton_default_opts()
        o.rtol, o.cg_rtol, o.max_newton, o.max_cg = rtol, cg_rtol, max_newton, max_cg
        o.cg_batch, o.use_graph, o.line_search, o.inner_precision = cg_batch, int(use_graph), int(line_search), 32
        reps, tot, err = abi.fe_batch_newton_solve(self.batch, u, self.count, o, stream)
        conv = lambda r: {"status": abi.STATUS_NAMES.get(r.status, r.status), "newton_iters": r.newton_iters,
                          "cg_iters": r.cg_iters_total, "r0": r.r0, "r_final": r.r_final,
                          "rel": r.r_final / r.r0 if r.r0 > 0 else 0.0, "halvings": r.line_search_halvings}
        total = conv(tot)
        total.update({"time_ms": tot.t_total_ms, "cg_ms": tot.t_cg_ms, "launches": tot.kernel_launches})
        if tot.status != abi.FE_OK:
            total["error"] = err
            if raise_on_error:
                raise FeodError(tot.status, "fe_batch_newton_solve", err)
        return [conv(r) for r in reps], total

    def close(self):
        if getattr(self, "batch", None):
            abi.fe_batch_destroy(self.batch)
            self.batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _compliance_autograd():
    import torch

    class ComplianceFn(torch.autograd.Function):
        """c(rho) = F^T u(rho) with R(u; rho) = 0, differentiable in rho by the adjoint method.

        forward: Newton solve from ``u0`` (the converged state is checkpointed, not the Newton
        history), then fe_compliance; backward: fe_compliance_gradient at the checkpointed state
        (adjoint CG J(u) lambda = F, then dc/drho = -lambda^T dR/drho from the quadrature-point
        dual-number VJP kernel), scaled by the incoming gradient.
        """

        @staticmethod
        def forward(ctx, rho, op: "Operator", u0, newton_kw: dict | None = None):
            op.set_design(rho.detach().contiguous())
            u = u0.detach().clone()
            op.newton_solve(u, **(newton_kw or {}))
            c = torch.empty((), dtype=torch.float64, device=op.device)
            abi.fe_compliance(op.ctx, u, c)
            ctx.op = op
            ctx.save_for_backward(u)
            return c

        @staticmethod
        def backward(ctx, grad_c):
            (u,) = ctx.saved_tensors
            op = ctx.op
            g = torch.empty(op.n_elements, dtype=torch.float64, device=op.device)
            abi.fe_compliance_gradient(op.ctx, u, float(grad_c), 1e-12, 50000, 64, g)
            return g, None, None, None

    return ComplianceFn


_COMPLIANCE = None


def __getattr__(name):
    global _COMPLIANCE
    if name == "ComplianceFn":
        if _COMPLIANCE is None:
            _COMPLIANCE = _compliance_autograd()
        return _COMPLIANCE
    raise AttributeError(name)
