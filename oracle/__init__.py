"""Oracle: a plain, slow, FP64 CPU reference for the operator of Eq. 1 and Eq. 2.

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference leg of ``bench.py`` may import or run it.  The CUDA library neither imports, links nor
calls anything here, and nothing here imports the CUDA library: the two meet only through the
seeded input arrays of ``paper_2506_00746_gb300.inputs``.

The element-level arithmetic lives in ``feod_oracle.c`` (dense per-element basis tables, the
analytic tangent of the pointwise operator, fixed-order global sums).  This module adds, on top of
it, the library-primitive steps the paper's method composes:

* ``assemble``  -- global sparse Jacobian from the element tangents K_e = B^T J_D B (Eq. 3),
  summed with scipy's COO->CSR conversion, then the Dirichlet convention (identity rows/columns);
* ``newton``    -- Newton's method on R(u) = 0 with a sparse direct solve and backtracking on
  ||R||_2 (the nonlinear solve that Eq. 2's Jacobian serves);
* ``adjoint_solve`` -- J(u) lambda = F (J is symmetric) for the compliance c = F^T u.
"""
from __future__ import annotations

import ctypes
import dataclasses
from ctypes import POINTER, c_double, c_int, c_int64

import numpy as np

from .build import build as _build

__all__ = [
    "Problem", "gauss_legendre", "gll_nodes", "lagrange", "node_coords", "residual", "load", "jv",
    "jv_partial", "residual_partial", "element_vectors", "element_matrices", "assemble",
    "adjoint_grad", "flux_work", "l2_error_exp", "exact_exp", "essential", "newton",
    "adjoint_solve", "set_threads",
]

_DP = POINTER(c_double)
_IP = POINTER(c_int64)


class _CProblem(ctypes.Structure):
    _fields_ = [("dim", c_int), ("n", c_int), ("order", c_int), ("q1d", c_int),
                ("vert", _DP), ("p", c_double), ("eps", c_double), ("f_kind", c_int),
                ("f_const", c_double), ("rho", _DP), ("kappa_eps", c_double),
                ("kappa_q", c_double)]


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        _LIB = _bind(_build())
    return _LIB


def _bind(path):
    lib = ctypes.CDLL(path)
    if lib is not None:
        P = POINTER(_CProblem)
        sig = {
            "orc_gauss_legendre": (c_int, [c_int, _DP, _DP]),
            "orc_gll_nodes": (c_int, [c_int, _DP]),
            "orc_lagrange": (c_int, [c_int, _DP, c_int, _DP, _DP, _DP]),
            "orc_node_coords": (c_int, [P, _DP]),
            "orc_residual": (c_int, [P, _DP, _DP]),
            "orc_jv": (c_int, [P, _DP, _DP, _DP]),
            "orc_jv_partial": (c_int, [P, _DP, _DP, _DP, c_int64, c_int64]),
            "orc_residual_partial": (c_int, [P, _DP, _DP, c_int64, c_int64]),
            "orc_element_vectors": (c_int, [P, _DP, _DP, _IP, c_int64, _DP, _DP, _IP]),
            "orc_element_matrices": (c_int, [P, _DP, c_int64, c_int64, _DP, _DP, _IP]),
            "orc_load": (c_int, [P, _DP]),
            "orc_adjoint_grad": (c_int, [P, _DP, _DP, _DP]),
            "orc_flux_work": (c_double, [P, _DP]),
            "orc_l2_error_exp": (c_double, [P, _DP, c_int]),
            "orc_exact_exp": (c_int, [c_int, c_int64, _DP, _DP]),
            "orc_set_threads": (c_int, [c_int]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
    return lib


class planted:
    """Context manager that swaps in a deliberately wrong oracle build (test use only)."""

    def __init__(self, plant: int):
        self.plant = plant

    def __enter__(self):
        global _LIB
        self._saved = _lib()
        _LIB = _bind(_build(plant=self.plant))
        return self

    def __exit__(self, *exc):
        global _LIB
        _LIB = self._saved
        return False


def _dp(a):
    return None if a is None else a.ctypes.data_as(_DP)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc} "
                           f"({ {1: 'bad argument', 2: 'det J <= 0', 3: 'out of memory'}.get(rc, '?') })")


@dataclasses.dataclass
class Problem:
    """The discrete p-Laplacian problem: lattice mesh, order, quadrature and the law's constants."""
    dim: int
    n: int
    order: int
    vertices: np.ndarray
    p: float = 3.0
    eps: float = 0.0
    f_kind: int = 0              # 0: f = f_const, 1: manufactured source of exp(x + y/2 + z/3)
    f_const: float = 1.0
    rho: np.ndarray | None = None
    kappa_eps: float = 1e-3
    kappa_q: float = 3.0
    q1d: int = 0                 # Gauss points per direction; 0 means order + 1

    def __post_init__(self):
        self.vertices = _f64(self.vertices)
        if self.rho is not None:
            self.rho = _f64(self.rho)
        self._c = _CProblem(self.dim, self.n, self.order, self.q1d, _dp(self.vertices), self.p,
                            self.eps, self.f_kind, self.f_const, _dp(self.rho), self.kappa_eps,
                            self.kappa_q)

    @property
    def n_dofs(self) -> int:
        return (self.order * self.n + 1) ** self.dim

    @property
    def n_elems(self) -> int:
        return self.n ** self.dim

    @property
    def nl(self) -> int:
        return (self.order + 1) ** self.dim

    def ref(self):
        return ctypes.byref(self._c)


def set_threads(n: int) -> int:
    return _lib().orc_set_threads(int(n))


def gauss_legendre(q: int):
    x = np.zeros(q); w = np.zeros(q)
    _check(_lib().orc_gauss_legendre(q, _dp(x), _dp(w)), "gauss_legendre")
    return x, w


def gll_nodes(k: int):
    x = np.zeros(k + 1)
    _check(_lib().orc_gll_nodes(k, _dp(x)), "gll_nodes")
    return x


def lagrange(nodes, pts):
    nodes = _f64(nodes); pts = _f64(pts)
    val = np.zeros((len(pts), len(nodes))); der = np.zeros_like(val)
    _check(_lib().orc_lagrange(len(nodes), _dp(nodes), len(pts), _dp(pts), _dp(val), _dp(der)),
           "lagrange")
    return val, der


def node_coords(P: Problem):
    xyz = np.zeros((P.n_dofs, P.dim))
    _check(_lib().orc_node_coords(P.ref(), _dp(xyz)), "node_coords")
    return xyz


def residual(P: Problem, u):
    u = _f64(u); r = np.zeros(P.n_dofs)
    _check(_lib().orc_residual(P.ref(), _dp(u), _dp(r)), "residual")
    return r


def load(P: Problem):
    F = np.zeros(P.n_dofs)
    _check(_lib().orc_load(P.ref(), _dp(F)), "load")
    return F


def jv(P: Problem, u, v):
    u = _f64(u); v = _f64(v); y = np.zeros(P.n_dofs)
    _check(_lib().orc_jv(P.ref(), _dp(u), _dp(v), _dp(y)), "jv")
    return y


def jv_partial(P: Problem, u, v, e0: int, e1: int, y=None):
    u = _f64(u); v = _f64(v)
    y = np.zeros(P.n_dofs) if y is None else y
    _check(_lib().orc_jv_partial(P.ref(), _dp(u), _dp(v), _dp(y), e0, e1), "jv_partial")
    return y


def residual_partial(P: Problem, u, e0: int, e1: int, r=None):
    u = _f64(u)
    r = np.zeros(P.n_dofs) if r is None else r
    _check(_lib().orc_residual_partial(P.ref(), _dp(u), _dp(r), e0, e1), "residual_partial")
    return r


def element_vectors(P: Problem, u, v, elems):
    """Per-element residuals r_e, Jacobian actions K_e v_e (v used unmasked) and DOF maps."""
    elems = np.ascontiguousarray(elems, dtype=np.int64)
    u = _f64(u); v = None if v is None else _f64(v)
    re = np.zeros((len(elems), P.nl)); ye = np.zeros_like(re)
    dofs = np.zeros((len(elems), P.nl), dtype=np.int64)
    _check(_lib().orc_element_vectors(P.ref(), _dp(u), _dp(v), elems.ctypes.data_as(_IP),
                                      len(elems), _dp(re), _dp(ye) if v is not None else None,
                                      dofs.ctypes.data_as(_IP)), "element_vectors")
    return re, (ye if v is not None else None), dofs


def element_matrices(P: Problem, u, e0: int = 0, e1: int | None = None):
    e1 = P.n_elems if e1 is None else e1
    u = _f64(u); cnt = e1 - e0
    K = np.zeros((cnt, P.nl, P.nl)); r = np.zeros((cnt, P.nl))
    dofs = np.zeros((cnt, P.nl), dtype=np.int64)
    _check(_lib().orc_element_matrices(P.ref(), _dp(u), e0, e1, _dp(K), _dp(r),
                                       dofs.ctypes.data_as(_IP)), "element_matrices")
    return K, r, dofs


def essential(P: Problem) -> np.ndarray:
    """Boolean mask of boundary DOFs, computed from the lattice numbering."""
    m = P.order * P.n + 1
    g = np.arange(P.n_dofs)
    mask = np.zeros(P.n_dofs, dtype=bool)
    for _ in range(P.dim):
        i = g % m
        mask |= (i == 0) | (i == m - 1)
        g = g // m
    return mask


def assemble(P: Problem, u, dirichlet: bool = True):
    """Global Jacobian J(u) (CSR) and residual R(u), element by element (Eq. 2, Eq. 3).

    With ``dirichlet`` the essential rows and columns become the identity and R is zero there.
    """
    import scipy.sparse as sp
    K, r, dofs = element_matrices(P, u)
    nl = P.nl
    rows = np.repeat(dofs, nl, axis=1).ravel()
    cols = np.tile(dofs, (1, nl)).ravel()
    J = sp.coo_matrix((K.ravel(), (rows, cols)), shape=(P.n_dofs, P.n_dofs)).tocsr()
    R = np.zeros(P.n_dofs)
    np.add.at(R, dofs.ravel(), r.ravel())
    if dirichlet:
        ess = essential(P)
        keep = sp.diags((~ess).astype(np.float64))
        J = (keep @ J @ keep + sp.diags(ess.astype(np.float64))).tocsr()
        R[ess] = 0.0
    return J, R


def adjoint_grad(P: Problem, u, lam):
    u = _f64(u); lam = _f64(lam); g = np.zeros(P.n_elems)
    _check(_lib().orc_adjoint_grad(P.ref(), _dp(u), _dp(lam), _dp(g)), "adjoint_grad")
    return g


def flux_work(P: Problem, u) -> float:
    u = _f64(u)
    return float(_lib().orc_flux_work(P.ref(), _dp(u)))


def l2_error_exp(P: Problem, u, qextra: int = 3) -> float:
    u = _f64(u)
    return float(_lib().orc_l2_error_exp(P.ref(), _dp(u), qextra))


def exact_exp(dim: int, x):
    x = _f64(x); out = np.zeros(len(x))
    _check(_lib().orc_exact_exp(dim, len(x), _dp(x), _dp(out)), "exact_exp")
    return out


def newton(P: Problem, u0, rtol: float = 1e-8, max_newton: int = 60, armijo: float = 1e-4,
           max_halvings: int = 20, history: list | None = None, linear: str = "direct",
           cg_rtol: float = 1e-4, cg_iters: list | None = None):
    """Newton's method for R(u) = 0 with backtracking on ||R||_2.

    Each step solves J(u) delta = -R(u) on the assembled sparse Jacobian: ``linear="direct"`` by a
    sparse direct solve, ``linear="cg"`` by scipy's conjugate gradients with the Jacobi (diagonal)
    preconditioner to ||J delta + R|| <= cg_rtol ||R|| (the inexact Newton step of the matrix-free
    solver; the iteration counts go to ``cg_iters``).  A step alpha*delta is accepted when
    ||R(u + alpha delta)|| <= (1 - armijo*alpha) ||R(u)||; otherwise alpha is halved (at most
    ``max_halvings`` times).  Stops when ||R(u_k)|| <= rtol * ||R(u_0)||.  Returns (u, list of
    residual norms).
    """
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    if linear not in ("direct", "cg"):
        raise ValueError("linear must be 'direct' or 'cg'")
    u = _f64(u0).copy()
    hist = [] if history is None else history
    r = residual(P, u)
    r0 = np.linalg.norm(r)
    hist.append(r0)
    if r0 == 0.0:
        return u, hist
    for _ in range(max_newton):
        if hist[-1] <= rtol * r0:
            break
        J, _ = assemble(P, u)
        if linear == "direct":
            delta = spla.spsolve(J.tocsc(), -r)
        else:
            count = [0]
            Minv = sp.diags(1.0 / J.diagonal())
            delta, info = spla.cg(J, -r, rtol=cg_rtol, maxiter=20000, M=Minv,
                                  callback=lambda _x: count.__setitem__(0, count[0] + 1))
            if info != 0:
                raise RuntimeError(f"oracle CG did not converge (info {info})")
            if cg_iters is not None:
                cg_iters.append(count[0])
        alpha, rn = 1.0, hist[-1]
        for _h in range(max_halvings + 1):
            trial = u + alpha * delta
            rt = residual(P, trial)
            nt = np.linalg.norm(rt)
            if nt <= (1.0 - armijo * alpha) * rn:
                break
            alpha *= 0.5
        u, r = trial, rt
        hist.append(nt)
    return u, hist


def adjoint_solve(P: Problem, u):
    """lambda with J(u) lambda = F, F the load vector with essential entries removed."""
    import scipy.sparse.linalg as spla
    J, _ = assemble(P, u)
    F = load(P)
    F[essential(P)] = 0.0
    return spla.spsolve(J.tocsc(), F)
