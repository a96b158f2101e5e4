"""ctypes binding of include/feod.h: the same entry points under the same names.

Argument marshalling only: every step of every call runs in the CUDA library.  Vectors are passed
as torch CUDA tensors (their data pointers); streams default to torch's current stream.  The
library must have been built (``paper_2506_00746_gb300.build.build()``); loading fails loudly
otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_char_p, c_double, c_int, c_int64, c_void_p

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfeod.so")


class FeodError(RuntimeError):
    """A library call returned a non-OK fe_status."""

    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: status {status} ({STATUS_NAMES.get(status, '?')}): {message}")
        self.status = status


STATUS_NAMES = {0: "FE_OK", 1: "FE_ERR_ARG", 2: "FE_ERR_MESH", 3: "FE_ERR_CUDA", 4: "FE_ERR_OOM",
                5: "FE_ERR_UNSUPPORTED", 6: "FE_ERR_NAN", 7: "FE_ERR_NOT_CONVERGED",
                8: "FE_ERR_BREAKDOWN", 9: "FE_ERR_STATE"}
FE_OK = 0


class fe_mesh(ctypes.Structure):
    _fields_ = [("dim", c_int), ("n", c_int * 3), ("vertices", POINTER(c_double)), ("natural_faces", c_int)]


def make_mesh(dim: int, n, vertices_ptr, natural_faces: int = 0) -> fe_mesh:
    """fe_mesh for a lattice of n elements per direction (an int: the same in every direction, or
    a sequence of dim counts)."""
    nn = [int(n)] * dim if isinstance(n, (int, np.integer)) else [int(x) for x in n]
    if len(nn) != dim:
        raise ValueError(f"n needs {dim} element counts")
    m = fe_mesh()
    m.dim = dim
    for d in range(3):
        m.n[d] = nn[d] if d < dim else 1
    m.vertices = vertices_ptr
    m.natural_faces = int(natural_faces)
    return m


class fe_problem(ctypes.Structure):
    _fields_ = [("p", c_double), ("eps", c_double), ("f_kind", c_int), ("f_const", c_double),
                ("rho", POINTER(c_double)), ("kappa_eps", c_double), ("kappa_q", c_double)]


class fe_setup_opts(ctypes.Structure):
    _fields_ = [("tile", c_int), ("per_element", c_int)]


class fe_newton_opts(ctypes.Structure):
    _fields_ = [("rtol", c_double), ("max_newton", c_int), ("max_cg", c_int), ("cg_rtol", c_double),
                ("inner_precision", c_int), ("line_search", c_int), ("armijo", c_double),
                ("max_halvings", c_int), ("cg_batch", c_int), ("use_graph", c_int), ("forcing", c_int),
                ("eta_max", c_double)]


FE_NEWTON_HIST = 64


class fe_newton_report(ctypes.Structure):
    _fields_ = [("newton_iters", c_int), ("cg_iters_total", c_int), ("line_search_halvings", c_int),
                ("status", c_int), ("r0", c_double), ("r_final", c_double), ("t_total_ms", c_double),
                ("t_cg_ms", c_double), ("kernel_launches", c_int64),
                ("r_hist", c_double * FE_NEWTON_HIST), ("cg_hist", c_int * FE_NEWTON_HIST)]


class fe_batch_item(ctypes.Structure):
    _fields_ = [("mesh", POINTER(fe_mesh)), ("order", c_int), ("prob", POINTER(fe_problem))]


class fe_batch_opts(ctypes.Structure):
    _fields_ = [("tune_cache", c_char_p), ("tune", c_int), ("retune", c_int), ("policy", c_int),
                ("tile", c_int * 4)]


_CTX = c_void_p
_BATCH = c_void_p
_SIGS = {
    "fe_setup": (c_int, [POINTER(fe_mesh), c_int, c_int, POINTER(fe_problem), POINTER(_CTX)]),
    "fe_setup_ex": (c_int, [POINTER(fe_mesh), c_int, c_int, POINTER(fe_problem), POINTER(fe_setup_opts),
                            POINTER(_CTX)]),
    "fe_num_dofs": (c_int, [_CTX, POINTER(c_int64), POINTER(c_int64)]),
    "fe_num_elements": (c_int, [_CTX, POINTER(c_int64)]),
    "fe_residual": (c_int, [_CTX, c_void_p, c_void_p, c_void_p]),
    "fe_linearize": (c_int, [_CTX, c_void_p, c_void_p]),
    "fe_jacobian_action": (c_int, [_CTX, c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
    "fe_jacobian_action_host": (c_int, [_CTX, c_void_p, c_void_p, c_int, c_void_p]),
    "fe_jacobian_action_noalloc": (c_int, [_CTX, c_void_p, c_void_p, c_int, c_void_p]),
    "fe_jacobian_diagonal": (c_int, [_CTX, c_void_p, c_void_p]),
    "fe_load_vector": (c_int, [_CTX, c_void_p, c_void_p]),
    "fe_node_coords": (c_int, [_CTX, c_void_p, c_void_p]),
    "fe_set_design": (c_int, [_CTX, c_void_p, c_void_p]),
    "fe_adjoint_vjp": (c_int, [_CTX, c_void_p, c_void_p, c_void_p, c_void_p]),
    "fe_newton_default_opts": (c_int, [POINTER(fe_newton_opts)]),
    "newton_solve": (c_int, [_CTX, c_void_p, POINTER(fe_newton_opts), POINTER(fe_newton_report), c_void_p]),
    "fe_cg_solve": (c_int, [_CTX, c_void_p, c_void_p, c_double, c_int, c_int, POINTER(c_int), c_void_p]),
    "fe_prof_enable": (c_int, [_CTX, c_int]),
    "fe_prof_reset": (c_int, [_CTX]),
    "fe_prof_read": (c_int, [_CTX, c_int, POINTER(c_char_p), POINTER(c_int64), POINTER(c_double),
                             POINTER(c_int)]),
    "fe_launch_count": (c_int, [_CTX, POINTER(c_int64)]),
    "fe_memory_bytes": (c_int, [_CTX, POINTER(c_int64)]),
    "fe_measure_fp64_peak": (c_int, [c_int, POINTER(c_double), POINTER(c_double), c_void_p]),
    "fe_dot": (c_int, [_CTX, c_void_p, c_void_p, c_int64, c_int64, c_void_p, c_void_p]),
    "fe_compliance": (c_int, [_CTX, c_void_p, c_void_p, c_void_p]),
    "fe_compliance_gradient": (c_int, [_CTX, c_void_p, c_double, c_double, c_int, c_int, c_void_p, POINTER(c_int),
                                       c_void_p]),
    "fe_axpby": (c_int, [_CTX, c_double, c_void_p, c_double, c_void_p, c_void_p]),
    "fe_pointwise_mul": (c_int, [_CTX, c_void_p, c_void_p, c_void_p, c_void_p]),
    "fe_reciprocal": (c_int, [_CTX, c_void_p, c_void_p, c_void_p]),
    "fe_face_size": (c_int, [_CTX, c_int, POINTER(c_int64)]),
    "fe_face_add": (c_int, [_CTX, c_int, c_void_p, c_void_p, c_void_p]),
    "fe_destroy": (None, [_CTX]),
    "fe_last_error": (c_char_p, [_CTX]),
    "fe_status_string": (c_char_p, [c_int]),
    "fe_element_matrices": (c_int, [_CTX, c_void_p, c_int, c_int64, c_int64, c_void_p, c_void_p]),
    "fe_selftest_wait_timeout": (c_int, [_CTX, c_void_p]),
    "fe_check_error": (c_int, [_CTX, c_void_p]),
    "fe_batch_create": (c_int, [POINTER(fe_batch_item), c_int, POINTER(fe_batch_opts), POINTER(_BATCH)]),
    "fe_batch_info": (c_int, [_BATCH, c_int, POINTER(c_int64), POINTER(c_int64), POINTER(c_int)]),
    "fe_batch_shape": (c_int, [_BATCH, POINTER(c_int64), POINTER(c_int), POINTER(c_int), POINTER(c_int),
                               POINTER(c_int64)]),
    "fe_batch_linearize": (c_int, [_BATCH, c_void_p, c_void_p]),
    "fe_batch_jacobian_action": (c_int, [_BATCH, c_void_p, c_void_p, c_void_p]),
    "fe_batch_newton_solve": (c_int, [_BATCH, c_void_p, POINTER(fe_newton_opts), POINTER(fe_newton_report),
                                      POINTER(fe_newton_report), c_void_p]),
    "fe_batch_destroy": (None, [_BATCH]),
    "fe_batch_last_error": (c_char_p, [_BATCH]),
}

_LIB = None


def library(path: str | None = None) -> ctypes.CDLL:
    """Load libfeod.so (once).  Raises FileNotFoundError if it has not been built."""
    global _LIB
    if _LIB is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise FileNotFoundError(f"{p} is missing: build the CUDA library first "
                                    "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(p)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def declared_symbols() -> list[str]:
    """Entry points this binding declares (the functions of include/feod.h)."""
    return list(_SIGS)


def check(status: int, where: str, ctx=None) -> None:
    if status != FE_OK:
        msg = library().fe_last_error(ctx)
        raise FeodError(status, where, msg.decode() if msg else "")


def ptr(t) -> c_void_p | None:
    """Device (or host) pointer of a torch tensor / None."""
    if t is None:
        return None
    return c_void_p(t.data_ptr())


def stream_handle(stream=None) -> c_void_p:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return c_void_p(s.cuda_stream)


# ---- same-name wrappers (argument marshalling only) -----------------------------------------

def fe_setup(mesh: fe_mesh, order: int, q1d: int, prob: fe_problem, opts: fe_setup_opts | None = None):
    ctx = _CTX()
    if opts is None:
        st = library().fe_setup(byref(mesh), order, q1d, byref(prob), byref(ctx))
    else:
        st = library().fe_setup_ex(byref(mesh), order, q1d, byref(prob), byref(opts), byref(ctx))
    check(st, "fe_setup")
    return ctx


def fe_num_dofs(ctx):
    nl, nf = c_int64(), c_int64()
    check(library().fe_num_dofs(ctx, byref(nl), byref(nf)), "fe_num_dofs", ctx)
    return nl.value, nf.value


def fe_num_elements(ctx):
    ne = c_int64()
    check(library().fe_num_elements(ctx, byref(ne)), "fe_num_elements", ctx)
    return ne.value


def fe_residual(ctx, u, r, stream=None):
    check(library().fe_residual(ctx, ptr(u), ptr(r), stream_handle(stream)), "fe_residual", ctx)


def fe_linearize(ctx, u, stream=None):
    check(library().fe_linearize(ctx, ptr(u), stream_handle(stream)), "fe_linearize", ctx)


def fe_jacobian_action(ctx, u, v, y, precision: int, stream=None):
    check(library().fe_jacobian_action(ctx, ptr(u), ptr(v), ptr(y), precision, stream_handle(stream)),
          "fe_jacobian_action", ctx)


def fe_jacobian_action_host(ctx, v_host, y_host, precision: int, stream=None):
    check(library().fe_jacobian_action_host(ctx, ptr(v_host), ptr(y_host), precision, stream_handle(stream)),
          "fe_jacobian_action_host", ctx)


def fe_jacobian_action_noalloc(ctx, v, y, precision: int, stream=None):
    """Allocation-free variant of the cached Jacobian action (static device scratch; see feod.h)."""
    check(library().fe_jacobian_action_noalloc(ctx, ptr(v), ptr(y), precision, stream_handle(stream)),
          "fe_jacobian_action_noalloc", ctx)


def fe_jacobian_diagonal(ctx, diag, stream=None):
    check(library().fe_jacobian_diagonal(ctx, ptr(diag), stream_handle(stream)), "fe_jacobian_diagonal", ctx)


def fe_load_vector(ctx, F, stream=None):
    check(library().fe_load_vector(ctx, ptr(F), stream_handle(stream)), "fe_load_vector", ctx)


def fe_node_coords(ctx, xyz, stream=None):
    check(library().fe_node_coords(ctx, ptr(xyz), stream_handle(stream)), "fe_node_coords", ctx)


def fe_set_design(ctx, rho, stream=None):
    check(library().fe_set_design(ctx, ptr(rho), stream_handle(stream)), "fe_set_design", ctx)


def fe_adjoint_vjp(ctx, u, lam, grad, stream=None):
    check(library().fe_adjoint_vjp(ctx, ptr(u), ptr(lam), ptr(grad), stream_handle(stream)), "fe_adjoint_vjp", ctx)


def fe_element_matrices(ctx, u, method: int, e0: int, count: int, K, stream=None):
    check(library().fe_element_matrices(ctx, ptr(u), method, e0, count, ptr(K), stream_handle(stream)),
          "fe_element_matrices", ctx)


def fe_check_error(ctx, stream=None):
    """Raise FeodError (FE_ERR_CUDA) if a kernel of the context reported a timed-out wait."""
    check(library().fe_check_error(ctx, stream_handle(stream)), "fe_check_error", ctx)


def fe_selftest_wait_timeout(ctx, stream=None):
    check(library().fe_selftest_wait_timeout(ctx, stream_handle(stream)), "fe_selftest_wait_timeout", ctx)


def fe_newton_default_opts() -> fe_newton_opts:
    o = fe_newton_opts()
    check(library().fe_newton_default_opts(byref(o)), "fe_newton_default_opts")
    return o


def newton_solve(ctx, u, opts: fe_newton_opts | None = None, stream=None) -> fe_newton_report:
    rep = fe_newton_report()
    st = library().newton_solve(ctx, ptr(u), byref(opts) if opts is not None else None, byref(rep),
                                stream_handle(stream))
    rep.status = st
    if st not in (FE_OK,):
        rep.error = library().fe_last_error(ctx).decode()
    return rep


def fe_cg_solve(ctx, b, x, rtol: float, max_iter: int, precision: int, stream=None) -> int:
    it = c_int()
    check(library().fe_cg_solve(ctx, ptr(b), ptr(x), rtol, max_iter, precision, byref(it), stream_handle(stream)),
          "fe_cg_solve", ctx)
    return it.value


def fe_prof_enable(ctx, enable: bool):
    check(library().fe_prof_enable(ctx, int(bool(enable))), "fe_prof_enable", ctx)


def fe_prof_reset(ctx):
    check(library().fe_prof_reset(ctx), "fe_prof_reset", ctx)


def fe_prof_read(ctx) -> dict:
    """{kernel name: (launches, total ms)} since the last reset."""
    lib = library()
    cnt = c_int()
    check(lib.fe_prof_read(ctx, -1, None, None, None, byref(cnt)), "fe_prof_read", ctx)
    out = {}
    for i in range(cnt.value):
        name, n, ms = c_char_p(), c_int64(), c_double()
        check(lib.fe_prof_read(ctx, i, byref(name), byref(n), byref(ms), byref(cnt)), "fe_prof_read", ctx)
        out[name.value.decode()] = (n.value, ms.value)
    return out


def fe_launch_count(ctx) -> int:
    n = c_int64()
    check(library().fe_launch_count(ctx, byref(n)), "fe_launch_count", ctx)
    return n.value


def fe_memory_bytes(ctx) -> int:
    n = c_int64()
    check(library().fe_memory_bytes(ctx, byref(n)), "fe_memory_bytes", ctx)
    return n.value


def fe_measure_fp64_peak(reps: int = 20, stream=None) -> tuple[float, float]:
    """(best, median) FP64 FMA rate of the current device in TFLOP/s."""
    best, med = c_double(), c_double()
    check(library().fe_measure_fp64_peak(reps, byref(best), byref(med), stream_handle(stream)),
          "fe_measure_fp64_peak")
    return best.value, med.value


def fe_dot(ctx, a, b, begin: int, end: int, out, stream=None):
    """out (a device double tensor of one entry) = a[begin:end] . b[begin:end]."""
    check(library().fe_dot(ctx, ptr(a), ptr(b), begin, end, ptr(out), stream_handle(stream)), "fe_dot", ctx)


def fe_compliance(ctx, u, out, stream=None):
    """out (a device double tensor of one entry) = F^T u."""
    check(library().fe_compliance(ctx, ptr(u), ptr(out), stream_handle(stream)), "fe_compliance", ctx)


def fe_compliance_gradient(ctx, u, scale: float, rtol: float, max_iter: int, precision: int, grad, stream=None) -> int:
    it = c_int()
    check(library().fe_compliance_gradient(ctx, ptr(u), scale, rtol, max_iter, precision, ptr(grad), byref(it),
                                           stream_handle(stream)), "fe_compliance_gradient", ctx)
    return it.value


def fe_axpby(ctx, alpha: float, x, beta: float, y, stream=None):
    check(library().fe_axpby(ctx, alpha, ptr(x), beta, ptr(y), stream_handle(stream)), "fe_axpby", ctx)


def fe_pointwise_mul(ctx, d, r, z, stream=None):
    check(library().fe_pointwise_mul(ctx, ptr(d), ptr(r), ptr(z), stream_handle(stream)), "fe_pointwise_mul", ctx)


def fe_reciprocal(ctx, x, y, stream=None):
    check(library().fe_reciprocal(ctx, ptr(x), ptr(y), stream_handle(stream)), "fe_reciprocal", ctx)


def fe_face_size(ctx, face: int) -> int:
    n = c_int64()
    check(library().fe_face_size(ctx, face, byref(n)), "fe_face_size", ctx)
    return n.value


def fe_face_add(ctx, face: int, y, buf, stream=None):
    check(library().fe_face_add(ctx, face, ptr(y), ptr(buf), stream_handle(stream)), "fe_face_add", ctx)


def fe_destroy(ctx):
    if ctx:
        library().fe_destroy(ctx)


def fe_last_error(ctx=None) -> str:
    m = library().fe_last_error(ctx)
    return m.decode() if m else ""


# ---- batched instances ---------------------------------------------------------------------

def _bcheck(status: int, where: str, batch=None) -> None:
    if status != FE_OK:
        msg = library().fe_batch_last_error(batch)
        raise FeodError(status, where, msg.decode() if msg else "")


def fe_batch_create(items, count: int, opts: fe_batch_opts | None = None):
    b = _BATCH()
    _bcheck(library().fe_batch_create(items, count, byref(opts) if opts is not None else None, byref(b)),
            "fe_batch_create")
    return b


def fe_batch_info(batch, i: int) -> tuple[int, int, int]:
    off, n, tile = c_int64(), c_int64(), c_int()
    _bcheck(library().fe_batch_info(batch, i, byref(off), byref(n), byref(tile)), "fe_batch_info", batch)
    return off.value, n.value, tile.value


def fe_batch_shape(batch) -> dict:
    tot, grid, thr, pol, ln = c_int64(), c_int(), c_int(), c_int(), c_int64()
    _bcheck(library().fe_batch_shape(batch, byref(tot), byref(grid), byref(thr), byref(pol), byref(ln)),
            "fe_batch_shape", batch)
    return {"total": tot.value, "grid": grid.value, "threads": thr.value, "policy": pol.value,
            "launches": ln.value}


def fe_batch_linearize(batch, u, stream=None):
    _bcheck(library().fe_batch_linearize(batch, ptr(u), stream_handle(stream)), "fe_batch_linearize", batch)


def fe_batch_jacobian_action(batch, v, y, stream=None):
    _bcheck(library().fe_batch_jacobian_action(batch, ptr(v), ptr(y), stream_handle(stream)),
            "fe_batch_jacobian_action", batch)


def fe_batch_newton_solve(batch, u, count: int, opts: fe_newton_opts | None = None, stream=None):
    reps = (fe_newton_report * count)()
    tot = fe_newton_report()
    st = library().fe_batch_newton_solve(batch, ptr(u), byref(opts) if opts is not None else None, reps,
                                         byref(tot), stream_handle(stream))
    tot.status = st
    err = library().fe_batch_last_error(batch).decode() if st != FE_OK else ""
    return list(reps), tot, err


def fe_batch_destroy(batch):
    if batch:
        library().fe_batch_destroy(batch)


def fe_batch_last_error(batch=None) -> str:
    m = library().fe_batch_last_error(batch)
    return m.decode() if m else ""
