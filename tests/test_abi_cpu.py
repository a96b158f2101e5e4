"""CPU-side checks of the boundary: the library builds, loads, and exports every entry point that
include/feod.h declares; the binding declares exactly those; host-side input recipes."""
from __future__ import annotations

import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "feod.h")


def _header_functions() -> set[str]:
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(", src, flags=re.M))
    return {n for n in names if n.startswith("fe_") or n == "newton_solve"}


@pytest.fixture(scope="module")
def lib_path():
    from paper_2506_00746_gb300.build import build
    return build()


def test_header_declares_the_boundary():
    names = _header_functions()
    for required in ("fe_setup", "fe_residual", "fe_jacobian_action", "fe_adjoint_vjp", "newton_solve",
                     "fe_linearize", "fe_destroy", "fe_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = _header_functions() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_binding_matches_header(lib_path):
    from paper_2506_00746_gb300 import abi
    lib = abi.library(lib_path)
    assert set(abi.declared_symbols()) == _header_functions()
    for name in abi.declared_symbols():
        assert hasattr(lib, name)


def _header_struct_fields(name: str) -> list[str]:
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + r"\s*;", src, flags=re.S).group(1)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if decl:
            fields.append(re.findall(r"([A-Za-z_][A-Za-z_0-9]*)\s*(?:\[\d+\])?\s*$", decl)[0])
    return fields


@pytest.mark.parametrize("name", ["fe_mesh", "fe_problem", "fe_setup_opts", "fe_newton_opts", "fe_batch_item",
                                  "fe_batch_opts"])
def test_binding_structs_match_header(name):
    """The ctypes structures list the header's fields in the header's order."""
    from paper_2506_00746_gb300 import abi
    assert [f[0] for f in getattr(abi, name)._fields_] == _header_struct_fields(name)


def test_setup_rejects_bad_arguments_without_gpu(lib_path):
    """Argument validation happens before any device call."""
    import ctypes
    from paper_2506_00746_gb300 import abi
    lib = abi.library(lib_path)
    V = np.zeros((4, 2))
    mesh = abi.make_mesh(2, 1, V.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    prob = abi.fe_problem(3.0, 0.0, 0, 1.0, None, 0.0, 1.0)
    ctx = ctypes.c_void_p()
    assert lib.fe_setup(ctypes.byref(mesh), 0, 0, ctypes.byref(prob), ctypes.byref(ctx)) == 5   # order 0
    assert lib.fe_setup(ctypes.byref(mesh), 7, 0, ctypes.byref(prob), ctypes.byref(ctx)) == 5   # order 7
    assert lib.fe_setup(ctypes.byref(mesh), 2, 5, ctypes.byref(prob), ctypes.byref(ctx)) == 5   # q1d
    bad = abi.fe_problem(1.5, 0.0, 0, 1.0, None, 0.0, 1.0)                                       # p < 2, eps = 0
    assert lib.fe_setup(ctypes.byref(mesh), 2, 0, ctypes.byref(bad), ctypes.byref(ctx)) == 1
    assert b"p >= 2" in lib.fe_last_error(None)
    assert lib.fe_setup(None, 2, 0, ctypes.byref(prob), ctypes.byref(ctx)) == 1
    bad_mesh = abi.make_mesh(2, (1, 0), V.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))   # n[1] = 0
    assert lib.fe_setup(ctypes.byref(bad_mesh), 2, 0, ctypes.byref(prob), ctypes.byref(ctx)) == 1
    bad_faces = abi.make_mesh(2, 1, V.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), natural_faces=16)  # z- in 2D
    assert lib.fe_setup(ctypes.byref(bad_faces), 2, 0, ctypes.byref(prob), ctypes.byref(ctx)) == 1
    assert b"natural_faces" in lib.fe_last_error(None)
    # the largest lattice: more than 2^30 - 1 DOFs is rejected before anything is read or allocated
    # (the vertex array is never touched, so a small one stands in)
    big = abi.make_mesh(3, (1100, 1100, 1100), V.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    prob3 = abi.fe_problem(3.0, 0.0, 0, 1.0, None, 0.0, 1.0)
    assert lib.fe_setup(ctypes.byref(big), 1, 0, ctypes.byref(prob3), ctypes.byref(ctx)) == 5
    assert b"DOFs exceed" in lib.fe_last_error(None)
    assert not ctx.value
    assert not ctx.value
    assert lib.fe_status_string(2) == b"invalid mesh (det J <= 0)"
    o = abi.fe_newton_default_opts()
    assert o.rtol == 1e-8 and o.inner_precision == 64 and o.line_search == 1


def test_input_recipes():
    from paper_2506_00746_gb300 import inputs as I
    V = I.lattice_vertices(3, 4, seed=0)
    h = 0.25
    idx = I.lattice_index(5, 3)
    base = idx.T * h
    shift = np.linalg.norm(V - base, axis=1)
    assert shift.max() <= 0.1 * h + 1e-15
    boundary = np.any((idx == 0) | (idx == 4), axis=0)
    assert np.all(shift[boundary] == 0.0) and np.all(shift[~boundary] > 0)
    u = I.smooth_field(3, 4, 2, seed=1)
    assert u.shape == (9 ** 3,)
    assert np.all(u[I.boundary_mask(3, 4, 2).astype(bool)] == 0.0)
    np.testing.assert_array_equal(I.smooth_field(3, 4, 2, seed=1), u)   # seeded
    assert I.WORKLOADS["3d_p3_k3_64"].n_dofs == 7_189_057
    assert I.WORKLOADS["2d_p3_k2_16x16"].n_dofs == 1089
    assert [I.sweep_workload(k).n_dofs for k in range(1, 7)] == [8_000_000, 8_120_601, 7_880_599, 8_120_601,
                                                                8_120_601, 7_880_599]
    b = I.batched_instances()
    assert len(b) == 64 and all(2.5 <= w.p <= 4.0 and 8 <= w.n <= 40 and 1 <= w.order <= 4 for w in b)
