"""The double-float operator (precision 48: FP32 word pairs on the FP32 pipes, FP64 vectors)
against the oracle.

Each double-float operation errs by a small multiple of 2^-48 relative to its operands, the kind of
bound one FP64 operation has with 2^-53, so the Jacobian action is held to the FP64 tolerance
(relative 2-norm error <= 1e-12 with a random direction v).  The CG and Newton modes built on it
are checked by FP64 residuals and the oracle's residual.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_2506_00746_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _setup(dim, n, k, p=3.0, tile_kernel=True, rho=False):
    import torch
    from paper_2506_00746_gb300 import Operator
    V = I.lattice_vertices(dim, n, seed=0)
    r = I.design_field(dim, n, seed=3) if rho else None
    op = Operator(dim, n, k, V, p=p, rho=r, tile_kernel=tile_kernel)
    P = O.Problem(dim, n, k, V, p=p, rho=r)
    u = I.smooth_field(dim, n, k, seed=1)
    v = I.uniform_vector(P.n_dofs, seed=2)
    return op, P, u, v, torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda()


# 2D and 3D, orders 1..6, ragged tiles, a single element; the 3D default tiles run the tile kernel
CASES = [(2, 16, 2), (2, 1, 1), (2, 9, 1), (2, 7, 3), (2, 4, 5), (2, 3, 6), (3, 1, 1), (3, 5, 1), (3, 4, 2),
         (3, 3, 3), (3, 5, 3), (3, 3, 4), (3, 3, 5), (3, 2, 6)]


@pytest.mark.parametrize("dim,n,k", CASES)
def test_double_float_jacobian_parity(dim, n, k):
    import torch
    op, P, u, v, ud, vd = _setup(dim, n, k)
    op.linearize(ud)
    y_ref = O.jv(P, u, v)
    y48 = op.jacobian_action(vd, precision=48)
    assert y48.dtype == torch.float64
    e48 = _rel(y48.cpu().numpy(), y_ref)
    assert e48 <= TOL64
    # far closer to the exact action than the FP32 operator
    e32 = _rel(op.jacobian_action(vd, precision=-32).cpu().numpy(), y_ref)
    assert e48 <= 1e-4 * e32
    assert torch.equal(op.jacobian_action(vd, precision=48), y48)          # deterministic
    op.close()


@pytest.mark.parametrize("n,k", [(7, 1), (5, 2), (6, 3), (4, 4), (3, 5), (2, 6)])
def test_double_float_tile_and_per_element_kernels(n, k):
    """The tile-level and the per-element double-float kernels both meet the FP64 tolerance and
    agree with each other to double-float rounding."""
    outs = []
    for tile_kernel in (True, False):
        op, P, u, v, ud, vd = _setup(3, n, k, tile_kernel=tile_kernel)
        op.linearize(ud)
        y = op.jacobian_action(vd, precision=48).cpu().numpy()
        assert _rel(y, O.jv(P, u, v)) <= TOL64
        outs.append(y)
        op.close()
    assert _rel(outs[0], outs[1]) <= 1e-13


def test_double_float_smooth_direction():
    """A smooth v makes J v a cancellation (the FP32 operator loses about (k n)^2 relative); the
    double-float operator keeps FP64-class accuracy."""
    import torch
    dim, n, k = 3, 6, 3
    op, P, u, _, ud, _ = _setup(dim, n, k)
    w = I.smooth_field(dim, n, k, seed=7)
    op.linearize(ud)
    y_ref = O.jv(P, u, w)
    wd = torch.from_numpy(w).cuda()
    e48 = _rel(op.jacobian_action(wd, precision=48).cpu().numpy(), y_ref)
    e64 = _rel(op.jacobian_action(wd, precision=64).cpu().numpy(), y_ref)
    e32 = _rel(op.jacobian_action(wd, precision=-32).cpu().numpy(), y_ref)
    assert e48 <= 1e-11 and e48 <= 1e-4 * e32, (e48, e64, e32)
    op.close()


def test_double_float_follows_relinearisation_and_design():
    """The double-float tangent is re-split after every change of the FP64 one."""
    import torch
    dim, n, k = 3, 3, 2
    op, P, u, v, ud, vd = _setup(dim, n, k, rho=True)
    op.linearize(ud)
    op.jacobian_action(vd, precision=48)
    u2 = I.smooth_field(dim, n, k, seed=11)
    op.linearize(torch.from_numpy(u2).cuda())
    assert _rel(op.jacobian_action(vd, precision=48).cpu().numpy(), O.jv(P, u2, v)) <= TOL64
    rho2 = I.design_field(dim, n, seed=12)
    op.set_design(torch.from_numpy(rho2).cuda())
    from paper_2506_00746_gb300 import FeodError
    with pytest.raises(FeodError):                    # the design change dropped the linearisation
        op.jacobian_action(vd, precision=48)
    op.linearize(ud)
    P2 = O.Problem(dim, n, k, I.lattice_vertices(dim, n, seed=0), p=3.0, rho=rho2)
    assert _rel(op.jacobian_action(vd, precision=48).cpu().numpy(), O.jv(P2, u, v)) <= TOL64
    op.close()


def test_double_float_rejects_stateless_and_noalloc():
    import ctypes

    import torch
    from paper_2506_00746_gb300 import FeodError, abi
    op, P, u, v, ud, vd = _setup(3, 2, 2)
    op.linearize(ud)
    with pytest.raises(FeodError):
        op.jacobian_action(vd, u=ud, precision=48)
    y = torch.empty_like(vd)
    lib = abi.library()
    st = lib.fe_jacobian_action_noalloc(op.ctx, ctypes.c_void_p(vd.data_ptr()), ctypes.c_void_p(y.data_ptr()), 48,
                                        None)
    assert abi.STATUS_NAMES[st] == "FE_ERR_ARG"
    # the context stays usable
    assert _rel(op.jacobian_action(vd, precision=48).cpu().numpy(), O.jv(P, u, v)) <= TOL64
    op.close()


def test_double_float_cg_solve_and_scaling():
    """CG with the double-float operator reaches an FP64-class relative residual (checked with the
    FP64 operator), and the power-of-two right-hand-side scaling makes the solve for b / 2^100
    exactly the solve for b, scaled."""
    import torch
    op, P, u, v, ud, vd = _setup(3, 5, 2)
    op.linearize(ud)
    b = vd.clone()
    x, it = op.cg_solve(b, rtol=1e-11, precision=48)
    r = b - op.jacobian_action(x, precision=64)
    assert torch.linalg.norm(r) <= 1e-10 * torch.linalg.norm(b), it
    x64, it64 = op.cg_solve(b, rtol=1e-11, precision=64)
    assert abs(it - it64) <= max(2, it64 // 20)
    assert torch.linalg.norm(x - x64) <= 1e-9 * torch.linalg.norm(x64)
    s = 2.0 ** -100
    xs, its = op.cg_solve(b * s, rtol=1e-11, precision=48)
    assert its == it and torch.equal(xs, x * s)
    op.close()


@pytest.mark.parametrize("dim,n,k", [(2, 12, 2), (3, 6, 3)])
def test_double_float_newton_matches_oracle(dim, n, k):
    import torch
    from paper_2506_00746_gb300 import Operator
    V = I.lattice_vertices(dim, n, seed=0)
    P = O.Problem(dim, n, k, V, p=3.0)
    u0 = I.smooth_field(dim, n, k, seed=1)
    r0 = np.linalg.norm(O.residual(P, u0))
    reps = {}
    for prec in (64, 48):
        op = Operator(dim, n, k, V, p=3.0)
        u = torch.from_numpy(u0).cuda()
        reps[prec] = op.newton_solve(u, rtol=1e-10, inner_precision=prec)
        assert reps[prec]["status"] == "FE_OK"
        assert np.linalg.norm(O.residual(P, u.cpu().numpy())) <= 1e-10 * r0 * 1.01
        op.close()
    assert reps[48]["newton_iters"] == reps[64]["newton_iters"]
    assert abs(reps[48]["cg_iters"] - reps[64]["cg_iters"]) <= max(3, reps[64]["cg_iters"] // 50)
