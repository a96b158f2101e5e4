"""Parity of the CUDA path (through the C ABI) with the oracle, on seeded inputs.

Tolerances (relative, vector 2-norm over all DOFs): FP64 results <= 1e-12; FP32 Jacobian actions
<= 1e-5 with a random direction v.  Cases span several tiles, ragged last tiles, a single element,
orders 1-6 in 2D and 3D, p in {2, 2.5, 3, 4}, eps > 0 and a design field.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_2506_00746_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _case(dim, n, k, p=3.0, eps=0.0, rho=False, tile=0, f_kind=0, seed=0):
    import torch
    from paper_2506_00746_gb300 import Operator
    V = I.lattice_vertices(dim, n, seed=seed)
    r = I.design_field(dim, n, seed=3) if rho else None
    op = Operator(dim, n, k, V, p=p, eps=eps, rho=r, tile=tile, f_kind=f_kind)
    P = O.Problem(dim, n, k, V, p=p, eps=eps, rho=r, f_kind=f_kind)
    u = I.smooth_field(dim, n, k, seed=1)
    v = I.uniform_vector(P.n_dofs, seed=2)
    return op, P, u, v, torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda()


CASES_3D = [(3, 1, 1), (3, 2, 1), (3, 5, 1), (3, 3, 2), (3, 4, 2), (3, 3, 3), (3, 5, 3), (3, 2, 4), (3, 3, 4),
            (3, 2, 5), (3, 3, 5), (3, 2, 6)]
CASES_2D = [(2, 16, 2), (2, 1, 1), (2, 9, 1), (2, 7, 3), (2, 5, 4), (2, 4, 5), (2, 3, 6)]


@pytest.mark.parametrize("dim,n,k", CASES_2D + CASES_3D)
def test_residual_and_jacobian_parity(dim, n, k):
    import torch
    op, P, u, v, ud, vd = _case(dim, n, k)
    assert _rel(op.residual(ud).cpu().numpy(), O.residual(P, u)) <= TOL64
    op.linearize(ud)
    y_ref = O.jv(P, u, v)
    assert _rel(op.jacobian_action(vd, precision=64).cpu().numpy(), y_ref) <= TOL64
    assert _rel(op.jacobian_action(vd, u=ud, precision=64).cpu().numpy(), y_ref) <= TOL64
    v32 = vd.float()
    y_ref32 = O.jv(P, u, v32.double().cpu().numpy())
    y32 = op.jacobian_action(v32, precision=32)
    assert _rel(y32.double().cpu().numpy(), y_ref32) <= TOL32
    # the mixed-precision CG operator (double vectors, FP32 arithmetic) is the same computation
    y32d = op.jacobian_action(v32.double(), precision=-32)
    assert torch.equal(y32d, y32.double())
    assert _rel(op.jacobian_action(v32, u=ud, precision=32).double().cpu().numpy(), y_ref32) <= TOL32
    op.close()


@pytest.mark.parametrize("dim,n,k", [(2, 16, 2), (2, 5, 4), (3, 3, 2), (3, 5, 3), (3, 2, 5)])
def test_diagonal_load_coords(dim, n, k):
    op, P, u, v, ud, vd = _case(dim, n, k)
    op.linearize(ud)
    J, _ = O.assemble(P, u)
    assert _rel(op.jacobian_diagonal().cpu().numpy(), J.diagonal()) <= TOL64
    F = O.load(P)
    F[O.essential(P)] = 0.0
    assert _rel(op.load_vector().cpu().numpy(), F) <= TOL64
    np.testing.assert_allclose(op.node_coords().cpu().numpy(), O.node_coords(P), rtol=0, atol=1e-15)
    op.close()


@pytest.mark.parametrize("p,eps", [(2.0, 0.0), (2.5, 0.0), (4.0, 0.0), (3.0, 1e-2), (1.5, 0.5), (3.7, 1e-3)])
@pytest.mark.parametrize("dim,n,k", [(2, 6, 2), (3, 3, 3)])
def test_laws(dim, n, k, p, eps):
    op, P, u, v, ud, vd = _case(dim, n, k, p=p, eps=eps)
    assert _rel(op.residual(ud).cpu().numpy(), O.residual(P, u)) <= TOL64
    op.linearize(ud)
    assert _rel(op.jacobian_action(vd, precision=64).cpu().numpy(), O.jv(P, u, v)) <= TOL64
    op.close()


@pytest.mark.parametrize("dim,n,k", [(2, 6, 2), (3, 3, 2), (3, 4, 3)])
def test_design_field_and_vjp(dim, n, k):
    op, P, u, v, ud, vd = _case(dim, n, k, rho=True)
    assert _rel(op.residual(ud).cpu().numpy(), O.residual(P, u)) <= TOL64
    op.linearize(ud)
    assert _rel(op.jacobian_action(vd, precision=64).cpu().numpy(), O.jv(P, u, v)) <= TOL64
    lam = I.uniform_vector(P.n_dofs, seed=9)
    import torch
    g = op.adjoint_vjp(ud, torch.from_numpy(lam).cuda()).cpu().numpy()
    assert _rel(g, O.adjoint_grad(P, u, lam)) <= TOL64
    op.close()


@pytest.mark.parametrize("tile", [1, 2, 3, 4])
def test_tile_shapes_agree(tile):
    """Every tile size (and so every halo pattern) gives the oracle's result."""
    op, P, u, v, ud, vd = _case(3, 7, 2, tile=tile)
    assert _rel(op.residual(ud).cpu().numpy(), O.residual(P, u)) <= TOL64
    op.linearize(ud)
    assert _rel(op.jacobian_action(vd, precision=64).cpu().numpy(), O.jv(P, u, v)) <= TOL64
    op.close()


@pytest.mark.parametrize("n,k", [(7, 1), (5, 2), (6, 3), (3, 3), (4, 4), (3, 5), (2, 6)])
def test_tile_and_per_element_jacobian_kernels(n, k):
    """The tile-level J v (sum factorisation over the whole tile) and the per-element J v (per
    element, staged in-tile G^T) both match the oracle."""
    import torch
    from paper_2506_00746_gb300 import Operator
    V = I.lattice_vertices(3, n, seed=0)
    P = O.Problem(3, n, k, V, p=3.0)
    u = I.smooth_field(3, n, k, seed=1)
    v = I.uniform_vector(P.n_dofs, seed=2)
    ud, vd = torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda()
    y_ref = O.jv(P, u, v)
    v32 = vd.float()
    y_ref32 = O.jv(P, u, v32.double().cpu().numpy())
    outs = []
    for tile_kernel in (True, False):
        op = Operator(3, n, k, V, p=3.0, tile_kernel=tile_kernel)
        op.linearize(ud)
        y64 = op.jacobian_action(vd, precision=64).cpu().numpy()
        y32 = op.jacobian_action(v32, precision=32).double().cpu().numpy()
        y32d = op.jacobian_action(v32.double(), precision=-32).cpu().numpy()
        assert _rel(y64, y_ref) <= TOL64
        assert _rel(y32, y_ref32) <= TOL32
        np.testing.assert_array_equal(y32d, y32)
        outs.append((y64, y32))
        op.close()
    assert _rel(outs[0][0], outs[1][0]) <= 1e-14
    assert _rel(outs[0][1], outs[1][1]) <= 1e-6


@pytest.mark.parametrize("n,k,p,eps,rho", [(7, 1, 3.0, 0.0, False), (5, 2, 2.5, 0.0, True), (5, 3, 3.0, 0.0, False),
                                           (3, 3, 1.5, 0.5, True), (4, 4, 4.0, 0.0, False), (3, 5, 3.7, 1e-3, False),
                                           (2, 6, 3.0, 0.0, True)])
def test_tile_and_per_element_residual_kernels(n, k, p, eps, rho):
    """The tile-level residual / tangent kernel (collocated stages, flux and dual tangent at each
    point) and the per-element one both match the oracle: R(u) alone, the tangent alone (through
    the cached FP64 and FP32 J v), and R with the tangent in one pass (Newton's fused call, through
    the FP32 J v it leaves cached).  Ragged last tiles (n not a multiple of the tile edge), the
    design factor and the generic power law are covered."""
    import torch
    from paper_2506_00746_gb300 import Operator
    V = I.lattice_vertices(3, n, seed=0)
    r = I.design_field(3, n, seed=3) if rho else None
    P = O.Problem(3, n, k, V, p=p, eps=eps, rho=r)
    u = I.smooth_field(3, n, k, seed=1)
    v = I.uniform_vector(P.n_dofs, seed=2)
    ud, vd = torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda()
    r_ref, y_ref = O.residual(P, u), O.jv(P, u, v)
    y_ref32 = O.jv(P, u, vd.float().double().cpu().numpy())
    outs = []
    for tile_kernel in (True, False):
        op = Operator(3, n, k, V, p=p, eps=eps, rho=r, tile_kernel=tile_kernel)
        res = op.residual(ud).cpu().numpy()
        assert _rel(res, r_ref) <= TOL64
        op.linearize(ud)
        y64 = op.jacobian_action(vd, precision=64).cpu().numpy()
        assert _rel(y64, y_ref) <= TOL64
        assert _rel(op.jacobian_action(vd.float(), precision=32).double().cpu().numpy(), y_ref32) <= TOL32
        # the fused residual + FP32 tangent of the mixed Newton step: one Newton step from u runs
        # it at u first; its reported initial residual norm is ||R(u)||
        w = ud.clone()
        rep = op.newton_solve(w, rtol=1e-30, max_newton=1, inner_precision=32, raise_on_error=False)
        assert abs(rep["r0"] - np.linalg.norm(r_ref)) <= 1e-12 * np.linalg.norm(r_ref)
        outs.append((res, y64))
        op.close()
    assert _rel(outs[0][0], outs[1][0]) <= 1e-13
    assert _rel(outs[0][1], outs[1][1]) <= 1e-13


def test_bitwise_reproducible():
    import torch
    op, P, u, v, ud, vd = _case(3, 6, 3)
    op.linearize(ud)
    a = op.jacobian_action(vd.float(), precision=32).clone()
    b = op.jacobian_action(vd.float(), precision=32).clone()
    assert torch.equal(a, b)
    r1 = op.residual(ud).clone()
    r2 = op.residual(ud).clone()
    assert torch.equal(r1, r2)
    op.close()


def test_zero_state_and_patch():
    """R(0) = -F; a linear field built from the library's own node coordinates passes the patch test."""
    import torch
    from paper_2506_00746_gb300 import Operator
    V = I.lattice_vertices(3, 4, seed=5)
    op = Operator(3, 4, 3, V, p=3.0, f_const=0.0)
    x = op.node_coords()
    a = torch.tensor([0.3, -0.7, 0.5], dtype=torch.float64, device=x.device)
    u = (x @ a + 0.2).contiguous()
    r = op.residual(u)
    assert r.abs().max().item() < 1e-13
    op.close()
    op, P, u, v, ud, vd = _case(3, 3, 2)
    r0 = op.residual(torch.zeros_like(ud)).cpu().numpy()
    F = O.load(P); F[O.essential(P)] = 0.0
    assert _rel(-r0, F) <= TOL64
    op.close()


def test_state_errors():
    import torch
    from paper_2506_00746_gb300 import FeodError
    op, P, u, v, ud, vd = _case(2, 4, 2)
    with pytest.raises(FeodError) as e:
        op.jacobian_action(vd, precision=64)          # nothing cached yet
    assert e.value.status == 9
    with pytest.raises(FeodError):
        op.adjoint_vjp(ud, vd)                        # no design field
    with pytest.raises(ValueError):
        op.residual(ud.float())
    op.close()


def test_inverted_element_is_rejected():
    from paper_2506_00746_gb300 import FeodError, Operator
    V = I.lattice_vertices(2, 3, jitter=0.0)
    V[5] = V[10] + np.array([0.2, 0.2])     # interior vertex (1,1) pushed past vertex (2,2)
    with pytest.raises(FeodError) as e:
        Operator(2, 3, 2, V, p=3.0)
    assert e.value.status == 2
