"""Subdomains: lattices of n[0] x n[1] x n[2] elements whose interface faces are natural (not
essential), the building block of the subdomain restriction P (Fig. 1) when one problem is split
across ranks.

A box of elements cut out of a cube problem is set up on its own (the cube's vertices of that box,
natural faces where the box meets the rest of the cube).  Its residual and Jacobian action must
equal the oracle's sums over the box's elements (the cube problem's element-range sums, the
direction's essential entries masked), restricted to the box's DOFs, with the Dirichlet
convention on the faces the box shares with the cube's boundary.  Two slabs that split the cube
must add up, on their interface plane, to the single-domain action.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_2506_00746_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _box_dofs(n, k, lo, hi):
    """Global DOF numbers (cube lattice (k n + 1)^3) of the box of elements [lo, hi) in local
    lexicographic order, and the box's DOF lattice shape."""
    m = k * n + 1
    rng = [np.arange(k * lo[d], k * hi[d] + 1) for d in range(3)]
    gz, gy, gx = np.meshgrid(rng[2], rng[1], rng[0], indexing="ij")
    return (gx + m * (gy + m * gz)).ravel(), tuple(len(r) for r in rng)


def _box_vertices(V, n, lo, hi):
    nv = n + 1
    idx = [np.arange(lo[d], hi[d] + 1) for d in range(3)]
    gz, gy, gx = np.meshgrid(idx[2], idx[1], idx[0], indexing="ij")
    return np.ascontiguousarray(V[(gx + nv * (gy + nv * gz)).ravel()])


def _natural(n, lo, hi):
    mask = 0
    for d in range(3):
        if lo[d] > 0:
            mask |= 1 << (2 * d)
        if hi[d] < n:
            mask |= 1 << (2 * d + 1)
    return mask


def _box_reference(P, u, v, n, lo, hi):
    """Oracle sums over the box's elements of r_e and K_e v_e (v's cube-essential entries zero)."""
    vm = v.copy()
    vm[O.essential(P)] = 0.0
    y = np.zeros(P.n_dofs)
    r = np.zeros(P.n_dofs)
    for ez in range(lo[2], hi[2]):
        for ey in range(lo[1], hi[1]):
            e0 = lo[0] + n * (ey + n * ez)
            e1 = hi[0] + n * (ey + n * ez)
            O.jv_partial(P, u, vm, e0, e1, y)
            O.residual_partial(P, u, e0, e1, r)
    return r, y


@pytest.mark.parametrize("n,k,lo,hi", [
    (6, 2, (0, 0, 0), (6, 6, 3)),       # bottom z-slab (natural z+)
    (6, 2, (0, 0, 3), (6, 6, 6)),       # top z-slab (natural z-)
    (7, 3, (2, 1, 0), (7, 5, 4)),       # interior box, ragged tiles, natural on four faces
    (5, 1, (1, 0, 1), (4, 5, 5)),       # order 1
])
def test_box_of_a_cube_against_oracle(n, k, lo, hi):
    import torch
    from paper_2506_00746_gb300 import Operator
    V = I.lattice_vertices(3, n, seed=0)
    P = O.Problem(3, n, k, V, p=3.0)
    u = I.smooth_field(3, n, k, seed=1)
    v = I.uniform_vector(P.n_dofs, seed=2)
    dofs, shape = _box_dofs(n, k, lo, hi)
    nb = tuple(hi[d] - lo[d] for d in range(3))
    op = Operator(3, nb, k, _box_vertices(V, n, lo, hi), p=3.0, natural_faces=_natural(n, lo, hi))
    assert op.n_dofs == len(dofs) and op.n_elements == nb[0] * nb[1] * nb[2]
    ess_cube = O.essential(P)[dofs]
    r_all, y_all = _box_reference(P, u, v, n, lo, hi)
    r_ref = np.where(ess_cube, 0.0, r_all[dofs])
    y_ref = np.where(ess_cube, v[dofs], y_all[dofs])
    ub = torch.from_numpy(u[dofs]).cuda()
    vb = torch.from_numpy(v[dofs]).cuda()
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert op.n_free == int((~ess_cube).sum())
    assert rel(op.residual(ub).cpu().numpy(), r_ref) <= 1e-12
    op.linearize(ub)
    assert rel(op.jacobian_action(vb, precision=64).cpu().numpy(), y_ref) <= 1e-12
    assert rel(op.jacobian_action(vb, precision=48).cpu().numpy(), y_ref) <= 1e-12
    assert rel(op.jacobian_action(vb, u=ub, precision=64).cpu().numpy(), y_ref) <= 1e-12
    # FP32: against the oracle's sums of the FP32-rounded direction
    v32 = v.astype(np.float32).astype(np.float64)
    _, y32_all = _box_reference(P, u, v32, n, lo, hi)
    y32_ref = np.where(ess_cube, v32[dofs], y32_all[dofs])
    y32 = op.jacobian_action(vb.float(), precision=32).double().cpu().numpy()
    assert rel(y32, y32_ref) <= 1e-5
    op.close()


def test_two_slabs_add_up_to_the_single_domain_action():
    """Slabs [0, 3) and [3, 6) in z: each slab's action on its own DOFs, the two summed on the
    interface plane's free DOFs, equals the single-domain action everywhere."""
    import torch
    from paper_2506_00746_gb300 import Operator
    n, k = 6, 3
    V = I.lattice_vertices(3, n, seed=0)
    u = I.smooth_field(3, n, k, seed=1)
    v = I.uniform_vector((k * n + 1) ** 3, seed=2)
    full = Operator(3, n, k, V, p=3.0)
    full.linearize(torch.from_numpy(u).cuda())
    y_full = full.jacobian_action(torch.from_numpy(v).cuda(), precision=64).cpu().numpy()
    full.close()
    y = np.zeros_like(v)
    plane = None
    for lo, hi in (((0, 0, 0), (6, 6, 3)), ((0, 0, 3), (6, 6, 6))):
        dofs, _ = _box_dofs(n, k, lo, hi)
        op = Operator(3, (6, 6, 3), k, _box_vertices(V, n, lo, hi), p=3.0, natural_faces=_natural(n, lo, hi))
        op.linearize(torch.from_numpy(u[dofs]).cuda())
        yb = op.jacobian_action(torch.from_numpy(v[dofs]).cuda(), precision=64).cpu().numpy()
        op.close()
        m = k * n + 1
        on_plane = (dofs // (m * m)) == k * 3
        if plane is None:
            plane = dofs[on_plane]
            y[dofs] = yb
        else:
            # interface plane: essential entries keep v, free entries take the sum of both slabs
            ess = O.essential(O.Problem(3, n, k, V))[plane]
            y[plane] = np.where(ess, yb[on_plane], y[plane] + yb[on_plane])
            y[dofs[~on_plane]] = yb[~on_plane]
    assert np.linalg.norm(y - y_full) <= 1e-13 * np.linalg.norm(y_full)
