"""The vector entry points (fe_dot, fe_axpby, fe_pointwise_mul, fe_reciprocal, fe_face_size,
fe_face_add) through the C ABI against numpy on the same inputs."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2506_00746_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _op(dim, n, k, natural=0):
    from paper_2506_00746_gb300 import Operator
    nn = (n,) * dim if isinstance(n, int) else n
    nv = int(np.prod([x + 1 for x in nn]))
    idx = np.indices([x + 1 for x in nn[::-1]]).reshape(dim, -1)[::-1]
    V = np.ascontiguousarray((idx / np.array(nn)[:, None]).T.astype(np.float64))
    assert V.shape == (nv, dim)
    return Operator(dim, nn, k, V, p=3.0, natural_faces=natural)


def test_dot_axpby_mul_reciprocal():
    import torch
    from paper_2506_00746_gb300 import abi
    op = _op(3, (5, 4, 6), 2)
    n = op.n_dofs
    a = I.uniform_vector(n, seed=1)
    b = I.uniform_vector(n, seed=2)
    ad, bd = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    for lo, hi in ((0, n), (17, n - 5), (n // 3, n // 3 + 1), (4, 4)):
        abi.fe_dot(op.ctx, ad, bd, lo, hi, out)
        ref = float(a[lo:hi] @ b[lo:hi])
        assert abs(out.item() - ref) <= 1e-14 * max(1.0, float(np.abs(a[lo:hi] * b[lo:hi]).sum()))
        first = out.item()
        abi.fe_dot(op.ctx, ad, bd, lo, hi, out)
        assert out.item() == first                      # fixed summation order
    with pytest.raises(abi.FeodError):
        abi.fe_dot(op.ctx, ad, bd, 0, n + 1, out)
    y = bd.clone()
    abi.fe_axpby(op.ctx, 0.75, ad, -1.5, y)
    np.testing.assert_allclose(y.cpu().numpy(), 0.75 * a - 1.5 * b, rtol=1e-15, atol=1e-15)
    y = torch.full_like(bd, float("nan"))
    abi.fe_axpby(op.ctx, 2.0, ad, 0.0, y)               # beta 0: y only written
    assert torch.equal(y, 2.0 * ad)
    z = torch.empty_like(ad)
    abi.fe_pointwise_mul(op.ctx, ad, bd, z)
    assert torch.equal(z, ad * bd)
    c = ad.abs() + 0.5
    abi.fe_reciprocal(op.ctx, c, z)
    assert torch.equal(z, 1.0 / c)
    op.close()


@pytest.mark.parametrize("dim,n,k,natural", [(3, (4, 3, 5), 2, 0b010110), (3, (3, 3, 3), 1, 0), (2, (6, 4), 3, 0b1001)])
def test_face_add(dim, n, k, natural):
    import torch
    from paper_2506_00746_gb300 import abi
    op = _op(dim, n, k, natural)
    m = [k * x + 1 for x in n]
    coords = np.indices(m[::-1]).reshape(dim, -1)[::-1]        # lattice coordinates, x fastest
    ess = np.zeros(op.n_dofs, dtype=bool)
    for d in range(dim):
        if not (natural >> (2 * d)) & 1:
            ess |= coords[d] == 0
        if not (natural >> (2 * d + 1)) & 1:
            ess |= coords[d] == m[d] - 1
    assert op.n_free == int((~ess).sum())
    y0 = I.uniform_vector(op.n_dofs, seed=3)
    for face in range(2 * dim):
        ax, side = face // 2, face % 2
        on = coords[ax] == (m[ax] - 1 if side else 0)
        size = abi.fe_face_size(op.ctx, face)
        assert size == int(on.sum())
        buf = I.uniform_vector(size, seed=10 + face)
        y = torch.from_numpy(y0).cuda()
        abi.fe_face_add(op.ctx, face, y, torch.from_numpy(buf).cuda())
        ref = y0.copy()
        g = np.flatnonzero(on)                # the face's DOFs in ascending order = lexicographic
        ref[g] = np.where(ess[g], y0[g], y0[g] + buf)
        assert torch.equal(y.cpu(), torch.from_numpy(ref))
    op.close()
