"""The Jacobian action on host buffers (fe_jacobian_action_host).  For 3D problems with several tile
layers it runs in z-chunks whose copies overlap the kernels; the result must be the device
action's, bit for bit, in every precision, and match the oracle within the usual tolerances.
Cases: ragged last tile layers, fewer and more tile layers than chunks, one-element tiles, pinned
and pageable host memory, and the one-piece path (2D, a single tile layer)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_2506_00746_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 48: 1e-12, 32: 1e-5, -32: 1e-5}


@pytest.mark.parametrize("dim,n,k", [(3, 5, 3), (3, 16, 2), (3, 40, 1), (3, 6, 4), (3, 3, 6), (3, 2, 3), (2, 9, 2)])
def test_host_action_equals_device_action(dim, n, k):
    import torch
    from paper_2506_00746_gb300 import Operator
    V = I.lattice_vertices(dim, n, seed=0)
    u = I.smooth_field(dim, n, k, seed=1)
    op = Operator(dim, n, k, V, p=3.0)
    P = O.Problem(dim, n, k, V, p=3.0)
    op.linearize(torch.from_numpy(u).cuda())
    v = I.uniform_vector(op.n_dofs, seed=2)
    ref64 = O.jv(P, u, v)
    ref32 = O.jv(P, u, v.astype(np.float32).astype(np.float64))
    for precision in (64, 48, 32, -32):
        dtype = torch.float32 if precision == 32 else torch.float64
        vd = torch.from_numpy(v).cuda().to(dtype)
        y_dev = op.jacobian_action(vd, precision=precision).cpu()
        for pinned in (True, False):
            vh = vd.cpu()
            yh = torch.full_like(vh, float("nan"))
            if pinned:
                vh, yh = vh.pin_memory(), yh.pin_memory()
            for _ in range(2):                       # twice in a row on the same buffers
                op.jacobian_action_host(vh, yh, precision=precision)
                assert torch.equal(yh, y_dev), (precision, pinned)
        ref = ref32 if precision in (32, -32) else ref64
        got = y_dev.double().numpy()
        assert np.linalg.norm(got - ref) <= TOL[precision] * np.linalg.norm(ref), precision
    op.close()
