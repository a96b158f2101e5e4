"""Element tangent matrices K_e = B^T J_D B (Eq. 3) formed three ways on the GPU -- the law's tangent
by hand (HND), forward AD at the quadrature point (RES), forward AD at the element level (ELM) --
each against the oracle's element matrices (hand-derived tangent, dense tables, FP64)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_2506_00746_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("order,p,design", [(1, 3.0, False), (2, 2.5, True), (3, 4.0, False), (3, 3.0, True)])
def test_element_matrices_match_oracle(order, p, design):
    import torch
    from paper_2506_00746_gb300 import Operator
    n = 3
    V = I.lattice_vertices(3, n, seed=0)
    rho = I.design_field(3, n, seed=3) if design else None
    op = Operator(3, n, order, V, p=p, rho=rho)
    u = I.smooth_field(3, n, order, seed=1)
    ud = torch.from_numpy(u).cuda()
    P = O.Problem(3, n, order, V, p=p, rho=rho)
    K_ref, _, _ = O.element_matrices(P, u)
    Ks = {}
    for method in ("hnd", "res", "elm"):
        K = op.element_matrices(ud, method).cpu().numpy()
        assert K.shape == K_ref.shape
        assert np.linalg.norm(K - K_ref) <= 1e-12 * np.linalg.norm(K_ref), method
        Ks[method] = K
    # a sub-range of elements gives the same rows as the full call
    part = op.element_matrices(ud, "elm", e0=5, count=7).cpu().numpy()
    np.testing.assert_array_equal(part, Ks["elm"][5:12])
    op.close()


def test_element_matrices_rejects():
    import torch
    from paper_2506_00746_gb300 import FeodError, Operator
    op = Operator(3, 2, 4, I.lattice_vertices(3, 2, seed=0))
    u = torch.zeros(op.n_dofs, dtype=torch.float64, device="cuda")
    with pytest.raises(FeodError):
        op.element_matrices(u, "res")           # order 4: not compiled for this experiment
    op.close()
    op = Operator(3, 2, 1, I.lattice_vertices(3, 2, seed=0))
    u = torch.zeros(op.n_dofs, dtype=torch.float64, device="cuda")
    with pytest.raises(FeodError):
        op.element_matrices(u, "res", e0=7, count=2)   # past the last element
    op.close()
