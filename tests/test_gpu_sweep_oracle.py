"""Error against the FP64 oracle per order on the order-sweep workloads: 3D p-Laplacian p = 3,
orders 1-6 on jittered hex lattices of about 8M DOFs (k n ~ 200), seeded smooth state and U[-1,1]
direction.  Per order, over the whole vector:
  * the FP64 residual against the oracle's R(u) (<= 1e-12 relative);
  * the FP64 and double-float Jacobian actions against the oracle's J(u) v (<= 1e-12 relative);
  * the FP32 action against the oracle's J(u) v at the same FP32-rounded direction (<= 1e-5);
  * the mixed-precision Newton solve (FP32 J v inside an FP64 CG): the oracle evaluates the
    residual of the GPU's solution and confirms ||R(u)|| <= 1e-8 ||R(u_0)||.
Each case prints one JSON line with the measured errors (pytest -s shows them)."""
from __future__ import annotations

import json

import numpy as np
import pytest

import oracle as O
from paper_2506_00746_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SWEEP = [(1, 199), (2, 100), (3, 66), (4, 50), (5, 40), (6, 33)]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("k,n", SWEEP)
def test_sweep_order_against_oracle(k, n):
    import torch
    from paper_2506_00746_gb300 import Operator
    V = I.lattice_vertices(3, n, seed=0)
    op = Operator(3, n, k, V, p=3.0)
    u0 = I.smooth_field(3, n, k, seed=1)
    v = I.uniform_vector(op.n_dofs, seed=2)
    ud, vd = torch.from_numpy(u0).cuda(), torch.from_numpy(v).cuda()
    r_gpu = op.residual(ud).cpu().numpy()
    op.linearize(ud)
    y64 = op.jacobian_action(vd, precision=64).cpu().numpy()
    y48 = op.jacobian_action(vd, precision=48).cpu().numpy()
    v32 = vd.float()
    y32 = op.jacobian_action(v32, precision=32).double().cpu().numpy()
    u = ud.clone()
    rep = op.newton_solve(u, rtol=1e-8, inner_precision=-32)
    uh = u.cpu().numpy()
    op.close()

    P = O.Problem(3, n, k, V, p=3.0)
    y_ref = O.jv(P, u0, v)
    y32_ref = O.jv(P, u0, v32.double().cpu().numpy())
    r_ref = O.residual(P, u0)
    r0 = float(np.linalg.norm(r_ref))
    r = float(np.linalg.norm(O.residual(P, uh)))
    out = {"order": k, "n": n, "n_dofs": int(P.n_dofs), "residual_rel_err": _rel(r_gpu, r_ref),
           "jv_f64_rel_err": _rel(y64, y_ref),
           "jv_double_float_rel_err": _rel(y48, y_ref), "jv_f32_rel_err": _rel(y32, y32_ref),
           "newton_mixed_steps": rep["newton_iters"], "newton_mixed_cg": rep["cg_iters"],
           "newton_mixed_rel_residual_gpu": rep["rel"], "newton_mixed_rel_residual_oracle": r / r0}
    print(json.dumps(out))
    assert out["residual_rel_err"] <= 1e-12
    assert out["jv_f64_rel_err"] <= 1e-12
    assert out["jv_double_float_rel_err"] <= 1e-12
    assert out["jv_f32_rel_err"] <= 1e-5
    assert rep["status"] == "FE_OK" and rep["rel"] <= 1e-8
    assert out["newton_mixed_rel_residual_oracle"] <= 1e-8 * 1.01
