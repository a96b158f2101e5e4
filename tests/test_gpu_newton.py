"""Newton-CG on the GPU (FP64 and mixed precision), checked by the oracle: the oracle evaluates
||R(u_gpu)|| independently, and the GPU solution matches the oracle's own Newton solution."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_2506_00746_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _setup(w: I.Workload):
    import torch
    from paper_2506_00746_gb300 import Operator
    V = I.lattice_vertices(w.dim, w.n, seed=w.mesh_seed)
    op = Operator(w.dim, w.n, w.order, V, p=w.p, eps=w.eps)
    P = O.Problem(w.dim, w.n, w.order, V, p=w.p, eps=w.eps)
    u0 = I.smooth_field(w.dim, w.n, w.order, seed=w.state_seed)
    return op, P, u0, torch.from_numpy(u0).cuda()


@pytest.mark.parametrize("precision", [64, -32, 32])
def test_newton_2d_config(precision):
    """2D p=3, 16x16 quads, order 2: Newton-CG to 1e-8 in FP64 and mixed precision."""
    w = I.WORKLOADS["2d_p3_k2_16x16"]
    op, P, u0, ud = _setup(w)
    u = ud.clone()
    rep = op.newton_solve(u, rtol=1e-8, inner_precision=precision)
    assert rep["rel"] <= 1e-8
    r0 = np.linalg.norm(O.residual(P, u0))
    ug = u.cpu().numpy()
    assert np.linalg.norm(O.residual(P, ug)) <= 1e-8 * r0 * 1.0001     # the oracle confirms the claim
    u_ref, hist = O.newton(P, u0, rtol=1e-13)
    assert np.linalg.norm(ug - u_ref) <= 1e-6 * np.linalg.norm(u_ref)
    op.close()


@pytest.mark.parametrize("precision", [64, -32, 32])
def test_newton_tight_matches_oracle(precision):
    w = I.Workload("3d_small", 3, 4, 2)
    op, P, u0, ud = _setup(w)
    u = ud.clone()
    rep = op.newton_solve(u, rtol=1e-12, cg_rtol=1e-6, inner_precision=precision)
    assert rep["rel"] <= 1e-12
    u_ref, _ = O.newton(P, u0, rtol=1e-13)
    assert np.linalg.norm(u.cpu().numpy() - u_ref) <= 1e-9 * np.linalg.norm(u_ref)
    op.close()


def test_newton_graph_and_plain_launches_agree():
    """Replaying CG batches as CUDA graphs, and the whole CG as one graph launch with a conditional
    WHILE node, give bitwise the same iterates as plain launches."""
    import torch
    w = I.Workload("3d_small", 3, 3, 3)
    op, P, u0, ud = _setup(w)
    for prec in (32, -32, 64):
        a, b, c = ud.clone(), ud.clone(), ud.clone()
        ra = op.newton_solve(a, inner_precision=prec, use_graph=1)
        rb = op.newton_solve(b, inner_precision=prec, use_graph=0, cg_batch=5)
        rc = op.newton_solve(c, inner_precision=prec, use_graph=2, cg_batch=3)    # device-side loop
        assert torch.equal(a, b) and torch.equal(a, c)
        assert ra["cg_hist"] == rb["cg_hist"] == rc["cg_hist"]
    op.close()


def test_newton_failure_paths():
    """Host-visible failures: iteration limits end the solve with a status, never a hang."""
    from paper_2506_00746_gb300 import FeodError
    w = I.Workload("3d_small", 3, 3, 2)
    op, P, u0, ud = _setup(w)
    u = ud.clone()
    rep = op.newton_solve(u, max_newton=1, raise_on_error=False)
    assert rep["status"] == "FE_ERR_NOT_CONVERGED" and rep["newton_iters"] == 1
    u = ud.clone()
    with pytest.raises(FeodError):
        op.newton_solve(u, max_newton=1)
    op.close()


def test_cg_solve_and_adjoint_homogeneity():
    """lambda solving J(u) lambda = F at the solution equals u/(p-1) (degree p-1 homogeneity)."""
    import torch
    from paper_2506_00746_gb300 import Operator
    dim, n, k, p = 3, 4, 2, 3.0
    V = I.lattice_vertices(dim, n, seed=0)
    rho = I.design_field(dim, n, seed=3)
    op = Operator(dim, n, k, V, p=p, rho=rho)
    u = torch.from_numpy(I.smooth_field(dim, n, k, seed=1)).cuda()
    op.newton_solve(u, rtol=1e-13, cg_rtol=1e-8)
    op.linearize(u)
    F = op.load_vector()
    lam, it = op.cg_solve(F, rtol=1e-13)
    assert it > 0
    assert torch.linalg.norm(lam - u / (p - 1)) <= 1e-9 * torch.linalg.norm(u)
    op.close()


def test_compliance_gradient_against_fd():
    """dc/drho from the autograd adjoint matches central differences on random directions."""
    import torch
    from paper_2506_00746_gb300 import ComplianceFn, Operator
    dim, n, k, p = 2, 6, 2, 3.0
    V = I.lattice_vertices(dim, n, seed=0)
    rho0 = I.design_field(dim, n, seed=3)
    op = Operator(dim, n, k, V, p=p, rho=rho0)
    u0 = torch.from_numpy(I.smooth_field(dim, n, k, seed=1)).cuda()
    kw = {"rtol": 1e-14, "cg_rtol": 1e-10}
    rho = torch.from_numpy(rho0).cuda().requires_grad_(True)
    c = ComplianceFn.apply(rho, op, u0, kw)
    c.backward()
    g = rho.grad.clone()
    # oracle adjoint gradient at the GPU solution
    P = O.Problem(dim, n, k, V, p=p, rho=rho0)
    u_ref, _ = O.newton(P, u0.cpu().numpy(), rtol=1e-14)
    lam = O.adjoint_solve(P, u_ref)
    g_ref = -O.adjoint_grad(P, u_ref, lam)
    assert np.linalg.norm(g.cpu().numpy() - g_ref) <= 1e-8 * np.linalg.norm(g_ref)
    # the objective c = F^T u (fe_compliance) against the oracle's load vector and solution
    F_ref = O.load(P)
    F_ref[O.essential(P)] = 0.0
    assert abs(c.item() - F_ref @ u_ref) <= 1e-10 * abs(F_ref @ u_ref)
    # fe_compliance_gradient scales by the incoming gradient
    from paper_2506_00746_gb300 import abi
    u = u0.clone()
    op.newton_solve(u, **kw)
    g2 = torch.empty_like(g)
    abi.fe_compliance_gradient(op.ctx, u, -0.5, 1e-12, 50000, 64, g2)
    assert torch.linalg.norm(g2 + 0.5 * g) <= 1e-12 * torch.linalg.norm(g)
    rng = np.random.default_rng(4)
    h = 1e-5
    for _ in range(4):
        d = torch.from_numpy(rng.standard_normal(n ** dim)).cuda()
        with torch.no_grad():
            cp = ComplianceFn.apply(rho.detach() + h * d, op, u0, kw)
            cm = ComplianceFn.apply(rho.detach() - h * d, op, u0, kw)
        fd = (cp - cm).item() / (2 * h)
        assert abs(fd - torch.dot(g, d).item()) <= 1e-6 * abs(torch.dot(g, d).item())
    op.close()


def test_cg_solve_fp32_accuracy_and_scaling():
    """FP32 CG: the FP64 operator confirms its solution's residual, and scaling b by 2^s gives
    bitwise 2^s x, also where b's entries lie far outside the FP32 range (the solver works on
    b divided by a power of two near its RMS)."""
    import torch
    w = I.Workload("3d_small", 3, 5, 2)
    op, P, u0, ud = _setup(w)
    op.linearize(ud)
    F = op.load_vector()
    b = -op.residual(ud)
    for rhs in (F, b):
        x, it = op.cg_solve(rhs, rtol=1e-6, precision=32)
        assert it > 0
        res = rhs - op.jacobian_action(x)
        assert torch.linalg.norm(res) <= 1e-5 * torch.linalg.norm(rhs)
        x64, _ = op.cg_solve(rhs, rtol=1e-12, precision=64)
        assert torch.linalg.norm(x - x64) <= 5e-4 * torch.linalg.norm(x64)
        for s in (-140, 150):
            xs, its = op.cg_solve(rhs * 2.0 ** s, rtol=1e-6, precision=32)
            assert its == it
            assert torch.equal(xs, x * 2.0 ** s)
    op.close()


def test_device_wait_timeout_is_reported_and_context_survives():
    """A bounded device wait that nothing completes gives up (about a second), the host reports
    FE_ERR_CUDA, and the same context computes correctly afterwards."""
    import torch
    from paper_2506_00746_gb300 import FeodError, abi
    w = I.Workload("3d_small", 3, 3, 2)
    op, P, u0, ud = _setup(w)
    with pytest.raises(FeodError) as ei:
        abi.fe_selftest_wait_timeout(op.ctx)
    assert ei.value.args and "FE_ERR_CUDA" in str(ei.value)
    op.linearize(ud)
    v = I.uniform_vector(op.n_dofs, seed=2)
    y = op.jacobian_action(torch.from_numpy(v).cuda()).cpu().numpy()
    y_ref = O.jv(P, u0, v)
    assert np.linalg.norm(y - y_ref) <= 1e-12 * np.linalg.norm(y_ref)
    # the word was cleared: fe_check_error finds nothing, a synchronous solve runs normally
    abi.fe_check_error(op.ctx)
    u = ud.clone()
    assert op.newton_solve(u, rtol=1e-8)["status"] == "FE_OK"
    op.close()


@pytest.mark.parametrize("precision", [64, 48, -32, 32])
def test_newton_eisenstat_walker_forcing(precision):
    """forcing 1 (Eisenstat-Walker choice 2): the same 1e-8 solution, confirmed by the oracle's
    residual, with fewer CG iterations in total than the fixed inner tolerance; every inner
    tolerance stays within [1e-6, eta_max], so no CG runs to its iteration limit."""
    import torch
    from paper_2506_00746_gb300 import FeodError, Operator
    V = I.lattice_vertices(3, 8, seed=0)
    op = Operator(3, 8, 3, V, p=3.0)
    P = O.Problem(3, 8, 3, V, p=3.0)
    u0 = I.smooth_field(3, 8, 3, seed=1)
    r0 = np.linalg.norm(O.residual(P, u0))
    reps = {}
    for forcing in (0, 1):
        u = torch.from_numpy(u0).cuda()
        reps[forcing] = op.newton_solve(u, rtol=1e-8, inner_precision=precision, forcing=forcing)
        assert reps[forcing]["status"] == "FE_OK" and reps[forcing]["rel"] <= 1e-8
        assert np.linalg.norm(O.residual(P, u.cpu().numpy())) <= 1e-8 * r0 * 1.01
    assert reps[1]["cg_iters"] < reps[0]["cg_iters"], reps
    with pytest.raises(FeodError):
        op.newton_solve(torch.from_numpy(u0).cuda(), forcing=1, eta_max=1.5)
    with pytest.raises(FeodError):
        op.newton_solve(torch.from_numpy(u0).cuda(), forcing=2)
    op.close()
