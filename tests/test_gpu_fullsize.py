"""Full-size parity: the 3D p=3 order-3 problem on 64^3 hexes (7,189,057 DOFs), in the launch
configuration the benchmark times.  The oracle computes sampled entries one by one from the
element-level definition (sum over the elements that contain the sampled DOF)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_2506_00746_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _elements_of(dof, n, k):
    """Elements (lexicographic) containing a global DOF of the (k n + 1)^3 lattice."""
    m = k * n + 1
    g = [dof % m, (dof // m) % m, dof // (m * m)]
    cands = []
    for d in range(3):
        c = []
        e = g[d] // k
        if g[d] % k == 0 and e >= 1:
            c.append(e - 1)
        if e < n:
            c.append(e)
        cands.append(c)
    return [ex + n * (ey + n * ez) for ez in cands[2] for ey in cands[1] for ex in cands[0]]


def _sampled(P, u, v, dofs, n, k):
    """Oracle values of R(u) and J(u) v at the sampled (free) DOFs."""
    vm = v.copy()
    vm[O.essential(P)] = 0.0
    elems = sorted({e for g in dofs for e in _elements_of(g, n, k)})
    re, ye, edofs = O.element_vectors(P, u, vm, elems)
    R = {g: 0.0 for g in dofs}; Y = {g: 0.0 for g in dofs}
    for i in range(len(elems)):
        for l, g in enumerate(edofs[i]):
            if g in R:
                R[g] += re[i, l]; Y[g] += ye[i, l]
    return np.array([R[g] for g in dofs]), np.array([Y[g] for g in dofs])


def test_config2_sampled_parity():
    import torch
    from paper_2506_00746_gb300 import Operator
    w = I.WORKLOADS["3d_p3_k3_64"]
    V = I.lattice_vertices(3, w.n, seed=w.mesh_seed)
    op = Operator(3, w.n, w.order, V, p=w.p)
    assert op.n_dofs == 7_189_057
    u = I.smooth_field(3, w.n, w.order, seed=w.state_seed)
    v = I.uniform_vector(op.n_dofs, seed=w.dir_seed)
    ud, vd = torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda()
    r = op.residual(ud).cpu().numpy()
    op.linearize(ud)
    y64 = op.jacobian_action(vd, precision=64).cpu().numpy()
    y48 = op.jacobian_action(vd, precision=48).cpu().numpy()
    v32 = vd.float()
    y32 = op.jacobian_action(v32, precision=32).double().cpu().numpy()
    P = O.Problem(3, w.n, w.order, V, p=w.p)
    ess = O.essential(P)
    rng = np.random.default_rng(7)
    free = np.flatnonzero(~ess)
    # random free DOFs plus the corners of tiles (DOFs shared by up to 8 elements) and a face
    m = w.order * w.n + 1
    tile_corner = [(6 + 6 * m + 6 * m * m), (12 + 12 * m + 12 * m * m), (96 + 96 * m + 96 * m * m)]
    dofs = sorted(set(rng.choice(free, 48, replace=False).tolist() + tile_corner + [m * m * 5 + m * 7 + 1]))
    R_ref, Y_ref = _sampled(P, u, v, dofs, w.n, w.order)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(r[dofs], R_ref) <= 1e-12
    assert rel(y64[dofs], Y_ref) <= 1e-12
    assert rel(y48[dofs], Y_ref) <= 1e-12          # double-float operator, FP64 tolerance
    assert rel(y48, y64) <= 1e-12
    _, Y32_ref = _sampled(P, u, v32.double().cpu().numpy(), dofs, w.n, w.order)
    assert rel(y32[dofs], Y32_ref) <= 1e-5
    # essential rows of J v return v, of R return 0
    eidx = np.flatnonzero(ess)[:1000]
    np.testing.assert_array_equal(y64[eidx], v[eidx])
    assert np.all(r[eidx] == 0.0)
    # properties that hold at any size: symmetry of the FP64 action
    w2 = torch.from_numpy(I.uniform_vector(op.n_dofs, seed=11)).cuda()
    w2[torch.from_numpy(ess).cuda()] = 0.0
    vm = vd.clone(); vm[torch.from_numpy(ess).cuda()] = 0.0
    a = torch.dot(w2, op.jacobian_action(vm, precision=64)).item()
    b = torch.dot(vm, op.jacobian_action(w2, precision=64)).item()
    assert abs(a - b) <= 1e-12 * abs(a)
    op.close()


def test_config2_whole_vector_parity():
    """R(u) and J(u) v at 64^3 order 3 over the whole vector against the oracle's whole-vector
    R and J v (element by element on the host cores): FP64 and double-float <= 1e-12, FP32 <= 1e-5
    (against the oracle's J v of the FP32-rounded direction)."""
    import torch
    from paper_2506_00746_gb300 import Operator
    w = I.WORKLOADS["3d_p3_k3_64"]
    V = I.lattice_vertices(3, w.n, seed=w.mesh_seed)
    op = Operator(3, w.n, w.order, V, p=w.p)
    u = I.smooth_field(3, w.n, w.order, seed=w.state_seed)
    v = I.uniform_vector(op.n_dofs, seed=w.dir_seed)
    ud, vd = torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda()
    r = op.residual(ud).cpu().numpy()
    op.linearize(ud)
    y64 = op.jacobian_action(vd, precision=64).cpu().numpy()
    y48 = op.jacobian_action(vd, precision=48).cpu().numpy()
    v32 = vd.float()
    y32 = op.jacobian_action(v32, precision=32).double().cpu().numpy()
    ym32 = op.jacobian_action(vd, precision=-32).cpu().numpy()
    op.close()
    P = O.Problem(3, w.n, w.order, V, p=w.p)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(r, O.residual(P, u)) <= 1e-12
    y_ref = O.jv(P, u, v)
    assert rel(y64, y_ref) <= 1e-12
    assert rel(y48, y_ref) <= 1e-12
    y32_ref = O.jv(P, u, v32.double().cpu().numpy())
    assert rel(y32, y32_ref) <= 1e-5
    assert rel(ym32, y32_ref) <= 1e-5


def test_design_fullsize_against_oracle():
    """The design case at full size (48^3 hexes, order 2, kappa(rho) = 1e-3 + rho^3, p = 3): the
    oracle evaluates the GPU's Newton solution (its own residual), the GPU's adjoint solution
    (its own J(u) lambda - F) and the GPU's gradient (its element-local adjoint formula at the
    GPU's u and lambda)."""
    import torch
    from paper_2506_00746_gb300 import Operator
    w = I.WORKLOADS["3d_design_k2_48"]
    V = I.lattice_vertices(3, w.n, seed=w.mesh_seed)
    rho = I.design_field(3, w.n, seed=3)
    op = Operator(3, w.n, w.order, V, p=w.p, rho=rho)
    assert op.n_dofs == 912_673
    u0 = I.smooth_field(3, w.n, w.order, seed=w.state_seed)
    ud = torch.from_numpy(u0).cuda()
    rep = op.newton_solve(ud, rtol=1e-10, cg_rtol=1e-6)
    assert rep["rel"] <= 1e-10
    op.linearize(ud)
    F = op.load_vector()
    lam, _ = op.cg_solve(F, rtol=1e-12)
    g = op.adjoint_vjp(ud, lam).cpu().numpy()
    u, lamh, Fh = ud.cpu().numpy(), lam.cpu().numpy(), F.cpu().numpy()
    P = O.Problem(3, w.n, w.order, V, p=w.p, rho=rho)
    nrm = np.linalg.norm
    assert nrm(O.residual(P, u)) <= 1e-10 * nrm(O.residual(P, u0)) * 1.01
    F_ref = O.load(P)
    F_ref[O.essential(P)] = 0.0          # the library's load vector is zero on essential DOFs
    assert nrm(Fh - F_ref) <= 1e-12 * nrm(F_ref)
    assert nrm(O.jv(P, u, lamh) - F_ref) <= 1e-10 * nrm(F_ref)
    g_ref = O.adjoint_grad(P, u, lamh)
    assert nrm(g - g_ref) <= 1e-12 * nrm(g_ref)
    op.close()


_R0_CACHE = {}


@pytest.mark.parametrize("precision", [-32, 32, 48, 64])
def test_config2_newton_verified_by_oracle(precision):
    """The full-size Newton solve (64^3 hexes, order 3, 7,189,057 DOFs) in each precision mode:
    the oracle evaluates ||R(u_gpu)|| on the host and confirms the GPU's 1e-8 claim."""
    import torch
    from paper_2506_00746_gb300 import Operator
    w = I.WORKLOADS["3d_p3_k3_64"]
    V = I.lattice_vertices(3, w.n, seed=w.mesh_seed)
    op = Operator(3, w.n, w.order, V, p=w.p)
    u0 = I.smooth_field(3, w.n, w.order, seed=w.state_seed)
    ud = torch.from_numpy(u0).cuda()
    rep = op.newton_solve(ud, rtol=1e-8, inner_precision=precision)
    assert rep["status"] == "FE_OK" and rep["rel"] <= 1e-8
    P = O.Problem(3, w.n, w.order, V, p=w.p)
    if "r0" not in _R0_CACHE:
        _R0_CACHE["r0"] = np.linalg.norm(O.residual(P, u0))
    r = np.linalg.norm(O.residual(P, ud.cpu().numpy()))
    assert r <= 1e-8 * _R0_CACHE["r0"] * 1.01
    op.close()
