"""Pins of the oracle against what the mathematics fixes (no GPU).

Each check is chosen so that a plausible slip in the oracle (a dropped term, a wrong sign or
index, a transposed Jacobian, a wrong weight) fails at least one of them:

* 1D rules against closed forms (tests/golden/rules_1d.json) and exactness properties;
* the patch test (linear fields are reproduced exactly for every p);
* p = 2 on an undistorted lattice equals the Kronecker-sum Laplacian built from exact 1D element
  matrices (closed forms for k <= 2, exact polynomial integration for k >= 3);
* symmetry of J, central finite differences of R against J v (Eq. 2 is the derivative of Eq. 1);
* the load vector sums to int f; K_e annihilates constants;
* O(h^{k+1}) L2 convergence to a manufactured solution;
* Newton's quadratic rate and the identity A(u).u = F.u at the solution;
* the adjoint of the compliance: lambda = u/(p-1) by homogeneity, and central differences of c(rho).
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2506_00746_gb300 import inputs as I

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "rules_1d.json")))


def _ev(expr: str) -> float:
    return float(eval(expr, {"sqrt": math.sqrt, "__builtins__": {}}))


# ------------------------------------------------------------------------------------------ 1D

@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_gauss_closed_forms(q):
    x, w = O.gauss_legendre(q)
    g = GOLDEN["gauss_legendre"][str(q)]
    np.testing.assert_allclose(x, [_ev(s) for s in g["x"]], rtol=0, atol=2e-16)
    np.testing.assert_allclose(w, [_ev(s) for s in g["w"]], rtol=0, atol=4e-16)


@pytest.mark.parametrize("q", range(1, 11))
def test_gauss_exactness(q):
    x, w = O.gauss_legendre(q)
    assert abs(w.sum() - 2.0) < 1e-14
    for deg in range(2 * q):                       # exact up to degree 2q-1
        exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
        assert abs(np.dot(w, x ** deg) - exact) < 1e-13
    deg = 2 * q                                    # and not beyond (guards a mis-sized rule)
    assert abs(np.dot(w, x ** deg) - 2.0 / (deg + 1)) > 1e-6


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_gll_closed_forms(k):
    x = O.gll_nodes(k)
    np.testing.assert_allclose(x, [_ev(s) for s in GOLDEN["gll_nodes"][str(k)]], rtol=0, atol=3e-16)


@pytest.mark.parametrize("k", range(2, 10))
def test_gll_are_roots_of_legendre_derivative(k):
    # independent check through numpy's Legendre series (not used by the oracle)
    x = O.gll_nodes(k)
    dP = np.polynomial.legendre.Legendre.basis(k).deriv()
    assert x[0] == -1.0 and x[-1] == 1.0
    assert np.all(np.diff(x) > 0)
    assert np.max(np.abs(dP(x[1:-1]))) < 1e-11 * k * k


@pytest.mark.parametrize("k", [1, 2, 3, 5, 7])
def test_lagrange_basis(k):
    nodes = O.gll_nodes(k)
    pts = np.linspace(-1, 1, 17)
    val, der = O.lagrange(nodes, pts)
    np.testing.assert_allclose(val.sum(axis=1), 1.0, atol=1e-13)   # partition of unity
    np.testing.assert_allclose(der.sum(axis=1), 0.0, atol=1e-11)
    v2, _ = O.lagrange(nodes, nodes)                              # cardinality
    np.testing.assert_allclose(v2, np.eye(k + 1), atol=1e-14)
    # interpolation of x^k is exact, so is its derivative
    np.testing.assert_allclose(val @ nodes ** k, pts ** k, atol=1e-12)
    np.testing.assert_allclose(der @ nodes ** k, k * pts ** (k - 1), atol=1e-10)


# ------------------------------------------------------------------------------ patch test

@pytest.mark.parametrize("dim,n,k", [(2, 3, 1), (2, 3, 2), (2, 2, 4), (3, 2, 1), (3, 2, 2), (3, 2, 3)])
@pytest.mark.parametrize("p", [2.0, 2.5, 3.0, 4.0])
def test_patch_linear_field(dim, n, k, p):
    """A linear field with its own boundary data and f = 0 is a discrete solution: interior R = 0."""
    V = I.lattice_vertices(dim, n, seed=11)
    P = O.Problem(dim, n, k, V, p=p, f_const=0.0)
    x = O.node_coords(P)
    a = np.array([0.3, -0.7, 0.5])[:dim]
    u = x @ a + 0.2
    r = O.residual(P, u)
    assert np.abs(r).max() < 2e-14
    # ... and the physical gradient is reproduced: the flux work is |a|^p * |box|
    assert abs(O.flux_work(P, u) - np.linalg.norm(a) ** p) < 1e-12


def test_patch_detects_nonlinear_field():
    """The patch test is not vacuous: a quadratic field leaves a residual."""
    V = I.lattice_vertices(2, 3, seed=11)
    P = O.Problem(2, 3, 2, V, p=3.0, f_const=0.0)
    x = O.node_coords(P)
    r = O.residual(P, x[:, 0] ** 2 + 0.2)
    assert np.abs(r).max() > 1e-3


# ------------------------------------------------------ the regularised law (eps > 0)

@pytest.mark.parametrize("dim,n,k", [(2, 3, 2), (3, 2, 2)])
@pytest.mark.parametrize("p,eps", [(1.5, 0.5), (2.5, 0.3), (3.0, 1e-2), (4.0, 0.5)])
def test_patch_linear_field_regularised(dim, n, k, p, eps):
    """eps > 0: the flux of a linear field a.x + b is still constant, (eps^2 + |a|^2)^((p-2)/2) a,
    so interior R = 0, and the flux work over the unit box is exactly
    (eps^2 + |a|^2)^((p-2)/2) |a|^2 (an eps-for-eps^2 slip changes it)."""
    V = I.lattice_vertices(dim, n, seed=11)
    P = O.Problem(dim, n, k, V, p=p, eps=eps, f_const=0.0)
    x = O.node_coords(P)
    a = np.array([0.3, -0.7, 0.5])[:dim]
    u = x @ a + 0.2
    assert np.abs(O.residual(P, u)).max() < 2e-14
    a2 = float(a @ a)
    expect = (eps * eps + a2) ** ((p - 2.0) / 2.0) * a2
    assert abs(O.flux_work(P, u) - expect) < 1e-12 * expect


@pytest.mark.parametrize("dim,n,k", [(2, 4, 2), (3, 2, 3)])
@pytest.mark.parametrize("p,eps", [(1.5, 0.5), (3.0, 0.5), (2.5, 1e-2)])
def test_symmetry_and_fd_regularised(dim, n, k, p, eps):
    """eps > 0 (including p < 2): J is symmetric and central differences of R match J v."""
    V = I.lattice_vertices(dim, n, seed=0)
    P = O.Problem(dim, n, k, V, p=p, eps=eps)
    u = I.smooth_field(dim, n, k, seed=1)
    ess = O.essential(P)
    v = I.uniform_vector(P.n_dofs, seed=2); v[ess] = 0.0
    w = I.uniform_vector(P.n_dofs, seed=3); w[ess] = 0.0
    Jv, Jw = O.jv(P, u, v), O.jv(P, u, w)
    assert abs(w @ Jv - v @ Jw) <= 1e-13 * abs(w @ Jv)
    h = 1e-5 * np.linalg.norm(u) / np.linalg.norm(v)
    fd = (O.residual(P, u + h * v) - O.residual(P, u - h * v)) / (2 * h)
    assert np.linalg.norm(fd - Jv) <= 1e-7 * np.linalg.norm(Jv)


# ----------------------------------------------------------------------- p = 2 Laplacian

def _exact_1d(k):
    """Exact 1D element stiffness/mass on [0,1] for GLL nodes, by polynomial integration."""
    from numpy.polynomial import Polynomial as Poly
    nodes = (np.real(np.polynomial.legendre.Legendre.basis(k).deriv().roots()) + 1.0) / 2.0
    nodes = np.concatenate([[0.0], np.sort(nodes), [1.0]]) if k > 1 else np.array([0.0, 1.0])
    basis = []
    for l in range(k + 1):
        others = np.delete(nodes, l)
        pl = Poly.fromroots(others)
        basis.append(pl / pl(nodes[l]))
    K = np.zeros((k + 1, k + 1)); M = np.zeros_like(K)
    for a in range(k + 1):
        for b in range(k + 1):
            K[a, b] = (basis[a].deriv() * basis[b].deriv()).integ()(1.0) - \
                      (basis[a].deriv() * basis[b].deriv()).integ()(0.0)
            M[a, b] = (basis[a] * basis[b]).integ()(1.0) - (basis[a] * basis[b]).integ()(0.0)
    return K, M


def test_exact_1d_matches_textbook():
    g = GOLDEN["element_1d_unit"]
    K1, M1 = _exact_1d(1)
    np.testing.assert_allclose(K1, g["k1_stiffness"], atol=1e-14)
    np.testing.assert_allclose(6 * M1, g["k1_mass_times_6"], atol=1e-14)
    K2, M2 = _exact_1d(2)
    np.testing.assert_allclose(3 * K2, g["k2_stiffness_times_3"], atol=1e-12)
    np.testing.assert_allclose(30 * M2, g["k2_mass_times_30"], atol=1e-12)


def _global_1d(n, k, h):
    K, M = _exact_1d(k)
    m = k * n + 1
    Kg = np.zeros((m, m)); Mg = np.zeros((m, m))
    for e in range(n):
        s = slice(k * e, k * e + k + 1)
        Kg[s, s] += K / h
        Mg[s, s] += M * h
    return Kg, Mg


@pytest.mark.parametrize("dim,n,k", [(2, 4, 1), (2, 3, 2), (2, 2, 3), (2, 2, 4), (3, 2, 1), (3, 2, 2),
                                     (3, 1, 3)])
def test_p2_is_kronecker_laplacian(dim, n, k):
    """p = 2 on the undistorted lattice: J equals K1 (x) M1 + M1 (x) K1 (Kronecker sum)."""
    V = I.lattice_vertices(dim, n, jitter=0.0)
    P = O.Problem(dim, n, k, V, p=2.0)
    u = I.smooth_field(dim, n, k, seed=3)
    J, _ = O.assemble(P, u, dirichlet=False)
    Kg, Mg = _global_1d(n, k, 1.0 / n)
    if dim == 2:
        ref = np.kron(Mg, Kg) + np.kron(Kg, Mg)          # index = ix + m*iy (x fastest)
    else:
        ref = (np.kron(Mg, np.kron(Mg, Kg)) + np.kron(Mg, np.kron(Kg, Mg)) +
               np.kron(Kg, np.kron(Mg, Mg)))
    np.testing.assert_allclose(J.toarray(), ref, atol=1e-12 * np.abs(ref).max())
    # R = K u - F at p = 2
    F = O.load(P)
    np.testing.assert_allclose(O.residual(P, u), np.where(O.essential(P), 0.0, ref @ u - F),
                               atol=1e-12)


def test_q1_laplacian_stencil():
    g = GOLDEN["q1_laplacian_2d"]
    n = 4
    P = O.Problem(2, n, 1, I.lattice_vertices(2, n, jitter=0.0), p=2.0)
    J, _ = O.assemble(P, np.zeros(P.n_dofs), dirichlet=False)
    row = J.getrow(2 + 5 * 2).toarray().ravel().reshape(5, 5)   # centre DOF (2,2)
    np.testing.assert_allclose(row[2, 2], _ev(g["centre"]), atol=1e-14)
    for (iy, ix) in [(1, 1), (1, 2), (1, 3), (2, 1), (2, 3), (3, 1), (3, 2), (3, 3)]:
        np.testing.assert_allclose(row[iy, ix], _ev(g["neighbour"]), atol=1e-14)


# --------------------------------------------------------------------- symmetry and FD

@pytest.mark.parametrize("dim,n,k", [(2, 4, 2), (2, 3, 4), (3, 2, 2), (3, 2, 3)])
@pytest.mark.parametrize("p", [2.5, 3.0, 4.0])
def test_symmetry_and_fd(dim, n, k, p):
    V = I.lattice_vertices(dim, n, seed=0)
    P = O.Problem(dim, n, k, V, p=p)
    u = I.smooth_field(dim, n, k, seed=1)
    ess = O.essential(P)
    v = I.uniform_vector(P.n_dofs, seed=2); v[ess] = 0.0
    w = I.uniform_vector(P.n_dofs, seed=3); w[ess] = 0.0
    Jv, Jw = O.jv(P, u, v), O.jv(P, u, w)
    assert abs(w @ Jv - v @ Jw) <= 1e-13 * abs(w @ Jv)
    J, _ = O.assemble(P, u)
    assert abs(J - J.T).max() <= 1e-14 * abs(J).max()
    np.testing.assert_allclose(J @ v, Jv, atol=1e-14 * np.abs(Jv).max())
    h = 1e-5 * np.linalg.norm(u) / np.linalg.norm(v)
    fd = (O.residual(P, u + h * v) - O.residual(P, u - h * v)) / (2 * h)
    assert np.linalg.norm(fd - Jv) <= 1e-7 * np.linalg.norm(Jv)


def _pins_hold() -> list[str]:
    """Run a compact set of the pins above against whatever oracle build is loaded."""
    failed = []
    V = I.lattice_vertices(2, 3, seed=11)
    P = O.Problem(2, 3, 2, V, p=3.0, f_const=0.0)
    x = O.node_coords(P)
    if np.abs(O.residual(P, x @ np.array([0.3, -0.7]) + 0.2)).max() > 2e-14:
        failed.append("patch")
    P = O.Problem(2, 3, 2, I.lattice_vertices(2, 3, jitter=0.0), p=2.0)
    J, _ = O.assemble(P, np.zeros(P.n_dofs), dirichlet=False)
    Kg, Mg = _global_1d(3, 2, 1.0 / 3)
    if np.abs(J.toarray() - (np.kron(Mg, Kg) + np.kron(Kg, Mg))).max() > 1e-12:
        failed.append("kronecker")
    if abs(O.load(O.Problem(2, 3, 2, V, p=3.0)).sum() - 1.0) > 1e-13:
        failed.append("load")
    P = O.Problem(2, 3, 2, V, p=1.5, eps=0.5, f_const=0.0)
    a = np.array([0.3, -0.7])
    if abs(O.flux_work(P, O.node_coords(P) @ a) - (0.25 + a @ a) ** -0.25 * (a @ a)) > 1e-12:
        failed.append("eps")
    P = O.Problem(2, 4, 2, I.lattice_vertices(2, 4, seed=0), p=3.0)
    u = I.smooth_field(2, 4, 2, seed=1)
    v = I.uniform_vector(P.n_dofs, seed=2); v[O.essential(P)] = 0.0
    h = 1e-5 * np.linalg.norm(u) / np.linalg.norm(v)
    fd = (O.residual(P, u + h * v) - O.residual(P, u - h * v)) / (2 * h)
    Jv = O.jv(P, u, v)
    if np.linalg.norm(fd - Jv) > 1e-7 * np.linalg.norm(Jv):
        failed.append("fd")
    return failed


def test_pins_hold_for_the_oracle():
    assert _pins_hold() == []


@pytest.mark.parametrize("plant", [1, 2, 3, 4, 5])
def test_pins_catch_planted_mistakes(plant):
    """Build the oracle with a deliberate slip and check that some pin fails."""
    with O.planted(plant):
        failed = _pins_hold()
    assert failed, f"planted mistake {plant} went unnoticed"


def test_load_and_constants():
    V = I.lattice_vertices(3, 3, seed=4)
    for f in (1.0, 2.5):
        P = O.Problem(3, 3, 2, V, p=3.0, f_const=f)
        assert abs(O.load(P).sum() - f) < 1e-13                 # sum_i phi_i = 1, |box| = 1
    P = O.Problem(3, 2, 3, I.lattice_vertices(3, 2, seed=4), p=3.0)
    u = I.smooth_field(3, 2, 3, seed=1)
    K, r, _ = O.element_matrices(P, u)
    assert np.abs(K @ np.ones(P.nl)).max() < 1e-13 * np.abs(K).max()
    assert np.abs(K - np.transpose(K, (0, 2, 1))).max() < 1e-14 * np.abs(K).max()
    # r_e sums to -int_e f: the flux part of sum_l r_l vanishes (sum of grad phi_l = 0)
    assert abs(r.sum() + 1.0) < 1e-12


# ------------------------------------------------------------------------- convergence

def _mms_solve(dim, n, k, p=3.0):
    V = I.lattice_vertices(dim, n, seed=5)
    P = O.Problem(dim, n, k, V, p=p, f_kind=1)
    x = O.node_coords(P)
    u0 = O.exact_exp(dim, x)                       # nodal interpolant: exact boundary data
    u, hist = O.newton(P, u0, rtol=1e-12)
    assert hist[-1] <= max(1e-11 * hist[0], 1e-12)
    return O.l2_error_exp(P, u)


@pytest.mark.parametrize("dim,k,ns", [(2, 1, (4, 8, 16)), (2, 2, (4, 8, 16)), (2, 3, (2, 4, 8)),
                                      (2, 4, (2, 4, 8)), (3, 1, (2, 4, 8)), (3, 2, (2, 4))])
def test_convergence_rate(dim, k, ns):
    errs = [_mms_solve(dim, n, k) for n in ns]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert abs(rates[-1] - (k + 1)) < 0.3, (errs, rates)


# ----------------------------------------------------------------------------- Newton

def test_newton_quadratic_and_work_identity():
    w = I.WORKLOADS["2d_p3_k2_16x16"]
    V = I.lattice_vertices(w.dim, w.n, seed=w.mesh_seed)
    P = O.Problem(w.dim, w.n, w.order, V, p=w.p)
    u0 = I.smooth_field(w.dim, w.n, w.order, seed=w.state_seed)
    u, hist = O.newton(P, u0, rtol=1e-13)
    assert hist[-1] <= 1e-13 * hist[0]
    # quadratic rate over the last steps that are above round-off
    h = [x for x in hist if x > 1e-14 * hist[0]]
    ratios = [h[i + 1] / h[i] ** 2 for i in range(len(h) - 3, len(h) - 1)]
    assert max(ratios) < 1e3 / hist[0], (hist, ratios)
    # A(u).u = F.u at the solution (u = 0 on the boundary), and A(u).u = int flux.grad u
    F = O.load(P)
    assert abs(O.flux_work(P, u) - F @ u) < 1e-10 * abs(F @ u)


# ------------------------------------------------------------------------------ adjoint

def _design_problem(dim=2, n=4, k=2, p=3.0, seed=3):
    V = I.lattice_vertices(dim, n, seed=0)
    rho = I.design_field(dim, n, seed=seed)
    return O.Problem(dim, n, k, V, p=p, rho=rho, kappa_eps=1e-3, kappa_q=3.0)


def test_adjoint_homogeneity():
    """eps = 0: A is positively homogeneous of degree p-1, so J(u)u = (p-1)F and lambda = u/(p-1)."""
    for p in (2.0, 3.0, 3.5):
        P = _design_problem(p=p)
        u, hist = O.newton(P, I.smooth_field(2, 4, 2, seed=1), rtol=1e-14)
        lam = O.adjoint_solve(P, u)
        np.testing.assert_allclose(lam, u / (p - 1.0), atol=1e-10 * np.abs(u).max())
        # closed form of the gradient: g_e = lambda^T dR/drho_e = kappa'(rho_e)/(p-1) int_e |grad u|^p
        # (the compliance gradient is -g); int_e |grad u|^p is the flux work of a problem whose design
        # factor is the indicator of element e (kappa_eps = 0, q = 1)
        g = O.adjoint_grad(P, u, lam)
        dk = P.kappa_q * P.rho ** (P.kappa_q - 1.0)
        work = np.array([O.flux_work(O.Problem(P.dim, P.n, P.order, P.vertices, p=p,
                                                rho=np.eye(P.n_elems)[e], kappa_eps=0.0, kappa_q=1.0), u)
                         for e in range(P.n_elems)])
        assert np.all(work > 0)
        np.testing.assert_allclose(g, dk / (p - 1.0) * work, rtol=1e-8)


def test_adjoint_against_central_differences():
    P = _design_problem(n=3)
    u0 = I.smooth_field(2, 3, 2, seed=1)
    u, _ = O.newton(P, u0, rtol=1e-14)
    F = O.load(P)
    lam = O.adjoint_solve(P, u)
    dc = -O.adjoint_grad(P, u, lam)                     # dc/drho = -lambda^T dR/drho
    rng = np.random.default_rng(4)
    rho0 = P.rho.copy()
    for _ in range(5):
        d = rng.standard_normal(P.n_elems)
        h = 1e-5
        cs = []
        for s in (+1, -1):
            Ps = O.Problem(P.dim, P.n, P.order, P.vertices, p=P.p, rho=rho0 + s * h * d,
                           kappa_eps=P.kappa_eps, kappa_q=P.kappa_q)
            us, _ = O.newton(Ps, u, rtol=1e-14)
            cs.append(F @ us)
        fd = (cs[0] - cs[1]) / (2 * h)
        assert abs(fd - dc @ d) <= 1e-6 * abs(dc @ d), (fd, dc @ d)
