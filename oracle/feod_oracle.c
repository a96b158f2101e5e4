/*
 * feod_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle for the finite element
 * operator of Eq. 1 (nonlinear action A_p(u) = P^T G^T B^T D(B G P u)) and its Jacobian
 * (Eq. 2, J_p(u) = P^T G^T B^T J_D(u_q) B G P), for the steady p-Laplacian
 * -div(kappa(|grad u|) grad u) = f with kappa = (eps^2 + |grad u|^2)^((p-2)/2).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load or call this code.  It shares no source, header, table or helper with the
 * CUDA library; the only things both sides see are the seeded input arrays.
 *
 * What it computes is the *definition* of the Galerkin residual and of its exact Jacobian:
 *   - element by element, with dense per-element basis tables phi_l(xi_q), grad phi_l(xi_q)
 *     (full tensor products, no sum factorisation),
 *   - physical gradients grad phi = J^{-T} grad_ref phi at every quadrature point,
 *   - the pointwise operator D and its derivative J_D written out by hand (the analytic
 *     tangent, the "hand-coded" column of Table 1), no dual numbers,
 *   - the element tangent K_e = B^T J_D B of Eq. 3 and the element residual r_e = B^T D(B u_e),
 *   - global sums in a fixed order (element parity colours, each colour's elements touch
 *     disjoint DOFs), then the Dirichlet convention: essential rows of R are zero, essential
 *     rows and columns of J are the identity.
 *
 * Discretisation (readings of the paper, which only names "continuous Galerkin" for the
 * p-Laplacian, Sec. "Automatic differentiation in finite element analysis"):
 *   - structured lattice of n^dim elements, vertices given by the caller (jittered), multilinear
 *     (Q1) geometry map from each element's 2^dim corner vertices, reference element [0,1]^dim;
 *   - nodal Lagrange basis of order k on Gauss-Lobatto-Legendre nodes, DOF lattice (k n + 1)^dim,
 *     lexicographic with x fastest; element (ex,ey,ez) has local node (a,b,c) at global lattice
 *     point (k ex + a, k ey + b, k ez + c);
 *   - q1d Gauss-Legendre points per direction;
 *   - essential DOFs: every DOF on the boundary of the box;
 *   - design problem: the flux is multiplied by kappa_rho(rho_e) = kappa_eps + rho_e^kappa_q.
 *   - at eps^2 + |grad u|^2 == 0 the flux and its derivative are taken as their limits
 *     (kappa = 0 for p > 2, kappa = 1 for p = 2, and the g g^T term of the tangent = 0).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_PTS 16

/* ORC_PLANT (default 0) compiles a deliberately wrong variant so that the test suite can show its
 * pins catch the mistake: 1 drops the (p-2) g g^T term of the tangent, 2 uses J^{-1} where
 * J^{-T} belongs, 3 flips the sign of the source term, 4 swaps two Gauss weights, 5 takes eps for
 * eps^2 in the regularised law (residual and tangent alike). */
#ifndef ORC_PLANT
#define ORC_PLANT 0
#endif

typedef struct {
    int dim, n, order, q1d;
    const double *vert;     /* [(n+1)^dim][dim], lexicographic x fastest */
    double p, eps;
    int f_kind;             /* 0: f = f_const; 1: manufactured source of u* = exp(a.x) */
    double f_const;
    const double *rho;      /* one value per element (ex fastest) or NULL */
    double kappa_eps, kappa_q;
} orc_problem;

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_MESH = 2, ORC_ERR_NOMEM = 3 };

/* ------------------------------------------------------------------------------------------ */
/* 1D rules on [-1,1]                                                                          */
/* ------------------------------------------------------------------------------------------ */

/* Legendre P_n(x) and P_n'(x) by Bonnet's recurrence (j+1)P_{j+1} = (2j+1) x P_j - j P_{j-1}. */
static void legendre(int n, double x, double *P, double *dP)
{
    double p0 = 1.0, p1 = x;
    if (n == 0) { *P = 1.0; *dP = 0.0; return; }
    for (int j = 1; j < n; ++j) {
        double p2 = ((2.0 * j + 1.0) * x * p1 - j * p0) / (j + 1.0);
        p0 = p1; p1 = p2;
    }
    *P = p1;
    /* derivative from (x^2-1) P_n' = n (x P_n - P_{n-1}); at |x| = 1 use P_n'(+-1) = (+-1)^{n+1} n(n+1)/2 */
    if (fabs(fabs(x) - 1.0) < 1e-300) {
        double s = (x > 0 || (n % 2 == 1)) ? 1.0 : -1.0;
        *dP = s * 0.5 * n * (n + 1.0);
    } else {
        *dP = n * (x * p1 - p0) / (x * x - 1.0);
    }
}

static void sort_asc(double *x, double *w, int n)
{
    for (int i = 1; i < n; ++i)
        for (int j = i; j > 0 && x[j] < x[j - 1]; --j) {
            double t = x[j]; x[j] = x[j - 1]; x[j - 1] = t;
            if (w) { t = w[j]; w[j] = w[j - 1]; w[j - 1] = t; }
        }
}

/* Gauss-Legendre: the q roots of P_q by Newton's method, weights 2 / ((1 - x^2) P_q'(x)^2). */
int orc_gauss_legendre(int q, double *x, double *w)
{
    if (q < 1 || q > ORC_MAX_PTS) return ORC_ERR_ARG;
    for (int i = 0; i < q; ++i) {
        double t = cos(M_PI * (i + 0.75) / (q + 0.5));
        for (int it = 0; it < 100; ++it) {
            double P, dP;
            legendre(q, t, &P, &dP);
            double dt = P / dP;
            t -= dt;
            if (fabs(dt) < 1e-17) break;
        }
        double P, dP;
        legendre(q, t, &P, &dP);
        x[i] = t;
        w[i] = 2.0 / ((1.0 - t * t) * dP * dP);
    }
    sort_asc(x, w, q);
    return ORC_OK;
}

/* Gauss-Lobatto-Legendre nodes of order k: -1, +1 and the k-1 roots of P_k'.  Newton on P_k'
 * with P_k'' from Legendre's equation (1-x^2) P'' = 2 x P' - k(k+1) P. */
int orc_gll_nodes(int k, double *x)
{
    if (k < 1 || k + 1 > ORC_MAX_PTS) return ORC_ERR_ARG;
    x[0] = -1.0; x[k] = 1.0;
    for (int i = 1; i < k; ++i) {
        double t = -cos(M_PI * i / k);
        for (int it = 0; it < 100; ++it) {
            double P, dP;
            legendre(k, t, &P, &dP);
            double d2P = (2.0 * t * dP - k * (k + 1.0) * P) / (1.0 - t * t);
            double dt = dP / d2P;
            t -= dt;
            if (fabs(dt) < 1e-17) break;
        }
        x[i] = t;
    }
    sort_asc(x, NULL, k + 1);
    return ORC_OK;
}

/* Lagrange basis on `nn` nodes evaluated at `np` points, product form:
 *   phi_l(x)  = prod_{m != l} (x - x_m) / (x_l - x_m)
 *   phi_l'(x) = sum_{j != l} 1/(x_l - x_j) prod_{m != l, j} (x - x_m) / (x_l - x_m)
 * val/der are [np][nn]. */
int orc_lagrange(int nn, const double *nodes, int np, const double *pts, double *val, double *der)
{
    if (nn < 1 || nn > ORC_MAX_PTS || np < 1) return ORC_ERR_ARG;
    for (int p = 0; p < np; ++p) {
        double x = pts[p];
        for (int l = 0; l < nn; ++l) {
            double v = 1.0;
            for (int m = 0; m < nn; ++m)
                if (m != l) v *= (x - nodes[m]) / (nodes[l] - nodes[m]);
            double d = 0.0;
            for (int j = 0; j < nn; ++j) {
                if (j == l) continue;
                double t = 1.0 / (nodes[l] - nodes[j]);
                for (int m = 0; m < nn; ++m)
                    if (m != l && m != j) t *= (x - nodes[m]) / (nodes[l] - nodes[m]);
                d += t;
            }
            val[p * nn + l] = v;
            der[p * nn + l] = d;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Element machinery                                                                           */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    int dim, k, d1, q1, nl, nq;
    double xi_q[ORC_MAX_PTS], w_q[ORC_MAX_PTS];          /* Gauss points / weights on [0,1]   */
    double phi[ORC_MAX_PTS * ORC_MAX_PTS];               /* [q][a] basis values on [0,1]      */
    double dphi[ORC_MAX_PTS * ORC_MAX_PTS];              /* [q][a] d/dxi on [0,1]             */
} rules1d;

static int make_rules(const orc_problem *P, int q1, rules1d *R)
{
    if (P->dim != 2 && P->dim != 3) return ORC_ERR_ARG;
    if (P->order < 1 || P->order + 1 > ORC_MAX_PTS || q1 < 1 || q1 > ORC_MAX_PTS) return ORC_ERR_ARG;
    R->dim = P->dim; R->k = P->order; R->d1 = P->order + 1; R->q1 = q1;
    R->nl = R->d1 * R->d1 * (P->dim == 3 ? R->d1 : 1);
    R->nq = q1 * q1 * (P->dim == 3 ? q1 : 1);
    double gx[ORC_MAX_PTS], gw[ORC_MAX_PTS], nodes[ORC_MAX_PTS], ref[ORC_MAX_PTS];
    if (orc_gauss_legendre(q1, gx, gw)) return ORC_ERR_ARG;
    if (orc_gll_nodes(P->order, nodes)) return ORC_ERR_ARG;
    /* map [-1,1] -> [0,1]: xi = (x+1)/2, weights halve, derivatives double */
    for (int q = 0; q < q1; ++q) { R->xi_q[q] = 0.5 * (gx[q] + 1.0); R->w_q[q] = 0.5 * gw[q]; }
    if (ORC_PLANT == 4 && q1 > 2) { double t = R->w_q[0]; R->w_q[0] = R->w_q[1]; R->w_q[1] = t; }
    for (int a = 0; a < R->d1; ++a) ref[a] = 0.5 * (nodes[a] + 1.0);
    orc_lagrange(R->d1, ref, q1, R->xi_q, R->phi, R->dphi);
    return ORC_OK;
}

static int64_t ipow(int64_t b, int e) { int64_t r = 1; while (e-- > 0) r *= b; return r; }

/* Element coordinates and global DOF numbers of its local nodes (a fastest). */
static void elem_coords(const orc_problem *P, int64_t e, int *ec)
{
    int64_t n = P->n;
    ec[0] = (int)(e % n); ec[1] = (int)((e / n) % n); ec[2] = P->dim == 3 ? (int)(e / (n * n)) : 0;
}

static void elem_dofs(const orc_problem *P, const rules1d *R, int64_t e, int64_t *dofs)
{
    int ec[3]; elem_coords(P, e, ec);
    int64_t m = (int64_t)P->order * P->n + 1;
    int d1 = R->d1, k = P->order;
    for (int l = 0; l < R->nl; ++l) {
        int a = l % d1, b = (l / d1) % d1, c = l / (d1 * d1);
        int64_t gx = (int64_t)k * ec[0] + a, gy = (int64_t)k * ec[1] + b, gz = (int64_t)k * ec[2] + c;
        dofs[l] = gx + m * (gy + (P->dim == 3 ? m * gz : 0));
    }
}

static int is_essential(const orc_problem *P, int64_t g)
{
    int64_t m = (int64_t)P->order * P->n + 1;
    for (int d = 0; d < P->dim; ++d) {
        int64_t i = g % m; g /= m;
        if (i == 0 || i == m - 1) return 1;
    }
    return 0;
}

/* Physical quantities at one quadrature point of one element. */
typedef struct {
    double x[3];            /* physical point                                  */
    double wdetJ;           /* quadrature weight times det J                   */
    double *grad;           /* [nl][dim] physical gradients of the basis       */
    double *val;            /* [nl] basis values                               */
} qpoint;

/* Evaluate geometry and the physical basis at quadrature point (qx,qy,qz) of element e.
 * Returns ORC_ERR_MESH if det J <= 0. */
static int eval_qpoint(const orc_problem *P, const rules1d *R, int64_t e, int q, qpoint *Q)
{
    const int dim = P->dim, d1 = R->d1, q1 = R->q1;
    int ec[3]; elem_coords(P, e, ec);
    int qi[3] = { q % q1, (q / q1) % q1, dim == 3 ? q / (q1 * q1) : 0 };
    double xi[3] = { R->xi_q[qi[0]], R->xi_q[qi[1]], dim == 3 ? R->xi_q[qi[2]] : 0.0 };
    double w = R->w_q[qi[0]] * R->w_q[qi[1]] * (dim == 3 ? R->w_q[qi[2]] : 1.0);

    /* multilinear map x(xi) = sum_corners N(xi) X_corner, N = prod (1-xi or xi) */
    double J[3][3] = {{0}}, x[3] = {0, 0, 0};
    int64_t nv = P->n + 1;
    int ncorner = dim == 3 ? 8 : 4;
    for (int c = 0; c < ncorner; ++c) {
        int ci[3] = { c & 1, (c >> 1) & 1, (c >> 2) & 1 };
        int64_t vi = (ec[0] + ci[0]) + nv * ((ec[1] + ci[1]) + (dim == 3 ? nv * (ec[2] + ci[2]) : 0));
        const double *X = P->vert + vi * dim;
        double N[3], dN[3];
        for (int d = 0; d < dim; ++d) {
            N[d] = ci[d] ? xi[d] : 1.0 - xi[d];
            dN[d] = ci[d] ? 1.0 : -1.0;
        }
        double Nall = 1.0;
        for (int d = 0; d < dim; ++d) Nall *= N[d];
        for (int a = 0; a < dim; ++a) {
            x[a] += Nall * X[a];
            for (int b = 0; b < dim; ++b) {
                double g = dN[b];
                for (int d = 0; d < dim; ++d) if (d != b) g *= N[d];
                J[a][b] += g * X[a];            /* J[a][b] = dx_a / dxi_b */
            }
        }
    }
    double det, inv[3][3];
    if (dim == 2) {
        det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        if (!(det > 0.0)) return ORC_ERR_MESH;
        inv[0][0] = J[1][1] / det; inv[0][1] = -J[0][1] / det;
        inv[1][0] = -J[1][0] / det; inv[1][1] = J[0][0] / det;
    } else {
        double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
        if (!(det > 0.0)) return ORC_ERR_MESH;
        inv[0][0] = c00 / det;
        inv[1][0] = c01 / det;
        inv[2][0] = c02 / det;
        inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
        inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
        inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
        inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
        inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
        inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    }
    for (int a = 0; a < 3; ++a) Q->x[a] = a < dim ? x[a] : 0.0;
    Q->wdetJ = w * det;

    /* dense basis table of this quadrature point: tensor products of the 1D tables */
    for (int l = 0; l < R->nl; ++l) {
        int li[3] = { l % d1, (l / d1) % d1, dim == 3 ? l / (d1 * d1) : 0 };
        double v[3], dv[3];
        for (int d = 0; d < dim; ++d) {
            v[d] = R->phi[qi[d] * d1 + li[d]];
            dv[d] = R->dphi[qi[d] * d1 + li[d]];
        }
        double val = 1.0, ref[3];
        for (int d = 0; d < dim; ++d) val *= v[d];
        for (int b = 0; b < dim; ++b) {
            double g = dv[b];
            for (int d = 0; d < dim; ++d) if (d != b) g *= v[d];
            ref[b] = g;
        }
        Q->val[l] = val;
        /* grad phi = J^{-T} grad_ref phi :  (grad phi)_i = sum_j inv[j][i] ref_j */
        for (int i = 0; i < dim; ++i) {
            double s = 0.0;
            for (int j = 0; j < dim; ++j) s += (ORC_PLANT == 2 ? inv[i][j] : inv[j][i]) * ref[j];
            Q->grad[l * dim + i] = s;
        }
    }
    return ORC_OK;
}

/* Source term f at a physical point. */
static const double MMS_A[3] = { 1.0, 0.5, 1.0 / 3.0 };
static double source(const orc_problem *P, const double *x)
{
    if (P->f_kind == 0) return ORC_PLANT == 3 ? -P->f_const : P->f_const;
    /* u* = exp(a.x): grad u* = a u*, flux = |a|^{p-2} a u*^{p-1}, div flux = (p-1)|a|^p u*^{p-1} */
    double ax = 0.0, a2 = 0.0;
    for (int d = 0; d < P->dim; ++d) { ax += MMS_A[d] * x[d]; a2 += MMS_A[d] * MMS_A[d]; }
    return -(P->p - 1.0) * pow(sqrt(a2), P->p) * exp((P->p - 1.0) * ax);
}

static double kappa_rho(const orc_problem *P, int64_t e)
{
    if (!P->rho) return 1.0;
    return P->kappa_eps + pow(P->rho[e], P->kappa_q);
}

/* Pointwise operator D: flux = kr * kappa(base) * g with base = eps^2 + |g|^2, and its exact
 * derivative C = kr * [kappa I + (p-2) base^{(p-4)/2} g g^T] (written out by hand). */
static void law(const orc_problem *P, double kr, const double *g, double *flux, double C[3][3])
{
    int dim = P->dim;
    double s = 0.0;
    for (int d = 0; d < dim; ++d) s += g[d] * g[d];
    double base = (ORC_PLANT == 5 ? P->eps : P->eps * P->eps) + s;
    double kap, kap2;
    if (base == 0.0) {
        kap = (P->p == 2.0) ? 1.0 : 0.0;
        kap2 = 0.0;
    } else {
        kap = pow(base, 0.5 * (P->p - 2.0));
        kap2 = (P->p - 2.0) * pow(base, 0.5 * (P->p - 4.0));
    }
    for (int d = 0; d < dim; ++d) flux[d] = kr * kap * g[d];
    if (C)
        for (int i = 0; i < dim; ++i)
            for (int j = 0; j < dim; ++j)
                C[i][j] = kr * ((i == j ? kap : 0.0) + (ORC_PLANT == 1 ? 0.0 : kap2) * g[i] * g[j]);
}

typedef struct {
    rules1d R;
    double *grad, *val;
    int64_t *dofs;
    double *ue, *ve, *ye;
} workspace;

static int ws_init(workspace *W, const orc_problem *P)
{
    int q1 = P->q1d > 0 ? P->q1d : P->order + 1;
    int rc = make_rules(P, q1, &W->R);
    if (rc) return rc;
    int nl = W->R.nl;
    W->grad = malloc(sizeof(double) * nl * 3);
    W->val = malloc(sizeof(double) * nl);
    W->dofs = malloc(sizeof(int64_t) * nl);
    W->ue = malloc(sizeof(double) * nl);
    W->ve = malloc(sizeof(double) * nl);
    W->ye = malloc(sizeof(double) * nl);
    if (!W->grad || !W->val || !W->dofs || !W->ue || !W->ve || !W->ye) return ORC_ERR_NOMEM;
    return ORC_OK;
}

static void ws_free(workspace *W)
{
    free(W->grad); free(W->val); free(W->dofs); free(W->ue); free(W->ve); free(W->ye);
}

/* Element residual r_e = sum_q wdetJ [flux(g) . grad phi_l - f phi_l]  (Eq. 1 / Eq. 3). */
static int elem_residual(const orc_problem *P, workspace *W, int64_t e, const double *ue, double *re)
{
    const rules1d *R = &W->R;
    int dim = P->dim, nl = R->nl;
    double kr = kappa_rho(P, e);
    qpoint Q = { {0}, 0, W->grad, W->val };
    for (int l = 0; l < nl; ++l) re[l] = 0.0;
    for (int q = 0; q < R->nq; ++q) {
        int rc = eval_qpoint(P, R, e, q, &Q);
        if (rc) return rc;
        double g[3] = {0, 0, 0}, flux[3];
        for (int l = 0; l < nl; ++l)
            for (int d = 0; d < dim; ++d) g[d] += ue[l] * Q.grad[l * dim + d];
        law(P, kr, g, flux, NULL);
        double f = source(P, Q.x);
        for (int l = 0; l < nl; ++l) {
            double t = 0.0;
            for (int d = 0; d < dim; ++d) t += flux[d] * Q.grad[l * dim + d];
            re[l] += Q.wdetJ * (t - f * Q.val[l]);
        }
    }
    return ORC_OK;
}

/* Element Jacobian action y_e = K_e v_e with K_e = B^T J_D B (Eq. 3), applied as
 * sum_q wdetJ grad phi_l . (C(g_u) g_v). */
static int elem_jv(const orc_problem *P, workspace *W, int64_t e, const double *ue, const double *ve,
                   double *ye)
{
    const rules1d *R = &W->R;
    int dim = P->dim, nl = R->nl;
    double kr = kappa_rho(P, e);
    qpoint Q = { {0}, 0, W->grad, W->val };
    for (int l = 0; l < nl; ++l) ye[l] = 0.0;
    for (int q = 0; q < R->nq; ++q) {
        int rc = eval_qpoint(P, R, e, q, &Q);
        if (rc) return rc;
        double gu[3] = {0, 0, 0}, gv[3] = {0, 0, 0}, flux[3], C[3][3];
        for (int l = 0; l < nl; ++l)
            for (int d = 0; d < dim; ++d) {
                gu[d] += ue[l] * Q.grad[l * dim + d];
                gv[d] += ve[l] * Q.grad[l * dim + d];
            }
        law(P, kr, gu, flux, C);
        double cg[3] = {0, 0, 0};
        for (int i = 0; i < dim; ++i)
            for (int j = 0; j < dim; ++j) cg[i] += C[i][j] * gv[j];
        for (int l = 0; l < nl; ++l) {
            double t = 0.0;
            for (int d = 0; d < dim; ++d) t += cg[d] * Q.grad[l * dim + d];
            ye[l] += Q.wdetJ * t;
        }
    }
    return ORC_OK;
}

static int64_t n_dofs(const orc_problem *P) { return ipow((int64_t)P->order * P->n + 1, P->dim); }
static int64_t n_elems(const orc_problem *P) { return ipow(P->n, P->dim); }

static int check_problem(const orc_problem *P)
{
    if (!P || !P->vert || (P->dim != 2 && P->dim != 3) || P->n < 1 || P->order < 1 ||
        P->order + 1 > ORC_MAX_PTS || P->q1d < 0 || P->q1d > ORC_MAX_PTS)
        return ORC_ERR_ARG;
    if (P->p < 2.0 && P->eps == 0.0) return ORC_ERR_ARG;   /* kappa unbounded at grad u = 0 */
    return ORC_OK;
}

/* The elements of colour c (parity pattern of (ex,ey,ez)) touch pairwise disjoint DOFs, so each
 * colour's scatter is race-free and every DOF receives its contributions in colour order. */
static int elem_in_colour(const orc_problem *P, int64_t e, int c)
{
    int ec[3]; elem_coords(P, e, ec);
    int col = (ec[0] & 1) | ((ec[1] & 1) << 1) | (P->dim == 3 ? (ec[2] & 1) << 2 : 0);
    return col == c;
}

/* Accumulate the element residuals or Jacobian actions of elements [e0, e1) into out.
 * mode 0: residual of u; mode 1: Jacobian action J(u) v with v given (already masked). */
static int accumulate(const orc_problem *P, int mode, const double *u, const double *v, double *out,
                      int64_t e0, int64_t e1)
{
    int ncol = P->dim == 3 ? 8 : 4;
    int err = ORC_OK;
    for (int c = 0; c < ncol; ++c) {
#pragma omp parallel
        {
            workspace W;
            int rc = ws_init(&W, P);
            if (rc) {
#pragma omp critical
                err = rc;
            }
#pragma omp for schedule(static)
            for (int64_t e = e0; e < e1; ++e) {
                if (rc || !elem_in_colour(P, e, c)) continue;
                elem_dofs(P, &W.R, e, W.dofs);
                for (int l = 0; l < W.R.nl; ++l) W.ue[l] = u ? u[W.dofs[l]] : 0.0;
                int r2;
                if (mode == 0) {
                    r2 = elem_residual(P, &W, e, W.ue, W.ye);
                } else {
                    for (int l = 0; l < W.R.nl; ++l) W.ve[l] = v[W.dofs[l]];
                    r2 = elem_jv(P, &W, e, W.ue, W.ve, W.ye);
                }
                if (r2) {
#pragma omp critical
                    err = r2;
                    continue;
                }
                for (int l = 0; l < W.R.nl; ++l) out[W.dofs[l]] += W.ye[l];
            }
            ws_free(&W);
        }
        if (err) return err;
    }
    return err;
}

/* ------------------------------------------------------------------------------------------ */
/* Exported entry points                                                                       */
/* ------------------------------------------------------------------------------------------ */

int orc_set_threads(int nt)
{
#ifdef _OPENMP
    if (nt > 0) omp_set_num_threads(nt);
    return omp_get_max_threads();
#else
    (void)nt;
    return 1;
#endif
}

/* Physical coordinates of every DOF: the geometry map at the element's GLL node. */
int orc_node_coords(const orc_problem *P, double *xyz)
{
    int rc = check_problem(P);
    if (rc) return rc;
    double nodes[ORC_MAX_PTS];
    orc_gll_nodes(P->order, nodes);
    int dim = P->dim, k = P->order;
    int64_t m = (int64_t)k * P->n + 1, nv = P->n + 1, N = n_dofs(P);
    for (int64_t g = 0; g < N; ++g) {
        int64_t gi[3] = { g % m, (g / m) % m, dim == 3 ? g / (m * m) : 0 };
        int ec[3]; double xi[3] = {0, 0, 0};
        for (int d = 0; d < dim; ++d) {
            int64_t el = gi[d] / k;
            if (el >= P->n) el = P->n - 1;
            ec[d] = (int)el;
            xi[d] = 0.5 * (nodes[gi[d] - (int64_t)k * el] + 1.0);
        }
        double x[3] = {0, 0, 0};
        for (int c = 0; c < (dim == 3 ? 8 : 4); ++c) {
            int ci[3] = { c & 1, (c >> 1) & 1, (c >> 2) & 1 };
            int64_t vi = (ec[0] + ci[0]) + nv * ((ec[1] + ci[1]) + (dim == 3 ? nv * (ec[2] + ci[2]) : 0));
            double Nall = 1.0;
            for (int d = 0; d < dim; ++d) Nall *= ci[d] ? xi[d] : 1.0 - xi[d];
            for (int a = 0; a < dim; ++a) x[a] += Nall * P->vert[vi * dim + a];
        }
        for (int a = 0; a < dim; ++a) xyz[g * dim + a] = x[a];
    }
    return ORC_OK;
}

/* Full residual R(u) = A(u) - F with essential entries set to zero (Eq. 1 plus the Dirichlet
 * convention).  u carries the boundary values. */
int orc_residual(const orc_problem *P, const double *u, double *r)
{
    int rc = check_problem(P);
    if (rc) return rc;
    int64_t N = n_dofs(P);
    memset(r, 0, sizeof(double) * N);
    rc = accumulate(P, 0, u, NULL, r, 0, n_elems(P));
    if (rc) return rc;
    for (int64_t g = 0; g < N; ++g) if (is_essential(P, g)) r[g] = 0.0;
    return ORC_OK;
}

/* Jacobian action y = J(u) v (Eq. 2) with the Dirichlet convention: the input is masked
 * (essential entries of v treated as zero) and essential rows return y_i = v_i. */
int orc_jv(const orc_problem *P, const double *u, const double *v, double *y)
{
    int rc = check_problem(P);
    if (rc) return rc;
    int64_t N = n_dofs(P);
    double *vm = malloc(sizeof(double) * N);
    if (!vm) return ORC_ERR_NOMEM;
    for (int64_t g = 0; g < N; ++g) vm[g] = is_essential(P, g) ? 0.0 : v[g];
    memset(y, 0, sizeof(double) * N);
    rc = accumulate(P, 1, u, vm, y, 0, n_elems(P));
    free(vm);
    if (rc) return rc;
    for (int64_t g = 0; g < N; ++g) if (is_essential(P, g)) y[g] = v[g];
    return ORC_OK;
}

/* Partial Jacobian action over the elements [e0, e1): adds their K_e v_e into y (no masking, no
 * Dirichlet finish).  Used to time a bounded sample of a full action. */
int orc_jv_partial(const orc_problem *P, const double *u, const double *v, double *y,
                   int64_t e0, int64_t e1)
{
    int rc = check_problem(P);
    if (rc) return rc;
    if (e0 < 0 || e1 > n_elems(P) || e0 > e1) return ORC_ERR_ARG;
    return accumulate(P, 1, u, v, y, e0, e1);
}

/* Residual over the elements [e0, e1) only (no Dirichlet finish); for timing samples. */
int orc_residual_partial(const orc_problem *P, const double *u, double *r, int64_t e0, int64_t e1)
{
    int rc = check_problem(P);
    if (rc) return rc;
    if (e0 < 0 || e1 > n_elems(P) || e0 > e1) return ORC_ERR_ARG;
    return accumulate(P, 0, u, NULL, r, e0, e1);
}

/* Element-level quantities of `count` listed elements: residual r_e, Jacobian action K_e v_e
 * (v given per global DOF, used unmasked) and the global DOFs of each local node.  Any output
 * pointer may be NULL.  Layout [count][nl]. */
int orc_element_vectors(const orc_problem *P, const double *u, const double *v, const int64_t *elems,
                        int64_t count, double *re, double *ye, int64_t *dofs)
{
    int rc = check_problem(P);
    if (rc) return rc;
    workspace W;
    rc = ws_init(&W, P);
    if (rc) { ws_free(&W); return rc; }
    int nl = W.R.nl;
    for (int64_t i = 0; i < count && !rc; ++i) {
        int64_t e = elems[i];
        if (e < 0 || e >= n_elems(P)) { rc = ORC_ERR_ARG; break; }
        elem_dofs(P, &W.R, e, W.dofs);
        for (int l = 0; l < nl; ++l) W.ue[l] = u ? u[W.dofs[l]] : 0.0;
        if (dofs) for (int l = 0; l < nl; ++l) dofs[i * nl + l] = W.dofs[l];
        if (re) rc = elem_residual(P, &W, e, W.ue, re + i * nl);
        if (!rc && ye && v) {
            for (int l = 0; l < nl; ++l) W.ve[l] = v[W.dofs[l]];
            rc = elem_jv(P, &W, e, W.ue, W.ve, ye + i * nl);
        }
    }
    ws_free(&W);
    return rc;
}

/* Element tangent matrices K_e = sum_q wdetJ grad phi_l^T C grad phi_m (Eq. 3, analytic C) and
 * element residuals of the elements [e0, e1).  K: [e1-e0][nl][nl], r: [e1-e0][nl],
 * dofs: [e1-e0][nl].  No Dirichlet convention applied. */
int orc_element_matrices(const orc_problem *P, const double *u, int64_t e0, int64_t e1, double *K,
                         double *r, int64_t *dofs)
{
    int rc = check_problem(P);
    if (rc) return rc;
    if (e0 < 0 || e1 > n_elems(P) || e0 > e1) return ORC_ERR_ARG;
    workspace W;
    rc = ws_init(&W, P);
    if (rc) { ws_free(&W); return rc; }
    const rules1d *R = &W.R;
    int dim = P->dim, nl = R->nl;
    qpoint Q = { {0}, 0, W.grad, W.val };
    for (int64_t e = e0; e < e1 && !rc; ++e) {
        int64_t i = e - e0;
        elem_dofs(P, R, e, W.dofs);
        for (int l = 0; l < nl; ++l) { W.ue[l] = u[W.dofs[l]]; dofs[i * nl + l] = W.dofs[l]; }
        rc = elem_residual(P, &W, e, W.ue, r + i * nl);
        if (rc) break;
        double *Ke = K + i * (int64_t)nl * nl;
        memset(Ke, 0, sizeof(double) * nl * nl);
        double kr = kappa_rho(P, e);
        for (int q = 0; q < R->nq && !rc; ++q) {
            rc = eval_qpoint(P, R, e, q, &Q);
            if (rc) break;
            double g[3] = {0, 0, 0}, flux[3], C[3][3];
            for (int l = 0; l < nl; ++l)
                for (int d = 0; d < dim; ++d) g[d] += W.ue[l] * Q.grad[l * dim + d];
            law(P, kr, g, flux, C);
            for (int m = 0; m < nl; ++m) {
                double cg[3] = {0, 0, 0};
                for (int a = 0; a < dim; ++a)
                    for (int b = 0; b < dim; ++b) cg[a] += C[a][b] * Q.grad[m * dim + b];
                for (int l = 0; l < nl; ++l) {
                    double t = 0.0;
                    for (int a = 0; a < dim; ++a) t += Q.grad[l * dim + a] * cg[a];
                    Ke[(int64_t)l * nl + m] += Q.wdetJ * t;
                }
            }
        }
    }
    ws_free(&W);
    return rc;
}

/* Load vector F_i = int f phi_i (no Dirichlet masking). */
int orc_load(const orc_problem *P, double *F)
{
    int rc = check_problem(P);
    if (rc) return rc;
    workspace W;
    rc = ws_init(&W, P);
    if (rc) { ws_free(&W); return rc; }
    const rules1d *R = &W.R;
    int64_t N = n_dofs(P), NE = n_elems(P);
    memset(F, 0, sizeof(double) * N);
    qpoint Q = { {0}, 0, W.grad, W.val };
    for (int64_t e = 0; e < NE && !rc; ++e) {
        elem_dofs(P, R, e, W.dofs);
        for (int q = 0; q < R->nq; ++q) {
            rc = eval_qpoint(P, R, e, q, &Q);
            if (rc) break;
            double f = source(P, Q.x);
            for (int l = 0; l < R->nl; ++l) F[W.dofs[l]] += Q.wdetJ * f * Q.val[l];
        }
    }
    ws_free(&W);
    return rc;
}

/* Design gradient of the residual contracted with lambda (essential entries of lambda ignored), per element:
 *   g_e = lambda_e^T dr_e/drho_e = kappa_rho'(rho_e) int_e kappa(|grad u|) grad u . grad lambda,
 * kappa_rho'(rho) = kappa_q rho^(kappa_q - 1).  (Adjoint load, local to quadrature points.) */
int orc_adjoint_grad(const orc_problem *P, const double *u, const double *lam, double *grad)
{
    int rc = check_problem(P);
    if (rc) return rc;
    if (!P->rho) return ORC_ERR_ARG;
    workspace W;
    rc = ws_init(&W, P);
    if (rc) { ws_free(&W); return rc; }
    const rules1d *R = &W.R;
    int dim = P->dim, nl = R->nl;
    int64_t NE = n_elems(P);
    qpoint Q = { {0}, 0, W.grad, W.val };
    for (int64_t e = 0; e < NE && !rc; ++e) {
        elem_dofs(P, R, e, W.dofs);
        /* essential rows of R are identically zero, so lambda's essential entries drop out */
        for (int l = 0; l < nl; ++l) {
            W.ue[l] = u[W.dofs[l]];
            W.ve[l] = is_essential(P, W.dofs[l]) ? 0.0 : lam[W.dofs[l]];
        }
        double dkr = P->kappa_q * pow(P->rho[e], P->kappa_q - 1.0);
        double acc = 0.0;
        for (int q = 0; q < R->nq; ++q) {
            rc = eval_qpoint(P, R, e, q, &Q);
            if (rc) break;
            double gu[3] = {0, 0, 0}, gl[3] = {0, 0, 0}, flux[3];
            for (int l = 0; l < nl; ++l)
                for (int d = 0; d < dim; ++d) {
                    gu[d] += W.ue[l] * Q.grad[l * dim + d];
                    gl[d] += W.ve[l] * Q.grad[l * dim + d];
                }
            law(P, 1.0, gu, flux, NULL);
            double t = 0.0;
            for (int d = 0; d < dim; ++d) t += flux[d] * gl[d];
            acc += Q.wdetJ * t;
        }
        grad[e] = dkr * acc;
    }
    ws_free(&W);
    return rc;
}

/* int kappa_rho kappa(|grad u|) |grad u|^2, i.e. int flux(grad u) . grad u (equals the energy
 * integral int kappa_rho |grad u|^p when eps = 0). */
double orc_flux_work(const orc_problem *P, const double *u)
{
    if (check_problem(P)) return NAN;
    workspace W;
    if (ws_init(&W, P)) { ws_free(&W); return NAN; }
    const rules1d *R = &W.R;
    int dim = P->dim, nl = R->nl;
    int64_t NE = n_elems(P);
    qpoint Q = { {0}, 0, W.grad, W.val };
    double total = 0.0;
    for (int64_t e = 0; e < NE; ++e) {
        elem_dofs(P, R, e, W.dofs);
        for (int l = 0; l < nl; ++l) W.ue[l] = u[W.dofs[l]];
        double kr = kappa_rho(P, e);
        for (int q = 0; q < R->nq; ++q) {
            if (eval_qpoint(P, R, e, q, &Q)) { ws_free(&W); return NAN; }
            double g[3] = {0, 0, 0}, flux[3];
            for (int l = 0; l < nl; ++l)
                for (int d = 0; d < dim; ++d) g[d] += W.ue[l] * Q.grad[l * dim + d];
            law(P, kr, g, flux, NULL);
            double t = 0.0;
            for (int d = 0; d < dim; ++d) t += flux[d] * g[d];
            total += Q.wdetJ * t;
        }
    }
    ws_free(&W);
    return total;
}

/* L2 error || u_h - u* || against the manufactured solution u* = exp(a.x), using a Gauss rule
 * with q1 + qextra points per direction. */
double orc_l2_error_exp(const orc_problem *P, const double *u, int qextra)
{
    if (check_problem(P)) return NAN;
    orc_problem P2 = *P;
    int q1 = (P->q1d > 0 ? P->q1d : P->order + 1) + qextra;
    if (q1 > ORC_MAX_PTS) return NAN;
    P2.q1d = q1;
    workspace W;
    if (ws_init(&W, &P2)) { ws_free(&W); return NAN; }
    const rules1d *R = &W.R;
    int dim = P->dim, nl = R->nl;
    int64_t NE = n_elems(P);
    qpoint Q = { {0}, 0, W.grad, W.val };
    double total = 0.0;
    for (int64_t e = 0; e < NE; ++e) {
        elem_dofs(P, R, e, W.dofs);
        for (int q = 0; q < R->nq; ++q) {
            if (eval_qpoint(&P2, R, e, q, &Q)) { ws_free(&W); return NAN; }
            double uh = 0.0;
            for (int l = 0; l < nl; ++l) uh += u[W.dofs[l]] * Q.val[l];
            double ax = 0.0;
            for (int d = 0; d < dim; ++d) ax += MMS_A[d] * Q.x[d];
            double err = uh - exp(ax);
            total += Q.wdetJ * err * err;
        }
    }
    ws_free(&W);
    return sqrt(total);
}

/* Value of the manufactured solution u* = exp(a.x) at given points [np][dim]. */
int orc_exact_exp(int dim, int64_t np, const double *x, double *out)
{
    if (dim != 2 && dim != 3) return ORC_ERR_ARG;
    for (int64_t i = 0; i < np; ++i) {
        double ax = 0.0;
        for (int d = 0; d < dim; ++d) ax += MMS_A[d] * x[i * dim + d];
        out[i] = exp(ax);
    }
    return ORC_OK;
}
