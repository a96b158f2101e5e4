// rules1d.cpp -- 1D quadrature, nodes and Lagrange tables for the library's basis operator B.
//
// Gauss-Legendre points/weights and the interior Gauss-Lobatto-Legendre nodes are computed with
// the Golub-Welsch method (Golub & Welsch, Math. Comp. 23, 1969): the nodes are the eigenvalues of
// the symmetric tridiagonal Jacobi matrix of the orthogonal polynomial family, the Gauss weights
// are mu_0 times the squared first components of the normalised eigenvectors.  The eigenproblem
// is solved with cyclic Jacobi rotations (dense, at most 8x8).  Lagrange values and derivatives
// use barycentric weights.
#include <cmath>
#include <vector>

namespace feod {

// Eigen-decomposition of a symmetric matrix A (n x n, row-major, destroyed) by cyclic Jacobi
// rotations.  On return lam[i] are the eigenvalues and V[:, i] the orthonormal eigenvectors.
static void jacobi_eigen(int n, std::vector<double> &A, std::vector<double> &lam, std::vector<double> &V)
{
    V.assign(n * n, 0.0);
    for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += A[p * n + q] * A[p * n + q];
        if (off < 1e-300) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                const double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {            // A <- A G (columns p, q)
                    const double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {            // A <- G^T A (rows p, q)
                    const double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {            // V <- V G
                    const double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    lam.resize(n);
    for (int i = 0; i < n; ++i) lam[i] = A[i * n + i];
}

static void sort_pairs(std::vector<double> &x, std::vector<double> &w)
{
    const int n = (int)x.size();
    for (int i = 1; i < n; ++i)
        for (int j = i; j > 0 && x[j] < x[j - 1]; --j) {
            std::swap(x[j], x[j - 1]);
            if (!w.empty()) std::swap(w[j], w[j - 1]);
        }
}

// Gauss-Legendre rule on [-1,1]: Jacobi matrix of the Legendre recurrence has zero diagonal and
// off-diagonal j / sqrt(4 j^2 - 1); mu_0 = int_{-1}^{1} 1 = 2.
void gauss_legendre(int q, std::vector<double> &x, std::vector<double> &w)
{
    std::vector<double> A(q * q, 0.0), lam, V;
    for (int j = 1; j < q; ++j) {
        const double b = j / std::sqrt(4.0 * j * j - 1.0);
        A[(j - 1) * q + j] = A[j * q + (j - 1)] = b;
    }
    jacobi_eigen(q, A, lam, V);
    x = lam;
    w.resize(q);
    for (int i = 0; i < q; ++i) w[i] = 2.0 * V[0 * q + i] * V[0 * q + i];
    sort_pairs(x, w);
    // the middle node of an odd rule is exactly 0 by symmetry
    if (q % 2 == 1) x[q / 2] = 0.0;
    for (int i = 0; i < q / 2; ++i) {          // enforce the exact symmetry of the rule
        const double a = 0.5 * (x[q - 1 - i] - x[i]), ww = 0.5 * (w[i] + w[q - 1 - i]);
        x[i] = -a; x[q - 1 - i] = a; w[i] = w[q - 1 - i] = ww;
    }
}

// Gauss-Lobatto-Legendre nodes of order k on [-1,1]: +-1 and the zeros of P_k', which are the
// zeros of the Jacobi polynomial P^{(1,1)}_{k-1}.  Its Jacobi matrix has zero diagonal and
// off-diagonal sqrt(j (j+2) / ((2j+1)(2j+3))), j = 1..k-2.
void gll_nodes(int k, std::vector<double> &x)
{
    x.assign(k + 1, 0.0);
    x[0] = -1.0; x[k] = 1.0;
    const int m = k - 1;
    if (m >= 1) {
        std::vector<double> A(m * m, 0.0), lam, V;
        for (int j = 1; j < m; ++j) {
            const double b = std::sqrt((double)j * (j + 2) / ((2.0 * j + 1.0) * (2.0 * j + 3.0)));
            A[(j - 1) * m + j] = A[j * m + (j - 1)] = b;
        }
        jacobi_eigen(m, A, lam, V);
        std::vector<double> none;
        sort_pairs(lam, none);
        for (int i = 0; i < m; ++i) x[i + 1] = lam[i];
        if (m % 2 == 1) x[1 + m / 2] = 0.0;
        for (int i = 0; i < m / 2; ++i) {
            const double a = 0.5 * (x[k - 1 - i] - x[1 + i]);
            x[1 + i] = -a; x[k - 1 - i] = a;
        }
    }
}

// Lagrange basis on `nodes` at `pts`: val[p*nn + l] = phi_l(pts[p]), der[p*nn + l] = phi_l'(pts[p]).
// Barycentric weights lambda_l = 1 / prod_{m != l} (x_l - x_m).  Away from the nodes
//   phi_l(x) = (lambda_l / (x - x_l)) / sum_m lambda_m / (x - x_m),
//   phi_l'(x) = phi_l(x) (sum_{m != l} 1 / (x - x_m)),
// and at a node x_j the values are delta_lj and the derivatives the differentiation matrix
//   D_jl = (lambda_l / lambda_j) / (x_j - x_l) (l != j),  D_jj = -sum_{l != j} D_jl.
void lagrange_tables(const std::vector<double> &nodes, const std::vector<double> &pts, std::vector<double> &val,
                     std::vector<double> &der)
{
    const int nn = (int)nodes.size(), np = (int)pts.size();
    std::vector<double> lam(nn, 1.0);
    for (int l = 0; l < nn; ++l) {
        double prod = 1.0;
        for (int m = 0; m < nn; ++m)
            if (m != l) prod *= nodes[l] - nodes[m];
        lam[l] = 1.0 / prod;
    }
    val.assign(np * nn, 0.0);
    der.assign(np * nn, 0.0);
    for (int p = 0; p < np; ++p) {
        const double x = pts[p];
        int hit = -1;
        for (int m = 0; m < nn; ++m)
            if (x == nodes[m]) hit = m;
        if (hit >= 0) {
            double diag = 0.0;
            for (int l = 0; l < nn; ++l) {
                val[p * nn + l] = (l == hit) ? 1.0 : 0.0;
                if (l != hit) {
                    const double d = (lam[l] / lam[hit]) / (nodes[hit] - nodes[l]);
                    der[p * nn + l] = d;
                    diag -= d;
                }
            }
            der[p * nn + hit] = diag;
            continue;
        }
        double denom = 0.0;
        for (int m = 0; m < nn; ++m) denom += lam[m] / (x - nodes[m]);
        double sinv = 0.0;
        for (int m = 0; m < nn; ++m) sinv += 1.0 / (x - nodes[m]);
        for (int l = 0; l < nn; ++l) {
            const double phi = (lam[l] / (x - nodes[l])) / denom;
            val[p * nn + l] = phi;
            der[p * nn + l] = phi * (sinv - 1.0 / (x - nodes[l]));
        }
    }
}

}  // namespace feod
