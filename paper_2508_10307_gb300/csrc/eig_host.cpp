// Host FP64 eigenvalues of a small dense symmetric matrix (the d x d patch covariance of
// the noise-level estimate, d = 64 C). Householder reduction to tridiagonal form, then
// implicit symmetric QR steps with a Wilkinson shift and deflation (Golub & Van Loan,
// "Matrix Computations", Sec. 8.3). Eigenvalues only.
#include <cmath>
#include <vector>

namespace htsvd {

namespace {

// A (n x n, row-major, symmetric; only the lower triangle i >= j is read and overwritten)
// -> diagonal d[n], off-diagonal e[n-1]. Step k reflects the trailing block B = A[k+1:, k+1:]
// with H = I - beta v v^T (H x = alpha e_1 for x = A[k+1:, k]): p = beta B v,
// w = p - (beta/2)(v^T p) v, B <- B - v w^T - w v^T.
void tridiagonalize(double* A, int n, double* d, double* e) {
    std::vector<double> v(n), p(n), w(n);
    for (int k = 0; k < n - 2; ++k) {
        const int m = n - k - 1;                  // size of the trailing block
        double* x = &v[0];
        double xn2 = 0.0;
        for (int i = 0; i < m; ++i) {
            x[i] = A[(size_t)(k + 1 + i) * n + k];
            xn2 += x[i] * x[i];
        }
        if (xn2 == 0.0) {
            e[k] = 0.0;
            continue;
        }
        double alpha = std::sqrt(xn2);
        if (x[0] > 0) alpha = -alpha;             // avoids cancellation in v_0
        x[0] -= alpha;
        double vtv = 0.0;
        for (int i = 0; i < m; ++i) vtv += x[i] * x[i];
        const double beta = 2.0 / vtv;
        // p = B v from the lower triangle: row i contributes its dot product to p_i and,
        // through symmetry, L_ij v_i to p_j (j < i)
        for (int i = 0; i < m; ++i) p[i] = 0.0;
        for (int i = 0; i < m; ++i) {
            const double* row = A + (size_t)(k + 1 + i) * n + (k + 1);
            const double vi = x[i];
            double s = 0.0;
            for (int j = 0; j < i; ++j) {
                s += row[j] * x[j];
                p[j] += row[j] * vi;
            }
            p[i] += s + row[i] * vi;
        }
        double vp = 0.0;
        for (int i = 0; i < m; ++i) {
            p[i] *= beta;
            vp += x[i] * p[i];
        }
        const double Kc = 0.5 * beta * vp;
        for (int i = 0; i < m; ++i) w[i] = p[i] - Kc * x[i];
        for (int i = 0; i < m; ++i) {
            double* row = A + (size_t)(k + 1 + i) * n + (k + 1);
            const double xi = x[i], wi = w[i];
            for (int j = 0; j <= i; ++j) row[j] -= xi * w[j] + wi * x[j];
        }
        e[k] = alpha;
    }
    for (int i = 0; i < n; ++i) d[i] = A[(size_t)i * n + i];
    if (n >= 2) e[n - 2] = A[(size_t)(n - 1) * n + (n - 2)];
}

// Eigenvalues of the symmetric tridiagonal (a, b) in place in a.
bool tridiagonal_eigenvalues(double* a, double* b, int n) {
    const double eps = 2.220446049250313e-16;
    int iter = 0;
    int hi = n - 1;
    while (hi > 0) {
        if (std::fabs(b[hi - 1]) <= eps * (std::fabs(a[hi - 1]) + std::fabs(a[hi]))) {
            b[hi - 1] = 0.0;
            --hi;
            continue;
        }
        int lo = hi - 1;
        while (lo > 0 && std::fabs(b[lo - 1]) > eps * (std::fabs(a[lo - 1]) + std::fabs(a[lo]))) --lo;
        if (++iter > 60 * n) return false;
        // Wilkinson shift from the trailing 2x2 block
        const double dd = 0.5 * (a[hi - 1] - a[hi]);
        const double bb = b[hi - 1];
        const double den = dd + (dd >= 0 ? 1.0 : -1.0) * std::sqrt(dd * dd + bb * bb);
        const double mu = a[hi] - (den != 0.0 ? bb * bb / den : 0.0);
        double x = a[lo] - mu, z = b[lo];
        for (int k = lo; k < hi; ++k) {
            const double r = std::sqrt(x * x + z * z);      // entries are far from overflow (covariances of bytes)
            const double c = r == 0.0 ? 1.0 : x / r, s = r == 0.0 ? 0.0 : z / r;
            if (k > lo) b[k - 1] = r;
            const double ak = a[k], ak1 = a[k + 1], bk = b[k];
            a[k] = c * c * ak + 2.0 * c * s * bk + s * s * ak1;
            a[k + 1] = s * s * ak - 2.0 * c * s * bk + c * c * ak1;
            b[k] = c * s * (ak1 - ak) + (c * c - s * s) * bk;
            if (k + 1 < hi) {
                x = b[k];
                z = s * b[k + 1];
                b[k + 1] = c * b[k + 1];
            }
        }
    }
    return true;
}

}  // namespace

// Eigenvalues (unsorted) of the symmetric n x n matrix A (row-major, overwritten). Returns false
// if the QR iteration did not converge.
bool symmetric_eigenvalues(double* A, int n, double* out) {
    std::vector<double> e(n > 1 ? n - 1 : 1, 0.0);
    tridiagonalize(A, n, out, e.data());
    return tridiagonal_eigenvalues(out, e.data(), n);
}

}  // namespace htsvd
