// Host FP64 eigenvalues of a small dense symmetric matrix (the d x d patch covariance of
// the noise-level estimate, d = 64 C). Householder reduction to tridiagonal form, then
// implicit-shift QR with a Wilkinson shift and deflation (Golub & Van Loan, "Matrix
// Computations", Secs. 8.3.1 and 8.3.5), carried out on the squared off-diagonal entries so
// that no square root is taken inside the chase. Eigenvalues only.
#include <cmath>
#include <vector>

namespace htsvd {

namespace {

// Two doubles as one vector value (GCC vector extension: SIMD on any target, no intrinsics).
typedef double v2d __attribute__((vector_size(16)));
inline v2d ld2(const double* p) {
    v2d r;
    __builtin_memcpy(&r, p, sizeof(r));
    return r;
}
inline void st2(double* p, v2d x) { __builtin_memcpy(p, &x, sizeof(x)); }

// A (n x n, row-major, symmetric; only the lower triangle i >= j is read and overwritten)
// -> diagonal d[n], off-diagonal e[n-1]. Step k reflects the trailing block B = A[k+1:, k+1:]
// with H = I - beta v v^T (H x = alpha e_1 for x = A[k+1:, k]): p = beta B v,
// w = p - (beta/2)(v^T p) v, B <- B - v w^T - w v^T. The rank-2 update of step k is deferred
// and applied to each row of the trailing triangle in the same pass that forms p of step k+1,
// so the triangle is read and written once per step; the pass runs on two-double vectors, two
// rows at a time. Its expressions are chains of multiply-adds (r - v w - w' v', p + a v + b v'), so
// that each entry costs four fused operations per row where a compiler contracts them: the pass
// is bound by floating-point issue, not by memory.
void tridiagonalize(double* A, int n, double* d, double* e) {
    std::vector<double> vb(n, 0.0), wb(n, 0.0), v(n), p(n);     // (vb, wb): deferred update, absolute indices
    bool pending = false;
    for (int k = 0; k < n; ++k) {
        if (pending) {                                            // column k, rows k..n-1
            const double vk = vb[k], wk = wb[k];
            for (int i = k; i < n; ++i) A[(size_t)i * n + k] -= vb[i] * wk + wb[i] * vk;
        }
        d[k] = A[(size_t)k * n + k];
        if (k >= n - 2) continue;                                 // the last 2x2 block needs no reflector
        const int m = n - k - 1;
        double xn2 = 0.0;
        for (int i = 0; i < m; ++i) {
            v[i] = A[(size_t)(k + 1 + i) * n + k];
            xn2 += v[i] * v[i];
        }
        double alpha = 0.0, beta = 0.0;
        if (xn2 != 0.0) {
            alpha = std::sqrt(xn2);
            if (v[0] > 0) alpha = -alpha;                         // avoids cancellation in v_0
            v[0] -= alpha;
            double vtv = 0.0;
            for (int i = 0; i < m; ++i) vtv += v[i] * v[i];
            beta = 2.0 / vtv;
        }
        e[k] = alpha;
        // one pass over the trailing lower triangle: deferred update of row i, then its part of
        // p = B v (row i gives its dot product to p_i and, by symmetry, L_ij v_i to p_j, j < i).
        // Rows go in pairs (i, i+1) so that each load of v, p and the deferred (vb, wb) serves both.
        const double* vo = vb.data() + k + 1;
        const double* wo = wb.data() + k + 1;
        const double* vv = v.data();
        double* pp = p.data();
        for (int i = 0; i < m; ++i) pp[i] = 0.0;
        const double pend = pending ? 1.0 : 0.0;     // the deferred update is zero at the first step
        int i = 0;
        for (; i + 2 <= m; i += 2) {
            double* ra = A + (size_t)(k + 1 + i) * n + (k + 1);
            double* rb = ra + n;
            const double va = vv[i], vb1 = vv[i + 1];
            const double voa = pend * vo[i], woa = pend * wo[i], vob = pend * vo[i + 1], wob = pend * wo[i + 1];
            const v2d VA = {va, va}, VB = {vb1, vb1};
            const v2d VOA = {voa, voa}, WOA = {woa, woa}, VOB = {vob, vob}, WOB = {wob, wob};
            v2d Sa0 = {0.0, 0.0}, Sa1 = {0.0, 0.0}, Sb0 = {0.0, 0.0}, Sb1 = {0.0, 0.0};
            double sa = 0.0, sb = 0.0;
            int j = 0;
            for (; j + 4 <= i; j += 4) {
                const v2d w0 = ld2(wo + j), w1 = ld2(wo + j + 2), o0 = ld2(vo + j), o1 = ld2(vo + j + 2);
                const v2d x0 = ld2(vv + j), x1 = ld2(vv + j + 2);
                const v2d a0 = (ld2(ra + j) - VOA * w0) - WOA * o0, a1 = (ld2(ra + j + 2) - VOA * w1) - WOA * o1;
                const v2d b0 = (ld2(rb + j) - VOB * w0) - WOB * o0, b1 = (ld2(rb + j + 2) - VOB * w1) - WOB * o1;
                st2(ra + j, a0);
                st2(ra + j + 2, a1);
                st2(rb + j, b0);
                st2(rb + j + 2, b1);
                Sa0 += a0 * x0;
                Sa1 += a1 * x1;
                Sb0 += b0 * x0;
                Sb1 += b1 * x1;
                st2(pp + j, (ld2(pp + j) + a0 * VA) + b0 * VB);
                st2(pp + j + 2, (ld2(pp + j + 2) + a1 * VA) + b1 * VB);
            }
            for (; j < i; ++j) {
                const double a0 = ra[j] - (voa * wo[j] + woa * vo[j]);
                const double b0 = rb[j] - (vob * wo[j] + wob * vo[j]);
                ra[j] = a0;
                rb[j] = b0;
                sa += a0 * vv[j];
                sb += b0 * vv[j];
                pp[j] += a0 * va + b0 * vb1;
            }
            // column i: the diagonal of row i and the last off-diagonal entry of row i+1
            const double da = ra[i] - (voa * wo[i] + woa * vo[i]);
            const double bi = rb[i] - (vob * wo[i] + wob * vo[i]);
            ra[i] = da;
            rb[i] = bi;
            const double db = rb[i + 1] - (vob * wo[i + 1] + wob * vo[i + 1]);
            rb[i + 1] = db;
            sb += bi * va;
            pp[i] += (((Sa0[0] + Sa0[1]) + (Sa1[0] + Sa1[1])) + sa) + da * va + bi * vb1;
            pp[i + 1] += (((Sb0[0] + Sb0[1]) + (Sb1[0] + Sb1[1])) + sb) + db * vb1;
        }
        for (; i < m; ++i) {                                      // the last row when m is odd
            double* row = A + (size_t)(k + 1 + i) * n + (k + 1);
            const double vi = vv[i], voi = pend * vo[i], woi = pend * wo[i];
            double s = 0.0;
            for (int j = 0; j < i; ++j) {
                const double r0 = row[j] - (voi * wo[j] + woi * vo[j]);
                row[j] = r0;
                s += r0 * vv[j];
                pp[j] += r0 * vi;
            }
            row[i] -= voi * wo[i] + woi * vo[i];
            pp[i] += s + row[i] * vi;
        }
        double vp = 0.0;
        for (int i = 0; i < m; ++i) {
            p[i] *= beta;
            vp += v[i] * p[i];
        }
        const double Kc = 0.5 * beta * vp;
        vb[k] = wb[k] = 0.0;
        for (int i = 0; i < m; ++i) {
            vb[k + 1 + i] = v[i];
            wb[k + 1 + i] = p[i] - Kc * v[i];
        }
        pending = beta != 0.0;
    }
    if (n >= 2) e[n - 2] = A[(size_t)(n - 1) * n + (n - 2)];
}

// State of one QR sweep in flight over the segment [lo, hi] with shift mu.
struct Sweep {
    double mu, gam, pi2, c2p, s2p;
};

// Step k of a sweep (k = lo starts it): reads a[k+1], e2[k]; writes a[k] and e2[k-1].
inline void sweep_step(double* a, double* e2, int lo, int k, Sweep& S) {
    if (k == lo) {
        S.gam = a[lo] - S.mu;
        S.pi2 = S.gam * S.gam;
        S.c2p = 1.0;
        S.s2p = 0.0;
    }
    const double b2 = e2[k];
    const double r2 = S.pi2 + b2;
    if (k > lo) e2[k - 1] = S.s2p * r2;
    const double nu = S.pi2 * (a[k + 1] - S.mu) - b2 * S.gam;
    const double gn = nu / r2;
    const double c2 = S.pi2 / r2, s2 = b2 / r2;
    a[k] = S.gam + (a[k + 1] - gn);
    S.pi2 = S.pi2 != 0.0 ? (nu * nu) / (r2 * S.pi2) : S.c2p * b2;
    S.c2p = c2;
    S.s2p = s2;
    S.gam = gn;
}

inline void sweep_end(double* a, double* e2, int hi, const Sweep& S) {
    e2[hi - 1] = S.s2p * S.pi2;
    a[hi] = S.mu + S.gam;
}

// Eigenvalues of the symmetric tridiagonal matrix (a, e2) in place in a, where e2 holds the
// SQUARES of the off-diagonal entries. One shifted QR step T - mu I = QR, T' = RQ + mu I with
// Givens rotations (c_k, s_k), written with gamma_k = c_{k-1} pi_k (pi_k: the k-th pivot of R
// before rotation k, c_0 = 1):
//   r_k^2 = pi_k^2 + b_k^2,  c_k^2 = pi_k^2 / r_k^2,  s_k^2 = b_k^2 / r_k^2,
//   gamma_{k+1} = c_k^2 (a_{k+1} - mu) - s_k^2 gamma_k,   a'_k = gamma_k + a_{k+1} - gamma_{k+1},
//   b'_{k-1}^2 = s_{k-1}^2 r_k^2,   pi_{k+1}^2 = gamma_{k+1}^2 / c_k^2 (= c_{k-1}^2 b_k^2 if c_k = 0),
// and at the end of the segment a'_hi = mu + gamma_hi, b'_{hi-1}^2 = s_{hi-1}^2 pi_hi^2.
// The chase is one long dependency chain through pi_k^2, so it is evaluated with a single
// division on that chain: with nu = pi_k^2 (a_{k+1} - mu) - b_k^2 gamma_k, gamma_{k+1} = nu / r_k^2
// and pi_{k+1}^2 = nu^2 / (r_k^2 pi_k^2); the other quotients are off the chain. Segments of four
// or more run two sweeps at once (shifts: both eigenvalues of the trailing 2x2 block), one
// trailing the other, so that two independent chains share the core.
bool tridiagonal_eigenvalues(double* a, double* e2, int n) {
    const double eps = 2.220446049250313e-16, eps2 = eps * eps;
    auto negligible = [&](int k) {
        const double t = std::fabs(a[k]) + std::fabs(a[k + 1]);
        return e2[k] <= eps2 * t * t;
    };
    int iter = 0;
    int hi = n - 1;
    while (hi > 0) {
        if (negligible(hi - 1)) {
            e2[hi - 1] = 0.0;
            --hi;
            continue;
        }
        int lo = hi - 1;
        while (lo > 0 && !negligible(lo - 1)) --lo;
        if (++iter > 60 * n) return false;
        // Wilkinson shift: the eigenvalue of the trailing 2x2 block nearer to a_hi
        const double dd = 0.5 * (a[hi - 1] - a[hi]);
        const double bb = e2[hi - 1];
        const double den = dd + (dd >= 0 ? 1.0 : -1.0) * std::sqrt(dd * dd + bb);
        const double mu = a[hi] - (den != 0.0 ? bb / den : 0.0);
        Sweep s1{mu, 0.0, 0.0, 0.0, 0.0};
        if (hi - lo < 3) {
            for (int k = lo; k < hi; ++k) sweep_step(a, e2, lo, k, s1);
            sweep_end(a, e2, hi, s1);
            continue;
        }
        // Two sweeps in flight: the second, shifted by the block's other eigenvalue, trails the
        // first by two positions (step k reads a[k+1] and e2[k], which the first sweep finished at
        // its step k+1), so the two dependency chains overlap.
        Sweep s2{(a[hi - 1] + a[hi]) - mu, 0.0, 0.0, 0.0, 0.0};
        for (int t = lo; t < hi + 2; ++t) {
            if (t < hi) sweep_step(a, e2, lo, t, s1);
            else if (t == hi) sweep_end(a, e2, hi, s1);
            if (t - 2 >= lo) sweep_step(a, e2, lo, t - 2, s2);
        }
        sweep_end(a, e2, hi, s2);
    }
    return true;
}

}  // namespace

// Eigenvalues (unsorted) of the symmetric n x n matrix A (row-major, overwritten). Returns false
// if the QR iteration did not converge.
bool symmetric_eigenvalues(double* A, int n, double* out) {
    std::vector<double> e(n > 1 ? n - 1 : 1, 0.0);
    tridiagonalize(A, n, out, e.data());
    for (double& x : e) x *= x;
    return tridiagonal_eigenvalues(out, e.data(), n);
}

}  // namespace htsvd
