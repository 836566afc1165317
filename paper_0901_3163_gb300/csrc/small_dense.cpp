// Host FP64 dense kernels for the small projected problems of one restart
// cycle (order m <= a few hundred): the eigenproblems of the regular and
// harmonic Ritz extractions, the Galerkin and least-squares solves, and
// the small factorisations of the deflation projection (arXiv:0901.3163,
// Sec. 1-2: Lan-DR uses regular Ritz vectors and a CG-type solve,
// MinRes-DR harmonic Ritz vectors and a minimum-residual solve).
//
// Methods: Householder tridiagonalisation followed by implicit symmetric QR
// steps with Wilkinson shifts (Golub & Van Loan, "Matrix Computations",
// Sec. 8.3); Householder QR for least squares; Cholesky; LU with partial
// pivoting; modified Gram-Schmidt.  All matrices are row-major.
#include "small_dense.h"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

namespace dlz {

namespace {

inline double sgn1(double x) { return x >= 0.0 ? 1.0 : -1.0; }

// Reduce symmetric a (n x n) to tridiagonal form Q^T a Q (Golub & Van Loan, Sec. 8.3.1),
// reading and updating the lower triangle only; returns d, e and, if want_q, Qt = Q^T
// (row i of Qt is column i of Q, so the later plane rotations touch two contiguous
// rows).  Q = H_0 H_1 ... is accumulated backwards (Qt = H_{n-3} ... H_0 as right
// products on the identity), so each reflector touches only the trailing block it
// acts on.  vl: the nonzero length of a Householder vector (the dense block of an
// arrowhead matrix ends early); loops stop there.
void tridiagonalise(int n, std::vector<double> &a, std::vector<double> &d, std::vector<double> &e,
                    std::vector<double> &Qt, bool want_q) {
    std::vector<double> v(n), p(n), q(n);
    std::vector<double> vs(want_q ? (size_t)n * n : 0), taus(n, 0.0);
    std::vector<int> vls(n, 0);
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;          // length of the column below the diagonal
        // a column with nothing below its subdiagonal is already reduced (the tridiagonal
        // tail of a restarted Lanczos matrix): no reflection needed
        double tail = 0.0;
        int vl = 1;
        for (int i = 1; i < m; ++i) {
            const double t = a[(size_t)(k + 1 + i) * n + k];
            tail += t * t;
            if (t != 0.0) vl = i + 1;
        }
        if (tail == 0.0) continue;
        const double x0 = a[(size_t)(k + 1) * n + k];
        const double alpha = -sgn1(x0) * std::sqrt(tail + x0 * x0);
        for (int i = 0; i < vl; ++i) v[i] = a[(size_t)(k + 1 + i) * n + k];
        v[0] -= alpha;
        double vn2 = 0.0;
        for (int i = 0; i < vl; ++i) vn2 += v[i] * v[i];
        if (vn2 == 0.0) continue;
        const double tau = 2.0 / vn2;
        // p = tau * A22 v from the lower triangle: rows i < vl give a dot over j < i and
        // an axpy into p[j < i]; rows i >= vl only a dot over j < vl
        for (int i = 0; i < m; ++i) p[i] = 0.0;
        for (int i = 0; i < vl; ++i) {
            const double *row = &a[(size_t)(k + 1 + i) * n + k + 1];
            const double vi = v[i];
            double s = 0.0;
            for (int j = 0; j < i; ++j) {
                s += row[j] * v[j];
                p[j] += row[j] * vi;
            }
            p[i] += s + row[i] * vi;
        }
        for (int i = vl; i < m; ++i) {
            const double *row = &a[(size_t)(k + 1 + i) * n + k + 1];
            double s = 0.0;
            for (int j = 0; j < vl; ++j) s += row[j] * v[j];
            p[i] = s;
        }
        double vp = 0.0;
        for (int i = 0; i < m; ++i) p[i] *= tau;
        for (int i = 0; i < vl; ++i) vp += v[i] * p[i];
        const double K = 0.5 * tau * vp;
        for (int i = 0; i < m; ++i) q[i] = p[i] - (i < vl ? K * v[i] : 0.0);
        // A22 -= v q^T + q v^T on the lower triangle (rows i >= vl: v[i] = 0, and only
        // the columns j < vl change)
        for (int i = 0; i < vl; ++i) {
            double *row = &a[(size_t)(k + 1 + i) * n + k + 1];
            const double vi = v[i], qi = q[i];
            for (int j = 0; j <= i; ++j) row[j] -= vi * q[j] + qi * v[j];
        }
        for (int i = vl; i < m; ++i) {
            double *row = &a[(size_t)(k + 1 + i) * n + k + 1];
            const double qi = q[i];
            for (int j = 0; j < vl; ++j) row[j] -= qi * v[j];
        }
        a[(size_t)(k + 1) * n + k] = alpha;
        for (int i = 1; i < vl; ++i) a[(size_t)(k + 1 + i) * n + k] = 0.0;
        if (want_q) {
            taus[k] = tau;
            vls[k] = vl;
            for (int i = 0; i < vl; ++i) vs[(size_t)k * n + i] = v[i];
        }
    }
    if (want_q) {
        Qt.assign((size_t)n * n, 0.0);
        for (int i = 0; i < n; ++i) Qt[(size_t)i * n + i] = 1.0;
        std::vector<double> w(n);
        for (int k = n - 3; k >= 0; --k) {
            if (taus[k] == 0.0) continue;
            // Qt <- Qt H_k: rows k+1..n-1, columns k+1..k+vl (the other columns of H_k
            // are those of the identity): Qt -= tau (Qt v) v^T
            const int m = n - k - 1, vl = vls[k];
            const double *vk = &vs[(size_t)k * n];
            for (int i = 0; i < m; ++i) {
                const double *row = &Qt[(size_t)(k + 1 + i) * n + k + 1];
                double s = 0.0;
                for (int j = 0; j < vl; ++j) s += row[j] * vk[j];
                w[i] = taus[k] * s;
            }
            for (int i = 0; i < m; ++i) {
                double *row = &Qt[(size_t)(k + 1 + i) * n + k + 1];
                const double wi = w[i];
                for (int j = 0; j < vl; ++j) row[j] -= wi * vk[j];
            }
        }
    }
    d.resize(n);
    e.assign(n > 1 ? n - 1 : 0, 0.0);
    for (int i = 0; i < n; ++i) d[i] = a[(size_t)i * n + i];
    for (int i = 0; i + 1 < n; ++i) e[i] = a[(size_t)(i + 1) * n + i];
}

// Implicit symmetric QR with Wilkinson shifts on (d, e); rotations accumulated into Q.
bool tridiagonal_qr(int n, std::vector<double> &d, std::vector<double> &e, std::vector<double> &Qt, bool want_q) {
    const double eps = 2.2e-16;
    int h = n - 1;
    long iter = 0;
    const long max_iter = 60L * n + 100;
    while (h > 0) {
        if (std::fabs(e[h - 1]) <= eps * (std::fabs(d[h - 1]) + std::fabs(d[h]))) {
            e[h - 1] = 0.0;
            --h;
            continue;
        }
        int l = h - 1;
        while (l > 0 && std::fabs(e[l - 1]) > eps * (std::fabs(d[l - 1]) + std::fabs(d[l]))) --l;
        if (l > 0) e[l - 1] = 0.0;
        if (++iter > max_iter) return false;
        // Wilkinson shift from the trailing 2x2 block of [l..h]
        const double delta = 0.5 * (d[h - 1] - d[h]);
        const double b = e[h - 1];
        const double mu = d[h] - b * b / (delta + sgn1(delta) * std::hypot(delta, b));
        double x = d[l] - mu, z = e[l];
        for (int k = l; k < h; ++k) {
            // plain square root unless x^2 + z^2 could over- or underflow
            const double r2 = x * x + z * z;
            const double r = (r2 > 1e-280 && r2 < 1e280) ? std::sqrt(r2) : std::hypot(x, z);
            const double ir = (r == 0.0) ? 0.0 : 1.0 / r;
            const double c = (r == 0.0) ? 1.0 : x * ir, s = z * ir;
            if (k > l) e[k - 1] = r;
            const double dk = d[k], dk1 = d[k + 1], ek = e[k];
            d[k] = c * c * dk + 2.0 * c * s * ek + s * s * dk1;
            d[k + 1] = s * s * dk - 2.0 * c * s * ek + c * c * dk1;
            e[k] = c * s * (dk1 - dk) + (c * c - s * s) * ek;
            if (k + 1 < h) {
                z = s * e[k + 1];            // bulge at (k, k+2)
                e[k + 1] = c * e[k + 1];
                x = e[k];
            }
            if (want_q) {
                // columns k, k+1 of Q = rows k, k+1 of Qt
                double *rk = &Qt[(size_t)k * n], *rk1 = &Qt[(size_t)(k + 1) * n];
                for (int r2 = 0; r2 < n; ++r2) {
                    const double qk = rk[r2], qk1 = rk1[r2];
                    rk[r2] = c * qk + s * qk1;
                    rk1[r2] = -s * qk + c * qk1;
                }
            }
        }
    }
    return true;
}

// Number of eigenvalues of the symmetric tridiagonal (d, e) below x: the negative
// pivots of the LDL^T factorisation of T - x I (Sturm sequence; Golub & Van Loan,
// Sec. 8.4), a zero pivot replaced by a tiny one.
int sturm_count(int n, const std::vector<double> &d, const std::vector<double> &e, double x, double tiny) {
    int cnt = 0;
    double q = 1.0;
    for (int i = 0; i < n; ++i) {
        q = d[i] - x - (i > 0 ? e[i - 1] * e[i - 1] / q : 0.0);
        if (q == 0.0) q = -tiny;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

// The j-th smallest eigenvalue (j = 0..n-1) of (d, e) by bisection inside [lo, hi]
// down to the spacing of doubles.
double bisect_eigenvalue(int n, const std::vector<double> &d, const std::vector<double> &e, int j, double lo,
                         double hi, double tiny) {
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi || hi - lo <= 2.2e-16 * std::max(std::fabs(lo), std::fabs(hi))) break;
        if (sturm_count(n, d, e, mid, tiny) > j) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

// Symmetrise a copy of A (against rounding in the caller) and scale it by a power of
// two so that its largest entry is near 1 (the sums of squares in the reduction then
// neither overflow nor underflow); returns the factor to multiply eigenvalues by, or
// 0 for non-finite input.
double symmetrised_scaled(int n, const double *A, std::vector<double> &a) {
    a.assign(A, A + (size_t)n * n);
    double amax = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            const double s = 0.5 * (a[(size_t)i * n + j] + a[(size_t)j * n + i]);
            a[(size_t)i * n + j] = a[(size_t)j * n + i] = s;
            amax = std::max(amax, std::fabs(s));
        }
    if (!std::isfinite(amax)) return 0.0;
    if (amax == 0.0 || (amax > 1e-100 && amax < 1e100)) return 1.0;
    int ex = 0;
    std::frexp(amax, &ex);
    for (double &v : a) v = std::ldexp(v, -ex);
    return std::ldexp(1.0, ex);
}

}  // namespace

bool sym_extremes(int n, const double *A, double *lo, double *hi) {
    if (n <= 0) return false;
    std::vector<double> a, d, e, Q;
    const double f = symmetrised_scaled(n, A, a);
    if (f == 0.0) return false;
    tridiagonalise(n, a, d, e, Q, false);
    // Gershgorin interval of the tridiagonal matrix
    double glo = 0.0, ghi = 0.0, scale = 0.0;
    for (int i = 0; i < n; ++i) {
        const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(e[i]) : 0.0);
        glo = (i == 0) ? d[i] - r : std::min(glo, d[i] - r);
        ghi = (i == 0) ? d[i] + r : std::max(ghi, d[i] + r);
        scale = std::max(scale, std::fabs(d[i]) + r);
    }
    if (!std::isfinite(scale)) return false;
    const double pad = 1e-14 * scale + 1e-300;
    glo -= pad;
    ghi += pad;
    const double tiny = 1e-300 + 1e-30 * scale;
    *lo = f * bisect_eigenvalue(n, d, e, 0, glo, ghi, tiny);
    *hi = f * bisect_eigenvalue(n, d, e, n - 1, glo, ghi, tiny);
    return true;
}

bool sym_eig(int n, const double *A, double *w, double *Z) {
    if (n <= 0) return true;
    std::vector<double> a, d, e, Q;
    const double f = symmetrised_scaled(n, A, a);
    if (f == 0.0) return false;
    const bool want_q = Z != nullptr;
    tridiagonalise(n, a, d, e, Q, want_q);
    if (!tridiagonal_qr(n, d, e, Q, want_q)) return false;
    std::vector<int> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return d[x] < d[y]; });
    for (int j = 0; j < n; ++j) {
        w[j] = f * d[idx[j]];
        if (want_q)
            for (int i = 0; i < n; ++i) Z[(size_t)i * n + j] = Q[(size_t)idx[j] * n + i];
    }
    return true;
}

bool lstsq(int rows, int cols, const double *T, const double *c, double *y, double *q) {
    if (rows <= cols || cols <= 0) return false;
    std::vector<double> a(T, T + (size_t)rows * cols), b(c, c + rows);
    std::vector<std::vector<double>> vs(cols);
    std::vector<double> taus(cols, 0.0);
    std::vector<int> ends(cols);
    for (int k = 0; k < cols; ++k) {
        // rows k..end-1 hold the nonzeros of column k (banded below the dense block)
        int end = rows;
        while (end > k + 1 && a[(size_t)(end - 1) * cols + k] == 0.0) --end;
        ends[k] = end;
        double alpha = 0.0;
        for (int i = k; i < end; ++i) alpha += a[(size_t)i * cols + k] * a[(size_t)i * cols + k];
        alpha = std::sqrt(alpha);
        std::vector<double> &v = vs[k];
        v.assign(rows - k, 0.0);
        if (alpha == 0.0) return false;
        alpha = -sgn1(a[(size_t)k * cols + k]) * alpha;
        for (int i = k; i < end; ++i) v[i - k] = a[(size_t)i * cols + k];
        v[0] -= alpha;
        double vn2 = 0.0;
        for (int i = k; i < end; ++i) vn2 += v[i - k] * v[i - k];
        const double tau = (vn2 == 0.0) ? 0.0 : 2.0 / vn2;
        taus[k] = tau;
        for (int j = k; j < cols; ++j) {
            double s = 0.0;
            for (int i = k; i < end; ++i) s += v[i - k] * a[(size_t)i * cols + j];
            if (s == 0.0) continue;
            s *= tau;
            for (int i = k; i < end; ++i) a[(size_t)i * cols + j] -= s * v[i - k];
        }
        double s = 0.0;
        for (int i = k; i < end; ++i) s += v[i - k] * b[i];
        s *= tau;
        for (int i = k; i < end; ++i) b[i] -= s * v[i - k];
    }
    for (int k = cols - 1; k >= 0; --k) {
        double s = b[k];
        for (int j = k + 1; j < cols; ++j) s -= a[(size_t)k * cols + j] * y[j];
        const double r = a[(size_t)k * cols + k];
        if (r == 0.0) return false;
        y[k] = s / r;
    }
    if (q) {
        // q = H_0 H_1 ... H_{cols-1} e_{rows-1}: the last column of the full Q
        std::vector<double> u(rows, 0.0);
        u[rows - 1] = 1.0;
        for (int k = cols - 1; k >= 0; --k) {
            const std::vector<double> &v = vs[k];
            double s = 0.0;
            for (int i = k; i < ends[k]; ++i) s += v[i - k] * u[i];
            s *= taus[k];
            for (int i = k; i < ends[k]; ++i) u[i] -= s * v[i - k];
        }
        for (int i = 0; i < rows; ++i) q[i] = u[i];
    }
    return true;
}

bool cholesky(int n, const double *A, double *L) {
    // the factor keeps the envelope of A (first nonzero column per row), so loops start there
    std::vector<int> first(n);
    for (int i = 0; i < n; ++i) {
        int f = 0;
        while (f < i && A[(size_t)i * n + f] == 0.0) ++f;
        first[i] = f;
    }
    for (int i = 0; i < n * n; ++i) L[i] = 0.0;
    for (int j = 0; j < n; ++j) {
        double s = A[(size_t)j * n + j];
        for (int k = first[j]; k < j; ++k) s -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(s > 0.0)) return false;
        const double ljj = std::sqrt(s);
        L[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            if (first[i] > j) continue;
            double t = A[(size_t)i * n + j];
            for (int k = std::max(first[i], first[j]); k < j; ++k) t -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = t / ljj;
        }
    }
    return true;
}

// first nonzero column of each row of a lower-triangular L (its envelope)
void envelope(int n, const double *L, std::vector<int> &first) {
    first.assign(n, 0);
    for (int i = 0; i < n; ++i) {
        int f = 0;
        while (f < i && L[(size_t)i * n + f] == 0.0) ++f;
        first[i] = f;
    }
}

void lower_solve(int n, const double *L, double *b, const int *first_in) {
    std::vector<int> own;
    const int *first = first_in;
    if (!first) { envelope(n, L, own); first = own.data(); }
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = first[i]; k < i; ++k) s -= L[(size_t)i * n + k] * b[k];
        b[i] = s / L[(size_t)i * n + i];
    }
}

void upper_t_solve(int n, const double *L, double *b, const int *first_in) {
    // solve L^T x = b
    std::vector<int> own;
    const int *first = first_in;
    if (!first) { envelope(n, L, own); first = own.data(); }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int k = i + 1; k < n; ++k)
            if (first[k] <= i) s -= L[(size_t)k * n + i] * b[k];
        b[i] = s / L[(size_t)i * n + i];
    }
}

void lower_solve_rows(int n, const double *L, double *B, int nrhs, const int *first) {
    // row i of X = (row i of B - sum_k L[i][k] row k of X) / L[i][i]: per column the
    // same operations, in the same order, as lower_solve
    for (int i = 0; i < n; ++i) {
        double *bi = B + (size_t)i * nrhs;
        for (int k = first[i]; k < i; ++k) {
            const double l = L[(size_t)i * n + k];
            const double *bk = B + (size_t)k * nrhs;
            for (int j = 0; j < nrhs; ++j) bi[j] -= l * bk[j];
        }
        const double d = L[(size_t)i * n + i];
        for (int j = 0; j < nrhs; ++j) bi[j] /= d;
    }
}

void upper_t_solve_rows(int n, const double *L, double *B, int nrhs, const int *first) {
    for (int i = n - 1; i >= 0; --i) {
        double *bi = B + (size_t)i * nrhs;
        for (int k = i + 1; k < n; ++k) {
            if (first[k] > i) continue;
            const double l = L[(size_t)k * n + i];
            const double *bk = B + (size_t)k * nrhs;
            for (int j = 0; j < nrhs; ++j) bi[j] -= l * bk[j];
        }
        const double d = L[(size_t)i * n + i];
        for (int j = 0; j < nrhs; ++j) bi[j] /= d;
    }
}

template <typename S>
static bool lu_factor_t(int n, S *A, int *piv) {
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = std::abs(A[(size_t)k * n + k]);
        for (int i = k + 1; i < n; ++i)
            if (std::abs(A[(size_t)i * n + k]) > best) { best = std::abs(A[(size_t)i * n + k]); p = i; }
        piv[k] = p;
        if (best == 0.0) return false;
        if (p != k)
            for (int j = 0; j < n; ++j) std::swap(A[(size_t)k * n + j], A[(size_t)p * n + j]);
        for (int i = k + 1; i < n; ++i) {
            const S f = A[(size_t)i * n + k] / A[(size_t)k * n + k];
            A[(size_t)i * n + k] = f;
            for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= f * A[(size_t)k * n + j];
        }
    }
    return true;
}

template <typename S>
static void lu_solve_t(int n, const S *LU, const int *piv, S *b) {
    for (int k = 0; k < n; ++k)
        if (piv[k] != k) std::swap(b[k], b[piv[k]]);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < i; ++k) b[i] -= LU[(size_t)i * n + k] * b[k];
    for (int i = n - 1; i >= 0; --i) {
        for (int k = i + 1; k < n; ++k) b[i] -= LU[(size_t)i * n + k] * b[k];
        b[i] /= LU[(size_t)i * n + i];
    }
}

bool lu_factor(int n, double *A, int *piv) { return lu_factor_t(n, A, piv); }
void lu_solve(int n, const double *LU, const int *piv, double *b) { lu_solve_t(n, LU, piv, b); }
bool lu_factor(int n, std::complex<double> *A, int *piv) { return lu_factor_t(n, A, piv); }
void lu_solve(int n, const std::complex<double> *LU, const int *piv, std::complex<double> *b) {
    lu_solve_t(n, LU, piv, b);
}

bool mgs_columns(int rows, int cols, double *P) {
    // on a column-major copy, so that every column is contiguous
    std::vector<double> Q((size_t)rows * cols);
    for (int r = 0; r < rows; ++r)
        for (int j = 0; j < cols; ++j) Q[(size_t)j * rows + r] = P[(size_t)r * cols + j];
    for (int j = 0; j < cols; ++j) {
        double *pj = &Q[(size_t)j * rows];
        for (int pass = 0; pass < 2; ++pass)
            for (int i = 0; i < j; ++i) {
                const double *pi = &Q[(size_t)i * rows];
                double s = 0.0;
                for (int r = 0; r < rows; ++r) s += pi[r] * pj[r];
                for (int r = 0; r < rows; ++r) pj[r] -= s * pi[r];
            }
        double nrm = 0.0;
        for (int r = 0; r < rows; ++r) nrm += pj[r] * pj[r];
        nrm = std::sqrt(nrm);
        if (!(nrm > 0.0)) return false;
        for (int r = 0; r < rows; ++r) pj[r] /= nrm;
    }
    for (int r = 0; r < rows; ++r)
        for (int j = 0; j < cols; ++j) P[(size_t)r * cols + j] = Q[(size_t)j * rows + r];
    return true;
}

}  // namespace dlz

extern "C" int dlz_host_symeig(int n, const double *A, double *w, double *Z) {
    if (n < 0 || (n > 0 && (!A || !w || !Z))) return DLZ_ERR_BADARG;
    return dlz::sym_eig(n, A, w, Z) ? DLZ_OK : DLZ_ERR_NONFINITE;
}

extern "C" int dlz_host_sym_extremes(int n, const double *A, double *lo, double *hi) {
    if (n <= 0 || !A || !lo || !hi) return DLZ_ERR_BADARG;
    return dlz::sym_extremes(n, A, lo, hi) ? DLZ_OK : DLZ_ERR_NONFINITE;
}

extern "C" int dlz_host_lstsq(int rows, int cols, const double *T, const double *c, double *y,
                              double *q) {
    if (rows <= cols || cols <= 0 || !T || !c || !y) return DLZ_ERR_BADARG;
    return dlz::lstsq(rows, cols, T, c, y, q) ? DLZ_OK : DLZ_ERR_BREAKDOWN;
}
