// Host FP64 complex dense helpers for the small problems of GMRES-DR (the
// non-hermitian deflated method the paper contrasts with, its refs. [1], [2]):
// the eigen-decomposition of a general complex matrix (harmonic Ritz pairs) and the
// least-squares solve of the (m+1) x m Arnoldi matrix.  Row-major storage.
//
// Eigen-decomposition (Golub & Van Loan, 7.4-7.6): Householder reduction to upper
// Hessenberg form, then single-shift QR iterations with Givens rotations (Wilkinson
// shift from the trailing 2 x 2 block, an exceptional shift every 12 iterations without
// deflation) to the Schur form T = Q^H A Q, and the eigenvectors of T by back
// substitution, mapped back by Q and normalised.
#include <algorithm>
#include <cmath>
#include <complex>
#include <limits>
#include <vector>

#include "small_dense.h"

namespace dlz {

namespace {

typedef std::complex<double> zc;

// Householder vector for x (length len): returns v (v[0] = 1 scaled) and beta with
// (I - beta v v^H) x = alpha e_1, |alpha| = ||x||.  beta = 0 when x is already e_1-aligned.
void householder(const zc *x, int len, std::vector<zc> &v, double &beta, zc &alpha) {
    double nrm2 = 0.0;
    for (int i = 0; i < len; ++i) nrm2 += std::norm(x[i]);
    const double nrm = std::sqrt(nrm2);
    v.assign(x, x + len);
    double tail = nrm2 - std::norm(x[0]);
    if (nrm == 0.0 || tail <= 0.0) {
        beta = 0.0;
        alpha = x[0];
        return;
    }
    const zc ph = std::abs(x[0]) > 0 ? x[0] / std::abs(x[0]) : zc(1.0, 0.0);
    alpha = -ph * nrm;
    v[0] = x[0] - alpha;
    double vn2 = std::norm(v[0]) + tail;
    beta = 2.0 / vn2;
}

}  // namespace

bool zgeev(int n, const zc *A, zc *w, zc *Z) {
    if (n <= 0) return true;
    for (int i = 0; i < n * n; ++i)
        if (!std::isfinite(A[i].real()) || !std::isfinite(A[i].imag())) return false;
    std::vector<zc> H(A, A + (size_t)n * n), Q((size_t)n * n, zc(0, 0));
    for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
    auto h = [&](int i, int j) -> zc & { return H[(size_t)i * n + j]; };
    auto q = [&](int i, int j) -> zc & { return Q[(size_t)i * n + j]; };
    // ---- Hessenberg reduction: H <- P H P, Q <- Q P for P = I - beta v v^H on rows/cols k+1..n-1
    std::vector<zc> v;
    for (int k = 0; k + 2 < n; ++k) {
        std::vector<zc> x(n - k - 1);
        for (int i = k + 1; i < n; ++i) x[i - k - 1] = h(i, k);
        double beta;
        zc alpha;
        householder(x.data(), n - k - 1, v, beta, alpha);
        if (beta == 0.0) continue;
        const int len = n - k - 1;
        for (int j = 0; j < n; ++j) {              // left: rows k+1.. of every column
            zc s = 0.0;
            for (int i = 0; i < len; ++i) s += std::conj(v[i]) * h(k + 1 + i, j);
            s *= beta;
            for (int i = 0; i < len; ++i) h(k + 1 + i, j) -= v[i] * s;
        }
        for (int i = 0; i < n; ++i) {              // right: columns k+1.. of every row
            zc s = 0.0;
            for (int j = 0; j < len; ++j) s += h(i, k + 1 + j) * v[j];
            s *= beta;
            for (int j = 0; j < len; ++j) h(i, k + 1 + j) -= s * std::conj(v[j]);
            zc sq = 0.0;
            for (int j = 0; j < len; ++j) sq += q(i, k + 1 + j) * v[j];
            sq *= beta;
            for (int j = 0; j < len; ++j) q(i, k + 1 + j) -= sq * std::conj(v[j]);
        }
        for (int i = k + 2; i < n; ++i) h(i, k) = 0.0;
    }
    // ---- shifted QR iterations to upper triangular form
    const double eps = std::numeric_limits<double>::epsilon();
    int hi = n - 1, iter = 0, total = 0;
    std::vector<double> cs(n);
    std::vector<zc> sn(n);
    while (hi > 0) {
        int l = hi;
        for (; l > 0; --l) {
            const double s = std::abs(h(l - 1, l - 1)) + std::abs(h(l, l));
            if (std::abs(h(l, l - 1)) <= eps * (s > 0 ? s : 1.0)) {
                h(l, l - 1) = 0.0;
                break;
            }
        }
        if (l == hi) {
            --hi;
            iter = 0;
            continue;
        }
        if (++total > 60 * n) return false;
        ++iter;
        zc mu;
        if (iter % 12 == 0) {
            mu = h(hi, hi) + std::abs(h(hi, hi - 1));     // exceptional shift
        } else {
            const zc a = h(hi - 1, hi - 1), b = h(hi - 1, hi), c = h(hi, hi - 1), d = h(hi, hi);
            const zc half = 0.5 * (a - d);
            const zc disc = std::sqrt(half * half + b * c);
            const zc m1 = 0.5 * (a + d) + disc, m2 = 0.5 * (a + d) - disc;
            mu = std::abs(m1 - d) < std::abs(m2 - d) ? m1 : m2;
        }
        for (int i = l; i <= hi; ++i) h(i, i) -= mu;
        // H - mu = G^H R: rotations on rows k, k+1 zero H(k+1, k)
        for (int k = l; k < hi; ++k) {
            const zc a = h(k, k), b = h(k + 1, k);
            const double r = std::sqrt(std::norm(a) + std::norm(b));
            double c;
            zc s;
            if (r == 0.0) {
                c = 1.0;
                s = 0.0;
            } else if (std::abs(a) == 0.0) {
                c = 0.0;
                s = std::conj(b) / r;
            } else {
                c = std::abs(a) / r;
                s = (a / std::abs(a)) * std::conj(b) / r;
            }
            cs[k] = c;
            sn[k] = s;
            for (int j = k; j < n; ++j) {          // the whole row (Schur form beyond the window)
                const zc u = h(k, j), t = h(k + 1, j);
                h(k, j) = c * u + s * t;
                h(k + 1, j) = -std::conj(s) * u + c * t;
            }
        }
        // R G + mu: rotations on columns k, k+1 (all rows above), and Q <- Q G
        for (int k = l; k < hi; ++k) {
            const double c = cs[k];
            const zc s = sn[k];
            for (int i = 0; i <= std::min(k + 1, hi); ++i) {
                const zc u = h(i, k), t = h(i, k + 1);
                h(i, k) = c * u + std::conj(s) * t;
                h(i, k + 1) = -s * u + c * t;
            }
            for (int i = 0; i < n; ++i) {
                const zc u = q(i, k), t = q(i, k + 1);
                q(i, k) = c * u + std::conj(s) * t;
                q(i, k + 1) = -s * u + c * t;
            }
        }
        for (int i = l; i <= hi; ++i) h(i, i) += mu;
    }
    for (int i = 0; i < n; ++i) w[i] = h(i, i);
    if (!Z) return true;
    // ---- eigenvectors of T by back substitution, then Z = Q z
    double tn = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = i; j < n; ++j) tn = std::max(tn, std::abs(h(i, j)));
    const double small = eps * (tn > 0 ? tn : 1.0);
    std::vector<zc> z(n);
    for (int i = 0; i < n; ++i) {
        std::fill(z.begin(), z.end(), zc(0, 0));
        z[i] = 1.0;
        for (int j = i - 1; j >= 0; --j) {
            zc s = 0.0;
            for (int l = j + 1; l <= i; ++l) s += h(j, l) * z[l];
            zc den = h(j, j) - h(i, i);
            if (std::abs(den) < small) den = small;
            z[j] = -s / den;
        }
        double nrm2 = 0.0;
        for (int r = 0; r < n; ++r) {
            zc s = 0.0;
            for (int l = 0; l <= i; ++l) s += q(r, l) * z[l];
            Z[(size_t)r * n + i] = s;
            nrm2 += std::norm(s);
        }
        const double inv = 1.0 / std::sqrt(nrm2);
        for (int r = 0; r < n; ++r) Z[(size_t)r * n + i] *= inv;
    }
    return true;
}

bool zlstsq(int rows, int cols, const zc *A, const zc *c, zc *y, zc *qperp) {
    // Householder QR of A (rows x cols, rows > cols): R y = (Q^H c)[:cols]
    std::vector<zc> R(A, A + (size_t)rows * cols), b(c, c + rows);
    std::vector<std::vector<zc>> vs(cols);
    std::vector<double> betas(cols);
    std::vector<zc> x;
    for (int k = 0; k < cols; ++k) {
        x.resize(rows - k);
        for (int i = k; i < rows; ++i) x[i - k] = R[(size_t)i * cols + k];
        zc alpha;
        householder(x.data(), rows - k, vs[k], betas[k], alpha);
        const std::vector<zc> &v = vs[k];
        const double beta = betas[k];
        if (beta == 0.0) continue;
        for (int j = k; j < cols; ++j) {
            zc s = 0.0;
            for (int i = k; i < rows; ++i) s += std::conj(v[i - k]) * R[(size_t)i * cols + j];
            s *= beta;
            for (int i = k; i < rows; ++i) R[(size_t)i * cols + j] -= v[i - k] * s;
        }
        zc s = 0.0;
        for (int i = k; i < rows; ++i) s += std::conj(v[i - k]) * b[i];
        s *= beta;
        for (int i = k; i < rows; ++i) b[i] -= v[i - k] * s;
    }
    for (int i = cols - 1; i >= 0; --i) {
        zc s = b[i];
        for (int j = i + 1; j < cols; ++j) s -= R[(size_t)i * cols + j] * y[j];
        const zc d = R[(size_t)i * cols + i];
        if (std::abs(d) == 0.0) return false;
        y[i] = s / d;
    }
    if (qperp && rows == cols + 1) {
        // the last column of the complete Q: H_0 H_1 ... H_{cols-1} e_last
        std::vector<zc> e(rows, zc(0, 0));
        e[rows - 1] = 1.0;
        for (int k = cols - 1; k >= 0; --k) {
            const std::vector<zc> &v = vs[k];
            const double beta = betas[k];
            if (beta == 0.0) continue;
            zc s = 0.0;
            for (int i = k; i < rows; ++i) s += std::conj(v[i - k]) * e[i];
            s *= beta;
            for (int i = k; i < rows; ++i) e[i] -= v[i - k] * s;
        }
        for (int i = 0; i < rows; ++i) qperp[i] = e[i];
    }
    return true;
}

bool zmgs_columns(int rows, int cols, zc *P) {
    for (int j = 0; j < cols; ++j) {
        for (int pass = 0; pass < 2; ++pass)
            for (int i = 0; i < j; ++i) {
                zc d = 0.0;
                for (int r = 0; r < rows; ++r) d += std::conj(P[(size_t)r * cols + i]) * P[(size_t)r * cols + j];
                for (int r = 0; r < rows; ++r) P[(size_t)r * cols + j] -= d * P[(size_t)r * cols + i];
            }
        double nrm2 = 0.0;
        for (int r = 0; r < rows; ++r) nrm2 += std::norm(P[(size_t)r * cols + j]);
        if (!(nrm2 > 0.0)) return false;
        const double inv = 1.0 / std::sqrt(nrm2);
        for (int r = 0; r < rows; ++r) P[(size_t)r * cols + j] *= inv;
    }
    return true;
}

}  // namespace dlz

extern "C" int dlz_host_zgeev(int n, const double *A, double *w, double *Z) {
    if (n < 0 || (n > 0 && (!A || !w))) return DLZ_ERR_BADARG;
    typedef std::complex<double> zc;
    return dlz::zgeev(n, reinterpret_cast<const zc *>(A), reinterpret_cast<zc *>(w), reinterpret_cast<zc *>(Z))
               ? DLZ_OK
               : DLZ_ERR_NONFINITE;
}

extern "C" int dlz_host_zlstsq(int rows, int cols, const double *A, const double *c, double *y, double *q) {
    if (rows <= cols || cols <= 0 || !A || !c || !y) return DLZ_ERR_BADARG;
    typedef std::complex<double> zc;
    return dlz::zlstsq(rows, cols, reinterpret_cast<const zc *>(A), reinterpret_cast<const zc *>(c),
                       reinterpret_cast<zc *>(y), reinterpret_cast<zc *>(q))
               ? DLZ_OK
               : DLZ_ERR_NONFINITE;
}
