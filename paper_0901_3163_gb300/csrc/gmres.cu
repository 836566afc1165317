// GMRES-DR(m,k) and D-GMRES(m) on the Wilson matrix D itself (non-hermitian), FP64:
// the deflated methods for non-hermitian systems that arXiv:0901.3163 contrasts its
// hermitian Lan-DR / MinRes-DR with (its refs. [1], [2]; Sec. 1).
//
// GMRES-DR: Arnoldi with classical Gram-Schmidt applied twice (the coefficients of both
// passes and the new norm stay on the device: no host round trip per step), then on
// the host the least-squares solve of the (m+1) x m Arnoldi matrix, the k harmonic Ritz
// pairs of smallest |theta| (eigenpairs of H_m + |h_{m+1,m}|^2 H_m^{-H} e_m e_m^H) and
// the restart V_{k+1} = V_{m+1} P with P = orthonormalise([[G_k; 0], q]), q spanning
// range(Hbar_m)^perp (the direction of the least-squares residual).  The kept space
// satisfies D V_k = V_{k+1} Hbar_k and is handed to D-GMRES.
// D-GMRES: for each later right-hand side, a minimum-residual projection over span(V_k)
// (y = argmin ||V_{k+1}^H r - Hbar_k y||), then one GMRES(m) cycle, repeated until the
// FP64 residual ||b - D x|| / ||b|| reaches tol.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "dlz_internal.cuh"
#include "krylov_util.cuh"
#include "reduce.cuh"
#include "small_dense.h"
#include "solvers.h"

namespace dlz {

namespace {

typedef std::complex<double> zc;

// Device work of an Arnoldi run with at most m steps.
struct ArnoldiBufs {
    DevBuf h1, h2, nrm, coef;
    int alloc(int m) {
        DLZ_TRY(h1.alloc((size_t)m * (m + 1) * sizeof(double2)));
        DLZ_TRY(h2.alloc((size_t)m * (m + 1) * sizeof(double2)));
        DLZ_TRY(nrm.alloc((size_t)(m + 1) * sizeof(double)));
        DLZ_TRY(coef.alloc((size_t)(m + 1) * (m + 2) * sizeof(double2)));
        return DLZ_OK;
    }
};

// Arnoldi steps j0 .. m-1 on the basis V ((m+1) vectors of n): w = D v_j, two passes of
// classical Gram-Schmidt against v_0 .. v_j (the negated coefficients of pass p go to
// h_p[j][0..j]), ||w||^2 to nrm[j], v_{j+1} = w / ||w||.  Then the new columns of Hbar
// on the host (H row-major (m+1) x m).  mvps: products with D.
int arnoldi(Op &op, double2 *V, long n, int j0, int m, double2 *w, ArnoldiBufs &ab, std::vector<zc> &H,
            long long &mvps) {
    double2 *h1 = ab.h1.as<double2>(), *h2 = ab.h2.as<double2>();
    double *nrm = ab.nrm.as<double>();
    for (int j = j0; j < m; ++j) {
        const double2 *vj = V + (size_t)j * n;
        DLZ_TRY(wilson64(op, w, vj, DLZ_D));
        ++mvps;
        double2 *c1 = h1 + (size_t)j * (m + 1), *c2 = h2 + (size_t)j * (m + 1);
        DLZ_TRY(v64::multidot(op, V, n, j + 1, w, c1, -1.0));
        DLZ_TRY(combine64(op, w, n, 1, V, n, j + 1, c1, 1, false, true));
        DLZ_TRY(v64::multidot(op, V, n, j + 1, w, c2, -1.0));
        DLZ_TRY(combine64(op, w, n, 1, V, n, j + 1, c2, 1, false, true));
        DLZ_TRY(v64::norm2_diff(op, w, nullptr, nrm + j));
        double2 *vn = V + (size_t)(j + 1) * n;
        const double *nj = nrm + j;
        const double2 *wc = w;
        DLZ_TRY(map(op, n, [=] __device__(long i) {
            const double s = 1.0 / sqrt(*nj);
            const double2 a = wc[i];
            vn[i] = make_double2(s * a.x, s * a.y);
        }));
    }
    if (j0 >= m) return DLZ_OK;
    std::vector<double2> a((size_t)m * (m + 1)), b((size_t)m * (m + 1));
    std::vector<double> nv(m);
    DLZ_TRY(d2h_sync(op, a.data(), h1, a.size() * sizeof(double2)));
    DLZ_TRY(d2h_sync(op, b.data(), h2, b.size() * sizeof(double2)));
    DLZ_TRY(d2h_sync(op, nv.data(), nrm, m * sizeof(double)));
    for (int j = j0; j < m; ++j) {
        for (int i = 0; i <= j; ++i) {
            const double2 u = a[(size_t)j * (m + 1) + i], v = b[(size_t)j * (m + 1) + i];
            H[(size_t)i * m + j] += zc(-(u.x + v.x), -(u.y + v.y));
        }
        if (!std::isfinite(nv[j])) return fail(DLZ_ERR_NONFINITE, "Arnoldi norm not finite");
        if (!(nv[j] > 0.0)) return fail(DLZ_ERR_BREAKDOWN, "Arnoldi breakdown (invariant subspace)");
        H[(size_t)(j + 1) * m + j] = std::sqrt(nv[j]);
    }
    return DLZ_OK;
}

// x += V_l y (l = y.size()); coef: device scratch of at least l complex values
int add_combination(Op &op, double2 *x, const double2 *V, long n, const std::vector<zc> &y, double2 *coef) {
    std::vector<double2> hy(y.size());
    for (size_t i = 0; i < y.size(); ++i) hy[i] = make_double2(y[i].real(), y[i].imag());
    DLZ_TRY(h2d(op, coef, hy.data(), hy.size() * sizeof(double2)));
    return combine64(op, x, n, 1, V, n, (int)y.size(), coef, 1, false, true);
}

// ||b - D x|| (relative to bnorm); r receives b - D x
int true_residual(Op &op, const double2 *b, const double2 *x, double2 *r, double *dev, double bnorm, double &rel,
                  long long &mvps) {
    DLZ_TRY(wilson64(op, r, x, DLZ_D));
    ++mvps;
    const long n = 12L * op.g.V;
    double2 *rr = r;
    DLZ_TRY(map(op, n, [=] __device__(long i) {
        const double2 u = b[i], v = rr[i];
        rr[i] = make_double2(u.x - v.x, u.y - v.y);
    }));
    DLZ_TRY(v64::norm2_diff(op, r, nullptr, dev));
    double h = 0.0;
    DLZ_TRY(d2h_sync(op, &h, dev, sizeof(double)));
    rel = std::sqrt(h) / bnorm;
    if (!std::isfinite(rel)) return fail(DLZ_ERR_NONFINITE, "residual is not finite");
    return DLZ_OK;
}

}  // namespace

int gmresdr64(Op &op, const double2 *b, double2 *x_out, const dlz_params &p, dlz_defl_s **defl_out, dlz_stats &st) {
    const int m = p.m, k = p.k;
    const long n = 12L * op.g.V;
    DevBuf Va, Vb, w, x, r, scal;
    DLZ_TRY(Va.alloc((size_t)(m + 1) * n * sizeof(double2)));
    DLZ_TRY(Vb.alloc((size_t)(m + 1) * n * sizeof(double2)));
    DLZ_TRY(w.alloc(n * sizeof(double2)));
    DLZ_TRY(x.alloc(n * sizeof(double2)));
    DLZ_TRY(r.alloc(n * sizeof(double2)));
    DLZ_TRY(scal.alloc(8 * sizeof(double)));
    ArnoldiBufs ab;
    DLZ_TRY(ab.alloc(m));
    double *dn = scal.as<double>();
    DLZ_TRY(v64::norm2_diff(op, b, nullptr, dn));
    double h = 0.0;
    DLZ_TRY(d2h_sync(op, &h, dn, sizeof(double)));
    const double bnorm = std::sqrt(h);
    if (!std::isfinite(bnorm)) return fail(DLZ_ERR_NONFINITE, "right-hand side is not finite");
    DLZ_TRY(v64::zero(op, x.as<double2>()));
    if (bnorm == 0.0) {
        DLZ_TRY(v64::copy(op, x_out, x.as<double2>()));
        st.converged = 1;
        return DLZ_OK;
    }
    double2 *V = Va.as<double2>(), *Vn = Vb.as<double2>();
    {
        const double s = 1.0 / bnorm;
        double2 *v0 = V;
        DLZ_TRY(map(op, n, [=] __device__(long i) { const double2 a = b[i]; v0[i] = make_double2(s * a.x, s * a.y); }));
    }
    std::vector<zc> H((size_t)(m + 1) * m, zc(0, 0)), c(m + 1, zc(0, 0)), theta;
    std::vector<zc> Pk;                 // (m+1) x (k+1) restart matrix of the last cycle
    c[0] = bnorm;
    int j0 = 0, cycle = 0;
    bool converged = false;
    double rel = 1.0;
    for (cycle = 0; cycle < p.max_cycles; ++cycle) {
        DLZ_TRY(arnoldi(op, V, n, j0, m, w.as<double2>(), ab, H, st.mvps));
        st.iterations += m - j0;
        // least squares and x update
        std::vector<zc> y(m), q(m + 1);
        if (!zlstsq(m + 1, m, H.data(), c.data(), y.data(), q.data()))
            return fail(DLZ_ERR_BREAKDOWN, "GMRES-DR least squares: singular Arnoldi matrix");
        std::vector<zc> s(c);
        for (int i = 0; i <= m; ++i)
            for (int j = 0; j < m; ++j) s[i] -= H[(size_t)i * m + j] * y[j];
        DLZ_TRY(add_combination(op, x.as<double2>(), V, n, y, ab.coef.as<double2>()));
        DLZ_TRY(true_residual(op, b, x.as<double2>(), r.as<double2>(), dn, bnorm, rel, st.mvps));
        st.true_residual = rel;
        // harmonic Ritz pairs: eig(H_m + |h_{m+1,m}|^2 f e_m^T), f = H_m^{-H} e_m
        std::vector<zc> Hm((size_t)m * m), Ht((size_t)m * m), f(m, zc(0, 0));
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                Hm[(size_t)i * m + j] = H[(size_t)i * m + j];
                Ht[(size_t)i * m + j] = std::conj(H[(size_t)j * m + i]);
            }
        std::vector<int> piv(m);
        if (!lu_factor(m, Ht.data(), piv.data())) return fail(DLZ_ERR_BREAKDOWN, "GMRES-DR: singular H_m");
        f[m - 1] = 1.0;
        lu_solve(m, Ht.data(), piv.data(), f.data());
        const double hm2 = std::norm(H[(size_t)m * m + (m - 1)]);
        for (int i = 0; i < m; ++i) Hm[(size_t)i * m + (m - 1)] += hm2 * f[i];
        std::vector<zc> ev(m), Z((size_t)m * m);
        if (!zgeev(m, Hm.data(), ev.data(), Z.data())) return fail(DLZ_ERR_NONFINITE, "GMRES-DR: harmonic eigenproblem");
        std::vector<int> order(m);
        for (int i = 0; i < m; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int bb) { return std::abs(ev[a]) < std::abs(ev[bb]); });
        theta.assign(k, zc(0, 0));
        // P = orthonormalise([[G_k; 0], q]), q phased like s
        Pk.assign((size_t)(m + 1) * (k + 1), zc(0, 0));
        for (int l = 0; l < k; ++l) {
            theta[l] = ev[order[l]];
            for (int i = 0; i < m; ++i) Pk[(size_t)i * (k + 1) + l] = Z[(size_t)i * m + order[l]];
        }
        zc ph(0, 0);
        for (int i = 0; i <= m; ++i) ph += std::conj(q[i]) * s[i];
        const zc u = std::abs(ph) > 0 ? ph / std::abs(ph) : zc(1, 0);
        for (int i = 0; i <= m; ++i) Pk[(size_t)i * (k + 1) + k] = q[i] * u;
        if (!zmgs_columns(m + 1, k + 1, Pk.data())) return fail(DLZ_ERR_BREAKDOWN, "GMRES-DR: dependent restart vectors");
        // V_{k+1} <- V_{m+1} P
        {
            std::vector<double2> pd(Pk.size());
            for (size_t i = 0; i < Pk.size(); ++i) pd[i] = make_double2(Pk[i].real(), Pk[i].imag());
            DLZ_TRY(h2d(op, ab.coef.as<double2>(), pd.data(), pd.size() * sizeof(double2)));
            DLZ_TRY(combine64(op, Vn, n, k + 1, V, n, m + 1, ab.coef.as<double2>(), k + 1, false, false));
        }
        // Hbar_k = P^H Hbar_m P[:m, :k]; c = P^H s
        std::vector<zc> HP((size_t)(m + 1) * k, zc(0, 0)), Hn((size_t)(m + 1) * m, zc(0, 0)), cn(m + 1, zc(0, 0));
        for (int i = 0; i <= m; ++i)
            for (int l = 0; l < k; ++l) {
                zc acc = 0.0;
                for (int j = 0; j < m; ++j) acc += H[(size_t)i * m + j] * Pk[(size_t)j * (k + 1) + l];
                HP[(size_t)i * k + l] = acc;
            }
        for (int a = 0; a <= k; ++a) {
            for (int l = 0; l < k; ++l) {
                zc acc = 0.0;
                for (int i = 0; i <= m; ++i) acc += std::conj(Pk[(size_t)i * (k + 1) + a]) * HP[(size_t)i * k + l];
                Hn[(size_t)a * m + l] = acc;
            }
            zc acc = 0.0;
            for (int i = 0; i <= m; ++i) acc += std::conj(Pk[(size_t)i * (k + 1) + a]) * s[i];
            cn[a] = acc;
        }
        H.swap(Hn);
        c.swap(cn);
        std::swap(V, Vn);
        j0 = k;
        if (rel <= p.tol) {
            converged = true;
            ++cycle;
            break;
        }
    }
    st.cycles = cycle;
    st.converged = converged ? 1 : 0;
    DLZ_TRY(v64::copy(op, x_out, x.as<double2>()));
    if (defl_out) {
        dlz_defl_s *d = new dlz_defl_s();
        d->op = &op;
        d->k = k;
        d->which = DLZ_D;
        int rc = d->V64.alloc((size_t)(k + 1) * n * sizeof(double2));
        if (rc != DLZ_OK) { delete d; return rc; }
        rc = [&]() -> int {
            DLZ_CUDA_TRY(cudaMemcpyAsync(d->V64.p, V, (size_t)(k + 1) * n * sizeof(double2), cudaMemcpyDeviceToDevice,
                                         op.stream));
            return DLZ_OK;
        }();
        if (rc != DLZ_OK) { delete d; return rc; }
        d->Hbar.assign((size_t)(k + 1) * k, zc(0, 0));
        for (int a = 0; a <= k; ++a)
            for (int l = 0; l < k; ++l) d->Hbar[(size_t)a * k + l] = H[(size_t)a * m + l];
        d->theta = theta;
        d->values.resize(k);
        for (int l = 0; l < k; ++l) d->values[l] = theta[l].real();
        // harmonic Ritz vector l = V_{k+1} P^H [g_l; 0]: coefficients (k+1) x k
        d->Z.assign((size_t)(k + 1) * k, zc(0, 0));
        for (int l = 0; l < k; ++l)
            for (int a = 0; a <= k; ++a) {
                zc acc = 0.0;
                for (int i = 0; i < m; ++i) acc += std::conj(Pk[(size_t)i * (k + 1) + a]) * Pk[(size_t)i * (k + 1) + l];
                d->Z[(size_t)a * k + l] = acc;
            }
        *defl_out = d;
    }
    DLZ_CUDA_TRY(cudaStreamSynchronize(op.stream));
    return converged ? DLZ_OK : DLZ_ERR_NOT_CONVERGED;
}

int dgmres64(Op &op, const dlz_defl_s *d, const double2 *b, double2 *x_out, const dlz_params &p, dlz_stats &st) {
    const int m = p.m;
    const long n = 12L * op.g.V;
    const int k = d ? d->k : 0;
    DevBuf Vb, w, x, r, scal, dots;
    DLZ_TRY(Vb.alloc((size_t)(m + 1) * n * sizeof(double2)));
    DLZ_TRY(w.alloc(n * sizeof(double2)));
    DLZ_TRY(x.alloc(n * sizeof(double2)));
    DLZ_TRY(r.alloc(n * sizeof(double2)));
    DLZ_TRY(scal.alloc(8 * sizeof(double)));
    DLZ_TRY(dots.alloc((size_t)(k + 2) * sizeof(double2)));
    ArnoldiBufs ab;
    DLZ_TRY(ab.alloc(m));
    double *dn = scal.as<double>();
    DLZ_TRY(v64::norm2_diff(op, b, nullptr, dn));
    double h = 0.0;
    DLZ_TRY(d2h_sync(op, &h, dn, sizeof(double)));
    const double bnorm = std::sqrt(h);
    if (!std::isfinite(bnorm)) return fail(DLZ_ERR_NONFINITE, "right-hand side is not finite");
    DLZ_TRY(v64::zero(op, x.as<double2>()));
    DLZ_TRY(v64::copy(op, r.as<double2>(), b));
    double rel = bnorm > 0 ? 1.0 : 0.0;
    bool converged = rel <= p.tol;
    double2 *V = Vb.as<double2>();
    int outer = 0;
    while (!converged && st.iterations < p.max_iter) {
        if (k > 0) {
            // minimum-residual projection over span(V_k): c = V_{k+1}^H r, y = lstsq(Hbar_k, c)
            DLZ_TRY(v64::multidot(op, d->V64.as<double2>(), n, k + 1, r.as<double2>(), dots.as<double2>(), 1.0));
            std::vector<double2> hc(k + 1);
            DLZ_TRY(d2h_sync(op, hc.data(), dots.p, (k + 1) * sizeof(double2)));
            std::vector<zc> cv(k + 1), y(k);
            for (int i = 0; i <= k; ++i) cv[i] = zc(hc[i].x, hc[i].y);
            if (!zlstsq(k + 1, k, d->Hbar.data(), cv.data(), y.data(), nullptr))
                return fail(DLZ_ERR_BREAKDOWN, "D-GMRES projection: singular Hbar_k");
            DLZ_TRY(add_combination(op, x.as<double2>(), d->V64.as<double2>(), n, y, ab.coef.as<double2>()));
            DLZ_TRY(true_residual(op, b, x.as<double2>(), r.as<double2>(), dn, bnorm, rel, st.mvps));
            if (rel <= p.tol) { converged = true; break; }
        }
        // one GMRES(m) cycle from r
        const double beta = rel * bnorm;
        {
            const double s = 1.0 / beta;
            double2 *v0 = V;
            const double2 *rr = r.as<double2>();
            DLZ_TRY(map(op, n, [=] __device__(long i) { const double2 a = rr[i]; v0[i] = make_double2(s * a.x, s * a.y); }));
        }
        std::vector<zc> H((size_t)(m + 1) * m, zc(0, 0)), c(m + 1, zc(0, 0)), y(m);
        c[0] = beta;
        DLZ_TRY(arnoldi(op, V, n, 0, m, w.as<double2>(), ab, H, st.mvps));
        st.iterations += m;
        if (!zlstsq(m + 1, m, H.data(), c.data(), y.data(), nullptr))
            return fail(DLZ_ERR_BREAKDOWN, "GMRES least squares: singular Arnoldi matrix");
        DLZ_TRY(add_combination(op, x.as<double2>(), V, n, y, ab.coef.as<double2>()));
        DLZ_TRY(true_residual(op, b, x.as<double2>(), r.as<double2>(), dn, bnorm, rel, st.mvps));
        converged = rel <= p.tol;
        ++outer;
    }
    st.cycles = outer;
    st.true_residual = rel;
    st.converged = converged ? 1 : 0;
    DLZ_TRY(v64::copy(op, x_out, x.as<double2>()));
    DLZ_CUDA_TRY(cudaStreamSynchronize(op.stream));
    return converged ? DLZ_OK : DLZ_ERR_NOT_CONVERGED;
}

// Residuals ||D y_l - theta_l y_l|| of the kept harmonic Ritz pairs of a GMRES-DR set
// (y_l = V_{k+1} Z[:, l] normalised), computed once in FP64.
int gmres_deflation_residuals(Op &op, dlz_defl_s *d) {
    if (!d->residuals.empty()) return DLZ_OK;
    const int k = d->k;
    const long n = 12L * op.g.V;
    DevBuf y, Dy, coef, scal;
    DLZ_TRY(y.alloc(n * sizeof(double2)));
    DLZ_TRY(Dy.alloc(n * sizeof(double2)));
    DLZ_TRY(coef.alloc((size_t)(k + 1) * sizeof(double2)));
    DLZ_TRY(scal.alloc(2 * sizeof(double)));
    d->residuals.resize(k);
    for (int l = 0; l < k; ++l) {
        std::vector<zc> z(k + 1);
        for (int a = 0; a <= k; ++a) z[a] = d->Z[(size_t)a * k + l];
        DLZ_TRY(v64::zero(op, y.as<double2>()));
        DLZ_TRY(add_combination(op, y.as<double2>(), d->V64.as<double2>(), n, z, coef.as<double2>()));
        DLZ_TRY(wilson64(op, Dy.as<double2>(), y.as<double2>(), DLZ_D));
        const zc th = d->theta[l];
        const double tr = th.real(), ti = th.imag();
        double2 *py = y.as<double2>(), *pdy = Dy.as<double2>();
        double *s2 = scal.as<double>();
        DLZ_TRY(reduce<2>(op, n, [=] __device__(long i, double (&acc)[2]) {
            const double2 a = py[i], b2 = pdy[i];
            const double rx = b2.x - (tr * a.x - ti * a.y), ry = b2.y - (tr * a.y + ti * a.x);
            acc[0] += rx * rx + ry * ry;
            acc[1] += a.x * a.x + a.y * a.y;
        }, [=] __device__(const double *res) { s2[0] = res[0]; s2[1] = res[1]; }));
        double hs[2];
        DLZ_TRY(d2h_sync(op, hs, s2, 2 * sizeof(double)));
        d->residuals[l] = std::sqrt(hs[0] / hs[1]);
    }
    return DLZ_OK;
}

}  // namespace dlz
