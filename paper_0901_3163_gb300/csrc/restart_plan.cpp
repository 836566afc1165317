// The FP64 small problem of a restart cycle (arXiv:0901.3163, Sec. 1-2): the
// Galerkin solve and regular Ritz pairs of Lan-DR, the least-squares solve and
// harmonic Ritz pairs of MinRes-DR, and the restart matrices (P, the new Tbar and c).
// Host code; the dense kernels are those of small_dense.cpp.
#include "restart_plan.h"

#include <algorithm>
#include <cmath>

#include "dlz_internal.cuh"
#include "small_dense.h"

namespace dlz {

int plan_solve(bool harmonic, int m, const std::vector<double> &T, const std::vector<double> &c, RestartPlan &o) {
    o.y.assign(m, 0.0);
    const double bm = T[(size_t)m * m + m - 1];
    if (!harmonic) {
        std::vector<double> LU((size_t)m * m);
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) LU[(size_t)i * m + j] = T[(size_t)i * m + j];
        std::vector<int> piv(m);
        std::copy(c.begin(), c.begin() + m, o.y.begin());
        if (!lu_factor(m, LU.data(), piv.data())) return fail(DLZ_ERR_BREAKDOWN, "T_m singular");
        lu_solve(m, LU.data(), piv.data(), o.y.data());
        o.rho = -bm * o.y[m - 1];
        return DLZ_OK;
    }
    o.q.assign(m + 1, 0.0);
    o.s.assign(m + 1, 0.0);
    if (!lstsq(m + 1, m, T.data(), c.data(), o.y.data(), o.q.data())) return fail(DLZ_ERR_BREAKDOWN, "least squares failed");
    for (int i = 0; i <= m; ++i) {
        double t = c[i];
        for (int j = 0; j < m; ++j) t -= T[(size_t)i * m + j] * o.y[j];
        o.s[i] = t;
    }
    return DLZ_OK;
}

int plan_finish(bool harmonic, int m, int k, const std::vector<double> &T, double &Anorm, RestartPlan &o) {
    std::vector<double> Tm((size_t)m * m);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) Tm[(size_t)i * m + j] = T[(size_t)i * m + j];
    std::vector<double> ev(m), G;
    // Lan-DR needs the Ritz vectors of T_m; MinRes-DR only its extreme eigenvalues (||A|| estimate)
    if (harmonic) {
        if (!sym_extremes(m, Tm.data(), &ev[0], &ev[m - 1])) return fail(DLZ_ERR_NONFINITE, "eig(T_m) failed");
    } else {
        G.resize((size_t)m * m);
        if (!sym_eig(m, Tm.data(), ev.data(), G.data())) return fail(DLZ_ERR_NONFINITE, "eig(T_m) failed");
    }
    Anorm = std::max(Anorm, std::max(std::fabs(ev[0]), std::fabs(ev[m - 1])));
    o.P.assign((size_t)(m + 1) * (k + 1), 0.0);
    o.Tn.assign((size_t)(m + 1) * m, 0.0);
    o.cn.assign(m + 1, 0.0);
    o.theta.assign(k, 0.0);
    o.res.assign(k, 0.0);
    const double bm = T[(size_t)m * m + m - 1];
    if (!harmonic) {
        for (int l = 0; l < k; ++l) {           // k algebraically smallest Ritz values
            o.theta[l] = ev[l];
            for (int i = 0; i < m; ++i) o.P[(size_t)i * (k + 1) + l] = G[(size_t)i * m + l];
            o.res[l] = std::fabs(bm * G[(size_t)(m - 1) * m + l]);
        }
        o.P[(size_t)m * (k + 1) + k] = 1.0;
        for (int l = 0; l < k; ++l) o.Tn[(size_t)l * m + l] = o.theta[l];
        for (int l = 0; l < k; ++l) o.Tn[(size_t)k * m + l] = bm * G[(size_t)(m - 1) * m + l];
        o.cn[k] = o.rho;
        return DLZ_OK;
    }
    std::vector<double> &q = o.q, &s = o.s;
    // harmonic Ritz pairs: T_m g = mu (Tbar^T Tbar) g, theta = 1/mu, via the Cholesky
    // factor L of Tbar^T Tbar: C = L^-1 T_m L^-T, g = L^-T z
    std::vector<double> M((size_t)m * m, 0.0), L((size_t)m * m), X, C((size_t)m * m);
    // M = Tbar^T Tbar from the nonzeros of each row of Tbar (dense (k+1) block + band)
    for (int r = 0; r <= m; ++r) {
        const double *row = &T[(size_t)r * m];
        int nz[1024];
        int cnt = 0;
        for (int j = 0; j < m; ++j)
            if (row[j] != 0.0) nz[cnt++] = j;
        for (int a = 0; a < cnt; ++a)
            for (int b = 0; b < cnt; ++b) M[(size_t)nz[a] * m + nz[b]] += row[nz[a]] * row[nz[b]];
    }
    if (!cholesky(m, M.data(), L.data())) return fail(DLZ_ERR_BREAKDOWN, "Tbar^T Tbar not positive definite");
    std::vector<int> env;
    envelope(m, L.data(), env);
    // X = L^-1 T_m, then C = L^-1 X^T (all columns at once)
    X = Tm;
    lower_solve_rows(m, L.data(), X.data(), m, env.data());
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) C[(size_t)i * m + j] = X[(size_t)j * m + i];
    lower_solve_rows(m, L.data(), C.data(), m, env.data());
    std::vector<double> mu(m), Zc((size_t)m * m);
    if (!sym_eig(m, C.data(), mu.data(), Zc.data())) return fail(DLZ_ERR_NONFINITE, "harmonic eigensolve failed");
    std::vector<int> idx(m);
    for (int i = 0; i < m; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return std::fabs(mu[a]) > std::fabs(mu[b]); });
    // nonzero column range [j0, j1) of each row of Tbar (a dense leading block, then the
    // band): the products with Tbar below skip only exact zeros
    std::vector<int> j0(m + 1), j1(m + 1);
    for (int r = 0; r <= m; ++r) {
        const double *row = &T[(size_t)r * m];
        int a = 0, b = m;
        while (a < m && row[a] == 0.0) ++a;
        while (b > a && row[b - 1] == 0.0) --b;
        j0[r] = a;
        j1[r] = b;
    }
    // g = L^-T z for the k selected z (all at once), each normalised
    std::vector<double> Gk((size_t)m * k), nr(k, 0.0);
    for (int i = 0; i < m; ++i)
        for (int l = 0; l < k; ++l) Gk[(size_t)i * k + l] = Zc[(size_t)i * m + idx[l]];
    upper_t_solve_rows(m, L.data(), Gk.data(), k, env.data());
    for (int i = 0; i < m; ++i)
        for (int l = 0; l < k; ++l) nr[l] += Gk[(size_t)i * k + l] * Gk[(size_t)i * k + l];
    for (int l = 0; l < k; ++l) nr[l] = std::sqrt(nr[l]);
    for (int i = 0; i < m; ++i)
        for (int l = 0; l < k; ++l) Gk[(size_t)i * k + l] /= nr[l];
    for (int l = 0; l < k; ++l) {
        o.theta[l] = 1.0 / mu[idx[l]];
        double r2 = 0;
        for (int r = 0; r <= m; ++r) {
            double t = 0;
            for (int j = j0[r]; j < j1[r]; ++j) t += T[(size_t)r * m + j] * Gk[(size_t)j * k + l];
            if (r < m) t -= o.theta[l] * Gk[(size_t)r * k + l];
            r2 += t * t;
        }
        o.res[l] = std::sqrt(r2);
    }
    double qs = 0;
    for (int i = 0; i <= m; ++i) qs += q[i] * s[i];
    if (qs < 0)
        for (double &t : q) t = -t;
    for (int i = 0; i < m; ++i)
        for (int l = 0; l < k; ++l) o.P[(size_t)i * (k + 1) + l] = Gk[(size_t)i * k + l];
    for (int i = 0; i <= m; ++i) o.P[(size_t)i * (k + 1) + k] = q[i];
    if (!mgs_columns(m + 1, k + 1, o.P.data())) return fail(DLZ_ERR_BREAKDOWN, "restart basis lost rank");
    // Tbar_k = P^T Tbar P[:m, :k] (k x k block symmetric, not diagonal); c <- P^T s
    std::vector<double> TP((size_t)(m + 1) * k, 0.0);
    for (int r = 0; r <= m; ++r)
        for (int l = 0; l < k; ++l) {
            double t = 0;
            for (int j = j0[r]; j < j1[r]; ++j) t += T[(size_t)r * m + j] * o.P[(size_t)j * (k + 1) + l];
            TP[(size_t)r * k + l] = t;
        }
    for (int a = 0; a <= k; ++a)
        for (int l = 0; l < k; ++l) {
            double t = 0;
            for (int r = 0; r <= m; ++r) t += o.P[(size_t)r * (k + 1) + a] * TP[(size_t)r * k + l];
            o.Tn[(size_t)a * m + l] = t;
        }
    for (int a = 0; a < k; ++a)
        for (int l = 0; l < a; ++l) {
            const double sym = 0.5 * (o.Tn[(size_t)a * m + l] + o.Tn[(size_t)l * m + a]);
            o.Tn[(size_t)a * m + l] = o.Tn[(size_t)l * m + a] = sym;
        }
    for (int a = 0; a <= k; ++a) {
        double t = 0;
        for (int r = 0; r <= m; ++r) t += o.P[(size_t)r * (k + 1) + a] * s[r];
        o.cn[a] = t;
    }
    return DLZ_OK;
}

}  // namespace dlz

extern "C" int dlz_host_restart_plan(int harmonic, int m, int k, const double *Tbar, const double *c, double *y,
                                     double *P, double *Tn, double *cn, double *theta, double *ritz_res,
                                     double *anorm) {
    if (m < 2 || k < 1 || k >= m || !Tbar || !c || !y || !P || !Tn || !cn || !theta || !ritz_res || !anorm)
        return dlz::fail(DLZ_ERR_BADARG, "restart plan: bad arguments");
    const std::vector<double> T(Tbar, Tbar + (size_t)(m + 1) * m), cv(c, c + m + 1);
    dlz::RestartPlan pl;
    int rc = dlz::plan_solve(harmonic != 0, m, T, cv, pl);
    if (rc) return rc;
    rc = dlz::plan_finish(harmonic != 0, m, k, T, *anorm, pl);
    if (rc) return rc;
    std::copy(pl.y.begin(), pl.y.end(), y);
    std::copy(pl.P.begin(), pl.P.end(), P);
    std::copy(pl.Tn.begin(), pl.Tn.end(), Tn);
    std::copy(pl.cn.begin(), pl.cn.end(), cn);
    std::copy(pl.theta.begin(), pl.theta.end(), theta);
    std::copy(pl.res.begin(), pl.res.end(), ritz_res);
    return DLZ_OK;
}
