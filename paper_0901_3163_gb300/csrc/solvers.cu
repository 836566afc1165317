// Solver drivers: Lan-DR(m,k), MinRes-DR(m,k), D-CG and D-MinRes
// (arXiv:0901.3163, Sec. 1-2) on the FP64 and FP32 device kernels.
//
// The host drives the cycle structure; inside a Lanczos cycle and inside the
// CG / MinRes loops every scalar (alpha_j, beta_j, the Givens rotation of
// MinRes, the CG step lengths) is produced and consumed on the device by the
// fused reduction kernels, so the host only synchronises at the end of a
// restart cycle (to solve the small projected problem) and every
// `check_every` iterations (to read a residual norm).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "dlz_internal.cuh"
#include "reduce.cuh"
#include "small_dense.h"
#include "solvers.h"
#include "krylov_util.cuh"

namespace dlz {

typedef std::complex<double> zc;

// ------------------------------------------------------------------ deflation set
int build_deflation(Op &op, int which, const double2 *Vk, int k, dlz_defl_s **out, const double *Hk) {
    dlz_defl_s *d = new dlz_defl_s();
    d->op = &op;
    d->k = k;
    d->which = which;
    const long n = 12L * op.g.V;
    int rc = d->V64.alloc((size_t)k * n * sizeof(double2));
    if (rc != DLZ_OK) { delete d; return rc; }
    rc = [&]() -> int {
        DLZ_CUDA_TRY(cudaMemcpyAsync(d->V64.p, Vk, (size_t)k * n * sizeof(double2), cudaMemcpyDeviceToDevice, op.stream));
        return DLZ_OK;
    }();
    if (rc != DLZ_OK) { delete d; return rc; }
    if (Hk) {
        // H = V_k^dag A V_k is the k x k block of the restarted projected matrix
        // (the Lanczos relation A V_k = V_{k+1} Tbar_k holds to the basis rounding)
        d->H.assign((size_t)k * k, zc(0, 0));
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) d->H[(size_t)i * k + j] = zc(0.5 * (Hk[(size_t)i * k + j] + Hk[(size_t)j * k + i]), 0.0);
        rc = deflation_factor(op, d);
    } else {
        rc = deflation_finish(op, d);
    }
    if (rc != DLZ_OK) { delete d; return rc; }
    *out = d;
    return DLZ_OK;
}

// H = V^dag A V, its LU factors, and the Rayleigh-Ritz pairs (values, residuals).
int deflation_finish(Op &op, dlz_defl_s *d) {
    const int k = d->k;
    const long n = 12L * op.g.V;
    if (k == 0) return DLZ_OK;
    DevBuf AV, tmp, dots, gram;
    DLZ_TRY(AV.alloc((size_t)n * sizeof(double2)));
    DLZ_TRY(tmp.alloc((size_t)n * sizeof(double2)));
    DLZ_TRY(dots.alloc((size_t)k * k * sizeof(double2)));
    DLZ_TRY(gram.alloc((size_t)k * k * sizeof(double2)));
    const double2 *V = d->V64.as<double2>();
    for (int j = 0; j < k; ++j) {
        double2 *avj = AV.as<double2>();
        DLZ_TRY(apply64(op, avj, V + (size_t)j * n, d->which, tmp.as<double2>()));
        DLZ_TRY(v64::multidot(op, V, n, k, avj, dots.as<double2>() + (size_t)j * k, 1.0));
        DLZ_TRY(v64::multidot(op, V, n, k, V + (size_t)j * n, gram.as<double2>() + (size_t)j * k, 1.0));
    }
    std::vector<double2> hd((size_t)k * k), gd((size_t)k * k);
    DLZ_TRY(d2h_sync(op, hd.data(), dots.p, hd.size() * sizeof(double2)));
    DLZ_TRY(d2h_sync(op, gd.data(), gram.p, gd.size() * sizeof(double2)));
    // dots[j*k + i] = <v_i, A v_j> = H[i][j]; hermitise (the same for the Gram matrix)
    d->H.assign((size_t)k * k, zc(0, 0));
    d->G.assign((size_t)k * k, zc(0, 0));
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
            const zc hij(hd[(size_t)j * k + i].x, hd[(size_t)j * k + i].y);
            const zc hji(hd[(size_t)i * k + j].x, hd[(size_t)i * k + j].y);
            d->H[(size_t)i * k + j] = 0.5 * (hij + std::conj(hji));
            const zc gij(gd[(size_t)j * k + i].x, gd[(size_t)j * k + i].y);
            const zc gji(gd[(size_t)i * k + j].x, gd[(size_t)i * k + j].y);
            d->G[(size_t)i * k + j] = 0.5 * (gij + std::conj(gji));
        }
    return deflation_factor(op, d);
}

// Cholesky factor G = L L^dag of a hermitian positive definite k x k matrix (row-major,
// L lower triangular); false if G is not positive definite.
static bool chol_lower(int k, const std::vector<zc> &G, std::vector<zc> &L) {
    L.assign((size_t)k * k, zc(0, 0));
    for (int j = 0; j < k; ++j) {
        double dj = G[(size_t)j * k + j].real();
        for (int p = 0; p < j; ++p) dj -= std::norm(L[(size_t)j * k + p]);
        if (!(dj > 0.0)) return false;
        const double ljj = std::sqrt(dj);
        L[(size_t)j * k + j] = ljj;
        for (int i = j + 1; i < k; ++i) {
            zc s = G[(size_t)i * k + j];
            for (int p = 0; p < j; ++p) s -= L[(size_t)i * k + p] * std::conj(L[(size_t)j * k + p]);
            L[(size_t)i * k + j] = s / ljj;
        }
    }
    return true;
}

// Rayleigh-Ritz pairs of a hermitian k x k H (row-major): the eigenpairs of H, or with a
// Gram matrix G = V^dag V (a basis orthonormal only to FP32 rounding; G may be null)
// those of H z = value G z, through C = L^-1 H L^-dag (G = L L^dag) and z = L^-dag u, so
// that each value is the Rayleigh quotient of y = V z and |y| = 1.  values ascending;
// Z row-major with column j the vector of values[j].  0, or a DLZ_ERR code with a message.
int rayleigh_ritz(int k, const std::vector<zc> &H, const std::vector<zc> *G, std::vector<double> &values,
                  std::vector<zc> &Zout) {
    std::vector<zc> L, C = H;
    const bool gen = G && !G->empty();
    if (gen) {
        if (!chol_lower(k, *G, L)) return fail(DLZ_ERR_BREAKDOWN, "deflation: V^dag V is not positive definite");
        // W = L^-1 H (forward substitution on every column), then C = L^-1 W^dag ...
        std::vector<zc> W = H;
        for (int c = 0; c < k; ++c)
            for (int i = 0; i < k; ++i) {
                zc s = W[(size_t)i * k + c];
                for (int p = 0; p < i; ++p) s -= L[(size_t)i * k + p] * W[(size_t)p * k + c];
                W[(size_t)i * k + c] = s / L[(size_t)i * k + i];
            }
        // ... C = (L^-1 (L^-1 H)^dag)^dag = L^-1 H L^-dag, hermitian
        std::vector<zc> Wd((size_t)k * k);
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) Wd[(size_t)i * k + j] = std::conj(W[(size_t)j * k + i]);
        for (int c = 0; c < k; ++c)
            for (int i = 0; i < k; ++i) {
                zc s = Wd[(size_t)i * k + c];
                for (int p = 0; p < i; ++p) s -= L[(size_t)i * k + p] * Wd[(size_t)p * k + c];
                Wd[(size_t)i * k + c] = s / L[(size_t)i * k + i];
            }
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j)
                C[(size_t)i * k + j] = 0.5 * (std::conj(Wd[(size_t)j * k + i]) + Wd[(size_t)i * k + j]);
    }
    // eigenvectors of the hermitian C via the real symmetric embedding
    // [[Re C, -Im C], [Im C, Re C]] (each eigenvalue twice)
    const int n2 = 2 * k;
    std::vector<double> E((size_t)n2 * n2), w(n2), Z((size_t)n2 * n2);
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
            const zc h = C[(size_t)i * k + j];
            E[(size_t)i * n2 + j] = h.real();
            E[(size_t)i * n2 + k + j] = -h.imag();
            E[(size_t)(k + i) * n2 + j] = h.imag();
            E[(size_t)(k + i) * n2 + k + j] = h.real();
        }
    if (!sym_eig(n2, E.data(), w.data(), Z.data()))
        return fail(DLZ_ERR_NONFINITE, "deflation: eigensolve of H failed");
    values.clear();
    std::vector<std::vector<zc>> chosen;
    for (int c = 0; c < n2 && (int)chosen.size() < k; ++c) {
        std::vector<zc> z(k);
        for (int i = 0; i < k; ++i) z[i] = zc(Z[(size_t)i * n2 + c], Z[(size_t)(k + i) * n2 + c]);
        for (const auto &q : chosen) {
            zc s(0, 0);
            for (int i = 0; i < k; ++i) s += std::conj(q[i]) * z[i];
            for (int i = 0; i < k; ++i) z[i] -= s * q[i];
        }
        double nr = 0;
        for (int i = 0; i < k; ++i) nr += std::norm(z[i]);
        nr = std::sqrt(nr);
        if (nr < 0.5) continue;   // the twin of an eigenvector already taken
        for (int i = 0; i < k; ++i) z[i] /= nr;
        chosen.push_back(z);
        values.push_back(w[c]);
    }
    if ((int)chosen.size() < k) return fail(DLZ_ERR_NONFINITE, "deflation: eigenvectors of H");
    if (gen) {
        // z = L^-dag u (back substitution with the conjugate transpose of L)
        for (auto &u : chosen)
            for (int i = k - 1; i >= 0; --i) {
                zc s = u[i];
                for (int p = i + 1; p < k; ++p) s -= std::conj(L[(size_t)p * k + i]) * u[p];
                u[i] = s / L[(size_t)i * k + i];
            }
    }
    Zout.resize((size_t)k * k);
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) Zout[(size_t)i * k + j] = chosen[j][i];   // column j = vector j
    return DLZ_OK;
}

// LU factors of H (the Galerkin projection, which needs no orthonormality) and the
// Rayleigh-Ritz pairs of the set.
int deflation_factor(Op &, dlz_defl_s *d) {
    const int k = d->k;
    if (k == 0) return DLZ_OK;
    d->Hlu = d->H;
    d->piv.assign(k, 0);
    if (!lu_factor(k, d->Hlu.data(), d->piv.data()))
        return fail(DLZ_ERR_BREAKDOWN, "deflation: H = V^dag A V is singular");
    DLZ_TRY(rayleigh_ritz(k, d->H, &d->G, d->values, d->Z));
    d->residuals.clear();   // computed on first request (deflation_residuals)
    return DLZ_OK;
}

// ||A y_j - value_j y_j|| for the Rayleigh-Ritz pairs, y = V Z (k MVPs).
int deflation_residuals(Op &op, dlz_defl_s *d) {
    const int k = d->k;
    const long n = 12L * op.g.V;
    if (k == 0 || (int)d->residuals.size() == k) return DLZ_OK;
    const double2 *V = d->V64.as<double2>();
    DevBuf Y, AY, coef, tmp;
    DLZ_TRY(tmp.alloc((size_t)n * sizeof(double2)));
    DLZ_TRY(Y.alloc((size_t)k * n * sizeof(double2)));
    DLZ_TRY(AY.alloc((size_t)k * n * sizeof(double2)));
    DLZ_TRY(coef.alloc((size_t)k * k * sizeof(double2)));
    std::vector<double2> zc2((size_t)k * k);
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j)
            zc2[(size_t)i * k + j] = make_double2(d->Z[(size_t)i * k + j].real(), d->Z[(size_t)i * k + j].imag());
    DLZ_TRY(h2d(op, coef.p, zc2.data(), zc2.size() * sizeof(double2)));
    DLZ_TRY(combine64(op, Y.as<double2>(), n, k, V, n, k, coef.p, k, false, false));
    for (int j = 0; j < k; ++j)
        DLZ_TRY(apply64(op, AY.as<double2>() + (size_t)j * n, Y.as<double2>() + (size_t)j * n, d->which,
                        tmp.as<double2>()));
    DevBuf res;
    DLZ_TRY(res.alloc((size_t)k * sizeof(double)));
    for (int j = 0; j < k; ++j) {
        const double2 *y = Y.as<double2>() + (size_t)j * n, *ay = AY.as<double2>() + (size_t)j * n;
        const double lam = d->values[j];
        double *o = res.as<double>() + j;
        DLZ_TRY(reduce<1>(op, n, [=] __device__(long i, double (&acc)[1]) {
            const double2 a = ay[i], b = y[i];
            const double rx = a.x - lam * b.x, ry = a.y - lam * b.y;
            acc[0] += rx * rx + ry * ry;
        }, [=] __device__(const double *r) { *o = sqrt(r[0]); }));
    }
    d->residuals.assign(k, 0.0);
    DLZ_TRY(d2h_sync(op, d->residuals.data(), res.p, (size_t)k * sizeof(double)));
    return DLZ_OK;
}

int deflation_v32(Op &op, dlz_defl_s *d) {
    if (d->k == 0 || d->V32.p) return DLZ_OK;
    const long n64 = 12L * op.g.V, n32 = 6L * op.g.V;
    DLZ_TRY(d->V32.alloc((size_t)d->k * n32 * sizeof(float4)));
    for (int j = 0; j < d->k; ++j)
        DLZ_TRY(convert64to32(op, d->V32.as<float4>() + (size_t)j * n32, d->V64.as<double2>() + (size_t)j * n64));
    return DLZ_OK;
}

// x0 = V H^-1 V^dag b  (b, x0 internal FP64; x0 overwritten)
int project64(Op &op, const dlz_defl_s *d, const double2 *b, double2 *x0, DevBuf &dots) {
    const int k = d->k;
    const long n = 12L * op.g.V;
    if (k == 0) return v64::zero(op, x0);
    DLZ_TRY(v64::multidot(op, d->V64.as<double2>(), n, k, b, dots.as<double2>(), 1.0));
    std::vector<double2> c(k);
    DLZ_TRY(d2h_sync(op, c.data(), dots.p, k * sizeof(double2)));
    std::vector<zc> z(k);
    for (int i = 0; i < k; ++i) z[i] = zc(c[i].x, c[i].y);
    lu_solve(k, d->Hlu.data(), d->piv.data(), z.data());
    for (int i = 0; i < k; ++i) c[i] = make_double2(z[i].real(), z[i].imag());
    DLZ_TRY(h2d(op, dots.p, c.data(), k * sizeof(double2)));
    return combine64(op, x0, n, 1, d->V64.as<double2>(), n, k, dots.p, 1, false, false);
}

// ------------------------------------------------------------------ D-MinRes (FP64)
struct MinresState {
    double beta, alpha, beta_next, inv_beta;
    double c, s, c_old, s_old, phibar;
    double eps, delta, gamma, tau;
};

static int minres_init(Op &op, MinresState *dst, double *d_norm) {
    // beta = phibar = ||r||, fresh rotations
    return map(op, 1, [=] __device__(long) {
        const double b = sqrt(*d_norm);
        MinresState s0;
        s0.beta = 0.0; s0.alpha = 0.0; s0.beta_next = b; s0.inv_beta = b > 0 ? 1.0 / b : 0.0;
        s0.c = 1.0; s0.s = 0.0; s0.c_old = 1.0; s0.s_old = 0.0; s0.phibar = b;
        s0.eps = s0.delta = s0.gamma = s0.tau = 0.0;
        *dst = s0;
    });
}

int dminres64(Op &op, const dlz_defl_s *d, const double2 *b_in, double2 *x_out, const dlz_params &p,
              dlz_stats &st, const double2 *x_init) {
    const long n = 12L * op.g.V;
    DevBuf bg, x, r, vp, v, w, d1, d2, scal, dots;
    DLZ_TRY(bg.alloc(n * sizeof(double2)));
    DLZ_TRY(x.alloc(n * sizeof(double2)));
    DLZ_TRY(r.alloc(n * sizeof(double2)));
    DLZ_TRY(vp.alloc(n * sizeof(double2)));
    DLZ_TRY(v.alloc(n * sizeof(double2)));
    DLZ_TRY(w.alloc(n * sizeof(double2)));
    DLZ_TRY(d1.alloc(n * sizeof(double2)));
    DLZ_TRY(d2.alloc(n * sizeof(double2)));
    DLZ_TRY(scal.alloc(64 * sizeof(double)));
    DLZ_TRY(dots.alloc((size_t)std::max(1, d ? d->k : 1) * sizeof(double2)));
    MinresState *ms = reinterpret_cast<MinresState *>(scal.as<double>());
    double *d_norm = scal.as<double>() + 32;
    HostScratch hs;
    DLZ_TRY(hs.ensure(32));
    DLZ_TRY(v64::gamma5(op, bg.as<double2>(), b_in));
    DLZ_TRY(v64::norm2_diff(op, bg.as<double2>(), nullptr, d_norm + 1));
    DLZ_TRY(d2h_sync(op, hs.p, d_norm + 1, sizeof(double)));
    const double bnorm = std::sqrt(hs.p[0]);
    if (!std::isfinite(bnorm)) return fail(DLZ_ERR_NONFINITE, "right-hand side is not finite");
    if (bnorm == 0.0) {
        DLZ_TRY(v64::zero(op, x_out));
        st.converged = 1; st.true_residual = 0.0;
        return DLZ_OK;
    }
    if (x_init) {
        // x = x_init + V H^-1 V^dag (gamma5 b - Q x_init)
        DLZ_TRY(v64::copy(op, x.as<double2>(), x_init));
        if (d && d->k > 0) {
            DLZ_TRY(wilson64(op, r.as<double2>(), x.as<double2>(), DLZ_Q));
            st.mvps += 1;
            const double2 *bgp = bg.as<double2>();
            double2 *rp = r.as<double2>();
            DLZ_TRY(map(op, n, [=] __device__(long i) {
                const double2 a = bgp[i], q = rp[i];
                rp[i] = make_double2(a.x - q.x, a.y - q.y);
            }));
            DLZ_TRY(project64(op, d, r.as<double2>(), d1.as<double2>(), dots));
            double2 *px0 = x.as<double2>();
            const double2 *pe = d1.as<double2>();
            DLZ_TRY(map(op, n, [=] __device__(long i) {
                const double2 a = px0[i], e = pe[i];
                px0[i] = make_double2(a.x + e.x, a.y + e.y);
            }));
        }
    } else if (d && d->k > 0) {
        DLZ_TRY(project64(op, d, bg.as<double2>(), x.as<double2>(), dots));
    } else {
        DLZ_TRY(v64::zero(op, x.as<double2>()));
    }
    bool converged = false;
    while (st.iterations < p.max_iter) {
        // r = gamma5 b - Q x ; start a MinRes run from x
        DLZ_TRY(wilson64(op, r.as<double2>(), x.as<double2>(), DLZ_Q));
        st.mvps += 1;
        {
            const double2 *bgp = bg.as<double2>();
            double2 *rp = r.as<double2>();
            DLZ_TRY(reduce<1>(op, n, [=] __device__(long i, double (&acc)[1]) {
                const double2 a = bgp[i], q = rp[i];
                const double2 t = make_double2(a.x - q.x, a.y - q.y);
                rp[i] = t;
                acc[0] += t.x * t.x + t.y * t.y;
            }, [=] __device__(const double *res) { *d_norm = res[0]; }));
        }
        DLZ_TRY(d2h_sync(op, hs.p, d_norm, sizeof(double)));
        const double rel0 = std::sqrt(hs.p[0]) / bnorm;
        st.true_residual = rel0;
        if (!std::isfinite(rel0)) return fail(DLZ_ERR_NONFINITE, "residual is not finite");
        if (rel0 <= p.tol) { converged = true; break; }
        DLZ_TRY(minres_init(op, ms, d_norm));
        double2 *pvp = vp.as<double2>(), *pv = v.as<double2>(), *pw = w.as<double2>();
        double2 *pd1 = d1.as<double2>(), *pd2 = d2.as<double2>();
        {
            const double2 *rp = r.as<double2>();
            DLZ_TRY(map(op, n, [=] __device__(long i) {
                const double inv = ms->inv_beta;
                const double2 t = rp[i];
                pv[i] = make_double2(t.x * inv, t.y * inv);
                pvp[i] = make_double2(0.0, 0.0);
                pd1[i] = make_double2(0.0, 0.0);
                pd2[i] = make_double2(0.0, 0.0);
            }));
        }
        double2 *px = x.as<double2>();
        int it_run = 0;
        bool stop_run = false;
        while (!stop_run && st.iterations < p.max_iter) {
            DLZ_TRY(wilson64(op, pw, pv, DLZ_Q));
            st.mvps += 1;
            // w -= beta_j v_{j-1}; alpha_j = <v_j, w>
            {
                const double2 *a_vp = pvp, *a_v = pv;
                double2 *a_w = pw;
                DLZ_TRY(reduce<1>(op, n, [=] __device__(long i, double (&acc)[1]) {
                    const double bt = ms->beta_next;
                    double2 t = a_w[i];
                    const double2 u = a_vp[i];
                    t.x -= bt * u.x; t.y -= bt * u.y;
                    a_w[i] = t;
                    const double2 q = a_v[i];
                    acc[0] += q.x * t.x + q.y * t.y;
                }, [=] __device__(const double *res) {
                    ms->beta = ms->beta_next;
                    ms->alpha = res[0];
                }));
            }
            // w -= alpha_j v_j; beta_{j+1} = ||w||; Givens update of the QR of Tbar_j
            {
                const double2 *a_v = pv;
                double2 *a_w = pw;
                DLZ_TRY(reduce<1>(op, n, [=] __device__(long i, double (&acc)[1]) {
                    const double al = ms->alpha;
                    double2 t = a_w[i];
                    const double2 q = a_v[i];
                    t.x -= al * q.x; t.y -= al * q.y;
                    a_w[i] = t;
                    acc[0] += t.x * t.x + t.y * t.y;
                }, [=] __device__(const double *res) {
                    MinresState s = *ms;
                    const double bn = sqrt(res[0]);
                    const double eps = s.s_old * s.beta;
                    const double deltabar = s.c_old * s.beta;
                    const double delta = s.c * deltabar + s.s * s.alpha;
                    const double gammabar = -s.s * deltabar + s.c * s.alpha;
                    const double gamma = hypot(gammabar, bn);
                    const double cn = gammabar / gamma, sn = bn / gamma;
                    s.tau = cn * s.phibar;
                    s.phibar = -sn * s.phibar;
                    s.eps = eps; s.delta = delta; s.gamma = gamma;
                    s.c_old = s.c; s.s_old = s.s; s.c = cn; s.s = sn;
                    s.beta_next = bn;
                    s.inv_beta = bn > 0 ? 1.0 / bn : 0.0;
                    *ms = s;
                }));
            }
            // d_j = (v_j - delta d_{j-1} - eps d_{j-2}) / gamma ; x += tau d_j ; v_{j+1} = w / beta_{j+1}
            {
                const double2 *a_v = pv, *a_d1 = pd1;
                double2 *a_d2 = pd2, *a_w = pw, *a_x = px;
                DLZ_TRY(map(op, n, [=] __device__(long i) {
                    const double de = ms->delta, ep = ms->eps, ig = 1.0 / ms->gamma, ta = ms->tau, ib = ms->inv_beta;
                    const double2 q = a_v[i], e1 = a_d1[i], e2 = a_d2[i];
                    double2 dn;
                    dn.x = (q.x - de * e1.x - ep * e2.x) * ig;
                    dn.y = (q.y - de * e1.y - ep * e2.y) * ig;
                    a_d2[i] = dn;
                    double2 xx = a_x[i];
                    xx.x += ta * dn.x; xx.y += ta * dn.y;
                    a_x[i] = xx;
                    const double2 t = a_w[i];
                    a_w[i] = make_double2(t.x * ib, t.y * ib);
                }));
            }
            // rotate: (v_prev, v, w) <- (v, w, v_prev) ; (d1, d2) <- (d2, d1)
            double2 *t0 = pvp; pvp = pv; pv = pw; pw = t0;
            std::swap(pd1, pd2);
            st.iterations++;
            ++it_run;
            if (it_run % p.check_every == 0 || st.iterations >= p.max_iter) {
                DLZ_TRY(d2h_sync(op, hs.p, ms, sizeof(MinresState)));
                const MinresState *hsm = reinterpret_cast<const MinresState *>(hs.p);
                if (!std::isfinite(hsm->phibar)) return fail(DLZ_ERR_NONFINITE, "MinRes residual not finite");
                if (std::fabs(hsm->phibar) <= 0.5 * p.tol * bnorm || hsm->beta_next == 0.0) stop_run = true;
            }
        }
    }
    DLZ_TRY(v64::copy(op, x_out, x.as<double2>()));
    if (!converged) {
        // final FP64 verification
        DLZ_TRY(wilson64(op, r.as<double2>(), x.as<double2>(), DLZ_Q));
        DLZ_TRY(v64::norm2_diff(op, bg.as<double2>(), r.as<double2>(), d_norm));
        DLZ_TRY(d2h_sync(op, hs.p, d_norm, sizeof(double)));
        st.true_residual = std::sqrt(hs.p[0]) / bnorm;
        converged = st.true_residual <= p.tol;
    }
    st.converged = converged ? 1 : 0;
    return converged ? DLZ_OK : DLZ_ERR_NOT_CONVERGED;
}

// ------------------------------------------------------------------ D-CG (FP64, normal equations)
struct CgState {
    double rr, alpha, beta, ss;
};

int dcg64(Op &op, const dlz_defl_s *d, const double2 *b_in, double2 *x_out, const dlz_params &p,
          dlz_stats &st, const double2 *x_init) {
    const long n = 12L * op.g.V;
    DevBuf x, r, s, pp, t, q, bd, scal, dots;
    DLZ_TRY(x.alloc(n * sizeof(double2)));
    DLZ_TRY(r.alloc(n * sizeof(double2)));
    DLZ_TRY(s.alloc(n * sizeof(double2)));
    DLZ_TRY(pp.alloc(n * sizeof(double2)));
    DLZ_TRY(t.alloc(n * sizeof(double2)));
    DLZ_TRY(q.alloc(n * sizeof(double2)));
    DLZ_TRY(bd.alloc(n * sizeof(double2)));
    DLZ_TRY(scal.alloc(64 * sizeof(double)));
    DLZ_TRY(dots.alloc((size_t)std::max(1, d ? d->k : 1) * sizeof(double2)));
    CgState *cs = reinterpret_cast<CgState *>(scal.as<double>());
    double *d_norm = scal.as<double>() + 32;
    HostScratch hs;
    DLZ_TRY(hs.ensure(32));
    const double2 *b = b_in;
    DLZ_TRY(v64::norm2_diff(op, b, nullptr, d_norm + 1));
    DLZ_TRY(d2h_sync(op, hs.p, d_norm + 1, sizeof(double)));
    const double bnorm = std::sqrt(hs.p[0]);
    if (!std::isfinite(bnorm)) return fail(DLZ_ERR_NONFINITE, "right-hand side is not finite");
    if (bnorm == 0.0) {
        DLZ_TRY(v64::zero(op, x_out));
        st.converged = 1; st.true_residual = 0.0;
        return DLZ_OK;
    }
    if (x_init) {
        // x = x_init + V H^-1 V^dag D^dag (b - D x_init)
        DLZ_TRY(v64::copy(op, x.as<double2>(), x_init));
        if (d && d->k > 0) {
            DLZ_TRY(wilson64(op, s.as<double2>(), x.as<double2>(), DLZ_D));
            const double2 *bp = b;
            double2 *sp = s.as<double2>();
            DLZ_TRY(map(op, n, [=] __device__(long i) {
                const double2 a = bp[i], q = sp[i];
                sp[i] = make_double2(a.x - q.x, a.y - q.y);
            }));
            DLZ_TRY(wilson64(op, bd.as<double2>(), s.as<double2>(), DLZ_DDAG));
            st.mvps += 2;
            DLZ_TRY(project64(op, d, bd.as<double2>(), t.as<double2>(), dots));
            double2 *px0 = x.as<double2>();
            const double2 *pe = t.as<double2>();
            DLZ_TRY(map(op, n, [=] __device__(long i) {
                const double2 a = px0[i], e = pe[i];
                px0[i] = make_double2(a.x + e.x, a.y + e.y);
            }));
        }
    } else if (d && d->k > 0) {
        DLZ_TRY(wilson64(op, bd.as<double2>(), b, DLZ_DDAG));    // b' = D^dag b
        st.mvps += 1;
        DLZ_TRY(project64(op, d, bd.as<double2>(), x.as<double2>(), dots));
    } else {
        DLZ_TRY(v64::zero(op, x.as<double2>()));
    }
    double2 *px = x.as<double2>(), *pr = r.as<double2>(), *ps = s.as<double2>(), *pp_ = pp.as<double2>();
    double2 *pt = t.as<double2>(), *pq = q.as<double2>();
    bool converged = false;
    while (st.iterations < p.max_iter) {
        // s = b - D x ; r = D^dag s ; p = r
        DLZ_TRY(wilson64(op, pt, px, DLZ_D));
        st.mvps += 1;
        DLZ_TRY(reduce<1>(op, n, [=] __device__(long i, double (&acc)[1]) {
            const double2 a = b[i], u = pt[i];
            const double2 v = make_double2(a.x - u.x, a.y - u.y);
            ps[i] = v;
            acc[0] += v.x * v.x + v.y * v.y;
        }, [=] __device__(const double *res) { *d_norm = res[0]; }));
        DLZ_TRY(d2h_sync(op, hs.p, d_norm, sizeof(double)));
        const double rel0 = std::sqrt(hs.p[0]) / bnorm;
        st.true_residual = rel0;
        if (!std::isfinite(rel0)) return fail(DLZ_ERR_NONFINITE, "residual is not finite");
        if (rel0 <= p.tol) { converged = true; break; }
        DLZ_TRY(wilson64(op, pr, ps, DLZ_DDAG));
        st.mvps += 1;
        DLZ_TRY(reduce<2>(op, n, [=] __device__(long i, double (&acc)[2]) {
            const double2 v = pr[i];
            pp_[i] = v;
            acc[0] += v.x * v.x + v.y * v.y;
            const double2 u = ps[i];
            acc[1] += u.x * u.x + u.y * u.y;
        }, [=] __device__(const double *res) { cs->rr = res[0]; cs->ss = res[1]; }));
        int it_run = 0;
        bool stop_run = false;
        while (!stop_run && st.iterations < p.max_iter) {
            DLZ_TRY(wilson64(op, pt, pp_, DLZ_D));               // t = D p
            DLZ_TRY(wilson64(op, pq, pt, DLZ_DDAG));             // q = D^dag t
            st.mvps += 2;
            DLZ_TRY(reduce<1>(op, n, [=] __device__(long i, double (&acc)[1]) {
                const double2 a = pp_[i], c = pq[i];
                acc[0] += a.x * c.x + a.y * c.y;
            }, [=] __device__(const double *res) { cs->alpha = cs->rr / res[0]; }));
            DLZ_TRY(reduce<2>(op, n, [=] __device__(long i, double (&acc)[2]) {
                const double al = cs->alpha;
                const double2 a = pp_[i], c = pq[i], tt = pt[i];
                double2 xx = px[i], rr_ = pr[i], ss_ = ps[i];
                xx.x += al * a.x; xx.y += al * a.y;
                rr_.x -= al * c.x; rr_.y -= al * c.y;
                ss_.x -= al * tt.x; ss_.y -= al * tt.y;
                px[i] = xx; pr[i] = rr_; ps[i] = ss_;
                acc[0] += rr_.x * rr_.x + rr_.y * rr_.y;
                acc[1] += ss_.x * ss_.x + ss_.y * ss_.y;
            }, [=] __device__(const double *res) {
                cs->beta = res[0] / cs->rr;
                cs->rr = res[0];
                cs->ss = res[1];
            }));
            DLZ_TRY(map(op, n, [=] __device__(long i) {
                const double be = cs->beta;
                const double2 rr_ = pr[i], a = pp_[i];
                pp_[i] = make_double2(rr_.x + be * a.x, rr_.y + be * a.y);
            }));
            st.iterations++;
            ++it_run;
            if (it_run % p.check_every == 0 || st.iterations >= p.max_iter) {
                DLZ_TRY(d2h_sync(op, hs.p, cs, sizeof(CgState)));
                const CgState *h = reinterpret_cast<const CgState *>(hs.p);
                if (!std::isfinite(h->ss)) return fail(DLZ_ERR_NONFINITE, "CG residual not finite");
                if (std::sqrt(h->ss) <= 0.5 * p.tol * bnorm || h->rr == 0.0) stop_run = true;
            }
        }
    }
    DLZ_TRY(v64::copy(op, x_out, px));
    if (!converged) {
        DLZ_TRY(wilson64(op, pt, px, DLZ_D));
        DLZ_TRY(v64::norm2_diff(op, b, pt, d_norm));
        DLZ_TRY(d2h_sync(op, hs.p, d_norm, sizeof(double)));
        st.true_residual = std::sqrt(hs.p[0]) / bnorm;
        converged = st.true_residual <= p.tol;
    }
    st.converged = converged ? 1 : 0;
    return converged ? DLZ_OK : DLZ_ERR_NOT_CONVERGED;
}

}  // namespace dlz

// Host entry of the Rayleigh-Ritz step (dlz.h: dlz_host_rayleigh_ritz).
extern "C" int dlz_host_rayleigh_ritz(int k, const double *H, const double *G, double *values, double *Z) {
    if (k < 1 || !H || !values) return dlz::fail(DLZ_ERR_BADARG, "rayleigh_ritz: k >= 1, H and values required");
    std::vector<std::complex<double>> h((size_t)k * k), g;
    for (size_t i = 0; i < h.size(); ++i) h[i] = std::complex<double>(H[2 * i], H[2 * i + 1]);
    if (G) {
        g.resize((size_t)k * k);
        for (size_t i = 0; i < g.size(); ++i) g[i] = std::complex<double>(G[2 * i], G[2 * i + 1]);
    }
    std::vector<double> w;
    std::vector<std::complex<double>> z;
    const int rc = dlz::rayleigh_ritz(k, h, G ? &g : nullptr, w, z);
    if (rc != DLZ_OK) return rc;
    for (int j = 0; j < k; ++j) values[j] = w[j];
    if (Z)
        for (size_t i = 0; i < z.size(); ++i) {
            Z[2 * i] = z[i].real();
            Z[2 * i + 1] = z[i].imag();
        }
    return DLZ_OK;
}

