/*
 * Wilson-Dirac operator as plain C loops, FP64 (test infrastructure only).
 *
 * The same definition as oracle/wilson.py (the Wilson matrix M of Sec. 2 of
 * arXiv:0901.3163), written out site by site so that large lattices can be
 * checked and timed on the host:
 *
 *   (D psi)(x) = psi(x) - kappa * sum_mu [ (1 - s gamma_mu) U_mu(x) psi(x+mu)
 *                                        + (1 + s gamma_mu) U_mu(x-mu)^dag psi(x-mu) ]
 *
 * s = +1 for D and s = -1 for D^dagger.  The 4x4 spin matrices are built from
 * the Pauli matrices (chiral basis) and applied as full matrices: no spin
 * projection.  Layouts: psi[V][4][3] complex, U[4][V][3][3] complex (row
 * major), site s = ((t*Lz + z)*Ly + y)*Lx + x.  Sites are independent, so the
 * OpenMP loop gives bit-identical results for any thread count.
 */
#include <complex.h>
#include <stddef.h>

typedef double _Complex cplx;

static void gamma_table(cplx g[4][4][4])
{
    /* sigma_1, sigma_2, sigma_3 */
    const cplx s[3][2][2] = {
        {{0, 1}, {1, 0}},
        {{0, -I}, {I, 0}},
        {{1, 0}, {0, -1}},
    };
    for (int m = 0; m < 4; ++m)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b)
                g[m][a][b] = 0;
    for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                g[k][a][2 + b] = -I * s[k][a][b];   /* upper right: -i sigma_k */
                g[k][2 + a][b] = I * s[k][a][b];    /* lower left:  +i sigma_k */
            }
    for (int a = 0; a < 2; ++a) {                   /* gamma_4 = [[0,1],[1,0]] */
        g[3][a][2 + a] = 1;
        g[3][2 + a][a] = 1;
    }
}

static long neighbour(const int c[4], const int dims[4], int mu, int step, int *wrapped_t)
{
    int d[4] = {c[0], c[1], c[2], c[3]};
    d[mu] += step;
    *wrapped_t = 0;
    if (d[mu] < 0) { d[mu] += dims[mu]; if (mu == 3) *wrapped_t = 1; }
    if (d[mu] >= dims[mu]) { d[mu] -= dims[mu]; if (mu == 3) *wrapped_t = 1; }
    return (((long)d[3] * dims[2] + d[2]) * dims[1] + d[1]) * dims[0] + d[0];
}

/* out = D in (dagger = 0) or D^dagger in (dagger = 1); arrays as interleaved re/im doubles. */
void oracle_wilson(const double *U_, const double *in_, double *out_,
                   const int *dims, double kappa, int bc_t, int dagger)
{
    const cplx *U = (const cplx *)U_;
    const cplx *in = (const cplx *)in_;
    cplx *out = (cplx *)out_;
    const long V = (long)dims[0] * dims[1] * dims[2] * dims[3];
    const double sgn = dagger ? -1.0 : 1.0;
    cplx g[4][4][4];
    gamma_table(g);
    cplx pm[4][4][4], pp[4][4][4];           /* 1 - s gamma_mu and 1 + s gamma_mu */
    for (int m = 0; m < 4; ++m)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                cplx one = (a == b) ? 1.0 : 0.0;
                pm[m][a][b] = one - sgn * g[m][a][b];
                pp[m][a][b] = one + sgn * g[m][a][b];
            }

#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; ++s) {
        int c[4];
        long r = s;
        c[0] = (int)(r % dims[0]); r /= dims[0];
        c[1] = (int)(r % dims[1]); r /= dims[1];
        c[2] = (int)(r % dims[2]); r /= dims[2];
        c[3] = (int)r;
        cplx acc[4][3] = {{0}};
        for (int mu = 0; mu < 4; ++mu) {
            int wt;
            /* forward: (1 - s g_mu) U_mu(x) psi(x + mu) */
            long sf = neighbour(c, dims, mu, +1, &wt);
            double ph = wt ? (double)bc_t : 1.0;
            const cplx *u = U + ((long)mu * V + s) * 9;
            const cplx *p = in + sf * 12;
            cplx h[4][3];
            for (int b = 0; b < 4; ++b)
                for (int i = 0; i < 3; ++i) {
                    cplx t = 0;
                    for (int j = 0; j < 3; ++j)
                        t += u[i * 3 + j] * p[b * 3 + j];
                    h[b][i] = ph * t;
                }
            for (int a = 0; a < 4; ++a)
                for (int i = 0; i < 3; ++i) {
                    cplx t = 0;
                    for (int b = 0; b < 4; ++b)
                        t += pm[mu][a][b] * h[b][i];
                    acc[a][i] += t;
                }
            /* backward: (1 + s g_mu) U_mu(x - mu)^dagger psi(x - mu) */
            long sb = neighbour(c, dims, mu, -1, &wt);
            ph = wt ? (double)bc_t : 1.0;
            u = U + ((long)mu * V + sb) * 9;
            p = in + sb * 12;
            for (int b = 0; b < 4; ++b)
                for (int i = 0; i < 3; ++i) {
                    cplx t = 0;
                    for (int j = 0; j < 3; ++j)
                        t += conj(u[j * 3 + i]) * p[b * 3 + j];
                    h[b][i] = ph * t;
                }
            for (int a = 0; a < 4; ++a)
                for (int i = 0; i < 3; ++i) {
                    cplx t = 0;
                    for (int b = 0; b < 4; ++b)
                        t += pp[mu][a][b] * h[b][i];
                    acc[a][i] += t;
                }
        }
        for (int a = 0; a < 4; ++a)
            for (int i = 0; i < 3; ++i)
                out[s * 12 + a * 3 + i] = in[s * 12 + a * 3 + i] - kappa * acc[a][i];
    }
}

/* Evaluate D (or D^dagger) at a list of sites only: out[j][12] for sites[j]. */
void oracle_wilson_sites(const double *U_, const double *in_, double *out_,
                         const int *dims, double kappa, int bc_t, int dagger,
                         const long *sites, long nsites)
{
    /* Reuse the full-site kernel on a one-site window is not possible without
     * the whole field, so evaluate the definition directly here as well. */
    const cplx *U = (const cplx *)U_;
    const cplx *in = (const cplx *)in_;
    cplx *out = (cplx *)out_;
    const long V = (long)dims[0] * dims[1] * dims[2] * dims[3];
    const double sgn = dagger ? -1.0 : 1.0;
    cplx g[4][4][4];
    gamma_table(g);
    for (long j = 0; j < nsites; ++j) {
        long s = sites[j];
        int c[4];
        long r = s;
        c[0] = (int)(r % dims[0]); r /= dims[0];
        c[1] = (int)(r % dims[1]); r /= dims[1];
        c[2] = (int)(r % dims[2]); r /= dims[2];
        c[3] = (int)r;
        cplx acc[4][3] = {{0}};
        for (int mu = 0; mu < 4; ++mu)
            for (int dir = 0; dir < 2; ++dir) {
                int wt;
                long sn = neighbour(c, dims, mu, dir == 0 ? +1 : -1, &wt);
                double ph = wt ? (double)bc_t : 1.0;
                const cplx *u = U + ((long)mu * V + (dir == 0 ? s : sn)) * 9;
                const cplx *p = in + sn * 12;
                cplx h[4][3];
                for (int b = 0; b < 4; ++b)
                    for (int i = 0; i < 3; ++i) {
                        cplx t = 0;
                        for (int k = 0; k < 3; ++k)
                            t += (dir == 0 ? u[i * 3 + k] : conj(u[k * 3 + i])) * p[b * 3 + k];
                        h[b][i] = ph * t;
                    }
                double sp = (dir == 0) ? -sgn : sgn;  /* 1 - s g (fwd), 1 + s g (bwd) */
                for (int a = 0; a < 4; ++a)
                    for (int i = 0; i < 3; ++i) {
                        cplx t = h[a][i];
                        for (int b = 0; b < 4; ++b)
                            t += sp * g[mu][a][b] * h[b][i];
                        acc[a][i] += t;
                    }
            }
        for (int a = 0; a < 4; ++a)
            for (int i = 0; i < 3; ++i)
                out[j * 12 + a * 3 + i] = in[s * 12 + a * 3 + i] - kappa * acc[a][i];
    }
}
