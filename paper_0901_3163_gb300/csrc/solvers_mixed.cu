// Mixed-precision D-MinRes and D-CG (arXiv:0901.3163, Sec. 2 methods):
// FP32 stencil and FP32 Krylov vectors inside, FP64 outside.
//
// Defect correction: the FP64 outer loop keeps x in FP64, recomputes the true
// residual r = b' - A x with the FP64 stencil, re-applies the Galerkin
// projection over the deflation set to it (which also removes the deflated
// directions that rounding lets back in), and hands r / ||r|| to an FP32
// MinRes (or CG on the normal equations) that reduces it by the factor
// `reliable_delta`; the FP32 correction is added to x in FP64.  All scalars
// of the inner iteration (alpha, beta, Givens rotations, step lengths) and all
// reductions are FP64; only vectors and the stencil are FP32.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "dlz_internal.cuh"
#include "krylov_util.cuh"
#include "prec.cuh"
#include "reduce.cuh"
#include "small_dense.h"
#include "solvers.h"

namespace dlz {

namespace {

// scalar scratch of the inner solvers (sized for either state: FusedState of the
// fused MinRes or CgFusedState of the fused CGNR)
struct InnerState {
    double beta, alpha, beta_next, inv_beta;
    double c, s, c_old, s_old, phibar;
    double eps, delta, gamma, tau;
    double rr, ss, pq;
    float fa, fb;
};

}  // namespace

}  // namespace dlz

// ------------------------------------------------------------------ batched form
// N <= kMaxBatch right-hand sides share every launch: the stencil processes all
// of them (links read once per site), and each fused reduction carries one
// accumulator per right-hand side.  Each right-hand side keeps its own FP64
// scalar recurrence (MinRes Givens rotations or CG step lengths); a right-hand
// side whose residual is already below tol enters with a zero vector and its
// scalars are held at a no-op.
namespace dlz {

namespace {

constexpr int kMaxBatch = 16;

}  // namespace

int dsolve_mixed_batch(Op &op, const dlz_defl_s *d, bool minres, const double2 *B, double2 *X, int N,
                       const dlz_params &p, dlz_stats *st, const double2 *X_init) {
    if (N < 1 || N > kMaxBatch) return fail(DLZ_ERR_BADARG, "batch size");
    if (minres && op.eo)
        return fail(DLZ_ERR_BADARG, "even-odd operators: FP32 D-MinRes is not built (use DLZ_F64, or D-CG)");
    const long n64 = 12L * op.g.V;
    const long n32 = 6L * op.g.V;
    DevBuf bp, x, r, tmp, corr, dots, scal, f32;
    DLZ_TRY(bp.alloc((size_t)N * n64 * sizeof(double2)));
    DLZ_TRY(x.alloc((size_t)N * n64 * sizeof(double2)));
    DLZ_TRY(r.alloc((size_t)N * n64 * sizeof(double2)));
    DLZ_TRY(tmp.alloc((size_t)N * n64 * sizeof(double2)));
    DLZ_TRY(corr.alloc(n64 * sizeof(double2)));
    DLZ_TRY(dots.alloc((size_t)std::max(1, d ? d->k : 1) * sizeof(double2)));
    DLZ_TRY(scal.alloc((size_t)(kMaxBatch * 24 + 4 * kMaxBatch) * sizeof(double)));
    DLZ_TRY(f32.alloc((size_t)8 * N * n32 * sizeof(float4)));
    float4 *w32[8];
    for (int i = 0; i < 8; ++i) w32[i] = f32.as<float4>() + (size_t)i * N * n32;
    DevBuf fpart, pdot;
    if (d && d->k > 0) {
        DLZ_TRY(pdot.alloc((size_t)N * d->k * sizeof(double2)));
        DLZ_TRY(reserve_multidot(op, d->k));
    }
    const long k1_blocks = std::max((long)((op.g.V + 127) / 128), minres ? 0L : cgnr_blocks_per_rhs(op, N)) * N;
    DLZ_TRY(fpart.alloc((size_t)2 * k1_blocks * sizeof(double)));   // K1 and K2a partials
    InnerState *ist = reinterpret_cast<InnerState *>(scal.as<double>());
    double *d_rn = scal.as<double>() + kMaxBatch * 24;        // ||r_q||
    double *d_inv = d_rn + kMaxBatch, *d_tol = d_inv + kMaxBatch, *d_bn = d_tol + kMaxBatch;
    HostScratch hs;
    DLZ_TRY(hs.ensure(1024));
    double2 *pbp = bp.as<double2>(), *px = x.as<double2>(), *pr = r.as<double2>(), *pt = tmp.as<double2>();
    // b'_q = gamma5 b_q (MinRes on Q) or b_q (CG on the normal equations, residual of D) ; ||b_q||
    {
        const long half = minres ? 6L * op.g.V : n64;
        DLZ_TRY(map(op, n64 * N, [=] __device__(long i) {
            double2 v = B[i];
            if ((i % n64) >= half) { v.x = -v.x; v.y = -v.y; }
            pbp[i] = v;
        }));
    }
    const int which = minres ? DLZ_Q : DLZ_D;
    DLZ_TRY(reduce<kMaxBatch>(op, n64, [=] __device__(long i, double (&acc)[kMaxBatch]) {
#pragma unroll
        for (int q = 0; q < kMaxBatch; ++q)
            if (q < N) { const double2 v = pbp[(size_t)q * n64 + i]; acc[q] += v.x * v.x + v.y * v.y; }
    }, [=] __device__(const double *res) { for (int q = 0; q < N; ++q) d_bn[q] = sqrt(res[q]); }));
    std::vector<double> bn(N);
    DLZ_TRY(d2h_sync(op, bn.data(), d_bn, N * sizeof(double)));
    for (int q = 0; q < N; ++q) {
        std::memset(&st[q], 0, sizeof(dlz_stats));
        if (!std::isfinite(bn[q])) return fail(DLZ_ERR_NONFINITE, "right-hand side is not finite");
    }
    if (X_init)
        DLZ_CUDA_TRY(cudaMemcpyAsync(px, X_init, (size_t)N * n64 * sizeof(double2), cudaMemcpyDeviceToDevice, op.stream));
    else
        DLZ_CUDA_TRY(cudaMemsetAsync(px, 0, (size_t)N * n64 * sizeof(double2), op.stream));
    std::vector<char> done(N, 0);
    std::vector<double> rn(N);
    int iters = 0, outer = 0;
    long long mv_batch = 0;
    auto residuals = [&]() -> int {
        DLZ_TRY(wilson64_batch(op, pt, px, which, N));
        mv_batch += 1;
        DLZ_TRY(reduce<kMaxBatch>(op, n64, [=] __device__(long i, double (&acc)[kMaxBatch]) {
#pragma unroll
            for (int q = 0; q < kMaxBatch; ++q) {
                if (q < N) {
                    const size_t o = (size_t)q * n64 + i;
                    const double2 a = pbp[o], c = pt[o];
                    const double2 t = make_double2(a.x - c.x, a.y - c.y);
                    pr[o] = t;
                    acc[q] += t.x * t.x + t.y * t.y;
                }
            }
        }, [=] __device__(const double *res) { for (int q = 0; q < N; ++q) d_rn[q] = sqrt(res[q]); }));
        DLZ_TRY(d2h_sync(op, rn.data(), d_rn, N * sizeof(double)));
        for (int q = 0; q < N; ++q)
            if (!std::isfinite(rn[q])) return fail(DLZ_ERR_NONFINITE, "residual is not finite");
        return DLZ_OK;
    };
    while (true) {
        DLZ_TRY(residuals());
        bool all = true;
        for (int q = 0; q < N; ++q) {
            if (!done[q] && (bn[q] == 0.0 || rn[q] <= p.tol * bn[q])) {
                done[q] = 1;
                st[q].iterations = iters;
                st[q].cycles = outer;
            }
            all = all && done[q];
        }
        if (all || iters >= p.max_iter) break;
        // normalised FP32 residuals (zero for finished right-hand sides) and inner tolerances.
        // The fused CG tracks |s| by a scalar recurrence whose rounding (about 1e-7 of
        // |s_0|^2 in all) levels off near a 3e-4 reduction of |s|, so its inner reduction
        // is held at 2e-3 or more: 1e-4 kept the inner solve running to max_iter on the
        // 24^3x48 workload, while 1e-3 took 7500 iterations per RHS there against 7524 with
        // the default 1e-2.
        const double delta = minres ? p.reliable_delta : std::max(p.reliable_delta, 2e-3);
        std::vector<double> inv(N), tl(N);
        for (int q = 0; q < N; ++q) {
            const bool open = !done[q] && rn[q] > p.tol * bn[q];
            inv[q] = open ? 1.0 / rn[q] : 0.0;
            tl[q] = open ? std::max(0.5 * p.tol * bn[q] / rn[q], delta) : 1.0;
        }
        DLZ_TRY(h2d(op, d_inv, inv.data(), N * sizeof(double)));
        DLZ_TRY(h2d(op, d_tol, tl.data(), N * sizeof(double)));
        {
            const int V = op.g.V;
            float4 *r32 = w32[0];
            DLZ_TRY(map(op, n32 * N, [=] __device__(long i) {
                const int q = (int)(i / n32);
                const long j = i % n32;
                const int c = (int)(j / V), s = (int)(j % V);
                const double sc = d_inv[q];
                const double2 *src = pr + (size_t)q * n64;
                const double2 a = src[(size_t)(2 * c) * V + s], b = src[(size_t)(2 * c + 1) * V + s];
                r32[i] = make_float4((float)(sc * a.x), (float)(sc * a.y), (float)(sc * b.x), (float)(sc * b.y));
            }));
        }
        // Galerkin projection of each open residual over the deflation set, in FP32
        // (Sec. 2: D-MinRes starts with it; repeated at every defect-correction restart):
        // e0 = V_k H^-1 V_k^dag r, u = r - Q e0; the inner MinRes then starts from e0.
        // D-CG: the projection is that of the normal equations, e0 = V_k H^-1 V_k^dag D^dag r
        // (H = V_k^dag D^dag D V_k), and the inner CG starts from s = r - D e0.
        const bool proj = d && d->k > 0;
        if (proj) {
            const int k = d->k;
            DLZ_TRY(deflation_v32(op, const_cast<dlz_defl_s *>(d)));
            const float4 *V32 = d->V32.as<float4>();
            double2 *pdots = pdot.as<double2>();
            const float4 *rhs32 = w32[0];
            if (!minres) {
                DLZ_TRY(wilson32_batch(op, w32[2], w32[0], DLZ_DDAG, N));
                rhs32 = w32[2];
            }
            // C = V_k^dag R for all N right-hand sides at once and E0 = V_k H^-1 C, both on
            // the tensor cores (tc_gemm.cu) when the shapes tile (k <= 128, 24 V % 32 == 0);
            // otherwise one CUDA-core multi-dot and combine per right-hand side
            const long len = 4L * n32;
            const bool tc = k <= 128 && len % 32 == 0;
            std::vector<double2> hc((size_t)N * k);
            if (tc) {
                DLZ_TRY(tc_dots32(op.tc, op.stream, hc.data(), reinterpret_cast<const float *>(V32), len, k,
                                  reinterpret_cast<const float *>(rhs32), len, N, len, &op.prof.launches));
            } else {
                for (int q = 0; q < N; ++q)
                    DLZ_TRY(multidot<P32>(op, V32, n32, k, rhs32 + (size_t)q * n32, pdots + (size_t)q * k, 1.0));
                DLZ_TRY(d2h_sync(op, hc.data(), pdots, hc.size() * sizeof(double2)));
            }
            std::vector<std::complex<double>> z(k);
            for (int q = 0; q < N; ++q) {
                for (int i = 0; i < k; ++i) z[i] = std::complex<double>(hc[(size_t)q * k + i].x, hc[(size_t)q * k + i].y);
                lu_solve(k, d->Hlu.data(), d->piv.data(), z.data());
                for (int i = 0; i < k; ++i) hc[(size_t)q * k + i] = make_double2(z[i].real(), z[i].imag());
            }
            if (tc) {
                std::vector<double> cf((size_t)2 * k * N);          // complex [k][N]
                for (int i = 0; i < k; ++i)
                    for (int q = 0; q < N; ++q) {
                        cf[2 * ((size_t)i * N + q)] = hc[(size_t)q * k + i].x;
                        cf[2 * ((size_t)i * N + q) + 1] = hc[(size_t)q * k + i].y;
                    }
                DLZ_TRY(tc_combine32(op.tc, op.stream, reinterpret_cast<float *>(w32[1]), len,
                                     reinterpret_cast<const float *>(V32), len, k, len, cf.data(), N, true,
                                     &op.prof.launches));
            } else {
                DLZ_TRY(h2d(op, pdots, hc.data(), hc.size() * sizeof(double2)));
                for (int q = 0; q < N; ++q)
                    DLZ_TRY(combine<P32>(op, w32[1] + (size_t)q * n32, n32, 1, V32, n32, k, pdots + (size_t)q * k, 1,
                                         false, false));
            }
            float4 *qe = w32[2], *r32 = w32[0];
            DLZ_TRY(wilson32_batch(op, qe, w32[1], which, N));
            DLZ_TRY(map(op, n32 * N, [=] __device__(long i) {
                const float4 a = r32[i], b = qe[i];
                r32[i] = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
            }));
        }
        const int it0 = iters;
        if (minres) {
            float4 *const bufs[6] = {w32[2], w32[3], w32[4], w32[5], w32[6], w32[7]};
            DLZ_TRY(minres_fused_batch(op, N, w32[0], w32[1], bufs, reinterpret_cast<FusedState *>(ist),
                                       fpart.as<double>(), d_tol, p, iters, hs, proj));
            mv_batch += iters - it0;
        } else {
            if (!proj) DLZ_CUDA_TRY(cudaMemsetAsync(w32[1], 0, (size_t)N * n32 * sizeof(float4), op.stream));
            float4 *const bufs[5] = {w32[2], w32[3], w32[4], w32[5], w32[6]};
            DLZ_TRY(cgnr_fused_batch(op, N, w32[0], w32[1], bufs, reinterpret_cast<CgFusedState *>(ist),
                                     fpart.as<double>(), d_tol, p, iters));
            mv_batch += 2L * (iters - it0);
        }
        // x_q += ||r_q|| e_q
        {
            const int V = op.g.V;
            const float4 *e32 = w32[1];
            DLZ_TRY(map(op, n32 * N, [=] __device__(long i) {
                const int q = (int)(i / n32);
                const double sc = d_inv[q] > 0.0 ? 1.0 / d_inv[q] : 0.0;
                const long j = i % n32;
                const int c = (int)(j / V), s = (int)(j % V);
                const float4 qv = e32[i];
                double2 *xq = px + (size_t)q * n64;
                double2 &a = xq[(size_t)(2 * c) * V + s];
                double2 &b = xq[(size_t)(2 * c + 1) * V + s];
                a.x += sc * qv.x; a.y += sc * qv.y; b.x += sc * qv.z; b.y += sc * qv.w;
            }));
        }
        ++outer;
    }
    DLZ_CUDA_TRY(cudaMemcpyAsync(X, px, (size_t)N * n64 * sizeof(double2), cudaMemcpyDeviceToDevice, op.stream));
    DLZ_CUDA_TRY(cudaStreamSynchronize(op.stream));
    int rc = DLZ_OK;
    for (int q = 0; q < N; ++q) {
        st[q].true_residual = bn[q] > 0 ? rn[q] / bn[q] : 0.0;
        st[q].converged = done[q] ? 1 : 0;
        if (!done[q]) { st[q].iterations = iters; st[q].cycles = outer; rc = DLZ_ERR_NOT_CONVERGED; }
        st[q].mvps = mv_batch;
    }
    return rc;
}

}  // namespace dlz
