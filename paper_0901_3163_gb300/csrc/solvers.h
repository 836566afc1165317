// Solver entry points between the C ABI (api.cu) and the kernels (solvers.cu).
#pragma once

#include <complex>
#include <vector>

#include "dlz_internal.cuh"

// The deflation set of Sec. 2: k orthonormal vectors (regular Ritz vectors
// of Lan-DR or the span of the harmonic Ritz vectors of MinRes-DR) and the
// projected operator H = V^dag A V used by the Galerkin projection of
// D-CG / D-MinRes.
struct dlz_defl_s {
    dlz::Op *op = nullptr;
    int k = 0;
    int which = DLZ_Q;                          // DLZ_Q or DLZ_DDAGD
    dlz::DevBuf V64;                            // k internal FP64 vectors
    dlz::DevBuf V32;                            // FP32 copy for the mixed-precision solvers
    std::vector<std::complex<double>> H;        // k x k, row-major
    std::vector<std::complex<double>> G;        // k x k Gram matrix V_k^dag V_k (empty: V_k
                                                // orthonormal to FP64 rounding)
    std::vector<std::complex<double>> Hlu;      // LU factors of H
    std::vector<int> piv;
    std::vector<double> values;                 // Rayleigh-Ritz values (ascending)
    std::vector<double> residuals;              // ||A y - value y|| (empty until requested)
    std::vector<std::complex<double>> Z;        // eigenvectors of H (column j <-> values[j]); GMRES-DR
                                                // sets: (k+1) x k coefficients of the harmonic Ritz
                                                // vectors in V_{k+1}
    // GMRES-DR sets (which == DLZ_D): V64 holds k + 1 vectors with D V_k = V_{k+1} Hbar
    std::vector<std::complex<double>> Hbar;     // (k+1) x k, row-major
    std::vector<std::complex<double>> theta;    // the kept harmonic Ritz values
};

// The operator object behind dlz_op_t.
struct dlz_op_s {
    dlz::Op op;
    ~dlz_op_s() {
        if (op.cap_stream) cudaStreamDestroy(op.cap_stream);
    }
};

namespace dlz {

// Rayleigh-Ritz pairs of a hermitian k x k H, with the Gram matrix G of a basis that is
// not orthonormal (G null or empty: the plain eigenpairs of H)
int rayleigh_ritz(int k, const std::vector<std::complex<double>> &H, const std::vector<std::complex<double>> *G,
                  std::vector<double> &values, std::vector<std::complex<double>> &Z);

int dr_solve(Op &op, bool harmonic, const double2 *b, double2 *x, const dlz_params &p,
             dlz_defl_s **defl_out, dlz_stats &st);
// x_init (may alias x, may be null): starting guess, corrected by the projection of
// its residual; null: x0 is the projection of the right-hand side.
int dminres64(Op &op, const dlz_defl_s *d, const double2 *b, double2 *x, const dlz_params &p,
              dlz_stats &st, const double2 *x_init = nullptr);
int dcg64(Op &op, const dlz_defl_s *d, const double2 *b, double2 *x, const dlz_params &p,
          dlz_stats &st, const double2 *x_init = nullptr);
// D-MinRes (minres) or D-CG in FP32 with FP64 defect correction on N <= 16
// right-hand sides at once (B, X: N internal FP64 vectors one after another; st: N
// entries); X_init (may alias X, may be null) is the starting guess.
int dsolve_mixed_batch(Op &op, const dlz_defl_s *d, bool minres, const double2 *B, double2 *X, int N,
                       const dlz_params &p, dlz_stats *st, const double2 *X_init = nullptr);
// Hk (k x k, may be null): V_k^dag A V_k known from the restart; else computed (k MVPs).
int build_deflation(Op &op, int which, const double2 *Vk, int k, dlz_defl_s **out, const double *Hk = nullptr);
int deflation_factor(Op &op, dlz_defl_s *d);
int prepare_kernels(Op &op);
struct FusedState;
struct HostScratch;
// Fused two-kernel FP32 MinRes on N right-hand sides (minres_fused.cu).
// e_init: e holds a starting guess (r is then the residual of that guess).
int minres_fused_batch(Op &op, int N, const float4 *r, float4 *e, float4 *const bufs[6],
                       FusedState *ms, double *partials, const double *d_tol,
                       const dlz_params &p, int &iters, HostScratch &hs, bool e_init = false);
// Fused FP32 CG on the normal equations for D e = s0 on N right-hand sides
// (cg_fused.cu); s0 is overwritten, e is updated in place (holds the start).
struct CgFusedState;
// blocks per right-hand side of the fused CGNR kernels for an N-RHS batch (the size of
// their partials arrays)
long cgnr_blocks_per_rhs(const Op &op, int N);
int cgnr_fused_batch(Op &op, int N, float4 *s0, float4 *e, float4 *const bufs[5], CgFusedState *ms,
                     double *partials, const double *d_tol, const dlz_params &p, int &iters);
// FP32 D-MinRes with FP64 defect correction on many lattices at once
// (minres_multi.cu); B[l], X[l]: nrhs[l] <= 16 internal FP64 vectors of lattice l,
// st: one entry per (lattice, right-hand side) in order.
int dminres_multi(int nlat, Op *const *ops, const dlz_defl_s *const *defls, const double2 *const *B,
                  double2 *const *X, const int *nrhs, const dlz_params &p, dlz_stats *st);
// GMRES-DR(m,k) and D-GMRES(m) on D, FP64 (gmres.cu); d may be null (plain GMRES(m)).
int gmresdr64(Op &op, const double2 *b, double2 *x, const dlz_params &p, dlz_defl_s **defl_out, dlz_stats &st);
int dgmres64(Op &op, const dlz_defl_s *d, const double2 *b, double2 *x, const dlz_params &p, dlz_stats &st);
int gmres_deflation_residuals(Op &op, dlz_defl_s *d);
// FP32 copy of the deflation basis (made on first use).
int deflation_v32(Op &op, dlz_defl_s *d);
int deflation_finish(Op &op, dlz_defl_s *d);
// Residuals of the Rayleigh-Ritz pairs (computed on first request: k MVPs).
int deflation_residuals(Op &op, dlz_defl_s *d);

}  // namespace dlz
