// Fused FP32 CG on the normal equations (CGNR) for a batch of right-hand sides:
// the inner solve of the mixed-precision D-CG (arXiv:0901.3163, Sec. 2: CG on
// D^dag D).  For D e = s0 it iterates, per right-hand side,
//   p = r + beta p,  t = D p,  alpha = |r|^2 / |t|^2,
//   e += alpha p,  s -= alpha t,  r = D^dag s,  beta = |r_new|^2 / |r|^2,
// with s the residual of D e = s0 (so |s| is the quantity the outer FP64 loop
// needs) and r = D^dag s the CG residual of D^dag D e = D^dag s0.
//
// Two full-vector kernels per iteration, each with its stencil:
//   K1:  p_new = r + beta p (formed on the fly at every site the stencil reads),
//        written once; t = D p_new; block partials of |t|^2.
//   K23: s_new = s - alpha t (formed on the fly likewise), written once;
//        e += alpha p_new; r = D^dag s_new; block partials of |r|^2 and |s_new|^2.
// plus one-block-per-RHS kernels that sum the partials in a fixed order and
// update the step lengths.  p and s alternate between two buffers (a stencil
// must not read what its own launch writes), so six iterations form a CUDA
// graph that is captured once and replayed.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "dlz_internal.cuh"
#include "krylov_util.cuh"
#include "reduce.cuh"
#include "solvers.h"
#include "wilson_site.cuh"

namespace dlz {

struct CgFusedState {        // one per right-hand side
    double gam;              // |r|^2
    double alpha, beta;
    double ss;               // |s|^2
    float f[4];              // f0 alpha, f1 beta (FP32 copies for the element updates)
};

namespace {

constexpr int kT = 128;

__device__ inline void load_ab(const float4 *__restrict__ A, const float4 *__restrict__ B, float cb, int V, int s,
                               float2 (&p)[12]) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const float4 a = A[(size_t)c * V + s], b = B[(size_t)c * V + s];
        p[2 * c] = make_float2(fmaf(cb, b.x, a.x), fmaf(cb, b.y, a.y));
        p[2 * c + 1] = make_float2(fmaf(cb, b.z, a.z), fmaf(cb, b.w, a.w));
    }
}

template <int MU, bool G5IN>
__device__ inline void hop_pair_ab(int s, const int (&c)[4], const Geom &g, int stride, const float4 *__restrict__ A,
                                   const float4 *__restrict__ B, float cb, const float4 *__restrict__ U,
                                   float2 (&acc)[12]) {
    const int L = g.L[MU];
    const int sf = (c[MU] == L - 1) ? s - (L - 1) * stride : s + stride;
    const float phf = (MU == 3 && c[3] == L - 1) ? (float)g.bc_t : 1.f;
    const int sb = (c[MU] == 0) ? s + (L - 1) * stride : s - stride;
    const float phb = (MU == 3 && c[3] == 0) ? (float)g.bc_t : 1.f;
    float2 p[12], u[9];
    load_ab(A, B, cb, g.V, sf, p);
    maybe_g5<G5IN>(p);
    load_link<float>(U, g.V, MU, s, u);
    hop_fwd<float, MU>(p, u, phf, acc);
    load_ab(A, B, cb, g.V, sb, p);
    maybe_g5<G5IN>(p);
    load_link<float>(U, g.V, MU, sb, u);
    hop_bwd<float, MU>(p, u, phb, acc);
}

// out = [g5]^G5OUT (1 - kappa H) [g5]^G5IN (A + cb B) at site s; self = (A + cb B)(s)
template <bool G5IN, bool G5OUT>
__device__ inline void wilson_site_ab(int s, const Geom &g, float kappa, const float4 *__restrict__ A,
                                      const float4 *__restrict__ B, float cb, const float4 *__restrict__ U,
                                      float2 (&out)[12], float2 (&self)[12]) {
    int c[4];
    int r = s;
    c[0] = r % g.L[0]; r /= g.L[0];
    c[1] = r % g.L[1]; r /= g.L[1];
    c[2] = r % g.L[2];
    c[3] = r / g.L[2];
    const int st1 = g.L[0], st2 = g.L[0] * g.L[1], st3 = st2 * g.L[2];
    float2 acc[12];
#pragma unroll
    for (int a = 0; a < 12; ++a) acc[a] = make_float2(0.f, 0.f);
    hop_pair_ab<0, G5IN>(s, c, g, 1, A, B, cb, U, acc);
    hop_pair_ab<1, G5IN>(s, c, g, st1, A, B, cb, U, acc);
    hop_pair_ab<2, G5IN>(s, c, g, st2, A, B, cb, U, acc);
    hop_pair_ab<3, G5IN>(s, c, g, st3, A, B, cb, U, acc);
    load_ab(A, B, cb, g.V, s, self);
#pragma unroll
    for (int a = 0; a < 12; ++a) out[a] = self[a];
    maybe_g5<G5IN>(out);
#pragma unroll
    for (int a = 0; a < 12; ++a) {
        out[a].x = out[a].x - kappa * acc[a].x;
        out[a].y = out[a].y - kappa * acc[a].y;
    }
    maybe_g5<G5OUT>(out);
}

__device__ inline float nrm(const float2 (&v)[12]) {
    float a = 0.f;
#pragma unroll
    for (int i = 0; i < 12; ++i) a += v[i].x * v[i].x + v[i].y * v[i].y;
    return a;
}

// block sum of up to two per-thread values into partials (FP64 across threads)
template <int NV>
__device__ inline void block_partials(float (&v)[NV], double *__restrict__ out, size_t stride) {
    __shared__ double sm[NV][kT / 32];
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        double a = (double)v[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if ((threadIdx.x & 31) == 0) sm[j][threadIdx.x >> 5] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            double t = 0.0;
#pragma unroll
            for (int w = 0; w < kT / 32; ++w) t += sm[j][w];
            out[j * stride] = t;
        }
    }
}

__global__ void __launch_bounds__(kT)
k_cg_k1(const float4 *__restrict__ R, const float4 *__restrict__ Pold, float4 *__restrict__ Pnew,
        float4 *__restrict__ T, const float4 *__restrict__ links, Geom g, float kappa, int N,
        const CgFusedState *__restrict__ st, double *__restrict__ partials) {
    const int q = blockIdx.x % N;
    const int s = (blockIdx.x / N) * blockDim.x + threadIdx.x;
    const size_t base = (size_t)q * 6 * g.V;
    float v[1] = {0.f};
    if (s < g.V) {
        const float bt = st[q].f[1];
        float2 o[12], self[12];
        wilson_site_ab<false, false>(s, g, kappa, R + base, Pold + base, bt, links, o, self);
        Field<float>::store(Pnew + base, g.V, s, self);
        Field<float>::store(T + base, g.V, s, o);
        v[0] = nrm(o);
    }
    const int nbq = gridDim.x / N;
    block_partials<1>(v, partials + (size_t)q * nbq + blockIdx.x / N, 0);
}

__global__ void __launch_bounds__(kT)
k_cg_k23(const float4 *__restrict__ S, const float4 *__restrict__ T, float4 *__restrict__ Snew,
         const float4 *__restrict__ Pnew, float4 *__restrict__ E, float4 *__restrict__ R,
         const float4 *__restrict__ links, Geom g, float kappa, int N, const CgFusedState *__restrict__ st,
         double *__restrict__ partials) {
    const int q = blockIdx.x % N;
    const int s = (blockIdx.x / N) * blockDim.x + threadIdx.x;
    const size_t base = (size_t)q * 6 * g.V;
    float v[2] = {0.f, 0.f};
    if (s < g.V) {
        const float al = st[q].f[0];
        float2 o[12], self[12];
        wilson_site_ab<true, true>(s, g, kappa, S + base, T + base, -al, links, o, self);
        Field<float>::store(Snew + base, g.V, s, self);
        Field<float>::store(R + base, g.V, s, o);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const size_t i = base + (size_t)c * g.V + s;
            const float4 p = Pnew[i];
            float4 e = E[i];
            e.x = fmaf(al, p.x, e.x); e.y = fmaf(al, p.y, e.y);
            e.z = fmaf(al, p.z, e.z); e.w = fmaf(al, p.w, e.w);
            E[i] = e;
        }
        v[0] = nrm(o);
        v[1] = nrm(self);
    }
    const int nbq = gridDim.x / N;
    block_partials<2>(v, partials + (size_t)q * nbq + blockIdx.x / N, (size_t)N * nbq);
}

__device__ inline double block_total(const double *__restrict__ p, int n) {
    double t = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) t += p[b];
    __shared__ double sm[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = t;
    __syncthreads();
    double a = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) a += sm[w];
    __syncthreads();
    return a;     // valid in thread 0
}

// alpha = |r|^2 / |t|^2 (one block per right-hand side)
__global__ void __launch_bounds__(256) k_cg_alpha(const double *__restrict__ partials, int nbq, CgFusedState *st) {
    const int q = blockIdx.x;
    const double tt = block_total(partials + (size_t)q * nbq, nbq);
    if (threadIdx.x == 0) {
        CgFusedState s = st[q];
        s.alpha = tt > 0.0 ? s.gam / tt : 0.0;
        s.f[0] = (float)s.alpha;
        st[q] = s;
    }
}

// |r_new|^2, |s_new|^2, beta (init: beta = 0)
__global__ void __launch_bounds__(256) k_cg_beta(const double *__restrict__ partials, int nbq, int N, int init,
                                                 CgFusedState *st) {
    const int q = blockIdx.x;
    const double rr = block_total(partials + (size_t)q * nbq, nbq);
    const double ss = block_total(partials + (size_t)N * nbq + (size_t)q * nbq, nbq);
    if (threadIdx.x == 0) {
        CgFusedState s = st[q];
        s.beta = (init || !(s.gam > 0.0)) ? 0.0 : rr / s.gam;
        s.gam = rr;
        s.ss = ss;
        s.f[1] = (float)s.beta;
        st[q] = s;
    }
}

}  // namespace

int cgnr_fused_batch(Op &op, int N, float4 *s0, float4 *e, float4 *const bufs[5], CgFusedState *ms,
                     double *partials, const double *d_tol, const dlz_params &p, int &iters) {
    const long n = 6L * op.g.V;
    const Geom g = op.g;
    const float kappa = (float)op.kappa;
    const float4 *links = op.gauge32.as<float4>();
    const unsigned blocks = (unsigned)(((g.V + kT - 1) / kT) * N);
    const int nbq = (int)(blocks / N);
    float4 *S[2] = {s0, bufs[0]}, *P[2] = {bufs[1], bufs[2]}, *T = bufs[3], *R = bufs[4];
    for (float4 *z : {P[0], P[1], T})
        DLZ_CUDA_TRY(cudaMemsetAsync(z, 0, (size_t)N * n * sizeof(float4), op.stream));
    DLZ_CUDA_TRY(cudaMemsetAsync(ms, 0, (size_t)N * sizeof(CgFusedState), op.stream));
    // r = D^dag s0 (K23 with alpha = 0), gamma = |r|^2, beta = 0
    k_cg_k23<<<blocks, kT, 0, op.stream>>>(S[0], T, S[1], P[0], e, R, links, g, kappa, N, ms, partials);
    k_cg_beta<<<N, 256, 0, op.stream>>>(partials, nbq, N, 1, ms);
    op.prof.launches += 2;
    DLZ_CUDA_TRY(cudaGetLastError());
    auto iteration = [&](const float4 *pold, float4 *pnew, const float4 *sc, float4 *sn) -> int {
        // K1 moves 96 reals per site and RHS (r, p read; p_new, t written) + links
        op.prof.stencil_start(op.stream, true, g.V, N, 96);
        k_cg_k1<<<blocks, kT, 0, op.stream>>>(R, pold, pnew, T, links, g, kappa, N, ms, partials);
        op.prof.stencil_stop(op.stream);
        k_cg_alpha<<<N, 256, 0, op.stream>>>(partials, nbq, ms);
        // K23 moves 168 reals per site and RHS (s, t, p_new, e read; s_new, e, r written)
        op.prof.stencil_start(op.stream, true, g.V, N, 168);
        k_cg_k23<<<blocks, kT, 0, op.stream>>>(sc, T, sn, pnew, e, R, links, g, kappa, N, ms, partials);
        op.prof.stencil_stop(op.stream);
        k_cg_beta<<<N, 256, 0, op.stream>>>(partials, nbq, N, 0, ms);
        op.prof.launches += 4;
        DLZ_CUDA_TRY(cudaGetLastError());
        return DLZ_OK;
    };
    GraphExec ge;
    auto six = [&]() -> int {
        // state entering the group: p in P[0], s in S[1]
        for (int sub = 0; sub < 6; ++sub) {
            const int a = sub & 1;
            DLZ_TRY(iteration(P[a], P[1 - a], S[1 - a], S[a]));
        }
        return DLZ_OK;
    };
    std::vector<CgFusedState> hsv(N);
    std::vector<double> tol(N);
    DLZ_TRY(d2h_sync(op, tol.data(), d_tol, N * sizeof(double)));
    int it = 0;
    while (it < p.max_iter - iters) {
        DLZ_TRY(run_graph(op, ge, six));
        it += 6;
        if (it % 12 == 0 || it >= p.max_iter - iters) {
            DLZ_TRY(d2h_sync(op, hsv.data(), ms, N * sizeof(CgFusedState)));
            bool all = true;
            for (int q = 0; q < N; ++q) {
                if (!std::isfinite(hsv[q].ss) || !std::isfinite(hsv[q].gam))
                    return fail(DLZ_ERR_NONFINITE, "inner CG residual not finite");
                all = all && std::sqrt(hsv[q].ss) <= tol[q];
            }
            if (all) break;
        }
    }
    ge.sample(op.prof);
    iters += it;
    return DLZ_OK;
}

}  // namespace dlz
