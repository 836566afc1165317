// Fused FP32 CG on the normal equations (CGNR) for a batch of right-hand sides:
// the inner solve of the mixed-precision D-CG (arXiv:0901.3163, Sec. 2: CG on
// D^dag D).  For D e = s0 it iterates, per right-hand side, CG on D^dag D e = D^dag s0
// with the norm of the residual of D e = s0 carried alongside:
//   p = r + beta p,  t = D p,  alpha = |r|^2 / |t|^2,
//   e += alpha p,  (s -= alpha t),  r -= alpha D^dag t,  beta = |r_new|^2 / |r|^2,
// s being the residual of D e = s0 (|s| is the quantity the inner stopping test needs)
// and r = D^dag s the CG residual (r starts as D^dag s0 and is then updated by the
// recurrence, as in CG on any hermitian matrix).  Since D p = D r + beta D p_old, the
// image t is carried too, so that each kernel applies its stencil to ONE vector:
//   K1:  t = D r + beta t (the stencil gathers r), p = r + beta p, and the previous
//        step's e += alpha p_old (K1 reads p_old anyway, so e is carried one step
//        behind and K23 touches neither p nor e); block partials of |t|^2.
//   K23: z = D^dag t (the stencil gathers t); r -= alpha z; block partials of |r|^2.  |s|^2 follows from |s_{k+1}|^2 = |s_k|^2 - alpha_k |r_k|^2,
//        so s is updated (and summed) only by the first K23 of a solve.
// Each kernel writes only vectors it does not gather (and only at its own site), so
// every vector is updated in place.  One-block-per-RHS kernels sum the partials in a
// fixed order and update the step lengths; six iterations form a CUDA graph that is
// captured once and replayed.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "dlz_internal.cuh"
#include "krylov_util.cuh"
#include "reduce.cuh"
#include "slab_walk.cuh"
#include "solvers.h"
#include "stage_gather.cuh"
#include "wilson_eo_site.cuh"
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

__device__ inline void axpy_store(float4 *__restrict__ P, size_t base, int V, int s, float a,
                                  const float2 (&x)[12], float2 (&y)[12]) {
    // y = x + a y at site s (y read from and written back to P)
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const size_t i = base + (size_t)c * V + s;
        const float4 q = P[i];
        const float2 x0 = x[2 * c], x1 = x[2 * c + 1];
        const float4 r = make_float4(fmaf(a, q.x, x0.x), fmaf(a, q.y, x0.y), fmaf(a, q.z, x1.x), fmaf(a, q.w, x1.y));
        P[i] = r;
        y[2 * c] = make_float2(r.x, r.y);
        y[2 * c + 1] = make_float2(r.z, r.w);
    }
}

// p = r + beta p at site s, and the deferred update of the previous step e += alpha p_old
// (e is carried one step behind, so that the kernel that reads p_old also moves e)
__device__ inline void pe_update(float4 *__restrict__ P, float4 *__restrict__ E, size_t base, int V, int s, float bt,
                                 float al, const float2 (&r)[12]) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const size_t i = base + (size_t)c * V + s;
        const float4 q = P[i];
        float4 e = E[i];
        e.x = fmaf(al, q.x, e.x); e.y = fmaf(al, q.y, e.y);
        e.z = fmaf(al, q.z, e.z); e.w = fmaf(al, q.w, e.w);
        E[i] = e;
        const float2 r0 = r[2 * c], r1 = r[2 * c + 1];
        P[i] = make_float4(fmaf(bt, q.x, r0.x), fmaf(bt, q.y, r0.y), fmaf(bt, q.z, r1.x), fmaf(bt, q.w, r1.y));
    }
}

// K1: t = D r + beta t, p = r + beta p, e += alpha p_old (the previous step's update);
// partial |t|^2.  Gathers r only.
template <bool STAGED>
__global__ void __launch_bounds__(kT, STAGED ? 3 : 6)
k_cg_k1(const float4 *__restrict__ R, float4 *__restrict__ P, float4 *__restrict__ T, float4 *__restrict__ E,
        const float4 *__restrict__ links, Geom g, SlabWalk w, float kappa, int N, const CgFusedState *__restrict__ st,
        double *__restrict__ partials, int *__restrict__ err) {
    extern __shared__ __align__(128) float4 stage_sm[];
    __shared__ __align__(8) uint64_t mbar;
    const int q = blockIdx.x % N;
    int s0, nb;
    slab_block(w, blockIdx.x / N, s0, nb);
    const int s = s0 + threadIdx.x;
    const size_t base = (size_t)q * 6 * g.V;
    if (threadIdx.x == 0 && nb > 0) {
        if (!STAGED) prefetch_planes_l2(R + base, 6, g.V, s0, nb);
        prefetch_planes_l2(T + base, 6, g.V, s0, nb);
        prefetch_planes_l2(P + base, 6, g.V, s0, nb);
        prefetch_planes_l2(E + base, 6, g.V, s0, nb);
        if (q == 0) prefetch_planes_l2(links, 12, g.V, s0, nb);
    }
    const bool ok = stage_begin<STAGED>(R + base, g, s0, nb, stage_sm, &mbar, err);
    float v[1] = {0.f};
    if ((int)threadIdx.x < nb && ok) {
        const float bt = st[q].f[1], al = st[q].f[0];
        float2 o[12], t[12], r[12];
        const PackedLinks<float> lk{links, g.V};
        if constexpr (STAGED) {
            const StagedGather32 ga = staged_gather(R + base, g, s0, stage_sm);
            wilson_site_g<float, false, false>(s, g, kappa, ga, lk, o);
            ga.get<0, 0>(s, false, r);
        } else {
            const GlobalGather<float> ga{R + base, g.V};
            wilson_site_g<float, false, false>(s, g, kappa, ga, lk, o);
            Field<float>::load(R + base, g.V, s, r);
        }
        axpy_store(T, base, g.V, s, bt, o, t);
        v[0] = nrm(t);
        pe_update(P, E, base, g.V, s, bt, al, r);
    }
    const int nbq = gridDim.x / N;
    block_partials<1>(v, partials + (size_t)q * nbq + blockIdx.x / N, 0);
}

// K23: r -= alpha D^dag t; partial |r|^2.  Gathers t only.  WITH_S (the first launch of
// a solve, alpha = 0): also s -= alpha t and the partial |s|^2; later |s|^2 follows from
// the scalar recurrence in k_cg_beta and s itself is not needed.
// (7 blocks of 128 threads per SM: 0.757 against 0.801 ms per launch with 6, on 24^3 x 48
// with 16 RHS; K1, which moves more vectors, is best at 6: 1.33 against 1.35 ms)
template <bool STAGED, bool WITH_S>
__global__ void __launch_bounds__(kT, STAGED ? 3 : 7)
k_cg_k23(const float4 *__restrict__ T, float4 *__restrict__ R, float4 *__restrict__ S,
         const float4 *__restrict__ links, Geom g, SlabWalk w, float kappa, int N,
         const CgFusedState *__restrict__ st, double *__restrict__ partials, int *__restrict__ err) {
    extern __shared__ __align__(128) float4 stage_sm[];
    __shared__ __align__(8) uint64_t mbar;
    const int q = blockIdx.x % N;
    int s0, nb;
    slab_block(w, blockIdx.x / N, s0, nb);
    const int s = s0 + threadIdx.x;
    const size_t base = (size_t)q * 6 * g.V;
    if (threadIdx.x == 0 && nb > 0) {
        if (!STAGED) prefetch_planes_l2(T + base, 6, g.V, s0, nb);
        prefetch_planes_l2(R + base, 6, g.V, s0, nb);
        if (WITH_S) prefetch_planes_l2(S + base, 6, g.V, s0, nb);
        if (q == 0) prefetch_planes_l2(links, 12, g.V, s0, nb);
    }
    const bool ok = stage_begin<STAGED>(T + base, g, s0, nb, stage_sm, &mbar, err);
    float v[2] = {0.f, 0.f};
    if ((int)threadIdx.x < nb && ok) {
        const float al = st[q].f[0];
        float2 z[12], tc[12];
        const PackedLinks<float> lk{links, g.V};
        if constexpr (STAGED) {
            const StagedGather32 ga = staged_gather(T + base, g, s0, stage_sm);
            wilson_site_g<float, true, true>(s, g, kappa, ga, lk, z);
            if (WITH_S) ga.get<0, 0>(s, false, tc);
        } else {
            const GlobalGather<float> ga{T + base, g.V};
            wilson_site_g<float, true, true>(s, g, kappa, ga, lk, z);
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const size_t i = base + (size_t)c * g.V + s;
            const float2 z0 = z[2 * c], z1 = z[2 * c + 1];
            float4 r = R[i];
            r.x = fmaf(-al, z0.x, r.x); r.y = fmaf(-al, z0.y, r.y);
            r.z = fmaf(-al, z1.x, r.z); r.w = fmaf(-al, z1.y, r.w);
            R[i] = r;
            v[0] += r.x * r.x + r.y * r.y + r.z * r.z + r.w * r.w;
            if constexpr (WITH_S) {
                float4 t;
                if constexpr (STAGED) t = make_float4(tc[2 * c].x, tc[2 * c].y, tc[2 * c + 1].x, tc[2 * c + 1].y);
                else t = T[i];
                float4 sv = S[i];
                sv.x = fmaf(-al, t.x, sv.x); sv.y = fmaf(-al, t.y, sv.y);
                sv.z = fmaf(-al, t.z, sv.z); sv.w = fmaf(-al, t.w, sv.w);
                S[i] = sv;
                v[1] += sv.x * sv.x + sv.y * sv.y + sv.z * sv.z + sv.w * sv.w;
            }
        }
    }
    const int nbq = gridDim.x / N;
    if constexpr (WITH_S) block_partials<2>(v, partials + (size_t)q * nbq + blockIdx.x / N, (size_t)N * nbq);
    else {
        float v1[1] = {v[0]};
        block_partials<1>(v1, partials + (size_t)q * nbq + blockIdx.x / N, 0);
    }
}

// Even-odd operator (Dhat on the even sites): each stencil is two launches, the odd
// hop (eo_hop32, gathering r or gamma5 t) and these Schur-step kernels at the even
// sites, which gather the odd field and carry the same updates as K1 and K23.
// K1b: t = Dhat r + beta t = (r - kappa^2 H_eo m) + beta t with m = H_oe r, p = r + beta p,
// e += alpha p_old as in K1.
__global__ void __launch_bounds__(kT, 6)
k_cg_eo_k1b(const float4 *__restrict__ R, const float4 *__restrict__ M, float4 *__restrict__ P, float4 *__restrict__ T,
            float4 *__restrict__ E, const float4 *__restrict__ links, Geom gf, SlabWalk w, float kappa2, int N,
            const CgFusedState *__restrict__ st, double *__restrict__ partials) {
    const int q = blockIdx.x % N;
    int c0, nb;
    slab_block(w, blockIdx.x / N, c0, nb);
    const int cb = c0 + threadIdx.x;
    const int Vh = gf.V >> 1;
    const size_t base = (size_t)q * 6 * Vh;
    if (threadIdx.x == 0 && nb > 0) {
        prefetch_planes_l2(R + base, 6, Vh, c0, nb);
        prefetch_planes_l2(T + base, 6, Vh, c0, nb);
        prefetch_planes_l2(P + base, 6, Vh, c0, nb);
        prefetch_planes_l2(E + base, 6, Vh, c0, nb);
    }
    float v[1] = {0.f};
    if ((int)threadIdx.x < nb) {
        const float bt = st[q].f[1], al = st[q].f[0];
        float2 o[12], t[12];
        wilson_eo_schur_site<float, false, false>(cb, gf, kappa2, R + base, M + base, links, o);
        axpy_store(T, base, Vh, cb, bt, o, t);
        v[0] = nrm(t);
        float2 r[12];
        Field<float>::load(R + base, Vh, cb, r);
        pe_update(P, E, base, Vh, cb, bt, al, r);
    }
    const int nbq = gridDim.x / N;
    block_partials<1>(v, partials + (size_t)q * nbq + blockIdx.x / N, 0);
}

// K23b: z = Dhat^dag t = gamma5 (gamma5 t - kappa^2 H_eo m), m = H_oe gamma5 t;
// r -= alpha z (WITH_S: s -= alpha t as in K23).
template <bool WITH_S>
__global__ void __launch_bounds__(kT, 6)
k_cg_eo_k23b(const float4 *__restrict__ T, const float4 *__restrict__ M, float4 *__restrict__ R,
             float4 *__restrict__ S, const float4 *__restrict__ links, Geom gf, SlabWalk w, float kappa2, int N,
             const CgFusedState *__restrict__ st, double *__restrict__ partials) {
    const int q = blockIdx.x % N;
    int c0, nb;
    slab_block(w, blockIdx.x / N, c0, nb);
    const int cb = c0 + threadIdx.x;
    const int Vh = gf.V >> 1;
    const size_t base = (size_t)q * 6 * Vh;
    if (threadIdx.x == 0 && nb > 0) {
        prefetch_planes_l2(T + base, 6, Vh, c0, nb);
        prefetch_planes_l2(R + base, 6, Vh, c0, nb);
        if (WITH_S) prefetch_planes_l2(S + base, 6, Vh, c0, nb);
    }
    float v[2] = {0.f, 0.f};
    if ((int)threadIdx.x < nb) {
        const float al = st[q].f[0];
        float2 z[12];
        wilson_eo_schur_site<float, true, true>(cb, gf, kappa2, T + base, M + base, links, z);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const size_t i = base + (size_t)c * Vh + cb;
            const float2 z0 = z[2 * c], z1 = z[2 * c + 1];
            float4 r = R[i];
            r.x = fmaf(-al, z0.x, r.x); r.y = fmaf(-al, z0.y, r.y);
            r.z = fmaf(-al, z1.x, r.z); r.w = fmaf(-al, z1.y, r.w);
            R[i] = r;
            v[0] += r.x * r.x + r.y * r.y + r.z * r.z + r.w * r.w;
            if constexpr (WITH_S) {
                const float4 t = T[i];
                float4 sv = S[i];
                sv.x = fmaf(-al, t.x, sv.x); sv.y = fmaf(-al, t.y, sv.y);
                sv.z = fmaf(-al, t.z, sv.z); sv.w = fmaf(-al, t.w, sv.w);
                S[i] = sv;
                v[1] += sv.x * sv.x + sv.y * sv.y + sv.z * sv.z + sv.w * sv.w;
            }
        }
    }
    const int nbq = gridDim.x / N;
    if constexpr (WITH_S) block_partials<2>(v, partials + (size_t)q * nbq + blockIdx.x / N, (size_t)N * nbq);
    else {
        float v1[1] = {v[0]};
        block_partials<1>(v1, partials + (size_t)q * nbq + blockIdx.x / N, 0);
    }
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

// e += alpha p for every right-hand side (n float4 per right-hand side): the update that
// K1 carries one step behind, made once after an inner solve's last step
__global__ void k_cg_flush_e(float4 *__restrict__ E, const float4 *__restrict__ P,
                             const CgFusedState *__restrict__ st, long n, int N) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)N * n) return;
    const float al = st[i / n].f[0];
    const float4 q = P[i];
    float4 e = E[i];
    e.x = fmaf(al, q.x, e.x); e.y = fmaf(al, q.y, e.y);
    e.z = fmaf(al, q.z, e.z); e.w = fmaf(al, q.w, e.w);
    E[i] = e;
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

// |r_new|^2, |s_new|^2, beta (init: beta = 0, |s|^2 summed).  After the first step
// |s|^2 follows from the recurrence of CG on the normal equations,
//   |s_{k+1}|^2 = |s_k - alpha_k t_k|^2 = |s_k|^2 - alpha_k |r_k|^2,
// since <s_k, t_k> = <s_k, D p_k> = <r_k, p_k> = |r_k|^2 and alpha_k |t_k|^2 = |r_k|^2; it
// only steers the inner stopping test (the outer loop recomputes the residual in FP64).
__global__ void __launch_bounds__(256) k_cg_beta(const double *__restrict__ partials, int nbq, int N, int init,
                                                 CgFusedState *st) {
    const int q = blockIdx.x;
    const double rr = block_total(partials + (size_t)q * nbq, nbq);
    const double ss = init ? block_total(partials + (size_t)N * nbq + (size_t)q * nbq, nbq) : 0.0;
    if (threadIdx.x == 0) {
        CgFusedState s = st[q];
        s.beta = (init || !(s.gam > 0.0)) ? 0.0 : rr / s.gam;
        s.ss = init ? ss : fmax(0.0, s.ss - s.alpha * s.gam);
        s.gam = rr;
        s.f[1] = (float)s.beta;
        st[q] = s;
    }
}

// The slab walk of the fused kernels for an N-RHS batch (~900 bytes per site and
// right-hand side: K23's streams); the even-odd kernels walk the even sites
SlabWalk cg_slab_walk(const Op &op, int N) {
    const Geom &g = op.eo ? op.gf : op.g;
    return make_slab_walk(g.L[0] * g.L[1] / (op.eo ? 2 : 1), g.L[2], g.L[3], N, 900.0);
}

// Whether the full-lattice kernels stage the gathered field in shared memory
// (DLZ_CG_STAGE=1, when the block's ranges fit).  Off by default: on 24^3 x 48 with 16
// right-hand sides the staged kernels took 2.17 (K23) and 1.67 ms (K1) per launch against
// 1.54 and 1.04 ms reading the neighbours from global memory (both in slabs of 4
// z-planes).  With 66 KB of shared memory per block only 3 blocks fit on an SM (12 warps
// against 24), and a block computes nothing until all of its copies have landed.
bool cg_staged(const Op &op) {
    if (op.eo || stage_bytes(op.g.L[0]) > 200 * 1024) return false;
    const char *env = std::getenv("DLZ_CG_STAGE");
    return env && env[0] == '1';
}

// dynamic shared memory of the staged kernels beyond 48 KB (set once, outside any graph
// capture)
int cg_prepare() {
    static int done = 0;
    if (done) return DLZ_OK;
    const int mx = 200 * 1024;
    DLZ_CUDA_TRY(cudaFuncSetAttribute(k_cg_k1<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    DLZ_CUDA_TRY(cudaFuncSetAttribute(k_cg_k23<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    DLZ_CUDA_TRY(cudaFuncSetAttribute(k_cg_k23<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    done = 1;
    return DLZ_OK;
}

}  // namespace

long cgnr_blocks_per_rhs(const Op &op, int N) {
    return slab_blocks(cg_slab_walk(op, N));
}

int cgnr_fused_batch(Op &op, int N, float4 *s0, float4 *e, float4 *const bufs[5], CgFusedState *ms,
                     double *partials, const double *d_tol, const dlz_params &p, int &iters) {
    const long n = 6L * op.g.V;
    const Geom g = op.g;
    const float kappa = (float)op.kappa;
    const float4 *links = op.gauge32.as<float4>();
    const SlabWalk w = cg_slab_walk(op, N);
    const unsigned blocks = (unsigned)(cgnr_blocks_per_rhs(op, N) * N);
    const int nbq = (int)(blocks / N);
    const bool staged = cg_staged(op);
    const int smem = staged ? stage_bytes(g.L[0]) : 0;
    int *err = op.stage_err.as<int>();
    if (staged) DLZ_TRY(cg_prepare());
    auto k1 = [&]() {
        if (staged)
            k_cg_k1<true><<<blocks, kT, smem, op.stream>>>(bufs[0], bufs[1], bufs[2], e, links, g, w, kappa, N,
                                                          ms,
                                                          partials, err);
        else
            k_cg_k1<false><<<blocks, kT, 0, op.stream>>>(bufs[0], bufs[1], bufs[2], e, links, g, w, kappa, N,
                                                          ms,
                                                        partials, err);
    };
    auto k23 = [&](bool with_s) {
        if (staged && with_s)
            k_cg_k23<true, true><<<blocks, kT, smem, op.stream>>>(bufs[2], bufs[0], s0, links, g, w,
                                                                 kappa, N, ms, partials, err);
        else if (staged)
            k_cg_k23<true, false><<<blocks, kT, smem, op.stream>>>(bufs[2], bufs[0], s0, links, g, w,
                                                                  kappa, N, ms, partials, err);
        else if (with_s)
            k_cg_k23<false, true><<<blocks, kT, 0, op.stream>>>(bufs[2], bufs[0], s0, links, g, w, kappa,
                                                               N, ms, partials, err);
        else
            k_cg_k23<false, false><<<blocks, kT, 0, op.stream>>>(bufs[2], bufs[0], s0, links, g, w,
                                                                kappa, N, ms, partials, err);
    };
    float4 *S = s0, *R = bufs[0], *P = bufs[1], *T = bufs[2];
    // p = t = 0 so that the first K1 (beta = 0) gives p = r, t = D r
    for (float4 *z : {P, T})
        DLZ_CUDA_TRY(cudaMemsetAsync(z, 0, (size_t)N * n * sizeof(float4), op.stream));
    DLZ_CUDA_TRY(cudaMemsetAsync(ms, 0, (size_t)N * sizeof(CgFusedState), op.stream));
    // r = D^dag s0; gamma = |r|^2, |s0|^2 (K23 with t = 0 and alpha = 0 would not form
    // D^dag s0, so the plain batched stencil does it, and K23 with alpha = 0 sums)
    DLZ_TRY(wilson32_batch(op, R, S, DLZ_DDAG, N));
    if (op.eo) {
        // t = 0: the odd hop of it is 0 and K23b only sums |r|^2 and |s|^2
        float4 *M = op.eo_tmp32.as<float4>();
        DLZ_CUDA_TRY(cudaMemsetAsync(M, 0, (size_t)N * n * sizeof(float4), op.stream));
        k_cg_eo_k23b<true><<<blocks, kT, 0, op.stream>>>(T, M, R, S, links, op.gf, w,
                                                         (float)(op.kappa * op.kappa), N, ms, partials);
    } else {
        k23(true);
    }
    k_cg_beta<<<N, 256, 0, op.stream>>>(partials, nbq, N, 1, ms);
    op.prof.launches += 2;
    DLZ_CUDA_TRY(cudaGetLastError());
    auto iteration = [&]() -> int {
        if (op.eo) {
            // even-odd: K1 = odd hop + K1b, K23 = odd hop + K23b (m: the odd work field).
            // Per even site and RHS, K1 moves 240 reals (r gathered by the hop, m written,
            // m gathered, r, t, p, e read, t, p, e written), K23 144 (t gathered by the hop,
            // m written, m gathered, r read and written); each pair reads every link twice
            // (192 reals per even site)
            float4 *M = op.eo_tmp32.as<float4>();
            const float kappa2 = (float)(op.kappa * op.kappa);
            op.prof.stencil_start(op.stream, true, g.V, N, 240, 1, 192);
            DLZ_TRY(eo_hop32(op, M, R, 1, false, N));
            k_cg_eo_k1b<<<blocks, kT, 0, op.stream>>>(R, M, P, T, e, links, op.gf, w, kappa2, N, ms, partials);
            op.prof.stencil_stop(op.stream);
            k_cg_alpha<<<N, 256, 0, op.stream>>>(partials, nbq, ms);
            op.prof.stencil_start(op.stream, true, g.V, N, 144, 2, 192);
            DLZ_TRY(eo_hop32(op, M, T, 1, true, N));
            k_cg_eo_k23b<false><<<blocks, kT, 0, op.stream>>>(T, M, R, S, links, op.gf, w, kappa2, N, ms,
                                                              partials);
            op.prof.stencil_stop(op.stream);
            k_cg_beta<<<N, 256, 0, op.stream>>>(partials, nbq, N, 0, ms);
            op.prof.launches += 4;
            DLZ_CUDA_TRY(cudaGetLastError());
            return DLZ_OK;
        }
        // K1 moves 168 reals per site and RHS (r gathered, t, p and e read and written) + links
        op.prof.stencil_start(op.stream, true, g.V, N, 168, 1);
        k1();
        op.prof.stencil_stop(op.stream);
        k_cg_alpha<<<N, 256, 0, op.stream>>>(partials, nbq, ms);
        // K23 moves 72 reals per site and RHS (t gathered; r read and written) + links
        op.prof.stencil_start(op.stream, true, g.V, N, 72, 2);
        k23(false);
        op.prof.stencil_stop(op.stream);
        k_cg_beta<<<N, 256, 0, op.stream>>>(partials, nbq, N, 0, ms);
        op.prof.launches += 4;
        DLZ_CUDA_TRY(cudaGetLastError());
        return DLZ_OK;
    };
    GraphExec ge;
    auto six = [&]() -> int {
        for (int sub = 0; sub < 6; ++sub) DLZ_TRY(iteration());
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
            if (staged) {
                // a staging wait that gave up leaves its block's sums out: stop at once
                int h_err = 0;
                DLZ_TRY(d2h_sync(op, &h_err, err, sizeof(int)));
                if (h_err) break;
            }
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
    // the last step's e += alpha p, which the next K1 would have made
    k_cg_flush_e<<<(unsigned)(((long)N * n + 255) / 256), 256, 0, op.stream>>>(e, P, ms, n, N);
    op.prof.launches++;
    DLZ_CUDA_TRY(cudaGetLastError());
    iters += it;
    if (staged) {
        int h_err = 0;
        DLZ_TRY(d2h_sync(op, &h_err, err, sizeof(int)));
        if (h_err) {
            DLZ_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), op.stream));
            return fail(DLZ_ERR_DEVICE_TIMEOUT, "a staging wait of the fused CGNR kernels gave up");
        }
    }
    return DLZ_OK;
}

}  // namespace dlz
