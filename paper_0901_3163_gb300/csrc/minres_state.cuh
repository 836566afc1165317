// State and per-site element updates of the fused FP32 MinRes iteration (the
// inner solve of the mixed-precision D-MinRes, arXiv:0901.3163 Sec. 2), shared by
// the one-lattice kernels (minres_fused.cu) and the multi-lattice kernels
// (minres_multi.cu).
#pragma once

#include "dlz_internal.cuh"
#include "wilson_site.cuh"

namespace dlz {

struct FusedState {          // one per right-hand side (FP64 scalars)
    double beta, alpha, beta_next, inv_beta;
    double c, s, c_old, s_old, phibar;
    double eps, delta, gamma, tau;
    double r0;               // ||r|| at the start of the inner solve
    // FP32 copies read by the element updates (no FP64 op or conversion per element):
    // f[0] 1/beta_j, f[1] beta_j, f[2] delta, f[3] eps, f[4] 1/gamma, f[5] tau, f[6] alpha,
    // f[7] 1/beta_{j-1}
    float f[8];
};

__host__ __device__ inline float4 f4(float a, float b, float c, float d) { return make_float4(a, b, c, d); }

__device__ inline void set_floats(FusedState &s) {
    s.f[0] = (float)s.inv_beta;
    s.f[1] = (float)s.beta_next;
    s.f[2] = (float)s.delta;
    s.f[3] = (float)s.eps;
    s.f[4] = (float)(1.0 / s.gamma);
    s.f[5] = (float)s.tau;
}

// beta_1 = ||r||, rotations reset, a no-op direction update for step 0; tolerances
// are relative to the normalised outer residual (norm 1)
__device__ inline void fused_init(FusedState &out, double b) {
    FusedState s0 = {};
    s0.beta_next = b;
    s0.inv_beta = b > 0 ? 1.0 / b : 0.0;
    s0.c = 1.0; s0.c_old = 1.0; s0.phibar = b; s0.gamma = 1.0; s0.r0 = 1.0;
    set_floats(s0);
    out = s0;
}

__device__ inline void fused_alpha(FusedState &s, double a) {
    s.beta = s.beta_next;
    s.alpha = a;
    s.f[6] = (float)a;
}

// beta_{j+1} = sqrt(r2) and the Givens rotation of step j
__device__ inline void fused_givens(FusedState &s, double r2) {
    const double bn = sqrt(r2);
    const double eps = s.s_old * s.beta;
    const double deltabar = s.c_old * s.beta;
    const double delta = s.c * deltabar + s.s * s.alpha;
    const double gammabar = -s.s * deltabar + s.c * s.alpha;
    double gamma = hypot(gammabar, bn);
    double cn = 1.0, sn = 0.0;
    if (gamma > 0.0) { cn = gammabar / gamma; sn = bn / gamma; }
    else gamma = 1.0;            // zero right-hand side: hold a no-op
    s.tau = cn * s.phibar;
    s.phibar = -sn * s.phibar;
    s.eps = eps; s.delta = delta; s.gamma = gamma;
    s.c_old = s.c; s.s_old = s.s; s.c = cn; s.s = sn;
    s.beta_next = bn;
    s.inv_beta = bn > 0 ? 1.0 / bn : 0.0;
    s.f[7] = s.f[0];             // 1/beta_j, to scale u_j into v_j in the next step
    set_floats(s);
}

// K1 at one site of one right-hand side (pointers at that right-hand side's
// vectors): w = Q u_j / beta_j - beta_j v_{j-1}; d_{j-1}, e updated; returns the
// site's share of Re <v_j, w>.
__device__ inline float minres_k1_site(int s, const Geom &g, float kappa, const float4 *__restrict__ Ub,
                                       const float4 *__restrict__ Up, float4 *__restrict__ W,
                                       const float4 *__restrict__ D2, float4 *__restrict__ D3,
                                       float4 *__restrict__ E, const float4 *__restrict__ links,
                                       const FusedState &st) {
    const float ib = st.f[0], bt = st.f[1], ibp = st.f[7];
    const float de = st.f[2], ep = st.f[3], ig = st.f[4], ta = st.f[5];
    float2 o[12];
    wilson_site<float, false, true>(s, g, kappa, Ub, links, o);   // Q u_j
    float facc = 0.f;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const size_t i = (size_t)c * g.V + s;
        const float4 u = Ub[i], up = Up[i], d2 = D2[i], d3 = D3[i];
        const float4 vj = f4(u.x * ib, u.y * ib, u.z * ib, u.w * ib);
        const float4 vp = f4(up.x * ibp, up.y * ibp, up.z * ibp, up.w * ibp);
        const float4 w = f4(o[2 * c].x * ib - bt * vp.x, o[2 * c].y * ib - bt * vp.y,
                            o[2 * c + 1].x * ib - bt * vp.z, o[2 * c + 1].y * ib - bt * vp.w);
        W[i] = w;
        facc += (vj.x * w.x + vj.y * w.y) + (vj.z * w.z + vj.w * w.w);
        const float4 dn = f4((vp.x - de * d2.x - ep * d3.x) * ig, (vp.y - de * d2.y - ep * d3.y) * ig,
                             (vp.z - de * d2.z - ep * d3.z) * ig, (vp.w - de * d2.w - ep * d3.w) * ig);
        D3[i] = dn;
        float4 ev = E[i];
        ev.x = fmaf(ta, dn.x, ev.x); ev.y = fmaf(ta, dn.y, ev.y);
        ev.z = fmaf(ta, dn.z, ev.z); ev.w = fmaf(ta, dn.w, ev.w);
        E[i] = ev;
    }
    return facc;
}

// K2a at one site: u_{j+1} = w - (alpha_j / beta_j) u_j over w; returns its ||.||^2 share.
// All 6 planes are loaded before any store so the loads overlap.
__device__ inline float minres_k2a_site(int s, int V, float4 *__restrict__ W, const float4 *__restrict__ Uc,
                                        const FusedState &st) {
    const float al = st.f[6] * st.f[0];
    float4 w[6], v[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        w[c] = W[(size_t)c * V + s];
        v[c] = Uc[(size_t)c * V + s];
    }
    float facc = 0.f;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const float4 t = f4(fmaf(-al, v[c].x, w[c].x), fmaf(-al, v[c].y, w[c].y),
                            fmaf(-al, v[c].z, w[c].z), fmaf(-al, v[c].w, w[c].w));
        W[(size_t)c * V + s] = t;
        facc += (t.x * t.x + t.y * t.y) + (t.z * t.z + t.w * t.w);
    }
    return facc;
}

// the direction update of the last step for one element: d_J from u_J, d_{J-1}, d_{J-2}; e += tau d_J
__device__ inline void minres_last_direction(float4 uj, float4 a, float4 b, float4 &ev, const FusedState &st) {
    const float de = st.f[2], ep = st.f[3], ig = st.f[4], ta = st.f[5];
    const float ibj = st.f[7];
    const float4 vp = f4(uj.x * ibj, uj.y * ibj, uj.z * ibj, uj.w * ibj);
    const float4 dn = f4((vp.x - de * a.x - ep * b.x) * ig, (vp.y - de * a.y - ep * b.y) * ig,
                         (vp.z - de * a.z - ep * b.z) * ig, (vp.w - de * a.w - ep * b.w) * ig);
    ev.x = fmaf(ta, dn.x, ev.x); ev.y = fmaf(ta, dn.y, ev.y);
    ev.z = fmaf(ta, dn.z, ev.z); ev.w = fmaf(ta, dn.w, ev.w);
}

// Block sum (FP64 over the threads) of facc stored at *out by thread 0.
template <int BT>
__device__ inline void block_partial_store(float facc, double *__restrict__ out) {
    __shared__ double sm[BT / 32];
    double acc = (double)facc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < BT / 32; ++w) t += sm[w];
        *out = t;
    }
}

// Block partials with the sum taken by the last block to finish.  Each block of
// right-hand side q stores its partial (FP64 over its threads) at slot[b], then
// counts itself in counter[q]; the block that brings the count to nbq adds all nbq
// partials of q in a fixed order and resets the counter (so the sum is deterministic
// and needs no second launch).  Returns true, with the sum in *total (thread 0), in
// that block only.  BT: threads per block.
template <int BT>
__device__ inline bool partial_then_last_sum(float facc, double *__restrict__ slot0, int b, int nbq,
                                             unsigned *__restrict__ counter, double *total) {
    __shared__ double sm[BT / 32];
    __shared__ bool last;
    double acc = (double)facc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < BT / 32; ++w) t += sm[w];
        slot0[b] = t;
        __threadfence();
        last = (atomicAdd(counter, 1u) == (unsigned)nbq - 1u);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double t = 0.0;
    for (int i = threadIdx.x; i < nbq; i += BT) t += __ldcg(&slot0[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
#pragma unroll
        for (int w = 0; w < BT / 32; ++w) a += sm[w];
        *total = a;
        *counter = 0u;
    }
    return true;
}

}  // namespace dlz
