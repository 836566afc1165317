// Per-site Wilson hopping term in the chiral basis, by spin projection.
//
// D psi(x) = psi(x) - kappa sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
//                                   + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ]
// (the Wilson matrix M of arXiv:0901.3163, Sec. 2).  With psi = (u0, u1, l0, l1)
// (spins 0..3, each a colour 3-vector) and gamma_k = [[0, -i s_k], [i s_k, 0]],
// gamma_4 = [[0, 1], [1, 0]], each (1 -+ gamma_mu) has rank 2: its image is fixed
// by a 2-spinor h = (h0, h1) built from psi, with the lower pair a fixed
// 2x2 map (entries 0, +-1, +-i) of the upper pair.  Colour and spin commute,
// so U is applied to h only (2 colour mat-vecs per hop instead of 4):
//
//   fwd mu=x: h = (u0 + i l1, u1 + i l0)   lower = (-i H1, -i H0)
//   fwd mu=y: h = (u0 + l1,   u1 - l0)     lower = (-H1,    H0)
//   fwd mu=z: h = (u0 + i l0, u1 - i l1)   lower = (-i H0,  i H1)
//   fwd mu=t: h = (u0 - l0,   u1 - l1)     lower = (-H0,   -H1)
//   bwd mu=x: h = (u0 - i l1, u1 - i l0)   lower = ( i H1,  i H0)
//   bwd mu=y: h = (u0 - l1,   u1 + l0)     lower = ( H1,   -H0)
//   bwd mu=z: h = (u0 - i l0, u1 + i l1)   lower = ( i H0, -i H1)
//   bwd mu=t: h = (u0 + l0,   u1 + l1)     lower = ( H0,    H1)
// where H = U h (forward) or U^dag h (backward).
#pragma once

#include "dlz_internal.cuh"

namespace dlz {

template <typename T> struct Field;
template <> struct Field<double> {
    typedef double2 vec;
    static constexpr int vec_per_site = 12;
    __host__ __device__ static inline void load(const double2 *__restrict__ p, int V, int s,
                                                double2 (&v)[12]) {
#pragma unroll
        for (int a = 0; a < 12; ++a) v[a] = p[(size_t)a * V + s];
    }
    __host__ __device__ static inline void store(double2 *__restrict__ p, int V, int s,
                                                 const double2 (&v)[12]) {
#pragma unroll
        for (int a = 0; a < 12; ++a) p[(size_t)a * V + s] = v[a];
    }
};
template <> struct Field<float> {
    typedef float4 vec;
    static constexpr int vec_per_site = 6;
    __host__ __device__ static inline void load(const float4 *__restrict__ p, int V, int s,
                                                float2 (&v)[12]) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            float4 q = p[(size_t)c * V + s];
            v[2 * c] = make_float2(q.x, q.y);
            v[2 * c + 1] = make_float2(q.z, q.w);
        }
    }
    __host__ __device__ static inline void store(float4 *__restrict__ p, int V, int s,
                                                 const float2 (&v)[12]) {
#pragma unroll
        for (int c = 0; c < 6; ++c)
            p[(size_t)c * V + s] = make_float4(v[2 * c].x, v[2 * c].y, v[2 * c + 1].x, v[2 * c + 1].y);
    }
};

// Link storage.  FP64: all 9 complex entries, double2 planes [4][9][V].
// FP32: the first two rows only ("12-real" form), float4 planes [4][3][V]
// holding (u00,u01), (u02,u10), (u11,u12); the third row of an SU(3) matrix is
// the complex conjugate of the cross product of the first two,
//   u2j = conj(u0k u1l - u0l u1k)  for (j,k,l) cyclic,
// so 48 instead of 72 bytes are read per link.
template <typename T> struct Link;
template <> struct Link<double> {
    typedef double2 vec;
    static constexpr int planes = 9;
    __host__ __device__ static inline void load(const double2 *__restrict__ U, int V, int mu, int s,
                                                double2 (&u)[9]) {
#pragma unroll
        for (int e = 0; e < 9; ++e) u[e] = U[(size_t)(mu * 9 + e) * V + s];
    }
};
template <> struct Link<float> {
    typedef float4 vec;
    static constexpr int planes = 3;
    __host__ __device__ static inline float2 cmul_conj_diff(float2 a, float2 b, float2 c, float2 d) {
        // conj(a b - c d)
        const float re = (a.x * b.x - a.y * b.y) - (c.x * d.x - c.y * d.y);
        const float im = (a.x * b.y + a.y * b.x) - (c.x * d.y + c.y * d.x);
        return make_float2(re, -im);
    }
    __host__ __device__ static inline void load(const float4 *__restrict__ U, int V, int mu, int s,
                                                float2 (&u)[9]) {
        const float4 q0 = U[(size_t)(mu * 3 + 0) * V + s];
        const float4 q1 = U[(size_t)(mu * 3 + 1) * V + s];
        const float4 q2 = U[(size_t)(mu * 3 + 2) * V + s];
        u[0] = make_float2(q0.x, q0.y);
        u[1] = make_float2(q0.z, q0.w);
        u[2] = make_float2(q1.x, q1.y);
        u[3] = make_float2(q1.z, q1.w);
        u[4] = make_float2(q2.x, q2.y);
        u[5] = make_float2(q2.z, q2.w);
        u[6] = cmul_conj_diff(u[1], u[5], u[2], u[4]);
        u[7] = cmul_conj_diff(u[2], u[3], u[0], u[5]);
        u[8] = cmul_conj_diff(u[0], u[4], u[1], u[3]);
    }
};

template <typename T>
__host__ __device__ inline void load_link(const typename Link<T>::vec *__restrict__ U, int V, int mu, int s,
                                          cx<T> (&u)[9]) {
    Link<T>::load(U, V, mu, s, u);
}

// Where a site function reads its links: (mu, s, u) loads U_mu(s).  PackedLinks reads the
// Link<T> storage (FP32: two rows, the third rebuilt in registers).
template <typename T> struct PackedLinks {
    const typename Link<T>::vec *__restrict__ U;
    int V;
    __host__ __device__ inline void operator()(int mu, int s, cx<T> (&u)[9]) const { Link<T>::load(U, V, mu, s, u); }
};

// Accumulate (1 - gamma_mu) U h-projection of p into acc (forward hop).
template <typename T, int MU>
__host__ __device__ inline void hop_fwd(const cx<T> (&p)[12], const cx<T> (&u)[9], T sign,
                                        cx<T> (&acc)[12]) {
    cx<T> h0[3], h1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cx<T> u0 = p[c], u1 = p[3 + c], l0 = p[6 + c], l1 = p[9 + c];
        if (MU == 0) { h0[c] = addI(u0, l1); h1[c] = addI(u1, l0); }
        if (MU == 1) { h0[c] = u0 + l1;      h1[c] = u1 - l0; }
        if (MU == 2) { h0[c] = addI(u0, l0); h1[c] = subI(u1, l1); }
        if (MU == 3) { h0[c] = u0 - l0;      h1[c] = u1 - l1; }
        h0[c].x *= sign; h0[c].y *= sign; h1[c].x *= sign; h1[c].y *= sign;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        cx<T> H0 = mk<T>(0, 0), H1 = mk<T>(0, 0);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            H0 = cfma(u[3 * i + j], h0[j], H0);
            H1 = cfma(u[3 * i + j], h1[j], H1);
        }
        acc[i] = acc[i] + H0;
        acc[3 + i] = acc[3 + i] + H1;
        if (MU == 0) { acc[6 + i] = subI(acc[6 + i], H1); acc[9 + i] = subI(acc[9 + i], H0); }
        if (MU == 1) { acc[6 + i] = acc[6 + i] - H1;      acc[9 + i] = acc[9 + i] + H0; }
        if (MU == 2) { acc[6 + i] = subI(acc[6 + i], H0); acc[9 + i] = addI(acc[9 + i], H1); }
        if (MU == 3) { acc[6 + i] = acc[6 + i] - H0;      acc[9 + i] = acc[9 + i] - H1; }
    }
}

// Accumulate (1 + gamma_mu) U^dag h-projection of p into acc (backward hop).
template <typename T, int MU>
__host__ __device__ inline void hop_bwd(const cx<T> (&p)[12], const cx<T> (&u)[9], T sign,
                                        cx<T> (&acc)[12]) {
    cx<T> h0[3], h1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cx<T> u0 = p[c], u1 = p[3 + c], l0 = p[6 + c], l1 = p[9 + c];
        if (MU == 0) { h0[c] = subI(u0, l1); h1[c] = subI(u1, l0); }
        if (MU == 1) { h0[c] = u0 - l1;      h1[c] = u1 + l0; }
        if (MU == 2) { h0[c] = subI(u0, l0); h1[c] = addI(u1, l1); }
        if (MU == 3) { h0[c] = u0 + l0;      h1[c] = u1 + l1; }
        h0[c].x *= sign; h0[c].y *= sign; h1[c].x *= sign; h1[c].y *= sign;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        cx<T> H0 = mk<T>(0, 0), H1 = mk<T>(0, 0);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            H0 = cfmaConj(u[3 * j + i], h0[j], H0);
            H1 = cfmaConj(u[3 * j + i], h1[j], H1);
        }
        acc[i] = acc[i] + H0;
        acc[3 + i] = acc[3 + i] + H1;
        if (MU == 0) { acc[6 + i] = addI(acc[6 + i], H1); acc[9 + i] = addI(acc[9 + i], H0); }
        if (MU == 1) { acc[6 + i] = acc[6 + i] + H1;      acc[9 + i] = acc[9 + i] - H0; }
        if (MU == 2) { acc[6 + i] = addI(acc[6 + i], H0); acc[9 + i] = subI(acc[9 + i], H1); }
        if (MU == 3) { acc[6 + i] = acc[6 + i] + H0;      acc[9 + i] = acc[9 + i] + H1; }
    }
}

// Bulk L2 prefetch (cp.async.bulk.prefetch.L2, a TMA operation) of a block's contiguous
// chunk of sites [s0, s0 + n) in each of `planes` planes of stride V (16-byte elements):
// one thread issues it at the start of a latency-bound stencil kernel, so the DRAM reads
// of the block's own site data overlap the neighbour gathers instead of following them.
// Addresses and sizes are multiples of 16 bytes as the instruction requires.
__device__ inline void prefetch_planes_l2(const void *base, int planes, long V, int s0, int n) {
#if defined(__CUDA_ARCH__)
    const unsigned bytes = (unsigned)n * 16u;
    for (int c = 0; c < planes; ++c) {
        const char *a = (const char *)base + ((size_t)c * V + s0) * 16;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(bytes) : "memory");
    }
#endif
}

template <bool G5> __host__ __device__ inline void maybe_g5(double2 (&v)[12]) {
    if (G5) {
#pragma unroll
        for (int a = 6; a < 12; ++a) { v[a].x = -v[a].x; v[a].y = -v[a].y; }
    }
}
template <bool G5> __host__ __device__ inline void maybe_g5(float2 (&v)[12]) {
    if (G5) {
#pragma unroll
        for (int a = 6; a < 12; ++a) { v[a].x = -v[a].x; v[a].y = -v[a].y; }
    }
}

// Where a site function reads the input spinors: get<MU, DIR>(n, wrapped, p) loads the
// spinor of site n, reached by the hop in direction MU (DIR = +1 forward, -1 backward)
// or the site itself (DIR = 0); `wrapped` when the hop crosses the lattice edge.  This
// one reads the field in global memory; the staged kernels read a shared-memory copy.
template <typename T> struct GlobalGather {
    const typename Field<T>::vec *__restrict__ in;
    int V;
    template <int MU, int DIR>
    __host__ __device__ inline void get(int n, bool, cx<T> (&p)[12]) const { Field<T>::load(in, V, n, p); }
};

template <typename T, int MU, bool G5IN, class G, class LK>
__host__ __device__ inline void hop_pair(int s, const int (&c)[4], const Geom &g, int stride, const G &ld,
                                         const LK &lk, cx<T> (&acc)[12]) {
    const int L = g.L[MU];
    // forward neighbour and the boundary phase of a hop across the time edge
    const bool wf = c[MU] == L - 1, wb = c[MU] == 0;
    const int sf = wf ? s - (L - 1) * stride : s + stride;
    const T phf = (MU == 3 && wf) ? (T)g.bc_t : (T)1;
    const int sb = wb ? s + (L - 1) * stride : s - stride;
    const T phb = (MU == 3 && wb) ? (T)g.bc_t : (T)1;
    cx<T> p[12], u[9];
    ld.template get<MU, 1>(sf, wf, p);
    maybe_g5<G5IN>(p);
    lk(MU, s, u);
    hop_fwd<T, MU>(p, u, phf, acc);
    ld.template get<MU, -1>(sb, wb, p);
    maybe_g5<G5IN>(p);
    lk(MU, sb, u);
    hop_bwd<T, MU>(p, u, phb, acc);
}

// out(s) = [gamma5]^G5OUT (1 - kappa H) [gamma5]^G5IN in, at one site, the input read
// through the gather ld and the links through lk.
template <typename T, bool G5IN, bool G5OUT, class G, class LK>
__host__ __device__ inline void wilson_site_g(int s, const Geom &g, T kappa, const G &ld, const LK &lk,
                                              cx<T> (&out)[12]) {
    int c[4];
    int r = s;
    c[0] = r % g.L[0]; r /= g.L[0];
    c[1] = r % g.L[1]; r /= g.L[1];
    c[2] = r % g.L[2];
    c[3] = r / g.L[2];
    const int st1 = g.L[0], st2 = g.L[0] * g.L[1], st3 = st2 * g.L[2];
    cx<T> acc[12];
#pragma unroll
    for (int a = 0; a < 12; ++a) acc[a] = mk<T>(0, 0);
    hop_pair<T, 0, G5IN>(s, c, g, 1, ld, lk, acc);
    hop_pair<T, 1, G5IN>(s, c, g, st1, ld, lk, acc);
    hop_pair<T, 2, G5IN>(s, c, g, st2, ld, lk, acc);
    hop_pair<T, 3, G5IN>(s, c, g, st3, ld, lk, acc);
    ld.template get<0, 0>(s, false, out);
    maybe_g5<G5IN>(out);
#pragma unroll
    for (int a = 0; a < 12; ++a) {
        out[a].x = out[a].x - kappa * acc[a].x;
        out[a].y = out[a].y - kappa * acc[a].y;
    }
    maybe_g5<G5OUT>(out);
}

// out(s) = [gamma5]^G5OUT (1 - kappa H) [gamma5]^G5IN in, at one site.
template <typename T, bool G5IN, bool G5OUT>
__host__ __device__ inline void wilson_site(int s, const Geom &g, T kappa,
                                            const typename Field<T>::vec *__restrict__ in,
                                            const typename Link<T>::vec *__restrict__ U, cx<T> (&out)[12]) {
    const GlobalGather<T> ld{in, g.V};
    const PackedLinks<T> lk{U, g.V};
    wilson_site_g<T, G5IN, G5OUT>(s, g, kappa, ld, lk, out);
}

}  // namespace dlz
